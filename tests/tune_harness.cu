// Host-only harness for the launch-variant tuner (tune.cuh), linked against libspdhss.so:
// the candidates' "timings" are host functions, nothing touches a GPU.  Prints "OK" and
// returns 0 when every scenario behaves as specified, else prints the failure.
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <stdexcept>
#include <string>
#include <thread>
#include <vector>

#include "tune.cuh"

using namespace spd;

namespace {

int g_fail = 0;
#define CHECK(c, what)                                      \
  do {                                                      \
    if (!(c)) {                                             \
      std::printf("FAIL %s: %s\n", what, #c);               \
      ++g_fail;                                             \
    }                                                       \
  } while (0)

}  // namespace

int main() {
  // the fastest candidate is kept; each candidate is timed once, on the first request only
  {
    int calls = 0;
    auto t = [&](int c) { ++calls; return c == 4 ? 0.5 : 1.0 + c; };
    const int a = tuned_variant("kind_a n64", {1, 2, 4, 8}, 2, t);
    CHECK(a == 4 && calls == 4, "first request");
    const int b = tuned_variant("kind_a n64", {1, 2, 4, 8}, 2, t);
    CHECK(b == 4 && calls == 4, "cached request");
    // another shape bucket is tuned on its own
    auto t2 = [&](int c) { ++calls; return c == 1 ? 0.1 : 1.0; };
    CHECK(tuned_variant("kind_a n128", {1, 2, 4, 8}, 2, t2) == 1 && calls == 8, "second key");
  }
  // ties keep the earlier candidate
  {
    auto t = [](int) { return 1.0; };
    CHECK(tuned_variant("kind_tie", {8, 2, 4}, 2, t) == 8, "tie");
  }
  // a candidate whose timing throws or fails is skipped; all failing -> the fallback
  {
    auto t = [](int c) -> double {
      if (c == 1) throw std::runtime_error("launch failed");
      return c == 2 ? -1.0 : 3.0;
    };
    CHECK(tuned_variant("kind_fail", {1, 2, 4}, 2, t) == 4, "skip failed candidates");
    auto none = [](int) -> double { throw std::runtime_error("launch failed"); };
    CHECK(tuned_variant("kind_none", {1, 2}, 2, none) == 2, "every candidate failed");
  }
  // a single candidate is not timed
  {
    int calls = 0;
    auto t = [&](int) { ++calls; return 1.0; };
    CHECK(tuned_variant("kind_one", {4}, 1, t) == 1 && calls == 0, "single candidate");
  }
  // SPDHSS_TUNE=0: the fallback, nothing timed, nothing cached
  {
    int calls = 0;
    auto t = [&](int c) { ++calls; return c == 8 ? 0.1 : 1.0; };
    setenv("SPDHSS_TUNE", "0", 1);
    CHECK(!tuning_enabled(), "tuning off");
    CHECK(tuned_variant("kind_off", {1, 8}, 1, t) == 1 && calls == 0, "tuning off");
    unsetenv("SPDHSS_TUNE");
    CHECK(tuning_enabled(), "tuning on");
    CHECK(tuned_variant("kind_off", {1, 8}, 1, t) == 8 && calls == 2, "tuned after off");
  }
  // concurrent first requests for one key: timed once, every caller gets the same choice
  {
    std::atomic<int> calls{0};
    std::vector<int> got(8, -1);
    std::vector<std::thread> th;
    for (int i = 0; i < 8; ++i)
      th.emplace_back([&, i] {
        got[i] = tuned_variant("kind_mt", {1, 2, 4}, 1, [&](int c) {
          ++calls;
          return c == 2 ? 0.2 : 0.9;
        });
      });
    for (auto& t : th) t.join();
    bool same = true;
    for (int v : got) same = same && v == 2;
    CHECK(same && calls.load() == 3, "concurrent first requests");
  }
  // the report: one line per tuned key, with the choice and every candidate's time
  {
    const std::string r = tuning_report();
    CHECK(r.find("kind_a n64 -> 4  (1:2.0000 2:3.0000 4:0.5000 8:9.0000 ms)") != std::string::npos,
          "report line");
    CHECK(r.find("kind_none -> 2") != std::string::npos, "report of a failed key");
    CHECK(r.find("kind_one") == std::string::npos, "untimed key not reported");
  }
  if (g_fail) return 1;
  std::printf("OK\n");
  return 0;
}
