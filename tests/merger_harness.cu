// Host-only harness for the launch merger of the batched level sweep (merge.cuh), linked
// against libspdhss.so.  Instances run on host threads and hand over "launches" whose
// merged form only records which instances it contained; nothing touches a GPU.  Prints
// "OK" and returns 0 when every scenario behaves as specified, else prints the failure.
#include <cstdio>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "merge.cuh"

using namespace spd;

namespace {

struct Launch {
  std::string key;
  std::vector<int> instances;
};

struct Log {
  std::mutex mu;
  std::vector<Launch> launches;
  void add(const std::string& key, const std::vector<int>& all) {
    std::lock_guard<std::mutex> g(mu);
    launches.push_back({key, all});
  }
};

int g_fail = 0;
#define CHECK(c, what)                                      \
  do {                                                      \
    if (!(c)) {                                             \
      std::printf("FAIL %s: %s\n", what, #c);               \
      ++g_fail;                                             \
    }                                                       \
  } while (0)

// one hand-over of `key` by the calling instance (its id is the descriptor)
void hand_over(Log& log, const std::string& key, bool fail = false) {
  std::vector<int> h = {merge_ctx().instance};
  defer_launch(key, h, [&log, key, fail](std::vector<int>& all, cudaStream_t) {
    log.add(key, all);
    if (fail) throw Error(SPDHSS_NOT_SPD, "planted failure in " + key);
  });
}

template <class F>
void run_instances(Merger& m, int count, F body) {
  std::vector<std::thread> th;
  for (int k = 0; k < count; ++k)
    th.emplace_back([&m, k, &body] {
      MergeCtx& c = merge_ctx();
      c.m = &m;
      c.instance = k;
      c.stage = c.step = 0;
      body(k);
      m.leave();
      c.m = nullptr;
    });
  for (auto& t : th) t.join();
}

bool same(const std::vector<int>& a, const std::vector<int>& b) { return a == b; }

}  // namespace

int main() {
  // 1. lockstep: every step of every stage becomes one launch holding all instances in
  //    instance order, stages in order
  {
    Log log;
    Merger m(nullptr, 4);
    run_instances(m, 4, [&](int) {
      for (int st = 0; st < 3; ++st) {
        merge_stage(1, st);
        for (const char* key : {"a", "b", "a"}) hand_over(log, std::string(key) + std::to_string(st));
      }
    });
    CHECK(log.launches.size() == 9, "lockstep count");
    const char* order[] = {"a0", "b0", "a0", "a1", "b1", "a1", "a2", "b2", "a2"};
    for (size_t i = 0; i < log.launches.size() && i < 9; ++i) {
      CHECK(log.launches[i].key == order[i], "lockstep order");
      CHECK(same(log.launches[i].instances, {0, 1, 2, 3}), "lockstep members");
    }
    CHECK(m.launches() == 9 && m.submissions() == 36, "lockstep counters");
  }
  // 2. uneven depths: instance k runs k + 1 stages and then leaves; nobody waits for it
  {
    Log log;
    Merger m(nullptr, 3);
    run_instances(m, 3, [&](int k) {
      for (int st = 0; st <= k; ++st) {
        merge_stage(1, st);
        hand_over(log, "s" + std::to_string(st));
      }
    });
    CHECK(log.launches.size() == 3, "uneven count");
    if (log.launches.size() == 3) {
      CHECK(same(log.launches[0].instances, {0, 1, 2}), "uneven stage 0");
      CHECK(same(log.launches[1].instances, {1, 2}), "uneven stage 1");
      CHECK(same(log.launches[2].instances, {2}), "uneven stage 2");
    }
  }
  // 3. an instance that runs ahead waits: instance 1 skips stage 0 entirely, so its stage-1
  //    hand-over is launched only after instance 0's stage-0 one, together with instance
  //    0's stage-1 hand-over
  {
    Log log;
    Merger m(nullptr, 2);
    run_instances(m, 2, [&](int k) {
      if (k == 0) {
        merge_stage(1, 0);
        hand_over(log, "x");
      }
      merge_stage(1, 1);
      hand_over(log, "y");
    });
    CHECK(log.launches.size() == 2, "ahead count");
    if (log.launches.size() == 2) {
      CHECK(log.launches[0].key == "x" && same(log.launches[0].instances, {0}), "ahead first");
      CHECK(log.launches[1].key == "y" && same(log.launches[1].instances, {0, 1}), "ahead merged");
    }
  }
  // 4. empty launcher calls keep the steps aligned (merge_skip); different kinds at the
  //    same step become separate launches
  {
    Log log;
    Merger m(nullptr, 2);
    run_instances(m, 2, [&](int k) {
      merge_stage(2, 0);
      hand_over(log, "a");
      if (k == 0) merge_skip();
      else hand_over(log, "b");
      hand_over(log, k == 0 ? "c" : "d");
    });
    CHECK(log.launches.size() == 4, "skip count");
    if (log.launches.size() == 4) {
      CHECK(log.launches[0].key == "a" && same(log.launches[0].instances, {0, 1}), "skip a");
      CHECK(log.launches[1].key == "b" && same(log.launches[1].instances, {1}), "skip b");
      // step 2: kinds c (instance 0) and d (instance 1), one launch each, in key order
      CHECK(log.launches[2].key == "c" && same(log.launches[2].instances, {0}), "skip c");
      CHECK(log.launches[3].key == "d" && same(log.launches[3].instances, {1}), "skip d");
    }
  }
  // 5. a failing merged launch reports its error to every instance in it, and the
  //    instances go on (or stop) independently
  {
    Log log;
    Merger m(nullptr, 3);
    std::mutex mu;
    std::vector<int> caught;
    run_instances(m, 3, [&](int k) {
      merge_stage(1, 0);
      try {
        hand_over(log, "bad", true);
      } catch (const Error& e) {
        std::lock_guard<std::mutex> g(mu);
        if (e.code == SPDHSS_NOT_SPD) caught.push_back(k);
        if (k == 1) return;   // this instance stops after the failure
      }
      merge_stage(1, 1);
      hand_over(log, "after");
    });
    CHECK(caught.size() == 3, "error reaches every member");
    CHECK(log.launches.size() == 2, "failure count");
    if (log.launches.size() == 2)
      CHECK(log.launches[1].key == "after" && same(log.launches[1].instances, {0, 2}),
            "survivors merge");
  }
  if (g_fail == 0) std::printf("OK\n");
  return g_fail == 0 ? 0 : 1;
}
