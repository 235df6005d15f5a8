// Launch-variant autotuning (see tune.cuh).
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>

#include "tune.cuh"

namespace spd {

namespace {
struct Entry {
  int choice;
  std::vector<std::pair<int, double>> times;
};
std::mutex g_tune_mu;
std::map<std::string, Entry> g_tune;
}  // namespace

bool tuning_enabled() {
  const char* e = std::getenv("SPDHSS_TUNE");
  return !(e && e[0] == '0');
}

int tuned_variant(const std::string& key, const std::vector<int>& cands, int fallback,
                  const std::function<double(int)>& time_ms) {
  if (!tuning_enabled() || cands.size() < 2) return fallback;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {   // no device (a host-only caller): one cache
    cudaGetLastError();
    dev = -1;
  }
  const std::string k = "dev" + std::to_string(dev) + " " + key;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(k);
  if (it != g_tune.end()) return it->second.choice;
  Entry e{fallback, {}};
  double best = 0.0;
  for (int c : cands) {
    double t = -1.0;
    try {
      t = time_ms(c);
    } catch (...) {
      cudaGetLastError();
      t = -1.0;
    }
    e.times.emplace_back(c, t);
    if (t > 0.0 && (best == 0.0 || t < best)) { best = t; e.choice = c; }
  }
  g_tune.emplace(k, e);
  return e.choice;
}

std::string tuning_report() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  std::string out;
  for (const auto& kv : g_tune) {
    out += kv.first + " -> " + std::to_string(kv.second.choice) + "  (";
    for (size_t i = 0; i < kv.second.times.size(); ++i) {
      char buf[64];
      std::snprintf(buf, sizeof(buf), "%s%d:%.4f", i ? " " : "", kv.second.times[i].first,
                    kv.second.times[i].second);
      out += buf;
    }
    out += " ms)\n";
  }
  return out;
}

}  // namespace spd
