// Cross-instance launch merging for the batched level sweep.
//
// Several independent instances (each its own points, kernel, tree and H^2 / SPD-HSS /
// ULV state) run the single-instance host code on one host thread each, all on one CUDA
// stream.  Every batched launcher (grouped GEMM, kernel tiles, proxy matrices, near field,
// Cholesky, TRSM, pivoted QR, reflectors, copies) hands its descriptors to the Merger
// instead of launching.  Once every instance still running is waiting in such a hand-over,
// the Merger concatenates the descriptors of each launcher kind (in instance order) and
// issues one launch per kind: the nodes of all instances at the same step of the level
// sweep go into one kernel launch.  Instances that run ahead or behind (other depths,
// other paths) simply form their own groups; nothing waits for a launch that is not
// coming, so the scheme cannot deadlock.  Kernels that are not batched over problems
// (tree construction, gathers, dots) are launched by the instance directly.
#pragma once

#include <condition_variable>
#include <exception>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

namespace spd {

// A launch handed over by one instance: its descriptors and launch parameters.
struct Deferred {
  int instance = 0;
  virtual ~Deferred() = default;
  // launch all entries of `group` (same key as this entry, in instance order) at once
  virtual void launch_merged(const std::vector<Deferred*>& group, cudaStream_t s) = 0;
};

class Merger {
 public:
  Merger(cudaStream_t s, int participants) : s_(s), live_(participants) {}
  // Hand over a launch; returns once the merged launch containing it has been issued on
  // the shared stream (rethrows the error of that merged launch, if any).
  void submit(const std::string& key, std::unique_ptr<Deferred> d);
  // The calling instance has finished (or failed) and submits nothing more.
  void leave();
  cudaStream_t stream() const { return s_; }
  int64_t launches() const { return launches_; }
  int64_t submissions() const { return submissions_; }

 private:
  struct Slot {
    std::string key;
    std::unique_ptr<Deferred> d;
    int64_t stage = 0, step = 0;
    bool done = false;
    std::exception_ptr err;
  };
  void flush();   // called with mu_ held when every live instance is waiting
  cudaStream_t s_;
  std::mutex mu_;
  std::condition_variable cv_;
  int live_;
  int waiting_ = 0;
  std::vector<Slot*> pending_;
  int64_t launches_ = 0, submissions_ = 0;
};

// Per host thread: the Merger of the instance running on it (null: launch directly), and
// its position in the sweep.  The Merger launches the waiting hand-overs at the earliest
// (stage, step) first, so instances that ran ahead wait for the others at the same step
// and their launches merge.  `stage` is set by the sweep (phase and level, or the PCG
// iteration) and must not decrease; `step` counts the batched launcher calls of the stage,
// empty ones included.
struct MergeCtx {
  Merger* m = nullptr;
  int instance = 0;
  bool bypass = false;   // set while the Merger itself issues a merged launch
  int64_t stage = 0;
  int64_t step = 0;
};
MergeCtx& merge_ctx();

inline bool merging() {
  const MergeCtx& c = merge_ctx();
  return c.m != nullptr && !c.bypass;
}

// Mark the start of a stage of the sweep (phase, level): no-op when not merging.
inline void merge_stage(int phase, int64_t level) {
  MergeCtx& c = merge_ctx();
  if (!c.m) return;
  c.stage = (int64_t)phase * (int64_t(1) << 40) + level;
  c.step = 0;
}
// A batched launcher was called with nothing to launch: keep the step count aligned.
inline void merge_skip() {
  MergeCtx& c = merge_ctx();
  if (c.m && !c.bypass) ++c.step;
}

// Descriptor vectors of one launcher kind: the merged launch concatenates them.
template <class P>
struct DeferredVec : Deferred {
  std::vector<P> h;
  std::function<void(std::vector<P>&, cudaStream_t)> fn;
  void launch_merged(const std::vector<Deferred*>& group, cudaStream_t s) override {
    std::vector<P> all;
    for (Deferred* d : group) {
      const auto* v = static_cast<const DeferredVec<P>*>(d);
      all.insert(all.end(), v->h.begin(), v->h.end());
    }
    fn(all, s);
  }
};

// Hand a launch over descriptor vector h to the calling thread's Merger; `fn` performs the
// real launch on the merged vector.  Returns false (and does nothing) when not merging.
template <class P, class F>
bool defer_launch(const std::string& key, const std::vector<P>& h, F fn) {
  if (!merging()) return false;
  std::unique_ptr<DeferredVec<P>> d(new DeferredVec<P>());
  d->h = h;
  d->fn = fn;
  merge_ctx().m->submit(key, std::move(d));
  return true;
}

}  // namespace spd
