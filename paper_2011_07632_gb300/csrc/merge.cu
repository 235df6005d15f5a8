// Cross-instance launch merging (see merge.cuh).
#include <algorithm>
#include <climits>

#include "merge.cuh"

namespace spd {

MergeCtx& merge_ctx() {
  static thread_local MergeCtx ctx;
  return ctx;
}

void Merger::submit(const std::string& key, std::unique_ptr<Deferred> d) {
  MergeCtx& ctx = merge_ctx();
  d->instance = ctx.instance;
  Slot slot;
  slot.key = key;
  slot.d = std::move(d);
  slot.stage = ctx.stage;
  slot.step = ctx.step++;
  std::unique_lock<std::mutex> lk(mu_);
  ++submissions_;
  pending_.push_back(&slot);
  ++waiting_;
  if (waiting_ >= live_) flush();
  cv_.wait(lk, [&] { return slot.done; });
  if (slot.err) std::rethrow_exception(slot.err);
}

void Merger::leave() {
  std::unique_lock<std::mutex> lk(mu_);
  --live_;
  if (waiting_ > 0 && waiting_ >= live_) flush();
}

void Merger::flush() {
  // the hand-overs at the earliest (stage, step), grouped by launcher kind
  int64_t st = INT64_MAX, sp = INT64_MAX;
  for (Slot* x : pending_)
    if (x->stage < st || (x->stage == st && x->step < sp)) { st = x->stage; sp = x->step; }
  std::map<std::string, std::vector<Slot*>> groups;
  std::vector<Slot*> rest;
  for (Slot* x : pending_) {
    if (x->stage == st && x->step == sp) groups[x->key].push_back(x);
    else rest.push_back(x);
  }
  MergeCtx& ctx = merge_ctx();
  const bool old = ctx.bypass;
  ctx.bypass = true;
  // the flushing thread may belong to any instance: launch on the shared stream
  StreamScope ss(s_);
  for (auto& kv : groups) {
    auto& v = kv.second;
    std::stable_sort(v.begin(), v.end(),
                     [](const Slot* a, const Slot* b) { return a->d->instance < b->d->instance; });
    std::vector<Deferred*> g;
    for (Slot* x : v) g.push_back(x->d.get());
    std::exception_ptr err;
    try {
      g[0]->launch_merged(g, s_);
    } catch (...) {
      err = std::current_exception();
    }
    ++launches_;
    for (Slot* x : v) {
      x->err = err;
      x->done = true;
      --waiting_;
    }
  }
  ctx.bypass = old;
  pending_.swap(rest);
  cv_.notify_all();
}

}  // namespace spd
