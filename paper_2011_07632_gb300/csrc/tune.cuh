// Launch-variant autotuning.  For a launch kind and a bucket of its shape, every candidate
// variant is timed once on a synthetic problem set of that shape (CUDA events on a private
// stream) and the fastest is kept for the rest of the process, per device.  Only variants
// that leave every problem's arithmetic unchanged are tuned, so results never depend on the
// choice, on timing noise or on which process made it.  SPDHSS_TUNE=0 turns tuning off
// (the launchers' fixed rules apply).
#pragma once

#include <functional>
#include <string>
#include <vector>

#include "common.cuh"

namespace spd {

bool tuning_enabled();
// the cached choice for `key` (device-qualified inside), timing each candidate with
// time_ms(candidate) on the first request; `fallback` when tuning is off or every timing
// failed
int tuned_variant(const std::string& key, const std::vector<int>& cands, int fallback,
                  const std::function<double(int)>& time_ms);
// one line per tuned key: "key -> chosen  (candidate:ms ...)"
std::string tuning_report();

}  // namespace spd
