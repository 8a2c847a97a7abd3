// Faults a kernel records in the plan's status words instead of faulting the GPU.
//
// counters[nq + 1] holds the sft_fault bits of the current execution and counters[nq + 3] the
// sft_fault_site of its first index fault; the execution's first kernel clears both.  The checked
// build (compiled with SFT_CHECKED) range-checks the gather, bin and candidate indexes of every
// kernel: an index outside its buffer records SFT_FAULT_INDEX and its site, and the access is
// skipped.  In the normal build index_ok is the constant true, so the checks compile to nothing.
#pragma once

#include "sft_internal.h"

namespace sft {

#ifdef SFT_CHECKED
constexpr bool kCheckedBuild = true;
#else
constexpr bool kCheckedBuild = false;
#endif

// (A record without status words, that of the no-alloc DFT, records nothing.)
__device__ __forceinline__ void record_fault(const DevPlan& d, int bits, int site) {
  if (d.counters == nullptr) return;
  atomicOr(d.counters + d.nq + 1, bits);
  if (site != SFT_SITE_NONE) atomicCAS(d.counters + d.nq + 3, 0, site);
}

// True when 0 <= i < lim (always, in the normal build); otherwise records the fault.
__device__ __forceinline__ bool index_ok(const DevPlan& d, int64_t i, int64_t lim, int site) {
  if constexpr (!kCheckedBuild) {
    return true;
  } else {
    if (i >= 0 && i < lim) return true;
    record_fault(d, SFT_FAULT_INDEX, site);
    return false;
  }
}

}  // namespace sft
