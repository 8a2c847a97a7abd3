// Batches: the transforms of many plans with one launch per stage.
//
// A batch holds device copies of its plans' records, the per-stage block prefixes (which blocks of
// each launch belong to which signal) and device arrays of the per-execution input and output
// pointers.  Each execution copies the pointers in from a pinned staging ring (so back-to-back
// executions on one stream never overwrite a staging slot the GPU has not read yet) and then runs
// the same stage sequence as a single plan, each stage launched once for the whole batch.
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "sft_internal.h"

namespace sft {

namespace {
constexpr int kRing = 8;
size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
}  // namespace

struct Batch {
  std::vector<Plan*> plans;
  int n = 0;
  DevPlan d0;
  LaunchSet ls;
  char* dev = nullptr;
  size_t device_bytes = 0;
  DevPlan* d_plans = nullptr;
  void** d_ptrs = nullptr;            // [4][n]: f, out_w, out_c, out_n
  void** pinned = nullptr;            // [kRing][4][n]
  cudaEvent_t ring_ev[kRing] = {};
  bool ring_used[kRing] = {};
  int ring_pos = 0;
  Profiler prof;
  int64_t launches = 0;
};

void free_batch(Batch& B) {
  profile_release(B.prof);
  for (int i = 0; i < kRing; ++i)
    if (B.ring_ev[i]) cudaEventDestroy(B.ring_ev[i]);
  if (B.pinned) cudaFreeHost(B.pinned);
  if (B.dev) cudaFree(B.dev);
  B.pinned = nullptr;
  B.dev = nullptr;
}

}  // namespace sft

struct sft_batch_s {
  sft::Batch B;
};

extern "C" {

sft_status sft_batch_create(sft_batch_t* out, const sft_plan_t* plans, int32_t n) {
  using namespace sft;
  if (!out || !plans || n < 1 || n > (1 << 20)) {
    set_error("sft_batch_create: need out, plans and 1 <= n <= 2^20");
    return SFT_EINVAL;
  }
  *out = nullptr;
  std::vector<Plan*> ps(n);
  for (int i = 0; i < n; ++i) {
    if (!plans[i]) { set_error("sft_batch_create: NULL plan"); return SFT_EINVAL; }
    ps[i] = sft_plan_internal(plans[i]);
  }
  const DevPlan& a = ps[0]->d;
  for (int i = 0; i < n; ++i) {
    const DevPlan& b = ps[i]->d;
    if (b.prec != a.prec || b.input != a.input || b.kappa != a.kappa) {
      set_error("sft_batch_create: plans must share precision, input type and kappa");
      return SFT_EINVAL;
    }
    for (int k = 0; k < i; ++k)
      if (ps[k] == ps[i]) {
        set_error("sft_batch_create: a plan may appear once (its scratch serves one signal)");
        return SFT_EINVAL;
      }
  }
  sft_batch_s* h = new (std::nothrow) sft_batch_s();
  if (!h) { set_error("host allocation failed"); return SFT_ENOMEM; }
  Batch& B = h->B;
  B.plans = ps;
  B.n = n;
  B.d0 = a;
  // block prefixes of every stage
  std::vector<int32_t> prefix((size_t)kStCount * (n + 1), 0);
  for (int k = 0; k < kStCount; ++k) {
    int64_t acc = 0;
    for (int i = 0; i < n; ++i) {
      prefix[(size_t)k * (n + 1) + i] = (int32_t)acc;
      acc += signal_blocks(ps[i]->d, k);
    }
    if (acc > 0x7fffffff) { delete h; set_error("sft_batch_create: batch too large"); return SFT_EINVAL; }
    prefix[(size_t)k * (n + 1) + n] = (int32_t)acc;
    B.ls.blocks[k] = (int32_t)acc;
  }
  B.ls.pmax = 0;
  for (int i = 0; i < n; ++i) B.ls.pmax = std::max(B.ls.pmax, ps[i]->d.pmax);
  const size_t o_plans = 0;
  const size_t o_prefix = align256(o_plans + sizeof(DevPlan) * (size_t)n);
  const size_t o_ptrs = align256(o_prefix + prefix.size() * sizeof(int32_t));
  const size_t total = align256(o_ptrs + 4 * (size_t)n * sizeof(void*));
  cudaError_t e = cudaMalloc((void**)&B.dev, total);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete h;
    set_error(std::string("sft_batch_create: cudaMalloc failed: ") + cudaGetErrorString(e));
    return SFT_ENOMEM;
  }
  B.device_bytes = total;
  std::vector<char> blob(o_ptrs, 0);
  for (int i = 0; i < n; ++i) memcpy(blob.data() + o_plans + sizeof(DevPlan) * i, &ps[i]->d, sizeof(DevPlan));
  memcpy(blob.data() + o_prefix, prefix.data(), prefix.size() * sizeof(int32_t));
  e = cudaMemcpy(B.dev, blob.data(), o_ptrs, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaHostAlloc((void**)&B.pinned, (size_t)kRing * 4 * n * sizeof(void*),
                                          cudaHostAllocDefault);
  for (int i = 0; e == cudaSuccess && i < kRing; ++i)
    e = cudaEventCreateWithFlags(&B.ring_ev[i], cudaEventDisableTiming);
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_batch(B);
    delete h;
    set_error(std::string("sft_batch_create: set-up failed: ") + cudaGetErrorString(e));
    return SFT_ECUDA;
  }
  B.d_plans = reinterpret_cast<DevPlan*>(B.dev + o_plans);
  B.d_ptrs = reinterpret_cast<void**>(B.dev + o_ptrs);
  const int32_t* dpre = reinterpret_cast<const int32_t*>(B.dev + o_prefix);
  for (int k = 0; k < kStCount; ++k) B.ls.blk[k] = dpre + (size_t)k * (n + 1);
  *out = h;
  return SFT_OK;
}

sft_status sft_batch_execute(sft_batch_t batch, const void* const* f_devs,
                             int64_t* const* out_freqs_devs, void* const* out_coefs_devs,
                             int32_t* const* out_count_devs, void* stream) {
  using namespace sft;
  if (!batch || !f_devs || !out_freqs_devs || !out_coefs_devs || !out_count_devs) {
    set_error("sft_batch_execute: NULL argument");
    return SFT_EINVAL;
  }
  Batch& B = batch->B;
  const int n = B.n;
  const size_t align = B.d0.input == SFT_IN_C64 ? 8 : 16;
  for (int i = 0; i < n; ++i) {
    if (!f_devs[i] || ((uintptr_t)f_devs[i] % align) || !out_freqs_devs[i] || !out_coefs_devs[i] ||
        !out_count_devs[i]) {
      set_error("sft_batch_execute: NULL or misaligned pointer for signal " + std::to_string(i));
      return SFT_EINVAL;
    }
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int slot = B.ring_pos;
  B.ring_pos = (B.ring_pos + 1) % kRing;
  if (B.ring_used[slot]) cudaEventSynchronize(B.ring_ev[slot]);
  void** stage = B.pinned + (size_t)slot * 4 * n;
  for (int i = 0; i < n; ++i) {
    stage[i] = const_cast<void*>(f_devs[i]);
    stage[n + i] = out_freqs_devs[i];
    stage[2 * n + i] = out_coefs_devs[i];
    stage[3 * n + i] = out_count_devs[i];
  }
  cudaError_t e = cudaMemcpyAsync(B.d_ptrs, stage, 4 * (size_t)n * sizeof(void*),
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaEventRecord(B.ring_ev[slot], st);
  B.ring_used[slot] = true;
  if (e != cudaSuccess) {
    set_error(std::string("sft_batch_execute: pointer upload failed: ") + cudaGetErrorString(e));
    return SFT_ECUDA;
  }
  BatchView bv;
  memset(&bv, 0, sizeof(bv));
  bv.plans = B.d_plans;
  bv.n = n;
  bv.f = const_cast<const void* const*>(B.d_ptrs);
  bv.out_w = reinterpret_cast<int64_t* const*>(B.d_ptrs + n);
  bv.out_c = reinterpret_cast<double2* const*>(B.d_ptrs + 2 * n);
  bv.out_n = reinterpret_cast<int32_t* const*>(B.d_ptrs + 3 * n);
  int launched = 0;
  e = run_stages(B.d0, bv, B.ls, st, profile_slot(B.prof), &launched);
  B.launches += launched;
  if (e != cudaSuccess) {
    set_error(std::string("sft_batch_execute: launch failed: ") + cudaGetErrorString(e));
    return SFT_ECUDA;
  }
  return SFT_OK;
}

sft_status sft_batch_destroy(sft_batch_t batch) {
  if (!batch) return SFT_OK;
  sft::free_batch(batch->B);
  delete batch;
  return SFT_OK;
}

sft_status sft_batch_profile(sft_batch_t batch, int32_t enable) {
  if (!batch) { sft::set_error("batch is NULL"); return SFT_EINVAL; }
  return sft::profile_enable(batch->B.prof, enable);
}

sft_status sft_batch_profile_read(sft_batch_t batch, double* stage_ms, int32_t* n_executions) {
  if (!batch || !stage_ms || !n_executions) { sft::set_error("NULL argument"); return SFT_EINVAL; }
  return sft::profile_read(batch->B.prof, stage_ms, n_executions);
}

int64_t sft_batch_launches(sft_batch_t batch) { return batch ? batch->B.launches : 0; }

size_t sft_batch_device_bytes(sft_batch_t batch) { return batch ? batch->B.device_bytes : 0; }

}  // extern "C"
