// C ABI (include/sft.h): plan life cycle and the stream-ordered execution of Algorithm 1.
#include <atomic>
#include <stdint.h>
#include <string.h>

#include <cmath>
#include <new>
#include <string>

#include "alloc_hook.h"
#include "guard.h"
#include "sft_internal.h"

namespace sft {

namespace {
thread_local std::string g_last_error;
}

void set_error(const std::string& msg) { g_last_error = msg; }

sft_tuning default_tuning() {
  sft_tuning t;
  t.resample_threads = 256;
  t.resample_regcap = 0;
  t.bin_threads = 256;
  for (int c = 0; c < 9; ++c) {
    const int M = 64 << c;
    t.dft_per_cta[c] = M >= 4096 ? 1 : 4096 / M;
  }
  t.dft_two_ctas = 1;
  return t;
}

bool tuning_valid(const sft_tuning& t, std::string* why) {
  auto pow2_in = [](int v, int lo, int hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; };
  if (!pow2_in(t.resample_threads, 64, kResampleMaxThreads)) {
    *why = "resample_threads must be 64, 128, 256 or 512";
    return false;
  }
  if (t.resample_regcap != 0 && t.resample_regcap != 1) { *why = "resample_regcap must be 0 or 1"; return false; }
  if (t.resample_regcap == 1 && t.resample_threads > 256) {
    *why = "resample_regcap = 1 needs resample_threads <= 256";
    return false;
  }
  if (!pow2_in(t.bin_threads, 64, kBinMaxThreads)) {
    *why = "bin_threads must be 64, 128, 256 or 512";
    return false;
  }
  for (int c = 0; c < 9; ++c) {
    const int M = 64 << c;
    const int hi = M >= 4096 ? 1 : 4096 / M;
    if (t.dft_per_cta[c] < 1 || t.dft_per_cta[c] > hi) {
      *why = "dft_per_cta[" + std::to_string(c) + "] must be in 1.." + std::to_string(hi);
      return false;
    }
  }
  if (t.dft_two_ctas != 0 && t.dft_two_ctas != 1) { *why = "dft_two_ctas must be 0 or 1"; return false; }
  return true;
}

// Blocks of each stage for one signal (matches the kernels' block shapes under tuning t).
int signal_blocks(const DevPlan& d, int kind, const sft_tuning& tu) {
  switch (kind) {
    case kStOne: return 1;
    case kStResample: {
      const int t = (d.kappa == 4 || d.kappa == 6) ? tu.resample_threads : kResampleGenericThreads;
      return (int)((d.m + t - 1) / t);
    }
    case kStBins: return (int)(((int64_t)d.nq * d.Ptot + tu.bin_threads - 1) / tu.bin_threads);
    case kStShift: return d.nq;
    case kStShiftRank:
    case kStGlobalRank:
    case kStFinalRank: return rank_blocks(d, kind);
    case kStReest: return d.prec == SFT_FP32 ? d.nq * d.K * d.nchunk : 0;
    case kStRefine: return d.prec == SFT_FP32 ? (d.s + kRefineThreads - 1) / kRefineThreads : 0;
    case kStRader: return d.rader ? d.nq * d.K * d.nsub : 0;
    default:
      if (kind >= kStBluestein0 && kind < kStCount) {
        const int M = fft_stage_length(kind);
        return bluestein_blocks(d, M, tu.dft_per_cta[fft_tune_class(M)]);
      }
      return 0;
  }
}

LaunchSet single_launch_set(const DevPlan& d) {
  LaunchSet ls;
  ls.tune = default_tuning();
  for (int k = 0; k < kStCount; ++k) {
    ls.blocks[k] = signal_blocks(d, k, ls.tune);
    ls.blk[k] = nullptr;
  }
  ls.pmax = d.pmax;
  ls.rlmax = d.rader ? d.rLmax : 0;
  ls.rtpt = d.rader ? d.rTpt : 0;
  ls.kmax = d.K;
  return ls;
}

cudaEvent_t* profile_slot(Profiler& pr) {
  if (pr.on && pr.recorded < kProfileCap) return &pr.events[(size_t)pr.recorded++ * (kStages + 1)];
  return nullptr;
}

void profile_release(Profiler& pr) {
  for (cudaEvent_t e : pr.events) cudaEventDestroy(e);
  pr.events.clear();
  pr.on = false;
  pr.recorded = 0;
}

sft_status profile_enable(Profiler& pr, int enable) {
  profile_release(pr);
  if (!enable) return SFT_OK;
  const size_t n = (size_t)kProfileCap * (kStages + 1);
  pr.events.resize(n);
  for (size_t i = 0; i < n; ++i) {
    if (cudaEventCreate(&pr.events[i]) != cudaSuccess) {
      pr.events.resize(i);
      profile_release(pr);
      set_error("cudaEventCreate failed");
      return SFT_ECUDA;
    }
  }
  pr.on = true;
  return SFT_OK;
}

sft_status profile_read(Profiler& pr, double* stage_ms, int32_t* n_executions) {
  for (int k = 0; k < kStages; ++k) stage_ms[k] = 0.0;
  *n_executions = pr.recorded;
  for (int r = 0; r < pr.recorded; ++r) {
    cudaEvent_t* ev = &pr.events[(size_t)r * (kStages + 1)];
    for (int k = 0; k < kStages; ++k) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev[k], ev[k + 1]) != cudaSuccess) {
        cudaGetLastError();
        set_error("profile events not complete (synchronise the stream first)");
        return SFT_ECUDA;
      }
      stage_ms[k] += ms;
    }
  }
  pr.recorded = 0;
  return SFT_OK;
}

// The stages of Algorithm 1 for every signal of bv, in stream order.  ev (optional) receives
// kStages + 1 events recorded between the stages.
cudaError_t run_stages(const DevPlan& d0, const BatchView& bv, const LaunchSet& ls,
                       cudaStream_t st, cudaEvent_t* ev, int* launched) {
  auto mark = [&](int k) { if (ev) cudaEventRecord(ev[k], st); };
  const bool fp64 = d0.prec == SFT_FP64;
  cudaError_t e = launch_zero(bv, ls, st);
  ++*launched;
  mark(0);
  if (e == cudaSuccess) { e = launch_resample(d0, bv, ls, st); ++*launched; }
  mark(1);
  if (e == cudaSuccess) e = launch_bluestein(d0, bv, ls, st, launched);
  mark(2);
  if (e == cudaSuccess) { e = launch_identify(d0, bv, ls, st); ++*launched; }
  mark(3);
  if (e == cudaSuccess) { e = launch_vote(d0, bv, ls, st); ++*launched; }
  mark(4);
  if (e == cudaSuccess) e = launch_select(bv, ls, st, launched);
  mark(5);
  if (e == cudaSuccess && !fp64 && d0.refine) { e = launch_refine(bv, ls, st); *launched += 3; }
  if (e == cudaSuccess) e = launch_finalize(bv, ls, st, launched);
  mark(6);
  return e;
}

}  // namespace sft

using sft::Plan;

struct sft_plan_s {
  Plan P;
};

namespace sft {
Plan* sft_plan_internal(sft_plan_t plan) { return &plan->P; }
}  // namespace sft

namespace sft {

// Allocation-failure injection: after `skip` more allocations succeed, the next `fail` ones
// return cudaErrorMemoryAllocation without allocating.
namespace {
std::atomic<int64_t> g_inject_skip{0}, g_inject_fail{0};

bool inject_failure() {
  if (g_inject_fail.load() <= 0) return false;
  if (g_inject_skip.fetch_sub(1) > 0) return false;
  g_inject_skip.store(0);
  return g_inject_fail.fetch_sub(1) > 0;
}
}  // namespace

cudaError_t dev_malloc(void** p, size_t bytes) {
  if (inject_failure()) { *p = nullptr; return cudaErrorMemoryAllocation; }
  return cudaMalloc(p, bytes);
}

cudaError_t dev_malloc_async(void** p, size_t bytes, cudaStream_t st) {
  if (inject_failure()) { *p = nullptr; return cudaErrorMemoryAllocation; }
  return cudaMallocAsync(p, bytes, st);
}

cudaError_t host_alloc(void** p, size_t bytes) {
  if (inject_failure()) { *p = nullptr; return cudaErrorMemoryAllocation; }
  return cudaHostAlloc(p, bytes, cudaHostAllocDefault);
}

}  // namespace sft

extern "C" {

sft_status sft_variant_init(sft_variant* v) {
  if (!v) { sft::set_error("variant is NULL"); return SFT_EINVAL; }
  v->kappa = SFT_DMSFT6;
  v->precision = SFT_FP32;
  v->input = SFT_IN_C64;
  v->K = 5;
  v->c_p = 3.0;
  v->alpha = 1.5;
  v->beta = 1.5;
  v->seed = 0;
  v->deterministic = 0;
  v->refine_fp64 = 1;
  v->pool = SFT_POOL_ALL;
  v->dft = SFT_DFT_AUTO;
  return SFT_OK;
}

sft_status sft_variant_theorem(sft_variant* v, int64_t N, double r) {
  if (!v) { sft::set_error("variant is NULL"); return SFT_EINVAL; }
  if (!(r >= 1.0) || (double)N < 36.0 * r) {
    sft::set_error("theorem parameters need r >= 1 and N >= 36 r");
    return SFT_EINVAL;
  }
  const double kPi = 3.14159265358979323846;
  const double half = std::ceil(6.0 * r * std::log((double)N) / (std::sqrt(2.0) * kPi)) + 1.0;
  if (half > sft::kMaxKappa) {
    sft::set_error("theorem half-width " + std::to_string((int64_t)half) + " exceeds 48");
    return SFT_EINVAL;
  }
  v->kappa = (int32_t)half;
  v->beta = 6.0 * std::sqrt(r);
  v->alpha = v->beta;
  return SFT_OK;
}

sft_status sft_plan(sft_plan_t* out, int64_t N, int32_t s, const sft_variant* v, int32_t n_shifts,
                    const int64_t* primes, int32_t n_primes, const int32_t* small_moduli,
                    int32_t n_small) {
  return sft::guarded("sft_plan", [&]() -> sft_status {
    if (!out) { sft::set_error("out is NULL"); return SFT_EINVAL; }
    *out = nullptr;
    sft_plan_s* h = new (std::nothrow) sft_plan_s();
    if (!h) { sft::set_error("host allocation failed"); return SFT_ENOMEM; }
    sft_status st = sft::build_plan(&h->P, N, s, v, n_shifts, primes, n_primes, small_moduli, n_small);
    if (st != SFT_OK) {
      sft::free_plan(&h->P);
      delete h;
      return st;
    }
    *out = h;
    return SFT_OK;
  });
}

sft_status sft_plan_destroy(sft_plan_t plan) {
  if (!plan) return SFT_OK;
  if (plan->P.solo) sft_batch_destroy(plan->P.solo);
  sft::profile_release(plan->P.prof);
  sft::free_plan(&plan->P);
  delete plan;
  return SFT_OK;
}

size_t sft_plan_device_bytes(sft_plan_t plan) { return plan ? plan->P.device_bytes : 0; }

sft_status sft_plan_info(sft_plan_t plan, sft_plan_desc* o) {
  if (!plan || !o) { sft::set_error("plan or out is NULL"); return SFT_EINVAL; }
  memset(o, 0, sizeof(*o));
  const sft::DevPlan& d = plan->P.d;
  o->N = d.N; o->s = d.s; o->kappa = d.kappa; o->K = d.K; o->n_small = d.nT; o->n_shifts = d.nq;
  o->n_sub = d.nsub;
  for (int j = 0; j < d.K; ++j) o->primes[j] = d.p[j];
  for (int l = 0; l < d.nT; ++l) o->small[l] = d.t[l];
  for (int i = 0; i < d.nq; ++i) o->shifts[i] = d.q[i];
  o->L = d.L; o->c1 = d.c1; o->nodes = d.m; o->fft_size = d.fftM;
  o->precision = d.prec; o->input = d.input;
  o->dft = d.rader ? SFT_DFT_RADER : SFT_DFT_CHIRP;
  return SFT_OK;
}

sft_status sft_plan_debug_buffer(sft_plan_t plan, int32_t which, void** dev_ptr, size_t* bytes) {
  if (!plan || !dev_ptr || !bytes) { sft::set_error("NULL argument"); return SFT_EINVAL; }
  const sft::DevPlan& d = plan->P.d;
  const size_t cs = d.prec == SFT_FP64 ? 16 : 8;
  switch (which) {
    case 0: *dev_ptr = d.samples; *bytes = (size_t)d.nq * d.m * cs; return SFT_OK;
    case 1: *dev_ptr = d.bins; *bytes = (size_t)d.nq * d.m * cs; return SFT_OK;
    case 2: *dev_ptr = d.cand; *bytes = (size_t)d.nq * d.Ptot * 8; return SFT_OK;
    case 3: *dev_ptr = d.resid; *bytes = (size_t)d.nq * d.Ptot * (d.nT > 0 ? d.nT : 1); return SFT_OK;
    case 4: *dev_ptr = d.counters; *bytes = (size_t)(d.nq + 4) * 4; return SFT_OK;
    case 5: *dev_ptr = d.voted; *bytes = (size_t)d.nq * d.vcap * sizeof(sft::Voted); return SFT_OK;
    default: sft::set_error("unknown buffer index"); return SFT_EINVAL;
  }
}

sft_status sft_debug_fail_allocations(int32_t skip, int32_t fail) {
  if (skip < 0 || fail < 0) { sft::set_error("sft_debug_fail_allocations: negative count"); return SFT_EINVAL; }
  sft::g_inject_fail.store(0);
  sft::g_inject_skip.store(skip);
  sft::g_inject_fail.store(fail);
  return SFT_OK;
}

int32_t sft_checked_build(void) {
#ifdef SFT_CHECKED
  return 1;
#else
  return 0;
#endif
}

sft_status sft_plan_faults(sft_plan_t plan, void* stream, int32_t* faults, int32_t* site) {
  if (!plan) { sft::set_error("plan is NULL"); return SFT_EINVAL; }
  const sft::DevPlan& d = plan->P.d;
  cudaStream_t st = (cudaStream_t)stream;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(st, &cap);
  if (e != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    sft::set_error("sft_plan_faults: the stream is being captured (or cannot be queried)");
    return SFT_EINVAL;
  }
  int32_t w[4] = {0, 0, 0, 0};                 // counters[nq .. nq + 3]
  e = cudaMemcpyAsync(w, d.counters + d.nq, sizeof(w), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    sft::set_error(std::string("sft_plan_faults: read failed: ") + cudaGetErrorString(e));
    return SFT_ECUDA;
  }
  if (faults) *faults = w[1];
  if (site) *site = w[3];
  return SFT_OK;
}

sft_status sft_plan_debug_limit(sft_plan_t plan, int32_t which, int32_t value) {
  if (!plan) { sft::set_error("plan is NULL"); return SFT_EINVAL; }
  Plan& P = plan->P;
  if (which != 0) { sft::set_error("sft_plan_debug_limit: unknown limit"); return SFT_EINVAL; }
  int64_t built = 0;                           // the voted list's built capacity: sum_j p_j
  for (int32_t pj : P.primes) built += pj;
  if (value < 1 || value > built) {
    sft::set_error("sft_plan_debug_limit: value must be in 1 .. sum_j p_j");
    return SFT_EINVAL;
  }
  P.d.vcap = value;
  const cudaError_t e = cudaMemcpy(P.d_dev, &P.d, sizeof(sft::DevPlan), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaGetLastError();
    sft::set_error(std::string("sft_plan_debug_limit: upload failed: ") + cudaGetErrorString(e));
    return SFT_ECUDA;
  }
  return SFT_OK;
}

sft_status sft_execute(sft_plan_t plan, const void* f_dev, int64_t* out_freqs_dev,
                       void* out_coefs_dev, int32_t* out_count_dev, void* stream) {
  if (!plan || !f_dev) { sft::set_error("plan or f is NULL"); return SFT_EINVAL; }
  const bool any = out_freqs_dev || out_coefs_dev || out_count_dev;
  const bool all = out_freqs_dev && out_coefs_dev && out_count_dev;
  if (any && !all) { sft::set_error("outputs must be all NULL or all non-NULL"); return SFT_EINVAL; }
  Plan& P = plan->P;
  const sft::DevPlan& d = P.d;
  const uintptr_t fa = (uintptr_t)f_dev;
  if (fa % (d.input == SFT_IN_C64 ? 8 : 16) != 0) {
    sft::set_error("f is not aligned to its element size");
    return SFT_EINVAL;
  }
  if (P.graph_on && all) {
    // replay of the plan's captured launches (its batch of one), after this call's pointer upload
    const int64_t before = sft_batch_launches(P.solo);
    void* cw = out_coefs_dev;
    const sft_status st = sft_batch_execute(P.solo, &f_dev, &out_freqs_dev, &cw, &out_count_dev,
                                            stream);
    P.launches += sft_batch_launches(P.solo) - before;
    return st;
  }
  sft::BatchView bv;
  memset(&bv, 0, sizeof(bv));
  bv.plans = P.d_dev;
  bv.n = 1;
  bv.f0 = f_dev;
  bv.out_w0 = out_freqs_dev;
  bv.out_c0 = reinterpret_cast<double2*>(out_coefs_dev);
  bv.out_n0 = out_count_dev;
  sft::LaunchSet ls = sft::single_launch_set(d);
  int launched = 0;
  cudaError_t e = sft::run_stages(d, bv, ls, (cudaStream_t)stream, sft::profile_slot(P.prof),
                                  &launched);
  P.launches += launched;
  if (e != cudaSuccess) {
    sft::set_error(std::string("CUDA launch failed: ") + cudaGetErrorString(e));
    return SFT_ECUDA;
  }
  return SFT_OK;
}

sft_status sft_plan_graph(sft_plan_t plan, int32_t enable) {
  if (!plan) { sft::set_error("plan is NULL"); return SFT_EINVAL; }
  Plan& P = plan->P;
  if (enable && !P.solo) {
    sft_plan_t one = plan;
    const sft_status st = sft_batch_create(&P.solo, &one, 1);
    if (st != SFT_OK) return st;
    sft_batch_graph(P.solo, 1);
  }
  P.graph_on = enable != 0;
  return SFT_OK;
}

sft_status sft_plan_profile(sft_plan_t plan, int32_t enable) {
  if (!plan) { sft::set_error("plan is NULL"); return SFT_EINVAL; }
  return sft::profile_enable(plan->P.prof, enable);
}

sft_status sft_plan_profile_read(sft_plan_t plan, double* stage_ms, int32_t* n_executions) {
  if (!plan || !stage_ms || !n_executions) { sft::set_error("NULL argument"); return SFT_EINVAL; }
  return sft::profile_read(plan->P.prof, stage_ms, n_executions);
}

int64_t sft_plan_launches(sft_plan_t plan) { return plan ? plan->P.launches : 0; }

sft_status sft_choose_moduli(int64_t N, int32_t s, int32_t K, double c_p, uint64_t seed,
                             int64_t* primes_out, int32_t* small_out, int32_t* n_small_out) {
  return sft::choose_moduli(N, s, K, c_p, seed, primes_out, small_out, n_small_out);
}

sft_status sft_choose_moduli_pool(int64_t N, int32_t s, int32_t K, double c_p, uint64_t seed,
                                  int32_t pool, int64_t* primes_out, int32_t* small_out,
                                  int32_t* n_small_out) {
  return sft::choose_moduli(N, s, K, c_p, seed, primes_out, small_out, n_small_out, pool);
}

sft_status sft_choose_moduli_deterministic(int64_t N, int32_t s, double c_p, int64_t* primes_out,
                                           int32_t* K_out, int32_t* small_out, int32_t* n_small_out) {
  return sft::choose_moduli_deterministic(N, s, c_p, primes_out, K_out, small_out, n_small_out);
}

const char* sft_last_error(void) { return sft::g_last_error.c_str(); }

void sft_tuning_default(sft_tuning* t) {
  if (t) *t = sft::default_tuning();
}

}  // extern "C"
