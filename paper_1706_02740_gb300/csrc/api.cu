// C ABI (include/sft.h): plan life cycle and the stream-ordered execution of Algorithm 1.
#include <stdint.h>
#include <string.h>

#include <new>
#include <string>

#include "sft_internal.h"

namespace sft {

namespace {
thread_local std::string g_last_error;
}

void set_error(const std::string& msg) { g_last_error = msg; }

}  // namespace sft

using sft::Plan;

struct sft_plan_s {
  Plan P;
};

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
  return SFT_OK;
}

sft_status sft_plan(sft_plan_t* out, int64_t N, int32_t s, const sft_variant* v, int32_t n_shifts,
                    const int64_t* primes, int32_t n_primes, const int32_t* small_moduli,
                    int32_t n_small) {
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
}

namespace {
void release_events(Plan& P) {
  for (cudaEvent_t e : P.events) cudaEventDestroy(e);
  P.events.clear();
  P.profiling = false;
  P.recorded = 0;
}
}  // namespace

sft_status sft_plan_destroy(sft_plan_t plan) {
  if (!plan) return SFT_OK;
  release_events(plan->P);
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

sft_status sft_execute(sft_plan_t plan, const void* f_dev, int64_t* out_freqs_dev,
                       void* out_coefs_dev, int32_t* out_count_dev, void* stream) {
  if (!plan || !f_dev) { sft::set_error("plan or f is NULL"); return SFT_EINVAL; }
  const bool any = out_freqs_dev || out_coefs_dev || out_count_dev;
  const bool all = out_freqs_dev && out_coefs_dev && out_count_dev;
  if (any && !all) { sft::set_error("outputs must be all NULL or all non-NULL"); return SFT_EINVAL; }
  sft::DevPlan d = plan->P.d;
  const uintptr_t fa = (uintptr_t)f_dev;
  if (fa % (d.input == SFT_IN_C64 ? 8 : 16) != 0) {
    sft::set_error("f is not aligned to its element size");
    return SFT_EINVAL;
  }
  d.aligned16 = (fa % 16) == 0;
  cudaStream_t st = (cudaStream_t)stream;
  double2* oc = reinterpret_cast<double2*>(out_coefs_dev);
  Plan& P = plan->P;
  cudaEvent_t* ev = nullptr;
  if (P.profiling && P.recorded < sft::kProfileCap)
    ev = &P.events[(size_t)P.recorded++ * (sft::kStages + 1)];
  auto mark = [&](int k) { if (ev) cudaEventRecord(ev[k], st); };
  const bool fp64 = d.prec == SFT_FP64;
  cudaError_t e = cudaMemsetAsync(d.counters, 0, (size_t)(d.nq + 4) * 4, st);
  mark(0);
  if (e == cudaSuccess) e = sft::launch_resample(d, f_dev, st);
  mark(1);
  if (e == cudaSuccess) e = sft::launch_bluestein(d, st);
  mark(2);
  if (e == cudaSuccess) e = sft::launch_identify(d, st);
  mark(3);
  if (e == cudaSuccess) e = sft::launch_vote(d, st);
  mark(4);
  if (e == cudaSuccess) e = sft::launch_select(d, out_count_dev, st);
  mark(5);
  if (e == cudaSuccess && !fp64) e = sft::launch_refine(d, st);
  if (e == cudaSuccess) e = sft::launch_finalize(d, out_freqs_dev, oc, st);
  mark(6);
  P.launches += 4 + sft::select_launches(d) + (fp64 ? 0 : sft::refine_launches(d)) +
                (out_freqs_dev ? sft::finalize_launches(d) : 0);
  if (e != cudaSuccess) {
    sft::set_error(std::string("CUDA launch failed: ") + cudaGetErrorString(e));
    return SFT_ECUDA;
  }
  return SFT_OK;
}

sft_status sft_plan_profile(sft_plan_t plan, int32_t enable) {
  if (!plan) { sft::set_error("plan is NULL"); return SFT_EINVAL; }
  Plan& P = plan->P;
  release_events(P);
  if (!enable) return SFT_OK;
  const size_t n = (size_t)sft::kProfileCap * (sft::kStages + 1);
  P.events.resize(n);
  for (size_t i = 0; i < n; ++i) {
    if (cudaEventCreate(&P.events[i]) != cudaSuccess) {
      P.events.resize(i);
      release_events(P);
      sft::set_error("cudaEventCreate failed");
      return SFT_ECUDA;
    }
  }
  P.profiling = true;
  return SFT_OK;
}

sft_status sft_plan_profile_read(sft_plan_t plan, double* stage_ms, int32_t* n_executions) {
  if (!plan || !stage_ms || !n_executions) { sft::set_error("NULL argument"); return SFT_EINVAL; }
  Plan& P = plan->P;
  for (int k = 0; k < sft::kStages; ++k) stage_ms[k] = 0.0;
  *n_executions = P.recorded;
  for (int r = 0; r < P.recorded; ++r) {
    cudaEvent_t* ev = &P.events[(size_t)r * (sft::kStages + 1)];
    for (int k = 0; k < sft::kStages; ++k) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev[k], ev[k + 1]) != cudaSuccess) {
        cudaGetLastError();
        sft::set_error("profile events not complete (synchronise the stream first)");
        return SFT_ECUDA;
      }
      stage_ms[k] += ms;
    }
  }
  P.recorded = 0;
  return SFT_OK;
}

int64_t sft_plan_launches(sft_plan_t plan) { return plan ? plan->P.launches : 0; }

sft_status sft_choose_moduli(int64_t N, int32_t s, int32_t K, double c_p, uint64_t seed,
                             int64_t* primes_out, int32_t* small_out, int32_t* n_small_out) {
  return sft::choose_moduli(N, s, K, c_p, seed, primes_out, small_out, n_small_out);
}

const char* sft_last_error(void) { return sft::g_last_error.c_str(); }

}  // extern "C"
