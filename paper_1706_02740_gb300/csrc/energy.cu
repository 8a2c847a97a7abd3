// Residual-energy check (sft_residual_energy): rho = 1 - sum_r |c_r|^2 / (||f||^2 / N), from
// Parseval's identity for f-hat = F f with F's 1/N normalisation (Section 2).
//
// Kernel 1: kEnergyBlocks CTAs stride over f.  A complex64 input accumulates |f_i|^2 per thread
// in double-single FP32 (each square split exactly with an FMA, sums carried with Knuth's
// two-sum), so no FP64 instruction touches the N-element stream; a complex128 input accumulates
// in FP64.  Each CTA reduces its threads in FP64 in a fixed tree and writes one partial.
// Kernel 2: one CTA adds the partials and the s returned |c_r|^2 in FP64, in index order.
#include "sft_internal.h"

namespace sft {

namespace {

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// (hi, lo) += x^2 + y^2 with the squares' rounding errors kept.
__device__ __forceinline__ void add_norm(float x, float y, float& hi, float& lo) {
  const float px = x * x, ex = fmaf(x, x, -px);
  const float py = y * y, ey = fmaf(y, y, -py);
  float s, t, u, v;
  two_sum(px, py, s, t);
  two_sum(hi, s, u, v);
  hi = u;
  lo += (v + t) + (ex + ey);
}

// Sum of the block's values in FP64, fixed order (shuffle tree, then one warp).
__device__ double block_sum(double v) {
  __shared__ double warp_part[kEnergyThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) warp_part[wid] = v;
  __syncthreads();
  v = 0.0;
  if (wid == 0) {
    v = lane < kEnergyThreads / 32 ? warp_part[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  return v;
}

__global__ void __launch_bounds__(kEnergyThreads) energy_partial_kernel(const DevPlan* dp,
                                                                       const void* f) {
  pdl_begin();
  const DevPlan& d = *dp;
  const int64_t N = d.N;
  const int64_t tid = (int64_t)blockIdx.x * kEnergyThreads + threadIdx.x;
  const int64_t stride = (int64_t)kEnergyBlocks * kEnergyThreads;
  double v;
  if (d.input == SFT_IN_C64) {
    float hi = 0.f, lo = 0.f;
    const float2* f2 = static_cast<const float2*>(f);
    if ((reinterpret_cast<uintptr_t>(f) & 15) == 0) {
      const float4* f4 = static_cast<const float4*>(f);
      const int64_t n4 = N >> 1;
      for (int64_t i = tid; i < n4; i += stride) {
        const float4 a = __ldg(f4 + i);
        add_norm(a.x, a.y, hi, lo);
        add_norm(a.z, a.w, hi, lo);
      }
      if ((N & 1) && tid == 0) {
        const float2 a = __ldg(f2 + N - 1);
        add_norm(a.x, a.y, hi, lo);
      }
    } else {
      for (int64_t i = tid; i < N; i += stride) {
        const float2 a = __ldg(f2 + i);
        add_norm(a.x, a.y, hi, lo);
      }
    }
    v = (double)hi + (double)lo;
  } else {
    const double2* f2 = static_cast<const double2*>(f);
    v = 0.0;
    for (int64_t i = tid; i < N; i += stride) {
      const double2 a = __ldg(f2 + i);
      v = fma(a.x, a.x, fma(a.y, a.y, v));
    }
  }
  v = block_sum(v);
  if (threadIdx.x == 0) d.epart[blockIdx.x] = v;
}

__global__ void __launch_bounds__(kEnergyThreads) energy_final_kernel(const DevPlan* dp,
                                                                     const double2* coefs,
                                                                     const int32_t* count,
                                                                     double* out) {
  pdl_begin();
  const DevPlan& d = *dp;
  double e = threadIdx.x < kEnergyBlocks ? d.epart[threadIdx.x] : 0.0;
  e = block_sum(e);
  __syncthreads();
  const int n = min(max(*count, 0), d.s);
  double c = 0.0;
  for (int r = threadIdx.x; r < n; r += kEnergyThreads) {
    const double2 z = coefs[r];
    c = fma(z.x, z.x, fma(z.y, z.y, c));
  }
  c = block_sum(c);
  if (threadIdx.x == 0) {
    const double fhat2 = e / (double)d.N;
    *out = fhat2 > 0.0 ? 1.0 - c / fhat2 : 0.0;
  }
}

static_assert(kEnergyBlocks <= kEnergyThreads, "the final CTA reads one partial per thread");

}  // namespace

}  // namespace sft

extern "C" sft_status sft_residual_energy(sft_plan_t plan, const void* f_dev, const void* coefs_dev,
                                          const int32_t* count_dev, double* out_dev, void* stream) {
  using namespace sft;
  if (!plan || !f_dev || !coefs_dev || !count_dev || !out_dev) {
    set_error("sft_residual_energy: NULL argument");
    return SFT_EINVAL;
  }
  Plan* P = sft_plan_internal(plan);
  if ((uintptr_t)f_dev % (P->d.input == SFT_IN_C64 ? 8 : 16) || (uintptr_t)coefs_dev % 16 ||
      (uintptr_t)out_dev % 8) {
    set_error("sft_residual_energy: misaligned buffer");
    return SFT_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  (void)launch_pdl(energy_partial_kernel, kEnergyBlocks, kEnergyThreads, 0, st, P->d_dev, f_dev);
  (void)launch_pdl(energy_final_kernel, 1, kEnergyThreads, 0, st, P->d_dev,
                   static_cast<const double2*>(coefs_dev), count_dev, out_dev);
  P->launches += 2;
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("sft_residual_energy: launch failed: ") + cudaGetErrorString(e));
    return SFT_ECUDA;
  }
  return SFT_OK;
}
