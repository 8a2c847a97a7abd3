// Kernel (f): re-estimation of the s returned coefficients (FP32 path).
//
// The bulk path's length-p measurements come from FP32 chirp convolutions whose rounding is spread
// over every bin.  For the s winners only, each needed bin
//     Y_j[b] = (1/p_j) sum_k h_q(-pi + 2 pi k / p_j) e^{-2 pi i k b / p_j},   b = w mod p_j,
// is recomputed directly from the same filtered samples with exactly rounded twiddles
// e^{-2 pi i ((k b) mod p_j) / p_j} and compensated (Neumaier) FP32 accumulation per lane, the
// lanes' partial sums combined in FP64.  The componentwise medians (eq. GSFT_Estimate), the sign
// (-1)^w and the division by g_hat_{w - q} (Lemma Periodic_Gaussian_FC) are then done in FP64, and
// the s pairs are re-ranked by the refined magnitudes (ties: smaller w).
#include <algorithm>

#include "cplx.cuh"
#include "sft_internal.h"

namespace sft {

namespace {

constexpr double kSqrt2Pi = 2.5066282746310002;

__device__ __forceinline__ void neumaier_add(float& s, float& c, float x) {
  const float t = s + x;
  if (fabsf(s) >= fabsf(x)) c += (s - t) + x;
  else c += (x - t) + s;
  s = t;
}

__global__ void __launch_bounds__(256) reestimate_kernel(DevPlan d) {
  const int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  const int n = d.counters[d.nq + 2];
  const int r = warp / d.K, jj = warp - (warp / d.K) * d.K;
  if (r >= n) return;
  const Pooled pw = d.winners[r];
  const int p = d.p[jj];
  const int b = (int)fmod64(pw.w, p);
  const float2* S = reinterpret_cast<const float2*>(d.samples) + (int64_t)pw.qi * d.m + d.nodeoff[jj];
  const float2* Wp = d.wp32 + (int64_t)jj * d.pmax;
  int idx = (int)(((int64_t)lane * b) % p);
  const int step = (int)(((int64_t)32 * b) % p);
  float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;
  for (int k = lane; k < p; k += 32) {
    const float2 a = S[k];
    const float2 w = __ldg(Wp + idx);
    neumaier_add(sr, cr, fmaf(a.x, w.x, -a.y * w.y));
    neumaier_add(si, ci, fmaf(a.x, w.y, a.y * w.x));
    idx += step;
    if (idx >= p) idx -= p;
  }
  double re = (double)sr + (double)cr, im = (double)si + (double)ci;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  if (lane == 0) d.ybuf[(int64_t)r * d.K + jj] = make_double2(re / p, im / p);
}

__device__ __forceinline__ void sort_d(double* a, int n) {
  for (int i = 1; i < n; ++i) {
    double v = a[i];
    int k = i - 1;
    while (k >= 0 && a[k] > v) { a[k + 1] = a[k]; --k; }
    a[k + 1] = v;
  }
}

__global__ void __launch_bounds__(256) finalize_kernel(DevPlan d) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = d.counters[d.nq + 2];
  if (r >= n) return;
  Pooled pw = d.winners[r];
  double re[kMaxK], im[kMaxK];
  for (int jj = 0; jj < d.K; ++jj) {
    const double2 y = d.ybuf[(int64_t)r * d.K + jj];
    re[jj] = y.x;
    im[jj] = y.y;
  }
  sort_d(re, d.K);
  sort_d(im, d.K);
  const int K = d.K;
  const double mre = (K & 1) ? re[K / 2] : 0.5 * (re[K / 2 - 1] + re[K / 2]);
  const double mim = (K & 1) ? im[K / 2] : 0.5 * (im[K / 2 - 1] + im[K / 2]);
  const double sg = (pw.w & 1) ? -1.0 : 1.0;
  const double x = d.c1 * (double)(pw.w - d.q[pw.qi]);
  const double inv_ghat = kSqrt2Pi * exp(0.5 * x * x);
  pw.cre = sg * mre * inv_ghat;
  pw.cim = sg * mim * inv_ghat;
  d.pool[r] = pw;   // the pool is free after the global selection; reuse it for refined winners
}

__global__ void __launch_bounds__(256) rerank_kernel(DevPlan d, int64_t* out_w, double2* out_c) {
  __shared__ double sm[256];
  __shared__ int64_t sw[256];
  const int n = d.counters[d.nq + 2];
  const int limit = max(n, d.s);
  for (int base = blockIdx.x * 256; base < limit; base += gridDim.x * 256) {
    const int i = base + threadIdx.x;
    double mi = 0;
    int64_t wi = 0;
    Pooled pi;
    if (i < n) {
      pi = d.pool[i];
      mi = pi.cre * pi.cre + pi.cim * pi.cim;
      wi = pi.w;
    }
    int rank = 0;
    for (int t0 = 0; t0 < n; t0 += 256) {
      __syncthreads();
      if (t0 + threadIdx.x < n) {
        const Pooled pt = d.pool[t0 + threadIdx.x];
        sm[threadIdx.x] = pt.cre * pt.cre + pt.cim * pt.cim;
        sw[threadIdx.x] = pt.w;
      }
      __syncthreads();
      const int lim = min(256, n - t0);
      if (i < n)
        for (int k = 0; k < lim; ++k)
          rank += (sm[k] > mi || (sm[k] == mi && sw[k] < wi)) ? 1 : 0;
    }
    if (i < n) {
      out_w[rank] = pi.w;
      out_c[rank] = make_double2(pi.cre, pi.cim);
    } else if (i < d.s) {
      out_w[i] = 0;
      out_c[i] = make_double2(0.0, 0.0);
    }
  }
}

}  // namespace

cudaError_t launch_refine(const DevPlan& d, int64_t* out_w, double2* out_c, int32_t* out_n,
                          cudaStream_t st) {
  (void)out_n;
  const int64_t warps = (int64_t)d.s * d.K;
  reestimate_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(d);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  finalize_kernel<<<(unsigned)((d.s + 255) / 256), 256, 0, st>>>(d);
  e = cudaGetLastError();
  if (e != cudaSuccess || !out_w) return e;
  const int g = (int)std::min<int64_t>((d.s + 255) / 256, 256);
  rerank_kernel<<<g, 256, 0, st>>>(d, out_w, out_c);
  return cudaGetLastError();
}

}  // namespace sft
