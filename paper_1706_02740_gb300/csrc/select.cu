// Kernel (e): selections of Algorithm 1.
//
// shift_select: per shift q, R_temp = the s voted frequencies of largest |z| (ties: smaller w);
// those inside [q - L, q + L) and B are divided by the modulated filter's Fourier coefficient
// g_hat_{w - q} = e^{-c1^2 (w - q)^2 / 2} / sqrt(2 pi) (Lemma Periodic_Gaussian_FC) and pooled.
// global_select: the s pooled pairs of largest |c| (ties: smaller w), in rank order.
//
// Lists are short (about s entries per shift), so each element's rank is counted directly against
// every other element of its list (keys are distinct: frequencies are distinct within a list),
// with the list staged through shared memory in tiles.  Ranks are exact and deterministic whatever
// order the atomics of the vote kernel produced.
#include <algorithm>

#include "cplx.cuh"
#include "sft_internal.h"

namespace sft {

namespace {

constexpr int kTile = 256;
constexpr double kSqrt2Pi = 2.5066282746310002;  // sqrt(2 pi)

// a precedes b: larger magnitude first, then the smaller frequency
__device__ __forceinline__ bool precedes(double ma, int64_t wa, double mb, int64_t wb) {
  return ma > mb || (ma == mb && wa < wb);
}

__global__ void __launch_bounds__(kTile) shift_select_kernel(DevPlan d) {
  __shared__ double sm[kTile];
  __shared__ int64_t sw[kTile];
  const int qi = blockIdx.y;
  const int n = min(d.counters[qi], d.vcap);
  const Voted* V = d.voted + (int64_t)qi * d.vcap;
  const int64_t q = d.q[qi];
  for (int base = blockIdx.x * kTile; base < n; base += gridDim.x * kTile) {
    const int i = base + threadIdx.x;
    double mi = 0;
    int64_t wi = 0;
    Voted vi;
    if (i < n) {
      vi = V[i];
      mi = vi.zre * vi.zre + vi.zim * vi.zim;
      wi = vi.w;
    }
    int rank = 0;
    for (int t0 = 0; t0 < n; t0 += kTile) {
      __syncthreads();
      if (t0 + threadIdx.x < n) {
        const Voted vt = V[t0 + threadIdx.x];
        sm[threadIdx.x] = vt.zre * vt.zre + vt.zim * vt.zim;
        sw[threadIdx.x] = vt.w;
      }
      __syncthreads();
      const int lim = min(kTile, n - t0);
      if (i < n)
        for (int k = 0; k < lim; ++k) rank += precedes(sm[k], sw[k], mi, wi) ? 1 : 0;
    }
    if (i < n && rank < d.s) {
      const int64_t lo = -((d.N + 1) / 2) + 1, hi = d.N / 2;
      if (wi >= q - d.L && wi < q + d.L && wi >= lo && wi <= hi) {
        const double x = d.c1 * (double)(wi - q);
        const double inv_ghat = kSqrt2Pi * exp(0.5 * x * x);
        Pooled pr;
        pr.w = wi;
        pr.cre = vi.zre * inv_ghat;
        pr.cim = vi.zim * inv_ghat;
        pr.qi = qi;
        pr.pad = 0;
        const int slot = atomicAdd(d.counters + d.nq, 1);
        if (slot < d.nq * d.s) d.pool[slot] = pr;
      }
    }
  }
}

// Rank the pool; write winners[rank] and, when out_w is given, the final output directly.
__global__ void __launch_bounds__(kTile) global_select_kernel(DevPlan d, int64_t* out_w,
                                                              double2* out_c, int32_t* out_n) {
  __shared__ double sm[kTile];
  __shared__ int64_t sw[kTile];
  const int n = min(d.counters[d.nq], d.nq * d.s);
  const int limit = max(n, d.s);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    d.counters[d.nq + 2] = min(n, d.s);
    if (out_n) *out_n = min(n, d.s);
  }
  for (int base = blockIdx.x * kTile; base < limit; base += gridDim.x * kTile) {
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
    for (int t0 = 0; t0 < n; t0 += kTile) {
      __syncthreads();
      if (t0 + threadIdx.x < n) {
        const Pooled pt = d.pool[t0 + threadIdx.x];
        sm[threadIdx.x] = pt.cre * pt.cre + pt.cim * pt.cim;
        sw[threadIdx.x] = pt.w;
      }
      __syncthreads();
      const int lim = min(kTile, n - t0);
      if (i < n)
        for (int k = 0; k < lim; ++k) rank += precedes(sm[k], sw[k], mi, wi) ? 1 : 0;
    }
    if (i < n && rank < d.s) {
      d.winners[rank] = pi;
      if (out_w) {
        out_w[rank] = pi.w;
        out_c[rank] = make_double2(pi.cre, pi.cim);
      }
    }
    if (out_w && i >= n && i < d.s) {
      out_w[i] = 0;
      out_c[i] = make_double2(0.0, 0.0);
    }
  }
}

}  // namespace

cudaError_t launch_select(const DevPlan& d, int64_t* out_w, double2* out_c, int32_t* out_n,
                          cudaStream_t st) {
  const int chunks = (int)std::min<int64_t>((d.vcap + kTile - 1) / kTile, 64);
  shift_select_kernel<<<dim3(chunks, d.nq), kTile, 0, st>>>(d);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t lim = std::max<int64_t>((int64_t)d.nq * d.s, d.s);
  const int g2 = (int)std::min<int64_t>((lim + kTile - 1) / kTile, 256);
  global_select_kernel<<<g2, kTile, 0, st>>>(d, out_w, out_c, out_n);
  return cudaGetLastError();
}

}  // namespace sft
