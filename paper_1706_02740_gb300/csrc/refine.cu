// Kernel (f): re-estimation of the s returned coefficients (FP32 path).
//
// The bulk path's length-p measurements come from FP32 chirp convolutions whose rounding is spread
// over every bin.  For the s winners only, each needed bin
//     Y_j[b] = (1/p_j) sum_k h_q(-pi + 2 pi k / p_j) e^{-2 pi i k b / p_j},   b = w mod p_j,
// is recomputed directly from the same filtered samples with twiddles e^{-2 pi i ((k b) mod p_j) / p_j}
// taken as products of two exactly rounded table entries.
//
// Work layout: one CTA of kReThreads threads per (shift, prime, chunk of kReChunk samples).  The
// CTA stages its chunk and the prime's twiddle table in shared memory, and each thread sums the
// chunk against one winner's twiddles in blocks of 16 terms: the block's twiddles factor as
// w^{(k0 + 16 m) b} w^{j b}, so a thread reads its 16 powers w^{j b} once per chunk and one block
// factor per 16 terms (exactly rounded table entries both), takes FMA sums within blocks and adds
// the block values with compensation (Neumaier), in FP32.  The chunk partials, kept as
// (sum, compensation) pairs, are combined exactly enough in double-single arithmetic.  The
// componentwise medians (eq. GSFT_Estimate), the sign (-1)^w and the division by g_hat_{w - q}
// (Lemma Periodic_Gaussian_FC) are done in FP64, spread over many CTAs.  All integer indexing is
// 32-bit.
#include <algorithm>

#include "checks.cuh"
#include "cplx.cuh"
#include "select_sort.cuh"
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

// Error-free two-sum in FP32 (Knuth): a + b = s + e exactly.
__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ int mod_p32(int64_t w, int p) {
  const int r = (int)w % p;
  return r < 0 ? r + p : r;
}

// Winner indices grouped by shift (one CTA per signal), for the re-estimation CTAs.
__global__ void __launch_bounds__(256) group_winners_kernel(BatchView bv) {
  pdl_begin();
  __shared__ int cnt[kMaxQ], cur[kMaxQ];
  int lb, nb;
  const DevPlan& d = bv.plans[batch_signal(bv, lb, nb)];
  const int n = d.counters[d.nq + 2];
  if (threadIdx.x < kMaxQ) cnt[threadIdx.x] = 0;
  __syncthreads();
  for (int r = threadIdx.x; r < n; r += 256) atomicAdd(&cnt[d.winners[r].qi], 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int q = 0; q < d.nq; ++q) {
      d.woff[q] = acc;
      cur[q] = acc;
      acc += cnt[q];
    }
    d.woff[d.nq] = acc;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < n; r += 256) d.wlist[atomicAdd(&cur[d.winners[r].qi], 1)] = r;
}

__global__ void __launch_bounds__(kReThreads) reestimate_kernel(BatchView bv) {
  pdl_begin();
  // [kReChunk] samples of this chunk, then the prime's [p] twiddles: each thread walks its own
  // residue sequence (k b) mod p, so the table reads scatter across the warp; shared memory serves
  // them with a few bank conflicts where the cached global table would take one line per lane.
  extern __shared__ float2 sm_re[];
  int lb, nb;
  const DevPlan& d = bv.plans[batch_signal(bv, lb, nb)];
  const int qk = lb / d.nchunk;
  const int c = lb - qk * d.nchunk;
  const int qi = qk / d.K;
  const int jj = qk - qi * d.K;
  const int beg = d.woff[qi], cnt = d.woff[qi + 1] - beg;
  if (cnt == 0) return;
  const int p = d.p[jj];
  const int k0 = c * kReChunk;
  const int klen = max(0, min(kReChunk, p - k0));
  // CTA-uniform checks (the checked build): the shift's winner range and the chunk of samples
  if (!index_ok(d, beg, d.s, SFT_SITE_REESTIMATE) || !index_ok(d, beg + cnt - 1, d.s, SFT_SITE_REESTIMATE) ||
      !index_ok(d, (int64_t)qi * d.m + d.nodeoff[jj] + k0 + max(klen, 1) - 1, (int64_t)d.nq * d.m,
                SFT_SITE_REESTIMATE))
    return;
  float2* S = sm_re;
  float2* Wt = sm_re + kReChunk;
  const float2* src = reinterpret_cast<const float2*>(d.samples) + (int64_t)qi * d.m + d.nodeoff[jj];
  for (int i = threadIdx.x; i < klen; i += kReThreads) S[i] = src[k0 + i];
  const float2* Wp = d.wp32 + (int64_t)jj * d.pmax;
  for (int i = threadIdx.x; i < p; i += kReThreads) Wt[i] = __ldg(Wp + i);
  __syncthreads();
  float4* part = reinterpret_cast<float4*>(d.ybuf);
  const float4* S4 = reinterpret_cast<const float4*>(S);
  for (int t = threadIdx.x; t < cnt; t += kReThreads) {
    const int r = d.wlist[beg + t];
    if (!index_ok(d, r, d.s, SFT_SITE_REESTIMATE)) continue;
    const int b = mod_p32(d.winners[r].w, p);
    // The chunk's sum in blocks of 16 consecutive k = k0 + 16 m + j:
    //     sum_m w^{(k0 + 16 m) b} * sum_{j<16} h_{k0 + 16 m + j} w^{j b},   w = e^{-2 pi i / p},
    // both factors exactly rounded table entries.  The inner sums are plain FMA chains of at most
    // 16 products; the block values are added with compensation.  Per block the rounding is a few
    // ulps of 16 terms, so the partial stays within ~eps * sqrt(p) * |h| of exact.
    float2 R[16];
    {
      int ij = 0;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        R[j] = Wt[ij];
        ij += b;
        if (ij >= p) ij -= p;
      }
    }
    int ib = (k0 * b) % p;                        // k0 b < 2^26: 32-bit
    const int b16 = (16 * b) % p;
    float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;
    for (int kb = 0; kb < klen; kb += 16) {
      float ur0 = 0.f, ui0 = 0.f, ur1 = 0.f, ui1 = 0.f;
      if (kb + 16 <= klen) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float4 h = S4[(kb >> 1) + q];     // h_{2q}, h_{2q+1} of this block
          const float2 r0 = R[2 * q], r1 = R[2 * q + 1];
          ur0 = fmaf(h.x, r0.x, ur0);
          ur0 = fmaf(-h.y, r0.y, ur0);
          ui0 = fmaf(h.x, r0.y, ui0);
          ui0 = fmaf(h.y, r0.x, ui0);
          ur1 = fmaf(h.z, r1.x, ur1);
          ur1 = fmaf(-h.w, r1.y, ur1);
          ui1 = fmaf(h.z, r1.y, ui1);
          ui1 = fmaf(h.w, r1.x, ui1);
        }
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          if (kb + j < klen) {
            const float2 h = S[kb + j];
            ur0 = fmaf(h.x, R[j].x, ur0);
            ur0 = fmaf(-h.y, R[j].y, ur0);
            ui0 = fmaf(h.x, R[j].y, ui0);
            ui0 = fmaf(h.y, R[j].x, ui0);
          }
        }
      }
      const float ur = ur0 + ur1, ui = ui0 + ui1;
      const float2 T = Wt[ib];
      neumaier_add(sr, cr, fmaf(ur, T.x, -ui * T.y));
      neumaier_add(si, ci, fmaf(ur, T.y, ui * T.x));
      ib += b16;
      if (ib >= p) ib -= p;
    }
    // partials of (winner, prime) are contiguous over the chunks: [r][K][nchunk]
    part[((int64_t)r * d.K + jj) * d.nchunk + c] = make_float4(sr, cr, si, ci);
  }
}

// Error-free two-sum in FP32 (Knuth): a + b = s + e exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Double-single sum, in chunk order, of one (winner, prime) bin's nc chunk partials (hi, lo) for
// the real and imaginary parts, returned in FP64; the loads of four chunks are issued together.
__device__ __forceinline__ void combine_chunks(const float4* pc, int nc, double& re, double& im) {
  float hr = 0.f, lr = 0.f, hi = 0.f, li = 0.f;
  for (int c0 = 0; c0 < nc; c0 += 4) {
    float4 v4[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v4[u] = c0 + u < nc ? pc[c0 + u] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (c0 + u >= nc) break;
      const float4 v = v4[u];
      float s, e;
      two_sum(hr, v.x, s, e);
      lr += e + v.y;
      two_sum(s, lr, hr, lr);
      two_sum(hi, v.z, s, e);
      li += e + v.w;
      two_sum(s, li, hi, li);
    }
  }
  re = (double)hr + (double)lr;
  im = (double)hi + (double)li;
}

// The refined coefficient of winner r from its K bins (FP64): componentwise medians, the sign
// (-1)^w and the division by g_hat_{w - q}; written back into winners[r].
template <int KCAP>
__device__ __forceinline__ void finish_winner(const DevPlan& d, int r, double* re, double* im) {
  Pooled pw = d.winners[r];
  const double mre = median_of<KCAP>(re, d.K);
  const double mim = median_of<KCAP>(im, d.K);
  const double sg = (pw.w & 1) ? -1.0 : 1.0;
  const double x = d.c1 * (double)(pw.w - d.q[pw.qi]);
  const double inv_ghat = kSqrt2Pi * exp(0.5 * x * x);
  pw.cre = sg * mre * inv_ghat;
  pw.cim = sg * mim * inv_ghat;
  d.winners[r] = pw;
}

// Refined coefficients of the kRefineThreads winners of a CTA, one thread per winner (any K up to
// kMaxK).
template <int KCAP>
__global__ void __launch_bounds__(kRefineThreads) refine_values_kernel(BatchView bv) {
  pdl_begin();
  int lb, nb;
  const DevPlan& d = bv.plans[batch_signal(bv, lb, nb)];
  const int n = d.counters[d.nq + 2];
  const int r = lb * kRefineThreads + threadIdx.x;
  if (r >= n) return;
  double re[KCAP], im[KCAP];
  const float4* part = reinterpret_cast<const float4*>(d.ybuf);
  for (int jj = 0; jj < d.K; ++jj) {
    const int p = d.p[jj];
    const int nc = (p + kReChunk - 1) / kReChunk;
    combine_chunks(part + ((int64_t)r * d.K + jj) * d.nchunk, nc, re[jj], im[jj]);
    const double inv_p = 1.0 / (double)p;
    re[jj] *= inv_p;
    im[jj] *= inv_p;
  }
  finish_winner<KCAP>(d, r, re, im);
}

// The same for K <= kFewK with the CTA's kRefineThreads x K (winner, prime) bins spread over
// kRefineFewThreads threads, so the chunk loads of all of a winner's bins are in flight at once
// (a lone transform's thousand winners otherwise wait on K rounds of loads each); the bins meet in
// shared memory and one thread per winner finishes it.  Same arithmetic, same bits.
constexpr int kRefineFewThreads = 256;
__global__ void __launch_bounds__(kRefineFewThreads) refine_values_few_kernel(BatchView bv) {
  pdl_begin();
  __shared__ double sre[kRefineThreads * kFewK], sim[kRefineThreads * kFewK];
  int lb, nb;
  const DevPlan& d = bv.plans[batch_signal(bv, lb, nb)];
  const int n = d.counters[d.nq + 2];
  const int r0 = lb * kRefineThreads;
  const int K = d.K;
  const float4* part = reinterpret_cast<const float4*>(d.ybuf);
  for (int q = threadIdx.x; q < kRefineThreads * K; q += kRefineFewThreads) {
    const int wl = q / K, jj = q - wl * K;
    if (r0 + wl >= n) continue;
    const int p = d.p[jj];
    const int nc = (p + kReChunk - 1) / kReChunk;
    double re, im;
    combine_chunks(part + ((int64_t)(r0 + wl) * K + jj) * d.nchunk, nc, re, im);
    const double inv_p = 1.0 / (double)p;
    sre[wl * kFewK + jj] = re * inv_p;
    sim[wl * kFewK + jj] = im * inv_p;
  }
  __syncthreads();
  const int wl = threadIdx.x;
  if (wl >= kRefineThreads || r0 + wl >= n) return;
  double re[kFewK], im[kFewK];
  for (int jj = 0; jj < K; ++jj) {
    re[jj] = sre[wl * kFewK + jj];
    im[jj] = sim[wl * kFewK + jj];
  }
  finish_winner<kFewK>(d, r0 + wl, re, im);
}

}  // namespace

cudaError_t launch_refine(const BatchView& bv, const LaunchSet& ls, cudaStream_t st) {
  BatchView v = bv;
  v.blk = ls.blk[kStOne];
  (void)launch_pdl(group_winners_kernel, ls.blocks[kStOne], 256, 0, st, v);
  v.blk = ls.blk[kStReest];
  const size_t smem = (size_t)(kReChunk + ls.pmax) * sizeof(float2);
  const cudaError_t e = ensure_dynamic_smem<reestimate_kernel>(smem);
  if (e != cudaSuccess) return e;
  (void)launch_pdl(reestimate_kernel, ls.blocks[kStReest], kReThreads, smem, st, v);
  v.blk = ls.blk[kStRefine];
  if (ls.kmax <= kFewK)
    (void)launch_pdl(refine_values_few_kernel, ls.blocks[kStRefine], kRefineFewThreads, 0, st, v);
  else
    (void)launch_pdl(refine_values_kernel<kMaxK>, ls.blocks[kStRefine], kRefineThreads, 0, st, v);
  return cudaGetLastError();
}

}  // namespace sft
