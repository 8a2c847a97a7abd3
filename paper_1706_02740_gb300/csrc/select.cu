// Kernel (e): selections of Algorithm 1.
//
// shift_select: per shift q, R_temp = the s voted frequencies of largest |z| (ties: smaller w);
// those inside [q - L, q + L) and B are divided by the modulated filter's Fourier coefficient
// g_hat_{w - q} = e^{-c1^2 (w - q)^2 / 2} / sqrt(2 pi) (Lemma Periodic_Gaussian_FC) and pooled.
// global_select: the s pooled pairs of largest |c| (ties: smaller w) become the winners.
// finalize: the winners in order, |c| descending, ties by the smaller frequency.
//
// Only membership matters at the first two points (the winners are put in order once, at the end),
// so a list of at most s entries is taken whole without sorting.  A longer list of up to kSortCap
// entries is sorted by one CTA (register/shuffle bitonic network on integer keys); a longer one
// still falls back to counting each element's rank against the whole list.  The kernels of both
// branches are launched and each checks the list length on the device.
#include <algorithm>

#include "checks.cuh"
#include "cplx.cuh"
#include "select_sort.cuh"
#include "sft_internal.h"

namespace sft {

namespace {

__device__ __forceinline__ bool in_band(const DevPlan& d, int64_t w, int64_t q) {
  const int64_t lo = -((d.N + 1) / 2) + 1, hi = d.N / 2;
  return w >= q - d.L && w < q + d.L && w >= lo && w <= hi;
}

// 1 / g_hat_{w - q} = sqrt(2 pi) e^{c1^2 (w - q)^2 / 2}; FP32 on the FP32 path (the winners are
// re-estimated and divided again in FP64 later), FP64 on the FP64 path.
__device__ __forceinline__ void pool_append(const DevPlan& d, const Voted& v, int qi) {
  const int64_t q = d.q[qi];
  if (!in_band(d, v.w, q)) return;
  Pooled pr;
  if (d.prec == SFT_FP32) {
    const float x = d.c1f * (float)(v.w - q);
    const float inv_ghat = 2.50662827463f * expf(0.5f * x * x);
    pr.cre = (double)((float)v.zre * inv_ghat);
    pr.cim = (double)((float)v.zim * inv_ghat);
  } else {
    const double x = d.c1 * (double)(v.w - q);
    const double inv_ghat = 2.5066282746310002 * exp(0.5 * x * x);
    pr.cre = v.zre * inv_ghat;
    pr.cim = v.zim * inv_ghat;
  }
  pr.w = v.w;
  pr.qi = qi;
  pr.pad = 0;
  const int slot = atomicAdd(d.counters + d.nq, 1);
  if (slot < d.nq * d.s) d.pool[slot] = pr;
  else record_fault(d, SFT_FAULT_POOL_FULL, SFT_SITE_NONE);
}

__device__ __forceinline__ uint64_t vkey(const Voted& v) {
  return mag_key(v.zre * v.zre + v.zim * v.zim);
}
__device__ __forceinline__ uint64_t pkey(const Pooled& p) {
  return mag_key(p.cre * p.cre + p.cim * p.cim);
}

__global__ void __launch_bounds__(kSortThreads) shift_select(BatchView bv) {
  pdl_begin();
  int lb, nb;
  const DevPlan& d = bv.plans[batch_signal(bv, lb, nb)];
  const int qi = lb;
  const int n = min(d.counters[qi], d.vcap);
  const Voted* V = d.voted + (int64_t)qi * d.vcap;
  if (n <= d.s) {
    for (int i = threadIdx.x; i < n; i += kSortThreads) pool_append(d, V[i], qi);
    return;
  }
  if (n > kSortCap) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Rec* S = reinterpret_cast<Rec*>(smem_raw);
  const int slots = sort_slots(n);
  for (int i = threadIdx.x; i < slots; i += kSortThreads) {
    if (i < n) {
      const Voted v = V[i];
      S[i].m = vkey(v);
      S[i].w = v.w;
      S[i].ix = i;
      S[i].pad = 0;
    } else {
      S[i] = pad_rec(i);
    }
  }
  __syncthreads();
  sort_smem(S, n);
  for (int i = threadIdx.x; i < d.s; i += kSortThreads) pool_append(d, V[S[i].ix], qi);
}

__global__ void __launch_bounds__(kRankThreads) shift_select_rank(BatchView bv) {
  pdl_begin();
  __shared__ uint64_t sm[kRankThreads];
  __shared__ int64_t sw[kRankThreads];
  int lb, nb;
  const DevPlan& d = bv.plans[batch_signal(bv, lb, nb)];
  const int chunks = nb / d.nq;
  const int qi = lb / chunks, chunk = lb - qi * chunks;
  const int n = min(d.counters[qi], d.vcap);
  if (n <= kSortCap || n <= d.s) return;
  const Voted* V = d.voted + (int64_t)qi * d.vcap;
  for (int base = chunk * kRankThreads; base < n; base += chunks * kRankThreads) {
    const int i = base + threadIdx.x;
    Voted vi;
    uint64_t mi = 0;
    int64_t wi = 0;
    if (i < n) {
      vi = V[i];
      mi = vkey(vi);
      wi = vi.w;
    }
    int rank = 0;
    for (int t0 = 0; t0 < n; t0 += kRankThreads) {
      __syncthreads();
      if (t0 + threadIdx.x < n) {
        const Voted vt = V[t0 + threadIdx.x];
        sm[threadIdx.x] = vkey(vt);
        sw[threadIdx.x] = vt.w;
      }
      __syncthreads();
      const int lim = min(kRankThreads, n - t0);
      if (i < n)
        for (int k = 0; k < lim; ++k) rank += precedes(sm[k], sw[k], mi, wi) ? 1 : 0;
    }
    if (i < n && rank < d.s) pool_append(d, vi, qi);
  }
}

__device__ __forceinline__ void set_count(const DevPlan& d, int n, int32_t* out_n, int lb) {
  if (lb == 0 && threadIdx.x == 0) {
    d.counters[d.nq + 2] = min(n, d.s);
    if (out_n) *out_n = min(n, d.s);
  }
}

__global__ void __launch_bounds__(kSortThreads) global_select(BatchView bv) {
  pdl_begin();
  int lb, nb;
  const int b = batch_signal(bv, lb, nb);
  const DevPlan& d = bv.plans[b];
  int32_t* out_n = batch_out_n(bv, b);
  const int n = min(d.counters[d.nq], d.nq * d.s);
  if (n <= d.s) {
    set_count(d, n, out_n, lb);
    for (int i = threadIdx.x; i < n; i += kSortThreads) d.winners[i] = d.pool[i];
    return;
  }
  if (n > kSortCap) return;
  set_count(d, n, out_n, lb);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Rec* S = reinterpret_cast<Rec*>(smem_raw);
  const int slots = sort_slots(n);
  for (int i = threadIdx.x; i < slots; i += kSortThreads) {
    if (i < n) {
      const Pooled p = d.pool[i];
      S[i].m = pkey(p);
      S[i].w = p.w;
      S[i].ix = i;
      S[i].pad = 0;
    } else {
      S[i] = pad_rec(i);
    }
  }
  __syncthreads();
  sort_smem(S, n);
  for (int i = threadIdx.x; i < d.s; i += kSortThreads) d.winners[i] = d.pool[S[i].ix];
}

__global__ void __launch_bounds__(kRankThreads) global_select_rank(BatchView bv) {
  pdl_begin();
  __shared__ uint64_t sm[kRankThreads];
  __shared__ int64_t sw[kRankThreads];
  int lb, nb;
  const int b = batch_signal(bv, lb, nb);
  const DevPlan& d = bv.plans[b];
  const int n = min(d.counters[d.nq], d.nq * d.s);
  if (n <= kSortCap || n <= d.s) return;
  set_count(d, n, batch_out_n(bv, b), lb);
  for (int base = lb * kRankThreads; base < n; base += nb * kRankThreads) {
    const int i = base + threadIdx.x;
    Pooled pi;
    uint64_t mi = 0;
    int64_t wi = 0;
    if (i < n) {
      pi = d.pool[i];
      mi = pkey(pi);
      wi = pi.w;
    }
    int rank = 0;
    for (int t0 = 0; t0 < n; t0 += kRankThreads) {
      __syncthreads();
      if (t0 + threadIdx.x < n) {
        const Pooled pt = d.pool[t0 + threadIdx.x];
        sm[threadIdx.x] = pkey(pt);
        sw[threadIdx.x] = pt.w;
      }
      __syncthreads();
      const int lim = min(kRankThreads, n - t0);
      if (i < n)
        for (int k = 0; k < lim; ++k) rank += precedes(sm[k], sw[k], mi, wi) ? 1 : 0;
    }
    if (i < n && rank < d.s) d.winners[rank] = pi;
  }
}

__global__ void __launch_bounds__(kSortThreads) finalize_sorted(BatchView bv) {
  pdl_begin();
  int lb, nb;
  const int b = batch_signal(bv, lb, nb);
  const DevPlan& d = bv.plans[b];
  int64_t* out_w = batch_out_w(bv, b);
  double2* out_c = batch_out_c(bv, b);
  const int n = d.counters[d.nq + 2];
  if (n > kSortCap || !out_w) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Rec* S = reinterpret_cast<Rec*>(smem_raw);
  const int slots = sort_slots(n);
  for (int i = threadIdx.x; i < slots; i += kSortThreads) {
    if (i < n) {
      const Pooled p = d.winners[i];
      S[i].m = pkey(p);
      S[i].w = p.w;
      S[i].ix = i;
      S[i].pad = 0;
    } else {
      S[i] = pad_rec(i);
    }
  }
  __syncthreads();
  sort_smem(S, n);
  for (int i = threadIdx.x; i < n; i += kSortThreads) {
    const Pooled p = d.winners[S[i].ix];
    out_w[i] = p.w;
    out_c[i] = make_double2(p.cre, p.cim);
  }
  for (int i = n + threadIdx.x; i < d.s; i += kSortThreads) {
    out_w[i] = 0;
    out_c[i] = make_double2(0.0, 0.0);
  }
}

__global__ void __launch_bounds__(kRankThreads) finalize_rank(BatchView bv) {
  pdl_begin();
  __shared__ uint64_t sm[kRankThreads];
  __shared__ int64_t sw[kRankThreads];
  int lb, nb;
  const int b = batch_signal(bv, lb, nb);
  const DevPlan& d = bv.plans[b];
  int64_t* out_w = batch_out_w(bv, b);
  double2* out_c = batch_out_c(bv, b);
  const int n = d.counters[d.nq + 2];
  if (n <= kSortCap || !out_w) return;
  const int limit = max(n, d.s);
  for (int base = lb * kRankThreads; base < limit; base += nb * kRankThreads) {
    const int i = base + threadIdx.x;
    Pooled pi;
    uint64_t mi = 0;
    int64_t wi = 0;
    if (i < n) {
      pi = d.winners[i];
      mi = pkey(pi);
      wi = pi.w;
    }
    int rank = 0;
    for (int t0 = 0; t0 < n; t0 += kRankThreads) {
      __syncthreads();
      if (t0 + threadIdx.x < n) {
        const Pooled pt = d.winners[t0 + threadIdx.x];
        sm[threadIdx.x] = pkey(pt);
        sw[threadIdx.x] = pt.w;
      }
      __syncthreads();
      const int lim = min(kRankThreads, n - t0);
      if (i < n)
        for (int k = 0; k < lim; ++k) rank += precedes(sm[k], sw[k], mi, wi) ? 1 : 0;
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

// Per-signal counters (voted counts, pool count, winner count) start at zero.
__global__ void __launch_bounds__(64) zero_kernel(BatchView bv) {
  pdl_begin();
  int lb, nb;
  const DevPlan& d = bv.plans[batch_signal(bv, lb, nb)];
  for (int i = threadIdx.x; i < d.nq + 4; i += 64) d.counters[i] = 0;
}


BatchView with_blk(const BatchView& bv, const LaunchSet& ls, int kind);

}  // namespace

namespace {
BatchView with_blk(const BatchView& bv, const LaunchSet& ls, int kind) {
  BatchView v = bv;
  v.blk = ls.blk[kind];
  return v;
}
}  // namespace

cudaError_t launch_zero(const BatchView& bv, const LaunchSet& ls, cudaStream_t st) {
  (void)launch_pdl(zero_kernel, ls.blocks[kStOne], 64, 0, st, with_blk(bv, ls, kStOne));
  return cudaGetLastError();
}

cudaError_t launch_select(const BatchView& bv, const LaunchSet& ls, cudaStream_t st, int* launched) {
  cudaError_t e = ensure_dynamic_smem<shift_select>(kSortSmem);
  if (e == cudaSuccess) e = ensure_dynamic_smem<global_select>(kSortSmem);
  if (e != cudaSuccess) return e;
  (void)launch_pdl(shift_select, ls.blocks[kStShift], kSortThreads, kSortSmem, st,
                   with_blk(bv, ls, kStShift));
  ++*launched;
  if (ls.blocks[kStShiftRank] > 0) {
    (void)launch_pdl(shift_select_rank, ls.blocks[kStShiftRank], kRankThreads, 0, st,
        with_blk(bv, ls, kStShiftRank));
    ++*launched;
  }
  (void)launch_pdl(global_select, ls.blocks[kStOne], kSortThreads, kSortSmem, st,
                   with_blk(bv, ls, kStOne));
  ++*launched;
  if (ls.blocks[kStGlobalRank] > 0) {
    (void)launch_pdl(global_select_rank, ls.blocks[kStGlobalRank], kRankThreads, 0, st,
        with_blk(bv, ls, kStGlobalRank));
    ++*launched;
  }
  return cudaGetLastError();
}

cudaError_t launch_finalize(const BatchView& bv, const LaunchSet& ls, cudaStream_t st,
                            int* launched) {
  cudaError_t e = ensure_dynamic_smem<finalize_sorted>(kSortSmem);
  if (e != cudaSuccess) return e;
  (void)launch_pdl(finalize_sorted, ls.blocks[kStOne], kSortThreads, kSortSmem, st,
                   with_blk(bv, ls, kStOne));
  ++*launched;
  if (ls.blocks[kStFinalRank] > 0) {
    (void)launch_pdl(finalize_rank, ls.blocks[kStFinalRank], kRankThreads, 0, st,
                     with_blk(bv, ls, kStFinalRank));
    ++*launched;
  }
  return cudaGetLastError();
}

int rank_blocks(const DevPlan& d, int kind) {
  if (kind == kStShiftRank)
    return d.vcap > kSortCap ? (int)std::min<int64_t>((d.vcap + kRankThreads - 1) / kRankThreads, 64) * d.nq : 0;
  if (kind == kStGlobalRank) {
    const int64_t lim = (int64_t)d.nq * d.s;
    return lim > kSortCap ? (int)std::min<int64_t>((lim + kRankThreads - 1) / kRankThreads, 256) : 0;
  }
  if (kind == kStFinalRank)
    return d.s > kSortCap ? (int)std::min<int64_t>((d.s + kRankThreads - 1) / kRankThreads, 256) : 0;
  return 0;
}

}  // namespace sft
