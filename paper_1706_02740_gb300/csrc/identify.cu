// Kernels (c) and (d) of the inner SFT (Appendix B reading): identification and estimation.
//
// identify: for each shift q, prime p_j and bin b, the residue of the bin's frequency modulo each
// small modulus t_l is the sub-bin of largest magnitude of the length-(p_j t_l) measurement that
// folds onto b.  By the prime-factor (Good-Thomas) index map, those t_l sub-bins are a length-t_l
// DFT over the node subsets offset by 2 pi k2 / t_l (k2 = 0 is the p_j nodes themselves):
//     X_r = (1/t) sum_{k2 < t} Z_{k2}[b] e^{-2 pi i k2 r / t},   r = frequency mod t,
// where Z_{k2} is the length-p_j measurement of subset k2.  The argmax breaks exact ties toward the
// smaller sub-bin index u = (r - b) p_j^{-1} mod t.  Garner's mixed-radix CRT of (b mod p_j,
// r_1 mod t_1, ...) then gives the representative in [0, p_j prod t), mapped to B or rejected.
// All integer work is exact.
//
// vote: a frequency w found in bin b of p_j counts one vote for every prime p_j' whose bin
// w mod p_j' reconstructed exactly w; it is kept when it has more than K/2 votes and is emitted
// once, by the smallest such j'.  Its estimate is (-1)^w times the componentwise medians of
// Z_0[w mod p_j'] over all K primes (eq. GSFT_Estimate).
#include "checks.cuh"
#include "cplx.cuh"
#include "select_sort.cuh"
#include "sft_internal.h"

namespace sft {

namespace {

// x mod t for 0 <= x < 2^63 and 2 <= t <= 64 in 32-bit arithmetic (a 64-bit '%' would run the
// FP64-based division routine).
__device__ __forceinline__ int mod_small(int64_t x, int t) {
  const uint64_t u = (uint64_t)x;
  const uint32_t hi = (uint32_t)(u >> 32), lo = (uint32_t)u;
  const uint32_t r32 = (0xFFFFFFFFu % (uint32_t)t + 1u) % (uint32_t)t;   // 2^32 mod t
  return (int)(((hi % (uint32_t)t) * r32 + lo % (uint32_t)t) % (uint32_t)t);
}

// w mod p (floor) for |w| < 2^31
__device__ __forceinline__ int mod_p(int64_t w, int p) {
  const int r = (int)w % p;
  return r < 0 ? r + p : r;
}

__device__ __forceinline__ void decode_bin(const DevPlan& d, int64_t gid, int& qi, int& j, int& b) {
  qi = (int)(gid / d.Ptot);
  const int bin = (int)(gid - (int64_t)qi * d.Ptot);
  int lo = 0, hi = d.K;                  // the prime whose bin range holds `bin`
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (d.poff[mid] <= bin) lo = mid;
    else hi = mid;
  }
  j = lo;
  b = bin - d.poff[j];
}

__device__ __forceinline__ float r_fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double r_fma(double a, double b, double c) { return fma(a, b, c); }

// Residue of bin b modulo a small modulus T: argmax over r of |X_r|^2 with
// X_r = sum_{k2 < T} Z_{k2}[b] e^{-2 pi i k2 r / T} (the 1/T factor does not change the argmax);
// exact ties go to the smaller sub-bin index u = (r - b) p^{-1} mod T.
// For odd T the terms k2 and T - k2 are paired: with A_k = z_k + z_{T-k}, B_k = z_k - z_{T-k},
// c = cos(2 pi k r / T), s = sin(2 pi k r / T),
//     X_r = z_0 + sum_k (c A_k - i s B_k),   X_{T-r} = z_0 + sum_k (c A_k + i s B_k),
// so each pair (r, T - r) costs two real-by-complex sums of (T-1)/2 terms instead of two complex
// sums of T - 1.  The comparison (largest |X|^2, then smallest u) does not depend on the order in
// which the r are visited.
template <int T, typename C, typename R>
__device__ __forceinline__ int residue_t(C z0, const C* Zl, int64_t p, const C* twl, int bt, int pinv) {
  C z[T];
  z[0] = z0;
#pragma unroll
  for (int k2 = 1; k2 < T; ++k2) z[k2] = __ldg(Zl + (int64_t)k2 * p);
  R best = (R)-1;
  int bestu = 1 << 30, bestr = 0;
  auto consider = [&](const C& X, int r, int u) {
    const R m2 = X.x * X.x + X.y * X.y;
    if (m2 > best || (m2 == best && u < bestu)) {
      best = m2;
      bestu = u;
      bestr = r;
    }
  };
  const int u0 = ((T - bt) % T) * pinv % T;      // u of r = 0; u of r +/- 1 moves by +/- pinv
  if constexpr (T == 2) {
    consider(cadd(z[0], z[1]), 0, u0);
    consider(csub(z[0], z[1]), 1, (u0 + pinv) % 2);
  } else {
    constexpr int H = (T - 1) / 2;
    // cos and sin of 2 pi m / T for m = 1..H from the table e^{-2 pi i m / T} (m > H follows by
    // symmetry: cos(2 pi (T - m) / T) = cos(2 pi m / T), sin(2 pi (T - m) / T) = -sin(2 pi m / T))
    R cs[H + 1], sn[H + 1];
#pragma unroll
    for (int m = 1; m <= H; ++m) {
      const C w = __ldg(twl + m);
      cs[m] = w.x;
      sn[m] = -w.y;
    }
    C A[H + 1], B[H + 1];
    C X0 = z[0];
#pragma unroll
    for (int k = 1; k <= H; ++k) {
      A[k] = cadd(z[k], z[T - k]);
      B[k] = csub(z[k], z[T - k]);
      X0 = cadd(X0, A[k]);
    }
    consider(X0, 0, u0);
    int up = u0, un = u0;
#pragma unroll
    for (int r = 1; r <= H; ++r) {
      C P = z[0], Q = czero<C>();
#pragma unroll
      for (int k = 1; k <= H; ++k) {
        const int m = (k * r) % T;
        const R c = m <= H ? cs[m] : cs[T - m], s = m <= H ? sn[m] : -sn[T - m];
        P.x = r_fma(A[k].x, c, P.x);
        P.y = r_fma(A[k].y, c, P.y);
        Q.x = r_fma(B[k].x, s, Q.x);
        Q.y = r_fma(B[k].y, s, Q.y);
      }
      up += pinv;
      if (up >= T) up -= T;
      un -= pinv;
      if (un < 0) un += T;
      consider(C{P.x + Q.y, P.y - Q.x}, r, up);           // X_r = P - i Q
      consider(C{P.x - Q.y, P.y + Q.x}, T - r, un);       // X_{T-r} = P + i Q
    }
  }
  return bestr;
}

template <typename C, typename R>
__device__ int residue_any(int t, C z0, const C* Zl, int64_t p, const C* twl, int bt, int pinv) {
  R best = (R)-1;
  int bestu = 1 << 30, bestr = 0;
  for (int r = 0; r < t; ++r) {
    C X = z0;
    int idx = 0;
    for (int k2 = 1; k2 < t; ++k2) {
      idx += r;
      if (idx >= t) idx -= t;
      X = cadd(X, cmul(__ldg(Zl + (int64_t)k2 * p), __ldg(twl + idx)));
    }
    const R m2 = X.x * X.x + X.y * X.y;
    const int u = (((r - bt) % t + t) % t) * pinv % t;
    if (m2 > best || (m2 == best && u < bestu)) {
      best = m2;
      bestu = u;
      bestr = r;
    }
  }
  return bestr;
}

// One small modulus with t = T known at compile time: its residue, then Garner's step
// x += M_x ((r - x) M_x^{-1} mod T), M_x *= T (divisions by T become multiplications).
template <int T, typename C, typename R>
__device__ __forceinline__ int crt_step(const DevPlan& d, int j, int l, int b, C z0, const C* Z,
                                        int64_t p, const C* tw, int64_t& x, int64_t& Mx) {
  const C* Zl = Z + (int64_t)(d.subbase[l] - 1) * p;
  const int r = residue_t<T, C, R>(z0, Zl, p, tw + d.twoff[l], b % T, d.pinv[j * d.nT + l]);
  const int xm = mod_small(x, T);
  const int v = ((r - xm + T) % T) * d.garner[j * d.nT + l] % T;
  x += Mx * v;
  Mx *= T;
  return r;
}

// The small moduli are the first primes 2, 3, 5, ... not among the p_j; when none of the p_j is
// one of them (every plan with p_1 > 13), they are the first nT of 2, 3, 5, 7, 11, 13 and the
// whole chain runs with compile-time moduli, fully unrolled; the residues are stored at the end.
__device__ __forceinline__ int prefix_t(int l) {
  return l == 0 ? 2 : l == 1 ? 3 : l == 2 ? 5 : l == 3 ? 7 : l == 4 ? 11 : 13;
}

template <int NT, typename C, typename R>
__device__ __forceinline__ void crt_prefix(const DevPlan& d, int j, int b, C z0, const C* Z,
                                           int64_t p, const C* tw, int64_t& x, uint8_t* resid) {
  int64_t Mx = p;
  int r[NT];
  if constexpr (NT >= 1) r[0] = crt_step<2, C, R>(d, j, 0, b, z0, Z, p, tw, x, Mx);
  if constexpr (NT >= 2) r[1] = crt_step<3, C, R>(d, j, 1, b, z0, Z, p, tw, x, Mx);
  if constexpr (NT >= 3) r[2] = crt_step<5, C, R>(d, j, 2, b, z0, Z, p, tw, x, Mx);
  if constexpr (NT >= 4) r[3] = crt_step<7, C, R>(d, j, 3, b, z0, Z, p, tw, x, Mx);
  if constexpr (NT >= 5) r[4] = crt_step<11, C, R>(d, j, 4, b, z0, Z, p, tw, x, Mx);
  if constexpr (NT >= 6) r[5] = crt_step<13, C, R>(d, j, 5, b, z0, Z, p, tw, x, Mx);
#pragma unroll
  for (int l = 0; l < NT; ++l) resid[l] = (uint8_t)r[l];
}

// One thread per bin.  The body is shared by the FP32 and FP64 kernels below.
template <typename R>
__device__ __forceinline__ void identify_bins(const BatchView& bv) {
  using C = typename Cx<R>::T;
  int lb, nb;
  const DevPlan& d = bv.plans[batch_signal(bv, lb, nb)];
  const int64_t gid = (int64_t)lb * blockDim.x + threadIdx.x;
  if (gid >= (int64_t)d.nq * d.Ptot) return;
  int qi, j, b;
  decode_bin(d, gid, qi, j, b);
  const int p = d.p[j];
  const int64_t zoff = (int64_t)qi * d.m + d.nodeoff[j] + b;
  if (!index_ok(d, b, p, SFT_SITE_SUBBIN) ||
      !index_ok(d, zoff + (int64_t)(d.nsub - 1) * p, (int64_t)d.nq * d.m, SFT_SITE_SUBBIN)) {
    d.cand[gid] = kNoFreq;
    return;
  }
  const C* Z = reinterpret_cast<const C*>(d.bins) + zoff;
  const C* tw = reinterpret_cast<const C*>(d.twsmall);
  const C z0 = __ldg(Z);
  int64_t x = b;
  int prefix = d.nT <= 6 ? d.nT : -1;                     // CTA-uniform: one plan per CTA
  for (int l = 0; l < d.nT && prefix >= 0; ++l)
    if (d.t[l] != prefix_t(l)) prefix = -1;
  if (prefix >= 0) {
    uint8_t* rs = d.resid + gid * d.nT;
    switch (prefix) {
      case 1: crt_prefix<1, C, R>(d, j, b, z0, Z, p, tw, x, rs); break;
      case 2: crt_prefix<2, C, R>(d, j, b, z0, Z, p, tw, x, rs); break;
      case 3: crt_prefix<3, C, R>(d, j, b, z0, Z, p, tw, x, rs); break;
      case 4: crt_prefix<4, C, R>(d, j, b, z0, Z, p, tw, x, rs); break;
      case 5: crt_prefix<5, C, R>(d, j, b, z0, Z, p, tw, x, rs); break;
      case 6: crt_prefix<6, C, R>(d, j, b, z0, Z, p, tw, x, rs); break;
      default: break;                                      // no small modulus: x = b
    }
  } else {
    int64_t Mx = p;
    for (int l = 0; l < d.nT; ++l) {
      const int t = d.t[l];
      const C* Zl = Z + (int64_t)(d.subbase[l] - 1) * p;   // Zl[k2 * p] = Z_{k2}[b], k2 >= 1
      const C* twl = tw + d.twoff[l];
      const int pinv = d.pinv[j * d.nT + l];
      const int bt = b % t;
      int r;
      switch (t) {
        case 2: r = residue_t<2, C, R>(z0, Zl, p, twl, bt, pinv); break;
        case 3: r = residue_t<3, C, R>(z0, Zl, p, twl, bt, pinv); break;
        case 5: r = residue_t<5, C, R>(z0, Zl, p, twl, bt, pinv); break;
        case 7: r = residue_t<7, C, R>(z0, Zl, p, twl, bt, pinv); break;
        case 11: r = residue_t<11, C, R>(z0, Zl, p, twl, bt, pinv); break;
        case 13: r = residue_t<13, C, R>(z0, Zl, p, twl, bt, pinv); break;
        default: r = residue_any<C, R>(t, z0, Zl, p, twl, bt, pinv); break;
      }
      d.resid[gid * d.nT + l] = (uint8_t)r;
      const int g = d.garner[j * d.nT + l];
      const int xm = mod_small(x, t);
      const int v = (((r - xm) % t + t) % t) * g % t;
      x += Mx * v;
      Mx *= t;
    }
  }
  const int64_t N = d.N;
  int64_t w = (x <= N / 2) ? x : x - d.Mj[j];
  d.cand[gid] = (w > -((N + 1) / 2)) ? w : kNoFreq;
}

// The FP32 kernel is held to kIdRegs registers.  The kernel waits on its sub-bin loads, so warps
// per SM count for more than the few spills of the unrolled chain at this cap: per 64 SFTs at
// N = 2^26, s = 1000, 64 registers (84 bytes of spills) measured 298 us, 72 (none) 309 us, 80 (none)
// 347 us, 56 (308 bytes) 298 us.  The FP64 kernel takes what it needs at up to 512 threads per CTA.
constexpr int kIdRegs = 64;

__global__ void __maxnreg__(kIdRegs) identify_kernel_fp32(BatchView bv) {
  pdl_begin();
  identify_bins<float>(bv);
}

__global__ void __launch_bounds__(kBinMaxThreads, 1) identify_kernel_fp64(BatchView bv) {
  pdl_begin();
  identify_bins<double>(bv);
}

// KCAP: capacity of the per-thread arrays (kFewK in registers, or kMaxK for many primes).
template <typename R, int KCAP>
__global__ void __launch_bounds__(kBinMaxThreads) vote_kernel(BatchView bv) {
  pdl_begin();
  using C = typename Cx<R>::T;
  int lb, nb;
  const DevPlan& d = bv.plans[batch_signal(bv, lb, nb)];
  const int64_t gid = (int64_t)lb * blockDim.x + threadIdx.x;
  if (gid >= (int64_t)d.nq * d.Ptot) return;
  const int64_t w = d.cand[gid];
  if (w == kNoFreq) return;
  int qi, j, b;
  decode_bin(d, gid, qi, j, b);
  const int64_t* cq = d.cand + (int64_t)qi * d.Ptot;
  // All K lookups are issued before any decision: a thread that left at the first match of an
  // earlier prime, or once the majority was out of reach, waited on each lookup in turn
  // (118 against 106 us per 64 SFTs).
  int cnt = 0, jmin = d.K;
  int bb[KCAP];
  for (int jj = 0; jj < d.K; ++jj) {
    bb[jj] = mod_p(w, d.p[jj]);
    if (!index_ok(d, d.poff[jj] + bb[jj], d.Ptot, SFT_SITE_VOTE)) continue;
    if (cq[d.poff[jj] + bb[jj]] == w) {
      ++cnt;
      if (jj < jmin) jmin = jj;
    }
  }
  if (cnt < d.K / 2 + 1 || jmin != j) return;
  const C* Zq = reinterpret_cast<const C*>(d.bins) + (int64_t)qi * d.m;
  R re[KCAP], im[KCAP];
  for (int jj = 0; jj < d.K; ++jj) {
    const C y = index_ok(d, (int64_t)d.nodeoff[jj] + bb[jj], d.m, SFT_SITE_VOTE)
                    ? Zq[d.nodeoff[jj] + bb[jj]] : czero<C>();
    re[jj] = y.x;
    im[jj] = y.y;
  }
  const double sg = (w & 1) ? -1.0 : 1.0;
  Voted rec;
  rec.w = w;
  rec.zre = sg * median_of<KCAP>(re, d.K);
  rec.zim = sg * median_of<KCAP>(im, d.K);
  rec.votes = cnt;
  rec.jmin = jmin;
  const int slot = atomicAdd(d.counters + qi, 1);
  if (slot < d.vcap) d.voted[(int64_t)qi * d.vcap + slot] = rec;
  else record_fault(d, SFT_FAULT_VOTED_FULL, SFT_SITE_NONE);
}

}  // namespace

cudaError_t launch_identify(const DevPlan& d0, const BatchView& bv, const LaunchSet& ls,
                            cudaStream_t st) {
  const unsigned grid = (unsigned)ls.blocks[kStBins];
  if (grid == 0) return cudaSuccess;
  BatchView v = bv;
  v.blk = ls.blk[kStBins];
  if (d0.prec == SFT_FP32)
    (void)launch_pdl(identify_kernel_fp32, grid, ls.tune.bin_threads, 0, st, v);
  else
    (void)launch_pdl(identify_kernel_fp64, grid, ls.tune.bin_threads, 0, st, v);
  return cudaGetLastError();
}

cudaError_t launch_vote(const DevPlan& d0, const BatchView& bv, const LaunchSet& ls,
                        cudaStream_t st) {
  const unsigned grid = (unsigned)ls.blocks[kStBins];
  if (grid == 0) return cudaSuccess;
  BatchView v = bv;
  v.blk = ls.blk[kStBins];
  const int t = ls.tune.bin_threads;
  const bool few = ls.kmax <= kFewK;
  if (d0.prec == SFT_FP32) {
    if (few) (void)launch_pdl(vote_kernel<float, kFewK>, grid, t, 0, st, v);
    else (void)launch_pdl(vote_kernel<float, kMaxK>, grid, t, 0, st, v);
  } else {
    if (few) (void)launch_pdl(vote_kernel<double, kFewK>, grid, t, 0, st, v);
    else (void)launch_pdl(vote_kernel<double, kMaxK>, grid, t, 0, st, v);
  }
  return cudaGetLastError();
}

}  // namespace sft
