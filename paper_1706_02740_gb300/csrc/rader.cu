// Kernel (b), Rader's form: the measurements E_c = (1/p) sum_k h_k e^{-2 pi i k c / p}, c < p, of
// every node subset (eq. DFT_GKlam_Comp), for every shift and prime, when every p - 1 is a
// product of 2, 3, 5, 7, 11 and 13.
//
// With g a primitive root modulo p and L = p - 1, the nonzero indices are the powers g^n, so for
// a_n = h_{g^n} and b_n = e^{-2 pi i g^{-n} / p} (n < L)
//     E_{g^{-m}} = h_0 / p + (1/p) sum_n a_n b_{m - n}     (a cyclic convolution of length L),
//     E_0 = (h_0 + sum_n a_n) / p.
// The convolution is FFT_L^{-1}(FFT_L(a) . FFT_L(b)); FFT_L(b) / (p L) = V is precomputed per prime
// (FP64 on the host), and the inverse is the forward FFT between two conjugations:
//     E_{g^{-m}} = h_0 / p + conj( FFT_L( conj( FFT_L(a) . V ) ) )[m].
// One transform per CTA: two shared-memory buffers of L elements (padded, one slot per 16) and
// out-of-place Stockham passes that alternate between them (one barrier per pass, one item of at
// most 16 values per thread at a time).  The radix of each pass comes from the plan's schedule at
// run time; each radix is a compile-time in-register DFT.  The samples h_1 .. h_{p-1} are first
// staged in order (coalesced loads) and the first pass gathers a_n from them through the table g^n
// (reading them from global memory in that order instead costs a 32-byte sector per 8-byte
// sample once a batch's samples exceed L2); the last pass of the first FFT multiplies by V
// and conjugates; the last pass of the second FFT writes conj(.) + h_0/p to shared memory at
// position g^{-m} - 1, from where the p outputs are stored contiguously.
#include <stdint.h>

#include "checks.cuh"
#include "cplx.cuh"
#include "fft_radix.cuh"
#include "sft_internal.h"

namespace sft {

namespace {

// v[r] *= w^r, w = e^{-2 pi i k / (S RAD)}, from the pass's table rows (exponents 1, 2, 3, 4, 8, 12
// below RAD, each row S entries): w^r for r = 4a + c is row(4a) x row(c), at most one product of
// two exactly rounded entries.
template <typename C, int RAD>
__device__ __forceinline__ void twiddle_rows(const C* __restrict__ W, int S, int k, C* v) {
  if constexpr (RAD == 2) {
    v[1] = cmul(v[1], __ldg(W + k));
  } else if constexpr (RAD == 3) {
    v[1] = cmul(v[1], __ldg(W + k));
    v[2] = cmul(v[2], __ldg(W + S + k));
  } else {
    const C w1 = __ldg(W + k), w2 = __ldg(W + S + k), w3 = __ldg(W + 2 * S + k);
    v[1] = cmul(v[1], w1);
    v[2] = cmul(v[2], w2);
    v[3] = cmul(v[3], w3);
#pragma unroll
    for (int a = 1; 4 * a < RAD; ++a) {
      const C P = __ldg(W + (2 + a) * S + k);   // w^{4a}
      v[4 * a] = cmul(v[4 * a], P);
      if (4 * a + 1 < RAD) v[4 * a + 1] = cmul(v[4 * a + 1], cmul(P, w1));
      if (4 * a + 2 < RAD) v[4 * a + 2] = cmul(v[4 * a + 2], cmul(P, w2));
      if (4 * a + 3 < RAD) v[4 * a + 3] = cmul(v[4 * a + 3], cmul(P, w3));
    }
  }
}

// Where a pass reads and writes.
enum { kRdSmem = 0, kRdGather = 1 };                   // in order, or a_n = h[g^n] (staged h)
enum { kWrSmem = 0, kWrFilter = 1, kWrScatter = 2 };   // plain, x V then conj, or permuted output

template <typename C>
struct RaderIO {
  const C* in;            // the transform's p samples (global)
  const int32_t* pin;     // g^n mod p
  const int32_t* pout;    // g^{-n} mod p
  const C* V;             // FFT(b) / (p L)
  C* a0;                  // shared slot for FFT(a)[0]
  C h0p;                  // h_0 / p
};

// One out-of-place Stockham pass of radix RAD over a length-L transform at sub-transform length S:
// item i < L / RAD reads elements i + r L/RAD (r < RAD), applies e^{-2 pi i r k / (S RAD)}
// (k = i mod S), takes a length-RAD DFT and writes element (i - k) RAD + k + r S.
template <typename C, int RAD, int RD, int WR>
__device__ __forceinline__ void rader_pass(const C* __restrict__ src, C* __restrict__ dst,
                                           const C* __restrict__ W, int L, int S, int lt, int tpt,
                                           const RaderIO<C>& io) {
  const int NI = L / RAD;
  // i = q S + k, advanced by tpt = tq S + tr per round (two divisions per pass, none per item)
  const int tq = tpt / S, tr = tpt - tq * S;
  int q = lt / S, k = lt - q * S;
  for (int i = lt; i < NI; i += tpt) {
    C v[RAD];
#pragma unroll
    for (int r = 0; r < RAD; ++r) {
      const int n = i + r * NI;
      if constexpr (RD == kRdGather) v[r] = src[pad16(__ldg(io.pin + n) - 1)];
      else v[r] = src[pad16(n)];
    }
    if (S > 1) twiddle_rows<C, RAD>(W, S, k, v);
    DFT<RAD, C>::run(v);
    const int j0 = q * S * RAD + k;
#pragma unroll
    for (int r = 0; r < RAD; ++r) {
      const int c = j0 + r * S;
      if constexpr (WR == kWrFilter) {
        if (c == 0) *io.a0 = v[r];
        dst[pad16(c)] = cconj(cmul(v[r], __ldg(io.V + c)));
      } else if constexpr (WR == kWrScatter) {
        dst[pad16(__ldg(io.pout + c) - 1)] = cadd(io.h0p, cconj(v[r]));
      } else {
        dst[pad16(c)] = v[r];
      }
    }
    q += tq;
    k += tr;
    if (k >= S) {
      k -= S;
      ++q;
    }
  }
}

template <typename C, int RD, int WR>
__device__ __forceinline__ void pass_any(int R, const C* src, C* dst, const C* W, int L, int S,
                                         int lt, int tpt, const RaderIO<C>& io) {
  switch (R) {
    case 2: rader_pass<C, 2, RD, WR>(src, dst, W, L, S, lt, tpt, io); break;
    case 3: rader_pass<C, 3, RD, WR>(src, dst, W, L, S, lt, tpt, io); break;
    case 4: rader_pass<C, 4, RD, WR>(src, dst, W, L, S, lt, tpt, io); break;
    case 5: rader_pass<C, 5, RD, WR>(src, dst, W, L, S, lt, tpt, io); break;
    case 6: rader_pass<C, 6, RD, WR>(src, dst, W, L, S, lt, tpt, io); break;
    case 7: rader_pass<C, 7, RD, WR>(src, dst, W, L, S, lt, tpt, io); break;
    case 8: rader_pass<C, 8, RD, WR>(src, dst, W, L, S, lt, tpt, io); break;
    case 10: rader_pass<C, 10, RD, WR>(src, dst, W, L, S, lt, tpt, io); break;
    case 11: rader_pass<C, 11, RD, WR>(src, dst, W, L, S, lt, tpt, io); break;
    case 12: rader_pass<C, 12, RD, WR>(src, dst, W, L, S, lt, tpt, io); break;
    case 13: rader_pass<C, 13, RD, WR>(src, dst, W, L, S, lt, tpt, io); break;
    case 14: rader_pass<C, 14, RD, WR>(src, dst, W, L, S, lt, tpt, io); break;
    default: rader_pass<C, 16, RD, WR>(src, dst, W, L, S, lt, tpt, io); break;
  }
}

// One transform per CTA (blockDim.x threads); the CTA of block x takes transform x of its signal,
// counted prime by prime (then shift, then node subset).  FP32 builds are held to 64
// registers (several CTAs per SM), FP64 builds to 128.
template <typename R>
__global__ void __launch_bounds__(512, sizeof(R) == 4 ? 2 : 1) rader_kernel(BatchView bv) {
  pdl_begin();
  using C = typename Cx<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ C a0;
  int lb, nb;
  const DevPlan& d = bv.plans[batch_signal(bv, lb, nb)];
  // prime-major order: the CTAs resident at one time mostly share a prime, so its tables
  // (twiddle rows, V, permutations: ~24 L bytes) stay in L1
  const int per_j = d.nq * d.nsub;
  if (lb >= per_j * d.K) return;                  // (the block count is exact; kept as a guard)
  const int j = lb / per_j;
  const int rem = lb - j * per_j;
  const int qi = rem / d.nsub;
  const int sub = rem - qi * d.nsub;
  const int p = d.p[j], L = p - 1;
  const int64_t off = (int64_t)qi * d.m + d.nodeoff[j] + (int64_t)sub * p;
  if (!index_ok(d, off + p - 1, (int64_t)d.nq * d.m, SFT_SITE_DFT)) return;   // whole CTA
  C* bufA = reinterpret_cast<C*>(smem_raw);
  C* bufB = bufA + rader_buf(d.rLmax);
  const int32_t* sch = d.rsched + j * kRaderSched;
  const int npass = sch[0];
  const C* Wj = reinterpret_cast<const C*>(d.rtw) + (int64_t)j * d.pmax;
  RaderIO<C> io;
  io.in = reinterpret_cast<const C*>(d.samples) + off;
  io.pin = d.rperm + (int64_t)j * 2 * d.pmax;
  io.pout = io.pin + d.pmax;
  io.V = reinterpret_cast<const C*>(d.rV) + (int64_t)j * d.pmax;
  io.a0 = &a0;
  const C h0 = __ldg(io.in);
  const R inv_p = (R)1 / (R)p;
  io.h0p = cscale(h0, inv_p);
  const int lt = threadIdx.x, tpt = blockDim.x;

  // h_1 .. h_{p-1} staged in order (coalesced loads); the first pass gathers a_n = h_{g^n} from it
  for (int n = lt; n < L; n += tpt) bufB[pad16(n)] = __ldg(io.in + 1 + n);
  __syncthreads();
  // forward FFT of a, then x V and conj in its last pass
  C* src = bufB;
  C* dst = bufA;
  int S = 1;
  for (int ps = 0; ps < npass; ++ps) {
    const int Rr = sch[1 + ps];
    const C* W = Wj + sch[16 + ps];
    const bool first = ps == 0, last = ps == npass - 1;
    if (first && last) pass_any<C, kRdGather, kWrFilter>(Rr, src, dst, W, L, S, lt, tpt, io);
    else if (first) pass_any<C, kRdGather, kWrSmem>(Rr, src, dst, W, L, S, lt, tpt, io);
    else if (last) pass_any<C, kRdSmem, kWrFilter>(Rr, src, dst, W, L, S, lt, tpt, io);
    else pass_any<C, kRdSmem, kWrSmem>(Rr, src, dst, W, L, S, lt, tpt, io);
    __syncthreads();
    C* t = src; src = dst; dst = t;
    S *= Rr;
  }
  // second forward FFT; its last pass writes h_0/p + conj(.) to position g^{-m} - 1
  S = 1;
  for (int ps = 0; ps < npass; ++ps) {
    const int Rr = sch[1 + ps];
    const C* W = Wj + sch[16 + ps];
    if (ps == npass - 1) pass_any<C, kRdSmem, kWrScatter>(Rr, src, dst, W, L, S, lt, tpt, io);
    else pass_any<C, kRdSmem, kWrSmem>(Rr, src, dst, W, L, S, lt, tpt, io);
    __syncthreads();
    C* t = src; src = dst; dst = t;
    S *= Rr;
  }
  // src now holds E_1 .. E_{p-1} in order
  C* out = reinterpret_cast<C*>(d.bins) + off;
  if (lt == 0) out[0] = cscale(cadd(h0, a0), inv_p);
  for (int n = lt; n < L; n += tpt) out[1 + n] = src[pad16(n)];
}

template <typename R>
cudaError_t launch_rader_prec(const BatchView& bv, const LaunchSet& ls, cudaStream_t st,
                              int* launched) {
  using C = typename Cx<R>::T;
  const unsigned grid = (unsigned)ls.blocks[kStRader];
  const int threads = ls.rtpt > 0 ? ls.rtpt : 256;
  const size_t smem = 2 * (size_t)rader_buf(ls.rlmax) * sizeof(C);
  cudaError_t e = ensure_dynamic_smem<rader_kernel<R>>(smem);
  if (e != cudaSuccess) return e;
  BatchView v = bv;
  v.blk = ls.blk[kStRader];
  (void)launch_pdl(rader_kernel<R>, grid, threads, smem, st, v);
  if (launched) ++*launched;
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_rader(const DevPlan& d0, const BatchView& bv, const LaunchSet& ls,
                         cudaStream_t st, int* launched) {
  if (ls.blocks[kStRader] == 0 || ls.rlmax < 1) return cudaSuccess;
  return d0.prec == SFT_FP32 ? launch_rader_prec<float>(bv, ls, st, launched)
                             : launch_rader_prec<double>(bv, ls, st, launched);
}

}  // namespace sft
