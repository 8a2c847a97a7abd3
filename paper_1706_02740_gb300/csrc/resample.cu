// Kernel (a): filtered samples h_q(x) = (1/N) sum_{i=-kappa}^{kappa} f_{(j'+i) mod N} g_q(x - y_{j'+i})
// at every node the inner SFT reads, for every shift q at once (eq. UntruncatedFiniteSum cut to
// the window of Lemma fewer_points_error; modulated filter g_q(x) = e^{iqx} g(x)).
//
// One thread per node.  The node's window of f (2 kappa + 1 complex values, contiguous except at
// the ends of f) is fetched once with 16-byte vector loads and reused by all shifts.  Writing
// x - y_{j'+i} = 2 pi (v0 - i) / N with the exact integer offset d0 = kN - j'P (v0 = d0 / P), the
// shift-q sample factors as
//     h_q(x) = e^{2 pi i q d0 / (P N)} * sum_i [f_{j'+i} G0 e^{-gamma (v0 - i)^2}] * e^{-2 pi i q i / N}
// (G0 = 1/(N c1), gamma = 2 pi^2 / (N c1)^2).  Only the n = 0 image of the periodic Gaussian is
// kept: the plan requires gamma (N - kappa - 1/2)^2 >= 40, so every other image is below e^{-40} of
// the window's central weight.  The table
// e^{-2 pi i (q i mod N) / N} is reduced exactly on the host; the node phase has
// |q d0 / (P N)| <= 1/4 and needs no reduction: the FP32 path forms it as the product of the two
// correctly rounded ratios d0/P and q/N, the FP64 path from the exact integer q d0.  The FP32
// path keeps FP64 and 64-bit integer division entirely off its instruction stream.
#include "checks.cuh"
#include "cplx.cuh"
#include "sft_internal.h"

namespace sft {

namespace {

struct NodeGeom {
  int64_t jp;   // nearest grid index reduced to [0, N)
  int32_t d0;   // kN - j'P (exact, |d0| <= P/2)
  int32_t PP;   // node modulus P (p_j or p_j t_l)
};

// Node k of modulus P sits at x = -pi + 2 pi k / P.  For the subset (l, k2) of prime p_j the node
// is -pi + 2 pi (k1/p + k2/t), i.e. k = (k1 t + k2 p) mod P, P = p t.  With N = Nq p + Nr and
// N = Nq' t + Nr',
//     kN / P = I + G / P (mod N),  I = k1 Nq + (k1 Nr) div p + k2 Nq' + (k2 Nr') div t,
//     G = ((k1 Nr) mod p) t + ((k2 Nr') mod t) p  in [0, 2P),
// so the nearest grid index (ties up) is j' = I + round(G / P) and d0 = kN - j'P = G - round(G/P) P,
// all in 32-bit integer arithmetic (no 64-bit division).
__device__ __forceinline__ void decode_node(const DevPlan& d, int64_t node, int& j, int& k1, NodeGeom& g) {
  {
    // the prime whose node range holds `node` (binary search: K may be large)
    int lo = 0, hi = d.K;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (d.nodeoff[mid] <= node) lo = mid;
      else hi = mid;
    }
    j = lo;
  }
  const int p = d.p[j];
  const int local = (int)(node - d.nodeoff[j]);
  const int sub = local / p;
  k1 = local - sub * p;
  const int a1 = k1 * d.Nrp[j];                 // < p^2
  const int q1 = a1 / p;
  const int F1 = a1 - q1 * p;
  int64_t I = (int64_t)k1 * d.Nqp[j] + q1;
  int G, PP;
  if (sub == 0) {
    PP = p;
    G = F1;
  } else {
    const int l = d.sub_l[sub];
    const int t = d.t[l];
    const int k2 = d.sub_k2[sub];
    const int a2 = k2 * d.Nrt[l];
    const int q2 = a2 / t;
    const int F2 = a2 - q2 * t;
    I += (int64_t)k2 * d.Nqt[l] + q2;
    PP = p * t;
    G = F1 * t + F2 * p;
  }
  const int rnd = (2 * G >= 3 * PP) ? 2 : ((2 * G >= PP) ? 1 : 0);
  g.d0 = G - rnd * PP;
  // I = floor(k1 N / p) + floor(k2 N / t) < 2N, so jp < 2N + 2: two reductions suffice (N >= 2)
  int64_t jp = I + rnd;
#pragma unroll
  for (int r = 0; r < 2; ++r)
    if (jp >= d.N) jp -= d.N;
  g.jp = jp;
  g.PP = PP;
}

// Node phase exp(2 pi i q d0 / (P N)) of shift qi (|q d0 / (P N)| <= 1/4, so it needs no reduction).
__device__ __forceinline__ float2 node_phase(const DevPlan& d, int qi, float v0, const NodeGeom&) {
  return expi_turns(v0 * d.qN32[qi]);
}
__device__ __forceinline__ double2 node_phase(const DevPlan& d, int qi, double, const NodeGeom& g) {
  const int64_t num = d.q[qi] * (int64_t)g.d0;           // exact
  return expi_turns((double)num / ((double)g.PP * (double)d.N));
}

template <typename R> __device__ __forceinline__ R gamma_of(const DevPlan& d);
template <> __device__ __forceinline__ float gamma_of<float>(const DevPlan& d) { return d.gamma32; }
template <> __device__ __forceinline__ double gamma_of<double>(const DevPlan& d) { return d.gamma; }
template <typename R> __device__ __forceinline__ R g0_of(const DevPlan& d);
template <> __device__ __forceinline__ float g0_of<float>(const DevPlan& d) { return d.G032; }
template <> __device__ __forceinline__ double g0_of<double>(const DevPlan& d) { return d.G0; }

template <typename IN> struct InLoad;
template <> struct InLoad<float2> {
  __device__ static __forceinline__ float2 one(const float2* f, int64_t i) { return __ldg(f + i); }
};
template <> struct InLoad<double2> {
  __device__ static __forceinline__ double2 one(const double2* f, int64_t i) { return __ldg(f + i); }
};

template <typename R, typename C, typename IN>
__device__ __forceinline__ C widen(IN v) {
  return cmake<C>((double)v.x, (double)v.y);
}
template <> __device__ __forceinline__ float2 widen<float, float2, float2>(float2 v) { return v; }
template <> __device__ __forceinline__ double2 widen<double, double2, double2>(double2 v) { return v; }

// Fetch the 2*KAPPA+1 window values f_{(jp+i) mod N}, i = -KAPPA..KAPPA, into win[].
template <int KAPPA, typename C, typename R, typename IN>
__device__ __forceinline__ void fetch_window(const DevPlan& d, const IN* f, int64_t jp, C* win) {
  constexpr int W = 2 * KAPPA + 1;
  const int64_t N = d.N;
  if constexpr (sizeof(IN) == 8) {
    if ((reinterpret_cast<uintptr_t>(f) & 15) == 0 && jp >= KAPPA && jp + KAPPA + 2 <= N) {
      const int64_t start = jp - KAPPA;
      const int64_t base = start & ~int64_t(1);
      const float4* v = reinterpret_cast<const float4*>(f + base);
      float2 e[W + 1];
#pragma unroll
      for (int h = 0; h < (W + 1) / 2; ++h) {
        float4 x = __ldg(v + h);
        e[2 * h] = make_float2(x.x, x.y);
        e[2 * h + 1] = make_float2(x.z, x.w);
      }
      if (start == base) {
#pragma unroll
        for (int i = 0; i < W; ++i) win[i] = widen<R, C, float2>(e[i]);
      } else {
#pragma unroll
        for (int i = 0; i < W; ++i) win[i] = widen<R, C, float2>(e[i + 1]);
      }
      return;
    }
  } else {
    if (jp >= KAPPA && jp + KAPPA < N) {
#pragma unroll
      for (int i = 0; i < W; ++i) win[i] = widen<R, C, IN>(InLoad<IN>::one(f, jp - KAPPA + i));
      return;
    }
  }
#pragma unroll
  for (int i = 0; i < W; ++i) {
    int64_t idx = jp - KAPPA + i;
    if (idx < 0) idx += N;
    if (idx >= N) idx -= N;
    win[i] = widen<R, C, IN>(InLoad<IN>::one(f, idx));
  }
}

// CAP = 0: the FP32 build fits 2 CTAs of 512 threads per SM (64 registers), the FP64 build is
// unlimited; CAP = 1: built for 5 CTAs of 256 threads (48 registers, more warps in flight for the
// gather; CTAs of at most 256 threads).
template <int KAPPA, typename R, typename IN, int CAP>
__global__ void __launch_bounds__(CAP ? 256 : kResampleMaxThreads, CAP ? 5 : (sizeof(R) == 4 ? 2 : 1))
resample_kernel(BatchView bv) {
  pdl_begin();
  using C = typename Cx<R>::T;
  constexpr int W = 2 * KAPPA + 1;
  int lb, nb;
  const int b = batch_signal(bv, lb, nb);
  const DevPlan& d = bv.plans[b];
  const int64_t node = (int64_t)lb * blockDim.x + threadIdx.x;
  if (node >= d.m) return;
  const IN* __restrict__ f = reinterpret_cast<const IN*>(batch_f(bv, b));
  int j, k1;
  NodeGeom g;
  decode_node(d, node, j, k1, g);
  if (!index_ok(d, g.jp, d.N, SFT_SITE_WINDOW)) return;

  C win[W];
  fetch_window<KAPPA, C, R, IN>(d, f, g.jp, win);

  // Gaussian weights G0 exp(-gamma (v0 - i)^2), v0 = d0 / P
  const R v0 = (R)g.d0 / (R)g.PP;
  const R gam = gamma_of<R>(d), G0 = g0_of<R>(d);
#pragma unroll
  for (int i = 0; i < W; ++i) {
    const R v = v0 - (R)(i - KAPPA);
    win[i] = cscale(win[i], G0 * r_exp(-gam * v * v));
  }

  const C* T = reinterpret_cast<const C*>(d.Ttab);
  C* out = reinterpret_cast<C*>(d.samples);
  const int nq = d.nq;
  const int64_t m = d.m;
  for (int qi = 0; qi < nq; ++qi) {
    C acc = czero<C>();
    const C* Tq = T + qi * W;
#pragma unroll
    for (int i = 0; i < W; ++i) acc = cadd(acc, cmul(win[i], __ldg(Tq + i)));
    out[(int64_t)qi * m + node] = cmul(acc, node_phase(d, qi, v0, g));
  }
}

// Shifts accumulated together by the wide-window kernel (a plan with more runs further groups,
// the window then read again from cache), and window taps loaded together.
constexpr int kWideShifts = 16;
constexpr int kWideChunk = 4;

// Taps of the shared shift-phase table: the window width rounded up to whole chunks.
__host__ __device__ constexpr int wide_taps(int W) { return (W + kWideChunk - 1) / kWideChunk * kWideChunk; }

// Shared-memory bytes of the wide-window kernel's table for nq shifts and half-width kappa.
template <typename C>
constexpr size_t wide_table_bytes(int nq, int kappa) {
  return (size_t)((nq + kWideShifts - 1) / kWideShifts) * kWideShifts * wide_taps(2 * kappa + 1) *
         sizeof(C);
}

// The shifts of one group times one tap's weighted sample: acc[t] += x T[t] for the group's 16
// table entries of the tap (consecutive in shared memory, read 16 bytes at a time).
__device__ __forceinline__ void wide_macs(float2 (&acc)[kWideShifts], float2 x, const float2* T) {
  const float4* T4 = reinterpret_cast<const float4*>(T);
#pragma unroll
  for (int h = 0; h < kWideShifts / 2; ++h) {
    const float4 w = T4[h];
    acc[2 * h] = cadd(acc[2 * h], cmul(x, make_float2(w.x, w.y)));
    acc[2 * h + 1] = cadd(acc[2 * h + 1], cmul(x, make_float2(w.z, w.w)));
  }
}
__device__ __forceinline__ void wide_macs(double2 (&acc)[kWideShifts], double2 x, const double2* T) {
#pragma unroll
  for (int t = 0; t < kWideShifts; ++t) acc[t] = cadd(acc[t], cmul(x, T[t]));
}

// Any window half-width up to kMaxKappa (theorem-parameter mode).  The shift-phase table
// e^{-2 pi i (q i mod N) / N} is staged tap-major in shared memory, [group][tap][16 shifts], with
// zeros for the shifts past nq and the taps past 2 kappa + 1, so the inner loop has no branches:
// per chunk of taps the window values are loaded first (independent loads in flight), then each
// weighted sample updates the group's 16 accumulators from its table row (uniform addresses).
template <typename R, typename IN>
__global__ void __launch_bounds__(kResampleGenericThreads, sizeof(R) == 4 ? 8 : 1)
resample_kernel_generic(BatchView bv) {
  pdl_begin();
  using C = typename Cx<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int lb, nb;
  const int b = batch_signal(bv, lb, nb);
  const DevPlan& d = bv.plans[b];
  const int KAPPA = d.kappa, W = 2 * KAPPA + 1, WP = wide_taps(W);
  const int groups = (d.nq + kWideShifts - 1) / kWideShifts;
  C* Ts = reinterpret_cast<C*>(smem_raw);
  {
    const C* Tg = reinterpret_cast<const C*>(d.Ttab);
    const int n = groups * WP * kWideShifts;
    for (int e = threadIdx.x; e < n; e += kResampleGenericThreads) {
      const int t = e % kWideShifts, row = e / kWideShifts;
      const int g = row / WP, i = row - g * WP;
      const int q = g * kWideShifts + t;
      Ts[e] = (q < d.nq && i < W) ? __ldg(Tg + q * W + i) : czero<C>();
    }
    __syncthreads();
  }
  const int64_t node = (int64_t)lb * kResampleGenericThreads + threadIdx.x;
  if (node >= d.m) return;
  const IN* __restrict__ f = reinterpret_cast<const IN*>(batch_f(bv, b));
  int j, k1;
  NodeGeom g;
  decode_node(d, node, j, k1, g);
  if (!index_ok(d, g.jp, d.N, SFT_SITE_WINDOW)) return;
  const R v0 = (R)g.d0 / (R)g.PP;
  const R gam = gamma_of<R>(d), G0 = g0_of<R>(d);
  C* out = reinterpret_cast<C*>(d.samples);
  const int64_t start = g.jp - KAPPA;
  const bool inside = start >= 0 && start + W <= d.N;       // no wrap around the ends of f
  for (int gr = 0; gr < groups; ++gr) {
    C acc[kWideShifts];
#pragma unroll
    for (int t = 0; t < kWideShifts; ++t) acc[t] = czero<C>();
    const C* Tgr = Ts + (size_t)gr * WP * kWideShifts;
    for (int i0 = 0; i0 < WP; i0 += kWideChunk) {
      C fw[kWideChunk];
#pragma unroll
      for (int u = 0; u < kWideChunk; ++u) {
        const int i = i0 + u;
        fw[u] = czero<C>();
        if (i < W) {
          int64_t idx = start + i;
          if (!inside) {
            if (idx < 0) idx += d.N;
            if (idx >= d.N) idx -= d.N;
          }
          fw[u] = widen<R, C, IN>(InLoad<IN>::one(f, idx));
        }
      }
#pragma unroll
      for (int u = 0; u < kWideChunk; ++u) {
        const int i = i0 + u;
        const R v = v0 - (R)(i - KAPPA);
        const C x = cscale(fw[u], G0 * r_exp(-gam * v * v));
        wide_macs(acc, x, Tgr + (size_t)i * kWideShifts);
      }
    }
#pragma unroll
    for (int t = 0; t < kWideShifts; ++t) {
      const int q = gr * kWideShifts + t;
      if (q < d.nq) out[(int64_t)q * d.m + node] = cmul(acc[t], node_phase(d, q, v0, g));
    }
  }
}

template <typename R, typename IN>
cudaError_t launch_typed(const DevPlan& d0, const BatchView& bv, const LaunchSet& ls,
                         cudaStream_t st) {
  const unsigned grid = (unsigned)ls.blocks[kStResample];
  if (grid == 0) return cudaSuccess;
  BatchView v = bv;
  v.blk = ls.blk[kStResample];
  const int t = ls.tune.resample_threads;
  const bool cap = ls.tune.resample_regcap != 0;
  if (d0.kappa == 6) {
    if (cap) (void)launch_pdl(resample_kernel<6, R, IN, 1>, grid, t, 0, st, v);
    else (void)launch_pdl(resample_kernel<6, R, IN, 0>, grid, t, 0, st, v);
  } else if (d0.kappa == 4) {
    if (cap) (void)launch_pdl(resample_kernel<4, R, IN, 1>, grid, t, 0, st, v);
    else (void)launch_pdl(resample_kernel<4, R, IN, 0>, grid, t, 0, st, v);
  } else {
    // room for the largest shift table of the batch (the signals share kappa; at most kMaxQ shifts)
    const size_t smem = wide_table_bytes<typename Cx<R>::T>(kMaxQ, d0.kappa);
    const cudaError_t e = ensure_dynamic_smem<resample_kernel_generic<R, IN>>(smem);
    if (e != cudaSuccess) return e;
    (void)launch_pdl(resample_kernel_generic<R, IN>, grid, kResampleGenericThreads, smem, st, v);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_resample(const DevPlan& d0, const BatchView& bv, const LaunchSet& ls,
                            cudaStream_t st) {
  if (d0.prec == SFT_FP32)
    return d0.input == SFT_IN_C64 ? launch_typed<float, float2>(d0, bv, ls, st)
                                  : launch_typed<float, double2>(d0, bv, ls, st);
  return d0.input == SFT_IN_C64 ? launch_typed<double, float2>(d0, bv, ls, st)
                                : launch_typed<double, double2>(d0, bv, ls, st);
}

}  // namespace sft
