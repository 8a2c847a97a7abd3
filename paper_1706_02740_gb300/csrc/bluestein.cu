// Kernel (b): the inner SFT's measurements E_c = (1/p) sum_k h(x_k) e^{-2 pi i k c / p}, c = 0..p-1,
// of every node subset (eq. DFT_GKlam_Comp), for every shift and prime at once.
//
// Each p_j is prime, so the length-p DFT is taken as a chirp convolution (Bluestein): with
// w_n = e^{-pi i n^2 / p},  E_c = (1/p) w_c sum_k (h_k w_k) conj(w_{c-k}),  a linear convolution
// done as a cyclic one of power-of-two length M >= 2p - 1:
//     E = w . conj( FFT( conj( FFT(h w, zero padded) . V ) ) ),
// V = FFT(conj(w) wrapped) / (M p) precomputed per prime in FP64 on the host (the inverse FFT is the
// forward one between two conjugations).  One transform lives in shared memory; the FFT is an
// in-place Stockham schedule whose passes hold 16 complex values per thread in registers (radix 16
// passes, then one radix 2/4/8 pass), with twiddles read from an exactly rounded table.  The
// shared-memory layout inserts one pad element after every 16 (index n -> n + n/16), so the
// strided stores of the first two passes hit distinct banks.
#include "cplx.cuh"
#include "sft_internal.h"

namespace sft {

namespace {

__device__ __forceinline__ int pad16(int n) { return n + (n >> 4); }
template <int M> constexpr int padded_len() { return M + M / 16; }

// e^{-2 pi i k / 16}, k = 0..15 (mathematical constants, correctly rounded).
__device__ __constant__ double kW16re[16] = {
    1.0, 0.92387953251128674, 0.70710678118654752, 0.38268343236508977,
    0.0, -0.38268343236508977, -0.70710678118654752, -0.92387953251128674,
    -1.0, -0.92387953251128674, -0.70710678118654752, -0.38268343236508977,
    0.0, 0.38268343236508977, 0.70710678118654752, 0.92387953251128674};
__device__ __constant__ double kW16im[16] = {
    0.0, -0.38268343236508977, -0.70710678118654752, -0.92387953251128674,
    -1.0, -0.92387953251128674, -0.70710678118654752, -0.38268343236508977,
    0.0, 0.38268343236508977, 0.70710678118654752, 0.92387953251128674,
    1.0, 0.92387953251128674, 0.70710678118654752, 0.38268343236508977};

__device__ __constant__ float kW16reF[16] = {
    1.0f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508977f,
    0.0f, -0.38268343236508977f, -0.70710678118654752f, -0.92387953251128674f,
    -1.0f, -0.92387953251128674f, -0.70710678118654752f, -0.38268343236508977f,
    0.0f, 0.38268343236508977f, 0.70710678118654752f, 0.92387953251128674f};
__device__ __constant__ float kW16imF[16] = {
    0.0f, -0.38268343236508977f, -0.70710678118654752f, -0.92387953251128674f,
    -1.0f, -0.92387953251128674f, -0.70710678118654752f, -0.38268343236508977f,
    0.0f, 0.38268343236508977f, 0.70710678118654752f, 0.92387953251128674f,
    1.0f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508977f};

template <typename C> __device__ __forceinline__ C w16(int k);
template <> __device__ __forceinline__ float2 w16<float2>(int k) {
  return make_float2(kW16reF[k], kW16imF[k]);
}
template <> __device__ __forceinline__ double2 w16<double2>(int k) {
  return make_double2(kW16re[k], kW16im[k]);
}

// In-register DFT of length R (forward), natural order in and out.
template <int R, typename C> struct DFT;
template <typename C> struct DFT<1, C> {
  __device__ static __forceinline__ void run(C*) {}
};
template <typename C> struct DFT<2, C> {
  __device__ static __forceinline__ void run(C* a) {
    C t = a[0];
    a[0] = cadd(t, a[1]);
    a[1] = csub(t, a[1]);
  }
};
template <typename C> struct DFT<4, C> {
  __device__ static __forceinline__ void run(C* a) {
    C t0 = cadd(a[0], a[2]), t1 = csub(a[0], a[2]);
    C t2 = cadd(a[1], a[3]), t3 = cmul_mi(csub(a[1], a[3]));
    a[0] = cadd(t0, t2);
    a[2] = csub(t0, t2);
    a[1] = cadd(t1, t3);
    a[3] = csub(t1, t3);
  }
};
// Radix-2 split of a length-R DFT into two of length R/2 (R = 8, 16).
template <int R, typename C> struct DFTsplit {
  __device__ static __forceinline__ void run(C* a) {
    C e[R / 2], o[R / 2];
#pragma unroll
    for (int i = 0; i < R / 2; ++i) { e[i] = a[2 * i]; o[i] = a[2 * i + 1]; }
    DFT<R / 2, C>::run(e);
    DFT<R / 2, C>::run(o);
#pragma unroll
    for (int k = 0; k < R / 2; ++k) {
      C t = cmul(o[k], w16<C>(k * (16 / R)));
      a[k] = cadd(e[k], t);
      a[k + R / 2] = csub(e[k], t);
    }
  }
};
template <typename C> struct DFT<8, C> {
  __device__ static __forceinline__ void run(C* a) { DFTsplit<8, C>::run(a); }
};
template <typename C> struct DFT<16, C> {
  __device__ static __forceinline__ void run(C* a) { DFTsplit<16, C>::run(a); }
};

// One Stockham pass of radix RAD over a length-M transform in shared memory s[0..M), current
// sub-transform length SPAN.  Item i in [0, M/RAD): reads s[i + r M/RAD], applies the twiddles
// e^{-2 pi i r k / (SPAN RAD)} (k = i mod SPAN), takes a radix-RAD DFT and writes
// s[(i - k) RAD + k + r SPAN].  All reads of the pass finish before any write (barrier), so the
// pass is in place.  Each of the TPT threads of the transform handles M / (RAD TPT) items.
template <typename C, int M, int RAD, int SPAN, int TPT>
__device__ __forceinline__ void stockham_pass(C* s, int lt, const C* __restrict__ W) {
  constexpr int ITEMS = M / RAD / TPT;
  C v[ITEMS * RAD];
#pragma unroll
  for (int it = 0; it < ITEMS; ++it) {
    const int i = lt + it * TPT;
    const int k = i & (SPAN - 1);
#pragma unroll
    for (int r = 0; r < RAD; ++r) v[it * RAD + r] = s[pad16(i + r * (M / RAD))];
    if (SPAN > 1) {
#pragma unroll
      for (int r = 1; r < RAD; ++r)
        v[it * RAD + r] = cmul(v[it * RAD + r], __ldg(W + r * k * (M / (SPAN * RAD))));
    }
    DFT<RAD, C>::run(&v[it * RAD]);
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < ITEMS; ++it) {
    const int i = lt + it * TPT;
    const int k = i & (SPAN - 1);
    const int j0 = (i - k) * RAD + k;
#pragma unroll
    for (int r = 0; r < RAD; ++r) s[pad16(j0 + r * SPAN)] = v[it * RAD + r];
  }
  __syncthreads();
}

template <typename C, int M, int SPAN, int TPT>
struct FFTPasses {
  __device__ static __forceinline__ void run(C* s, int lt, const C* W) {
    constexpr int RAD = (M / SPAN) >= 16 ? 16 : (M / SPAN);
    stockham_pass<C, M, RAD, SPAN, TPT>(s, lt, W);
    FFTPasses<C, M, SPAN * RAD, TPT>::run(s, lt, W);
  }
};
template <typename C, int M, int TPT>
struct FFTPasses<C, M, M, TPT> {
  __device__ static __forceinline__ void run(C*, int, const C*) {}
};

// FP32 transforms up to M = 8192 are limited to 64 registers so that two CTAs share an SM.
template <typename R, int M>
__global__ void __launch_bounds__((M / 16) > 256 ? (M / 16) : 256,
                                  (sizeof(R) == 4 && M <= 8192) ? 2 : 1)
bluestein_kernel(DevPlan d) {
  using C = typename Cx<R>::T;
  constexpr int TPT = M / 16;                      // threads per transform
  constexpr int G = (M >= 4096) ? 1 : 4096 / M;    // transforms per CTA
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int g = threadIdx.x / TPT;
  const int lt = threadIdx.x - g * TPT;
  const int64_t per_q = (int64_t)d.K * d.nsub;
  const int64_t total = per_q * d.nq;
  const int64_t tid = (int64_t)blockIdx.x * G + g;
  const bool active = tid < total;
  int qi = 0, j = 0, sub = 0;
  if (active) {
    qi = (int)(tid / per_q);
    const int rem = (int)(tid - (int64_t)qi * per_q);
    j = rem / d.nsub;
    sub = rem - j * d.nsub;
  }
  const int p = d.p[j];
  const int64_t off = (int64_t)qi * d.m + d.nodeoff[j] + (int64_t)sub * p;
  const C* in = reinterpret_cast<const C*>(d.samples) + off;
  C* out = reinterpret_cast<C*>(d.bins) + off;
  const C* chirp = reinterpret_cast<const C*>(d.chirp) + (int64_t)j * d.pmax;
  const C* vhat = reinterpret_cast<const C*>(d.vhat) + (int64_t)j * M;
  const C* W = reinterpret_cast<const C*>(d.fftw);
  C* s = buf + g * padded_len<M>();

  for (int n = lt; n < M; n += TPT)
    s[pad16(n)] = (active && n < p) ? cmul(in[n], __ldg(chirp + n)) : czero<C>();
  __syncthreads();
  FFTPasses<C, M, 1, TPT>::run(s, lt, W);
  for (int n = lt; n < M; n += TPT) s[pad16(n)] = cconj(cmul(s[pad16(n)], __ldg(vhat + n)));
  __syncthreads();
  FFTPasses<C, M, 1, TPT>::run(s, lt, W);
  if (active)
    for (int c = lt; c < p; c += TPT) out[c] = cmul(cconj(s[pad16(c)]), __ldg(chirp + c));
}

template <typename R, int M>
cudaError_t launch_M(const DevPlan& d, cudaStream_t st) {
  using C = typename Cx<R>::T;
  constexpr int G = (M >= 4096) ? 1 : 4096 / M;
  constexpr int threads = (M / 16) * G;
  const size_t smem = (size_t)G * padded_len<M>() * sizeof(C);
  cudaError_t e = cudaFuncSetAttribute(bluestein_kernel<R, M>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t total = (int64_t)d.K * d.nsub * d.nq;
  const unsigned grid = (unsigned)((total + G - 1) / G);
  bluestein_kernel<R, M><<<grid, threads, smem, st>>>(d);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_prec(const DevPlan& d, cudaStream_t st) {
  switch (d.fftM) {
    case 64: return launch_M<R, 64>(d, st);
    case 128: return launch_M<R, 128>(d, st);
    case 256: return launch_M<R, 256>(d, st);
    case 512: return launch_M<R, 512>(d, st);
    case 1024: return launch_M<R, 1024>(d, st);
    case 2048: return launch_M<R, 2048>(d, st);
    case 4096: return launch_M<R, 4096>(d, st);
    case 8192: return launch_M<R, 8192>(d, st);
    case 16384:
      if constexpr (sizeof(R) == 4) return launch_M<R, 16384>(d, st);
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_bluestein(const DevPlan& d, cudaStream_t st) {
  return d.prec == SFT_FP32 ? launch_prec<float>(d, st) : launch_prec<double>(d, st);
}

}  // namespace sft
