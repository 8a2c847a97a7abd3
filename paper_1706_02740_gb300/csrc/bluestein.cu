// Kernel (b): the inner SFT's measurements E_c = (1/p) sum_k h(x_k) e^{-2 pi i k c / p}, c = 0..p-1,
// of every node subset (eq. DFT_GKlam_Comp), for every shift and prime at once.
//
// Each p_j is prime, so the length-p DFT is taken as a chirp convolution (Bluestein): with
// w_n = e^{-pi i n^2 / p},  E_c = (1/p) w_c sum_k (h_k w_k) conj(w_{c-k}),  a linear convolution
// done as a cyclic one of length M >= 2p - 1, M = r 2^k with r = 1, 3, 5 or 7 (the smallest):
//     E = w . conj( FFT( conj( FFT(h w, zero padded) . V ) ) ),
// V = FFT(conj(w) wrapped) / (M p) precomputed per prime in FP64 on the host (the inverse FFT is the
// forward one between two conjugations).  One transform lives in shared memory; the FFT is an
// in-place Stockham schedule whose passes hold at most 16 complex values per thread in registers:
// a radix-2 first pass, radix-16 passes, then the passes that M needs (radix 2/4/8, or 3/6/12,
// 5/10 or 7/14, possibly followed by a radix 2 or 4), with twiddles read from exactly rounded
// per-pass tables.  The radix 5 and 7 butterflies pair the terms k and T - k (real cosine and sine
// sums); 6, 10, 12 and 14 are prime-factor compositions without internal twiddles.  Since
// p <= M/2, the first FFT's radix-2 pass only duplicates its input and is skipped.
// The shared-memory layout inserts one pad element after every 16 (index n -> n + n/16), so the
// strided stores of the short-span passes hit distinct banks.
#include <stdint.h>
#include <string.h>

#include <mutex>
#include <string>

#include "checks.cuh"
#include "cplx.cuh"
#include "fft_radix.cuh"
#include "sft_internal.h"

namespace sft {

namespace {

// Where a pass takes its input and puts its output.  The chirp convolution folds its pointwise
// steps into the passes: the first FFT's first pass reads the chirp-multiplied samples (zero from p
// on) from the first p entries of shared memory, and the second FFT's last pass writes conj(.) times
// the chirp straight to the p outputs.  Other passes read and write shared memory.
enum { kFromSmem = 0, kFromInput = 1 };
enum { kToSmem = 0, kToOutput = 1 };

template <typename C>
struct ChirpIO {
  const C* in;
  const C* chirp;
  const C* vhat;
  C* out;
  int p;          // 0 for an inactive transform slot: nothing is read or written
};

// v[r] *= w^r, w = e^{-2 pi i k / (SPAN RAD)}, r = 4a + c, from the pass's table rows w^1, w^2, w^3
// (and w^4, w^8, w^12 below RAD): w^r is w^c, (w^4)^a, or their product, so every twiddle is at
// most one rounding away from the exactly rounded table.  Lanes with consecutive k read
// consecutive table entries.
template <typename C, int M, int RAD, int SPAN>
__device__ __forceinline__ void apply_twiddles(const C* __restrict__ W, int k, C* v) {
  constexpr int base = fft_tw_offset(M, SPAN);
  if constexpr (RAD == 2) {
    v[1] = cmul(v[1], __ldg(W + base + k));
  } else if constexpr (RAD == 3) {
    v[1] = cmul(v[1], __ldg(W + base + k));
    v[2] = cmul(v[2], __ldg(W + base + SPAN + k));
  } else {
    const C w1 = __ldg(W + base + k), w2 = __ldg(W + base + SPAN + k),
            w3 = __ldg(W + base + 2 * SPAN + k);
    v[1] = cmul(v[1], w1);
    v[2] = cmul(v[2], w2);
    v[3] = cmul(v[3], w3);
#pragma unroll
    for (int a = 1; 4 * a < RAD; ++a) {
      const C P = __ldg(W + base + (2 + a) * SPAN + k);     // w^{4a}
      v[4 * a] = cmul(v[4 * a], P);
      if (4 * a + 1 < RAD) v[4 * a + 1] = cmul(v[4 * a + 1], cmul(P, w1));
      if (4 * a + 2 < RAD) v[4 * a + 2] = cmul(v[4 * a + 2], cmul(P, w2));
      if (4 * a + 3 < RAD) v[4 * a + 3] = cmul(v[4 * a + 3], cmul(P, w3));
    }
  }
}

// One Stockham pass of radix RAD over a length-M transform, current sub-transform length SPAN.
// Item i in [0, M/RAD): takes element i + r M/RAD, applies the twiddles e^{-2 pi i r k / (SPAN RAD)}
// (k = i mod SPAN), takes a radix-RAD DFT and puts element (i - k) RAD + k + r SPAN.  All reads of
// the pass finish before any shared-memory write (barrier), so the pass is in place.  Each of the
// TPT threads of the transform handles M / (RAD TPT) items, rounded up (a radix-16 pass of a
// length 3 2^k has 3/4 of an item per thread: the rest of the threads only wait at the barrier).
//
// LOAD == kFromInput is the first pass after the radix-2 first pass of a transform whose input
// x vanishes from p <= M/2 on: that radix-2 pass only duplicates (y[2i] = y[2i + 1] = x[i]), so it
// is never run and this pass reads y[n] = x[n / 2] from the first p entries of shared memory.
// (Forming x = h w from global memory inside this pass instead of a staging sweep measured slower:
// length 6144, 589 against 480 us per 16 SFTs.)
// Offsets of an item's elements: (a + 16 e) >> 4 = (a >> 4) + e, so when the element stride d is
// a multiple of 16, pad16(a + r d) = pad16(a) + r (d + d / 16): one padded base per item and
// compile-time offsets instead of a shift and an add per access.
template <typename C, int M, int RAD, int SPAN, int TPT, int LOAD, int STORE>
__device__ __forceinline__ void stockham_pass(C* s, int lt, const C* __restrict__ W,
                                              const ChirpIO<C>& io) {
  constexpr int NI = M / RAD;              // items of the pass
  constexpr int ITEMS = (NI + TPT - 1) / TPT;
  constexpr bool EVEN = NI % TPT == 0;
  constexpr int STRIDE = M / RAD;          // input stride of an item's elements
  C v[ITEMS * RAD];
#pragma unroll
  for (int it = 0; it < ITEMS; ++it) {
    const int i = lt + it * TPT;
    const int k = i % SPAN;
    if (!EVEN && i >= NI) continue;
    if (LOAD == kFromInput) {
      // element n = i + r STRIDE reads x[n / 2] = x[(i >> 1) + r STRIDE / 2] (STRIDE is even)
      const int m0 = i >> 1, pm0 = pad16(m0);
#pragma unroll
      for (int r = 0; r < RAD; ++r) {
        const int m = m0 + r * (STRIDE / 2);
        const int pm = (STRIDE / 2) % 16 == 0 ? pm0 + r * ((STRIDE / 2) + (STRIDE / 2) / 16)
                                               : pad16(m);
        v[it * RAD + r] = (m < io.p) ? s[pm] : czero<C>();
      }
    } else {
      const int p0 = pad16(i);
#pragma unroll
      for (int r = 0; r < RAD; ++r) {
        const int pn = STRIDE % 16 == 0 ? p0 + r * (STRIDE + STRIDE / 16) : pad16(i + r * STRIDE);
        v[it * RAD + r] = s[pn];
      }
    }
    apply_twiddles<C, M, RAD, SPAN>(W, k, &v[it * RAD]);
    DFT<RAD, C>::run(&v[it * RAD]);
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < ITEMS; ++it) {
    const int i = lt + it * TPT;
    const int k = i % SPAN;
    if (!EVEN && i >= NI) continue;
    const int j0 = (i - k) * RAD + k;
    if (STORE == kToOutput) {
#pragma unroll
      for (int r = 0; r < RAD; ++r) {
        const int c = j0 + r * SPAN;
        if (c < io.p) io.out[c] = cmul(cconj(v[it * RAD + r]), __ldg(io.chirp + c));
      }
    } else {
      const int p0 = pad16(j0);
#pragma unroll
      for (int r = 0; r < RAD; ++r) {
        const int pc = SPAN % 16 == 0 ? p0 + r * (SPAN + SPAN / 16) : pad16(j0 + r * SPAN);
        s[pc] = v[it * RAD + r];
      }
    }
  }
  if (STORE == kToSmem) __syncthreads();
}

// The passes from sub-transform length SPAN (>= 2) to M.
template <typename C, int M, int SPAN, int TPT, int LOAD, int STORE>
struct FFTPasses {
  __device__ static __forceinline__ void run(C* s, int lt, const C* W, const ChirpIO<C>& io) {
    constexpr int RAD = fft_radix(M, SPAN);
    constexpr bool last = SPAN * RAD == M;
    stockham_pass<C, M, RAD, SPAN, TPT, LOAD, last ? STORE : kToSmem>(s, lt, W, io);
    FFTPasses<C, M, SPAN * RAD, TPT, kFromSmem, STORE>::run(s, lt, W, io);
  }
};
template <typename C, int M, int TPT, int LOAD, int STORE>
struct FFTPasses<C, M, M, TPT, LOAD, STORE> {
  __device__ static __forceinline__ void run(C*, int, const C*, const ChirpIO<C>&) {}
};

// The radix-2 first pass (SPAN 1, no twiddles) in shared memory: y[2i] = x[i] + x[i + M/2],
// y[2i + 1] = x[i] - x[i + M/2].  (Fusing the filter product into this pass, or into the previous
// pass's stores, keeps 16 more values in flight and spills at the 64-register budget.)
template <typename C, int M, int TPT>
__device__ __forceinline__ void radix2_first(C* s, int lt) {
  constexpr int ITEMS = M / 2 / TPT;
  static_assert(ITEMS * TPT == M / 2, "whole items per thread");
  C v[2 * ITEMS];
#pragma unroll
  for (int it = 0; it < ITEMS; ++it) {
    const int i = lt + it * TPT;
    const int pi = pad16(i);
    const C a = s[pi], b = s[pi + M / 2 + M / 32];       // pad16(i + M/2), M/2 a multiple of 16
    v[2 * it] = cadd(a, b);
    v[2 * it + 1] = csub(a, b);
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < ITEMS; ++it) {
    const int i = lt + it * TPT;
    const int pe = pad16(2 * i);                          // 2i even: 2i + 1 pads to pe + 1
    s[pe] = v[2 * it];
    s[pe + 1] = v[2 * it + 1];
  }
  __syncthreads();
}

// A CTA holds blockDim.x / fft_tpt(M) transforms, at most max(fft_tpt(M), 256) threads.  MINB is
// the builds' CTAs-per-SM target, which holds every FP32 build to 64 registers: two CTAs of 512
// threads (M = 5120 .. 8192) or four of 256 (M <= 4096; the earlier 128-register build of these
// lengths ran the mixed 4096-signal batch's transforms in 32.4 against 24.0 ms).
template <int M> constexpr int dft_max_threads() { return fft_tpt(M) > 256 ? fft_tpt(M) : 256; }

template <typename R, int M, int MINB>
__global__ void __launch_bounds__(dft_max_threads<M>(), MINB)
bluestein_kernel(BatchView bv) {
  pdl_begin();
  using C = typename Cx<R>::T;
  constexpr int TPT = fft_tpt(M);                  // threads per transform
  const int G = blockDim.x / TPT;                  // transforms per CTA
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  int lb, nb;
  const DevPlan& d = bv.plans[batch_signal(bv, lb, nb)];
  const int g = threadIdx.x / TPT;
  const int lt = threadIdx.x - g * TPT;
  const int per_q = d.K * d.nsub;
  const int total = per_q * d.nq;
  const int tid = lb * G + g;
  const bool active = tid < total;
  int qi = 0, j = 0, sub = 0;
  if (active) {
    qi = tid / per_q;
    const int rem = tid - qi * per_q;
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
  const bool inside = active && index_ok(d, off + p - 1, (int64_t)d.nq * d.m, SFT_SITE_DFT);
  const ChirpIO<C> io{in, chirp, vhat, out, inside ? p : 0};
  // p <= M/2: at most 8 (or 7, 6, 5) input elements per thread.  (The unroll factors of this and
  // the filter sweep are the largest that keep the FP32 builds free of register spills.)
#pragma unroll 4
  for (int it = 0; it < M / 2 / TPT; ++it) {
    const int n = lt + it * TPT;
    if (n < io.p) s[pad16(n)] = cmul(__ldg(in + n), __ldg(chirp + n));
  }
  __syncthreads();
  FFTPasses<C, M, 2, TPT, kFromInput, kToSmem>::run(s, lt, W, io);
  // the filter product, conjugated, in its own sweep: folded into the radix-2 pass below it adds
  // sixteen loads in flight per thread (spills at 64 registers) and, fenced to fewer, measured
  // slower (length 6144: 675 against 480 us per 16 SFTs)
#pragma unroll 8
  for (int it = 0; it < M / TPT; ++it) {
    const int n = lt + it * TPT;
    s[pad16(n)] = cconj(cmul(s[pad16(n)], __ldg(vhat + n)));
  }
  __syncthreads();
  radix2_first<C, M, TPT>(s, lt);
  FFTPasses<C, M, 2, TPT, kFromSmem, kToOutput>::run(s, lt, W, io);
}
template <typename R, int M, int MINB>
cudaError_t launch_MB(const BatchView& bv, const LaunchSet& ls, cudaStream_t st, int* launched) {
  using C = typename Cx<R>::T;
  const int stage = fft_stage(M);
  const unsigned grid = (unsigned)ls.blocks[stage];
  if (grid == 0) return cudaSuccess;
  const int G = ls.tune.dft_per_cta[fft_tune_class(M)];
  const int threads = fft_tpt(M) * G;
  const size_t smem = (size_t)G * padded_len<M>() * sizeof(C);
  cudaError_t e = ensure_dynamic_smem<bluestein_kernel<R, M, MINB>>(smem);
  if (e != cudaSuccess) return e;
  BatchView v = bv;
  v.blk = ls.blk[stage];
  (void)launch_pdl(bluestein_kernel<R, M, MINB>, grid, threads, smem, st, v);
  if (launched) ++*launched;
  return cudaGetLastError();
}

template <typename R, int M>
cudaError_t launch_M(const BatchView& bv, const LaunchSet& ls, cudaStream_t st, int* launched) {
  if constexpr (sizeof(R) == 4 && M == 8192) {
    if (!ls.tune.dft_two_ctas) return launch_MB<R, M, 1>(bv, ls, st, launched);
  }
  constexpr int MINB = sizeof(R) != 4 ? 1 : fft_tpt(M) <= 256 ? 4 : fft_tpt(M) <= 512 ? 2 : 1;
  return launch_MB<R, M, MINB>(bv, ls, st, launched);
}

template <typename R>
cudaError_t launch_prec(const BatchView& bv, const LaunchSet& ls, cudaStream_t st, int* launched) {
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = launch_M<R, 64>(bv, ls, st, launched);
  if (e == cudaSuccess) e = launch_M<R, 128>(bv, ls, st, launched);
  if (e == cudaSuccess) e = launch_M<R, 256>(bv, ls, st, launched);
  if (e == cudaSuccess) e = launch_M<R, 512>(bv, ls, st, launched);
  if (e == cudaSuccess) e = launch_M<R, 1024>(bv, ls, st, launched);
  if (e == cudaSuccess) e = launch_M<R, 2048>(bv, ls, st, launched);
  if (e == cudaSuccess) e = launch_M<R, 4096>(bv, ls, st, launched);
  if (e == cudaSuccess) e = launch_M<R, 8192>(bv, ls, st, launched);
  if constexpr (sizeof(R) == 4)
    if (e == cudaSuccess) e = launch_M<R, 16384>(bv, ls, st, launched);
  if (e == cudaSuccess) e = launch_M<R, 96>(bv, ls, st, launched);
  if (e == cudaSuccess) e = launch_M<R, 192>(bv, ls, st, launched);
  if (e == cudaSuccess) e = launch_M<R, 384>(bv, ls, st, launched);
  if (e == cudaSuccess) e = launch_M<R, 768>(bv, ls, st, launched);
  if (e == cudaSuccess) e = launch_M<R, 1536>(bv, ls, st, launched);
  if (e == cudaSuccess) e = launch_M<R, 3072>(bv, ls, st, launched);
  if (e == cudaSuccess) e = launch_M<R, 6144>(bv, ls, st, launched);
  if (e == cudaSuccess) e = launch_M<R, 640>(bv, ls, st, launched);
  if (e == cudaSuccess) e = launch_M<R, 1280>(bv, ls, st, launched);
  if (e == cudaSuccess) e = launch_M<R, 2560>(bv, ls, st, launched);
  if (e == cudaSuccess) e = launch_M<R, 5120>(bv, ls, st, launched);
  if (e == cudaSuccess) e = launch_M<R, 896>(bv, ls, st, launched);
  if (e == cudaSuccess) e = launch_M<R, 1792>(bv, ls, st, launched);
  if (e == cudaSuccess) e = launch_M<R, 3584>(bv, ls, st, launched);
  if (e == cudaSuccess) e = launch_M<R, 7168>(bv, ls, st, launched);
  if constexpr (sizeof(R) == 4) {
    if (e == cudaSuccess) e = launch_M<R, 12288>(bv, ls, st, launched);
    if (e == cudaSuccess) e = launch_M<R, 10240>(bv, ls, st, launched);
    if (e == cudaSuccess) e = launch_M<R, 14336>(bv, ls, st, launched);
  }
  return e;
}

}  // namespace

// The DFT stage: the chirp-convolution launches of every length class present, then the Rader
// launch when some signal takes that form.
cudaError_t launch_bluestein(const DevPlan& d0, const BatchView& bv, const LaunchSet& ls,
                             cudaStream_t st, int* launched) {
  cudaError_t e = d0.prec == SFT_FP32 ? launch_prec<float>(bv, ls, st, launched)
                                      : launch_prec<double>(bv, ls, st, launched);
  if (e == cudaSuccess && ls.blocks[kStRader] > 0) e = launch_rader(d0, bv, ls, st, launched);
  return e;
}

int bluestein_blocks(const DevPlan& d, int M, int per_cta) {
  if (d.fftM != M) return 0;
  const int total = d.nq * d.K * d.nsub;
  return (total + per_cta - 1) / per_cta;
}

// ---------------------------------------------------------------------------------------------
// Batched DFT that allocates nothing (sft_dft_noalloc).
//
// Its tables (the chirp, the transformed filter and the FFT twiddles) live in one file-scope
// device array of a fixed size; every GPU that loads the library holds it until the process
// exits.  They are built on the device by the two kernels below the first time a length is used
// on a device, and rebuilt when the length changes; the transforms themselves run through the
// same chirp-convolution kernel as the sparse transform.
// ---------------------------------------------------------------------------------------------
namespace {

constexpr int kNoAllocMaxN = 8191;           // longest transform: 2n - 1 <= 16384
constexpr int kNoAllocMaxM = 16384;
constexpr int kNoAllocChirp = 8192;
constexpr size_t kNoAllocHead = (sizeof(DevPlan) + 4095) / 4096 * 4096;   // the launch's plan record
static_assert(sizeof(DevPlan) <= kNoAllocHead, "plan record must fit the head of the array");
constexpr size_t kNoAllocBytes =
    kNoAllocHead + sizeof(float2) * ((size_t)kNoAllocChirp + 2 * (size_t)kNoAllocMaxM);
constexpr int kMaxDevices = 64;

// plan record [20 KiB] | chirp [8192] | filter spectrum [16384] | twiddles [16384] (complex64):
// 340 KiB in all
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
unsigned char* g_noalloc_ptr[kMaxDevices];  // device address of g_noalloc_scratch, per device
int g_noalloc_n[kMaxDevices];           // length the tables currently hold (0 = none)

// Twiddles in the per-pass layout of the chirp convolution's FFT (entry e^{-2 pi i e_t k / (SPAN R)}
// of the pass at SPAN, row t, column k), the chirp w_k = e^{-pi i (k^2 mod 2n) / n} (k < n)
// and the wrapped conjugate chirp V (V[k] = V[M - k] = conj(w_k), zero elsewhere), in FP64 then
// rounded.
__global__ void noalloc_tables_kernel(int n, int M, float2* chirp, float2* V, float2* W) {
  pdl_begin();
  const int entries = fft_tw_entries(M);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
    double s, c;
    if (i < entries) {
      int span = 2, off = 0;
      while (true) {
        const int R = fft_radix(M, span), rows = fft_tw_rows(R);
        if (i < off + rows * span) {
          const int row = (i - off) / span, k = (i - off) - row * span;
          sincospi(-2.0 * (double)(fft_tw_exp(row) * k) / (double)(span * R), &s, &c);
          W[i] = make_float2((float)c, (float)s);
          break;
        }
        off += rows * span;
        span *= R;
      }
    }
    int k = -1;
    if (i < n) k = i;
    else if (i > M - n) k = M - i;
    float2 v = make_float2(0.f, 0.f);
    if (k >= 0) {
      const int r = (k * k) % (2 * n);                 // k < 8192: k^2 < 2^26
      sincospi(-(double)r / (double)n, &s, &c);
      v = make_float2((float)c, -(float)s);
      if (i < n) chirp[i] = make_float2((float)c, (float)s);
    }
    V[i] = v;
  }
}

// Filter spectrum: FFT_M(V) / (M n), one CTA, the same shared-memory Stockham passes.
template <int M>
__global__ void __launch_bounds__(M / 16) noalloc_filter_kernel(int n, float2* V, const float2* W) {
  pdl_begin();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* s = reinterpret_cast<float2*>(smem_raw);
  constexpr int TPT = M / 16;
  const int lt = threadIdx.x;
  for (int i = lt; i < M; i += TPT) s[pad16(i)] = V[i];
  __syncthreads();
  const ChirpIO<float2> io{nullptr, nullptr, nullptr, nullptr, 0};
  radix2_first<float2, M, TPT>(s, lt);
  FFTPasses<float2, M, 2, TPT, kFromSmem, kToSmem>::run(s, lt, W, io);
  const float scale = (float)(1.0 / ((double)M * (double)n));
  for (int i = lt; i < M; i += TPT) V[i] = cscale(s[pad16(i)], scale);
}

// The launch record of one call, written on the device (the fields the chirp-convolution kernel
// reads; the rest of the record stays zero).  Its arguments travel by value with the launch, so
// the call copies nothing from host memory.
__global__ void noalloc_record_kernel(DevPlan* rec, int n, int batch, int M, void* in, void* out,
                                      const float2* base) {
  pdl_begin();
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  rec->prec = SFT_FP32;
  rec->K = 1;
  rec->nsub = 1;
  rec->nq = batch;
  rec->p[0] = n;
  rec->nodeoff[0] = 0;
  rec->nodeoff[1] = n;
  rec->m = n;
  rec->pmax = n;
  rec->fftM = M;
  rec->samples = in;
  rec->bins = out;
  rec->chirp = base;
  rec->vhat = base + kNoAllocChirp;
  rec->fftw = base + kNoAllocChirp + kNoAllocMaxM;
  rec->counters = nullptr;          // no status words
}

template <int M>
cudaError_t noalloc_build(int n, float2* base, cudaStream_t st) {
  float2* chirp = base;
  float2* V = base + kNoAllocChirp;
  float2* W = V + kNoAllocMaxM;
  (void)launch_pdl(noalloc_tables_kernel, (M + 255) / 256, 256, 0, st, n, M, chirp, V, W);
  const size_t smem = (size_t)padded_len<M>() * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(noalloc_filter_kernel<M>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  (void)launch_pdl(noalloc_filter_kernel<M>, 1, M / 16, smem, st, n, V, W);
  return cudaGetLastError();
}

cudaError_t noalloc_build_any(int n, int M, float2* base, cudaStream_t st) {
  switch (M) {
    case 64: return noalloc_build<64>(n, base, st);
    case 128: return noalloc_build<128>(n, base, st);
    case 256: return noalloc_build<256>(n, base, st);
    case 512: return noalloc_build<512>(n, base, st);
    case 1024: return noalloc_build<1024>(n, base, st);
    case 2048: return noalloc_build<2048>(n, base, st);
    case 4096: return noalloc_build<4096>(n, base, st);
    case 8192: return noalloc_build<8192>(n, base, st);
    case 16384: return noalloc_build<16384>(n, base, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

}  // namespace sft

extern "C" sft_status sft_dft_noalloc(int32_t n, int32_t batch, const void* in_dev, void* out_dev,
                                      void* stream) {
  using namespace sft;
  if (n < 2 || n > kNoAllocMaxN) {
    set_error("sft_dft_noalloc: length must be in 2..8191 (the static table holds at most 8191)");
    return SFT_EINVAL;
  }
  if (batch < 1 || !in_dev || !out_dev || ((uintptr_t)in_dev % 8) || ((uintptr_t)out_dev % 8)) {
    set_error("sft_dft_noalloc: need batch >= 1 and non-NULL 8-byte aligned buffers");
    return SFT_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    set_error("sft_dft_noalloc: no usable current device");
    return SFT_ECUDA;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int M = 64;
  while (M < 2 * n - 1) M <<= 1;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_error(std::string("sft_dft_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
      return SFT_ECUDA;
    }
    g_noalloc_ptr[dev] = reinterpret_cast<unsigned char*>(p);
  }
  DevPlan* rec = reinterpret_cast<DevPlan*>(g_noalloc_ptr[dev]);
  float2* base = reinterpret_cast<float2*>(g_noalloc_ptr[dev] + kNoAllocHead);
  if (g_noalloc_n[dev] != n) {
    // building the tables must run now, not in a graph that may never be launched
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(st, &cap);
    if (e != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
      (void)cudaGetLastError();
      set_error("sft_dft_noalloc: the first call with a new length (which builds the tables) "
                "must not be made while the stream is being captured");
      return SFT_EINVAL;
    }
    e = noalloc_build_any(n, M, base, st);
    if (e != cudaSuccess) {
      g_noalloc_n[dev] = 0;
      set_error(std::string("sft_dft_noalloc: table build failed: ") + cudaGetErrorString(e));
      return SFT_ECUDA;
    }
    g_noalloc_n[dev] = n;
  }
  (void)launch_pdl(noalloc_record_kernel, 1, 32, 0, st, rec, (int)n, (int)batch, M,
                   const_cast<void*>(in_dev), out_dev, (const float2*)base);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("sft_dft_noalloc: record launch failed: ") + cudaGetErrorString(e));
    return SFT_ECUDA;
  }
  // the host's view of the same record, for the block count
  DevPlan d;
  memset(&d, 0, sizeof(d));
  d.K = 1;
  d.nsub = 1;
  d.nq = batch;
  d.fftM = M;
  BatchView bv;
  memset(&bv, 0, sizeof(bv));
  bv.plans = rec;
  bv.n = 1;
  LaunchSet ls;
  memset(&ls, 0, sizeof(ls));
  ls.tune = default_tuning();
  ls.kmax = 1;
  int lg = 0;
  while ((1 << lg) < M) ++lg;
  ls.blocks[kStBluestein0 + lg - 6] = bluestein_blocks(d, M, ls.tune.dft_per_cta[lg - 6]);
  e = launch_prec<float>(bv, ls, st, nullptr);
  if (e != cudaSuccess) {
    set_error(std::string("sft_dft_noalloc: launch failed: ") + cudaGetErrorString(e));
    return SFT_ECUDA;
  }
  return SFT_OK;
}
