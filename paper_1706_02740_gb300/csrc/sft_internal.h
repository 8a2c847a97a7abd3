// Internal declarations shared by the plan, the kernels and the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/sft.h"

namespace sft {

constexpr int kMaxK = SFT_MAX_K;          // prime moduli (the deterministic inner SFT needs many)
constexpr int kFewK = 16;                 // per-thread median arrays in registers up to this K
constexpr int kMaxT = SFT_MAX_SMALL;      // small moduli
constexpr int kMaxQ = SFT_MAX_SHIFTS;     // shifts
constexpr int kMaxKappa = 48;             // window half-width
constexpr int kMaxSub = 128;              // node subsets per prime: 1 + sum_l (t_l - 1)
constexpr int kMaxFFT32 = 16384;          // chirp convolution length, FP32 (128 KiB of smem)
constexpr int kMaxFFT64 = 8192;           // FP64 (128 KiB of smem)
constexpr int64_t kNoFreq = INT64_MIN;    // "no frequency" marker in candidate arrays
// Rader's form: cyclic convolutions of length L = p - 1 over two shared-memory buffers of
// rader_buf(L) elements each (one transform per CTA).
constexpr int kRaderMaxL32 = 13600;
constexpr int kRaderMaxL64 = 6800;
constexpr int kRaderSched = 32;           // per prime: [0] passes, [1..15] radices, [16..30] row offsets
constexpr int kRaderMaxPasses = 15;
__host__ __device__ constexpr int rader_buf(int L) { return L + (L - 1) / 16; }

// Record of one voted frequency of one shift (written by the vote/median kernel).
struct Voted {
  int64_t w;       // frequency in B
  double zre, zim; // median estimate (FP64 storage; FP32 path values are FP32-exact)
  int32_t votes;
  int32_t jmin;
};

// Record of one in-band, filter-divided coefficient (per-shift top-s, Algorithm 1's R-hat).
struct Pooled {
  int64_t w;
  double cre, cim;
  int32_t qi;      // shift index
  int32_t pad;
};

// Everything a kernel needs about a plan (read by the kernels from device memory).
struct DevPlan {
  int64_t N;
  int32_t s, kappa, K, nT, nq, nsub;
  int32_t prec, input;
  int32_t refine;             // FP32 path: re-estimate the winners (sft_variant.refine_fp64)
  int64_t m;                  // distinct nodes: nsub * sum_j p_j
  int32_t Ptot;               // sum_j p_j
  int32_t fftM, fftLog2;      // chirp convolution length (r 2^k, r = 1, 3, 5, 7), floor(log2 fftM);
                              // 0 when the plan takes Rader's form
  int32_t rader;              // 1: the length-p_j DFTs by Rader's algorithm (every p_j - 1 13-smooth)
  int32_t rLmax;              // largest p_j - 1 of a Rader plan
  int32_t rTpt;               // threads per Rader transform chosen for this plan's schedules
  int32_t p[kMaxK];
  int64_t nodeoff[kMaxK + 1]; // first node of prime j
  int32_t poff[kMaxK + 1];    // first bin of prime j
  int64_t Mj[kMaxK];          // p_j * prod(t)
  int32_t t[kMaxT];
  int32_t subbase[kMaxT];     // node subset index of (l, k2 = 1)
  int32_t twoff[kMaxT];       // offset of l's twiddles in twsmall
  int8_t sub_l[kMaxSub];      // small-modulus index of subset u (-1 for u = 0)
  int8_t sub_k2[kMaxSub];     // offset numerator k2 of subset u
  int64_t q[kMaxQ];
  int64_t L;
  double c1;
  double gamma;               // 2 pi^2 / (N c1)^2: Gaussian exponent per squared grid offset
  double G0;                  // 1 / (N c1): weight prefactor
  float gamma32, G032, c1f;   // the same, rounded once to FP32
  float qN32[kMaxQ];          // q / N rounded to FP32 (node phase of the FP32 path)
  // N = Nq p_j + Nr and N = Nq t_l + Nr: 32-bit pieces of the window-centre computation
  int32_t Nqp[kMaxK], Nrp[kMaxK];
  int32_t Nqt[kMaxT], Nrt[kMaxT];
  int32_t nchunk;             // sample chunks of the re-estimation (ceil(pmax / kReChunk))
  int32_t vcap;               // capacity of each shift's voted list
  // device tables
  const void* Ttab;           // [nq][2 kappa + 1] exp(-2 pi i (q i mod N) / N)   (prec type)
  const void* chirp;          // [K][pmax] exp(-pi i (n^2 mod 2p) / p)           (prec type)
  const void* vhat;           // [K][fftM] FFT of the conjugate chirp / (M p)    (prec type)
  const void* fftw;           // [fftM] per-pass FFT twiddles (fft_tw_offset)     (prec type)
  const void* twsmall;        // [sum_l t_l] exp(-2 pi i n / t_l)                (prec type)
  const float2* wp32;         // [K][pmax] exp(-2 pi i n / p_j) for the FP32 re-estimation
  const int32_t* garner;      // [K][nT] (p_j t_1 .. t_{l-1})^{-1} mod t_l
  const int32_t* pinv;        // [K][nT] p_j^{-1} mod t_l
  const int32_t* rsched;      // [K][kRaderSched] Rader pass schedule of p_j - 1
  const int32_t* rperm;       // [K][2][pmax]: g^n mod p_j and g^{-n} mod p_j, n < p_j - 1
  const void* rV;             // [K][pmax]: FFT(b) / (p (p - 1)), b_n = e^{-2 pi i g^{-n} / p} (prec type)
  const void* rtw;            // [K][pmax]: twiddle rows of the length p_j - 1 FFT passes (prec type)
  int32_t pmax;
  // scratch
  void* samples;              // [nq][m] prec complex
  void* bins;                 // [nq][m] prec complex
  int64_t* cand;              // [nq][Ptot]
  uint8_t* resid;             // [nq][Ptot][nT]
  int32_t* counters;          // [0..nq): voted counts, [nq]: pool count, [nq+1]: status word
  Voted* voted;               // [nq][vcap]
  Pooled* pool;               // [nq * s]
  Pooled* winners;            // [s]
  double2* ybuf;              // [s][K][nchunk] partial sums of the re-estimated bins
  int32_t* wlist;             // [s] winner indices grouped by shift
  int32_t* woff;              // [nq + 1] start of each shift's group in wlist
  double* epart;              // [kEnergyBlocks] partial sums of |f|^2 (residual-energy check)
};

constexpr int kReChunk = 512;   // samples per re-estimation CTA (the prime's table is staged once per chunk)
constexpr int kReThreads = 256; // its threads: one winner each per round
constexpr int kResampleMaxThreads = 512;      // largest CTA of the kappa = 4 / 6 resampling kernel
constexpr int kResampleGenericThreads = 128;
constexpr int kBinMaxThreads = 512;    // identify / vote: one thread per bin, at most 512 per CTA
constexpr int kRefineThreads = 64;
constexpr int kEnergyBlocks = 304;     // residual-energy check: two CTAs per SM, fixed reduction order
constexpr int kEnergyThreads = 512;

// ---------------------------------------------------------------------------------------------
// Batches.  One launch of a stage covers every signal of a batch; each signal has its own plan
// (tables and scratch).  Blocks never straddle signals: blk[b] .. blk[b+1] are signal b's blocks
// in this launch (a signal may have none).  A single signal needs no prefix (blk == nullptr).
// ---------------------------------------------------------------------------------------------
struct BatchView {
  const DevPlan* plans;       // [n] device copies of the plans
  int32_t n;
  const int32_t* blk;         // [n + 1] block prefix of this launch, or nullptr when n == 1
  const void* const* f;       // [n] input pointers (device array), or nullptr: f0
  int64_t* const* out_w;      // [n] or nullptr: out_w0
  double2* const* out_c;      // [n] or nullptr: out_c0
  int32_t* const* out_n;      // [n] or nullptr: out_n0
  const void* f0;
  int64_t* out_w0;
  double2* out_c0;
  int32_t* out_n0;
};

#ifdef __CUDACC__
// Signal of this block, its block index within the signal and the signal's block count.
__device__ __forceinline__ int batch_signal(const BatchView& bv, int& lb, int& nb) {
  if (!bv.blk) {
    lb = blockIdx.x;
    nb = gridDim.x;
    return 0;
  }
  int lo = 0, hi = bv.n;
  const int x = blockIdx.x;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (bv.blk[mid] <= x) lo = mid;
    else hi = mid;
  }
  lb = x - bv.blk[lo];
  nb = bv.blk[lo + 1] - bv.blk[lo];
  return lo;
}
__device__ __forceinline__ const void* batch_f(const BatchView& bv, int b) {
  return bv.f ? bv.f[b] : bv.f0;
}
__device__ __forceinline__ int64_t* batch_out_w(const BatchView& bv, int b) {
  return bv.out_w ? bv.out_w[b] : bv.out_w0;
}
__device__ __forceinline__ double2* batch_out_c(const BatchView& bv, int b) {
  return bv.out_c ? bv.out_c[b] : bv.out_c0;
}
__device__ __forceinline__ int32_t* batch_out_n(const BatchView& bv, int b) {
  return bv.out_n ? bv.out_n[b] : bv.out_n0;
}
#endif

// Stages whose per-signal block counts a launch set records.
enum StageKind {
  kStOne = 0,        // one block per signal (counters, global selection, final order)
  kStResample,       // nodes / resampling threads per block
  kStBins,           // shifts * sum p / bin threads per block
  kStShift,          // one block per shift
  kStShiftRank,      // rank fallback of long voted lists (0 for signals that never need it)
  kStGlobalRank,     // rank fallback of long pools
  kStReest,          // shifts * K * chunks
  kStRefine,         // s / 64
  kStFinalRank,      // rank fallback of the final order
  kStRader,          // Rader's form: one transform per block
  kStBluestein0,     // + log2(M) - 6: chirp-convolution lengths 2^k, 64..16384
  kStBluestein3 = kStBluestein0 + 9,   // + log2(M / 96): lengths M = 3 2^k, 96..12288
  kStBluestein5 = kStBluestein3 + 8,   // + log2(M / 640): lengths M = 5 2^k, 640..10240
  kStBluestein7 = kStBluestein5 + 5,   // + log2(M / 896): lengths M = 7 2^k, 896..14336
  kStCount = kStBluestein7 + 5
};

// Host-side description of one execution's launches: total blocks of each stage and the device
// prefix array (nullptr for a single signal).
struct LaunchSet {
  int32_t blocks[kStCount];
  const int32_t* blk[kStCount];
  int32_t pmax;               // largest prime over the signals (shared-memory sizing)
  int32_t rlmax;              // largest p - 1 over the signals in Rader's form (0: none)
  int32_t rtpt;               // threads per Rader transform (largest rTpt over those signals)
  int32_t kmax;               // most prime moduli of any signal (per-thread median arrays)
  sft_tuning tune;            // launch geometry (block shapes; never changes results)
};

// Built-in launch geometry, and the validity check of a caller's (message in *why).
sft_tuning default_tuning();
bool tuning_valid(const sft_tuning& t, std::string* why);

// The chirp convolution's FFT length M is r 2^k with r in {1, 3, 5, 7}: the smallest such length
// >= 2p - 1 (fft_length).  After the radix-2 first pass (no twiddles) the passes run at
// sub-transform lengths SPAN = 2, 2 R_1, ... with radix R = fft_radix(M, SPAN) until SPAN = M:
// radix 16 while at least 16 r is left, then the largest r 2^j <= 16 that divides what is left
// (r = 3: 3, 6, 12; r = 5: 5, 10; r = 7: 7, 14; r = 1: 2, 4, 8), then a last radix 2 or 4 where
// M needs it.  Threads per transform fft_tpt(M) = M / R_r, R_r the largest r 2^j <= 16 (16, 12,
// 10 or 14), so no pass holds more than 16 values per thread.  The pass at SPAN owns
// fft_tw_rows(R) rows of SPAN entries: row t, column k holds e^{-2 pi i e_t k / (SPAN R)} with
// exponents e_t = 1, 2, 3, 4, 8, 12 (those below R); every power r' = 4a + c < R is then one
// product (w^4)^a w^c of two entries.  The rows of all passes are stored one after the other
// (fft_tw_offset); together they hold fewer than M entries.
__host__ __device__ constexpr int fft_odd(int M) {
  return M % 7 == 0 ? 7 : M % 5 == 0 ? 5 : M % 3 == 0 ? 3 : 1;
}
__host__ __device__ constexpr int fft_odd_radix(int r) {   // the largest r 2^j <= 16
  int R = r;
  while (2 * R <= 16) R *= 2;
  return R;
}
__host__ __device__ constexpr int fft_radix(int M, int span) {
  const int rem = M / span, r = fft_odd(M);
  if (r == 1 || rem % r != 0) return rem >= 16 ? 16 : rem;
  if (rem % (16 * r) == 0) return 16;
  int R = r;
  while (2 * R <= 16 && rem % (2 * R) == 0) R *= 2;
  return R;
}
__host__ __device__ constexpr int fft_tpt(int M) { return M / fft_odd_radix(fft_odd(M)); }
__host__ __device__ constexpr int fft_log2(int x) { return x <= 1 ? 0 : 1 + fft_log2(x / 2); }
__host__ __device__ constexpr int fft_tw_rows(int R) {
  return R >= 13 ? 6 : R >= 9 ? 5 : R >= 5 ? 4 : R == 4 ? 3 : R == 3 ? 2 : 1;
}
__host__ __device__ constexpr int fft_tw_exp(int t) { return t < 3 ? t + 1 : 4 * (t - 2); }
__host__ __device__ constexpr int fft_tw_offset(int M, int span) {
  int off = 0;
  for (int s = 2; s < span; s *= fft_radix(M, s)) off += fft_tw_rows(fft_radix(M, s)) * s;
  return off;
}
__host__ __device__ constexpr int fft_tw_entries(int M) { return fft_tw_offset(M, M); }
// The smallest admissible length >= n (0 if none is <= maxM): 2^k >= 64, 3 2^k >= 96,
// 5 2^k >= 640 or 7 2^k >= 896.
inline int fft_length(int64_t n, int maxM) {
  int64_t best = 0;
  for (int64_t base : {64, 96, 640, 896})
    for (int64_t m = base; m <= maxM; m <<= 1)
      if (m >= n) {
        if (best == 0 || m < best) best = m;
        break;
      }
  return (int)best;
}
// Launch class of a length (one stage kind per length), and the entry of sft_tuning::dft_per_cta
// it takes: that of the power-of-two length with the same threads per transform.
inline int fft_stage(int M) {
  switch (fft_odd(M)) {
    case 3: return kStBluestein3 + fft_log2(M / 96);
    case 5: return kStBluestein5 + fft_log2(M / 640);
    case 7: return kStBluestein7 + fft_log2(M / 896);
    default: return kStBluestein0 + fft_log2(M) - 6;
  }
}
inline int fft_tune_class(int M) { return fft_log2(fft_tpt(M)) - 2; }
inline int fft_stage_length(int kind) {
  if (kind >= kStBluestein7) return 896 << (kind - kStBluestein7);
  if (kind >= kStBluestein5) return 640 << (kind - kStBluestein5);
  if (kind >= kStBluestein3) return 96 << (kind - kStBluestein3);
  return 64 << (kind - kStBluestein0);
}
// Programmatic dependent launch.  Every kernel of the library begins with pdl_begin(): it waits
// until the kernel before it on the stream has completed and its writes are visible, then lets the
// kernel after it be scheduled.  launch_pdl allows that overlap on streams that are not being
// captured, so the next kernel's blocks are set up while this one's last blocks run (the wait
// keeps every data dependence): one SFT through direct launches took 0.171 instead of 0.191 ms.
// Launches captured into a CUDA graph are plain (the graph already closes the launch gaps; with
// programmatic edges it measured 0.180 instead of 0.176 ms); pdl_begin() is then a no-op.
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_begin() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
#endif
template <typename... P, typename... A>
inline cudaError_t launch_pdl(void (*kernel)(P...), unsigned grid, unsigned block, size_t smem,
                              cudaStream_t st, A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
    (void)cudaGetLastError();           // (a refused query must not read as a launch failure)
    cap = cudaStreamCaptureStatusActive;
  }
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = cap == cudaStreamCaptureStatusNone ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<P>(args)...);
}

int bluestein_blocks(const DevPlan& d, int M, int per_cta);   // chirp-convolution blocks of one signal
int rank_blocks(const DevPlan& d, int kind);     // blocks of the rank fallbacks (0 when not needed)

constexpr int kStages = 6;
constexpr int kProfileCap = 4096;

// Per-stage timing with CUDA events (plans and batches).
struct Profiler {
  bool on = false;
  std::vector<cudaEvent_t> events;   // kProfileCap * (kStages + 1)
  int recorded = 0;
};

// Where a plan's device memory comes from when it is not cudaMalloc (the server's arena).
struct DeviceMemory {
  virtual ~DeviceMemory() = default;
  virtual void* alloc(size_t bytes) = 0;                         // nullptr when it does not fit
  virtual void release(void* p) = 0;
  virtual cudaError_t upload(void* dst, const void* src, size_t bytes) = 0;  // host -> device, done on return
};

struct Plan {
  DevPlan d;
  DevPlan* d_dev = nullptr;   // device copy of d (inside the plan's allocation)
  Profiler prof;
  int64_t launches = 0;
  double alpha = 0, beta = 0;
  uint64_t seed = 0;
  std::vector<int64_t> shifts;
  std::vector<int32_t> primes, small;
  size_t device_bytes = 0;
  size_t want_bytes = 0;         // device bytes the last build asked for (set even when it failed)
  std::vector<void*> allocations;
  DeviceMemory* mem = nullptr;   // nullptr: allocations came from cudaMalloc
  int device = 0;
  sft_batch_t solo = nullptr;    // batch of this plan alone, for CUDA-graph execution
  bool graph_on = false;
};

// Kernel launch wrappers: one launch per stage for all signals of bv (each returns
// cudaGetLastError()).  `d0` is the first signal's plan (batches share precision, input type and
// window half-width; the chirp-convolution launch is repeated per length class present).
cudaError_t launch_zero(const BatchView& bv, const LaunchSet& ls, cudaStream_t st);
cudaError_t launch_resample(const DevPlan& d0, const BatchView& bv, const LaunchSet& ls,
                            cudaStream_t st);
cudaError_t launch_bluestein(const DevPlan& d0, const BatchView& bv, const LaunchSet& ls,
                             cudaStream_t st, int* launched);
cudaError_t launch_rader(const DevPlan& d0, const BatchView& bv, const LaunchSet& ls,
                         cudaStream_t st, int* launched);
cudaError_t launch_identify(const DevPlan& d0, const BatchView& bv, const LaunchSet& ls,
                            cudaStream_t st);
cudaError_t launch_vote(const DevPlan& d0, const BatchView& bv, const LaunchSet& ls,
                        cudaStream_t st);
cudaError_t launch_select(const BatchView& bv, const LaunchSet& ls, cudaStream_t st, int* launched);
cudaError_t launch_refine(const BatchView& bv, const LaunchSet& ls, cudaStream_t st);
cudaError_t launch_finalize(const BatchView& bv, const LaunchSet& ls, cudaStream_t st,
                            int* launched);

// Engine (api.cu): the stage sequence for one signal or a batch.
int signal_blocks(const DevPlan& d, int kind, const sft_tuning& t);
LaunchSet single_launch_set(const DevPlan& d);
cudaError_t run_stages(const DevPlan& d0, const BatchView& bv, const LaunchSet& ls,
                       cudaStream_t st, cudaEvent_t* ev, int* launched);

#ifdef __CUDACC__
// Raise kernel KERNEL's dynamic shared-memory limit to at least `bytes` on the current device,
// calling the runtime only when the limit must grow.  The kernel itself is the template argument,
// so every kernel keeps its own record (kernels of one signature share a type, not a record).
template <auto KERNEL>
cudaError_t ensure_dynamic_smem(size_t bytes) {
  constexpr int kDevices = 64;
  static int granted[kDevices] = {};            // bytes granted so far (updates are idempotent)
  if (bytes <= 48 * 1024) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < kDevices && granted[dev] >= (int)bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(KERNEL, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess && dev >= 0 && dev < kDevices) granted[dev] = (int)bytes;
  return e;
}
#endif

cudaEvent_t* profile_slot(Profiler& pr);
sft_status profile_enable(Profiler& pr, int enable);
sft_status profile_read(Profiler& pr, double* stage_ms, int32_t* n_executions);
void profile_release(Profiler& pr);

// Host plan construction (plan.cpp).
sft_status build_plan(Plan* P, int64_t N, int32_t s, const sft_variant* v, int32_t n_shifts,
                      const int64_t* primes, int32_t n_primes, const int32_t* small,
                      int32_t n_small, DeviceMemory* mem = nullptr);
void free_plan(Plan* P);
sft_status choose_moduli(int64_t N, int32_t s, int32_t K, double c_p, uint64_t seed,
                         int64_t* primes_out, int32_t* small_out, int32_t* n_small_out,
                         int pool = SFT_POOL_ALL);
sft_status choose_moduli_deterministic(int64_t N, int32_t s, double c_p, int64_t* primes_out,
                                       int32_t* K_out, int32_t* small_out, int32_t* n_small_out);

// Thread-local error text.
void set_error(const std::string& msg);

// The plan behind a C handle (api.cu).
Plan* sft_plan_internal(sft_plan_t plan);

}  // namespace sft
