/*
 * sft.h — C ABI of the GB300 Gaussian-filtered discrete sparse Fourier transform.
 *
 * Problem (Section 2 and Algorithm 1 of Merhi, Zhang, Iwen, Christlieb, "A New Class of Fully
 * Discrete Sparse Fourier Transforms"): given the N samples f_j = f(-pi + 2 pi j / N) of a
 * length-N vector, any N >= 2, return a near best s-term approximation of its DFT
 *     f_hat = F f,   F[w, j] = (-1)^w exp(-2 pi i w j / N) / N,   w in B = (-ceil(N/2), floor(N/2)],
 * as at most s (frequency, coefficient) pairs.  The method (Algorithm 1) filters f with ceil(c2)
 * modulated periodic Gaussians, evaluates each filtered function at the off-grid nodes of an
 * unequally spaced SFT from a short window of f (Section 3.1, Lemma fewer_points_error), runs that
 * SFT (prime-modulus DFT measurements, CRT identification, majority vote, median estimates,
 * Appendix B), keeps each shift's in-band frequencies divided by the filter's Fourier coefficient,
 * and returns the s largest.
 *
 * Conventions shared by every entry point
 *  - Every pointer argument named *_dev is a CUDA device pointer on the current device; every
 *    other pointer is host memory.  The caller owns all buffers it passes; the plan owns its own
 *    device tables and scratch and frees them in sft_plan_destroy.
 *  - An input signal (f_dev, f_devs[i]) may also be page-locked host memory that the device can
 *    address (cudaHostAlloc / cudaMallocHost under unified addressing): the transform reads only
 *    the 2 kappa + 1 samples around each node, so it then fetches those windows over the
 *    CPU-GPU link instead of the whole signal being copied first.  Results are the same bits.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Execution entry
 *    points only enqueue work and return; results are valid after the stream is synchronised.
 *  - No entry point throws or aborts.  Each returns an sft_status; on failure the plan is left
 *    usable (or untouched) and sft_last_error() gives a thread-local message.
 *  - A plan is not re-entrant: two executions of one plan must not overlap on the GPU (they share
 *    the plan's scratch).  Distinct plans may run concurrently on distinct streams.
 */
#ifndef SFT_H
#define SFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SFT_OK = 0,
  SFT_EINVAL = 1,    /* invalid argument or plan parameters */
  SFT_ENOMEM = 2,    /* device or host allocation failed (nothing leaked) */
  SFT_ECUDA = 3,     /* a CUDA runtime call failed */
  SFT_ETIMEOUT = 4,  /* a bounded wait ran out (sft_server_wait's time limit) */
  SFT_EBUSY = 5      /* server full: request not admitted */
} sft_status;

/* Window half-widths of the paper's DMSFT-4 and DMSFT-6 implementations (Section 5). */
enum { SFT_DMSFT4 = 4, SFT_DMSFT6 = 6 };

typedef enum { SFT_FP32 = 0, SFT_FP64 = 1 } sft_precision;
typedef enum { SFT_IN_C64 = 0, SFT_IN_C128 = 1 } sft_input_type;
/* Pool of the randomized inner SFT's primes (sft_variant.pool). */
typedef enum { SFT_POOL_ALL = 0, SFT_POOL_SMOOTH = 1 } sft_pool;
/* How the length-p_j DFTs of the measurements are taken (sft_variant.dft). */
typedef enum { SFT_DFT_AUTO = 0, SFT_DFT_CHIRP = 1, SFT_DFT_RADER = 2 } sft_dft;

/*
 * Method parameters.  Fill with sft_variant_init() and override fields.
 *  kappa      window half-width: each filtered sample uses f_{j'-kappa..j'+kappa} (Lemma
 *             fewer_points_error); SFT_DMSFT4 or SFT_DMSFT6, or any 1..48.
 *  alpha,beta passband / filter parameters of Lemma Periodic_Gaussian_Decay and Algorithm 1:
 *             c1 = beta sqrt(ln N)/N, L = ceil(N/(alpha sqrt(ln N))), ceil(alpha sqrt(ln N)/2) shifts.
 *  K, c_p     number of prime moduli p_j of the inner SFT and their size, p_j >= c_p * s.
 *  seed       selects the primes (the randomized inner SFT reads a random subset of moduli).
 *  deterministic
 *             0: the randomized inner SFT (K primes drawn by `seed` from the 4K smallest primes
 *             >= max(ceil(c_p s), 5)).  1: the deterministic inner SFT (the paper's Algorithm 3
 *             of the cited work, Lemma SFT_Ident_Coef_Est_in_Noise): the K smallest primes
 *             >= max(ceil(c_p s), 5) with K = 2 (s - 1) L + 1, L = floor(log_{p_1}(N - 1)).  Two
 *             distinct frequencies of B differ by less than N, so they share a residue modulo at
 *             most L of the primes; every frequency of an s-sparse spectrum then sits alone in its
 *             bin for a strict majority of the primes, and an exactly s-sparse input is recovered
 *             exactly whatever the input (O(s^2 log N) samples).  The given K and seed are
 *             ignored; SFT_EINVAL if K would exceed SFT_MAX_K.
 *  precision  SFT_FP32: window sums and DFTs in FP32 with FP32 accumulation, phases reduced exactly
 *             as integers; the s winners are then re-estimated from the samples with exact
 *             twiddles and compensated accumulation, medians and division in FP64.
 *             SFT_FP64: every stage in FP64.
 *  refine_fp64
 *             FP32 path only (ignored for SFT_FP64): 1 (default) runs the re-estimation of the s
 *             winners described above; 0 returns the FP32 medians divided by the filter's
 *             coefficient as they are (three fewer kernels; the coefficients then carry the FP32
 *             DFTs' rounding, about 1e-6 of the largest bin, instead of meeting 1e-5 relative).
 *             Plans of one batch must agree on it.
 *  input      element type of f: SFT_IN_C64 (interleaved float re,im) or SFT_IN_C128 (double).
 *  pool       randomized inner SFT only: SFT_POOL_ALL draws the K primes from the 4K smallest
 *             primes >= max(ceil(c_p s), 5); SFT_POOL_SMOOTH from the 4K smallest such primes
 *             whose p - 1 has no prime factor above 13, so that every length-p DFT can be taken
 *             by Rader's algorithm (below).  Any K distinct primes serve the randomized inner SFT
 *             (Lemma SFT_Ident_Coef_Est_in_Noise); the smooth pool reaches a little higher (its
 *             mean prime is about 1.15 c_p s near c_p s = 3000 against 1.03 c_p s).
 *  dft        how the length-p DFTs are taken.  SFT_DFT_CHIRP: a chirp convolution (Bluestein)
 *             over an FFT of length r 2^k >= 2p - 1 (p <= 8192 FP32, 4096 FP64).
 *             SFT_DFT_RADER: Rader's algorithm, a cyclic convolution of length p - 1 over a
 *             mixed-radix FFT of that length (every p - 1 must be a product of 2, 3, 5, 7, 11,
 *             13; p <= 13313 FP32, 6657 FP64); about half the work of the chirp form.
 *             SFT_DFT_AUTO (default): Rader when every p_j allows it, else the chirp form.
 */
typedef struct {
  int32_t kappa;
  int32_t precision;
  int32_t input;
  int32_t K;
  double c_p;
  double alpha;
  double beta;
  uint64_t seed;
  int32_t deterministic;
  int32_t refine_fp64;
  int32_t pool;
  int32_t dft;
} sft_variant;

/*
 * Theorem-parameter mode (Theorem total_convolution_error): every filtered sample is then within
 * 3 ||f||_p N^{-r} of (g * f)(x).  Sets v->beta = 6 sqrt(r), v->kappa = ceil(6 r ln N / (sqrt(2) pi))
 * + 1 (the theorem's window half-width) and v->alpha = v->beta (band-edge filter gain e^{-1/2},
 * which meets Section 4's lower bound on alpha); other fields are unchanged.  Host only.
 * SFT_EINVAL for r < 1, N < 36 r (outside the theorem's range) or a half-width above 48.
 */
sft_status sft_variant_theorem(sft_variant* v, int64_t N, double r);

typedef struct sft_plan_s* sft_plan_t;

/* Plan description returned by sft_plan_info (host memory, filled by the library). */
#define SFT_MAX_K 512
#define SFT_MAX_SMALL 12
#define SFT_MAX_SHIFTS 32
typedef struct {
  int64_t N;
  int32_t s;
  int32_t kappa;
  int32_t K;                          /* number of prime moduli p_j */
  int32_t n_small;                    /* number of small moduli t_l */
  int32_t n_shifts;                   /* ceil(c2) */
  int32_t n_sub;                      /* node subsets per prime: 1 + sum_l (t_l - 1) */
  int64_t primes[SFT_MAX_K];
  int32_t small[SFT_MAX_SMALL];
  int64_t shifts[SFT_MAX_SHIFTS];     /* q_1 .. q_{n_shifts} */
  int64_t L;                          /* band half-width ceil(N/(alpha sqrt(ln N))) */
  double c1;                          /* Gaussian width beta sqrt(ln N)/N */
  int64_t nodes;                      /* distinct nodes m = n_sub * sum_j p_j */
  int32_t fft_size;                   /* chirp-convolution length: the smallest of 2^k >= 64,
                                         3 2^k >= 96, 5 2^k >= 640, 7 2^k >= 896 that is
                                         >= 2 p_K - 1; 0 when the plan uses Rader's form */
  int32_t precision;
  int32_t input;
  int32_t dft;                        /* SFT_DFT_CHIRP or SFT_DFT_RADER: the form in use */
} sft_plan_desc;

/* Fill *v with the defaults: kappa 6 (DMSFT-6), FP32, complex64 input, K 5, c_p 3,
 * alpha = beta = 1.5, seed 0, randomized inner SFT, refine_fp64 1, SFT_POOL_ALL, SFT_DFT_AUTO.
 * Returns SFT_EINVAL if v is NULL. */
sft_status sft_variant_init(sft_variant* v);

/*
 * Build a plan for length-N inputs and sparsity s (Algorithm 1, its set-up lines: c1, c2, L and the
 * shifts q_j = -ceil(N/2) + 1 + (2j - 1) L).
 *  n_shifts      0 = ceil(alpha sqrt(ln N)/2); otherwise that many shifts (must still cover B).
 *  primes        NULL = K primes chosen by v->seed from v->pool (the 4K smallest primes
 *                >= max(c_p s, 5), or the 4K smallest of those whose p - 1 is 13-smooth);
 *                else n_primes distinct primes (1 <= n_primes <= SFT_MAX_K) used as given.
 *  small_moduli  NULL = the smallest primes, none equal to a p_j, until p_1 prod(t) >= N;
 *                else n_small pairwise-coprime moduli >= 2, coprime to every p_j, p_1 prod >= N.
 * Requires 2 <= N < 2^31, 1 <= s <= N, 2 kappa + 1 <= N, and every p_j within the limits of the
 * DFT form (v->dft: chirp p <= 8192 FP32 / 4096 FP64; Rader p <= 13313 FP32 / 6657 FP64).
 * (Theorem MainTHM is stated for s >= 2; s = 1 is accepted, since Algorithm 1 itself is defined
 * for it: one term per shift, the largest kept.)
 * Allocates the plan's device tables and scratch on the current device (sft_plan_device_bytes).
 * On failure *out is set to NULL and nothing is leaked.
 */
sft_status sft_plan(sft_plan_t* out, int64_t N, int32_t s, const sft_variant* v, int32_t n_shifts,
                    const int64_t* primes, int32_t n_primes, const int32_t* small_moduli,
                    int32_t n_small);

/*
 * Run Algorithm 1 on f_dev (N elements of the plan's input type, 8-byte aligned; 16-byte
 * alignment enables vector loads) and write, on `stream`:
 *   out_freqs_dev[0..s)   int64 frequencies in B, sorted by |coefficient| descending, ties by the
 *                         smaller frequency (Section 2's tie-break for R_s^opt);
 *   out_coefs_dev[0..s)   complex128 (interleaved double re,im) coefficient estimates in the
 *                         f_hat = F f convention;
 *   out_count_dev[0]      int32 number of pairs written (<= s; unused slots are zeroed).
 * Any of the three may be NULL only if all are NULL (a dry run that still executes every stage).
 */
sft_status sft_execute(sft_plan_t plan, const void* f_dev, int64_t* out_freqs_dev,
                       void* out_coefs_dev, int32_t* out_count_dev, void* stream);

/*
 * Host-only, no device work: the moduli sft_plan would choose for (N, s, K, c_p, seed) when given
 * NULL primes and NULL small moduli (Monte Carlo inner SFT: K primes drawn by a SplitMix64-seeded
 * partial Fisher-Yates shuffle from the 4K smallest primes >= max(ceil(c_p s), 5), ascending; then
 * the smallest primes t != p_j until p_1 prod(t) >= N).  primes_out holds K entries, small_out
 * SFT_MAX_SMALL; *n_small_out receives the count.  SFT_EINVAL on bad arguments.
 */
sft_status sft_choose_moduli(int64_t N, int32_t s, int32_t K, double c_p, uint64_t seed,
                             int64_t* primes_out, int32_t* small_out, int32_t* n_small_out);

/* Host only: as sft_choose_moduli with the primes drawn from `pool` (SFT_POOL_ALL gives the same
 * moduli as sft_choose_moduli; SFT_POOL_SMOOTH the 4K smallest primes >= max(ceil(c_p s), 5) whose
 * p - 1 has no prime factor above 13). */
sft_status sft_choose_moduli_pool(int64_t N, int32_t s, int32_t K, double c_p, uint64_t seed,
                                  int32_t pool, int64_t* primes_out, int32_t* small_out,
                                  int32_t* n_small_out);

/* Host only: the moduli of the deterministic inner SFT (sft_variant.deterministic = 1) for N, s,
 * c_p: the K smallest primes >= max(ceil(c_p s), 5), K = 2 (s - 1) floor(log_{p_1}(N - 1)) + 1,
 * written to primes_out (room for SFT_MAX_K) with *K_out = K, and the small moduli as for
 * sft_choose_moduli.  SFT_EINVAL on bad arguments or when K would exceed SFT_MAX_K. */
sft_status sft_choose_moduli_deterministic(int64_t N, int32_t s, double c_p, int64_t* primes_out,
                                           int32_t* K_out, int32_t* small_out, int32_t* n_small_out);

/*
 * Batches: the transforms of n signals, each with its own plan, with one kernel launch per stage
 * for the whole batch (Algorithm 1 is unchanged per signal).  Plans may
 * differ in N, s and moduli but must share precision, input type and kappa, and each plan may
 * appear once (its scratch serves one signal).  The batch keeps device copies of the plans'
 * records, so plans must outlive the batch and must not be executed on their own while an
 * execution of the batch is in flight.
 */
typedef struct sft_batch_s* sft_batch_t;

/* Create a batch of plans[0..n) (1 <= n <= 2^20); *out receives the handle, which the caller owns
 * and releases with sft_batch_destroy (the plans stay the caller's).  Starts from the tuning
 * table's entry for the plans' shape class, else sft_tuning_default.  On failure *out is NULL and
 * nothing is held: SFT_EINVAL for a NULL argument, a NULL or repeated plan, plans that differ in
 * precision, input type, kappa or refine_fp64, or a launch that would exceed 2^31 - 1 blocks;
 * SFT_ENOMEM when device or pinned host memory cannot be had; SFT_ECUDA on another failed call. */
sft_status sft_batch_create(sft_batch_t* out, const sft_plan_t* plans, int32_t n);

/*
 * One execution: f_devs[i] is signal i's input (N_i elements of the shared input type); its
 * results go to out_freqs_devs[i][0..s_i), out_coefs_devs[i][0..s_i) (complex128) and
 * out_count_devs[i][0], as for sft_execute.  All five arrays are host arrays of n device pointers;
 * they are copied at the call.  Executions of one batch must not overlap on the GPU.
 */
sft_status sft_batch_execute(sft_batch_t batch, const void* const* f_devs,
                             int64_t* const* out_freqs_devs, void* const* out_coefs_devs,
                             int32_t* const* out_count_devs, void* stream);

/* Release the batch's device and host resources (NULL is a no-op; its plans are not touched).
 * The caller must ensure no execution of the batch is still running on the GPU. */
sft_status sft_batch_destroy(sft_batch_t batch);

/*
 * One-shot form of the three calls above: the transforms of plans[0..n) with one launch per stage,
 * enqueued on `stream` with the same arguments as sft_batch_execute; the call returns without
 * waiting (results are valid after the stream is synchronised).  The call's own device array (the
 * plans' records, block prefixes and pointer tables, about 20 KB per plan) comes from the
 * stream-ordered allocator (cudaMallocAsync on `stream`) and is released in stream order after
 * the last stage (cudaFreeAsync), so nothing outlives the call on the host.  It is not meant for
 * stream capture.  For repeated executions of the same plans create a batch once (graph replay,
 * tuning).  Errors: those of sft_batch_create and sft_batch_execute (nothing runs), or SFT_ENOMEM
 * / SFT_ECUDA when the allocation or a launch fails.
 */
sft_status sft_execute_batch(const sft_plan_t* plans, const void* const* f_devs,
                             int64_t* const* out_freqs_devs, void* const* out_coefs_devs,
                             int32_t* const* out_count_devs, int32_t n, void* stream);

/*
 * Launch geometry of a batch's kernels.  It changes how work is split into CTAs, never what is
 * computed: every valid choice gives the same results, bit for bit.
 *   resample_threads  nodes per CTA of the kappa = 4 / 6 resampling kernel: 64, 128, 256 or 512
 *                     (other kappa use a fixed 128).
 *   resample_regcap   1: that kernel's build limited to 48 registers (five 256-thread CTAs per SM,
 *                     more warps in flight for the gather; needs resample_threads <= 256);
 *                     0: the default build (64 registers on the FP32 path).
 *   bin_threads       bins per CTA of residue identification and vote: 64, 128, 256 or 512.
 *   dft_per_cta[c]    chirp-convolution transforms per CTA for the lengths with 4 << c threads
 *                     per transform (c = 0..8): the power of two M = 64 << c, and 3 << (c + 4),
 *                     5 << (c + 3), 7 << (c + 3) where the plan's primes choose those; at most
 *                     max(M/16, 256) threads per CTA, so 1 <= dft_per_cta[c] <= max(1, 4096 / M).
 *   dft_two_ctas      FP32, M = 8192: 1 = the build limited to 64 registers so that two CTAs share
 *                     an SM; 0 = one CTA per SM with up to 128 registers.
 * sft_tuning_default fills the built-in choice (host only, no device call).
 */
typedef struct {
  int32_t resample_threads;
  int32_t resample_regcap;
  int32_t bin_threads;
  int32_t dft_per_cta[9];
  int32_t dft_two_ctas;
} sft_tuning;

/* Fill *t with the built-in launch geometry (host only; a NULL t is ignored). */
void sft_tuning_default(sft_tuning* t);

/* Validate and apply a launch geometry (SFT_EINVAL, nothing changed, if invalid).  Waits for the
 * device to finish (cudaDeviceSynchronize) before it rewrites the batch's launch tables, and drops
 * a captured graph (sft_batch_graph recaptures at the next execution). */
sft_status sft_batch_set_tuning(sft_batch_t batch, const sft_tuning* t);
/* Copy the batch's current launch geometry to *t (SFT_EINVAL for a NULL argument). */
sft_status sft_batch_get_tuning(sft_batch_t batch, sft_tuning* t);

/*
 * Autotuner: times each knob's candidates on this batch and these buffers (as for
 * sft_batch_execute; outputs are overwritten), one knob at a time with the others at their best
 * so far, from the per-stage CUDA-event times of `reps` executions per candidate after one
 * untimed execution, and applies the fastest.  The choice is copied to *chosen when it is not
 * NULL and stored in the tuning table (below) when the batch's plans share one shape class.
 * Synchronous (returns after the device has finished).  Profiling state is restored.
 */
sft_status sft_batch_autotune(sft_batch_t batch, const void* const* f_devs,
                              int64_t* const* out_freqs_devs, void* const* out_coefs_devs,
                              int32_t* const* out_count_devs, void* stream, int32_t reps,
                              sft_tuning* chosen);

/*
 * Table of tuned launch geometries (process-wide, thread-safe; host only, no device call), keyed
 * by a shape class: floor(log2 N), floor(log2 s), kappa and precision.  sft_batch_autotune stores
 * its choice under the class of a batch whose plans all share one, and sft_batch_create starts such
 * a batch from the class's entry (else from sft_tuning_default).  Entries change launch geometry
 * only, never results.
 *   _put / _get   set or read the entry of the class of (N, s, kappa, precision); SFT_EINVAL on a
 *                 bad key or tuning, or (get) when the class has no entry.
 *   _save         write the table to a text file (a header line, then one line per entry: the
 *                 four key fields and the tuning's 13 integers, in struct order), through a
 *                 temporary file renamed over `path`.
 *   _load         merge the entries of such a file; SFT_EINVAL, nothing merged, on any bad line.
 *   _size, _clear the number of entries; empty the table.
 */
sft_status sft_tuning_table_put(int64_t N, int32_t s, int32_t kappa, int32_t precision,
                                const sft_tuning* t);
sft_status sft_tuning_table_get(int64_t N, int32_t s, int32_t kappa, int32_t precision,
                                sft_tuning* t);
sft_status sft_tuning_table_save(const char* path);
sft_status sft_tuning_table_load(const char* path);
int32_t sft_tuning_table_size(void);
void sft_tuning_table_clear(void);

/*
 * enable = 1: the next execution captures the batch's kernel launches once as a CUDA graph (on a
 * private stream, so capturing runs nothing) and every execution replays it on the caller's
 * stream after uploading that execution's pointers; per-stage profiling is off while graphs are
 * on.  enable = 0 drops the graph and returns to direct launches.  Results are identical either
 * way.
 */
sft_status sft_batch_graph(sft_batch_t batch, int32_t enable);

/* Per-stage timing and launch count of a batch, as sft_plan_profile / _read / _launches
 * (SFT_EINVAL for a NULL argument; _launches is 0 for NULL), and the device bytes the batch holds
 * beside its plans (0 for NULL). */
sft_status sft_batch_profile(sft_batch_t batch, int32_t enable);
sft_status sft_batch_profile_read(sft_batch_t batch, double* stage_ms, int32_t* n_executions);
int64_t sft_batch_launches(sft_batch_t batch);
size_t sft_batch_device_bytes(sft_batch_t batch);

/* Release every device and host resource of the plan (NULL is a no-op).  The caller must ensure
 * no execution of the plan is still running on the GPU. */
sft_status sft_plan_destroy(sft_plan_t plan);

/* Device bytes held by the plan (tables + scratch), for admission by memory budget. */
size_t sft_plan_device_bytes(sft_plan_t plan);

/* Copy the plan's parameters into *out (host). */
sft_status sft_plan_info(sft_plan_t plan, sft_plan_desc* out);

/*
 * Expose one of the plan's intermediate device buffers (valid after an execution has completed),
 * for stage-by-stage checks.  which:
 *   0 samples  filtered samples h_q(x), [n_shifts][nodes] complex (FP32 or FP64 per precision);
 *              node order: prime j, then node subset u (u = 0: the p_j nodes -pi + 2 pi k/p_j;
 *              u >= 1: the p_j nodes offset by 2 pi k2 / t_l), then k = 0..p_j-1.
 *   1 bins     length-p_j DFTs of every node subset, same layout as samples (eq. DFT_GKlam_Comp).
 *   2 cand     int64 [n_shifts][sum_j p_j]: frequency identified in bin b of modulus p_j, or
 *              INT64_MIN when the CRT representative lies outside B.
 *   3 residues uint8 [n_shifts][sum_j p_j][n_small]: residue of bin b modulo each t_l.
 *   4 counters int32 [n_shifts + 4]: entry i < n_shifts is the length of shift i's voted list,
 *              entry n_shifts the length of the pooled in-band list, n_shifts + 1 the status
 *              word (sft_fault bits), n_shifts + 2 the winner count, n_shifts + 3 the site of
 *              the first index fault (sft_fault_site).
 *   5 voted    [n_shifts][capacity] records of 32 bytes: int64 frequency, double re and im of the
 *              median estimate (with the (-1)^w factor), int32 vote count, int32 first prime index
 *              that found it; shift i's first counters[i] records are valid, in no fixed order.
 * *bytes receives the buffer size.  Returns SFT_EINVAL for an unknown index.
 */
sft_status sft_plan_debug_buffer(sft_plan_t plan, int32_t which, void** dev_ptr, size_t* bytes);

/*
 * Faults the kernels record instead of faulting the GPU.  Each execution clears the plan's status
 * words first (its first kernel), and a kernel that meets one of these conditions sets its bit
 * and carries on without the access or record in question, so the result is then incomplete:
 *   SFT_FAULT_VOTED_FULL  a shift's voted list was full (its capacity is sum_j p_j, which no
 *                         execution reaches unless lowered by sft_plan_debug_limit); records
 *                         past it were dropped.
 *   SFT_FAULT_POOL_FULL   the pooled in-band list (n_shifts * s records) was full.
 *   SFT_FAULT_INDEX       checked build only (libsft_checked.so, compiled with SFT_CHECKED): an
 *                         index fell outside its buffer; the access was skipped.  The site of the
 *                         first such fault is kept (sft_fault_site).
 * The normal build compiles no index checks; its kernels and results are those of the checked
 * build whenever the latter records nothing.
 */
typedef enum {
  SFT_FAULT_VOTED_FULL = 1,
  SFT_FAULT_POOL_FULL = 2,
  SFT_FAULT_INDEX = 4
} sft_fault;

typedef enum {
  SFT_SITE_NONE = 0,
  SFT_SITE_WINDOW = 1,      /* resampling: a node's window centre j' outside [0, N) */
  SFT_SITE_DFT = 2,         /* a transform's samples or bins outside the plan's buffers */
  SFT_SITE_SUBBIN = 3,      /* identification: a bin's sub-bins outside the bins buffer */
  SFT_SITE_VOTE = 4,        /* vote: a candidate lookup or a median bin outside its buffer */
  SFT_SITE_REESTIMATE = 5   /* re-estimation: a chunk of samples or a winner outside its buffer */
} sft_fault_site;

/* 1 when the loaded library is the checked build, else 0. */
int32_t sft_checked_build(void);

/*
 * Read the plan's status words after its last execution (by sft_execute or in a batch): enqueues
 * the read on `stream` and waits for the stream.  *faults receives the sft_fault bits (0: none),
 * *site the sft_fault_site of the first index fault (0: none); either may be NULL.  SFT_EINVAL on
 * a NULL plan or while `stream` is being captured into a graph, SFT_ECUDA if the read fails.
 */
sft_status sft_plan_faults(sft_plan_t plan, void* stream, int32_t* faults, int32_t* site);

/*
 * Test hook: lower one of the plan's list capacities so that the kernels' capacity checks can be
 * exercised (which = 0: the voted list's capacity per shift, 1 <= value <= sum_j p_j; the buffer
 * keeps its size, so every access stays inside it).  Takes effect for executions by sft_execute
 * with graph replay off and for batches created afterwards.  SFT_EINVAL on a bad argument.
 */
sft_status sft_plan_debug_limit(sft_plan_t plan, int32_t which, int32_t value);

/*
 * Test hook: the library's device and pinned-host allocations (plans, batches, sft_execute_batch,
 * the server's arena and slots) go through one counter; after `skip` more of them succeed, the
 * next `fail` ones report cudaErrorMemoryAllocation without allocating, so that each caller's
 * SFT_ENOMEM path and rollback can be checked.  sft_debug_fail_allocations(0, 0) turns it off.
 * Process-wide; not for use while other threads allocate through the library.  SFT_EINVAL on a
 * negative count.
 */
sft_status sft_debug_fail_allocations(int32_t skip, int32_t fail);

/*
 * Residual-energy check of a result (after the execution that produced it, in stream order).  With
 * f-hat = F f, F[w, j] = (-1)^w e^{-2 pi i w j / N} / N (Section 2), Parseval's identity gives
 * ||f-hat||_2^2 = ||f||_2^2 / N, so for the returned terms c_0..c_{count-1}
 *     rho = 1 - (sum_r |c_r|^2) / (||f||_2^2 / N)
 * is the fraction of the spectrum's energy the s-term approximation leaves out (the tail and the
 * noise, when the estimates are exact; a negative rho flags over-estimated coefficients).  f_dev is
 * the input of that execution (N elements of the plan's input type), coefs_dev / count_dev its
 * outputs; *out_dev (one double, device memory) receives rho.  Reads f once; the sums of |f|^2 are
 * formed in double-single FP32 (complex64 input) or FP64 (complex128) per thread and combined in
 * FP64 in a fixed order, so the result is deterministic.  Two kernel launches on `stream`.
 */
sft_status sft_residual_energy(sft_plan_t plan, const void* f_dev, const void* coefs_dev,
                               const int32_t* count_dev, double* out_dev, void* stream);

/*
 * enable = 1: later sft_execute calls of this plan (with non-NULL outputs) replay its kernel
 * launches as one CUDA graph, captured at the first such call on a private stream (capturing runs
 * nothing): one graph launch instead of a dozen kernel launches, so the device no longer waits on
 * the host between stages.  Each call still uploads its own pointers first (stream-ordered), so
 * inputs and outputs may change from call to call.  Per-stage profiling is off while graphs are
 * on.  enable = 0 returns to direct launches.  Results are identical either way.
 */
sft_status sft_plan_graph(sft_plan_t plan, int32_t enable);

/*
 * Per-stage timing of this plan's executions with CUDA events recorded on the execution stream
 * between the stages (enable = 1 creates the events, 0 releases them).  Stages: 0 resampling,
 * 1 chirp-convolution DFTs, 2 residues + CRT, 3 vote + medians, 4 selections, 5 re-estimation.
 * At most 4096 executions are recorded between two reads; later ones are not timed.
 */
sft_status sft_plan_profile(sft_plan_t plan, int32_t enable);

/* After the stream has been synchronised: the summed milliseconds of each stage (stage_ms[0..6))
 * over the executions recorded since the previous read, and their number; then resets. */
sft_status sft_plan_profile_read(sft_plan_t plan, double* stage_ms, int32_t* n_executions);

/* Total number of kernels this plan has launched (all executions so far). */
int64_t sft_plan_launches(sft_plan_t plan);

/*
 * Serving loop.  A server owns one device-memory arena of `mem_budget` bytes from which it carves
 * the plans of the requests it admits (tables, filter constants and scratch stay resident for
 * later requests of the same N and s), a scheduler thread and `max_inflight` non-blocking
 * streams.  Requests of any N and s are queued in arrival order; whenever a stream is free the
 * scheduler takes up to `max_batch` queued requests whose plans it can hold (building plans, and
 * evicting least recently used idle plans when the arena is full) and runs them as one batched
 * execution (one launch per stage for all of them, as sft_batch_execute).  Requests that arrive
 * while others run join the next batch, and batches on different streams overlap on the device.
 * A request waits at the head of the queue until memory frees up; one whose plan does not fit
 * the whole arena fails with SFT_ENOMEM.  Each result is the one sft_execute gives for a plan of
 * the same N, s and variant, bit for bit, whatever else ran with it.
 *
 * Every plan uses `variant`.  Tuning `tune` (sft_tuning_default when tune.resample_threads is 0)
 * sets the launch geometry.  mem_budget covers the plans; each stream adds a small record
 * buffer (< 1 MiB at max_batch = 256).
 */
typedef struct sft_server_s* sft_server_t;
typedef int64_t sft_request_t;

typedef struct {
  size_t mem_budget;      /* device bytes for plans (the arena); >= 1 MiB */
  int32_t max_batch;      /* requests per batched execution, 1..256 */
  int32_t max_inflight;   /* batched executions in flight at once (streams), 1..8 */
  sft_variant variant;
  sft_tuning tune;
  int32_t build_threads;  /* threads that build new plans beside the scheduler, 0..16 (0: the
                             scheduler builds them itself, holding up the queue meanwhile) */
  int32_t reserved;
} sft_server_config;

typedef struct {
  int32_t state;          /* 0 queued, 1 running, 2 done, 3 failed */
  int32_t status;         /* sft_status: SFT_OK, or why the request failed */
  int32_t batch_size;     /* requests in the batched execution that served it (0 until launched) */
  int32_t plan_reused;    /* 1 if its plan was resident already, 0 if built for it */
  double queued_ms;       /* submission -> launch of its batch (host clock) */
  double latency_ms;      /* submission -> results complete in device memory (host clock) */
  double build_ms;        /* host time spent building its plan (0 when a resident plan served) */
} sft_request_info;

typedef struct {
  int64_t submitted, completed, failed, batches;
  int64_t plans_built, plans_reused, plans_evicted;
  int64_t kernel_launches;
  size_t arena_bytes, arena_used, arena_peak;
  int32_t resident_plans, max_batch_seen;
  double build_ms_total;  /* host time spent building plans */
} sft_server_stats;

/* Default configuration: 8 GiB, max_batch 64, max_inflight 2, sft_variant_init, default tuning,
 * 2 build threads.  A request whose (N, s) has no idle resident plan has its plan built by a
 * build thread (tables of primes seen before come from a host cache) while the requests behind
 * it are batched; it joins the next batch once the plan is ready. */
void sft_server_config_init(sft_server_config* cfg);

/* Allocate the arena and the streams, start the scheduler.  SFT_EINVAL for a bad configuration,
 * SFT_ENOMEM if the arena cannot be allocated. */
sft_status sft_server_create(sft_server_t* out, const sft_server_config* cfg);

/*
 * Queue one transform.  f_dev holds N elements of the variant's input type and must be fully
 * written before the call (synchronise the producing stream first); the outputs are laid out as
 * for sft_execute.  All four buffers are the caller's and must stay valid until the request is
 * done or failed.  *id receives the request's handle.  Never blocks on the device.
 */
sft_status sft_server_submit(sft_server_t server, int64_t N, int32_t s, const void* f_dev,
                             int64_t* out_freqs_dev, void* out_coefs_dev, int32_t* out_count_dev,
                             sft_request_t* id);

/* State and timings of a request (SFT_EINVAL for an unknown or released handle). */
sft_status sft_server_query(sft_server_t server, sft_request_t id, sft_request_info* info);

/* Block until the request has finished, done or failed (SFT_OK; sft_server_query tells which and
 * why), or timeout_ms has passed (SFT_ETIMEOUT; timeout_ms < 0 waits without limit).  SFT_EINVAL
 * for an unknown handle.  A done request's results are complete in device memory and visible to
 * every stream. */
sft_status sft_server_wait(sft_server_t server, sft_request_t id, int32_t timeout_ms);

/* Non-blocking completion test: *done = 1 once the request has finished, else 0.  Returns SFT_OK
 * while it is pending or when it is done, the request's own failure status when it failed, and
 * SFT_EINVAL for an unknown handle or a NULL argument. */
sft_status sft_server_poll(sft_server_t server, sft_request_t id, int32_t* done);

/* Forget a finished request's record (SFT_EBUSY while it is queued or running). */
sft_status sft_server_release(sft_server_t server, sft_request_t id);

/* Snapshot of the server's counters and arena usage into *out (SFT_EINVAL for a NULL argument). */
sft_status sft_server_stats_read(sft_server_t server, sft_server_stats* out);

/* Finish every queued and running request, stop the scheduler, free everything. */
sft_status sft_server_destroy(sft_server_t server);

/*
 * Batched DFT that allocates no device memory, for callers that cannot call cudaMalloc: code that
 * runs while another component owns the device's memory (a host framework's caching allocator, a
 * plug-in with a fixed memory budget, or a phase where allocating would stall or fragment the
 * heap).  The paper has no counterpart: it is a stand-alone use of this library's prime-length DFT
 * (the chirp-convolution kernel of the measurements).
 *
 * Computes, for b = 0..batch-1 and c = 0..n-1,
 *     out[b n + c] = (1/n) sum_{k=0}^{n-1} in[b n + k] e^{-2 pi i k c / n}
 * on complex64 vectors (interleaved float re,im, 8-byte aligned, caller-owned), any length
 * 2 <= n <= 8191 (prime or not), in FP32, on `stream`.
 *
 * The kernel's tables (chirp, filter spectrum, FFT twiddles) and its launch record live in one
 * fixed 340 KiB array in device memory that the library declares statically: every GPU that
 * loads the library holds it until the process exits, and nothing is allocated at any call.  The
 * first call on a device looks up that array's address, and the first call with a given n (on
 * that device, since the last call with another n) builds the tables for n on `stream`.  Such a
 * call must not be made while `stream` is being captured (it returns SFT_EINVAL then): make it
 * before any capture.  Every call enqueues two kernels on `stream` (one writes the call's launch
 * record into the array, the other runs the transforms) and copies nothing from host memory.
 * All calls share the array, which keeps the last call's record and tables, so calls that
 * overlap on the GPU (different streams, or another n while one is in flight) race; serialise
 * them.  Returns SFT_EINVAL for n outside 2..8191, batch < 1 or NULL/misaligned buffers.
 */
sft_status sft_dft_noalloc(int32_t n, int32_t batch, const void* in_dev, void* out_dev,
                           void* stream);

/* Thread-local description of the last failure in this thread ("" if none). */
const char* sft_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SFT_H */
