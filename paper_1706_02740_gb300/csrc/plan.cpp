// Host side of a plan: Algorithm 1's parameters, the inner SFT's moduli, and the constant tables
// the kernels read (all computed in FP64 with integer-exact phase reduction, then stored in the
// plan's precision).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <complex>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <stdexcept>
#include <thread>
#include <string>
#include <tuple>
#include <vector>

#include "alloc_hook.h"
#include "host_fft.h"
#include "int_math.h"
#include "prime_tables.h"
#include "rader_plan.h"
#include "sft_internal.h"

namespace sft {

namespace {

// SplitMix64 (Steele, Lea and Flood, 2014; constants as published by Vigna).
uint64_t splitmix64(uint64_t* state) {
  *state += 0x9E3779B97F4A7C15ULL;
  uint64_t z = *state;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// The inner SFT's K primes: a seeded partial Fisher-Yates draw from a pool of 4K primes
// >= max(ceil(c_p s), 5), returned ascending (randomized inner SFT reading a random subset of
// moduli).  SFT_POOL_ALL: the 4K smallest such primes; SFT_POOL_SMOOTH: the 4K smallest whose
// p - 1 has no prime factor above 13.
std::vector<int32_t> choose_primes(int32_t s, int K, double c_p, uint64_t seed,
                                   int pool_kind = SFT_POOL_ALL) {
  int64_t lo = std::max<int64_t>((int64_t)ceil(c_p * (double)s), 5);
  std::vector<int64_t> pool;
  for (int64_t n = lo; (int)pool.size() < 4 * K; ++n)
    if (is_prime(n) && (pool_kind != SFT_POOL_SMOOTH || smooth13(n - 1))) pool.push_back(n);
  uint64_t state = seed;
  for (int i = 0; i < K; ++i) {
    uint64_t r = splitmix64(&state);
    size_t j = (size_t)i + (size_t)(r % (uint64_t)(pool.size() - (size_t)i));
    std::swap(pool[i], pool[j]);
  }
  std::vector<int32_t> out(pool.begin(), pool.begin() + K);
  std::sort(out.begin(), out.end());
  return out;
}

// Smallest primes t, none equal to a p_j, until p_1 * prod(t) >= N.
// The deterministic inner SFT's moduli: the K smallest primes >= max(ceil(c_p s), 5) with
// K = 2 (s - 1) L + 1, L = floor(log_{p_1}(N - 1)) (the largest L with p_1^L <= N - 1).
std::vector<int32_t> deterministic_primes(int64_t N, int32_t s, double c_p, int* K_out) {
  int64_t n = std::max<int64_t>((int64_t)ceil(c_p * (double)s), 5);
  while (!is_prime(n)) ++n;
  const int64_t p1 = n;
  int64_t L = 0;
  for (__int128 pw = p1; pw <= (__int128)(N - 1); pw *= p1) ++L;
  const int64_t K = 2 * (int64_t)(s - 1) * L + 1;
  *K_out = K > (int64_t)kMaxK ? -1 : (int)K;
  std::vector<int32_t> out;
  if (*K_out < 0) return out;
  for (int64_t m = p1; (int)out.size() < K; ++m)
    if (is_prime(m)) out.push_back((int32_t)m);
  return out;
}

std::vector<int32_t> choose_small(int64_t N, const std::vector<int32_t>& primes) {
  std::vector<int32_t> T;
  int64_t prod = primes[0];
  for (int32_t t = 2; prod < N; ++t) {
    if (is_prime(t) && std::find(primes.begin(), primes.end(), t) == primes.end()) {
      T.push_back(t);
      prod *= t;
    }
  }
  return T;
}

// Per-prime tables (csrc/prime_tables.h), cached on the host across plans: a plan for a new N
// whose primes were seen before only assembles them.  Bounded to kPrimeCache entries, oldest
// dropped first.
constexpr size_t kPrimeCache = 512;
std::mutex g_prime_mu;
std::map<std::tuple<int64_t, int, bool>, std::shared_ptr<const PrimeTables>> g_prime_tables;
std::deque<std::tuple<int64_t, int, bool>> g_prime_order;

std::shared_ptr<const PrimeTables> prime_tables(int64_t p, int M, bool rader) {
  const auto key = std::make_tuple(p, rader ? 0 : M, rader);
  {
    std::lock_guard<std::mutex> g(g_prime_mu);
    auto it = g_prime_tables.find(key);
    if (it != g_prime_tables.end()) return it->second;
  }
  auto T = compute_prime_tables(p, M, rader);
  std::lock_guard<std::mutex> g(g_prime_mu);
  if (g_prime_tables.emplace(key, T).second) {
    g_prime_order.push_back(key);
    while (g_prime_order.size() > kPrimeCache) {
      g_prime_tables.erase(g_prime_order.front());
      g_prime_order.pop_front();
    }
  }
  return T;
}

std::shared_ptr<const PrimeTables> cached_prime_tables(int64_t p, int M, bool rader) {
  std::lock_guard<std::mutex> g(g_prime_mu);
  auto it = g_prime_tables.find(std::make_tuple(p, rader ? 0 : M, rader));
  return it == g_prime_tables.end() ? nullptr : it->second;
}

// The tables of every prime of a plan.  A plan for a new length often brings several primes not
// seen before, each an FFT of up to 16384 points on the host: those are computed concurrently, at
// most kTableThreads at a time (this thread takes one of each group; a thread that cannot start,
// or whose computation throws, leaves its prime to this thread afterwards).
constexpr size_t kTableThreads = 8;

std::vector<std::shared_ptr<const PrimeTables>> all_prime_tables(const std::vector<int32_t>& primes,
                                                                 int M, bool rader) {
  std::vector<std::shared_ptr<const PrimeTables>> tabs(primes.size());
  std::vector<size_t> missing;
  for (size_t j = 0; j < primes.size(); ++j) {
    tabs[j] = cached_prime_tables(primes[j], M, rader);
    if (!tabs[j]) missing.push_back(j);
  }
  for (size_t next = 0; next < missing.size(); next += kTableThreads) {
    const size_t n = std::min(missing.size() - next, kTableThreads);
    std::vector<std::thread> th;
    for (size_t i = 1; i < n; ++i) {
      const size_t j = missing[next + i];
      try {
        th.emplace_back([&tabs, &primes, j, M, rader] {
          try {
            tabs[j] = prime_tables(primes[j], M, rader);
          } catch (...) {
          }
        });
      } catch (...) {
        break;
      }
    }
    tabs[missing[next]] = prime_tables(primes[missing[next]], M, rader);
    for (auto& t : th) t.join();
    for (size_t i = 1; i < n; ++i) {
      const size_t j = missing[next + i];
      if (!tabs[j]) tabs[j] = prime_tables(primes[j], M, rader);
    }
  }
  return tabs;
}

template <typename T>
void put(std::vector<char>& blob, size_t off, const std::vector<cd>& v, bool fp64) {
  if (fp64) {
    double* d = reinterpret_cast<double*>(blob.data() + off);
    for (size_t i = 0; i < v.size(); ++i) { d[2 * i] = v[i].real(); d[2 * i + 1] = v[i].imag(); }
  } else {
    float* d = reinterpret_cast<float*>(blob.data() + off);
    for (size_t i = 0; i < v.size(); ++i) {
      d[2 * i] = (float)v[i].real(); d[2 * i + 1] = (float)v[i].imag();
    }
  }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

namespace {

sft_status build_plan_body(Plan* P, int64_t N, int32_t s, const sft_variant* v, int32_t n_shifts,
                           const int64_t* primes_in, int32_t n_primes, const int32_t* small_in,
                           int32_t n_small, DeviceMemory* mem) {
  DevPlan& d = P->d;
  memset(&d, 0, sizeof(d));
  if (!v) { set_error("variant is NULL"); return SFT_EINVAL; }
  if (N < 2 || N >= (int64_t(1) << 31)) { set_error("need 2 <= N < 2^31"); return SFT_EINVAL; }
  if (s < 1 || s > N) { set_error("need 1 <= s <= N"); return SFT_EINVAL; }
  if (v->kappa < 1 || v->kappa > kMaxKappa) { set_error("kappa must be in 1..48"); return SFT_EINVAL; }
  if (2 * (int64_t)v->kappa + 1 > N) { set_error("window 2*kappa+1 exceeds N"); return SFT_EINVAL; }
  if (v->precision != SFT_FP32 && v->precision != SFT_FP64) { set_error("bad precision"); return SFT_EINVAL; }
  if (v->input != SFT_IN_C64 && v->input != SFT_IN_C128) { set_error("bad input type"); return SFT_EINVAL; }
  if (!(v->alpha >= 1.0) || !(v->beta > 0.0) || !(v->c_p > 0.0)) {
    set_error("need alpha >= 1, beta > 0, c_p > 0"); return SFT_EINVAL;
  }
  const bool fp64 = v->precision == SFT_FP64;

  // ---- Algorithm 1 set-up: c1, c2, L, shifts
  const double lnN = log((double)N);
  const double c1 = v->beta * sqrt(lnN) / (double)N;
  const int64_t L = (int64_t)ceil((double)N / (v->alpha * sqrt(lnN)));
  int64_t nq = n_shifts > 0 ? n_shifts : (int64_t)ceil(v->alpha * sqrt(lnN) / 2.0);
  if (nq < 1 || nq > kMaxQ) { set_error("number of shifts out of range 1..32"); return SFT_EINVAL; }
  if (2 * nq * L < N) { set_error("the bands [q-L, q+L) do not cover B"); return SFT_EINVAL; }
  const int64_t ceil_half = (N + 1) / 2;

  // ---- moduli
  std::vector<int32_t> primes;
  if (primes_in) {
    if (n_primes < 1 || n_primes > kMaxK) { set_error("n_primes must be 1.." + std::to_string(kMaxK)); return SFT_EINVAL; }
    for (int i = 0; i < n_primes; ++i) {
      if (primes_in[i] < 2 || primes_in[i] > (1 << 20) || !is_prime(primes_in[i])) {
        set_error("primes must be primes in [2, 2^20]"); return SFT_EINVAL;
      }
      primes.push_back((int32_t)primes_in[i]);
    }
    std::sort(primes.begin(), primes.end());
    if (std::adjacent_find(primes.begin(), primes.end()) != primes.end()) {
      set_error("primes must be distinct"); return SFT_EINVAL;
    }
  } else if (v->deterministic) {
    if (v->c_p * (double)s > 1.0e6) { set_error("c_p * s too large"); return SFT_EINVAL; }
    int Kd = 0;
    primes = deterministic_primes(N, s, v->c_p, &Kd);
    if (Kd < 0) {
      set_error("deterministic mode needs more than " + std::to_string(kMaxK) + " primes here");
      return SFT_EINVAL;
    }
  } else {
    if (v->K < 1 || v->K > kMaxK) { set_error("K must be 1.." + std::to_string(kMaxK)); return SFT_EINVAL; }
    if (v->c_p * (double)s > 1.0e6) { set_error("c_p * s too large"); return SFT_EINVAL; }
    if (v->pool != SFT_POOL_ALL && v->pool != SFT_POOL_SMOOTH) { set_error("bad prime pool"); return SFT_EINVAL; }
    primes = choose_primes(s, v->K, v->c_p, v->seed, v->pool);
  }
  std::vector<int32_t> small;
  if (small_in) {
    if (n_small < 0 || n_small > kMaxT) { set_error("n_small must be 0..12"); return SFT_EINVAL; }
    for (int i = 0; i < n_small; ++i) {
      if (small_in[i] < 2 || small_in[i] > 64) { set_error("small moduli must be in 2..64"); return SFT_EINVAL; }
      small.push_back(small_in[i]);
    }
  } else {
    small = choose_small(N, primes);
    if ((int)small.size() > kMaxT) { set_error("too many small moduli"); return SFT_EINVAL; }
  }
  for (size_t a = 0; a < small.size(); ++a)
    for (size_t b = a + 1; b < small.size(); ++b)
      if (gcd64(small[a], small[b]) != 1) { set_error("small moduli must be pairwise coprime"); return SFT_EINVAL; }
  for (int32_t p : primes)
    for (int32_t t : small)
      if (gcd64(p, t) != 1) { set_error("every p_j must be coprime to every small modulus"); return SFT_EINVAL; }
  {
    // p_1 * prod(t) >= N, computed without overflow
    int64_t prod = primes[0];
    for (int32_t t : small) { if (prod >= N) break; prod *= t; }
    if (prod < N) { set_error("p_1 * prod(small moduli) must be >= N"); return SFT_EINVAL; }
  }
  const int K = (int)primes.size();
  const int nT = (int)small.size();
  int nsub = 1;
  for (int32_t t : small) nsub += t - 1;
  if (nsub > kMaxSub) { set_error("too many node subsets (sum of t_l - 1 must be < 128)"); return SFT_EINVAL; }
  const int32_t pmax = primes.back();
  if (v->dft != SFT_DFT_AUTO && v->dft != SFT_DFT_CHIRP && v->dft != SFT_DFT_RADER) {
    set_error("bad DFT form"); return SFT_EINVAL;
  }
  // Rader's form when every p_j - 1 has a pass schedule and the two buffers fit shared memory
  std::vector<std::vector<int>> rsched(primes.size());
  bool rader_ok = v->dft != SFT_DFT_CHIRP;
  for (size_t j = 0; rader_ok && j < primes.size(); ++j)
    rader_ok = primes[j] >= 3 && (primes[j] - 1) <= (fp64 ? kRaderMaxL64 : kRaderMaxL32) &&
               rader_schedule(primes[j] - 1, rsched[j]);
  if (v->dft == SFT_DFT_RADER && !rader_ok) {
    set_error(std::string("Rader's form needs every p_j - 1 to have no prime factor above 13 and "
                          "p_j <= ") + (fp64 ? "6801 (FP64)" : "13601 (FP32)"));
    return SFT_EINVAL;
  }
  const bool rader = rader_ok;
  const int M = rader ? 0 : fft_length(2 * (int64_t)pmax - 1, fp64 ? kMaxFFT64 : kMaxFFT32);
  if (!rader && M == 0) {
    set_error(fp64 ? "FP64 plans need every p_j <= 4096 (chirp form; Rader's form reaches 6801 "
                     "when every p_j - 1 is 13-smooth)"
                   : "FP32 plans need every p_j <= 8192 (chirp form; Rader's form reaches 13601 "
                     "when every p_j - 1 is 13-smooth)");
    return SFT_EINVAL;
  }
  const int logM = rader ? 0 : fft_log2(M);

  // ---- fill the device-plan scalars
  d.N = N; d.s = s; d.kappa = v->kappa; d.K = K; d.nT = nT; d.nq = (int32_t)nq; d.nsub = nsub;
  d.prec = v->precision; d.input = v->input;
  d.refine = (v->precision == SFT_FP32 && v->refine_fp64) ? 1 : 0;
  d.fftM = M; d.fftLog2 = logM; d.pmax = pmax;
  d.rader = rader ? 1 : 0;
  d.rLmax = rader ? pmax - 1 : 0;
  d.rTpt = rader ? rader_threads(rsched, primes, pmax - 1, fp64) : 0;
  int64_t sump = 0;
  for (int j = 0; j < K; ++j) {
    d.p[j] = primes[j];
    d.poff[j] = (int32_t)sump;
    d.nodeoff[j] = sump * nsub;
    sump += primes[j];
    int64_t Mj = primes[j];
    for (int32_t t : small) Mj *= t;
    d.Mj[j] = Mj;
  }
  d.poff[K] = (int32_t)sump;
  d.nodeoff[K] = sump * nsub;
  d.Ptot = (int32_t)sump;
  d.m = sump * nsub;
  int sb = 1, tw = 0;
  d.sub_l[0] = -1; d.sub_k2[0] = 0;
  for (int l = 0; l < nT; ++l) {
    d.t[l] = small[l];
    d.subbase[l] = sb;
    d.twoff[l] = tw;
    for (int k2 = 1; k2 < small[l]; ++k2) { d.sub_l[sb] = (int8_t)l; d.sub_k2[sb] = (int8_t)k2; ++sb; }
    tw += small[l];
  }
  std::vector<int64_t> shifts;
  for (int64_t jq = 1; jq <= nq; ++jq) shifts.push_back(-ceil_half + 1 + (2 * jq - 1) * L);
  for (int i = 0; i < nq; ++i) d.q[i] = shifts[i];
  d.L = L;
  d.c1 = c1;
  d.G0 = 1.0 / ((double)N * c1);
  d.gamma = 2.0 * kPi * kPi / (((double)N * c1) * ((double)N * c1));
  d.vcap = (int32_t)sump;
  d.gamma32 = (float)d.gamma;
  d.G032 = (float)d.G0;
  d.c1f = (float)c1;
  for (int i = 0; i < nq; ++i) d.qN32[i] = (float)((double)shifts[i] / (double)N);
  for (int j = 0; j < K; ++j) {
    d.Nqp[j] = (int32_t)(N / primes[j]);
    d.Nrp[j] = (int32_t)(N % primes[j]);
  }
  for (int l = 0; l < nT; ++l) {
    d.Nqt[l] = (int32_t)(N / small[l]);
    d.Nrt[l] = (int32_t)(N % small[l]);
  }
  d.nchunk = (pmax + kReChunk - 1) / kReChunk;
  {
    const double far = (double)N - v->kappa - 0.5;
    if (d.gamma * far * far < 40.0) {
      set_error("N too small for these filter parameters (periodic images of g would matter)");
      return SFT_EINVAL;
    }
  }

  // ---- constant tables (host, FP64), laid out in one blob
  const size_t cs = fp64 ? 16 : 8;
  const int W = 2 * v->kappa + 1;
  size_t off = 0;
  const size_t o_T = off;      off = align256(off + (size_t)nq * W * cs);
  const size_t o_chirp = off;  off = align256(off + (size_t)K * pmax * cs);
  const size_t o_vhat = off;   off = align256(off + (size_t)K * M * cs);
  const size_t o_fftw = off;   off = align256(off + (size_t)M * cs);
  const size_t o_tws = off;    off = align256(off + (size_t)std::max(tw, 1) * cs);
  const size_t o_wp = off;     off = align256(off + (size_t)K * pmax * 8);
  const size_t o_gar = off;    off = align256(off + (size_t)K * std::max(nT, 1) * 4);
  const size_t o_pinv = off;   off = align256(off + (size_t)K * std::max(nT, 1) * 4);
  const size_t rk = rader ? (size_t)K : 0;
  const size_t o_rsch = off;   off = align256(off + rk * kRaderSched * 4);
  const size_t o_rperm = off;  off = align256(off + rk * 2 * pmax * 4);
  const size_t o_rV = off;     off = align256(off + rk * pmax * cs);
  const size_t o_rtw = off;    off = align256(off + rk * pmax * cs);
  const size_t table_bytes = off;
  std::vector<char> blob(table_bytes, 0);
  {
    std::vector<cd> Tt((size_t)nq * W);
    for (int qi = 0; qi < nq; ++qi)
      for (int i = -v->kappa; i <= v->kappa; ++i)
        Tt[(size_t)qi * W + (i + v->kappa)] = expi_turns(-(shifts[qi] % N) * i, N);
    put<cd>(blob, o_T, Tt, fp64);
  }
  {
    std::vector<cd> ch((size_t)K * pmax, cd(0, 0)), vh((size_t)K * M), wp((size_t)K * pmax, cd(0, 0));
    std::vector<cd> rv(rader ? (size_t)K * pmax : 0, cd(0, 0)), rt(rader ? (size_t)K * pmax : 0, cd(1, 0));
    int32_t* sch = reinterpret_cast<int32_t*>(blob.data() + o_rsch);
    int32_t* perm = reinterpret_cast<int32_t*>(blob.data() + o_rperm);
    const std::vector<std::shared_ptr<const PrimeTables>> tabs = all_prime_tables(primes, M, rader);
    for (int j = 0; j < K; ++j) {
      const std::shared_ptr<const PrimeTables>& T = tabs[j];
      std::copy(T->wp.begin(), T->wp.end(), wp.begin() + (size_t)j * pmax);
      if (!rader) {
        std::copy(T->chirp.begin(), T->chirp.end(), ch.begin() + (size_t)j * pmax);
        std::copy(T->vhat.begin(), T->vhat.end(), vh.begin() + (size_t)j * M);
        continue;
      }
      std::copy(T->pin.begin(), T->pin.end(), perm + (size_t)j * 2 * pmax);
      std::copy(T->pout.begin(), T->pout.end(), perm + (size_t)j * 2 * pmax + pmax);
      std::copy(T->rv.begin(), T->rv.end(), rv.begin() + (size_t)j * pmax);
      std::copy(T->rt.begin(), T->rt.end(), rt.begin() + (size_t)j * pmax);
      int32_t* sj = sch + (size_t)j * kRaderSched;
      sj[0] = (int32_t)T->sched.size();
      for (size_t i = 0; i < T->sched.size(); ++i) {
        sj[1 + i] = T->sched[i];
        sj[16 + i] = T->toff[i];
      }
    }
    put<cd>(blob, o_chirp, ch, fp64);
    put<cd>(blob, o_vhat, vh, fp64);
    put<cd>(blob, o_wp, wp, false);
    if (rader) {
      put<cd>(blob, o_rV, rv, fp64);
      put<cd>(blob, o_rtw, rt, fp64);
    }
  }
  {
    std::vector<cd> fw(M, cd(1, 0));
    for (int span = 2; span < M; span *= fft_radix(M, span)) {
      const int R = fft_radix(M, span), base = fft_tw_offset(M, span);
      for (int row = 0; row < fft_tw_rows(R); ++row)
        for (int k = 0; k < span; ++k)
          fw[(size_t)base + (size_t)row * span + k] =
              expi_turns(-(int64_t)fft_tw_exp(row) * k, (int64_t)span * R);
    }
    put<cd>(blob, o_fftw, fw, fp64);
    std::vector<cd> ts(std::max(tw, 1), cd(1, 0));
    for (int l = 0; l < nT; ++l)
      for (int n = 0; n < small[l]; ++n) ts[d.twoff[l] + n] = expi_turns(-n, small[l]);
    put<cd>(blob, o_tws, ts, fp64);
    int32_t* gar = reinterpret_cast<int32_t*>(blob.data() + o_gar);
    int32_t* pin = reinterpret_cast<int32_t*>(blob.data() + o_pinv);
    for (int j = 0; j < K; ++j) {
      int64_t Mprev = primes[j];
      for (int l = 0; l < nT; ++l) {
        gar[j * nT + l] = (int32_t)inv_mod(Mprev % small[l], small[l]);
        pin[j * nT + l] = (int32_t)inv_mod(primes[j] % small[l], small[l]);
        Mprev *= small[l];
      }
    }
  }

  // ---- scratch layout
  size_t soff = align256(table_bytes);
  const size_t o_samples = soff; soff = align256(soff + (size_t)nq * d.m * cs);
  const size_t o_bins = soff;    soff = align256(soff + (size_t)nq * d.m * cs);
  const size_t o_cand = soff;    soff = align256(soff + (size_t)nq * sump * 8);
  const size_t o_resid = soff;   soff = align256(soff + (size_t)nq * sump * std::max(nT, 1));
  const size_t o_cnt = soff;     soff = align256(soff + (size_t)(nq + 4) * 4);
  const size_t o_voted = soff;   soff = align256(soff + (size_t)nq * d.vcap * sizeof(Voted));
  const size_t o_pool = soff;    soff = align256(soff + (size_t)nq * s * sizeof(Pooled));
  const size_t o_win = soff;     soff = align256(soff + (size_t)s * sizeof(Pooled));
  const size_t o_ybuf = soff;    soff = align256(soff + (size_t)d.nchunk * s * K * sizeof(double2));
  const size_t o_wlist = soff;   soff = align256(soff + (size_t)s * 4);
  const size_t o_woff = soff;    soff = align256(soff + (size_t)(nq + 1) * 4);
  const size_t o_epart = soff;   soff = align256(soff + (size_t)kEnergyBlocks * sizeof(double));
  const size_t o_self = soff;    soff = align256(soff + sizeof(DevPlan));
  const size_t total = soff;

  char* base = nullptr;
  cudaError_t e = cudaSuccess;
  P->mem = mem;
  P->want_bytes = total;
  if (mem) {
    base = static_cast<char*>(mem->alloc(total));
    if (!base) {
      set_error("plan needs " + std::to_string(total) + " device bytes: not available in the arena");
      return SFT_ENOMEM;
    }
  } else {
    e = dev_malloc((void**)&base, total);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error(std::string("cudaMalloc of plan memory failed: ") + cudaGetErrorString(e));
      return SFT_ENOMEM;
    }
  }
  P->allocations.push_back(base);
  e = mem ? mem->upload(base, blob.data(), table_bytes)
          : cudaMemcpy(base, blob.data(), table_bytes, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    set_error(std::string("copy of plan tables failed: ") + cudaGetErrorString(e));
    free_plan(P);
    return SFT_ECUDA;
  }
  d.Ttab = base + o_T; d.chirp = base + o_chirp; d.vhat = base + o_vhat; d.fftw = base + o_fftw;
  d.twsmall = base + o_tws; d.wp32 = reinterpret_cast<const float2*>(base + o_wp);
  d.garner = reinterpret_cast<const int32_t*>(base + o_gar);
  d.pinv = reinterpret_cast<const int32_t*>(base + o_pinv);
  if (rader) {
    d.rsched = reinterpret_cast<const int32_t*>(base + o_rsch);
    d.rperm = reinterpret_cast<const int32_t*>(base + o_rperm);
    d.rV = base + o_rV;
    d.rtw = base + o_rtw;
  }
  d.samples = base + o_samples; d.bins = base + o_bins;
  d.cand = reinterpret_cast<int64_t*>(base + o_cand);
  d.resid = reinterpret_cast<uint8_t*>(base + o_resid);
  d.counters = reinterpret_cast<int32_t*>(base + o_cnt);
  d.voted = reinterpret_cast<Voted*>(base + o_voted);
  d.pool = reinterpret_cast<Pooled*>(base + o_pool);
  d.winners = reinterpret_cast<Pooled*>(base + o_win);
  d.ybuf = reinterpret_cast<double2*>(base + o_ybuf);
  d.wlist = reinterpret_cast<int32_t*>(base + o_wlist);
  d.woff = reinterpret_cast<int32_t*>(base + o_woff);
  d.epart = reinterpret_cast<double*>(base + o_epart);
  P->d_dev = reinterpret_cast<DevPlan*>(base + o_self);
  e = mem ? mem->upload(P->d_dev, &d, sizeof(DevPlan))
          : cudaMemcpy(P->d_dev, &d, sizeof(DevPlan), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    set_error(std::string("copy of the plan record failed: ") + cudaGetErrorString(e));
    free_plan(P);
    return SFT_ECUDA;
  }
  P->device_bytes = total;
  P->alpha = v->alpha; P->beta = v->beta; P->seed = v->seed;
  P->shifts = shifts; P->primes = primes; P->small = small;
  cudaGetDevice(&P->device);
  return SFT_OK;
}

}  // namespace

sft_status choose_moduli_deterministic(int64_t N, int32_t s, double c_p, int64_t* primes_out,
                                       int32_t* K_out, int32_t* small_out, int32_t* n_small_out) {
  if (!primes_out || !K_out || !small_out || !n_small_out) { set_error("NULL output"); return SFT_EINVAL; }
  if (N < 2 || s < 1 || s > N || !(c_p > 0.0) || c_p * (double)s > 1.0e6) {
    set_error("need N >= 2, 1 <= s <= N, c_p > 0");
    return SFT_EINVAL;
  }
  int K = 0;
  std::vector<int32_t> pr = deterministic_primes(N, s, c_p, &K);
  if (K < 0) { set_error("deterministic mode needs more than " + std::to_string(kMaxK) + " primes here"); return SFT_EINVAL; }
  std::vector<int32_t> sm = choose_small(N, pr);
  if ((int)sm.size() > kMaxT) { set_error("too many small moduli"); return SFT_EINVAL; }
  for (int j = 0; j < K; ++j) primes_out[j] = pr[j];
  *K_out = K;
  for (size_t l = 0; l < sm.size(); ++l) small_out[l] = sm[l];
  *n_small_out = (int32_t)sm.size();
  return SFT_OK;
}

sft_status choose_moduli(int64_t N, int32_t s, int32_t K, double c_p, uint64_t seed,
                         int64_t* primes_out, int32_t* small_out, int32_t* n_small_out, int pool) {
  if (!primes_out || !small_out || !n_small_out) { set_error("NULL output"); return SFT_EINVAL; }
  if (N < 2 || N >= (int64_t(1) << 31) || s < 1 || s > N) { set_error("need 2 <= N < 2^31, 1 <= s <= N"); return SFT_EINVAL; }
  if (K < 1 || K > kMaxK || !(c_p > 0.0) || c_p * (double)s > 1.0e6) { set_error("bad K or c_p"); return SFT_EINVAL; }
  if (pool != SFT_POOL_ALL && pool != SFT_POOL_SMOOTH) { set_error("bad prime pool"); return SFT_EINVAL; }
  std::vector<int32_t> pr = choose_primes(s, K, c_p, seed, pool);
  std::vector<int32_t> sm = choose_small(N, pr);
  if ((int)sm.size() > kMaxT) { set_error("too many small moduli"); return SFT_EINVAL; }
  for (int j = 0; j < K; ++j) primes_out[j] = pr[j];
  for (size_t l = 0; l < sm.size(); ++l) small_out[l] = sm[l];
  *n_small_out = (int32_t)sm.size();
  return SFT_OK;
}

// The plan build's host containers can throw (std::bad_alloc); no exception leaves the library:
// the device memory taken so far is released and the failure becomes a status.
sft_status build_plan(Plan* P, int64_t N, int32_t s, const sft_variant* v, int32_t n_shifts,
                      const int64_t* primes_in, int32_t n_primes, const int32_t* small_in,
                      int32_t n_small, DeviceMemory* mem) {
  try {
    return build_plan_body(P, N, s, v, n_shifts, primes_in, n_primes, small_in, n_small, mem);
  } catch (const std::bad_alloc&) {
    free_plan(P);
    set_error("host allocation failed while building the plan");
    return SFT_ENOMEM;
  } catch (const std::exception& e) {
    free_plan(P);
    set_error(std::string("plan build failed: ") + e.what());
    return SFT_EINVAL;
  }
}

void free_plan(Plan* P) {
  for (void* a : P->allocations) {
    if (P->mem) P->mem->release(a);
    else cudaFree(a);
  }
  P->allocations.clear();
}

}  // namespace sft
