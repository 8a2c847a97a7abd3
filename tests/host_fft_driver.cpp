// Host-compiled check of the plan's FP64 host FFTs (csrc/host_fft.h) against the defining sum
// X_k = sum_n a_n e^{-2 pi i n k / M}, evaluated in long double with the exponent n k reduced
// exactly modulo M.  Lengths: every chirp-convolution length r 2^k (r = 1, 3, 5, 7) up to the FP32
// limit, through host_fft, and Rader lengths p - 1 through host_fft_mixed.  Up to 4096 every bin
// is checked; above, 97 bins spread over the spectrum (each O(M)).  Prints one line per length:
//   kind M err bound
// with err = ||X - X_ref||_2 / ||X_ref||_2 over the checked bins, and first the turns and twiddles
// as "turns 0 err bound" (absolute error in units of u = 2^-53).  Exits non-zero if any error is
// above its bound.
#include <cmath>
#include <cstdio>
#include <vector>

#include "../paper_1706_02740_gb300/csrc/host_fft.h"

using namespace sft;

namespace {

using ld = long double;
const ld kPiL = 3.14159265358979323846264338327950288L;
const double kEps = 0x1p-53;

uint64_t g_state = 0x243F6A8885A308D3ULL;
double uniform() {                       // xorshift64*, mapped to [-1, 1)
  g_state ^= g_state >> 12;
  g_state ^= g_state << 25;
  g_state ^= g_state >> 27;
  const uint64_t v = g_state * 0x2545F4914F6CDD1DULL;
  return (double)(v >> 11) * 0x1p-52 - 1.0;
}

// e^{-2 pi i j / M} for j < M in long double.
void ref_table(int64_t M, std::vector<ld>& c, std::vector<ld>& s) {
  c.resize(M);
  s.resize(M);
  for (int64_t j = 0; j < M; ++j) {
    const ld t = 2 * kPiL * (ld)j / (ld)M;
    c[j] = cosl(t);
    s[j] = -sinl(t);
  }
}

// Relative L2 error of X against the defining sum over the checked bins.
double dft_error(const std::vector<cd>& a, const std::vector<cd>& X) {
  const int64_t M = (int64_t)a.size();
  std::vector<ld> c, s;
  ref_table(M, c, s);
  std::vector<int64_t> bins;
  if (M <= 4096) {
    for (int64_t k = 0; k < M; ++k) bins.push_back(k);
  } else {
    for (int64_t i = 0; i < 97; ++i) bins.push_back((i * M) / 97 + (i % 5));
    bins.push_back(M - 1);
  }
  ld num = 0, den = 0;
  for (int64_t k : bins) {
    ld re = 0, im = 0;
    for (int64_t n = 0; n < M; ++n) {
      const int64_t j = (n * k) % M;
      re += (ld)a[n].real() * c[j] - (ld)a[n].imag() * s[j];
      im += (ld)a[n].real() * s[j] + (ld)a[n].imag() * c[j];
    }
    const ld dr = (ld)X[k].real() - re, di = (ld)X[k].imag() - im;
    num += dr * dr + di * di;
    den += re * re + im * im;
  }
  return (double)sqrtl(num / den);
}

std::vector<cd> random_vector(int64_t M) {
  std::vector<cd> a(M);
  for (auto& v : a) v = cd(uniform(), uniform());
  return a;
}

// Absolute error bound of a computed turn e^{i t}, t = 2 pi r / den in [0, 2 pi): kPi carries a
// relative error below u, the product and the quotient one rounding each, so |t^ - t| <= 3 u t,
// and sincos adds at most 1 ulp (u for values below 1): (3 t_max + 1) u.  expi_turns: t_max = 2 pi;
// half_turn_twiddles: pi / 4 when 8 divides M (octant symmetries are exact), else pi.
const double kMuTurn = (6 * M_PI + 1) * kEps;

// Relative L2 error bound of a decimation-in-time FFT with stage radices r_i, to first order in u:
// the sum over stages of eta_r = sqrt(r) (mu + (2 sqrt(2) + r - 1) u).  Each stage output is a sum
// of r twiddled terms: twiddle error mu, complex product sqrt(2) gamma_2 ~ 2 sqrt(2) u (Higham,
// Accuracy and Stability of Numerical Algorithms, Lemma 3.5), recursive summation gamma_{r-1}
// (Lemma 3.4 form); sqrt(r) is Cauchy-Schwarz over a stage that scales norms by sqrt(r).  For
// r = 2 this is sqrt(2) (mu + 3.83 u), above the eta = mu + gamma_4 (sqrt(2) + mu) of Higham's
// Theorem 24.2 for the radix-2 FFT.
double dit_bound(const std::vector<int64_t>& radices) {
  double b = 0;
  for (int64_t r : radices)
    b += std::sqrt((double)r) * (kMuTurn + (2 * std::sqrt(2.0) + (double)(r - 1)) * kEps);
  return b;
}

std::vector<int64_t> factor_smallest_first(int64_t L) {
  std::vector<int64_t> f;
  for (int64_t r = 2; L > 1;) {
    if (L % r == 0) { f.push_back(r); L /= r; }
    else ++r;
  }
  return f;
}

bool check_turns() {
  // expi_turns reduces num exactly modulo den: compare with the long double turn for numerators far
  // beyond den, of both signs (the Rader chirp uses -(n^2 mod 2p), the twiddles -t k).
  double worst = 0;
  for (int64_t den : {7LL, 96LL, 4099LL, 2LL * 16411, 1LL << 20, 1000003LL}) {
    for (int64_t i = -40; i <= 40; ++i) {
      const int64_t num = i * 7919 * 104729 + i;
      const cd e = expi_turns(num, den);
      const int64_t r = ((num % den) + den) % den;
      const ld t = 2 * kPiL * (ld)r / (ld)den;
      const double err =
          (double)fmaxl(fabsl((ld)e.real() - cosl(t)), fabsl((ld)e.imag() - sinl(t)));
      if (err > worst) worst = err;
    }
  }
  std::printf("turns 0 %.3e %.3e\n", worst / kEps, kMuTurn / kEps);
  bool ok = worst <= kMuTurn;
  // half_turn_twiddles: e^{-2 pi i k / M}, k < M / 2, octant symmetries exact.
  for (size_t M : {2, 4, 6, 8, 12, 24, 64, 96, 640, 896, 4096, 7168, 16384}) {
    std::vector<double> w;
    half_turn_twiddles(M, w);
    worst = 0;
    for (size_t k = 0; k < M / 2; ++k) {
      const ld t = 2 * kPiL * (ld)k / (ld)M;
      const double err =
          (double)fmaxl(fabsl((ld)w[2 * k] - cosl(t)), fabsl((ld)w[2 * k + 1] + sinl(t)));
      if (err > worst) worst = err;
    }
    const double bound = ((M % 8 == 0 ? 3 * M_PI / 4 : 3 * M_PI) + 1) * kEps;
    std::printf("twiddles %zu %.3e %.3e\n", M, worst / kEps, bound / kEps);
    if (!(worst <= bound)) ok = false;
  }
  return ok;
}

}  // namespace

int main() {
  bool ok = check_turns();
  std::vector<int64_t> chirp = {1, 2, 4, 8, 16, 32};
  for (int64_t base : {64, 96, 640, 896})
    for (int64_t m = base; m <= kMaxFFT32; m <<= 1) chirp.push_back(m);
  for (int64_t M : chirp) {
    const std::vector<cd> a = random_vector(M);
    std::vector<cd> X = a;
    host_fft(X);
    std::vector<int64_t> rad(fft_log2((int)(M / fft_odd((int)M))), 2);
    if (fft_odd((int)M) > 1) rad.push_back(fft_odd((int)M));
    const double err = dft_error(a, X), bound = dit_bound(rad);
    std::printf("chirp %lld %.3e %.3e\n", (long long)M, err, bound);
    if (!(err <= bound)) ok = false;
  }
  // Rader lengths p - 1: smooth ones, ones with a large prime factor, and lengths near the FP32
  // limit of Rader's form.
  for (int64_t L : {1LL, 2LL, 6LL, 10LL, 96LL, 1008LL, 2 * 3 * 683LL, 2 * 3 * 5 * 137LL,
                    2 * 4099LL, 12 * 1000LL, 2LL * 5 * 1327, 13596LL}) {
    const std::vector<cd> a = random_vector(L);
    std::vector<cd> X = a;
    host_fft_mixed(X);
    const double err = dft_error(a, X), bound = dit_bound(factor_smallest_first(L));
    std::printf("rader %lld %.3e %.3e\n", (long long)L, err, bound);
    if (!(err <= bound)) ok = false;
  }
  std::printf(ok ? "ok\n" : "FAILED\n");
  return ok ? 0 : 1;
}
