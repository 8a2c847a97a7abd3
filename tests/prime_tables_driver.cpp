// Host-compiled check of the per-prime DFT tables (csrc/prime_tables.h): each form's length-p DFT
// E_c = (1/p) sum_k x_k e^{-2 pi i k c / p} is run on the host in FP64 from the tables exactly as
// the kernels combine them, and compared with the defining sum in long double.
//   chirp form (w = chirp, V = vhat):
//     E = w . conj( FFT_M( conj( FFT_M(x w, zero padded) . V ) ) )
//   Rader's form (a_n = x_{g^n}, V = rv):
//     E_{g^{-m}} = x_0 / p + conj( FFT_L( conj( FFT_L(a) . V ) ) )_m,  E_0 = (x_0 + sum_n a_n) / p
// Also the re-estimation twiddles wp against e^{-2 pi i n / p} (within the turns' bound), and the
// permutations g^n, g^{-n} as inverse bijections of 1 .. p - 1.  Prints "chirp p M err" /
// "rader p err" and "ok"; exits non-zero when an error exceeds 1e-13 (relative L2, a hundredth of
// the FP64 path's tolerance; a wrong index, wrap or scale in a table gives an error of order one)
// or a permutation is wrong.
#include <cmath>
#include <cstdio>
#include <vector>

#include "../paper_1706_02740_gb300/csrc/prime_tables.h"

using namespace sft;

namespace {

using ld = long double;
const ld kPiL = 3.14159265358979323846264338327950288L;
const double kTol = 1e-13;

uint64_t g_state = 0x6A09E667F3BCC909ULL;
double uniform() {                       // xorshift64*, mapped to [-1, 1)
  g_state ^= g_state >> 12;
  g_state ^= g_state << 25;
  g_state ^= g_state >> 27;
  return (double)((g_state * 0x2545F4914F6CDD1DULL) >> 11) * 0x1p-52 - 1.0;
}

// Relative L2 error of E against (1/p) sum_k x_k e^{-2 pi i k c / p}, kc reduced exactly mod p.
double dft_error(const std::vector<cd>& x, const std::vector<cd>& E) {
  const int64_t p = (int64_t)x.size();
  std::vector<ld> c(p), s(p);
  for (int64_t j = 0; j < p; ++j) {
    c[j] = cosl(2 * kPiL * (ld)j / (ld)p);
    s[j] = -sinl(2 * kPiL * (ld)j / (ld)p);
  }
  ld num = 0, den = 0;
  for (int64_t k = 0; k < p; ++k) {
    ld re = 0, im = 0;
    for (int64_t n = 0; n < p; ++n) {
      const int64_t j = (n * k) % p;
      re += (ld)x[n].real() * c[j] - (ld)x[n].imag() * s[j];
      im += (ld)x[n].real() * s[j] + (ld)x[n].imag() * c[j];
    }
    re /= (ld)p;
    im /= (ld)p;
    const ld dr = (ld)E[k].real() - re, di = (ld)E[k].imag() - im;
    num += dr * dr + di * di;
    den += re * re + im * im;
  }
  return (double)sqrtl(num / den);
}

std::vector<cd> random_vector(int64_t n) {
  std::vector<cd> a(n);
  for (auto& v : a) v = cd(uniform(), uniform());
  return a;
}

// wp[n] = e^{-2 pi i n / p} within the turns' bound (6 pi + 1) 2^-53 (three roundings in the
// argument, one in sincos).
bool check_wp(const PrimeTables& T, int64_t p) {
  const ld bound = (6 * kPiL + 1) * 0x1p-53L;
  for (int64_t n = 0; n < p; ++n) {
    const ld t = 2 * kPiL * (ld)n / (ld)p;
    if (fabsl((ld)T.wp[n].real() - cosl(t)) > bound || fabsl((ld)T.wp[n].imag() + sinl(t)) > bound)
      return false;
  }
  return true;
}

}  // namespace

int main() {
  bool ok = true;
  for (int64_t p : {3LL, 5LL, 7LL, 13LL, 97LL, 1009LL, 3001LL, 3079LL, 3137LL, 4099LL, 8191LL}) {
    const int M = fft_length(2 * p - 1, kMaxFFT32);
    const auto T = compute_prime_tables(p, M, false);
    const std::vector<cd> x = random_vector(p);
    std::vector<cd> a(M, cd(0, 0));
    for (int64_t n = 0; n < p; ++n) a[n] = x[n] * T->chirp[n];
    host_fft(a);
    for (int i = 0; i < M; ++i) a[i] = std::conj(a[i] * T->vhat[i]);
    host_fft(a);
    std::vector<cd> E(p);
    for (int64_t c = 0; c < p; ++c) E[c] = T->chirp[c] * std::conj(a[c]);
    const double err = dft_error(x, E);
    const bool wp = check_wp(*T, p);
    std::printf("chirp %lld %d %.3e\n", (long long)p, M, err);
    if (!(err <= kTol) || !wp) ok = false;
  }
  for (int64_t p : {5LL, 7LL, 13LL, 97LL, 3001LL, 3137LL, 7681LL, 12289LL, 13313LL}) {
    const int64_t L = p - 1;
    const auto T = compute_prime_tables(p, 0, true);
    // g^n and g^{-n}: inverse bijections of 1 .. p - 1
    std::vector<char> seen_in(p, 0), seen_out(p, 0);
    for (int64_t n = 0; n < L; ++n) {
      const int64_t u = T->pin[n], v = T->pout[n];
      if (u < 1 || u >= p || v < 1 || v >= p || seen_in[u] || seen_out[v] || (u * v) % p != 1) {
        std::printf("rader %lld: permutation entry %lld wrong\n", (long long)p, (long long)n);
        return 1;
      }
      seen_in[u] = seen_out[v] = 1;
    }
    const std::vector<cd> x = random_vector(p);
    std::vector<cd> A(L);
    cd sum(0, 0);
    for (int64_t n = 0; n < L; ++n) {
      A[n] = x[T->pin[n]];
      sum += A[n];
    }
    host_fft_mixed(A);
    for (int64_t k = 0; k < L; ++k) A[k] = std::conj(A[k] * T->rv[k]);
    host_fft_mixed(A);
    std::vector<cd> E(p);
    E[0] = (x[0] + sum) / (double)p;
    for (int64_t m = 0; m < L; ++m) E[T->pout[m]] = x[0] / (double)p + std::conj(A[m]);
    const double err = dft_error(x, E);
    const bool wp = check_wp(*T, p);
    std::printf("rader %lld %.3e\n", (long long)p, err);
    if (!(err <= kTol) || !wp) ok = false;
  }
  std::printf(ok ? "ok\n" : "FAILED\n");
  return ok ? 0 : 1;
}
