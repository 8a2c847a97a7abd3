// Host-compiled check of the plan's integer helpers (csrc/int_math.h) against brute force:
//   is_prime   against a sieve of Eratosthenes below 2^21 and known large primes and composites;
//   gcd64      against the largest common divisor found by search, signs and zeros included;
//   inv_mod    for every modulus m <= 3000 and every a coprime to m (negative a too):
//              a inv = 1 (mod m), inv in [0, m) (the Garner constants of the CRT come from it);
//   smooth13   against trial factorisation up to 2 10^5.
// Prints "ok" and exits 0, or names the first failure and exits 1.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../paper_1706_02740_gb300/csrc/int_math.h"

using namespace sft;

int main() {
  const int top = 1 << 21;
  std::vector<char> comp(top, 0);
  comp[0] = comp[1] = 1;
  for (int i = 2; (int64_t)i * i < top; ++i)
    if (!comp[i])
      for (int j = i * i; j < top; j += i) comp[j] = 1;
  for (int64_t n = -5; n < top; ++n)
    if (is_prime(n) != (n >= 0 && !comp[n])) {
      std::printf("is_prime(%lld)\n", (long long)n);
      return 1;
    }
  for (int64_t n : {2147483647LL, 4194301LL, 1000003LL, 999999999989LL})
    if (!is_prime(n)) { std::printf("is_prime(%lld) false\n", (long long)n); return 1; }
  for (int64_t n : {2147483649LL, 4194303LL, 1000001LL, 999999999987LL, 3LL * 1000003LL})
    if (is_prime(n)) { std::printf("is_prime(%lld) true\n", (long long)n); return 1; }

  for (int64_t a = -60; a <= 60; ++a)
    for (int64_t b = -60; b <= 60; ++b) {
      int64_t want = 0;
      for (int64_t d = 1; d <= 60; ++d)
        if (a % d == 0 && b % d == 0) want = d;
      if (a == 0 && b == 0) want = 0;
      if (gcd64(a, b) != want) {
        std::printf("gcd64(%lld, %lld) = %lld, want %lld\n", (long long)a, (long long)b,
                    (long long)gcd64(a, b), (long long)want);
        return 1;
      }
    }

  for (int64_t m = 1; m <= 3000; ++m)
    for (int64_t a = 0; a < m; ++a) {
      if (gcd64(a, m) != 1) continue;
      const int64_t v = inv_mod(a, m);
      if (v < 0 || v >= m || (m > 1 && (a * v) % m != 1) || inv_mod(a - 7 * m, m) != v) {
        std::printf("inv_mod(%lld, %lld) = %lld\n", (long long)a, (long long)m, (long long)v);
        return 1;
      }
    }

  for (int64_t n = -3; n <= 200000; ++n) {
    bool want = n >= 1;
    int64_t r = n;
    for (int64_t f = 2; want && r > 1 && f * f <= r; ++f)
      while (r % f == 0) {
        if (f > 13) want = false;
        r /= f;
      }
    if (want && r > 13) want = false;
    if (smooth13(n) != want) { std::printf("smooth13(%lld)\n", (long long)n); return 1; }
  }
  std::printf("ok\n");
  return 0;
}
