// Integer helpers of the plan: primality, gcd, modular inverse (the Garner constants of the
// residue reconstruction) and 13-smoothness (Rader's pass schedules).
#pragma once

#include <stdint.h>

#include <initializer_list>

namespace sft {

// Trial division.
inline bool is_prime(int64_t n) {
  if (n < 2) return false;
  if (n < 4) return true;
  if (n % 2 == 0) return false;
  for (int64_t i = 3; i * i <= n; i += 2)
    if (n % i == 0) return false;
  return true;
}

// Greatest common divisor (non-negative) by Euclid's algorithm.
inline int64_t gcd64(int64_t a, int64_t b) {
  while (b) {
    int64_t t = a % b;
    a = b;
    b = t;
  }
  return a < 0 ? -a : a;
}

// Inverse of a modulo m (a, m coprime, m >= 1) by the extended Euclidean algorithm.
inline int64_t inv_mod(int64_t a, int64_t m) {
  if (m == 1) return 0;
  int64_t g = m, x = 0, x1 = 1, a1 = ((a % m) + m) % m;
  while (a1) {
    int64_t qq = g / a1;
    int64_t t = g - qq * a1; g = a1; a1 = t;
    t = x - qq * x1; x = x1; x1 = t;
  }
  return ((x % m) + m) % m;
}

// True when n >= 1 has no prime factor above 13.
inline bool smooth13(int64_t n) {
  if (n < 1) return false;
  for (int64_t t : {2, 3, 5, 7, 11, 13})
    while (n % t == 0) n /= t;
  return n == 1;
}

}  // namespace sft
