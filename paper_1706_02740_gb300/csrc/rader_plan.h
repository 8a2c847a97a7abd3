// Host planning of Rader's form for a prime p: the pass schedule of the length-(p - 1) FFTs, the
// threads per transform, and the primitive root whose powers order the nonzero indices.
#pragma once

#include <stdint.h>

#include <algorithm>
#include <vector>

#include "sft_internal.h"

namespace sft {

// Pass schedule of a length-L mixed-radix FFT for Rader's form: the radices multiply to L and each
// is one of the in-register DFTs (2, 3, 4, 5, 6, 7, 8, 10, 11, 12, 13, 14, 16): every 7, 5 and 3
// takes a factor 2 (14, 10) or 4 (12) or 2 (6) while any is left, 11 and 13 stand alone, the
// remaining powers of two go in radix-16 passes and one last 8, 4 or 2; largest radix first.
// False when L has a prime factor above 13, L < 2 or the schedule is too long.
inline bool rader_schedule(int L, std::vector<int>& rad) {
  rad.clear();
  if (L < 2) return false;
  int e[6] = {0, 0, 0, 0, 0, 0};
  const int f[6] = {2, 3, 5, 7, 11, 13};
  int n = L;
  for (int i = 0; i < 6; ++i)
    while (n % f[i] == 0) { n /= f[i]; ++e[i]; }
  if (n != 1) return false;
  int a2 = e[0];
  for (int i = 0; i < e[3]; ++i) { if (a2 > 0) { rad.push_back(14); --a2; } else rad.push_back(7); }
  for (int i = 0; i < e[2]; ++i) { if (a2 > 0) { rad.push_back(10); --a2; } else rad.push_back(5); }
  for (int i = 0; i < e[1]; ++i) {
    if (a2 >= 2) { rad.push_back(12); a2 -= 2; }
    else if (a2 == 1) { rad.push_back(6); --a2; }
    else rad.push_back(3);
  }
  for (int i = 0; i < e[4]; ++i) rad.push_back(11);
  for (int i = 0; i < e[5]; ++i) rad.push_back(13);
  while (a2 >= 4) { rad.push_back(16); a2 -= 4; }
  if (a2 > 0) rad.push_back(1 << a2);
  std::sort(rad.begin(), rad.end(), [](int x, int y) { return x > y; });
  return (int)rad.size() <= kRaderMaxPasses;
}

// Threads per Rader transform (one transform per CTA): the whole-warp count in 32..512 that
// maximises resident CTAs per SM over the pass iterations of the plan's transforms.  A CTA's
// threads take a pass's L/R items in ceil(L/(R t)) rounds; residency is bounded by shared memory
// (two buffers of rader_buf(Lmax) elements), registers (64 a thread FP32, 128 FP64) and 2048
// threads per SM.  Ties go to fewer threads.
inline int rader_threads(const std::vector<std::vector<int>>& sched,
                         const std::vector<int32_t>& primes, int Lmax, bool fp64) {
  const double smem = 2.0 * rader_buf(Lmax) * (fp64 ? 16 : 8) + 1024;
  const int regs = fp64 ? 128 : 64;
  int best_t = 256;
  double best = -1;
  for (int t = 32; t <= 512; t += 32) {
    const int by_smem = (int)((228.0 * 1024) / smem);
    const int ctas = std::min(std::min(by_smem, 65536 / (regs * t)), std::min(2048 / t, 32));
    if (ctas < 1) continue;
    int64_t rounds = 0;
    for (size_t j = 0; j < primes.size(); ++j) {
      const int L = primes[j] - 1;
      for (int R : sched[j]) rounds += (L / R + t - 1) / t;
    }
    const double rate = (double)ctas / (double)rounds;
    if (rate > best * (1 + 1e-9)) { best = rate; best_t = t; }
  }
  return best_t;
}

// b^e mod m by repeated squaring (m^2 must fit in int64).
inline int64_t pow_mod(int64_t b, int64_t e, int64_t m) {
  int64_t r = 1 % m;
  b %= m;
  while (e) {
    if (e & 1) r = r * b % m;
    b = b * b % m;
    e >>= 1;
  }
  return r;
}

// Smallest primitive root modulo the prime p (p - 1 13-smooth): g with g^((p-1)/q) != 1 for every
// prime q dividing p - 1.
inline int64_t primitive_root(int64_t p) {
  std::vector<int64_t> qs;
  int64_t n = p - 1;
  for (int64_t q : {2, 3, 5, 7, 11, 13})
    if (n % q == 0) { qs.push_back(q); while (n % q == 0) n /= q; }
  for (int64_t g = 2; g < p; ++g) {
    bool ok = true;
    for (int64_t q : qs) ok = ok && pow_mod(g, (p - 1) / q, p) != 1;
    if (ok) return g;
  }
  return 1;   // p = 2
}

}  // namespace sft
