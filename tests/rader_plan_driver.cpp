// Host-compiled check of Rader's-form planning (csrc/rader_plan.h) for every prime p with
// 3 <= p <= kRaderMaxL32 + 1:
//   * rader_schedule(p - 1) succeeds exactly when p - 1 has no prime factor above 13; its radices
//     multiply to p - 1, each is one the Rader kernel has an in-register DFT for (2, 3, 4, 5, 6, 7,
//     8, 10, 11, 12, 13, 14, 16), largest first, at most one lone power of two below 16;
//   * primitive_root(p) has order exactly p - 1 (its powers run through every nonzero residue,
//     brute force) and no smaller g does;
//   * the two transform buffers of the longest admissible lengths fit one CTA's shared memory;
//   * rader_threads picks a whole-warp count in 32..512 for seeded sets of five smooth primes.
// Prints "sched p g G | radices" for a few primes, "primes P smooth S maxpasses X maxroot G" and
// "ok"; exits non-zero on the first failure.
#include <cstdio>
#include <vector>

#include "../paper_1706_02740_gb300/csrc/rader_plan.h"

using namespace sft;

namespace {

bool has_dft(int R) {
  for (int r : {2, 3, 4, 5, 6, 7, 8, 10, 11, 12, 13, 14, 16})
    if (r == R) return true;
  return false;
}

bool smooth13(int L) {
  for (int f : {2, 3, 5, 7, 11, 13})
    while (L % f == 0) L /= f;
  return L == 1;
}

// Order of g modulo p by walking its powers.
int64_t order_of(int64_t g, int64_t p) {
  int64_t x = g % p, k = 1;
  while (x != 1) {
    x = x * g % p;
    ++k;
    if (k > p) return -1;
  }
  return k;
}

}  // namespace

int main() {
  const int top = kRaderMaxL32 + 1;
  std::vector<char> composite(top + 1, 0);
  std::vector<int> primes;
  for (int i = 2; i <= top; ++i) {
    if (composite[i]) continue;
    primes.push_back(i);
    for (int64_t j = (int64_t)i * i; j <= top; j += i) composite[j] = 1;
  }
  int n_smooth = 0, max_passes = 0;
  int64_t max_root = 0;
  std::vector<int> smooth_primes;
  for (int p : primes) {
    if (p < 3) continue;
    const int L = p - 1;
    std::vector<int> rad;
    const bool ok = rader_schedule(L, rad);
    if (ok != smooth13(L)) {
      std::printf("p = %d: schedule %d but smooth %d\n", p, (int)ok, (int)smooth13(L));
      return 1;
    }
    if (!ok) continue;
    ++n_smooth;
    smooth_primes.push_back(p);
    int64_t prod = 1;
    int lone_pow2 = 0;
    for (size_t i = 0; i < rad.size(); ++i) {
      if (!has_dft(rad[i]) || (i > 0 && rad[i] > rad[i - 1])) {
        std::printf("p = %d: radix %d at pass %zu\n", p, rad[i], i);
        return 1;
      }
      if (rad[i] == 2 || rad[i] == 4 || rad[i] == 8) ++lone_pow2;
      prod *= rad[i];
    }
    if (prod != L || lone_pow2 > 1 || (int)rad.size() > kRaderMaxPasses) {
      std::printf("p = %d: radices multiply to %lld, %d lone powers of two, %zu passes\n", p,
                  (long long)prod, lone_pow2, rad.size());
      return 1;
    }
    if ((int)rad.size() > max_passes) max_passes = (int)rad.size();
    const int64_t g = primitive_root(p);
    if (order_of(g, p) != L) {
      std::printf("p = %d: g = %lld has order %lld\n", p, (long long)g, (long long)order_of(g, p));
      return 1;
    }
    for (int64_t h = 2; h < g; ++h)
      if (order_of(h, p) == L) {
        std::printf("p = %d: %lld is a smaller primitive root than %lld\n", p, (long long)h,
                    (long long)g);
        return 1;
      }
    if (pow_mod(g, p - 2, p) * g % p != 1) {
      std::printf("p = %d: inverse of g by Fermat fails\n", p);
      return 1;
    }
    if (g > max_root) max_root = g;
    if (p == 13 || p == 3001 || p == 3137 || p == 8191 || p == 12289) {
      std::printf("sched %d g %lld |", p, (long long)g);
      for (int R : rad) std::printf(" %d", R);
      std::printf("\n");
    }
  }
  // both transform buffers of the longest lengths in one CTA (227 KiB opt-in shared memory)
  const long long smem32 = 2LL * rader_buf(kRaderMaxL32) * 8;
  const long long smem64 = 2LL * rader_buf(kRaderMaxL64) * 16;
  if (smem32 > 227 * 1024 || smem64 > 227 * 1024) {
    std::printf("buffers %lld / %lld bytes exceed a CTA's shared memory\n", smem32, smem64);
    return 1;
  }
  // thread counts for seeded sets of five smooth primes (xorshift64 draws), FP64 within its limit
  std::vector<int> smooth64;
  for (int p : smooth_primes)
    if (p - 1 <= kRaderMaxL64) smooth64.push_back(p);
  uint64_t state = 0x9E3779B97F4A7C15ULL;
  for (int trial = 0; trial < 200; ++trial) {
    std::vector<int32_t> set;
    std::vector<std::vector<int>> sched;
    int pmax = 0;
    const bool fp64 = trial & 1;
    for (int k = 0; k < 5; ++k) {
      state ^= state << 13;
      state ^= state >> 7;
      state ^= state << 17;
      const std::vector<int>& pool = fp64 ? smooth64 : smooth_primes;
      const int p = pool[state % pool.size()];
      set.push_back(p);
      sched.emplace_back();
      rader_schedule(p - 1, sched.back());
      if (p > pmax) pmax = p;
    }
    const int t = rader_threads(sched, set, pmax - 1, fp64);
    if (t < 32 || t > 512 || t % 32) {
      std::printf("trial %d: %d threads\n", trial, t);
      return 1;
    }
  }
  std::printf("primes %zu smooth %d maxpasses %d maxroot %lld\n", primes.size(), n_smooth,
              max_passes, (long long)max_root);
  std::printf("ok\n");
  return 0;
}
