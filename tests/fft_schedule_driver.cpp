// Host-compiled check of the chirp-convolution FFT schedule declared in csrc/sft_internal.h (the
// same constexpr functions the kernels instantiate).  Prints one line per admissible length:
//   M tpt radices... | rows entries
// and exits non-zero on the first broken invariant.
#include <cstdio>
#include <vector>

#include "../paper_1706_02740_gb300/csrc/sft_internal.h"

using namespace sft;

int main() {
  std::vector<int> lengths;
  for (int base : {64, 96, 640, 896})
    for (int m = base; m <= kMaxFFT32; m <<= 1) lengths.push_back(m);
  for (int M : lengths) {
    const int tpt = fft_tpt(M);
    if (M % 2 || (M / 2) % tpt) { std::printf("radix-2 pass of %d uneven over %d threads\n", M, tpt); return 1; }
    std::printf("%d %d", M, tpt);
    int span = 2, passes = 0;
    while (span < M) {
      const int R = fft_radix(M, span);
      if (R < 2 || R > 16 || M % (span * R)) { std::printf(" bad radix %d at span %d\n", R, span); return 1; }
      const int items = M / R;
      const int per_thread = (items + tpt - 1) / tpt;
      if (per_thread * R > 16) { std::printf(" %d values per thread at span %d\n", per_thread * R, span); return 1; }
      if (fft_tw_rows(R) < 1 || fft_tw_rows(R) > 6) { std::printf(" rows\n"); return 1; }
      std::printf(" %d", R);
      span *= R;
      ++passes;
    }
    if (span != M) { std::printf(" schedule ends at %d\n", span); return 1; }
    if (fft_tw_entries(M) >= M) { std::printf(" table %d >= %d\n", fft_tw_entries(M), M); return 1; }
    std::printf(" | %d\n", fft_tw_entries(M));
  }
  // the length chosen for 2p - 1 is admissible, >= 2p - 1 and the smallest such
  for (int p = 5; p <= 8192; ++p) {
    const int M = fft_length(2 * p - 1, kMaxFFT32);
    if (M < 2 * p - 1) { std::printf("length %d < 2p - 1 for p = %d\n", M, p); return 1; }
    for (int L : lengths)
      if (L >= 2 * p - 1 && L < M) { std::printf("length %d not minimal for p = %d\n", M, p); return 1; }
  }
  std::printf("ok\n");
  return 0;
}
