// The host FFTs that make a plan's FP64 tables: the chirp filter's spectrum (lengths r 2^k,
// r = 1, 3, 5, 7) and Rader's V (lengths whose prime factors are small), with the exactly reduced
// turns e^{2 pi i num / den} they and the other tables are built from.
#pragma once

#include <math.h>
#include <stddef.h>
#include <stdint.h>

#include <complex>
#include <vector>

#include "sft_internal.h"

namespace sft {

using cd = std::complex<double>;
constexpr double kPi = 3.14159265358979323846;

// exp(2 pi i num / den), num reduced exactly modulo den first.
inline cd expi_turns(int64_t num, int64_t den) {
  int64_t r = ((num % den) + den) % den;
  double a = 2.0 * kPi * (double)r / (double)den, sn, cs;
  sincos(a, &sn, &cs);
  return cd(cs, sn);
}

// e^{-2 pi i j / n} for j = 0 .. n - 1, by expi_turns (which reduces its argument exactly, so
// entry (t k) mod n equals expi_turns(-t k, n)).
inline std::vector<cd> twiddle_table(int64_t n) {
  std::vector<cd> W(n);
  for (int64_t j = 0; j < n; ++j) W[j] = expi_turns(-j, n);
  return W;
}

// e^{-2 pi i k / M} for k < M/2 as interleaved (re, im): for M a multiple of 8 the first octant
// from sincos and the rest by the exact symmetries cos(pi/2 - t) = sin t, sin(pi/2 - t) = cos t
// and cos(pi/2 + t) = -sin t, sin(pi/2 + t) = cos t.
inline void half_turn_twiddles(size_t M, std::vector<double>& w) {
  w.assign(M, 0.0);
  if (M % 8 != 0) {
    for (size_t k = 0; k < M / 2; ++k) {
      double sn, cs;
      sincos(2.0 * kPi * (double)k / (double)M, &sn, &cs);
      w[2 * k] = cs;
      w[2 * k + 1] = -sn;
    }
    return;
  }
  const size_t e = M / 8, q = M / 4;
  std::vector<double> co(e + 1), si(e + 1);
  for (size_t k = 0; k <= e; ++k) sincos(2.0 * kPi * (double)k / (double)M, &si[k], &co[k]);
  auto cos_sin = [&](size_t k, double& c, double& sv) {      // k <= M/4
    if (k <= e) { c = co[k]; sv = si[k]; }
    else { c = si[q - k]; sv = co[q - k]; }
  };
  for (size_t k = 0; k < M / 2; ++k) {
    double c, sv;
    if (k <= q) {
      cos_sin(k, c, sv);
    } else {
      double c2, s2;
      cos_sin(k - q, c2, s2);
      c = -s2;
      sv = c2;
    }
    w[2 * k] = c;
    w[2 * k + 1] = -sv;
  }
}

// In-place iterative FFT (forward, exp(-2 pi i n k / M)), M a power of two: bit reversal, one
// radix-2 stage when log2 M is odd, then the radix-2 stages in pairs (one pass over the data per
// pair, four points per butterfly group), in plain double arithmetic on the interleaved array.
inline void host_fft_pow2(std::vector<cd>& va) {
  const size_t M = va.size();
  for (size_t i = 1, j = 0; i < M; ++i) {
    size_t bit = M >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(va[i], va[j]);
  }
  if (M < 2) return;
  std::vector<double> w;
  half_turn_twiddles(M, w);
  double* a = reinterpret_cast<double*>(va.data());
  size_t len = 2;
  size_t lg = 0;
  while ((size_t(1) << lg) < M) ++lg;
  if (lg & 1) {
    for (size_t i = 0; i < M; i += 2) {
      double* u = a + 2 * i;
      double* v = u + 2;
      const double vr = v[0], vi = v[1];
      v[0] = u[0] - vr;
      v[1] = u[1] - vi;
      u[0] += vr;
      u[1] += vi;
    }
    len = 4;
  }
  // the stages of sub-transform lengths len and 2 len together: points x0..x3 at k, k + len/2,
  // k + len, k + 3 len/2; twiddle w^k of length len, then w^k and w^{k + len/2} of length 2 len
  for (; len <= M / 2; len <<= 2) {
    const size_t h = len / 2, s1 = M / len, s2 = M / (2 * len);
    for (size_t k = 0; k < h; ++k) {
      const double w1r = w[2 * k * s1], w1i = w[2 * k * s1 + 1];
      const double w2r = w[2 * k * s2], w2i = w[2 * k * s2 + 1];
      const double w3r = w[2 * (k + h) * s2], w3i = w[2 * (k + h) * s2 + 1];
      for (size_t i = k; i < M; i += 2 * len) {
        double* x0 = a + 2 * i;
        double* x1 = a + 2 * (i + h);
        double* x2 = a + 2 * (i + len);
        double* x3 = a + 2 * (i + len + h);
        const double t1r = x1[0] * w1r - x1[1] * w1i, t1i = x1[0] * w1i + x1[1] * w1r;
        const double t3r = x3[0] * w1r - x3[1] * w1i, t3i = x3[0] * w1i + x3[1] * w1r;
        const double y0r = x0[0] + t1r, y0i = x0[1] + t1i, y1r = x0[0] - t1r, y1i = x0[1] - t1i;
        const double y2r = x2[0] + t3r, y2i = x2[1] + t3i, y3r = x2[0] - t3r, y3i = x2[1] - t3i;
        const double u2r = y2r * w2r - y2i * w2i, u2i = y2r * w2i + y2i * w2r;
        const double u3r = y3r * w3r - y3i * w3i, u3i = y3r * w3i + y3i * w3r;
        x0[0] = y0r + u2r;
        x0[1] = y0i + u2i;
        x2[0] = y0r - u2r;
        x2[1] = y0i - u2i;
        x1[0] = y1r + u3r;
        x1[1] = y1i + u3i;
        x3[0] = y1r - u3r;
        x3[1] = y1i - u3i;
      }
    }
  }
}

// Forward FFT of length M = r 2^k (r = 1, 3, 5, 7), used once per plan to transform the chirp
// filter.  For r > 1, one decimation in time: with A_t the length-M' (M' = M / r) transforms of
// a[r n + t], X[k + M' u] = sum_t e^{-2 pi i t (k + M' u) / M} A_t[k], u = 0..r-1.
inline void host_fft(std::vector<cd>& a) {
  const size_t M = a.size();
  const int r = fft_odd((int)M);
  if (r == 1) { host_fft_pow2(a); return; }
  const size_t Mp = M / r;
  std::vector<std::vector<cd>> A(r, std::vector<cd>(Mp));
  for (int t = 0; t < r; ++t) {
    for (size_t n = 0; n < Mp; ++n) A[t][n] = a[r * n + t];
    host_fft_pow2(A[t]);
  }
  const std::vector<cd> W = twiddle_table((int64_t)M);
  for (size_t k = 0; k < Mp; ++k)
    for (int u = 0; u < r; ++u) {
      const int64_t kk = (int64_t)(k + Mp * u);
      cd x = A[0][k];
      for (int t = 1; t < r; ++t) x += W[((int64_t)t * kk) % (int64_t)M] * A[t][k];
      a[kk] = x;
    }
}

// Forward DFT of any length whose prime factors are small, by recursive decimation in time on
// the smallest prime factor r: with A_t the transforms of a[r n + t] (length m = L / r),
// X[k + m u] = sum_t e^{-2 pi i t (k + m u) / L} A_t[k].  Twiddles come from one table of the
// top-level length L0 (exact reductions): e^{-2 pi i j / L} is entry j (L0 / L).
inline void host_fft_mixed_with(std::vector<cd>& a, const std::vector<cd>& W, int64_t stride) {
  const int64_t L = (int64_t)a.size();
  if (L <= 1) return;
  int64_t r = 2;
  while (L % r) ++r;
  const int64_t m = L / r;
  std::vector<std::vector<cd>> A(r, std::vector<cd>(m));
  for (int64_t t = 0; t < r; ++t) {
    for (int64_t n = 0; n < m; ++n) A[t][n] = a[r * n + t];
    host_fft_mixed_with(A[t], W, stride * r);
  }
  for (int64_t k = 0; k < m; ++k)
    for (int64_t u = 0; u < r; ++u) {
      const int64_t kk = k + m * u;
      cd x = A[0][k];
      for (int64_t t = 1; t < r; ++t) x += W[((t * kk) % L) * stride] * A[t][k];
      a[kk] = x;
    }
}

inline void host_fft_mixed(std::vector<cd>& a) {
  if (a.size() <= 1) return;
  const std::vector<cd> W = twiddle_table((int64_t)a.size());
  host_fft_mixed_with(a, W, 1);
}

}  // namespace sft
