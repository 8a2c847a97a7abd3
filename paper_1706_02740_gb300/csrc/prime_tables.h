// The constant tables of one prime p for the measurements' DFTs of length p, computed once on the
// host in FP64 with exactly reduced turns: the chirp form's chirp and filter spectrum at
// convolution length M, or Rader's form's permutations, V and twiddle rows.
#pragma once

#include <stdint.h>

#include <complex>
#include <memory>
#include <vector>

#include "host_fft.h"
#include "rader_plan.h"
#include "sft_internal.h"

namespace sft {

// Per-prime constant tables (FP64).  The re-estimation twiddles e^{-2 pi i n / p}; in
// the chirp form the chirp e^{-pi i n^2 / p} and FFT_M of its wrapped conjugate / (M p); in
// Rader's form the permutations g^n, g^{-n}, V = FFT(b) / (p (p - 1)) and the pass schedule with
// its twiddle rows.
struct PrimeTables {
  std::vector<cd> wp;
  std::vector<cd> chirp, vhat;
  std::vector<int32_t> pin, pout;
  std::vector<cd> rv, rt;
  std::vector<int> sched;
  std::vector<int32_t> toff;
};

inline std::shared_ptr<const PrimeTables> compute_prime_tables(int64_t p, int M, bool rader) {
  auto T = std::make_shared<PrimeTables>();
  T->wp.resize(p);
  for (int64_t n = 0; n < p; ++n) T->wp[n] = expi_turns(-n, p);
  if (!rader) {
    T->chirp.resize(p);
    std::vector<cd> V(M, cd(0, 0));
    for (int64_t n = 0; n < p; ++n) {
      const cd w = expi_turns(-((n * n) % (2 * p)), 2 * p);  // exp(-pi i n^2 / p)
      T->chirp[n] = w;
      V[n] = std::conj(w);
      if (n > 0) V[M - n] = std::conj(w);
    }
    host_fft(V);
    T->vhat.resize(M);
    for (int n = 0; n < M; ++n) T->vhat[n] = V[n] / ((double)M * (double)p);
    return T;
  }
  // Rader's form: L = p - 1, g a primitive root; a_n = h_{g^n}, b_n = e^{-2 pi i g^{-n} / p} and
  // E_{g^{-m}} = h_0 / p + (a (*) b)[m] / p (cyclic convolution), E_0 = (h_0 + sum_n a_n) / p.
  const int64_t L = p - 1;
  rader_schedule((int)L, T->sched);
  const int64_t g = primitive_root(p), ginv = pow_mod(g, p - 2, p);
  T->pin.resize(L);
  T->pout.resize(L);
  std::vector<cd> b(L);
  int64_t x = 1, y = 1;
  for (int64_t n = 0; n < L; ++n) {
    T->pin[n] = (int32_t)x;                 // g^n mod p
    T->pout[n] = (int32_t)y;                // g^{-n} mod p
    b[n] = expi_turns(-y, p);
    x = x * g % p;
    y = y * ginv % p;
  }
  host_fft_mixed(b);
  T->rv.resize(L);
  for (int64_t k = 0; k < L; ++k) T->rv[k] = b[k] / ((double)p * (double)L);
  T->rt.assign(L, cd(1, 0));
  int64_t span = 1, off = 0;
  for (int R : T->sched) {
    T->toff.push_back((int32_t)off);
    for (int row = 0; row < fft_tw_rows(R); ++row)
      for (int64_t k = 0; k < span; ++k)
        T->rt[off + (size_t)row * span + k] = expi_turns(-(int64_t)fft_tw_exp(row) * k, span * R);
    off += (int64_t)fft_tw_rows(R) * span;
    span *= R;
  }
  return T;
}

}  // namespace sft
