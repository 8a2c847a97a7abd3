// In-register DFTs of the small radices of the shared-memory FFTs (the chirp convolution's and
// Rader's), natural order in and out, and the padded shared-memory index map.
#pragma once

#include "cplx.cuh"

namespace sft {

namespace {

__device__ __forceinline__ int pad16(int n) { return n + (n >> 4); }
template <int M> constexpr int padded_len() { return M + M / 16; }

// Constants of the radix-8 and radix-16 butterflies: cos(pi/8), sin(pi/8), sqrt(1/2).
constexpr double kC8 = 0.92387953251128674;
constexpr double kS8 = 0.38268343236508977;
constexpr double kH = 0.70710678118654752;
// sqrt(3)/2, the sine of the radix-3 butterfly.
constexpr double kS3 = 0.86602540378443865;
// cos(2 pi m / T) and sin(2 pi m / T), m = 1..(T-1)/2, of the odd prime butterflies T = 5, 7, 11,
// 13 (the exact values rounded to double).
__host__ __device__ constexpr double odd_cos(int T, int m) {
  return T == 5 ? (m == 1 ? 0.30901699437494742 : -0.80901699437494742)
       : T == 7 ? (m == 1 ? 0.62348980185873353 : m == 2 ? -0.22252093395631440 : -0.90096886790241913)
       : T == 11 ? (m == 1 ? 0.84125353283118117 : m == 2 ? 0.41541501300188643
                    : m == 3 ? -0.14231483827328514 : m == 4 ? -0.65486073394528506
                    : -0.95949297361449739)
       : (m == 1 ? 0.88545602565320990 : m == 2 ? 0.56806474673115580
          : m == 3 ? 0.12053668025532305 : m == 4 ? -0.35460488704253563
          : m == 5 ? -0.74851074817110110 : -0.97094181742605203);
}
__host__ __device__ constexpr double odd_sin(int T, int m) {
  return T == 5 ? (m == 1 ? 0.95105651629515357 : 0.58778525229247313)
       : T == 7 ? (m == 1 ? 0.78183148246802981 : m == 2 ? 0.97492791218182361 : 0.43388373911755812)
       : T == 11 ? (m == 1 ? 0.54064081745559758 : m == 2 ? 0.90963199535451837
                    : m == 3 ? 0.98982144188093273 : m == 4 ? 0.75574957435425828
                    : 0.28173255684142970)
       : (m == 1 ? 0.46472317204376855 : m == 2 ? 0.82298386589365639
          : m == 3 ? 0.99270887409805399 : m == 4 ? 0.93501624268541482
          : m == 5 ? 0.66312265824079520 : 0.23931566428755777);
}

__device__ __forceinline__ float r_fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double r_fma(double a, double b, double c) { return fma(a, b, c); }

// a (c - i s) for constants c, s
template <typename C, typename R>
__device__ __forceinline__ C mul_cs(C a, R c, R s) {
  return C{r_fma(a.x, c, a.y * s), r_fma(a.y, c, -a.x * s)};
}
// a e^{-i pi / 4} = a (1 - i) / sqrt 2
template <typename C> __device__ __forceinline__ C mul_w8_1(C a) {
  using R = decltype(a.x);
  return C{(a.x + a.y) * (R)kH, (a.y - a.x) * (R)kH};
}
// a e^{-3 i pi / 4} = a (-1 - i) / sqrt 2
template <typename C> __device__ __forceinline__ C mul_w8_3(C a) {
  using R = decltype(a.x);
  return C{(a.y - a.x) * (R)kH, -(a.x + a.y) * (R)kH};
}

// In-register forward DFT of length R, natural order in and out.  The multiplications by 1 and
// -i are written out, so only the nontrivial twiddles cost multiplications.
template <int R, typename C> struct DFT;
template <typename C> struct DFT<2, C> {
  __device__ static __forceinline__ void run(C* a) {
    C t = a[0];
    a[0] = cadd(t, a[1]);
    a[1] = csub(t, a[1]);
  }
};
template <typename C> struct DFT<4, C> {
  __device__ static __forceinline__ void run(C* a) {
    C t0 = cadd(a[0], a[2]), t1 = csub(a[0], a[2]);
    C t2 = cadd(a[1], a[3]), t3 = cmul_mi(csub(a[1], a[3]));
    a[0] = cadd(t0, t2);
    a[2] = csub(t0, t2);
    a[1] = cadd(t1, t3);
    a[3] = csub(t1, t3);
  }
};
// 8 = 2 x 4: X[k] = E[k] + w8^k O[k], X[k + 4] = E[k] - w8^k O[k].
template <typename C> struct DFT<8, C> {
  __device__ static __forceinline__ void run(C* a) {
    C e[4] = {a[0], a[2], a[4], a[6]}, o[4] = {a[1], a[3], a[5], a[7]};
    DFT<4, C>::run(e);
    DFT<4, C>::run(o);
    o[1] = mul_w8_1(o[1]);
    o[2] = cmul_mi(o[2]);
    o[3] = mul_w8_3(o[3]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      a[k] = cadd(e[k], o[k]);
      a[k + 4] = csub(e[k], o[k]);
    }
  }
};
// X0 = a0 + a1 + a2, X1,2 = a0 - (a1 + a2)/2 -/+ i (sqrt 3 / 2)(a1 - a2).
template <typename C> struct DFT<3, C> {
  __device__ static __forceinline__ void run(C* a) {
    using R = decltype(a[0].x);
    const C t = cadd(a[1], a[2]), d = csub(a[1], a[2]);
    const C m = C{r_fma(t.x, (R)-0.5, a[0].x), r_fma(t.y, (R)-0.5, a[0].y)};
    a[0] = cadd(a[0], t);
    a[1] = C{r_fma(d.y, (R)kS3, m.x), r_fma(d.x, -(R)kS3, m.y)};
    a[2] = C{r_fma(d.y, -(R)kS3, m.x), r_fma(d.x, (R)kS3, m.y)};
  }
};
// Odd prime T = 5, 7, 11, 13 with the terms k and T - k paired: A_k = a_k + a_{T-k}, B_k = a_k - a_{T-k},
//     X_r = a_0 + sum_k (cos(2 pi k r / T) A_k - i sin(2 pi k r / T) B_k),
//     X_{T-r} = a_0 + sum_k (cos(2 pi k r / T) A_k + i sin(2 pi k r / T) B_k),   k, r = 1..(T-1)/2.
template <int T, typename C>
__device__ __forceinline__ void dft_odd_prime(C* a) {
  using R = decltype(a[0].x);
  constexpr int H = (T - 1) / 2;
  C A[H + 1], B[H + 1];
  C X0 = a[0];
#pragma unroll
  for (int k = 1; k <= H; ++k) {
    A[k] = cadd(a[k], a[T - k]);
    B[k] = csub(a[k], a[T - k]);
    X0 = cadd(X0, A[k]);
  }
  C out[T];
  out[0] = X0;
#pragma unroll
  for (int r = 1; r <= H; ++r) {
    C P = a[0], Q = C{(R)0, (R)0};
#pragma unroll
    for (int k = 1; k <= H; ++k) {
      const int m = (k * r) % T;
      const R c = (R)(m <= H ? odd_cos(T, m) : odd_cos(T, T - m));
      const R sn = (R)(m <= H ? odd_sin(T, m) : -odd_sin(T, T - m));
      P.x = r_fma(A[k].x, c, P.x);
      P.y = r_fma(A[k].y, c, P.y);
      Q.x = r_fma(B[k].x, sn, Q.x);
      Q.y = r_fma(B[k].y, sn, Q.y);
    }
    out[r] = C{P.x + Q.y, P.y - Q.x};          // P - i Q
    out[T - r] = C{P.x - Q.y, P.y + Q.x};      // P + i Q
  }
#pragma unroll
  for (int r = 0; r < T; ++r) a[r] = out[r];
}
template <typename C> struct DFT<5, C> {
  __device__ static __forceinline__ void run(C* a) { dft_odd_prime<5>(a); }
};
template <typename C> struct DFT<7, C> {
  __device__ static __forceinline__ void run(C* a) { dft_odd_prime<7>(a); }
};
template <typename C> struct DFT<11, C> {
  __device__ static __forceinline__ void run(C* a) { dft_odd_prime<11>(a); }
};
template <typename C> struct DFT<13, C> {
  __device__ static __forceinline__ void run(C* a) { dft_odd_prime<13>(a); }
};
// Prime-factor (Good-Thomas) forms, no twiddles: for R = R1 R2 with gcd(R1, R2) = 1, input
// n = (R2 n1 + R1 n2) mod R and output k = (k1 R2 (R2^-1 mod R1) + k2 R1 (R1^-1 mod R2)) mod R
// turn the length-R DFT into length-R1 DFTs over n1 and length-R2 DFTs over n2.
// 6 = 2 x 3: n = (3 n1 + 2 n2) mod 6, k = (3 k1 + 4 k2) mod 6.
template <typename C> struct DFT<6, C> {
  __device__ static __forceinline__ void run(C* a) {
    C u[3] = {a[0], a[2], a[4]}, v[3] = {a[3], a[5], a[1]};
    DFT<3, C>::run(u);
    DFT<3, C>::run(v);
    // k = (3 k1 + 4 k2) mod 6 for k1 = 0, 1 and k2 = 0, 1, 2
    a[0] = cadd(u[0], v[0]); a[3] = csub(u[0], v[0]);
    a[4] = cadd(u[1], v[1]); a[1] = csub(u[1], v[1]);
    a[2] = cadd(u[2], v[2]); a[5] = csub(u[2], v[2]);
  }
};
// 2T = 2 x T (T = 5, 7): n = (T n1 + 2 n2) mod 2T, k = (T k1 + 2 (2^-1 mod T) k2) mod 2T.
template <int T, typename C>
__device__ __forceinline__ void dft_two_odd(C* a) {
  constexpr int N = 2 * T, I2 = (T + 1) / 2;     // 2^-1 mod T
  C u[T], v[T];
#pragma unroll
  for (int n2 = 0; n2 < T; ++n2) {
    u[n2] = a[(2 * n2) % N];
    v[n2] = a[(T + 2 * n2) % N];
  }
  DFT<T, C>::run(u);
  DFT<T, C>::run(v);
#pragma unroll
  for (int k2 = 0; k2 < T; ++k2) {
    a[(2 * I2 * k2) % N] = cadd(u[k2], v[k2]);
    a[(T + 2 * I2 * k2) % N] = csub(u[k2], v[k2]);
  }
}
template <typename C> struct DFT<10, C> {
  __device__ static __forceinline__ void run(C* a) { dft_two_odd<5>(a); }
};
template <typename C> struct DFT<14, C> {
  __device__ static __forceinline__ void run(C* a) { dft_two_odd<7>(a); }
};
// 12 = 3 x 4: n = (4 n1 + 3 n2) mod 12, k = (4 k1 + 9 k2) mod 12.
template <typename C> struct DFT<12, C> {
  __device__ static __forceinline__ void run(C* a) {
    C y[3][4];
#pragma unroll
    for (int n1 = 0; n1 < 3; ++n1) {
      C t[4];
#pragma unroll
      for (int n2 = 0; n2 < 4; ++n2) t[n2] = a[(4 * n1 + 3 * n2) % 12];
      DFT<4, C>::run(t);
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) y[n1][k2] = t[k2];
    }
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) {
      C t[3] = {y[0][k2], y[1][k2], y[2][k2]};
      DFT<3, C>::run(t);
#pragma unroll
      for (int k1 = 0; k1 < 3; ++k1) a[(4 * k1 + 9 * k2) % 12] = t[k1];
    }
  }
};
// 16 = 4 x 4 with n = n1 + 4 n2, k = k2 + 4 k1: length-4 DFTs over n2, twiddles w16^{n1 k2},
// length-4 DFTs over n1.
template <typename C> struct DFT<16, C> {
  __device__ static __forceinline__ void run(C* a) {
    using R = decltype(a[0].x);
    C y[4][4];
#pragma unroll
    for (int n1 = 0; n1 < 4; ++n1) {
      C t[4] = {a[n1], a[n1 + 4], a[n1 + 8], a[n1 + 12]};
      DFT<4, C>::run(t);
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) y[n1][k2] = t[k2];
    }
    y[1][1] = mul_cs(y[1][1], (R)kC8, (R)kS8);     // w16^1
    y[1][2] = mul_w8_1(y[1][2]);                  // w16^2
    y[1][3] = mul_cs(y[1][3], (R)kS8, (R)kC8);     // w16^3
    y[2][1] = mul_w8_1(y[2][1]);                  // w16^2
    y[2][2] = cmul_mi(y[2][2]);                   // w16^4
    y[2][3] = mul_w8_3(y[2][3]);                  // w16^6
    y[3][1] = mul_cs(y[3][1], (R)kS8, (R)kC8);     // w16^3
    y[3][2] = mul_w8_3(y[3][2]);                  // w16^6
    y[3][3] = mul_cs(y[3][3], (R)-kC8, (R)-kS8);   // w16^9
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) {
      C t[4] = {y[0][k2], y[1][k2], y[2][k2], y[3][k2]};
      DFT<4, C>::run(t);
#pragma unroll
      for (int k1 = 0; k1 < 4; ++k1) a[k2 + 4 * k1] = t[k1];
    }
  }
};


}  // namespace

}  // namespace sft
