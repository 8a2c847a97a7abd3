/* The C ABI used from plain C (no Python, no torch): an exactly 4-sparse spectrum at N = 2^20,
 * synthesised on the host from its definition f[j] = sum_k c_k (-1)^{w_k} e^{2 pi i w_k j / N}
 * (the inverse of f_hat = F f), copied to the device, transformed, and read back.  Prints
 * "C-ABI OK" when the frequencies come back exactly and every coefficient within 1e-5. */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime.h>

#include "sft.h"

#define S 4
static const double kPi = 3.14159265358979323846;

static int fail(const char* what) {
  fprintf(stderr, "%s: %s\n", what, sft_last_error());
  return 1;
}

int main(void) {
  const int64_t N = (int64_t)1 << 20;
  const int64_t w[S] = {-77777, 5, 123456, 400000};
  const double cre[S] = {1.0, 0.5, -0.75, 0.25}, cim[S] = {0.5, -1.0, 0.0, 0.8};
  float* f = (float*)malloc((size_t)N * 2 * sizeof(float));
  if (!f) return 1;
  for (int64_t j = 0; j < N; ++j) {
    double re = 0.0, im = 0.0;
    for (int k = 0; k < S; ++k) {
      const int64_t wk = ((w[k] % N) + N) % N;
      const double a = 2.0 * kPi * (double)((wk * j) % N) / (double)N;
      const double sg = (w[k] % 2 == 0) ? 1.0 : -1.0;
      re += sg * (cre[k] * cos(a) - cim[k] * sin(a));
      im += sg * (cre[k] * sin(a) + cim[k] * cos(a));
    }
    f[2 * j] = (float)re;
    f[2 * j + 1] = (float)im;
  }
  void *f_dev = NULL, *c_dev = NULL;
  int64_t* w_dev = NULL;
  int32_t* n_dev = NULL;
  if (cudaMalloc(&f_dev, (size_t)N * 8) != cudaSuccess || cudaMalloc((void**)&w_dev, S * 8) != cudaSuccess ||
      cudaMalloc(&c_dev, S * 16) != cudaSuccess || cudaMalloc((void**)&n_dev, 4) != cudaSuccess) {
    fprintf(stderr, "cudaMalloc failed\n");
    return 1;
  }
  cudaMemcpy(f_dev, f, (size_t)N * 8, cudaMemcpyHostToDevice);
  sft_variant v;
  if (sft_variant_init(&v) != SFT_OK) return fail("sft_variant_init");
  v.c_p = 4.0;
  v.seed = 11;
  sft_plan_t plan = NULL;
  if (sft_plan(&plan, N, S, &v, 0, NULL, 0, NULL, 0) != SFT_OK) return fail("sft_plan");
  if (sft_execute(plan, f_dev, w_dev, c_dev, n_dev, NULL) != SFT_OK) return fail("sft_execute");
  if (cudaDeviceSynchronize() != cudaSuccess) {
    fprintf(stderr, "device error\n");
    return 1;
  }
  int64_t wo[S];
  double co[2 * S];
  int32_t n = 0;
  cudaMemcpy(wo, w_dev, sizeof(wo), cudaMemcpyDeviceToHost);
  cudaMemcpy(co, c_dev, sizeof(co), cudaMemcpyDeviceToHost);
  cudaMemcpy(&n, n_dev, 4, cudaMemcpyDeviceToHost);
  if (n != S) {
    fprintf(stderr, "count %d\n", n);
    return 1;
  }
  for (int r = 0; r < S; ++r) {
    int k = 0;
    while (k < S && w[k] != wo[r]) ++k;
    if (k == S) {
      fprintf(stderr, "unexpected frequency %lld\n", (long long)wo[r]);
      return 1;
    }
    const double er = co[2 * r] - cre[k], ei = co[2 * r + 1] - cim[k];
    const double mag = sqrt(cre[k] * cre[k] + cim[k] * cim[k]);
    if (sqrt(er * er + ei * ei) > 1e-5 * mag) {
      fprintf(stderr, "coefficient of %lld off by %g\n", (long long)wo[r], sqrt(er * er + ei * ei));
      return 1;
    }
  }
  sft_plan_destroy(plan);
  cudaFree(f_dev);
  cudaFree(w_dev);
  cudaFree(c_dev);
  cudaFree(n_dev);
  free(f);
  printf("C-ABI OK\n");
  return 0;
}
