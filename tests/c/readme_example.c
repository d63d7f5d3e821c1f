/* The README's C usage example as a complete program: build a seeded series on
 * the host, copy it to the device, run the whole method through vl_fit, read
 * the order and B0 back and print them.  tests/test_c_example.py builds this
 * file against include/varlingam_gb300.h and the shared library, runs it and
 * compares its output with the Python binding on the same series.
 *
 *   readme_example M N SEED PREC     (PREC: 0 = FP64 path, 1 = mixed)
 */
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "varlingam_gb300.h"

/* 64-bit linear congruential generator (Knuth's MMIX constants); the test
 * regenerates the same numbers in Python. */
static uint64_t lcg_state;
static double lcg_uniform(void) {
  lcg_state = lcg_state * 6364136223846793005ULL + 1442695040888963407ULL;
  return (double)(lcg_state >> 11) * (1.0 / 9007199254740992.0);
}

int main(int argc, char** argv) {
  if (argc != 5) {
    fprintf(stderr, "usage: %s M N SEED PREC\n", argv[0]);
    return 2;
  }
  const int m = atoi(argv[1]), n = atoi(argv[2]), p = 1;
  lcg_state = strtoull(argv[3], NULL, 10);
  const vl_precision prec = atoi(argv[4]) ? VL_PREC_MIXED : VL_PREC_FP64;
  /* x_t = 0.3 x_{t-1} + e_t with uniform shocks on [-1, 1], e_t(i) feeding
   * variable i + 1 as well (a chain of instantaneous effects) */
  double* X = (double*)malloc(sizeof(double) * m * n);
  for (int t = 0; t < n; ++t) {
    double carry = 0.0;
    for (int i = 0; i < m; ++i) {
      const double e = 2.0 * lcg_uniform() - 1.0;
      const double prev = t ? X[(size_t)i * n + t - 1] : 0.0;
      X[(size_t)i * n + t] = 0.3 * prev + e + 0.5 * carry;
      carry = e;
    }
  }
  double *dX, *dM, *dB0, *dBtau;
  int32_t* dOrder;
  cudaMalloc((void**)&dX, sizeof(double) * m * n);
  cudaMalloc((void**)&dM, sizeof(double) * p * m * m);
  cudaMalloc((void**)&dB0, sizeof(double) * m * m);
  cudaMalloc((void**)&dBtau, sizeof(double) * p * m * m);
  cudaMalloc((void**)&dOrder, sizeof(int32_t) * m);
  cudaMemcpy(dX, X, sizeof(double) * m * n, cudaMemcpyHostToDevice);

  /* --- the README example --- */
  vl_handle h;
  if (vl_create(&h, /*device=*/0, /*cuda_stream=*/NULL, /*workspace_bytes=*/0) != VL_OK) {
    fprintf(stderr, "vl_create failed\n");
    return 1;
  }
  vl_fit(h, dX, /*ldx=*/n, m, n, p, prec, dM, dOrder, dB0, dBtau, /*D=*/NULL);
  if (vl_sync(h) != VL_OK) {
    fprintf(stderr, "%s\n", vl_last_error(h));
    return 1;
  }
  vl_destroy(h);
  /* --- end of the example --- */

  int32_t* order = (int32_t*)malloc(sizeof(int32_t) * m);
  double* B0 = (double*)malloc(sizeof(double) * m * m);
  cudaMemcpy(order, dOrder, sizeof(int32_t) * m, cudaMemcpyDeviceToHost);
  cudaMemcpy(B0, dB0, sizeof(double) * m * m, cudaMemcpyDeviceToHost);
  printf("order");
  for (int i = 0; i < m; ++i) printf(" %d", order[i]);
  printf("\nB0");
  for (int i = 0; i < m * m; ++i) printf(" %.17g", B0[i]);
  printf("\n");
  cudaFree(dX);
  cudaFree(dM);
  cudaFree(dB0);
  cudaFree(dBtau);
  cudaFree(dOrder);
  free(X);
  free(order);
  free(B0);
  return 0;
}
