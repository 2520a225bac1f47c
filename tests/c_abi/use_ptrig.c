/* A plain C99 client of libptrig: allocates device buffers with the CUDA
 * runtime, evaluates sin, cos, tan and sincos through the C ABI, and checks
 * the results on the host against sin^2 + cos^2 = 1, tan = sin / cos and a
 * few exact values of the method (sin 0 = 0, cos 0 = 1, sin(pi/4) = cos(pi/4)).
 * Prints "ok" and exits 0 on success. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime_api.h>

#include "ptrig.h"

#define N 100003

static int check(ptrig_status s, const char *what) {
  if (s != PTRIG_OK) {
    fprintf(stderr, "%s: %s\n", what, ptrig_status_string(s));
    return 1;
  }
  return 0;
}

int main(void) {
  float *hx = malloc(N * sizeof(float)), *hs = malloc(N * sizeof(float));
  float *hc = malloc(N * sizeof(float)), *ht = malloc(N * sizeof(float));
  float *hs2 = malloc(N * sizeof(float)), *hc2 = malloc(N * sizeof(float));
  float *dx, *ds, *dc, *dt, *ds2, *dc2;
  int i, bad = 0;
  if (!hx || !hs || !hc || !ht || !hs2 || !hc2) return 2;
  for (i = 0; i < N; ++i) hx[i] = (float)(-300.0 + 600.0 * (double)i / (N - 1));
  hx[0] = 0.0f;
  hx[1] = 0.78539816f; /* pi/4 rounded to float */
  if (cudaMalloc((void **)&dx, N * sizeof(float)) || cudaMalloc((void **)&ds, N * sizeof(float)) ||
      cudaMalloc((void **)&dc, N * sizeof(float)) || cudaMalloc((void **)&dt, N * sizeof(float)) ||
      cudaMalloc((void **)&ds2, N * sizeof(float)) || cudaMalloc((void **)&dc2, N * sizeof(float)))
    return 3;
  if (cudaMemcpy(dx, hx, N * sizeof(float), cudaMemcpyHostToDevice)) return 3;
  bad |= check(ptrig_sin_f32(dx, ds, N, NULL), "ptrig_sin_f32");
  bad |= check(ptrig_cos_f32(dx, dc, N, NULL), "ptrig_cos_f32");
  bad |= check(ptrig_tan_f32(dx, dt, N, NULL), "ptrig_tan_f32");
  bad |= check(ptrig_sincos_f32(dx, ds2, dc2, N, NULL), "ptrig_sincos_f32");
  bad |= check(ptrig_sin_f32(NULL, ds, 4, NULL) == PTRIG_ERR_INVALID_ARG ? PTRIG_OK : PTRIG_ERR_CUDA,
               "NULL input must be rejected");
  if (cudaDeviceSynchronize()) return 4;
  cudaMemcpy(hs, ds, N * sizeof(float), cudaMemcpyDeviceToHost);
  cudaMemcpy(hc, dc, N * sizeof(float), cudaMemcpyDeviceToHost);
  cudaMemcpy(ht, dt, N * sizeof(float), cudaMemcpyDeviceToHost);
  cudaMemcpy(hs2, ds2, N * sizeof(float), cudaMemcpyDeviceToHost);
  cudaMemcpy(hc2, dc2, N * sizeof(float), cudaMemcpyDeviceToHost);
  for (i = 0; i < N; ++i) {
    const double s = hs[i], c = hc[i], t = ht[i];
    if (fabs(s * s + c * c - 1.0) > 1e-6) bad = 1;
    if (fabs(c) > 1e-2 && fabs(t - s / c) > 1e-5 * fabs(t) + 1e-6) bad = 1;
    if (hs2[i] != hs[i] || hc2[i] != hc[i]) bad = 1;
  }
  if (hs[0] != 0.0f || hc[0] != 1.0f || fabs((double)hs[1] - (double)hc[1]) > 1e-6) bad = 1;
  cudaFree(dx);
  cudaFree(ds);
  cudaFree(dc);
  cudaFree(dt);
  cudaFree(ds2);
  cudaFree(dc2);
  printf(bad ? "mismatch (version %d)\n" : "ok (version %d)\n", ptrig_version());
  return bad;
}
