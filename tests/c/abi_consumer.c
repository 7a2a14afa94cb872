/* A plain C consumer of the library (no Python, no PyTorch): builds a plan for
 * a 6 x 16 detector, 41 wire steps of 1 um and 101 bins of 1 um, reconstructs
 * a deterministic image stack on the GPU through dr_reconstruct, and checks a
 * property the method fixes: where a pixel's swept depths lie inside the
 * bins, its bins add up to I_first - I_last (the differences telescope).
 * Prints "abi consumer ok" and exits 0 on success. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime.h>

#include "dr.h"

#define H 6
#define W 16
#define K 41
#define B 101

static int fail(const char *what, int st) {
  fprintf(stderr, "%s: status %d (%s): %s\n", what, st, dr_status_string((dr_status)st),
          dr_last_error());
  return 1;
}

int main(void) {
  dr_geometry g = {{0, 0, 0}, {0, 0, 1}, {-1.5, 510.0, -0.5}, {0, 0, 0.2}, {0.2, 0, 0},
                   H, W, {1, 0, 0}, 0.026, DR_EDGE_LEADING};
  double wires[K][3], edges[B + 1];
  for (int k = 0; k < K; ++k) {
    wires[k][0] = 0.0;
    wires[k][1] = 0.5;
    wires[k][2] = -0.020 + 0.001 * k;
  }
  for (int j = 0; j <= B; ++j) edges[j] = (-50.5 + j) * 1e-3;
  dr_plan_t *plan = NULL;
  int st = dr_plan(&g, &wires[0][0], K, edges, B, NULL, &plan);
  if (st != DR_OK) return fail("dr_plan", st);
  dr_plan_info info;
  if ((st = dr_plan_get_info(plan, &info)) != DR_OK) return fail("dr_plan_get_info", st);

  static uint16_t img[K][H][W];
  for (int k = 0; k < K; ++k)
    for (int r = 0; r < H; ++r)
      for (int c = 0; c < W; ++c)  /* a deterministic, non-monotone pattern */
        img[k][r][c] = (uint16_t)(1000 + (k * 37 + r * 11 + c * 5) % 97 + (k > 20 ? 300 : 0));
  uint16_t *d_img = NULL;
  float *d_out = NULL;
  if (cudaMalloc((void **)&d_img, sizeof img) != cudaSuccess ||
      cudaMalloc((void **)&d_out, sizeof(float) * B * H * W) != cudaSuccess)
    return fail("cudaMalloc", DR_ERR_CUDA);
  if (cudaMemcpy(d_img, img, sizeof img, cudaMemcpyHostToDevice) != cudaSuccess)
    return fail("cudaMemcpy", DR_ERR_CUDA);
  if ((st = dr_reconstruct(plan, d_img, d_out, NULL)) != DR_OK) return fail("dr_reconstruct", st);
  if (cudaDeviceSynchronize() != cudaSuccess) return fail("synchronize", DR_ERR_CUDA);
  if ((st = dr_plan_check(plan)) != DR_OK) return fail("dr_plan_check", st);
  static float out[B][H][W];
  if (cudaMemcpy(out, d_out, sizeof out, cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail("cudaMemcpy back", DR_ERR_CUDA);
  /* the swept depths lie inside the bins for this geometry */
  if (!(info.depth_min > edges[0] && info.depth_max < edges[B])) {
    fprintf(stderr, "depths [%g, %g] outside the bins\n", info.depth_min, info.depth_max);
    return 1;
  }
  int bad = 0;
  for (int r = 0; r < H; ++r)
    for (int c = 0; c < W; ++c) {
      double sum = 0.0, sabs = 0.0;
      for (int j = 0; j < B; ++j) sum += out[j][r][c];
      for (int k = 0; k + 1 < K; ++k) sabs += fabs((double)img[k][r][c] - img[k + 1][r][c]);
      const double want = (double)img[0][r][c] - (double)img[K - 1][r][c];
      if (fabs(sum - want) > 1e-5 * (sabs > 1 ? sabs : 1)) {
        if (bad < 5) fprintf(stderr, "pixel (%d,%d): sum %.6f, want %.1f\n", r, c, sum, want);
        ++bad;
      }
    }
  cudaFree(d_img);
  cudaFree(d_out);
  dr_plan_destroy(plan);
  if (bad) return 1;
  printf("abi consumer ok: kernel %d, %d x %d pixels, K=%d, B=%d, library %s\n", info.kernel, H,
         W, K, B, dr_version());
  return 0;
}
