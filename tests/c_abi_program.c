/* A plain C caller of the library's C ABI (include/sfb.h), with no Python
 * and no PyTorch: it describes the 2-subdomain tiny workload (two 8x8 Darcy
 * subdomains under an 8x8 Taylor-Hood Stokes subdomain, 2 linear mortar
 * elements per edge, N_term = 2 per KL region, tensor 2-point collocation),
 * runs the host set-up calls and prints what they return. It makes no call
 * that needs a GPU. tests/test_c_abi_program.py builds it with gcc and
 * compares its output with the Python binding's. */
#include <stddef.h>
#include <stdio.h>
#include <stdlib.h>

#include "sfb.h"

#define CHECK(call)                                                        \
  do {                                                                     \
    sfb_status st_ = (call);                                               \
    if (st_ != SFB_OK) {                                                   \
      fprintf(stderr, "%s failed: %d %s\n", #call, (int)st_,               \
              ctx ? sfb_last_error(ctx) : "");                             \
      return 1;                                                            \
    }                                                                      \
  } while (0)

int main(void) {
  sfb_ctx* ctx = NULL;
  const int32_t nx[2] = {8, 8}, ny[2] = {8, 8};
  const int32_t msd[2] = {2, 2}, mdv[1] = {2}, mdh[1] = {0};
  const double source[2] = {0.0, 0.0};
  sfb_problem prob = {{0.0, 1.0, 0.0, 0.5}, {0.0, 1.0, 0.5, 1.0}, 2, 1, nx, ny, 8, 8, 1,
                      msd, mdv, mdh, 1.0, 1.0, 1.0, 1.0, 0.0, source};
  CHECK(sfb_create(&prob, NULL, &ctx));
  int64_t n_lambda = 0;
  int32_t n_darcy = 0;
  CHECK(sfb_sizes(ctx, &n_lambda, &n_darcy));
  sfb_kl_region reg[2];
  for (int i = 0; i < 2; ++i) {
    reg[i].sigma2 = 1.0;
    reg[i].eta1 = 0.25;
    reg[i].eta2 = 0.125;
    reg[i].mean_y = 0.0;
    reg[i].n_term = 2;
    reg[i].n_modes_x = 0;
    reg[i].n_modes_y = 0;
  }
  double eig[4];
  CHECK(sfb_kl_setup(ctx, reg, 2, eig));
  sfb_collocation col = {0, 2, 0, 0, NULL, 1, NULL};
  int64_t n_pts = 0;
  CHECK(sfb_collocation_setup(ctx, &col, &n_pts));
  double* y = (double*)malloc(sizeof(double) * (size_t)n_pts * 4);
  double* w = (double*)malloc(sizeof(double) * (size_t)n_pts);
  CHECK(sfb_collocation_points(ctx, y, w));
  double wsum = 0.0;
  for (int64_t l = 0; l < n_pts; ++l) wsum += w[l];
  size_t ws_fp64 = 0, ws_mixed = 0;
  CHECK(sfb_workspace_size(ctx, SFB_FP64, n_pts, &ws_fp64));
  CHECK(sfb_workspace_size(ctx, SFB_MIXED, n_pts, &ws_mixed));
  int32_t threads = 0, ctas = 0, gbuf = 0, tcgen05 = 0, split = 0;
  CHECK(sfb_basis_launch_shape(SFB_MIXED, 0, 0, &threads, &ctas, &gbuf, &tcgen05, &split));
  printf("n_lambda %lld\n", (long long)n_lambda);
  printf("n_darcy %d\n", (int)n_darcy);
  printf("eig %.17g %.17g %.17g %.17g\n", eig[0], eig[1], eig[2], eig[3]);
  printf("n_pts %lld\n", (long long)n_pts);
  printf("weight_sum %.17g\n", wsum);
  printf("workspace_fp64 %zu\n", ws_fp64);
  printf("workspace_mixed %zu\n", ws_mixed);
  printf("shape %d %d %d %d %d\n", (int)threads, (int)ctas, (int)gbuf, (int)tcgen05, (int)split);
  /* struct layouts, for the binding's mirrors: size and the last member's offset */
  printf("layout_problem %zu %zu\n", sizeof(sfb_problem), offsetof(sfb_problem, source));
  printf("layout_kl_region %zu %zu\n", sizeof(sfb_kl_region), offsetof(sfb_kl_region, n_modes_y));
  printf("layout_collocation %zu %zu\n", sizeof(sfb_collocation), offsetof(sfb_collocation, m_dim));
  printf("layout_basis_stats %zu %zu\n", sizeof(sfb_basis_stats), offsetof(sfb_basis_stats, mean_refine_steps));
  /* an out-of-order call is an error status, not a crash */
  if (sfb_moments(ctx, SFB_FIELD_DARCY_P, y, w) == SFB_OK) {
    fprintf(stderr, "moments before any solve should fail\n");
    return 1;
  }
  free(y);
  free(w);
  sfb_destroy(ctx);
  return 0;
}
