/*
 * The C ABI of include/exx.h used from plain C (no Python, no torch):
 *
 *   exx_c_example spectrum n h
 *       host only: the band-limited kernel spectrum octant; prints Ghat at
 *       k = 0 and k = (n, n, n)
 *   exx_c_example apply n h norb psi.bin vx.bin
 *       FP64 plan (f_i = 2, alpha = 1/4, band-limited kernel) on host buffers:
 *       reads psi[norb][n][n][n] (doubles), writes vx (doubles), prints E_x
 *
 * Exit status 0 on success, 1 on a usage or file error, 2 on a library error.
 */
#include <stdio.h>
#include <stdlib.h>

#include "exx.h"

static int fail(const char* what, exx_status_t s, exx_plan_t plan) {
  fprintf(stderr, "%s: %s %s\n", what, exx_status_string(s), plan ? exx_last_error(plan) : "");
  return 2;
}

int main(int argc, char** argv) {
  if (argc == 4) {
    const int n = atoi(argv[2]);
    const double h = atof(argv[3]);
    const size_t m = (size_t)n + 1;
    double* G = (double*)malloc(m * m * m * sizeof(double));
    if (G == NULL) return 1;
    exx_status_t s = exx_kernel_spectrum(n, h, EXX_KERNEL_SINC, 0.0, G);
    if (s != EXX_OK) return fail("exx_kernel_spectrum", s, NULL);
    printf("%.17g %.17g\n", G[0], G[m * m * m - 1]);
    free(G);
    return 0;
  }
  if (argc != 7) {
    fprintf(stderr, "usage: %s spectrum n h | apply n h norb psi.bin vx.bin\n", argv[0]);
    return 1;
  }
  const int n = atoi(argv[2]);
  const double h = atof(argv[3]);
  const int norb = atoi(argv[4]);
  const size_t cnt = (size_t)norb * n * n * n;
  double* psi = (double*)malloc(cnt * sizeof(double));
  double* vx = (double*)malloc(cnt * sizeof(double));
  double* occ = (double*)malloc((size_t)norb * sizeof(double));
  if (psi == NULL || vx == NULL || occ == NULL) return 1;
  FILE* f = fopen(argv[5], "rb");
  if (f == NULL || fread(psi, sizeof(double), cnt, f) != cnt) return 1;
  fclose(f);
  for (int i = 0; i < norb; ++i) occ[i] = 2.0;

  const int grid[3] = {n, n, n};
  const double hh[3] = {h, h, h};
  exx_plan_t plan = NULL;
  exx_status_t s = exx_plan_create(&plan, grid, hh, 0.25, occ, norb, EXX_FP64, EXX_KERNEL_SINC, 0,
                                   NULL);
  if (s != EXX_OK) return fail("exx_plan_create", s, NULL);
  double E = 0.0;
  s = exx_apply_host(plan, psi, vx, &E, NULL);
  if (s != EXX_OK) return fail("exx_apply_host", s, plan);
  exx_plan_destroy(plan);

  f = fopen(argv[6], "wb");
  if (f == NULL || fwrite(vx, sizeof(double), cnt, f) != cnt) return 1;
  fclose(f);
  printf("%.17g\n", E);
  free(psi);
  free(vx);
  free(occ);
  return 0;
}
