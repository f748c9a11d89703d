/* A C caller of libhmc, used by the tests to exercise the C ABI without
 * Python: it reads phi and b from a file, applies M[phi; m_s] and solves
 * (M M^dagger) x = b with FP64 CG on the device, and writes M b and x back.
 *
 *   hmc_example n m nt in.bin out.bin
 *
 * in.bin:  N doubles (phi), then N complex doubles (b), N = 2 n m nt.
 * out.bin: N complex doubles (M b), N complex doubles (x).
 * kappa = 1, U = 2, beta = 4, m_s = 0.3, relative tolerance 1e-12.
 * Without a GPU it prints the status hmc_create returns and exits 0. */
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime_api.h>

#include "hmc.h"

static int fail(const char* what) {
  fprintf(stderr, "hmc_example: %s\n", what);
  return 1;
}

int main(int argc, char** argv) {
  if (argc != 6) return fail("usage: hmc_example n m nt in.bin out.bin");
  hmc_lattice lat;
  lat.n = atoi(argv[1]);
  lat.m = atoi(argv[2]);
  lat.nt = atoi(argv[3]);
  lat.kappa = 1.0;
  lat.U = 2.0;
  lat.beta = 4.0;
  const size_t N = 2 * (size_t)lat.n * (size_t)lat.m * (size_t)lat.nt;
  printf("abi %d\n", hmc_abi_version());
  hmc_ctx* ctx = NULL;
  hmc_status st = hmc_create(&ctx, &lat, NULL);
  printf("create %d %s\n", (int)st, hmc_status_string(st));
  if (st != HMC_OK) return 0;

  double* host = (double*)malloc(sizeof(double) * 3 * N);
  double* out = (double*)malloc(sizeof(double) * 4 * N);
  if (!host || !out) return fail("out of host memory");
  FILE* f = fopen(argv[4], "rb");
  if (!f || fread(host, sizeof(double), 3 * N, f) != 3 * N) return fail("cannot read the input file");
  fclose(f);

  double *phi, *b, *mb, *x;
  if (cudaMalloc((void**)&phi, sizeof(double) * N) != cudaSuccess ||
      cudaMalloc((void**)&b, sizeof(double) * 2 * N) != cudaSuccess ||
      cudaMalloc((void**)&mb, sizeof(double) * 2 * N) != cudaSuccess ||
      cudaMalloc((void**)&x, sizeof(double) * 2 * N) != cudaSuccess)
    return fail("cudaMalloc failed");
  cudaMemcpy(phi, host, sizeof(double) * N, cudaMemcpyHostToDevice);
  cudaMemcpy(b, host + N, sizeof(double) * 2 * N, cudaMemcpyHostToDevice);
  cudaMemset(x, 0, sizeof(double) * 2 * N);

  st = hmc_apply_M(ctx, phi, 0.3, b, mb, 64);
  printf("apply_M %d\n", (int)st);
  hmc_solve_info info;
  st = hmc_solve_cg(ctx, phi, 0.3, 0.0, b, x, 1e-12, 10000, &info);
  printf("solve_cg %d iters %d true_rel_res %.3e\n", (int)st, info.iters, info.true_rel_res);
  cudaMemcpy(out, mb, sizeof(double) * 2 * N, cudaMemcpyDeviceToHost);
  cudaMemcpy(out + 2 * N, x, sizeof(double) * 2 * N, cudaMemcpyDeviceToHost);
  f = fopen(argv[5], "wb");
  if (!f || fwrite(out, sizeof(double), 4 * N, f) != 4 * N) return fail("cannot write the output file");
  fclose(f);

  cudaFree(phi);
  cudaFree(b);
  cudaFree(mb);
  cudaFree(x);
  hmc_destroy(ctx);
  free(host);
  free(out);
  return 0;
}
