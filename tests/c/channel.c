/* A 2-D channel stepped through the C ABI alone (no Python): a plug velocity inlet and a
 * pressure outlet, 200 steps; checks the count invariant N = N0 + injected - deleted and
 * that both buffers acted.  Prints "ok" and exits 0 on success. */
#include <stdio.h>
#include <stdlib.h>

#include "sphbuf.h"

#define CHECK(call)                                                                     \
  do {                                                                                  \
    sphbuf_status s_ = (call);                                                          \
    if (s_ != SPHBUF_OK) {                                                              \
      fprintf(stderr, "%s failed: %s (%s)\n", #call, sphbuf_status_string(s_),          \
              dom ? sphbuf_error_message(dom) : "");                                    \
      return 1;                                                                         \
    }                                                                                   \
  } while (0)

int main(void) {
  const double dp = 0.01, L = 1.0, W = 0.3, U = 1.0;
  const int nx = (int)(L / dp + 0.5), ny = (int)(W / dp + 0.5);
  sphbuf_domain_t dom = NULL;
  sphbuf_domain_desc desc = {0};
  desc.dim = 2;
  desc.lo[0] = -0.15;
  desc.lo[1] = -0.1;
  desc.hi[0] = L + 0.15;
  desc.hi[1] = W + 0.1;
  desc.dp = dp;
  desc.h_over_dp = 1.3;
  desc.rho0 = 1000.0;
  desc.c0 = 10.0;
  desc.nu = 1e-2;
  desc.dt = 0.25 * 1.3 * dp / (10.0 + U);
  desc.capacity = 2 * (uint64_t)nx * ny;
  CHECK(sphbuf_create_domain(&desc, NULL, &dom));

  /* three wall layers below and above the channel, from x = -0.1 to L + 0.1 */
  const int nwx = (int)((L + 0.2) / dp + 0.5);
  double *wall = malloc(sizeof(double) * 2 * 6 * nwx);
  int nw = 0;
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < nwx; ++i) {
      const double x = -0.1 + (i + 0.5) * dp;
      wall[2 * nw] = x;
      wall[2 * nw + 1] = -(k + 0.5) * dp;
      ++nw;
      wall[2 * nw] = x;
      wall[2 * nw + 1] = W + (k + 0.5) * dp;
      ++nw;
    }
  CHECK(sphbuf_set_walls(dom, wall, (uint64_t)nw));

  /* inlet box [0, 4 dp] x [0, W] with its normal along +x (the inflow direction); outlet box
   * [L - 4 dp, L] x [0, W] with its normal along +x (the outflow direction) */
  const double normal[3] = {1.0, 0.0, 0.0};
  double R[9];
  CHECK(sphbuf_rotation_from_normal(normal, 0.0, R));
  const double ext[3] = {4 * dp, W, 0.0};
  const double o_in[3] = {2 * dp, 0.5 * W, 0.0}, o_out[3] = {L - 2 * dp, 0.5 * W, 0.0};
  sphbuf_bc_params vin = {U, 0.0, 0.0, 0.0, 0.0, 0.0};
  sphbuf_bc_params pout = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  int k_in = -1, k_out = -1;
  CHECK(sphbuf_add_inout_buffer(dom, o_in, R, ext, SPHBUF_VELOCITY_INLET, &vin, &k_in));
  CHECK(sphbuf_add_inout_buffer(dom, o_out, R, ext, SPHBUF_PRESSURE_OUTLET, &pout, &k_out));

  /* fluid on the lattice, moving at U */
  const uint64_t n0 = (uint64_t)nx * ny;
  double *pos = malloc(sizeof(double) * 2 * n0);
  float *vel = malloc(sizeof(float) * 2 * n0);
  float *rho = malloc(sizeof(float) * n0);
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      const size_t q = (size_t)j * nx + i;
      pos[2 * q] = (i + 0.5) * dp;
      pos[2 * q + 1] = (j + 0.5) * dp;
      vel[2 * q] = (float)U;
      vel[2 * q + 1] = 0.0f;
      rho[q] = 1000.0f;
    }
  CHECK(sphbuf_set_fluid(dom, pos, vel, rho, n0));
  CHECK(sphbuf_use_graph(dom, 1));
  CHECK(sphbuf_step(dom, 200));
  CHECK(sphbuf_sync(dom));

  uint64_t n = 0, inj[2], del[2];
  double mi, mo, q;
  CHECK(sphbuf_count(dom, &n));
  CHECK(sphbuf_read_counters(dom, k_in, &inj[0], &del[0], &mi, &mo, &q));
  CHECK(sphbuf_read_counters(dom, k_out, &inj[1], &del[1], &mi, &mo, &q));
  printf("n0 %llu n %llu injected %llu deleted %llu\n", (unsigned long long)n0, (unsigned long long)n,
         (unsigned long long)(inj[0] + inj[1]), (unsigned long long)(del[0] + del[1]));
  const int ok = n == n0 + inj[0] + inj[1] - del[0] - del[1] && inj[0] > 0 && del[1] > 0;
  CHECK(sphbuf_destroy(dom));
  dom = NULL;
  free(wall);
  free(pos);
  free(vel);
  free(rho);
  if (!ok) {
    fprintf(stderr, "count invariant or buffer activity failed\n");
    return 1;
  }
  printf("ok\n");
  return 0;
}
