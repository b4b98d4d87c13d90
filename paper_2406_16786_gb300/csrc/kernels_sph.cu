// WCSPH neighbour passes (Sec. 2, Sec. 4): density (Eq. (9) / Eq. (4)), force (Eqs. (5)-(8),
// (18)) fused with the kick, the boundary velocity (Eqs. (19), (23)-(26)) and the drift.
//
// Neighbour lists.  One thread per particle of the sorted set A.  Its candidates are the
// particles of the 3^d cells around its cell, one contiguous range per (dy, dz) row (the three
// x-cells of a row are adjacent in the sorted order), plus the wall particles of the same
// cells.  The neighbour-list pass tests every candidate once and appends the in-range ones,
// packed into 32 bits, to the particle's own list (16-byte stores of 4 entries); the density
// and force passes then loop over exactly those neighbours (~80 of ~475 candidates in 3-D), so
// a warp no longer runs the interaction for candidates that only some of its lanes accept.
// Lists are built in a fixed order, so every sum is evaluated in the same order on every run
// (the step is deterministic).
//
// Wall neighbours carry the mirrored state of i (rho_j = rho_i, p_j = p_i, v_j = -v_i), the
// reading of the cited one-sided Riemann solver with no-slip walls.  The intermediate
// velocity of Eq. (4) is taken along -e_ij, consistent with U_L = -v_i . e_ij of Eq. (7):
// (v_i - v*) . e_ij = v_ij . e_ij / 2 + (p_i - p_j) / (2 rho_bar c0).
#include "sph_bodies.cuh"

namespace sphbuf {

namespace {

// Single-domain kernels and their multi-domain (batched) twins: block b of a batched launch
// works for domain map[b].x as its block map[b].y of map[b].z; the domain's descriptor is
// copied to shared memory first.  The batched twins come in two register budgets: the
// single-domain one (for blocks of up to 256 threads) and 64 registers for blocks of 512
// (NAME##_batch512); the autotuner picks the block size.
#define SPHBUF_PAIR(NAME, BODY, BOUNDS)                                                          \
  template <int D>                                                                             \
  __global__ void __launch_bounds__ BOUNDS NAME(DomainDev d) {                                 \
    BODY<D>(d, blockIdx.x, gridDim.x);                                                         \
  }                                                                                            \
  template <int D>                                                                             \
  __global__ void __launch_bounds__ BOUNDS NAME##_batch(BatchDev b) {                          \
    __shared__ DomainDev sd;                                                                   \
    const int4 m = b.map[blockIdx.x];                                                          \
    load_domain(sd, b.doms + m.x);                                                             \
    BODY<D>(sd, (unsigned)m.y, (unsigned)m.z);                                                 \
  }                                                                                            \
  template <int D>                                                                             \
  __global__ void __launch_bounds__(512, 2) NAME##_batch512(BatchDev b) {                      \
    __shared__ DomainDev sd;                                                                   \
    const int4 m = b.map[blockIdx.x];                                                          \
    load_domain(sd, b.doms + m.x);                                                             \
    BODY<D>(sd, (unsigned)m.y, (unsigned)m.z);                                                 \
  }

SPHBUF_PAIR(k_neighbours, neighbours_body, (kThreads, 4))
SPHBUF_PAIR(k_density_deferred, density_deferred_body, (kThreads, 4))
template <int D, bool TVF>
__global__ void __launch_bounds__(kThreads, 4) k_force(DomainDev d, int fused) {
  force_body<D, TVF>(d, blockIdx.x, gridDim.x, fused != 0);
}
template <int D, bool TVF, int BIG>
__global__ void __launch_bounds__(BIG ? 512 : kThreads, BIG ? 2 : 4) k_force_batch(BatchDev b, int fused) {
  __shared__ DomainDev sd;
  const int4 m = b.map[blockIdx.x];
  load_domain(sd, b.doms + m.x);
  force_body<D, TVF>(sd, (unsigned)m.y, (unsigned)m.z, fused != 0);
}
// the drift epilogues, with (fused != 0) or without the buffer decisions
#define SPHBUF_PAIR_F(NAME, BODY, BOUNDS)                                                        \
  template <int D>                                                                             \
  __global__ void __launch_bounds__ BOUNDS NAME(DomainDev d, int fused) {                      \
    BODY<D>(d, blockIdx.x, gridDim.x, fused != 0);                                             \
  }                                                                                            \
  template <int D>                                                                             \
  __global__ void __launch_bounds__ BOUNDS NAME##_batch(BatchDev b, int fused) {               \
    __shared__ DomainDev sd;                                                                   \
    const int4 m = b.map[blockIdx.x];                                                          \
    load_domain(sd, b.doms + m.x);                                                             \
    BODY<D>(sd, (unsigned)m.y, (unsigned)m.z, fused != 0);                                     \
  }                                                                                            \
  template <int D>                                                                             \
  __global__ void __launch_bounds__(512, 2) NAME##_batch512(BatchDev b, int fused) {           \
    __shared__ DomainDev sd;                                                                   \
    const int4 m = b.map[blockIdx.x];                                                          \
    load_domain(sd, b.doms + m.x);                                                             \
    BODY<D>(sd, (unsigned)m.y, (unsigned)m.z, fused != 0);                                     \
  }
SPHBUF_PAIR_F(k_drift, drift_body, (kThreads))
SPHBUF_PAIR(k_begin, begin_body, (32))
SPHBUF_PAIR(k_viscous, viscous_body, (kThreads, 4))
SPHBUF_PAIR_F(k_dual_finish, dual_finish_body, (kThreads))
#undef SPHBUF_PAIR_F

template <int D>
__global__ void __launch_bounds__(kThreads, 4) k_acoustic(DomainDev d, int sub) {
  acoustic_body<D>(d, blockIdx.x, gridDim.x, sub);
}
template <int D>
__global__ void __launch_bounds__(512, 2) k_acoustic_batch(BatchDev b, int sub) {
  __shared__ DomainDev sd;
  const int4 m = b.map[blockIdx.x];
  load_domain(sd, b.doms + m.x);
  acoustic_body<D>(sd, (unsigned)m.y, (unsigned)m.z, sub);
}
#undef SPHBUF_PAIR

int grid_for(const DomainDev& d, int per_sm) { return d.sm_count * per_sm; }


}  // namespace

int launch_neighbours(const DomainDev& d, cudaStream_t s) {
  if (d.g.dim == 2)
    k_neighbours<2><<<grid_for(d, 8), kThreads, 0, s>>>(d);
  else
    k_neighbours<3><<<grid_for(d, 8), kThreads, 0, s>>>(d);
  return 1;
}

int launch_density(const DomainDev& d, cudaStream_t s) {
  // the fluid particles' Eq. (9) is computed by the neighbour pass; this is the rest
  if (d.g.dim == 2)
    k_density_deferred<2><<<grid_for(d, 4), kThreads, 0, s>>>(d);
  else
    k_density_deferred<3><<<grid_for(d, 4), kThreads, 0, s>>>(d);
  return 1;
}

namespace {

template <int D>
void launch_force_t(const DomainDev& d, bool tvf, bool fused, cudaStream_t s) {
  const int g = grid_for(d, 8);
  if (tvf)
    k_force<D, true><<<g, kThreads, 0, s>>>(d, fused ? 1 : 0);
  else
    k_force<D, false><<<g, kThreads, 0, s>>>(d, fused ? 1 : 0);
}

template <int D>
void launch_dual_t(const DomainDev& d, bool fused, cudaStream_t s) {
  const int grid = grid_for(d, 8);
  k_viscous<D><<<grid, kThreads, 0, s>>>(d);
  for (int q = 0; q < d.P.dual_n; ++q) k_acoustic<D><<<grid, kThreads, 0, s>>>(d, q);
  k_dual_finish<D><<<grid, kThreads, 0, s>>>(d, fused ? 1 : 0);
}

template <int D, int BIG>
void launch_batch_force_b(const BatchDev& b, int nblocks, int threads, bool tvf, bool fused, cudaStream_t s) {
  if (tvf)
    k_force_batch<D, true, BIG><<<nblocks, threads, 0, s>>>(b, fused ? 1 : 0);
  else
    k_force_batch<D, false, BIG><<<nblocks, threads, 0, s>>>(b, fused ? 1 : 0);
}

template <int D>
void launch_batch_force_t(const BatchDev& b, int nblocks, int threads, bool tvf, bool fused, cudaStream_t s) {
  if (threads > kThreads)
    launch_batch_force_b<D, 1>(b, nblocks, threads, tvf, fused, s);
  else
    launch_batch_force_b<D, 0>(b, nblocks, threads, tvf, fused, s);
}

}  // namespace

int launch_force(const DomainDev& d, bool fused, cudaStream_t s) {
  const bool tvf = d.P.tvf_lambda > 0.f;
  if (d.g.dim == 2)
    launch_force_t<2>(d, tvf, fused, s);
  else
    launch_force_t<3>(d, tvf, fused, s);
  return 1;
}

int launch_drift(const DomainDev& d, bool fused, cudaStream_t s) {
  const int g = d.sm_count * 8;
  if (d.g.dim == 2) {
    k_begin<2><<<1, 32, 0, s>>>(d);
    k_drift<2><<<g, kThreads, 0, s>>>(d, fused ? 1 : 0);
  } else {
    k_begin<3><<<1, 32, 0, s>>>(d);
    k_drift<3><<<g, kThreads, 0, s>>>(d, fused ? 1 : 0);
  }
  return 2;
}

int launch_dual(const DomainDev& d, bool fused, cudaStream_t s) {
  if (d.g.dim == 2)
    launch_dual_t<2>(d, fused, s);
  else
    launch_dual_t<3>(d, fused, s);
  return d.P.dual_n + 2;
}

int launch_batch_sph(Kern k, int dim, const BatchDev& b, int nblocks, cudaStream_t s, bool tvf, int sub, bool fused,
                     int threads) {
  const bool big = threads > kThreads;
  const int f = fused ? 1 : 0;
  if (k == K_BEGIN) {
    if (dim == 2)
      k_begin_batch<2><<<nblocks, 32, 0, s>>>(b);
    else
      k_begin_batch<3><<<nblocks, 32, 0, s>>>(b);
    return 1;
  }
  if (k == K_ACOUSTIC) {
    if (dim == 2)
      k_acoustic_batch<2><<<nblocks, threads, 0, s>>>(b, sub);
    else
      k_acoustic_batch<3><<<nblocks, threads, 0, s>>>(b, sub);
    return 1;
  }
  if (k == K_FORCE) {
    // the transport-velocity kernel also serves domains with lambda = 0 (p_max stays 0)
    if (dim == 2)
      launch_batch_force_t<2>(b, nblocks, threads, tvf, fused, s);
    else
      launch_batch_force_t<3>(b, nblocks, threads, tvf, fused, s);
    return 1;
  }
#define SPHBUF_CASE(KID, NAME)                                                                                \
  case KID:                                                                                                   \
    if (dim == 2)                                                                                             \
      big ? NAME##_batch512<2><<<nblocks, threads, 0, s>>>(b) : NAME##_batch<2><<<nblocks, threads, 0, s>>>(b); \
    else                                                                                                      \
      big ? NAME##_batch512<3><<<nblocks, threads, 0, s>>>(b) : NAME##_batch<3><<<nblocks, threads, 0, s>>>(b); \
    return 1;
#define SPHBUF_CASE_F(KID, NAME)                                                          \
  case KID:                                                                               \
    if (dim == 2)                                                                         \
      big ? NAME##_batch512<2><<<nblocks, threads, 0, s>>>(b, f)                          \
          : NAME##_batch<2><<<nblocks, threads, 0, s>>>(b, f);                            \
    else                                                                                  \
      big ? NAME##_batch512<3><<<nblocks, threads, 0, s>>>(b, f)                          \
          : NAME##_batch<3><<<nblocks, threads, 0, s>>>(b, f);                            \
    return 1;
  switch (k) {
    SPHBUF_CASE(K_NEIGHBOURS, k_neighbours)
    SPHBUF_CASE(K_DENSITY_DEFER, k_density_deferred)
    SPHBUF_CASE(K_VISCOUS, k_viscous)
    SPHBUF_CASE_F(K_DUAL_FINISH, k_dual_finish)
    SPHBUF_CASE_F(K_DRIFT, k_drift)
    default:
      return 0;
  }
#undef SPHBUF_CASE
#undef SPHBUF_CASE_F
}

}  // namespace sphbuf
