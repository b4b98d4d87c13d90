// Device bodies of the WCSPH passes (Sec. 2, Sec. 4), shared by the per-phase kernels
// (kernels_sph.cu) and the persistent batched step (kernels_persist.cu).  Loads of data that
// another block may have written go through SPHBUF_LDG: the read-only path (__ldg) between
// launches, coherent loads inside the persistent step (see kernels_persist.cu).
#pragma once

#include "decide.cuh"

namespace sphbuf {

namespace {

constexpr int kThreads = 256;

// Step prologue, run by one thread of the step's first kernel: per-step constants.  (The
// deferred-particle count is not reset here: the other blocks of the neighbour pass add to it
// while this runs; the rebuild's last pass zeroes it at the end of every step.)
__device__ __forceinline__ void begin_step(const DomainDev& d) {
  StepState* st = d.st;
  st->n_inj = 0;
  st->n_del = 0;
  // Eq. (10): p_max = lambda rho0 v_max^2 with v_max of the last force pass (0 at the start)
  const double vmax = (double)__uint_as_float(st->vmax_bits);
  st->p_max = (float)((double)d.P.tvf_lambda * d.P.rho0_d * vmax * vmax);
  st->vmax_bits = 0u;
  const double t = (double)st->step * d.P.dt_d;
  for (int k = 0; k < d.nbuf; ++k) {
    const BufDev& b = d.bufs[k];
    const double q = (double)st->flux_fx[k] * kFluxUnit;  // flux of the previous step
    st->flux_last[k] = q;
    st->flux_fx[k] = 0;
    double pb;
    if (b.wk) {
      // Eq. (31) as P = P_d + R_p Q, C dP_d/dt = Q - P_d / R_d; explicit Euler with the
      // flux of the previous step: P_d <- P_d + dt ((Q - P_d / R_d) / C)
      double pd = st->wk_pd[k];
      if (st->step > 0)
        pd = SPHBUF_DADD(pd, SPHBUF_DMUL(d.P.dt_d, SPHBUF_DDIV(SPHBUF_DSUB(q, SPHBUF_DDIV(pd, b.wk_rd)), b.wk_c)));
      st->wk_pd[k] = pd;
      pb = SPHBUF_DADD(pd, SPHBUF_DMUL(b.wk_rp, q));
    } else {
      pb = b.p_b0 + b.p_amp * sin(b.p_omega * t + b.p_phase);
    }
    st->pb_d[k] = pb;
    st->pb[k] = (float)pb;
    st->rho_pb[k] = (float)(d.P.rho0_d + (pb - d.P.p_bg_d) / d.P.c0sq_d);
  }
}

// ---------------------------------------------------------------- per-pair arithmetic
// Eq. (9) term, or the Eq. (4) term for a buffer particle i.  (rx, ry, rz) = r_i - r_j.
template <int D>
__device__ __forceinline__ float density_term(const Phys& P, bool buffer_i, bool wall, float rx, float ry, float rz,
                                              float r, const float vi[3], float rho_i, float p_i, const float vj[3],
                                              float rho_j) {
  if (!buffer_i) return kernel_w(r * P.inv_h, P);
  const float inv_r = 1.f / r;
  float vx, vy, vz, p_j;
  if (wall) {
    vx = 2.f * vi[0], vy = 2.f * vi[1], vz = 2.f * vi[2];
    rho_j = rho_i;
    p_j = p_i;
  } else {
    vx = vi[0] - vj[0], vy = vi[1] - vj[1], vz = vi[2] - vj[2];
    p_j = P.c0sq * (rho_j - P.rho0) + P.p_bg;
  }
  const float vij_e = (vx * rx + vy * ry + vz * rz) * inv_r;
  const float term = 0.5f * vij_e + (p_i - p_j) / ((rho_i + rho_j) * P.c0);
  return P.mass / rho_j * term * kernel_dw(r * P.inv_h, P);
}

// Eq. (5) / (18) pair term added to a.  pb2 = 2 p_b (0 for non-buffer particles).  With TVF
// the pair's term of Eq. (10)'s sum, 2 m/(rho_i rho_j) dW/dr e_ij, is added to tb.
template <bool TVF>
__device__ __forceinline__ void force_term(const Phys& P, bool wall, float rx, float ry, float rz, float r2,
                                           const float vi[3], float rho_i, float p_i, float pb2, const float vj[3],
                                           float rho_j, float a[3], float tb[3]) {
  // 1/r and r from the hardware reciprocal square root, and m / (rho_i rho_j) from the fast
  // reciprocal: a few ulp each, far inside the FP32 pass's tolerance against FP64, where the
  // correctly rounded sqrt and divisions cost about a sixth of the pair's instructions
  const float inv_r = rsqrtf(r2), r = r2 * inv_r;
  float vx, vy, vz, p_j;
  if (wall) {
    // mirrored wall state: v_ij = 2 v_i, rho_j = rho_i, p_j = p_i
    vx = 2.f * vi[0], vy = 2.f * vi[1], vz = 2.f * vi[2];
    rho_j = rho_i;
    p_j = p_i;
  } else {
    vx = vi[0] - vj[0], vy = vi[1] - vj[1], vz = vi[2] - vj[2];
    p_j = P.c0sq * (rho_j - P.rho0) + P.p_bg;
  }
  const float dU = -(vx * rx + vy * ry + vz * rz) * inv_r;  // U_L - U_R
  const float beta = fminf(3.f * fmaxf(dU, 0.f), P.c0);
  const float pstar = 0.5f * (p_i + p_j) + 0.25f * beta * (rho_i + rho_j) * dU;
  const float m_rr = __fdividef(P.mass, rho_i * rho_j) * kernel_dw(r * P.inv_h, P);
  const float ce = m_rr * (pb2 - 2.f * pstar) * inv_r;  // along r_ij (e_ij = r_ij / r)
  const float cv = m_rr * 2.f * P.eta * inv_r;
  a[0] += ce * rx + cv * vx;
  a[1] += ce * ry + cv * vy;
  a[2] += ce * rz + cv * vz;
  if (TVF) {
    const float ct = 2.f * m_rr * inv_r;
    tb[0] += ct * rx;
    tb[1] += ct * ry;
    tb[2] += ct * rz;
  }
}

// Calls fn(wall, j, rx, ry, rz) for every particle of the 3^d cells around cell c (global
// memory; the per-particle fallback path).  The cell ranges index the sorted particles, or
// the index list of live slots when the last rebuild kept the slots.
template <int D, typename Fn>
__device__ __forceinline__ void for_each_near(const DomainDev& d, const int c[3], const float fi[3], Fn&& fn,
                                              unsigned first = 0, unsigned stride = 1) {
  const Grid& g = d.g;
  const float cs = g.cs;
  const bool indirect = d.P.reuse && !d.st->full;
  const int x0 = max(c[0] - 1, 0), x1 = min(c[0] + 1, g.nx - 1);
  for (int wall = 0; wall < 2; ++wall) {
    const unsigned* start = wall ? d.W.start : d.cell_start;
    const int* cell = wall ? d.W.cell : d.A.cell;
    const float* const* F = wall ? d.W.f : (const float* const*)d.A.f;
    for (int dz = (D == 3 ? -1 : 0); dz <= (D == 3 ? 1 : 0); ++dz) {
      const int z = c[2] + dz;
      if (z < 0 || z >= g.nz) continue;
      for (int dy = -1; dy <= 1; ++dy) {
        const int y = c[1] + dy;
        if (y < 0 || y >= g.ny) continue;
        const int rb = (z * g.ny + y) * g.nx;
        const unsigned j1 = start[rb + x1 + 1];
        for (unsigned k = start[rb + x0] + first; k < j1; k += stride) {
          const unsigned j = (indirect && !wall) ? d.order[k] : k;
          if (!SPHBUF_IN_BOUNDS(d, wall ? j < d.W.start[g.ncell] : j < d.st->n, 5, j)) continue;
          const int xoff = cell[j] - rb - c[0];
          const float rx = fi[0] - F[0][j] - (float)xoff * cs;
          const float ry = fi[1] - (float)dy * cs - F[1][j];
          const float rz = (D == 3) ? fi[2] - (float)dz * cs - F[2][j] : 0.f;
          fn(wall, j, rx, ry, rz);
        }
      }
    }
  }
}

// Drift + fold + escape check of the force/drift epilogue; writes B[i].  fused: the buffer
// decisions (Algorithms 1-3) of the particle are taken here from its post-drift state, when
// the cell it was sorted into (c) is a candidate cell of some buffer (decide.cuh); n is the
// particle count of the step (duplicates go to B[n + slot]).  (A run-time flag, so that the
// steps with and without the fused decisions run the same code.)
template <int D>
__device__ __forceinline__ void drift_store(const DomainDev& d, bool fused, unsigned i, unsigned n, const int c[3],
                                            const float fi[3], const float v[3], const float adv[3], float rho,
                                            uint8_t lab) {
  const Grid& g = d.g;
  if (lab == kDead) {
    // a slot kept (with kept neighbour lists) for a particle deleted since the last full
    // rebuild: it stays dead and in place until that rebuild drops it
    d.B.cell[i] = (c[2] * g.ny + c[1]) * g.nx + c[0];
#pragma unroll
    for (int x = 0; x < D; ++x) {
      d.B.f[x][i] = fi[x];
      d.B.v[x][i] = 0.f;
    }
    d.B.rho[i] = d.P.rho0;
    d.B.id[i] = d.A.id[i];
    d.B.label[i] = kDead;
#pragma unroll
    for (int x = 0; x < D; ++x) d.disp[x][i] = 0.f;
    d.B.bflag[i] = 0;
    return;
  }
  int cn[3] = {c[0], c[1], c[2]};
  float fn[3] = {fi[0], fi[1], fi[2]};
  bool finite = true;
#pragma unroll
  for (int x = 0; x < D; ++x) finite &= move_fold(fn[x], cn[x], __fmul_rn(adv[x], d.P.dt), g.cs);
  bool inside = cn[0] >= 0 && cn[0] < g.nx && cn[1] >= 0 && cn[1] < g.ny && cn[2] >= 0 && cn[2] < g.nz;
  if (!finite) {
    latch(d.st, 6 /* SPHBUF_ERR_NAN */);
    inside = false;
  }
  if (!inside && lab != kDead) {
    atomicAdd(&d.st->escaped_total, 1ull);
    lab = kDead;
  }
  const unsigned id = d.A.id[i];
  if (fused) {
    const int lin0 = (c[2] * g.ny + c[1]) * g.nx + c[0];
    const unsigned bits =
        SPHBUF_IN_BOUNDS(d, lin0 >= 0 && lin0 < g.ncell, 9, lin0) ? SPHBUF_LDG(d.cand_mask + lin0) : 0u;
    decide_fused<D>(d, __activemask(), n, bits, i, id, lab, cn, fn, inside, v, rho);
  }
  const int lin = inside ? (cn[2] * g.ny + cn[1]) * g.nx + cn[0] : 0;
  d.B.cell[i] = lin;
#pragma unroll
  for (int x = 0; x < D; ++x) {
    d.B.f[x][i] = fn[x];
    d.B.v[x][i] = v[x];
  }
  d.B.rho[i] = rho;
  d.B.id[i] = id;
  d.B.label[i] = lab;
  d.B.bflag[i] = d.A.bflag[i];
  if (d.P.reuse) {
    // displacement since the last full list build relative to the period's reference
    // velocity, its largest length this step, and the range of the drift velocities
    float s2 = 0.f;
#pragma unroll
    for (int x = 0; x < D; ++x) {
      const float dx = d.disp[x][i] + (adv[x] - d.st->u0[x]) * d.P.dt;
      d.disp[x][i] = dx;
      s2 += dx * dx;
    }
    const unsigned am = __activemask();
    const bool lead = (threadIdx.x & 31) == __ffs(am) - 1;
    const unsigned wmax = __reduce_max_sync(am, __float_as_uint(sqrtf(s2)));
    if (lead) atomicMax(&d.st->path_bits, wmax);
    // the range over every particle (so that u0, and with it the step on which lists are
    // built again, depends on the state alone, not on which warp took which particles); each
    // warp adds to one of kRangeCopies copies, which keeps the atomics off one address
    const unsigned copy = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) % (unsigned)kRangeCopies;
#pragma unroll
    for (int x = 0; x < D; ++x) {
      const unsigned k = float_to_key(adv[x]);
      const unsigned hi = __reduce_max_sync(am, k), lo = __reduce_max_sync(am, ~k);
      if (lead) {
        atomicMax(&d.st->v_hi[copy][x], hi);
        atomicMax(&d.st->v_lo[copy][x], lo);
      }
    }
  }
}

// Kick, boundary velocity, flux, drift for centre particle i with acceleration a.  With TVF
// (Eq. (10)) a fluid particle (label 0) drifts with v - dt p_max tb, the buffer particles (the
// in-/outlet boundary layers, reading A23) with v; v_max of the pass is recorded.
template <int D, bool TVF>
__device__ __forceinline__ void finish_force(const DomainDev& d, bool fused, unsigned i, unsigned n, const int c[3], const float fi[3],
                                             const float vi[3], float rho_i, uint8_t lab, const float a[3],
                                             const float tb[3], bool near_core = false) {
  const Phys& P = d.P;
  float v[3] = {vi[0] + a[0] * P.dt, vi[1] + a[1] * P.dt, D == 3 ? vi[2] + a[2] * P.dt : 0.f};
  if (lab != 0 && lab != kDead) {
    const int k = (int)lab - 1;
    const BufDev& b = d.bufs[k];
    if (b.vel_bc) {
      // Eqs. (23)-(26): v = U profile(Y', Z') along u, from the start-of-step position
      float X[3];
      local_coords<D>(b, c, fi, d.g.cs, X, D);
      float rr = X[1] * X[1];
      if (D == 3) rr += X[2] * X[2];
      const float prof = b.inv_hw2 > 0.f ? b.umax * fmaxf(1.f - rr * b.inv_hw2, 0.f) : b.umax;
#pragma unroll
      for (int x = 0; x < D; ++x) v[x] = prof * b.u[x];
    } else {
      // Eq. (19): v = (v . u) u
      float vn = v[0] * b.u[0] + v[1] * b.u[1];
      if (D == 3) vn += v[2] * b.u[2];
#pragma unroll
      for (int x = 0; x < D; ++x) v[x] = vn * b.u[x];
    }
    float vn = v[0] * b.u[0] + v[1] * b.u[1];
    if (D == 3) vn += v[2] * b.u[2];
    atomicAdd(reinterpret_cast<unsigned long long*>(&d.st->flux_fx[k]),
              (unsigned long long)__double2ll_rn((double)(vn * b.flux_scale) * kFluxScale));
  }
  if (TVF) {
    // reading A27: the inner fluid is label 0 and neither core nor within 2h of a core
    // boundary particle; the flags go with the particle for the next step's temporal test
    const uint8_t cf = d.core[i];
    const bool bnd = (cf & 1u) || near_core;
    float adv[3] = {v[0], v[1], v[2]};
    if (lab == 0 && !bnd) {
      const float s = P.dt * d.st->p_max;
#pragma unroll
      for (int x = 0; x < D; ++x) adv[x] = v[x] - s * tb[x];
    }
    float sp = v[0] * v[0] + v[1] * v[1];
    if (D == 3) sp += v[2] * v[2];
    const unsigned bits = __float_as_uint(sqrtf(sp));  // non-negative: bits order like values
    const unsigned am = __activemask();
    const unsigned wmax = __reduce_max_sync(am, bits);
    if ((threadIdx.x & 31) == __ffs(am) - 1) atomicMax(&d.st->vmax_bits, wmax);
    drift_store<D>(d, fused, i, n, c, fi, v, adv, rho_i, lab);
    if (lab != kDead)
      d.B.bflag[i] = (uint8_t)(2u | ((cf >> 1) & 1u) | ((cf & 1u) << 2) | (bnd ? 8u : 0u));
  } else {
    drift_store<D>(d, fused, i, n, c, fi, v, v, rho_i, lab);
  }
}

__device__ __forceinline__ float boundary_pressure2(const DomainDev& d, uint8_t lab, float p_i) {
  // Eq. (18): 2 p_b with p_b(t) prescribed, or p_b = p_i for velocity buffers (Sec. 4.2)
  if (lab == 0 || lab == kDead) return 0.f;
  const int k = (int)lab - 1;
  return 2.f * (d.bufs[k].vel_bc ? p_i : d.st->pb[k]);
}

// ---------------------------------------------------------------- fallback: one particle from the cells
template <int D, bool TVF>
__device__ void force_one(const DomainDev& d, bool fused, unsigned i, unsigned n) {
  const Phys& P = d.P;
  int c[3];
  cell_coords(d.A.cell[i], d.g, c);
  const float fi[3] = {d.A.f[0][i], d.A.f[1][i], D == 3 ? d.A.f[2][i] : 0.f};
  const float vi[3] = {d.A.v[0][i], d.A.v[1][i], D == 3 ? d.A.v[2][i] : 0.f};
  const uint8_t lab = d.A.label[i];
  const float rho_i = d.vr4[i].w;
  const float p_i = P.c0sq * (rho_i - P.rho0) + P.p_bg;
  const float pb2 = boundary_pressure2(d, lab, p_i);
  float a[3] = {0.f, 0.f, 0.f}, tb[3] = {0.f, 0.f, 0.f};
  bool near_core = false;
  for_each_near<D>(d, c, fi, [&](int wall, unsigned j, float rx, float ry, float rz) {
    const float r2 = rx * rx + ry * ry + rz * rz;
    if (r2 < P.two_h_sq && r2 > 0.f) {
      float vj[3] = {0.f, 0.f, 0.f};
      float rho_j = rho_i;
      if (!wall) {
        const float4 v = d.vr4[j];
        vj[0] = v.x, vj[1] = v.y, vj[2] = v.z;
        rho_j = v.w;
        if (TVF) near_core |= (d.core[j] & 1u) != 0;
      }
      force_term<TVF>(P, wall, rx, ry, rz, r2, vi, rho_i, p_i, pb2, vj, rho_j, a, tb);
    }
  });
  finish_force<D, TVF>(d, fused, i, n, c, fi, vi, rho_i, lab, a, tb, near_core);
}

// ---------------------------------------------------------------- neighbour lists
// Packed neighbour: index j (bits 0-30) | wall (bit 31).  The pair's geometry comes from the
// cells packed in both particles' position copies (pos4.w), so an entry stays valid when
// either particle moves to another cell (lists kept over several steps).

// Unpacks one entry of the particle in packed cell ci at offset fi and calls
// fn(wall, j, rx, ry, rz), r = r_i - r_j.
template <int D, typename Fn>
__device__ __forceinline__ void visit_entry(const DomainDev& d, unsigned ent, unsigned ci, const float fi[3],
                                            Fn&& fn, unsigned who = kNoSlot, unsigned site = 3) {
  const float cs = d.g.cs;
  const unsigned j = ent & 0x7FFFFFFFu;
  const int wall = (int)(ent >> 31);
  if (!SPHBUF_IN_BOUNDS_AT(d, wall ? j < d.W.start[d.g.ncell] : j < d.st->n, site + 100 * wall, j, who)) return;
  const float4 p = SPHBUF_LDG((wall ? d.wpos4 : d.pos4) + j);
  const unsigned cj = __float_as_uint(p.w);
  const float rx = fi[0] - p.x - (packed_cx(cj) - packed_cx(ci)) * cs;
  const float ry = fi[1] - (packed_cyf(cj) - packed_cyf(ci)) * cs - p.y;
  const float rz = (D == 3) ? fi[2] - (packed_czf(cj) - packed_czf(ci)) * cs - p.z : 0.f;
  fn(wall, j, rx, ry, rz);
}

// Calls fn for the cnt listed neighbours of particle i (16-byte loads of 4 entries, the next
// four loaded while the current four are visited).  The list was written by an earlier launch.
template <int D, typename Fn>
__device__ __forceinline__ void for_each_listed(const DomainDev& d, unsigned i, int cnt, unsigned ci, const float fi[3],
                                                Fn&& fn, unsigned site = 3) {
  const uint4* lst = reinterpret_cast<const uint4*>(d.nb + (size_t)i * d.nb_cap);
  uint4 nq = make_uint4(0u, 0u, 0u, 0u);
  if (cnt > 0) nq = SPHBUF_LDG(lst);
  for (int e = 0; e < cnt; e += 4) {
    const uint4 q = nq;
    if (e + 4 < cnt) nq = SPHBUF_LDG(lst + (e >> 2) + 1);
    visit_entry<D>(d, q.x, ci, fi, fn, i, site);
    if (e + 1 < cnt) visit_entry<D>(d, q.y, ci, fi, fn, i, site);
    if (e + 2 < cnt) visit_entry<D>(d, q.z, ci, fi, fn, i, site);
    if (e + 3 < cnt) visit_entry<D>(d, q.w, ci, fi, fn, i, site);
  }
}

// Boundary identification of reading A27 (the transport velocity's inner fluid): particle i
// is a candidate when its position divergence psi = -sum_j V_j r_ij . grad_i W_ij falls below
// 0.75 d, and core when it was a candidate in the previous step too (or has no previous step);
// core[i] holds bit 0 core, bit 1 candidate for the force pass.
__device__ __forceinline__ void identify_boundary(const DomainDev& d, unsigned i, float psi) {
  const bool cand = psi < d.P.psi_cand;
  const uint8_t prev = d.A.bflag[i];
  const bool before = (prev & 2u) ? (prev & 1u) != 0 : cand;
  d.core[i] = (uint8_t)((cand && before ? 1u : 0u) | (cand ? 2u : 0u));
}

// The position of list entry ent (fluid slot or wall), for the pipelined walk below.
__device__ __forceinline__ float4 entry_pos(const DomainDev& d, unsigned ent, unsigned who, unsigned site) {
  const unsigned j = ent & 0x7FFFFFFFu;
  const int wall = (int)(ent >> 31);
  if (!SPHBUF_IN_BOUNDS_AT(d, wall ? j < d.W.start[d.g.ncell] : j < d.st->n, site + 100 * wall, j, who))
    return make_float4(0.f, 0.f, 0.f, __uint_as_float(0xFFFFFFFFu));
  return SPHBUF_LDG((wall ? d.wpos4 : d.pos4) + j);
}

// Density, Eq. (9), for particle i of the fluid (not in a buffer) from its list; writes
// vr4[i] = (v_i, rho_i).  The sum runs in list order, as in every other pass.
template <int D, bool OWN>
__device__ __forceinline__ void density_fluid(const DomainDev& d, unsigned i, int cnt) {
  const Phys& P = d.P;
  const float4 pi = d.pos4[i];
  const float fi[3] = {pi.x, pi.y, pi.z};
  const unsigned ci = __float_as_uint(pi.w);
  const bool tvf = P.tvf_lambda > 0.f;
  const unsigned site = OWN ? 11 : 12;
  float s = 0.f, psi = 0.f;
  // software pipeline over the chunks of four entries: the positions of chunk k + 1 and the
  // entries of chunk k + 2 are in flight while chunk k is summed
  const uint4* lst = reinterpret_cast<const uint4*>(d.nb + (size_t)i * d.nb_cap);
  auto ld = [&](int c) { return OWN ? lst[c] : SPHBUF_LDG(lst + c); };
  const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
  const uint4 q = cnt > 0 ? ld(0) : zero;
  uint4 nq = cnt > 4 ? ld(1) : zero;
  float4 p[4];
  {
    const unsigned e4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) p[k] = k < cnt ? entry_pos(d, e4[k], i, site) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  const float cs = d.g.cs;
  for (int e = 0; e < cnt; e += 4) {
    float4 pn[4];
    {
      const unsigned e4[4] = {nq.x, nq.y, nq.z, nq.w};
#pragma unroll
      for (int k = 0; k < 4; ++k)
        pn[k] = e + 4 + k < cnt ? entry_pos(d, e4[k], i, site) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const uint4 nnq = e + 8 < cnt ? ld((e >> 2) + 2) : zero;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (e + k < cnt) {
        const unsigned cj = __float_as_uint(p[k].w);
        const float rx = fi[0] - p[k].x - (packed_cx(cj) - packed_cx(ci)) * cs;
        const float ry = fi[1] - (packed_cyf(cj) - packed_cyf(ci)) * cs - p[k].y;
        const float rz = (D == 3) ? fi[2] - (packed_czf(cj) - packed_czf(ci)) * cs - p[k].z : 0.f;
        const float r2 = rx * rx + ry * ry + rz * rz;
        const float r = r2 * rsqrtf(r2);  // (listed pairs have r > 0)
        s += kernel_w(r * P.inv_h, P);
        if (tvf) psi -= P.vol * r * kernel_dw(r * P.inv_h, P);
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) p[k] = pn[k];
    nq = nnq;
  }
  const float4 v = d.vel4[i];
  d.vr4[i] = make_float4(v.x, v.y, v.z, P.rho0 * (s + P.w_self) * P.inv_sum_w0);
  if (tvf) identify_boundary(d, i, psi);
}

// Eq. (9) for fluid particle i from its list, or, for a buffer particle (the Eq. (4) rate) or
// an overflowed list (strong compression: it reads its cells directly), an entry in the
// deferred list for density_deferred_body.  Every active lane of the warp calls it.
template <int D, bool OWN>
__device__ __forceinline__ void density_or_defer(const DomainDev& d, unsigned i, int cnt) {
  const int lane = threadIdx.x & 31;
  const bool defer = d.A.label[i] != 0 || cnt > d.nb_cap;
  const unsigned am = __activemask();
  const unsigned m = __ballot_sync(am, defer);
  if (m) {
    const int leader = __ffs(m) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(&d.st->n_defer, (unsigned)__popc(m));
    base = __shfl_sync(am, base, leader);
    if (defer) d.deferred[base + __popc(m & ((1u << lane) - 1u))] = i;
  }
  if (!defer) density_fluid<D, OWN>(d, i, cnt);
}

// One candidate of the neighbour-list pass: appends j to the particle's list when within 2h.
// The last four entries are held in q0..q3 (oldest first) and stored 16 bytes at a time.
struct ListTail {
  unsigned q0, q1, q2, q3;
  int cnt;
};

__device__ __forceinline__ void list_append(ListTail& t, bool in, unsigned ent, uint4* lst, int cap) {
  t.q0 = in ? t.q1 : t.q0;
  t.q1 = in ? t.q2 : t.q1;
  t.q2 = in ? t.q3 : t.q2;
  t.q3 = in ? ent : t.q3;
  t.cnt += in;
  if (in && (t.cnt & 3) == 0 && t.cnt <= cap) lst[(t.cnt >> 2) - 1] = make_uint4(t.q0, t.q1, t.q2, t.q3);
}

// One particle's neighbour search: tests every candidate of the 3^d cells around cell c once
// (one 16-byte load each) and appends those within r2max to the particle's list (contiguous
// per particle, 16-byte stores of 4 entries, branch-free appends); returns the count.
// INDIRECT: the fluid candidates are read through the index list `order` (kept lists: the
// slots are not sorted), otherwise the cell ranges index the sorted particles directly.
// (Skipping rows and end cells that cannot hold a neighbour, per particle, was slower: the
// lanes of a warp rarely agree on the skip.)
template <int D, bool INDIRECT>
__device__ __forceinline__ int search_list(const DomainDev& d, unsigned i, const int c[3], const float4 pi,
                                           float r2max) {
  const Grid& g = d.g;
  const float cs = g.cs;
  const int cap = d.nb_cap;
  const float cxf = packed_cx(__float_as_uint(pi.w));
  uint4* lst = reinterpret_cast<uint4*>(d.nb + (size_t)i * cap);
  ListTail t{0u, 0u, 0u, 0u, 0};
  // x of particle i from its grid row's origin: enough for the inclusion test (its rounding,
  // ~1e-7 of the row length, moves only pairs at the list radius by O(1e-5) of it); the
  // density and force passes recompute r_ij from the cell offsets
  const float ox = pi.x + cxf * cs;
#pragma unroll 1
  for (int wall = 0; wall < 2; ++wall) {
    const unsigned* start = wall ? d.W.start : d.cell_start;
    const float4* P4 = wall ? d.wpos4 : d.pos4;
#pragma unroll 1
    for (int dz = (D == 3 ? -1 : 0); dz <= (D == 3 ? 1 : 0); ++dz) {
      const int z = c[2] + dz;
      if (z < 0 || z >= g.nz) continue;
#pragma unroll 1
      for (int dy = -1; dy <= 1; ++dy) {
        const int y = c[1] + dy;
        if (y < 0 || y >= g.ny) continue;
        const int x0 = max(c[0] - 1, 0), x1 = min(c[0] + 1, g.nx - 1);
        const int rb = (z * g.ny + y) * g.nx;
        const unsigned tag = (unsigned)wall << 31;
        const float oy = pi.y - (float)dy * cs;
        const float oz = (D == 3) ? pi.z - (float)dz * cs : 0.f;
        const unsigned k1 = SPHBUF_LDG(start + rb + x1 + 1);
        unsigned k = SPHBUF_LDG(start + rb + x0);
        for (; k < k1; ++k) {
          const unsigned j = (INDIRECT && !wall) ? SPHBUF_LDG(d.order + k) : k;
          if (!SPHBUF_IN_BOUNDS(d, wall ? j < d.W.start[g.ncell] : j < d.st->n, wall ? 2 : 1, j)) continue;
          const float4 p = SPHBUF_LDG(P4 + j);
          const float rx = ox - (p.x + packed_cx(__float_as_uint(p.w)) * cs);
          const float ry = oy - p.y;
          const float rz = (D == 3) ? oz - p.z : 0.f;
          const float r2 = rx * rx + ry * ry + rz * rz;
          list_append(t, r2 < r2max && r2 > 0.f, j | tag, lst, cap);
        }
      }
    }
  }
  // the last (cnt mod 4) entries are q(4 - r) .. q3
  const int r = t.cnt & 3;
  if (r && t.cnt < cap)
    lst[t.cnt >> 2] = make_uint4(r == 1 ? t.q3 : (r == 2 ? t.q2 : t.q1), r == 2 ? t.q3 : t.q2, t.q3, 0u);
  d.nb_cnt[i] = (unsigned)t.cnt;
  return t.cnt;
}

// Dynamic share-out of a pass over the particles: the blocks of the pass (nblk of them for
// this domain) take chunks of blockDim.x particles from the domain's counter st->sched[k]
// until none is left, so that blocks whose chunks are costly (the every-step search region of
// kept lists, strongly compressed regions) do not hold up the end of the pass; body(i) runs
// for i = chunk * blockDim.x + threadIdx.x (i may reach past n).  Every block takes part,
// with n = 0 once an error is latched; the last block to finish resets the counter and the
// done count for the pass's next launch.
template <typename Body>
__device__ __forceinline__ void for_each_chunk(const DomainDev& d, int k, unsigned n, unsigned nblk, Body&& body) {
  __shared__ unsigned s_chunk;
  const unsigned nch = (n + blockDim.x - 1) / blockDim.x;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_chunk = atomicAdd(&d.st->sched[k], 1u);
    __syncthreads();
    const unsigned c = s_chunk;
    if (c >= nch) break;
    body(c * blockDim.x + threadIdx.x);
  }
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&d.st->sched_done[k], 1u) == nblk - 1u) {
      atomicExch(&d.st->sched[k], 0u);
      atomicExch(&d.st->sched_done[k], 0u);
    }
  }
}

// Neighbour-list pass, then Eq. (9) from the list for a fluid particle (deferred otherwise).
// Lists rebuilt every step (reuse off): every particle searches the sorted cells.  Kept lists
// (reuse on): after a full rebuild every particle searches (radius 2h + skin, displacements
// restart from 0); after a rebuild that kept the slots, only the particles whose cell lies in
// the every-step region around the buffers (where duplicates appear and parents are recycled)
// search, through the index list, and the others keep their lists; dead slots are skipped
// (their density copy is a harmless rho0 at rest, since listed dead slots add nothing).
template <int D>
__device__ __forceinline__ void neighbours_body(const DomainDev& d, unsigned bid, unsigned nblk) {
  if (bid == 0 && threadIdx.x == 0) begin_step(d);
  const unsigned n = d.st->status ? 0u : d.st->n;
  const Grid g = d.g;
  const bool reuse = d.P.reuse != 0;
  const bool full = !reuse || d.st->full != 0;
  const float r2max = d.P.list_r2;
  for_each_chunk(d, 0, n, nblk, [&](unsigned i) {
    if (i >= n) return;
    const int lin = d.A.cell[i];
    if (!SPHBUF_IN_BOUNDS(d, (lin >= 0 && lin < d.g.ncell) || d.A.label[i] == kDead, 6, i)) return;
    if (reuse && !full && d.A.label[i] == kDead) {
      d.nb_cnt[i] = 0u;
      d.vr4[i] = make_float4(0.f, 0.f, 0.f, d.P.rho0);
      if (d.P.tvf_lambda > 0.f) d.core[i] = 0;
      return;
    }
    const bool fresh = full || SPHBUF_LDG(d.s_mask + lin) != 0;
    int cnt;
    if (fresh) {
      int c[3];
      cell_coords(lin, g, c);
      const float4 pi = d.pos4[i];
      cnt = full ? search_list<D, false>(d, i, c, pi, r2max) : search_list<D, true>(d, i, c, pi, r2max);
      if (reuse && full)
        for (int x = 0; x < D; ++x) d.disp[x][i] = 0.f;
    } else {
      cnt = (int)d.nb_cnt[i];
    }
    // Eq. (9) right away, while a new list and the neighbours' positions are in cache
    if (fresh)
      density_or_defer<D, true>(d, i, cnt);
    else
      density_or_defer<D, false>(d, i, cnt);
  });
}

// The deferred particles of the density pass: Eq. (4) rate for buffer particles (the Riemann
// intermediate velocity of reading A9 against the neighbours' start-of-step velocity and
// density, density_term), Eq. (9) from the cells for fluid particles with an overflowed list.
template <int D>
__device__ __forceinline__ void density_deferred_body(const DomainDev& d, unsigned bid, unsigned nblk) {
  if (d.st->status) return;
  const unsigned nd = d.st->n_defer;
  const Phys P = d.P;
  const int cap = d.nb_cap;
  // eight lanes per deferred particle share its neighbours (the buffer particles, tens of
  // thousands, would leave the GPU waiting on one long neighbour loop per thread), then a
  // reduction over the eight in a fixed order (the group's first lane's)
  constexpr unsigned G = 8;
  const unsigned lane = threadIdx.x & (G - 1);
  const unsigned grp = (bid * blockDim.x + threadIdx.x) / G, ngrp = (nblk * blockDim.x) / G;
  // every lane of a warp runs the same number of rounds (the shuffles need all 32)
  const unsigned rounds = (nd + ngrp - 1) / ngrp;
  for (unsigned r = 0; r < rounds; ++r) {
    const unsigned e = grp + r * ngrp;
    const bool live = e < nd;
    const unsigned i = live && SPHBUF_IN_BOUNDS(d, d.deferred[e] < d.st->n, 7, d.deferred[e]) ? d.deferred[e] : 0u;
    const int cnt = live ? (int)d.nb_cnt[i] : 0;
    const float4 pi = d.pos4[i];
    const float fi[3] = {pi.x, pi.y, pi.z};
    const uint8_t lab = d.A.label[i];
    const bool buf = lab != 0;
    const float4 vi4 = d.vel4[i];
    const float rho_i = vi4.w;
    const float p_i = P.c0sq * (rho_i - P.rho0) + P.p_bg;
    const float vi[3] = {vi4.x, vi4.y, vi4.z};
    float s = 0.f, psi = 0.f;
    const bool tvf = P.tvf_lambda > 0.f;
    auto term = [&](int wall, unsigned j, float rx, float ry, float rz) {
      const float r2 = rx * rx + ry * ry + rz * rz;
      if (tvf) {
        const float r = sqrtf(r2);
        psi -= P.vol * r * kernel_dw(r * P.inv_h, P);
      }
      if (!buf) {
        s += kernel_w(sqrtf(r2) * P.inv_h, P);
      } else {
        float vj[3] = {0.f, 0.f, 0.f};
        float rho_j = rho_i;
        if (!wall) {
          const float4 v = SPHBUF_LDG(d.vel4 + j);
          vj[0] = v.x, vj[1] = v.y, vj[2] = v.z;
          rho_j = v.w;
        }
        s += density_term<D>(P, true, wall, rx, ry, rz, sqrtf(r2), vi, rho_i, p_i, vj, rho_j);
      }
    };
    if (cnt <= cap) {
      const unsigned* lst = d.nb + (size_t)i * cap;
      for (int k = (int)lane; k < cnt; k += (int)G)
        visit_entry<D>(d, SPHBUF_LDG(lst + k), __float_as_uint(pi.w), fi, term, i, 15);
    } else {
      int c[3];
      cell_coords(d.A.cell[i], d.g, c);
      for_each_near<D>(
          d, c, fi,
          [&](int wall, unsigned j, float rx, float ry, float rz) {
            const float r2 = rx * rx + ry * ry + rz * rz;
            if (r2 < P.two_h_sq && r2 > 0.f) term(wall, j, rx, ry, rz);
          },
          lane, G);
    }
#pragma unroll
    for (int o = (int)G / 2; o > 0; o >>= 1) {
      s += __shfl_xor_sync(0xFFFFFFFFu, s, o, (int)G);
      psi += __shfl_xor_sync(0xFFFFFFFFu, psi, o, (int)G);
    }
    if (live && lane == 0 && tvf) identify_boundary(d, i, psi);
    if (live && lane == 0) {
      // (in the dual-criteria scheme the buffer particles keep their density here; their
      // continuity is integrated by the acoustic steps)
      const float rb = P.dual_n > 0 ? rho_i : rho_i + P.dt * (2.f * rho_i * s);
      d.vr4[i] = make_float4(vi[0], vi[1], vi[2], buf ? rb : P.rho0 * (s + P.w_self) * P.inv_sum_w0);
    }
  }
}

// Force pass over the lists: Eqs. (5)-(8), (18), then kick, boundary velocity and drift
// (with the transport velocity of Eq. (10) when TVF).
template <int D, bool TVF>
__device__ __forceinline__ void force_body(const DomainDev& d, unsigned bid, unsigned nblk, bool fused) {
  const unsigned n = d.st->status ? 0u : d.st->n;
  const Phys P = d.P;
  const int cap = d.nb_cap;
  for_each_chunk(d, 1, n, nblk, [&](unsigned i) {
    if (i >= n) return;
    const int cnt = (int)d.nb_cnt[i];
    if (cnt > cap) {
      force_one<D, TVF>(d, fused, i, n);
      return;
    }
    const float4 pi = d.pos4[i];
    const float fi[3] = {pi.x, pi.y, pi.z};
    const float4 vi4 = d.vr4[i];
    const float vi[3] = {vi4.x, vi4.y, vi4.z};
    const uint8_t lab = d.A.label[i];
    const float rho_i = vi4.w;
    const float p_i = P.c0sq * (rho_i - P.rho0) + P.p_bg;
    const float pb2 = boundary_pressure2(d, lab, p_i);
    float a[3] = {0.f, 0.f, 0.f}, tb[3] = {0.f, 0.f, 0.f};
    bool near_core = false;
    for_each_listed<D>(d, i, cnt, __float_as_uint(pi.w), fi, [&](int wall, unsigned j, float rx, float ry, float rz) {
      const float r2 = rx * rx + ry * ry + rz * rz;
      float vj[3] = {0.f, 0.f, 0.f};
      float rho_j = rho_i;
      if (!wall) {
        const float4 v = SPHBUF_LDG(d.vr4 + j);
        vj[0] = v.x, vj[1] = v.y, vj[2] = v.z;
        rho_j = v.w;
        // (kept lists reach beyond 2h: the layer test takes the pairs within 2h only)
        if (TVF && r2 < P.two_h_sq) near_core |= (SPHBUF_LDG(d.core + j) & 1u) != 0;
      }
      force_term<TVF>(P, wall, rx, ry, rz, r2, vi, rho_i, p_i, pb2, vj, rho_j, a, tb);
    }, 13);
    int c[3];
    cell_coords(d.A.cell[i], d.g, c);
    finish_force<D, TVF>(d, fused, i, n, c, fi, vi, rho_i, lab, a, tb, near_core);
  });
}

// Kinematic steps start with a launch of their own for the step constants (begin_body): the
// drift that follows takes the fused buffer decisions, which read them (rho0 + p_b / c0^2)
// and add to the list counts that begin_step resets.
template <int D>
__device__ __forceinline__ void begin_body(const DomainDev& d, unsigned bid, unsigned) {
  if (bid == 0 && threadIdx.x == 0) begin_step(d);
}

template <int D>
__device__ __forceinline__ void drift_body(const DomainDev& d, unsigned bid, unsigned nblk, bool fused) {
  if (d.st->status) return;
  const unsigned n = d.st->n;
  for (unsigned i = bid * blockDim.x + threadIdx.x; i < n; i += nblk * blockDim.x) {
    int c[3];
    cell_coords(d.A.cell[i], d.g, c);
    const float fi[3] = {d.A.f[0][i], d.A.f[1][i], D == 3 ? d.A.f[2][i] : 0.f};
    const float v[3] = {d.A.v[0][i], d.A.v[1][i], D == 3 ? d.A.v[2][i] : 0.f};
    drift_store<D>(d, fused, i, n, c, fi, v, v, d.A.rho[i], d.A.label[i]);
  }
}

// ---------------------------------------------------------------- dual-criteria time stepping
// One advection step = the neighbour lists and the density re-initialisation (Eq. (9)) of the
// step, the viscous acceleration once (viscous_body), dual_n acoustic steps (acoustic_body:
// continuity, Eq. (4), and the pressure part of Eq. (5) with Eq. (18) from the current state;
// kick, boundary velocity, density and position update), then the positions are folded back
// into their cells and written to B (dual_finish_body).  During the acoustic steps the
// configuration of the lists is fixed and the offsets stay relative to the cells of the
// advection step (they may leave [0, cs)); pos4/vr4 and pos_b/vr_b alternate.

// Viscous part of Eq. (5) for the pair (walls: v_ij = 2 v_i, rho_j = rho_i).
__device__ __forceinline__ void viscous_term(const Phys& P, bool wall, float rx, float ry, float rz, float r2,
                                             const float vi[3], float rho_i, const float vj[3], float rho_j,
                                             float a[3]) {
  const float r = sqrtf(r2), inv_r = 1.f / r;
  float vx, vy, vz;
  if (wall) {
    vx = 2.f * vi[0], vy = 2.f * vi[1], vz = 2.f * vi[2];
    rho_j = rho_i;
  } else {
    vx = vi[0] - vj[0], vy = vi[1] - vj[1], vz = vi[2] - vj[2];
  }
  const float cv = P.mass / (rho_i * rho_j) * kernel_dw(r * P.inv_h, P) * 2.f * P.eta * inv_r;
  a[0] += cv * vx;
  a[1] += cv * vy;
  a[2] += cv * vz;
}

template <int D>
__device__ __forceinline__ void viscous_body(const DomainDev& d, unsigned bid, unsigned nblk) {
  if (d.st->status) return;
  const unsigned n = d.st->n;
  const Phys P = d.P;
  const int cap = d.nb_cap;
  for (unsigned i = bid * blockDim.x + threadIdx.x; i < n; i += nblk * blockDim.x) {
    const int cnt = (int)d.nb_cnt[i];
    const float4 pi = d.pos4[i];
    const float fi[3] = {pi.x, pi.y, pi.z};
    const float4 vi4 = d.vr4[i];
    const float vi[3] = {vi4.x, vi4.y, vi4.z};
    const float rho_i = vi4.w;
    float a[3] = {0.f, 0.f, 0.f};
    auto fn = [&](int wall, unsigned j, float rx, float ry, float rz) {
      const float r2 = rx * rx + ry * ry + rz * rz;
      float vj[3] = {0.f, 0.f, 0.f};
      float rho_j = rho_i;
      if (!wall) {
        const float4 v = SPHBUF_LDG(d.vr4 + j);
        vj[0] = v.x, vj[1] = v.y, vj[2] = v.z;
        rho_j = v.w;
      }
      viscous_term(P, wall, rx, ry, rz, r2, vi, rho_i, vj, rho_j, a);
    };
    if (cnt <= cap) {
      for_each_listed<D>(d, i, cnt, __float_as_uint(pi.w), fi, fn);
    } else {
      int c[3];
      cell_coords(d.A.cell[i], d.g, c);
      for_each_near<D>(d, c, fi, [&](int wall, unsigned j, float rx, float ry, float rz) {
        const float r2 = rx * rx + ry * ry + rz * rz;
        if (r2 < P.two_h_sq && r2 > 0.f) fn(wall, j, rx, ry, rz);
      });
    }
    d.av[i] = make_float4(a[0], a[1], a[2], 0.f);
  }
}

// Acoustic step sub (0-based) of the advection step: reads state sub % 2, writes the other.
template <int D>
__device__ __forceinline__ void acoustic_body(const DomainDev& d, unsigned bid, unsigned nblk, int sub) {
  if (d.st->status) return;
  const unsigned n = d.st->n;
  const Phys P = d.P;
  Phys Pp = P;
  Pp.eta = 0.f;  // pressure part only (the viscous one is in av)
  const float4* pc = (sub & 1) ? d.pos_b : d.pos4;
  const float4* sc = (sub & 1) ? d.vr_b : d.vr4;
  float4* pn = (sub & 1) ? d.pos4 : d.pos_b;
  float4* sn = (sub & 1) ? d.vr4 : d.vr_b;
  const float dt = P.dt_ac;
  const float inv_n = 1.f / (float)P.dual_n;
  const Grid& g = d.g;
  const int cap = d.nb_cap;
  for (unsigned i = bid * blockDim.x + threadIdx.x; i < n; i += nblk * blockDim.x) {
    int cnt = (int)d.nb_cnt[i];
    if (cnt > cap) {
      // an overflowed list has no fixed configuration for the acoustic steps
      latch(d.st, 2 /* SPHBUF_ERR_CAPACITY */);
      cnt = cap;
    }
    const float4 pi = pc[i];
    const float fi[3] = {pi.x, pi.y, pi.z};
    const float cxf = pi.w;  // the packed cell, carried over to the next acoustic state
    const unsigned ci = __float_as_uint(pi.w);
    const float4 si = sc[i];
    const float vi[3] = {si.x, si.y, si.z};
    const float rho_i = si.w;
    const float p_i = P.c0sq * (rho_i - P.rho0) + P.p_bg;
    const uint8_t lab = d.A.label[i];
    const float pb2 = boundary_pressure2(d, lab, p_i);
    float a[3] = {0.f, 0.f, 0.f}, tb[3] = {0.f, 0.f, 0.f};
    float srho = 0.f;
    const uint4* lst = reinterpret_cast<const uint4*>(d.nb + (size_t)i * d.nb_cap);
    auto one = [&](unsigned ent) {
      const unsigned j = ent & 0x7FFFFFFFu;
      const int wall = (int)(ent >> 31);
      const float4 p = wall ? SPHBUF_LDG(d.wpos4 + j) : pc[j];
      const unsigned cj = __float_as_uint(p.w);
      const float rx = fi[0] - p.x - (packed_cx(cj) - packed_cx(ci)) * g.cs;
      const float ry = fi[1] - (packed_cyf(cj) - packed_cyf(ci)) * g.cs - p.y;
      const float rz = (D == 3) ? fi[2] - (packed_czf(cj) - packed_czf(ci)) * g.cs - p.z : 0.f;
      const float r2 = rx * rx + ry * ry + rz * rz;
      float vj[3] = {0.f, 0.f, 0.f};
      float rho_j = rho_i;
      if (!wall) {
        const float4 v = sc[j];
        vj[0] = v.x, vj[1] = v.y, vj[2] = v.z;
        rho_j = v.w;
      }
      force_term<false>(Pp, wall, rx, ry, rz, r2, vi, rho_i, p_i, pb2, vj, rho_j, a, tb);
      srho += density_term<D>(P, true, wall, rx, ry, rz, sqrtf(r2), vi, rho_i, p_i, vj, rho_j);
    };
    for (int e = 0; e < cnt; e += 4) {
      const uint4 q = SPHBUF_LDG(lst + (e >> 2));
      one(q.x);
      if (e + 1 < cnt) one(q.y);
      if (e + 2 < cnt) one(q.z);
      if (e + 3 < cnt) one(q.w);
    }
    const float4 av = d.av[i];
    float v[3] = {vi[0] + dt * (a[0] + av.x), vi[1] + dt * (a[1] + av.y), D == 3 ? vi[2] + dt * (a[2] + av.z) : 0.f};
    if (lab != 0) {
      const int k = (int)lab - 1;
      const BufDev& b = d.bufs[k];
      int c[3];
      cell_coords(d.A.cell[i], g, c);
      if (b.vel_bc) {
        float X[3];
        local_coords<D>(b, c, fi, g.cs, X, D);
        float rr = X[1] * X[1];
        if (D == 3) rr += X[2] * X[2];
        const float prof = b.inv_hw2 > 0.f ? b.umax * fmaxf(1.f - rr * b.inv_hw2, 0.f) : b.umax;
#pragma unroll
        for (int x = 0; x < D; ++x) v[x] = prof * b.u[x];
      } else {
        float vn = v[0] * b.u[0] + v[1] * b.u[1];
        if (D == 3) vn += v[2] * b.u[2];
#pragma unroll
        for (int x = 0; x < D; ++x) v[x] = vn * b.u[x];
      }
      float vn = v[0] * b.u[0] + v[1] * b.u[1];
      if (D == 3) vn += v[2] * b.u[2];
      atomicAdd(reinterpret_cast<unsigned long long*>(&d.st->flux_fx[k]),
                (unsigned long long)__double2ll_rn((double)(vn * b.flux_scale * inv_n) * kFluxScale));
    }
    const float rho_n = rho_i + dt * (2.f * rho_i * srho);
    float f[3];
#pragma unroll
    for (int x = 0; x < 3; ++x) f[x] = x < D ? __fadd_rn(fi[x], __fmul_rn(v[x], dt)) : 0.f;
    pn[i] = make_float4(f[0], f[1], f[2], cxf);
    sn[i] = make_float4(v[0], v[1], v[2], rho_n);
  }
}

// After the acoustic steps: offsets folded back into [0, cs), the particles written to B.
template <int D>
__device__ __forceinline__ void dual_finish_body(const DomainDev& d, unsigned bid, unsigned nblk, bool fused) {
  if (d.st->status) return;
  const unsigned n = d.st->n;
  const bool odd = d.P.dual_n & 1;
  const float4* pc = odd ? d.pos_b : d.pos4;
  const float4* sc = odd ? d.vr_b : d.vr4;
  const float zero[3] = {0.f, 0.f, 0.f};
  for (unsigned i = bid * blockDim.x + threadIdx.x; i < n; i += nblk * blockDim.x) {
    int c[3];
    cell_coords(d.A.cell[i], d.g, c);
    const float4 p = pc[i];
    const float4 s = sc[i];
    const float f[3] = {p.x, p.y, p.z};
    const float v[3] = {s.x, s.y, s.z};
    drift_store<D>(d, fused, i, n, c, f, v, zero, s.w, d.A.label[i]);
  }
}

}  // namespace

}  // namespace sphbuf
