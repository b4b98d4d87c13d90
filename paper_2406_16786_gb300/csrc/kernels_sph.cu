// WCSPH neighbour passes (Sec. 2, Sec. 4): density (Eq. (9) / Eq. (4)), force (Eqs. (5)-(8),
// (18)) fused with the kick, the boundary velocity (Eqs. (19), (23)-(26)) and the drift.
//
// One thread per particle of the sorted set A; neighbours come from the 3^d cells around the
// particle's cell, read as one contiguous range per (dy, dz) row (the three x-cells of a row
// are adjacent in the sorted order).  Wall neighbours use the static wall list.
//
// Wall neighbours carry the mirrored state of i (rho_j = rho_i, p_j = p_i, v_j = -v_i), the
// reading of the cited one-sided Riemann solver with no-slip walls.  The intermediate
// velocity of Eq. (4) is taken along -e_ij, consistent with U_L = -v_i . e_ij of Eq. (7):
// (v_i - v*) . e_ij = v_ij . e_ij / 2 + (p_i - p_j) / (2 rho_bar c0).
#include "kernels.cuh"

namespace sphbuf {

namespace {

// Step prologue, run by one thread of the step's first kernel: per-step constants.
__device__ void begin_step(const DomainDev& d) {
  StepState* st = d.st;
  st->n_inj = 0;
  st->n_del = 0;
  const double t = (double)st->step * d.P.dt_d;
  for (int k = 0; k < d.nbuf; ++k) {
    const BufDev& b = d.bufs[k];
    const double pb = b.p_b0 + b.p_amp * sin(b.p_omega * t + b.p_phase);
    st->pb[k] = (float)pb;
    st->rho_pb[k] = (float)(d.P.rho0_d + pb / d.P.c0sq_d);
    st->flux[k] = 0.0;
  }
}

// Calls fn(j, rx, ry, rz) for every sorted particle j in the 3^d cells around cell c of a
// particle at in-cell offset fi; (rx, ry, rz) = r_i - r_j.
template <int D, typename Fn>
__device__ __forceinline__ void for_each_fluid(const DomainDev& d, const int c[3], const float fi[3],
                                               Fn&& fn) {
  const Grid& g = d.g;
  const float cs = g.cs;
  const int x0 = max(c[0] - 1, 0), x1 = min(c[0] + 1, g.nx - 1);
  const int zlo = (D == 3) ? -1 : 0, zhi = (D == 3) ? 1 : 0;
  for (int dz = zlo; dz <= zhi; ++dz) {
    const int z = c[2] + dz;
    if (z < 0 || z >= g.nz) continue;
    for (int dy = -1; dy <= 1; ++dy) {
      const int y = c[1] + dy;
      if (y < 0 || y >= g.ny) continue;
      const int row = (z * g.ny + y) * g.nx;
      const unsigned j0 = __ldg(d.cell_start + row + x0);
      const unsigned j1 = __ldg(d.cell_start + row + x1 + 1);
      const float oy = fi[1] - (float)dy * cs;
      const float oz = (D == 3) ? fi[2] - (float)dz * cs : 0.f;
      for (unsigned j = j0; j < j1; ++j) {
        const int xj = __ldg(d.A.cell + j) - row;
        const float rx = fi[0] - __ldg(d.A.f[0] + j) - (float)(xj - c[0]) * cs;
        const float ry = oy - __ldg(d.A.f[1] + j);
        const float rz = (D == 3) ? oz - __ldg(d.A.f[2] + j) : 0.f;
        fn(j, rx, ry, rz);
      }
    }
  }
}

template <int D, typename Fn>
__device__ __forceinline__ void for_each_wall(const DomainDev& d, const int c[3], const float fi[3],
                                              Fn&& fn) {
  const Grid& g = d.g;
  const float cs = g.cs;
  const int x0 = max(c[0] - 1, 0), x1 = min(c[0] + 1, g.nx - 1);
  const int zlo = (D == 3) ? -1 : 0, zhi = (D == 3) ? 1 : 0;
  for (int dz = zlo; dz <= zhi; ++dz) {
    const int z = c[2] + dz;
    if (z < 0 || z >= g.nz) continue;
    for (int dy = -1; dy <= 1; ++dy) {
      const int y = c[1] + dy;
      if (y < 0 || y >= g.ny) continue;
      const int row = (z * g.ny + y) * g.nx;
      const unsigned j0 = __ldg(d.W.start + row + x0);
      const unsigned j1 = __ldg(d.W.start + row + x1 + 1);
      const float oy = fi[1] - (float)dy * cs;
      const float oz = (D == 3) ? fi[2] - (float)dz * cs : 0.f;
      for (unsigned j = j0; j < j1; ++j) {
        const int xj = __ldg(d.W.cell + j) - row;
        const float rx = fi[0] - __ldg(d.W.f[0] + j) - (float)(xj - c[0]) * cs;
        const float ry = oy - __ldg(d.W.f[1] + j);
        const float rz = (D == 3) ? oz - __ldg(d.W.f[2] + j) : 0.f;
        fn(j, rx, ry, rz);
      }
    }
  }
}

template <int D>
__global__ void __launch_bounds__(256) k_density(DomainDev d) {
  if (blockIdx.x == 0 && threadIdx.x == 0) begin_step(d);
  if (d.st->status) return;
  const unsigned n = d.st->n;
  const Phys P = d.P;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int c[3];
    cell_coords(d.A.cell[i], d.g, c);
    float fi[3] = {d.A.f[0][i], d.A.f[1][i], D == 3 ? d.A.f[2][i] : 0.f};
    const uint8_t lab = d.A.label[i];
    if (lab == 0) {
      // Eq. (9): rho0 sum_j W_ij / sum W0 (self included through j = i)
      float s = 0.f;
      auto add = [&](unsigned, float rx, float ry, float rz) {
        const float r2 = rx * rx + ry * ry + rz * rz;
        if (r2 < P.two_h_sq) s += kernel_w(sqrtf(r2) * P.inv_h, P);
      };
      for_each_fluid<D>(d, c, fi, add);
      for_each_wall<D>(d, c, fi, add);
      d.rho_new[i] = P.rho0 * s * P.inv_sum_w0;
    } else {
      // Eq. (4) for buffer particles: drho/dt = 2 rho_i sum_j m/rho_j (v_i - v*) . grad W
      const float vi[3] = {d.A.v[0][i], d.A.v[1][i], D == 3 ? d.A.v[2][i] : 0.f};
      const float rho_i = d.A.rho[i];
      const float p_i = P.c0sq * (rho_i - P.rho0);
      float acc = 0.f;
      for_each_fluid<D>(d, c, fi, [&](unsigned j, float rx, float ry, float rz) {
        const float r2 = rx * rx + ry * ry + rz * rz;
        if (r2 < P.two_h_sq && r2 > 0.f) {
          const float r = sqrtf(r2), inv_r = 1.f / r;
          const float vx = vi[0] - __ldg(d.A.v[0] + j), vy = vi[1] - __ldg(d.A.v[1] + j);
          const float vz = (D == 3) ? vi[2] - __ldg(d.A.v[2] + j) : 0.f;
          const float rho_j = __ldg(d.A.rho + j);
          const float p_j = P.c0sq * (rho_j - P.rho0);
          const float vij_e = (vx * rx + vy * ry + vz * rz) * inv_r;
          const float term = 0.5f * vij_e + (p_i - p_j) / ((rho_i + rho_j) * P.c0);
          acc += P.mass / rho_j * term * kernel_dw(r * P.inv_h, P);
        }
      });
      for_each_wall<D>(d, c, fi, [&](unsigned, float rx, float ry, float rz) {
        const float r2 = rx * rx + ry * ry + rz * rz;
        if (r2 < P.two_h_sq && r2 > 0.f) {
          const float r = sqrtf(r2), inv_r = 1.f / r;
          const float vi_e = (vi[0] * rx + vi[1] * ry + vi[2] * rz) * inv_r;  // mirrored: v_ij = 2 v_i
          acc += P.mass / rho_i * vi_e * kernel_dw(r * P.inv_h, P);
        }
      });
      d.rho_new[i] = rho_i + P.dt * (2.f * rho_i * acc);
    }
  }
}

// Drift + fold + escape check of the force/drift epilogue; writes B[i].
template <int D>
__device__ __forceinline__ void drift_store(const DomainDev& d, unsigned i, const int c[3], const float fi[3],
                                            const float v[3], float rho, uint8_t lab) {
  const Grid& g = d.g;
  int cn[3] = {c[0], c[1], c[2]};
  float fn[3] = {fi[0], fi[1], fi[2]};
  bool finite = true;
#pragma unroll
  for (int x = 0; x < D; ++x) finite &= move_fold(fn[x], cn[x], __fmul_rn(v[x], d.P.dt), g.cs);
  bool inside = cn[0] >= 0 && cn[0] < g.nx && cn[1] >= 0 && cn[1] < g.ny && cn[2] >= 0 && cn[2] < g.nz;
  if (!finite) {
    latch(d.st, 6 /* SPHBUF_ERR_NAN */);
    inside = false;
  }
  if (!inside && lab != kDead) {
    atomicAdd(&d.st->escaped_total, 1ull);
    lab = kDead;
  }
  const int lin = inside ? (cn[2] * g.ny + cn[1]) * g.nx + cn[0] : 0;
  d.B.cell[i] = lin;
#pragma unroll
  for (int x = 0; x < D; ++x) {
    d.B.f[x][i] = fn[x];
    d.B.v[x][i] = v[x];
  }
  d.B.rho[i] = rho;
  d.B.id[i] = d.A.id[i];
  d.B.label[i] = lab;
}

template <int D>
__global__ void __launch_bounds__(256) k_force(DomainDev d) {
  if (d.st->status) return;
  const unsigned n = d.st->n;
  const Phys P = d.P;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int c[3];
    cell_coords(d.A.cell[i], d.g, c);
    const float fi[3] = {d.A.f[0][i], d.A.f[1][i], D == 3 ? d.A.f[2][i] : 0.f};
    const float vi[3] = {d.A.v[0][i], d.A.v[1][i], D == 3 ? d.A.v[2][i] : 0.f};
    const uint8_t lab = d.A.label[i];
    const float rho_i = d.rho_new[i];
    const float p_i = P.c0sq * (rho_i - P.rho0);
    const int k = (int)lab - 1;
    // Eq. (18): boundary pressure p_b(t), or p_i for velocity buffers (Sec. 4.2)
    float pb2 = 0.f;
    if (lab != 0) pb2 = 2.f * (d.bufs[k].vel_bc ? p_i : d.st->pb[k]);
    float ax = 0.f, ay = 0.f, az = 0.f;
    const float two_eta = 2.f * P.eta;
    for_each_fluid<D>(d, c, fi, [&](unsigned j, float rx, float ry, float rz) {
      const float r2 = rx * rx + ry * ry + rz * rz;
      if (r2 < P.two_h_sq && r2 > 0.f) {
        const float r = sqrtf(r2), inv_r = 1.f / r;
        const float vx = vi[0] - __ldg(d.A.v[0] + j), vy = vi[1] - __ldg(d.A.v[1] + j);
        const float vz = (D == 3) ? vi[2] - __ldg(d.A.v[2] + j) : 0.f;
        const float rho_j = __ldg(d.rho_new + j);
        const float p_j = P.c0sq * (rho_j - P.rho0);
        const float dU = -(vx * rx + vy * ry + vz * rz) * inv_r;  // U_L - U_R
        const float beta = fminf(3.f * fmaxf(dU, 0.f), P.c0);
        const float pstar = 0.5f * (p_i + p_j) + 0.25f * beta * (rho_i + rho_j) * dU;
        const float dw = kernel_dw(r * P.inv_h, P);
        const float m_rr = P.mass / (rho_i * rho_j) * dw;
        const float ce = m_rr * (pb2 - 2.f * pstar) * inv_r;  // along r_ij (e_ij = r_ij / r)
        const float cv = m_rr * two_eta * inv_r;
        ax += ce * rx + cv * vx;
        ay += ce * ry + cv * vy;
        az += ce * rz + cv * vz;
      }
    });
    for_each_wall<D>(d, c, fi, [&](unsigned, float rx, float ry, float rz) {
      const float r2 = rx * rx + ry * ry + rz * rz;
      if (r2 < P.two_h_sq && r2 > 0.f) {
        const float r = sqrtf(r2), inv_r = 1.f / r;
        // mirrored wall state: v_ij = 2 v_i, rho_j = rho_i, p_j = p_i
        const float vx = 2.f * vi[0], vy = 2.f * vi[1], vz = 2.f * vi[2];
        const float dU = -(vx * rx + vy * ry + vz * rz) * inv_r;
        const float beta = fminf(3.f * fmaxf(dU, 0.f), P.c0);
        const float pstar = p_i + 0.5f * beta * rho_i * dU;
        const float dw = kernel_dw(r * P.inv_h, P);
        const float m_rr = P.mass / (rho_i * rho_i) * dw;
        const float ce = m_rr * (pb2 - 2.f * pstar) * inv_r;
        const float cv = m_rr * two_eta * inv_r;
        ax += ce * rx + cv * vx;
        ay += ce * ry + cv * vy;
        az += ce * rz + cv * vz;
      }
    });
    float v[3] = {vi[0] + ax * P.dt, vi[1] + ay * P.dt, D == 3 ? vi[2] + az * P.dt : 0.f};
    if (lab != 0) {
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
      atomicAdd(&d.st->flux[k], (double)(vn * b.flux_scale));
    }
    drift_store<D>(d, i, c, fi, v, rho_i, lab);
  }
}

template <int D>
__global__ void __launch_bounds__(256) k_drift(DomainDev d) {
  if (blockIdx.x == 0 && threadIdx.x == 0) begin_step(d);
  if (d.st->status) return;
  const unsigned n = d.st->n;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int c[3];
    cell_coords(d.A.cell[i], d.g, c);
    const float fi[3] = {d.A.f[0][i], d.A.f[1][i], D == 3 ? d.A.f[2][i] : 0.f};
    const float v[3] = {d.A.v[0][i], d.A.v[1][i], D == 3 ? d.A.v[2][i] : 0.f};
    drift_store<D>(d, i, c, fi, v, d.A.rho[i], d.A.label[i]);
  }
}

int grid_for(const DomainDev& d, int per_sm) { return d.sm_count * per_sm; }

}  // namespace

int launch_density(const DomainDev& d, cudaStream_t s) {
  if (d.g.dim == 2)
    k_density<2><<<grid_for(d, 4), 256, 0, s>>>(d);
  else
    k_density<3><<<grid_for(d, 4), 256, 0, s>>>(d);
  return 1;
}

int launch_force(const DomainDev& d, cudaStream_t s) {
  if (d.g.dim == 2)
    k_force<2><<<grid_for(d, 4), 256, 0, s>>>(d);
  else
    k_force<3><<<grid_for(d, 4), 256, 0, s>>>(d);
  return 1;
}

int launch_drift(const DomainDev& d, cudaStream_t s) {
  if (d.g.dim == 2)
    k_drift<2><<<grid_for(d, 8), 256, 0, s>>>(d);
  else
    k_drift<3><<<grid_for(d, 8), 256, 0, s>>>(d);
  return 1;
}

}  // namespace sphbuf
