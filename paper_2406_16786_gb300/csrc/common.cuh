// Shared device-side definitions of the sphbuf library (GB300, sm_103a).
//
// Data layout in HBM (structure of arrays, one array per field, capacity-sized):
//   cell  int32   linear cell index (cz * ny + cy) * nx + cx, cell size cs = 2h
//   f[d]  float   offset inside the cell, [0, cs32)
//   v[d]  float   velocity
//   rho   float   density
//   id    uint32  particle id
//   label uint8   0 fluid, k + 1 buffer k, 255 dead (dropped by the next rebuild)
// Two copies exist: A (sorted by (cell, id), read by the neighbour passes) and B (written
// by the force/drift pass in A's order; new particles are appended; the rebuild sorts B
// back into A).  Walls are a third, static, sorted set with their own cell_start.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

// Loads of data written by an earlier launch: the read-only data path (__ldg).  A translation
// unit whose kernel also writes that data in the same launch (the persistent batched step)
// defines SPHBUF_LDG as a coherent load before including the kernel bodies.
#ifndef SPHBUF_LDG
#define SPHBUF_LDG(p) __ldg(p)
#endif

namespace sphbuf {

constexpr int kMaxBuffers = 32;
constexpr int kRangeCopies = 64;  // copies of the drift-velocity range (StepState::v_hi, v_lo)
constexpr uint8_t kDead = 255;
constexpr unsigned kNoSlot = 0xFFFFFFFFu;
constexpr int kScanItems = 16;      // cells per thread in the scan kernels
constexpr int kScanThreads = 256;
constexpr int kScanTile = kScanItems * kScanThreads;

enum Kind : int { KIND_INFLOW = 0, KIND_OUTFLOW = 1, KIND_BIDIR = 2 };

// Per-buffer constants (FP32 copies follow the header's FP32 decision contract).
struct BufDev {
  int kind;
  int vel_bc;          // 1 velocity BC, 0 pressure BC
  int label;           // k + 1
  int cO[3];
  float fO[3];
  float R[3][3];
  float ha, hb, hc;    // a/2, b/2, c/2
  float da, db, dc;    // a/2 + cs, b/2 + cs, c/2 + cs (outflow candidate region)
  float shift[3];      // fl32(-a R[0][x]): recycling move
  float u[3];          // FP32 boundary normal R^T e_x
  float umax, inv_hw2; // velocity profile; inv_hw2 = 1/R^2, 0 = plug
  float flux_scale;    // dp^d / a
  int box_lo[3], box_hi[3];  // cell-coordinate bounds containing the box (relabel prefilter)
  double p_b0, p_amp, p_omega, p_phase;
  // time-varying frame (Sec. 5.3): the buffer's particles turn by M32 about the pivot
  // (cC, fC) after each buffer update; the frame fields above are re-derived every step
  int rotating;
  int cC[3];
  float fC[3];
  float M32[3][3];
  // RCR Windkessel pressure (Eq. (31)) instead of p_b(t): parameters R_p, C, R_d
  int wk;
  double wk_rp, wk_c, wk_rd;
};

// Volume fluxes are summed as 64-bit fixed-point integers (unit 2^-50 m^d/s): integer
// atomics make the sum independent of the order of the additions.
constexpr double kFluxScale = 1125899906842624.0;     // 2^50
constexpr double kFluxUnit = 1.0 / 1125899906842624.0;  // 2^-50

// FP64 state of a rotating buffer's frame (Sec. 5.3): Q_n = M Q_{n-1}, R_n = R_0 Q_n^T,
// O'_n = C + Q_n (O'_0 - C).
struct RotDev {
  double M[9];   // rotation by omega dt (row-major)
  double Q[9];   // accumulated rotation of the current step
  double C[3];   // pivot
  double O0[3];  // origin at step 0
  double R0[9];  // frame at step 0
  double a;      // extent along X' (recycling shift)
};

// FP64 arithmetic without contraction, identical on host and device (the host code is
// compiled with -ffp-contract=off; device code uses the round-to-nearest intrinsics).
#ifdef __CUDA_ARCH__
#define SPHBUF_DMUL(a, b) __dmul_rn((a), (b))
#define SPHBUF_DADD(a, b) __dadd_rn((a), (b))
#define SPHBUF_DSUB(a, b) __dsub_rn((a), (b))
#define SPHBUF_DDIV(a, b) __ddiv_rn((a), (b))
#else
#define SPHBUF_DMUL(a, b) ((a) * (b))
#define SPHBUF_DADD(a, b) ((a) + (b))
#define SPHBUF_DSUB(a, b) ((a) - (b))
#define SPHBUF_DDIV(a, b) ((a) / (b))
#endif

// The frame-dependent FP32 constants of the decision contract from an FP64 frame (origin O,
// row-major R): cO = floor((O - lo) / cs), fO = fl((O - lo) - cO cs), R32 = fl(R),
// shift = fl(-a R[0][x]), u = fl(R[0][x]).
__host__ __device__ inline void frame_constants(BufDev& v, const double O[3], const double R[9], double a,
                                                const double lo[3], double cs, int D) {
  for (int x = 0; x < 3; ++x) {
    v.cO[x] = 0;
    v.fO[x] = 0.f;
    if (x < D) {
      const double t = SPHBUF_DSUB(O[x], lo[x]);
      const double c = floor(SPHBUF_DDIV(t, cs));
      v.cO[x] = (int)c;
      v.fO[x] = (float)SPHBUF_DSUB(t, SPHBUF_DMUL(c, cs));
    }
  }
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) v.R[r][c] = (float)R[3 * r + c];
  for (int x = 0; x < 3; ++x) {
    v.shift[x] = x < D ? (float)SPHBUF_DMUL(-a, R[x]) : 0.f;
    v.u[x] = x < D ? (float)R[x] : 0.f;
  }
}

// Frame of the current step from the rotation state (module header order).
__host__ __device__ inline void rotated_frame(const RotDev& q, double O[3], double R[9]) {
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c)
      R[3 * r + c] = SPHBUF_DADD(SPHBUF_DADD(SPHBUF_DMUL(q.R0[3 * r], q.Q[3 * c]), SPHBUF_DMUL(q.R0[3 * r + 1], q.Q[3 * c + 1])),
                                 SPHBUF_DMUL(q.R0[3 * r + 2], q.Q[3 * c + 2]));
  const double d0 = SPHBUF_DSUB(q.O0[0], q.C[0]), d1 = SPHBUF_DSUB(q.O0[1], q.C[1]), d2 = SPHBUF_DSUB(q.O0[2], q.C[2]);
  for (int x = 0; x < 3; ++x)
    O[x] = SPHBUF_DADD(q.C[x], SPHBUF_DADD(SPHBUF_DADD(SPHBUF_DMUL(q.Q[3 * x], d0), SPHBUF_DMUL(q.Q[3 * x + 1], d1)),
                                           SPHBUF_DMUL(q.Q[3 * x + 2], d2)));
}

// Q <- M Q (module header order).
__host__ __device__ inline void advance_rotation(RotDev& q) {
  double T[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c)
      T[3 * r + c] = SPHBUF_DADD(SPHBUF_DADD(SPHBUF_DMUL(q.M[3 * r], q.Q[c]), SPHBUF_DMUL(q.M[3 * r + 1], q.Q[3 + c])),
                                 SPHBUF_DMUL(q.M[3 * r + 2], q.Q[6 + c]));
  for (int e = 0; e < 9; ++e) q.Q[e] = T[e];
}

// Cell coordinates packed into 32 bits (x: bits 0-10, y: bits 11-21, z: bits 22-31), carried
// as the .w word of the position copies the neighbour passes read (pos4, wpos4): the geometry
// of a listed pair comes from both particles' own cells, so a list entry holds only the index.
// Grids are therefore limited to 2048 x 2048 x 1024 cells.
constexpr int kMaxCellsX = 2048, kMaxCellsY = 2048, kMaxCellsZ = 1024;
__host__ __device__ inline unsigned pack_cell(int cx, int cy, int cz) {
  return (unsigned)cx | ((unsigned)cy << 11) | ((unsigned)cz << 22);
}
// x of a packed cell as a float (exact: the 11 bits placed in the mantissa of 2^23, minus 2^23)
__device__ __forceinline__ float packed_cx(unsigned pc) {
  return __int_as_float(0x4B000000 | (int)(pc & 0x7FFu)) - 8388608.f;
}
// Order-preserving unsigned key of a float (and back): keys compare like the values.
__device__ __forceinline__ unsigned float_to_key(float v) {
  const unsigned b = __float_as_uint(v);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key_to_float(unsigned k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}
// y and z likewise (exact; no integer-to-float conversion)
__device__ __forceinline__ float packed_cyf(unsigned pc) {
  return __int_as_float(0x4B000000 | (int)((pc >> 11) & 0x7FFu)) - 8388608.f;
}
__device__ __forceinline__ float packed_czf(unsigned pc) {
  return __int_as_float(0x4B000000 | (int)(pc >> 22)) - 8388608.f;
}

struct Grid {
  int dim;
  int nx, ny, nz;
  long long ncell;
  float cs;  // cs32
};

struct Phys {
  float h, inv_h, two_h_sq, alpha, rho0, c0, c0sq, eta, mass, dt, inv_sum_w0, w_self;
  float p_bg;  // background pressure of the EoS: p = c0^2 (rho - rho0) + p_bg
  float tvf_lambda;  // transport velocity (Eq. (10)): p_max = lambda rho0 v_max^2; 0 = off
  float psi_cand;    // boundary candidates: position divergence below 0.75 d (reading A27)
  float vol;         // particle volume dp^d
  float dt_ac;       // acoustic step of the dual-criteria scheme (dt / dual_n)
  int dual_n;        // acoustic steps per advection step; 0 = single-rate kick-drift
  // neighbour lists kept over steps (0 = rebuilt every step): lists hold the pairs within
  // list_r2 = (2h + skin)^2 and are rebuilt when twice the largest displacement since the last
  // full build (relative to a reference velocity) exceeds the skin, or after reuse_max steps
  int reuse;
  float list_r2, skin;
  int reuse_max;
  double rho0_d, c0sq_d, dt_d, p_bg_d;
  double lo_d[3], cs_d;  // grid origin and cell size in FP64 (frames of rotating buffers)
  unsigned capacity;
  unsigned list_cap;
};

// Device-resident step bookkeeping (one per domain).
struct StepState {
  unsigned n;          // particles in the sorted arrays (A)
  unsigned n_inj;      // injections of the current step
  unsigned n_del;      // deletions of the current step
  unsigned next_id;
  unsigned n_occ;      // occupied cells of the current cell-linked list
  unsigned n_defer;    // particles deferred by the fluid density pass this step
  unsigned long long step;
  int status;          // latched error code (sphbuf_status), 0 = OK
  unsigned long long escaped_total;
  unsigned long long injected[kMaxBuffers];
  unsigned long long deleted[kMaxBuffers];
  float pb[kMaxBuffers];      // p_b(t_n)
  float rho_pb[kMaxBuffers];  // fl32(rho0 + p_b(t_n) / c0^2)
  long long flux_fx[kMaxBuffers];  // volume flux through buffer k in the current step (fixed point)
  double flux_last[kMaxBuffers];   // flux of the previous step (the one p_b(t_n) used)
  double pb_d[kMaxBuffers];        // p_b(t_n) in FP64
  double wk_pd[kMaxBuffers];       // Windkessel distal pressure P_d (Eq. (31) split)
  unsigned vmax_bits;              // largest particle speed of the current force pass (float bits)
  float p_max;                     // Eq. (10) background pressure of the current step
  // kept neighbour lists: full = the last rebuild sorted the state (its next step searches
  // every particle's neighbours); otherwise the slots kept their order, dead particles their
  // slots, and the index list `order` holds the live particles sorted by (cell, id)
  int full;
  unsigned n_live;                 // live particles (n counts slots)
  unsigned path_bits;              // largest |disp| of this step's drift (float bits)
  // reference velocity of the current reuse period, and the range of the drift velocities
  // seen in it (order-preserving keys, both maximised from 0: hi = key(v), lo = ~key(v))
  float u0[3];
  unsigned v_hi[kRangeCopies][3], v_lo[kRangeCopies][3];  // copies that spread the atomics
  unsigned since_full;             // steps since the last full build
  unsigned long long list_builds;  // full builds so far
  // dynamic share-out of the neighbour (0) and force (1) passes: the next chunk to take and
  // the blocks done; zero between launches (the last block of a launch resets them)
  unsigned sched[2];
  unsigned sched_done[2];
};

struct Particles {
  int* cell;
  float* f[3];
  float* v[3];
  float* rho;
  unsigned* id;
  uint8_t* label;
  // boundary identification of the transport velocity (reading A27), set by the last force
  // pass with the transport velocity: bit 0 candidate, bit 1 set (a previous step exists),
  // bit 2 core, bit 3 boundary particle
  uint8_t* bflag;
};

struct Walls {
  const int* cell;
  const float* f[3];
  const unsigned* start;  // wall cell_start[ncell + 1]
};

// Decision list entry: buffer k, particle index in B, particle id; for injections also the
// parent's state before recycling (the duplicate's state).
struct Decision {
  unsigned k;
  unsigned idx;
  unsigned id;
  int cell;
  float f[3];
  float v[3];
  float rho;
};

struct InjRecord {
  unsigned k;
  unsigned parent;
  unsigned child;
};

__device__ __forceinline__ void latch(StepState* st, int code) { atomicCAS(&st->status, 0, code); }

__device__ __forceinline__ void cell_coords(int lin, const Grid& g, int c[3]) {
  c[0] = lin % g.nx;
  int t = lin / g.nx;
  c[1] = t % g.ny;
  c[2] = t / g.ny;
}

// FP32 move + fold of the decision contract: f <- fl(f + delta), then at most 8 folds.
// Returns false for a non-finite result.
__device__ __forceinline__ bool move_fold(float& f, int& c, float delta, float cs) {
  f = __fadd_rn(f, delta);
#pragma unroll 1
  for (int it = 0; it < 8; ++it) {
    if (f >= cs) {
      f = __fadd_rn(f, -cs);
      c += 1;
    } else if (f < 0.f) {
      f = __fadd_rn(f, cs);
      c -= 1;
    } else {
      break;
    }
  }
  return isfinite(f);
}

// The cell part of X - O' in the contract's FP32 order: fl(fl(c - cO) cs) per axis.
template <int D>
__device__ __forceinline__ void cell_part(const BufDev& b, const int c[3], float cs, float cp[3]) {
#pragma unroll
  for (int x = 0; x < 3; ++x) cp[x] = x < D ? __fmul_rn(__int2float_rn(c[x] - b.cO[x]), cs) : 0.f;
}

// X' = R (X - O') rows [0, nrow) from the cell part cp and the offset f:
// Delta = fl(cp + fl(f - fO)), X'_r = fl(fl(fl(R_r0 Delta_0) + fl(R_r1 Delta_1)) + fl(R_r2 Delta_2)).
template <int D>
__device__ __forceinline__ void local_from_part(const BufDev& b, const float cp[3], const float f[3], float X[3],
                                                int nrow) {
  float Dl[3];
#pragma unroll
  for (int x = 0; x < D; ++x) Dl[x] = __fadd_rn(cp[x], __fadd_rn(f[x], -b.fO[x]));
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    if (r >= D || r >= nrow) break;
    float acc = __fmul_rn(b.R[r][0], Dl[0]);
    acc = __fadd_rn(acc, __fmul_rn(b.R[r][1], Dl[1]));
    if (D == 3) acc = __fadd_rn(acc, __fmul_rn(b.R[r][2], Dl[2]));
    X[r] = acc;
  }
}

// Local coordinates X' = R (X - O') in the contract's FP32 order, rows [0, nrow).
template <int D>
__device__ __forceinline__ void local_coords(const BufDev& b, const int c[3], const float f[3],
                                             float cs, float X[3], int nrow) {
  float Dl[3];
#pragma unroll
  for (int x = 0; x < D; ++x)
    Dl[x] = __fadd_rn(__fmul_rn(__int2float_rn(c[x] - b.cO[x]), cs), __fadd_rn(f[x], -b.fO[x]));
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    if (r >= D || r >= nrow) break;
    float acc = __fmul_rn(b.R[r][0], Dl[0]);
    acc = __fadd_rn(acc, __fmul_rn(b.R[r][1], Dl[1]));
    if (D == 3) acc = __fadd_rn(acc, __fmul_rn(b.R[r][2], Dl[2]));
    X[r] = acc;
  }
}

template <int D>
__device__ __forceinline__ bool in_box(const BufDev& b, const float X[3]) {
  bool in = fabsf(X[0]) < b.ha && fabsf(X[1]) < b.hb;
  if (D == 3) in = in && fabsf(X[2]) < b.hc;
  return in;
}

// Wendland C2: W = alpha (1 - q/2)^4 (2q + 1); dW/dr = -(5 alpha / h) q (1 - q/2)^3.
__device__ __forceinline__ float kernel_w(float q, const Phys& P) {
  float t = fmaxf(1.f - 0.5f * q, 0.f);
  float t2 = t * t;
  return P.alpha * t2 * t2 * (2.f * q + 1.f);
}
__device__ __forceinline__ float kernel_dw(float q, const Phys& P) {
  float t = fmaxf(1.f - 0.5f * q, 0.f);
  return -5.f * P.alpha * P.inv_h * q * t * t * t;
}

}  // namespace sphbuf
