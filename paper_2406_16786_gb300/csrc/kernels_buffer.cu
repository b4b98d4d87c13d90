// The arbitrary-positioned buffer (Sec. 3, Algorithms 1-3) on the GPU as a launch of its own:
// the form for rotating buffers (Sec. 5.3), for the all-particle check and on request; by
// default the decisions are fused into the drift (decide.cuh).
//
// Only the particles listed in the cells around each buffer's box are visited (four candidate
// cells per warp, eight lanes per cell, four particles per lane loaded before any is tested;
// the cells' particle ranges come from the last rebuild).  Each is transformed into
// the buffer's local frame (Eqs. (11), (15)) with the FP32 decision contract and compared on
// the normal axis only.  Crossings are compacted with a warp ballot: each warp with crossings
// reserves its range of the step's global lists with one atomic per list and its lanes write
// their records at once.  The deciding thread does everything that does not depend on the
// order of the injections: it writes the duplicate (the parent's state before recycling,
// label 0) at the tail of B, recycles the parent by -a u (Eqs. (16)-(17)), resets its density
// for pressure buffers (Eq. (22)) and marks deleted particles dead.  The ids of the
// duplicates follow the (buffer, parent id) order and are assigned by the first pass of the
// rebuild (rank_injections, in apply.cuh), which needs every decision of the step.
// The full-domain variant takes the same decisions over every particle and every buffer.
#include "decide.cuh"

namespace sphbuf {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kBufThreads = 256;

// What the test of one particle of B needs (its id, velocity and density are read only when
// it crossed a face).
struct Cand {
  uint8_t lab;
  int cell;
  float f[3];
};

template <int D>
__device__ __forceinline__ void load_cand(const DomainDev& d, unsigned i, bool ok, Cand& p) {
  p.lab = kDead;
  p.cell = 0;
#pragma unroll
  for (int x = 0; x < 3; ++x) p.f[x] = 0.f;
  if (!ok) return;
  p.lab = d.B.label[i];
  p.cell = d.B.cell[i];
#pragma unroll
  for (int x = 0; x < D; ++x) p.f[x] = d.B.f[x][i];
}

// The buffers' constants and this step's recycled density, in shared memory.
struct BlockShared {
  BufDev bufs[kMaxBuffers];
  float rho_pb[kMaxBuffers];
  unsigned n, bad;
};

// Algorithms 1-3 for particle i of B (test state p) against buffer k; the warp stages the
// decisions.  (lin_c, c_c, cp_c): a cell, its coordinates and its cell part for buffer k,
// used when the particle is still in that cell (the cell it was sorted into).  A particle of
// a rotating inflow buffer then turns with the buffer about its pivot (Sec. 5.3), after any
// recycling: positions in the FP32 contract (offset from the pivot, rotated row by row, moved
// by the difference), velocities rotated row by row.  ROT: some buffer of the domain rotates
// (the turn is compiled out otherwise).
template <int D, bool ROT>
__device__ __forceinline__ void decide(const DomainDev& d, BlockShared& sm, int k, unsigned i, const Cand& p, int lin_c,
                                       const int c_c[3], const float cp_c[3]) {
  const BufDev& b = sm.bufs[k];
  const Grid& g = d.g;
  bool inj = false, del = false;
  int c[3] = {c_c[0], c_c[1], c_c[2]};
  const bool test = (b.kind == KIND_OUTFLOW) ? (p.lab != kDead) : (p.lab == (uint8_t)b.label);
  if (test) {
    float cp[3] = {cp_c[0], cp_c[1], cp_c[2]};
    if (p.cell != lin_c) {
      cell_coords(p.cell, g, c);
      cell_part<D>(b, c, g.cs, cp);
    }
    float X[3];
    if (b.kind == KIND_OUTFLOW) {
      // Algorithm 2: candidates within one cell of the box, deleted once X' > a/2
      local_from_part<D>(b, cp, p.f, X, D);
      bool cand = fabsf(X[0]) < b.da && fabsf(X[1]) < b.db;
      if (D == 3) cand = cand && fabsf(X[2]) < b.dc;
      del = cand && X[0] > b.ha;
    } else {
      // Algorithms 1 and 3: buffer particles crossing X' = a/2 generate; Algorithm 3 deletes
      // those crossing X' = -a/2
      local_from_part<D>(b, cp, p.f, X, 1);
      inj = X[0] > b.ha;
      if (b.kind == KIND_BIDIR) del = X[0] < -b.ha;
    }
  }
  const bool rot = ROT && test && b.rotating;
  if (!__any_sync(kFull, inj || del || rot)) return;
  Decision rec;
  rec.k = (unsigned)k;
  rec.idx = i;
  rec.id = 0;
  rec.cell = p.cell;
  rec.rho = 0.f;
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    rec.f[x] = p.f[x];
    rec.v[x] = 0.f;
  }
  if (inj || del) rec.id = d.B.id[i];
  if (inj || rot) {
#pragma unroll
    for (int x = 0; x < D; ++x) rec.v[x] = d.B.v[x][i];
  }
  if (inj) rec.rho = d.B.rho[i];
  stage<D, true>(d, kFull, sm.n, inj, rec);
  float fw[3] = {p.f[0], p.f[1], p.f[2]};
  bool ok = true;
  if (inj) {
    // recycle the parent: r' - [a, 0, 0]^T mapped back, i.e. r - a u (after the record
    // captured the duplicate's state)
#pragma unroll
    for (int x = 0; x < D; ++x) ok &= move_fold(fw[x], c[x], b.shift[x], g.cs);
  }
  if (ROT && rot) {
    float Dv[3] = {0.f, 0.f, 0.f}, Dn[3], vn[3];
#pragma unroll
    for (int x = 0; x < D; ++x)
      Dv[x] = __fadd_rn(__fmul_rn(__int2float_rn(c[x] - b.cC[x]), g.cs), __fadd_rn(fw[x], -b.fC[x]));
#pragma unroll
    for (int r = 0; r < D; ++r) {
      float acc = __fmul_rn(b.M32[r][0], Dv[0]);
      float vac = __fmul_rn(b.M32[r][0], rec.v[0]);
      acc = __fadd_rn(acc, __fmul_rn(b.M32[r][1], Dv[1]));
      vac = __fadd_rn(vac, __fmul_rn(b.M32[r][1], rec.v[1]));
      if (D == 3) {
        acc = __fadd_rn(acc, __fmul_rn(b.M32[r][2], Dv[2]));
        vac = __fadd_rn(vac, __fmul_rn(b.M32[r][2], rec.v[2]));
      }
      Dn[r] = acc;
      vn[r] = vac;
    }
#pragma unroll
    for (int x = 0; x < D; ++x) {
      ok &= move_fold(fw[x], c[x], __fadd_rn(Dn[x], -Dv[x]), g.cs);
      d.B.v[x][i] = vn[x];
    }
  }
  if (inj || rot) {
#pragma unroll
    for (int x = 0; x < D; ++x) d.B.f[x][i] = fw[x];
    const bool inside = ok && c[0] >= 0 && c[0] < g.nx && c[1] >= 0 && c[1] < g.ny && c[2] >= 0 && c[2] < g.nz;
    if (inside) {
      d.B.cell[i] = (c[2] * g.ny + c[1]) * g.nx + c[0];
    } else {
      d.B.label[i] = kDead;
      atomicAdd(&d.st->escaped_total, 1ull);
    }
  }
  if (inj && !b.vel_bc) d.B.rho[i] = sm.rho_pb[k];  // Eq. (22)
  if (del) d.B.label[i] = kDead;
  stage<D, false>(d, kFull, sm.n, del, rec);
}

// Decisions (restricted to candidate cells, or over all particles), then the block's lists
// and duplicates.  CPW: candidate cells per warp (the cell tile), 32 / CPW lanes per cell.
template <int D, bool FULL, bool ROT, int CPW>
__device__ __forceinline__ void buffer_body(const DomainDev& d, unsigned bid, unsigned nblk) {
  static_assert(CPW == 1 || CPW == 2 || CPW == 4 || CPW == 8, "cells per warp");
  constexpr unsigned L = 32 / CPW;  // lanes per cell
  __shared__ BlockShared sm;
  const int lane = threadIdx.x & 31;
  const unsigned warp = (bid * blockDim.x + threadIdx.x) >> 5;
  const unsigned nwarps = (nblk * blockDim.x) >> 5;
  // CPW candidate cells per warp, L lanes per cell; the first cells' particle ranges are
  // requested before the block copies the buffers' constants
  const unsigned grp = lane / L, gl = lane % L;
  const unsigned nseg = (unsigned)d.nseg;
  unsigned s0 = warp * CPW;
  uint4 r = make_uint4(0, 0, 0, 0);  // (first particle, end, cell, buffer)
  if constexpr (!FULL) {
    if (s0 + grp < nseg) r = d.seg_range[s0 + grp];
  }
  if (threadIdx.x == 0) {
    sm.n = d.st->n;
    sm.bad = d.st->status != 0;
  }
  {
    const int words = d.nbuf * (int)(sizeof(BufDev) / sizeof(int));
    const int* src = reinterpret_cast<const int*>(d.bufs);
    int* dst = reinterpret_cast<int*>(sm.bufs);
    for (int w = threadIdx.x; w < words; w += blockDim.x) dst[w] = src[w];
    if (threadIdx.x < (unsigned)d.nbuf) sm.rho_pb[threadIdx.x] = d.st->rho_pb[threadIdx.x];
  }
  __syncthreads();
  if (sm.bad) return;
  if constexpr (FULL) {
    const unsigned n = sm.n;
    for (unsigned base = warp * 32; base < n; base += nwarps * 32) {
      const unsigned i = base + lane;
      Cand p;
      load_cand<D>(d, i, i < n, p);
      const int none[3] = {0, 0, 0};
      const float zero[3] = {0.f, 0.f, 0.f};
      for (int kk = 0; kk < d.nbuf; ++kk) decide<D, ROT>(d, sm, kk, i, p, -1, none, zero);
    }
  } else {
    // four particles per lane are loaded before any is tested (cells of up to 4 L particles
    // take one pass)
    while (s0 < nseg) {
      const unsigned j0 = r.x, j1 = r.y;
      const int lin = (int)r.z, kc = (int)r.w;
      // next cells' ranges, requested before this group is tested
      const unsigned s1 = s0 + nwarps * CPW;
      r = make_uint4(0, 0, 0, 0);
      if (s1 + grp < nseg) r = d.seg_range[s1 + grp];
      // the cell's coordinates and cell part, shared by its particles that stayed in it
      int cc[3];
      float cp[3];
      cell_coords(lin, d.g, cc);
      cell_part<D>(sm.bufs[kc], cc, d.g.cs, cp);
      const unsigned passes = __reduce_max_sync(kFull, (j1 - j0 + 4 * L - 1) / (4 * L));
      for (unsigned it = 0; it < passes; ++it) {
        Cand p[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const unsigned i = j0 + it * 4 * L + q * L + gl;
          load_cand<D>(d, i, i < j1, p[q]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) decide<D, ROT>(d, sm, kc, j0 + it * 4 * L + q * L + gl, p[q], lin, cc, cp);
      }
      s0 = s1;
    }
  }
}

template <int D, bool FULL, bool ROT>
__global__ void __launch_bounds__(kBufThreads, 4) k_buffer(DomainDev d) {
  buffer_body<D, FULL, ROT, 4>(d, blockIdx.x, gridDim.x);
}

// batched: any block size up to 512 and a cell tile of CPW cells per warp (the autotuner's)
template <int D, bool FULL, bool ROT, int CPW>
__global__ void __launch_bounds__(512) k_buffer_batch(BatchDev b) {
  __shared__ DomainDev sd;
  const int4 m = b.map[blockIdx.x];
  load_domain(sd, b.doms + m.x);
  buffer_body<D, FULL, ROT, CPW>(sd, (unsigned)m.y, (unsigned)m.z);
}

template <int D>
__global__ void __launch_bounds__(256) k_identify(DomainDev d) {
  const unsigned n = d.st->n;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int c[3];
    cell_coords(d.B.cell[i], d.g, c);
    const float f[3] = {d.B.f[0][i], d.B.f[1][i], D == 3 ? d.B.f[2][i] : 0.f};
    uint8_t lab = d.B.label[i];
    for (int k = 0; k < d.nbuf; ++k) {
      const BufDev& b = d.bufs[k];
      if (b.kind != KIND_INFLOW) continue;
      float X[3];
      local_coords<D>(b, c, f, d.g.cs, X, D);
      if (in_box<D>(b, X)) lab = (uint8_t)b.label;
    }
    d.B.label[i] = lab;
  }
}

// Blocks of k_buffer resident at once (at most one wave: every block reserves its list ranges
// as soon as its own decisions end).
template <typename K>
int one_wave(const DomainDev& d, K kernel) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBufThreads, 0) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  return d.sm_count * per_sm;
}

}  // namespace

int launch_identify(const DomainDev& d, cudaStream_t s) {
  if (d.g.dim == 2)
    k_identify<2><<<d.sm_count * 8, 256, 0, s>>>(d);
  else
    k_identify<3><<<d.sm_count * 8, 256, 0, s>>>(d);
  return 1;
}

namespace {

template <int D, bool FULL, bool ROT>
void launch_decide_t(const DomainDev& d, cudaStream_t s) {
  const int wave = one_wave(d, k_buffer<D, FULL, ROT>);
  int blocks = wave;
  if (!FULL) {
    const int cells_per_block = 4 * (kBufThreads / 32);
    blocks = std::max(1, std::min(wave, (d.nseg + cells_per_block - 1) / cells_per_block));
  }
  k_buffer<D, FULL, ROT><<<blocks, kBufThreads, 0, s>>>(d);
}

template <int D, bool FULL, bool ROT>
void launch_batch_tile(const BatchDev& b, int nblocks, int threads, int cpw, cudaStream_t s) {
  switch (FULL ? 4 : cpw) {
    case 1:
      k_buffer_batch<D, FULL, ROT, 1><<<nblocks, threads, 0, s>>>(b);
      break;
    case 2:
      k_buffer_batch<D, FULL, ROT, 2><<<nblocks, threads, 0, s>>>(b);
      break;
    case 8:
      k_buffer_batch<D, FULL, ROT, 8><<<nblocks, threads, 0, s>>>(b);
      break;
    default:
      k_buffer_batch<D, FULL, ROT, 4><<<nblocks, threads, 0, s>>>(b);
  }
}

template <int D, bool FULL>
void launch_batch_t(const BatchDev& b, int nblocks, bool rot, int threads, int cpw, cudaStream_t s) {
  if (rot)
    launch_batch_tile<D, FULL, true>(b, nblocks, threads, cpw, s);
  else
    launch_batch_tile<D, FULL, false>(b, nblocks, threads, cpw, s);
}

}  // namespace

int launch_decide(const DomainDev& d, bool full_domain, cudaStream_t s) {
  const bool rot = d.any_rot != 0;
  if (d.g.dim == 2) {
    if (full_domain)
      rot ? launch_decide_t<2, true, true>(d, s) : launch_decide_t<2, true, false>(d, s);
    else
      rot ? launch_decide_t<2, false, true>(d, s) : launch_decide_t<2, false, false>(d, s);
  } else {
    if (full_domain)
      rot ? launch_decide_t<3, true, true>(d, s) : launch_decide_t<3, true, false>(d, s);
    else
      rot ? launch_decide_t<3, false, true>(d, s) : launch_decide_t<3, false, false>(d, s);
  }
  return 1;
}


int launch_batch_buffer(Kern k, int dim, const BatchDev& b, int nblocks, bool rot, int threads, int cpw,
                        cudaStream_t s) {
  if (k != K_BUFFER && k != K_BUFFER_FULL) return 0;
  const bool full = k == K_BUFFER_FULL;
  if (dim == 2)
    full ? launch_batch_t<2, true>(b, nblocks, rot, threads, cpw, s)
         : launch_batch_t<2, false>(b, nblocks, rot, threads, cpw, s);
  else
    full ? launch_batch_t<3, true>(b, nblocks, rot, threads, cpw, s)
         : launch_batch_t<3, false>(b, nblocks, rot, threads, cpw, s);
  return 1;
}

}  // namespace sphbuf
