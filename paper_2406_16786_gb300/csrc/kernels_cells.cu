// Cell-linked list rebuild (the end of each step, Sec. 3.1) as a counting sort, fused with the
// relabelling of outflow and bidirectional buffers (Algorithms 2-3, after the rebuild).
//
//   hist    slot_i = atomicAdd(count[cell_i], 1) for every live particle of B (the first
//           threads name the step's duplicates first, see apply.cuh)
//   scan    cell_start = exclusive prefix sum of count (3 passes over tiles of 4096 cells;
//           count is re-zeroed on the way)
//   keys    tmp_id[cell_start[cell_i] + slot_i] = id_i  (the cell's ids, in arbitrary order)
//   scatter rank_i = #{ids of the same cell smaller than id_i}; A[cell_start + rank] = B[i]
//           with the relabel test applied on the way
//   finalize particle count, next id, and the particle ranges of the buffers' candidate cells
// The result is sorted by (cell, id) whatever order the atomics took, so it is
// deterministic and identical to a plain sort.
#include "cells_bodies.cuh"

namespace sphbuf {

namespace {

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const unsigned* __restrict__ cnt,
                                                              unsigned* __restrict__ part,
                                                              const int* status) {
  if (status && *status) return;
  const size_t base = (size_t)blockIdx.x * kScanTile + (size_t)threadIdx.x * kScanItems;
  const uint4* p = reinterpret_cast<const uint4*>(cnt + base);
  unsigned s = 0;
#pragma unroll
  for (int q = 0; q < kScanItems / 4; ++q) {
    const uint4 v = p[q];
    s += v.x + v.y + v.z + v.w;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
  __shared__ unsigned ws[kScanThreads / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) t += ws[w];
    part[blockIdx.x] = t;
  }
}

// Exclusive scan of the per-tile sums, one block.
__global__ void __launch_bounds__(1024) k_scan_top(unsigned* part, int ntiles, const int* status) {
  if (status && *status) return;
  __shared__ unsigned ws[32];
  __shared__ unsigned carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int b0 = 0; b0 < ntiles; b0 += 1024) {
    const int t = b0 + threadIdx.x;
    const unsigned v = t < ntiles ? part[t] : 0u;
    unsigned x = v;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
      unsigned s = ws[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xFFFFFFFFu, s, o);
        if (lane >= o) s += y;
      }
      ws[lane] = s;
    }
    __syncthreads();
    const unsigned incl = x + (w > 0 ? ws[w - 1] : 0u);
    if (t < ntiles) part[t] = carry + incl - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += incl;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(unsigned* __restrict__ cnt,
                                                            const unsigned* __restrict__ part,
                                                            unsigned* __restrict__ start,
                                                            const int* status) {
  if (status && *status) return;
  const size_t base = (size_t)blockIdx.x * kScanTile + (size_t)threadIdx.x * kScanItems;
  uint4* p = reinterpret_cast<uint4*>(cnt + base);
  unsigned v[kScanItems];
#pragma unroll
  for (int q = 0; q < kScanItems / 4; ++q) {
    const uint4 t = p[q];
    v[4 * q] = t.x;
    v[4 * q + 1] = t.y;
    v[4 * q + 2] = t.z;
    v[4 * q + 3] = t.w;
    p[q] = make_uint4(0, 0, 0, 0);
  }
  unsigned s = 0;
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) s += v[q];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned x = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  __shared__ unsigned ws[kScanThreads / 32];
  if (lane == 31) ws[w] = x;
  __syncthreads();
  unsigned wpre = 0;
  for (int q = 0; q < w; ++q) wpre += ws[q];
  unsigned run = part[blockIdx.x] + wpre + x - s;
  uint4* o = reinterpret_cast<uint4*>(start + base);
#pragma unroll
  for (int q = 0; q < kScanItems / 4; ++q) {
    uint4 t;
    t.x = run;
    run += v[4 * q];
    t.y = run;
    run += v[4 * q + 1];
    t.z = run;
    run += v[4 * q + 2];
    t.w = run;
    run += v[4 * q + 3];
    o[q] = t;
  }
}

void scan_cells(unsigned* cnt, unsigned* part, unsigned* start, int tiles, const int* status,
                cudaStream_t s) {
  k_scan_reduce<<<tiles, kScanThreads, 0, s>>>(cnt, part, status);
  k_scan_top<<<1, 1024, 0, s>>>(part, tiles, status);
  k_scan_down<<<tiles, kScanThreads, 0, s>>>(cnt, part, start, status);
}

// ---- single-domain kernels
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce_occ(DomainDev d) {
  if (d.st->status) return;
  scan_reduce_occ_body(d.cnt, d.scan_part, d.scan_part_occ, blockIdx.x);
}
__global__ void __launch_bounds__(1024) k_scan_top_occ(DomainDev d) {
  if (d.st->status) return;
  scan_top_occ_body(d.scan_part, d.scan_part_occ, d.scan_tiles, &d.st->n_occ);
}
__global__ void __launch_bounds__(kScanThreads) k_scan_down_occ(DomainDev d) {
  if (d.st->status) return;
  scan_down_occ_body(d.cnt, d.scan_part, d.scan_part_occ, d.cell_start, d.occ_list, blockIdx.x);
}
__global__ void __launch_bounds__(256) k_hist(DomainDev d, int force_full) {
  hist_body(d, blockIdx.x, gridDim.x, force_full);
}
__global__ void __launch_bounds__(256) k_keys(DomainDev d) { keys_body(d, blockIdx.x, gridDim.x); }
template <int D>
__global__ void __launch_bounds__(256) k_scatter(DomainDev d) {
  scatter_body<D>(d, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(256) k_finalize(DomainDev d, int count_step) {
  finalize_body(d, count_step, blockIdx.x, gridDim.x);
}

// ---- batched twins (block -> (domain, local block, blocks of the domain))
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce_occ_batch(BatchDev b) {
  const int4 m = b.map[blockIdx.x];
  const DomainDev* d = b.doms + m.x;
  if (d->st->status) return;
  scan_reduce_occ_body(d->cnt, d->scan_part, d->scan_part_occ, (unsigned)m.y);
}
__global__ void __launch_bounds__(1024) k_scan_top_occ_batch(BatchDev b) {
  const int4 m = b.map[blockIdx.x];
  const DomainDev* d = b.doms + m.x;
  if (d->st->status) return;
  scan_top_occ_body(d->scan_part, d->scan_part_occ, d->scan_tiles, &d->st->n_occ);
}
__global__ void __launch_bounds__(kScanThreads) k_scan_down_occ_batch(BatchDev b) {
  const int4 m = b.map[blockIdx.x];
  const DomainDev* d = b.doms + m.x;
  if (d->st->status) return;
  scan_down_occ_body(d->cnt, d->scan_part, d->scan_part_occ, d->cell_start, d->occ_list, (unsigned)m.y);
}
// (the particle kernels of the rebuild take any block size up to 512: the autotuner's)
__global__ void __launch_bounds__(512) k_hist_batch(BatchDev b, int force_full) {
  __shared__ DomainDev sd;
  const int4 m = b.map[blockIdx.x];
  load_domain(sd, b.doms + m.x);
  hist_body(sd, (unsigned)m.y, (unsigned)m.z, force_full);
}
__global__ void __launch_bounds__(512) k_keys_batch(BatchDev b) {
  __shared__ DomainDev sd;
  const int4 m = b.map[blockIdx.x];
  load_domain(sd, b.doms + m.x);
  keys_body(sd, (unsigned)m.y, (unsigned)m.z);
}
template <int D>
__global__ void __launch_bounds__(512) k_scatter_batch(BatchDev b) {
  __shared__ DomainDev sd;
  const int4 m = b.map[blockIdx.x];
  load_domain(sd, b.doms + m.x);
  scatter_body<D>(sd, (unsigned)m.y, (unsigned)m.z);
}
__global__ void __launch_bounds__(256) k_finalize_batch(BatchDev b) {
  const int4 m = b.map[blockIdx.x];
  finalize_body(b.doms[m.x], 1, (unsigned)m.y, (unsigned)m.z);
}

__global__ void __launch_bounds__(256) k_ingest(DomainDev d, const float* __restrict__ frac,
                                                const float* __restrict__ vel, unsigned n, int ids_given,
                                                int labels_given, int nbuf) {
  const int D = d.g.dim;
  unsigned bad = 0, mx = 0;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int c = d.B.cell[i];
    if (c < 0 || (long long)c >= d.g.ncell) bad |= 1u;
    for (int x = 0; x < D; ++x) {
      const float f = frac[(size_t)i * D + x];
      if (!(f >= 0.f && f < d.g.cs)) bad |= 2u;
      d.B.f[x][i] = f;
      d.B.v[x][i] = vel[(size_t)i * D + x];
    }
    if (labels_given) {
      const uint8_t lab = d.B.label[i];
      if (lab != 0 && (lab == kDead || (int)lab > nbuf)) bad |= 4u;
    } else {
      d.B.label[i] = 0;
    }
    if (!ids_given) d.B.id[i] = i;
    d.B.bflag[i] = 0;
    mx = max(mx, d.B.id[i]);
  }
  bad = __reduce_or_sync(0xFFFFFFFFu, bad);
  mx = __reduce_max_sync(0xFFFFFFFFu, mx);
  if ((threadIdx.x & 31) == 0) {
    if (bad) atomicOr(&d.io[0], bad);
    atomicMax(&d.io[1], mx);
  }
}

__global__ void __launch_bounds__(256) k_ingest_staged(DomainDev d, const int* __restrict__ cell,
                                                       const float* __restrict__ frac, const float* __restrict__ vel,
                                                       const float* __restrict__ rho, const unsigned* __restrict__ id,
                                                       const uint8_t* __restrict__ label, unsigned n, int nbuf) {
  const int D = d.g.dim;
  unsigned bad = 0, mx = 0;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int c = cell[i];
    if (c < 0 || (long long)c >= d.g.ncell) bad |= 1u;
    d.B.cell[i] = c;
    for (int x = 0; x < D; ++x) {
      const float f = frac[(size_t)i * D + x];
      if (!(f >= 0.f && f < d.g.cs)) bad |= 2u;
      d.B.f[x][i] = f;
      d.B.v[x][i] = vel[(size_t)i * D + x];
    }
    d.B.rho[i] = rho[i];
    const uint8_t lab = label ? label[i] : (uint8_t)0;
    if (lab != 0 && (lab == kDead || (int)lab > nbuf)) bad |= 4u;
    d.B.label[i] = lab;
    const unsigned q = id ? id[i] : i;
    d.B.id[i] = q;
    d.B.bflag[i] = 0;
    mx = max(mx, q);
  }
  bad = __reduce_or_sync(0xFFFFFFFFu, bad);
  mx = __reduce_max_sync(0xFFFFFFFFu, mx);
  if ((threadIdx.x & 31) == 0) {
    if (bad) atomicOr(&d.io[0], bad);
    atomicMax(&d.io[1], mx);
  }
}

// The checks of the staged arrays decided: the state takes (n, next_id), or no particles
// and SPHBUF_ERR_INVALID_ARG.
__global__ void k_ingest_finish(DomainDev d, unsigned n, unsigned next_id) {
  StepState* st = d.st;
  const bool ok = n == 0 || (d.io[0] == 0 && next_id > d.io[1]);
  st->n = ok ? n : 0u;
  st->n_live = st->n;
  st->full = 1;
  st->n_inj = 0;
  st->n_del = 0;
  st->next_id = next_id;
  st->status = ok ? 0 : 1 /* SPHBUF_ERR_INVALID_ARG */;
  for (int k = 0; k < 2; ++k) st->sched[k] = st->sched_done[k] = 0u;
}

__global__ void __launch_bounds__(256) k_egest_staged(DomainDev d, int* __restrict__ cell, float* __restrict__ frac,
                                                      float* __restrict__ vel, float* __restrict__ rho,
                                                      unsigned* __restrict__ id, uint8_t* __restrict__ label,
                                                      unsigned* n_out, unsigned cap) {
  const int D = d.g.dim;
  // the live particles in (cell, id) order: the state itself after a full rebuild, through
  // the index list when the slots were kept
  const unsigned n = d.st->n_live;
  const bool full = d.st->full != 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) *n_out = n;
  const unsigned m = min(n, cap);
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    const unsigned o = full ? i : d.order[i];
    cell[i] = d.A.cell[o];
    for (int x = 0; x < D; ++x) {
      frac[(size_t)i * D + x] = d.A.f[x][o];
      vel[(size_t)i * D + x] = d.A.v[x][o];
    }
    rho[i] = d.A.rho[o];
    id[i] = d.A.id[o];
    label[i] = d.A.label[o];
  }
}

// B[k] = A[order[k]] for the live particles (a sorted copy of a state whose slots were kept;
// B is free between steps).
__global__ void __launch_bounds__(256) k_view(DomainDev d) {
  const int D = d.g.dim;
  const unsigned n = d.st->n_live;
  for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const unsigned o = d.order[k];
    d.B.cell[k] = d.A.cell[o];
    for (int x = 0; x < D; ++x) {
      d.B.f[x][k] = d.A.f[x][o];
      d.B.v[x][k] = d.A.v[x][o];
    }
    d.B.rho[k] = d.A.rho[o];
    d.B.id[k] = d.A.id[o];
    d.B.label[k] = d.A.label[o];
  }
}

__global__ void __launch_bounds__(256) k_egest(DomainDev d, Particles P, float* __restrict__ frac,
                                               float* __restrict__ vel, unsigned n) {
  const int D = d.g.dim;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    for (int x = 0; x < D; ++x) {
      if (frac) frac[(size_t)i * D + x] = P.f[x][i];
      if (vel) vel[(size_t)i * D + x] = P.v[x][i];
    }
  }
}

__global__ void k_decode(DomainDev d, double* out, double lo0, double lo1, double lo2, double cs) {
  const unsigned n = d.st->n_live;
  const bool full = d.st->full != 0;
  const int D = d.g.dim;
  const double lo[3] = {lo0, lo1, lo2};
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const unsigned o = full ? i : d.order[i];
    int c[3];
    cell_coords(d.A.cell[o], d.g, c);
    for (int x = 0; x < D; ++x) out[(size_t)i * D + x] = lo[x] + (double)c[x] * cs + (double)d.A.f[x][o];
  }
}

// ---- stand-alone cell-linked list on caller-provided device arrays
__global__ void k_hist_raw(const int32_t* cell, const uint8_t* label, unsigned n, long long ncell,
                           unsigned* cnt, unsigned* slot, int* bad) {
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int c = cell[i];
    if (label && label[i] == kDead) {
      slot[i] = kNoSlot;
    } else if (c < 0 || (long long)c >= ncell) {
      slot[i] = kNoSlot;
      atomicExch(bad, 1);
    } else {
      slot[i] = atomicAdd(cnt + c, 1u);
    }
  }
}

__global__ void k_keys_raw(const int32_t* cell, const uint32_t* id, unsigned n, const unsigned* slot,
                           const unsigned* start, unsigned* tmp) {
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const unsigned sl = slot[i];
    if (sl != kNoSlot) tmp[start[cell[i]] + sl] = id[i];
  }
}

// Rank of each particle among its cell's ids: O(m) loads per particle of a cell of m, so the
// stand-alone entry points accept at most kMaxPerCellRaw particles in one cell (a larger cell
// sets the input flag and is left unsorted instead of running for minutes).
constexpr unsigned kMaxPerCellRaw = 1024;

__global__ void k_order_raw(const int32_t* cell, const uint32_t* id, unsigned n, const unsigned* slot,
                            const unsigned* start, const unsigned* tmp, uint32_t* order, int* bad) {
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (slot[i] == kNoSlot) continue;
    const int c = cell[i];
    const unsigned s0 = start[c], s1 = start[c + 1], my = id[i];
    if (s1 - s0 > kMaxPerCellRaw) {
      atomicExch(bad, 1);
      continue;
    }
    unsigned rank = 0;
    for (unsigned p = s0; p < s1; ++p) rank += tmp[p] < my;
    order[s0 + rank] = i;
  }
}

}  // namespace

int finalize_blocks(const DomainDev& d) { return d.nseg > 256 ? (d.nseg + 255) / 256 : 1; }

int launch_rebuild(const DomainDev& d, bool count_step, bool force_full, cudaStream_t s) {
  const int blocks = d.sm_count * 8;
  k_hist<<<blocks, 256, 0, s>>>(d, force_full ? 1 : 0);
  k_scan_reduce_occ<<<d.scan_tiles, kScanThreads, 0, s>>>(d);
  k_scan_top_occ<<<1, 1024, 0, s>>>(d);
  k_scan_down_occ<<<d.scan_tiles, kScanThreads, 0, s>>>(d);
  k_keys<<<blocks, 256, 0, s>>>(d);
  if (d.g.dim == 2)
    k_scatter<2><<<blocks, 256, 0, s>>>(d);
  else
    k_scatter<3><<<blocks, 256, 0, s>>>(d);
  k_finalize<<<finalize_blocks(d), 256, 0, s>>>(d, count_step ? 1 : 0);
  return 7;
}

int launch_batch_cells(Kern k, int dim, const BatchDev& b, int nblocks, int threads, cudaStream_t s,
                       bool force_full) {
  switch (k) {
    case K_HIST:
      k_hist_batch<<<nblocks, threads, 0, s>>>(b, force_full ? 1 : 0);
      return 1;
    case K_SCAN_REDUCE:
      k_scan_reduce_occ_batch<<<nblocks, kScanThreads, 0, s>>>(b);
      return 1;
    case K_SCAN_TOP:
      k_scan_top_occ_batch<<<nblocks, 1024, 0, s>>>(b);
      return 1;
    case K_SCAN_DOWN:
      k_scan_down_occ_batch<<<nblocks, kScanThreads, 0, s>>>(b);
      return 1;
    case K_KEYS:
      k_keys_batch<<<nblocks, threads, 0, s>>>(b);
      return 1;
    case K_SCATTER:
      if (dim == 2)
        k_scatter_batch<2><<<nblocks, threads, 0, s>>>(b);
      else
        k_scatter_batch<3><<<nblocks, threads, 0, s>>>(b);
      return 1;
    case K_FINALIZE:
      k_finalize_batch<<<nblocks, 256, 0, s>>>(b);
      return 1;
    default:
      return 0;
  }
}

int batch_threads(Kern k) {
  switch (k) {
    case K_SCAN_TOP:
      return 1024;
    case K_BEGIN:
      return 32;
    default:
      return 256;
  }
}

bool batch_tunable(Kern k) {
  switch (k) {
    case K_NEIGHBOURS:
    case K_DENSITY_DEFER:
    case K_FORCE:
    case K_DRIFT:
    case K_VISCOUS:
    case K_ACOUSTIC:
    case K_DUAL_FINISH:
    case K_BUFFER:
    case K_BUFFER_FULL:
    case K_HIST:
    case K_KEYS:
    case K_SCATTER:
      return true;
    default:
      return false;  // the scans (tiles of 4096 cells, 256 threads), the per-domain single blocks
  }
}

void launch_ingest(const DomainDev& d, const float* frac, const float* vel, unsigned n, int ids_given,
                   int labels_given, int nbuf, cudaStream_t s) {
  k_ingest<<<d.sm_count * 4, 256, 0, s>>>(d, frac, vel, n, ids_given, labels_given, nbuf);
}

void launch_ingest_staged(const DomainDev& d, const int* cell, const float* frac, const float* vel, const float* rho,
                          const unsigned* id, const uint8_t* label, unsigned n, unsigned next_id, int nbuf,
                          cudaStream_t s) {
  cudaMemsetAsync(d.io, 0, 4 * sizeof(unsigned), s);
  if (n) k_ingest_staged<<<d.sm_count * 4, 256, 0, s>>>(d, cell, frac, vel, rho, id, label, n, nbuf);
  k_ingest_finish<<<1, 1, 0, s>>>(d, n, next_id);
}

void launch_egest_staged(const DomainDev& d, int* cell, float* frac, float* vel, float* rho, unsigned* id,
                         uint8_t* label, unsigned* n_out, unsigned cap, cudaStream_t s) {
  k_egest_staged<<<d.sm_count * 4, 256, 0, s>>>(d, cell, frac, vel, rho, id, label, n_out, cap);
}

void launch_egest(const DomainDev& d, const Particles& P, float* frac, float* vel, unsigned n, cudaStream_t s) {
  k_egest<<<d.sm_count * 4, 256, 0, s>>>(d, P, frac, vel, n);
}

void launch_view(const DomainDev& d, cudaStream_t s) { k_view<<<d.sm_count * 4, 256, 0, s>>>(d); }

namespace {
__global__ void __launch_bounds__(256) k_gather_u8(DomainDev d, const uint8_t* __restrict__ src,
                                                   uint8_t* __restrict__ dst, unsigned n) {
  for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) dst[k] = src[d.order[k]];
}
}  // namespace

void launch_gather_u8(const DomainDev& d, const uint8_t* src, uint8_t* dst, unsigned n, cudaStream_t s) {
  k_gather_u8<<<d.sm_count * 4, 256, 0, s>>>(d, src, dst, n);
}

void launch_decode_positions(const DomainDev& d, double* pos_out, const double lo[3], double cs,
                             cudaStream_t s) {
  k_decode<<<d.sm_count * 4, 256, 0, s>>>(d, pos_out, lo[0], lo[1], lo[2], cs);
}

cudaError_t cell_list_build(const int32_t* cell, const uint32_t* id, const uint8_t* label, uint64_t n,
                            uint64_t ncell, uint32_t* cell_start, uint32_t* order, cudaStream_t s,
                            int* bad_input) {
  *bad_input = 0;
  const long long pad = ((long long)ncell + 1 + kScanTile - 1) / kScanTile * kScanTile;
  const int tiles = (int)(pad / kScanTile);
  unsigned *cnt = nullptr, *part = nullptr, *start = nullptr, *slot = nullptr, *tmp = nullptr;
  int* bad = nullptr;
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t r) {
    if (e == cudaSuccess && r != cudaSuccess) e = r;
  };
  chk(cudaMallocAsync((void**)&cnt, (size_t)pad * sizeof(unsigned), s));
  chk(cudaMallocAsync((void**)&part, (size_t)tiles * sizeof(unsigned), s));
  chk(cudaMallocAsync((void**)&start, (size_t)(pad + 1) * sizeof(unsigned), s));
  chk(cudaMallocAsync((void**)&slot, (size_t)(n ? n : 1) * sizeof(unsigned), s));
  chk(cudaMallocAsync((void**)&tmp, (size_t)(n ? n : 1) * sizeof(unsigned), s));
  chk(cudaMallocAsync((void**)&bad, sizeof(int), s));
  if (e == cudaSuccess) {
    chk(cudaMemsetAsync(cnt, 0, (size_t)pad * sizeof(unsigned), s));
    chk(cudaMemsetAsync(bad, 0, sizeof(int), s));
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * 8;
    const unsigned nn = (unsigned)n;
    k_hist_raw<<<blocks, 256, 0, s>>>(cell, label, nn, (long long)ncell, cnt, slot, bad);
    scan_cells(cnt, part, start, tiles, nullptr, s);
    k_keys_raw<<<blocks, 256, 0, s>>>(cell, id, nn, slot, start, tmp);
    k_order_raw<<<blocks, 256, 0, s>>>(cell, id, nn, slot, start, tmp, order, bad);
    chk(cudaGetLastError());
    chk(cudaMemcpyAsync(cell_start, start, (size_t)(ncell + 1) * sizeof(unsigned), cudaMemcpyDeviceToDevice, s));
    int hbad = 0;
    chk(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    chk(cudaStreamSynchronize(s));
    *bad_input = hbad;
  }
  if (cnt) cudaFreeAsync(cnt, s);
  if (part) cudaFreeAsync(part, s);
  if (start) cudaFreeAsync(start, s);
  if (slot) cudaFreeAsync(slot, s);
  if (tmp) cudaFreeAsync(tmp, s);
  if (bad) cudaFreeAsync(bad, s);
  return e;
}

// ---- the same cell-linked list with its scratch in a fixed, file-scope device array
//
// For callers that cannot allocate device memory.  Layout of the array (32-bit words):
//   count[kNaPad] | start[kNaPad + 1] | part[kNaTiles] | slot[kNaMaxN] | tmp[kNaMaxN] | flag[1]
// A GPU holds this array (about 16 MiB) from the library's first use on it (when its device
// code is loaded there) until the process exits.
namespace {

constexpr unsigned long long kNaMaxN = 1ull << 20;          // particles per call
constexpr unsigned long long kNaMaxCells = (1ull << 20) - 1;  // cells per call
constexpr size_t kNaPad = ((kNaMaxCells + 1 + kScanTile - 1) / kScanTile) * kScanTile;
constexpr size_t kNaTiles = kNaPad / kScanTile;
constexpr size_t kNaCount = 0;
constexpr size_t kNaStart = kNaCount + kNaPad;
constexpr size_t kNaPart = kNaStart + kNaPad + 4;  // keeps the next block 16-byte aligned
constexpr size_t kNaSlot = kNaPart + ((kNaTiles + 3) / 4) * 4;
constexpr size_t kNaTmp = kNaSlot + kNaMaxN;
constexpr size_t kNaFlag = kNaTmp + kNaMaxN;
constexpr size_t kNaWords = kNaFlag + 4;

static __device__ __align__(256) unsigned g_noalloc_scratch[kNaWords];

// Device address of the scratch array on the current device, looked up on every call
// (cudaGetSymbolAddress allocates nothing; a cached address would go stale after a
// cudaDeviceReset reloads the module).  The first lookup on a device loads the library's
// device code there if it was not loaded yet, which is when the array is reserved.
cudaError_t noalloc_scratch(unsigned** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<unsigned*>(p);
  return cudaSuccess;
}

}  // namespace

unsigned long long cell_list_noalloc_max_particles() { return kNaMaxN; }
unsigned long long cell_list_noalloc_max_cells() { return kNaMaxCells; }

cudaError_t cell_list_build_noalloc(const int32_t* cell, const uint32_t* id, const uint8_t* label, uint64_t n,
                                    uint64_t ncell, uint32_t* cell_start, uint32_t* order, cudaStream_t s,
                                    int* bad_input) {
  *bad_input = 0;
  unsigned* base = nullptr;
  cudaError_t e = noalloc_scratch(&base);
  if (e != cudaSuccess) return e;
  const long long pad = ((long long)ncell + 1 + kScanTile - 1) / kScanTile * kScanTile;
  const int tiles = (int)(pad / kScanTile);
  unsigned* cnt = base + kNaCount;
  unsigned* start = base + kNaStart;
  unsigned* part = base + kNaPart;
  unsigned* slot = base + kNaSlot;
  unsigned* tmp = base + kNaTmp;
  int* bad = reinterpret_cast<int*>(base + kNaFlag);
  // the array keeps the previous call's contents: clear the counters and the error flag
  e = cudaMemsetAsync(cnt, 0, (size_t)pad * sizeof(unsigned), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = (sms > 0 ? sms : 1) * 8;
  const unsigned nn = (unsigned)n;
  k_hist_raw<<<blocks, 256, 0, s>>>(cell, label, nn, (long long)ncell, cnt, slot, bad);
  scan_cells(cnt, part, start, tiles, nullptr, s);
  k_keys_raw<<<blocks, 256, 0, s>>>(cell, id, nn, slot, start, tmp);
  k_order_raw<<<blocks, 256, 0, s>>>(cell, id, nn, slot, start, tmp, order, bad);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(cell_start, start, (size_t)(ncell + 1) * sizeof(unsigned), cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return e;
  int hbad = 0;
  e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  *bad_input = hbad;
  return e;
}

}  // namespace sphbuf
