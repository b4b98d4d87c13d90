// Device bodies of the cell-linked list rebuild (counting sort, relabel, finalize), shared
// by the per-phase kernels (kernels_cells.cu) and the persistent batched step
// (kernels_persist.cu).
#pragma once

#include "apply.cuh"
#include "kernels.cuh"

namespace sphbuf {

namespace {

// ---- domain scan: cell_start plus the ordered list of occupied cells (the work list of the
// tiled neighbour passes)
__device__ __forceinline__ unsigned block_excl_scan(unsigned x, unsigned* ws, unsigned* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) ws[w] = incl;
  __syncthreads();
  unsigned wpre = 0, tot = 0;
  for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
    if (q < w) wpre += ws[q];
    tot += ws[q];
  }
  __syncthreads();
  if (total) *total = tot;
  return wpre + incl - x;
}

__device__ __forceinline__ void scan_reduce_occ_body(const unsigned* __restrict__ cnt, unsigned* __restrict__ part,
                                                     unsigned* __restrict__ part_occ, unsigned tile) {
  __shared__ unsigned ws[kScanThreads / 32];
  const size_t base = (size_t)tile * kScanTile + (size_t)threadIdx.x * kScanItems;
  const uint4* p = reinterpret_cast<const uint4*>(cnt + base);
  unsigned s = 0, o = 0;
#pragma unroll
  for (int q = 0; q < kScanItems / 4; ++q) {
    const uint4 v = p[q];
    s += v.x + v.y + v.z + v.w;
    o += (v.x > 0) + (v.y > 0) + (v.z > 0) + (v.w > 0);
  }
  unsigned ts = 0, to = 0;
  block_excl_scan(s, ws, &ts);
  block_excl_scan(o, ws, &to);
  if (threadIdx.x == 0) {
    part[tile] = ts;
    part_occ[tile] = to;
  }
}

// Exclusive scans of both per-tile sums (one block); the total occupied count goes to *n_occ.
__device__ __forceinline__ void scan_top_occ_body(unsigned* part, unsigned* part_occ, int ntiles, unsigned* n_occ) {
  __shared__ unsigned ws[32];
  unsigned carry = 0, carry_o = 0;
  for (int b0 = 0; b0 < ntiles; b0 += blockDim.x) {
    const int t = b0 + threadIdx.x;
    const unsigned v = t < ntiles ? part[t] : 0u;
    const unsigned vo = t < ntiles ? part_occ[t] : 0u;
    unsigned tot = 0, toto = 0;
    const unsigned ex = block_excl_scan(v, ws, &tot);
    const unsigned exo = block_excl_scan(vo, ws, &toto);
    if (t < ntiles) {
      part[t] = carry + ex;
      part_occ[t] = carry_o + exo;
    }
    carry += tot;
    carry_o += toto;
  }
  if (threadIdx.x == 0) *n_occ = carry_o;
}

__device__ __forceinline__ void scan_down_occ_body(unsigned* __restrict__ cnt, const unsigned* __restrict__ part,
                                                   const unsigned* __restrict__ part_occ, unsigned* __restrict__ start,
                                                   unsigned* __restrict__ occ_list, unsigned tile) {
  __shared__ unsigned ws[kScanThreads / 32];
  const size_t base = (size_t)tile * kScanTile + (size_t)threadIdx.x * kScanItems;
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
  unsigned s = 0, o = 0;
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) {
    s += v[q];
    o += v[q] > 0;
  }
  unsigned run = part[tile] + block_excl_scan(s, ws, nullptr);
  unsigned orun = part_occ[tile] + block_excl_scan(o, ws, nullptr);
  uint4* out = reinterpret_cast<uint4*>(start + base);
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
    out[q] = t;
  }
#pragma unroll
  for (int q = 0; q < kScanItems; ++q)
    if (v[q]) occ_list[orun++] = (unsigned)(base + q);
}

// force_full: this step's rebuild must sort (kinematic steps and the commit's rebuild);
// otherwise, with kept neighbour lists, the first thread decides: a full rebuild once twice
// the largest displacement since the last one, relative to the period's reference velocity
// u0 (walls included, whose relative displacement is -u0 t), exceeds the lists' skin (a pair
// may then have come within 2h unlisted) or after reuse_max steps, else the slots keep their
// order.  At a full rebuild the next period's u0 is set from the range of this period's drift
// velocities; any constant u0 keeps the test exact, the middle of the range makes it tightest.
__device__ __forceinline__ void hist_body(const DomainDev& d, unsigned bid, unsigned nblk, int force_full) {
  if (d.st->status) return;
  if (bid == 0 && threadIdx.x == 0) {
    StepState* st = d.st;
    int full = 1;
    if (d.P.reuse && !force_full) {
      // a pair's distance changed by at most |disp_i| + |disp_j| (both relative to u0); a
      // wall particle's displacement relative to u0 is -u0 t
      float u2 = 0.f;
      for (int x = 0; x < d.g.dim; ++x) u2 += st->u0[x] * st->u0[x];
      const float wall = d.W.start[d.g.ncell] ? sqrtf(u2) * (float)(st->since_full + 1) * d.P.dt : 0.f;
      const float path = fmaxf(__uint_as_float(st->path_bits), wall);
      full = (2.f * path > d.P.skin || st->since_full + 1 >= (unsigned)d.P.reuse_max) ? 1 : 0;
    }
    if (full) {
      // the next period's reference velocity: the middle of the range of the drift
      // velocities of this one, zero (the walls) included
      for (int x = 0; x < 3; ++x) {
        unsigned khi = 0u, klo = 0u;
        for (int q = 0; q < kRangeCopies; ++q) {
          khi = max(khi, st->v_hi[q][x]);
          klo = max(klo, st->v_lo[q][x]);
          st->v_hi[q][x] = st->v_lo[q][x] = 0u;
        }
        float u = 0.f;
        if (khi) {
          const float hi = fmaxf(key_to_float(khi), 0.f), lo = fminf(key_to_float(~klo), 0.f);
          u = 0.5f * (hi + lo);
        }
        st->u0[x] = u;
      }
    }
    st->full = full;
    st->path_bits = 0u;
    st->since_full = full ? 0u : st->since_full + 1u;
    if (full) st->list_builds += 1;
  }
  rank_injections(d, bid, nblk);
  const unsigned n = d.st->n + d.st->n_inj;
  const unsigned lane = threadIdx.x & 31u;
  for (unsigned i = bid * blockDim.x + threadIdx.x; i < n; i += nblk * blockDim.x) {
    // consecutive particles mostly share a cell (B is in the last rebuild's order): one
    // atomic per cell and warp; the slots inside a cell are only an arrival order (the
    // scatter ranks each cell's particles by id)
    const bool dead = d.B.label[i] == kDead;
    const int c = d.B.cell[i];
    if (!SPHBUF_IN_BOUNDS(d, dead || (c >= 0 && c < d.g.ncell), 10, i)) return;
    const unsigned act = __activemask();
    const unsigned peers = __match_any_sync(act, dead ? 0xFFFFFFFFu : (unsigned)c);
    const int leader = __ffs(peers) - 1;
    unsigned base = 0;
    if (!dead && (int)lane == leader) base = atomicAdd(d.cnt + c, (unsigned)__popc(peers));
    base = __shfl_sync(act, base, leader);
    d.slot[i] = dead ? kNoSlot : base + (unsigned)__popc(peers & ((1u << lane) - 1u));
  }
}

__device__ __forceinline__ void keys_body(const DomainDev& d, unsigned bid, unsigned nblk) {
  if (d.st->status) return;
  const unsigned n = d.st->n + d.st->n_inj;
  for (unsigned i = bid * blockDim.x + threadIdx.x; i < n; i += nblk * blockDim.x) {
    const unsigned sl = d.slot[i];
    if (sl != kNoSlot) d.tmp_id[d.cell_start[d.B.cell[i]] + sl] = d.B.id[i];
  }
}

// The particle's label after the relabel of Algorithms 2-3 (in-box particles join the
// outflow / bidirectional buffer, others leave it).
template <int D>
__device__ __forceinline__ uint8_t relabelled(const DomainDev& d, const int c[3], const float f[3], uint8_t lab) {
  for (int q = 0; q < d.nrelabel; ++q) {
    const BufDev& b = d.bufs[d.relabel_ids[q]];
    const bool near = c[0] >= b.box_lo[0] && c[0] <= b.box_hi[0] && c[1] >= b.box_lo[1] && c[1] <= b.box_hi[1] &&
                      c[2] >= b.box_lo[2] && c[2] <= b.box_hi[2];
    if (!near && lab != (uint8_t)b.label) continue;
    float X[3];
    local_coords<D>(b, c, f, d.g.cs, X, D);
    if (in_box<D>(b, X))
      lab = (uint8_t)b.label;
    else if (lab == (uint8_t)b.label)
      lab = 0;
  }
  return lab;
}

// Full rebuild: A[cell_start + rank] = B[i], rank = the particle's place by id in its cell,
// relabelled on the way; dead particles are dropped; the index list is the identity.
// Kept slots (kept neighbour lists, no full rebuild this step): A[i] = B[i] for every slot,
// dead ones included (their position copy is put far outside the grid, so listed dead slots
// add nothing), and the index list takes each live slot at its sorted place.
template <int D>
__device__ __forceinline__ void scatter_body(const DomainDev& d, unsigned bid, unsigned nblk) {
  if (d.st->status) return;
  const unsigned n = d.st->n + d.st->n_inj;
  const bool full = d.st->full != 0;
  const Grid& g = d.g;
  for (unsigned i = bid * blockDim.x + threadIdx.x; i < n; i += nblk * blockDim.x) {
    const bool live = d.slot[i] != kNoSlot;
    if (full && !live) continue;
    const int lin = d.B.cell[i];
    unsigned dst = i;
    if (live) {
      const unsigned s0 = d.cell_start[lin], s1 = d.cell_start[lin + 1];
      const unsigned my = d.B.id[i];
      unsigned rank = 0;
      for (unsigned p = s0; p < s1; ++p) rank += SPHBUF_LDG(d.tmp_id + p) < my;
      if (!SPHBUF_IN_BOUNDS(d, s0 + rank < s1, 8, s0 + rank)) continue;
      if (full) {
        dst = s0 + rank;
        d.order[dst] = dst;
      } else {
        d.order[s0 + rank] = i;
      }
    }
    float f[3] = {0.f, 0.f, 0.f}, v[3] = {0.f, 0.f, 0.f};
    d.A.cell[dst] = lin;
#pragma unroll
    for (int x = 0; x < D; ++x) {
      f[x] = d.B.f[x][i];
      v[x] = d.B.v[x][i];
      d.A.f[x][dst] = f[x];
      d.A.v[x][dst] = v[x];
    }
    const float rho = d.B.rho[i];
    d.A.rho[dst] = rho;
    d.A.id[dst] = d.B.id[i];
    d.A.bflag[dst] = d.B.bflag[i];
    int c[3];
    cell_coords(lin, g, c);
    if (live) {
      d.pos4[dst] = make_float4(f[0], f[1], f[2], __uint_as_float(pack_cell(c[0], c[1], c[2])));
      d.A.label[dst] = d.nrelabel ? relabelled<D>(d, c, f, d.B.label[i]) : d.B.label[i];
    } else {
      d.pos4[dst] = make_float4(0.f, 0.f, 0.f, __uint_as_float(pack_cell(kMaxCellsX - 1, kMaxCellsY - 1, kMaxCellsZ - 1)));
      d.A.label[dst] = kDead;
    }
    d.vel4[dst] = make_float4(v[0], v[1], v[2], rho);
  }
}

__device__ __forceinline__ void finalize_body(const DomainDev& d, int count_step, unsigned bid, unsigned nblk) {
  StepState* st = d.st;
  if (st->status) return;
  if (bid == 0 && threadIdx.x == 0) {
    // slots: the sorted live particles after a full rebuild, the kept slots plus this step's
    // duplicates otherwise
    st->n_live = d.cell_start[d.g.ncell];
    st->n = st->full ? st->n_live : st->n + min(st->n_inj, d.P.list_cap);
    st->next_id += min(st->n_inj, d.P.list_cap);
    // the next step's neighbour pass counts its deferred particles from zero (reset here, in
    // a launch of its own, not by that pass's first block while the others add to it)
    st->n_defer = 0;
    if (count_step) {
      st->step += 1;
      // Sec. 5.3: re-establish the frames of rotating buffers for the next step (their
      // particles turned in this step's buffer update)
      for (int k = 0; k < d.nbuf; ++k) {
        BufDev* b = const_cast<BufDev*>(d.bufs) + k;
        if (!b->rotating) continue;
        RotDev& q = d.rot[k];
        advance_rotation(q);
        double O[3], R[9];
        rotated_frame(q, O, R);
        frame_constants(*b, O, R, q.a, d.P.lo_d, d.P.cs_d, d.g.dim);
      }
    }
  }
  // (first particle, end, cell, buffer) of the candidate cell segments
  for (unsigned s = bid * blockDim.x + threadIdx.x; s < (unsigned)d.nseg; s += nblk * blockDim.x) {
    const int lin0 = d.seg_lin[2 * s];
    d.seg_range[s] = make_uint4(d.cell_start[lin0], d.cell_start[d.seg_lin[2 * s + 1]], (unsigned)lin0,
                                (unsigned)d.seg_buf[s]);
  }
}

}  // namespace

}  // namespace sphbuf
