// Algorithms 1-3 (Sec. 3): the list records of the step's decisions and the decision of one
// particle whose post-drift state is in registers.
//
// Two forms share this code.  The buffer kernel (kernels_buffer.cu) visits the candidate
// cells after the drift; the fused form decides inside the drift epilogue of the step
// (drift_store in kernels_sph.cu), for the particles whose cell (the one they were sorted
// into) is a candidate cell of some buffer (a bit per buffer in the per-cell mask
// DomainDev::cand_mask).  Both take every decision from the particle's post-drift state,
// compare X' with the FP32 decision contract, and compact the records with a warp ballot:
// the lanes that reach the ballot together reserve their ranges of the step's lists with one
// atomic per list.  The duplicates' ids are assigned by the rebuild (apply.cuh).
#pragma once

#include "kernels.cuh"

namespace sphbuf {

// Writes injection `slot` of the step: its record and its duplicate at B[n + slot] (the
// parent's state before recycling, label 0; id assigned by the rebuild).
template <int D>
__device__ __forceinline__ void write_injection(const DomainDev& d, const Decision& e, unsigned slot, unsigned n) {
  if (slot >= d.P.list_cap || (unsigned long long)n + slot >= d.P.capacity) {
    latch(d.st, 2 /* SPHBUF_ERR_CAPACITY */);
    return;
  }
  d.inj[slot] = e;
  const unsigned dst = n + slot;
  d.B.cell[dst] = e.cell;
#pragma unroll
  for (int x = 0; x < D; ++x) {
    d.B.f[x][dst] = e.f[x];
    d.B.v[x][dst] = e.v[x];
  }
  d.B.rho[dst] = e.rho;
  d.B.id[dst] = kNoSlot;
  d.B.label[dst] = 0;  // the duplicate is ordinary fluid (Algorithm 1)
#pragma unroll
  for (int x = 0; x < D; ++x) d.disp[x][dst] = 0.f;
  d.B.bflag[dst] = 0;
}

__device__ __forceinline__ void write_deletion(const DomainDev& d, const Decision& e, unsigned slot) {
  if (slot >= d.P.list_cap) {
    latch(d.st, 2 /* SPHBUF_ERR_CAPACITY */);
    return;
  }
  d.del[slot] = e;
}

// Warp-ballot compaction of one record per flagged lane among the lanes of `am` (which all
// call it): one atomic per list and warp, then each flagged lane writes its record (and, for
// an injection, its duplicate).
template <int D, bool INJ>
__device__ __forceinline__ void stage(const DomainDev& d, unsigned am, unsigned n, bool flag, const Decision& rec) {
  const unsigned m = __ballot_sync(am, flag);
  if (m == 0) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(m) - 1;
  unsigned base = 0;
  if (lane == leader) base = atomicAdd(INJ ? &d.st->n_inj : &d.st->n_del, (unsigned)__popc(m));
  base = __shfl_sync(am, base, leader);
  if (!flag) return;
  atomicAdd(INJ ? &d.st->injected[rec.k] : &d.st->deleted[rec.k], 1ull);
  const unsigned r = base + __popc(m & ((1u << lane) - 1u));
  if (INJ)
    write_injection<D>(d, rec, r, n);
  else
    write_deletion(d, rec, r);
}

// The test of Algorithms 1-3 against buffer b for a particle with label lab at (c, f) after
// the drift: Algorithm 1 (inflow) and 3 (bidirectional) test the buffer's own particles on
// X' = a/2 (injection) and, for Algorithm 3, X' = -a/2 (deletion); Algorithm 2 (outflow)
// deletes any live particle of the candidate region (reading A4) beyond X' = a/2.
template <int D>
__device__ __forceinline__ void buffer_test(const BufDev& b, uint8_t lab, const int c[3], const float f[3], float cs,
                                            bool& inj, bool& del) {
  inj = false;
  del = false;
  const bool test = (b.kind == KIND_OUTFLOW) ? (lab != kDead) : (lab == (uint8_t)b.label);
  if (!test) return;
  float X[3];
  if (b.kind == KIND_OUTFLOW) {
    local_coords<D>(b, c, f, cs, X, D);
    bool cand = fabsf(X[0]) < b.da && fabsf(X[1]) < b.db;
    if (D == 3) cand = cand && fabsf(X[2]) < b.dc;
    del = cand && X[0] > b.ha;
  } else {
    local_coords<D>(b, c, f, cs, X, 1);
    inj = X[0] > b.ha;
    if (b.kind == KIND_BIDIR) del = X[0] < -b.ha;
  }
}

// Fused form: the decisions of particle i (id `id`, post-drift state lab, c, f, v, rho, with
// `inside` false once it left the grid) against the buffers of `bits` (the candidate buffers
// of the cell it was sorted into), from that state.  Every lane of `am` calls it.  An
// injection records the parent's state, writes its duplicate and recycles the parent by
// -a u (Eqs. (16)-(17)), with rho0 + p_b / c0^2 for a pressure buffer (Eq. (22)); a deletion
// marks the particle dead.  The state in registers is updated in place for the caller's
// store.  (Buffers' candidate regions are disjoint, so at most one buffer acts on a particle.)
template <int D>
__device__ __forceinline__ void decide_fused(const DomainDev& d, unsigned am, unsigned n, unsigned bits, unsigned i,
                                             unsigned id, uint8_t& lab, int c[3], float f[3], bool& inside,
                                             const float v[3], float& rho) {
  if (!__any_sync(am, bits != 0u)) return;
  const Grid& g = d.g;
  const uint8_t lab0 = lab;
  const int c0[3] = {c[0], c[1], c[2]};
  const float f0[3] = {f[0], f[1], f[2]};
  const float rho0 = rho;
  unsigned rem = bits;
  while (__any_sync(am, rem != 0u)) {
    const int k = rem ? __ffs(rem) - 1 : 0;
    const bool have = rem != 0u;
    rem &= rem - 1u;
    bool inj = false, del = false;
    const BufDev* b = d.bufs + k;
    if (have) buffer_test<D>(*b, lab0, c0, f0, g.cs, inj, del);
    if (!__any_sync(am, inj || del)) continue;
    Decision rec;
    rec.k = (unsigned)k;
    rec.idx = i;
    rec.id = id;
    rec.cell = (c0[2] * g.ny + c0[1]) * g.nx + c0[0];
    rec.rho = rho0;
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      rec.f[x] = f0[x];
      rec.v[x] = x < D ? v[x] : 0.f;
    }
    stage<D, true>(d, am, n, inj, rec);
    if (inj) {
      // recycle the parent: r' - [a, 0, 0]^T mapped back, i.e. r - a u
      bool ok = true;
#pragma unroll
      for (int x = 0; x < D; ++x) ok &= move_fold(f[x], c[x], b->shift[x], g.cs);
      const bool in = ok && c[0] >= 0 && c[0] < g.nx && c[1] >= 0 && c[1] < g.ny && c[2] >= 0 && c[2] < g.nz;
      if (!in) {
        inside = false;
        lab = kDead;
        atomicAdd(&d.st->escaped_total, 1ull);
      }
      if (!b->vel_bc) rho = d.st->rho_pb[k];  // Eq. (22)
    }
    if (del) lab = kDead;
    stage<D, false>(d, am, n, del, rec);
  }
}

}  // namespace sphbuf
