// The arbitrary-positioned buffer (Sec. 3, Algorithms 1-3) on the GPU.
//
// decide: for each buffer, only the particles listed in the cells around its box are
//   visited (one warp per run of consecutive candidate cells); each is transformed into the
//   buffer's local frame (Eqs. (11), (15)) with the FP32 decision contract and compared on
//   the normal axis only.  Crossings are compacted with a warp ballot + one atomic per
//   warp into the injection / deletion lists.  Deleted particles are marked dead in place.
// apply: injections are ranked by (buffer, parent id) (tile-wise comparison in shared
//   memory); rank r appends a duplicate with id next_id + r at the tail of B and recycles
//   the parent by -a u (Eqs. (16)-(17)); pressure buffers reset its density (Eq. (22)).
#include "kernels.cuh"

namespace sphbuf {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ void emit(bool flag, unsigned k, unsigned i, unsigned id, Decision* list,
                                     unsigned* counter, unsigned long long* per_buffer, unsigned cap,
                                     StepState* st) {
  const unsigned m = __ballot_sync(kFull, flag);
  if (m == 0) return;
  const int lane = threadIdx.x & 31;
  unsigned base = 0;
  if (lane == 0) {
    base = atomicAdd(counter, (unsigned)__popc(m));
    atomicAdd(per_buffer, (unsigned long long)__popc(m));
  }
  base = __shfl_sync(kFull, base, 0);
  if (flag) {
    const unsigned r = base + __popc(m & ((1u << lane) - 1u));
    if (r < cap)
      list[r] = Decision{k, i, id};
    else
      latch(st, 2 /* SPHBUF_ERR_CAPACITY */);
  }
}

// Algorithms 1-3 for particle i (in B) against buffer b.
template <int D>
__device__ __forceinline__ void decide_one(const DomainDev& d, const BufDev& b, unsigned i, bool& inj,
                                           bool& del) {
  const uint8_t lab = d.B.label[i];
  const bool test = (b.kind == KIND_OUTFLOW) ? (lab != kDead) : (lab == (uint8_t)b.label);
  if (!test) return;
  int c[3];
  cell_coords(d.B.cell[i], d.g, c);
  const float f[3] = {d.B.f[0][i], d.B.f[1][i], D == 3 ? d.B.f[2][i] : 0.f};
  float X[3];
  if (b.kind == KIND_OUTFLOW) {
    // Algorithm 2: candidates within one cell of the box, deleted once X' > a/2
    local_coords<D>(b, c, f, d.g.cs, X, D);
    bool cand = fabsf(X[0]) < b.da && fabsf(X[1]) < b.db;
    if (D == 3) cand = cand && fabsf(X[2]) < b.dc;
    del = cand && X[0] > b.ha;
  } else {
    // Algorithms 1 and 3: buffer particles crossing X' = a/2 generate; Algorithm 3 deletes
    // those crossing X' = -a/2
    local_coords<D>(b, c, f, d.g.cs, X, 1);
    inj = X[0] > b.ha;
    if (b.kind == KIND_BIDIR) del = X[0] < -b.ha;
  }
}

template <int D>
__device__ __forceinline__ void decide_emit(const DomainDev& d, int k, unsigned i, bool valid) {
  const BufDev& b = d.bufs[k];
  bool inj = false, del = false;
  if (valid) decide_one<D>(d, b, i, inj, del);
  const unsigned id = valid ? d.B.id[i] : 0u;
  emit(inj, (unsigned)k, i, id, d.inj, &d.st->n_inj, &d.st->injected[k], d.P.list_cap, d.st);
  if (del) d.B.label[i] = kDead;
  emit(del, (unsigned)k, i, id, d.del, &d.st->n_del, &d.st->deleted[k], d.P.list_cap, d.st);
}

// Restricted decisions: one warp per candidate segment (run of consecutive cells).
template <int D>
__global__ void __launch_bounds__(256) k_decide(DomainDev d) {
  if (d.st->status) return;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int s = warp; s < d.nseg; s += nwarps) {
    const int lin0 = d.seg_lin[2 * s], lin1 = d.seg_lin[2 * s + 1];
    const int k = d.seg_buf[s];
    const unsigned j0 = d.cell_start[lin0], j1 = d.cell_start[lin1];
    for (unsigned base = j0; base < j1; base += 32) {
      const unsigned i = base + lane;
      decide_emit<D>(d, k, i, i < j1);
    }
  }
}

// Full-domain decisions: every particle against every buffer (same result).
template <int D>
__global__ void __launch_bounds__(256) k_decide_full(DomainDev d) {
  if (d.st->status) return;
  const unsigned n = d.st->n;
  const int lane = threadIdx.x & 31;
  const unsigned warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned nwarps = (gridDim.x * blockDim.x) >> 5;
  for (unsigned base = warp * 32; base < n; base += nwarps * 32) {
    const unsigned i = base + lane;
    for (int k = 0; k < d.nbuf; ++k) decide_emit<D>(d, k, i, i < n);
  }
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

constexpr int kApplyThreads = 256;

template <int D>
__global__ void __launch_bounds__(kApplyThreads) k_apply(DomainDev d) {
  if (d.st->status) return;
  StepState* st = d.st;
  const unsigned n_inj = min(st->n_inj, d.P.list_cap);
  const unsigned n = st->n;
  if (n_inj == 0) return;
  if ((unsigned long long)n + n_inj > d.P.capacity) {
    if (threadIdx.x == 0 && blockIdx.x == 0) latch(st, 2 /* SPHBUF_ERR_CAPACITY */);
    return;
  }
  __shared__ unsigned long long keys[kApplyThreads];
  const Grid& g = d.g;
  for (unsigned e0 = blockIdx.x * kApplyThreads; e0 < n_inj; e0 += gridDim.x * kApplyThreads) {
    const unsigned e = e0 + threadIdx.x;
    Decision me{0, 0, 0};
    unsigned long long key = ~0ull;
    if (e < n_inj) {
      me = d.inj[e];
      key = ((unsigned long long)me.k << 32) | me.id;
    }
    unsigned rank = 0;
    for (unsigned t0 = 0; t0 < n_inj; t0 += kApplyThreads) {
      __syncthreads();
      const unsigned te = t0 + threadIdx.x;
      if (te < n_inj) {
        const Decision o = d.inj[te];
        keys[threadIdx.x] = ((unsigned long long)o.k << 32) | o.id;
      } else {
        keys[threadIdx.x] = ~0ull;
      }
      __syncthreads();
      const unsigned cnt = min((unsigned)kApplyThreads, n_inj - t0);
      for (unsigned q = 0; q < cnt; ++q) rank += keys[q] < key;
    }
    if (e < n_inj) {
      const unsigned i = me.idx;
      const unsigned dst = n + rank;
      const unsigned child = st->next_id + rank;
      // duplicate: same state as the crossing particle, ordinary fluid (Algorithm 1)
      d.B.cell[dst] = d.B.cell[i];
#pragma unroll
      for (int x = 0; x < D; ++x) {
        d.B.f[x][dst] = d.B.f[x][i];
        d.B.v[x][dst] = d.B.v[x][i];
      }
      d.B.rho[dst] = d.B.rho[i];
      d.B.id[dst] = child;
      d.B.label[dst] = 0;
      d.inj_sorted[rank] = InjRecord{me.k, me.id, child};
      // recycle the parent: r' - [a, 0, 0]^T mapped back, i.e. r - a u
      const BufDev& b = d.bufs[me.k];
      int c[3];
      cell_coords(d.B.cell[i], g, c);
      bool ok = true;
#pragma unroll
      for (int x = 0; x < D; ++x) {
        float fx = d.B.f[x][i];
        ok &= move_fold(fx, c[x], b.shift[x], g.cs);
        d.B.f[x][i] = fx;
      }
      const bool inside = ok && c[0] >= 0 && c[0] < g.nx && c[1] >= 0 && c[1] < g.ny && c[2] >= 0 && c[2] < g.nz;
      if (inside) {
        d.B.cell[i] = (c[2] * g.ny + c[1]) * g.nx + c[0];
      } else {
        d.B.label[i] = kDead;
        atomicAdd(&st->escaped_total, 1ull);
      }
      if (!b.vel_bc) d.B.rho[i] = st->rho_pb[me.k];  // Eq. (22)
    }
  }
}

}  // namespace

int launch_identify(const DomainDev& d, cudaStream_t s) {
  if (d.g.dim == 2)
    k_identify<2><<<d.sm_count * 8, 256, 0, s>>>(d);
  else
    k_identify<3><<<d.sm_count * 8, 256, 0, s>>>(d);
  return 1;
}

int launch_decide(const DomainDev& d, bool full_domain, cudaStream_t s) {
  if (full_domain) {
    if (d.g.dim == 2)
      k_decide_full<2><<<d.sm_count * 8, 256, 0, s>>>(d);
    else
      k_decide_full<3><<<d.sm_count * 8, 256, 0, s>>>(d);
    return 1;
  }
  if (d.nseg == 0) return 0;
  const int warps = 8;
  int blocks = (d.nseg + warps - 1) / warps;
  if (blocks > d.sm_count * 16) blocks = d.sm_count * 16;
  if (d.g.dim == 2)
    k_decide<2><<<blocks, 32 * warps, 0, s>>>(d);
  else
    k_decide<3><<<blocks, 32 * warps, 0, s>>>(d);
  return 1;
}

int launch_apply(const DomainDev& d, cudaStream_t s) {
  if (d.g.dim == 2)
    k_apply<2><<<d.sm_count, kApplyThreads, 0, s>>>(d);
  else
    k_apply<3><<<d.sm_count, kApplyThreads, 0, s>>>(d);
  return 1;
}

}  // namespace sphbuf
