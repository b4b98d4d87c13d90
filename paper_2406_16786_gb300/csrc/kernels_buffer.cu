// The arbitrary-positioned buffer (Sec. 3, Algorithms 1-3) on the GPU: one launch per step.
//
// decide: only the particles listed in the cells around each buffer's box are visited (four
//   candidate cells per warp, eight lanes per cell; label, cell and offset are loaded
//   together); each is transformed into the buffer's local frame (Eqs. (11), (15)) with the
//   FP32 decision contract and compared on the normal axis only.  Crossings are compacted with
//   a warp ballot and one atomic per warp into the injection / deletion lists.  The deciding
//   thread also does the work that does not depend on the injection order: it records the
//   parent's state (the duplicate's state), recycles the parent by -a u (Eqs. (16)-(17)),
//   resets its density for pressure buffers (Eq. (22)), and marks deleted particles dead.
// apply: the last block to finish (atomic ticket after a fence) ranks the injections by
//   (buffer, parent id) with a bitonic sort in shared memory (a pairwise rank count for very
//   long lists) and writes duplicate r at the tail of B with id next_id + r.
// The full-domain variant takes the same decisions over every particle and every buffer.
#include "kernels.cuh"

namespace sphbuf {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kBufThreads = 256;
constexpr int kSortCap = 2048;  // injections ranked by the in-block bitonic sort

// Warp-ballot compaction of one record per flagged lane into `list` (lanes may belong to
// different buffers; each flagged lane also counts itself in its buffer's counter).
__device__ __forceinline__ void emit(bool flag, const Decision& rec, Decision* list, unsigned* counter,
                                     unsigned long long* per_buffer, unsigned cap, StepState* st) {
  const unsigned m = __ballot_sync(kFull, flag);
  if (m == 0) return;
  const int lane = threadIdx.x & 31;
  unsigned base = 0;
  if (lane == 0) base = atomicAdd(counter, (unsigned)__popc(m));
  base = __shfl_sync(kFull, base, 0);
  if (flag) {
    atomicAdd(per_buffer, 1ull);
    const unsigned r = base + __popc(m & ((1u << lane) - 1u));
    if (r < cap)
      list[r] = rec;
    else
      latch(st, 2 /* SPHBUF_ERR_CAPACITY */);
  }
}

// Algorithms 1-3 for particle i of B against buffer k; the warp emits the decisions.
template <int D>
__device__ __forceinline__ void decide_emit(const DomainDev& d, int k, unsigned i, bool valid) {
  const BufDev& b = d.bufs[k];
  const Grid& g = d.g;
  bool inj = false, del = false;
  Decision rec;
  rec.k = (unsigned)k;
  rec.idx = i;
  rec.id = 0;
  rec.cell = 0;
  rec.rho = 0.f;
#pragma unroll
  for (int x = 0; x < 3; ++x) rec.f[x] = rec.v[x] = 0.f;
  int c[3] = {0, 0, 0};
  if (valid) {
    // independent loads, issued together
    const uint8_t lab = d.B.label[i];
    rec.cell = d.B.cell[i];
#pragma unroll
    for (int x = 0; x < 3; ++x) rec.f[x] = x < D ? d.B.f[x][i] : 0.f;
    rec.id = d.B.id[i];
    const bool test = (b.kind == KIND_OUTFLOW) ? (lab != kDead) : (lab == (uint8_t)b.label);
    if (test) {
      cell_coords(rec.cell, g, c);
      float X[3];
      if (b.kind == KIND_OUTFLOW) {
        // Algorithm 2: candidates within one cell of the box, deleted once X' > a/2
        local_coords<D>(b, c, rec.f, g.cs, X, D);
        bool cand = fabsf(X[0]) < b.da && fabsf(X[1]) < b.db;
        if (D == 3) cand = cand && fabsf(X[2]) < b.dc;
        del = cand && X[0] > b.ha;
      } else {
        // Algorithms 1 and 3: buffer particles crossing X' = a/2 generate; Algorithm 3 deletes
        // those crossing X' = -a/2
        local_coords<D>(b, c, rec.f, g.cs, X, 1);
        inj = X[0] > b.ha;
        if (b.kind == KIND_BIDIR) del = X[0] < -b.ha;
      }
    }
  }
  if (inj) {
#pragma unroll
    for (int x = 0; x < 3; ++x) rec.v[x] = x < D ? d.B.v[x][i] : 0.f;
    rec.rho = d.B.rho[i];
  }
  emit(inj, rec, d.inj, &d.st->n_inj, &d.st->injected[k], d.P.list_cap, d.st);
  if (inj) {
    // recycle the parent: r' - [a, 0, 0]^T mapped back, i.e. r - a u (same thread, after the
    // record captured the duplicate's state)
    bool ok = true;
#pragma unroll
    for (int x = 0; x < D; ++x) {
      float fx = rec.f[x];
      ok &= move_fold(fx, c[x], b.shift[x], g.cs);
      d.B.f[x][i] = fx;
    }
    const bool inside = ok && c[0] >= 0 && c[0] < g.nx && c[1] >= 0 && c[1] < g.ny && c[2] >= 0 && c[2] < g.nz;
    if (inside) {
      d.B.cell[i] = (c[2] * g.ny + c[1]) * g.nx + c[0];
    } else {
      d.B.label[i] = kDead;
      atomicAdd(&d.st->escaped_total, 1ull);
    }
    if (!b.vel_bc) d.B.rho[i] = d.st->rho_pb[k];  // Eq. (22)
  }
  if (del) d.B.label[i] = kDead;
  emit(del, rec, d.del, &d.st->n_del, &d.st->deleted[k], d.P.list_cap, d.st);
}

// Writes duplicate number r from its record.
template <int D>
__device__ __forceinline__ void write_duplicate(const DomainDev& d, const Decision* e, unsigned rank, unsigned n,
                                                unsigned next_id) {
  const unsigned dst = n + rank;
  const unsigned child = next_id + rank;
  d.B.cell[dst] = __ldcg(&e->cell);
#pragma unroll
  for (int x = 0; x < D; ++x) {
    d.B.f[x][dst] = __ldcg(&e->f[x]);
    d.B.v[x][dst] = __ldcg(&e->v[x]);
  }
  d.B.rho[dst] = __ldcg(&e->rho);
  d.B.id[dst] = child;
  d.B.label[dst] = 0;  // the duplicate is ordinary fluid (Algorithm 1)
  d.inj_sorted[rank] = InjRecord{__ldcg(&e->k), __ldcg(&e->id), child};
}

__device__ __forceinline__ unsigned long long inj_key(unsigned k, unsigned id) {
  return ((unsigned long long)k << 32) | id;
}

// Ranks the step's injections and writes the duplicates; run by one block.
template <int D>
__device__ void apply_all(const DomainDev& d, unsigned long long* keys, unsigned* idx) {
  StepState* st = d.st;
  const unsigned n_inj = min(__ldcg(&st->n_inj), d.P.list_cap);
  const unsigned n = st->n;
  const unsigned next_id = st->next_id;
  if (n_inj == 0 || __ldcg(&st->status)) return;
  if ((unsigned long long)n + n_inj > d.P.capacity) {
    if (threadIdx.x == 0) latch(st, 2 /* SPHBUF_ERR_CAPACITY */);
    return;
  }
  const Decision* inj = d.inj;
  if (n_inj <= (unsigned)kSortCap) {
    unsigned p2 = 1;
    while (p2 < n_inj) p2 <<= 1;
    for (unsigned e = threadIdx.x; e < p2; e += blockDim.x) {
      keys[e] = e < n_inj ? inj_key(__ldcg(&inj[e].k), __ldcg(&inj[e].id)) : ~0ull;
      idx[e] = e;
    }
    // bitonic sort of (key, entry) pairs, ascending keys (keys are distinct)
    for (unsigned size = 2; size <= p2; size <<= 1) {
      for (unsigned stride = size >> 1; stride > 0; stride >>= 1) {
        __syncthreads();
        for (unsigned t = threadIdx.x; t < (p2 >> 1); t += blockDim.x) {
          const unsigned lo = 2 * t - (t & (stride - 1));
          const unsigned hi = lo + stride;
          const bool up = (lo & size) == 0;
          const unsigned long long a = keys[lo], b = keys[hi];
          if ((a > b) == up) {
            keys[lo] = b;
            keys[hi] = a;
            const unsigned ti = idx[lo];
            idx[lo] = idx[hi];
            idx[hi] = ti;
          }
        }
      }
    }
    __syncthreads();
    for (unsigned r = threadIdx.x; r < n_inj; r += blockDim.x) write_duplicate<D>(d, inj + idx[r], r, n, next_id);
  } else {
    // long lists: rank = number of smaller keys
    for (unsigned e = threadIdx.x; e < n_inj; e += blockDim.x) {
      const unsigned long long key = inj_key(__ldcg(&inj[e].k), __ldcg(&inj[e].id));
      unsigned rank = 0;
      for (unsigned q = 0; q < n_inj; ++q) rank += inj_key(__ldcg(&inj[q].k), __ldcg(&inj[q].id)) < key;
      write_duplicate<D>(d, inj + e, rank, n, next_id);
    }
  }
}

// Decisions (restricted to candidate cells, or over all particles), then the duplicates by
// the last block to finish.
template <int D, bool FULL>
__device__ __forceinline__ void buffer_body(const DomainDev& d, unsigned bid, unsigned nblk) {
  __shared__ unsigned long long s_keys[kSortCap];
  __shared__ unsigned s_idx[kSortCap];
  __shared__ int s_last;
  const int lane = threadIdx.x & 31;
  const unsigned warp = (bid * blockDim.x + threadIdx.x) >> 5;
  const unsigned nwarps = (nblk * blockDim.x) >> 5;
  // every block takes part in the completion count, even after an error was latched
  if (d.st->status) {
  } else if (FULL) {
    const unsigned n = d.st->n;
    for (unsigned base = warp * 32; base < n; base += nwarps * 32) {
      const unsigned i = base + lane;
      for (int k = 0; k < d.nbuf; ++k) decide_emit<D>(d, k, i, i < n);
    }
  } else {
    // four candidate cells per warp, eight lanes per cell
    const unsigned grp = lane >> 3, gl = lane & 7;
    const unsigned nseg = (unsigned)d.nseg;
    for (unsigned s0 = warp * 4; s0 < nseg; s0 += nwarps * 4) {
      const unsigned s = s0 + grp;
      unsigned j0 = 0, j1 = 0;
      int k = 0;
      if (s < nseg) {
        const int lin0 = d.seg_lin[2 * s], lin1 = d.seg_lin[2 * s + 1];
        k = d.seg_buf[s];
        j0 = d.cell_start[lin0];
        j1 = d.cell_start[lin1];
      }
      const unsigned iters = __reduce_max_sync(kFull, (j1 - j0 + 7) >> 3);
      for (unsigned it = 0; it < iters; ++it) {
        const unsigned i = j0 + it * 8 + gl;
        decide_emit<D>(d, k, i, i < j1);
      }
    }
  }
  // the last block to finish writes the step's duplicates
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&d.st->done_blocks, 1u) == nblk - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  apply_all<D>(d, s_keys, s_idx);
  if (threadIdx.x == 0) d.st->done_blocks = 0;
}

template <int D, bool FULL>
__global__ void __launch_bounds__(kBufThreads) k_buffer(DomainDev d) {
  buffer_body<D, FULL>(d, blockIdx.x, gridDim.x);
}

template <int D, bool FULL>
__global__ void __launch_bounds__(kBufThreads) k_buffer_batch(BatchDev b) {
  __shared__ DomainDev sd;
  const int4 m = b.map[blockIdx.x];
  load_domain(sd, b.doms + m.x);
  buffer_body<D, FULL>(sd, (unsigned)m.y, (unsigned)m.z);
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

// Blocks of k_buffer resident at once (one wave: the last block's apply starts as soon as the
// decisions end).
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

int launch_decide(const DomainDev& d, bool full_domain, cudaStream_t s) {
  int blocks;
  if (full_domain) {
    blocks = d.g.dim == 2 ? one_wave(d, k_buffer<2, true>) : one_wave(d, k_buffer<3, true>);
  } else {
    const int cells_per_block = 4 * (kBufThreads / 32);
    blocks = (d.nseg + cells_per_block - 1) / cells_per_block;
    const int wave = d.g.dim == 2 ? one_wave(d, k_buffer<2, false>) : one_wave(d, k_buffer<3, false>);
    if (blocks > wave) blocks = wave;
    if (blocks < 1) blocks = 1;
  }
  if (d.g.dim == 2) {
    if (full_domain)
      k_buffer<2, true><<<blocks, kBufThreads, 0, s>>>(d);
    else
      k_buffer<2, false><<<blocks, kBufThreads, 0, s>>>(d);
  } else {
    if (full_domain)
      k_buffer<3, true><<<blocks, kBufThreads, 0, s>>>(d);
    else
      k_buffer<3, false><<<blocks, kBufThreads, 0, s>>>(d);
  }
  return 1;
}

int launch_apply(const DomainDev&, cudaStream_t) { return 0; }  // applied inside k_buffer

int launch_batch_buffer(Kern k, int dim, const BatchDev& b, int nblocks, cudaStream_t s) {
  if (k == K_BUFFER) {
    if (dim == 2)
      k_buffer_batch<2, false><<<nblocks, kBufThreads, 0, s>>>(b);
    else
      k_buffer_batch<3, false><<<nblocks, kBufThreads, 0, s>>>(b);
    return 1;
  }
  if (k == K_BUFFER_FULL) {
    if (dim == 2)
      k_buffer_batch<2, true><<<nblocks, kBufThreads, 0, s>>>(b);
    else
      k_buffer_batch<3, true><<<nblocks, kBufThreads, 0, s>>>(b);
    return 1;
  }
  return 0;
}

}  // namespace sphbuf
