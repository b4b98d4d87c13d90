// The batched step as one persistent launch: every phase of a single-rate step with the
// buffer decisions fused into the force pass (neighbour lists + Eq. (9), deferred densities,
// force + kick + BC + drift + Algorithms 1-3, and the rebuild's histogram, three scans, keys,
// scatter + relabel, finalize) runs in one cooperative launch whose blocks are all resident;
// a grid barrier separates the phases.  Each phase walks the same block maps as the per-phase
// batched kernels (virtual blocks shared out over the domains), block by block, with the
// domain's descriptor in shared memory.
//
// Loads: inside one launch a phase reads what an earlier phase wrote in other blocks
// (densities, neighbour lists, decision records, the cell list), so the kernel bodies are
// compiled here with coherent loads (SPHBUF_LDG) instead of the read-only data path.
//
// Barrier: one arrival counter and one generation word in device memory, zeroed before every
// launch.  A block's first thread fences, arrives, and the last arrival opens the next
// generation; the others spin on the generation with a bounded number of iterations.  A
// spin that runs out (or finds the abort word set by another block) sets the abort word,
// latches SPHBUF_ERR_TIMEOUT in every domain of the batch and returns, so every block leaves
// the kernel after at most one bounded wait per barrier.
#define SPHBUF_LDG(p) (*(p))

#include "cells_bodies.cuh"
#include "sph_bodies.cuh"

namespace sphbuf {

namespace {

constexpr int kPersistThreads = 256;

enum PersistPhase : int {
  P_NEIGHBOURS,
  P_DENSITY,
  P_FORCE,
  P_HIST,
  P_SCAN_REDUCE,
  P_SCAN_TOP,
  P_SCAN_DOWN,
  P_KEYS,
  P_SCATTER,
  P_FINALIZE,
  P_COUNT
};

// Waits until every block of the grid has arrived (see the file comment); false when the
// wait gave up.  `gen` is this block's count of barriers passed in the launch.
__device__ __forceinline__ bool grid_barrier(const PersistDev& p, unsigned& gen) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned* vgen = p.bar + 1;
    volatile int* vabort = reinterpret_cast<volatile int*>(p.bar + 2);
    __threadfence();
    const unsigned arrived = atomicAdd(p.bar, 1u) + 1u;
    if (arrived == gridDim.x) {
      atomicExch(p.bar, 0u);
      __threadfence();
      atomicExch(p.bar + 1, gen + 1u);
    } else {
      long long it = 0;
      while (*vgen == gen) {
        if (*vabort || it >= p.spin_limit) {
          ok = 0;
          break;
        }
        ++it;
        __nanosleep(100);
      }
    }
    if (!ok) {
      atomicExch(p.bar + 2, 1u);
      for (int q = 0; q < p.ndom; ++q) atomicCAS(&p.doms[q].st->status, 0, 5 /* SPHBUF_ERR_TIMEOUT */);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  ++gen;
  return s_ok != 0;
}

template <int D, bool TVF>
__device__ __forceinline__ void run_phase(int ph, const DomainDev& d, unsigned lb, unsigned nb) {
  switch (ph) {
    case P_NEIGHBOURS:
      neighbours_body<D>(d, lb, nb);
      break;
    case P_DENSITY:
      density_deferred_body<D>(d, lb, nb);
      break;
    case P_FORCE:
      force_body<D, TVF>(d, lb, nb, true);
      break;
    case P_HIST:
      hist_body(d, lb, nb, 0);
      break;
    case P_SCAN_REDUCE:
      if (!d.st->status) scan_reduce_occ_body(d.cnt, d.scan_part, d.scan_part_occ, lb);
      break;
    case P_SCAN_TOP:
      if (!d.st->status) scan_top_occ_body(d.scan_part, d.scan_part_occ, d.scan_tiles, &d.st->n_occ);
      break;
    case P_SCAN_DOWN:
      if (!d.st->status) scan_down_occ_body(d.cnt, d.scan_part, d.scan_part_occ, d.cell_start, d.occ_list, lb);
      break;
    case P_KEYS:
      keys_body(d, lb, nb);
      break;
    case P_SCATTER:
      scatter_body<D>(d, lb, nb);
      break;
    default:
      finalize_body(d, 1, lb, nb);
  }
}

template <int D, bool TVF>
__global__ void __launch_bounds__(kPersistThreads, 3) k_step_persistent(PersistDev p) {
  __shared__ DomainDev sd;
  unsigned gen = 0;
  for (int ph = 0; ph < P_COUNT; ++ph) {
    if (ph > 0 && !grid_barrier(p, gen)) return;
    const int4* map = p.map[ph];
    for (int vb = blockIdx.x; vb < p.nvb[ph]; vb += gridDim.x) {
      const int4 m = map[vb];
      load_domain(sd, p.doms + m.x);
      run_phase<D, TVF>(ph, sd, (unsigned)m.y, (unsigned)m.z);
      __syncthreads();
    }
  }
}

template <int D, bool TVF>
int grid_of() {
  int per_sm = 0, dev = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_persistent<D, TVF>, kPersistThreads, 0) !=
          cudaSuccess ||
      cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  return per_sm * sms;
}

template <int D, bool TVF>
cudaError_t launch_t(const PersistDev& p, int grid, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kPersistThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_step_persistent<D, TVF>, p);
}

}  // namespace

static_assert(P_COUNT == kPersistPhases, "phases of the persistent step");

const int kPersistKern[kPersistPhases] = {K_NEIGHBOURS, K_DENSITY_DEFER, K_FORCE, K_HIST,    K_SCAN_REDUCE,
                                          K_SCAN_TOP,   K_SCAN_DOWN,     K_KEYS,  K_SCATTER, K_FINALIZE};

int persistent_grid(int dim, bool tvf) {
  if (dim == 2) return tvf ? grid_of<2, true>() : grid_of<2, false>();
  return tvf ? grid_of<3, true>() : grid_of<3, false>();
}

cudaError_t launch_persistent(const PersistDev& p, int dim, bool tvf, int grid, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(p.bar, 0, 4 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  if (dim == 2) return tvf ? launch_t<2, true>(p, grid, s) : launch_t<2, false>(p, grid, s);
  return tvf ? launch_t<3, true>(p, grid, s) : launch_t<3, false>(p, grid, s);
}

}  // namespace sphbuf
