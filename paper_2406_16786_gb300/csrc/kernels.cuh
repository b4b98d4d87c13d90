// Host-side launchers of the sphbuf kernels (one translation unit per kernel family).
#pragma once

#include "common.cuh"

namespace sphbuf {

struct DomainDev {
  Grid g;
  Phys P;
  Particles A, B;
  Walls W;
  unsigned* cell_start;   // A's cell-linked list, ncell_pad + 1 entries
  unsigned* cnt;          // per-cell counters (zero between rebuilds), ncell_pad entries
  unsigned* scan_part;    // per-tile partial sums
  unsigned* scan_part_occ;  // per-tile occupied-cell counts
  unsigned* occ_list;     // occupied cells in increasing order (st->n_occ entries)
  unsigned* slot;         // per-particle slot from the histogram, capacity
  unsigned* tmp_id;       // ids scattered to their cell's range, capacity
  float4* vr4;            // density pass output (vx, vy, vz, new rho) in A order, capacity
  float4* pos_b;          // dual-criteria scheme: second copy of pos4 and vr4 (acoustic steps
  float4* vr_b;           //   alternate between the two), and the viscous acceleration of
  float4* av;             //   the advection step
  unsigned* io;           // 8 words: host-transfer checks (error bits, largest id), bounds-check record
  unsigned* deferred;     // particles left by the fluid density pass (buffer or overflowed list)
  float4* pos4;           // A-order copies for the neighbour passes: (fx, fy, fz, cell x)
  float4* vel4;           //   and (vx, vy, vz, rho); written by the rebuild scatter
  const float4* wpos4;    // walls: (fx, fy, fz, cell x)
  unsigned* nb;           // neighbour lists, nb_cap entries per particle (16-byte aligned)
  unsigned* nb_cnt;       // neighbours found per particle (above nb_cap: direct path)
  int nb_cap;             // multiple of 4
  Decision* inj;          // decisions of the current step, list_cap each
  Decision* del;
  InjRecord* inj_sorted;  // injections in (buffer, parent id) order
  const BufDev* bufs;     // nbuf entries (frame fields of rotating buffers rewritten per step)
  RotDev* rot;            // kMaxBuffers entries: frame state of rotating buffers
  int any_rot;            // some buffer rotates (selects the buffer kernel with the turn)
  int nbuf;
  const int* relabel_ids; // buffers that relabel (outflow, bidirectional)
  int nrelabel;
  const int* seg_lin;     // candidate cell segments: [lin0, lin1) pairs
  const int* seg_buf;     // buffer of each segment
  uint4* seg_range;       // (cell_start[lin0], cell_start[lin1], lin0, buffer) of each segment
  int nseg;
  const unsigned* cand_mask;  // per cell: bit k set when the cell is a candidate cell of buffer k
  const uint8_t* s_mask;      // per cell: 1 where kept lists are rebuilt every step (candidate
                              //   cells and two rings of cells around them)
  unsigned* order;            // live particles' slots sorted by (cell, id) (kept lists)
  float* disp[3];             // per slot (kept lists): displacement since the last full list
                              //   build relative to the period's reference velocity
                              //   StepState::u0 (x < d allocated); only the slot's own drift
                              //   reads and writes it, so it stays in place between full
                              //   builds and is reset at each
  uint8_t* core;              // per slot, from the density pass with the transport velocity:
                              //   bit 0 core boundary particle, bit 1 candidate (reading A27)
  StepState* st;
  long long ncell_pad;
  int scan_tiles;
  int sm_count;
};

// Multi-domain (batched) launches: block b works for domain map[b].x as its local block
// map[b].y of map[b].z.
struct BatchDev {
  const DomainDev* doms;
  const int4* map;
};

enum Kern : int {
  K_BEGIN,  // step constants before a kinematic drift (one block per domain)
  K_NEIGHBOURS,
  K_DENSITY_DEFER,
  K_FORCE,
  K_DRIFT,
  K_VISCOUS,
  K_ACOUSTIC,
  K_DUAL_FINISH,
  K_BUFFER,
  K_BUFFER_FULL,
  K_HIST,
  K_SCAN_REDUCE,
  K_SCAN_TOP,
  K_SCAN_DOWN,
  K_KEYS,
  K_SCATTER,
  K_FINALIZE,
  K_COUNT
};

// The persistent batched step (kernels_persist.cu): one cooperative launch per step whose
// phases walk the per-kernel block maps of the batch, separated by grid barriers.
constexpr int kPersistPhases = 10;
extern const int kPersistKern[kPersistPhases];  // the Kern whose block map each phase walks
struct PersistDev {
  const DomainDev* doms;
  const int4* map[kPersistPhases];
  int nvb[kPersistPhases];
  unsigned* bar;         // 4 words: arrivals, generation, abort (zeroed before each launch)
  long long spin_limit;  // iterations a barrier wait may spin (about 100 ns each)
  int ndom;
};
int persistent_grid(int dim, bool tvf);  // resident blocks of the persistent step (0: error)
cudaError_t launch_persistent(const PersistDev& p, int dim, bool tvf, int grid, cudaStream_t s);

// Bounds-checked build (compiled with -DSPHBUF_CHECK, see build.py): SPHBUF_IN_BOUNDS(d, cond,
// site, index) is cond; when cond is false the first failing site and index go to io[2] and
// io[3] and SPHBUF_ERR_BOUNDS is latched, and the caller skips the access.  Without the flag
// the checks compile to nothing.  Sites: 1 fluid candidate, 2 wall candidate (neighbour
// search); 3 fluid entry, 4 wall entry (list visit); 5 cell walk; 6 particle cell; 7 deferred
// particle; 8 index-list place; 9 cell of the candidate mask; 10 rebuild cell.
// SPHBUF_IN_BOUNDS_AT(d, cond, site, index, who) also records the particle `who` with its
// list count, cell and the state's sort flag (io[4..7]).
#ifdef SPHBUF_CHECK
__device__ __forceinline__ bool bounds_ok(const DomainDev& d, bool cond, unsigned site, unsigned index,
                                          unsigned who) {
  if (!cond) {
    if (atomicCAS(&d.io[2], 0u, site) == 0u) {
      d.io[3] = index;
      d.io[4] = who;
      if (who != kNoSlot) {
        d.io[5] = d.nb_cnt[who];
        d.io[6] = (unsigned)d.A.cell[who];
      }
      d.io[7] = (unsigned)d.st->full | ((unsigned)d.st->since_full << 8);
    }
    latch(d.st, 8 /* SPHBUF_ERR_BOUNDS */);
  }
  return cond;
}
#define SPHBUF_IN_BOUNDS(d, cond, site, index) bounds_ok((d), (cond), (site), (unsigned)(index), kNoSlot)
#define SPHBUF_IN_BOUNDS_AT(d, cond, site, index, who) bounds_ok((d), (cond), (site), (unsigned)(index), (who))
#else
#define SPHBUF_IN_BOUNDS(d, cond, site, index) true
#define SPHBUF_IN_BOUNDS_AT(d, cond, site, index, who) true
#endif

// Copies one domain descriptor into shared memory (whole block; ends with a barrier).
__device__ __forceinline__ void load_domain(DomainDev& dst, const DomainDev* src) {
  const int words = (int)(sizeof(DomainDev) / sizeof(int));
  const int* s = reinterpret_cast<const int*>(src);
  int* t = reinterpret_cast<int*>(&dst);
  for (int q = threadIdx.x; q < words; q += blockDim.x) t[q] = s[q];
  __syncthreads();
}

// Batched launches with `threads` per block (up to 512).  fused: the buffer decisions
// (Algorithms 1-3) in the drift epilogue (decide.cuh); cpw: candidate cells per warp of the
// buffer kernel (1, 2, 4 or 8).
int launch_batch_sph(Kern k, int dim, const BatchDev& b, int nblocks, cudaStream_t s, bool tvf, int sub, bool fused,
                     int threads);
int launch_batch_buffer(Kern k, int dim, const BatchDev& b, int nblocks, bool rot, int threads, int cpw,
                        cudaStream_t s);
int launch_batch_cells(Kern k, int dim, const BatchDev& b, int nblocks, int threads, cudaStream_t s,
                       bool force_full = false);
int batch_threads(Kern k);  // threads per block of the batched kernels whose block size is fixed
bool batch_tunable(Kern k);  // may the autotuner choose the block size of this kernel?

// sph (kernels_sph.cu)
int launch_neighbours(const DomainDev& d, cudaStream_t s);  // starts the step (step constants)
int launch_density(const DomainDev& d, cudaStream_t s);  // two kernels: fluid, then deferred
int launch_force(const DomainDev& d, bool fused, cudaStream_t s);
int launch_drift(const DomainDev& d, bool fused, cudaStream_t s);
int launch_dual(const DomainDev& d, bool fused, cudaStream_t s);  // viscous, acoustic steps, fold (dual_n > 0)
// buffer (kernels_buffer.cu)
int launch_identify(const DomainDev& d, cudaStream_t s);
int launch_decide(const DomainDev& d, bool full_domain, cudaStream_t s);
// cells (kernels_cells.cu)
// force_full: sort the state whatever the kept-list policy says (kinematic steps, commits)
int launch_rebuild(const DomainDev& d, bool count_step, bool force_full, cudaStream_t s);
int finalize_blocks(const DomainDev& d);  // blocks of the finalize pass (candidate segments / 256)
// Host transfers: the AoS frac / vel arrays staged in device memory <-> the SoA state.
// ingest: B <- staged arrays (cell, rho, id, label already copied), with the checks of
// sphbuf_write_particles (io[0] bits: 1 cell, 2 offset, 4 label; io[1] = largest id).
void launch_ingest(const DomainDev& d, const float* frac, const float* vel, unsigned n, int ids_given,
                   int labels_given, int nbuf, cudaStream_t s);
// egest: staged AoS arrays <- P (the sorted state: A, or B after launch_view).
void launch_egest(const DomainDev& d, const Particles& P, float* frac, float* vel, unsigned n, cudaStream_t s);
// view: B <- the live particles of A in (cell, id) order through the index list (for reads of a
// state whose slots were kept by the last rebuild).
void launch_view(const DomainDev& d, cudaStream_t s);
// dst[k] = src[order[k]] for the n live particles (a per-slot byte field in sorted order).
void launch_gather_u8(const DomainDev& d, const uint8_t* src, uint8_t* dst, unsigned n, cudaStream_t s);
// Pipelined host transfers.  ingest_staged: B <- arrays of n particles staged in device memory
// (id / label NULL: 0..n-1 / 0), with the checks of sphbuf_write_particles; a failed check
// latches SPHBUF_ERR_INVALID_ARG and leaves the domain with no particles, otherwise n and
// next_id become the state's.  egest_staged: rows [0, min(n, cap)) of A into staged arrays and
// n (the particle count, from the device state) into *n_out.
void launch_ingest_staged(const DomainDev& d, const int* cell, const float* frac, const float* vel, const float* rho,
                          const unsigned* id, const uint8_t* label, unsigned n, unsigned next_id, int nbuf,
                          cudaStream_t s);
void launch_egest_staged(const DomainDev& d, int* cell, float* frac, float* vel, float* rho, unsigned* id,
                         uint8_t* label, unsigned* n_out, unsigned cap, cudaStream_t s);
void launch_decode_positions(const DomainDev& d, double* pos_out, const double lo[3], double cs,
                             cudaStream_t s);
cudaError_t cell_list_build(const int32_t* cell, const uint32_t* id, const uint8_t* label,
                            uint64_t n, uint64_t ncell, uint32_t* cell_start, uint32_t* order,
                            cudaStream_t s, int* bad_input);
// Same list with scratch in a fixed file-scope device array (no allocation).
unsigned long long cell_list_noalloc_max_particles();
unsigned long long cell_list_noalloc_max_cells();
cudaError_t cell_list_build_noalloc(const int32_t* cell, const uint32_t* id, const uint8_t* label,
                                    uint64_t n, uint64_t ncell, uint32_t* cell_start, uint32_t* order,
                                    cudaStream_t s, int* bad_input);

}  // namespace sphbuf
