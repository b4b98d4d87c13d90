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
  float* rho_new;         // density pass output, capacity
  float4* pos4;           // A-order copies for the neighbour passes: (fx, fy, fz, cell x)
  float4* vel4;           //   and (vx, vy, vz, rho); written by the rebuild scatter
  const float4* wpos4;    // walls: (fx, fy, fz, cell x)
  unsigned* nb;           // neighbour lists, nb_cap entries per particle (16-byte aligned)
  unsigned* nb_cnt;       // neighbours found per particle (above nb_cap: direct path)
  int nb_cap;             // multiple of 4
  Decision* inj;          // decisions of the current step, list_cap each
  Decision* del;
  InjRecord* inj_sorted;  // injections in (buffer, parent id) order
  const BufDev* bufs;     // nbuf entries
  int nbuf;
  const int* relabel_ids; // buffers that relabel (outflow, bidirectional)
  int nrelabel;
  const int* seg_lin;     // candidate cell segments: [lin0, lin1) pairs
  const int* seg_buf;     // buffer of each segment
  int nseg;
  StepState* st;
  long long ncell_pad;
  int scan_tiles;
  int sm_count;
};

// sph (kernels_sph.cu)
int launch_neighbours(const DomainDev& d, cudaStream_t s);  // starts the step (step constants)
int launch_density(const DomainDev& d, cudaStream_t s);
int launch_force(const DomainDev& d, cudaStream_t s);
int launch_drift(const DomainDev& d, cudaStream_t s);
// buffer (kernels_buffer.cu)
int launch_identify(const DomainDev& d, cudaStream_t s);
int launch_decide(const DomainDev& d, bool full_domain, cudaStream_t s);
int launch_apply(const DomainDev& d, cudaStream_t s);
// cells (kernels_cells.cu)
int launch_rebuild(const DomainDev& d, bool count_step, cudaStream_t s);
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
