// Ids of the step's duplicates (Algorithm 1 generation, reading A5 of the numbering): the
// duplicate written for injection e at B[n + e] gets id next_id + r, r = the rank of
// (buffer, parent id) among the step's injections.  Run by the first threads of the rebuild's
// histogram pass before their share of the histogram; it needs every decision of the step,
// so it cannot run inside the buffer kernel without a grid-wide wait.  The count costs
// O(n_inj) reads per injection (cached), small next to the histogram for the few to a few
// thousand injections of a step.
#pragma once

#include "kernels.cuh"

namespace sphbuf {

__device__ __forceinline__ unsigned long long injection_key(const Decision* e) {
  return ((unsigned long long)SPHBUF_LDG(&e->k) << 32) | SPHBUF_LDG(&e->id);
}

// Thread t of the domain's blocks names injection t (grid-stride): rank = the number of
// smaller keys (keys are distinct), read through L1 from the step's injection list.
__device__ __forceinline__ void rank_injections(const DomainDev& d, unsigned bid, unsigned nblk) {
  const StepState* st = d.st;
  const unsigned n_inj = min(st->n_inj, d.P.list_cap);
  const unsigned n = st->n, next_id = st->next_id;
  const Decision* inj = d.inj;
  for (unsigned e = bid * blockDim.x + threadIdx.x; e < n_inj; e += nblk * blockDim.x) {
    const unsigned long long key = injection_key(inj + e);
    unsigned r = 0;
    for (unsigned q = 0; q < n_inj; ++q) r += injection_key(inj + q) < key;
    const unsigned child = next_id + r;
    d.B.id[n + e] = child;
    d.inj_sorted[r] = InjRecord{SPHBUF_LDG(&inj[e].k), SPHBUF_LDG(&inj[e].id), child};
  }
}

}  // namespace sphbuf
