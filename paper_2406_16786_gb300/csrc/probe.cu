// Launch-latency floor of a kernel with a given grid: the time a kernel that does nothing, or
// only one or two dependent loads per thread, takes when timed like the step's phases (CUDA
// events around one launch on the stream).  It is the floor against which the buffer update,
// a kernel of a few microseconds moving a few MB, is read.
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/sphbuf.h"

namespace {

__global__ void k_probe(const unsigned* __restrict__ idx, const unsigned* __restrict__ val, unsigned n, int loads,
                        unsigned* out) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned v = 0;
  if (loads >= 1) v = __ldg(idx + (t * 2654435761u) % n) % n;  // a scattered index
  if (loads >= 2) v = __ldg(val + v);                         // then what it points at
  if (v == 0xFFFFFFFFu) out[0] = v;                           // never true: keeps the loads
}

// idx[i] = (i * 40503) mod n: in range, scattered.
__global__ void k_probe_fill(unsigned* idx, unsigned n) {
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    idx[i] = (unsigned)(((unsigned long long)i * 40503ull) % n);
}

}  // namespace

extern "C" sphbuf_status sphbuf_probe_launch_floor(int blocks, int threads, int loads, int flush_l2, int reps,
                                                    void* cuda_stream, double* us_per_launch) {
  if (blocks < 1 || threads < 32 || threads > 1024 || loads < 0 || loads > 2 || reps < 1 || !us_per_launch)
    return SPHBUF_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const unsigned n = 1u << 24;             // 64 MB per array
  const size_t flush_bytes = 256u << 20;   // twice the L2
  unsigned *idx = nullptr, *val = nullptr, *out = nullptr;
  void* flush = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  sphbuf_status st = SPHBUF_ERR_CUDA;
  double total = 0.0;
  if (cudaMalloc(&idx, n * sizeof(unsigned)) != cudaSuccess) goto done;
  if (cudaMalloc(&val, n * sizeof(unsigned)) != cudaSuccess) goto done;
  if (cudaMalloc(&out, sizeof(unsigned)) != cudaSuccess) goto done;
  if (flush_l2 && cudaMalloc(&flush, flush_bytes) != cudaSuccess) goto done;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) goto done;
  k_probe_fill<<<1024, 256, 0, s>>>(idx, n);
  k_probe_fill<<<1024, 256, 0, s>>>(val, n);
  for (int r = -3; r < reps; ++r) {  // three untimed launches first
    if (flush_l2) cudaMemsetAsync(flush, r & 0xFF, flush_bytes, s);
    cudaEventRecord(e0, s);
    k_probe<<<blocks, threads, 0, s>>>(idx, val, n, loads, out);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) goto done;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (r >= 0) total += ms;
  }
  if (cudaGetLastError() != cudaSuccess) goto done;
  *us_per_launch = 1e3 * total / reps;
  st = SPHBUF_OK;
done:
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(idx);
  cudaFree(val);
  cudaFree(out);
  cudaFree(flush);
  return st;
}
