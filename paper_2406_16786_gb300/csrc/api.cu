// C ABI of the sphbuf library: domain set-up, buffer frames, step orchestration, read-back.
// See include/sphbuf.h for the contract of every entry point.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "sphbuf.h"

using namespace sphbuf;

namespace {

constexpr int kPhases = 5;
// Neighbour lists pack particle indices into 25 bits (see kernels_sph.cu).
constexpr uint64_t kMaxParticles = (1ull << 25) - 1;

struct BufHost {
  double origin[3], R[9], extent[3];
  int bc;
  sphbuf_bc_params prm;
  bool rotating = false;
  RotDev rot{};
  double wk_pd0 = 0;  // initial Windkessel distal pressure
  double r_min = 0, r_max = 0;  // distances from the pivot swept by the dilated box
};

}  // namespace

struct sphbuf_domain {
  sphbuf_domain_desc desc{};
  DomainDev dev{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;
  double cs = 0;
  float cs32 = 0;
  int dims[3] = {1, 1, 1};
  long long ncell = 0;
  double mass_d = 0;
  std::vector<BufHost> bufs;
  std::vector<BufDev> bufs_dev;
  std::vector<void*> allocs;
  void* seg_mem = nullptr;
  unsigned* cand_mask = nullptr;  // per cell: candidate buffers (bit k), for the fused decisions
  uint8_t* s_mask = nullptr;      // per cell: kept neighbour lists are rebuilt every step there
  float* xfer = nullptr;          // staging of the blocking transfers' AoS arrays (2 x capacity x dim)
  std::vector<int> seg_host, segbuf_host;
  void* wall_mem = nullptr;
  uint64_t launches = 0;
  uint64_t graph_launches = 0;  // kernels in the instantiated graph
  bool committed = false;
  bool need_rebuild = false;
  bool labels_given = false;
  bool stepped = false;
  bool timing = false;
  cudaEvent_t ev[kPhases + 1] = {};
  double acc_ms[kPhases] = {};
  uint64_t timed_steps = 0;
  bool use_graph = false;
  cudaGraphExec_t graph = nullptr;
  unsigned graph_phases = 0;
  // pipelined host transfers (set up by the first asynchronous call): copies on two streams
  // of their own, staged in device memory, ordered against the domain's stream by events
  struct PendingRead {
    uint64_t* n_out;
    uint64_t cap;
    int slot;
  };
  cudaStream_t io_h2d = nullptr, io_d2h = nullptr;
  cudaEvent_t ev_ingest = nullptr, ev_h2d = nullptr, ev_egest = nullptr, ev_d2h = nullptr;
  unsigned char* in_stage = nullptr;
  unsigned char* out_stage = nullptr;
  unsigned* n_pinned = nullptr;  // host ring of the particle counts of pending reads
  int ring_next = 0;
  std::vector<PendingRead> reads;
  bool ingest_pending = false;
  uint64_t w_n = 0;
  uint32_t w_next_id = 0;
  bool w_ids = false, w_labels = false;
  std::string err;
};

namespace {

sphbuf_status fail(sphbuf_domain* d, sphbuf_status s, const std::string& msg) {
  if (d) d->err = msg;
  return s;
}

sphbuf_status cuda_fail(sphbuf_domain* d, cudaError_t e, const char* what) {
  return fail(d, SPHBUF_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                              \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail(d, e_, #call);    \
  } while (0)

template <typename T>
cudaError_t dalloc(sphbuf_domain* d, T** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
  if (e == cudaSuccess) {
    d->allocs.push_back(q);
    *p = static_cast<T*>(q);
  }
  return e;
}

double wendland_alpha(int dim, double h) {
  return dim == 2 ? 7.0 / (4.0 * M_PI * h * h) : 21.0 / (16.0 * M_PI * h * h * h);
}

double wendland_w(double r, double h, int dim) {
  const double q = r / h;
  const double t = std::max(1.0 - 0.5 * q, 0.0);
  return wendland_alpha(dim, h) * t * t * t * t * (2.0 * q + 1.0);
}

// Reference sum of Eq. (9): W over the full-support lattice of spacing dp, self included.
double lattice_sum_w0(int dim, double dp, double h) {
  const int m = (int)std::ceil(2.0 * h / dp) + 1;
  double s = 0;
  for (int i = -m; i <= m; ++i)
    for (int j = -m; j <= m; ++j)
      for (int k = (dim == 3 ? -m : 0); k <= (dim == 3 ? m : 0); ++k) {
        const double r = std::sqrt((double)(i * i + j * j + k * k)) * dp;
        if (r < 2.0 * h) s += wendland_w(r, h, dim);
      }
  return s;
}

// Host encoding of a global FP64 position into (cell coordinate, FP32 offset) per axis.
bool encode_axis(double x, double lo, double cs, float cs32, int n, int* c_out, float* f_out) {
  const double t = x - lo;
  double c = std::floor(t / cs);
  float f = (float)(t - c * cs);
  if (f >= cs32) {
    f = f - cs32;
    c += 1;
  }
  if (f < 0.f) {
    f = f + cs32;
    c -= 1;
  }
  if (f >= cs32) {
    f = 0.f;
    c += 1;
  }
  if (!(c >= 0 && c < n)) return false;
  *c_out = (int)c;
  *f_out = f;
  return true;
}

// Separating-axis test of two oriented boxes (centre, frame rows, half extents); 2-D uses
// the in-plane axes only.
bool obb_overlap(int dim, const double c1[3], const double R1[9], const double h1[3], const double c2[3],
                 const double R2[9], const double h2[3]) {
  std::vector<std::array<double, 3>> axes;
  auto row = [](const double R[9], int r) { return std::array<double, 3>{R[3 * r], R[3 * r + 1], R[3 * r + 2]}; };
  const int nr = dim;
  for (int r = 0; r < nr; ++r) axes.push_back(row(R1, r));
  for (int r = 0; r < nr; ++r) axes.push_back(row(R2, r));
  if (dim == 3)
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        auto u = row(R1, a), v = row(R2, b);
        std::array<double, 3> w{u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
        const double nn = std::sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
        if (nn > 1e-9) axes.push_back({w[0] / nn, w[1] / nn, w[2] / nn});
      }
  for (auto& ax : axes) {
    if (dim == 2) ax[2] = 0;
    auto proj = [&](const double R[9], const double h[3]) {
      double s = 0;
      for (int r = 0; r < nr; ++r) s += h[r] * std::fabs(R[3 * r] * ax[0] + R[3 * r + 1] * ax[1] + R[3 * r + 2] * ax[2]);
      return s;
    };
    const double dist = std::fabs((c2[0] - c1[0]) * ax[0] + (c2[1] - c1[1]) * ax[1] + (c2[2] - c1[2]) * ax[2]);
    if (dist > proj(R1, h1) + proj(R2, h2)) return false;
  }
  return true;
}

// Distances from a point C to the nearest and farthest points of an oriented box (centre O,
// frame rows R, half extents h).
void box_distances(int dim, const double C[3], const double O[3], const double R[9], const double h[3],
                   double* dmin, double* dmax) {
  double s2 = 0;
  for (int r = 0; r < dim; ++r) {
    double q = 0;
    for (int x = 0; x < dim; ++x) q += R[3 * r + x] * (C[x] - O[x]);
    const double e = std::max(std::fabs(q) - h[r], 0.0);
    s2 += e * e;
  }
  *dmin = std::sqrt(s2);
  double best = 0;
  const int ncorner = 1 << dim;
  for (int m = 0; m < ncorner; ++m) {
    double p2 = 0;
    for (int x = 0; x < dim; ++x) {
      double cx = O[x] - C[x];
      for (int r = 0; r < dim; ++r) cx += ((m >> r) & 1 ? h[r] : -h[r]) * R[3 * r + x];
      p2 += cx * cx;
    }
    best = std::max(best, p2);
  }
  *dmax = std::sqrt(best);
}

// Does the region swept by rotating buffer b (a shell about its pivot) meet the box?
bool swept_overlaps_box(int dim, const BufHost& b, const double O[3], const double R[9], const double h[3]) {
  double dmin = 0, dmax = 0;
  box_distances(dim, b.rot.C, O, R, h, &dmin, &dmax);
  return dmin <= b.r_max && dmax >= b.r_min;
}

sphbuf_status upload_buffers(sphbuf_domain* d) {
  CK(cudaMemcpy(const_cast<BufDev*>(d->dev.bufs), d->bufs_dev.data(), d->bufs_dev.size() * sizeof(BufDev),
                cudaMemcpyHostToDevice));
  std::vector<double> pd(d->bufs.size(), 0.0);
  for (size_t k = 0; k < d->bufs.size(); ++k) pd[k] = d->bufs[k].wk_pd0;
  if (!pd.empty())
    CK(cudaMemcpy(reinterpret_cast<char*>(d->dev.st) + offsetof(StepState, wk_pd), pd.data(), pd.size() * sizeof(double),
                  cudaMemcpyHostToDevice));
  std::vector<RotDev> rot(d->bufs.size());
  for (size_t k = 0; k < d->bufs.size(); ++k) rot[k] = d->bufs[k].rot;
  if (!rot.empty()) CK(cudaMemcpy(d->dev.rot, rot.data(), rot.size() * sizeof(RotDev), cudaMemcpyHostToDevice));
  std::vector<int> rel;
  for (size_t k = 0; k < d->bufs_dev.size(); ++k)
    if (d->bufs_dev[k].kind != KIND_INFLOW) rel.push_back((int)k);
  if (!rel.empty())
    CK(cudaMemcpy(const_cast<int*>(d->dev.relabel_ids), rel.data(), rel.size() * sizeof(int), cudaMemcpyHostToDevice));
  d->dev.nbuf = (int)d->bufs_dev.size();
  d->dev.nrelabel = (int)rel.size();
  return SPHBUF_OK;
}

// Candidate cells of every buffer (Sec. 3.1: the local cell-linked lists around the box):
// cells that can hold, before this step's drift, a particle the decision has to see.
// Inflow/bidirectional: box dilated by one cell (movement within a step); outflow: box
// dilated by the candidate margin cs plus one cell.  A cell is kept when its centre passes
// the separating-axis test on the box axes against the dilated box (a superset of the cells
// the region touches).  One [lin, lin + 1) segment per candidate cell.
sphbuf_status build_segments(sphbuf_domain* d) {
  const int D = d->desc.dim;
  const double cs = d->cs;
  std::vector<int> seg;
  std::vector<int> segbuf;
  for (size_t k = 0; k < d->bufs.size(); ++k) {
    const BufHost& b = d->bufs[k];
    if (b.rotating) {
      // Sec. 5.3: every cell the dilated box can reach while it turns about the pivot, i.e.
      // cells whose centre lies within [r_min - rad, r_max + rad] of the pivot
      const double rad = 0.5 * cs * std::sqrt((double)D);
      int lo_c[3] = {0, 0, 0}, hi_c[3] = {0, 0, 0};
      for (int x = 0; x < D; ++x) {
        lo_c[x] = std::max(0, (int)std::floor((b.rot.C[x] - b.r_max - rad - d->desc.lo[x]) / cs));
        hi_c[x] = std::min(d->dims[x] - 1, (int)std::floor((b.rot.C[x] + b.r_max + rad - d->desc.lo[x]) / cs));
      }
      for (int cz = lo_c[2]; cz <= hi_c[2]; ++cz)
        for (int cy = lo_c[1]; cy <= hi_c[1]; ++cy)
          for (int cx = lo_c[0]; cx <= hi_c[0]; ++cx) {
            const int cc[3] = {cx, cy, cz};
            double r2 = 0;
            for (int x = 0; x < D; ++x) {
              const double e = d->desc.lo[x] + (cc[x] + 0.5) * cs - b.rot.C[x];
              r2 += e * e;
            }
            const double r = std::sqrt(r2);
            if (r > b.r_max + rad || r < b.r_min - rad) continue;
            const int lin = (cz * d->dims[1] + cy) * d->dims[0] + cx;
            seg.push_back(lin);
            seg.push_back(lin + 1);
            segbuf.push_back((int)k);
          }
      continue;
    }
    const double dil = (d->bufs_dev[k].kind == KIND_OUTFLOW) ? 2.0 * cs : cs;
    double half[3] = {0.5 * b.extent[0] + dil, 0.5 * b.extent[1] + dil, D == 3 ? 0.5 * b.extent[2] + dil : 0.0};
    // AABB of the dilated box in cell coordinates
    int lo_c[3] = {0, 0, 0}, hi_c[3] = {0, 0, 0};
    for (int x = 0; x < D; ++x) {
      double ext = 0;
      for (int r = 0; r < D; ++r) ext += half[r] * std::fabs(b.R[3 * r + x]);
      ext += cs;
      lo_c[x] = std::max(0, (int)std::floor((b.origin[x] - ext - d->desc.lo[x]) / cs));
      hi_c[x] = std::min(d->dims[x] - 1, (int)std::floor((b.origin[x] + ext - d->desc.lo[x]) / cs));
    }
    double rad[3] = {0, 0, 0};
    for (int r = 0; r < D; ++r)
      for (int x = 0; x < D; ++x) rad[r] += 0.5 * cs * std::fabs(b.R[3 * r + x]);
    for (int cz = lo_c[2]; cz <= hi_c[2]; ++cz)
      for (int cy = lo_c[1]; cy <= hi_c[1]; ++cy)
        for (int cx = lo_c[0]; cx <= hi_c[0]; ++cx) {
          const int cc[3] = {cx, cy, cz};
          double ctr[3] = {0, 0, 0};
          for (int x = 0; x < D; ++x) ctr[x] = d->desc.lo[x] + (cc[x] + 0.5) * cs - b.origin[x];
          bool keep = true;
          for (int r = 0; r < D; ++r) {
            double X = 0;
            for (int x = 0; x < D; ++x) X += b.R[3 * r + x] * ctr[x];
            if (std::fabs(X) > half[r] + rad[r]) keep = false;
          }
          if (!keep) continue;
          const int lin = (cz * d->dims[1] + cy) * d->dims[0] + cx;
          seg.push_back(lin);
          seg.push_back(lin + 1);
          segbuf.push_back((int)k);
        }
  }
  if (d->seg_mem) {
    cudaFree(d->seg_mem);
    d->seg_mem = nullptr;
  }
  // per-cell mask of the candidate buffers: the fused form decides a particle against the
  // buffers whose candidate cells hold the cell it was sorted into
  std::vector<unsigned> mask((size_t)d->ncell, 0u);
  for (size_t q = 0; q < segbuf.size(); ++q)
    for (int lin = seg[2 * q]; lin < seg[2 * q + 1]; ++lin) mask[(size_t)lin] |= 1u << segbuf[q];
  if (!d->cand_mask) CK(cudaMalloc(&d->cand_mask, std::max<size_t>((size_t)d->ncell, 1) * sizeof(unsigned)));
  CK(cudaMemcpy(d->cand_mask, mask.data(), mask.size() * sizeof(unsigned), cudaMemcpyHostToDevice));
  d->dev.cand_mask = d->cand_mask;
  // every-step region of kept neighbour lists: the candidate cells (duplicates appear there,
  // parents are recycled there) and two rings of cells around them, so that no kept list
  // (radius 2h + skin < 2 cells) can reach a particle that appeared or jumped in this step
  std::vector<uint8_t> smask((size_t)d->ncell, 0);
  for (size_t lin = 0; lin < mask.size(); ++lin) {
    if (!mask[lin]) continue;
    const int cx = (int)(lin % d->dims[0]), cy = (int)((lin / d->dims[0]) % d->dims[1]),
              cz = (int)(lin / ((size_t)d->dims[0] * d->dims[1]));
    for (int dz = (D == 3 ? -2 : 0); dz <= (D == 3 ? 2 : 0); ++dz)
      for (int dy = -2; dy <= 2; ++dy)
        for (int dx = -2; dx <= 2; ++dx) {
          const int x = cx + dx, y = cy + dy, z = cz + dz;
          if (x < 0 || y < 0 || z < 0 || x >= d->dims[0] || y >= d->dims[1] || z >= d->dims[2]) continue;
          smask[((size_t)z * d->dims[1] + y) * d->dims[0] + x] = 1;
        }
  }
  if (!d->s_mask) CK(cudaMalloc(&d->s_mask, std::max<size_t>((size_t)d->ncell, 1)));
  CK(cudaMemcpy(d->s_mask, smask.data(), smask.size(), cudaMemcpyHostToDevice));
  d->dev.s_mask = d->s_mask;
  const size_t nseg = segbuf.size();
  // [seg_range: 4 nseg words, 16-byte aligned][seg_lin: 2 nseg][seg_buf: nseg]; the ranges
  // are written by every rebuild (the first one runs before the first step)
  const size_t bytes = (4 * nseg + 2 * nseg + nseg) * sizeof(int);
  CK(cudaMalloc(&d->seg_mem, std::max<size_t>(bytes, 16)));
  int* p = static_cast<int*>(d->seg_mem);
  CK(cudaMemset(p, 0, std::max<size_t>(bytes, 16)));
  if (nseg) {
    CK(cudaMemcpy(p + 4 * nseg, seg.data(), 2 * nseg * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(p + 6 * nseg, segbuf.data(), nseg * sizeof(int), cudaMemcpyHostToDevice));
  }
  d->dev.seg_range = reinterpret_cast<uint4*>(p);
  d->dev.seg_lin = p + 4 * nseg;
  d->dev.seg_buf = p + 6 * nseg;
  d->dev.nseg = (int)nseg;
  d->seg_host = seg;
  d->segbuf_host = segbuf;
  return SPHBUF_OK;
}

template <typename T>
sphbuf_status set_state_field(sphbuf_domain* d, size_t offset, T value) {
  CK(cudaMemcpyAsync(reinterpret_cast<char*>(d->dev.st) + offset, &value, sizeof(T), cudaMemcpyHostToDevice,
                     d->stream));
  CK(cudaStreamSynchronize(d->stream));
  return SPHBUF_OK;
}

sphbuf_status read_state(sphbuf_domain* d, StepState* out) {
  CK(cudaStreamSynchronize(d->stream));
  CK(cudaMemcpy(out, d->dev.st, sizeof(StepState), cudaMemcpyDeviceToHost));
  if (out->status) {
    const char* what = out->status == SPHBUF_ERR_CAPACITY      ? "particle or decision-list capacity exceeded"
                       : out->status == SPHBUF_ERR_NAN         ? "non-finite particle position"
                       : out->status == SPHBUF_ERR_TIMEOUT     ? "a grid-barrier wait of the persistent batched step "
                                                                 "ran out of its spin limit"
                       : out->status == SPHBUF_ERR_BOUNDS      ? "an index check failed (bounds-checked build)"
                       : out->status == SPHBUF_ERR_INVALID_ARG ? "asynchronously written arrays failed the checks "
                                                                 "(cell, offset, label or next_id)"
                                                               : "device-side error";
    if (out->status == SPHBUF_ERR_BOUNDS) {
      unsigned io[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      cudaMemcpy(io, d->dev.io, sizeof(io), cudaMemcpyDeviceToHost);
      return fail(d, SPHBUF_ERR_BOUNDS,
                  std::string(what) + ": site " + std::to_string(io[2]) + ", index " + std::to_string(io[3]) +
                      ", particle " + std::to_string(io[4]) + " (list count " + std::to_string(io[5]) + ", cell " +
                      std::to_string(io[6]) + "), sorted " + std::to_string(io[7] & 255u) + ", steps since sort " +
                      std::to_string(io[7] >> 8));
    }
    return fail(d, (sphbuf_status)out->status, what);
  }
  return SPHBUF_OK;
}

// Device staging of the pipelined transfers: the six particle arrays of up to C particles
// (cell, frac rows, vel rows, rho, id, label) and a count word.
struct Stage {
  int* cell;
  float* frac;
  float* vel;
  float* rho;
  unsigned* id;
  uint8_t* label;
  unsigned* count;
};

size_t stage_bytes(size_t C, int D) { return ((13 * C + 8 * C * (size_t)D + 15) / 16) * 16 + 16; }

Stage stage_of(unsigned char* base, size_t C, int D) {
  Stage s;
  s.cell = reinterpret_cast<int*>(base);
  s.frac = reinterpret_cast<float*>(base + 4 * C);
  s.vel = reinterpret_cast<float*>(base + 4 * C + 4 * C * D);
  s.rho = reinterpret_cast<float*>(base + 4 * C + 8 * C * D);
  s.id = reinterpret_cast<unsigned*>(base + 8 * C + 8 * C * D);
  s.label = base + 12 * C + 8 * C * D;
  s.count = reinterpret_cast<unsigned*>(base + stage_bytes(C, D) - 16);
  return s;
}

constexpr int kIoRing = 64;  // pending asynchronous reads at most

sphbuf_status ensure_io(sphbuf_domain* d) {
  if (d->io_h2d) return SPHBUF_OK;
  const size_t C = d->desc.capacity;
  const int D = d->desc.dim;
  // each piece only once (a call that failed half-way is retried by the next one)
  if (!d->in_stage) CK(dalloc(d, &d->in_stage, stage_bytes(C, D)));
  if (!d->out_stage) CK(dalloc(d, &d->out_stage, stage_bytes(C, D)));
  if (!d->n_pinned)
    CK(cudaHostAlloc(reinterpret_cast<void**>(&d->n_pinned), kIoRing * sizeof(unsigned), cudaHostAllocDefault));
  for (cudaEvent_t* e : {&d->ev_ingest, &d->ev_h2d, &d->ev_egest, &d->ev_d2h})
    if (!*e) CK(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  if (!d->io_d2h) CK(cudaStreamCreateWithFlags(&d->io_d2h, cudaStreamNonBlocking));
  CK(cudaStreamCreateWithFlags(&d->io_h2d, cudaStreamNonBlocking));  // set last: marks the set-up done
  return SPHBUF_OK;
}

sphbuf_status commit(sphbuf_domain* d) {
  sphbuf_status s;
  if (!d->committed) {
    if ((s = upload_buffers(d)) != SPHBUF_OK) return s;
    if ((s = build_segments(d)) != SPHBUF_OK) return s;
    if (!d->dev.W.start) {
      // no walls: an empty wall list
      unsigned* ws = nullptr;
      CK(dalloc(d, &ws, (size_t)d->ncell + 1));
      CK(cudaMemset(ws, 0, ((size_t)d->ncell + 1) * sizeof(unsigned)));
      d->dev.W.start = ws;
      float4* wp4 = nullptr;
      CK(dalloc(d, &wp4, 1));
      d->dev.wpos4 = wp4;
    }
    d->committed = true;
  }
  if (d->need_rebuild) {
    if (d->ingest_pending) {
      // the staged arrays of an asynchronous write, once their copies have landed
      CK(cudaStreamWaitEvent(d->stream, d->ev_h2d, 0));
      const Stage in = stage_of(d->in_stage, d->desc.capacity, d->desc.dim);
      launch_ingest_staged(d->dev, in.cell, in.frac, in.vel, in.rho, d->w_ids ? in.id : nullptr,
                           d->w_labels ? in.label : nullptr, (unsigned)d->w_n, d->w_next_id, (int)d->bufs.size(),
                           d->stream);
      CK(cudaGetLastError());
      CK(cudaEventRecord(d->ev_ingest, d->stream));
      d->launches += d->w_n ? 2 : 1;
      d->ingest_pending = false;
    }
    if (!d->labels_given) d->launches += launch_identify(d->dev, d->stream);
    d->launches += launch_rebuild(d->dev, false, true, d->stream);
    CK(cudaGetLastError());
    d->need_rebuild = false;
  }
  return SPHBUF_OK;
}

// Are the step's buffer decisions fused into the drift epilogue?  Not for the all-particle
// check, on request (SPHBUF_PHASE_BUFFER_KERNEL), or when a buffer rotates (its particles turn
// in the buffer kernel).
bool fused_decisions(unsigned phases, bool any_rot) {
  return (phases & SPHBUF_PHASE_BUFFER) && !(phases & (SPHBUF_PHASE_FULL_CHECK | SPHBUF_PHASE_BUFFER_KERNEL)) &&
         !any_rot;
}

// Enqueues the kernels of one step; returns the number of kernels launched.
int enqueue_step(sphbuf_domain* d, unsigned phases, bool timed) {
  const DomainDev& v = d->dev;
  cudaStream_t s = d->stream;
  const bool fused = fused_decisions(phases, v.any_rot != 0);
  // phases timed: [neighbour lists, density, force (or drift), buffer update, rebuild]; the
  // fused decisions are timed with the force (or drift) phase
  int k = 0;
  if (timed) cudaEventRecord(d->ev[0], s);
  if (phases & SPHBUF_PHASE_PHYSICS) {
    k += launch_neighbours(v, s);
    if (timed) cudaEventRecord(d->ev[1], s);
    k += launch_density(v, s);
    if (timed) cudaEventRecord(d->ev[2], s);
    k += v.P.dual_n > 0 ? launch_dual(v, fused, s) : launch_force(v, fused, s);
  } else {
    if (timed) cudaEventRecord(d->ev[1], s);
    if (timed) cudaEventRecord(d->ev[2], s);
    k += launch_drift(v, fused, s);
  }
  if (timed) cudaEventRecord(d->ev[3], s);
  if ((phases & SPHBUF_PHASE_BUFFER) && !fused) {
    k += launch_decide(v, (phases & SPHBUF_PHASE_FULL_CHECK) != 0, s);
  }
  if (timed) cudaEventRecord(d->ev[4], s);
  // kinematic steps use no lists: they end with a sorted state
  k += launch_rebuild(v, true, (phases & SPHBUF_PHASE_KINEMATIC) != 0, s);
  if (timed) cudaEventRecord(d->ev[5], s);
  return k;
}

}  // namespace

extern "C" {

const char* sphbuf_status_string(sphbuf_status s) {
  switch (s) {
    case SPHBUF_OK: return "ok";
    case SPHBUF_ERR_INVALID_ARG: return "invalid argument";
    case SPHBUF_ERR_CAPACITY: return "capacity exceeded";
    case SPHBUF_ERR_OVERLAP: return "buffer regions overlap";
    case SPHBUF_ERR_CUDA: return "CUDA error";
    case SPHBUF_ERR_TIMEOUT: return "device wait timed out";
    case SPHBUF_ERR_NAN: return "non-finite value";
    case SPHBUF_ERR_STATE: return "call not valid in the current state";
    case SPHBUF_ERR_BOUNDS: return "index out of bounds (bounds-checked build)";
  }
  return "unknown status";
}

const char* sphbuf_error_message(sphbuf_domain_t d) { return d ? d->err.c_str() : ""; }

sphbuf_status sphbuf_create_domain(const sphbuf_domain_desc* desc, void* cuda_stream, sphbuf_domain_t* out) {
  if (!desc || !out) return SPHBUF_ERR_INVALID_ARG;
  *out = nullptr;
  if (desc->dim != 2 && desc->dim != 3) return SPHBUF_ERR_INVALID_ARG;
  if (!(desc->dp > 0) || !(desc->h_over_dp > 0) || !(desc->rho0 > 0) || !(desc->c0 > 0) || !(desc->dt > 0) ||
      !(desc->nu >= 0) || desc->capacity == 0 || desc->capacity > kMaxParticles)
    return SPHBUF_ERR_INVALID_ARG;
  auto* d = new sphbuf_domain();
  d->desc = *desc;
  const int D = desc->dim;
  d->cs = 2.0 * (desc->h_over_dp * desc->dp);
  d->cs32 = (float)d->cs;
  for (int x = 0; x < 3; ++x) {
    if (x < D) {
      if (!(desc->hi[x] > desc->lo[x])) {
        delete d;
        return SPHBUF_ERR_INVALID_ARG;
      }
      d->dims[x] = (int)std::ceil((desc->hi[x] - desc->lo[x]) / d->cs);
    } else {
      d->dims[x] = 1;
    }
  }
  d->ncell = (long long)d->dims[0] * d->dims[1] * d->dims[2];
  if (d->ncell >= (1ll << 31) - kScanTile || d->dims[0] > kMaxCellsX || d->dims[1] > kMaxCellsY ||
      d->dims[2] > kMaxCellsZ) {
    delete d;
    return SPHBUF_ERR_INVALID_ARG;
  }
  cudaGetDevice(&d->device);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d->device);
  if (cuda_stream) {
    d->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&d->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete d;
      return SPHBUF_ERR_CUDA;
    }
    d->own_stream = true;
  }
  DomainDev& v = d->dev;
  v.sm_count = sms > 0 ? sms : 1;
  v.g.dim = D;
  v.g.nx = d->dims[0];
  v.g.ny = d->dims[1];
  v.g.nz = d->dims[2];
  v.g.ncell = d->ncell;
  v.g.cs = d->cs32;
  const double h = desc->h_over_dp * desc->dp;
  Phys& P = v.P;
  P.h = (float)h;
  P.inv_h = (float)(1.0 / h);
  P.two_h_sq = (float)(4.0 * h * h);
  P.alpha = (float)wendland_alpha(D, h);
  P.rho0 = (float)desc->rho0;
  P.c0 = (float)desc->c0;
  P.c0sq = (float)(desc->c0 * desc->c0);
  P.eta = (float)(desc->rho0 * desc->nu);
  d->mass_d = desc->rho0 * std::pow(desc->dp, D);
  P.mass = (float)d->mass_d;
  P.dt = (float)desc->dt;
  P.inv_sum_w0 = (float)(1.0 / lattice_sum_w0(D, desc->dp, h));
  P.w_self = (float)wendland_w(0.0, h, D);
  P.rho0_d = desc->rho0;
  P.c0sq_d = desc->c0 * desc->c0;
  P.dt_d = desc->dt;
  for (int x = 0; x < 3; ++x) P.lo_d[x] = desc->lo[x];
  P.cs_d = d->cs;
  P.capacity = (unsigned)desc->capacity;
  P.list_cap = (unsigned)std::max<uint64_t>(1024, std::min<uint64_t>(desc->capacity, 1ull << 22));
  P.psi_cand = (float)(0.75 * D);
  P.vol = (float)std::pow(desc->dp, D);
  P.reuse = 0;
  P.list_r2 = P.two_h_sq;
  P.skin = 0.f;
  P.reuse_max = 1;
  const size_t C = desc->capacity;
  v.ncell_pad = (d->ncell + 1 + kScanTile - 1) / kScanTile * kScanTile;
  v.scan_tiles = (int)(v.ncell_pad / kScanTile);
  cudaError_t e = cudaSuccess;
  auto A = [&](cudaError_t r) {
    if (e == cudaSuccess) e = r;
  };
  for (Particles* p : {&v.A, &v.B}) {
    A(dalloc(d, &p->cell, C));
    for (int x = 0; x < 3; ++x) {
      p->f[x] = nullptr;
      p->v[x] = nullptr;
      if (x < D) {
        A(dalloc(d, &p->f[x], C));
        A(dalloc(d, &p->v[x], C));
      }
    }
    A(dalloc(d, &p->rho, C));
    A(dalloc(d, &p->id, C));
    A(dalloc(d, &p->label, C));
    A(dalloc(d, &p->bflag, C));
  }
  A(dalloc(d, &v.order, C));
  for (int x = 0; x < 3; ++x) {
    v.disp[x] = nullptr;
    if (x < D) A(dalloc(d, &v.disp[x], C));
  }
  A(dalloc(d, &v.core, C));
  A(dalloc(d, &v.vr4, C));
  A(dalloc(d, &v.deferred, C));
  // neighbour lists of the density pass, reused by the force pass (~80 neighbours in 3-D and
  // ~20 in 2-D at h = 1.3 dp on the lattice; headroom for compression)
  v.nb_cap = D == 3 ? 128 : 48;
  A(dalloc(d, &v.nb, C * (size_t)v.nb_cap));
  A(dalloc(d, &v.pos4, C));
  A(dalloc(d, &v.vel4, C));
  A(dalloc(d, &v.nb_cnt, C));
  A(dalloc(d, &v.slot, C));
  A(dalloc(d, &v.tmp_id, C));
  A(dalloc(d, &v.cell_start, (size_t)v.ncell_pad + 1));
  A(dalloc(d, &v.cnt, (size_t)v.ncell_pad));
  A(dalloc(d, &v.scan_part, (size_t)v.scan_tiles));
  A(dalloc(d, &v.scan_part_occ, (size_t)v.scan_tiles));
  A(dalloc(d, &v.occ_list, std::min<size_t>((size_t)d->ncell, C) + 1));
  A(dalloc(d, &v.inj, P.list_cap));
  A(dalloc(d, &v.del, P.list_cap));
  A(dalloc(d, &v.inj_sorted, P.list_cap));
  BufDev* bd = nullptr;
  A(dalloc(d, &bd, kMaxBuffers));
  v.bufs = bd;
  A(dalloc(d, &v.rot, kMaxBuffers));
  int* rel = nullptr;
  A(dalloc(d, &rel, kMaxBuffers));
  v.relabel_ids = rel;
  A(dalloc(d, &v.st, 1));
  A(dalloc(d, &v.io, 8));
  if (e == cudaSuccess) {
    A(cudaMemset(v.io, 0, 8 * sizeof(unsigned)));
    // list entries that no search has written read as an index beyond any particle (caught by
    // the bounds-checked build), and list counts start at 0
    A(cudaMemset(v.nb, 0xFF, C * (size_t)v.nb_cap * sizeof(unsigned)));
    A(cudaMemset(v.nb_cnt, 0, C * sizeof(unsigned)));
    A(cudaMemset(v.cnt, 0, (size_t)v.ncell_pad * sizeof(unsigned)));
    A(cudaMemset(v.cell_start, 0, ((size_t)v.ncell_pad + 1) * sizeof(unsigned)));
    A(cudaMemset(v.st, 0, sizeof(StepState)));
  }
  for (int q = 0; q <= kPhases && e == cudaSuccess; ++q) A(cudaEventCreate(&d->ev[q]));
  if (e != cudaSuccess) {
    sphbuf_destroy(d);
    return SPHBUF_ERR_CUDA;
  }
  *out = d;
  return SPHBUF_OK;
}

sphbuf_status sphbuf_destroy(sphbuf_domain_t d) {
  if (!d) return SPHBUF_ERR_INVALID_ARG;
  if (d->stream) cudaStreamSynchronize(d->stream);
  for (cudaStream_t s : {d->io_h2d, d->io_d2h})
    if (s) {
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    }
  for (cudaEvent_t e : {d->ev_ingest, d->ev_h2d, d->ev_egest, d->ev_d2h})
    if (e) cudaEventDestroy(e);
  if (d->n_pinned) cudaFreeHost(d->n_pinned);
  if (d->graph) cudaGraphExecDestroy(d->graph);
  for (void* p : d->allocs) cudaFree(p);
  if (d->seg_mem) cudaFree(d->seg_mem);
  if (d->cand_mask) cudaFree(d->cand_mask);
  if (d->s_mask) cudaFree(d->s_mask);
  for (int q = 0; q <= kPhases; ++q)
    if (d->ev[q]) cudaEventDestroy(d->ev[q]);
  if (d->own_stream) cudaStreamDestroy(d->stream);
  delete d;
  return SPHBUF_OK;
}

sphbuf_status sphbuf_set_walls(sphbuf_domain_t d, const double* pos, uint64_t n) {
  if (!d || (!pos && n)) return SPHBUF_ERR_INVALID_ARG;
  if (n > kMaxParticles) return fail(d, SPHBUF_ERR_CAPACITY, "too many wall particles");
  if (d->stepped) return fail(d, SPHBUF_ERR_STATE, "walls must be set before the first step");
  const int D = d->desc.dim;
  std::vector<int> cell(n);
  std::vector<float> f((size_t)n * 3, 0.f);
  for (uint64_t i = 0; i < n; ++i) {
    int c[3] = {0, 0, 0};
    for (int x = 0; x < D; ++x)
      if (!encode_axis(pos[i * D + x], d->desc.lo[x], d->cs, d->cs32, d->dims[x], &c[x], &f[i * 3 + x]))
        return fail(d, SPHBUF_ERR_INVALID_ARG, "wall particle outside the grid box");
    cell[i] = (c[2] * d->dims[1] + c[1]) * d->dims[0] + c[0];
  }
  std::vector<uint64_t> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](uint64_t a, uint64_t b) { return cell[a] < cell[b]; });
  std::vector<unsigned> start((size_t)d->ncell + 1, 0);
  for (uint64_t i = 0; i < n; ++i) start[cell[i] + 1]++;
  for (long long c = 0; c < d->ncell; ++c) start[c + 1] += start[c];
  std::vector<int> sc(n);
  std::vector<float> sf[3];
  for (int x = 0; x < D; ++x) sf[x].resize(n);
  for (uint64_t p = 0; p < n; ++p) {
    sc[p] = cell[order[p]];
    for (int x = 0; x < D; ++x) sf[x][p] = f[order[p] * 3 + x];
  }
  if (d->wall_mem) {
    cudaFree(d->wall_mem);
    d->wall_mem = nullptr;
  }
  // packed copy for the neighbour passes: (fx, fy, fz, cell x)
  std::vector<float4> w4(n);
  for (uint64_t p = 0; p < n; ++p) {
    w4[p].x = sf[0][p];
    w4[p].y = sf[1][p];
    w4[p].z = D == 3 ? sf[2][p] : 0.f;
    w4[p].w = [&] {
      const unsigned pc = pack_cell(sc[p] % d->dims[0], (sc[p] / d->dims[0]) % d->dims[1], sc[p] / (d->dims[0] * d->dims[1]));
      float f;
      std::memcpy(&f, &pc, sizeof f);
      return f;
    }();
  }
  const size_t nn = std::max<uint64_t>(n, 1);
  const size_t bytes =
      nn * sizeof(float4) + nn * sizeof(int) + 3 * nn * sizeof(float) + ((size_t)d->ncell + 1) * sizeof(unsigned) + 64;
  CK(cudaMalloc(&d->wall_mem, bytes));
  char* p = static_cast<char*>(d->wall_mem);
  float4* wp4 = reinterpret_cast<float4*>(p);
  int* wc = reinterpret_cast<int*>(p + nn * sizeof(float4));
  float* wf = reinterpret_cast<float*>(p + nn * sizeof(float4) + nn * sizeof(int));
  unsigned* ws = reinterpret_cast<unsigned*>(p + nn * sizeof(float4) + nn * sizeof(int) + 3 * nn * sizeof(float));
  if (n) CK(cudaMemcpy(wp4, w4.data(), n * sizeof(float4), cudaMemcpyHostToDevice));
  if (n) CK(cudaMemcpy(wc, sc.data(), n * sizeof(int), cudaMemcpyHostToDevice));
  for (int x = 0; x < D; ++x)
    if (n) CK(cudaMemcpy(wf + x * nn, sf[x].data(), n * sizeof(float), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ws, start.data(), start.size() * sizeof(unsigned), cudaMemcpyHostToDevice));
  d->dev.W.cell = wc;
  for (int x = 0; x < 3; ++x) d->dev.W.f[x] = x < D ? wf + x * nn : nullptr;
  d->dev.W.start = ws;
  d->dev.wpos4 = wp4;
  return SPHBUF_OK;
}

sphbuf_status sphbuf_write_particles(sphbuf_domain_t d, const int32_t* cell, const float* frac, const float* vel,
                                     const float* rho, const uint32_t* id, const uint8_t* label, uint64_t n,
                                     uint32_t next_id) {
  if (!d || (n && (!cell || !frac || !vel || !rho))) return SPHBUF_ERR_INVALID_ARG;
  if (n > d->desc.capacity) return fail(d, SPHBUF_ERR_CAPACITY, "more particles than the domain capacity");
  const int D = d->desc.dim;
  CK(cudaStreamSynchronize(d->stream));
  d->ingest_pending = false;  // replaces a pending asynchronous write
  Particles& B = d->dev.B;
  cudaStream_t s = d->stream;
  if (n) {
    // copy the arrays as they are (the AoS frac / vel into the transfer staging), then check
    // and transpose them on the device
    if (!d->xfer) CK(dalloc(d, &d->xfer, 2 * (size_t)d->desc.capacity * D));
    float* sf = d->xfer;
    float* sv = sf + (size_t)n * D;
    CK(cudaMemcpyAsync(B.cell, cell, n * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(sf, frac, n * D * sizeof(float), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(sv, vel, n * D * sizeof(float), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(B.rho, rho, n * sizeof(float), cudaMemcpyHostToDevice, s));
    if (id) CK(cudaMemcpyAsync(B.id, id, n * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
    if (label) CK(cudaMemcpyAsync(B.label, label, n, cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(d->dev.io, 0, 4 * sizeof(unsigned), s));
    launch_ingest(d->dev, sf, sv, (unsigned)n, id != nullptr, label != nullptr, (int)d->bufs.size(), s);
    CK(cudaGetLastError());
    unsigned io[4] = {0, 0, 0, 0};
    CK(cudaMemcpyAsync(io, d->dev.io, sizeof(io), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const char* why = (io[0] & 1u)         ? "cell index outside the grid"
                      : (io[0] & 2u)       ? "in-cell offset outside [0, cs)"
                      : (io[0] & 4u)       ? "label names no buffer"
                      : (next_id <= io[1]) ? "next_id must exceed every id"
                                           : nullptr;
    if (why) {
      // the arrays were checked after they were copied: leave the domain empty
      StepState st;
      CK(cudaMemcpy(&st, d->dev.st, sizeof(StepState), cudaMemcpyDeviceToHost));
      st.n = 0;
      st.n_live = 0;
      st.full = 1;
      st.n_inj = 0;
      st.n_del = 0;
      for (int k = 0; k < 2; ++k) st.sched[k] = st.sched_done[k] = 0u;
      CK(cudaMemcpy(d->dev.st, &st, sizeof(StepState), cudaMemcpyHostToDevice));
      d->labels_given = true;
      d->need_rebuild = true;
      return fail(d, SPHBUF_ERR_INVALID_ARG, why);
    }
  }
  StepState st;
  CK(cudaMemcpy(&st, d->dev.st, sizeof(StepState), cudaMemcpyDeviceToHost));
  st.n = (unsigned)n;
  st.n_live = (unsigned)n;
  st.full = 1;
  st.n_inj = 0;
  st.n_del = 0;
  st.next_id = next_id;
  st.status = 0;
  for (int k = 0; k < 2; ++k) st.sched[k] = st.sched_done[k] = 0u;
  CK(cudaMemcpy(d->dev.st, &st, sizeof(StepState), cudaMemcpyHostToDevice));
  d->labels_given = label != nullptr;
  d->need_rebuild = true;
  return SPHBUF_OK;
}

sphbuf_status sphbuf_write_particles_async(sphbuf_domain_t d, const int32_t* cell, const float* frac,
                                           const float* vel, const float* rho, const uint32_t* id,
                                           const uint8_t* label, uint64_t n, uint32_t next_id) {
  if (!d || (n && (!cell || !frac || !vel || !rho))) return SPHBUF_ERR_INVALID_ARG;
  if (n > d->desc.capacity) return fail(d, SPHBUF_ERR_CAPACITY, "more particles than the domain capacity");
  if (d->ingest_pending)
    return fail(d, SPHBUF_ERR_STATE, "the previous asynchronous write has not been taken by a step or read yet");
  sphbuf_status s = ensure_io(d);
  if (s != SPHBUF_OK) return s;
  const int D = d->desc.dim;
  const Stage in = stage_of(d->in_stage, d->desc.capacity, D);
  cudaStream_t q = d->io_h2d;
  // the staging is free once the previous ingest has read it
  CK(cudaStreamWaitEvent(q, d->ev_ingest, 0));
  if (n) {
    CK(cudaMemcpyAsync(in.cell, cell, n * sizeof(int32_t), cudaMemcpyHostToDevice, q));
    CK(cudaMemcpyAsync(in.frac, frac, n * D * sizeof(float), cudaMemcpyHostToDevice, q));
    CK(cudaMemcpyAsync(in.vel, vel, n * D * sizeof(float), cudaMemcpyHostToDevice, q));
    CK(cudaMemcpyAsync(in.rho, rho, n * sizeof(float), cudaMemcpyHostToDevice, q));
    if (id) CK(cudaMemcpyAsync(in.id, id, n * sizeof(uint32_t), cudaMemcpyHostToDevice, q));
    if (label) CK(cudaMemcpyAsync(in.label, label, n, cudaMemcpyHostToDevice, q));
  }
  CK(cudaEventRecord(d->ev_h2d, q));
  d->ingest_pending = true;
  d->w_n = n;
  d->w_next_id = next_id;
  d->w_ids = id != nullptr;
  d->w_labels = label != nullptr;
  d->labels_given = label != nullptr;
  d->need_rebuild = true;
  return SPHBUF_OK;
}

sphbuf_status sphbuf_read_particles_async(sphbuf_domain_t d, int32_t* cell, float* frac, float* vel, float* rho,
                                          uint32_t* id, uint8_t* label, uint64_t cap, uint64_t* n_out) {
  if (!d || !cell || !frac || !vel || !rho || !id || !label) return SPHBUF_ERR_INVALID_ARG;
  if (!d->committed && !d->need_rebuild) return fail(d, SPHBUF_ERR_STATE, "no particles written");
  sphbuf_status s = SPHBUF_OK;
  if (d->need_rebuild && (s = commit(d)) != SPHBUF_OK) return s;
  if ((s = ensure_io(d)) != SPHBUF_OK) return s;
  if (d->reads.size() >= (size_t)kIoRing && (s = sphbuf_io_wait(d)) != SPHBUF_OK) return s;
  const int D = d->desc.dim;
  const uint64_t rows = std::min<uint64_t>(cap, d->desc.capacity);
  const Stage out = stage_of(d->out_stage, d->desc.capacity, D);
  // the staging is free once the previous read's copies have left it
  CK(cudaStreamWaitEvent(d->stream, d->ev_d2h, 0));
  launch_egest_staged(d->dev, out.cell, out.frac, out.vel, out.rho, out.id, out.label, out.count, (unsigned)rows,
                      d->stream);
  CK(cudaGetLastError());
  d->launches += 1;
  CK(cudaEventRecord(d->ev_egest, d->stream));
  cudaStream_t q = d->io_d2h;
  CK(cudaStreamWaitEvent(q, d->ev_egest, 0));
  if (rows) {
    CK(cudaMemcpyAsync(cell, out.cell, rows * sizeof(int32_t), cudaMemcpyDeviceToHost, q));
    CK(cudaMemcpyAsync(frac, out.frac, rows * D * sizeof(float), cudaMemcpyDeviceToHost, q));
    CK(cudaMemcpyAsync(vel, out.vel, rows * D * sizeof(float), cudaMemcpyDeviceToHost, q));
    CK(cudaMemcpyAsync(rho, out.rho, rows * sizeof(float), cudaMemcpyDeviceToHost, q));
    CK(cudaMemcpyAsync(id, out.id, rows * sizeof(uint32_t), cudaMemcpyDeviceToHost, q));
    CK(cudaMemcpyAsync(label, out.label, rows, cudaMemcpyDeviceToHost, q));
  }
  const int slot = d->ring_next;
  d->ring_next = (d->ring_next + 1) % kIoRing;
  CK(cudaMemcpyAsync(d->n_pinned + slot, out.count, sizeof(unsigned), cudaMemcpyDeviceToHost, q));
  CK(cudaEventRecord(d->ev_d2h, q));
  d->reads.push_back({n_out, cap, slot});
  return SPHBUF_OK;
}

sphbuf_status sphbuf_io_wait(sphbuf_domain_t d) {
  if (!d) return SPHBUF_ERR_INVALID_ARG;
  if (d->io_h2d) CK(cudaStreamSynchronize(d->io_h2d));
  if (d->io_d2h) CK(cudaStreamSynchronize(d->io_d2h));
  sphbuf_status ret = SPHBUF_OK;
  for (const sphbuf_domain::PendingRead& r : d->reads) {
    const uint64_t n = d->n_pinned[r.slot];
    if (r.n_out) *r.n_out = n;
    if (n > r.cap && ret == SPHBUF_OK)
      ret = fail(d, SPHBUF_ERR_CAPACITY, "host arrays of an asynchronous read smaller than the particle count");
  }
  d->reads.clear();
  StepState st;
  sphbuf_status s = read_state(d, &st);
  return ret != SPHBUF_OK ? ret : s;
}

sphbuf_status sphbuf_set_fluid(sphbuf_domain_t d, const double* pos, const float* vel, const float* rho, uint64_t n) {
  if (!d || (n && (!pos || !vel || !rho))) return SPHBUF_ERR_INVALID_ARG;
  if (d->stepped) return fail(d, SPHBUF_ERR_STATE, "set_fluid is only valid before the first step");
  const int D = d->desc.dim;
  std::vector<int32_t> cell(n);
  std::vector<float> f((size_t)n * D);
  for (uint64_t i = 0; i < n; ++i) {
    int c[3] = {0, 0, 0};
    for (int x = 0; x < D; ++x)
      if (!encode_axis(pos[i * D + x], d->desc.lo[x], d->cs, d->cs32, d->dims[x], &c[x], &f[i * D + x]))
        return fail(d, SPHBUF_ERR_INVALID_ARG, "fluid particle outside the grid box");
    cell[i] = (c[2] * d->dims[1] + c[1]) * d->dims[0] + c[0];
  }
  return sphbuf_write_particles(d, cell.data(), f.data(), vel, rho, nullptr, nullptr, n, (uint32_t)n);
}

sphbuf_status sphbuf_rotation_from_normal(const double normal[3], double roll, double out_R[9]) {
  if (!normal || !out_R) return SPHBUF_ERR_INVALID_ARG;
  const double nn = std::sqrt(normal[0] * normal[0] + normal[1] * normal[1] + normal[2] * normal[2]);
  if (!(nn > 0) || !std::isfinite(nn)) return SPHBUF_ERR_INVALID_ARG;
  const double dvec[3] = {normal[0] / nn, normal[1] / nn, normal[2] / nn};
  // Eq. (12): n = e_x x d / |e_x x d| = (0, -d_z, d_y) / |.|
  const double ax[3] = {0.0, -dvec[2], dvec[1]};
  const double an = std::sqrt(ax[1] * ax[1] + ax[2] * ax[2]);
  double R[9];
  if (an < 1e-12) {
    for (int q = 0; q < 9; ++q) R[q] = 0;
    if (dvec[0] > 0) {
      R[0] = R[4] = R[8] = 1.0;
    } else {
      R[0] = -1.0;
      R[4] = -1.0;
      R[8] = 1.0;
    }
  } else {
    const double n0 = ax[0] / an, n1 = ax[1] / an, n2 = ax[2] / an;
    // Eq. (13)
    const double S[9] = {0, -n2, n1, n2, 0, -n0, -n1, n0, 0};
    double S2[9];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) S2[3 * r + c] = S[3 * r] * S[c] + S[3 * r + 1] * S[3 + c] + S[3 * r + 2] * S[6 + c];
    const double th = std::acos(std::max(-1.0, std::min(1.0, dvec[0])));
    const double sn = std::sin(th), cm = 1.0 - std::cos(th);
    // Eq. (14) with the sign reading: R = I - S sin + S^2 (1 - cos), so that R d = e_x
    for (int q = 0; q < 9; ++q) R[q] = ((q % 4) == 0 ? 1.0 : 0.0) - S[q] * sn + S2[q] * cm;
  }
  const double c = std::cos(roll), s = std::sin(roll);
  const double Rx[9] = {1, 0, 0, 0, c, s, 0, -s, c};
  for (int r = 0; r < 3; ++r)
    for (int q = 0; q < 3; ++q) out_R[3 * r + q] = Rx[3 * r] * R[q] + Rx[3 * r + 1] * R[3 + q] + Rx[3 * r + 2] * R[6 + q];
  return SPHBUF_OK;
}

sphbuf_status sphbuf_add_inout_buffer(sphbuf_domain_t d, const double origin[3], const double rotation[9],
                                      const double extent[3], sphbuf_bc_type bc, const sphbuf_bc_params* params,
                                      int* out_id) {
  if (!d || !origin || !rotation || !extent) return SPHBUF_ERR_INVALID_ARG;
  if (d->stepped || d->committed) return fail(d, SPHBUF_ERR_STATE, "buffers must be added before the first step");
  if ((int)bc < 0 || (int)bc > 5) return fail(d, SPHBUF_ERR_INVALID_ARG, "unknown boundary type");
  if (d->bufs.size() >= (size_t)kMaxBuffers) return fail(d, SPHBUF_ERR_CAPACITY, "too many buffers");
  const int D = d->desc.dim;
  BufHost b{};
  std::memcpy(b.origin, origin, sizeof(b.origin));
  std::memcpy(b.R, rotation, sizeof(b.R));
  std::memcpy(b.extent, extent, sizeof(b.extent));
  if (D == 2) {
    b.origin[2] = 0;
    b.extent[2] = 0;
    b.R[2] = b.R[5] = b.R[6] = b.R[7] = 0;
    b.R[8] = 1;
  }
  b.bc = (int)bc;
  if (params) b.prm = *params;
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double dot = 0;
      for (int x = 0; x < 3; ++x) dot += b.R[3 * r + x] * b.R[3 * c + x];
      if (std::fabs(dot - (r == c ? 1.0 : 0.0)) > 1e-9) return fail(d, SPHBUF_ERR_INVALID_ARG, "frame not orthonormal");
    }
  const double det = b.R[0] * (b.R[4] * b.R[8] - b.R[5] * b.R[7]) - b.R[1] * (b.R[3] * b.R[8] - b.R[5] * b.R[6]) +
                     b.R[2] * (b.R[3] * b.R[7] - b.R[4] * b.R[6]);
  if (det < 0) return fail(d, SPHBUF_ERR_INVALID_ARG, "frame is not a rotation (det < 0)");
  for (int x = 0; x < D; ++x)
    if (!(b.extent[x] > 0)) return fail(d, SPHBUF_ERR_INVALID_ARG, "extent must be positive");
  // candidate regions (box dilated by 2 cs) must not overlap
  const double dil = 2.0 * d->cs;
  const double h1[3] = {0.5 * b.extent[0] + dil, 0.5 * b.extent[1] + dil, D == 3 ? 0.5 * b.extent[2] + dil : 0};
  for (const BufHost& o : d->bufs) {
    const double h2[3] = {0.5 * o.extent[0] + dil, 0.5 * o.extent[1] + dil, D == 3 ? 0.5 * o.extent[2] + dil : 0};
    if (obb_overlap(D, b.origin, b.R, h1, o.origin, o.R, h2) || (o.rotating && swept_overlaps_box(D, o, b.origin, b.R, h1)))
      return fail(d, SPHBUF_ERR_OVERLAP, "candidate regions of two buffers overlap");
  }
  const int k = (int)d->bufs.size();
  BufDev v{};
  v.kind = (bc == SPHBUF_VELOCITY_INLET || bc == SPHBUF_PRESSURE_INLET) ? KIND_INFLOW
           : (bc == SPHBUF_PRESSURE_OUTLET || bc == SPHBUF_VELOCITY_OUTLET) ? KIND_OUTFLOW
                                                                              : KIND_BIDIR;
  v.vel_bc = (bc == SPHBUF_VELOCITY_INLET || bc == SPHBUF_VELOCITY_OUTLET || bc == SPHBUF_BIDIR_VELOCITY) ? 1 : 0;
  v.label = k + 1;
  const double cs = d->cs;
  for (int x = 0; x < 3; ++x) {
    v.cO[x] = 0;
    v.fO[x] = 0.f;
    if (x < D) {
      const double t = b.origin[x] - d->desc.lo[x];
      const double c = std::floor(t / cs);
      v.cO[x] = (int)c;
      v.fO[x] = (float)(t - c * cs);
    }
  }
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) v.R[r][c] = (float)b.R[3 * r + c];
  const double a = b.extent[0];
  v.ha = (float)(0.5 * a);
  v.hb = (float)(0.5 * b.extent[1]);
  v.hc = (float)(0.5 * b.extent[2]);
  v.da = (float)(0.5 * a + cs);
  v.db = (float)(0.5 * b.extent[1] + cs);
  v.dc = (float)(0.5 * b.extent[2] + cs);
  for (int x = 0; x < 3; ++x) {
    v.shift[x] = x < D ? (float)(-a * b.R[x]) : 0.f;
    v.u[x] = x < D ? (float)b.R[x] : 0.f;
  }
  v.umax = (float)b.prm.umax;
  v.inv_hw2 = b.prm.half_width > 0 ? (float)(1.0 / (b.prm.half_width * b.prm.half_width)) : 0.f;
  v.flux_scale = (float)(std::pow(d->desc.dp, D) / a);
  // cell bounds that contain the box (with one cell of margin): relabel prefilter
  for (int x = 0; x < 3; ++x) {
    if (x >= D) {
      v.box_lo[x] = 0;
      v.box_hi[x] = 0;
      continue;
    }
    double ext = 0;
    for (int r = 0; r < D; ++r) ext += 0.5 * b.extent[r] * std::fabs(b.R[3 * r + x]);
    v.box_lo[x] = (int)std::floor((b.origin[x] - ext - d->desc.lo[x]) / cs) - 1;
    v.box_hi[x] = (int)std::floor((b.origin[x] + ext - d->desc.lo[x]) / cs) + 1;
  }
  v.p_b0 = b.prm.p_b;
  v.p_amp = b.prm.p_amp;
  v.p_omega = b.prm.p_omega;
  v.p_phase = b.prm.p_phase;
  d->bufs.push_back(b);
  d->bufs_dev.push_back(v);
  if (out_id) *out_id = k;
  return SPHBUF_OK;
}

sphbuf_status sphbuf_set_buffer_rotation(sphbuf_domain_t d, int buffer_id, const double pivot[3], const double axis[3],
                                         double omega) {
  if (!d || !pivot) return SPHBUF_ERR_INVALID_ARG;
  if (d->stepped || d->committed) return fail(d, SPHBUF_ERR_STATE, "rotation must be set before the first step");
  if (buffer_id < 0 || buffer_id >= (int)d->bufs.size()) return fail(d, SPHBUF_ERR_INVALID_ARG, "no such buffer");
  if (d->dev.P.reuse) return fail(d, SPHBUF_ERR_INVALID_ARG, "kept neighbour lists serve domains without rotating buffers");
  BufHost& b = d->bufs[buffer_id];
  BufDev& v = d->bufs_dev[buffer_id];
  if (v.kind != KIND_INFLOW) return fail(d, SPHBUF_ERR_INVALID_ARG, "only inflow buffers may rotate");
  if (b.rotating) return fail(d, SPHBUF_ERR_STATE, "rotation already set");
  if (!std::isfinite(omega)) return fail(d, SPHBUF_ERR_INVALID_ARG, "omega must be finite");
  const int D = d->desc.dim;
  const double C[3] = {pivot[0], pivot[1], D == 3 ? pivot[2] : 0.0};
  for (int x = 0; x < 3; ++x)
    if (!std::isfinite(C[x])) return fail(d, SPHBUF_ERR_INVALID_ARG, "pivot must be finite");
  // M: rotation by omega dt (about z in 2-D; about the unit axis in 3-D, Rodrigues' formula),
  // FP64 with the products and sums in the order written (the frames of later steps, and so
  // the FP32 decisions, depend on its rounding)
  const double phi = omega * d->desc.dt;
  const double s = std::sin(phi), c = std::cos(phi);
  double M[9];
  if (D == 2) {
    const double m2[9] = {c, -s, 0.0, s, c, 0.0, 0.0, 0.0, 1.0};
    std::memcpy(M, m2, sizeof(M));
  } else {
    if (!axis) return fail(d, SPHBUF_ERR_INVALID_ARG, "a 3-D rotation needs an axis");
    const double nn = std::sqrt((axis[0] * axis[0] + axis[1] * axis[1]) + axis[2] * axis[2]);
    if (!(nn > 0) || !std::isfinite(nn)) return fail(d, SPHBUF_ERR_INVALID_ARG, "rotation axis must be non-zero");
    const double n0 = axis[0] / nn, n1 = axis[1] / nn, n2 = axis[2] / nn, t = 1.0 - c;
    const double m3[9] = {(t * n0) * n0 + c,      (t * n0) * n1 - s * n2, (t * n0) * n2 + s * n1,
                          (t * n0) * n1 + s * n2, (t * n1) * n1 + c,      (t * n1) * n2 - s * n0,
                          (t * n0) * n2 - s * n1, (t * n1) * n2 + s * n0, (t * n2) * n2 + c};
    std::memcpy(M, m3, sizeof(M));
  }
  BufHost nb = b;
  RotDev& q = nb.rot;
  std::memcpy(q.M, M, sizeof(M));
  for (int e = 0; e < 9; ++e) q.Q[e] = (e % 4 == 0) ? 1.0 : 0.0;
  std::memcpy(q.C, C, sizeof(C));
  std::memcpy(q.O0, b.origin, sizeof(q.O0));
  std::memcpy(q.R0, b.R, sizeof(q.R0));
  q.a = b.extent[0];
  // distances from the pivot swept by the box dilated by 2 cs
  const double dil = 2.0 * d->cs;
  const double hd[3] = {0.5 * b.extent[0] + dil, 0.5 * b.extent[1] + dil, D == 3 ? 0.5 * b.extent[2] + dil : 0.0};
  box_distances(D, C, b.origin, b.R, hd, &nb.r_min, &nb.r_max);
  nb.rotating = true;
  for (size_t o = 0; o < d->bufs.size(); ++o) {
    if ((int)o == buffer_id) continue;
    const BufHost& ob = d->bufs[o];
    const double ho[3] = {0.5 * ob.extent[0] + dil, 0.5 * ob.extent[1] + dil, D == 3 ? 0.5 * ob.extent[2] + dil : 0.0};
    bool hit = swept_overlaps_box(D, nb, ob.origin, ob.R, ho);
    if (ob.rotating) {
      double dd = 0;
      for (int x = 0; x < D; ++x) dd += (C[x] - ob.rot.C[x]) * (C[x] - ob.rot.C[x]);
      hit = hit || std::sqrt(dd) <= nb.r_max + ob.r_max;
    }
    if (hit) return fail(d, SPHBUF_ERR_OVERLAP, "the rotating buffer's swept region meets another buffer's");
  }
  b = nb;
  v.rotating = 1;
  d->dev.any_rot = 1;
  for (int x = 0; x < 3; ++x) {
    v.cC[x] = 0;
    v.fC[x] = 0.f;
    if (x < D) {
      const double t = C[x] - d->desc.lo[x];
      const double cc = std::floor(t / d->cs);
      v.cC[x] = (int)cc;
      v.fC[x] = (float)(t - cc * d->cs);
    }
  }
  for (int r = 0; r < 3; ++r)
    for (int cc = 0; cc < 3; ++cc) v.M32[r][cc] = (float)M[3 * r + cc];
  return SPHBUF_OK;
}

sphbuf_status sphbuf_set_background_pressure(sphbuf_domain_t d, double p_bg) {
  if (!d) return SPHBUF_ERR_INVALID_ARG;
  if (d->stepped || d->committed) return fail(d, SPHBUF_ERR_STATE, "the background pressure must be set before the first step");
  if (!std::isfinite(p_bg)) return fail(d, SPHBUF_ERR_INVALID_ARG, "background pressure must be finite");
  d->dev.P.p_bg = (float)p_bg;
  d->dev.P.p_bg_d = p_bg;
  return SPHBUF_OK;
}

sphbuf_status sphbuf_set_dual_time_stepping(sphbuf_domain_t d, int n_acoustic) {
  if (!d) return SPHBUF_ERR_INVALID_ARG;
  if (d->stepped || d->committed) return fail(d, SPHBUF_ERR_STATE, "the time stepping must be set before the first step");
  if (n_acoustic < 0 || n_acoustic > 4096) return fail(d, SPHBUF_ERR_INVALID_ARG, "n_acoustic must be in [0, 4096]");
  if (n_acoustic > 0 && d->dev.P.reuse)
    return fail(d, SPHBUF_ERR_INVALID_ARG, "kept neighbour lists serve single-rate domains");
  DomainDev& v = d->dev;
  if (n_acoustic > 0 && !v.pos_b) {
    const size_t C = d->desc.capacity;
    CK(dalloc(d, &v.pos_b, C));
    CK(dalloc(d, &v.vr_b, C));
    CK(dalloc(d, &v.av, C));
  }
  v.P.dual_n = n_acoustic;
  v.P.dt_ac = n_acoustic > 0 ? (float)(d->desc.dt / n_acoustic) : 0.f;
  return SPHBUF_OK;
}

sphbuf_status sphbuf_set_transport_velocity(sphbuf_domain_t d, double lambda) {
  if (!d) return SPHBUF_ERR_INVALID_ARG;
  if (d->stepped || d->committed) return fail(d, SPHBUF_ERR_STATE, "the transport velocity must be set before the first step");
  if (!(lambda >= 0) || !std::isfinite(lambda)) return fail(d, SPHBUF_ERR_INVALID_ARG, "lambda must be finite and >= 0");
  d->dev.P.tvf_lambda = (float)lambda;
  return SPHBUF_OK;
}

sphbuf_status sphbuf_set_list_reuse(sphbuf_domain_t d, double skin_over_h, int max_steps) {
  if (!d) return SPHBUF_ERR_INVALID_ARG;
  if (d->stepped) return fail(d, SPHBUF_ERR_STATE, "kept neighbour lists are chosen before the first step");
  if (!(skin_over_h >= 0.0) || skin_over_h > 1.0 || max_steps < 1)
    return fail(d, SPHBUF_ERR_INVALID_ARG, "skin must be in [0, h], max_steps >= 1");
  if (skin_over_h > 0.0 && (d->dev.any_rot || d->dev.P.dual_n > 0))
    return fail(d, SPHBUF_ERR_INVALID_ARG, "kept neighbour lists serve single-rate domains without rotating buffers");
  Phys& P = d->dev.P;
  const double h = d->desc.h_over_dp * d->desc.dp;
  P.reuse = skin_over_h > 0.0 ? 1 : 0;
  P.skin = (float)(skin_over_h * h);
  P.list_r2 = P.reuse ? (float)((2.0 * h + skin_over_h * h) * (2.0 * h + skin_over_h * h)) : P.two_h_sq;
  P.reuse_max = max_steps;
  if (d->graph) {
    cudaGraphExecDestroy(d->graph);
    d->graph = nullptr;
  }
  return SPHBUF_OK;
}

sphbuf_status sphbuf_read_boundary_flags(sphbuf_domain_t d, uint8_t* flags, uint64_t cap, uint64_t* n_out) {
  if (!d) return SPHBUF_ERR_INVALID_ARG;
  StepState st;
  sphbuf_status s = read_state(d, &st);
  if (s != SPHBUF_OK) return s;
  const uint64_t n = st.n_live;
  if (n_out) *n_out = n;
  if (!flags || !n) return SPHBUF_OK;
  if (n > cap) return fail(d, SPHBUF_ERR_CAPACITY, "host array smaller than the particle count");
  const uint8_t* src = d->dev.A.bflag;
  if (!st.full) {
    launch_gather_u8(d->dev, d->dev.A.bflag, d->dev.B.bflag, (unsigned)n, d->stream);
    CK(cudaGetLastError());
    src = d->dev.B.bflag;
  }
  CK(cudaMemcpyAsync(flags, src, n, cudaMemcpyDeviceToHost, d->stream));
  CK(cudaStreamSynchronize(d->stream));
  return SPHBUF_OK;
}

sphbuf_status sphbuf_read_list_builds(sphbuf_domain_t d, uint64_t* builds) {
  if (!d || !builds) return SPHBUF_ERR_INVALID_ARG;
  StepState st;
  sphbuf_status s = read_state(d, &st);
  *builds = st.list_builds;
  return s;
}

sphbuf_status sphbuf_set_windkessel(sphbuf_domain_t d, int buffer_id, double r_p, double compliance, double r_d,
                                    double p_d0) {
  if (!d) return SPHBUF_ERR_INVALID_ARG;
  if (d->stepped || d->committed) return fail(d, SPHBUF_ERR_STATE, "the Windkessel must be set before the first step");
  if (buffer_id < 0 || buffer_id >= (int)d->bufs.size()) return fail(d, SPHBUF_ERR_INVALID_ARG, "no such buffer");
  BufDev& v = d->bufs_dev[buffer_id];
  if (v.vel_bc) return fail(d, SPHBUF_ERR_INVALID_ARG, "a Windkessel drives a pressure buffer");
  if (!(r_p >= 0) || !(compliance > 0) || !(r_d > 0) || !std::isfinite(r_p) || !std::isfinite(compliance) ||
      !std::isfinite(r_d) || !std::isfinite(p_d0))
    return fail(d, SPHBUF_ERR_INVALID_ARG, "Windkessel parameters: R_p >= 0, C > 0, R_d > 0, finite");
  v.wk = 1;
  v.wk_rp = r_p;
  v.wk_c = compliance;
  v.wk_rd = r_d;
  d->bufs[buffer_id].wk_pd0 = p_d0;
  return SPHBUF_OK;
}

sphbuf_status sphbuf_read_boundary_pressure(sphbuf_domain_t d, int buffer_id, double* p_b, double* p_d, double* q_prev) {
  if (!d) return SPHBUF_ERR_INVALID_ARG;
  if (buffer_id < 0 || buffer_id >= (int)d->bufs.size()) return fail(d, SPHBUF_ERR_INVALID_ARG, "no such buffer");
  StepState st;
  sphbuf_status s = read_state(d, &st);
  if (s != SPHBUF_OK) return s;
  if (p_b) *p_b = st.pb_d[buffer_id];
  if (p_d) *p_d = st.wk_pd[buffer_id];
  if (q_prev) *q_prev = st.flux_last[buffer_id];
  return SPHBUF_OK;
}

sphbuf_status sphbuf_step_phases(sphbuf_domain_t d, int nsteps, unsigned phases) {
  if (!d || nsteps < 0) return SPHBUF_ERR_INVALID_ARG;
  const bool phys = phases & SPHBUF_PHASE_PHYSICS, kin = phases & SPHBUF_PHASE_KINEMATIC;
  if (phys == kin) return fail(d, SPHBUF_ERR_INVALID_ARG, "exactly one of PHYSICS or KINEMATIC is required");
  if (phases & ~31u) return fail(d, SPHBUF_ERR_INVALID_ARG, "unknown phase bits");
  if (d->dev.P.reuse && (phases & (SPHBUF_PHASE_FULL_CHECK | SPHBUF_PHASE_BUFFER_KERNEL)))
    return fail(d, SPHBUF_ERR_INVALID_ARG, "kept neighbour lists need the decisions fused into the drift");
  if (!d->committed && !d->need_rebuild) return fail(d, SPHBUF_ERR_STATE, "no particles written");
  sphbuf_status s = commit(d);
  if (s != SPHBUF_OK) return s;
  d->stepped = true;
  for (int q = 0; q < nsteps; ++q) {
    if (d->timing) {
      d->launches += enqueue_step(d, phases, true);
      CK(cudaEventSynchronize(d->ev[kPhases]));
      for (int p = 0; p < kPhases; ++p) {
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, d->ev[p], d->ev[p + 1]));
        d->acc_ms[p] += ms;
      }
      d->timed_steps++;
    } else if (d->use_graph) {
      if (!d->graph || d->graph_phases != phases) {
        if (d->graph) {
          cudaGraphExecDestroy(d->graph);
          d->graph = nullptr;
        }
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(d->stream, cudaStreamCaptureModeThreadLocal));
        const int nk = enqueue_step(d, phases, false);
        CK(cudaStreamEndCapture(d->stream, &g));
        CK(cudaGraphInstantiate(&d->graph, g, 0));
        cudaGraphDestroy(g);
        d->graph_phases = phases;
        d->graph_launches = (uint64_t)nk;
      }
      CK(cudaGraphLaunch(d->graph, d->stream));
      d->launches += d->graph_launches;
    } else {
      d->launches += enqueue_step(d, phases, false);
    }
  }
  CK(cudaGetLastError());
  return SPHBUF_OK;
}

sphbuf_status sphbuf_step(sphbuf_domain_t d, int nsteps) { return sphbuf_step_phases(d, nsteps, SPHBUF_STEP_DEFAULT); }

sphbuf_status sphbuf_use_graph(sphbuf_domain_t d, int enable) {
  if (!d) return SPHBUF_ERR_INVALID_ARG;
  d->use_graph = enable != 0;
  return SPHBUF_OK;
}

sphbuf_status sphbuf_sync(sphbuf_domain_t d) {
  if (!d) return SPHBUF_ERR_INVALID_ARG;
  if (!d->committed) {
    CK(cudaStreamSynchronize(d->stream));
    return SPHBUF_OK;
  }
  StepState st;
  return read_state(d, &st);
}

sphbuf_status sphbuf_count(sphbuf_domain_t d, uint64_t* n) {
  if (!d || !n) return SPHBUF_ERR_INVALID_ARG;
  StepState st;
  sphbuf_status s = read_state(d, &st);
  *n = st.n_live;
  return s;
}

sphbuf_status sphbuf_grid_info(sphbuf_domain_t d, int32_t dims[3], double* cs, uint64_t* ncell) {
  if (!d) return SPHBUF_ERR_INVALID_ARG;
  if (dims)
    for (int x = 0; x < 3; ++x) dims[x] = d->dims[x];
  if (cs) *cs = d->cs;
  if (ncell) *ncell = (uint64_t)d->ncell;
  return SPHBUF_OK;
}

sphbuf_status sphbuf_read_particles(sphbuf_domain_t d, int32_t* cell, float* frac, float* vel, float* rho,
                                    uint32_t* id, uint8_t* label, uint64_t cap, uint64_t* n_out) {
  if (!d) return SPHBUF_ERR_INVALID_ARG;
  if (d->need_rebuild) {
    sphbuf_status s = commit(d);
    if (s != SPHBUF_OK) return s;
  }
  StepState st;
  sphbuf_status s = read_state(d, &st);
  if (s != SPHBUF_OK) return s;
  const uint64_t n = st.n_live;
  if (n_out) *n_out = n;
  if (n > cap && (cell || frac || vel || rho || id || label))
    return fail(d, SPHBUF_ERR_CAPACITY, "host arrays smaller than the particle count");
  const int D = d->desc.dim;
  if (!n) return SPHBUF_OK;
  cudaStream_t st_ = d->stream;
  // the live particles in (cell, id) order: the state itself, or (slots kept by the last
  // rebuild) a copy through the index list in B, which is free between steps
  if (!st.full) {
    launch_view(d->dev, st_);
    CK(cudaGetLastError());
  }
  const Particles& A = st.full ? d->dev.A : d->dev.B;
  if (frac || vel) {
    // gather the AoS arrays on the device (into the transfer staging), then copy each array
    // once
    if (!d->xfer) CK(dalloc(d, &d->xfer, 2 * (size_t)d->desc.capacity * D));
    float* sf = d->xfer;
    float* sv = sf + (size_t)n * D;
    launch_egest(d->dev, A, frac ? sf : nullptr, vel ? sv : nullptr, (unsigned)n, st_);
    CK(cudaGetLastError());
    if (frac) CK(cudaMemcpyAsync(frac, sf, n * D * sizeof(float), cudaMemcpyDeviceToHost, st_));
    if (vel) CK(cudaMemcpyAsync(vel, sv, n * D * sizeof(float), cudaMemcpyDeviceToHost, st_));
  }
  if (cell) CK(cudaMemcpyAsync(cell, A.cell, n * sizeof(int), cudaMemcpyDeviceToHost, st_));
  if (rho) CK(cudaMemcpyAsync(rho, A.rho, n * sizeof(float), cudaMemcpyDeviceToHost, st_));
  if (id) CK(cudaMemcpyAsync(id, A.id, n * sizeof(uint32_t), cudaMemcpyDeviceToHost, st_));
  if (label) CK(cudaMemcpyAsync(label, A.label, n, cudaMemcpyDeviceToHost, st_));
  CK(cudaStreamSynchronize(st_));
  return SPHBUF_OK;
}

sphbuf_status sphbuf_read_positions(sphbuf_domain_t d, double* pos, uint64_t cap, uint64_t* n_out) {
  if (!d) return SPHBUF_ERR_INVALID_ARG;
  StepState st;
  sphbuf_status s = read_state(d, &st);
  if (s != SPHBUF_OK) return s;
  const uint64_t n = st.n_live;
  if (n_out) *n_out = n;
  if (!pos || !n) return SPHBUF_OK;
  if (n > cap) return fail(d, SPHBUF_ERR_CAPACITY, "host array smaller than the particle count");
  double* tmp = nullptr;
  CK(cudaMalloc(&tmp, n * d->desc.dim * sizeof(double)));
  launch_decode_positions(d->dev, tmp, d->desc.lo, d->cs, d->stream);
  cudaError_t e = cudaStreamSynchronize(d->stream);
  if (e == cudaSuccess) e = cudaMemcpy(pos, tmp, n * d->desc.dim * sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(tmp);
  if (e != cudaSuccess) return cuda_fail(d, e, "read_positions");
  return SPHBUF_OK;
}

sphbuf_status sphbuf_read_cell_start(sphbuf_domain_t d, uint32_t* cell_start, uint64_t cap) {
  if (!d || !cell_start) return SPHBUF_ERR_INVALID_ARG;
  if (cap < (uint64_t)d->ncell + 1) return fail(d, SPHBUF_ERR_CAPACITY, "cell_start needs ncell + 1 entries");
  StepState st;
  sphbuf_status s = read_state(d, &st);
  if (s != SPHBUF_OK) return s;
  CK(cudaMemcpy(cell_start, d->dev.cell_start, ((size_t)d->ncell + 1) * sizeof(unsigned), cudaMemcpyDeviceToHost));
  return SPHBUF_OK;
}

sphbuf_status sphbuf_read_counters(sphbuf_domain_t d, int k, uint64_t* injected, uint64_t* deleted, double* mass_in,
                                   double* mass_out, double* flux_q) {
  if (!d || k < 0 || (size_t)k >= d->bufs.size()) return SPHBUF_ERR_INVALID_ARG;
  StepState st;
  sphbuf_status s = read_state(d, &st);
  if (s != SPHBUF_OK) return s;
  if (injected) *injected = st.injected[k];
  if (deleted) *deleted = st.deleted[k];
  if (mass_in) *mass_in = (double)st.injected[k] * d->mass_d;
  if (mass_out) *mass_out = (double)st.deleted[k] * d->mass_d;
  if (flux_q) *flux_q = (double)st.flux_fx[k] * kFluxUnit;
  return SPHBUF_OK;
}

sphbuf_status sphbuf_read_global(sphbuf_domain_t d, uint64_t* escaped, uint64_t* steps, uint32_t* next_id) {
  if (!d) return SPHBUF_ERR_INVALID_ARG;
  StepState st;
  sphbuf_status s = read_state(d, &st);
  if (escaped) *escaped = st.escaped_total;
  if (steps) *steps = st.step;
  if (next_id) *next_id = st.next_id;
  return s;
}

sphbuf_status sphbuf_last_decisions(sphbuf_domain_t d, uint32_t* inj_buffer, uint32_t* inj_parent, uint32_t* inj_new,
                                    uint64_t* n_inj, uint32_t* del_buffer, uint32_t* del_id, uint64_t* n_del,
                                    uint64_t cap) {
  if (!d) return SPHBUF_ERR_INVALID_ARG;
  StepState st;
  sphbuf_status s = read_state(d, &st);
  if (s != SPHBUF_OK) return s;
  const uint64_t ni = std::min(st.n_inj, d->dev.P.list_cap), nd = std::min(st.n_del, d->dev.P.list_cap);
  if (n_inj) *n_inj = ni;
  if (n_del) *n_del = nd;
  if ((ni > cap && (inj_buffer || inj_parent || inj_new)) || (nd > cap && (del_buffer || del_id)))
    return fail(d, SPHBUF_ERR_CAPACITY, "host arrays smaller than the decision lists");
  if (ni && (inj_buffer || inj_parent || inj_new)) {
    std::vector<InjRecord> r(ni);
    CK(cudaMemcpy(r.data(), d->dev.inj_sorted, ni * sizeof(InjRecord), cudaMemcpyDeviceToHost));
    for (uint64_t q = 0; q < ni; ++q) {
      if (inj_buffer) inj_buffer[q] = r[q].k;
      if (inj_parent) inj_parent[q] = r[q].parent;
      if (inj_new) inj_new[q] = r[q].child;
    }
  }
  if (nd && (del_buffer || del_id)) {
    std::vector<Decision> r(nd);
    CK(cudaMemcpy(r.data(), d->dev.del, nd * sizeof(Decision), cudaMemcpyDeviceToHost));
    for (uint64_t q = 0; q < nd; ++q) {
      if (del_buffer) del_buffer[q] = r[q].k;
      if (del_id) del_id[q] = r[q].id;
    }
  }
  return SPHBUF_OK;
}

sphbuf_status sphbuf_enable_phase_timing(sphbuf_domain_t d, int enable) {
  if (!d) return SPHBUF_ERR_INVALID_ARG;
  d->timing = enable != 0;
  return SPHBUF_OK;
}

sphbuf_status sphbuf_read_phase_times(sphbuf_domain_t d, double ms[5], uint64_t* steps) {
  if (!d || !ms) return SPHBUF_ERR_INVALID_ARG;
  CK(cudaStreamSynchronize(d->stream));
  for (int p = 0; p < kPhases; ++p) {
    ms[p] = d->acc_ms[p];
    d->acc_ms[p] = 0;
  }
  if (steps) *steps = d->timed_steps;
  d->timed_steps = 0;
  return SPHBUF_OK;
}

// ---------------------------------------------------------------- batched domains
struct sphbuf_batch {
  std::vector<sphbuf_domain*> doms;
  int dual_n = 0;    // acoustic steps per step (the same for every domain of the batch)
  bool tvf = false;  // some domain advects with the transport velocity (Eq. (10))
  bool rot = false;  // some domain has a rotating buffer
  std::vector<uint64_t> n0;  // particles per domain when the batch was made (block shares)
  int dim = 0;
  int sm_count = 1;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  DomainDev* d_doms = nullptr;
  int4* d_maps[K_COUNT] = {};
  int nblocks[K_COUNT] = {};
  int mult = 8;
  // launch configuration per kernel (the autotuner's): threads per block, blocks per SM (the
  // particle kernels' grid is blocks_per_sm x SMs, shared out over the domains by work), and
  // the buffer kernel's cell tile (candidate cells per warp)
  int thr[K_COUNT] = {};
  int mk[K_COUNT] = {};
  int cpw = 4;
  // persistent form of the default step (one cooperative launch, grid barriers)
  bool persistent = false;
  bool kin_step = false;  // the step being enqueued is kinematic (its rebuild sorts)
  long long spin_limit = 1ll << 24;
  unsigned* d_bar = nullptr;
  int pgrid = 0;
  // per-kernel timing (autotuner): an event pair around every launch of a step
  bool ktime = false;
  std::vector<cudaEvent_t> kev;
  std::vector<int> kid;
  size_t kpos = 0;
  bool use_graph = false;
  cudaGraphExec_t graph = nullptr;
  unsigned graph_phases = 0;
  uint64_t graph_launches = 0;
  cudaEvent_t ev[kPhases + 1] = {};
  cudaEvent_t done = nullptr;
  std::vector<cudaEvent_t> dom_ev;
  std::string err;
};

static sphbuf_status batch_fail(sphbuf_batch* b, sphbuf_status s, const std::string& msg) {
  if (b) b->err = msg;
  return s;
}

#define BCK(call)                                                                            \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) return batch_fail(b, SPHBUF_ERR_CUDA, std::string(#call) + ": " + \
                                             cudaGetErrorString(e_));                        \
  } while (0)

// Block maps of every batched kernel: domain d gets a share of the blocks proportional to
// its work (particles for the particle kernels, candidate cells for the buffer kernel, scan
// tiles for the scans, one block for the per-domain single-block kernels).
static sphbuf_status batch_build_maps(sphbuf_batch* b) {
  const int nd = (int)b->doms.size();
  double total_n = 0;
  for (uint64_t v : b->n0) total_n += (double)std::max<uint64_t>(v, 1);
  for (int k = 0; k < K_COUNT; ++k) {
    const double T = (double)b->sm_count * b->mk[k];
    std::vector<int4> map;
    for (int q = 0; q < nd; ++q) {
      const DomainDev& v = b->doms[q]->dev;
      int cnt = 1;
      switch (k) {
        case K_BUFFER: {
          const int cells_per_block = b->cpw * (b->thr[k] / 32);
          cnt = std::max(1, (v.nseg + cells_per_block - 1) / cells_per_block);
          break;
        }
        case K_SCAN_REDUCE:
        case K_SCAN_DOWN:
          cnt = v.scan_tiles;
          break;
        case K_SCAN_TOP:
        case K_BEGIN:
          cnt = 1;
          break;
        case K_FINALIZE:
          cnt = finalize_blocks(v);
          break;
        default:
          cnt = std::max(1, (int)std::lround(T * (double)std::max<uint64_t>(b->n0[q], 1) / total_n));
      }
      for (int l = 0; l < cnt; ++l) map.push_back(make_int4(q, l, cnt, 0));
    }
    if (b->d_maps[k]) cudaFree(b->d_maps[k]);
    b->d_maps[k] = nullptr;
    BCK(cudaMalloc(&b->d_maps[k], map.size() * sizeof(int4)));
    BCK(cudaMemcpy(b->d_maps[k], map.data(), map.size() * sizeof(int4), cudaMemcpyHostToDevice));
    b->nblocks[k] = (int)map.size();
  }
  b->mult = b->mk[K_NEIGHBOURS];
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return SPHBUF_OK;
}

// Every blocks-per-SM multiplier m to m (particle kernels), block sizes left as they are.
static void batch_set_mult(sphbuf_batch* b, int m) {
  for (int k = 0; k < K_COUNT; ++k) b->mk[k] = m;
}

static int batch_launch_k(sphbuf_batch* b, Kern k, bool fused, int sub) {
  const BatchDev bd{b->d_doms, b->d_maps[k]};
  const int n = b->nblocks[k];
  switch (k) {
    case K_BEGIN:
    case K_NEIGHBOURS:
    case K_DENSITY_DEFER:
    case K_FORCE:
    case K_DRIFT:
    case K_VISCOUS:
    case K_ACOUSTIC:
    case K_DUAL_FINISH:
      return launch_batch_sph(k, b->dim, bd, n, b->stream, b->tvf, sub, fused, b->thr[k]);
    case K_BUFFER:
    case K_BUFFER_FULL:
      return launch_batch_buffer(k, b->dim, bd, n, b->rot, b->thr[k], b->cpw, b->stream);
    default:
      return launch_batch_cells(k, b->dim, bd, n, b->thr[k], b->stream, b->kin_step);
  }
}

static int batch_launch(sphbuf_batch* b, Kern k, bool fused = false, int sub = 0) {
  if (!b->ktime) return batch_launch_k(b, k, fused, sub);
  if (b->kev.size() < 2 * (b->kpos + 1)) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    b->kev.push_back(e0);
    b->kev.push_back(e1);
  }
  cudaEventRecord(b->kev[2 * b->kpos], b->stream);
  const int r = batch_launch_k(b, k, fused, sub);
  cudaEventRecord(b->kev[2 * b->kpos + 1], b->stream);
  if (b->kid.size() <= b->kpos) b->kid.resize(b->kpos + 1);
  b->kid[b->kpos++] = (int)k;
  return r;
}

// One batched step; phases timed as for a single domain.
static int batch_enqueue_step(sphbuf_batch* b, unsigned phases, bool timed) {
  cudaStream_t s = b->stream;
  const bool fused = fused_decisions(phases, b->rot);
  b->kin_step = (phases & SPHBUF_PHASE_KINEMATIC) != 0;
  int k = 0;
  if (b->persistent && !timed && !b->ktime && phases == SPHBUF_STEP_DEFAULT) {
    PersistDev p{};
    p.doms = b->d_doms;
    for (int q = 0; q < kPersistPhases; ++q) {
      p.map[q] = b->d_maps[kPersistKern[q]];
      p.nvb[q] = b->nblocks[kPersistKern[q]];
    }
    p.bar = b->d_bar;
    p.spin_limit = b->spin_limit;
    p.ndom = (int)b->doms.size();
    return launch_persistent(p, b->dim, b->tvf, b->pgrid, s) == cudaSuccess ? 1 : -1;
  }
  if (timed) cudaEventRecord(b->ev[0], s);
  if (phases & SPHBUF_PHASE_PHYSICS) {
    k += batch_launch(b, K_NEIGHBOURS);
    if (timed) cudaEventRecord(b->ev[1], s);
    k += batch_launch(b, K_DENSITY_DEFER);
    if (timed) cudaEventRecord(b->ev[2], s);
    if (b->dual_n > 0) {
      k += batch_launch(b, K_VISCOUS);
      for (int q = 0; q < b->dual_n; ++q) k += batch_launch(b, K_ACOUSTIC, false, q);
      k += batch_launch(b, K_DUAL_FINISH, fused);
    } else {
      k += batch_launch(b, K_FORCE, fused);
    }
  } else {
    if (timed) cudaEventRecord(b->ev[1], s);
    if (timed) cudaEventRecord(b->ev[2], s);
    k += batch_launch(b, K_BEGIN);
    k += batch_launch(b, K_DRIFT, fused);
  }
  if (timed) cudaEventRecord(b->ev[3], s);
  if ((phases & SPHBUF_PHASE_BUFFER) && !fused)
    k += batch_launch(b, (phases & SPHBUF_PHASE_FULL_CHECK) ? K_BUFFER_FULL : K_BUFFER);
  if (timed) cudaEventRecord(b->ev[4], s);
  for (Kern r : {K_HIST, K_SCAN_REDUCE, K_SCAN_TOP, K_SCAN_DOWN, K_KEYS, K_SCATTER, K_FINALIZE}) k += batch_launch(b, r);
  if (timed) cudaEventRecord(b->ev[5], s);
  return k;
}

static sphbuf_status batch_run(sphbuf_batch* b, int nsteps, unsigned phases, bool timed, double* acc_ms) {
  // order after the domains' pending work
  for (size_t q = 0; q < b->doms.size(); ++q) {
    BCK(cudaEventRecord(b->dom_ev[q], b->doms[q]->stream));
    BCK(cudaStreamWaitEvent(b->stream, b->dom_ev[q], 0));
  }
  uint64_t launched = 0;
  for (int s = 0; s < nsteps; ++s) {
    if (timed) {
      launched += (uint64_t)batch_enqueue_step(b, phases, true);
      BCK(cudaEventSynchronize(b->ev[kPhases]));
      for (int p = 0; p < kPhases; ++p) {
        float ms = 0;
        BCK(cudaEventElapsedTime(&ms, b->ev[p], b->ev[p + 1]));
        if (acc_ms) acc_ms[p] += ms;
      }
    } else if (b->use_graph) {
      if (!b->graph || b->graph_phases != phases) {
        if (b->graph) {
          cudaGraphExecDestroy(b->graph);
          b->graph = nullptr;
        }
        cudaGraph_t g = nullptr;
        BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        const int nk = batch_enqueue_step(b, phases, false);
        const cudaError_t le = cudaGetLastError();
        const cudaError_t ce = cudaStreamEndCapture(b->stream, &g);
        if (nk < 0 || le != cudaSuccess || ce != cudaSuccess) {
          if (g) cudaGraphDestroy(g);
          return batch_fail(b, SPHBUF_ERR_CUDA, std::string("capturing the batched step: ") +
                                                    cudaGetErrorString(le != cudaSuccess ? le : ce));
        }
        b->graph_launches = (uint64_t)nk;
        BCK(cudaGraphInstantiate(&b->graph, g, 0));
        cudaGraphDestroy(g);
        b->graph_phases = phases;
      }
      BCK(cudaGraphLaunch(b->graph, b->stream));
      launched += b->graph_launches;
    } else {
      const int nk = batch_enqueue_step(b, phases, false);
      if (nk < 0) return batch_fail(b, SPHBUF_ERR_CUDA, std::string("persistent step launch: ") +
                                                        cudaGetErrorString(cudaGetLastError()));
      launched += (uint64_t)nk;
    }
  }
  BCK(cudaGetLastError());
  // the domains' later work waits for the batch
  BCK(cudaEventRecord(b->done, b->stream));
  for (sphbuf_domain* d : b->doms) {
    BCK(cudaStreamWaitEvent(d->stream, b->done, 0));
    d->launches += launched;  // every kernel of the batch works for every domain
    d->stepped = true;
  }
  return SPHBUF_OK;
}

sphbuf_status sphbuf_batch_create(sphbuf_domain_t* domains, int n, void* cuda_stream, sphbuf_batch_t* out) {
  if (!domains || n <= 0 || !out) return SPHBUF_ERR_INVALID_ARG;
  *out = nullptr;
  auto* b = new sphbuf_batch();
  b->dim = domains[0] ? domains[0]->desc.dim : 0;
  for (int q = 0; q < n; ++q) {
    sphbuf_domain* d = domains[q];
    if (!d || d->desc.dim != b->dim) {
      delete b;
      return SPHBUF_ERR_INVALID_ARG;
    }
    for (int r = 0; r < q; ++r)
      if (domains[r] == d) {
        delete b;
        return SPHBUF_ERR_INVALID_ARG;
      }
    if (!d->committed && !d->need_rebuild) {
      delete b;
      return SPHBUF_ERR_STATE;
    }
    sphbuf_status s = commit(d);
    if (s != SPHBUF_OK) {
      delete b;
      return s;
    }
    StepState st;
    s = read_state(d, &st);
    if (s != SPHBUF_OK) {
      delete b;
      return s;
    }
    if (q == 0) b->dual_n = d->dev.P.dual_n;
    if (d->dev.P.dual_n != b->dual_n) {
      delete b;
      return SPHBUF_ERR_INVALID_ARG;
    }
    b->doms.push_back(d);
    b->n0.push_back(st.n);
    if (d->dev.P.tvf_lambda > 0.f) b->tvf = true;
    if (d->dev.any_rot) b->rot = true;
  }
  b->sm_count = b->doms[0]->dev.sm_count;
  if (cuda_stream) {
    b->stream = static_cast<cudaStream_t>(cuda_stream);
  } else if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) == cudaSuccess) {
    b->own_stream = true;
  } else {
    delete b;
    return SPHBUF_ERR_CUDA;
  }
  std::vector<DomainDev> host(n);
  for (int q = 0; q < n; ++q) host[q] = b->doms[q]->dev;
  bool ok = cudaMalloc(&b->d_doms, n * sizeof(DomainDev)) == cudaSuccess &&
            cudaMemcpy(b->d_doms, host.data(), n * sizeof(DomainDev), cudaMemcpyHostToDevice) == cudaSuccess;
  for (int p = 0; ok && p <= kPhases; ++p) ok = cudaEventCreate(&b->ev[p]) == cudaSuccess;
  ok = ok && cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) == cudaSuccess;
  b->dom_ev.assign(n, nullptr);
  for (int q = 0; ok && q < n; ++q) ok = cudaEventCreateWithFlags(&b->dom_ev[q], cudaEventDisableTiming) == cudaSuccess;
  for (int k = 0; k < K_COUNT; ++k) b->thr[k] = batch_threads((Kern)k);
  batch_set_mult(b, 8);
  if (!ok || batch_build_maps(b) != SPHBUF_OK) {
    sphbuf_batch_destroy(b);
    return SPHBUF_ERR_CUDA;
  }
  *out = b;
  return SPHBUF_OK;
}

static bool batch_phases_ok(unsigned phases) {
  const bool phys = phases & SPHBUF_PHASE_PHYSICS, kin = phases & SPHBUF_PHASE_KINEMATIC;
  return phys != kin && !(phases & ~31u);
}

sphbuf_status sphbuf_batch_step(sphbuf_batch_t b, int nsteps, unsigned phases) {
  if (!b || nsteps < 0) return SPHBUF_ERR_INVALID_ARG;
  if (!batch_phases_ok(phases)) return batch_fail(b, SPHBUF_ERR_INVALID_ARG, "bad phase mask");
  for (sphbuf_domain* d : b->doms) {
    if (d->need_rebuild) return batch_fail(b, SPHBUF_ERR_STATE, "a domain was rewritten after batching");
    if (d->dev.P.reuse && (phases & (SPHBUF_PHASE_FULL_CHECK | SPHBUF_PHASE_BUFFER_KERNEL)))
      return batch_fail(b, SPHBUF_ERR_INVALID_ARG, "kept neighbour lists need the decisions fused into the drift");
  }
  return batch_run(b, nsteps, phases, false, nullptr);
}

sphbuf_status sphbuf_batch_use_graph(sphbuf_batch_t b, int enable) {
  if (!b) return SPHBUF_ERR_INVALID_ARG;
  b->use_graph = enable != 0;
  return SPHBUF_OK;
}

// Runs nsteps plain batched steps with an event pair around every launch; acc[k] receives
// kernel k's milliseconds summed over its launches and the steps.
static sphbuf_status batch_time_kernels(sphbuf_batch* b, int nsteps, unsigned phases, std::vector<double>& acc) {
  acc.assign(K_COUNT, 0.0);
  const bool graph = b->use_graph;
  b->use_graph = false;
  b->ktime = true;
  sphbuf_status s = SPHBUF_OK;
  for (int q = 0; q < nsteps && s == SPHBUF_OK; ++q) {
    b->kpos = 0;
    s = batch_run(b, 1, phases, false, nullptr);
    if (s == SPHBUF_OK && cudaStreamSynchronize(b->stream) != cudaSuccess)
      s = batch_fail(b, SPHBUF_ERR_CUDA, "autotune: stream synchronisation failed");
    for (size_t e = 0; s == SPHBUF_OK && e < b->kpos; ++e) {
      float ms = 0;
      if (cudaEventElapsedTime(&ms, b->kev[2 * e], b->kev[2 * e + 1]) == cudaSuccess) acc[b->kid[e]] += ms;
    }
  }
  b->ktime = false;
  b->use_graph = graph;
  return s;
}

sphbuf_status sphbuf_batch_autotune(sphbuf_batch_t b, int trial_steps, unsigned phases, int* best_m,
                                    double ms_per_step[5]) {
  if (!b || trial_steps <= 0) return SPHBUF_ERR_INVALID_ARG;
  if (!batch_phases_ok(phases)) return batch_fail(b, SPHBUF_ERR_INVALID_ARG, "bad phase mask");
  const int threads_c[] = {64, 128, 256, 512};
  const int mult_c[] = {1, 2, 4, 8, 16};
  std::vector<double> best(K_COUNT, 1e300), acc;
  std::vector<int> bt(K_COUNT), bm(K_COUNT);
  // every (block size, blocks per SM) pair for all tunable kernels at once; each kernel keeps
  // the pair under which it ran fastest (the kernels' times do not depend on one another's
  // launch shapes)
  for (int t : threads_c)
    for (int m : mult_c) {
      for (int k = 0; k < K_COUNT; ++k)
        if (batch_tunable((Kern)k)) b->thr[k] = t;
      batch_set_mult(b, m);
      sphbuf_status s = batch_build_maps(b);
      if (s == SPHBUF_OK) s = batch_time_kernels(b, trial_steps, phases, acc);
      if (s != SPHBUF_OK) return s;
      for (int k = 0; k < K_COUNT; ++k)
        if (batch_tunable((Kern)k) && acc[k] > 0.0 && acc[k] < best[k]) {
          best[k] = acc[k];
          bt[k] = t;
          bm[k] = m;
        }
    }
  for (int k = 0; k < K_COUNT; ++k) {
    const bool ran = batch_tunable((Kern)k) && best[k] < 1e300;
    b->thr[k] = ran ? bt[k] : batch_threads((Kern)k);
    b->mk[k] = ran ? bm[k] : 8;
  }
  // the buffer kernel's cell tile, when the phases launch it
  if (best[K_BUFFER] < 1e300) {
    double bb = 1e300;
    int bc = 4;
    for (int c : {1, 2, 4, 8}) {
      b->cpw = c;
      sphbuf_status s = batch_build_maps(b);
      if (s == SPHBUF_OK) s = batch_time_kernels(b, trial_steps, phases, acc);
      if (s != SPHBUF_OK) return s;
      if (acc[K_BUFFER] > 0.0 && acc[K_BUFFER] < bb) {
        bb = acc[K_BUFFER];
        bc = c;
      }
    }
    b->cpw = bc;
  }
  sphbuf_status s = batch_build_maps(b);
  if (s != SPHBUF_OK) return s;
  double ph[kPhases] = {0, 0, 0, 0, 0};
  s = batch_run(b, trial_steps, phases, true, ph);
  if (s != SPHBUF_OK) return s;
  if (best_m) *best_m = b->mk[K_NEIGHBOURS];
  if (ms_per_step)
    for (int p = 0; p < kPhases; ++p) ms_per_step[p] = ph[p] / trial_steps;
  return SPHBUF_OK;
}

sphbuf_status sphbuf_batch_set_grid(sphbuf_batch_t b, int m) {
  if (!b || m < 1 || m > 32) return SPHBUF_ERR_INVALID_ARG;
  BCK(cudaStreamSynchronize(b->stream));
  batch_set_mult(b, m);
  return batch_build_maps(b);
}

// Public kernel ids of sphbuf_batch_config and the library's kernels.
static const Kern kTuned[SPHBUF_KERNEL_COUNT] = {K_NEIGHBOURS, K_DENSITY_DEFER, K_FORCE,   K_DRIFT,
                                                 K_VISCOUS,    K_ACOUSTIC,      K_DUAL_FINISH, K_BUFFER,
                                                 K_BUFFER_FULL, K_HIST,         K_KEYS,    K_SCATTER};

sphbuf_status sphbuf_batch_get_config(sphbuf_batch_t b, sphbuf_batch_config* cfg) {
  if (!b || !cfg) return SPHBUF_ERR_INVALID_ARG;
  for (int q = 0; q < SPHBUF_KERNEL_COUNT; ++q) {
    cfg->threads[q] = b->thr[kTuned[q]];
    cfg->blocks_per_sm[q] = b->mk[kTuned[q]];
  }
  cfg->cells_per_warp = b->cpw;
  return SPHBUF_OK;
}

sphbuf_status sphbuf_batch_set_config(sphbuf_batch_t b, const sphbuf_batch_config* cfg) {
  if (!b || !cfg) return SPHBUF_ERR_INVALID_ARG;
  for (int q = 0; q < SPHBUF_KERNEL_COUNT; ++q) {
    const int t = cfg->threads[q], m = cfg->blocks_per_sm[q];
    if (t < 32 || t > 512 || t % 32 || m < 1 || m > 32)
      return batch_fail(b, SPHBUF_ERR_INVALID_ARG, "threads must be a multiple of 32 in 32..512, blocks per SM 1..32");
  }
  const int c = cfg->cells_per_warp;
  if (c != 1 && c != 2 && c != 4 && c != 8) return batch_fail(b, SPHBUF_ERR_INVALID_ARG, "cells per warp: 1, 2, 4 or 8");
  BCK(cudaStreamSynchronize(b->stream));
  for (int q = 0; q < SPHBUF_KERNEL_COUNT; ++q) {
    b->thr[kTuned[q]] = cfg->threads[q];
    b->mk[kTuned[q]] = cfg->blocks_per_sm[q];
  }
  b->cpw = c;
  return batch_build_maps(b);
}

sphbuf_status sphbuf_batch_set_persistent(sphbuf_batch_t b, int enable, long long spin_limit) {
  if (!b) return SPHBUF_ERR_INVALID_ARG;
  if (enable && (b->rot || b->dual_n > 0))
    return batch_fail(b, SPHBUF_ERR_INVALID_ARG,
                      "the persistent step serves single-rate batches without rotating buffers");
  BCK(cudaStreamSynchronize(b->stream));
  if (enable && !b->d_bar) BCK(cudaMalloc(&b->d_bar, 4 * sizeof(unsigned)));
  if (enable) {
    b->pgrid = persistent_grid(b->dim, b->tvf);
    if (b->pgrid <= 0) return batch_fail(b, SPHBUF_ERR_CUDA, "no resident grid for the persistent step");
  }
  b->persistent = enable != 0;
  b->spin_limit = spin_limit < 0 ? (1ll << 24) : spin_limit;
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return SPHBUF_OK;
}

sphbuf_status sphbuf_batch_sync(sphbuf_batch_t b) {
  if (!b) return SPHBUF_ERR_INVALID_ARG;
  BCK(cudaStreamSynchronize(b->stream));
  for (sphbuf_domain* d : b->doms) {
    StepState st;
    sphbuf_status s = read_state(d, &st);
    if (s != SPHBUF_OK) return batch_fail(b, s, d->err);
  }
  return SPHBUF_OK;
}

sphbuf_status sphbuf_batch_destroy(sphbuf_batch_t b) {
  if (!b) return SPHBUF_ERR_INVALID_ARG;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (int k = 0; k < K_COUNT; ++k)
    if (b->d_maps[k]) cudaFree(b->d_maps[k]);
  for (cudaEvent_t e : b->kev) cudaEventDestroy(e);
  if (b->d_bar) cudaFree(b->d_bar);
  if (b->d_doms) cudaFree(b->d_doms);
  for (int p = 0; p <= kPhases; ++p)
    if (b->ev[p]) cudaEventDestroy(b->ev[p]);
  if (b->done) cudaEventDestroy(b->done);
  for (cudaEvent_t e : b->dom_ev)
    if (e) cudaEventDestroy(e);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
  return SPHBUF_OK;
}

sphbuf_status sphbuf_candidate_count(sphbuf_domain_t d, int k, uint64_t* cells, uint64_t* particles) {
  if (!d || k < 0 || (size_t)k >= d->bufs.size()) return SPHBUF_ERR_INVALID_ARG;
  if (!d->committed) return fail(d, SPHBUF_ERR_STATE, "no cell-linked list yet");
  StepState st;
  sphbuf_status s = read_state(d, &st);
  if (s != SPHBUF_OK) return s;
  std::vector<unsigned> start((size_t)d->ncell + 1);
  CK(cudaMemcpy(start.data(), d->dev.cell_start, start.size() * sizeof(unsigned), cudaMemcpyDeviceToHost));
  uint64_t nc = 0, np = 0;
  for (size_t q = 0; q < d->segbuf_host.size(); ++q) {
    if (d->segbuf_host[q] != k) continue;
    const int l0 = d->seg_host[2 * q], l1 = d->seg_host[2 * q + 1];
    nc += (uint64_t)(l1 - l0);
    np += start[l1] - start[l0];
  }
  if (cells) *cells = nc;
  if (particles) *particles = np;
  return SPHBUF_OK;
}

sphbuf_status sphbuf_read_launch_count(sphbuf_domain_t d, uint64_t* launches) {
  if (!d || !launches) return SPHBUF_ERR_INVALID_ARG;
  *launches = d->launches;
  return SPHBUF_OK;
}

sphbuf_status sphbuf_cell_list_build(const int32_t* cell, const uint32_t* id, const uint8_t* label, uint64_t n,
                                     uint64_t ncell, uint32_t* cell_start, uint32_t* order, void* cuda_stream) {
  if ((n && (!cell || !id || !order)) || !cell_start || ncell == 0 || n >= 0xF0000000ull ||
      ncell >= (1ull << 31) - kScanTile)
    return SPHBUF_ERR_INVALID_ARG;
  int bad = 0;
  cudaError_t e = sphbuf::cell_list_build(cell, id, label, n, ncell, cell_start, order,
                                          static_cast<cudaStream_t>(cuda_stream), &bad);
  if (e != cudaSuccess) return SPHBUF_ERR_CUDA;
  return bad ? SPHBUF_ERR_INVALID_ARG : SPHBUF_OK;
}

sphbuf_status sphbuf_cell_list_build_noalloc(const int32_t* cell, const uint32_t* id, const uint8_t* label,
                                             uint64_t n, uint64_t ncell, uint32_t* cell_start, uint32_t* order,
                                             void* cuda_stream) {
  if ((n && (!cell || !id || !order)) || !cell_start || ncell == 0) return SPHBUF_ERR_INVALID_ARG;
  if (n > sphbuf::cell_list_noalloc_max_particles() || ncell > sphbuf::cell_list_noalloc_max_cells())
    return SPHBUF_ERR_CAPACITY;
  int bad = 0;
  cudaError_t e = sphbuf::cell_list_build_noalloc(cell, id, label, n, ncell, cell_start, order,
                                                  static_cast<cudaStream_t>(cuda_stream), &bad);
  if (e != cudaSuccess) return SPHBUF_ERR_CUDA;
  return bad ? SPHBUF_ERR_INVALID_ARG : SPHBUF_OK;
}

}  // extern "C"
