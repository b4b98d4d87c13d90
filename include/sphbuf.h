/*
 * sphbuf.h - C ABI of the GB300 (sm_103a) open-boundary SPH library.
 *
 * The library runs, on one GPU, the per-step hot path of the arbitrary-positioned
 * in-/outflow buffer of Zhang, Fan, Ren, Qian & Hu, "Generalized and high-efficiency
 * arbitrary-positioned buffer for smoothed particle hydrodynamics" (arXiv 2406.16786),
 * inside a plain weakly-compressible SPH step:
 *
 *   1 density  - Eq. (9) summation for fluid particles, Eq. (4) continuity for buffer
 *                particles (Sec. 4: no re-initialisation near the open boundary);
 *   2 force    - Eq. (5) Riemann momentum with the Eq. (8) limiter; Eq. (18) for buffer
 *                particles; kick, Eqs. (23)-(26) velocity BC or Eq. (19) projection; drift;
 *   3 decide   - Algorithms 1-3: local-frame transform (Eqs. (11), (15)) of the particles in
 *                the cells around each buffer and the normal-axis test X' > a/2 / X' < -a/2;
 *   4 apply    - duplicate + recycle (Eqs. (16)-(17), density Eq. (22)), delete;
 *   5 rebuild  - counting-sort cell-linked list, sorted by (cell, id);
 *   6 relabel  - outflow / bidirectional buffers after the rebuild (Algorithms 2-3).
 *
 * Conventions
 * -----------
 * Grid: cell size cs = 2 h, h = h_over_dp * dp; nx = ceil((hi_x - lo_x) / cs) (same for y, z;
 * nz = 1 in 2-D); linear cell index lin = (cz * ny + cy) * nx + cx.
 * Particle positions are stored cell-relative: an int32 linear cell index plus an FP32
 * offset f in [0, cs32) per axis (cs32 = FP32 rounding of cs).  Global x = lo + c cs + f.
 * Particle arrays are structure-of-arrays on the host side of this ABI: frac and vel are
 * n x dim row-major (x, y[, z] per particle).  Labels: 0 = fluid, k + 1 = particle of
 * buffer k, 255 = never returned (deleted).
 * Buffer frame: row-major R (3 x 3, FP64) with X' = R (X - O'); R's first row is the unit
 * normal, pointing in the inflow direction for inlets and bidirectional buffers and in
 * the outflow direction for outlets (Sec. 3.1-3.2).  In 2-D only the upper-left 2 x 2
 * block and the first two components of origin are used.
 *
 * FP32 decision contract (bit-exact with an FP32 restatement of Algorithms 1-3):
 *   cO = floor((O - lo) / cs) and fO = fl32((O - lo) - cO cs) per axis (FP64 host math);
 *   D = fl(fl(fl(c - cO) * cs32) + fl(f - fO));  X'_r = ((R_r0 D0 + R_r1 D1) + R_r2 D2)
 *   with every product and sum rounded to FP32 separately; thresholds fl32(a/2), fl32(b/2),
 *   fl32(c/2); outflow candidates additionally need |X'| < fl32(a/2 + cs), |Y'| < fl32(b/2 + cs)
 *   (|Z'| < fl32(c/2 + cs)).  Moves (drift fl(v * fl32(dt)), recycling fl32(-a R[0][x])) use
 *   f = fl(f + delta) then at most 8 folds {f >= cs32: f -= cs32, c++; f < 0: f += cs32, c--}.
 *   Injections are numbered in (buffer, parent id) order: new id = next_id + rank.
 *
 * Ownership: the library allocates and frees all device memory of a domain; host pointers
 * passed in are only read (or written, for read_* calls) during the call, except those of
 * the asynchronous transfers, which are used until sphbuf_io_wait returns.
 * Threads: calls on one domain (or batch) must not overlap; different domains may be used
 * from different host threads.
 * Errors: every call returns a status.  Asynchronous device-side errors (capacity overflow,
 * NaN positions) are latched in the domain and returned by the next synchronising call
 * (sphbuf_sync or any sphbuf_read_*); once latched, later steps do no work.  No call traps
 * or aborts.  sphbuf_error_message gives a one-line text for the domain's last error.
 */
#ifndef SPHBUF_H
#define SPHBUF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sphbuf_domain *sphbuf_domain_t; /* opaque, library-owned */

typedef enum {
  SPHBUF_OK = 0,
  SPHBUF_ERR_INVALID_ARG = 1, /* bad pointer, size, dimension, non-orthonormal frame, ... */
  SPHBUF_ERR_CAPACITY = 2,    /* particle capacity or per-step list capacity exceeded */
  SPHBUF_ERR_OVERLAP = 3,     /* two buffers' candidate regions overlap */
  SPHBUF_ERR_CUDA = 4,        /* a CUDA runtime call failed */
  SPHBUF_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
  SPHBUF_ERR_NAN = 6,         /* a non-finite position was met */
  SPHBUF_ERR_STATE = 7,       /* call not valid now (e.g. add_inout_buffer after the first step) */
  SPHBUF_ERR_BOUNDS = 8       /* an index check of the bounds-checked build failed (the library
                                 built with SPHBUF_CHECK=1); the failing site and index are in
                                 the domain's error message */
} sphbuf_status;

typedef enum {
  SPHBUF_VELOCITY_INLET = 0,  /* unidirectional inflow buffer (Algorithm 1), velocity BC */
  SPHBUF_PRESSURE_OUTLET = 1, /* unidirectional outflow buffer (Algorithm 2), pressure BC */
  SPHBUF_PRESSURE_INLET = 2,  /* Algorithm 1 with the pressure BC (PIVO inlet, Sec. 5.1) */
  SPHBUF_VELOCITY_OUTLET = 3, /* Algorithm 2 with the velocity BC (PIVO outlet, Sec. 5.1) */
  SPHBUF_BIDIR_PRESSURE = 4,  /* bidirectional buffer (Algorithm 3), pressure BC */
  SPHBUF_BIDIR_VELOCITY = 5   /* bidirectional buffer (Algorithm 3), velocity BC */
} sphbuf_bc_type;

/* Phase masks for sphbuf_step_phases.  Exactly one of PHYSICS / KINEMATIC is required.
 * The rebuild and relabel always close a step. */
#define SPHBUF_PHASE_PHYSICS 1u     /* density, force, kick + BC velocity, drift */
#define SPHBUF_PHASE_KINEMATIC 2u   /* drift only, with the stored velocity (no BC) */
#define SPHBUF_PHASE_BUFFER 4u      /* decisions + apply (Algorithms 1-3); by default fused into
                                       the drift of the step: each particle sorted into a
                                       candidate cell of a buffer (Sec. 3.1's local cells) is
                                       decided right after its drift */
#define SPHBUF_PHASE_FULL_CHECK 8u  /* decisions over all particles instead of the cells around
                                       each buffer, in a kernel of their own (same result; for
                                       timing comparisons) */
#define SPHBUF_PHASE_BUFFER_KERNEL 16u /* decisions in a kernel of their own after the drift,
                                          visiting the candidate cells (same result as the fused
                                          form; the form always used for rotating buffers) */
#define SPHBUF_STEP_DEFAULT (SPHBUF_PHASE_PHYSICS | SPHBUF_PHASE_BUFFER)

typedef struct {
  int dim;                  /* 2 or 3 */
  double lo[3], hi[3];      /* grid box, global coordinates (m); must contain every particle;
                               cut into cells of 2h, at most 2048 x 2048 x 1024 of them
                               (SPHBUF_ERR_INVALID_ARG otherwise) */
  double dp;                /* initial particle spacing (m) */
  double h_over_dp;         /* smoothing length / dp (1.3 in the paper, Sec. 3) */
  double rho0, c0, nu, dt;  /* reference density, artificial sound speed, kinematic viscosity,
                               fixed time step */
  uint64_t capacity;        /* maximum number of fluid particles, at most 2^25 - 1 (walls too) */
} sphbuf_domain_desc;

typedef struct {
  double umax;       /* velocity BC: peak speed U of the profile (Eqs. (23)-(24)) */
  double half_width; /* velocity BC: profile radius R in U (1 - (Y'^2 + Z'^2)/R^2); 0 = plug U */
  double p_b;        /* pressure BC: p_b(t) = p_b + p_amp sin(p_omega t + p_phase) (Eq. (18)) */
  double p_amp, p_omega, p_phase;
} sphbuf_bc_params;

const char *sphbuf_status_string(sphbuf_status s);

/* Last error text of a domain ("" if none).  Valid until the next call on the domain. */
const char *sphbuf_error_message(sphbuf_domain_t d);

/* Creates an empty domain and allocates its device memory (capacity-sized) on the current
 * CUDA device.  cuda_stream: a cudaStream_t on which every later call of this domain
 * enqueues its work; NULL makes the domain create (and later destroy) a private
 * non-blocking stream. */
sphbuf_status sphbuf_create_domain(const sphbuf_domain_desc *desc, void *cuda_stream,
                                   sphbuf_domain_t *out);
sphbuf_status sphbuf_destroy(sphbuf_domain_t d);

/* Fixed wall particles (3 layers, Sec. 3), FP64 global positions n x dim.  Replaces any
 * previous walls.  Only before the first step. */
sphbuf_status sphbuf_set_walls(sphbuf_domain_t d, const double *pos, uint64_t n);

/* Fluid particles from FP64 global positions (n x dim), FP32 velocity (n x dim) and density
 * (n); ids 0..n-1, labels 0; inflow buffer particles are identified at the first step
 * (Algorithm 1).  Only before the first step. */
sphbuf_status sphbuf_set_fluid(sphbuf_domain_t d, const double *pos, const float *vel,
                               const float *rho, uint64_t n);

/* Fluid particles in the native cell-relative encoding (see Conventions).  id NULL means
 * 0..n-1.  label NULL means 0 everywhere and Algorithm 1's identification runs at the next
 * step; a non-NULL label array is taken as is (restart).  next_id: first id for new
 * particles (>= every id).  Allowed before the first step and between steps (restart).
 * The arrays are copied to the device as they are and checked there (cell inside the grid,
 * offsets in [0, cs32), labels naming a buffer, next_id above every id); a check that fails
 * returns SPHBUF_ERR_INVALID_ARG and leaves the domain with no particles.  Pinned host
 * arrays make the copies direct. */
sphbuf_status sphbuf_write_particles(sphbuf_domain_t d, const int32_t *cell, const float *frac,
                                     const float *vel, const float *rho, const uint32_t *id,
                                     const uint8_t *label, uint64_t n, uint32_t next_id);

/* Pipelined host transfers (overlap the copies of one step with the work of another).
 * sphbuf_write_particles_async: the arrays of sphbuf_write_particles, copied to a device
 * staging area on a stream of the domain's own, so that the copies overlap the work already
 * enqueued on the domain's stream; the next step (or read) waits for them, checks the arrays
 * on the device and takes them into the state.  A failed check is latched: the next
 * synchronising call returns SPHBUF_ERR_INVALID_ARG, and the domain is left with no
 * particles.  Only one asynchronous write may wait for a step: another one before that
 * returns SPHBUF_ERR_STATE; a synchronous write replaces it.
 * sphbuf_read_particles_async: after the work enqueued so far, the device gathers the sorted
 * state (as sphbuf_read_particles) into a second staging area and the first cap rows of each
 * array (frac, vel: cap x dim) are copied to the host on another stream, overlapping later
 * steps; rows past the particle count hold unspecified values.  All six arrays are required.
 * *n_out (may be NULL) receives the particle count when sphbuf_io_wait returns, which
 * returns SPHBUF_ERR_CAPACITY if the count exceeded cap (only cap rows were copied).
 * Up to 64 reads may be pending; the 65th waits for the others first.
 * sphbuf_io_wait: waits for every pending asynchronous copy and for the domain's stream,
 * fills n_out of the pending reads and returns any latched error.
 * Host arrays: page-locked (cudaHostAlloc, cudaHostRegister, torch pin_memory) for the copies
 * to be asynchronous; the caller keeps them valid and unchanged until sphbuf_io_wait returns.
 * The first asynchronous call allocates two staging areas of (13 + 8 dim) bytes per particle
 * of capacity, two streams and four events, held until sphbuf_destroy. */
sphbuf_status sphbuf_write_particles_async(sphbuf_domain_t d, const int32_t *cell, const float *frac,
                                           const float *vel, const float *rho, const uint32_t *id,
                                           const uint8_t *label, uint64_t n, uint32_t next_id);
sphbuf_status sphbuf_read_particles_async(sphbuf_domain_t d, int32_t *cell, float *frac, float *vel,
                                          float *rho, uint32_t *id, uint8_t *label, uint64_t cap,
                                          uint64_t *n_out);
sphbuf_status sphbuf_io_wait(sphbuf_domain_t d);

/* Adds one in-/outlet buffer: box centre O' (origin), frame R (rotation, see Conventions),
 * extent = (a, b, c): width along X', length along Y', height along Z' (c unused in 2-D).
 * R must be orthonormal with det +1 (tolerance 1e-9).  Candidate regions of two buffers
 * (box dilated by 2 cs) must not overlap.  Only before the first step.  *out_id = k. */
sphbuf_status sphbuf_add_inout_buffer(sphbuf_domain_t d, const double origin[3],
                                      const double rotation[9], const double extent[3],
                                      sphbuf_bc_type bc, const sphbuf_bc_params *params,
                                      int *out_id);

/* Time-varying frame of inflow buffer buffer_id (Sec. 5.3, the rotating sprinkler: the
 * buffer turns with the constant angular velocity omega, theta = omega t + theta_0).  After
 * the particle generation of each step the buffer's particles (positions and velocities) are
 * rotated by omega dt about pivot (about the z axis in 2-D, about axis in 3-D; axis need not
 * be unit length and is ignored in 2-D), and the frame is re-established for the next step:
 * with M the rotation by omega dt and Q_n = M^n, the frame of step n is
 * O'_n = pivot + Q_n (O'_0 - pivot), R_n = R_0 Q_n^T (FP64 recurrence, the FP32 decision
 * constants re-derived each step).  Positions move in the FP32 contract: offset from the
 * pivot D, D' = fl32(M) D row by row, move by D' - D.  The candidate cells are those the
 * box (dilated by 2 cs) can reach while it turns.  Errors: SPHBUF_ERR_INVALID_ARG (not an
 * inflow buffer, no axis in 3-D, non-finite input), SPHBUF_ERR_STATE (after the first step or
 * set twice), SPHBUF_ERR_OVERLAP (the swept region meets another buffer's candidate region).
 * Only before the first step. */
sphbuf_status sphbuf_set_buffer_rotation(sphbuf_domain_t d, int buffer_id, const double pivot[3],
                                         const double axis[3], double omega);

/* Background pressure of the equation of state: p = c0^2 (rho - rho0) + p_bg (Eq. (3) plus
 * a constant, default 0).  Only pressure differences and the open-boundary term of Eq. (18)
 * act on the flow, so a p_bg above the largest expected suction keeps every pressure
 * positive and avoids the tensile instability of plain WCSPH where the gauge pressure goes
 * negative (the regularisation the paper obtains from its transport-velocity formulation,
 * Eq. (10)).  Prescribed buffer pressures p_b are absolute (include p_bg); a recycled
 * pressure-buffer particle gets rho = rho0 + (p_b - p_bg) / c0^2 (Eq. (22)).  Errors:
 * SPHBUF_ERR_INVALID_ARG (non-finite), SPHBUF_ERR_STATE (after the first step). */
sphbuf_status sphbuf_set_background_pressure(sphbuf_domain_t d, double p_bg);

/* Dual-criteria time stepping (Sec. 2.2): each step (of the descriptor's dt, the advection
 * step) fixes the neighbour configuration, re-initialises the density of the fluid particles
 * by Eq. (9) (buffer particles keep theirs), evaluates the viscous acceleration once, then
 * runs n_acoustic acoustic steps of dt / n_acoustic: continuity (Eq. (4)) for every particle
 * and the pressure part of Eq. (5) with Eq. (18) from the current state, kick, boundary
 * velocity, density and position update.  The buffer update and the cell-list rebuild run
 * once per step.  A buffer's flux is the mean over the acoustic steps.  n_acoustic = 0 (the
 * default) is the single-rate kick-drift step.  A particle whose neighbour list overflowed
 * (strong compression) latches SPHBUF_ERR_CAPACITY in this mode.  Batches need the same
 * n_acoustic in every domain.  Errors: SPHBUF_ERR_INVALID_ARG (outside [0, 4096]),
 * SPHBUF_ERR_STATE (after the first step), SPHBUF_ERR_CUDA (allocation). */
sphbuf_status sphbuf_set_dual_time_stepping(sphbuf_domain_t d, int n_acoustic);

/* Transport-velocity formulation (Eq. (10)): fluid particles (label 0) are advected with
 * v - dt p_max sum_j 2 m/(rho_i rho_j) dW/dr_ij e_ij instead of v, p_max = lambda rho0 v_max^2
 * with v_max the largest particle speed of the previous step's force pass (0 at the first
 * step); their momentum velocity stays v.  The buffer particles (the in-/outlet layers) are
 * advected with v.  lambda = 0 (the default) turns it off; the paper takes 5 to 10.
 * Errors: SPHBUF_ERR_INVALID_ARG (negative or non-finite), SPHBUF_ERR_STATE (after the first
 * step). */
sphbuf_status sphbuf_set_transport_velocity(sphbuf_domain_t d, double lambda);

/* RCR Windkessel outlet (Eq. (31), the aorta outlets of Sec. 6.2) for pressure buffer
 * buffer_id: its boundary pressure is computed each step from the volume flux Q through the
 * buffer instead of p_b(t).  Eq. (31) is taken as P = P_d + R_p Q with C dP_d/dt = Q - P_d / R_d
 * (the same model), integrated explicitly once per step with the flux of the previous step:
 * P_d(n) = P_d(n-1) + dt ((Q(n-1) - P_d(n-1) / R_d) / C) (n >= 1, FP64 in this order; P_d(0) =
 * p_d0, Q(-1) = 0) and p_b(t_n) = P_d(n) + R_p Q(n-1).  Q is the flux the force pass measures:
 * sum over the buffer's particles of (v . u) dp^dim / a, positive along u (outward for an
 * outlet), m^dim/s.  Units SI: r_p, r_d in Pa s / m^dim, compliance in m^dim / Pa.  Errors:
 * SPHBUF_ERR_INVALID_ARG (velocity buffer, r_p < 0, compliance or r_d <= 0, non-finite),
 * SPHBUF_ERR_STATE (after the first step).  Only before the first step. */
sphbuf_status sphbuf_set_windkessel(sphbuf_domain_t d, int buffer_id, double r_p, double compliance,
                                    double r_d, double p_d0);

/* Boundary pressure of buffer buffer_id for the current (last begun) step: p_b (FP64), the
 * Windkessel distal pressure P_d (0 without a Windkessel) and the flux Q of the step before,
 * which p_b was computed from.  Any pointer may be NULL.  Synchronises the domain's stream. */
sphbuf_status sphbuf_read_boundary_pressure(sphbuf_domain_t d, int buffer_id, double *p_b, double *p_d,
                                            double *q_prev);

/* Rodrigues frame of Eqs. (12)-(14): R with R n = e_x (reading: I - S sin + S^2 (1 - cos),
 * the transpose of the printed formula, so that X' = R (X - O') has X' along n), followed by
 * a roll about X': R <- Rx(roll) R.  n need not be unit length. */
sphbuf_status sphbuf_rotation_from_normal(const double normal[3], double roll, double out_R[9]);

/* Kept neighbour lists (a Verlet skin; the paper has no counterpart: its neighbour search is a
 * cell-linked list, Sec. 3.1, and the results here differ from it only by the order of the
 * FP32 sums): with skin_over_h > 0 the lists hold the pairs within
 * 2h + skin (skin = skin_over_h h, at most h) and are kept over steps.  A step whose rebuild
 * keeps the lists also keeps the particles' slots (no sort; deleted particles stay as dead
 * slots, duplicates are appended), except where the lists must change: the particles in the
 * buffers' candidate cells and two rings of cells around them search their neighbours again
 * every step (through a list of the live particles sorted by (cell, id), rebuilt every step).
 * A full rebuild (sort, every list searched again) follows once a pair may have come within
 * 2h unlisted: each particle's displacement since the last full rebuild is measured relative
 * to a reference velocity fixed for the period (the middle of the range of the previous
 * period's drift velocities, zero included; a pair's distance changes by at most the sum of
 * the two relative displacements, and a wall particle's is the reference velocity times the
 * time), and the rebuild follows once twice the largest of them exceeds the skin; also after
 * max_steps steps, after a kinematic step and after particles are written.
 * Results differ from lists rebuilt every step only by the order of the FP32 sums.  Reads
 * and counts always give the live particles sorted by (cell, id).  skin_over_h = 0 turns it
 * off (the default).  Only before the first step.  Errors: SPHBUF_ERR_INVALID_ARG (skin
 * outside [0, 1] h, max_steps < 1, rotating buffers or dual-criteria stepping; later steps
 * with SPHBUF_PHASE_BUFFER_KERNEL or SPHBUF_PHASE_FULL_CHECK are refused too),
 * SPHBUF_ERR_STATE (after the first step). */
sphbuf_status sphbuf_set_list_reuse(sphbuf_domain_t d, double skin_over_h, int max_steps);
/* Boundary identification of the transport velocity (the TVF of Eq. (10) advects the inner
 * fluid; Sec. 2.2 identifies about three layers of boundary particles with a cited
 * spatio-temporal method; this library's reading): a particle is a candidate when its
 * position divergence -sum_j V_j r_ij . grad_i W_ij (V_j = dp^d, fluid and wall neighbours)
 * is below 0.75 d, core when it was a candidate in the previous physics step too (or has no
 * previous step), and a boundary particle when it is core or a fluid neighbour within 2h is
 * core; the transport velocity moves only label-0 particles that are not boundary particles.
 * Writes, for the live particles in the order of sphbuf_read_particles, the flags of the last
 * step with the transport velocity: bit 0 candidate, bit 1 set once identified, bit 2 core,
 * bit 3 boundary particle (all 0 before such a step).  Synchronises. */
sphbuf_status sphbuf_read_boundary_flags(sphbuf_domain_t d, uint8_t *flags, uint64_t cap, uint64_t *n_out);
/* Full neighbour-list builds so far (with lists rebuilt every step: one per rebuild). */
sphbuf_status sphbuf_read_list_builds(sphbuf_domain_t d, uint64_t *builds);

/* Runs nsteps full steps (SPHBUF_STEP_DEFAULT), asynchronously on the domain's stream. */
sphbuf_status sphbuf_step(sphbuf_domain_t d, int nsteps);
/* Runs nsteps steps of the given phases (SPHBUF_PHASE_* mask). */
sphbuf_status sphbuf_step_phases(sphbuf_domain_t d, int nsteps, unsigned phases);

/* Captures the launches of one step (for a phase mask) into a CUDA graph and replays it
 * for later steps with that mask.  enable = 0 returns to plain launches. */
sphbuf_status sphbuf_use_graph(sphbuf_domain_t d, int enable);

/* Waits for the domain's stream and returns any latched device-side error. */
sphbuf_status sphbuf_sync(sphbuf_domain_t d);

/* Number of fluid particles after the last step (synchronises). */
sphbuf_status sphbuf_count(sphbuf_domain_t d, uint64_t *n);

/* Grid description. */
sphbuf_status sphbuf_grid_info(sphbuf_domain_t d, int32_t dims[3], double *cs, uint64_t *ncell);

/* Copies the sorted particle state to host arrays of capacity cap (synchronises).  Any
 * pointer may be NULL.  Order: by (cell, id).  frac / vel are gathered into n x dim rows on
 * the device and copied once each. */
sphbuf_status sphbuf_read_particles(sphbuf_domain_t d, int32_t *cell, float *frac, float *vel,
                                    float *rho, uint32_t *id, uint8_t *label, uint64_t cap,
                                    uint64_t *n_out);
/* FP64 global positions lo + c cs + f (n x dim), same order (synchronises). */
sphbuf_status sphbuf_read_positions(sphbuf_domain_t d, double *pos, uint64_t cap, uint64_t *n_out);
/* cell_start[ncell + 1] of the current cell-linked list (synchronises). */
sphbuf_status sphbuf_read_cell_start(sphbuf_domain_t d, uint32_t *cell_start, uint64_t cap);

/* Per-buffer counters since creation (synchronises): injected / deleted particle counts, the
 * corresponding masses (count x rho0 dp^dim) and the volume flux through the buffer at the
 * last step, Q_k = sum over its particles of (v . u) dp^dim / a (m^3/s in 3-D). */
sphbuf_status sphbuf_read_counters(sphbuf_domain_t d, int buffer_id, uint64_t *injected,
                                   uint64_t *deleted, double *mass_in, double *mass_out,
                                   double *flux_q);
/* Domain-wide counters (synchronises): escaped particles, completed steps, next new id. */
sphbuf_status sphbuf_read_global(sphbuf_domain_t d, uint64_t *escaped, uint64_t *steps,
                                 uint32_t *next_id);

/* Decisions of the last step (synchronises): injections sorted by (buffer, parent id) with
 * their new ids, and deletions (unordered).  Arrays of capacity cap; NULL allowed. */
sphbuf_status sphbuf_last_decisions(sphbuf_domain_t d, uint32_t *inj_buffer, uint32_t *inj_parent,
                                    uint32_t *inj_new, uint64_t *n_inj, uint32_t *del_buffer,
                                    uint32_t *del_id, uint64_t *n_del, uint64_t cap);

/* Phase timing: when enabled, every step records CUDA events around its phases on the
 * domain's stream (plain launches, no graph); sphbuf_read_phase_times returns the accumulated
 * milliseconds per phase [neighbour lists, density, force (or kinematic drift), buffer update
 * (decisions + apply), rebuild + relabel] and resets them (synchronises). */
sphbuf_status sphbuf_enable_phase_timing(sphbuf_domain_t d, int enable);
sphbuf_status sphbuf_read_phase_times(sphbuf_domain_t d, double ms[5], uint64_t *steps);

/* Candidate set of buffer k for the current cell-linked list (synchronises): the number of
 * cells the decision visits and the particles listed in them (Sec. 3.1's local cells). */
sphbuf_status sphbuf_candidate_count(sphbuf_domain_t d, int buffer_id, uint64_t *cells,
                                     uint64_t *particles);

/* Number of kernel launches this domain has issued (graph replays count every kernel
 * node of the graph). */
sphbuf_status sphbuf_read_launch_count(sphbuf_domain_t d, uint64_t *launches);

/* Stand-alone counting-sort cell-linked list (the rebuild of step 5) on DEVICE arrays:
 * cell[n] (linear cell index in [0, ncell)), id[n], optional label[n] (entries equal to 255
 * are skipped; NULL = none skipped).  Writes cell_start[ncell + 1] (exclusive prefix sum of
 * the per-cell counts) and order[n_kept]: order[p] = input index of the particle in sorted
 * slot p, sorted by (cell, id).  Ids within one cell must be distinct; at most 1024 particles
 * may share one cell (a particle is ranked inside its cell by comparing it with every other
 * particle of the cell).  Scratch memory is allocated and freed on the stream
 * (cudaMallocAsync).  Returns INVALID_ARG for a cell index outside [0, ncell) or a cell with
 * more than 1024 particles (checked on the device, reported at the end of the call, which
 * synchronises the stream; order[] is then incomplete). */
sphbuf_status sphbuf_cell_list_build(const int32_t *cell, const uint32_t *id, const uint8_t *label,
                                     uint64_t n, uint64_t ncell, uint32_t *cell_start,
                                     uint32_t *order, void *cuda_stream);

/* ---------------------------------------------------------------- batched domains
 * Many independent domains (same dim, same device) stepped together: every kernel of the
 * step is launched once for all domains, its blocks split among the domains in proportion
 * to their work (particles, candidate cells, scan tiles).  Results are identical to stepping
 * each domain alone.  The batch enqueues on its own stream (cuda_stream, or a private one if
 * NULL) after the domains' pending work, and each domain's stream waits for the batch's
 * steps, so sphbuf_read_* on a domain after sphbuf_batch_step sees the new state.  Domains
 * must not be stepped on their own while they belong to a batch; a domain's particles are
 * committed (Algorithm 1 identification, first cell list) when the batch is created.  The
 * batch does not own the domains: destroy the batch before its domains. */
typedef struct sphbuf_batch *sphbuf_batch_t;

sphbuf_status sphbuf_batch_create(sphbuf_domain_t *domains, int n, void *cuda_stream,
                                  sphbuf_batch_t *out);
/* nsteps steps with the given phase mask (see sphbuf_step_phases) for every domain. */
sphbuf_status sphbuf_batch_step(sphbuf_batch_t b, int nsteps, unsigned phases);
/* Capture one batched step into a CUDA graph and replay it (enable = 1), or plain launches. */
sphbuf_status sphbuf_batch_use_graph(sphbuf_batch_t b, int enable);
/* Launch configuration of a batch's kernels (the autotuner's choice).  For each kernel of
 * sphbuf_kernel: threads per block (a multiple of 32 in 32..512) and blocks per SM (1..32;
 * the kernel's grid is blocks_per_sm x SMs blocks, shared out over the domains in
 * proportion to their particles, or to their candidate cells for the buffer kernel);
 * cells_per_warp: candidate cells one warp of the buffer kernel visits at a time (its cell
 * tile: 1, 2, 4 or 8, with 32 / cells_per_warp lanes per cell).  The scans of the cell-list
 * rebuild (tiles of 4096 cells) and the single-block kernels are not configurable.  A
 * configuration changes launch shapes only, never results. */
typedef enum {
  SPHBUF_KERNEL_NEIGHBOURS = 0,  /* neighbour lists + Eq. (9) */
  SPHBUF_KERNEL_DENSITY = 1,     /* deferred densities (Eq. (4), overflowed lists) */
  SPHBUF_KERNEL_FORCE = 2,       /* force, kick, BC velocity, drift (+ fused decisions) */
  SPHBUF_KERNEL_DRIFT = 3,       /* kinematic drift (+ fused decisions) */
  SPHBUF_KERNEL_VISCOUS = 4,     /* dual-criteria scheme: viscous acceleration */
  SPHBUF_KERNEL_ACOUSTIC = 5,    /* dual-criteria scheme: acoustic step */
  SPHBUF_KERNEL_DUAL_FINISH = 6, /* dual-criteria scheme: fold + store (+ fused decisions) */
  SPHBUF_KERNEL_BUFFER = 7,      /* decisions in a kernel of their own (candidate cells) */
  SPHBUF_KERNEL_BUFFER_FULL = 8, /* decisions over all particles */
  SPHBUF_KERNEL_HIST = 9,        /* rebuild: histogram */
  SPHBUF_KERNEL_KEYS = 10,       /* rebuild: keys */
  SPHBUF_KERNEL_SCATTER = 11,    /* rebuild: scatter + relabel */
  SPHBUF_KERNEL_COUNT = 12
} sphbuf_kernel;

typedef struct {
  int threads[SPHBUF_KERNEL_COUNT];
  int blocks_per_sm[SPHBUF_KERNEL_COUNT];
  int cells_per_warp;
} sphbuf_batch_config;

/* Autotuner: runs trial_steps real steps (the domains advance) with the given phase mask for
 * every pair (threads in {64, 128, 256, 512}) x (blocks per SM in {1, 2, 4, 8, 16}), timing
 * every kernel launch with CUDA events, and gives each kernel the pair under which it ran
 * fastest; then, when the phases launch the buffer kernel, the cell tile in {1, 2, 4, 8}.
 * *best_m receives the neighbour kernel's blocks per SM (may be NULL); ms_per_step (may be
 * NULL) the per-phase milliseconds of trial_steps steps with the chosen configuration.
 * Read the choice with sphbuf_batch_get_config (e.g. to cache it per workload size). */
sphbuf_status sphbuf_batch_autotune(sphbuf_batch_t b, int trial_steps, unsigned phases, int *best_m,
                                    double ms_per_step[5]);
sphbuf_status sphbuf_batch_get_config(sphbuf_batch_t b, sphbuf_batch_config *cfg);
/* Applies a configuration (e.g. a cached autotuner result) without trial steps; synchronises
 * the batch's stream.  SPHBUF_ERR_INVALID_ARG for a value outside the ranges above. */
sphbuf_status sphbuf_batch_set_config(sphbuf_batch_t b, const sphbuf_batch_config *cfg);
/* Sets the blocks per SM of every configurable kernel to m (1..32) without trial steps,
 * block sizes unchanged; the domains do not advance.  SPHBUF_ERR_INVALID_ARG outside 1..32. */
sphbuf_status sphbuf_batch_set_grid(sphbuf_batch_t b, int m);
/* Persistent form of the batch's default step (SPHBUF_STEP_DEFAULT): every phase (neighbour
 * lists, densities, force with the fused decisions, the cell-list rebuild) in one cooperative
 * launch whose blocks all stay resident, with a grid-wide barrier between phases, instead
 * of one launch per phase (other phase masks keep the per-phase launches; results are
 * identical either way).  Each barrier wait spins at most spin_limit iterations of about
 * 100 ns (< 0: the default, 2^24); a wait that runs out makes every block of the launch
 * return and latches SPHBUF_ERR_TIMEOUT in every domain of the batch, reported by the next
 * synchronising call (the domains then need new particles written to step again).
 * SPHBUF_ERR_INVALID_ARG for a batch with rotating buffers or dual-criteria stepping. */
sphbuf_status sphbuf_batch_set_persistent(sphbuf_batch_t b, int enable, long long spin_limit);
/* Waits for the batch's stream and returns the first latched error of its domains. */
sphbuf_status sphbuf_batch_sync(sphbuf_batch_t b);
sphbuf_status sphbuf_batch_destroy(sphbuf_batch_t b);

/* The same cell-linked list as sphbuf_cell_list_build, for callers that must not allocate
 * device memory: for example a host program whose GPU memory is already fully reserved by
 * another allocator, or a latency-bound loop in which cudaMalloc / cudaFree (which can
 * synchronise the device) are not acceptable.  This call performs no cudaMalloc, cudaFree or
 * other allocating call; its scratch lives in a fixed array inside the library (about 16 MiB).
 * A GPU holds that array from the library's first use on it (when the library's device code
 * is loaded there, which may be lazy) until the process exits: a caller that hands all the
 * remaining device memory to another allocator should make one call (or any other library
 * call that launches work) on that device first.  The paper has no counterpart of this entry
 * point.
 *   Limits: n <= 1048576 particles and ncell <= 1048575 cells; larger sizes return
 *   SPHBUF_ERR_CAPACITY without doing any work.
 *   Inputs, outputs and errors as for sphbuf_cell_list_build (the call synchronises the stream).
 *   Every call looks up the array's address on the device current at the call (no
 *   allocation); the first call on a device may load the library's device code there, so
 *   make that first call before any stream capture.
 *   All calls share the one array and it keeps the last call's contents (each call clears the
 *   parts that must start at zero): calls whose work overlaps on the GPU, from several streams
 *   or threads, race and give wrong results; serialise them. */
sphbuf_status sphbuf_cell_list_build_noalloc(const int32_t *cell, const uint32_t *id,
                                             const uint8_t *label, uint64_t n, uint64_t ncell,
                                             uint32_t *cell_start, uint32_t *order,
                                             void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* SPHBUF_H */
