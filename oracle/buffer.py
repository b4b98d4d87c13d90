"""The arbitrary-positioned buffer (Sec. 3, Algorithms 1-3) and the full step, in FP64.

Every particle is tested against every buffer at every step: the restriction of the
candidates to the local cell-linked lists (Sec. 3.1) is an acceleration that must not
change the result, so the oracle uses the plain definition.

Labels: 0 = ordinary fluid, k + 1 = particle of buffer k.

Per-step order (the paper fixes only a partial order: generation/deletion during the step,
cell-list rebuild at the end, relabelling after the rebuild):
  1 density   (Eq. (9) for non-buffer fluid, Eq. (4) for buffer particles)
  2 force     (Eq. (5); Eq. (18) for buffer particles)
  3 integrate (kick; velocity BC Eqs. (23)-(26) or pressure-BC projection Eq. (19); drift)
  4 decide    (Algorithms 1-3 on the new positions)
  5 apply     (duplicate + recycle Eqs. (16)-(17), density Eq. (22); delete)
  6 rebuild   (cell-linked list: sort by (cell, id))
  7 relabel   (outflow and bidirectional buffers, Algorithms 2-3)

Readings where the paper is silent:
* Outflow candidates (Sec. 3.1 "about one layer of cells" around the box): a particle is a
  candidate of outflow buffer k when |X'| < a/2 + cs, |Y'| < b/2 + cs (|Z'| < c/2 + cs),
  cs = 2h the cell size; it is deleted when also X' > a/2.
* Ties: all inequalities are strict, as printed; X' = a/2 neither injects nor deletes.
* Order of new particles: injections are taken in (buffer, parent id) order; duplicate number
  r of a step gets id next_id + r, the parent's state and label 0.
* Recycling moves the parent by -a u (u = R^T e_x), which is Eqs. (16)-(17) applied to
  X' - [a, 0, 0]^T.  Pressure buffers then set rho = rho0 + p_b / c0^2 (Eq. (22)); velocity
  buffers keep rho (Sec. 4.2).
* p_b(t) = p_b + p_amp sin(p_omega t + p_phase), evaluated once per step at t_n = n dt.
* Velocity profile, Eqs. (23)-(24): v_X' = U (1 - (Y'^2 + Z'^2)/R^2), clipped at 0, or U
  everywhere when R = 0 (plug); Y' only in 2-D.
* Particles leaving the grid box are removed and counted as escaped.
"""
from __future__ import annotations

import math
from typing import List

import numpy as np

from . import frames, moving, sph

VELOCITY_INLET, PRESSURE_OUTLET, PRESSURE_INLET, VELOCITY_OUTLET, BIDIR_PRESSURE, BIDIR_VELOCITY = range(6)
INFLOW = (VELOCITY_INLET, PRESSURE_INLET)
OUTFLOW = (PRESSURE_OUTLET, VELOCITY_OUTLET)
BIDIR = (BIDIR_PRESSURE, BIDIR_VELOCITY)
VELOCITY_BC = (VELOCITY_INLET, VELOCITY_OUTLET, BIDIR_VELOCITY)
PRESSURE_BC = (PRESSURE_OUTLET, PRESSURE_INLET, BIDIR_PRESSURE)


class Buffer:
    """FP64 description of buffer k (any object with BufferSpec attributes)."""

    def __init__(self, k: int, spec, dim: int):
        self.k = k
        self.label = k + 1
        self.dim = dim
        self.origin = np.asarray(spec.origin, dtype=np.float64)[:3]
        R = np.asarray(spec.rotation, dtype=np.float64).reshape(3, 3)
        self.R3 = R
        self.R = R[:dim, :dim]
        self.extent = np.asarray(spec.extent, dtype=np.float64)
        self.bc = int(spec.bc)
        self.umax = float(spec.umax)
        self.half_width = float(spec.half_width)
        self.p_b0 = float(spec.p_b)
        self.p_amp = float(getattr(spec, "p_amp", 0.0))
        self.p_omega = float(getattr(spec, "p_omega", 0.0))
        self.p_phase = float(getattr(spec, "p_phase", 0.0))
        self.u = frames.normal(self.R)
        pivot = getattr(spec, "pivot", None)
        self.pivot = None if pivot is None else np.asarray(pivot, dtype=np.float64)[:3]
        axis = getattr(spec, "axis", None)
        self.axis = (0.0, 0.0, 1.0) if axis is None else np.asarray(axis, dtype=np.float64)[:3]
        self.omega = float(getattr(spec, "omega", 0.0))
        if self.pivot is not None and self.bc not in INFLOW:
            raise ValueError("only inflow buffers may have a time-varying frame")
        # RCR Windkessel (Eq. (31)): p_b from the flux instead of p_b(t); see windkessel_step
        wk_c = getattr(spec, "wk_c", None)
        self.wk = wk_c is not None
        if self.wk and self.bc not in PRESSURE_BC:
            raise ValueError("a Windkessel drives a pressure buffer")
        self.wk_rp = float(getattr(spec, "wk_rp", 0.0))
        self.wk_c = float(wk_c) if self.wk else 0.0
        self.wk_rd = float(getattr(spec, "wk_rd", 0.0))
        self.wk_pd = float(getattr(spec, "wk_pd0", 0.0))
        self.pb_now = self.wk_pd  # p_b of the current step (Windkessel buffers)

    def windkessel_step(self, q_prev: float, dt: float, first: bool):
        """Eq. (31) as P = P_d + R_p Q, C dP_d/dt = Q - P_d / R_d (the same RCR model), one
        explicit Euler step with the flux of the previous step (reading):
        P_d <- P_d + dt ((Q - P_d / R_d) / C) (not at the first step); p_b = P_d + R_p Q."""
        if not first:
            self.wk_pd = self.wk_pd + dt * ((q_prev - self.wk_pd / self.wk_rd) / self.wk_c)
        self.pb_now = self.wk_pd + self.wk_rp * q_prev

    def set_frame(self, R3, origin):
        """Re-establish the local frame (Sec. 5.3): new rotation and origin."""
        self.R3 = np.asarray(R3, dtype=np.float64)
        self.R = self.R3[:self.dim, :self.dim]
        self.origin = np.asarray(origin, dtype=np.float64)[:3]
        self.u = frames.normal(self.R)

    def p_b(self, t: float) -> float:
        if self.wk:
            return self.pb_now
        return self.p_b0 + self.p_amp * math.sin(self.p_omega * t + self.p_phase)

    def flux(self, vel, label, dp: float) -> float:
        """Volume flux through the buffer: sum over its particles of (v . u) dp^d / a."""
        m = label == self.label
        return float(np.sum(vel[m] @ self.u) * dp ** self.dim / self.extent[0])

    def local(self, pos: np.ndarray) -> np.ndarray:
        return frames.to_local(self.R, self.origin, pos)

    def profile(self, Xp: np.ndarray) -> np.ndarray:
        """Eqs. (23)-(24) scaled by U (reading above)."""
        if self.half_width <= 0.0:
            return np.full(Xp.shape[0], self.umax)
        rr = Xp[:, 1] ** 2
        if self.dim == 3:
            rr = rr + Xp[:, 2] ** 2
        return self.umax * np.clip(1.0 - rr / self.half_width ** 2, 0.0, None)


def decide(buffers: List[Buffer], pos, label, cs: float):
    """Algorithms 1-3 (generation and deletion) for all particles and all buffers.

    Returns (inj, dels): lists of (k, particle index).
    """
    inj, dels = [], []
    for b in buffers:
        Xp = b.local(pos)
        ha = 0.5 * b.extent[0]
        if b.bc in INFLOW:
            idx = np.nonzero((label == b.label) & (Xp[:, 0] > ha))[0]
            inj += [(b.k, int(i)) for i in idx]
        elif b.bc in OUTFLOW:
            cand = (np.abs(Xp[:, 0]) < ha + cs) & (np.abs(Xp[:, 1]) < 0.5 * b.extent[1] + cs)
            if b.dim == 3:
                cand &= np.abs(Xp[:, 2]) < 0.5 * b.extent[2] + cs
            idx = np.nonzero(cand & (Xp[:, 0] > ha))[0]
            dels += [(b.k, int(i)) for i in idx]
        else:
            mine = label == b.label
            inj += [(b.k, int(i)) for i in np.nonzero(mine & (Xp[:, 0] > ha))[0]]
            dels += [(b.k, int(i)) for i in np.nonzero(mine & (Xp[:, 0] < -ha))[0]]
    return inj, dels


def identify_inflow(buffers: List[Buffer], pos, label):
    """Algorithm 1 identification (once, over all fluid): in-box particles join buffer k."""
    for b in buffers:
        if b.bc in INFLOW:
            label[frames.in_box(b.local(pos), b.extent, b.dim)] = b.label
    return label


def relabel(buffers: List[Buffer], pos, label):
    """Algorithms 2-3 identification after the rebuild (outflow and bidirectional buffers)."""
    for b in buffers:
        if b.bc in OUTFLOW or b.bc in BIDIR:
            inside = frames.in_box(b.local(pos), b.extent, b.dim)
            label[(~inside) & (label == b.label)] = 0
            label[inside] = b.label
    return label


def cell_coords(pos, lo, cs, dims, dim):
    c = np.zeros((pos.shape[0], 3), dtype=np.int64)
    for a in range(dim):
        c[:, a] = np.floor((pos[:, a] - lo[a]) / cs).astype(np.int64)
    return c


def linear_cell(c, dims):
    nx, ny, _ = dims
    return (c[:, 2] * ny + c[:, 1]) * nx + c[:, 0]


def in_grid(c, dims, dim):
    ok = np.ones(c.shape[0], dtype=bool)
    for a in range(dim):
        ok &= (c[:, a] >= 0) & (c[:, a] < dims[a])
    return ok


def sort_cells(lin, ids, ncell):
    """Cell-linked list: permutation sorting by (cell, id) and cell_start[ncell + 1]."""
    order = np.lexsort((ids, lin))
    counts = np.bincount(lin, minlength=ncell)
    cell_start = np.zeros(ncell + 1, dtype=np.int64)
    np.cumsum(counts, out=cell_start[1:])
    return order, cell_start


class OracleSim:
    """Full FP64 step of the WCSPH + buffer method; state kept sorted by (cell, id)."""

    def __init__(self, case, pos=None, vel=None, rho=None, ids=None, labels=None, next_id=None,
                 step_index=0):
        self.dim = int(case.dim)
        self.P = sph.make_params(case.dim, case.dp, case.h_over_dp, case.rho0, case.c0, case.nu, case.dt,
                                 getattr(case, "p_bg", 0.0), getattr(case, "tvf_lambda", 0.0))
        self.vmax = 0.0  # largest particle speed after the last force pass (Eq. (10)'s v_max)
        self.lo = np.asarray(case.lo, dtype=np.float64)
        self.hi = np.asarray(case.hi, dtype=np.float64)
        self.cs = 2.0 * (float(case.h_over_dp) * float(case.dp))
        d = self.dim
        self.dims = [int(math.ceil((self.hi[a] - self.lo[a]) / self.cs)) for a in range(3)]
        if d == 2:
            self.dims[2] = 1
        self.ncell = self.dims[0] * self.dims[1] * self.dims[2]
        self.pos = np.array(case.fluid_pos if pos is None else pos, dtype=np.float64)[:, :d].copy()
        self.vel = np.array(case.fluid_vel if vel is None else vel, dtype=np.float64)[:, :d].copy()
        self.rho = np.array(case.fluid_rho if rho is None else rho, dtype=np.float64).copy()
        n = self.pos.shape[0]
        self.id = np.arange(n, dtype=np.int64) if ids is None else np.asarray(ids, dtype=np.int64).copy()
        self.label = np.zeros(n, dtype=np.int64) if labels is None else np.asarray(labels, dtype=np.int64).copy()
        self.labels_given = labels is not None
        self.next_id = int(n if next_id is None else next_id)
        self.wall = np.array(case.wall_pos, dtype=np.float64)[:, :d].copy()
        self.buffers = [Buffer(k, s, d) for k, s in enumerate(case.buffers)]
        self.step_index = int(step_index)
        # time-varying frames (Sec. 5.3): the frame of step n is the n-th of the recurrence
        self.moving = {b.k: moving.MovingFrame(d, b.R3, b.origin, b.pivot, b.axis, b.omega, self.P.dt)
                       for b in self.buffers if b.pivot is not None}
        for k, mf in self.moving.items():
            for _ in range(self.step_index):
                mf.advance()
            self.buffers[k].set_frame(*mf.frame())
        K = len(self.buffers)
        self.flux = np.zeros(K)  # volume flux of the last step per buffer (0 before the first)
        self.dp = float(case.dp)
        self.injected = np.zeros(K, dtype=np.int64)
        self.deleted = np.zeros(K, dtype=np.int64)
        self.escaped = 0
        self.last_inj = []  # (k, parent_id, new_id)
        self.last_del = []  # (k, id)
        self.cell_start = None
        self.n0 = n
        # boundary identification of the transport velocity (reading A27): the previous step's
        # candidate flag per particle (-1: none yet) and the last boundary flags
        self.cand_prev = np.full(n, -1, dtype=np.int64)
        self.boundary = np.zeros(n, dtype=bool)

    # ------------------------------------------------------------------ helpers
    @property
    def n(self):
        return self.pos.shape[0]

    @property
    def t(self):
        return self.step_index * self.P.dt

    def _take(self, idx):
        self.pos = self.pos[idx]
        self.vel = self.vel[idx]
        self.rho = self.rho[idx]
        self.id = self.id[idx]
        self.label = self.label[idx]
        self.cand_prev = self.cand_prev[idx]
        self.boundary = self.boundary[idx]

    def rebuild(self):
        c = cell_coords(self.pos, self.lo, self.cs, self.dims, self.dim)
        ok = in_grid(c, self.dims, self.dim)
        self.escaped += int((~ok).sum())
        self._take(np.nonzero(ok)[0])
        c = c[ok]
        lin = linear_cell(c, self.dims)
        order, self.cell_start = sort_cells(lin, self.id, self.ncell)
        self._take(order)
        self.cell = lin[order]

    def commit(self):
        """Set-up: Algorithm 1 identification (unless labels were given), rebuild, relabel."""
        if not self.labels_given:
            identify_inflow(self.buffers, self.pos, self.label)
        self.rebuild()
        relabel(self.buffers, self.pos, self.label)

    def p_bc(self, rho_new):
        """Boundary pressure per particle for Eq. (18): p_b(t) or p_i (velocity BC); NaN if none."""
        out = np.full(self.n, np.nan)
        p = sph.eos(rho_new, self.P)
        for b in self.buffers:
            m = self.label == b.label
            if b.bc in PRESSURE_BC:
                out[m] = b.p_b(self.t)
            else:
                out[m] = p[m]
        return out

    # ------------------------------------------------------------------ phases
    def physics(self):
        """Steps 1-3: density, force, kick + boundary velocity, drift (FP64)."""
        P = self.P
        ff, fw = sph.neighbor_pairs(self.pos, self.wall, P.h)
        is_buf = self.label != 0
        rho_sum = sph.density_summation(P, self.n, ff, fw)
        drho = sph.continuity_rate(P, self.vel, self.rho, ff, fw)
        rho_new = np.where(is_buf, self.rho + P.dt * drho, rho_sum)
        acc = sph.acceleration(P, self.vel, rho_new, self.p_bc(rho_new), ff, fw)
        v = self.vel + acc * P.dt
        for b in self.buffers:
            m = self.label == b.label
            if not np.any(m):
                continue
            if b.bc in VELOCITY_BC:
                prof = b.profile(b.local(self.pos[m]))
                v[m] = prof[:, None] * b.u[None, :]
            else:
                un = v[m] @ b.u
                v[m] = un[:, None] * b.u[None, :]
        for b in self.buffers:
            self.flux[b.k] = b.flux(v, self.label, self.dp)
        self.acc = acc
        adv = v
        if P.tvf_lambda > 0.0:
            # Eq. (10): advect the inner fluid with the transport velocity
            # v - dt p_max sum_j 2 m/(rho_i rho_j) dW/dr e_ij, p_max = lambda rho0 v_max^2 with
            # v_max of the previous step; the buffer particles and the identified boundary
            # particles (reading A27, from the step's start positions) keep v
            psi = sph.position_divergence(P, self.n, ff, fw)
            cand, _, self.boundary = sph.boundary_layers(P, psi, self.cand_prev, ff)
            self.cand_prev = cand.astype(np.int64)
            p_max = P.tvf_lambda * P.rho0 * self.vmax * self.vmax
            shift = P.dt * p_max * sph.transport_sum(P, rho_new, ff, fw)
            inner = (self.label == 0) & ~self.boundary
            adv = np.where(inner[:, None], v - shift, v)
        self.vmax = float(np.linalg.norm(v, axis=1).max()) if v.shape[0] else 0.0
        self.vel = v
        self.pos = self.pos + adv * P.dt
        self.rho = rho_new

    def dual_physics(self, n_ac: int):
        """Dual-criteria time stepping (Sec. 2.2, the cited dual-criteria scheme; reading A26):
        one advection step of dt = P.dt made of n_ac acoustic steps of dt / n_ac.

        At the advection step the configuration (the neighbour pairs) is fixed and the
        density of the fluid particles is re-initialised by Eq. (9) (buffer particles keep
        theirs); the viscous acceleration is evaluated once.  Each acoustic step then takes,
        from the current state with the pairs' distances recomputed: the continuity rate of
        Eq. (4) for every particle and the pressure part of Eq. (5) with Eq. (18); v += dt_ac
        (a_p + a_v), the boundary velocity of the buffer particles (Eqs. (19), (23)-(26), from
        the acoustic step's start position), rho += dt_ac drho/dt, r += dt_ac v.  The flux of
        a buffer is the mean over the acoustic steps."""
        P = self.P
        ff, fw = sph.neighbor_pairs(self.pos, self.wall, P.h)
        is_buf = self.label != 0
        rho = np.where(is_buf, self.rho, sph.density_summation(P, self.n, ff, fw))
        nan = np.full(self.n, np.nan)
        a_v = sph.acceleration(P, self.vel, rho, nan, ff, fw, pressure=False)
        dt = P.dt / n_ac
        v, pos = self.vel.copy(), self.pos.copy()
        flux = np.zeros(len(self.buffers))
        for _ in range(n_ac):
            ffs, fws = sph.moved(ff, pos, pos), sph.moved(fw, pos, self.wall)
            drho = sph.continuity_rate(P, v, rho, ffs, fws)
            a_p = sph.acceleration(P, v, rho, self.p_bc(rho), ffs, fws, viscous=False)
            vn = v + dt * (a_p + a_v)
            for b in self.buffers:
                m = self.label == b.label
                if not np.any(m):
                    continue
                if b.bc in VELOCITY_BC:
                    prof = b.profile(b.local(pos[m]))
                    vn[m] = prof[:, None] * b.u[None, :]
                else:
                    un = vn[m] @ b.u
                    vn[m] = un[:, None] * b.u[None, :]
            for b in self.buffers:
                flux[b.k] += b.flux(vn, self.label, self.dp) / n_ac
            rho = rho + dt * drho
            pos = pos + dt * vn
            v = vn
        self.flux[:] = flux
        self.vel, self.pos, self.rho = v, pos, rho

    def kinematic(self):
        """Drift only with the current velocity (used by the lockstep tests)."""
        self.pos = self.pos + self.vel * self.P.dt

    def buffer_update(self):
        """Steps 4-5: decisions (Algorithms 1-3) and their application."""
        inj, dels = decide(self.buffers, self.pos, self.label, self.cs)
        t = self.t
        inj.sort(key=lambda kv: (kv[0], int(self.id[kv[1]])))
        new_pos, new_vel, new_rho, new_id = [], [], [], []
        self.last_inj = []
        for r, (k, i) in enumerate(inj):
            b = self.buffers[k]
            nid = self.next_id + r
            new_pos.append(self.pos[i].copy())
            new_vel.append(self.vel[i].copy())
            new_rho.append(self.rho[i])
            new_id.append(nid)
            self.last_inj.append((k, int(self.id[i]), nid))
            self.pos[i] = self.pos[i] - b.extent[0] * b.u
            if b.bc in PRESSURE_BC:
                self.rho[i] = self.P.rho0 + (b.p_b(t) - self.P.p_bg) / (self.P.c0 * self.P.c0)
            self.injected[k] += 1
        self.next_id += len(inj)
        self.last_del = [(k, int(self.id[i])) for k, i in dels]
        for k, _ in dels:
            self.deleted[k] += 1
        keep = np.ones(self.n, dtype=bool)
        keep[[i for _, i in dels]] = False
        self._take(np.nonzero(keep)[0])
        if new_pos:
            self.pos = np.concatenate([self.pos, np.array(new_pos)])
            self.vel = np.concatenate([self.vel, np.array(new_vel)])
            self.rho = np.concatenate([self.rho, np.array(new_rho)])
            self.id = np.concatenate([self.id, np.array(new_id, dtype=np.int64)])
            self.label = np.concatenate([self.label, np.zeros(len(new_pos), dtype=np.int64)])
            self.cand_prev = np.concatenate([self.cand_prev, np.full(len(new_pos), -1, dtype=np.int64)])
            self.boundary = np.concatenate([self.boundary, np.zeros(len(new_pos), dtype=bool)])
        # Sec. 5.3: after the generation, the particles of a rotating buffer turn with it
        for k, mf in self.moving.items():
            m = self.label == self.buffers[k].label
            if m.any():
                self.pos[m], self.vel[m] = moving.rotate64(self.pos[m], self.vel[m], mf.C, mf.M, self.dim)

    def advance_frames(self):
        """Re-establish the rotating buffers' frames for the next step (Sec. 5.3)."""
        for k, mf in self.moving.items():
            mf.advance()
            self.buffers[k].set_frame(*mf.frame())

    def drop_escaped(self):
        c = cell_coords(self.pos, self.lo, self.cs, self.dims, self.dim)
        ok = in_grid(c, self.dims, self.dim)
        if not ok.all():
            self.escaped += int((~ok).sum())
            self._take(np.nonzero(ok)[0])

    def begin_step(self):
        """Boundary pressures of the step: Windkessel buffers from the last step's flux."""
        for b in self.buffers:
            if b.wk:
                b.windkessel_step(float(self.flux[b.k]), self.P.dt, self.step_index == 0)
        self.flux[:] = 0.0

    def step(self, nsteps=1, physics=True, buffer=True, dual=0):
        for _ in range(nsteps):
            self.begin_step()
            if physics and dual:
                self.dual_physics(dual)
            elif physics:
                self.physics()
            else:
                self.kinematic()
            self.drop_escaped()
            if buffer:
                self.buffer_update()
            else:
                self.last_inj, self.last_del = [], []
            self.rebuild()
            relabel(self.buffers, self.pos, self.label)
            self.advance_frames()
            self.step_index += 1
