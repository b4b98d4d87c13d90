"""FP32 decision mode: Algorithms 1-3 on the cell-relative FP32 state, bit-for-bit defined.

The FP64 decisions of ``buffer`` and an FP32 implementation can disagree for a particle
within rounding distance of a threshold.  So that a decision can be compared exactly, both
sides take it in FP32 from the same stored state with the operation order below; every
product and sum is rounded to FP32 on its own (no fused multiply-add).  fl() = round to
nearest FP32.

State per particle: integer cell coordinates c (grid anchored at lo, cell size cs = 2h)
and an in-cell offset f in [0, cs32), FP32.

Constants of buffer k, from FP64 inputs (origin O, frame R, extent a, b, c):
  cO_x = floor((O_x - lo_x) / cs);  fO_x = fl((O_x - lo_x) - cO_x cs)
  R32 = fl(R) (upper-left d x d block);   ha, hb, hc = fl(a/2), fl(b/2), fl(c/2)
  da, db, dc = fl(a/2 + cs), fl(b/2 + cs), fl(c/2 + cs)   (candidate region, reading in
  ``buffer``);  s_x = fl(-a R[0][x])   (recycling shift -a u, Eqs. (16)-(17))
Local coordinates (Eqs. (11)/(15)):
  D_x = fl( fl( fl(c_x - cO_x) * cs32 ) + fl(f_x - fO_x) )
  X'_r = fl( fl( fl(R32[r][0] D_0) + fl(R32[r][1] D_1) ) + fl(R32[r][2] D_2) )  (2-D: 2 terms)
Move by Delta (drift fl(v dt32), or recycling s):  f <- fl(f + Delta), then repeat at most 8
  times: if f >= cs32 { f <- fl(f - cs32); c += 1 } else if f < 0 { f <- fl(f + cs32); c -= 1 }
  else stop.
"""
from __future__ import annotations

import math
from typing import List

import numpy as np

from . import buffer as B
from . import moving as MV

F32 = np.float32


class Grid32:
    def __init__(self, dim, lo, hi, dp, h_over_dp):
        self.dim = int(dim)
        self.lo = np.asarray(lo, dtype=np.float64)
        self.cs = 2.0 * (float(h_over_dp) * float(dp))
        self.cs32 = F32(self.cs)
        hi = np.asarray(hi, dtype=np.float64)
        self.dims = [int(math.ceil((hi[a] - self.lo[a]) / self.cs)) for a in range(3)]
        if self.dim == 2:
            self.dims[2] = 1
        self.ncell = self.dims[0] * self.dims[1] * self.dims[2]

    def coords(self, cell):
        nx, ny, _ = self.dims
        cell = np.asarray(cell, dtype=np.int64)
        return np.stack([cell % nx, (cell // nx) % ny, cell // (nx * ny)], axis=1)

    def linear(self, c):
        nx, ny, _ = self.dims
        return (c[:, 2] * ny + c[:, 1]) * nx + c[:, 0]

    def in_grid(self, c):
        ok = np.ones(c.shape[0], dtype=bool)
        for a in range(self.dim):
            ok &= (c[:, a] >= 0) & (c[:, a] < self.dims[a])
        return ok


class Buffer32:
    def __init__(self, b: B.Buffer, g: Grid32):
        d = g.dim
        self.b = b
        self.k = b.k
        self.label = b.label
        self.bc = b.bc
        self.cO = np.zeros(3, dtype=np.int64)
        self.fO = np.zeros(3, dtype=F32)
        for x in range(d):
            t = b.origin[x] - g.lo[x]
            c = math.floor(t / g.cs)
            self.cO[x] = c
            self.fO[x] = F32(t - c * g.cs)
        self.R32 = b.R3[:d, :d].astype(F32)
        a, bb, cc = (float(v) for v in b.extent[:3])
        self.ha, self.hb, self.hc = F32(0.5 * a), F32(0.5 * bb), F32(0.5 * cc)
        self.da, self.db, self.dc = F32(0.5 * a + g.cs), F32(0.5 * bb + g.cs), F32(0.5 * cc + g.cs)
        self.shift = np.array([F32(-a * b.R3[0][x]) for x in range(d)], dtype=F32)


def local32(g: Grid32, b32: Buffer32, c, f):
    """X', Y' (, Z') in FP32 with the operation order of the module header."""
    d = g.dim
    D = np.empty((c.shape[0], d), dtype=F32)
    for x in range(d):
        cx = (c[:, x] - b32.cO[x]).astype(F32)
        D[:, x] = (cx * g.cs32) + (f[:, x] - b32.fO[x])
    out = np.empty_like(D)
    R = b32.R32
    for r in range(d):
        acc = R[r, 0] * D[:, 0]
        for x in range(1, d):
            acc = acc + R[r, x] * D[:, x]
        out[:, r] = acc
    return out


def move32(g: Grid32, c, f, delta):
    """f <- fl(f + delta), then fold back into [0, cs32) (module header).  In place."""
    d = g.dim
    for x in range(d):
        fx = (f[:, x] + delta[:, x]).astype(F32)
        cx = c[:, x].copy()
        for _ in range(8):
            up = fx >= g.cs32
            dn = fx < F32(0)
            if not (up.any() or dn.any()):
                break
            fx[up] = fx[up] - g.cs32
            cx[up] += 1
            fx[dn] = fx[dn] + g.cs32
            cx[dn] -= 1
        f[:, x] = fx
        c[:, x] = cx


def in_box32(X, b32: Buffer32, dim):
    m = (np.abs(X[:, 0]) < b32.ha) & (np.abs(X[:, 1]) < b32.hb)
    if dim == 3:
        m &= np.abs(X[:, 2]) < b32.hc
    return m


def decide32(g: Grid32, bufs: List[Buffer32], c, f, label):
    inj, dels = [], []
    for b in bufs:
        X = local32(g, b, c, f)
        if b.bc in B.INFLOW:
            inj += [(b.k, int(i)) for i in np.nonzero((label == b.label) & (X[:, 0] > b.ha))[0]]
        elif b.bc in B.OUTFLOW:
            cand = (np.abs(X[:, 0]) < b.da) & (np.abs(X[:, 1]) < b.db)
            if g.dim == 3:
                cand &= np.abs(X[:, 2]) < b.dc
            dels += [(b.k, int(i)) for i in np.nonzero(cand & (X[:, 0] > b.ha))[0]]
        else:
            mine = label == b.label
            inj += [(b.k, int(i)) for i in np.nonzero(mine & (X[:, 0] > b.ha))[0]]
            dels += [(b.k, int(i)) for i in np.nonzero(mine & (X[:, 0] < -b.ha))[0]]
    return inj, dels


class Fp32Sim:
    """Kinematic (drift-only) steps with the buffer update, entirely in FP32 mode.

    State arrays: cell (linear, int64), frac (n, d) FP32, vel (n, d) FP32, rho FP32,
    id int64, label int64; kept sorted by (cell, id) after each rebuild.
    """

    def __init__(self, case, cell, frac, vel, rho, ids=None, labels=None, next_id=None, step_index=0):
        self.g = Grid32(case.dim, case.lo, case.hi, case.dp, case.h_over_dp)
        d = self.g.dim
        self.dt = float(case.dt)
        self.dt32 = F32(case.dt)
        self.rho0 = float(case.rho0)
        self.c0 = float(case.c0)
        self.p_bg = float(getattr(case, "p_bg", 0.0))
        self.c = self.g.coords(cell)
        self.f = np.array(frac, dtype=F32)[:, :d].copy()
        self.vel = np.array(vel, dtype=F32)[:, :d].copy()
        self.rho = np.array(rho, dtype=F32).copy()
        n = self.f.shape[0]
        self.id = np.arange(n, dtype=np.int64) if ids is None else np.asarray(ids, dtype=np.int64).copy()
        self.label = np.zeros(n, dtype=np.int64) if labels is None else np.asarray(labels, dtype=np.int64).copy()
        self.labels_given = labels is not None
        self.next_id = int(n if next_id is None else next_id)
        self.bufs64 = [B.Buffer(k, s, d) for k, s in enumerate(case.buffers)]
        self.step_index = int(step_index)
        # time-varying frames (Sec. 5.3; oracle/moving.py): FP64 recurrence, FP32 rotation
        self.moving = {b.k: MV.MovingFrame(d, b.R3, b.origin, b.pivot, b.axis, b.omega, self.dt)
                       for b in self.bufs64 if b.pivot is not None}
        self.pivot32 = {k: MV.encode_point(self.g, mf.C) for k, mf in self.moving.items()}
        self.M32 = {k: np.array(mf.M, dtype=F32) for k, mf in self.moving.items()}
        for k, mf in self.moving.items():
            for _ in range(self.step_index):
                mf.advance()
            self.bufs64[k].set_frame(*mf.frame())
        self.bufs = [Buffer32(b, self.g) for b in self.bufs64]
        K = len(self.bufs)
        self.injected = np.zeros(K, dtype=np.int64)
        self.deleted = np.zeros(K, dtype=np.int64)
        self.escaped = 0
        self.last_inj, self.last_del = [], []
        self.n0 = n

    @property
    def n(self):
        return self.f.shape[0]

    @property
    def cell(self):
        return self.g.linear(self.c)

    def _take(self, idx):
        for name in ("c", "f", "vel", "rho", "id", "label"):
            setattr(self, name, getattr(self, name)[idx])

    def rebuild(self):
        ok = self.g.in_grid(self.c)
        self.escaped += int((~ok).sum())
        self._take(np.nonzero(ok)[0])
        lin = self.g.linear(self.c)
        order, self.cell_start = B.sort_cells(lin, self.id, self.g.ncell)
        self._take(order)

    def identify(self):
        for b in self.bufs:
            if b.bc in B.INFLOW:
                self.label[in_box32(local32(self.g, b, self.c, self.f), b, self.g.dim)] = b.label

    def relabel(self):
        for b in self.bufs:
            if b.bc in B.OUTFLOW or b.bc in B.BIDIR:
                inside = in_box32(local32(self.g, b, self.c, self.f), b, self.g.dim)
                self.label[(~inside) & (self.label == b.label)] = 0
                self.label[inside] = b.label

    def commit(self):
        if not self.labels_given:
            self.identify()
        self.rebuild()
        self.relabel()

    def drift(self):
        delta = (self.vel * self.dt32).astype(F32)
        move32(self.g, self.c, self.f, delta)
        ok = self.g.in_grid(self.c)
        if not ok.all():
            self.escaped += int((~ok).sum())
            self._take(np.nonzero(ok)[0])

    def buffer_update(self):
        inj, dels = decide32(self.g, self.bufs, self.c, self.f, self.label)
        t = self.step_index * self.dt
        inj.sort(key=lambda kv: (kv[0], int(self.id[kv[1]])))
        n_new = len(inj)
        self.last_inj = []
        if n_new:
            par = np.array([i for _, i in inj], dtype=np.int64)
            ks = [k for k, _ in inj]
            nc = self.c[par].copy()
            nf = self.f[par].copy()
            nv = self.vel[par].copy()
            nr = self.rho[par].copy()
            nid = self.next_id + np.arange(n_new, dtype=np.int64)
            self.last_inj = [(k, int(self.id[i]), int(nid[r])) for r, (k, i) in enumerate(inj)]
            shifts = np.stack([self.bufs[k].shift for k in ks]).astype(F32)
            pc = self.c[par].copy()
            pf = self.f[par].copy()
            move32(self.g, pc, pf, shifts)
            self.c[par] = pc
            self.f[par] = pf
            for k, i in inj:
                b64 = self.bufs64[k]
                if b64.bc in B.PRESSURE_BC:
                    self.rho[i] = F32(self.rho0 + (b64.p_b(t) - self.p_bg) / (self.c0 * self.c0))
                self.injected[k] += 1
            self.next_id += n_new
        self.last_del = [(k, int(self.id[i])) for k, i in dels]
        for k, _ in dels:
            self.deleted[k] += 1
        keep = np.ones(self.n, dtype=bool)
        keep[[i for _, i in dels]] = False
        self._take(np.nonzero(keep)[0])
        if n_new:
            self.c = np.concatenate([self.c, nc])
            self.f = np.concatenate([self.f, nf])
            self.vel = np.concatenate([self.vel, nv])
            self.rho = np.concatenate([self.rho, nr])
            self.id = np.concatenate([self.id, nid])
            self.label = np.concatenate([self.label, np.zeros(n_new, dtype=np.int64)])
        # Sec. 5.3: the particles of a rotating buffer turn with it after the generation
        for k in self.moving:
            m = np.nonzero(self.label == self.bufs[k].label)[0]
            if m.size:
                cc, ff, vv = self.c[m].copy(), self.f[m].copy(), self.vel[m].copy()
                cC, fC = self.pivot32[k]
                MV.rotate32(self.g, cc, ff, vv, cC, fC, self.M32[k])
                self.c[m], self.f[m], self.vel[m] = cc, ff, vv

    def advance_frames(self):
        for k, mf in self.moving.items():
            mf.advance()
            self.bufs64[k].set_frame(*mf.frame())
            self.bufs[k] = Buffer32(self.bufs64[k], self.g)

    def step(self, nsteps=1, buffer=True):
        for _ in range(nsteps):
            # kinematic steps measure no flux: Windkessel buffers see Q = 0
            for b in self.bufs64:
                if b.wk:
                    b.windkessel_step(0.0, self.dt, self.step_index == 0)
            self.drift()
            if buffer:
                self.buffer_update()
            else:
                self.last_inj, self.last_del = [], []
            self.rebuild()
            self.relabel()
            self.advance_frames()
            self.step_index += 1
