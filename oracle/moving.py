"""Time-varying buffer frames (Sec. 5.3, the rotating sprinkler).  Test infrastructure.

The paper turns an inflow buffer with a constant angular velocity omega: after the particle
generation of a step has been done in the current local frame, the positions and velocities
of the buffer's particles are rotated, and the local frame is re-established at the new
position of the buffer for the next step's generation.  With the angle theta = omega t +
theta_0 this is, per step of length dt, one rotation by omega dt about the pivot C (about
the z axis in 2-D, about a unit axis n in 3-D).

Frame of step n (Q_0 = I, M = rotation by omega dt):
  Q_n = M Q_{n-1},   R_n = R_0 Q_n^T,   O'_n = C + Q_n (O'_0 - C),
so X'_n = R_n (X - O'_n) = R_0 (Q_n^T (X - C) - (O'_0 - C)): a particle turned with the buffer
keeps its local coordinates.

FP64 arithmetic is written out in a fixed order, every product and sum rounded on its own
(a CUDA implementation reproduces it bit for bit with __dmul_rn / __dadd_rn), so that the
FP32 decision constants derived from the frame are the same on both sides:
  M, 3-D (n = a / |a|, |a| = sqrt((a0 a0 + a1 a1) + a2 a2), s = sin(omega dt),
          c = cos(omega dt), t = 1 - c):
     M_00 = (t n0) n0 + c          M_01 = (t n0) n1 - s n2      M_02 = (t n0) n2 + s n1
     M_10 = (t n0) n1 + s n2       M_11 = (t n1) n1 + c         M_12 = (t n1) n2 - s n0
     M_20 = (t n0) n2 - s n1       M_21 = (t n1) n2 + s n0      M_22 = (t n2) n2 + c
  M, 2-D = [[c, -s, 0], [s, c, 0], [0, 0, 1]]
  (A B)_rc = (A_r0 B_0c + A_r1 B_1c) + A_r2 B_2c;   (R_0 Q^T)_rc = (R0_r0 Q_c0 + R0_r1 Q_c1) + R0_r2 Q_c2
  O'_x = C_x + ((Q_x0 d_0 + Q_x1 d_1) + Q_x2 d_2),  d = O'_0 - C
FP32 rotation of a particle (the contract of fp32.py; pivot encoded like a buffer origin:
cC = floor((C - lo) / cs), fC = fl((C - lo) - cC cs)):
  D_x = fl(fl(fl(c_x - cC_x) cs32) + fl(f_x - fC_x))
  D'_r = fl(fl(fl(M32_r0 D_0) + fl(M32_r1 D_1)) + fl(M32_r2 D_2))   (2-D: the first two terms)
  the particle moves by fl(D'_x - D_x) (fp32.move32); v'_r = same rows applied to v.
"""
from __future__ import annotations

import math

import numpy as np

F32 = np.float32


def step_rotation(dim: int, axis, omega: float, dt: float):
    """M, the rotation by omega dt (3x3 nested lists of Python floats)."""
    phi = omega * dt
    s, c = math.sin(phi), math.cos(phi)
    if dim == 2:
        return [[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]]
    a = [float(v) for v in axis]
    nn = math.sqrt((a[0] * a[0] + a[1] * a[1]) + a[2] * a[2])
    if not nn > 0.0:
        raise ValueError("rotation axis must be non-zero")
    n0, n1, n2 = a[0] / nn, a[1] / nn, a[2] / nn
    t = 1.0 - c
    return [[(t * n0) * n0 + c, (t * n0) * n1 - s * n2, (t * n0) * n2 + s * n1],
            [(t * n0) * n1 + s * n2, (t * n1) * n1 + c, (t * n1) * n2 - s * n0],
            [(t * n0) * n2 - s * n1, (t * n1) * n2 + s * n0, (t * n2) * n2 + c]]


def matmul3(A, B):
    return [[(A[r][0] * B[0][c] + A[r][1] * B[1][c]) + A[r][2] * B[2][c] for c in range(3)] for r in range(3)]


class MovingFrame:
    """The frame recurrence of one rotating buffer (FP64, module header order)."""

    def __init__(self, dim, R0, O0, pivot, axis, omega, dt):
        self.dim = int(dim)
        self.R0 = [[float(R0[r][c]) for c in range(3)] for r in range(3)]
        self.O0 = [float(O0[x]) for x in range(3)]
        self.C = [float(pivot[x]) for x in range(3)]
        if self.dim == 2:
            self.O0[2] = 0.0
            self.C[2] = 0.0
        self.M = step_rotation(self.dim, axis if axis is not None else (0.0, 0.0, 1.0), omega, dt)
        self.Q = [[1.0 if r == c else 0.0 for c in range(3)] for r in range(3)]
        self.steps = 0

    def advance(self):
        self.Q = matmul3(self.M, self.Q)
        self.steps += 1

    def frame(self):
        """(R_n as a 3x3 array, O'_n as a 3-vector) of the current step."""
        Q, R0 = self.Q, self.R0
        R = [[(R0[r][0] * Q[c][0] + R0[r][1] * Q[c][1]) + R0[r][2] * Q[c][2] for c in range(3)] for r in range(3)]
        d = [self.O0[x] - self.C[x] for x in range(3)]
        O = [self.C[x] + ((Q[x][0] * d[0] + Q[x][1] * d[1]) + Q[x][2] * d[2]) for x in range(3)]
        return np.array(R, dtype=np.float64), np.array(O, dtype=np.float64)


def rotate64(pos, vel, pivot, M, dim):
    """FP64 rotation of positions about the pivot and of velocities (rows = particles)."""
    Md = np.asarray(M, dtype=np.float64)[:dim, :dim]
    C = np.asarray(pivot, dtype=np.float64)[:dim]
    return C + (pos - C) @ Md.T, vel @ Md.T


def encode_point(g, p):
    """(cC, fC) of a point, the buffer-origin encoding of fp32.py."""
    cC = np.zeros(3, dtype=np.int64)
    fC = np.zeros(3, dtype=F32)
    for x in range(g.dim):
        t = float(p[x]) - float(g.lo[x])
        c = math.floor(t / g.cs)
        cC[x] = c
        fC[x] = F32(t - c * g.cs)
    return cC, fC


def rotate32(g, c, f, v, cC, fC, M32):
    """FP32 rotation of particles (c, f, v: rows = particles), in place."""
    from .fp32 import move32

    d = g.dim
    D = np.empty((c.shape[0], d), dtype=F32)
    for x in range(d):
        D[:, x] = ((c[:, x] - cC[x]).astype(F32) * g.cs32) + (f[:, x] - fC[x])
    Dn = np.empty_like(D)
    vn = np.empty_like(v)
    for r in range(d):
        acc = M32[r][0] * D[:, 0]
        vac = M32[r][0] * v[:, 0]
        for x in range(1, d):
            acc = acc + M32[r][x] * D[:, x]
            vac = vac + M32[r][x] * v[:, x]
        Dn[:, r] = acc
        vn[:, r] = vac
    move32(g, c, f, (Dn - D).astype(F32))
    v[:, :] = vn
