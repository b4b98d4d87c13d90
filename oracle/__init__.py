"""CPU oracle for the arbitrary-positioned open-boundary buffer in a WCSPH step.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously-correct restatement of
"Generalized and high-efficiency arbitrary-positioned buffer for smoothed particle
hydrodynamics" (Zhang, Fan, Ren, Qian, Hu; arXiv 2406.16786).  Only the test-suite, the
smoke check and the benchmark's CPU-baseline leg may import it; the CUDA library never does,
and this package imports nothing from the CUDA path.  It takes its inputs as plain arrays
(or any object with the attributes of a case description).

Modules
-------
kernel   Wendland C2 kernel and its derivative (Sec. 3: support 2h, h = 1.3 dp).
frames   local frames: Eq. (11) 2-D rotation, Eqs. (12)-(15) 3-D Rodrigues frame, the
         inverse maps Eqs. (16)-(17) and the boundary normal Eqs. (20)-(21).
sph      the Riemann-based WCSPH step in FP64: Eqs. (3)-(9), (18), (19), (22)-(26).
buffer   Algorithms 1-3 (generation/recycling, deletion, relabelling) in FP64 on global
         positions, the cell-linked list, and the full-step driver ``OracleSim``.
fp32     the FP32 decision mode: the same decisions taken on the cell-relative FP32 state
         with a fixed operation order and no fused multiply-add, for bit-exact comparison.
analytic closed forms used as pins: plane Poiseuille Eq. (27), RMSEP Eq. (28), Womersley
         Eq. (29).

Readings where the paper is silent or inconsistent are stated where they are used and
collected in the repository's design notes.  Parity status per function:

* kernel, frames, analytic: pinned by quadrature, closed forms, library routines.
* buffer decisions (FP64 and FP32): pinned by brute-force predicates on tiny inputs,
  count invariants and the inlet injection schedule.
* sph one-step arithmetic: pinned by closed-form special cases (uniform lattice density,
  two-particle forces, rest state) and by the converged Poiseuille profile.
"""

from . import analytic, buffer, frames, fp32, kernel, sph  # noqa: F401

__all__ = ["analytic", "buffer", "frames", "fp32", "kernel", "sph"]
