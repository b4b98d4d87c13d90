"""3-D pressure-driven pipe flow through two bidirectional pressure buffers (the Sec. 6.1
set-up at steady pressure): pipe R = 0.5 mm, L = 4 mm at -45 deg, eta = 3.536e-4 Pa s,
dp = d/20, c0 = 0.1 m/s, a 0.1 Pa pressure difference, driven once forward (inlet high) and
once in reverse (outlet high), so that each buffer both generates and deletes.  After 6000
steps (about five viscous times R^2/nu) the mid-pipe velocity profile matches the Poiseuille
profile v = dP (R^2 - r^2) / (4 eta L), the limit of Eq. (29) at small alpha: centre speed
within 4 %, RMSEP (Eq. (28), lanes r <= R - dp) within 8 %, and the two directions mirror
each other."""
import math

import numpy as np
import pytest

from oracle import analytic
from paper_2406_16786_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

R, L, D = 5e-4, 4e-3, 1e-3
RHO, ETA = 1000.0, 3.536e-4
E = np.array([1.0, -1.0, 0.0]) / math.sqrt(2.0)


def _profile(dom, dp, nl):
    st = dom.read()
    pos = dom.positions()
    s = pos @ E
    r = np.linalg.norm(pos - s[:, None] * E[None, :], axis=1)
    mid = (s > L / 3) & (s < 2 * L / 3)
    va = st["vel"].astype(np.float64) @ E
    edges = np.linspace(0.0, R, nl + 1)
    return np.array([va[mid & (r >= edges[q]) & (r < edges[q + 1])].mean() for q in range(nl)])


def _run(p_in, p_out):
    from paper_2406_16786_gb300.domain import Domain

    dp = D / 20
    c = wl.pipe_case(name="pipe_poiseuille", length=L, radius=R, dp=dp, axis=(1.0, -1.0, 0.0),
                     inlet_bc=wl.BIDIR_PRESSURE, outlet_bc=wl.BIDIR_PRESSURE, p_in=p_in, p_amp=0.0, p_omega=0.0,
                     p_out=p_out, c0=0.1, nu=ETA / RHO, rho0=RHO, umax_est=0.0044, seed=61)
    dom = Domain.from_case(c)
    dom.use_graph(True)
    n0 = dom.count()
    dom.step(6000)
    nl = 10
    prof = _profile(dom, dp, nl)
    n1 = dom.count()
    dom.close()
    rc = (np.arange(nl) + 0.5) * (R / nl)
    exact = (p_in - p_out) * (R * R - rc * rc) / (4 * ETA * L)
    return prof, exact, rc, dp, n0, n1


def test_pressure_driven_pipe_both_directions():
    fwd, exact, rc, dp, n0, n1 = _run(0.1, 0.0)
    rev, exact_r, _, _, m0, m1 = _run(0.0, 0.1)
    keep = rc <= R - dp
    for prof, ex in ((fwd, exact), (rev, exact_r)):
        assert abs(prof[0] - ex[0]) < 0.04 * abs(ex[0])
        assert analytic.rmsep(ex[keep], prof[keep]) < 0.08
    # the buffers swap roles: the reverse run mirrors the forward one
    assert np.abs(fwd + rev).max() < 0.02 * np.abs(exact).max()
    # particle count held within 1 % (generation balances deletion)
    assert abs(n1 - n0) < 0.01 * n0 and abs(m1 - m0) < 0.01 * m0
