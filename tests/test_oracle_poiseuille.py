"""Pin of the oracle's full step against the plane Poiseuille closed form (Sec. 5.1, Eq. (27)).

Sloped (30 deg) VIPO channel: parabolic velocity inlet, pressure outlet p_b = 0, no-slip walls.
Scaled to Re = 1 (d = 1 mm, U = 1 mm/s, nu = 1e-6) and d/dp = 20 so that it converges in a
few thousand steps on the CPU; c0 is raised to keep the density variation near 1 % (Sec. 2.1).
Checks: RMSEP (Eq. (28)) of the time-averaged mid-channel profile and the inlet pressure,
which must approach the Poiseuille pressure drop (the paper's VIPO expectation, Sec. 5.1).
"""
import numpy as np
import pytest

from oracle import analytic
from oracle import buffer as OB
from paper_2406_16786_gb300 import workloads as wl

D, L, U, NU, RHO0, C0 = 1e-3, 4e-3, 1e-3, 1e-6, 1000.0, 0.06


def vipo_case(dp=D / 20):
    return wl.straight_channel_case(length=L, width=D, dp=dp, angle_deg=30.0, inlet_bc=wl.VELOCITY_INLET,
                                    outlet_bc=wl.PRESSURE_OUTLET, umax=U, profile="parabolic", c0=C0, nu=NU,
                                    rho0=RHO0, init_velocity="bc")


@pytest.mark.slow
def test_vipo_converges_to_poiseuille():
    case = vipo_case()
    eta = RHO0 * NU
    dP = 8.0 * eta * L * U / D ** 2  # pressure drop that drives U at the centre line
    sim = OB.OracleSim(case)
    sim.commit()
    b0 = sim.buffers[0]
    a = b0.extent[0]
    ys = (np.arange(20) + 0.5) * case.dp - 0.5 * D
    acc_v, acc_p, nsamp = np.zeros(20), 0.0, 0
    for s in range(2200):
        sim.step(1)
        if s >= 1600 and s % 50 == 0:
            loc = b0.local(sim.pos)
            mid = np.abs(loc[:, 0] - (0.5 * L - 0.5 * a)) < 2 * case.dp
            lane = np.clip(np.round((loc[mid, 1] + 0.5 * D) / case.dp - 0.5).astype(int), 0, 19)
            vx = sim.vel[mid] @ b0.u
            acc_v += np.bincount(lane, weights=vx, minlength=20) / np.maximum(np.bincount(lane, minlength=20), 1)
            p = (sim.rho - RHO0) * C0 ** 2
            acc_p += p[sim.label == 1].mean()
            nsamp += 1
    v = acc_v / nsamp
    exact = analytic.poiseuille_plane(ys, dP, eta, L, D)
    keep = np.abs(ys) <= 0.5 * D - case.dp  # measuring points away from the walls
    err = analytic.rmsep(exact[keep], v[keep])
    assert err < 0.02, err
    # inlet buffer centre sits a/2 + a/2 upstream of the outlet buffer's span: p ~ dP (1 - a / L)
    assert acc_p / nsamp == pytest.approx(dP * (1 - a / L), rel=0.1)
    assert sim.escaped == 0
    assert sim.n == sim.n0 + sim.injected.sum() - sim.deleted.sum()


@pytest.mark.slow
def test_vipo_converges_to_poiseuille_dual_time_stepping():
    # the same channel with the dual-criteria scheme (reading A26): advection step four times
    # the single-rate step (viscous limit 0.25 h^2/nu), two acoustic steps of CFL 0.5 each
    case = vipo_case()
    case.dt = 4.0 * case.dt
    case.dual_substeps = 2
    eta = RHO0 * NU
    dP = 8.0 * eta * L * U / D ** 2
    sim = OB.OracleSim(case)
    sim.commit()
    b0 = sim.buffers[0]
    a = b0.extent[0]
    ys = (np.arange(20) + 0.5) * case.dp - 0.5 * D
    acc_v, nsamp = np.zeros(20), 0
    for s in range(550):
        sim.step(1, dual=case.dual_substeps)
        if s >= 400 and s % 12 == 0:
            loc = b0.local(sim.pos)
            mid = np.abs(loc[:, 0] - (0.5 * L - 0.5 * a)) < 2 * case.dp
            lane = np.clip(np.round((loc[mid, 1] + 0.5 * D) / case.dp - 0.5).astype(int), 0, 19)
            vx = sim.vel[mid] @ b0.u
            acc_v += np.bincount(lane, weights=vx, minlength=20) / np.maximum(np.bincount(lane, minlength=20), 1)
            nsamp += 1
    v = acc_v / nsamp
    exact = analytic.poiseuille_plane(ys, dP, eta, L, D)
    keep = np.abs(ys) <= 0.5 * D - case.dp
    assert analytic.rmsep(exact[keep], v[keep]) < 0.02
    assert sim.escaped == 0
    assert sim.n == sim.n0 + sim.injected.sum() - sim.deleted.sum()
