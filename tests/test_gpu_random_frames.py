"""Bit-exact buffer decisions over randomly drawn frames and buffer types.

Twelve seeded cases: 2-D channels at uniformly drawn angles and 3-D pipes along uniformly
drawn axes with drawn rolls, each with an inlet and an outlet of drawn types (all six), a
drawn width and a velocity field that crosses both faces of both buffers.  Six kinematic
steps (drift, Algorithms 1-3, rebuild, relabel) per case, GPU against the FP32-mode oracle:
injection list, deletion set, sorted state and cell_start identical.
"""
import numpy as np
import pytest

from oracle import fp32 as OF
from paper_2406_16786_gb300 import _ffi
from paper_2406_16786_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
KIN = _ffi.PHASE_KINEMATIC | _ffi.PHASE_BUFFER
INLETS = [wl.VELOCITY_INLET, wl.PRESSURE_INLET, wl.BIDIR_PRESSURE, wl.BIDIR_VELOCITY]
OUTLETS = [wl.PRESSURE_OUTLET, wl.VELOCITY_OUTLET, wl.BIDIR_PRESSURE, wl.BIDIR_VELOCITY]


def _bits(a):
    return np.ascontiguousarray(a, dtype=np.float32).view(np.int32)


def _case(seed):
    rng = np.random.default_rng(9000 + seed)
    ib, ob = int(rng.choice(INLETS)), int(rng.choice(OUTLETS))
    if seed % 2 == 0:
        c = wl.straight_channel_case(length=float(rng.uniform(0.5, 1.0)), width=float(rng.uniform(0.15, 0.35)),
                                     dp=0.01, angle_deg=float(rng.uniform(0.0, 360.0)), inlet_bc=ib, outlet_bc=ob,
                                     umax=1.0, profile="parabolic", p_in=2.0, p_out=0.0, c0=10.0, nu=1e-2,
                                     seed=500 + seed, init_velocity="bc")
    else:
        ax = rng.standard_normal(3)
        c = wl.pipe_case(length=float(rng.uniform(0.3, 0.5)), radius=float(rng.uniform(0.05, 0.08)), dp=0.01,
                         axis=tuple(ax / np.linalg.norm(ax)), roll=float(rng.uniform(0.0, 2.0 * np.pi)),
                         inlet_bc=ib, outlet_bc=ob, p_in=2.0, p_amp=1.0, p_omega=2.0, umax=1.0, c0=3.0,
                         seed=500 + seed, init_velocity="profile")
    # along the axis (one way or the other, per seed) plus a shear: both faces see crossings
    e = c.buffers[0].rotation[0, : c.dim]
    sgn = 1.0 if rng.uniform() < 0.7 else -1.0
    c.fluid_vel = sgn * 6.0 * e[None, :] + wl.shear_velocity(c, u0=10.0, seed=seed)
    return c


@pytest.mark.parametrize("seed", range(12))
def test_random_frames_bit_exact(seed):
    from paper_2406_16786_gb300.domain import Domain

    c = _case(seed)
    cell, frac = wl.encode_positions(c.fluid_pos, c.lo, c.cs, c.grid_dims())
    vel = c.fluid_vel.astype(np.float32)
    rho = c.fluid_rho.astype(np.float32)
    dom = Domain.from_case(c)
    dom.use_graph(True)
    sim = OF.Fp32Sim(c, cell, frac, vel, rho)
    sim.commit()
    total = 0
    for _ in range(6):
        dom.step(1, KIN)
        sim.step(1)
        inj, dels = dom.last_decisions()
        assert inj == sim.last_inj
        assert sorted(dels) == sorted(sim.last_del)
        total += len(inj) + len(dels)
        g = dom.read()
        assert np.array_equal(g["id"].astype(np.int64), sim.id)
        assert np.array_equal(g["cell"].astype(np.int64), sim.cell)
        assert np.array_equal(_bits(g["frac"]), _bits(sim.f))
        assert np.array_equal(g["label"].astype(np.int64), sim.label)
        assert np.array_equal(dom.cell_start().astype(np.int64), sim.cell_start)
    assert total > 0
    dom.close()
