"""The largest buffer count (32): a 2-D channel carrying 32 buffers of all six types along its
length, kinematic steps bit-exact against the FP32-mode oracle; a 33rd buffer is refused
with SPHBUF_ERR_CAPACITY."""
import numpy as np
import pytest

from oracle import fp32 as OF
from paper_2406_16786_gb300 import _ffi
from paper_2406_16786_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
KIN = _ffi.PHASE_KINEMATIC | _ffi.PHASE_BUFFER
TYPES = [wl.VELOCITY_INLET, wl.PRESSURE_OUTLET, wl.PRESSURE_INLET, wl.VELOCITY_OUTLET, wl.BIDIR_PRESSURE,
         wl.BIDIR_VELOCITY]


def _case():
    dp, a, pitch = 0.01, 0.04, 0.15
    c = wl.straight_channel_case(length=32 * pitch + 0.1, width=0.2, dp=dp, angle_deg=17.0, umax=1.0,
                                 profile="parabolic", c0=10.0, nu=1e-2, seed=71, init_velocity="bc")
    frame = c.buffers[0].rotation
    e_s = frame[0]
    start = c.buffers[0].origin - 0.5 * a * e_s
    bufs = []
    for q in range(32):
        bc = TYPES[q % 6]
        # outflow boxes face along the flow, inflow and bidirectional ones too (into the channel)
        bufs.append(wl.BufferSpec(origin=start + (0.05 + q * pitch) * e_s, rotation=frame.copy(),
                                  extent=np.array([a, 0.2, 0.0]), bc=bc, umax=1.0, half_width=0.1, p_b=0.5 * q))
    c.buffers = bufs
    c.fluid_vel = 8.0 * e_s[None, :2] + wl.shear_velocity(c, u0=6.0, seed=72)
    return c


def _bits(a):
    return np.ascontiguousarray(a, dtype=np.float32).view(np.int32)


def test_thirty_two_buffers_bit_exact():
    from paper_2406_16786_gb300.domain import Domain, SphbufError

    c = _case()
    cell, frac = wl.encode_positions(c.fluid_pos, c.lo, c.cs, c.grid_dims())
    vel = c.fluid_vel.astype(np.float32)
    rho = c.fluid_rho.astype(np.float32)
    dom = Domain.from_case(c)
    assert dom.nbuf == 32
    extra = wl.BufferSpec(origin=c.buffers[-1].origin + 0.15 * c.buffers[0].rotation[0],
                          rotation=c.buffers[0].rotation, extent=np.array([0.04, 0.2, 0.0]), bc=wl.PRESSURE_OUTLET)
    with pytest.raises(SphbufError) as e:
        dom.add_buffer(extra)
    assert e.value.status == 2
    dom.use_graph(True)
    sim = OF.Fp32Sim(c, cell, frac, vel, rho)
    sim.commit()
    per_buffer = np.zeros(32, np.int64)
    for _ in range(6):
        dom.step(1, KIN)
        sim.step(1)
        inj, dels = dom.last_decisions()
        assert inj == sim.last_inj
        assert sorted(dels) == sorted(sim.last_del)
        for k, _, _ in inj:
            per_buffer[k] += 1
        for k, _ in dels:
            per_buffer[k] += 1
        g = dom.read()
        assert np.array_equal(g["id"].astype(np.int64), sim.id)
        assert np.array_equal(g["cell"].astype(np.int64), sim.cell)
        assert np.array_equal(_bits(g["frac"]), _bits(sim.f))
        assert np.array_equal(g["label"].astype(np.int64), sim.label)
    assert (per_buffer > 0).sum() >= 24  # most buffers decided something
    dom.close()
