"""Rotating inflow buffer (Sec. 5.3, sprinkler): the GPU's kinematic steps, in graph replay,
bit-exact against the FP32-mode oracle (decisions, sorted state, cell_start), in 2-D and in
3-D about an oblique axis, with fluid at rest around the swept region; the full-domain
decision variant gives the same results.  Sixty full steps against the FP64 oracle (same
ids and generation count; measured rho 1.4e-7, v 9e-6 / 4e-6, positions 2.4e-5 / 6.9e-6 cs
in 2-D / 3-D).  Plus the set-up checks of the entry point."""
import numpy as np
import pytest

from paper_2406_16786_gb300 import _ffi
from paper_2406_16786_gb300 import workloads as wl
from tests import sampled

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dim", [2, 3])
def test_rotating_buffer_kinematic_bit_exact(dim):
    c = wl.sprinkler_case(dim=dim, dp=0.004 if dim == 3 else 0.002, umax=1.0, omega=30.0, axis=(0.2, 0.3, 1.0),
                          ambient=True, domain_radius=0.16 if dim == 3 else 0.3)
    # 0.6 dp per step along the nozzle: a generation every other step or so
    vel = c.fluid_vel * (0.6 * c.dp / c.dt)
    assert sampled.kinematic_bit_exact(c, vel, 12, full_check_too=True) > 0


def test_rotation_entry_point_checks():
    from paper_2406_16786_gb300.domain import Domain, SphbufError

    c = wl.sprinkler_case(dim=2)
    d = Domain(c.dim, c.lo, c.hi, c.dp, c.h_over_dp, c.rho0, c.c0, c.nu, c.dt, c.capacity)
    spec = c.buffers[0]
    k = d.add_buffer(wl.BufferSpec(origin=spec.origin, rotation=spec.rotation, extent=spec.extent, bc=spec.bc,
                                   umax=spec.umax, half_width=spec.half_width))
    # an outlet may not rotate
    out = wl.BufferSpec(origin=np.array([-0.2, 0.0, 0.0]), rotation=wl.frame_2d(np.pi), extent=spec.extent,
                        bc=wl.PRESSURE_OUTLET)
    ko = d.add_buffer(out)
    with pytest.raises(SphbufError):
        d.set_buffer_rotation(ko, np.zeros(3), None, 1.0)
    # the outlet at x = -0.2 lies outside the nozzle's swept annulus (radii ~0.08-0.12 m about
    # the origin), so the nozzle may rotate; a buffer inside the annulus is then rejected
    d.set_buffer_rotation(k, np.zeros(3), None, 1.0)
    near = wl.BufferSpec(origin=np.array([0.0, 0.1, 0.0]), rotation=wl.frame_2d(0.5 * np.pi), extent=spec.extent,
                         bc=wl.PRESSURE_OUTLET)
    with pytest.raises(SphbufError):
        d.add_buffer(near)
    d.close()


@pytest.mark.parametrize("dim", [2, 3])
def test_rotating_buffer_physics_tracks_fp64_oracle(dim):
    """Full steps (density, force, the nozzle's velocity profile in its turning frame, drift,
    generation, the turn, rebuild) against the FP64 oracle: same ids and generation count,
    fields within FP32 rounding accumulated over the steps."""
    from oracle import buffer as OB
    from paper_2406_16786_gb300.domain import Domain

    c = wl.sprinkler_case(dim=dim, dp=0.004 if dim == 2 else 0.008, umax=1.0, omega=30.0, axis=(0.2, 0.3, 1.0),
                          ambient=True, domain_radius=0.2)
    cell, frac = wl.encode_positions(c.fluid_pos, c.lo, c.cs, c.grid_dims())
    vel32 = c.fluid_vel.astype(np.float32)
    rho32 = c.fluid_rho.astype(np.float32)
    dom = Domain.from_case(c)
    dom.use_graph(True)
    pos0 = wl.decode_positions(cell, frac, c.lo, c.cs, c.grid_dims())
    ora = OB.OracleSim(c, pos=pos0, vel=vel32.astype(np.float64), rho=rho32.astype(np.float64))
    ora.commit()
    steps = 60
    for _ in range(steps):
        dom.step(1)
        ora.step(1)
    g = dom.read()
    gp = dom.positions()
    assert sorted(g["id"].tolist()) == sorted(ora.id.tolist())
    assert dom.counters(0)["injected"] == int(ora.injected[0]) > 0
    o, q = np.argsort(g["id"]), np.argsort(ora.id)
    rho_g, rho_o = g["rho"][o].astype(np.float64), ora.rho[q]
    v_g, v_o = g["vel"][o].astype(np.float64), ora.vel[q]
    e_rho = np.linalg.norm(rho_g - rho_o) / np.linalg.norm(rho_o)
    e_v = np.linalg.norm(v_g - v_o) / np.linalg.norm(v_o)
    e_p = np.max(np.linalg.norm(gp[o] - ora.pos[q], axis=1)) / c.cs
    print("rotating physics dim %d: n %d inj %d rho %.2e v %.2e pos %.2e cs" % (dim, g["id"].size,
                                                                              int(ora.injected[0]), e_rho, e_v, e_p))
    assert e_rho < 1e-5 and e_v < 1e-4 and e_p < 1e-4
    dom.close()
