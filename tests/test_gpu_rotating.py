"""Rotating inflow buffer (Sec. 5.3, sprinkler): the GPU's kinematic steps, in graph replay,
bit-exact against the FP32-mode oracle (decisions, sorted state, cell_start), in 2-D and in
3-D about an oblique axis, with fluid at rest around the swept region; the full-domain
decision variant gives the same results.  Plus the set-up checks of the entry point."""
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
