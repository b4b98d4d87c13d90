"""The 2-D bent channel (inlet leg at +30 deg, bend of radius 2 m, outlet leg at -15 deg;
parabolic velocity inlet, pressure outlet) at its full size, dp = 0.005 (0.38 M particles):

* kinematic steps with every particle moving along the centre line at 0.6 dp per step, so
  that both buffers decide every step: bit-exact against the FP32-mode oracle, and the
  full-domain decision variant equal to the restricted one;
* one physics step from the paper's start (rest, inlet buffer on its profile): sampled
  particles against the FP64 oracle with the one-step tolerances.
"""
import pytest

from paper_2406_16786_gb300 import workloads as wl
from tests import sampled

pytestmark = pytest.mark.gpu


def test_bent_channel_kinematic_bit_exact_and_full_check():
    c0 = wl.config2()
    c = wl.config2(init_velocity="tangent", speed=0.6 * c0.dp / c0.dt)
    assert sampled.kinematic_bit_exact(c, c.fluid_vel, 4, full_check_too=True) > 0


def test_bent_channel_physics_step_sampled():
    assert sampled.physics_step_sampled(wl.config2()) > 1000
