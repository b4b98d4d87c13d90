"""Background pressure of the EoS (reading A22): one full GPU step against the FP64 oracle
with p = c0^2 (rho - rho0) + p_bg, on a 3-D pipe with two bidirectional pressure buffers whose
absolute pressures carry p_bg, and on the 2-D bent channel's physics set-up."""
import dataclasses
import math

import pytest

from paper_2406_16786_gb300 import workloads as wl
from tests import sampled

pytestmark = pytest.mark.gpu


def test_background_pressure_one_step_pipe():
    pbg = 200.0
    c = wl.pipe_case(length=0.5, radius=0.08, dp=0.01, axis=(1.0, -0.4, 0.3), inlet_bc=wl.BIDIR_PRESSURE,
                     outlet_bc=wl.BIDIR_PRESSURE, p_in=pbg, p_amp=50.0, p_omega=math.pi, p_out=pbg, c0=3.0,
                     seed=71, umax=0.05, init_velocity="profile")
    c.p_bg = pbg
    assert sampled.physics_step_sampled(c, sample_size=800) > 500


def test_background_pressure_one_step_channel():
    c = wl.bent_channel_case(dp=0.02)
    c.p_bg = 500.0
    c.buffers[1] = dataclasses.replace(c.buffers[1], p_b=500.0)
    assert sampled.physics_step_sampled(c, sample_size=800) > 500
