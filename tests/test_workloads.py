"""The seeded synthetic inputs have the recipe the design states: lattice spacing dp with a
uniform +-0.01 dp jitter, three wall layers (at least the 2h support), buffer depth a = 4 dp
(Sec. 3), the stated particle counts, and identical arrays for identical seeds."""
import math

import numpy as np

from paper_2406_16786_gb300 import workloads as wl


def _lattice_residual(x, dp):
    """Distance of each coordinate from the nearest lattice site (k + 1/2) dp, in units of dp."""
    q = x / dp - 0.5
    return np.abs(q - np.round(q))


def test_config1_channel_recipe():
    c = wl.config1()
    assert c.dim == 2 and c.dp == 0.025
    assert c.fluid_pos.shape == (400 * 40, 2)  # 10 m x 1 m at dp 0.025
    res = _lattice_residual(c.fluid_pos, c.dp)
    assert res.max() <= 0.01 + 1e-9
    assert 0.004 < res.mean() < 0.006  # uniform on [0, 0.01]: mean 0.005
    # walls: three layers above and below the channel, thicker than the support 2h = 2.6 dp
    y = c.wall_pos[:, 1]
    assert np.all(np.abs(y) > 0.5)
    layers = np.unique(np.round((np.abs(y) - 0.5) / c.dp - 0.5).astype(int))
    assert list(layers) == [0, 1, 2] and 3 * c.dp >= 2 * c.h_over_dp * c.dp
    assert _lattice_residual(c.wall_pos, c.dp).max() < 1e-9  # walls are not jittered
    # two buffers of depth a = 4 dp spanning the width: velocity inlet, pressure outlet
    assert [b.bc for b in c.buffers] == [wl.VELOCITY_INLET, wl.PRESSURE_OUTLET]
    for b in c.buffers:
        assert math.isclose(b.extent[0], 4 * c.dp) and math.isclose(b.extent[1], 1.0)
    # the same seed gives the same arrays
    d = wl.config1()
    assert np.array_equal(c.fluid_pos, d.fluid_pos) and np.array_equal(c.fluid_vel, d.fluid_vel)


def test_config3_pipe_recipe_and_bench_size():
    c = wl.config3(length=0.5)
    assert c.dim == 3 and c.dp == 0.01
    n = c.fluid_pos.shape[0]
    per_layer = n // 50
    assert n == 50 * per_layer
    # lattice points inside a disc of radius 0.5 m: pi R^2 / dp^2 to a fraction of a percent
    assert abs(per_layer / (math.pi * 0.25 / 1e-4) - 1) < 0.005
    # the bench pipe (L = 5.09 m) therefore holds about 4.0 M fluid particles
    assert abs(509 * per_layer - 4.0e6) < 0.01e6
    # both buffers are bidirectional pressure buffers of depth 4 dp whose frames map the
    # inflow normal onto e_x; the pipe axis is (1,1,1)/sqrt3
    axis = np.ones(3) / math.sqrt(3.0)
    assert [b.bc for b in c.buffers] == [wl.BIDIR_PRESSURE, wl.BIDIR_PRESSURE]
    signs = []
    for b in c.buffers:
        assert math.isclose(b.extent[0], 4 * c.dp)
        R = b.rotation
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-12) and math.isclose(np.linalg.det(R), 1.0)
        signs.append(float(R[0] @ axis))
    assert np.allclose(sorted(signs), [-1.0, 1.0])  # inlet along +axis, outlet's inflow along -axis
    # the fluid starts on the developed profile: 0.06 m/s on the axis, along the axis
    speed = np.linalg.norm(c.fluid_vel, axis=1)
    assert 0.055 < speed.max() <= 0.06 + 1e-12
    along = c.fluid_vel @ axis
    assert np.allclose(along, speed)


def test_config5_batched_star_channels():
    cases = wl.config5()
    assert len(cases) == 64
    ns = np.array([c.fluid_pos.shape[0] for c in cases])
    # sizes drawn log-uniform in [10 k, 500 k]; the lattice fill lands within ~10 % of the draw
    assert ns.min() > 0.85 * 10_000 and ns.max() < 1.15 * 500_000
    assert abs(ns.sum() / 6.93e6 - 1) < 0.01
    assert all(c.dim == 2 for c in cases)
    arms = [len(c.buffers) for c in cases]
    assert min(arms) == 1 and max(arms) == 6
    for c in cases:
        if len(c.buffers) == 1:
            assert c.buffers[0].bc == wl.BIDIR_PRESSURE  # a dead-end arm with an oscillating buffer
        else:
            assert c.buffers[0].bc == wl.VELOCITY_INLET
            assert all(b.bc == wl.PRESSURE_OUTLET for b in c.buffers[1:])
        for b in c.buffers:
            assert math.isclose(b.extent[0], 4 * c.dp)


def test_config4_tjunction_recipe_at_a_coarser_spacing():
    # the same geometry at dp = 0.02 (0.4 M particles) scales to the 15.4 M of dp = 0.006
    c = wl.tjunction_case(dp=0.02)
    n = c.fluid_pos.shape[0]
    assert abs(n * (0.02 / 0.006) ** 3 / 15.4e6 - 1) < 0.015
    assert [b.bc for b in c.buffers] == [wl.VELOCITY_INLET, wl.PRESSURE_OUTLET, wl.PRESSURE_OUTLET]
    normals = [b.rotation[0] for b in c.buffers]
    angles = [math.degrees(math.acos(np.clip(normals[0] @ u, -1.0, 1.0))) for u in normals]
    assert np.allclose(angles, [0.0, 0.0, 60.0], atol=1e-9)  # main outlet along the pipe, branch at 60 deg
    assert np.allclose([b.extent[1] for b in c.buffers], [1.0, 1.0, 0.6])  # main R 0.5, branch R 0.3
    for b in c.buffers:
        assert math.isclose(b.extent[0], 4 * c.dp)


def test_config2_bent_channel_recipe():
    c = wl.config2()
    assert c.dim == 2 and c.dp == 0.005
    assert abs(c.fluid_pos.shape[0] / 0.38e6 - 1) < 0.01
    inlet, outlet = c.buffers
    assert (inlet.bc, outlet.bc) == (wl.VELOCITY_INLET, wl.PRESSURE_OUTLET)
    deg = [math.degrees(math.atan2(b.rotation[0][1], b.rotation[0][0])) for b in c.buffers]
    assert np.allclose(deg, [30.0, -15.0], atol=1e-9)
    assert (inlet.umax, inlet.half_width) == (1.5, 0.5)  # parabolic profile over the 1 m width
    assert math.isclose(inlet.extent[0], 4 * c.dp) and math.isclose(outlet.extent[0], 4 * c.dp)
