"""Pins of the local frames (oracle.frames): Eqs. (11)-(17), (20)-(21) and reading of Eq. (14)."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import frames


def _dirs(n, seed=3):
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((n, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def test_rotation_maps_normal_to_ex_and_is_proper():
    for d in _dirs(50):
        R = frames.rotation_3d(d)
        assert np.allclose(R @ d, [1, 0, 0], atol=1e-14)
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(R) - 1.0) < 1e-13


def test_rodrigues_is_the_shortest_arc_rotation():
    # a single aligned pair: scipy returns the minimal-angle rotation taking d to e_x,
    # which is Rodrigues' formula about n = e_x x d
    for d in _dirs(20, seed=5):
        C, _ = Rotation.align_vectors([[1.0, 0.0, 0.0]], [d])
        assert np.allclose(C.as_matrix(), frames.rotation_3d(d), atol=1e-13)


def test_printed_sign_turns_ex_onto_d():
    # documents the sign reading: I + S sin + S^2 (1 - cos) is the transpose
    d = _dirs(1, seed=9)[0]
    S = frames.skew(frames.rotation_axis(d))
    th = math.acos(d[0])
    printed = np.eye(3) + S * math.sin(th) + S @ S * (1 - math.cos(th))
    assert np.allclose(printed @ [1, 0, 0], d, atol=1e-14)
    assert np.allclose(printed.T, frames.rotation_3d(d), atol=1e-14)


@pytest.mark.parametrize("theta_deg", [-75.0, -15.0, 0.0, 30.0, 120.0, 179.0])
def test_3d_frame_reduces_to_2d_matrix(theta_deg):
    th = math.radians(theta_deg)
    d = np.array([math.cos(th), math.sin(th), 0.0])
    R = frames.rotation_3d(d)
    assert np.allclose(R[:2, :2], frames.rotation_2d(th), atol=1e-14)
    assert abs(R[2, 2] - 1.0) < 1e-14


def test_degenerate_axis():
    assert np.allclose(frames.rotation_3d([2.0, 0, 0]), np.eye(3))
    R = frames.rotation_3d([-1.0, 0, 0])
    assert np.allclose(R @ [-1.0, 0, 0], [1, 0, 0])
    assert abs(np.linalg.det(R) - 1) < 1e-14


def test_skew_is_cross_product():
    rng = np.random.default_rng(1)
    n, v = rng.standard_normal(3), rng.standard_normal(3)
    assert np.allclose(frames.skew(n) @ v, np.cross(n, v))


def test_normal_and_inverse_map():
    rng = np.random.default_rng(2)
    for d in _dirs(10, seed=4):
        R = frames.roll_about_x(frames.rotation_3d(d), rng.uniform(0, 2 * math.pi))
        assert np.allclose(frames.normal(R), d, atol=1e-14)
        O = rng.standard_normal(3)
        X = rng.standard_normal((7, 3))
        assert np.allclose(frames.to_global(R, O, frames.to_local(R, O, X)), X, atol=1e-13)
        # X' of O' + s d is (s, 0, 0)
        Xp = frames.to_local(R, O, O[None, :] + 0.7 * d[None, :])
        assert np.allclose(Xp, [[0.7, 0, 0]], atol=1e-14)
    th = 0.4
    assert np.allclose(frames.normal(frames.rotation_2d(th)), [math.cos(th), math.sin(th)])


def test_in_box_strict():
    ext = np.array([4.0, 2.0, 6.0])
    Xp = np.array([[1.999, 0.999, 2.999], [2.0, 0, 0], [0, 1.0, 0], [0, 0, -3.0], [-1.9, -0.9, 0]])
    assert list(frames.in_box(Xp, ext, 3)) == [True, False, False, False, True]
    assert list(frames.in_box(Xp[:, :2], ext, 2)) == [True, False, False, True, True]
