"""Pins of the boundary identification of the transport velocity (reading A27, oracle/sph.py).

* The kernel term of psi integrates to d over a full support (integration by parts of
  div r = d: the integral of r |dW/dr| over the support is d times the integral of W), by
  quadrature independent of any lattice.
* On a lattice, psi of an inner particle lies within 3 % of d, and a particle on a flat free
  face (half its support empty) lies between d/2 and the candidate threshold 0.75 d, while the
  next row lies above it.
* A block with a free face has exactly three identified rows at that face (the core row and
  the rows within 2h = 2.6 dp of it) and none inside.
* A block inside three layers of wall particles has no boundary particle (walls fill the
  support).
* Temporal filter: a candidate that was not a candidate in the previous step is not core; a
  particle without a previous step counts the current one.
"""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import kernel, sph

DP = 0.01


def _params(dim):
    return sph.make_params(dim, DP, 1.3, 1000.0, 10.0, 1e-3, 1e-4)


def _block(dim, m):
    ax = np.arange(m) * DP
    return np.stack(np.meshgrid(*([ax] * dim), indexing="ij"), axis=-1).reshape(-1, dim)


@pytest.mark.parametrize("dim", [2, 3])
def test_kernel_term_integrates_to_d(dim):
    h = 1.3 * DP
    shell = (lambda r: 2.0 * math.pi * r) if dim == 2 else (lambda r: 4.0 * math.pi * r * r)
    val, _ = integrate.quad(lambda r: -r * float(kernel.dW(r, h, dim)) * shell(r), 0.0, 2.0 * h, limit=200)
    assert abs(val - dim) < 1e-8


@pytest.mark.parametrize("dim", [2, 3])
def test_psi_inside_and_at_a_free_face(dim):
    P = _params(dim)
    m = 15 if dim == 2 else 9
    g = _block(dim, m)
    ff, fw = sph.neighbor_pairs(g, np.zeros((0, dim)), P.h)
    psi = sph.position_divergence(P, g.shape[0], ff, fw) / dim
    c = (m // 2) * DP
    line = np.all(np.abs(g[:, 1:] - c) < 1e-9, axis=1)
    rows = [psi[line & (np.abs(g[:, 0] - q * DP) < 1e-9)][0] for q in range(4)]
    assert abs(rows[3] - 1.0) < 0.03
    assert 0.5 < rows[0] < sph.PSI_CANDIDATE
    assert rows[1] > sph.PSI_CANDIDATE


@pytest.mark.parametrize("dim", [2, 3])
def test_three_rows_at_a_free_face(dim):
    P = _params(dim)
    m = 15 if dim == 2 else 11
    g = _block(dim, m)
    ff, fw = sph.neighbor_pairs(g, np.zeros((0, dim)), P.h)
    psi = sph.position_divergence(P, g.shape[0], ff, fw)
    cand, core, bnd = sph.boundary_layers(P, psi, None, ff)
    # depth = distance in rows to the nearest face
    depth = np.min(np.concatenate([g / DP, (m - 1) - g / DP], axis=1), axis=1).round().astype(int)
    assert np.array_equal(bnd, depth <= 2)
    assert np.array_equal(core, depth == 0)


def test_walls_fill_the_support():
    dim = 2
    P = _params(dim)
    m = 12
    g = _block(dim, m)
    ax = np.arange(-3, m + 3) * DP
    full = np.stack(np.meshgrid(ax, ax, indexing="ij"), axis=-1).reshape(-1, 2)
    inside = np.all((full >= -1e-9) & (full <= (m - 1) * DP + 1e-9), axis=1)
    walls = full[~inside]
    ff, fw = sph.neighbor_pairs(g, walls, P.h)
    psi = sph.position_divergence(P, g.shape[0], ff, fw)
    _, _, bnd = sph.boundary_layers(P, psi, None, ff)
    assert not bnd.any()
    assert np.all(psi / dim > 0.95)


def test_temporal_filter():
    dim = 2
    P = _params(dim)
    g = _block(dim, 12)
    ff, fw = sph.neighbor_pairs(g, np.zeros((0, dim)), P.h)
    psi = sph.position_divergence(P, g.shape[0], ff, fw)
    cand, core, bnd = sph.boundary_layers(P, psi, None, ff)
    assert cand.any() and np.array_equal(core, cand)
    # the previous step had no candidate: nothing is core, nothing is a boundary particle
    _, core0, bnd0 = sph.boundary_layers(P, psi, np.zeros(g.shape[0], dtype=np.int64), ff)
    assert not core0.any() and not bnd0.any()
    # no previous step for half of the particles: those count the current step
    prev = np.where(np.arange(g.shape[0]) % 2 == 0, -1, 0)
    _, core1, _ = sph.boundary_layers(P, psi, prev, ff)
    assert np.array_equal(core1, cand & (prev < 0))
