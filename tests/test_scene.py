"""Checks of the seeded input generator (mesh, areas, SH transfer)."""
import math

import numpy as np
import pytest

from paper_2203_12339_gb300 import scene


@pytest.mark.parametrize("nu", [1, 2, 3, 8, 16])
def test_icosphere_counts_and_closed_surface(nu):
    unit, tris = scene.icosphere_unit(nu)
    n = 10 * nu * nu + 2
    assert unit.shape == (n, 3)
    assert tris.shape == (20 * nu * nu, 3)
    # Euler characteristic of a closed genus-0 surface: V - E + F = 2
    edges = {tuple(sorted(e)) for t in tris.tolist() for e in ((t[0], t[1]), (t[1], t[2]), (t[2], t[0]))}
    assert n - len(edges) + len(tris) == 2
    # every edge has exactly two incident faces with opposite orientation
    directed = {(t[a], t[(a + 1) % 3]) for t in tris.tolist() for a in range(3)}
    assert len(directed) == 3 * len(tris)
    assert all((b, a) in directed for (a, b) in directed)
    assert np.allclose(np.linalg.norm(unit, axis=1), 1.0)


def test_icosphere_outward_and_pole_ids():
    m = scene.icosphere(8)
    c = m.pos[m.tris].mean(1)
    e1 = m.pos[m.tris[:, 1]] - m.pos[m.tris[:, 0]]
    e2 = m.pos[m.tris[:, 2]] - m.pos[m.tris[:, 0]]
    assert np.all((np.cross(e1, e2) * c).sum(1) > 0)
    assert np.allclose(m.pos[10 * 64], [0, 0, 20.0])
    assert np.allclose(m.pos[10 * 64 + 1], [0, 0, -20.0])


def test_areas_converge_to_sphere():
    a16 = scene.icosphere(16).area.sum()
    a64 = scene.icosphere(64).area.sum()
    full = 4 * math.pi * scene.MESH_SCALE_MM ** 2
    assert abs(a64 - full) < abs(a16 - full) / 10
    assert abs(a64 - full) / full < 1e-4


def test_displacement_seeded_and_bounded():
    a = scene.icosphere(16, 0.1, 3, 1).pos
    b = scene.icosphere(16, 0.1, 3, 1).pos
    c = scene.icosphere(16, 0.1, 3, 2).pos
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    rad = np.linalg.norm(a, axis=1) / scene.MESH_SCALE_MM
    assert rad.min() >= 0.9 - 1e-12 and rad.max() <= 1.1 + 1e-12


def _sphere_quadrature(n_t=96, n_p=192):
    x, w = np.polynomial.legendre.leggauss(n_t)
    phi = (np.arange(n_p) + 0.5) * 2 * math.pi / n_p
    ct = np.repeat(x, n_p)
    st = np.sqrt(1 - ct * ct)
    ph = np.tile(phi, n_t)
    dirs = np.stack([st * np.cos(ph), st * np.sin(ph), ct], 1)
    wt = np.repeat(w, n_p) * (2 * math.pi / n_p)
    return dirs, wt


def test_sh_orthonormal_by_quadrature():
    dirs, wt = _sphere_quadrature()
    Y = scene.sh_real(5, dirs)
    G = (Y * wt) @ Y.T
    assert np.max(np.abs(G - np.eye(25))) < 1e-12


def test_sh_transfer_is_clamped_cosine_projection():
    # Funk-Hecke: int Y_j(w) max(n.w, 0) dw = Ahat_l Y_j(n); checked by direct quadrature
    dirs, wt = _sphere_quadrature(400, 800)
    Y = scene.sh_real(5, dirs)
    rng = np.random.default_rng(0)
    n = rng.standard_normal((4, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    T = scene.sh_transfer(n, 25)
    for q in range(4):
        cosw = np.maximum(dirs @ n[q], 0.0)
        direct = (Y * (cosw * wt)) .sum(1)
        assert np.max(np.abs(direct - T[:, q])) < 2e-4


def test_batched_sizes():
    nu = scene.batched_nus()
    assert nu.shape == (256,) and nu.min() >= 8 and nu.max() <= 64
    assert np.array_equal(nu, scene.batched_nus())
