"""Pins for the oracle's point sets (Section 2, Fig. 1)."""
import os

import numpy as np
import pytest

from oracle.elements import element
from oracle.points import tet_nodes, tri_face_points, tri_solution_points
from oracle.polys import gauss_legendre, gauss_lobatto

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    return np.loadtxt(os.path.join(GOLDEN, name), comments="#")


def _same_set(a, b, tol):
    d = np.linalg.norm(a[:, None, :] - b[None, :, :], axis=2)
    return d.min(axis=1).max() < tol and d.min(axis=0).max() < tol


def test_tet_p4_solution_points_match_fig1c():
    """Fig. 1(c) prints the 35 p=4 alpha-optimised solution points."""
    gold = _load("tet_p4_solution_points.txt")
    assert gold.shape == (35, 3)
    pts = tet_nodes(4)
    assert pts.shape == (35, 3)
    assert _same_set(pts, gold, 2e-15)


def test_tet_p4_flux_points_match_fig1b():
    """Fig. 1(b): the flux points are the 34 distinct surface locations,
    and every one of them is also a solution point (Fig. 1(c))."""
    gold = _load("tet_p4_flux_points.txt")
    el = element("tet", 4)
    assert el.nfpts == 4 * 15
    uniq = np.unique(np.round(el.fpts, 12), axis=0)
    assert uniq.shape == (34, 3)
    assert _same_set(el.fpts, gold, 2e-15)
    d = np.linalg.norm(el.fpts[:, None] - el.upts[None], axis=2)
    assert d.min(axis=1).max() < 1e-14


def test_tet_p4_face_points_differ_from_2d_alpha():
    """The triangle set on tet faces uses the 3D alpha; the 2D optimum
    (alpha 0.1001 at p=4) does not reproduce the printed -0.551583572090994."""
    face = tri_face_points(4)
    assert np.isclose(face, -0.551583572090994, rtol=0, atol=2e-15).any()
    alt = tri_solution_points(4)
    assert not np.isclose(alt, -0.551583572090994, rtol=0, atol=1e-9).any()


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_tri_and_tet_sets_are_symmetric(p):
    """Both sets are invariant under the element's vertex permutations, so
    conforming faces see the same physical points from either side."""
    t2 = tri_face_points(p)
    bary = np.stack([-(t2[:, 0] + t2[:, 1]) / 2, (1 + t2[:, 0]) / 2,
                     (1 + t2[:, 1]) / 2], axis=1)
    for perm in ([1, 0, 2], [0, 2, 1], [2, 1, 0], [1, 2, 0]):
        b = bary[:, perm]
        q = np.stack([2 * b[:, 1] - 1, 2 * b[:, 2] - 1], axis=1)
        assert _same_set(q, t2, 1e-13)
    t3 = tet_nodes(p)
    lam = np.concatenate([-(t3.sum(1, keepdims=True) + 1) / 2,
                          (1 + t3) / 2], axis=1)
    for perm in ([1, 0, 2, 3], [0, 1, 3, 2], [3, 2, 1, 0]):
        b = lam[:, perm]
        assert _same_set(2 * b[:, 1:] - 1, t3, 1e-13)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 8])
def test_gauss_legendre_exactness(n):
    x, w = gauss_legendre(n)
    assert abs(w.sum() - 2) < 1e-14
    for k in range(2 * n):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-14


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_gauss_lobatto_exactness(n):
    x, w = gauss_lobatto(n)
    assert x[0] == -1 and x[-1] == 1
    for k in range(2 * n - 2):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-14
    # p=4 edge points of Fig. 1 are the interior GLL points of order 4
    if n == 5:
        assert np.allclose(x[1:4], [-np.sqrt(3 / 7), 0, np.sqrt(3 / 7)],
                           atol=1e-15)


def test_point_counts_match_element_formulas():
    for p in range(1, 6):
        assert element("hex", p).nupts == (p + 1) ** 3
        assert element("hex", p).nfpts == 6 * (p + 1) ** 2
        assert element("pri", p).nupts == (p + 1) ** 2 * (p + 2) // 2
        assert element("pri", p).nfpts == (p + 1) * (p + 2) + 3 * (p + 1) ** 2
        assert element("tet", p).nupts == (p + 1) * (p + 2) * (p + 3) // 6
        assert element("tet", p).nfpts == 2 * (p + 1) * (p + 2)
