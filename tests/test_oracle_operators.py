"""Pins for the oracle's bases and FR operators (Section 2, Eqs. disu and
FRfinal)."""
import itertools

import numpy as np
import pytest
from numpy.polynomial import legendre as L

from oracle import bases
from oracle.elements import element, hex_rule, pri_rule, tet_rule
from oracle.polys import gauss_lobatto, gauss_legendre, lagrange_matrix

TYPES = ["hex", "pri", "tet"]


def _monomials(name, p):
    """Exponent triples spanning the element's solution space."""
    r = range(p + 1)
    if name == "hex":
        return list(itertools.product(r, r, r))
    if name == "pri":
        return [(a, b, c) for a in r for b in r for c in r if a + b <= p]
    return [(a, b, c) for a in r for b in r for c in r if a + b + c <= p]


def _mono(x, e):
    return x[:, 0] ** e[0] * x[:, 1] ** e[1] * x[:, 2] ** e[2]


def _dmono(x, e, d):
    if e[d] == 0:
        return np.zeros(len(x))
    f = list(e)
    f[d] -= 1
    return e[d] * _mono(x, f)


@pytest.mark.parametrize("name", TYPES)
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_orthonormal_under_exact_quadrature(name, p):
    el = element(name, p)
    rule = {"hex": hex_rule, "pri": pri_rule, "tet": tet_rule}[name]
    x, w = rule(p + 2)
    B = el.basis(x)
    G = (B * w[:, None]).T @ B
    assert np.abs(G - np.eye(len(G))).max() < 1e-13


@pytest.mark.parametrize("name", TYPES)
def test_basis_gradients_against_finite_differences(name):
    el = element(name, 3)
    rng = np.random.default_rng(0)
    x = el.upts * 0.7 + 0.01 * rng.standard_normal(el.upts.shape)
    G = el.grad(x)
    h = 1e-6
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        fd = (el.basis(x + e) - el.basis(x - e)) / (2 * h)
        assert np.abs(fd - G[d]).max() < 1e-7 * max(1.0, np.abs(G[d]).max())


@pytest.mark.parametrize("name", TYPES + ["hex-gll"])
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_interpolation_and_derivative_are_exact(name, p):
    """Eq. (disu) and the grad l term of Eq. (FRfinal) are exact on the
    element's polynomial space."""
    name, _, fam = name.partition("-")
    el = element(name, p, fam or "gl")
    for e in _monomials(name, p):
        f = _mono(el.upts, e)
        assert np.abs(el.M0 @ f - _mono(el.fpts, e)).max() < 1e-13
        for d in range(3):
            assert np.abs(el.D[d] @ f - _dmono(el.upts, e, d)).max() < 2e-13


def _radau_derivs(p, x):
    """g_R'(x) = (P'_{p+1} + P'_p)/2 and g_L'(x) for g_L = (-1)^{p+1}
    (P_{p+1} - P_p)/2, Huynh (2007) DG correction functions."""
    cp1 = [0] * (p + 1) + [1]
    cp = [0] * p + [1]
    dp1 = L.legval(x, L.legder(cp1))
    dp = L.legval(x, L.legder(cp))
    return 0.5 * (dp1 + dp), (-1) ** (p + 1) * 0.5 * (dp1 - dp)


@pytest.mark.parametrize("family", ["gl", "gll"])
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_hex_lift_equals_tensor_radau(p, family):
    """The DG lift built from face quadrature equals the tensor-product
    Radau correction of Huynh (2007): for a flux point on x=+1 at (y_j,z_k)
    the lift at (x_a,y_b,z_c) is g_R'(x_a) d_jb d_kc, on x=-1 it is
    -g_L'(x_a) d_jb d_kc (outward normal -x).  The correction function does
    not depend on the solution points: the same formula holds at the
    Gauss-Lobatto points."""
    el = element("hex", p, family)
    x1 = (gauss_legendre(p + 1) if family == "gl" else gauss_lobatto(p + 1))[0]
    gr, gl = _radau_derivs(p, x1)
    n = p + 1
    ref = np.zeros_like(el.LIFT)
    for s in range(el.nfpts):
        f = el.fpts[s]
        nrm = el.fpts_norm[s]
        d = int(np.nonzero(nrm)[0][0])
        others = [k for k in range(3) if k != d]
        for z in range(el.nupts):
            u = el.upts[z]
            if all(abs(u[k] - f[k]) < 1e-14 for k in others):
                a = int(np.argmin(np.abs(x1 - u[d])))
                ref[z, s] = gr[a] if nrm[d] > 0 else -gl[a]
    assert np.abs(ref - el.LIFT).max() < 1e-12
    assert n ** 3 == el.nupts


@pytest.mark.parametrize("name", TYPES)
@pytest.mark.parametrize("p", [1, 2, 3])
def test_lift_reproduces_face_integrals(name, p):
    """int_element v LIFT_s = int_face(s) v l_s for every monomial v of the
    solution space; checked with an independent volume rule and the
    closed-form face integrals of monomials."""
    el = element(name, p)
    rule = {"hex": hex_rule, "pri": pri_rule, "tet": tet_rule}[name]
    xq, wq = rule(p + 3)
    Lq = el.basis(xq) @ el.vdm_inv            # nodal basis at quad points
    lift_q = Lq @ el.LIFT                     # (nq, nf)
    for e in _monomials(name, p):
        v = _mono(xq, e)
        lhs = (wq * v) @ lift_q
        # right-hand side: face integral of v times the face Lagrange basis,
        # by a dense rule on each face
        rhs = np.zeros(el.nfpts)
        for fi, face in enumerate(el.faces):
            st, w2 = el._face_rule(face)
            xf = face.map(st)
            Vf = el._face_basis(face, el.face_points(face))
            lf = el._face_basis(face, st) @ np.linalg.inv(Vf)
            rhs[el.face_fpts[fi]] = (w2 * face.scale * _mono(xf, e)) @ lf
        assert np.abs(lhs - rhs).max() < 1e-12


def test_lagrange_matrix_identity():
    x = gauss_legendre(5)[0]
    assert np.abs(lagrange_matrix(x, x) - np.eye(5)).max() < 1e-15


@pytest.mark.parametrize("name", TYPES)
def test_integration_weights(name):
    el = element(name, 3)
    vol = {"hex": 8.0, "pri": 4.0, "tet": 4.0 / 3.0}[name]
    assert abs(el.W.sum() - vol) < 1e-13
    # integrates the solution space exactly: int x^2 over the element
    e = (2, 0, 0)
    exact = {"hex": 8.0 / 3.0, "pri": 2.0 / 3.0 * 2, "tet": None}[name]
    val = el.W @ _mono(el.upts, e)
    if exact is not None:
        # prism: int_tri x^2 = 2/3 (reference triangle), times length 2
        assert abs(val - exact) < 1e-13
    else:
        # tet: int x^2 over the reference tet = 2/5 * 4/3 ... by quadrature
        xq, wq = tet_rule(8)
        assert abs(val - wq @ xq[:, 0] ** 2) < 1e-13


def test_bases_module_sizes():
    for p in range(5):
        assert len(bases.tri_modes(p)) == (p + 1) * (p + 2) // 2
        assert len(bases.tet_modes(p)) == (p + 1) * (p + 2) * (p + 3) // 6


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_gll_flux_points_are_solution_points(p):
    """Gauss-Lobatto hexahedra (Section 3.1, "Matrix multiplications", last
    paragraph): every flux point is a solution point, so the interpolation
    of Eq. (disu) is a gather -- each row of M0 one 1 at the coinciding
    solution point, zeros elsewhere."""
    el = element("hex", p, "gll")
    for f in range(el.nfpts):
        d = np.linalg.norm(el.upts - el.fpts[f], axis=1)
        z = int(np.argmin(d))
        assert d[z] < 1e-15
        row = np.zeros(el.nupts)
        row[z] = 1.0
        assert np.abs(el.M0[f] - row).max() < 1e-13


def test_gll_family_is_hexahedra_only():
    for name in ("pri", "tet"):
        with pytest.raises(ValueError):
            element(name, 2, "gll")
