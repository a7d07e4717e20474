"""Pins for the oracle's anti-aliased flux (Section 3.2, "Anti-aliasing":
the transformed flux is taken at the points of a volume quadrature rule and
projected onto the solution space by least squares instead of collocated).

* the rules integrate every monomial of total degree <= qdeg exactly
  (closed forms: products of 2/(k+1) on the cube, the barycentric formula
  a! b! c! d! n! |T| / (a+b+c+d+n)! on the simplices);
* the projection reproduces the solution space (P B = I for qdeg >= 2p) and
  is the exact L2 projection for integrands within the rule's degree;
* for a flux that lies in the solution space the anti-aliased right-hand
  side equals the collocated one and the closed form -div f;
* free stream, discrete conservation, and that it does change the
  right-hand side of a nonlinear flow.
"""
from math import factorial

import numpy as np
import pytest

from frinputs import box_hex, curved_box_hex, ics, mixed_box
from oracle.elements import element
from oracle.fr import FRSystem
from oracle.mesh import FRMesh
from oracle.physics import prim_to_cons

TYPES = ["hex", "pri", "tet"]


def _exact_monomial(t, a, b, c):
    """Integral of x^a y^b z^c over the reference element."""
    line = lambda k: 0.0 if k % 2 else 2.0 / (k + 1)  # noqa: E731
    if t == "hex":
        return line(a) * line(b) * line(c)
    raise AssertionError


def _bary_integral(lam_pows, dim, measure):
    n = sum(lam_pows)
    num = np.prod([factorial(k) for k in lam_pows]) * factorial(dim)
    return num * measure / factorial(n + dim)


@pytest.mark.parametrize("t", TYPES)
@pytest.mark.parametrize("qdeg", [1, 2, 4, 6, 9, 12])
def test_rule_exact_to_its_degree(t, qdeg):
    el = element(t, 2)
    x, w = el.quadrature(qdeg)
    rng = np.random.default_rng(qdeg)
    for _ in range(12):
        k = rng.integers(0, qdeg + 1)
        if t == "hex":
            a = rng.integers(0, k + 1)
            b = rng.integers(0, k - a + 1)
            c = k - a - b
            val = np.sum(w * x[:, 0] ** a * x[:, 1] ** b * x[:, 2] ** c)
            ref = _exact_monomial(t, a, b, c)
        elif t == "tet":
            # barycentric coordinates of the reference tetrahedron
            lam = np.stack([-(1 + x[:, 0] + x[:, 1] + x[:, 2]) / 2,
                            (1 + x[:, 0]) / 2, (1 + x[:, 1]) / 2,
                            (1 + x[:, 2]) / 2], axis=1)
            pw = rng.multinomial(k, [0.25] * 4)
            val = np.sum(w * np.prod(lam ** pw, axis=1))
            ref = _bary_integral(pw, 3, 4.0 / 3.0)
        else:  # prism = triangle x line
            lam = np.stack([-(x[:, 0] + x[:, 1]) / 2, (1 + x[:, 0]) / 2,
                            (1 + x[:, 1]) / 2], axis=1)
            kz = rng.integers(0, k + 1)
            pw = rng.multinomial(k - kz, [1 / 3] * 3)
            val = np.sum(w * np.prod(lam ** pw, axis=1) * x[:, 2] ** kz)
            ref = _bary_integral(pw, 2, 2.0) * (0.0 if kz % 2 else 2.0 / (kz + 1))
        assert abs(val - ref) < 1e-14 * max(1.0, abs(ref)), (pw if t != "hex" else (a, b, c), val, ref)


@pytest.mark.parametrize("t", TYPES)
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_projection_reproduces_solution_space(t, p):
    el = element(t, p)
    for qdeg in (2 * p, 3 * p):
        _, _, B, P = el.aa_operators(qdeg)
        assert np.abs(P @ B - np.eye(el.nupts)).max() < 1e-13


def _monomials(x, d, rng, n=4):
    """x^d (outside both Q_p and P_p for d > p), then a few random
    monomials of total degree exactly d, at points x."""
    out = [x[:, 0] ** d]
    for _ in range(n):
        a = rng.integers(0, d + 1)
        b = rng.integers(0, d - a + 1)
        c = d - a - b
        out.append(x[:, 0] ** a * x[:, 1] ** b * x[:, 2] ** c)
    return out


@pytest.mark.parametrize("t", TYPES)
def test_projection_is_the_exact_l2_projection(t):
    """For f of degree d <= qdeg - p the rule integrates phi_k f exactly, so
    the projection equals the one taken with a far higher rule (degree 30);
    the collocated values (the aliased form) differ once d >= p + 2."""
    p, qdeg = 3, 9
    el = element(t, p)
    xq, _, _, P = el.aa_operators(qdeg)
    xh, _, _, Ph = el.aa_operators(30)
    for d in (4, 5, qdeg - p):
        seed = 100 + d
        fq = _monomials(xq, d, np.random.default_rng(seed))
        fh = _monomials(xh, d, np.random.default_rng(seed))
        fu = _monomials(el.upts, d, np.random.default_rng(seed))
        for i, (a, b, c) in enumerate(zip(fq, fh, fu)):
            proj, exact = P @ a, Ph @ b
            assert np.abs(proj - exact).max() < 1e-12 * np.abs(exact).max()
            if i == 0 and d >= p + 2:
                # x^d aliases at collocation (at Gauss points interpolation
                # of degree p + 1 still equals the projection)
                assert np.abs(c - exact).max() > 1e-6


def _x_flow(x, gamma=1.4):
    """rho = 1, velocity (x, 0, 0), p = 1: every flux component is a
    polynomial of degree <= 3 in x."""
    one = np.ones(len(x))
    v = np.zeros((len(x), 3))
    v[:, 0] = x[:, 0]
    return prim_to_cons(one, v, one, gamma)


def _x_flow_rhs(x, gamma, mu):
    """Closed form of -div(f - f_v) for _x_flow: the viscous stress
    tau_xx = 4 mu / 3 is uniform, the temperature is uniform (no heat flux),
    so the viscous part contributes d/dx (u tau_xx) = 4 mu / 3 to energy."""
    X = x[..., 0]
    r = np.zeros(x.shape[:-1] + (5,))
    r[..., 0] = -1.0
    r[..., 1] = -2.0 * X
    r[..., 4] = -(gamma / (gamma - 1.0) + 1.5 * X ** 2) + 4.0 * mu / 3.0
    return r


def _state(m, fn):
    return {t: fn(m.upts_x[t].reshape(-1, 3)).reshape(m.ne[t], -1, 5)
            for t in m.types}


EXTRAP = {k: ("extrap",) for k in range(6)}


@pytest.mark.parametrize("mesh", ["hex", "mixed"])
@pytest.mark.parametrize("p", [3, 4])
@pytest.mark.parametrize("physics", ["euler", "ns"])
def test_polynomial_flux_equals_collocation_and_closed_form(mesh, p, physics):
    if mesh == "hex":
        spec = box_hex((3, 2, 2), periodic=(1, 2))
    else:
        spec = mixed_box(n=3, x_pri=0.34, x_tet=0.67, perturb=0.0)
    m = FRMesh(spec.as_dict(), p)
    mu = 0.05 if physics == "ns" else 0.0
    u = _state(m, _x_flow)
    r_col = FRSystem(m, physics, mu=mu, bcs=EXTRAP).rhs(u)
    r_aa = FRSystem(m, physics, mu=mu, bcs=EXTRAP, antialias=3 * p).rhs(u)
    for t in m.types:
        exact = _x_flow_rhs(m.upts_x[t], 1.4, mu)
        assert np.abs(r_aa[t] - exact).max() < 1e-10
        assert np.abs(r_col[t] - exact).max() < 1e-10


@pytest.mark.parametrize("spec_name", ["perturbed_hex", "mixed", "curved"])
@pytest.mark.parametrize("p", [2, 3])
def test_free_stream_with_antialiasing(spec_name, p):
    """Perturbed trilinear hexahedra: the metric's cofactors lie in the
    tensor space Q_2, so their projection is exact for p >= 2; curved
    elements: the curl-form metric is itself in Q_p."""
    spec = {"perturbed_hex": lambda: box_hex((3, 3, 2), perturb=0.1),
            "mixed": lambda: mixed_box(n=3, x_pri=0.34, x_tet=0.67, perturb=0.05),
            "curved": lambda: curved_box_hex((3, 3, 2))}[spec_name]()
    m = FRMesh(spec.as_dict(), p)
    bcs = {k: ("extrap",) for k in range(6)}
    s = FRSystem(m, "ns", mu=0.02, pr=0.71, bcs=bcs, antialias=3 * p)
    r = s.rhs(_state(m, ics.uniform))
    for t in r:
        assert np.abs(r[t]).max() < 1e-10, (t, np.abs(r[t]).max())


@pytest.mark.parametrize("spec_name", ["perturbed_hex", "curved"])
def test_conservation_with_antialiasing(spec_name):
    spec = {"perturbed_hex": lambda: box_hex((3, 3, 2), perturb=0.1),
            "curved": lambda: curved_box_hex((3, 3, 2))}[spec_name]()
    m = FRMesh(spec.as_dict(), 3)
    s = FRSystem(m, "ns", mu=0.02, pr=0.71, antialias=9)
    u = _state(m, lambda x: ics.taylor_green(2 * np.pi * x, mach=0.3))
    r = s.rhs(u)
    el = m.el["hex"]
    tot = np.einsum("q,eq,eqk->k", el.W, m.detJ["hex"], r["hex"])
    scale = np.einsum("q,eq,eqk->k", el.W, m.detJ["hex"], np.abs(r["hex"]))
    assert np.all(np.abs(tot) < 1e-13 * scale.max()), tot / scale.max()


def test_antialiasing_changes_a_nonlinear_rhs():
    """On an under-resolved nonlinear flow the projected flux differs from
    the collocated one (the aliasing error it removes), and the difference
    shrinks as the rule's degree grows (the projection converges)."""
    m = FRMesh(box_hex((2, 2, 2), perturb=0.1).as_dict(), 3)
    u = _state(m, lambda x: ics.taylor_green(2 * np.pi * x, mach=0.3))
    r0 = FRSystem(m, "euler").rhs(u)["hex"]
    r = {q: FRSystem(m, "euler", antialias=q).rhs(u)["hex"] for q in (9, 15, 30)}
    scale = np.abs(r0).max()
    assert np.abs(r[9] - r0).max() > 1e-3 * scale
    assert np.abs(r[15] - r[30]).max() < np.abs(r[9] - r[30]).max()
