"""Pins that tie the oracle's right-hand side to things other than itself.

* brute force: a 50-digit mpmath evaluation of the Section 2 definitions on
  1-2 element periodic meshes with discontinuous states (``brute_mp``);
* FR-DG equals nodal DG: the weak-form DG residual with Gauss quadrature,
  coded without correction functions (``weak_dg``; Huynh's equivalence of FR
  with the DG correction function and nodal DG, Eq. FRfinal);
* heat conduction: a quiescent gas at constant pressure whose internal
  energy varies, e = e0 + a cos x, has exactly dE/dt = kappa e'' =
  -kappa a cos x with kappa = mu gamma / Pr, all other components 0;
* a manufactured Navier-Stokes state whose exact right-hand side -div F
  is derived symbolically (sympy) from the textbook fluxes;
* the LDG penalty is dissipative: it changes the mass-weighted inner
  product <u, R> by exactly -tau sum w |dA| |u- - u+|^2.

Each pin has a companion that plants a plausible mistake in the oracle (on
the CPU, by monkeypatching) and shows the pin fails.
"""
import numpy as np
import pytest
import sympy as sp
from scipy.spatial import cKDTree

import oracle.fr as ofr
from frinputs import box_hex, ics
from oracle import physics as oph
from oracle.fr import FRSystem
from oracle.mesh import FRMesh

import brute_mp
import weak_dg

# a sheared parallelepiped map: physical normals differ from reference ones
SHEAR = [[1.0, 0.3, 0.1], [0.2, 1.1, -0.15], [-0.1, 0.25, 0.9]]
GAMMA, MU, PRANDTL = 1.4, 0.05, 0.72


def _per_var(a, b):
    return np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)


def _match(m, pos, keys):
    """Oracle (element, point) order of the keyed points: elements by
    centroid, then points within each element by position (Gauss-Lobatto
    points of neighbouring elements coincide on their shared faces)."""
    els = sorted({k[0] for k in keys})
    cen = {e: np.mean([pos[k] for k in keys if k[0] == e], axis=0) for e in els}
    order = []
    for i, oc in enumerate(m.upts_x["hex"].mean(axis=1)):
        e = min(els, key=lambda f: np.linalg.norm(cen[f] - oc))
        ks = [k for k in keys if k[0] == e]
        d, j = cKDTree(np.array([pos[k] for k in ks])).query(m.upts_x["hex"][i])
        assert d.max() < 1e-12 and len(set(j.tolist())) == len(j)
        order += [ks[q] for q in j]
    return order


def _oracle_on_points(spec, p, physics, keys, pos, state, family="gl", **kw):
    """Oracle RHS at its own points and the matching keys."""
    m = FRMesh(spec, p, family=family)
    s = FRSystem(m, physics, gamma=GAMMA, mu=MU, pr=PRANDTL, **kw)
    order = _match(m, pos, keys)
    u = np.array([state[k] for k in order]).reshape(m.ne["hex"], -1, 5)
    idx = np.array([keys.index(k) for k in order])
    return s.rhs({"hex": u})["hex"].reshape(-1, 5), idx


def _brute_case(p, n, physics, seed=7, family="gl"):
    br = brute_mp.BruteFR(p, SHEAR, n, gamma=GAMMA, mu=MU, pr=PRANDTL,
                          family=family)
    pos = br.points()
    keys = sorted(pos)
    st = brute_mp.random_state(keys, seed, amp=0.3 if p < 3 else 0.1)
    R = br.rhs(st, physics)
    rb = np.array([[float(c) for c in R[k]] for k in keys])
    return keys, pos, st, rb


# ------------------------------------------------------------- brute force
@pytest.mark.parametrize("physics", ["euler", "ns"])
@pytest.mark.parametrize("family,p,n", [("gl", 1, (2, 1, 1)), ("gl", 2, (2, 1, 1)),
                                        ("gl", 2, (1, 1, 1)), ("gll", 1, (2, 1, 1)),
                                        ("gll", 2, (2, 1, 1)), ("gll", 3, (1, 1, 1))])
def test_brute_force_small_meshes(physics, family, p, n):
    """Section 2 definitions at 50 digits vs the FP64 oracle: every
    interface carries a jump (random state per point), every face is
    sheared, and one- and two-element periodic meshes pair elements with
    themselves and with each other; Gauss-Legendre and Gauss-Lobatto
    hexahedron points."""
    keys, pos, st, rb = _brute_case(p, n, physics, family=family)
    r, idx = _oracle_on_points(brute_mp.spec_for(SHEAR, n), p, physics,
                               keys, pos, st, family=family)
    assert _per_var(r, rb[idx]).max() < 1e-13


def _rusanov_speed_without_c(ul, ur, n, gamma):
    fl = np.einsum("...j,...jv->...v", n, oph.euler_flux(ul, gamma))
    fr = np.einsum("...j,...jv->...v", n, oph.euler_flux(ur, gamma))
    _, vl, _ = oph.primitives(ul, gamma)
    _, vr, _ = oph.primitives(ur, gamma)
    lam = np.maximum(np.abs(np.sum(vl * n, -1)), np.abs(np.sum(vr * n, -1)))
    return 0.5 * (fl + fr) - 0.5 * lam[..., None] * (ur - ul)


def _rusanov_reference_normal(ul, ur, n, gamma):
    """Wave speed along the dominant reference axis instead of the physical
    unit normal (a plausible indexing slip on sheared elements)."""
    nr = np.zeros_like(n)
    k = np.argmax(np.abs(n), axis=-1)
    np.put_along_axis(nr, k[..., None],
                      np.sign(np.take_along_axis(n, k[..., None], -1)), -1)
    fl = np.einsum("...j,...jv->...v", n, oph.euler_flux(ul, gamma))
    fr = np.einsum("...j,...jv->...v", n, oph.euler_flux(ur, gamma))
    rl, vl, pl = oph.primitives(ul, gamma)
    rr, vr, pr_ = oph.primitives(ur, gamma)
    lam = np.maximum(np.abs(np.sum(vl * nr, -1)) + np.sqrt(gamma * pl / rl),
                     np.abs(np.sum(vr * nr, -1)) + np.sqrt(gamma * pr_ / rr))
    return 0.5 * (fl + fr) - 0.5 * lam[..., None] * (ur - ul)


@pytest.mark.parametrize("planted", [_rusanov_speed_without_c,
                                     _rusanov_reference_normal])
def test_brute_force_catches_planted_wave_speed(planted, monkeypatch):
    keys, pos, st, rb = _brute_case(2, (2, 1, 1), "euler")
    monkeypatch.setattr(ofr, "rusanov", planted)
    r, idx = _oracle_on_points(brute_mp.spec_for(SHEAR, (2, 1, 1)), 2, "euler",
                               keys, pos, st)
    assert _per_var(r, rb[idx]).max() > 1e-4


def test_brute_force_catches_planted_heat_flux(monkeypatch):
    """kappa = mu / Pr instead of mu gamma / Pr."""
    keys, pos, st, rb = _brute_case(2, (2, 1, 1), "ns")
    orig = ofr.viscous_flux
    monkeypatch.setattr(ofr, "viscous_flux",
                        lambda u, g, gamma, mu, pr: orig(u, g, gamma, mu, pr * gamma))
    r, idx = _oracle_on_points(brute_mp.spec_for(SHEAR, (2, 1, 1)), 2, "ns",
                               keys, pos, st)
    assert _per_var(r, rb[idx])[4] > 1e-3


# --------------------------------------------------- FR-DG == weak-form DG
def _weak_case(p, n, physics, seed=11):
    dg = weak_dg.WeakDG(p, SHEAR, n, gamma=GAMMA, mu=MU, pr=PRANDTL)
    pos = dg.points()
    keys = sorted(pos)
    st = brute_mp.random_state(keys, seed, amp=0.3 if p < 3 else 0.08)
    N = p + 1
    order = [(a, b, c) for c in range(N) for b in range(N) for a in range(N)]
    u = {e: np.array([st[(e,) + z] for z in order]) for e in dg.elems}
    R = dg.rhs(u, physics)
    Rk = {(e,) + z: R[e][i] for e in dg.elems for i, z in enumerate(order)}
    return keys, pos, st, np.array([Rk[k] for k in keys])


@pytest.mark.parametrize("physics", ["euler", "ns"])
@pytest.mark.parametrize("p,n", [(1, (2, 1, 1)), (2, (2, 2, 1)), (3, (3, 2, 2)),
                                 (4, (2, 1, 2))])
def test_fr_dg_equals_weak_form_nodal_dg(physics, p, n):
    keys, pos, st, rw = _weak_case(p, n, physics)
    r, idx = _oracle_on_points(brute_mp.spec_for(SHEAR, n), p, physics,
                               keys, pos, st)
    assert _per_var(r, rw[idx]).max() < 1e-12


def test_weak_form_catches_planted_lift_scaling():
    """The correction scaled by 1/2 (a plausible slip in the Radau weights)
    leaves conservation intact but breaks the DG equivalence."""
    keys, pos, st, rw = _weak_case(3, (3, 2, 2), "euler")
    m = FRMesh(brute_mp.spec_for(SHEAR, (3, 2, 2)), 3)
    s = FRSystem(m, "euler", gamma=GAMMA)
    X = np.array([pos[k] for k in keys])
    _, idx = cKDTree(X).query(m.upts_x["hex"].reshape(-1, 3))
    u = np.array([st[keys[i]] for i in idx]).reshape(m.ne["hex"], -1, 5)
    el = m.el["hex"]
    saved = el.LIFT
    try:
        el.LIFT = 0.5 * saved
        r = s.rhs({"hex": u})["hex"].reshape(-1, 5)
    finally:
        el.LIFT = saved
    assert _per_var(r, rw[idx]).max() > 1e-3


# ------------------------------------------------------- heat conduction
def _heat_error(n, p, pr_oracle=PRANDTL, mu=0.1):
    m = FRMesh(box_hex((n, 1, 1), hi=(2 * np.pi, 1.0, 1.0)).as_dict(), p)
    x = m.upts_x["hex"][..., 0]
    e0, a, p0 = 2.5, 0.25, 1.0
    u = np.zeros(x.shape + (5,))
    u[..., 0] = p0 / ((GAMMA - 1) * (e0 + a * np.cos(x)))
    u[..., 4] = p0 / (GAMMA - 1)
    r = FRSystem(m, "ns", gamma=GAMMA, mu=mu, pr=pr_oracle).rhs({"hex": u})["hex"]
    exact = -mu * GAMMA / PRANDTL * a * np.cos(x)
    return (np.abs(r[..., 4] - exact).max() / np.abs(exact).max(),
            np.abs(r[..., :4]).max())


def test_heat_conduction_converges_to_kappa_laplacian():
    """Quiescent gas, p = const, e = 2.5 + 0.25 cos x: dE/dt -> -kappa a cos x
    (kappa = mu gamma / Pr) under refinement (BR1 second derivatives: order
    about p - 1 in the maximum norm), the other components -> 0."""
    e8, o8 = _heat_error(8, 3)
    e16, o16 = _heat_error(16, 3)
    assert e16 < 0.02 and e8 / e16 > 2.8, (e8, e16)
    assert o16 < 1e-4 and o8 / o16 > 4


def test_heat_conduction_catches_planted_kappa():
    e16, _ = _heat_error(16, 3, pr_oracle=PRANDTL * GAMMA)
    assert e16 > 0.2


# ---------------------------------------------- manufactured NS solution
def _manufactured():
    X, Y, Z = sp.symbols("x y z")
    q = sp.Rational
    rho = 1 + q(1, 5) * sp.sin(X) * sp.cos(Y)
    vel = [q(3, 10) + q(1, 5) * sp.sin(Y) + q(1, 10) * sp.sin(X),
           q(1, 5) * sp.cos(X) + q(1, 10) * sp.cos(Y),
           q(1, 10) * sp.sin(X + Y)]
    P = 1 + q(1, 10) * sp.cos(X) * sp.cos(2 * Y)
    G, M, PR = q(7, 5), q(1, 10), q(18, 25)
    xs = (X, Y, Z)
    cons = [rho] + [rho * v for v in vel] + [P / (G - 1) + rho * sum(v * v for v in vel) / 2]
    dv = [[sp.diff(vel[i], xs[j]) for j in range(3)] for i in range(3)]
    div = dv[0][0] + dv[1][1] + dv[2][2]
    tau = [[M * (dv[i][j] + dv[j][i]) - (q(2, 3) * M * div if i == j else 0)
            for j in range(3)] for i in range(3)]
    e = P / ((G - 1) * rho)
    F = []
    for j in range(3):
        inv = ([rho * vel[j]] + [rho * vel[i] * vel[j] + (P if i == j else 0)
                                 for i in range(3)] + [(cons[4] + P) * vel[j]])
        vis = ([0] + [tau[i][j] for i in range(3)]
               + [sum(vel[i] * tau[i][j] for i in range(3)) + M * G / PR * sp.diff(e, xs[j])])
        F.append([inv[k] - vis[k] for k in range(5)])
    R = [-sum(sp.diff(F[j][k], xs[j]) for j in range(3)) for k in range(5)]
    return sp.lambdify(xs, cons, "numpy"), sp.lambdify(xs, R, "numpy")


def _mms_error(n, p, fu, fr):
    m = FRMesh(box_hex((n, n, 1), hi=(2 * np.pi, 2 * np.pi, 1.0)).as_dict(), p)
    x = m.upts_x["hex"]

    def ev(f):
        v = f(x[..., 0], x[..., 1], x[..., 2])
        return np.stack([np.broadcast_to(c, x.shape[:-1]) for c in v], -1)
    r = FRSystem(m, "ns", gamma=1.4, mu=0.1, pr=0.72).rhs({"hex": ev(fu)})["hex"]
    return _per_var(r.reshape(-1, 5), ev(fr).reshape(-1, 5))


def _viscous_without_two_thirds(u, gu, gamma, mu, pr):
    F = _ORIG_VISCOUS(u, gu, gamma, mu, pr)
    rho = u[..., 0]
    v = u[..., 1:4] / rho[..., None]
    gv = (gu[..., :, 1:4] - v[..., None, :] * gu[..., :, 0:1]) / rho[..., None, None]
    div = np.einsum("...ii->...", gv)
    for i in range(3):
        F[..., i, 1 + i] += 2.0 / 3.0 * mu * div
        F[..., i, 4] += v[..., i] * 2.0 / 3.0 * mu * div
    return F


_ORIG_VISCOUS = ofr.viscous_flux


def test_manufactured_navier_stokes_converges():
    """Every conserved variable's discrete RHS converges to the symbolic
    -div(F_inviscid - F_viscous) of a smooth compressible state with
    shear, divergence and temperature gradients."""
    fu, fr = _manufactured()
    e8 = _mms_error(8, 3, fu, fr)
    e16 = _mms_error(16, 3, fu, fr)
    assert e16.max() < 0.01, e16
    assert (e8 / e16).min() > 3.2, e8 / e16


def test_manufactured_catches_planted_stress(monkeypatch):
    fu, fr = _manufactured()
    monkeypatch.setattr(ofr, "viscous_flux", _viscous_without_two_thirds)
    assert _mms_error(16, 3, fu, fr)[1] > 0.02


# ---------------------------------------------------- LDG penalty sign
def _ldg_inner_products(tau):
    m = FRMesh(box_hex((3, 2, 2), perturb=0.1).as_dict(), 3)
    x = m.upts_x["hex"].reshape(-1, 3)
    rng = np.random.Generator(np.random.PCG64(5))
    u = ics.taylor_green(2 * np.pi * x, mach=0.3).reshape(m.ne["hex"], -1, 5)
    u = u * (1 + 0.05 * rng.uniform(-1, 1, u.shape))     # jumps at every face
    ur = {"hex": u}
    r0 = FRSystem(m, "ns", mu=0.02, ldg=(0.5, 0.0)).rhs(ur)["hex"]
    r1 = FRSystem(m, "ns", mu=0.02, ldg=(0.5, tau)).rhs(ur)["hex"]
    el = m.el["hex"]
    lhs = np.einsum("z,ez,ezk,ezk->", el.W, m.detJ["hex"], u, r1 - r0)
    # independent face weights: Gauss-Legendre products at the face points
    xg, wg = np.polynomial.legendre.leggauss(el.p + 1)
    wface = np.tile(np.outer(wg, wg).ravel(), 6)
    uf = np.einsum("fz,ezk->efk", el.M0, u).reshape(-1, 5)
    w_all = np.tile(wface, m.ne["hex"])
    jump = uf[m.pair_l] - uf[m.pair_r]
    expect = -abs(tau) * np.sum(w_all[m.pair_l] * m.fm_all[m.pair_l]
                                * np.sum(jump * jump, axis=1))
    return lhs, expect


def test_ldg_penalty_is_dissipative():
    """The penalty tau (u- - u+) added to the common normal flux changes
    sum_e sum_z W_z J_z u_z . R_z by exactly -tau sum_pairs w |dA| |u- - u+|^2
    (DG lift, Gauss face quadrature at the flux points): never positive."""
    lhs, expect = _ldg_inner_products(0.1)
    assert expect < 0
    assert abs(lhs - expect) < 1e-10 * abs(expect)


def test_ldg_pin_catches_planted_penalty_sign():
    lhs, expect = _ldg_inner_products(-0.1)    # tau (u+ - u-): anti-dissipative
    assert lhs > 0 and abs(lhs - expect) > abs(expect)
