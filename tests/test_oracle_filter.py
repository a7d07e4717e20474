"""Pins for the oracle's entropy filter (Section 3.2) and the filter-strength
predictor."""
import numpy as np
import pytest

from frinputs import box_hex, ics
from oracle import entropy_filter as EF
from oracle import mlp
from oracle import rk
from oracle.fr import FRSystem
from oracle.mesh import FRMesh

POST = ics.SHU_OSHER_POST


def _shu_osher(n=32, p=3):
    spec = box_hex((n, 1, 1), lo=(-5, 0, 0), hi=(5, 10 / n, 10 / n),
                   periodic=(1, 2))
    m = FRMesh(spec.as_dict(), p)
    bcs = {0: ("state", POST[0], POST[1], 0, 0, POST[2]), 1: ("extrap",)}
    s = FRSystem(m, "euler", bcs=bcs)
    u = {"hex": ics.shu_osher(m.upts_x["hex"].reshape(-1, 3)).reshape(
        m.ne["hex"], -1, 5)}
    return m, s, u


@pytest.mark.parametrize("name", ["hex", "pri", "tet"])
def test_zero_strength_is_identity_and_mean_is_kept(name):
    from oracle.elements import element
    el = element(name, 3)
    op = EF.FilterOperators(el)
    rng = np.random.default_rng(0)
    u = 1.0 + 0.1 * rng.standard_normal((el.nupts, 5))
    uhat = op.Vinv @ u
    vu, vf = op.evaluate(uhat, 0.0)
    assert np.abs(vu - u).max() < 1e-13
    assert np.abs(vf - el.M0 @ u).max() < 1e-13
    for z in (0.5, 3.0, 36.0):
        vu, _ = op.evaluate(uhat, z)
        assert np.abs(el.W @ vu - el.W @ u).max() < 1e-13
    # strongest filter leaves essentially the mean
    vu, _ = op.evaluate(uhat, 1e3)
    assert np.abs(vu - (el.W @ u) / el.W.sum()).max() < 1e-12


def test_root_find_returns_minimal_feasible_strength():
    """On a synthetic monotone margin the root-find returns the root to the
    stated tolerance, from the plain bracket and from guesses either side."""
    root = 2.7182818

    def g(z):
        return np.tanh(z - root)
    for guess in (None, 0.1, 2.0, 3.0, 30.0):
        for gtol in (EF.TAU_S, None):
            z, n, fb = EF.find_zeta(g, guess, gtol=gtol)
            assert not fb and g(z) >= 0
            assert abs(z - root) <= 2e-6 * root
            assert g(z) <= EF.TAU_S or g(z * (1 - 2e-6)) < 0
    z, n, fb = EF.find_zeta(lambda z: -1.0)
    assert fb and z == EF.ZETA_MAX
    z, n, fb = EF.find_zeta(lambda z: 1.0)
    assert z == 0.0 and n == 1
    # a good guess needs fewer evaluations than the plain bracket
    n_plain = EF.find_zeta(g)[1]
    n_guess = EF.find_zeta(g, root * 1.05)[1]
    assert n_guess < n_plain


def test_margin_stop_ends_at_the_first_feasible_point_within_tau():
    """With gtol the search ends as soon as the feasible end's margin is at
    most gtol, and never returns an infeasible strength."""
    root = 0.37

    def g(z):
        return 1e-3 * (z - root)          # margin 1e-8 is 1e-5 past the root
    z, n, fb = EF.find_zeta(g, gtol=1e-8)
    assert 0.0 <= g(z) <= 1e-8
    z2, n2, _ = EF.find_zeta(g, gtol=None)
    assert n <= n2 and abs(z2 - root) <= 1e-6 * root


def test_filtered_elements_are_feasible_minimal_and_match_a_scan():
    m, s, u = _shu_osher(n=64)
    dt = 2e-3
    smin = EF.element_smin(s, u)
    R = s.rhs(u)
    assert np.isfinite(R["hex"]).all()
    nxt = {"hex": u["hex"] + 0.5 * dt * R["hex"]}
    out, z, n, fb = EF.filter_state(s, nxt, smin)
    zt = z["hex"]
    assert (zt > 0).any() and not fb["hex"].any()
    op = EF.FilterOperators(m.el["hex"])
    g = s.gamma
    for e in np.nonzero(zt > 0)[0][:8]:
        uhat = op.Vinv @ nxt["hex"][e]
        mr = max(np.dot(op.el.W, nxt["hex"][e][:, 0]) / op.el.W.sum(), 1e-8)
        pe = (g - 1) * (nxt["hex"][e][:, 4] - 0.5 * np.sum(
            nxt["hex"][e][:, 1:4] ** 2, axis=1) / nxt["hex"][e][:, 0])
        mp = max(np.dot(op.el.W, pe) / op.el.W.sum(), 1e-8)

        def gfun(zz):
            vu, vf = op.evaluate(uhat, zz)
            return EF.margin(vu, vf, smin["hex"][e], g, mr, mp)
        assert gfun(zt[e]) >= 0
        assert gfun(zt[e]) <= EF.TAU_S or gfun(zt[e] * (1 - 2e-6)) < 0
        scan = np.linspace(0, EF.ZETA_MAX, 3601)
        first = scan[np.argmax([gfun(q) >= 0 for q in scan])]
        assert first - 0.01 <= zt[e] <= first + 1e-9


def test_filter_keeps_shu_osher_finite_where_plain_rk4_fails():
    m, s, u0 = _shu_osher(n=64)
    dt = 2e-3
    u = u0
    for _ in range(6):
        u, _ = EF.rk4_step_filtered(s, u, dt)
    assert np.isfinite(u["hex"]).all()
    assert u["hex"][..., 0].min() > 0
    v = u0
    with np.errstate(all="ignore"):
        for _ in range(10):
            v = rk.step(s.rhs, v, dt, "rk4")
    assert not np.isfinite(v["hex"]).all()


def test_filter_conserves_mass_per_element():
    m, s, u = _shu_osher(n=64)
    smin = EF.element_smin(s, u)
    R = s.rhs(u)
    nxt = {"hex": u["hex"] + 1e-3 * R["hex"]}
    out, z, _, _ = EF.filter_state(s, nxt, smin)
    J = m.detJ["hex"]
    W = m.el["hex"].W
    a = np.einsum("z,ez,ezk->ek", W, J, nxt["hex"])
    b = np.einsum("z,ez,ezk->ek", W, J, out["hex"])
    assert np.abs(a - b).max() < 1e-12 * np.abs(a).max()


def test_mlp_backward_matches_finite_differences():
    rng = np.random.default_rng(3)
    theta = mlp.init(seed=5, mean=rng.normal(size=4),
                     std=rng.uniform(0.5, 2, 4))
    x = rng.normal(size=(17, 4))
    zs = np.exp(rng.normal(size=17))
    loss, g = mlp.loss_and_grad(theta, x, zs)
    h = 1e-6
    idx = list(range(0, mlp.NTRAIN, 37)) + [mlp.NTRAIN - 1]
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss_and_grad(tp, x, zs)[0]
              - mlp.loss_and_grad(tm, x, zs)[0]) / (2 * h)
        assert abs(fd - g[i]) < 1e-7 * max(1.0, abs(g[i])), i
    assert np.all(g[mlp.NTRAIN:] == 0)
