"""Pins for the oracle's Runge-Kutta schemes (Section 2; Section 3.5)."""
import numpy as np
import pytest

from oracle import rk


def _order_conditions(A, b):
    c = A.sum(axis=1)
    return {
        "b": b.sum() - 1.0,
        "bc": b @ c - 1 / 2,
        "bc2": b @ c ** 2 - 1 / 3,
        "bAc": b @ A @ c - 1 / 6,
        "bc3": b @ c ** 3 - 1 / 4,
        "bcAc": (b * c) @ A @ c - 1 / 8,
        "bAc2": b @ A @ c ** 2 - 1 / 12,
        "bAAc": b @ A @ A @ c - 1 / 24,
    }


@pytest.mark.parametrize("scheme", ["rk4", "rk45"])
def test_fourth_order_conditions(scheme):
    A, b = rk.tableau(scheme)
    for name, v in _order_conditions(A, b).items():
        assert abs(v) < 1e-12, (scheme, name, v)


def test_rk45_embedded_pair_is_third_order_not_fourth():
    A, _ = rk.tableau("rk45")
    bh = rk.RK45_BHAT
    cond = _order_conditions(A, bh)
    for k in ("b", "bc", "bc2", "bAc"):
        assert abs(cond[k]) < 1e-12
    assert max(abs(cond[k]) for k in ("bc3", "bcAc", "bAc2", "bAAc")) > 1e-6


def test_rk45_is_two_register_form():
    """Stage i only needs sum_{j<i-1} b_j k_j and a_{i,i-1} k_{i-1}."""
    A, b = rk.tableau("rk45")
    for i in range(2, 5):
        assert np.allclose(A[i, :i - 1], b[:i - 1], rtol=0, atol=0)


@pytest.mark.parametrize("scheme", ["rk4", "rk45"])
def test_linear_step_matches_stability_polynomial(scheme):
    A, b = rk.tableau(scheme)
    lam = -0.7 + 0.3j
    dt = 0.4
    z = lam * dt
    # stability polynomial R(z) = 1 + z b^T (I - z A)^{-1} 1
    R = 1 + z * b @ np.linalg.solve(np.eye(len(b)) - z * A, np.ones(len(b)))
    u = {"x": np.array([1.0 + 0.0j])}
    out = rk.step(lambda v: {"x": lam * v["x"]}, u, dt, scheme)
    assert abs(out["x"][0] - R) < 1e-15
    # both are fourth order: R(z) agrees with exp(z) through z^4
    taylor = sum(z ** k / np.prod(range(1, k + 1)) for k in range(5))
    assert abs(R - taylor) < (1 if scheme == "rk4" else 5e-3) * abs(z) ** 5


# ---------------------------------------------------------- adaptive stepping
def test_embedded_error_matches_stability_polynomials():
    """On u' = lambda u the estimate is (R(z) - Rhat(z)) u0, R and Rhat the
    stability polynomials of b and bhat."""
    A, b = rk.tableau("rk45")
    lam, dt = -0.9 + 0.4j, 0.3
    z = lam * dt
    one = np.ones(len(b))
    w = np.linalg.solve(np.eye(len(b)) - z * A, one)
    R, Rh = 1 + z * b @ w, 1 + z * rk.RK45_BHAT @ w
    u = {"x": np.array([2.0 + 0.0j])}
    u1, e = rk.embedded_step(lambda v: {"x": lam * v["x"]}, u, dt)
    assert abs(u1["x"][0] - 2.0 * R) < 1e-14
    assert abs(e["x"][0] - 2.0 * (R - Rh)) < 1e-15


def test_embedded_error_is_fourth_order_in_dt():
    """Local error estimate of a third-order embedded method: O(dt^4)."""
    rhs = lambda v: {"x": -v["x"] ** 2 + np.sin(v["x"])}  # noqa: E731
    u = {"x": np.array([0.7])}
    es = [abs(rk.embedded_step(rhs, u, dt)[1]["x"][0]) for dt in (0.05, 0.025, 0.0125)]
    rates = [np.log2(es[i] / es[i + 1]) for i in range(2)]
    assert all(3.8 < r < 4.2 for r in rates), rates


def test_error_norm_of_the_scale_is_one():
    u0 = {"a": np.array([[1.0, -2.0]]), "b": np.array([3.0])}
    u1 = {"a": np.array([[0.5, -4.0]]), "b": np.array([-1.0])}
    atol, rtol = 1e-3, 1e-2
    e = {t: atol + rtol * np.maximum(np.abs(u0[t]), np.abs(u1[t])) for t in u0}
    assert abs(rk.error_norm(u0, u1, e, atol, rtol) - 1.0) < 1e-15
    e["b"] = -2 * e["b"]   # one of three components doubled: sqrt((1+1+4)/3)
    assert abs(rk.error_norm(u0, u1, e, atol, rtol) - np.sqrt(2.0)) < 1e-15


def _integrate(rhs, u, t_end, dt, atol, rtol):
    st = {"err_prev": 1.0, "rejected": False}
    t, acc, rej = 0.0, 0, 0
    while t < t_end - 1e-14:
        dt = min(dt, t_end - t)
        u, ok, err, dt_next = rk.adaptive_step(rhs, u, dt, atol, rtol, st)
        if ok:
            t += dt
            acc += 1
        else:
            rej += 1
        dt = dt_next
    return u, acc, rej


def test_adaptive_integration_tracks_the_tolerance():
    """y' = -y on [0, 3]: the global error follows the tolerance and a
    too-large first step is rejected and shrunk."""
    rhs = lambda v: {"y": -v["y"]}  # noqa: E731
    errs = []
    for tol in (1e-5, 1e-7, 1e-9):
        y, acc, rej = _integrate(rhs, {"y": np.array([1.0])}, 3.0, 1e-3, tol, tol)
        errs.append(abs(y["y"][0] - np.exp(-3.0)))
        assert errs[-1] < 30 * tol
        assert rej <= 1
    assert errs[0] > errs[1] > errs[2]
    y, acc, rej = _integrate(rhs, {"y": np.array([1.0])}, 3.0, 2.5, 1e-8, 1e-8)
    assert rej >= 1 and abs(y["y"][0] - np.exp(-3.0)) < 3e-7
