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
