"""Shared helpers for the tests: build the oracle and the library on the same
seeded inputs and compare them.  Inputs come from ``frinputs``; the oracle
and the library each compute their own points, operators and metrics."""
import numpy as np

from frinputs import box_hex, mixed_box  # noqa: F401


def oracle_state(om, fn):
    return {t: fn(om.upts_x[t].reshape(-1, 3)).reshape(om.ne[t], -1, 5)
            for t in om.types}


def lib_state(gm, fn):
    out = {}
    for t in gm.types:
        x = gm.points(t)
        out[t] = fn(x.reshape(-1, 3)).reshape(x.shape[0], x.shape[1], 5)
    return out


def rel_l2(a, b, uref=1.0):
    """Per conserved variable: ||a - b||_2 / max(||b||_2, ||rho_b||_2 uref)
    over all solution points of all element types."""
    num = np.zeros(5)
    den = np.zeros(5)
    rho = 0.0
    for t in b:
        d = (a[t] - b[t]).reshape(-1, 5)
        r = b[t].reshape(-1, 5)
        num += np.sum(d * d, axis=0)
        den += np.sum(r * r, axis=0)
        rho += np.sum(r[:, 0] ** 2)
    den = np.maximum(np.sqrt(den), np.sqrt(rho) * uref)
    return np.sqrt(num) / np.where(den > 0, den, 1.0)


def rel_l2_rhs(a, b, floor=1e-3):
    """Relative L2 of right-hand sides per conserved variable, each
    normalised by its own norm ||b_k||_2 over all solution points.  A
    component whose norm is below ``floor`` times the largest per-variable
    norm is normalised by that floor instead: such a component is (close
    to) zero in exact arithmetic -- e.g. the w-momentum RHS of a
    z-invariant flow -- so its computed value is rounding of the O(1) flux
    terms that cancel in it, and relative to itself it has no meaning."""
    num = np.zeros(5)
    den = np.zeros(5)
    for t in b:
        d = (a[t] - b[t]).reshape(-1, 5)
        r = b[t].reshape(-1, 5)
        num += np.sum(d * d, axis=0)
        den += np.sum(r * r, axis=0)
    den = np.sqrt(den)
    den = np.maximum(den, floor * max(den.max(), 1e-300))
    return np.sqrt(num) / den
