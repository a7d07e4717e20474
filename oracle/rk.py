"""Explicit Runge-Kutta integration for the oracle (test infrastructure only).

Section 2 ends with "a suitable explicit time integration scheme"; Section
3.5 names low-storage Runge-Kutta methods with embedded pairs.  Two schemes:

* RK4: the classical four-stage, fourth-order method (Butcher tableau).
* RK45: Kennedy, Carpenter & Lewis (2000) RK4(3)5[2R+]C, a five-stage
  fourth-order two-register scheme with an embedded third-order pair; its
  coefficients are the published ones.  Stage i uses
  U_i = u^n + dt sum_{j<i-1} b_j k_j + dt a_{i,i-1} k_{i-1}.

Both are written here as full Butcher tableaux and stepped stage by stage.
Pins (tests/test_oracle_rk.py): order conditions up to order 4 hold to
1e-12; on u' = lambda u one step equals the stability polynomial.
"""
import numpy as np

RK4_A = np.array([[0, 0, 0, 0], [0.5, 0, 0, 0], [0, 0.5, 0, 0], [0, 0, 1, 0]],
                 float)
RK4_B = np.array([1 / 6, 1 / 3, 1 / 3, 1 / 6])

RK45_SUB = np.array([970286171893 / 4311952581923,
                     6584761158862 / 12103376702013,
                     2251764453980 / 15575788980749,
                     26877169314380 / 34165994151039])
RK45_B = np.array([1153189308089 / 22510343858157,
                   1772645290293 / 4653164025191,
                   -1672844663538 / 4480602732383,
                   2114624349019 / 3568978502595,
                   5198255086312 / 14908931495163])
RK45_BHAT = np.array([1016888040809 / 7410784769900,
                      11231460423587 / 58533540763752,
                      -1563879915014 / 6823010717585,
                      606302364029 / 971179775848,
                      1097981568119 / 3980877426909])


def rk45_tableau():
    s = 5
    A = np.zeros((s, s))
    for i in range(1, s):
        A[i, :i - 1] = RK45_B[:i - 1]
        A[i, i - 1] = RK45_SUB[i - 1]
    return A, RK45_B.copy()


def tableau(scheme):
    if scheme == "rk4":
        return RK4_A.copy(), RK4_B.copy()
    if scheme == "rk45":
        return rk45_tableau()
    raise ValueError(scheme)


def step(rhs, u, dt, scheme):
    """One step of ``scheme`` for a dict-of-arrays state ``u``."""
    A, b = tableau(scheme)
    ks = []
    for i in range(len(b)):
        ui = {t: u[t] + dt * sum(A[i, j] * ks[j][t] for j in range(i)
                                 if A[i, j] != 0.0)
              for t in u}
        ks.append(rhs(ui))
    return {t: u[t] + dt * sum(b[j] * ks[j][t] for j in range(len(b)))
            for t in u}


# ------------------------------------------------------------------------
# Adaptive step-size control with the embedded pair (Section 3.5, "Adaptive
# Time Stepping": the embedded estimate of the local error, normalised,
# decides acceptance and grows or shrinks the step; the paper cites Hairer,
# Norsett & Wanner for the method).  Readings taken here (the paper gives no
# formulas):
#   error estimate  e = u_{n+1} - uhat_{n+1} = dt sum_i (b_i - bhat_i) k_i
#   norm            err = sqrt(mean_c (e_c / (atol + rtol max(|u_n,c|, |u_{n+1},c|)))^2)
#                   over every component c of every element type; accept when
#                   err <= 1
#   step control    PI controller with exponents 0.7/k and 0.4/k, k = 4 (the
#                   estimate is O(dt^4)): accepted steps take
#                   dt * clip(0.9 err^-0.175 err_prev^0.1, 0.2, 5) (at most 1
#                   right after a rejection), rejected steps
#                   dt * max(0.2, 0.9 err^-0.25); err_prev starts at 1.
ADAPT_SAFETY = 0.9
ADAPT_FACMIN = 0.2
ADAPT_FACMAX = 5.0
ADAPT_ALPHA = 0.7 / 4.0
ADAPT_BETA = 0.4 / 4.0


def embedded_step(rhs, u, dt):
    """One RK4(3)5[2R+] step: (u_{n+1}, dt sum_i (b_i - bhat_i) k_i)."""
    A, b = rk45_tableau()
    d = b - RK45_BHAT
    ks = []
    for i in range(len(b)):
        ui = {t: u[t] + dt * sum(A[i, j] * ks[j][t] for j in range(i)
                                 if A[i, j] != 0.0)
              for t in u}
        ks.append(rhs(ui))
    u1 = {t: u[t] + dt * sum(b[j] * ks[j][t] for j in range(len(b))) for t in u}
    e = {t: dt * sum(d[j] * ks[j][t] for j in range(len(b))) for t in u}
    return u1, e


def error_norm(u0, u1, e, atol, rtol):
    """Root mean square of e scaled by atol + rtol max(|u0|, |u1|)."""
    s, n = 0.0, 0
    for t in u0:
        sc = atol + rtol * np.maximum(np.abs(u0[t]), np.abs(u1[t]))
        s += float(np.sum((e[t] / sc) ** 2))
        n += e[t].size
    return float(np.sqrt(s / n))


def next_dt(dt, err, err_prev, after_reject):
    """Step size after a step of size dt with normalised error err."""
    if err <= 1.0:
        fac = ADAPT_SAFETY * max(err, 1e-10) ** -ADAPT_ALPHA * err_prev ** ADAPT_BETA
        fac = min(max(fac, ADAPT_FACMIN), ADAPT_FACMAX)
        if after_reject:
            fac = min(fac, 1.0)
    else:
        fac = max(ADAPT_FACMIN, ADAPT_SAFETY * err ** -0.25)
    return dt * fac


def adaptive_step(rhs, u, dt, atol, rtol, state):
    """One attempted adaptive step.  state: {"err_prev", "rejected"} (updated).
    Returns (u_next, accepted, err, dt_next); u_next is u when rejected."""
    u1, e = embedded_step(rhs, u, dt)
    err = error_norm(u, u1, e, atol, rtol)
    accepted = err <= 1.0
    dt_next = next_dt(dt, err, state["err_prev"], state["rejected"])
    if accepted:
        state["err_prev"] = max(err, 1e-4)
        state["rejected"] = False
        return u1, True, err, dt_next
    state["rejected"] = True
    return u, False, err, dt_next
