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
