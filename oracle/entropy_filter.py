"""Entropy filter for the oracle (test infrastructure only).

Section 3.2 of the paper: a modal filter is applied selectively to elements
that violate positivity of density, positivity of pressure or a minimum
entropy condition; its strength is found iteratively per element so that as
little filtering as possible is applied (Dzanic & Witherden 2022).  The
paper gives no formulas; the reading used here:

* modal coefficients u^ = V^{-1} u in the element's orthonormal basis;
  filter u^_k <- sigma_k(zeta) u^_k, sigma_k = exp(-zeta (d_k / p)^2), d_k the
  total degree of mode k; the mean (d = 0) is untouched, so the element mean
  is conserved;
* constraints, checked at the solution points and at the flux points of the
  filtered polynomial: rho >= 1e-8, p >= 1e-8 and
  s = p rho^{-gamma} >= s_min - 1e-8 |s_min|, where s_min is the minimum of s
  over the stage input at the element's solution points, at its own flux
  points and at the partner flux points across its faces (admissible points
  only; with none the entropy condition is dropped);
* feasibility margin g(zeta) = min over those points of
  (rho - 1e-8)/rho_mean, (p - 1e-8)/p_mean,
  (s - s_min + tau |s_min|)/|s_min| with tau = 1e-8 (2^-20 when the
  state being compared is FP32, whose resolution is coarser than 1e-8);
  elements with g(0) >= 0 are left alone; otherwise zeta* is the root of g
  found by the Illinois method on a bracket [lo, hi] with g(lo) < 0 <=
  g(hi), stopped when hi - lo <= 1e-6 hi, when g(hi) <= tau (the feasible
  end meets the constraints with no more slack than the tolerance they
  already carry, so further filtering could not be told from none) or
  after 24 evaluations; the result is the feasible end hi.  The plain bracket is [0, zeta_max], zeta_max = 36
  (exp(-36) ~ 2e-16); with a start guess z0 the bracket is opened at z0,
  then z0 / r or r z0 (r = 1.25 unless given), then by halving / doubling.
  If g(zeta_max) < 0
  the element is filtered with zeta_max and counted as a fallback.

Parity: pinned by the tests in tests/test_oracle_filter.py (identity at
zeta = 0, mean conservation, feasibility of the result, minimality
(g(zeta* (1 - 2e-6)) < 0 or g(zeta*) <= tau), agreement with a brute-force
scan).
"""
import numpy as np

from .physics import primitives

ZETA_MAX = 36.0
EPS_POS = 1e-8
TAU_S = 1e-8
REL_TOL = 1e-6
MAX_EVALS = 24


def mode_degrees(el):
    """Total polynomial degree of each orthonormal mode of the element."""
    from . import bases
    p = el.p
    if el.name == "hex":
        return np.array([i + j + k for i, j, k in bases.hex_modes(p)], float)
    if el.name == "pri":
        return np.array([i + j + k for (i, j), k in bases.pri_modes(p)],
                        float)
    return np.array([i + j + k for i, j, k in bases.tet_modes(p)], float)


class FilterOperators:
    """Per element type: modal transform and filtered evaluation at the
    solution and flux points."""

    def __init__(self, el):
        self.el = el
        self.Vinv = el.vdm_inv                       # modal <- nodal
        self.Vu = el.basis(el.upts)                  # nodal <- modal
        self.Vf = el.basis(el.fpts)
        self.deg = mode_degrees(el)
        self.p = el.p

    def sigma(self, zeta):
        return np.exp(-zeta * (self.deg / self.p) ** 2)

    def evaluate(self, uhat, zeta):
        """Filtered values at solution and flux points, uhat (nm, 5)."""
        s = self.sigma(zeta)[:, None] * uhat
        return self.Vu @ s, self.Vf @ s


def entropy(u, gamma):
    """s = p rho^-gamma at admissible points (rho > 0, p > 0), +inf at the
    others so that they do not lower the minimum."""
    rho, _, p = primitives(u, gamma)
    ok = (rho > 0) & (p > 0)
    return np.where(ok, p * np.where(ok, rho, 1.0) ** (-gamma), np.inf)


def element_smin(system, u):
    """s_min per element from the stage input u: own solution points, own
    flux points and partner flux points across each face."""
    m, g = system.m, system.gamma
    uf = system.interp(u)
    sf = entropy(uf, g)
    partner = np.arange(len(sf))
    partner[m.pair_l] = m.pair_r
    partner[m.pair_r] = m.pair_l
    sf_both = np.minimum(sf, sf[partner])
    out = {}
    for t in m.types:
        n = m.ne[t] * m.el[t].nfpts
        fpart = sf_both[m.foff[t]:m.foff[t] + n].reshape(m.ne[t], -1)
        sm = np.minimum(entropy(u[t], g).min(axis=1), fpart.min(axis=1))
        out[t] = np.where(np.isfinite(sm), sm, 0.0)
    return out


def margin(vals_u, vals_f, smin, gamma, rho_mean, p_mean, tau=TAU_S):
    """Feasibility margin g of one element (scalar)."""
    allv = np.concatenate([vals_u, vals_f])
    rho, _, p = primitives(allv, gamma)
    s = p * np.abs(rho) ** (-gamma)
    s = np.where(rho > 0, s, -np.inf)
    m_rho = (rho.min() - EPS_POS) / rho_mean
    m_p = (p.min() - EPS_POS) / p_mean
    if smin > 0:
        m_s = (s.min() - smin + tau * smin) / smin
    else:
        m_s = np.inf
    g = min(m_rho, m_p, m_s)
    return g if np.isfinite(g) or g == np.inf else -np.inf


def find_zeta(gfun, guess=None, ratio=1.25, gtol=TAU_S):
    """Smallest feasible zeta by a bracketed Illinois iteration.

    g(0) is evaluated first in every case (it decides whether the element
    is filtered at all).  Without a guess the bracket is [0, zeta_max].
    With a guess z0 the bracket is opened around it: z0, then z0 / ratio
    or ratio z0, then repeated halving / doubling.  The search ends as soon
    as a feasible point has margin <= gtol, when the bracket is within
    1e-6 relative, or after 24 evaluations.  Returns (zeta, evaluations,
    fallback).  ratio: first bracket step around a guess."""
    evals = 0

    def G(z):
        nonlocal evals
        evals += 1
        return gfun(z)

    def close(gh):
        return gtol is not None and gh <= gtol

    g0 = G(0.0)
    if g0 >= 0:
        return 0.0, evals, False
    lo, glo = 0.0, g0
    if guess is None or not (0.0 < guess < ZETA_MAX):
        hi, ghi = ZETA_MAX, G(ZETA_MAX)
        if ghi < 0:
            return ZETA_MAX, evals, True
    else:
        gz = G(guess)
        if gz >= 0:
            hi, ghi = guess, gz
            z = guess / ratio
            while not close(ghi):
                gz = G(z)
                if gz < 0:
                    lo, glo = z, gz
                    break
                hi, ghi = z, gz
                if z < 1e-6:
                    return hi, evals, False
                z = z * 0.5
        else:
            lo, glo = guess, gz
            z = min(ratio * guess, ZETA_MAX)
            while True:
                gz = G(z)
                if gz >= 0:
                    hi, ghi = z, gz
                    break
                lo, glo = z, gz
                if z >= ZETA_MAX:
                    return ZETA_MAX, evals, True
                z = min(2.0 * z, ZETA_MAX)
    side = 0
    g_hi = ghi      # the margin at hi (ghi is halved by the Illinois rule)
    while not close(g_hi) and hi - lo > REL_TOL * hi and evals < MAX_EVALS:
        z = (lo * ghi - hi * glo) / (ghi - glo)
        if not (lo < z < hi):
            z = 0.5 * (lo + hi)
        gz = G(z)
        if gz >= 0:
            hi, ghi, g_hi = z, gz, gz
            if side == 1:
                glo *= 0.5
            side = 1
        else:
            lo, glo = z, gz
            if side == -1:
                ghi *= 0.5
            side = -1
    return hi, evals, False


def features(op, uhat, vu, vf, smin, gamma):
    """The four predictor inputs of an element, from its unfiltered state:
    log10 of the share of density-mode energy above degree p, min/mean
    density, min/mean pressure (clipped to [-30, 30]) and log10 of the
    entropy-bound violation (s_min - min s)/s_min, floored at 1e-14 (0 when
    a point is not admissible)."""
    e = uhat[:, 0] ** 2
    hi = e[op.deg > op.p].sum()
    tot = e[op.deg >= 1].sum()
    f0 = np.log10((hi + 1e-30) / (tot + 1e-30))
    allv = np.concatenate([vu, vf])
    rho, _, p = primitives(allv, gamma)
    W = op.el.W
    rmean = max(np.dot(W, vu[:, 0]) / W.sum(), EPS_POS)
    pmean = max(np.dot(W, primitives(vu, gamma)[2]) / W.sum(), EPS_POS)
    f1 = rho.min() / rmean
    f2 = p.min() / pmean
    ok = (rho > 0) & (p > 0)
    if smin > 0 and ok.all():
        f3 = max((smin - np.min(p * rho ** (-gamma))) / smin, 1e-14)
    else:
        f3 = 1.0
    f = np.clip(np.array([f0, f1, f2]), -30.0, 30.0)
    return np.concatenate([f, [np.log10(f3)]])


def filter_state(system, u, smin, predictor=None, record=None, tau=TAU_S,
                 ratio=1.25):
    """Filter every element of u (dict of (ne, nu, 5)) that violates the
    constraints; returns (filtered u, zeta per element, evaluations per
    element, fallback flags).  predictor(features) -> start guess; record,
    if given, receives (features, zeta*) of every filtered element."""
    m, g = system.m, system.gamma
    out, zetas, evals, falls = {}, {}, {}, {}
    for t in m.types:
        op = FilterOperators(m.el[t])
        ut = u[t].copy()
        ne = m.ne[t]
        zt = np.zeros(ne)
        et = np.zeros(ne, int)
        ft = np.zeros(ne, bool)
        for e in range(ne):
            uhat = op.Vinv @ u[t][e]
            mean_rho = np.dot(op.el.W, u[t][e][:, 0]) / op.el.W.sum()
            pe = primitives(u[t][e], g)[2]
            mean_p = max(np.dot(op.el.W, pe) / op.el.W.sum(), EPS_POS)
            mean_rho = max(mean_rho, EPS_POS)

            def gfun(z, uhat=uhat, e=e, mr=mean_rho, mp=mean_p):
                vu, vf = op.evaluate(uhat, z)
                return margin(vu, vf, smin[t][e], g, mr, mp, tau)
            guess = None
            if predictor is not None or record is not None:
                vu0, vf0 = op.evaluate(uhat, 0.0)
                if margin(vu0, vf0, smin[t][e], g, mean_rho, mean_p,
                          tau) < 0:
                    feat = features(op, uhat, vu0, vf0, smin[t][e], g)
                    if predictor is not None:
                        guess = float(predictor(feat))
                else:
                    feat = None
            z, n, fb = find_zeta(gfun, guess, ratio, tau)
            zt[e], et[e], ft[e] = z, n, fb
            if z > 0:
                ut[e] = op.evaluate(uhat, z)[0]
                if record is not None and feat is not None and not fb:
                    record.append((feat, z))
        out[t], zetas[t], evals[t], falls[t] = ut, zt, et, ft
    return out, zetas, evals, falls


def rk4_step_filtered(system, u, dt, predictor=None, record=None,
                      tau=TAU_S, ratio=1.25):
    """Classical RK4 with the entropy filter applied to every stage value
    (the state that enters the next right-hand side)."""
    b = (1 / 6, 1 / 3, 1 / 3, 1 / 6)
    c = (0.5, 0.5, 1.0)
    acc = {t: u[t].copy() for t in u}
    stage_in = u
    stats = []
    for s in range(4):
        smin = element_smin(system, stage_in)
        R = system.rhs(stage_in)
        for t in u:
            acc[t] = acc[t] + dt * b[s] * R[t]
        if s < 3:
            nxt = {t: u[t] + dt * c[s] * R[t] for t in u}
        else:
            nxt = acc
        nxt, z, n, fb = filter_state(system, nxt, smin, predictor, record,
                                     tau, ratio)
        stats.append((z, n, fb))
        stage_in = nxt
    return stage_in, stats
