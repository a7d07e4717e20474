"""Pins for the oracle's LDG viscous scheme (reading of the local DG flux of
Cockburn and Shu; the paper names no viscous scheme): beta-biased common
solution and viscous flux along a fixed interface orientation, plus the
penalty tau (u- - u+).

* beta = tau = 0 is BR1;
* the orientation: every interface's "-" side is the lower global element;
* states that are polynomials of the solution space have no jumps, so the
  steady shear keeps its closed form (R = (0, 0, 0, 0, mu));
* a uniform flow stays uniform; the scheme is conservative (both sides of an
  interface see one common flux) for any beta and tau;
* the bias does act on an under-resolved flow, and reversing it (beta ->
  -beta) on the mirrored orientation is the same scheme.
"""
import numpy as np
import pytest

from frinputs import box_hex, ics, mixed_box
from oracle.fr import FRSystem
from oracle.mesh import FRMesh


def _state(m, fn):
    return {t: fn(m.upts_x[t].reshape(-1, 3)).reshape(m.ne[t], -1, 5)
            for t in m.types}


def _tgv(x):
    return ics.taylor_green(2 * np.pi * x, mach=0.3)


def test_zero_bias_zero_penalty_is_br1():
    m = FRMesh(box_hex((3, 3, 2), perturb=0.1).as_dict(), 3)
    u = _state(m, _tgv)
    a = FRSystem(m, "ns", mu=0.02, pr=0.71).rhs(u)["hex"]
    b = FRSystem(m, "ns", mu=0.02, pr=0.71, ldg=(0.0, 0.0)).rhs(u)["hex"]
    assert np.array_equal(a, b)


@pytest.mark.parametrize("name", ["hex", "mixed"])
def test_interface_orientation_lower_element_first(name):
    spec = {"hex": lambda: box_hex((3, 2, 2), perturb=0.1),
            "mixed": lambda: mixed_box(n=3, x_pri=0.34, x_tet=0.67)}[name]()
    m = FRMesh(spec.as_dict(), 2)
    eoff, n = {}, 0
    for t in m.types:
        eoff[t] = n
        n += m.ne[t]

    def element(g):
        for t in m.types:
            lo = m.foff[t]
            hi = lo + m.ne[t] * m.el[t].nfpts
            if lo <= g < hi:
                return eoff[t] + (g - lo) // m.el[t].nfpts
        raise AssertionError
    el = np.array([element(g) for g in m.pair_l])
    er = np.array([element(g) for g in m.pair_r])
    assert np.all(el <= er)


def test_steady_shear_closed_form_with_ldg():
    mu = 0.05
    m = FRMesh(box_hex((3, 2, 2), periodic=(0, 2)).as_dict(), 3)
    bcs = {2: ("state", 1.0, 0.0, 0.0, 0.0, 1.0),
           3: ("state", 1.0, 1.0, 0.0, 0.0, 1.0)}
    r = FRSystem(m, "ns", mu=mu, bcs=bcs, ldg=(0.5, 0.1)).rhs(_state(m, ics.shear))
    expect = np.array([0, 0, 0, 0, mu])
    assert np.abs(r["hex"] - expect).max() < 1e-11


@pytest.mark.parametrize("ldg", [(0.5, 0.1), (-0.3, 0.05)])
def test_free_stream_and_conservation_with_ldg(ldg):
    spec = box_hex((3, 3, 2), perturb=0.1)
    m = FRMesh(spec.as_dict(), 3)
    s = FRSystem(m, "ns", mu=0.02, pr=0.71, ldg=ldg)
    assert np.abs(s.rhs(_state(m, ics.uniform))["hex"]).max() < 1e-10
    r = s.rhs(_state(m, _tgv))["hex"]
    el = m.el["hex"]
    tot = np.einsum("q,eq,eqk->k", el.W, m.detJ["hex"], r)
    scale = np.einsum("q,eq,eqk->k", el.W, m.detJ["hex"], np.abs(r))
    assert np.all(np.abs(tot) < 1e-13 * scale.max()), tot / scale.max()


def test_bias_acts_and_reverses_with_the_orientation():
    """On an under-resolved flow LDG differs from BR1; swapping every
    interface's sides and the sign of beta gives back the same scheme."""
    m = FRMesh(box_hex((2, 2, 2), perturb=0.1).as_dict(), 2)
    u = _state(m, _tgv)
    br1 = FRSystem(m, "ns", mu=0.05, pr=0.71).rhs(u)["hex"]
    a = FRSystem(m, "ns", mu=0.05, pr=0.71, ldg=(0.5, 0.0)).rhs(u)["hex"]
    assert np.abs(a - br1).max() > 1e-3 * np.abs(br1).max()
    m.pair_l, m.pair_r = m.pair_r.copy(), m.pair_l.copy()
    b = FRSystem(m, "ns", mu=0.05, pr=0.71, ldg=(-0.5, 0.0)).rhs(u)["hex"]
    assert np.abs(a - b).max() < 1e-11 * np.abs(a).max()
