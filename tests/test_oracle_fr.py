"""Pins for the oracle's FR right-hand side (Section 2 and Section 3.4)."""
import numpy as np
import pytest

from frinputs import box_hex, ics, mixed_box
from oracle.fr import FRSystem
from oracle.mesh import FRMesh, MeshError
from oracle.physics import prim_to_cons
from oracle import rk


def _state(m, fn):
    return {t: fn(m.upts_x[t].reshape(-1, 3)).reshape(m.ne[t], -1, 5)
            for t in m.types}


def _maxabs(r):
    return max(np.abs(v).max() for v in r.values())


def _uniform_bcs(n, state=(1.0, 0.3, -0.2, 0.5, 1.0)):
    return {k: ("state",) + tuple(state) for k in range(n)}


@pytest.mark.parametrize("family", ["gl", "gll"])
@pytest.mark.parametrize("p", [2, 3])
@pytest.mark.parametrize("physics", ["euler", "ns"])
def test_freestream_preserved_on_perturbed_hexes(p, physics, family):
    """Section 3.4: a uniform flow stays uniform on a mesh whose interior
    nodes are perturbed by 10% (metric from the vertex map)."""
    m = FRMesh(box_hex((3, 3, 3), perturb=0.1).as_dict(), p, family=family)
    s = FRSystem(m, physics, mu=0.01)
    assert _maxabs(s.rhs(_state(m, ics.uniform))) < 1e-11


@pytest.mark.parametrize("physics", ["euler", "ns"])
def test_freestream_preserved_on_jittered_mixed_mesh(physics):
    m = FRMesh(mixed_box(n=5, x_pri=0.4, x_tet=0.8, perturb=0.05).as_dict(), 3)
    s = FRSystem(m, physics, mu=0.01, bcs=_uniform_bcs(4))
    assert _maxabs(s.rhs(_state(m, ics.uniform))) < 1e-11


def _integral(m, r):
    return sum(np.einsum("z,ez,ezk->k", m.el[t].W, m.detJ[t], r[t])
               for t in m.types)


@pytest.mark.parametrize("family", ["gl", "gll"])
@pytest.mark.parametrize("physics", ["euler", "ns"])
def test_discrete_conservation_periodic_hex(physics, family):
    """Sum over elements of int J R = 0 on a periodic mesh: the common
    fluxes of both sides of every interface cancel."""
    m = FRMesh(box_hex((3, 3, 2), perturb=0.1).as_dict(), 3, family=family)
    s = FRSystem(m, physics, mu=0.02)
    u = _state(m, lambda x: ics.taylor_green(2 * np.pi * x, mach=0.3))
    r = s.rhs(u)
    scale = max(np.abs(_integral(m, {t: np.abs(r[t]) for t in r})))
    assert np.abs(_integral(m, r)).max() < 1e-12 * scale


@pytest.mark.parametrize("layout", [(0.5, 1.0), (0.0, 1.0), (0.0, 0.0)])
@pytest.mark.parametrize("physics", ["euler", "ns"])
def test_discrete_conservation_mixed_periodic(layout, physics):
    """Same on fully periodic hex|prism, all-prism and all-tet meshes: the
    hex|prism quad interfaces, prism|prism triangles and tet|tet triangles
    (whose reference faces have different areas) must cancel exactly."""
    x_pri, x_tet = layout
    spec = mixed_box(n=3, x_pri=x_pri, x_tet=x_tet, perturb=0.05,
                     periodic_x=True)
    m = FRMesh(spec.as_dict(), 2)
    s = FRSystem(m, physics, mu=0.02)
    u = _state(m, lambda x: ics.taylor_green(2 * np.pi * x, mach=0.3))
    r = s.rhs(u)
    scale = max(np.abs(_integral(m, {t: np.abs(r[t]) for t in r})))
    assert np.abs(_integral(m, r)).max() < 1e-12 * scale


@pytest.mark.parametrize("p", [2, 3])
@pytest.mark.parametrize("physics", ["euler", "ns"])
def test_steady_shear_hex(p, physics):
    """u = (y, 0, 0), rho = 1, p const is a steady Euler solution; with
    viscosity mu the energy equation gains exactly +mu (viscous heating
    mu (du/dy)^2, no heat flux since the temperature is uniform)."""
    mu = 0.05
    spec = box_hex((3, 2, 2), periodic=(0, 2))
    m = FRMesh(spec.as_dict(), p)
    bcs = {2: ("state", 1.0, 0.0, 0.0, 0.0, 1.0),
           3: ("state", 1.0, 1.0, 0.0, 0.0, 1.0)}
    s = FRSystem(m, physics, mu=mu, bcs=bcs)
    r = s.rhs(_state(m, ics.shear))
    expect = np.zeros(5)
    if physics == "ns":
        expect[4] = mu
    for t in r:
        assert np.abs(r[t] - expect).max() < 1e-11


@pytest.mark.parametrize("physics", ["euler", "ns"])
def test_steady_shear_mixed_affine(physics):
    """w = x shear on the unperturbed (affine) hex/prism/tet mesh."""
    mu = 0.05
    m = FRMesh(mixed_box(n=5, x_pri=0.4, x_tet=0.8, perturb=0.0).as_dict(), 2)

    def state(x):
        v = np.zeros((len(x), 3))
        v[:, 2] = x[:, 0]
        return prim_to_cons(np.ones(len(x)), v, np.ones(len(x)), 1.4)
    bcs = {0: ("state", 1.0, 0.0, 0.0, 0.0, 1.0),
           1: ("state", 1.0, 0.0, 0.0, 1.0, 1.0),
           2: ("state", 1.0, 0.0, 0.0, 0.8, 1.0),
           3: ("state", 1.0, 0.0, 0.0, 0.8, 1.0)}
    s = FRSystem(m, physics, mu=mu, bcs=bcs)
    r = s.rhs(_state(m, state))
    expect = np.zeros(5)
    if physics == "ns":
        expect[4] = mu
    for t in r:
        assert np.abs(r[t] - expect).max() < 1e-10


def test_planted_lift_error_is_caught():
    """A plausible mistake planted in the oracle (the correction term with
    the wrong sign) breaks the conservation pin."""
    m = FRMesh(box_hex((3, 3, 2), perturb=0.1).as_dict(), 2)
    s = FRSystem(m, "euler")
    u = _state(m, lambda x: ics.taylor_green(2 * np.pi * x, mach=0.3))
    ok = np.abs(_integral(m, s.rhs(u))).max()
    for t in m.types:
        m.el[t].LIFT = -m.el[t].LIFT
    try:
        bad = np.abs(_integral(m, s.rhs(u))).max()
    finally:
        for t in m.types:
            m.el[t].LIFT = -m.el[t].LIFT
    assert ok < 1e-12 and bad > 1e-6


def test_gll_family_rejects_prisms():
    with pytest.raises(MeshError):
        FRMesh(mixed_box(n=3, x_pri=0.34, x_tet=0.67).as_dict(), 2, family="gll")


def test_nonconforming_mesh_is_rejected():
    spec = box_hex((2, 2, 2), periodic=(0, 1))      # z sides unlisted
    spec.bfaces = []
    with pytest.raises(MeshError):
        FRMesh(spec.as_dict(), 2)


def _vortex_error(n, p, t_end, dt):
    lz = 10.0 / n
    spec = box_hex((n, n, 1), lo=(0, 0, 0), hi=(10.0, 10.0, lz))
    m = FRMesh(spec.as_dict(), p)
    s = FRSystem(m, "euler")
    u = _state(m, ics.isentropic_vortex)
    nsteps = int(round(t_end / dt))
    for _ in range(nsteps):
        u = rk.step(s.rhs, u, dt, "rk4")
    ex = _state(m, lambda x: ics.isentropic_vortex(x, t=nsteps * dt))
    err = sum(np.einsum("z,ez,ez->", m.el[t].W, m.detJ[t],
                        (u[t][..., 0] - ex[t][..., 0]) ** 2)
              for t in m.types)
    return np.sqrt(err / (100.0 * lz))


@pytest.mark.slow
@pytest.mark.parametrize("p", [2, 3])
def test_isentropic_vortex_converges_at_order_p_plus_1(p):
    """Density error of the advected isentropic vortex against its closed
    form falls at about order p+1 (observed order > p + 0.3 from 16^2 to
    32^2 elements; coarser meshes are pre-asymptotic for a unit-radius
    vortex)."""
    e1 = _vortex_error(16, p, 0.05, 0.005)
    e2 = _vortex_error(32, p, 0.05, 0.005)
    order = np.log2(e1 / e2)
    assert order > p + 0.3, (e1, e2, order)


@pytest.mark.parametrize("physics", ["euler", "ns"])
def test_prescribed_boundary_state_keeps_exact_shear_steady(physics):
    """The steady shear u = (y, 0, 0) with its own values prescribed point by
    point on the y boundaries ('prescribed' condition): R = 0 (Euler) and
    R = (0, 0, 0, 0, mu) (NS), as with the constant-state condition; and a
    constant prescribed state equals the 'state' condition exactly."""
    mu = 0.05
    spec = box_hex((3, 2, 2), periodic=(0, 2))

    def exact(x):
        return np.column_stack([np.ones(len(x)), x[:, 1], 0 * x[:, 0], 0 * x[:, 0],
                                np.ones(len(x))])
    m = FRMesh(spec.as_dict(), 3)
    s = FRSystem(m, physics, mu=mu, bcs={2: ("prescribed", exact), 3: ("prescribed", exact)})
    r = s.rhs(_state(m, ics.shear))
    expect = np.zeros(5)
    if physics == "ns":
        expect[4] = mu
    assert np.abs(r["hex"] - expect).max() < 1e-11
    const = (1.0, 0.3, 0.1, -0.2, 1.2)
    a = FRSystem(m, physics, mu=mu, bcs={2: ("prescribed", lambda x: np.tile(const, (len(x), 1))),
                                        3: ("state",) + const}).rhs(_state(m, ics.shear))
    b = FRSystem(m, physics, mu=mu, bcs={2: ("state",) + const,
                                        3: ("state",) + const}).rhs(_state(m, ics.shear))
    assert np.array_equal(a["hex"], b["hex"])
