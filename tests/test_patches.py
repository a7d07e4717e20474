"""The element-patch property that the full-size GPU parity tests rely on:
the oracle's right-hand side of an element evaluated on the 5x5x5 block of
elements around it equals that element's right-hand side on the whole
mesh (Euler and Navier-Stokes), whatever the block's boundary condition."""
import numpy as np
import pytest

from frinputs import box_hex, ics
from oracle.fr import FRSystem
from oracle.mesh import FRMesh

from patches import box_patch


@pytest.mark.parametrize("physics", ["euler", "ns"])
def test_patch_rhs_equals_whole_mesh_rhs(physics):
    n, p = 7, 2
    spec = box_hex((n, n, n), hi=(2 * np.pi,) * 3, perturb=0.1)

    def ic(x):
        return ics.flow3d(x / (2 * np.pi))
    m = FRMesh(spec.as_dict(), p)
    r = FRSystem(m, physics, mu=0.01, pr=0.71).rhs(
        {"hex": ic(m.upts_x["hex"].reshape(-1, 3)).reshape(m.ne["hex"], -1, 5)})["hex"]
    for c in [(3, 3, 3), (2, 4, 2)]:
        sub, ids, mid = box_patch(spec, (n, n, n), c)
        o = FRMesh(sub, p)
        ro = FRSystem(o, physics, mu=0.01, pr=0.71, bcs={0: ("extrap",)}).rhs(
            {"hex": ic(o.upts_x["hex"].reshape(-1, 3)).reshape(o.ne["hex"], -1, 5)})["hex"]
        assert np.array_equal(o.upts_x["hex"][mid], m.upts_x["hex"][ids[mid]])
        assert np.abs(ro[mid] - r[ids[mid]]).max() <= 1e-14 * np.abs(r[ids[mid]]).max()
        # the block's corner element does see the block boundary
        assert np.abs(ro[0] - r[ids[0]]).max() > 1e-6 * np.abs(r[ids[0]]).max()


def test_patch_must_lie_inside_the_box():
    spec = box_hex((5, 5, 5))
    with pytest.raises(ValueError):
        box_patch(spec, (5, 5, 5), (1, 2, 2))
