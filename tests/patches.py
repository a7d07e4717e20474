"""Element patches of a box mesh (test infrastructure, no FR arithmetic).

The right-hand side of one element depends on its own state, its face
neighbours' traces and, for Navier-Stokes, the neighbours' corrected
gradients, which involve their own face neighbours' traces: two layers of
elements.  The oracle evaluated on the 5 x 5 x 5 block of elements around
an element, with any boundary condition on the block's outer faces, gives
that element's right-hand side exactly as on the whole mesh.  This lets the
oracle check full-size meshes on sampled elements.
"""
import numpy as np


def box_patch(spec, n, centre, radius=2):
    """Sub-mesh of the box_hex spec (n cells per direction, element order i
    fastest) made of the elements within `radius` cells of `centre` (no
    periodic wrap: the block must lie inside the box).  Returns (sub-spec
    dict with tag-0 boundary faces, global element ids in sub-mesh order,
    local index of the centre element)."""
    nx, ny, nz = n
    ci, cj, ck = centre
    for c, m in zip(centre, n):
        if c - radius < 0 or c + radius >= m:
            raise ValueError("patch leaves the box")
    ids = []
    for k in range(ck - radius, ck + radius + 1):
        for j in range(cj - radius, cj + radius + 1):
            for i in range(ci - radius, ci + radius + 1):
                ids.append(i + nx * (j + ny * k))
    ids = np.array(ids)
    conn = np.asarray(spec.elements["hex"])[ids]
    used, inv = np.unique(conn, return_inverse=True)
    nodes = np.asarray(spec.nodes)[used]
    conn = inv.reshape(conn.shape)
    # faces that appear once are the block's outer faces
    faces = [(0, 3, 7, 4), (1, 2, 6, 5), (0, 1, 5, 4), (3, 2, 6, 7),
             (0, 1, 2, 3), (4, 5, 6, 7)]
    count = {}
    for e in range(len(conn)):
        for f in faces:
            key = tuple(sorted(int(conn[e, v]) for v in f))
            count[key] = count.get(key, 0) + 1
    bf = [(k, 0) for k, c in count.items() if c == 1]
    sub = {"nodes": nodes, "elements": {"hex": conn}, "periodic": [],
           "bfaces": bf, "maps": {}}
    mid = len(ids) // 2
    return sub, ids, mid
