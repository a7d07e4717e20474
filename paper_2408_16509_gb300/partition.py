"""Sub-meshes of a partitioned mesh (Section 3.3, "Mixed Elements and Domain
Decomposition").  The library partitions the elements (fr_partition) and
lists each part's faces that border another part (fr_partition_faces);
this module only assembles, for every part, the mesh description of its
elements with those faces as boundary faces of an exchange condition."""
import numpy as np

from ._binding import ETYPES, FRMesh

EXCHANGE_TAG = 1 << 20       # boundary tag of the faces between parts
ORDER = [t for t in ("hex", "pri", "tet")]


def _as_dict(spec):
    return spec.as_dict() if hasattr(spec, "as_dict") else dict(spec)


def split(spec, nparts, mode="weighted", weights=None, order=1, halo_last=False):
    """Partition `spec` into nparts and return (sub_specs, element_ids):
    sub_specs[r] is a mesh description of part r (all nodes kept, its
    elements, the original boundary faces plus its exchange faces tagged
    EXCHANGE_TAG); element_ids[r][t] are the indices, within type t of the
    full mesh, of part r's elements (for scattering solutions).  halo_last:
    each type's elements that border another part come after the others,
    so that a stage's interior work (fr_rk_stage part 1) is one contiguous
    range and can overlap the exchange."""
    d = _as_dict(spec)
    host = FRMesh(d, order, bcs={k: ("extrap",) for k in _tags(d)}, device=-1)
    part = host.partition(nparts, mode, weights)
    halo = {}
    if halo_last:
        types0 = [t for t in ORDER if t in d["elements"] and len(d["elements"][t])]
        offs0 = np.cumsum([0] + [len(d["elements"][t]) for t in types0])
        for i, t in enumerate(types0):
            nbr = host.adjacency(t)
            mine = part[offs0[i]:offs0[i + 1]]
            other = np.where(nbr >= 0, part[np.maximum(nbr, 0)], mine[:, None])
            halo[t] = np.any(other != mine[:, None], axis=1)
    subs, ids = [], []
    types = [t for t in ORDER if t in d["elements"] and len(d["elements"][t])]
    offs = np.cumsum([0] + [len(d["elements"][t]) for t in types])
    for r in range(nparts):
        el, mp, idr = {}, {}, {}
        for i, t in enumerate(types):
            sel = np.nonzero(part[offs[i]:offs[i + 1]] == r)[0]
            if halo_last:
                sel = np.concatenate([sel[~halo[t][sel]], sel[halo[t][sel]]])
            idr[t] = sel
            if len(sel):
                el[t] = np.asarray(d["elements"][t])[sel]
                if t in (d.get("maps") or {}):
                    order_t, mconn = d["maps"][t]
                    mp[t] = (order_t, np.asarray(mconn)[sel])
        faces = host.partition_faces(part, r)
        bf = list(d.get("bfaces", [])) + [(tuple(int(v) for v in f if v >= 0), EXCHANGE_TAG)
                                          for f in faces]
        subs.append({"nodes": d["nodes"], "elements": el, "periodic": d.get("periodic", []),
                     "bfaces": bf, "maps": mp})
        ids.append(idr)
    host.close()
    return subs, ids, part


def _tags(d):
    return sorted({int(tag) for _, tag in d.get("bfaces", [])})


def exchange_bcs(bcs):
    """The boundary conditions of a part: the mesh's own plus the exchange."""
    out = dict(bcs or {})
    out[EXCHANGE_TAG] = ("exchange",)
    return out


def scatter(u, ids):
    """Per-part solutions {type: (ne_r, nupts, 5)} from a full-mesh one."""
    return [{t: u[t][idr[t]] for t in idr if len(idr[t])} for idr in ids]


def gather(parts, ids, like):
    """Full-mesh arrays from per-part ones (the inverse of scatter)."""
    out = {t: np.empty_like(like[t]) for t in like}
    for p, idr in zip(parts, ids):
        for t in idr:
            if len(idr[t]):
                out[t][idr[t]] = p[t]
    return out


__all__ = ["EXCHANGE_TAG", "split", "exchange_bcs", "scatter", "gather", "ETYPES"]
