"""ctypes binding of ``libfrgb.so`` (the C ABI declared in include/frgb.h).

Argument marshalling only: every step of the right-hand side and of the
Runge-Kutta update runs in the library's CUDA kernels.  There is no CPU
path; if the library has not been built, loading raises immediately.
"""
import ctypes as C
import os

import numpy as np

from .build import LIB

FR_OK = 0
ERRORS = {-1: "FR_EINVAL", -2: "FR_ENOMEM", -3: "FR_ECUDA", -4: "FR_EMESH",
          -5: "FR_ENONFINITE", -6: "FR_EFILTER", -7: "FR_ETIMEOUT"}
ETYPES = {"hex": 0, "pri": 1, "tet": 2}
# map nodes of curved elements per (type, map order)
MAP_NODES = {("hex", 2): 27, ("hex", 3): 64, ("pri", 2): 18, ("pri", 3): 40,
             ("tet", 2): 10, ("tet", 3): 20}
PHYSICS = {"euler": 0, "ns": 1}
PRECISION = {"fp64": 0, "fp32": 1, "mixed": 2}
VARIANTS = {"auto": 0, "dense": 1, "sumfact": 2, "sumfact_vertex": 3,
            "tensor": 4}
SCHEMES = {"rk4": 0, "rk45": 1}
BC_KIND = {"state": 0, "extrap": 1, "exchange": 2, "prescribed": 3}
VARIANT_NAMES = {v: k for k, v in VARIANTS.items()}
FR_DTYPE_F64, FR_DTYPE_F32 = 0, 1
FR_KC_COUNT = 8


class FRError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code
        self.name = ERRORS.get(code, str(code))


class EtypeDesc(C.Structure):
    _fields_ = [("etype", C.c_int), ("n_elem", C.c_int64),
                ("conn", C.POINTER(C.c_int64)), ("map_order", C.c_int),
                ("map_conn", C.POINTER(C.c_int64))]


class BCDesc(C.Structure):
    _fields_ = [("tag", C.c_int), ("kind", C.c_int),
                ("state", C.c_double * 5)]


class MeshDesc(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("nodes", C.POINTER(C.c_double)),
                ("n_etypes", C.c_int), ("etypes", C.POINTER(EtypeDesc)),
                ("order", C.c_int), ("physics", C.c_int),
                ("gamma", C.c_double), ("mu", C.c_double),
                ("prandtl", C.c_double), ("n_periodic", C.c_int),
                ("periodic", (C.c_double * 3) * 3),
                ("n_bfaces", C.c_int64),
                ("bface_nodes", C.POINTER(C.c_int64)),
                ("bface_tags", C.POINTER(C.c_int)),
                ("n_bcs", C.c_int), ("bcs", C.POINTER(BCDesc)),
                ("precision", C.c_int), ("device", C.c_int),
                ("point_family", C.c_int)]


_lib = None


def load():
    """Load the compiled library (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB):
        raise RuntimeError(
            f"CUDA library {LIB} is missing: build it with "
            "paper_2408_16509_gb300.build.build() (nvcc for sm_103a)")
    lib = C.CDLL(LIB)
    P, I, D = C.c_void_p, C.c_int, C.c_double
    sigs = {
        "fr_mesh_create": (I, [C.POINTER(MeshDesc), C.POINTER(P)]),
        "fr_mesh_destroy": (I, [P]),
        "fr_get_info": (I, [P, I, C.POINTER(C.c_int64), C.POINTER(I),
                            C.POINTER(I)]),
        "fr_get_points": (I, [P, I, P]),
        "fr_set_solution": (I, [P, I, P]),
        "fr_get_solution": (I, [P, I, P]),
        "fr_set_solution_device": (I, [P, I, P, I]),
        "fr_get_solution_device": (I, [P, I, P, I]),
        "fr_rhs": (I, [P, D, P, P]),
        "fr_stats": (I, [P, C.POINTER(Stats), I]),
        "fr_get_schedule": (I, [P, C.POINTER(Schedule)]),
        "fr_set_schedule": (I, [P, C.POINTER(Schedule)]),
        "fr_exchange_faces": (I, [P, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                  P, P, P, P]),
        "fr_exchange_setup": (I, [P, I, I, P, P, P, P, P, P, P]),
        "fr_exchange_list": (I, [P, P, C.POINTER(C.c_int64)]),
        "fr_exchange_pack": (I, [P, I, P]),
        "fr_exchange_unpack": (I, [P, I, P]),
        "fr_rk_stage": (I, [P, I, D, I, I, I]),
        "fr_set_bc_state": (I, [P, I, BC_FN, D, P]),
        "fr_probe_fma": (I, [I, I, C.c_int64, C.POINTER(D), C.POINTER(D)]),
        "fr_check_conversions": (I, [I, C.c_uint64, C.c_int64, C.POINTER(C.c_int64)]),
        "fr_get_rhs": (I, [P, I, P]),
        "fr_rk_step": (I, [P, I, D, I]),
        "fr_rk_adaptive_step": (I, [P, C.POINTER(AdaptCtl), C.POINTER(D),
                                    C.POINTER(I), C.POINTER(D)]),
        "fr_set_stream": (I, [P, P]),
        "fr_sync": (I, [P]),
        "fr_last_error": (C.c_char_p, []),
        "fr_get_operator": (I, [P, I, I, P]),
        "fr_get_metrics": (I, [P, I, P, P]),
        "fr_get_pairs": (I, [P, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
        "fr_get_adjacency": (I, [P, I, P]),
        "fr_get_boundary_points": (I, [P, P, P]),
        "fr_get_interfaces": (I, [P, P, P]),
        "fr_partition": (I, [P, I, I, P, P]),
        "fr_partition_faces": (I, [P, P, I, P, C.POINTER(C.c_int64)]),
        "fr_group_create": (I, [P, I, C.POINTER(C.c_void_p)]),
        "fr_group_destroy": (I, [P]),
        "fr_group_rhs": (I, [P]),
        "fr_group_rk_step": (I, [P, I, D, I]),
        "fr_profile_step": (I, [P, I, D, P, P]),
        "fr_set_antialias": (I, [P, I]),
        "fr_set_viscous_scheme": (I, [P, D, D]),
        "fr_set_kernel_variant": (I, [P, I]),
        "fr_get_tuning": (I, [P, C.POINTER(I), P]),
        "fr_set_solution_static": (I, [P, I, P]),
        "fr_filter_enable": (I, [P, I, C.c_int64]),
        "fr_filter_set_mlp": (I, [P, P, C.c_int64]),
        "fr_filter_stats": (I, [P, P, I]),
        "fr_filter_samples": (I, [P, P, C.c_int64, C.POINTER(C.c_int64)]),
        "fr_mlp_train": (I, [I, P, P, C.c_int64, P, I, C.c_float, P]),
        "fr_mlp_loss_grad": (I, [I, P, P, P, C.c_int64, P, P]),
        "fr_filter_last": (I, [P, I, P, P]),
        "fr_filter_solution": (I, [P, P]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc):
    if rc != FR_OK:
        raise FRError(rc, load().fr_last_error().decode())


class Stats(C.Structure):
    """fr_stats_t."""
    _fields_ = [("rhs_calls", C.c_uint64), ("rk_steps", C.c_uint64),
                ("rk_attempts", C.c_uint64), ("rk_rejected", C.c_uint64),
                ("stages", C.c_uint64), ("filtered", C.c_uint64),
                ("filter_evals", C.c_uint64), ("filter_fallbacks", C.c_uint64),
                ("predictor_used", C.c_uint64), ("ms_device", C.c_double),
                ("ms_kernel", C.c_double * FR_KC_COUNT),
                ("launches", C.c_int * FR_KC_COUNT),
                ("kernel_family", C.c_int), ("t_last", C.c_double)]


BC_FN = C.CFUNCTYPE(None, C.c_int64, C.POINTER(C.c_double), C.c_double,
                    C.POINTER(C.c_double), C.c_void_p)


class Schedule(C.Structure):
    """fr_schedule_t."""
    _fields_ = [("tile_grad", C.c_int * 3), ("tile_vol", C.c_int * 3),
                ("tensor_grad", C.c_int * 3), ("tensor_vol", C.c_int * 3),
                ("face_block", C.c_int), ("parallel_types", C.c_int),
                ("ms_default", C.c_float), ("ms_tuned", C.c_float),
                ("structured", C.c_int * 3)]


class AdaptCtl(C.Structure):
    """fr_adapt_t: tolerances and the PI controller's memory."""
    _fields_ = [("atol", C.c_double), ("rtol", C.c_double),
                ("err_prev", C.c_double), ("after_reject", C.c_int)]


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


class FRMesh:
    """A discretised mesh living on one GPU (see include/frgb.h).

    spec: dict with ``nodes``, ``elements`` ({'hex'|'pri'|'tet': conn}),
    ``periodic`` (translation vectors) and ``bfaces`` ([(node ids, tag)]).
    bcs: {tag: ('state', rho, u, v, w, p) | ('extrap',)}.
    family: hexahedron line points, 'gl' (Gauss-Legendre) or 'gll'
    (Gauss-Lobatto: flux points among the solution points).
    """

    def __init__(self, spec, order, physics="euler", gamma=1.4, mu=0.0,
                 prandtl=0.72, bcs=None, precision="fp64", device=0,
                 family="gl"):
        lib = load()
        if hasattr(spec, "as_dict"):
            spec = spec.as_dict()
        nodes = np.ascontiguousarray(spec["nodes"], np.float64)
        self._keep = [nodes]
        ets = []
        maps = spec.get("maps", {}) or {}
        for name, conn in spec["elements"].items():
            conn = np.ascontiguousarray(conn, np.int64)
            if len(conn) == 0:
                continue
            self._keep.append(conn)
            morder, mconn = maps.get(name, (1, None))
            mptr = None
            if morder >= 2:
                mconn = np.ascontiguousarray(mconn, np.int64)
                nmap = MAP_NODES.get((name, int(morder)))
                if nmap is None or mconn.shape != (len(conn), nmap):
                    raise FRError(-1, f"{name} map of order {morder}: map connectivity "
                                      f"of shape {mconn.shape}, expected ({len(conn)}, {nmap})")
                self._keep.append(mconn)
                mptr = mconn.ctypes.data_as(C.POINTER(C.c_int64))
            ets.append(EtypeDesc(ETYPES[name], len(conn),
                                 conn.ctypes.data_as(C.POINTER(C.c_int64)),
                                 int(morder), mptr))
        et_arr = (EtypeDesc * len(ets))(*ets)
        bfl = spec.get("bfaces", [])
        bnodes = np.full((max(len(bfl), 1), 4), -1, np.int64)
        btags = np.zeros(max(len(bfl), 1), np.int32)
        for i, (ids, tag) in enumerate(bfl):
            bnodes[i, :len(ids)] = ids
            btags[i] = tag
        self._keep += [bnodes, btags]
        bcs = bcs or {}
        bc_list = []
        presc = {}
        for tag, bc in bcs.items():
            st = (C.c_double * 5)(*(bc[1:6] if bc[0] == "state" else [0] * 5))
            if bc[0] == "prescribed":
                presc[int(tag)] = bc[1]
            bc_list.append(BCDesc(int(tag), BC_KIND[bc[0]], st))
        bc_arr = (BCDesc * max(len(bc_list), 1))(*bc_list)
        per = ((C.c_double * 3) * 3)()
        pv = spec.get("periodic", [])
        for i, T in enumerate(pv):
            for k in range(3):
                per[i][k] = float(T[k])
        d = MeshDesc()
        d.n_nodes = len(nodes)
        d.nodes = nodes.ctypes.data_as(C.POINTER(C.c_double))
        d.n_etypes = len(ets)
        d.etypes = et_arr
        d.order = int(order)
        d.physics = PHYSICS[physics]
        d.gamma, d.mu, d.prandtl = float(gamma), float(mu), float(prandtl)
        d.n_periodic = len(pv)
        d.periodic = per
        d.n_bfaces = len(bfl)
        d.bface_nodes = bnodes.ctypes.data_as(C.POINTER(C.c_int64))
        d.bface_tags = btags.ctypes.data_as(C.POINTER(C.c_int))
        d.n_bcs = len(bc_list)
        d.bcs = bc_arr
        d.precision = PRECISION[precision]
        d.device = int(device)
        d.point_family = {"gl": 0, "gll": 1}[family]
        h = C.c_void_p()
        _check(lib.fr_mesh_create(C.byref(d), C.byref(h)))
        self._h = h
        self._keep = None
        self.precision = precision
        self.physics = physics
        for tag, fn in presc.items():
            if device >= 0 and fn is not None:   # None: set later (set_bc_state)
                self.set_bc_state(tag, fn)
        self.types = [t for t in ("hex", "pri", "tet") if self.info(t)[0] > 0]

    def close(self):
        if getattr(self, "_h", None):
            load().fr_mesh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self, etype):
        ne, nu, nf = C.c_int64(), C.c_int(), C.c_int()
        _check(load().fr_get_info(self._h, ETYPES[etype], C.byref(ne),
                                  C.byref(nu), C.byref(nf)))
        return ne.value, nu.value, nf.value

    def points(self, etype):
        ne, nu, _ = self.info(etype)
        out = np.empty((ne, nu, 3), np.float64)
        _check(load().fr_get_points(self._h, ETYPES[etype], _ptr(out)))
        return out

    def set_solution(self, u):
        """u: {etype: (n_elem, nupts, 5) float64 host array}."""
        for t, a in u.items():
            a = np.ascontiguousarray(a, np.float64)
            _check(load().fr_set_solution(self._h, ETYPES[t], _ptr(a)))

    def get_solution(self):
        out = {}
        for t in self.types:
            ne, nu, _ = self.info(t)
            a = np.empty((ne, nu, 5), np.float64)
            _check(load().fr_get_solution(self._h, ETYPES[t], _ptr(a)))
            out[t] = a
        return out

    @staticmethod
    def _dtype(tensor):
        name = str(tensor.dtype)
        if name.endswith("float64"):
            return FR_DTYPE_F64
        if name.endswith("float32"):
            return FR_DTYPE_F32
        raise ValueError(f"unsupported dtype {tensor.dtype} (float64 or float32)")

    def set_solution_device(self, etype, tensor):
        """tensor: CUDA float64 or float32 contiguous (n_elem, nupts, 5)."""
        _check(load().fr_set_solution_device(self._h, ETYPES[etype],
                                             C.c_void_p(tensor.data_ptr()),
                                             self._dtype(tensor)))

    def get_solution_device(self, etype, tensor):
        _check(load().fr_get_solution_device(self._h, ETYPES[etype],
                                             C.c_void_p(tensor.data_ptr()),
                                             self._dtype(tensor)))

    def rhs(self, t=0.0):
        """One right-hand-side evaluation at the current solution (fr_rhs
        with a host output): {etype: (n_elem, nupts, 5) float64}."""
        sizes = [(tp,) + self.info(tp)[:2] for tp in self.types]
        flat = np.empty(sum(ne * nu * 5 for _, ne, nu in sizes), np.float64)
        _check(load().fr_rhs(self._h, float(t), _ptr(flat), None))
        out, off = {}, 0
        for tp, ne, nu in sizes:
            out[tp] = flat[off:off + ne * nu * 5].reshape(ne, nu, 5)
            off += ne * nu * 5
        return out

    def get_rhs(self):
        """The last right-hand side (fr_get_rhs)."""
        out = {}
        for t in self.types:
            ne, nu, _ = self.info(t)
            a = np.empty((ne, nu, 5), np.float64)
            _check(load().fr_get_rhs(self._h, ETYPES[t], _ptr(a)))
            out[t] = a
        return out

    def rhs_device(self, t=0.0, out=None):
        """Right-hand side on the device: into `out` (a CUDA float64 tensor of
        all types' [n_elem][nupts][5] blocks in mesh order) when given, else
        left in the library's own buffers."""
        dev = None if out is None else C.c_void_p(out.data_ptr())
        _check(load().fr_rhs(self._h, float(t), None, dev))

    def stats(self, reset=False):
        """Counters and timings (fr_stats) as a dict."""
        st = Stats()
        _check(load().fr_stats(self._h, C.byref(st), int(bool(reset))))
        names = self.KERNEL_CLASSES
        return {"rhs_calls": st.rhs_calls, "rk_steps": st.rk_steps,
                "rk_attempts": st.rk_attempts, "rk_rejected": st.rk_rejected,
                "stages": st.stages, "filtered": st.filtered,
                "filter_evals": st.filter_evals,
                "filter_fallbacks": st.filter_fallbacks,
                "predictor_used": st.predictor_used, "ms_device": st.ms_device,
                "kernel_ms": {n: st.ms_kernel[k] for k, n in enumerate(names)},
                "launches": {n: st.launches[k] for k, n in enumerate(names)},
                "kernel_family": VARIANT_NAMES.get(st.kernel_family, st.kernel_family),
                "t_last": st.t_last}

    def rk_step(self, scheme, dt, nsteps=1):
        _check(load().fr_rk_step(self._h, SCHEMES[scheme], float(dt),
                                 int(nsteps)))

    def rk_adaptive_step(self, dt, ctl):
        """One attempted adaptive RK45 step (fr_rk_adaptive_step).  `ctl` is
        an AdaptCtl, updated in place.  Returns (accepted, err, dt_next)."""
        d = C.c_double(float(dt))
        acc = C.c_int(0)
        err = C.c_double(0.0)
        _check(load().fr_rk_adaptive_step(self._h, C.byref(ctl), C.byref(d),
                                          C.byref(acc), C.byref(err)))
        return bool(acc.value), err.value, d.value

    def integrate_adaptive(self, t_end, dt, atol, rtol, max_attempts=100000):
        """Adaptive RK45 steps from t = 0 to t_end (the last step shortened
        to land on t_end).  Returns a list of (t_after, dt, accepted, err)."""
        ctl = AdaptCtl(atol, rtol, 1.0, 0)
        t, log = 0.0, []
        for _ in range(max_attempts):
            if t >= t_end - 1e-14 * max(1.0, abs(t_end)):
                break
            h = min(dt, t_end - t)
            ok, err, dt = self.rk_adaptive_step(h, ctl)
            if ok:
                t += h
            log.append((t, h, ok, err))
        return log

    KERNEL_CLASSES = ("face_ucommon", "bnd_ucommon", "grad", "face_flux",
                      "bnd_flux", "volume", "filter", "aa_flux")

    def profile_step(self, scheme, dt):
        """One RK step with per-launch CUDA events: returns
        {kernel class: (summed ms, launches)}."""
        ms = np.zeros(len(self.KERNEL_CLASSES), np.float64)
        n = np.zeros(len(self.KERNEL_CLASSES), np.int32)
        _check(load().fr_profile_step(self._h, SCHEMES[scheme], float(dt),
                                      _ptr(ms), _ptr(n)))
        return {k: (float(ms[i]), int(n[i]))
                for i, k in enumerate(self.KERNEL_CLASSES)}

    def tuning(self):
        """(active kernel family, {family: ms per tuned step})."""
        a = C.c_int()
        ms = np.zeros(5, np.float32)
        _check(load().fr_get_tuning(self._h, C.byref(a), _ptr(ms)))
        names = {v: k for k, v in VARIANTS.items()}
        return names[a.value], {names[i]: float(ms[i]) for i in range(1, 5)
                                if ms[i] > 0}

    def set_bc_state(self, tag, fn, t=0.0):
        """States of an FR_BC_PRESCRIBED condition (fr_set_bc_state):
        fn(x (n, 3), t) or fn(x) returns the primitive state (n, 5)."""
        err = []

        def cb(n, x, tt, prim, ctx):
            try:
                xs = np.ctypeslib.as_array(x, shape=(n, 3))
                try:
                    w = fn(xs.copy(), tt)
                except TypeError:
                    w = fn(xs.copy())
                np.ctypeslib.as_array(prim, shape=(n, 5))[:] = np.asarray(w, float)
            except Exception as exc:  # noqa: BLE001 - reported after the call
                err.append(exc)
                np.ctypeslib.as_array(prim, shape=(n, 5))[:] = np.nan
        cfun = BC_FN(cb)
        rc = load().fr_set_bc_state(self._h, int(tag), cfun, float(t), None)
        if err:
            raise err[0]
        _check(rc)

    def schedule(self):
        """Tiles and schedule of the kernels (fr_get_schedule): per element
        type {'grad': tile, 'vol': tile, 'tensor_grad': bool, 'tensor_vol':
        bool, 'structured': bool}, plus 'face_block', 'parallel_types',
        'ms_default', 'ms_tuned'."""
        sc = Schedule()
        _check(load().fr_get_schedule(self._h, C.byref(sc)))
        out = {"face_block": sc.face_block,
               "parallel_types": bool(sc.parallel_types),
               "ms_default": sc.ms_default, "ms_tuned": sc.ms_tuned}
        for name, k in ETYPES.items():
            if sc.tile_grad[k] >= 0:
                out[name] = {"grad": sc.tile_grad[k], "vol": sc.tile_vol[k],
                             "tensor_grad": bool(sc.tensor_grad[k]),
                             "tensor_vol": bool(sc.tensor_vol[k]),
                             "structured": bool(sc.structured[k])}
        return out

    def set_schedule(self, tiles=None, face_block=256, parallel_types=False):
        """tiles: {etype: (grad tile, vol tile)}; others keep 0 (default)."""
        sc = Schedule()
        cur = self.schedule()
        for name, k in ETYPES.items():
            if name in cur:
                g, v = (tiles or {}).get(name, (cur[name]["grad"], cur[name]["vol"]))
                sc.tile_grad[k], sc.tile_vol[k] = int(g), int(v)
        sc.face_block = int(face_block)
        sc.parallel_types = int(bool(parallel_types))
        _check(load().fr_set_schedule(self._h, C.byref(sc)))

    def set_variant(self, name):
        """Kernel family: 'auto', 'dense', 'sumfact', 'sumfact_vertex' or
        'tensor' (tensor-core prisms / tetrahedra, FP32 values)."""
        _check(load().fr_set_kernel_variant(self._h, VARIANTS[name]))

    def filter_enable(self, on=True, sample_capacity=0):
        _check(load().fr_filter_enable(self._h, int(on), int(sample_capacity)))

    def filter_set_mlp(self, params):
        if params is None:
            _check(load().fr_filter_set_mlp(self._h, None, 0))
            return
        p = np.ascontiguousarray(params, np.float32)
        _check(load().fr_filter_set_mlp(self._h, _ptr(p), len(p)))

    def filter_solution(self, smin=None):
        """smin: {etype: (n_elem,) bound} or None (bound from the state)."""
        if smin is None:
            _check(load().fr_filter_solution(self._h, None))
            return
        a = np.ascontiguousarray(
            np.concatenate([np.asarray(smin[t], np.float64)
                            for t in self.types]))
        _check(load().fr_filter_solution(self._h, _ptr(a)))

    def filter_last(self, etype="hex"):
        ne, _, _ = self.info(etype)
        z = np.zeros(ne, np.float32)
        n = np.zeros(ne, np.int32)
        _check(load().fr_filter_last(self._h, ETYPES[etype], _ptr(z), _ptr(n)))
        return z, n

    def filter_stats(self, reset=False):
        out = np.zeros(5, np.uint64)
        _check(load().fr_filter_stats(self._h, _ptr(out), int(reset)))
        return dict(zip(("filtered", "evals", "fallbacks", "samples",
                         "guessed"), (int(v) for v in out)))

    def filter_samples(self, max_samples=1 << 22):
        out = np.empty((max_samples, 5), np.float32)
        n = C.c_int64()
        _check(load().fr_filter_samples(self._h, _ptr(out), int(max_samples),
                                        C.byref(n)))
        return out[:n.value].copy()

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, a raw cudaStream_t int, or None."""
        ptr = getattr(stream, "cuda_stream", stream)
        _check(load().fr_set_stream(self._h, C.c_void_p(ptr or 0)))

    def sync(self):
        _check(load().fr_sync(self._h))

    _aa_qdeg = 0

    def set_viscous_scheme(self, beta=0.0, tau=0.0):
        """Viscous coupling: beta = tau = 0 is BR1, (0.5, 0.1) the usual LDG
        (fr_set_viscous_scheme)."""
        _check(load().fr_set_viscous_scheme(self._h, float(beta), float(tau)))

    def set_antialias(self, qdeg):
        """Anti-aliased flux (Section 3.2): transformed flux projected from a
        volume rule of degree qdeg; 0 restores collocation."""
        _check(load().fr_set_antialias(self._h, int(qdeg)))
        self._aa_qdeg = int(qdeg)

    OPS = {"M0": 0, "D": 1, "LIFT": 2, "W": 3, "upts": 4, "fpts": 5,
           "aa_qpts": 6, "aa_qwts": 7, "aa_B": 8, "aa_P": 9}

    def operator(self, etype, which):
        """Reference-element data built by the library (FR_OP_*)."""
        ne, nu, nf = self.info(etype)
        nq = (self._aa_qdeg // 2 + 1) ** 3
        shape = {"M0": (nf, nu), "D": (3, nu, nu), "LIFT": (nu, nf),
                 "W": (nu,), "upts": (nu, 3), "fpts": (nf, 3),
                 "aa_qpts": (nq, 3), "aa_qwts": (nq,), "aa_B": (nq, nu),
                 "aa_P": (nu, nq)}[which]
        out = np.empty(shape, np.float64)
        _check(load().fr_get_operator(self._h, ETYPES[etype],
                                      self.OPS[which], _ptr(out)))
        return out

    def metrics(self, etype):
        ne, nu, _ = self.info(etype)
        S = np.empty((ne, 9, nu), np.float64)
        rj = np.empty((ne, nu), np.float64)
        _check(load().fr_get_metrics(self._h, ETYPES[etype], _ptr(S),
                                     _ptr(rj)))
        return S, rj

    def pair_counts(self):
        a, b = C.c_int64(), C.c_int64()
        _check(load().fr_get_pairs(self._h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def boundary_points(self):
        """(x [nb][3], kind [nb]) of the boundary flux points."""
        _, nb = self.pair_counts()
        x = np.empty((nb, 3), np.float64)
        k = np.empty(nb, np.int32)
        _check(load().fr_get_boundary_points(self._h, _ptr(x), _ptr(k)))
        return x, k

    def interfaces(self):
        """(left, right) global element indices of every interior flux-point
        pair (fr_get_interfaces)."""
        n, _ = self.pair_counts()
        a = np.empty(n, np.int64)
        b = np.empty(n, np.int64)
        _check(load().fr_get_interfaces(self._h, _ptr(a), _ptr(b)))
        return a, b

    def n_elements(self):
        return sum(self.info(t)[0] for t in self.types)

    def exchange_faces(self):
        """This part's exchange faces (fr_exchange_faces): (points per face,
        centroids [nf][3], point positions [np][3], |S^T n~| [np])."""
        nf, npt = C.c_int64(), C.c_int64()
        _check(load().fr_exchange_faces(self._h, C.byref(nf), C.byref(npt),
                                        None, None, None, None))
        fn = np.empty(nf.value, np.int32)
        cen = np.empty((nf.value, 3), np.float64)
        px = np.empty((npt.value, 3), np.float64)
        pm = np.empty(npt.value, np.float64)
        _check(load().fr_exchange_faces(self._h, C.byref(nf), C.byref(npt),
                                        _ptr(fn), _ptr(cen), _ptr(px), _ptr(pm)))
        return fn, cen, px, pm

    def exchange_setup(self, rank, per_rank):
        """Match with the other ranks (fr_exchange_setup).  per_rank: every
        rank's exchange_faces() tuple, in rank order.  Returns the points
        exchanged with each rank."""
        nr = len(per_rank)
        fpr = np.array([len(x[0]) for x in per_rank], np.int64)
        ppr = np.array([len(x[3]) for x in per_rank], np.int64)
        fn = np.ascontiguousarray(np.concatenate([x[0] for x in per_rank]), np.int32)
        cen = np.ascontiguousarray(np.concatenate([np.reshape(x[1], (-1, 3)) for x in per_rank]))
        px = np.ascontiguousarray(np.concatenate([np.reshape(x[2], (-1, 3)) for x in per_rank]))
        pm = np.ascontiguousarray(np.concatenate([x[3] for x in per_rank]), np.float64)
        counts = np.zeros(nr, np.int64)
        _check(load().fr_exchange_setup(self._h, int(rank), nr, _ptr(fpr), _ptr(ppr),
                                        _ptr(fn), _ptr(cen), _ptr(px), _ptr(pm),
                                        _ptr(counts)))
        return counts

    def exchange_list(self):
        """Boundary-point indices of the exchanged points in message order."""
        n = C.c_int64()
        _check(load().fr_exchange_list(self._h, None, C.byref(n)))
        out = np.empty(n.value, np.int32)
        _check(load().fr_exchange_list(self._h, _ptr(out), C.byref(n)))
        return out

    def exchange_pack(self, what, tensor):
        """Gather the traces of kind what (0 solution, 1 gradient) into a
        CUDA tensor [n][nv] on the handle's stream."""
        _check(load().fr_exchange_pack(self._h, int(what), C.c_void_p(tensor.data_ptr())))

    def exchange_unpack(self, what, tensor):
        _check(load().fr_exchange_unpack(self._h, int(what), C.c_void_p(tensor.data_ptr())))

    def rk_stage(self, scheme, dt, stage, phase, part=0):
        """One phase of one RK stage (fr_rk_stage); part 1 interior, 2
        exchange-adjacent, 0 both."""
        _check(load().fr_rk_stage(self._h, SCHEMES[scheme], float(dt), int(stage),
                                  int(phase), int(part)))

    def adjacency(self, etype):
        """[ne][nfaces] global index of the neighbour across each face, -1
        on a boundary (fr_get_adjacency)."""
        ne = self.info(etype)[0]
        nf = {"hex": 6, "pri": 5, "tet": 4}[etype]
        out = np.empty((ne, nf), np.int64)
        _check(load().fr_get_adjacency(self._h, ETYPES[etype], _ptr(out)))
        return out

    def partition(self, nparts, mode="weighted", weights=None):
        """Part of every element (global index order) by recursive
        coordinate bisection; mode 'weighted' (weights per type hex, pri,
        tet) or 'balanced' (fr_partition)."""
        part = np.empty(self.n_elements(), np.int32)
        w = None if weights is None else np.ascontiguousarray(weights, np.float64)
        _check(load().fr_partition(self._h, int(nparts), {"weighted": 0, "balanced": 1}[mode],
                                   None if w is None else _ptr(w), _ptr(part)))
        return part

    def partition_faces(self, part, rank):
        """Node ids [n][4] of the faces of part `rank` that border another
        part (fr_partition_faces)."""
        part = np.ascontiguousarray(part, np.int32)
        n = C.c_int64()
        _check(load().fr_partition_faces(self._h, _ptr(part), int(rank), None, C.byref(n)))
        out = np.empty((n.value, 4), np.int64)
        if n.value:
            _check(load().fr_partition_faces(self._h, _ptr(part), int(rank), _ptr(out),
                                             C.byref(n)))
        return out


class FRGroup:
    """Partitions of one mesh run together on one device (fr_group_*): the
    right-hand side and RK steps of the whole mesh, with the traces of
    exchange faces pushed between the members at every coupling point."""

    def __init__(self, members):
        self.members = list(members)
        arr = (C.c_void_p * len(self.members))(*[m._h for m in self.members])
        h = C.c_void_p()
        _check(load().fr_group_create(arr, len(self.members), C.byref(h)))
        self._h = h

    def rhs(self):
        _check(load().fr_group_rhs(self._h))
        return [m.get_rhs() for m in self.members]

    def rk_step(self, scheme, dt, nsteps=1):
        _check(load().fr_group_rk_step(self._h, SCHEMES[scheme], float(dt), int(nsteps)))

    def close(self):
        if getattr(self, "_h", None):
            load().fr_group_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def probe_fma(dtype="fp64", iters=None, device=0):
    """Fused multiply-add throughput of the device (fr_probe_fma): returns
    (TFLOP/s, ms, flops) of one timed launch."""
    code = {"fp64": FR_DTYPE_F64, "fp32": FR_DTYPE_F32}[dtype]
    if iters is None:
        iters = 20000 if dtype == "fp64" else 400000
    ms, fl = C.c_double(), C.c_double()
    _check(load().fr_probe_fma(int(device), code, int(iters), C.byref(ms),
                               C.byref(fl)))
    return fl.value / (ms.value * 1e-3) / 1e12, ms.value, fl.value


def check_conversions(n, seed=1, device=0):
    """Number of the n seeded patterns on which the library's FP32 <-> FP64
    conversions differ from the hardware's (fr_check_conversions)."""
    bad = C.c_int64()
    _check(load().fr_check_conversions(int(device), int(seed), int(n), C.byref(bad)))
    return bad.value


def mlp_train(x, zstar, params, epochs, lr, device=0):
    """Train the filter-strength predictor on the GPU (fr_mlp_train)."""
    x = np.ascontiguousarray(x, np.float32)
    z = np.ascontiguousarray(zstar, np.float32)
    p = np.ascontiguousarray(params, np.float32).copy()
    hist = np.zeros(epochs, np.float32)
    _check(load().fr_mlp_train(int(device), _ptr(x), _ptr(z), len(z), _ptr(p),
                               int(epochs), float(lr), _ptr(hist)))
    return p, hist


def mlp_loss_grad(params, x, zstar, device=0):
    """Loss and gradient of the predictor objective on the GPU."""
    x = np.ascontiguousarray(x, np.float32)
    z = np.ascontiguousarray(zstar, np.float32)
    p = np.ascontiguousarray(params, np.float32)
    loss = np.zeros(1, np.float32)
    g = np.zeros(len(p), np.float32)
    _check(load().fr_mlp_loss_grad(int(device), _ptr(p), _ptr(x), _ptr(z),
                                   len(z), _ptr(loss), _ptr(g)))
    return float(loss[0]), g
