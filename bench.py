#!/usr/bin/env python
"""Benchmark: FR right-hand side + RK update throughput on one GB300.

Workload (the Navier-Stokes Taylor-Green vortex of the paper's Section 5
in the mixed-precision configuration, the largest that fits one GPU):
periodic [0, 2 pi]^3 box of 48^3 hexahedra whose interior nodes are
perturbed by up to 10% of the spacing (seed 20240829), p = 4 (125
Gauss-Legendre solution points per element, 13.8 M points), Re = 1600,
Ma = 0.1, Pr = 0.71, constant viscosity, BR1 gradients, Rusanov inviscid
flux, RK4(3)5[2R+] with dt = 2.5e-4 (1e-3 exceeds the explicit limit at
this h and p).  A "step" is one RK step (five right-hand-side stages).
Metric: GDOF-stage/s = solution points x 5 variables x stages / s / 1e9.
The headline value is the plain FP64 form; the mixed form (FP32 values,
FP64 RK registers) and the FP32 form are reported beside it with their
relative L2 error per conserved variable against the FP64 form after the
same steps.

--impl reference times the CPU FP64 oracle (plain numpy) on the same
workload, on bounded samples (4^3-element boxes of the same shape), one
single-threaded replica per host core.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_CELLS = 48
ORDER = 4
RE, MACH, PR = 1600.0, 0.1, 0.71
DT = 2.5e-4
STAGES = 5
SAMPLE_CELLS = 4     # per direction, CPU oracle samples
# the Navier-Stokes TGV at one-GPU size of the paper's subsonic case
C2_CELLS, C2_ORDER, C2_DT = 32, 3, 1e-3
L2_BYTES = 129e6


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ workload
def workload_spec(n):
    from frinputs import box_hex
    return box_hex((n, n, n), hi=(2 * np.pi,) * 3, perturb=0.1)


def tgv(x):
    from frinputs import ics
    return ics.taylor_green(x, mach=MACH)


def config(precision):
    nu = (ORDER + 1) ** 3
    return {"workload": f"ns-tgv-hex{N_CELLS}^3-p{ORDER}-rk45",
            "elements": N_CELLS ** 3, "order": ORDER,
            "solution_points": N_CELLS ** 3 * nu,
            "physics": "navier-stokes BR1 + Rusanov", "scheme": "RK4(3)5[2R+]",
            "dt": DT, "re": RE, "mach": MACH, "precision": precision,
            "mesh_perturbation": 0.1,
            "l2": f"inputs larger than L2 (state register "
                  f"{N_CELLS ** 3 * nu * 5 * 8 / 1e6:.0f} MB in FP64, step working "
                  f"set > 5 GB); no flush"}


# ------------------------------------------------------ byte/flop models
def kernel_models(nu, nf, ne, w, wr, npair):
    """Algorithmic DRAM bytes and floating-point operations per launch of
    each kernel class for an RK4(3)5[2R+] stage i > 0 of the Navier-Stokes
    right-hand side on hexahedra (sum-factorised operators), N = p + 1.
    w: bytes of a trace/stage value, wr: bytes of a solution register."""
    n = round(nu ** (1.0 / 3.0))
    # FP64 values: 15 gradient components per flux point go to the face
    # kernel; FP32 values: 5 viscous normal-flux values q per flux point
    # (plus the 5 solution traces the grad kernel reads to form q)
    gf = 15 if w == 8 else 10
    bytes_ = {
        # u(5) + metrics(10) + du(5 per flux pt) in, grad(15) + gradf out
        "grad": ne * (w * (5 * nu + 10 * nu + 5 * nf + 15 * nu + gf * nf)),
        # u(5) + grad(15) + metrics(10) + F^C(5/fpt) in; Y and u_f out;
        # solution register X in and out
        "volume": ne * (w * (5 * nu + 15 * nu + 10 * nu + 5 * nf + 5 * nu
                             + 5 * nf) + wr * 10 * nu),
        "face_ucommon": npair * (w * 20 + 8),
        "face_flux": npair * (w * (2 * (20 if w == 8 else 10) + 5 + 10) + 8),
    }
    flops = {
        "grad": ne * (2 * nu * (15 * n + 30 + 45) + 15 * nu
                      + 2 * nf * 15 * n),
        "volume": ne * (nu * (30 + 150 + 90 + 2 * 5 * (3 * n + 6) + 25)
                        + 2 * nf * 5 * n + 5 * nf + 2 * nf * 5 * n),
        "face_ucommon": npair * 10,
        "face_flux": npair * 330,
    }
    return bytes_, flops


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of a dominant
# kernel per element and launch, from one ncu capture on a smaller case of the
# same kernel (inputs well above L2, so traffic grows with the elements) and
# scaled by the elements of a launch.  Keyed by (kernel class, precision,
# order); each entry records the sha256 of the library's CUDA sources the
# capture ran, and the bench reports it only while they are unchanged (a
# changed kernel reports null), with the profile that holds the capture.
TRAFFIC = {
    # k_hex_vol<double, double, 5, 2, NS>: 32^3 elements, p = 4, two launches
    ("volume", "fp64", 4): (53324.6,
                           "686cfcca827c9ddaf043d9eaa9600573a3627d36daac1e196544fe4da21f742b",
                           "profiles/k_hex_vol_fp64_tgv32_p4_traffic.md"),
}


def _sources_sha():
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2408_16509_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh", ".inc")):
            with open(os.path.join(d, f), "rb") as fh:
                h.update(f.encode())
                h.update(fh.read())
    return h.hexdigest()


def traffic_of(kernel, precision, p, ne):
    """(bytes per launch, profile) of a recorded capture, or (None, why)."""
    rec = TRAFFIC.get((kernel, precision, p))
    if rec is None:
        return None, "no capture recorded for this kernel"
    per_elem, sha, prof = rec
    if sha != _sources_sha():
        return None, "kernel sources changed since " + prof
    return per_elem * ne, prof


def roofline(prof, models, peaks, src, precision, alu, order=None, ne=None):
    """Roofline record of the dominant kernel class: the bound is whichever
    of DRAM bytes / HBM peak and flops / arithmetic peak takes longer.
    alu: {"fp64": (TFLOP/s, source), "fp32": (...)} measured in this run."""
    bytes_, flops = models
    dom = max((k for k in prof if prof[k][1] > 0), key=lambda k: prof[k][0])
    t = prof[dom][0] / prof[dom][1] * 1e-3
    b, f = bytes_.get(dom), flops.get(dom)
    bw = b / t / 1e9 if b else None
    fl = f / t / 1e12 if f else None
    fpeak, fsrc = alu["fp64" if precision == "fp64" else "fp32"]
    t_mem = b / (peaks["hbm_gbs"] * 1e9) if b else 0.0
    t_alu = f / (fpeak * 1e12) if f else 0.0
    if t_alu > t_mem:
        out = {"kernel": dom, "bound": "alu", "achieved": fl, "peak": fpeak,
               "unit": "TFLOP/s", "frac": fl / fpeak, "peak_source": fsrc}
    else:
        out = {"kernel": dom, "bound": "hbm", "achieved": bw,
               "peak": peaks["hbm_gbs"], "unit": "GB/s",
               "frac": bw / peaks["hbm_gbs"],
               "peak_source": src + " hbm_gbs (MEASURED_PEAKS.json), burst copy"}
    out["traffic"], out["traffic_source"] = (
        traffic_of(dom, precision, order, ne) if ne else (None, "not recorded"))
    out.update({"launches_per_step": prof[dom][1], "kernel_ms": t * 1e3,
                "algorithmic_bytes": b, "algorithmic_flops": f,
                "achieved_gbs": bw, "achieved_tflops": fl,
                "attainable_ms": max(t_mem, t_alu) * 1e3})
    return out


def alu_peaks(fr, device):
    """FMA throughput of this GPU in FP64 and FP32 (fr_probe_fma, CUDA
    events), with the SM clocks sampled during the probes."""
    sampler = ClockSampler(device)
    sampler.start()
    out = {}
    for dt in ("fp64", "fp32"):
        best = max(fr.probe_fma(dt, device=device)[0] for _ in range(3))
        out[dt] = (best, f"fr_probe_fma {dt} FMA chains, best of 3 launches, this run")
    clocks = sampler.stop()
    return out, clocks


# ------------------------------------------------------------ our arm
def aggregate(ms_local, units_local, dist=None, device="cpu"):
    """Whole-job figures over ranks running independent replicas: the
    slowest rank's time and the units processed by all ranks."""
    if dist is None:
        return float(ms_local), float(units_local)
    import torch
    mx = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    sm = torch.tensor([float(units_local)], dtype=torch.float64, device=device)
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx.item()), float(sm.item())



METRIC = "GDOF-stage/s per GB300 (plain FP64 vs mixed-prec/batched) at stated L2 error"


def measure(fr, torch, precision, steps, warmup, device, dist, n=None,
            order=ORDER, dt=DT):
    spec = workload_spec(n or N_CELLS)
    mesh = fr.FRMesh(spec, order, physics="ns", gamma=1.4, mu=1.0 / RE,
                     prandtl=PR, precision=precision, device=device)
    stream = torch.cuda.Stream(device=device)
    mesh.set_stream(stream)
    x = mesh.points("hex")
    ne, nu, nf = mesh.info("hex")
    u0 = tgv(x.reshape(-1, 3)).reshape(ne, nu, 5)
    mesh.set_solution({"hex": u0})
    for _ in range(warmup):             # the first one tunes and builds the graph
        mesh.rk_step("rk45", dt, 1)
    mesh.set_solution({"hex": u0})
    sampler = ClockSampler(device)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    mesh.rk_step("rk45", dt, steps)
    t1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = t0.elapsed_time(t1)
    ms, units = aggregate(ms, ne * nu * 5 * STAGES * steps, dist, "cuda")
    if dist:
        dist.barrier()
    final = mesh.get_solution()["hex"]
    tuning = mesh.tuning()
    prof = {}
    reps = 3
    for _ in range(reps):
        for k, (t, c) in mesh.profile_step("rk45", dt).items():
            a = prof.setdefault(k, [0.0, 0])
            a[0] += t / reps
            a[1] = c
    return {"mesh": mesh, "u0": u0, "ms": ms, "clocks": clocks, "prof": prof,
            "final": final, "tuning": tuning, "units": units,
            "schedule": mesh.schedule()}


def _rel_l2_arrays(a, b):
    """Per conserved variable: ||a - b|| / max(||b||, ||rho_b||)."""
    d = (a - b).reshape(-1, 5)
    r = b.reshape(-1, 5)
    den = np.maximum(np.linalg.norm(r, axis=0), np.linalg.norm(r[:, 0]))
    return (np.linalg.norm(d, axis=0) / den).tolist()


def _e2e(fr, torch, mesh, u0, steps, world, dist, warmup=3):
    """Same metric through the C ABI with host buffers: every step copies
    the state in from pinned memory, runs one RK step and copies it out."""
    import ctypes
    lib = fr.load()
    host_in = torch.from_numpy(np.ascontiguousarray(u0)).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    hin, hout = host_in.numpy(), host_out.numpy()
    ne, nu, _ = mesh.info("hex")
    e2e_steps = max(3, min(steps, 10))
    # untimed passes first (at least as many as the warm-up steps, at least
    # 3, and at least 1 s of them): the first passes through freshly pinned
    # buffers copy 553 MB (48^3, p = 4) in 26-30 ms each way instead of 3
    t0, n = time.perf_counter(), 0
    while n < max(3, warmup) or time.perf_counter() - t0 < 1.0:
        rc = lib.fr_set_solution(mesh._h, 0, hin.ctypes.data_as(ctypes.c_void_p))
        rc |= lib.fr_rk_step(mesh._h, 1, DT, 1)
        rc |= lib.fr_get_solution(mesh._h, 0, hout.ctypes.data_as(ctypes.c_void_p))
        if rc:
            raise RuntimeError(lib.fr_last_error().decode())
        n += 1
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    for _ in range(e2e_steps):
        rc = lib.fr_set_solution(mesh._h, 0, hin.ctypes.data_as(ctypes.c_void_p))
        rc |= lib.fr_rk_step(mesh._h, 1, DT, 1)
        rc |= lib.fr_get_solution(mesh._h, 0, hout.ctypes.data_as(ctypes.c_void_p))
        if rc:
            raise RuntimeError(lib.fr_last_error().decode())
    e2e_s = time.perf_counter() - w0
    if dist:
        tt = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_s = float(tt.item())
    val = ne * nu * 5 * STAGES * e2e_steps * world / e2e_s / 1e9
    return {"value": val, "unit": "GDOF-stage/s",
            "h2d_bytes_per_step": int(hin.nbytes),
            "d2h_bytes_per_step": int(hout.nbytes), "steps": e2e_steps}


def run_ours(args):
    import torch

    import paper_2408_16509_gb300 as fr

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    fr.build()
    peaks, src = _peaks()
    alu, probe_clocks = alu_peaks(fr, local)
    r = measure(fr, torch, args.precision, args.steps, args.warmup, local, dist)
    mesh, prof, ms = r["mesh"], r["prof"], r["ms"]
    ne, nu, nf = mesh.info("hex")
    value = r["units"] / (ms * 1e-3) / 1e9     # all replicas / slowest rank
    launches_per_step = sum(c for _, c in prof.values())
    e2e = _e2e(fr, torch, mesh, r["u0"], args.steps, world, dist, args.warmup)
    npair, _ = mesh.pair_counts()

    def widths(prec):
        return (8 if prec == "fp64" else 4), (4 if prec == "fp32" else 8)
    w, wr = widths(args.precision)
    order = round(nu ** (1.0 / 3.0)) - 1
    roof = roofline(prof, kernel_models(nu, nf, ne, w, wr, npair), peaks, src,
                    args.precision, alu, order, ne)
    line = {
        "metric": METRIC,
        "value": value, "unit": "GDOF-stage/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp32": "f32",
                  "mixed": "f32 (f64 RK registers)"}[args.precision],
        "data": "synthetic (seeded perturbed mesh, analytic TGV state)",
        "config": config(args.precision),
        "clocks": r["clocks"],
        "e2e": e2e,
        "gpu_launches": launches_per_step * args.steps,
        "kernel_ms_per_step": {k: v[0] for k, v in prof.items() if v[1]},
        "kernel_family": {"active": r["tuning"][0],
                          "tuned_ms_per_step": r["tuning"][1],
                          "schedule": r["schedule"]},
        "roofline": roof,
        "alu_probe": {"fp64_tflops": alu["fp64"][0], "fp32_tflops": alu["fp32"][0],
                      "clocks": probe_clocks},
        "l2_error": {args.precision: "reference form of this line; parity with the "
                     "FP64 oracle is gated per variable in the -m gpu tests"},
    }
    ref_final = r["final"] if args.precision == "fp64" else None
    mesh.close()
    if args.variants and world == 1:
        line["variants"] = {}
        finals = {}
        for prec in ("fp64", "mixed", "fp32"):
            if prec == args.precision:
                continue
            v = measure(fr, torch, prec, args.steps, args.warmup, local, None)
            finals[prec] = v["final"]
            w2, wr2 = widths(prec)
            line["variants"][prec] = {
                "value": v["units"] / (v["ms"] * 1e-3) / 1e9,
                "ms_per_step": v["ms"] / args.steps,
                "roofline": roofline(
                    v["prof"], kernel_models(nu, nf, ne, w2, wr2, npair), peaks,
                    src, prec, alu, order, ne),
                "kernel_ms_per_step": {k: x[0] for k, x in v["prof"].items() if x[1]},
                "kernel_family": {"active": v["tuning"][0],
                                  "tuned_ms_per_step": v["tuning"][1],
                                  "schedule": v["schedule"]},
                "clocks": v["clocks"]}
            v["mesh"].close()
        if ref_final is None and "fp64" in finals:
            ref_final = finals["fp64"]
        if ref_final is not None:
            for prec, fin in finals.items():
                if prec == "fp64":
                    continue
                err = _rel_l2_arrays(fin, ref_final)
                line["variants"][prec]["rel_l2_vs_fp64"] = err
                line["l2_error"][prec] = {
                    "rel_l2_per_variable_vs_fp64_after_steps": err,
                    "steps": args.steps, "tolerance": 1e-5}
    if args.configs and world == 1:
        line["configs"] = other_configs(fr, torch, local)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# ------------------------------------------------------- other workloads
def _timed_steps(torch, mesh, stream, scheme, dt, steps):
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(stream)
    mesh.rk_step(scheme, dt, steps)
    t1.record(stream)
    torch.cuda.synchronize()
    return t0.elapsed_time(t1)


def _gdofs(mesh, stages, steps, ms):
    pts = sum(mesh.info(t)[0] * mesh.info(t)[1] for t in mesh.types)
    return pts * 5 * stages * steps / (ms * 1e-3) / 1e9


def _state(mesh, fn):
    out = {}
    for t in mesh.types:
        x = mesh.points(t)
        out[t] = fn(x.reshape(-1, 3)).reshape(x.shape[0], x.shape[1], 5)
    return out


def _rel_l2(a, b):
    num = np.zeros(5)
    den = np.zeros(5)
    rho = 0.0
    for t in b:
        d = (a[t] - b[t]).reshape(-1, 5)
        r = b[t].reshape(-1, 5)
        num += (d * d).sum(0)
        den += (r * r).sum(0)
        rho += (r[:, 0] ** 2).sum()
    return (np.sqrt(num) / np.maximum(np.sqrt(den), np.sqrt(rho))).tolist()


def config_vortex(fr, torch, device):
    """Isentropic vortex, 8^3 hexes on [0,10]^3, p=2, Euler, RK4,
    dt 0.01 x 100, FP64; error against the closed form."""
    from frinputs import box_hex, ics
    mesh = fr.FRMesh(box_hex((8, 8, 8), hi=(10.0, 10.0, 10.0)), 2,
                     physics="euler", device=device)
    st = torch.cuda.Stream(device=device)
    mesh.set_stream(st)
    mesh.set_solution(_state(mesh, ics.isentropic_vortex))
    mesh.rk_step("rk4", 0.01, 3)
    mesh.set_solution(_state(mesh, ics.isentropic_vortex))
    ms = _timed_steps(torch, mesh, st, "rk4", 0.01, 100)
    exact = _state(mesh, lambda x: ics.isentropic_vortex(x, t=1.0))
    err = _rel_l2(mesh.get_solution(), exact)
    out = {"gdof_stage_s": _gdofs(mesh, 4, 100, ms), "ms_per_step": ms / 100,
           "rel_l2_vs_closed_form_t1": err, "precision": "fp64"}
    mesh.close()
    return out


def config_tgv_adaptive(fr, torch, device, attempts=30):
    """TGV 32^3 p=3 (the bench workload) in FP32 with adaptive RK45 steps
    (Section 3.5): atol = rtol = 1e-6 from dt = 1e-3.  Every attempt is one
    graph (stages + embedded error + norm) plus the host's accept / reject
    decision; the time covers all attempts, rejected ones included."""
    spec = workload_spec(C2_CELLS)
    mesh = fr.FRMesh(spec, C2_ORDER, physics="ns", gamma=1.4, mu=1.0 / RE,
                     prandtl=PR, precision="fp32", device=device)
    st = torch.cuda.Stream(device=device)
    mesh.set_stream(st)
    mesh.set_solution(_state(mesh, tgv))
    mesh.rk_step("rk45", 1e-3, 2)     # tuning and warm-up
    ctl = fr.AdaptCtl(1e-6, 1e-6, 1.0, 0)
    dt, log = 1e-3, []
    for _ in range(3):                # warm-up attempts (graph build)
        ok, err, dt = mesh.rk_adaptive_step(dt, ctl)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(st)
    for _ in range(attempts):
        h = dt
        ok, err, dt = mesh.rk_adaptive_step(h, ctl)
        log.append((ok, err, h))
    t1.record(st)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    fixed = _timed_steps(torch, mesh, st, "rk45", 1e-4, attempts)
    acc = [x for x in log if x[0]]
    out = {"attempts": attempts, "accepted": len(acc),
           "rejected": attempts - len(acc),
           "ms_per_attempt": ms / attempts,
           "ms_per_fixed_step": fixed / attempts,
           "gdof_stage_s": _gdofs(mesh, 5, attempts, ms),
           "dt_first_last": [log[0][2], log[-1][2]],
           "err_mean_accepted": float(np.mean([x[1] for x in acc])) if acc else None,
           "tolerance": 1e-6}
    mesh.close()
    return out


def config_tgv32(fr, torch, device, steps=20):
    """TGV on 32^3 perturbed hexes, p=3, RK45 dt 1e-3: FP64, FP32 and
    mixed, the reduced forms against the FP64 form after the same steps."""
    out, fin = {}, {}
    for prec in ("fp64", "fp32", "mixed"):
        r = measure(fr, torch, prec, steps, 3, device, None, n=C2_CELLS,
                    order=C2_ORDER, dt=C2_DT)
        fin[prec] = r["final"]
        ne, nu, _ = r["mesh"].info("hex")
        out[prec] = {"gdof_stage_s": r["units"] / (r["ms"] * 1e-3) / 1e9,
                     "ms_per_step": r["ms"] / steps,
                     "kernel_family": r["tuning"][0],
                     "kernel_ms_per_step": {k: v[0] for k, v in r["prof"].items() if v[1]}}
        r["mesh"].close()
    for prec in ("fp32", "mixed"):
        out[prec]["rel_l2_vs_fp64_after_steps"] = _rel_l2_arrays(fin[prec], fin["fp64"])
    out["steps"] = steps
    return out


def config_mixed_elements(fr, torch, device, steps=20, cells=40, variant="auto",
                          qdeg=0):
    """40^3 cells: hexes x < 0.5, 2 prisms per cell 0.5 <= x < 0.8, 6 tets
    x >= 0.8 (5% jitter), p=3, NS Re 1000, Ma 0.2, RK4, FP32.  `cells` and
    `variant` (kernel family) serve profiling runs (--only mixed)."""
    from frinputs import ics, mixed_box
    spec = mixed_box(n=cells)
    pinf = 1.0 / (1.4 * 0.04)
    far = ("state", 1.0, 1.0, 0.0, 0.0, pinf)
    mesh = fr.FRMesh(spec, 3, physics="ns", mu=1e-3, prandtl=PR,
                     bcs={0: far, 1: far, 2: far, 3: far}, precision="fp32",
                     device=device)
    st = torch.cuda.Stream(device=device)
    mesh.set_stream(st)
    mesh.set_variant(variant)
    if qdeg:
        mesh.set_antialias(qdeg)
    mesh.set_solution(_state(mesh, lambda x: ics.perturbed_uniform(x)))
    mesh.rk_step("rk4", 2e-4, 2)
    ms = _timed_steps(torch, mesh, st, "rk4", 2e-4, steps)
    prof = mesh.profile_step("rk4", 2e-4)
    active, tuned = mesh.tuning()
    out = {"gdof_stage_s": _gdofs(mesh, 4, steps, ms), "ms_per_step": ms / steps,
           "elements": {t: mesh.info(t)[0] for t in mesh.types},
           "schedule": mesh.schedule(),
           "kernel_ms_per_step": {k: v[0] for k, v in prof.items() if v[1]},
           "kernel_family": {"active": active, "tuned_ms_per_step": tuned}}
    mesh.close()
    return out


def config_tgv_curved(fr, torch, device, steps=10, precisions=("fp64", "fp32")):
    """TGV on 32^3 curved hexahedra (quadratic maps, Section 3.4; nodes moved
    by 5% of the cell size in a smooth field) on [0, 2 pi]^3, p=3, NS Re
    1600, RK45 dt 1e-3: FP64 and FP32 beside the straight-element workload.
    Curved elements run the table-metric families only."""
    from frinputs import curved_box_hex
    t_setup = time.perf_counter()
    spec = curved_box_hex((C2_CELLS,) * 3, hi=(2 * np.pi,) * 3)
    out = {}
    for prec in precisions:
        t0 = time.perf_counter()
        mesh = fr.FRMesh(spec, C2_ORDER, physics="ns", gamma=1.4, mu=1.0 / RE,
                         prandtl=PR, precision=prec, device=device)
        setup_s = time.perf_counter() - t0
        st = torch.cuda.Stream(device=device)
        mesh.set_stream(st)
        u0 = _state(mesh, tgv)
        mesh.set_solution(u0)
        mesh.rk_step("rk45", 1e-3, 2)
        mesh.set_solution(u0)
        ms = _timed_steps(torch, mesh, st, "rk45", 1e-3, steps)
        active, _ = mesh.tuning()
        out[prec] = {"gdof_stage_s": _gdofs(mesh, 5, steps, ms),
                     "ms_per_step": ms / steps, "kernel_family": active,
                     "mesh_setup_s": setup_s}
        mesh.close()
    out["spec_s"] = time.perf_counter() - t_setup
    return out


def config_tgv_antialias(fr, torch, device, steps=10, qdeg=9,
                         precisions=("fp64", "fp32")):
    """TGV 32^3 p=3 (the bench workload) with the anti-aliased flux of
    Section 3.2: transformed flux at the 125 points of a degree-9 Gauss rule,
    projected back by least squares.  FP64 and FP32, beside collocation."""
    spec = workload_spec(C2_CELLS)
    out = {"qdeg": qdeg}
    for prec in precisions:
        mesh = fr.FRMesh(spec, C2_ORDER, physics="ns", gamma=1.4, mu=1.0 / RE,
                         prandtl=PR, precision=prec, device=device)
        mesh.set_antialias(qdeg)
        st = torch.cuda.Stream(device=device)
        mesh.set_stream(st)
        u0 = _state(mesh, tgv)
        mesh.set_solution(u0)
        mesh.rk_step("rk45", 1e-3, 2)
        mesh.set_solution(u0)
        ms = _timed_steps(torch, mesh, st, "rk45", 1e-3, steps)
        prof = mesh.profile_step("rk45", 1e-3)
        active, _ = mesh.tuning()
        out[prec] = {"gdof_stage_s": _gdofs(mesh, 5, steps, ms),
                     "ms_per_step": ms / steps, "kernel_family": active,
                     "kernel_ms_per_step": {k: v[0] for k, v in prof.items() if v[1]}}
        mesh.close()
    return out


def config_tgv_partitioned(fr, torch, device, steps=10, parts=(2, 4),
                           precisions=("fp64", "fp32")):
    """TGV 32^3 p=3 (the bench workload) split by recursive coordinate
    bisection into 2 and 4 parts that run as one group on this GPU: each
    stage pushes the exchange faces' solution traces, then the gradient
    traces (FP64) or viscous normal fluxes (FP32), into the partners'
    receive buffers.  Against the unpartitioned mesh: the cost of the
    decomposition and exchange, and the difference after the steps."""
    from paper_2408_16509_gb300 import partition
    spec = workload_spec(C2_CELLS)
    out = {}
    for prec in precisions:
        kw = dict(physics="ns", gamma=1.4, mu=1.0 / RE, prandtl=PR,
                  precision=prec, device=device)
        whole = fr.FRMesh(spec, C2_ORDER, **kw)
        whole.set_variant("sumfact")
        st = torch.cuda.Stream(device=device)
        whole.set_stream(st)
        u0 = _state(whole, tgv)
        whole.set_solution(u0)
        whole.rk_step("rk45", 1e-3, 2)
        whole.set_solution(u0)
        ms_whole = _timed_steps(torch, whole, st, "rk45", 1e-3, steps)
        ref = whole.get_solution()
        rec = {"whole_ms_per_step": ms_whole / steps}
        for k in parts:
            subs, ids, _ = partition.split(spec, k, "weighted")
            members = []
            for sp in subs:
                g = fr.FRMesh(sp, C2_ORDER, bcs=partition.exchange_bcs({}), **kw)
                g.set_variant("sumfact")
                g.set_stream(st)
                members.append(g)
            grp = fr.FRGroup(members)
            for g, ur in zip(members, partition.scatter(u0, ids)):
                g.set_solution(ur)
            grp.rk_step("rk45", 1e-3, 2)
            for g, ur in zip(members, partition.scatter(u0, ids)):
                g.set_solution(ur)
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            t0.record(st)
            grp.rk_step("rk45", 1e-3, steps)
            t1.record(st)
            torch.cuda.synchronize()
            ms = t0.elapsed_time(t1)
            got = partition.gather([g.get_solution() for g in members], ids, ref)
            nb = [g.pair_counts()[1] for g in members]
            rec[f"{k}_parts"] = {
                "ms_per_step": ms / steps,
                "gdof_stage_s": _gdofs(whole, 5, steps, ms),
                "exchange_points": int(sum(nb)),
                "rel_l2_vs_whole": _rel_l2(got, ref)}
            grp.close()
            for g in members:
                g.close()
        whole.close()
        out[prec] = rec
    return out


def config_shu_osher(fr, torch, device, steps=40):
    """256x8x8 hexes on [-5,5]x[0,0.3125]^2, p=3, Euler, RK4 dt 9e-4, FP32,
    entropy filter: plain root-find, then the predictor trained on the
    run's own filter solves."""
    from frinputs import box_hex, ics
    post = ics.SHU_OSHER_POST
    spec = box_hex((256, 8, 8), lo=(-5.0, 0, 0), hi=(5.0, 0.3125, 0.3125),
                   periodic=(1, 2))
    bcs = {0: ("state", post[0], post[1], 0.0, 0.0, post[2]), 1: ("extrap",)}
    mesh = fr.FRMesh(spec, 3, physics="euler", bcs=bcs, precision="fp32",
                     device=device)
    st = torch.cuda.Stream(device=device)
    mesh.set_stream(st)
    mesh.set_solution(_state(mesh, ics.shu_osher))
    mesh.filter_enable(True, sample_capacity=1 << 20)
    mesh.filter_solution()
    mesh.filter_samples()
    mesh.rk_step("rk4", 9e-4, 40)            # warm-up and training data
    samp = mesh.filter_samples()
    start = mesh.get_solution()
    mesh.filter_stats(reset=True)
    ms_plain = _timed_steps(torch, mesh, st, "rk4", 9e-4, steps)
    plain = mesh.filter_stats(reset=True)
    prof = mesh.profile_step("rk4", 9e-4)
    mesh.filter_stats(reset=True)
    out = {"samples": int(len(samp)),
           "plain": {"gdof_stage_s": _gdofs(mesh, 4, steps, ms_plain),
                     "ms_per_step": ms_plain / steps,
                     "evals_per_filtered": plain["evals"] / max(1, plain["filtered"]),
                     "filtered_per_step": plain["filtered"] / steps,
                     "kernel_ms_one_step": {k: v[0] for k, v in prof.items()
                                            if v[1]}}}
    if len(samp) > 100:
        x = samp[:, :4].astype(np.float64)
        z = samp[:, 4].astype(np.float64)
        theta = np.zeros(1257)
        rng = np.random.default_rng(0)
        theta[0:128] = rng.normal(0, 0.5, 128)
        theta[160:1184] = rng.normal(0, 1 / np.sqrt(32), 1024)
        theta[1216:1248] = rng.normal(0, 1 / np.sqrt(32), 32)
        theta[1249:1253] = x.mean(0)
        theta[1253:1257] = x.std(0) + 1e-6
        th, hist = fr.mlp_train(x, z, theta, epochs=2000, lr=3e-3)
        rms = float(np.sqrt(hist[-1]))
        ratio = float(np.clip(np.exp(1.5 * rms), 1.02, 2.0))
        mesh.filter_set_mlp(np.concatenate([th, [ratio]]).astype(np.float32))
        mesh.set_solution(start)
        mesh.filter_stats(reset=True)
        ms_mlp = _timed_steps(torch, mesh, st, "rk4", 9e-4, steps)
        lrn = mesh.filter_stats(reset=True)
        out["learned"] = {"gdof_stage_s": _gdofs(mesh, 4, steps, ms_mlp),
                          "ms_per_step": ms_mlp / steps,
                          "evals_per_filtered": lrn["evals"] / max(1, lrn["filtered"]),
                          "filtered_per_step": lrn["filtered"] / steps,
                          "train_loss": [float(hist[0]), float(hist[-1])],
                          "bracket_ratio": ratio}
    mesh.close()
    return out


def other_configs(fr, torch, device):
    out = {}
    for name, fn in (("vortex_8^3_p2_fp64", config_vortex),
                     ("tgv_32^3_p3", config_tgv32),
                     ("mixed_elements_40^3_p3_fp32", config_mixed_elements),
                     ("tgv_32^3_p3_fp32_adaptive", config_tgv_adaptive),
                     ("tgv_32^3_p3_curved", config_tgv_curved),
                     ("tgv_32^3_p3_antialias_q9", config_tgv_antialias),
                     ("tgv_32^3_p3_partitioned", config_tgv_partitioned),
                     ("shu_osher_256x8x8_p3_filter", config_shu_osher)):
        try:
            out[name] = fn(fr, torch, device)
        except Exception as exc:  # a failing side workload must not hide the rest
            out[name] = {"error": repr(exc)[:300]}
    return out


# ------------------------------------------------------ oracle baseline
# One single-threaded oracle replica: `warmup` untimed RK45 steps, then RK45
# steps of a SAMPLE_CELLS^3 box of the workload until `budget` seconds or
# `max_steps` steps.  The oracle is a serial numpy program; the all-cores
# figure runs one replica per core at the same time (weak scaling).
ORACLE_SAMPLE = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
import numpy as np
from frinputs import box_hex, ics
from oracle.mesh import FRMesh
from oracle.fr import FRSystem
from oracle import rk
n = {n}
spec = box_hex((n, n, n), hi=(2*np.pi,)*3, perturb=0.1)
m = FRMesh(spec.as_dict(), {p})
s = FRSystem(m, "ns", gamma=1.4, mu=1/{re}, pr={pr})
u = {{"hex": ics.taylor_green(m.upts_x["hex"].reshape(-1,3), mach={mach}).reshape(m.ne["hex"], -1, 5)}}
for _ in range({warmup}):
    u = rk.step(s.rhs, u, {dt}, "rk45")
steps = 0
t0 = time.perf_counter()
while True:
    u = rk.step(s.rhs, u, {dt}, "rk45")
    steps += 1
    el = time.perf_counter() - t0
    if el > {budget} or steps >= {max_steps}:
        break
npts = m.ne["hex"] * m.el["hex"].nupts
print(json.dumps({{"steps": steps, "seconds": el, "npts": int(npts)}}))
"""


def _cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return "unknown"


def _oracle_replicas(nrep, budget, max_steps, warmup=0):
    """Run nrep single-threaded oracle replicas at once (fresh interpreters,
    no CUDA); returns (GDOF-stage/s over all replicas, per-replica records)."""
    code = ORACLE_SAMPLE.format(root=ROOT, n=SAMPLE_CELLS, p=ORDER, re=RE, pr=PR,
                                mach=MACH, dt=DT, budget=budget,
                                max_steps=max_steps, warmup=warmup)
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    procs = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True, env=env)
             for _ in range(nrep)]
    recs = []
    for pr_ in procs:
        out, err = pr_.communicate(timeout=min(budget * 20, 3000.0) + 600)
        if pr_.returncode != 0:
            raise RuntimeError(err[-300:])
        recs.append(json.loads(out.strip().splitlines()[-1]))
    units = sum(r["npts"] * 5 * STAGES * r["steps"] for r in recs)
    wall = max(r["seconds"] for r in recs)
    return units / wall / 1e9, recs


def cpu_baseline(budget):
    cores = os.cpu_count() or 1
    try:
        one, r1 = _oracle_replicas(1, budget, 200)
        allc, ra = _oracle_replicas(cores, budget, 200)
    except Exception as exc:  # noqa: BLE001 - reported, not fatal
        return {"value": None, "error": repr(exc)[:300]}
    return {"value": allc, "unit": "GDOF-stage/s", "cores": cores,
            "kind": "oracle", "one_core": one, "cpu_model": _cpu_model(),
            "nproc": cores,
            "sample": f"{SAMPLE_CELLS}^3-element boxes of the same workload "
                      f"(p={ORDER}, NS TGV, RK45 dt {DT}), numpy FP64: one "
                      f"single-threaded replica per core, each about {budget:.0f} s "
                      f"({ra[0]['steps']} steps on the first); 1 core alone: "
                      f"{r1[0]['steps']} steps in {r1[0]['seconds']:.1f} s"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    val, recs = _oracle_replicas(cores, 1e9, args.steps, warmup=args.warmup)
    wall = max(r["seconds"] for r in recs)
    cb = {"value": val, "unit": "GDOF-stage/s", "cores": cores, "kind": "oracle",
          "cpu_model": _cpu_model(),
          "sample": f"{cores} single-threaded replicas, each {args.warmup} untimed "
                    f"+ {args.steps} timed RK45 steps of a {SAMPLE_CELLS}^3-element "
                    f"box of the workload (p={ORDER}), numpy FP64"}
    line = {"impl": "reference", "metric": METRIC,
            "value": val, "unit": "GDOF-stage/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": wall * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": config("fp64"),
            "cpu_baseline": cb,
            "e2e": {"value": val, "unit": "GDOF-stage/s",
                    "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    global N_CELLS
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64",
                    choices=["fp64", "fp32", "mixed"])
    ap.add_argument("--variants", type=int, default=1,
                    help="also time the other precision modes (N=1 only)")
    ap.add_argument("--configs", type=int, default=1,
                    help="also time the other workloads (N=1 only)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--only", default=None,
                    choices=["vortex", "tgv32", "mixed", "shu_osher", "adaptive",
                             "curved", "antialias", "partitioned"],
                    help="run one side workload alone and print its record "
                         "(profiling aid; not a contract line)")
    ap.add_argument("--size", type=int, default=N_CELLS,
                    help="hexahedra per direction of the main workload (smaller "
                         "sizes for profiling captures; the contract line is 48)")
    ap.add_argument("--cells", type=int, default=40,
                    help="cells per direction of the mixed-element box (--only mixed)")
    ap.add_argument("--qdeg", type=int, default=0,
                    help="anti-aliasing rule degree of the mixed-element run (--only mixed)")
    ap.add_argument("--precisions", default="fp64,fp32",
                    help="precisions of the curved / anti-aliased runs (--only)")
    ap.add_argument("--variant", default="auto",
                    help="kernel family of the mixed-element run (--only mixed)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    N_CELLS = args.size
    if args.only:
        import torch
        import paper_2408_16509_gb300 as fr
        fr.build()
        dev = 0
        torch.cuda.set_device(dev)
        fns = {"vortex": config_vortex, "tgv32": config_tgv32,
               "adaptive": config_tgv_adaptive,
               "curved": lambda f, t, d: config_tgv_curved(
                   f, t, d, precisions=tuple(args.precisions.split(","))),
               "antialias": lambda f, t, d: config_tgv_antialias(
                   f, t, d, precisions=tuple(args.precisions.split(","))),
               "partitioned": lambda f, t, d: config_tgv_partitioned(
                   f, t, d, precisions=tuple(args.precisions.split(","))),
               "shu_osher": config_shu_osher,
               "mixed": lambda f, t, d: config_mixed_elements(
                   f, t, d, steps=args.steps, cells=args.cells,
                   variant=args.variant, qdeg=args.qdeg)}
        rec = fns[args.only](fr, torch, dev)
        print(json.dumps({"only": args.only, "record": rec}), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
