#!/usr/bin/env python
"""Benchmark: FR right-hand side + RK update throughput on one GB300.

Workload (the Navier-Stokes Taylor-Green vortex of the paper's Section 5,
at the size of a single-GPU run): periodic [0, 2 pi]^3 box of 32^3
hexahedra whose interior nodes are perturbed by up to 10% of the spacing
(seed 20240829), p = 3 (64 Gauss-Legendre solution points per element),
Re = 1600, Ma = 0.1, Pr = 0.71, constant viscosity, BR1 gradients, Rusanov
inviscid flux, RK4(3)5[2R+] with dt = 1e-3.  A "step" is one RK step
(five right-hand-side stages).  Metric: GDOF-stage/s = solution points x 5
variables x stages / second / 1e9.

--impl reference times the CPU FP64 oracle (plain numpy) on the same
workload, on a bounded sample (an 8^3-element box of the same shape).
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

N_CELLS = 32
ORDER = 3
RE, MACH, PR = 1600.0, 0.1, 0.71
DT = 1e-3
STAGES = 5
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
    return {"workload": f"ns-tgv-hex{N_CELLS}^3-p{ORDER}-rk45",
            "elements": N_CELLS ** 3, "order": ORDER,
            "solution_points": N_CELLS ** 3 * (ORDER + 1) ** 3,
            "physics": "navier-stokes BR1 + Rusanov", "scheme": "RK4(3)5[2R+]",
            "dt": DT, "re": RE, "mach": MACH, "precision": precision,
            "mesh_perturbation": 0.1,
            "l2": "inputs larger than L2 (state register 84 MB, step working "
                  "set > 1 GB); no flush"}


# ------------------------------------------------------ byte/flop models
FP64_TFLOPS_PROBE = 1.058   # measured DFMA throughput on this GB300 pool
FP32_TFLOPS_PROBE = 77.8    # measured FFMA throughput on this GB300 pool


def kernel_models(nu, nf, ne, w, wr, npair):
    """Algorithmic DRAM bytes and floating-point operations per launch of
    each kernel class for an RK4(3)5[2R+] stage i > 0 of the Navier-Stokes
    right-hand side on hexahedra (sum-factorised operators), N = p + 1.
    w: bytes of a trace/stage value, wr: bytes of a solution register."""
    n = round(nu ** (1.0 / 3.0))
    bytes_ = {
        # u(5) + metrics(10) + du(5 per flux pt) in, grad(15) + gradf(15) out
        "grad": ne * (w * (5 * nu + 10 * nu + 5 * nf + 15 * nu + 15 * nf)),
        # u(5) + grad(15) + metrics(10) + F^C(5/fpt) in; Y and u_f out;
        # solution register X in and out
        "volume": ne * (w * (5 * nu + 15 * nu + 10 * nu + 5 * nf + 5 * nu
                             + 5 * nf) + wr * 10 * nu),
        "face_ucommon": npair * (w * 20 + 8),
        "face_flux": npair * (w * (2 * 20 + 5 + 10) + 8),
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


def roofline(prof, models, peaks, src, precision):
    """Roofline record of the dominant kernel class: the bound is whichever
    of DRAM bytes / HBM peak and flops / arithmetic peak takes longer."""
    bytes_, flops = models
    dom = max((k for k in prof if prof[k][1] > 0), key=lambda k: prof[k][0])
    t = prof[dom][0] / prof[dom][1] * 1e-3
    b, f = bytes_.get(dom), flops.get(dom)
    bw = b / t / 1e9 if b else None
    fl = f / t / 1e12 if f else None
    if precision == "fp64":
        fpeak, fsrc = FP64_TFLOPS_PROBE, "FP64 FMA probe on this pool"
    else:
        fpeak, fsrc = FP32_TFLOPS_PROBE, "FP32 FMA probe on this pool"
    t_mem = b / (peaks["hbm_gbs"] * 1e9) if b else 0.0
    t_alu = f / (fpeak * 1e12) if f else 0.0
    if t_alu > t_mem:
        out = {"kernel": dom, "bound": "alu", "achieved": fl, "peak": fpeak,
               "unit": "TFLOP/s", "frac": fl / fpeak, "traffic": None,
               "peak_source": fsrc}
    else:
        out = {"kernel": dom, "bound": "hbm", "achieved": bw,
               "peak": peaks["hbm_gbs"], "unit": "GB/s",
               "frac": bw / peaks["hbm_gbs"], "traffic": None,
               "peak_source": src + " hbm_gbs (MEASURED_PEAKS.json)"}
    out.update({"launches_per_step": prof[dom][1], "kernel_ms": t * 1e3,
                "algorithmic_bytes": b, "algorithmic_flops": f,
                "achieved_gbs": bw, "achieved_tflops": fl,
                "attainable_ms": max(t_mem, t_alu) * 1e3})
    return out


# ------------------------------------------------------------ our arm
def measure(fr, torch, precision, steps, warmup, device, dist):
    spec = workload_spec(N_CELLS)
    mesh = fr.FRMesh(spec, ORDER, physics="ns", gamma=1.4, mu=1.0 / RE,
                     prandtl=PR, precision=precision, device=device)
    stream = torch.cuda.Stream(device=device)
    mesh.set_stream(stream)
    x = mesh.points("hex")
    ne, nu, nf = mesh.info("hex")
    u0 = tgv(x.reshape(-1, 3)).reshape(ne, nu, 5)
    mesh.set_solution({"hex": u0})
    for _ in range(warmup):             # the first one builds the CUDA graph
        mesh.rk_step("rk45", DT, 1)
    mesh.set_solution({"hex": u0})
    sampler = ClockSampler(device)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    mesh.rk_step("rk45", DT, steps)
    t1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = t0.elapsed_time(t1)
    if dist:
        tt = torch.tensor([ms], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
        dist.barrier()
    final = mesh.get_solution()["hex"]
    prof = {}
    reps = 3
    for _ in range(reps):
        for k, (t, n) in mesh.profile_step("rk45", DT).items():
            a = prof.setdefault(k, [0.0, 0])
            a[0] += t / reps
            a[1] = n
    return mesh, u0, ms, clocks, prof, final


def run_ours(args):
    import ctypes

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
    mesh, u0, ms, clocks, prof, final = measure(
        fr, torch, args.precision, args.steps, args.warmup, local, dist)
    ne, nu, nf = mesh.info("hex")
    units_per_step = ne * nu * 5 * STAGES
    value = units_per_step * args.steps * world / (ms * 1e-3) / 1e9
    launches_per_step = sum(n for _, n in prof.values())
    # end-to-end through the C ABI with pinned host buffers: every step
    # copies the state in, runs one RK step and copies the state out
    lib = fr.load()
    host_in = torch.from_numpy(np.ascontiguousarray(u0)).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    hin, hout = host_in.numpy(), host_out.numpy()
    e2e_steps = max(3, min(args.steps, 10))
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    for _ in range(e2e_steps):
        rc = lib.fr_set_solution(mesh._h, 0, hin.ctypes.data_as(ctypes.c_void_p))
        rc |= lib.fr_rk_step(mesh._h, 1, DT, 1)
        rc |= lib.fr_get_solution(mesh._h, 0,
                                  hout.ctypes.data_as(ctypes.c_void_p))
        if rc:
            raise RuntimeError(lib.fr_last_error().decode())
    e2e_s = time.perf_counter() - w0
    if dist:
        tt = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_s = float(tt.item())
    e2e = units_per_step * e2e_steps * world / e2e_s / 1e9
    npair, _ = mesh.pair_counts()
    w = 8 if args.precision == "fp64" else 4
    wr = 4 if args.precision == "fp32" else 8
    roof = roofline(prof, kernel_models(nu, nf, ne, w, wr, npair), peaks,
                    src, args.precision)
    line = {
        "metric": "GDOF-stage/s per GB300 (NS FR RHS + RK update)",
        "value": value, "unit": "GDOF-stage/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp32": "f32",
                  "mixed": "f32 (f64 RK registers)"}[args.precision],
        "data": "synthetic (seeded perturbed mesh, analytic TGV state)",
        "config": config(args.precision),
        "clocks": clocks,
        "e2e": {"value": e2e, "unit": "GDOF-stage/s",
                "h2d_bytes_per_step": int(hin.nbytes),
                "d2h_bytes_per_step": int(hout.nbytes)},
        "gpu_launches": launches_per_step * args.steps,
        "kernel_ms_per_step": {k: v[0] for k, v in prof.items() if v[1]},
        "roofline": roof,
    }
    mesh.close()
    if args.variants and world == 1:
        line["variants"] = {}
        for prec in ("fp64", "fp32", "mixed"):
            if prec == args.precision:
                continue
            m2, _, ms2, _, prof2, fin2 = measure(
                fr, torch, prec, args.steps, args.warmup, local, None)
            w2 = 8 if prec == "fp64" else 4
            wr2 = 4 if prec == "fp32" else 8
            if args.precision == "fp64":
                ref, oth = final, fin2
            else:
                ref, oth = fin2, final
            d = (oth - ref).reshape(-1, 5)
            r = ref.reshape(-1, 5)
            den = np.maximum(np.linalg.norm(r, axis=0),
                             np.linalg.norm(r[:, 0]))
            line["variants"][prec] = {
                "value": units_per_step * args.steps / (ms2 * 1e-3) / 1e9,
                "ms_per_step": ms2 / args.steps,
                "rel_l2_vs_fp64_after_steps": (np.linalg.norm(d, axis=0)
                                               / den).tolist(),
                "roofline": roofline(
                    prof2, kernel_models(nu, nf, ne, w2, wr2, npair), peaks,
                    src, prec),
                "kernel_ms_per_step": {k: v[0] for k, v in prof2.items()
                                       if v[1]}}
            m2.close()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# ------------------------------------------------------ oracle baseline
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


def cpu_baseline(budget):
    n = 8
    code = ORACLE_SAMPLE.format(root=ROOT, n=n, p=ORDER, re=RE, pr=PR,
                                mach=MACH, dt=DT, budget=budget, max_steps=50)
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    r = subprocess.run([sys.executable, "-c", code], capture_output=True,
                       text=True, env=env, timeout=budget * 10 + 120)
    if r.returncode != 0:
        return {"value": None, "error": r.stderr[-300:]}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    val = d["npts"] * 5 * STAGES * d["steps"] / d["seconds"] / 1e9
    return {"value": val, "unit": "GDOF-stage/s", "cores": 1,
            "kind": "oracle",
            "sample": f"{n}^3-element box of the same workload (p={ORDER}, "
                      f"NS TGV, RK45), {d['steps']} steps in "
                      f"{d['seconds']:.1f} s, numpy FP64, 1 thread"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cb = cpu_baseline(args.cpu_seconds)
    val = cb.get("value")
    line = {"impl": "reference",
            "metric": "GDOF-stage/s per GB300 (NS FR RHS + RK update)",
            "value": val, "unit": "GDOF-stage/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": config("fp64"),
            "cpu_baseline": cb,
            "e2e": {"value": val, "unit": "GDOF-stage/s",
                    "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64",
                    choices=["fp64", "fp32", "mixed"])
    ap.add_argument("--variants", type=int, default=1,
                    help="also time the other precision modes (N=1 only)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
