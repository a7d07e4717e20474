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
def kernel_models(nu, nf, ne, w, np_, nb):
    """Compulsory DRAM bytes per launch of each kernel class (RK45 stage
    i > 0, Navier-Stokes): see the design doc, kernel table."""
    per_elem = {
        "grad": w * (5 * nu + 5 * nf + 10 * nu + 15 * nu + 15 * nf),
        "volume": w * (5 * nu + 15 * nu + 5 * nf + 10 * nu + 5 * nu
                       + 10 * nu + 5 * nf),
    }
    per_pair = {
        "face_ucommon": w * 20 + 8,
        "face_flux": w * (2 * 20 + 5 + 10) + 8,
    }
    return {"grad": per_elem["grad"] * ne, "volume": per_elem["volume"] * ne,
            "face_ucommon": per_pair["face_ucommon"] * np_,
            "face_flux": per_pair["face_flux"] * np_}


# ------------------------------------------------------------ our arm
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
    spec = workload_spec(N_CELLS)
    mesh = fr.FRMesh(spec, ORDER, physics="ns", gamma=1.4, mu=1.0 / RE,
                     prandtl=PR, precision=args.precision, device=local)
    stream = torch.cuda.Stream(device=local)
    mesh.set_stream(stream)
    x = mesh.points("hex")
    ne, nu, nf = mesh.info("hex")
    u0 = tgv(x.reshape(-1, 3)).reshape(ne, nu, 5)
    mesh.set_solution({"hex": u0})
    npts = ne * nu
    units_per_step = npts * 5 * STAGES
    # warm-up (builds the CUDA graph)
    for _ in range(args.warmup):
        mesh.rk_step("rk45", DT, 1)
    sampler = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    mesh.rk_step("rk45", DT, args.steps)
    t1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = t0.elapsed_time(t1)
    if dist:
        tt = torch.tensor([ms], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
        dist.barrier()
    value = units_per_step * args.steps * world / (ms * 1e-3) / 1e9
    # per-kernel device times of one step, launched one by one with events
    prof = {}
    reps = 3
    for _ in range(reps):
        for k, (t, n) in mesh.profile_step("rk45", DT).items():
            a = prof.setdefault(k, [0.0, 0])
            a[0] += t / reps
            a[1] = n
    launches_per_step = sum(n for _, n in prof.values())
    # end-to-end through the C ABI with pinned host buffers
    host_in = torch.from_numpy(np.ascontiguousarray(u0)).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    hin = host_in.numpy()
    hout = host_out.numpy()
    e2e_steps = max(2, min(args.steps, 10))
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    import ctypes
    lib = fr.load()
    for _ in range(e2e_steps):
        rc = lib.fr_set_solution(mesh._h, 0, hin.ctypes.data_as(ctypes.c_void_p))
        rc |= lib.fr_rk_step(mesh._h, 1, DT, 1)
        rc |= lib.fr_get_solution(mesh._h, 0, hout.ctypes.data_as(ctypes.c_void_p))
        if rc:
            raise RuntimeError(lib.fr_last_error().decode())
    e2e_s = time.perf_counter() - w0
    e2e = units_per_step * e2e_steps * world / e2e_s / 1e9
    # roofline of the dominant kernel
    peaks, src = _peaks()
    w = 8 if args.precision == "fp64" else 4
    npair, nb = mesh.pair_counts()
    models = kernel_models(nu, nf, ne, w, npair, nb)
    dom = max((k for k in prof if prof[k][1] > 0), key=lambda k: prof[k][0])
    dom_ms = prof[dom][0] / prof[dom][1]
    bytes_per_launch = models.get(dom)
    achieved = bytes_per_launch / (dom_ms * 1e-3) / 1e9 if bytes_per_launch else None
    roof = {"kernel": dom, "bound": "hbm", "achieved": achieved,
            "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"] if achieved else None,
            "traffic": None, "peak_source": src,
            "kernel_ms": dom_ms,
            "algorithmic_bytes_per_launch": bytes_per_launch}
    line = {
        "metric": "GDOF-stage/s per GB300 (NS FR RHS + RK update)",
        "value": value, "unit": "GDOF-stage/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32",
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
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
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
