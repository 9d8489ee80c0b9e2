"""Benchmark of the hex8 element-assembly hot path on B300.

One step = the whole hot path over one synthetic workload: consistent-tangent CSR
assembly with the residual fused (gather, shape gradients, constitutive update, R_e and
K_e, coloured scatter), the matrix-free tangent product K.v, and the FP64 residual norm.
Workload (default): 128^3 hex8 unidirectional-fibre RVE (2,097,152 elements, 6,440,067
DOFs, 513,599,625 CSR non-zeros), compressible neo-Hookean per phase, 1% uniaxial stretch
plus 1e-4 noise, FP64.  Metric: elements per second of that step (higher is better).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl jetsci|reference]

Prints one JSON line (rank 0).  With N > 1 (torchrun), each rank runs its own replica of the
workload (independent problems, no data-path collective: weak scaling); the timed region is
bracketed by barriers and the max over ranks is reported.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "hex8 elem/s (residual+tangent, K·v) at 128³, surrogate vs plain, % of HBM peak"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="jetsci", choices=["jetsci", "reference"])
    ap.add_argument("--n", type=int, default=128, help="elements per side of the RVE")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "df64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle sample")
    return ap.parse_args()


# ------------------------------------------------------------------------------ helpers
def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0, "sm_max_mhz": 2032.0}, \
        "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle sampling in a background process during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(prob, target_seconds):
    """The FP64 oracle (single-threaded C, as it stands) on a bounded sample of the same
    workload: the first M elements in element order (a contiguous slab of the RVE), one
    step = tangent CSR + residual + element-loop K.v + norm; pattern setup not timed."""
    import oracle

    def run(m):
        conn = prob.conn[:m]
        used = np.unique(conn)
        remap = -np.ones(prob.n_nodes, dtype=np.int64)
        remap[used] = np.arange(len(used))
        sub_conn = remap[conn].astype(np.int32)
        sub_coords = prob.coords[used]
        dofs = (3 * used[:, None] + np.arange(3)).ravel()
        om = oracle.Mesh(sub_coords, sub_conn, prob.phase[:m], prob.materials)
        rp, col = oracle.csr_pattern(sub_conn, len(used))
        u, v = prob.u[dofs], prob.v[dofs]
        t0 = time.perf_counter()
        vals, R = oracle.tangent_csr(om, u, rp, col)
        oracle.apply_tangent(om, u, v)
        oracle.norm2(R)
        return time.perf_counter() - t0

    m = 512
    dt = run(m)
    m = int(min(prob.n_elem, max(m, m * target_seconds / max(dt, 1e-6))))
    dt = run(m)
    return {"value": m / dt, "unit": "elem/s", "cores": 1, "kind": "oracle",
            "sample": f"first {m} elements (contiguous slab) of the same workload, FP64, one step "
                      f"(tangent CSR + residual + K.v + norm) in {dt:.1f} s"}


def make_problem(n, precision):
    from paper_2604_22087_b300 import inputs as I
    return I.fibre_composite(n, seed=2, law=I.LAW_NEO_HOOKEAN)


# ------------------------------------------------------------------------------ reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return
    prob = make_problem(args.n, args.precision)
    per = max(1.0, 60.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        cpu_baseline(prob, min(per, 2.0))
    vals = [cpu_baseline(prob, per) for _ in range(args.steps)]
    v = statistics.median(x["value"] for x in vals)
    cb = dict(vals[-1])
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "elem/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * prob.n_elem / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(prob, args),
            "cpu_baseline": cb, "e2e": {"value": v, "unit": "elem/s", "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_dict(prob, args):
    return {"workload": f"fibre RVE {args.n}^3 hex8 neo-Hookean, 1% stretch + 1e-4 noise, "
                        f"step = tangent CSR (+R) + matrix-free K.v + ||R||",
            "n_elem": prob.n_elem, "n_dof": prob.n_dof, "precision": args.precision,
            "fibre_fraction": prob.meta.get("fibre_fraction"),
            "l2": "inputs larger than L2 (CSR values 4.1 GB FP64 written every step)"}


# ------------------------------------------------------------------------------ main arm
def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2604_22087_b300 import jetsci as J

    prec = {"fp64": J.FP64, "fp32": J.FP32, "df64": J.DF64}[args.precision]
    prob = make_problem(args.n, args.precision)
    mesh = J.Mesh.of(prob)
    stream = torch.cuda.Stream()
    u = torch.as_tensor(prob.u).cuda()
    v = torch.as_tensor(prob.v).cuda()
    R = mesh.new_vector()
    y = mesh.new_vector()
    vals = mesh.new_values(prec)
    nrm = torch.empty(1, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        mesh.tangent_csr(u, vals=vals, R=R, precision=prec, stream=stream)
        if ev is not None:
            ev[1].record(stream)
        mesh.apply_tangent(u, v, y=y, precision=prec, stream=stream)
        mesh.norm2(R, out=nrm, stream=stream)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(max(3, args.warmup)):
        step()
    barrier()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        t0.record(stream)
        for k in range(args.steps):
            step(evs[k])
        t1.record(stream)
        t1.synchronize()
    barrier()
    ms_total = t0.elapsed_time(t1)
    ms_tangent = statistics.mean(a.elapsed_time(b) for a, b in evs)
    tmax = torch.tensor([ms_total], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    ms_total = float(tmax.item())
    ms_step = ms_total / args.steps
    value = world * prob.n_elem / (ms_step * 1e-3)
    assert mesh.check() == 0

    # ---- end to end through the public API with host buffers (pinned), copies timed
    u_h = torch.as_tensor(prob.u).pin_memory()
    v_h = torch.as_tensor(prob.v).pin_memory()
    y_h = torch.empty(prob.n_dof, dtype=torch.float64).pin_memory()
    n_h = torch.empty(1, dtype=torch.float64).pin_memory()

    def e2e_step():
        with torch.cuda.stream(stream):
            u.copy_(u_h, non_blocking=True)
            v.copy_(v_h, non_blocking=True)
        step()
        with torch.cuda.stream(stream):
            y_h.copy_(y, non_blocking=True)
            n_h.copy_(nrm, non_blocking=True)

    e2e_step()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    e1.synchronize()
    barrier()
    e2e_ms = e0.elapsed_time(e1) / args.steps
    emax = torch.tensor([e2e_ms], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(emax, op=dist.ReduceOp.MAX)
    e2e_ms = float(emax.item())

    forms = {}
    if not args.no_forms and rank == 0:
        forms = measure_forms(J, mesh, prob, stream, u, v)

    if rank == 0:
        peaks, peak_kind = load_peaks()
        clocks = clk.summary()
        # dominant kernel: the tangent assembly (FP64 pipe bound in FP64)
        fp64_peak = 4.0 * 148 * peaks.get("sm_max_mhz", 2032.0) * 1e6 / 1e12  # 2 DFMA/clk/SM
        flops = TANGENT_FP64_FLOP_PER_ELEM * prob.n_elem
        achieved = flops / (ms_tangent * 1e-3) / 1e12
        hbm_bytes = TANGENT_BYTES_PER_ELEM_FP64 * prob.n_elem
        line = {
            "metric": METRIC, "value": value, "unit": "elem/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32", "df64": "f32x2"}[args.precision],
            "data": "synthetic", "config": config_dict(prob, args),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                         "frac": achieved / fp64_peak, "traffic": None, "kernel": "k_tangent<double,double>",
                         "peak_source": "2 DFMA/clk/SM x 148 SMs x sm_max_mhz (FP64 pipe)",
                         "hbm_achieved_gbs": hbm_bytes / (ms_tangent * 1e-3) / 1e9,
                         "hbm_frac": hbm_bytes / (ms_tangent * 1e-3) / 1e9 / peaks["hbm_gbs"],
                         "hbm_peak_kind": peak_kind, "ms_per_launch_group": ms_tangent},
            "e2e": {"value": world * prob.n_elem / (e2e_ms * 1e-3), "unit": "elem/s",
                    "h2d_bytes_per_step": 2 * prob.n_dof * 8, "d2h_bytes_per_step": prob.n_dof * 8 + 8},
            "gpu_launches": args.steps * (2 * mesh.n_colours + 2),
            "clocks": clocks,
            "forms": forms,
        }
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(prob, args.cpu_seconds)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


# Algorithmic work per element of the dominant kernel (derivation in the design doc).
TANGENT_FP64_FLOP_PER_ELEM = 26_000.0
TANGENT_BYTES_PER_ELEM_FP64 = 2160.0


def measure_forms(J, mesh, prob, stream, u, v, reps=5):
    """Per-call device times of the individual entry points (ms) and elem/s."""
    import torch
    out = {}
    R = mesh.new_vector()
    y = mesh.new_vector()

    def timeit(fn):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b) / reps
        return {"ms": ms, "elem_per_s": prob.n_elem / (ms * 1e-3)}

    for name, p in (("fp64", J.FP64), ("fp32", J.FP32)):
        vals = mesh.new_values(p)
        out[f"residual_{name}"] = timeit(lambda: mesh.residual(u, R=R, precision=p, stream=stream))
        out[f"tangent_csr_{name}"] = timeit(lambda: mesh.tangent_csr(u, vals=vals, R=R, precision=p, stream=stream))
        out[f"apply_mf_{name}"] = timeit(lambda: mesh.apply_tangent(u, v, y=y, precision=p, stream=stream))
        out[f"spmv_csr_{name}"] = timeit(lambda: mesh.apply_tangent(None, v, y=y, mode=J.CSR, vals=vals,
                                                                    precision=p, stream=stream))
        del vals
        torch.cuda.empty_cache()
    return out


if __name__ == "__main__":
    main()
