"""Benchmark of the hex8 element-assembly hot path on B300.

One step = the whole hot path over one synthetic workload: consistent-tangent CSR assembly
with the residual fused (gather, shape gradients, constitutive update, R_e and K_e, coloured
scatter; the call also stores the neo-Hookean state per Gauss point), the tangent product K.v
both from the assembled CSR matrix and matrix-free (at that stored linearisation, as a
Newton-Krylov product at one iterate would be), and the FP64 residual norm.  Workload (default): 128^3 hex8 unidirectional-fibre RVE (2,097,152
elements, 6,440,067 DOFs, 513,599,625 CSR non-zeros), compressible neo-Hookean per phase at a
1% uniaxial stretch plus 1e-4 noise, FP64.  Metric: elements per second of that step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl jetsci|reference] [--no-newton]

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank runs its own replica of the
workload (independent problems, no data-path collective: weak scaling); the timed region is
bracketed by barriers and the max over ranks is reported.  Besides the headline, the line
carries per-form timings with errors against the FP64 oracle on sampled rows (FP64, FP32,
TF32 tensor-core and surrogate forms), surrogate training, the 64^3 adjoint workload and
Newton iteration counts per tangent precision on the same RVE (all after the timed region).
"""
from __future__ import annotations

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

METRIC = "hex8 elem/s (residual+tangent, K·v) at 128³, surrogate vs plain, % of HBM peak"

# Work per element of the dominant kernel, k_tangent<double,double>:
# executed FP64 operations of the formulation (ncu on the 64^3 fibre RVE: 5,432 DFMA x 2 +
# 192 DADD + 1,252 DMUL per element; the pair form accumulated entry by entry, with the
# geometric term mu L_ab read from the reference-Laplacian cache) and the algorithmic bytes
# (write-once CSR values 1,959 + slot map and masks 96 + u, R and connectivity 82 + the
# reference-geometry cache 1,216 + the stored linearisation 768 + L_ab 288).
TANGENT_FP64_FLOP_PER_ELEM = 12_308.0
# The same operations counted as FP64-pipe instructions (5,432 DFMA + 192 DADD + 1,252 DMUL):
# each takes one slot of the pipe (2 per clock per SM), whatever its flop count.
TANGENT_FP64_INSTR_PER_ELEM = 6_876.0
TANGENT_BYTES_PER_ELEM_FP64 = 4_409.0
# DRAM bytes (read + write) per element of k_tangent<double,double> from one ncu capture of the
# 64^3 fibre RVE (profiles/k_tangent_fp64_fibre64.md), scaled by the element count (the
# coloured read-modify-writes re-read CSR rows once per colour, so traffic grows with elements).
TANGENT_DRAM_BYTES_PER_ELEM_FP64 = 14_617.0
# FP32-value element kernels are bound by instruction issue (4 warp instructions per clock per SM),
# not by a math pipe or DRAM: warp instructions per element from one ncu capture each of the 64^3 fibre
# RVE (profiles/k_tangent_fp32_fibre64.md, k_gather_rows_fp32_fibre64.md, k_apply_mf_fp32_fibre64.md,
# k_residual_fp32_fibre64.md), with their DRAM bytes per element and the algorithmic bytes (FP32
# tangent: the write-once FP32 CSR values 980 + slot map 64 + u, R and connectivity 82 + L_ab 288;
# matrix-free K.v: u, v, coordinates and the y write 98 + connectivity and phase 33).
FP32_FORMS = {
    "tangent_csr_fp32": {"warp_instr": 778.0 + 348.0, "dram_bytes": 2638.0 + 3529.0, "alg_bytes": 1414.0,
                         "kernels": "k_tangent<float,float,1> (element pass) + k_gather_rows<float> (row pass)"},
    "apply_matrix_free_fp32": {"warp_instr": 314.0, "dram_bytes": 858.0, "alg_bytes": 131.0,
                               "kernels": "k_apply_mf<float,0> (eight colour launches)"},
    "residual_fp32": {"warp_instr": 245.0, "dram_bytes": 662.0, "alg_bytes": 107.0,
                      "kernels": "k_residual<float,0> (eight colour launches)"},
    # TF32: the tensor-core element pass (profiles/k_tf32_tangent_fibre64.md, tensor pipe active
    # 20.7% of its cycles) + the same row pass; the same algorithmic bytes as the FP32 tangent
    "tangent_csr_tf32": {"warp_instr": 474.0 + 348.0, "dram_bytes": 2642.0 + 3529.0, "alg_bytes": 1414.0,
                         "kernels": "k_tf32 (tensor-core element pass) + k_gather_rows<float> (row pass)",
                         "tensor_pipe_active_element_pass": 0.207},
}
# Algorithmic bytes per CSR non-zero of the sparse product: the value plus a third of a column
# index (a node's three rows share one column list); v and y are per-row and stay in L2.
SPMV_BYTES_PER_NNZ = {"fp64": 8.0 + 4.0 / 3.0, "fp32": 4.0 + 4.0 / 3.0}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="jetsci", choices=["jetsci", "reference"])
    ap.add_argument("--n", type=int, default=128, help="elements per side of the RVE")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip surrogate training and the adjoint workload")
    ap.add_argument("--no-newton", action="store_true", help="skip the Newton iteration counts")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle sample")
    ap.add_argument("--partition", default="replicas", choices=["replicas", "slab"],
                    help="N > 1: one replica of the workload per rank (weak scaling, default), or one mesh "
                         "split into z-slabs over the ranks with a halo exchange (strong scaling)")
    return ap.parse_args()


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0, "sm_max_mhz": 2032.0}, \
        "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling in a background process."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx, self.proc, self.lines = device_index, None, []

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


def max_over_ranks(ms, world, device):
    """The largest per-rank time (ms): every rank runs its own replica, so the job finishes
    when the slowest rank does.  A plain all-reduce(MAX) over the default process group."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(n_elem_per_rank, world, ms_step):
    """Whole-job throughput: the elements all ranks processed in one step over the slowest
    rank's step time (elements per second)."""
    return world * n_elem_per_rank / (ms_step * 1e-3)


def make_problem(n):
    from paper_2604_22087_b300 import inputs as I
    return I.fibre_composite(n, seed=2, law=I.LAW_NEO_HOOKEAN)


def config_dict(prob, n):
    return {"workload": f"fibre RVE {n}^3 hex8 neo-Hookean (50% fibres, E 3.5/70 GPa), 1% stretch + 1e-4 noise; "
                        f"step = tangent CSR with fused residual + K.v (CSR SpMV, and matrix-free at the linearisation the tangent stored) + ||R||, FP64",
            "n_elem": prob.n_elem, "n_dof": prob.n_dof, "fibre_fraction": prob.meta.get("fibre_fraction"),
            "l2": l2_note(n)}


def l2_note(n):
    # an n^3 grid of hex8 elements couples (3n+1)^3 node pairs, 9 values each
    gb = 9 * (3 * n + 1) ** 3 * 8 / 1e9
    if gb > 0.126:
        return f"inputs larger than L2 (CSR values {gb:.1f} GB written and read every step)"
    return f"inputs fit in L2 ({gb * 1e3:.1f} MB of CSR values): a parity-size case, not a timed workload"


# ------------------------------------------------------------------------------ CPU oracle
class OracleSlab:
    """The first m elements of the workload (a contiguous slab of the RVE) set up once for the
    FP64 oracle (sub-mesh, CSR pattern, u and v restricted to its nodes)."""

    def __init__(self, prob, m):
        import oracle
        self.m = m
        conn = prob.conn[:m]
        used = np.unique(conn)
        remap = -np.ones(prob.n_nodes, dtype=np.int64)
        remap[used] = np.arange(len(used))
        sub_conn = remap[conn].astype(np.int32)
        dofs = (3 * used[:, None] + np.arange(3)).ravel()
        self.om = oracle.Mesh(prob.coords[used], sub_conn, prob.phase[:m], prob.materials)
        self.rp, self.col = oracle.csr_pattern(sub_conn, len(used))
        self.u, self.v = prob.u[dofs], prob.v[dofs]

    def step(self):
        """One step of the oracle (single-threaded C, as it stands): tangent CSR + residual +
        element-loop K.v + CSR K.v + norm.  Returns seconds."""
        import oracle
        t0 = time.perf_counter()
        vals, R = oracle.tangent_csr(self.om, self.u, self.rp, self.col)
        oracle.apply_tangent(self.om, self.u, self.v)
        oracle.spmv(self.rp, self.col, vals, self.v)
        oracle.norm2(R)
        return time.perf_counter() - t0


def calibrated_m(prob, target_seconds):
    """A 512-element slab, and the element count one oracle step covers in about target_seconds
    (from the 512-element step's time)."""
    small = OracleSlab(prob, 512)
    dt = min(small.step() for _ in range(2))
    return small, int(min(prob.n_elem, max(512, 512 * target_seconds / max(dt, 1e-6))))


def calibrated_slab(prob, target_seconds):
    """A slab sized so that one oracle step takes about target_seconds, and a 512-element one."""
    small, m = calibrated_m(prob, target_seconds)
    return small, (OracleSlab(prob, m) if m > 512 else small)


def host_cores():
    """Cores this process may run on (its affinity set), else the machine's count."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def baseline_line(slab, dt):
    return {"value": slab.m / dt, "unit": "elem/s", "cores": 1, "kind": "oracle",
            "sample": f"first {slab.m} elements (a contiguous slab) of the same workload, FP64, one step "
                      f"(tangent CSR + residual + element K.v + CSR K.v + norm) in {dt:.1f} s, one thread",
            "host_cores": host_cores()}


class _SlabArrays:
    """Elements [e0, e0 + m) of the workload as plain arrays (picklable for a worker process)."""

    def __init__(self, prob, e0, m):
        conn = prob.conn[e0:e0 + m]
        used = np.unique(conn)
        remap = -np.ones(prob.n_nodes, dtype=np.int64)
        remap[used] = np.arange(len(used))
        dofs = (3 * used[:, None] + np.arange(3)).ravel()
        self.m = m
        self.coords, self.conn = prob.coords[used], remap[conn].astype(np.int32)
        self.phase, self.materials = prob.phase[e0:e0 + m], prob.materials
        self.u, self.v = prob.u[dofs], prob.v[dofs]


def _oracle_worker(arrays, pipe):
    """One process of the all-core legs: sets up its slab (not timed), then for every "go"
    message runs one oracle step (single-threaded, as it stands) and sends its time back, until
    it receives "stop"."""
    import oracle
    om = oracle.Mesh(arrays.coords, arrays.conn, arrays.phase, arrays.materials)
    rp, col = oracle.csr_pattern(arrays.conn, len(arrays.coords))
    pipe.send("ready")
    while pipe.recv() == "go":
        t0 = time.perf_counter()
        vals, R = oracle.tangent_csr(om, arrays.u, rp, col)
        oracle.apply_tangent(om, arrays.u, arrays.v)
        oracle.spmv(rp, col, vals, arrays.v)
        oracle.norm2(R)
        pipe.send(time.perf_counter() - t0)


class OraclePool:
    """The oracle on every host core: one spawned process per core (at most max_workers), each
    with its own slab of m elements spread over the workload.  step() runs one oracle step in
    every process at once and returns (wall seconds from the common start to the last finish,
    per-process seconds)."""

    def __init__(self, prob, per_worker_elems, max_workers=64):
        import multiprocessing as mp
        self.P = max(1, min(host_cores(), max_workers))
        self.m = int(max(512, min(per_worker_elems, prob.n_elem // self.P)))
        starts = [int(k * (prob.n_elem - self.m) / max(1, self.P - 1)) for k in range(self.P)] if self.P > 1 else [0]
        ctx = mp.get_context("spawn")
        self.procs, self.pipes = [], []
        try:
            for e0 in starts:
                a, b = ctx.Pipe()
                pr = ctx.Process(target=_oracle_worker, args=(_SlabArrays(prob, e0, self.m), b), daemon=True)
                pr.start()
                self.procs.append(pr)
                self.pipes.append(a)
            deadline = time.perf_counter() + 600.0
            for a, pr in zip(self.pipes, self.procs):
                if self._receive(a, pr, deadline) != "ready":
                    raise RuntimeError("oracle worker failed")
        except BaseException:
            self.close()
            raise

    @staticmethod
    def _receive(a, pr, deadline):
        # a worker that died (or never answers) must not block the bench
        while not a.poll(0.2):
            if not pr.is_alive() or time.perf_counter() > deadline:
                raise RuntimeError(f"oracle worker exited or timed out (exit code {pr.exitcode})")
        return a.recv()

    def step(self):
        t0 = time.perf_counter()
        for a in self.pipes:
            a.send("go")
        dts = [self._receive(a, pr, t0 + 600.0) for a, pr in zip(self.pipes, self.procs)]
        return time.perf_counter() - t0, dts

    def close(self):
        for a in self.pipes:
            try:
                a.send("stop")
            except (BrokenPipeError, OSError):
                pass
        for pr in self.procs:
            pr.join(timeout=30)
            if pr.is_alive():
                pr.terminate()


def cpu_baseline_all_cores(prob, per_worker_elems, max_workers=64):
    """The same oracle step on every host core at once (OraclePool), one step.  value = all
    processes' elements / wall time from the common start to the last finish."""
    pool = OraclePool(prob, per_worker_elems, max_workers)
    try:
        wall, dts = pool.step()
    finally:
        pool.close()
    P, m = pool.P, pool.m
    return {"value": P * m / wall, "unit": "elem/s", "cores": P, "kind": "oracle", "host_cores": host_cores(),
            "sample": f"{P} processes at once, one per core, each the single-threaded oracle step on its own "
                      f"{m}-element slab of the same workload ({P * m} elements), wall {wall:.1f} s "
                      f"(per-process {min(dts):.1f}-{max(dts):.1f} s)"}


def cpu_baseline(prob, target_seconds):
    """The FP64 oracle on a bounded sample of the same workload, single-threaded and on every
    host core; slab set-up is not timed."""
    _, slab = calibrated_slab(prob, target_seconds)
    line = baseline_line(slab, slab.step())
    try:
        line["all_cores"] = cpu_baseline_all_cores(prob, max(512, slab.m // 2))
    except Exception as ex:  # report, do not hide
        line["all_cores"] = {"error": repr(ex)}
    return line


def run_reference(args, rank):
    """The oracle as it stands on the machine's host cores: every step runs one single-threaded oracle
    step in each of one process per core, each on its own slab of the workload sized so that the
    whole --warmup + --steps run takes a few minutes; value = the elements all processes stepped
    over the step's wall time (median over the timed steps)."""
    if rank != 0:
        return
    prob = make_problem(args.n)
    per = max(1.0, min(20.0, 100.0 / max(1, args.steps + args.warmup)))
    _, m = calibrated_m(prob, per)  # the elements one core steps in about `per` seconds
    pool = OraclePool(prob, m)
    try:
        for _ in range(args.warmup):
            pool.step()
        walls, per_proc = [], []
        for _ in range(args.steps):
            w, dts = pool.step()
            walls.append(w)
            per_proc += dts
    finally:
        pool.close()
    wall = statistics.median(walls)
    elems = pool.P * pool.m
    v = elems / wall
    cb = {"value": v, "unit": "elem/s", "cores": pool.P, "kind": "oracle", "host_cores": host_cores(),
          "sample": f"{pool.P} processes at once, one per host core, each the single-threaded oracle step "
                    f"(tangent CSR + residual + element K.v + CSR K.v + norm) on its own {pool.m}-element slab of "
                    f"the same workload ({elems} elements per step); median wall {wall:.2f} s over {args.steps} "
                    f"steps (per-process {min(per_proc):.2f}-{max(per_proc):.2f} s)"}
    # ms_per_step is the measured wall time of one step (the work each timed step did); the full
    # mesh at this rate would take n_elem / value seconds per step.
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "elem/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall,
            "ms_per_step_note": (f"one step = the oracle on {pool.P} host cores over the whole {prob.n_elem}-element "
                                 f"mesh ({pool.P} slabs that tile it)" if elems == prob.n_elem else
                                 f"one step = the oracle on {pool.P} host cores over {elems} elements of the workload; "
                                 f"the full {prob.n_elem}-element mesh at this rate would take "
                                 f"{prob.n_elem / v:.1f} s per step (extrapolated, not run)"),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(prob, args.n), "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "elem/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------ helpers
def timeit(fn, stream, reps=5):
    import torch
    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b) / reps


class SampledOracle:
    """Oracle rows of R, K and K.v at a fixed sample of nodes (computed element by element)."""

    def __init__(self, prob, n_nodes=24, seed=0):
        import oracle
        self.om = oracle.Mesh.of(prob)
        g = np.random.default_rng(seed)
        self.nodes = np.concatenate([[0, prob.n_nodes - 1], g.choice(prob.n_nodes, n_nodes - 2, replace=False)])
        self.rows = oracle.sampled_rows(self.om, prob.u, prob.v, self.nodes)

    def errors(self, R, vals, y, rowptr, col):
        """Max errors over the sample, each relative to the sample's max |reference|."""
        eR = ey = eK = 0.0
        sR = max(np.max(np.abs(self.rows[n][0])) for n in self.nodes)
        sy = max(np.max(np.abs(self.rows[n][1])) for n in self.nodes)
        sK = 0.0
        for n in self.nodes:
            Rn, Kvn, krow = self.rows[n]
            if R is not None:
                eR = max(eR, np.max(np.abs(R[3 * n:3 * n + 3] - Rn)))
            if y is not None:
                ey = max(ey, np.max(np.abs(y[3 * n:3 * n + 3] - Kvn)))
            if vals is not None:
                for i in range(3):
                    r = 3 * n + i
                    cs = col[rowptr[r]:rowptr[r + 1]]
                    kref = np.array([krow[c][i] for c in cs])
                    sK = max(sK, np.max(np.abs(kref)))
                    eK = max(eK, np.max(np.abs(vals[rowptr[r]:rowptr[r + 1]].astype(np.float64) - kref)))
        out = {}
        if R is not None:
            out["R"] = eR / sR
        if vals is not None:
            out["K"] = eK / sK
        if y is not None:
            out["Kv"] = ey / sy
        return out


def gather_rows(t, nodes):
    idx = np.concatenate([[3 * n, 3 * n + 1, 3 * n + 2] for n in nodes])
    out = np.zeros(int(t.numel()))
    out[idx] = t[idx].cpu().numpy()
    return out


def gather_vals(vals, rowptr, nodes):
    out = np.zeros(int(vals.numel()), dtype=np.float64)
    for n in nodes:
        a, b = int(rowptr[3 * n]), int(rowptr[3 * n + 3])
        out[a:b] = vals[a:b].double().cpu().numpy()
    return out


# ------------------------------------------------------------------------------ extras
def train_surrogate(J, torch, I, n_samples=1 << 20, epochs=50, batch=4096):
    """Surrogate trained on 2^20 neo-Hookean labels (|E_ij| <= 0.05) by the library's kernels."""
    E6, ph = I.strain_samples(n_samples, seed=5)
    E6d, phd = torch.as_tensor(E6).cuda(), torch.as_tensor(ph).cuda()
    mats = I.composite_materials(I.LAW_NEO_HOOKEAN)
    Sd = J.Surrogate.label(mats, E6d, phd)
    sc = np.array([[I.MATRIX_E * 0.05] * 6, [I.INCLUSION_E * 0.05] * 6])
    s = J.Surrogate(I.mlp_init(5), in_scale=0.05, range_=0.05, out_scale=sc, out_shift=np.zeros((2, 6)))
    order = torch.as_tensor(I.minibatch_order(n_samples, epochs, seed=5)).cuda()
    steps = epochs * (n_samples // batch)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = s.train(E6d, phd, Sd, order, n_steps=steps, batch=batch, lr_max=3e-3, lr_min=1e-5)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    Et, pt = I.strain_samples(1 << 16, seed=99)
    Etd, ptd = torch.as_tensor(Et).cuda(), torch.as_tensor(pt).cuda()
    S_true = J.Surrogate.label(mats, Etd, ptd).cpu().numpy()
    S, D = s.eval(Etd, ptd)
    S = S.cpu().numpy()
    scale = sc[pt]
    rms = float(np.sqrt(np.mean(((S - S_true) / scale) ** 2)))
    rel_max = float(np.max(np.abs(S - S_true)) / np.max(np.abs(S_true)))
    l = losses.cpu().numpy()
    info = {"samples": n_samples, "epochs": epochs, "batch": batch, "steps": steps, "seconds": dt,
            "steps_per_s": steps / dt, "loss_first": float(l[:10].mean()), "loss_last": float(l[-100:].mean()),
            "stress_rms_err_normalised": rms, "stress_max_err_rel": rel_max}
    return s, info


def adjoint_workload(J, torch, I, stream):
    """64^3 linear-elastic mesh with a lognormal per-element modulus: dLoss/dE for
    L = 1/2 ||R(u; E)||^2, checked by central differences (h = 1e-6 E_e and 1e-2 E_e) on 32
    random elements and against the oracle gradient on the same elements."""
    import oracle
    prob = I.lognormal_problem(64, seed=4)
    mesh = J.Mesh.of(prob)
    u, E = torch.as_tensor(prob.u).cuda(), torch.as_tensor(prob.E_elem).cuda()
    R = mesh.new_vector()
    g = torch.empty(prob.n_elem, dtype=torch.float64, device="cuda")
    out = {"workload": "lognormal E 64^3 linear elastic (262,144 elements)"}
    for name, p in (("fp64", J.FP64), ("fp32", J.FP32)):
        ms_r = timeit(lambda: mesh.residual(u, R=R, precision=p, E_elem=E, stream=stream), stream)
        # the gradient pass that recomputes R_e(u; E = 1), and the one from the element vectors
        # the residual call kept (u = None: the backward pass right after the forward residual)
        ms_gr = timeit(lambda: mesh.material_grad(u, R, E_elem=E, g=g, precision=p, stream=stream), stream)
        ms_g = timeit(lambda: mesh.material_grad(None, R, E_elem=E, g=g, precision=p, stream=stream), stream)
        out[f"residual_{name}_ms"] = ms_r
        out[f"grad_{name}_ms"] = ms_g
        out[f"grad_recompute_{name}_ms"] = ms_gr
        out[f"forward_backward_{name}_elem_per_s"] = prob.n_elem / ((ms_r + ms_g) * 1e-3)
        if name == "fp64":
            g64 = g.clone()
        else:
            g32 = g.clone()
    rng = np.random.default_rng(7)
    sample = rng.choice(prob.n_elem, 32, replace=False)

    def central_differences(rel_h):
        fd = []
        for e in sample:
            h = rel_h * float(prob.E_elem[e])
            Ls = []
            for sgn in (1, -1):
                Ep = E.clone()
                Ep[e] += sgn * h
                Rp = mesh.residual(u, E_elem=Ep)
                Ls.append(0.5 * float(mesh.norm2(Rp).item()) ** 2)
            fd.append((Ls[0] - Ls[1]) / (2 * h))
        return np.array(fd)

    # h = 1e-6 E_e as the workload states, and h = 1e-2 E_e: L is exactly quadratic in E_e, so the
    # larger step has no truncation error either and lifts the difference of L above its rounding
    fd = central_differences(1e-6)
    fd_exact = central_differences(1e-2)
    gs = g64.cpu().numpy()[sample]
    # oracle gradient on the sampled elements: R at their nodes from the adjacent elements
    om = oracle.Mesh.of(prob)
    ptr, eidx = oracle.node_elements(prob.conn, prob.n_nodes)
    g_ref = []
    for e in sample:
        nodes = prob.conn[e].astype(np.int64)
        Rn = np.zeros(24)
        for a, n in enumerate(nodes):
            for e2 in eidx[ptr[n]:ptr[n + 1]]:
                Re = oracle.element_of(om, int(e2), prob.u, tangent=False)
                a2 = int(np.where(prob.conn[e2] == n)[0][0])
                Rn[3 * a:3 * a + 3] += Re[3 * a2:3 * a2 + 3]
        Re = oracle.element_of(om, int(e), prob.u, tangent=False)
        g_ref.append(float(Rn @ Re) / float(prob.E_elem[e]))
    g_ref = np.array(g_ref)
    scale = np.max(np.abs(g_ref))
    out["fd_max_rel_err_fp64"] = float(np.max(np.abs(gs - fd)) / scale)
    out["fd_h1e-2_max_rel_err_fp64"] = float(np.max(np.abs(gs - fd_exact)) / scale)
    out["oracle_max_rel_err_fp64"] = float(np.max(np.abs(gs - g_ref)) / scale)
    out["oracle_max_rel_err_fp32"] = float(np.max(np.abs(g32.cpu().numpy()[sample] - g_ref)) / scale)
    mesh.close()
    return out


def newton_counts(J, torch, I, prob, mesh, stretch=0.01):
    """Newton steps and CG iterations to a 1e-10 relative FP64 residual, per tangent precision.

    Roller conditions with a 1% stretch; the initial guess is the affine stretch u = stretch X_1 e_1
    (it meets the rollers exactly).  Inexact Newton: Jacobi-CG to 1e-6 relative per step.
    """
    n = round(prob.n_elem ** (1.0 / 3.0))
    dofs, vals = I.roller_bcs(prob.coords, stretch)
    u0 = np.zeros(prob.n_dof)
    u0[0::3] = stretch * prob.coords[:, 0]
    out = {"workload": f"fibre RVE {n}^3 neo-Hookean, rollers, 1% stretch from the affine guess, "
                       f"rtol 1e-10, Jacobi-CG rtol 1e-6"}
    for name, p in (("fp64", J.FP64), ("fp32", J.FP32), ("tf32", J.TF32)):
        u = torch.as_tensor(u0).cuda()
        t0 = time.perf_counter()
        info = J.newton_solve(mesh, u, dofs, vals, tangent_precision=p, rtol=1e-10, max_newton=20, cg_rtol=1e-6,
                              max_cg=50000, raise_on_fail=False)
        out[name] = {"newton_iters": info.newton_iters, "cg_iters_total": info.cg_iters_total,
                     "cg_capped": info.cg_capped, "final_rel_residual": info.final_rel_residual,
                     "seconds": time.perf_counter() - t0,
                     "device_seconds": {"residual": info.seconds_residual, "tangent": info.seconds_tangent,
                                        "solve": info.seconds_solve},
                     "history": [info.residual_history[k] for k in range(min(info.newton_iters + 1, 32))]}
    return out



# ------------------------------------------------------------------------------ slab arm
def main_slab(args, rank, world, local):
    """One 128^3 mesh split over the ranks into z-slabs of owned nodes (each rank holds every
    element touching its nodes: a one-element ghost layer).  A step is the headline step on
    every rank's sub-mesh, preceded by the halo exchange of u and v (NCCL point-to-point), with
    the norm from the ranks' owned sums of squares (all-gather, fixed-order sum).  Strong
    scaling: value = the mesh's elements / the slowest rank's step time."""
    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2604_22087_b300 import jetsci as J
    from paper_2604_22087_b300 import slab as S

    prob = make_problem(args.n)
    s = S.decompose(prob.coords, prob.conn, world)[rank]
    part = S.SlabMesh(s, prob.coords, prob.phase, prob.materials)
    mesh = part.mesh
    stream = torch.cuda.Stream()
    u = torch.as_tensor(s.scatter_owned(prob.u)).cuda()
    v = torch.as_tensor(s.scatter_owned(prob.v)).cuda()
    R, y, y2 = mesh.new_vector(), mesh.new_vector(), mesh.new_vector()
    vals = mesh.new_values(J.FP64)
    own = torch.empty(1, dtype=torch.float64, device="cuda")
    out = {}
    torch.cuda.synchronize()

    def step():
        with torch.cuda.stream(stream):
            if world > 1:
                S.exchange(s, u)
                S.exchange(s, v)
            mesh.tangent_csr(u, vals=vals, R=R, stream=stream)
            mesh.apply_tangent(None, v, y=y2, mode=J.CSR, vals=vals, stream=stream)
            mesh.apply_tangent(None, v, y=y, stream=stream)
            part.mesh.norm2(part.owned(R), out=own, stream=stream)
            out["norm"] = S.norm2_device(s, own) if world > 1 else own

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(max(3, args.warmup)):
        step()
    barrier()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        t0.record(stream)
        for _ in range(args.steps):
            step()
        t1.record(stream)
        t1.synchronize()
    barrier()
    ms_step = max_over_ranks(t0.elapsed_time(t1) / args.steps, world, "cuda")
    norm = float(out["norm"].item())

    # end to end: the owned part of u and v from pinned host memory, the owned rows of the CSR
    # product and the norm back, every step
    n_own = s.n_owned_dof
    u_h = torch.as_tensor(prob.u[s.dofs()[:n_own]]).pin_memory()
    v_h = torch.as_tensor(prob.v[s.dofs()[:n_own]]).pin_memory()
    y_h = torch.empty(n_own, dtype=torch.float64).pin_memory()
    n_h = torch.empty(1, dtype=torch.float64).pin_memory()

    def e2e_step():
        with torch.cuda.stream(stream):
            u[:n_own].copy_(u_h, non_blocking=True)
            v[:n_own].copy_(v_h, non_blocking=True)
        step()
        with torch.cuda.stream(stream):
            y_h.copy_(y2[:n_own], non_blocking=True)
            n_h.copy_(out["norm"], non_blocking=True)

    e2e_step()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    e1.synchronize()
    barrier()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, "cuda")
    if rank == 0:
        halo = sum(len(x) for x in s.recv.values())
        line = {"metric": METRIC, "value": prob.n_elem / (ms_step * 1e-3), "unit": "elem/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
                "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": dict(config_dict(prob, args.n), partition=f"z-slabs over {world} ranks, owner computes, "
                               f"one-element ghost layer; rank 0: {len(s.elems)} elements, {s.n_owned} owned "
                               f"nodes, {halo} halo DOFs received per exchange"),
                "e2e": {"value": prob.n_elem / (e2e_ms * 1e-3), "unit": "elem/s",
                        "h2d_bytes_per_step": 16 * n_own, "d2h_bytes_per_step": 8 * n_own + 8,
                        "note": "rank 0's owned u, v in and owned CSR product rows and the norm out"},
                "gpu_launches": args.steps * (2 * mesh.n_colours + 3), "clocks": clk.summary(),
                "residual_norm": norm, "device_flags": mesh.check()}
        print(json.dumps(line), flush=True)
    part.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


# ------------------------------------------------------------------------------ main arm
def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.partition == "slab":
        main_slab(args, rank, world, local)
        return
    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2604_22087_b300 import inputs as I
    from paper_2604_22087_b300 import jetsci as J

    prob = make_problem(args.n)
    mesh = J.Mesh.of(prob)
    stream = torch.cuda.Stream()
    u = torch.as_tensor(prob.u).cuda()
    v = torch.as_tensor(prob.v).cuda()
    R = mesh.new_vector()
    y = mesh.new_vector()
    y2 = mesh.new_vector()
    vals = mesh.new_values(J.FP64)
    nrm = torch.empty(1, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        mesh.tangent_csr(u, vals=vals, R=R, stream=stream)
        if ev is not None:
            ev[1].record(stream)
        mesh.apply_tangent(None, v, y=y2, mode=J.CSR, vals=vals, stream=stream)
        # matrix-free K(u) v at the linearisation the tangent call just stored (same u)
        mesh.apply_tangent(None, v, y=y, stream=stream)
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
    ms_tangent = statistics.mean(a.elapsed_time(b) for a, b in evs)
    ms_step = max_over_ranks(t0.elapsed_time(t1), world, "cuda") / args.steps
    value = weak_scaling_value(prob.n_elem, world, ms_step)
    flags = mesh.check()

    # ---- end to end through the public API with pinned host buffers, copies timed
    u_h = torch.as_tensor(prob.u).pin_memory()
    v_h = torch.as_tensor(prob.v).pin_memory()
    y_h = torch.empty(prob.n_dof, dtype=torch.float64).pin_memory()
    n_h = torch.empty(1, dtype=torch.float64).pin_memory()

    # Every step copies its inputs u and v from pinned host memory and its results (the CSR
    # product y2 and the norm) back, all inside the timed region, overlapped with the compute on
    # a second stream: u is double-buffered and step k+1's copy runs during step k; v goes in
    # while the tangent is assembled (the CSR product is the first call that reads v); y2 comes
    # back while the matrix-free product and the norm run.  A step ends when both streams are.
    cs = torch.cuda.Stream()
    ub = [u, torch.empty_like(u)]
    ev_u = [torch.cuda.Event(), torch.cuda.Event()]
    ev_v, ev_y = torch.cuda.Event(), torch.cuda.Event()

    def copy_u(k):
        with torch.cuda.stream(cs):
            ub[k % 2].copy_(u_h, non_blocking=True)
            ev_u[k % 2].record(cs)

    def e2e_step(k, last):
        uk = ub[k % 2]
        cs.wait_stream(stream)  # v, y2 and the other u buffer are no longer in use
        if not last:
            copy_u(k + 1)
        with torch.cuda.stream(cs):
            v.copy_(v_h, non_blocking=True)
            ev_v.record(cs)
        stream.wait_event(ev_u[k % 2])
        mesh.tangent_csr(uk, vals=vals, R=R, stream=stream)
        stream.wait_event(ev_v)
        mesh.apply_tangent(None, v, y=y2, mode=J.CSR, vals=vals, stream=stream)
        ev_y.record(stream)
        with torch.cuda.stream(cs):
            cs.wait_event(ev_y)
            y_h.copy_(y2, non_blocking=True)
        mesh.apply_tangent(None, v, y=y, stream=stream)  # at the linearisation of the tangent at uk
        mesh.norm2(R, out=nrm, stream=stream)
        with torch.cuda.stream(stream):
            n_h.copy_(nrm, non_blocking=True)
        stream.wait_stream(cs)

    def e2e_run(n_steps):
        cs.wait_stream(stream)
        copy_u(0)
        for k in range(n_steps):
            e2e_step(k, k == n_steps - 1)

    e2e_run(1)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    e2e_run(args.steps)
    e1.record(stream)
    e1.synchronize()
    barrier()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, "cuda")

    extra = {}
    if rank == 0 and not args.no_forms:
        extra["forms"] = measure_forms(J, torch, I, mesh, prob, stream, u, v, vals, args)
    if rank == 0 and not args.no_extras:
        try:
            extra["adjoint"] = adjoint_workload(J, torch, I, stream)
        except Exception as ex:  # report, do not hide
            extra["adjoint"] = {"error": repr(ex)}
    if rank == 0 and not args.no_newton:
        extra["newton"] = newton_counts(J, torch, I, prob, mesh)

    if rank == 0:
        peaks, peak_kind = load_peaks()
        clocks = clk.summary()
        fp64_peak = 4.0 * 148 * peaks.get("sm_max_mhz", 2032.0) * 1e6 / 1e12  # 2 DFMA / clk / SM
        achieved = TANGENT_FP64_FLOP_PER_ELEM * prob.n_elem / (ms_tangent * 1e-3) / 1e12
        hbm = TANGENT_BYTES_PER_ELEM_FP64 * prob.n_elem / (ms_tangent * 1e-3) / 1e9
        line = {
            "metric": METRIC, "value": value, "unit": "elem/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config_dict(prob, args.n),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                         "frac": achieved / fp64_peak,
                         "traffic": TANGENT_DRAM_BYTES_PER_ELEM_FP64 * prob.n_elem,
                         "traffic_note": "bytes per tangent call (8 colour launches), ncu at 64^3 scaled by elements",
                         "kernel": "k_tangent<double,double>",
                         "peak_source": "FP64 pipe: 2 DFMA/clk/SM (measured FP64 FMA rate) x 2 flop x 148 SMs x the maximum SM clock",
                         "flop_note": "achieved counts the flops this formulation executes (12,308 per element); "
                                      "the pair form that accumulated the geometric term per Gauss point executed "
                                      "16,860 for the same tangent, so fewer flops in less time can lower frac",
                         "ms_per_launch_group": ms_tangent,
                         "fp64_pipe_instr_frac": TANGENT_FP64_INSTR_PER_ELEM * prob.n_elem / (ms_tangent * 1e-3) /
                                                 (2.0 * 148 * peaks.get("sm_max_mhz", 2032.0) * 1e6),
                         "fp64_pipe_instr_note": "FP64-pipe instructions (DFMA, DADD, DMUL: 6,876 per element, ncu) "
                                                 "per second over the pipe's 2 per clock per SM: the share of the "
                                                 "pipe's issue slots the executed work fills (frac counts a DADD or "
                                                 "DMUL as 1 flop against a peak of 2)",
                         "hbm_achieved_gbs": hbm,
                         "hbm_frac": hbm / peaks["hbm_gbs"], "hbm_peak_kind": peak_kind},
            "e2e": {"value": world * prob.n_elem / (e2e_ms * 1e-3), "unit": "elem/s",
                    "h2d_bytes_per_step": 2 * prob.n_dof * 8, "d2h_bytes_per_step": prob.n_dof * 8 + 8,
                    "note": "in: u and v from pinned host memory; out: the CSR product y and ||R||. The "
                            "residual R, the CSR values and the matrix-free product stay on the device "
                            "(a device-resident Newton driver reads only the norm)"},
            # per step: k_tangent and k_apply_mf once per colour, k_spmv, two norm passes
            "gpu_launches": args.steps * (2 * mesh.n_colours + 3),
            "clocks": clocks, "device_flags": flags,
        }
        line.update(extra)
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(prob, args.cpu_seconds)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def measure_forms(J, torch, I, mesh, prob, stream, u, v, vals64, args):
    """Per-entry-point device times (ms, elem/s) and errors vs the FP64 oracle on sampled rows."""
    out = {}
    so = SampledOracle(prob)
    rp, col = mesh.pattern()
    rp_h, col_h = rp.cpu().numpy(), col.cpu().numpy()
    R = mesh.new_vector()
    y = mesh.new_vector()

    def rec(name, ms, extra=None):
        d = {"ms": ms, "elem_per_s": prob.n_elem / (ms * 1e-3)}
        if extra:
            d.update(extra)
        out[name] = d

    for name, p in (("fp64", J.FP64), ("df64", J.DF64), ("fp32", J.FP32), ("tf32", J.TF32)):
        vv = vals64 if p in (J.FP64, J.DF64) else mesh.new_values(p)
        rec(f"residual_{name}", timeit(lambda: mesh.residual(u, R=R, precision=p, stream=stream), stream))
        ms = timeit(lambda: mesh.tangent_csr(u, vals=vv, R=R, precision=p, stream=stream), stream)
        torch.cuda.synchronize()
        err = so.errors(gather_rows(R, so.nodes), gather_vals(vv, rp_h, so.nodes), None, rp_h, col_h)
        rec(f"tangent_csr_{name}", ms, {"err_vs_oracle": err})
        ms = timeit(lambda: mesh.apply_tangent(u, v, y=y, precision=p, stream=stream), stream)
        torch.cuda.synchronize()
        rec(f"apply_matrix_free_{name}", ms, {"err_vs_oracle": so.errors(None, None, gather_rows(y, so.nodes), rp_h, col_h)})
        if p in (J.FP64, J.DF64):
            # at the linearisation stored by the tangent call above (u not read again)
            mesh.tangent_csr(u, vals=vv, R=R, precision=p, stream=stream)
            ms = timeit(lambda: mesh.apply_tangent(None, v, y=y, precision=p, stream=stream), stream)
            torch.cuda.synchronize()
            rec(f"apply_matrix_free_{name}_stored_linearisation", ms,
                {"err_vs_oracle": so.errors(None, None, gather_rows(y, so.nodes), rp_h, col_h)})
        if p in (J.FP64, J.FP32):
            # 100 back-to-back products on the assembled matrix (the paper's repeated-SpMV
            # comparison, Section V); ms is per product
            ms = timeit(lambda: mesh.apply_tangent(None, v, y=y, mode=J.CSR, vals=vv, precision=p, stream=stream),
                        stream, reps=100)
            torch.cuda.synchronize()
            gbs = SPMV_BYTES_PER_NNZ[name] * mesh.nnz / (ms * 1e-3) / 1e9
            rec(f"spmv_csr_{name}", ms, {"err_vs_oracle": so.errors(None, None, gather_rows(y, so.nodes), rp_h, col_h),
                                         "algorithmic_gbs": gbs, "products_timed": 100})
        if p not in (J.FP64, J.DF64):
            del vv
            torch.cuda.empty_cache()
    # The same step with two-float (DF64) element arithmetic on the FP32 pipes: tangent CSR with
    # fused R (FP64 values), CSR K.v, matrix-free DF64 K.v at the linearisation the tangent stored,
    # and the FP64 norm.  An FP64-accurate alternative reported beside the IEEE FP64 headline,
    # never in its place.
    nrm = torch.empty(1, dtype=torch.float64, device="cuda")
    y2 = mesh.new_vector()

    def df64_step():
        mesh.tangent_csr(u, vals=vals64, R=R, precision=J.DF64, stream=stream)
        mesh.apply_tangent(None, v, y=y2, mode=J.CSR, vals=vals64, precision=J.DF64, stream=stream)
        # at the linearisation the two-float tangent stored, as in the FP64 step
        mesh.apply_tangent(None, v, y=y, precision=J.DF64, stream=stream)
        mesh.norm2(R, out=nrm, stream=stream)

    ms = timeit(df64_step, stream)
    torch.cuda.synchronize()
    err = so.errors(gather_rows(R, so.nodes), gather_vals(vals64, rp_h, so.nodes), gather_rows(y, so.nodes), rp_h,
                    col_h)
    rec("step_df64", ms, {"err_vs_oracle": err})

    # The same step with FP32 element arithmetic (FP32 CSR values, matrix-free FP32 K.v from u).
    vals32 = mesh.new_values(J.FP32)

    def fp32_step():
        mesh.tangent_csr(u, vals=vals32, R=R, precision=J.FP32, stream=stream)
        mesh.apply_tangent(None, v, y=y2, mode=J.CSR, vals=vals32, precision=J.FP32, stream=stream)
        mesh.apply_tangent(u, v, y=y, precision=J.FP32, stream=stream)
        mesh.norm2(R, out=nrm, stream=stream)

    rec("step_fp32", timeit(fp32_step, stream))

    # The surrogate step's calls (tangent CSR + R, CSR K.v, norm) with the plain law in FP32: the
    # like-for-like comparison for the surrogate, which also runs FP32 element arithmetic.
    def fp32_csr_step():
        mesh.tangent_csr(u, vals=vals32, R=R, precision=J.FP32, stream=stream)
        mesh.apply_tangent(None, v, y=y2, mode=J.CSR, vals=vals32, precision=J.FP32, stream=stream)
        mesh.norm2(R, out=nrm, stream=stream)

    rec("step_fp32_csr_only", timeit(fp32_csr_step, stream))
    del vals32
    torch.cuda.empty_cache()

    # The calls a surrogate step has (tangent CSR + R, CSR K.v, norm; there is no matrix-free
    # surrogate product), in plain FP64, for a like-for-like comparison with step_surrogate.
    def fp64_csr_step():
        mesh.tangent_csr(u, vals=vals64, R=R, stream=stream)
        mesh.apply_tangent(None, v, y=y2, mode=J.CSR, vals=vals64, stream=stream)
        mesh.norm2(R, out=nrm, stream=stream)

    rec("step_fp64_csr_only", timeit(fp64_csr_step, stream))
    # the FP32 forms against their own bound (instruction issue) and against HBM
    peaks, _ = load_peaks()
    issue_peak = 4.0 * 148 * peaks.get("sm_max_mhz", 2032.0) * 1e6  # warp instructions per second
    for name, f in FP32_FORMS.items():
        sec = out[name]["ms"] * 1e-3
        out[name]["roofline"] = {
            "bound": "issue", "kernels": f["kernels"],
            "issue_frac": f["warp_instr"] * prob.n_elem / sec / issue_peak,
            "warp_instr_per_elem": f["warp_instr"],
            "hbm_frac_algorithmic": f["alg_bytes"] * prob.n_elem / sec / 1e9 / peaks["hbm_gbs"],
            "hbm_frac_dram": f["dram_bytes"] * prob.n_elem / sec / 1e9 / peaks["hbm_gbs"],
            "dram_bytes_per_elem": f["dram_bytes"], "algorithmic_bytes_per_elem": f["alg_bytes"],
            **{k: v for k, v in f.items() if k.startswith("tensor_pipe")},
            "note": "issue_frac: ncu warp instructions per element x elements / time over 4 per clock per SM "
                    "at the maximum SM clock; hbm_frac_*: algorithmic and ncu DRAM bytes per element over "
                    "the measured HBM peak"}
    if not args.no_extras:
        s, tinfo = train_surrogate(J, torch, I)
        out["surrogate_training"] = tinfo
        J.attach_surrogate(mesh, s)
        vv = mesh.new_values(J.SURROGATE)
        ms = timeit(lambda: mesh.tangent_csr(u, vals=vv, R=R, precision=J.SURROGATE, stream=stream), stream)
        torch.cuda.synchronize()
        fb = J.surrogate_fallbacks(mesh)
        err = so.errors(gather_rows(R, so.nodes), gather_vals(vv, rp_h, so.nodes), None, rp_h, col_h)
        rec("tangent_csr_surrogate", ms, {"err_vs_oracle_neo_hookean": err, "fallback_gauss_points": fb,
                                          "gauss_points": 8 * prob.n_elem})
        rec("residual_surrogate", timeit(lambda: mesh.residual(u, R=R, precision=J.SURROGATE, stream=stream), stream))

        def surrogate_step():
            mesh.tangent_csr(u, vals=vv, R=R, precision=J.SURROGATE, stream=stream)
            mesh.apply_tangent(None, v, y=y2, mode=J.CSR, vals=vv, precision=J.SURROGATE, stream=stream)
            mesh.norm2(R, out=nrm, stream=stream)

        ms = timeit(surrogate_step, stream)
        rec("step_surrogate", ms, {"vs_step_fp64_csr_only": out["step_fp64_csr_only"]["ms"] / ms,
                                   "vs_step_fp32_csr_only": out["step_fp32_csr_only"]["ms"] / ms})
        J.attach_surrogate(mesh, None)
        del vv
        torch.cuda.empty_cache()
    return out


if __name__ == "__main__":
    main()
