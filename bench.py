"""Benchmark: stiffness nonzeros assembled per second, surrogate vs exact, on one GB300.

One step = the whole hot path once: surrogate assembly of the stiffness
matrix (basis and pair tables, coefficient field, sum-factorised quadrature of
the frame and sample rows, per-offset spline interpolation, surrogate fill
with the kernel-preserving diagonal) followed by one stencil SpMV with it.
The exact Gauss-quadrature assembly of the same patch is timed the same way
and reported beside it, and so are the mass matrix of the same patch (its
symmetric surrogate and exact assembly), the kappa adjoint and the batch of
256 patches (outside the timed region).  Default workload: 3-D patch, p = 4, 96^3 elements
(10^6 DoFs, 6.8e8 nonzeros), M = 8, q = 3, FP64 values (x_i = xi_i + 0.03 prod sin(pi xi_j),
kappa = exp(0.5 sin(2 pi x) cos(2 pi y) sin(2 pi z))), synthetic and seeded.  Beside it the line
reports the FP32-value precision tier of the same patch and the 64^3 p = 3 FP64 patch.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload NAME]

Under torchrun (N > 1) every rank assembles its own replica of the workload
(the benchmark is one patch; replicas only) and the time is the max over ranks.
``--impl reference`` times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import iga_workloads as W  # noqa: E402

METRIC = "stiffness nonzeros assembled/s, surrogate vs exact on GB300 at stated entry error"
UNIT = "nnz/s"
FP64_FLOPS_PER_SM_CLK = 4          # 2 FP64 FMA per SM per clock (1.25 TFLOP/s nominal at 2.07 GHz, 152 SMs)
FP32_FLOPS_PER_SM_CLK = 256        # 128 FP32 FMA per SM per clock (80.5 TFLOP/s at 2.07 GHz)


# ---------------------------------------------------------------------------
# distributed helpers (rank 0 prints; time is the max over ranks)
# ---------------------------------------------------------------------------
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def init_dist(world: int, backend: str):
    if world <= 1:
        return None
    import torch.distributed as dist
    if not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)
    return dist


def barrier(dist, device=None):
    if dist is not None:
        if device is not None:
            dist.barrier(device_ids=[device.index]) if device.type == "cuda" else dist.barrier()
        else:
            dist.barrier()


def max_over_ranks(dist, value: float, device) -> float:
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_value(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Whole-job throughput: units all ranks processed / max time over ranks."""
    return units_per_rank * world / seconds_max


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        # raw nvidia-smi samples; IGA_BENCH_LOG_DIR keeps them where the caller wants them
        log_dir = os.environ.get("IGA_BENCH_LOG_DIR") or tempfile.gettempdir()
        self.path = os.path.join(log_dir, f"clocks_bench_{os.getpid()}.csv")
        self.gpu = gpu_index

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = max(smax, float(parts[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if parts[5 + k].lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# algorithmic work model of the quadrature stages (what the kernels execute)
# ---------------------------------------------------------------------------
def _union_count(p, m, M):
    """Sample rows per direction with per-offset domains: the lattice p + aM in the
    cardinal range [p, m-p-1] and the p + 1 first and last cardinal indices."""
    c0, c1 = p, m - p - 1
    return len(set(range(c0, c1 + 1, M)) | set(range(c0, min(c0 + p, c1) + 1)) | set(range(max(c1 - p, c0), c1 + 1)))


def _boxes(prob, M, surrogate, domains="common"):
    """Row boxes of the assembly: whole patch (exact) or frame slabs + one-row sample boxes."""
    p, m, dim = prob.p, list(prob.m), prob.dim
    if not surrogate:
        return [[(0, md) for md in m]], 0
    k0 = p if domains == "per_offset" else 2 * p
    k1 = [md - k0 - 1 for md in m]
    if any(b < k0 for b in k1):
        return [[(0, md) for md in m]], 0
    boxes = []
    full = [(0, md) for md in m]
    inner = [(k0, b - k0 + 1) for b in k1]
    for d in reversed(range(dim)):
        for lo, R in ((0, k0), (k1[d] + 1, m[d] - 1 - k1[d])):
            bx = []
            for e in range(dim):
                if e == d:
                    bx.append((lo, R))
                elif e > d:
                    bx.append(inner[e])
                else:
                    bx.append(full[e])
            boxes.append(bx)
    if domains == "per_offset":
        ns = [_union_count(p, md, M) for md in m]
    else:
        ns = [(b - k0) // M + 1 + (1 if (b - k0) % M else 0) for b in k1]
    return boxes, int(np.prod(ns))


def box_sym(n_boxes, surrogate, symmetric=True):
    """Symmetry mode of each explicit box (the order of `_boxes`): +1 computes the upper offsets,
    -1 the lower ones, 0 all.  The stiffness matrix is symmetric; exact assembly (or a surrogate
    without Omega~) mirrors over the whole patch, the surrogate over the two frame slabs normal to
    the slowest direction (the first two boxes).  Off with the tensor-core stage X."""
    sym = [0] * n_boxes
    if not symmetric:
        return sym
    if not surrogate or n_boxes == 1:
        sym[0] = 1
    elif n_boxes >= 2:
        sym[0], sym[1] = 1, -1
    return sym


def stage_fmas(prob, M, surrogate, domains="common", symmetric=True):
    """Multiply-adds that stage Z / Y / X need (per launch), closed form over the boxes.  A symmetric
    box needs the partial sums of the offsets on its side only: stage Z the delta_2 of that sign,
    stage Y with delta_2 = 0 the delta_1 of that sign, stage X on the centre line (delta_2 = delta_1
    = 0) the delta_0 of that sign."""
    p, dim = prob.p, prob.dim
    Q, Wd = p + 1, 2 * p + 1
    n_el = list(prob.n_el)

    def cnt(i, ne, mode):     # Gauss point x partner pairs of row i: mode 0 all, +1 delta >= 0, -1 delta <= 0
        n = 0
        for a in range(p + 1):
            if 0 <= i - p + a < ne:
                n += Q * (Q if mode == 0 else (a + 1 if mode > 0 else p - a + 1))
        return n

    def G(lo, R, ne):         # Gauss points of the box in one direction
        elo = max(0, lo - p)
        ehi = min(ne - 1, lo + R - 1)
        return (ehi - elo + 1) * Q

    boxes, nsamp = _boxes(prob, M, surrogate, domains)
    syms = box_sym(len(boxes), surrogate and nsamp > 0, symmetric)
    samp_box = [(2 * p, 1)] * dim           # every sample box: one row, p + 1 elements per direction
    tot = {"stage_z": 0, "stage_y": 0, "stage_x": 0}
    items = [(b, 1, sg) for b, sg in zip(boxes, syms)] + ([(samp_box, nsamp, 0)] if nsamp else [])
    for bx, mult, sg in items:
        rows = [range(bx[d][0], bx[d][0] + bx[d][1]) for d in range(dim)]
        s_all = [sum(cnt(i, n_el[d], 0) for i in rows[d]) for d in range(dim)]
        s_sym = [sum(cnt(i, n_el[d], sg) for i in rows[d]) for d in range(dim)]
        g = [G(bx[d][0], bx[d][1], n_el[d]) for d in range(dim)]
        R = [bx[d][1] for d in range(dim)]
        # lines of the slower offsets: (full, centre) = delta strictly on the box's side, delta = 0
        nf, nc = (Wd, 0) if sg == 0 else (p, 1)
        if dim == 3:
            tot["stage_z"] += mult * 8 * s_sym[2] * g[1] * g[0]
            tot["stage_y"] += mult * 9 * g[0] * R[2] * (nf * s_all[1] + nc * s_sym[1])
            tot["stage_x"] += mult * 4 * R[2] * (nf * R[1] * Wd * s_all[0]
                                                 + nc * R[1] * (nf * s_all[0] + nc * s_sym[0]))
        else:
            tot["stage_y"] += mult * 4 * g[0] * s_sym[1]
            tot["stage_x"] += mult * 4 * R[1] * (nf * s_all[0] + nc * s_sym[0])
    return tot


# FP32 flops of one double-float multiply-accumulate (arith.cuh, PolDF::mac):
# 1 FMUL + 3 FFMA + 8 FADD/FSUB = 15 flops in 12 instructions, so the FP32 pipe
# caps this instruction mix at 15 / 24 = 62.5 % of its FFMA peak.
DF64_FLOPS_PER_MAC = 15


def kernel_work(prob, wl, arith: str, surrogate=True, domains="common"):
    """Per-launch algorithmic work: flops of the contraction stages in the arithmetic
    they run in, bytes for the SpMV."""
    esz = 8 if wl.dtype == "f64" else 4
    # the tensor-core stage X (df64_tc, bf16x3) writes every offset: no symmetric boxes
    tc = arith in ("df64_tc", "bf16x3")
    fm = stage_fmas(prob, wl.M, surrogate, domains, symmetric=not tc)
    if tc:
        # stage X runs on the tensor cores (no FP32-pipe figure); stages Z and Y in the CUDA-core
        # arithmetic of the mode: double-float for df64_tc, FP32 for bf16x3
        fm = {k: v for k, v in fm.items() if k != "stage_x"}
    if arith == "fp64":
        work = {k: {"bound": "alu", "pipe": "fp64", "flops": 2.0 * v} for k, v in fm.items() if v}
    elif arith in ("df64", "df64_tc"):
        work = {k: {"bound": "alu", "pipe": "fp32 (double-float)", "flops": float(DF64_FLOPS_PER_MAC) * v}
                for k, v in fm.items() if v}
    else:
        work = {k: {"bound": "alu", "pipe": "fp32", "flops": 2.0 * v} for k, v in fm.items() if v}
    work["spmv"] = {"bound": "hbm", "bytes": float(prob.S * prob.N * esz + 2 * prob.N * esz)}
    return work


def alu_peak_tflops(pipe: str, sm_mhz: float) -> float:
    """152 SMs x flops per SM per clock x clock: FP64 2 FMA/clk (4 flops), FP32 128 FMA/clk (256 flops)."""
    per_clk = FP64_FLOPS_PER_SM_CLK if pipe == "fp64" else FP32_FLOPS_PER_SM_CLK
    return 152 * per_clk * sm_mhz * 1e6 / 1e12


def source_hash(rel_paths) -> str:
    """Hash of the source files that define a kernel (a path or a list of paths)."""
    h = hashlib.sha256()
    for rel in ([rel_paths] if isinstance(rel_paths, str) else rel_paths):
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


_CSRC = "paper_1904_06971_gb300/csrc/"
_QUAD = [_CSRC + "quad_bodies.cuh", _CSRC + "k_quad.cu", _CSRC + "arith.cuh"]
KERNEL_SOURCE = {"stage_z": _QUAD, "stage_y": _QUAD, "stage_x": _QUAD, "coef": _CSRC + "k_tables.cu",
                 "fill": _CSRC + "k_spline.cu", "spmv": _CSRC + "k_spmv.cu"}


def ncu_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the current source."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path))
        rec = d.get(workload, {}).get(kernel)
        if rec and rec.get("source_sha") == source_hash(KERNEL_SOURCE.get(kernel, "bench.py")):
            return float(rec["dram_bytes_per_launch"])
    except (ValueError, KeyError, OSError):
        return None
    return None


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            return json.load(open(path)), "measured"
        except ValueError:
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ---------------------------------------------------------------------------
# CPU oracle leg
# ---------------------------------------------------------------------------
class OracleTimer:
    """The oracle's surrogate assembly timed on a bounded sample of one workload.

    The setup (exact quadrature of every sample row, the interpolation solves) is
    timed once in full; each step times `rows` seeded random rows of the
    surrogate and extrapolates them to all N rows."""

    def __init__(self, wl, domains):
        import oracle
        from oracle import per_offset
        self.wl, self.domains = wl, domains
        prob = wl.problem
        t0 = time.perf_counter()
        if domains == "per_offset":
            self.setup = per_offset.per_offset_setup(prob, wl.M, wl.q)
            self.n_setup = int(np.prod([len(u) for u in self.setup.union]))
            self._rows = lambda rows: per_offset.per_offset_rows(prob, wl.M, wl.q, rows, self.setup)
        else:
            self.setup = oracle.surrogate_setup(prob, wl.M, wl.q)
            self.n_setup = int(np.prod([len(s) for s in self.setup.samples])) if not self.setup.empty else 0
            self._rows = lambda rows: oracle.surrogate_rows(prob, wl.M, wl.q, rows, self.setup)
        self.t_setup = time.perf_counter() - t0
        self.cores = oracle.num_threads()

    def step(self, rows_budget: int, seed: int):
        prob = self.wl.problem
        rows = W.sample_rows(prob.N, rows_budget, seed=seed)
        t0 = time.perf_counter()
        self._rows(rows)
        t_rows = time.perf_counter() - t0
        t_full = self.t_setup + t_rows * prob.N / len(rows)
        sample = (f"oracle surrogate assembly ({self.domains} domains): all {self.n_setup} exact sample rows "
                  f"({self.t_setup:.2f} s, timed once) plus {len(rows)} of {prob.N} rows (seeded uniform, seed "
                  f"{seed}), time extrapolated to all rows")
        return prob.nnz / t_full, t_rows, sample


def cpu_baseline(wl, domains, target_s: float = 15.0):
    timer = OracleTimer(wl, domains)
    # calibrate the row count so that the sampled rows cost about target_s seconds
    _, t64, _ = timer.step(64, seed=0)
    k = int(min(wl.problem.N, max(64, (target_s - timer.t_setup) / max(t64 / 64, 1e-6))))
    v, t_rows, sample = timer.step(k, seed=1)
    return {"value": v, "unit": UNIT, "cores": timer.cores, "kind": "oracle", "sample": sample,
            "seconds": timer.t_setup + t_rows}


def reference_rows(timer, steps_total: int, budget_s: float = 150.0, cap_s: float = 15.0) -> int:
    """Rows per reference step: calibrated like the cpu_baseline leg (a timed pilot of 64 rows) so that
    one step costs min(cap_s, budget_s / steps_total) seconds of row work; the per-call overhead is then
    amortised as in the baseline leg and the whole run stays within a few minutes."""
    _, t64, _ = timer.step(64, seed=10 ** 6)
    per_step = min(cap_s, max(1.0, budget_s / max(1, steps_total)))
    return int(min(timer.wl.problem.N, max(64, per_step / max(t64 / 64, 1e-6))))


def run_reference(args, wl):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    timer = OracleTimer(wl, args.domains)
    rows = args.ref_rows or reference_rows(timer, args.warmup + args.steps)
    vals = []
    sample = ""
    for k in range(args.warmup + args.steps):
        v, _, sample = timer.step(rows, seed=k)
        if k >= args.warmup:
            vals.append(v)
    value = float(np.mean(vals))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": wl.problem.nnz / value * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded); FP64 CPU oracle on the host cores",
        "config": config_of(wl, world, args.domains),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": timer.cores, "kind": "oracle", "sample": sample,
                         "rows_per_step": rows},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def config_of(wl, world, domains="common"):
    prob = wl.problem
    return {"workload": wl.name, "dim": prob.dim, "p": prob.p, "n_el": list(prob.n_el), "M": wl.M, "q": wl.q,
            "domains": domains,
            "map": f"{prob.map_kind} amp {prob.map_amp}",
            "kappa": f"{prob.kappa_kind} a {prob.kappa_a} b {prob.kappa_b}",
            "N": prob.N, "nnz": prob.nnz, "slots": prob.S * prob.N, "values": wl.dtype,
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
            "l2": "256 MiB L2 flush written between timed steps; each step writes > 1 GB"}


# ---------------------------------------------------------------------------
# GPU leg
# ---------------------------------------------------------------------------
def adjoint_report(iga, torch, dev, steps: int, warmup: int):
    """Gradient of L = ybar^T A~(c) x with respect to the 16^3 B-spline control values of
    kappa and x on the 48^3, p = 3 workload: forward (assembly + SpMV) and backward
    (iga_kappa_gradient + SpMV), CUDA events, inputs resident."""
    wl = W.CFG_3D_P3_BSPLINE
    prob = wl.problem
    gen = torch.Generator(device="cpu").manual_seed(wl.seed)
    x = torch.randn(prob.N, generator=gen, dtype=torch.float64).to(dev)
    ybar = torch.randn(prob.N, generator=gen, dtype=torch.float64).to(dev)
    ctrl = torch.tensor(prob.kappa_ctrl, dtype=torch.float64, device=dev)
    out = {"workload": wl.name, "controls": ctrl.numel(), "unit": "ms"}
    for M, key in ((wl.M, "surrogate"), (0, "exact")):
        A = iga.assemble_surrogate(prob, M, wl.q, kappa_ctrl=ctrl) if M else iga.assemble_exact(prob, kappa_ctrl=ctrl)
        y = torch.empty_like(x)
        gx = torch.empty_like(x)

        def fwd():
            if M:
                iga.assemble_surrogate(prob, M, wl.q, out=A, kappa_ctrl=ctrl)
            else:
                iga.assemble_exact(prob, out=A, kappa_ctrl=ctrl)
            A.apply(x, y)

        def bwd():
            iga.kappa_gradient(prob, ybar, x, M, wl.q, kappa_ctrl=ctrl)
            A.apply(ybar, gx)

        res = {}
        for name, fn in (("forward", fwd), ("backward", bwd)):
            for _ in range(warmup):
                fn()
            torch.cuda.synchronize()
            iga.profile_read()
            iga.profile_enable(True)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(steps):
                fn()
            b.record()
            torch.cuda.synchronize()
            iga.profile_enable(False)
            prof = iga.profile_read()
            res[name + "_ms"] = a.elapsed_time(b) / steps
            res[name + "_kernels"] = {k: round(v[1] / steps, 4) for k, v in prof.items() if v[0]}
        out[key] = res
        A.destroy()
    return out


def mass_report(iga, torch, wl, steps: int, warmup: int):
    """Mass matrix of the bench workload's patch (Sec. 8): the symmetric surrogate
    (eq. DefinitionOfSurrogateMatrixSymmetric, same M and q) against the exact
    assembly, CUDA events, matrices resident; entry error of the surrogate."""
    prob = wl.problem
    stream = torch.cuda.current_stream()
    out = {"workload": wl.name, "unit": "nnz/s"}
    mats = {}
    for key in ("surrogate", "exact"):
        A = iga.assemble_mass_surrogate(prob, wl.M, wl.q, dtype=wl.dtype) if key == "surrogate" \
            else iga.assemble_mass(prob, dtype=wl.dtype)

        def step():
            if key == "surrogate":
                iga.assemble_mass_surrogate(prob, wl.M, wl.q, dtype=wl.dtype, out=A)
            else:
                iga.assemble_mass(prob, dtype=wl.dtype, out=A)

        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        iga.profile_read()
        iga.profile_enable(True)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            step()
        b.record(stream)
        torch.cuda.synchronize()
        iga.profile_enable(False)
        prof = iga.profile_read()
        ms = a.elapsed_time(b) / steps
        out[key] = {"value": prob.nnz / (ms * 1e-3), "ms_per_step": ms,
                    "kernels": {k: round(v[1] / steps, 4) for k, v in prof.items() if v[0]}}
        mats[key] = A
    vs, ve = mats["surrogate"].values(), mats["exact"].values()
    out["entry_error"] = ((vs.double() - ve.double()).abs().max() / ve.double().abs().max()).item()
    out["speedup_vs_exact"] = out["exact"]["ms_per_step"] / out["surrogate"]["ms_per_step"]
    del vs, ve
    for A in mats.values():
        A.destroy()
    return out


def batch_report(iga, torch, steps: int, warmup: int):
    """The 256-patch batching workload (FP32 values): eager per-patch assembly on one
    stream against the autotuned graph replay (one graph launch per step)."""
    items = W.batch_items()
    nnz = sum(prob.nnz for prob, _, _ in items)
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    mats = iga.assemble_batch(items, dtype="f32")            # creates the matrices
    torch.cuda.synchronize()
    t_create = time.perf_counter() - t0

    def eager():
        for (prob, M, q), A in zip(items, mats):
            iga.assemble_surrogate(prob, M, q, dtype="f32", out=A)

    def timed(fn):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = iga.launch_count()
        a.record(stream)
        for _ in range(steps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / steps, (iga.launch_count() - l0) // steps

    ms_eager, k_eager = timed(eager)

    def tuned(branches_ok, persistent_ok):
        # a fresh autotune restricted to the given candidate kinds, then timed cached replays
        iga.batch_release()
        iga.batch_set_modes(branches_ok, persistent_ok)
        t0 = time.perf_counter()
        iga.assemble_batch(items, dtype="f32", out=mats)      # capture + autotune
        torch.cuda.synchronize()
        t_tune = time.perf_counter() - t0
        branches, kernels, _, tuned_ms = iga.batch_info()
        persistent, bps, chunk = iga.batch_mode()
        ms, _ = timed(lambda: iga.assemble_batch(items, dtype="f32", out=mats))
        iga.batch_status()
        out = {"value": nnz / (ms * 1e-3), "ms_per_batch": ms, "kind": "persistent" if persistent else "branches",
               "branches": branches, "kernels_per_launch": kernels, "graph_launches_per_batch": 1,
               "capture_and_tune_s": t_tune, "tuned_replay_ms": tuned_ms}
        if persistent:
            out.update({"blocks_per_sm": bps, "items_per_claim": chunk})
        return out

    try:
        best = tuned(True, True)
        only_persistent = tuned(False, True)
        only_branches = tuned(True, False)
    finally:
        iga.batch_set_modes(True, True)
        iga.batch_release()
    for A in mats:
        A.destroy()
    return {"workload": "256 patches: 192 2-D (p 2..5, 16..256 el/dir) + 64 3-D (p 2..4, 8..48 el/dir), M in {4,8}, "
                        "q 3, FP32 values, seed 0",
            "patches": len(items), "nnz": nnz, "unit": "nnz/s",
            "graph": best, "persistent_only": only_persistent, "branches_only": only_branches,
            "eager_one_stream": {"value": nnz / (ms_eager * 1e-3), "ms_per_batch": ms_eager,
                                 "kernel_launches_per_batch": k_eager},
            "create_s": t_create}


def _time_steps(torch, step, steps: int, warmup: int, stream, profile_iga=None):
    """Mean CUDA-event time (ms) of `step` on `stream`, 256 MiB L2 flush between steps."""
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    if profile_iga is not None:
        profile_iga.profile_read()
        profile_iga.profile_enable(True)
    evs = []
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    prof = None
    if profile_iga is not None:
        profile_iga.profile_enable(False)
        prof = {k: round(v[1] / steps, 4) for k, v in profile_iga.profile_read().items() if v[0]}
    del flush
    return float(np.mean([a.elapsed_time(b) for a, b in evs])), prof


def fp32_tier_report(iga, torch, wl, A64, E64, exact_solution, args, steps: int = 10, warmup: int = 3):
    """The FP32-value precision tier of the same patch: surrogate (+ SpMV) and exact steps, the entry
    error of the FP32 matrices against the FP64 matrices of the same method (the FP64 values are parity-
    tested against the FP64 oracle at 1e-12; the FP32 ones at 1e-5), and the discrete-solution error of
    the FP32 surrogate's CG with FP64-residual iterative refinement against u_h of the exact FP64 matrix."""
    prob = wl.problem
    stream = torch.cuda.current_stream()
    gen = torch.Generator(device="cpu").manual_seed(0)
    x = torch.randn(prob.N, generator=gen, dtype=torch.float64).to(dtype=torch.float32, device="cuda")
    y = torch.empty_like(x)
    A = iga.assemble_surrogate(prob, wl.M, wl.q, dtype="f32")
    E = iga.assemble_exact(prob, dtype="f32")

    def s_step():
        iga.assemble_surrogate(prob, wl.M, wl.q, dtype="f32", out=A)
        A.apply(x, y)

    def e_step():
        iga.assemble_exact(prob, dtype="f32", out=E)
        E.apply(x, y)

    ms_s, prof_s = _time_steps(torch, s_step, steps, warmup, stream, iga)
    ms_e, _ = _time_steps(torch, e_step, max(3, steps // 2), warmup, stream)
    out = {"workload": wl.name.replace("_M8_q3", "_M8_q3_f32"), "values": "f32",
           "arith": {"contractions": iga.get_arithmetic("f32"), "fill": "fp32", "diagonal": "compensated fp32",
                     "spmv": "f32"},
           "unit": UNIT, "surrogate": {"value": prob.nnz / (ms_s * 1e-3), "ms_per_step": ms_s, "kernels": prof_s},
           "exact": {"value": prob.nnz / (ms_e * 1e-3), "ms_per_step": ms_e},
           "speedup_surrogate_vs_exact": ms_e / ms_s}
    vs32, vs64 = A.values().double(), A64.values()
    scale = vs64.abs().max().item()
    out["entry_error_vs_fp64_surrogate"] = float((vs32 - vs64).abs().max().item() / scale)
    del vs32
    ve32, ve64 = E.values().double(), E64.values()
    out["exact_entry_error_vs_fp64_exact"] = float((ve32 - ve64).abs().max().item() / ve64.abs().max().item())
    del ve32
    vs32 = A.values().double()
    out["surrogate_vs_exact_fp64_max_rel"] = float((vs32 - ve64).abs().max().item() / ve64.abs().max().item())
    del vs32, vs64, ve64
    if not args.no_solve:
        f = torch.from_numpy(W.rhs_vector(prob.N, seed=wl.seed)).to("cuda")
        u_e, _, _ = exact_solution(f)
        u_s, it_s, res_s = A.cg(f, tol=args.cg_tol, maxit=args.cg_maxit)
        err = u_s - u_e
        Ee = E64.apply(err).double()
        Eu = E64.apply(u_e).double()
        out["solution_error"] = {"rel_l2": float(err.norm() / u_e.norm()),
                                 "rel_energy": float(torch.sqrt(torch.dot(err, Ee) / torch.dot(u_e, Eu))),
                                 "cg_iters": it_s, "cg_rel_residual": res_s,
                                 "solver": "FP32 CG inner solves, FP64 residuals (iterative refinement)",
                                 "reference": "u_h of the exact FP64 matrix"}
    # the same steps with stage X of the cardinal rows on the tensor cores (BF16x3 parts, FP32 accumulation)
    saved = iga.get_arithmetic("f32")
    try:
        iga.set_arithmetic("f32", "bf16x3")
        At = iga.assemble_surrogate(prob, wl.M, wl.q, dtype="f32")
        Et = iga.assemble_exact(prob, dtype="f32")

        def s_step_tc():
            iga.assemble_surrogate(prob, wl.M, wl.q, dtype="f32", out=At)
            At.apply(x, y)

        def e_step_tc():
            iga.assemble_exact(prob, dtype="f32", out=Et)
            Et.apply(x, y)

        ms_st, prof_st = _time_steps(torch, s_step_tc, steps, warmup, stream, iga)
        ms_et, prof_et = _time_steps(torch, e_step_tc, max(3, steps // 2), warmup, stream, iga)
        tc = {"arith": "bf16x3 tensor-core stage X (cardinal rows), FP32 elsewhere",
              "surrogate": {"value": prob.nnz / (ms_st * 1e-3), "ms_per_step": ms_st, "kernels": prof_st},
              "exact": {"value": prob.nnz / (ms_et * 1e-3), "ms_per_step": ms_et, "kernels": prof_et},
              "speedup_surrogate_vs_exact": ms_et / ms_st}
        vt, v64 = At.values().double(), A64.values()
        tc["entry_error_vs_fp64_surrogate"] = float((vt - v64).abs().max().item() / v64.abs().max().item())
        vc = A.values().double()
        tc["entry_error_vs_fp32_cuda_cores"] = float((vt - vc).abs().max().item() / vc.abs().max().item())
        del vt, vc, v64
        vt, v64 = Et.values().double(), E64.values()
        tc["exact_entry_error_vs_fp64_exact"] = float((vt - v64).abs().max().item() / v64.abs().max().item())
        del vt, v64
        out["tensor_core"] = tc
        At.destroy()
        Et.destroy()
    finally:
        iga.set_arithmetic("f32", saved)
    A.destroy()
    E.destroy()
    return out


def equal_accuracy_report(iga, torch, wl, E, ms_exact, args, Ms=(2, 4, 6, 8, 12, 16), freqs=(20, 1), steps: int = 5,
                          warmup: int = 3):
    """Surrogate vs exact at equal accuracy of the discrete solution (Sec. 7.3): for the manufactured
    solutions u = prod sin(k pi x_d) (k = 20 and k = 1, the paper's high- and low-frequency loads;
    iga_manufactured_load) the discretisation error ||u - u_h||_a of the exact matrix (Galerkin
    orthogonality: a(u,u) - F.u_h) and, per sampling length M, the consistency error ||u_h - u~_h||_A of
    the surrogate, both relative to ||u||_a; the paper's rule of thumb keeps the consistency error at or
    below 5 % of the discretisation error.  Reports the surrogate step time per M and the speed-up over
    the exact step at the largest M that satisfies the rule.  When the discretisation error is below what
    FP64 resolves in a(u,u) - F.u_h (relative square under 1e-12), it is reported as unresolved."""
    prob = wl.problem
    stream = torch.cuda.current_stream()
    gen = torch.Generator(device="cpu").manual_seed(0)
    tdt = torch.float64 if wl.dtype == "f64" else torch.float32
    x = torch.randn(prob.N, generator=gen, dtype=torch.float64).to(dtype=tdt, device="cuda")
    y = torch.empty_like(x)
    times = {}
    for M in Ms:
        A = iga.assemble_surrogate(prob, M, wl.q, dtype=wl.dtype)

        def step():
            iga.assemble_surrogate(prob, M, wl.q, dtype=wl.dtype, out=A)
            A.apply(x, y)

        times[M], _ = _time_steps(torch, step, steps, warmup, stream)
        A.destroy()
    out = {"workload": wl.name, "norm": "energy a(.,.), relative to ||u||_a", "exact_ms_per_step": ms_exact,
           "rule": "consistency <= 5% of discretisation",
           "surrogate_ms_per_step": {str(M): times[M] for M in Ms}, "solutions": []}
    for k in freqs:
        F, en = iga.manufactured_load(prob, freq=k)
        energy = en.item()
        u_h, it_h, _ = E.cg(F, tol=args.cg_tol, maxit=args.cg_maxit)
        d2 = (energy - torch.dot(F, u_h).item()) / energy
        disc = float(np.sqrt(d2)) if d2 > 1e-12 else None
        rows = []
        for M in Ms:
            A = iga.assemble_surrogate(prob, M, wl.q, dtype=wl.dtype)
            u_s, it_s, _ = A.cg(F, tol=args.cg_tol, maxit=args.cg_maxit)
            d = (u_s - u_h).to(tdt)
            cons = float(np.sqrt(max(torch.dot(d.double(), E.apply(d).double()).item(), 0.0) / energy))
            rows.append({"M": M, "q": wl.q, "consistency_rel_energy": cons,
                         "consistency_over_discretisation": (cons / disc) if disc else None,
                         "speedup_vs_exact": ms_exact / times[M], "cg_iters": it_s})
            A.destroy()
        ok = [r for r in rows if r["consistency_over_discretisation"] is not None
              and r["consistency_over_discretisation"] <= 0.05]
        best = max(ok, key=lambda r: r["M"]) if ok else None
        out["solutions"].append({
            "u": f"prod_d sin({k} pi x_d)", "discretisation_rel_energy": disc,
            "discretisation_note": None if disc else "below FP64 resolution of a(u,u) - F.u_h",
            "exact_cg_iters": it_h, "per_M": rows, "largest_M_within_rule": best["M"] if best else None,
            "speedup_at_equal_accuracy": best["speedup_vs_exact"] if best else None})
    return out


def side_report(iga, torch, wl, steps: int, warmup: int):
    """Surrogate (+ SpMV) and exact steps of another workload, with the surrogate's entry error."""
    prob = wl.problem
    stream = torch.cuda.current_stream()
    gen = torch.Generator(device="cpu").manual_seed(0)
    tdt = torch.float64 if wl.dtype == "f64" else torch.float32
    x = torch.randn(prob.N, generator=gen, dtype=torch.float64).to(dtype=tdt, device="cuda")
    y = torch.empty_like(x)
    A = iga.assemble_surrogate(prob, wl.M, wl.q, dtype=wl.dtype)
    E = iga.assemble_exact(prob, dtype=wl.dtype)

    def s_step():
        iga.assemble_surrogate(prob, wl.M, wl.q, dtype=wl.dtype, out=A)
        A.apply(x, y)

    def e_step():
        iga.assemble_exact(prob, dtype=wl.dtype, out=E)
        E.apply(x, y)

    ms_s, prof_s = _time_steps(torch, s_step, steps, warmup, stream, iga)
    ms_e, prof_e = _time_steps(torch, e_step, steps, warmup, stream, iga)
    vs, ve = A.values().double(), E.values().double()
    err = float((vs - ve).abs().max().item() / ve.abs().max().item())
    del vs, ve
    A.destroy()
    E.destroy()
    return {"workload": wl.name, "values": wl.dtype, "unit": UNIT, "nnz": prob.nnz,
            "surrogate": {"value": prob.nnz / (ms_s * 1e-3), "ms_per_step": ms_s, "kernels": prof_s},
            "exact": {"value": prob.nnz / (ms_e * 1e-3), "ms_per_step": ms_e, "kernels": prof_e},
            "speedup_surrogate_vs_exact": ms_e / ms_s, "surrogate_vs_exact_max_rel": err}


def run_gpu(args, wl):
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = init_dist(world, "nccl")
    import paper_1904_06971_gb300 as iga
    iga.load()
    if args.arith:
        # the contraction arithmetic of the workload's value type
        if wl.dtype == "f64" and args.arith in ("fp32", "bf16x3"):
            raise SystemExit("--arith fp32 / bf16x3 apply to FP32-value workloads")
        iga.set_arithmetic(wl.dtype, args.arith)
    prob = wl.problem
    stream = torch.cuda.current_stream()
    primary = args.domains
    other = "common" if primary == "per_offset" else "per_offset"
    A = iga.assemble_surrogate(prob, wl.M, wl.q, dtype=wl.dtype, domains=primary)
    E = iga.assemble_exact(prob, dtype=wl.dtype)
    tdt = A.torch_dtype
    gen = torch.Generator(device="cpu").manual_seed(0)
    x = torch.randn(prob.N, generator=gen, dtype=torch.float64).to(dtype=tdt, device=dev)
    y = torch.empty_like(x)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)     # 256 MiB > L2

    def surr_step(mat, domains):
        def step():
            iga.assemble_surrogate(prob, wl.M, wl.q, dtype=wl.dtype, out=mat, domains=domains)
            mat.apply(x, y)
        return step

    def step_exact():
        iga.assemble_exact(prob, dtype=wl.dtype, out=E)
        E.apply(x, y)

    def timed(step, K, W_, profile=False, clocks=None):
        for _ in range(W_):
            step()
        torch.cuda.synchronize()
        barrier(dist, dev)
        if profile:
            iga.profile_read()
            iga.profile_enable(True)
        if clocks:
            clocks.start()
        l0 = iga.launch_count()
        evs = []
        t0 = time.perf_counter()
        for _ in range(K):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step()
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        barrier(dist, dev)
        launches = iga.launch_count() - l0
        clk = clocks.stop() if clocks else None
        prof = None
        if profile:
            iga.profile_enable(False)
            prof = iga.profile_read()
        ms = float(np.mean([a.elapsed_time(b) for a, b in evs]))
        return ms, launches, prof, clk, wall

    clocks = Clocks(local) if rank == 0 else None
    if args.mode == "exact":            # profiling helper: the exact step alone
        ms_e, launches_e, prof_e, _, _ = timed(step_exact, args.steps, args.warmup, profile=True)
        if rank == 0:
            print(json.dumps({"mode": "exact", "ms_per_step": ms_e, "kernels": prof_e}))
        return 0
    ms_s, launches, prof, clk, _ = timed(surr_step(A, primary), args.steps, args.warmup, profile=True, clocks=clocks)
    if args.mode == "surrogate":        # profiling helper: the surrogate step alone
        if rank == 0:
            print(json.dumps({"mode": "surrogate", "domains": primary, "ms_per_step": ms_s, "kernels": prof}))
        return 0
    ms_e, launches_e, prof_e, _, _ = timed(step_exact, max(3, args.steps // 2), args.warmup, profile=True)
    ms_s_max = max_over_ranks(dist, ms_s, dev)
    ms_e_max = max_over_ranks(dist, ms_e, dev)
    # the other choice of interpolation domains, for comparison
    B = iga.assemble_surrogate(prob, wl.M, wl.q, dtype=wl.dtype, domains=other)
    ms_o, _, prof_o, _, _ = timed(surr_step(B, other), max(3, args.steps // 2), args.warmup, profile=True)
    ms_o_max = max_over_ranks(dist, ms_o, dev)

    # end to end through the public API with host buffers (pinned), copies inside the timed region
    xh = torch.empty(prob.N, dtype=tdt, pin_memory=True)
    xh.copy_(x.cpu())
    yh = torch.empty(prob.N, dtype=tdt, pin_memory=True)
    xn, yn = xh.numpy(), yh.numpy()
    esz = 8 if wl.dtype == "f64" else 4

    def step_e2e():
        iga.assemble_surrogate(prob, wl.M, wl.q, dtype=wl.dtype, out=A, domains=primary)
        A.apply_host(xn, yn)

    for _ in range(args.warmup):
        step_e2e()
    torch.cuda.synchronize()
    barrier(dist, dev)
    K2 = max(3, args.steps // 2)
    t0 = time.perf_counter()
    for _ in range(K2):
        step_e2e()
    t_e2e = (time.perf_counter() - t0) / K2
    t_e2e = max_over_ranks(dist, t_e2e, dev)

    ref_solution = {}

    def exact_solution(f):
        """u_h of the exact FP64-quadrature matrix for the seeded load (one CG solve, reused)."""
        if "u" not in ref_solution:
            ref_solution["u"] = E.cg(f, tol=args.cg_tol, maxit=args.cg_maxit)
        return ref_solution["u"]

    def accuracy(mat, exact=None):
        """Stated entry error max |A~ - A| / max |A| over all stored entries (GPU copies), the
        row sums, and the discrete-solution error of CG on both matrices with one load vector."""
        exact = E if exact is None else exact
        vs, ve = mat.values(), exact.values()
        entry_err = float((vs.double() - ve.double()).abs().max().item() / ve.double().abs().max().item())
        del vs, ve
        ones = torch.ones(prob.N, dtype=mat.torch_dtype, device=dev)
        rowsum = float(mat.apply(ones).double().abs().max().item())
        solution = None
        if not args.no_solve:
            f = torch.from_numpy(W.rhs_vector(prob.N, seed=wl.seed)).to(dev)
            u_e, it_e, res_e = exact_solution(f)
            u_s, it_s, res_s = mat.cg(f, tol=args.cg_tol, maxit=args.cg_maxit)
            err = u_s - u_e
            Ee = E.apply(err.to(tdt)).double()
            Eu = E.apply(u_e.to(tdt)).double()
            solution = {"rel_l2": float(err.norm() / u_e.norm()),
                        "rel_energy": float(torch.sqrt(torch.dot(err, Ee) / torch.dot(u_e, Eu))),
                        "cg_iters": {"exact": it_e, "surrogate": it_s}, "cg_rel_residual": max(res_e, res_s),
                        "load": "f_i ~ U[-1,1] (seeded), homogeneous Dirichlet",
                        "reference": "u_h of the exact FP64 matrix"}
        return {"surrogate_vs_exact_max_rel": entry_err, "row_sum_max_abs": rowsum}, solution

    entry, solution = accuracy(A)
    entry_o, solution_o = accuracy(B)
    B.destroy()
    extra = {}
    if not args.no_extra and wl.name == W.CFG_3D_P4_F64.name:
        extra["fp32_tier"] = fp32_tier_report(iga, torch, wl, A, E, exact_solution, args)
    if not args.no_extra:
        extra["p3_64cube"] = side_report(iga, torch, W.CFG_3D_P3, steps=8, warmup=3)
    if not args.no_solve and not args.no_extra:
        extra["equal_accuracy"] = equal_accuracy_report(iga, torch, wl, E, ms_e_max, args)

    if rank != 0:
        return 0
    peaks, peak_kind = measured_peaks()
    arith = iga.get_arithmetic(wl.dtype)
    work = kernel_work(prob, wl, arith, surrogate=True, domains=primary)
    per_kernel = {k: {"launches": v[0], "ms": v[1]} for k, v in prof.items() if v[0]}
    dominant = max(per_kernel, key=lambda k: per_kernel[k]["ms"])
    dom = per_kernel[dominant]
    avg_ms = dom["ms"] / dom["launches"]
    sm_mhz = (clk or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
    if dominant in work and work[dominant]["bound"] == "alu":
        pipe = work[dominant]["pipe"]
        achieved = work[dominant]["flops"] / (avg_ms * 1e-3) / 1e12
        peak = alu_peak_tflops("fp64" if pipe == "fp64" else "fp32", float(peaks.get("sm_max_mhz", 2070.0)))
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "kernel": dominant, "pipe": pipe,
                "peak_source": ("derived: 152 SMs x 2 FP64 FMA/clk x max SM clock (nominal 1.25 TFLOP/s)"
                                if pipe == "fp64" else
                                "derived: 152 SMs x 128 FP32 FMA/clk x max SM clock; the double-float "
                                "instruction mix caps at 0.625 of it")}
    elif dominant in work:
        achieved = work[dominant]["bytes"] / (avg_ms * 1e-3) / 1e9
        peak = float(peaks["hbm_gbs"])
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "kernel": dominant, "peak_source": f"{peak_kind} hbm_gbs"}
    else:
        roof = {"bound": "alu", "achieved": None, "peak": None, "unit": "TFLOP/s", "frac": None, "kernel": dominant}
    roof["traffic"] = ncu_traffic(dominant, wl.name + ("" if primary == "common" else "_" + primary))
    roof["avg_launch_ms"] = avg_ms
    # SpMV against HBM, from the same timed region
    if "spmv" in per_kernel:
        sp = per_kernel["spmv"]
        gbs = work["spmv"]["bytes"] / (sp["ms"] / sp["launches"] * 1e-3) / 1e9
        spmv_roof = {"achieved": gbs, "peak": float(peaks["hbm_gbs"]), "unit": "GB/s",
                     "frac": gbs / float(peaks["hbm_gbs"]), "ms": sp["ms"] / sp["launches"]}
    else:
        spmv_roof = None

    value = aggregate_value(prob.nnz, world, ms_s_max * 1e-3)
    exact_value = aggregate_value(prob.nnz, world, ms_e_max * 1e-3)
    base = None
    if world == 1 and not args.no_cpu_baseline:
        base = cpu_baseline(wl, primary, target_s=args.cpu_seconds)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_s_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": wl.dtype,
        "arith": {"contractions": arith,
                  "coefficients": (arith if prob.map_kind == "sinprod" and prob.kappa_kind in ("const", "sin2d", "expsin3d")
                                   else "fp64"),
                  "fill": "df64" if wl.dtype == "f64" else "fp32", "diagonal": "fp64" if wl.dtype == "f64" else
                  "compensated fp32", "spmv": wl.dtype},
        "data": "synthetic (seeded map/coefficient family, x ~ N(0,1))",
        "config": config_of(wl, world, primary),
        "exact": {"value": exact_value, "unit": UNIT, "ms_per_step": ms_e_max,
                  "kernels": {k: {"launches": v[0], "ms": v[1]} for k, v in prof_e.items() if v[0]}},
        "speedup_surrogate_vs_exact": ms_e_max / ms_s_max,
        "entry_error": entry,
        "solution_error": solution,
        other + "_domains": {"value": aggregate_value(prob.nnz, world, ms_o_max * 1e-3), "unit": UNIT,
                             "ms_per_step": ms_o_max, "speedup_vs_exact": ms_e_max / ms_o_max,
                             "entry_error": entry_o, "solution_error": solution_o,
                             "kernels": {k: {"launches": v[0], "ms": v[1]} for k, v in prof_o.items() if v[0]}},
        "kernels": per_kernel,
        "roofline": roof,
        "spmv_roofline": spmv_roof,
        "cpu_baseline": base,
        "e2e": {"value": aggregate_value(prob.nnz, world, t_e2e), "unit": UNIT,
                "h2d_bytes_per_step": prob.N * esz, "d2h_bytes_per_step": prob.N * esz},
        **extra,
        "adjoint": adjoint_report(iga, torch, dev, steps=5, warmup=3) if not args.no_adjoint else None,
        "batch": batch_report(iga, torch, steps=5, warmup=3) if not args.no_batch else None,
        "mass": mass_report(iga, torch, wl, steps=5, warmup=3) if not args.no_mass else None,
        "gpu_launches": launches,
        "clocks": clk,
    }
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--workload", default=W.CFG_3D_P4_F64.name, choices=sorted(W.WORKLOADS))
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="CPU work budget of the oracle baseline")
    ap.add_argument("--ref-rows", type=int, default=0,
                    help="rows per step of the reference (oracle) arm (0: calibrated like the cpu_baseline leg)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-solve", action="store_true", help="skip the CG solution-error report")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the kappa-gradient timing")
    ap.add_argument("--no-batch", action="store_true", help="skip the 256-patch batch timing")
    ap.add_argument("--no-mass", action="store_true", help="skip the mass-matrix timing")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the FP32-tier and 64^3 p = 3 reports beside the headline")
    ap.add_argument("--cg-tol", type=float, default=1e-10)
    ap.add_argument("--cg-maxit", type=int, default=20000)
    ap.add_argument("--arith", default=None, choices=["df64", "df64_tc", "fp64", "fp32", "bf16x3"],
                    help="contraction arithmetic of the workload's value type (default: the library's)")
    ap.add_argument("--domains", choices=["common", "per_offset"], default="common",
                    help="interpolation domains of the headline surrogate (the other is reported beside it)")
    ap.add_argument("--mode", choices=["both", "surrogate", "exact"], default="both",
                    help="profiling helper: time only one of the two steps and print a short line")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    wl = W.WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, wl)
    return run_gpu(args, wl)


if __name__ == "__main__":
    sys.exit(main())
