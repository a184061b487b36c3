#!/usr/bin/env python3
"""Benchmark of the batched 3x3 symmetric eigendecomposition hot path on GB300.

One step = the FP32 precision form of the method on one batch, forward (eigenvalues, D, Euler
angles) and adjoint (packed gradient for random cotangents of eigenvalues and D), through the
C-ABI (kd_eig3_sym, kd_eig3_sym_adjoint). Workload per GPU: 2^24 packed 3x3 FP32 matrices
R diag(lam) R^T with Haar R in four groups (N(0,1) eigenvalues; a pair equal to 1e-6; a
near-triple with spread 1e-7; exactly diagonal), each scaled by 10^u, u ~ U[-15, 15], seed = rank.

Prints ONE JSON line (rank 0): the whole-job rate (matrices/s, fwd+bwd), the roofline of the
dominant kernel against the measured HBM copy bandwidth, a breakdown (the forward and adjoint
alone, the FP64 plain form on the same matrices, the other invariant modes, each group of the
workload alone, array-of-structures records), an end-to-end rate with host buffers, the clocks
seen while timing, the CPU oracle timed on the host cores, and under `configs` the other
workloads (plain FP64, the mixed 2x2 + 3x3 graph, the differentiation workload, the
structure-tensor field, the last sharded over the ranks).

  python bench.py [--gpus N --steps K --warmup W]      (N > 1: launched by torch.distributed.run)
  python bench.py --impl reference ...                 (the CPU oracle as the reference arm)
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "3x3 eigendecomps/s fwd & fwd+bwd, % of HBM roofline, FP32 form vs FP64 plain"
WORKLOAD = ("precision form: 2^24 symmetric 3x3 FP32 built as R diag(lam) R^T with Haar R in four "
            "equal groups (lam N(0,1); two equal to 1e-6; near-triple 1e-7; exactly diagonal), "
            "scaled by 10^u, u~U[-15,15]")
FWD_BYTES = 24 + 12 + 36 + 12      # A in; lam, D, angles out (per matrix)
BWD_BYTES = 24 + 12 + 36 + 24      # A, lam_bar, D_bar in; A_bar out
FALLBACK_HBM_GBS = 6800.0
# FP32 / MUFU operations per voxel that the fused structure-tensor loss needs by the method's
# steps (one decomposition and the loss gradient), itemised in the header of csrc/kd_stloss.cu
ST_ALGO_OPS = 410


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", choices=["kdiag", "reference"], default="kdiag")
    p.add_argument("--n", type=int, default=1 << 24, help="matrices per GPU")
    p.add_argument("--e2e-steps", type=int, default=10)
    p.add_argument("--cpu-seconds", type=float, default=10.0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--all-configs", action="store_true",
                   help="time the other workloads too (the default; kept for older command lines)")
    p.add_argument("--no-configs", action="store_true",
                   help="skip the other workloads (plain FP64, mixed 2x2+3x3 graph, differentiation, tensor field)")
    p.add_argument("--configs", default="plain_fp64,mixed,differentiation,tensor_field",
                   help="the comma-separated subset of the other workloads to run")
    p.add_argument("--small", action="store_true",
                   help="reduced sizes of the other workloads (1/8 to 1/16 of each) for profiler captures")
    p.add_argument("--no-groups", action="store_true",
                   help="skip the per-group and per-invariant-mode timings of the headline workload")
    return p.parse_args()


# ---------------------------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------------------------

def whole_job_rate(elapsed: float, units_per_rank: int, world: int, device="cpu"):
    """Weak scaling: every rank processed units_per_rank units in its own `elapsed` seconds; the
    job took the slowest rank's time. Returns (units/s over all ranks, max elapsed). With
    world > 1 the process group must be initialised (NCCL on GPUs, gloo in tests)."""
    if world > 1:
        import torch
        import torch.distributed as tdist
        t = torch.tensor([float(elapsed)], dtype=torch.float64, device=device)
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        elapsed = float(t.item())
    return world * units_per_rank / elapsed, elapsed


def shard_range(n_total: int, rank: int, world: int):
    """Contiguous [start, end) of a global batch owned by `rank` (sizes differ by at most one)."""
    base, extra = divmod(n_total, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# The sources each profiled kernel is compiled from: a committed ncu figure counts only while
# these files are unchanged since the capture.
KERNEL_SOURCES = {
    "k_eig3_fwd": ("kd_eig3_fwd.cu", "kd_soa.cuh", "kd_method.cuh", "kd_internal.h"),
    "k_eig3_adj": ("kd_eig3_adj.cu", "kd_soa.cuh", "kd_method.cuh", "kd_internal.h"),
    "k_eig2_fwd": ("kd_eig2.cu", "kd_soa.cuh", "kd_method.cuh", "kd_internal.h"),
    "k_st_fwd_bwd": ("kd_stloss.cu", "kd_method.cuh", "kd_internal.h"),
}


def kernel_sha(kernel: str) -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_1306_6291_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profile_figure(tag: str, kernel: str, key: str):
    """A per-unit figure from a committed ncu summary under profiles/ (a line
    '<TAG> kernel=<name> src_sha=<sha> <key>=<value>'), or None when absent or taken on other
    sources of that kernel."""
    sha = kernel_sha(kernel)
    for f in glob.glob(os.path.join(ROOT, "profiles", "*.md")) + glob.glob(os.path.join(ROOT, "profiles", "*.txt")):
        for line in open(f):
            if not line.startswith(tag + " "):
                continue
            kv = dict(t.split("=", 1) for t in line.split()[1:] if "=" in t)
            if kv.get("kernel") == kernel and kv.get("src_sha") == sha and key in kv:
                return float(kv[key])
    return None


def traffic_for(kernel: str, n: int):
    """DRAM bytes (read + write) per launch of n matrices from the committed capture, or None."""
    b = profile_figure("TRAFFIC", kernel, "bytes_per_matrix")
    return None if b is None else b * n


class ClockSampler:
    """nvidia-smi samples every 100 ms while running (started before warm-up, stopped after
    the timed region)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = []
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((int(f[0]), float(f[1]), float(f[2]), f[3], float(f[4]), f[5:9]))
            except ValueError:
                continue
        idx = {r[0] for r in rows}
        if len(idx) > 1:
            rows = [r for r in rows if r[0] == self.index]
        if not rows:
            return None
        load = [r for r in rows if r[4] >= 50] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in load for k in range(4) if r[5][k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[1] for r in load), "sm_max_mhz": max(r[2] for r in load),
                "reasons": reasons, "samples_under_load": len(load)}


# ---------------------------------------------------------------------------------------------
# reference arm: the CPU oracle as it stands
# ---------------------------------------------------------------------------------------------

def oracle_step(A_rows, lb, Db):
    import oracle
    oracle.eig3(A_rows)
    oracle.eig3_adjoint(A_rows, lb, Db)


def make_host_workload(n, seed):
    import numpy as np
    import torch

    import workloads as W
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    A, _ = W.sym3_precision(n, seed=seed, device=dev)
    rows = A.t().contiguous().double().cpu().numpy()
    rng = np.random.default_rng(seed)
    return rows, rng


def cpu_baseline(A_rows, seconds: float):
    """The oracle (FP64 method forward + analytic adjoint) on the host cores, on a bounded sample
    of the workload: passes over its first m matrices until about `seconds` of work."""
    import numpy as np

    import oracle
    rng = np.random.default_rng(0)
    m = A_rows.shape[0]
    lb, Db = rng.standard_normal((m, 3)), rng.standard_normal((m, 3, 3))
    oracle_step(A_rows[:1024], lb[:1024], Db[:1024])      # thread pool start-up, untimed
    done, t0 = 0, time.perf_counter()
    while True:
        oracle_step(A_rows, lb, Db)
        done += m
        dt = time.perf_counter() - t0
        if dt >= seconds:
            break
    return {"value": done / dt, "unit": "matrices/s", "cores": oracle.get_threads(), "kind": "oracle",
            "sample": f"{done // m} passes over the first {m} matrices of the workload ({done} matrices); "
                      f"FP64 method oracle forward (lam, D, angles) + analytic adjoint, {dt:.1f} s"}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import numpy as np

    import oracle
    oracle.build()
    # the other ranks exit at once, so rank 0 times the oracle on all the host cores it may use
    # (torchrun sets OMP_NUM_THREADS=1 for every rank)
    oracle.set_threads(len(os.sched_getaffinity(0)) or os.cpu_count() or 1)
    A_rows, rng = make_host_workload(args.n, 0)
    # per step a bounded sample, sized so that warm-up + steps take about a minute
    m = 4096
    lb, Db = rng.standard_normal((m, 3)), rng.standard_normal((m, 3, 3))
    t = time.perf_counter()
    oracle_step(A_rows[:m], lb, Db)
    per = (time.perf_counter() - t) / m
    budget = 60.0 / max(1, args.steps + args.warmup)
    m = int(max(256, min(args.n, budget / max(per, 1e-9))))
    lb, Db = rng.standard_normal((m, 3)), rng.standard_normal((m, 3, 3))
    for i in range(args.warmup):
        s = (i * m) % max(1, args.n - m)
        oracle_step(A_rows[s:s + m], lb, Db)
    t = time.perf_counter()
    for i in range(args.steps):
        s = ((i + args.warmup) * m) % max(1, args.n - m)
        oracle_step(A_rows[s:s + m], lb, Db)
    dt = time.perf_counter() - t
    value = m * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "matrices/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": args.n, "seed": 0, "step": "forward + adjoint",
                       "sample_per_step": m},
            "cpu_baseline": {"value": value, "unit": "matrices/s", "cores": oracle.get_threads(), "kind": "oracle",
                             "sample": f"{m} matrices of the workload per step (FP64 method oracle forward + "
                                       f"analytic adjoint)"},
            "e2e": {"value": value, "unit": "matrices/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------------------------
# the other workloads (--all-configs)
# ---------------------------------------------------------------------------------------------

def _time(fn, reps, stream):
    import torch
    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3 / reps


def run_all_configs(dev, peak, which=("plain_fp64", "mixed", "differentiation", "tensor_field"), small=False):
    """Throughput and HBM-roofline fraction of each workload (algorithmic bytes per unit over the
    measured copy bandwidth). Inputs are generated before timing; every call goes through the C-ABI.
    `small` shrinks every workload (for profiler captures, which must stay a few GB)."""
    import torch

    import workloads as W
    from paper_1306_6291_gb300 import kdiag as K
    stream = torch.cuda.current_stream(dev)
    h = stream.cuda_stream
    out = {}

    def chk(s, what):
        if s != K.KD_OK:
            raise K.KdError(s, what)

    # plain FP64 form, entries U[-1, 1]: 65,536 matrices, and 2^24 for a bandwidth-relevant size
    for n in ((65536,) if small else (65536, 1 << 24)) if "plain_fp64" in which else ():
        A = W.sym3_uniform(n, seed=0, device=dev)
        lam, D, ang = (torch.empty(k, n, device=dev, dtype=torch.float64) for k in (3, 9, 3))
        t = _time(lambda: chk(K.kd_eig3_sym(A.data_ptr(), K.KD_F64, n, n, lam.data_ptr(), D.data_ptr(),
                                            ang.data_ptr(), K.KD_F64, None, None, h), "f64"), 20 if n > 65536 else 200,
                  stream)
        out[f"plain_fp64_n{n}"] = {"matrices_per_s": n / t, "ms": 1e3 * t, "bytes_per_matrix": 168,
                                   "hbm_frac": 168 * n / t / 1e9 / peak, "bound": "FP64 pipe"}
        del A, lam, D, ang

    # mixed 2^25 2x2 + 2^25 3x3 FP32, one CUDA graph with one launch per size
    if "mixed" in which:
        out.update(_cfg_mixed(dev, peak, 1 << (22 if small else 25)))
    if "differentiation" in which:
        out.update(_cfg_differentiation(dev, peak, 1 << (23 if small else 26)))
    if "tensor_field" in which:
        out.update(_cfg_tensor_field(dev, peak, (256, 256, 128) if small else (512, 512, 256)))
    return out


def _chk(s, what):
    from paper_1306_6291_gb300 import kdiag as K
    if s != K.KD_OK:
        raise K.KdError(s, what)


def _cfg_mixed(dev, peak, n):
    import torch

    import workloads as W
    from paper_1306_6291_gb300 import kdiag as K
    stream = torch.cuda.current_stream(dev)
    h = stream.cuda_stream
    chk = _chk
    out = {}
    A2 = W.sym2_normal_ties(n, seed=0, device=dev)
    A3 = W.sym3_normal(n, seed=1, device=dev)
    l2, p2 = torch.empty(2, n, device=dev), torch.empty(n, device=dev)
    l3, a3 = torch.empty(3, n, device=dev), torch.empty(3, n, device=dev)
    s2 = torch.cuda.Stream(dev)
    s2.wait_stream(stream)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s2):
        with torch.cuda.graph(g, stream=s2):
            hh = torch.cuda.current_stream().cuda_stream
            chk(K.kd_eig2_sym(A2.data_ptr(), K.KD_F32, n, n, l2.data_ptr(), p2.data_ptr(), None, K.KD_F32, None, hh),
                "eig2")
            chk(K.kd_eig3_sym(A3.data_ptr(), K.KD_F32, n, n, l3.data_ptr(), None, a3.data_ptr(), K.KD_F32, None,
                              None, hh), "eig3")
    stream.wait_stream(s2)
    t = _time(g.replay, 20, stream)
    t2 = _time(lambda: chk(K.kd_eig2_sym(A2.data_ptr(), K.KD_F32, n, n, l2.data_ptr(), p2.data_ptr(), None,
                                         K.KD_F32, None, h), "eig2"), 20, stream)
    # roofline of the graph: the 2x2 launch's bytes at the copy bandwidth plus the 3x3 launch's
    # executed instruction slots (committed ncu capture) at the SMs' issue rate (4 schedulers per
    # SM, one instruction per cycle, 2070 MHz)
    slots = profile_figure("INST", "k_eig3_fwd", "thread_slots_per_matrix_lam_ang_normal")
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    roof_s = None if slots is None else 24 * n / (peak * 1e9) + slots * n / 32 / (sms * 4 * 2.07e9)
    out["mixed_2x2_3x3_graph" + ("" if n == 1 << 25 else f"_2e{n.bit_length() - 1}")] = {
        "pairs_per_s": n / t, "ms": 1e3 * t, "bytes_per_pair": 24 + 48, "hbm_frac": 72 * n / t / 1e9 / peak,
        "eig2_alone_ms": 1e3 * t2, "eig2_hbm_frac": 24 * n / t2 / 1e9 / peak,
        "eig3_issue_slots_per_matrix": slots, "roofline_ms": None if roof_s is None else 1e3 * roof_s,
        "roofline_frac": None if roof_s is None else roof_s / t,
        "bound": "2x2 half HBM, 3x3 half issue (48 B against "
                 + ("about 500" if slots is None else f"{slots:.0f}") + " instruction slots per matrix)"}
    return out


def _cfg_differentiation(dev, peak, n):
    """Eigen-gaps >= 1e-3, forward (lam, D) and adjoint (lam_bar, D_bar)."""
    import torch

    import workloads as W
    from paper_1306_6291_gb300 import kdiag as K
    stream = torch.cuda.current_stream(dev)
    h = stream.cuda_stream
    chk = _chk
    out = {}
    A = W.sym3_normal_gapped(n, seed=0, device=dev)
    gen = torch.Generator(device=dev).manual_seed(1)
    lb, Db = torch.randn(3, n, generator=gen, device=dev), torch.randn(9, n, generator=gen, device=dev)
    lam, D, Ab = torch.empty(3, n, device=dev), torch.empty(9, n, device=dev), torch.empty(6, n, device=dev)
    tf = _time(lambda: chk(K.kd_eig3_sym(A.data_ptr(), K.KD_F32, n, n, lam.data_ptr(), D.data_ptr(), None, K.KD_F32,
                                         None, None, h), "fwd"), 10, stream)
    tb = _time(lambda: chk(K.kd_eig3_sym_adjoint(A.data_ptr(), K.KD_F32, n, n, lb.data_ptr(), Db.data_ptr(), None,
                                                 Ab.data_ptr(), None, h), "adj"), 10, stream)
    out[f"differentiation_2e{n.bit_length() - 1}"] = {
        "fwd_matrices_per_s": n / tf, "fwd_ms": 1e3 * tf, "fwd_hbm_frac": 72 * n / tf / 1e9 / peak,
        "fwd_bwd_matrices_per_s": n / (tf + tb), "bwd_ms": 1e3 * tb, "bwd_hbm_frac": 96 * n / tb / 1e9 / peak,
        "fwd_bwd_hbm_frac": 168 * n / (tf + tb) / 1e9 / peak}
    return out


def _cfg_tensor_field(dev, peak, shape, rank=0, world=1):
    """BF16 structure tensors of a smoothed random field, loss forward + backward. With world > 1
    every rank builds the same field (seed 0) and takes its shard_range of the voxels; the fused
    call on the shard plus one all_reduce of the two sums is the timed step, and the rate is the
    field's voxels over the slowest rank's time (strong scaling of one field)."""
    import math

    import torch

    import workloads as W
    from paper_1306_6291_gb300 import kdiag as K
    stream = torch.cuda.current_stream(dev)
    h = stream.cuda_stream
    chk = _chk
    out = {}
    S = W.structure_tensor_field(shape, seed=0, device=dev)
    n = S.shape[1]
    a, b = shard_range(n, rank, world)
    m = b - a
    wv = (1 / math.sqrt(3),) * 3
    ws = K.st_loss_workspace(max(m, 1), dev)
    loss = torch.empty(2, device=dev, dtype=torch.float64)
    gS = torch.empty_like(S)
    off = 2 * a   # bytes (BF16 planes): the shard is a plane view with ld = n
    pS, pG = S.data_ptr() + off, gS.data_ptr() + off

    def fused(a_, b_):
        chk(K.kd_st_loss_fwd_bwd(pS, K.KD_BF16, b_ - a_, n, wv, 1.0, ws.data_ptr(), ws.numel() * 8,
                                 loss.data_ptr(), pG, None, h), "st fwd_bwd")
        return loss

    def step():
        return sharded_st_loss(n, rank, world, fused)

    tf = _time(lambda: chk(K.kd_st_loss_fwd(pS, K.KD_BF16, m, n, wv, ws.data_ptr(), ws.numel() * 8,
                                            loss.data_ptr(), None, h), "st fwd"), 10, stream)
    tb = _time(lambda: chk(K.kd_st_loss_bwd(pS, K.KD_BF16, m, n, wv, 1.0, pG, None, h), "st bwd"), 10, stream)
    if world > 1:
        import torch.distributed as tdist
        tdist.barrier()
    tfb = _time(step, 10, stream)
    if world > 1:
        t = torch.tensor([tfb], dtype=torch.float64, device=dev)
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        tfb = float(t.item())
    sums = step().tolist()
    # issue roofline: the fused kernel's executed instruction slots per voxel (committed ncu
    # capture) over the SMs' issue rate (4 warp schedulers per SM, one instruction per cycle each,
    # at the maximum SM clock, 2070 MHz); and the same for the algorithmic operation count of the
    # method's steps (ST_ALGO_OPS, derived in the loss kernel's source)
    slots = profile_figure("INST", "k_st_fwd_bwd", "thread_slots_per_voxel")
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    issue_rate = world * sms * 4 * 2.07e9 * 32   # thread instructions per second, all ranks
    issue_s = None if slots is None else slots * n / issue_rate
    algo_s = ST_ALGO_OPS * n / issue_rate
    out["tensor_field_" + "x".join(str(d) for d in shape)] = {
        "voxels_per_s_fwd_bwd": n / tfb, "fused_ms": 1e3 * tfb, "bytes_per_voxel": 24, "ranks": world,
        "hbm_frac": 24 * n / tfb / 1e9 / (peak * world), "separate_fwd_ms": 1e3 * tf, "separate_bwd_ms": 1e3 * tb,
        "separate_voxels_per_s": m / (tf + tb), "bound": "issue (one decomposition + adjoint per voxel)",
        "loss_sums": sums,
        "algorithmic_ops_per_voxel": ST_ALGO_OPS, "algorithmic_issue_ms": 1e3 * algo_s,
        "algorithmic_issue_frac": algo_s / tfb,
        "executed_slots_per_voxel": slots, "executed_issue_ms": None if issue_s is None else 1e3 * issue_s,
        "executed_issue_frac": None if issue_s is None else issue_s / tfb}
    return out


def time_groups_and_modes(K, P, n, stream, h, grp, tensors=None):
    """Forward and adjoint of each group of the precision workload alone (the groups are
    contiguous quarters of the batch: plane views with ld = n), of the whole batch with the other
    invariant modes, and of the whole batch as array-of-structures records (A, lam_bar, D_bar
    given as row copies of the planes). Fractions are of the algorithmic bytes at the measured
    copy bandwidth."""
    import torch
    peak, _ = hbm_peak()
    q = n // 4
    out = {}
    if q * 4 == n and q > 0:
        import workloads as W
        for k, name in enumerate(W.GROUPS):
            off = 4 * k * q   # bytes: FP32 planes

            def f(off=off):
                _chk(K.kd_eig3_sym(P["A"] + off, K.KD_F32, q, n, P["lam"] + off, P["D"] + off, P["ang"] + off,
                                   K.KD_F32, None, None, h), "group fwd")

            def b(off=off):
                _chk(K.kd_eig3_sym_adjoint(P["A"] + off, K.KD_F32, q, n, P["lb"] + off, P["Db"] + off, None,
                                           P["Ab"] + off, None, h), "group adj")
            tf, tb = _time(f, 20, stream), _time(b, 20, stream)
            out[f"group_{name}"] = {"fwd_ms": 1e3 * tf, "fwd_hbm_frac": FWD_BYTES * q / tf / 1e9 / peak,
                                    "bwd_ms": 1e3 * tb, "bwd_hbm_frac": BWD_BYTES * q / tb / 1e9 / peak}
    modes = {"fp32_inv64": K.make_opts(invariants=K.KD_INV_F64),
             "fp32_ff": K.make_opts(invariants=K.KD_INV_FLOAT_FLOAT)}
    for key, o in modes.items():
        tf = _time(lambda o=o: _chk(K.kd_eig3_sym(P["A"], K.KD_F32, n, n, P["lam"], P["D"], P["ang"], K.KD_F32,
                                                  None, o, h), key), 10, stream)
        tb = _time(lambda o=o: _chk(K.kd_eig3_sym_adjoint(P["A"], K.KD_F32, n, n, P["lb"], P["Db"], None, P["Ab"], o,
                                                          h), key), 10, stream)
        out[f"fwd_{key}_ms"] = 1e3 * tf
        out[f"fwd_{key}_hbm_frac"] = FWD_BYTES * n / tf / 1e9 / peak
        out[f"bwd_{key}_ms"] = 1e3 * tb
        out[f"bwd_{key}_hbm_frac"] = BWD_BYTES * n / tb / 1e9 / peak
    if tensors is not None:
        A, lb, Db = tensors
        RA, Rlb, RDb = (x.t().contiguous() for x in (A, lb, Db))
        Rl, RD, Ra, RAb = (torch.empty(n, k, device=A.device) for k in (3, 9, 3, 6))
        o = K.make_opts(layout=K.KD_LAYOUT_AOS)
        tf = _time(lambda: _chk(K.kd_eig3_sym(RA.data_ptr(), K.KD_F32, n, n, Rl.data_ptr(), RD.data_ptr(),
                                              Ra.data_ptr(), K.KD_F32, None, o, h), "aos fwd"), 10, stream)
        tb = _time(lambda: _chk(K.kd_eig3_sym_adjoint(RA.data_ptr(), K.KD_F32, n, n, Rlb.data_ptr(), RDb.data_ptr(),
                                                      None, RAb.data_ptr(), o, h), "aos adj"), 10, stream)
        out["fwd_fp32_aos_ms"] = 1e3 * tf
        out["fwd_fp32_aos_hbm_frac"] = FWD_BYTES * n / tf / 1e9 / peak
        out["bwd_fp32_aos_ms"] = 1e3 * tb
        out["bwd_fp32_aos_hbm_frac"] = BWD_BYTES * n / tb / 1e9 / peak
        del RA, Rlb, RDb, Rl, RD, Ra, RAb
        torch.cuda.empty_cache()
    return out


def sharded_st_loss(n_total, rank, world, loss_shard):
    """The structure-tensor loss of a field split over `world` ranks: rank r takes the contiguous
    range shard_range(n_total, r, world) and `loss_shard(start, end)` returns its two sums as a
    float64 tensor (2,); with world > 1 one all_reduce adds the ranks' sums (the only exchange
    step of the path). Returns the sums of the whole field (on every rank)."""
    a, b = shard_range(n_total, rank, world)
    part = loss_shard(a, b)
    if world > 1:
        import torch.distributed as tdist
        tdist.all_reduce(part, op=tdist.ReduceOp.SUM)
    return part


# ---------------------------------------------------------------------------------------------
# kdiag arm
# ---------------------------------------------------------------------------------------------

def run_kdiag(args, rank, world, local):
    import numpy as np
    import torch

    import workloads as W
    from paper_1306_6291_gb300 import kdiag as K

    dist = world > 1
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if dist:
        import torch.distributed as tdist
        tdist.init_process_group("nccl", device_id=dev)
    K.load()
    n = args.n
    A, _grp = W.sym3_precision(n, seed=rank, device=dev)
    g = torch.Generator(device=dev).manual_seed(1000 + rank)
    lb = torch.randn(3, n, generator=g, device=dev)
    Db = torch.randn(9, n, generator=g, device=dev)
    lam = torch.empty(3, n, device=dev)
    D = torch.empty(9, n, device=dev)
    ang = torch.empty(3, n, device=dev)
    Ab = torch.empty(6, n, device=dev)
    stream = torch.cuda.current_stream(dev)
    h = stream.cuda_stream
    P = {k: v.data_ptr() for k, v in dict(A=A, lb=lb, Db=Db, lam=lam, D=D, ang=ang, Ab=Ab).items()}

    def fwd():
        s = K.kd_eig3_sym(P["A"], K.KD_F32, n, n, P["lam"], P["D"], P["ang"], K.KD_F32, None, None, h)
        if s != K.KD_OK:
            raise K.KdError(s, "kd_eig3_sym")

    def bwd():
        s = K.kd_eig3_sym_adjoint(P["A"], K.KD_F32, n, n, P["lb"], P["Db"], None, P["Ab"], None, h)
        if s != K.KD_OK:
            raise K.KdError(s, "kd_eig3_sym_adjoint")

    sampler = ClockSampler(local)
    sampler.start()
    for _ in range(args.warmup):
        fwd()
        bwd()
    torch.cuda.synchronize()
    if dist:
        tdist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for e0, e1, e2 in ev:
        e0.record(stream)
        fwd()
        e1.record(stream)
        bwd()
        e2.record(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    if dist:
        tdist.barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    elapsed = t_start.elapsed_time(t_end) / 1e3
    fwd_s = sum(e0.elapsed_time(e1) for e0, e1, _ in ev) / 1e3 / args.steps
    bwd_s = sum(e1.elapsed_time(e2) for _, e1, e2 in ev) / 1e3 / args.steps
    value, elapsed = whole_job_rate(elapsed, n * args.steps, world, dev)

    # FP64 plain form on the same matrices (forward), and the forward alone
    A64 = A.double()
    l64, D64, a64 = (torch.empty(k, n, device=dev, dtype=torch.float64) for k in (3, 9, 3))
    reps = 5

    def fwd64():
        s = K.kd_eig3_sym(A64.data_ptr(), K.KD_F64, n, n, l64.data_ptr(), D64.data_ptr(), a64.data_ptr(), K.KD_F64,
                          None, None, h)
        if s != K.KD_OK:
            raise K.KdError(s, "kd_eig3_sym f64")

    fwd64()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fwd64()
    e1.record(stream)
    torch.cuda.synchronize()
    f64_s = e0.elapsed_time(e1) / 1e3 / reps
    del A64, l64, D64, a64
    torch.cuda.empty_cache()

    # per group of the workload (each group alone, through plane views with ld = n) and the other
    # invariant modes of the forward on the whole batch
    groups = None if args.no_groups else time_groups_and_modes(K, P, n, stream, h, _grp, (A, lb, Db))

    # end to end with host buffers through the public host API (kdiag.eig3_host): pinned inputs,
    # chunks rotating over three streams so that host-to-device copies, both calls and
    # device-to-host copies of every output overlap; the timed region starts with the data on
    # the host and ends with every output back on the host
    # (outputs and the device workspace are allocated once, as a caller repeating the call would)
    hA, hlb, hDb = (x.cpu().pin_memory() for x in (A, lb, Db))
    chunk, nst = 1 << 20, 3
    ws = K.eig3_host_workspace(torch.float32, min(chunk, n), nst, dev)
    hout = K.eig3_host(hA, hlb, hDb, chunk=chunk, streams=nst, workspace=ws)   # warm-up
    torch.cuda.synchronize()
    if dist:
        tdist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        K.eig3_host(hA, hlb, hDb, chunk=chunk, streams=nst, workspace=ws, out=hout)
    e2e_s = (time.perf_counter() - t0) / args.e2e_steps
    e2e_value, _ = whole_job_rate(e2e_s * args.e2e_steps, n * args.e2e_steps, world, dev)
    h2d = (6 + 3 + 9) * 4 * n
    d2h = (3 + 9 + 3 + 6) * 4 * n

    peak, peak_kind = hbm_peak()
    kern = {"k_eig3_fwd": (fwd_s, FWD_BYTES), "k_eig3_adj": (bwd_s, BWD_BYTES)}
    dom = max(kern, key=lambda k: kern[k][0])
    dsec, dbytes = kern[dom]
    achieved = dbytes * n / dsec / 1e9
    result = None
    if rank == 0:
        result = {
            "metric": METRIC, "value": value, "unit": "matrices/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_per_gpu": n, "seed": "rank", "step": "forward + adjoint",
                       "form": "FP32 precision form (FP32 invariants, Jacobi refinement)",
                       "l2": "inputs larger than L2 (403 MB of A per GPU vs 129 MB L2)",
                       "parallelism": f"independent batch per GPU x{world}"},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_source": f"{peak_kind} HBM copy bandwidth",
                         "bytes_per_matrix": dbytes, "traffic": traffic_for(dom, n)},
            "breakdown": {
                "fwd_fp32_ms": 1e3 * fwd_s, "fwd_fp32_matrices_per_s": n / fwd_s,
                "fwd_fp32_hbm_frac": FWD_BYTES * n / fwd_s / 1e9 / peak,
                "bwd_fp32_ms": 1e3 * bwd_s, "bwd_fp32_matrices_per_s": n / bwd_s,
                "bwd_fp32_hbm_frac": BWD_BYTES * n / bwd_s / 1e9 / peak,
                "fwd_fp64_plain_ms": 1e3 * f64_s, "fwd_fp64_plain_matrices_per_s": n / f64_s,
                "fp32_fwd_speedup_over_fp64_plain": f64_s / fwd_s,
            },
            "e2e": {"value": e2e_value, "unit": "matrices/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h,
                    "path": "kdiag.eig3_host -> kd_eig3_sym_host: pinned host (6, n) planes, chunks of 2^20 "
                            "on 3 rotating streams: strided H2D / kd_eig3_sym + kd_eig3_sym_adjoint / strided D2H "
                            "of lam, D, angles, A_bar"},
            "gpu_launches": 2 * args.steps,
            "clocks": clocks,
        }
        if groups is not None:
            result["breakdown"].update(groups)
        if world == 1 and not args.no_cpu_baseline:
            rows = A[:, : min(n, 1 << 22)].t().contiguous().double().cpu().numpy()
            result["cpu_baseline"] = cpu_baseline(rows, args.cpu_seconds)
    if not args.no_configs:
        del A, lb, Db, lam, D, ang, Ab, hA, hlb, hDb, ws, hout
        torch.cuda.empty_cache()
        which = tuple(args.configs.split(","))
        cs = ClockSampler(local)
        cs.start()
        # the tensor field runs on every rank (the field sharded over the ranks, one all_reduce
        # of the two loss sums); the other workloads on rank 0 (per-GPU figures)
        cfg = {}
        if "tensor_field" in which:
            cfg.update(_cfg_tensor_field(dev, peak, (256, 256, 128) if args.small else (512, 512, 256),
                                         rank, world))
        if rank == 0:
            cfg.update(run_all_configs(dev, peak, tuple(c for c in which if c != "tensor_field"), args.small))
        torch.cuda.synchronize()
        cclk = cs.stop()
        if rank == 0:
            cfg["clocks"] = cclk
            result["configs"] = cfg
    if dist:
        tdist.barrier()
        tdist.destroy_process_group()
    if result is not None:
        print(json.dumps(result), flush=True)
    return 0


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_kdiag(args, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
