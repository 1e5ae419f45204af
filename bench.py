#!/usr/bin/env python
"""SpGEMM benchmark on one or more GB300s (one process per GPU).

Workload (default): C = A*A with A an R-MAT matrix of scale 20 (1,048,576
vertices), edge factor 8, (a, b, c, d) = (0.57, 0.19, 0.19, 0.05), duplicates
merged, self-loops kept, values uniform(0, 1).  One step runs every product
of the workload once: the flat product in plus-times FP64 and in boolean
or-and, and the same two on a 32 x 32 virtual 2D Sparse SUMMA grid.  The
smaller R-MAT scale-18 workload (flat and 16 x 16 grid, plus-times FP64 and
min-plus FP32) is timed after it and reported under "secondary".
Metric: GFLOPS = 2 * flops / time, flops = sum_j sum_{k in B(:,j)} nnz(A(:,k)).

Multi-GPU: every rank computes its own copy of the workload (independent
problems, no collective on the data path); value = all ranks' flops / the
slowest rank's time ("weak" scaling).

--impl reference times the CPU oracle (plain Gustavson, OpenMP over columns)
on a bounded column sample of the same workload, on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1006_2183_gb300 import gen  # noqa: E402

METRIC = "SpGEMM GFLOPS (2*flops/s)"
UNIT = "GFLOPS"
SCALE, EF, SEED = 20, 8, 0x2005
GRID = 32
SEMIRINGS = "pt64,bool"
# the secondary workload: R-MAT scale 18, 16 x 16 grid, plus-times FP64 and min-plus FP32
SECONDARY = (18, 16, "pt64,mp32")
# R-MAT seeds of the A*A workloads by scale (scale 20 is the larger flat + 32 x 32 grid configuration)
SEED_OF_SCALE = {18: 0x1802, 20: 0x2005}
# semiring ids of the C ABI: name and value width in bytes
SR_NAME = {0: "pt64", 1: "mp32", 2: "bool", 3: "pti64"}
SR_WIDTH = {0: 8, 1: 4, 2: 1, 3: 8}
L2_FLUSH_BYTES = 512 << 20
# oracle sample: every CPU_STRIDE[scale]-th output column (a few seconds on the host cores)
CPU_STRIDE = {18: 4, 20: 8}


def _train_predictor(sp, ctx):
    """Predictor trained on exact symbolic counts of R-MAT and ER squares of scales 14-18,
    drawn from seeds disjoint from the measured workloads."""
    import torch
    Xs, ys = [], []
    for M in (gen.rmat(14, 8, 0x7000), gen.erdos_renyi(16384, 16384, 8, 0x7100), gen.rmat(16, 4, 0x7200),
              gen.rmat(15, 16, 0x7300), gen.rmat(17, 8, 0x7400), gen.rmat(18, 8, 0x7500),
              gen.erdos_renyi(65536, 65536, 16, 0x7600)):
        d = sp.Matrix.from_host(ctx, M, sp.PLUS_TIMES_F64)
        X, y = sp.spgemm_predictor_features(ctx, d, d)
        keep = y > 0
        Xs.append(X[keep])
        ys.append(torch.log1p(y[keep].double()).float())
    X, y = torch.cat(Xs), torch.cat(ys)
    sp.spgemm_predictor_set(ctx, np.random.default_rng(11).normal(0, 0.2, sp.NPARAM).astype(np.float32))
    for _ in range(400):
        loss, _ = sp.spgemm_predictor_train_step(ctx, X, y, 3e-3)
    return {"loss": loss, "samples": int(X.shape[0]),
            "matrices": "R-MAT scales 14-18 and ER 2^14, 2^16 squares, seeds 0x7000-0x7600"}


def _same_outputs(ctx, Xs, Ys, sr) -> bool:
    """Exact equality of two lists of device products: column pointers, rows, and values
    (bit-exact for int64, boolean and min-plus; within 1e-13 relative for plus-times FP64)."""
    import torch
    torch.cuda.current_stream().wait_stream(ctx.stream)
    for X, Y in zip(Xs, Ys):
        mx, nx, zx, cpx, irx, vx = X.export()
        my, ny, zy, cpy, iry, vy = Y.export()
        if (mx, nx, zx) != (my, ny, zy) or not torch.equal(cpx, cpy) or not torch.equal(irx, iry):
            return False
        if sr == 0:
            if not bool(((vx - vy).abs() <= 1e-13 * vy.abs()).all()):
                return False
        elif not torch.equal(vx, vy):
            return False
    return True


def _timed_arm(ctx, fn, steps, warmup, flush):
    """Median device time of fn() (CUDA events on the context stream, L2 flushed before
    each run) over `steps` runs after `warmup` untimed runs; returns (ms, last result)."""
    import torch
    st = ctx.stream
    for _ in range(warmup):
        r = fn()
        del r
    ts = []
    r = None
    for _ in range(steps):
        del r
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        r = fn()
        e1.record(st)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts), r


def learned_vs_plain(sp, ctx, steps: int, warmup: int, flush, c5=None) -> dict:
    """The a9 + a10 comparison.  Per batched workload five arms, each timed on the device
    (CUDA events, L2 flushed, median of `steps` after `warmup`) and checked against the
    plain arm's output, exactly:
      plain            one spgemm_multiply per product, in sequence;
      batched          spgemm_batch, exact symbolic pass, autotuned thresholds;
      learned_batched  spgemm_batch with the predictor sizing the output (no symbolic
                       pass for the hash tiers), autotuned thresholds;
      auto             spgemm_batch with what the autotuner chose, predictor included;
      graph_replay     spgemm_batch_plan once, then one spgemm_batch_execute per call: the
                       numeric pass replayed from a CUDA graph (same structure, new values).
    A speedup is reported only where the outputs are identical."""
    import oracle
    train = _train_predictor(sp, ctx)
    out = {"predictor": train, "timing": f"CUDA events, median of {steps} after {warmup} warm-up runs, "
                                          "L2 flushed before each",
           "arms": {"plain": "one spgemm_multiply per product, in sequence",
                    "batched": "one spgemm_batch call (one launch per tier over all products), no CUDA graph",
                    "learned_batched": "spgemm_batch with the nnz predictor sizing the output, no CUDA graph",
                    "auto": "spgemm_batch with the autotuner's thresholds and predictor choice, no CUDA graph",
                    "graph_replay": "spgemm_batch_plan once, then one spgemm_batch_execute per call: the numeric "
                                    "launches replayed from one CUDA graph (fixed structure)"}}
    work = {}
    pairs = gen.batch_pairs(512, 0x4004)
    As = [sp.Matrix.from_host(ctx, a, sp.PLUS_TIMES_I64) for a, _ in pairs]
    Bs = [sp.Matrix.from_host(ctx, b, sp.PLUS_TIMES_I64) for _, b in pairs]
    fl = sum(int(oracle.flops_per_col(a, b).sum()) for a, b in pairs)
    work["batch512_int64"] = (As, Bs, sp.PLUS_TIMES_I64, fl,
                              "512 uneven int64 pairs, n_i = 2^U(10,16), ER or R-MAT, edge factor in {4,8,16,32}")
    Ab = gen.rmat(20, 16, 0x4F00, gen.OR_AND_BOOL)
    F = gen.frontier(Ab.m, 128, 0x4F01, 1, 1000)
    work["bfs_step_bool"] = ([sp.Matrix.from_host(ctx, Ab, sp.OR_AND_BOOL)], [sp.Matrix.from_host(ctx, F, sp.OR_AND_BOOL)],
                             sp.OR_AND_BOOL, int(oracle.flops_per_col(Ab, F).sum()),
                             "boolean R-MAT scale 20 (edge factor 16) times a 2^20 x 128 frontier")
    for name, (As_, Bs_, sr, flops, desc) in work.items():
        tuned = sp.default_opts(use_predictor=1)
        tuned = sp.spgemm_autotune(ctx, As_, Bs_, sr, tuned)
        thr = dict(warp_max_flops=tuned.warp_max_flops, block_max_flops=tuned.block_max_flops,
                   dense_part_flops=tuned.dense_part_flops)
        o_b, o_l = sp.default_opts(use_predictor=0, **thr), sp.default_opts(use_predictor=1, **thr)
        t_p, Cp = _timed_arm(ctx, lambda: [sp.spgemm_multiply(ctx, a, b, sr) for a, b in zip(As_, Bs_)], steps,
                             warmup, flush)
        rec = {"workload": desc, "flops": flops, "tuned": {**thr, "use_predictor": tuned.use_predictor},
               "plain_ms": t_p}
        for arm, fn in (("batched", lambda: sp.spgemm_batch(ctx, As_, Bs_, sr, o_b)),
                        ("learned_batched", lambda: sp.spgemm_batch(ctx, As_, Bs_, sr, o_l)),
                        ("auto", lambda: sp.spgemm_batch(ctx, As_, Bs_, sr, tuned))):
            t, C = _timed_arm(ctx, fn, steps, warmup, flush)
            same = _same_outputs(ctx, C, Cp, sr)
            rec[arm] = {"ms": t, "identical": same, "speedup": t_p / t if same else None}
            del C
        plan = sp.spgemm_batch_plan(ctx, As_, Bs_, sr, o_b)
        t, _ = _timed_arm(ctx, lambda: plan.execute(), steps, warmup, flush)
        same = _same_outputs(ctx, plan.outputs(), Cp, sr)
        rec["graph_replay"] = {"ms": t, "identical": same, "speedup": t_p / t if same else None,
                               "note": "numeric pass only, replayed from a CUDA graph on a fixed structure"}
        del plan, Cp
        rec["predictor_gain"] = rec["batched"]["ms"] / rec["learned_batched"]["ms"]
        out[name] = rec
    # Galerkin triple product R*(A*P), FP64: two dependent products
    N = 128
    A, P = gen.grid3d_laplacian(N), gen.aggregation_2x2x2(N)
    R = gen.transpose_host(P)
    dA, dP, dR = (sp.Matrix.from_host(ctx, M, sp.PLUS_TIMES_F64) for M in (A, P, R))
    sr = sp.PLUS_TIMES_F64
    # the two products differ (fine-grid operator times aggregation, then restriction
    # times a coarse operator), so each is tuned on its own
    AP0 = sp.spgemm_multiply(ctx, dA, dP, sr)
    tuned1 = sp.spgemm_autotune(ctx, [dA], [dP], sr, sp.default_opts(use_predictor=1))
    tuned2 = sp.spgemm_autotune(ctx, [dR], [AP0], sr, sp.default_opts(use_predictor=1))
    del AP0

    def thr(t):
        return dict(warp_max_flops=t.warp_max_flops, block_max_flops=t.block_max_flops,
                    dense_part_flops=t.dense_part_flops)
    fl = A.nnz + 32 * 64 ** 3 - 24 * 64 ** 2   # flops(A*P) = nnz(A), flops(R*(AP)) = nnz(AP)
    t_p, Cp = _timed_arm(ctx, lambda: [sp.spgemm_multiply(ctx, dR, sp.spgemm_multiply(ctx, dA, dP, sr), sr)],
                         steps, warmup, flush)
    rec = {"workload": "R*(A*P), 7-point Laplacian on 128^3, 2x2x2 aggregation", "flops": fl,
           "tuned": [{**thr(t), "use_predictor": t.use_predictor} for t in (tuned1, tuned2)], "plain_ms": t_p}
    arms = (("batched", sp.default_opts(use_predictor=0, **thr(tuned1)), sp.default_opts(use_predictor=0, **thr(tuned2))),
            ("learned_batched", sp.default_opts(use_predictor=1, **thr(tuned1)),
             sp.default_opts(use_predictor=1, **thr(tuned2))),
            ("auto", tuned1, tuned2))
    for arm, o1, o2 in arms:
        t, C = _timed_arm(ctx, lambda o1=o1, o2=o2: [sp.spgemm_batch(ctx, [dR], sp.spgemm_batch(ctx, [dA], [dP], sr, o1),
                                                                     sr, o2)[0]],
                          steps, warmup, flush)
        same = _same_outputs(ctx, C, Cp, sr)
        rec[arm] = {"ms": t, "identical": same, "speedup": t_p / t if same else None}
        del C
    p1 = sp.spgemm_batch_plan(ctx, [dA], [dP], sr, sp.default_opts(**thr(tuned1)))
    p1.execute()
    p2 = sp.spgemm_batch_plan(ctx, [dR], p1.outputs(), sr, sp.default_opts(**thr(tuned2)))
    t, _ = _timed_arm(ctx, lambda: (p1.execute(), p2.execute()), steps, warmup, flush)
    same = _same_outputs(ctx, p2.outputs(), Cp, sr)
    rec["graph_replay"] = {"ms": t, "identical": same, "speedup": t_p / t if same else None,
                           "note": "numeric passes only, replayed from CUDA graphs on a fixed structure"}
    rec["predictor_gain"] = rec["batched"]["ms"] / rec["learned_batched"]["ms"]
    out["galerkin128_fp64"] = rec
    del p1, p2, Cp
    # the large skewed squaring (R-MAT scale 20 flat A*A): predictor on vs off
    if c5 is not None:
        for sr, M in c5:
            t_p, Cp = _timed_arm(ctx, lambda: [sp.spgemm_multiply(ctx, M, M, sr)], max(3, steps // 2), 3, flush)
            t_l, Cl = _timed_arm(ctx, lambda: [sp.spgemm_multiply(ctx, M, M, sr, sp.default_opts(use_predictor=1))],
                                 max(3, steps // 2), 3, flush)
            same = _same_outputs(ctx, Cl, Cp, sr)
            out[f"rmat20_flat_{SR_NAME[sr]}"] = {"plain_ms": t_p, "learned_ms": t_l, "identical": same,
                                                 "speedup": t_p / t_l if same else None}
            del Cp, Cl
    return out


def aggregate_ranks(local_ms: float, flops_step: int, steps: int, world: int, device=None):
    """Whole-job time and GFLOPS over `world` replicas: every rank ran `steps` steps of
    `flops_step` flops; the job took as long as its slowest rank (max over ranks).
    Returns (max time in ms, GFLOPS of all ranks' flops over that time)."""
    tot_ms = float(local_ms)
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([tot_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_ms = float(t.item())
        dist.barrier()
    return tot_ms, 2.0 * flops_step * steps * world / (tot_ms / 1e3) / 1e9


def imbalance(bf: np.ndarray) -> dict:
    """Load imbalance of Section 7.1 (max flops of any processor / mean) from the
    block-product flops bf[s, J, I] of a g x g grid: per stage with SUMMA's pairing
    A(I,s)B(s,J) and with Sparse Cannon's A(I,k)B(k,J), k = (I+J+s) mod g (the
    pairing of the paper's Fig. 25/26 simulation), and over all stages."""
    g = bf.shape[0]
    I, J = np.meshgrid(np.arange(g), np.arange(g), indexing="ij")

    def ratio(x):
        mu = x.mean()
        return float(x.max() / mu) if mu > 0 else 1.0
    summa = [ratio(bf[s]) for s in range(g)]
    cannon = [ratio(bf[(I + J + s) % g, J, I]) for s in range(g)]
    return {"overall": ratio(bf.sum(axis=0)), "per_stage_mean_summa": float(np.mean(summa)),
            "per_stage_max_summa": float(np.max(summa)), "per_stage_mean_cannon": float(np.mean(cannon)),
            "per_stage_max_cannon": float(np.max(cannon))}


def summa_imbalance(sp, ctx, M, g: int, seed: int = 0x5EED) -> dict:
    """Block-work imbalance of the virtual grid for A*A, as given and after a random
    symmetric permutation A' = PAP^T (Section 5.3.3), both computed on the device."""
    import torch
    out = {"grid": g, "plain": imbalance(sp.spgemm_summa_block_flops(ctx, M, M, g))}
    perm = torch.from_numpy(np.random.default_rng(seed).permutation(M.shape()[0]).astype(np.int32)).to(ctx.device)
    Mp = sp.spgemm_mat_permute(ctx, M, perm, perm)
    out["permuted"] = imbalance(sp.spgemm_summa_block_flops(ctx, Mp, Mp, g))
    out["paper_context"] = ("Sparse Cannon on R-MAT scale 20 (a=0.6, b=c=d=0.13), 256 processors, permuted: "
                            "per-stage mean 1.46, overall below 1.1 (Section 7.1, Figs. 25-26)")
    return out


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=int, default=SCALE)
    ap.add_argument("--grid", type=int, default=GRID, help="virtual SUMMA grid size g (g x g blocks)")
    ap.add_argument("--workload", default="rmat_square",
                    choices=["rmat_square", "restriction", "tallskinny", "summa_pipeline"],
                    help="rmat_square: the default A*A step; restriction: A S^T and S (A S^T) of orders 2, 4, 8 "
                         "(Section 6.2.3); tallskinny: R-MAT times n x n/2^13 ER with c2 = 1 .. 10^5 per column "
                         "(Section 6.2.2); summa_pipeline: R-MAT A*A on the g x g grid with merges every "
                         "1, 2, 4, 8 stages, one stream vs two streams (Sections 7.2-7.3)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the learned+batched vs plain comparison on the batched workloads")
    ap.add_argument("--semirings", default=SEMIRINGS,
                    help="comma list of pt64 (plus-times FP64), mp32 (min-plus FP32), bool (or-and)")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the secondary R-MAT scale-18 workload")
    ap.add_argument("--products", default="flat,summa",
                    help="comma list of product kinds in a step: flat, summa")
    ap.add_argument("--opt", action="append", default=[],
                    help="library option for every product, e.g. --opt range_table_slots=4096")
    return ap.parse_args()


CPU_STRIDE_1T = 64   # the single-thread oracle sample: every 64th output column


def cpu_single_thread(oracle, A) -> dict:
    """The oracle on one host thread, over every CPU_STRIDE_1T-th output column of A*A
    (plus-times FP64), for the single-thread figure beside the all-cores baseline."""
    cols = np.arange(0, A.n, CPU_STRIDE_1T)
    lens = np.diff(A.colptr)
    fl = int(sum(lens[A.rowidx[A.colptr[j]:A.colptr[j + 1]]].sum() for j in cols))
    t0 = time.perf_counter()
    oracle.spgemm_columns(A, A, oracle.PT_F64, cols, nthreads=1)
    dt = time.perf_counter() - t0
    return {"value": 2.0 * fl / dt / 1e9, "unit": UNIT, "cores": 1,
            "sample": f"every {CPU_STRIDE_1T}th output column ({len(cols)} columns, {fl} flops), {dt:.2f} s wall"}


def flops_of(A) -> int:
    lens = np.diff(A.colptr)
    return int(lens[A.rowidx].sum())


def kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in ("kernels.cu", "kernels.cuh", "common.cuh"):
        with open(os.path.join(ROOT, "paper_1006_2183_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(scale: int):
    """DRAM bytes per launch of the dominant kernel from the committed ncu summary,
    or None when the kernels changed since it was captured (or no capture exists)."""
    path = os.path.join(ROOT, "profiles", f"k_slab_num_pt64_rmat{scale}.md")
    if not os.path.exists(path):
        return None
    kv = {}
    for ln in open(path):
        if ":" in ln and ln.startswith("- "):
            k, v = ln[2:].split(":", 1)
            kv[k.strip()] = v.strip().strip("`")
    if kv.get("kernel source sha256/16") != kernel_source_hash():
        return None
    try:
        return float(kv["dram bytes per launch"])
    except (KeyError, ValueError):
        return None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (200 ms) while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        rows = []
        for ln in open(self.path):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        mx = max(r[1] for r in rows)
        loaded = [r[0] for r in rows]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[2]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(rows)}


# ---------------------------------------------------------------- reference arm (CPU oracle)
def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    seed = SEED_OF_SCALE.get(args.scale, SEED)
    A = gen.rmat(args.scale, EF, seed, gen.PLUS_TIMES_F64)
    n = A.n
    # bounded sample: every 4th output column of the flat plus-times FP64 product
    stride = CPU_STRIDE.get(args.scale, 4)
    cols = np.arange(0, n, stride)
    lens = np.diff(A.colptr)
    fl_cols = np.array([lens[A.rowidx[A.colptr[j]:A.colptr[j + 1]]].sum() for j in cols], np.int64)
    flops = int(fl_cols.sum())
    cores = oracle.max_threads()
    times = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.spgemm_columns(A, A, oracle.PT_F64, cols)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
    tot = sum(times)
    value = 2.0 * flops * len(times) / tot / 1e9
    sample = (f"every {stride}th output column ({len(cols)} columns, {flops} flops) of the flat plus-times "
              f"FP64 product")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"rmat{args.scale}_AxA", "scale": args.scale, "edge_factor": EF,
                       "abcd": [0.57, 0.19, 0.19, 0.05], "seed": seed, "grid": args.grid,
                       "products": [f"{k}_{s}" for k in args.products.split(",") if k
                                    for s in args.semirings.split(",") if s],
                       "flops_per_product": flops_of(A), "nnz_A": A.nnz,
                       "reference_sample": "the oracle computes the sampled columns of the flat plus-times FP64 "
                                           "product; blocking and the semiring change only the order of the same "
                                           "column work"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_sweep(args) -> None:
    """The second workloads of Section 6.2 and the stage pipeline of Sections 7.2-7.3 on one
    GPU: every case timed on the device
    (CUDA events on the context stream around the public product call, L2 flushed
    before each run), one JSON line with the aggregate and the per-case numbers."""
    import torch
    from paper_1006_2183_gb300 import build as _build
    _build.build()
    from paper_1006_2183_gb300 import spgemm as sp
    import oracle
    ctx = sp.Context()
    dev = ctx.device
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    sr = sp.PLUS_TIMES_F64
    cases = []   # (name, callable returning the product, flops)
    if args.workload == "restriction":
        A = gen.rmat(args.scale, EF, SEED, gen.PLUS_TIMES_F64)
        dA = sp.Matrix.from_host(ctx, A, sr)
        for order in (2, 4, 8):
            S = gen.restriction(A.n, order, 0x6202 + order)
            St = gen.transpose_host(S)
            dS, dSt = sp.Matrix.from_host(ctx, S, sr), sp.Matrix.from_host(ctx, St, sr)
            fl_ast = A.nnz   # one S^T entry per row of S^T: flops(A S^T) = nnz(A)
            cases.append((f"A*S^T order {order}", lambda dSt=dSt: sp.spgemm_multiply(ctx, dA, dSt, sr), fl_ast))
            ASt = sp.spgemm_multiply(ctx, dA, dSt, sr)
            fl_sast = ASt.shape()[2]   # flops(S (A S^T)) = nnz(A S^T): one S entry per column
            cases.append((f"S*(A*S^T) order {order}",
                          lambda dS=dS, ASt=ASt: sp.spgemm_multiply(ctx, dS, ASt, sr), fl_sast))
        workload = {"workload": f"rmat{args.scale}_restriction", "scale": args.scale, "edge_factor": EF,
                    "seed": SEED, "orders": [2, 4, 8]}
    elif args.workload == "summa_pipeline":
        A = gen.rmat(args.scale, EF, SEED, gen.PLUS_TIMES_F64)
        dA = sp.Matrix.from_host(ctx, A, sr)
        mctx = sp.Context(stream=torch.cuda.Stream())
        g = args.grid
        fl = flops_of(A)
        for every in (1, 2, 4, 8):
            if every >= g:
                continue
            o = sp.default_opts(summa_merge_every=every)
            cases.append((f"one stream, merge every {every}",
                          lambda o=o: sp.spgemm_summa_blocked(ctx, dA, dA, g, sr, o), fl))
            cases.append((f"two streams, merge every {every}",
                          lambda o=o: sp.spgemm_summa_pipelined(ctx, mctx, dA, dA, g, sr, o), fl))
        cases.append((f"one stream, one merge after stage {g}",
                      lambda: sp.spgemm_summa_blocked(ctx, dA, dA, g, sr), fl))
        workload = {"workload": f"rmat{args.scale}_AxA_summa{g}_pipeline", "scale": args.scale, "edge_factor": EF,
                    "seed": SEED, "grid": g}
    else:
        n_scale = args.scale
        A = gen.rmat(n_scale, EF, SEED, gen.PLUS_TIMES_F64)
        dA = sp.Matrix.from_host(ctx, A, sr)
        k = max(1, A.n >> 13)
        for c2 in (1, 10, 100, 1000, 10000, 100000):
            if c2 > A.n:
                continue
            F = gen.erdos_renyi(A.n, k, c2, 0x6302 + c2, gen.PLUS_TIMES_F64)
            dF = sp.Matrix.from_host(ctx, F, sr)
            fl = int(oracle.flops_per_col(A, F).sum())
            cases.append((f"c2 = {c2}", lambda dF=dF: sp.spgemm_multiply(ctx, dA, dF, sr), fl))
        workload = {"workload": f"rmat{args.scale}_times_tall_skinny_er", "scale": args.scale, "edge_factor": EF,
                    "seed": SEED, "k": k, "c2": [1, 10, 100, 1000, 10000, 100000]}
    st = ctx.stream
    out = []
    tot_ms = tot_fl = 0.0
    for name, fn, fl in cases:
        for _ in range(max(3, args.warmup)):
            fn()
        ts = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            C = fn()
            e1.record(st)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
            del C
        ms = statistics.median(ts)
        out.append({"case": name, "flops": fl, "ms": ms, "gflops": 2 * fl / ms / 1e6})
        tot_ms += ms
        tot_fl += fl
    line = {"metric": METRIC, "value": 2 * tot_fl / tot_ms / 1e6, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": tot_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(workload, l2="flushed before every timed run (512 MiB write)"), "cases": out}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm
SRS = {"pt64": 0, "mp32": 1, "bool": 2}


def run_workload(sp, ctx, scale, grid, semirings, kinds, steps, warmup, lib_opts, flush, world, local, sample=True):
    """R-MAT(scale) A*A: every (product kind, semiring) once per step.  W warm-up steps,
    then `steps` steps timed with CUDA events on the context stream, L2 flushed before
    each; every product's result is freed once its nnz is read (inside the step).
    Returns the measurement and the objects the other legs reuse."""
    import torch
    import torch.distributed as dist
    seed = SEED_OF_SCALE.get(scale, SEED)
    A64 = gen.rmat(scale, EF, seed, gen.PLUS_TIMES_F64)
    wanted = [x for x in semirings.split(",") if x]
    # the same pattern in every semiring: FP64 values, their FP32 rounding, boolean ones
    host = {sp.PLUS_TIMES_F64: A64, sp.MIN_PLUS_F32: A64.with_vals(A64.vals.astype(np.float32)),
            sp.OR_AND_BOOL: A64.with_vals(np.ones(A64.nnz, dtype=np.uint8))}
    mats = {SRS[nm]: sp.Matrix.from_host(ctx, host[SRS[nm]], SRS[nm]) for nm in wanted}
    products = [(k, SRS[nm]) for k in kinds for nm in wanted]

    def run_product(kind, sr, M):
        if kind == "flat":
            ctx.timing_group(0)
            plan = sp.spgemm_plan(ctx, M, M, sr, lib_opts)
            return sp.spgemm_numeric(plan), plan
        ctx.timing_group(1)
        return sp.spgemm_summa_blocked(ctx, M, M, grid, sr, lib_opts), None

    def step():
        nz = []
        for kind, sr in products:
            C, plan = run_product(kind, sr, mats[sr])
            nz.append(C.shape()[2])
            del C, plan
        return nz

    step()   # one untimed run of every product first (errors surface here, before any timing)
    for _ in range(max(3, warmup)):
        step()
    torch.cuda.synchronize()
    st = ctx.stream
    ctx.timing(True)
    l0 = sp.launch_count()
    times = []
    nz = None
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) if sample else _NoClock() as clk:
        for _ in range(steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            nz = step()
            e1.record(st)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    launches = sp.launch_count() - l0
    phases = ctx.phase_ms()
    ctx.timing(False)
    flops1 = flops_of(A64)
    nnz_seen = dict(zip(products, nz))
    tot_ms, value = aggregate_ranks(sum(times), flops1 * len(products), steps, world, ctx.device)
    hbm, _ = peaks()
    pipe = {}
    for (kind, sr) in products:
        w = SR_WIDTH[sr]
        byt = (A64.n + 1) * 8 + A64.nnz * (4 + w) + (A64.n + 1) * 8 + nnz_seen[(kind, sr)] * (4 + w)
        pipe[f"{kind}_{SR_NAME[sr]}"] = {"compulsory_bytes": byt, "nnz_C": nnz_seen[(kind, sr)]}
    byt_step = sum(v["compulsory_bytes"] for v in pipe.values())
    return {"A64": A64, "host": host, "mats": mats, "products": products, "run_product": run_product,
            "seed": seed, "flops1": flops1, "value": value, "tot_ms": tot_ms, "ms_per_step": tot_ms / steps,
            "phases": phases, "launches": launches, "clocks": clk.summary(), "nnz_seen": nnz_seen, "pipe": pipe,
            "pipeline_frac": byt_step / (tot_ms / steps / 1e3) / 1e9 / hbm,
            "phase_tab": {f"{['flat', 'summa', 'g2', 'g3'][g]}:{SR_NAME[s_]}:{p_}": round(v[0] / max(1, steps), 4)
                          for (g, s_, p_), v in phases.items() if v[1]}}


class _NoClock:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False

    def summary(self):
        return None


def slab_roofline(sp, ctx, W, lib_opts, scale):
    """Roofline of the slab-tier numeric kernel of the flat plus-times FP64 product:
    its compulsory bytes (C's entries of the tier written once, the tier's B columns
    and A read once, column pointers) over its mean CUDA-event time in the timed
    region (the numeric_dense phase brackets exactly its one launch)."""
    A64 = W["A64"]
    M = W["mats"][sp.PLUS_TIMES_F64]
    ms, cnt = W["phases"].get((0, sp.PLUS_TIMES_F64, "numeric_dense"), (0.0, 0))
    if not cnt:
        return None
    plan = sp.spgemm_plan(ctx, M, M, sp.PLUS_TIMES_F64, lib_opts)
    sp.spgemm_symbolic(plan)
    ts = plan.tier_stats()
    del plan
    nnz_d, bnnz_d, cols_d = ts["nnz"][3], ts["bnnz"][3], ts["cols"][3]
    alg = nnz_d * 12 + bnnz_d * 12 + cols_d * 16 + A64.nnz * 12 + 8 * (A64.n + 1)
    per_launch_ms = ms / cnt
    hbm, peak_kind = peaks()
    ach = alg / (per_launch_ms / 1e3) / 1e9
    return {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
            "traffic": profiled_traffic(scale), "kernel": "k_slab_num<PT64>", "peak_kind": peak_kind,
            "alg_bytes_per_launch": alg, "ms_per_launch": per_launch_ms, "launches_timed": cnt}


def e2e_leg(sp, ctx, W, steps, warmup, flush, world):
    """The step's products through the public API with host buffers: every step copies A
    from pinned host memory to the device and every C back into one reused pinned
    buffer, inside the timed region (wall clock).  A product's copy back runs on a side
    stream while the next product computes; a result is released once its copy has
    completed, and the step ends when the last copy has."""
    import torch as _t
    A64, host, products, run_product = W["A64"], W["host"], W["products"], W["run_product"]
    dev = ctx.device
    st = ctx.stream
    pinned = {}
    for sr in {sr for _, sr in products}:
        H = host[sr]
        pinned[sr] = (_t.from_numpy(H.colptr).pin_memory(), _t.from_numpy(H.rowidx).pin_memory(),
                      _t.from_numpy(np.ascontiguousarray(H.vals)).pin_memory())
    h2d = sum(sum(t.numel() * t.element_size() for t in pinned[sr]) for _, sr in products)
    nzmax = max(W["nnz_seen"].values())
    out_cp = _t.empty(A64.n + 1, dtype=_t.int64).pin_memory()
    out_ir = _t.empty(nzmax, dtype=_t.int32).pin_memory()
    out_v = _t.empty(nzmax * 8, dtype=_t.uint8).pin_memory()   # viewed per semiring
    d2h = sum((A64.n + 1) * 8 + nz * (4 + SR_WIDTH[sr]) for (kind, sr), nz in W["nnz_seen"].items())
    side = _t.cuda.Stream()
    # the copies back are the longer part: start them as early as possible (the flat
    # products first, the smaller boolean result leading) and end the step on a short
    # one (the boolean SUMMA result last)
    order = sorted(products, key=lambda p: (p[0] != "flat", (p[1] == sp.OR_AND_BOOL) != (p[0] == "flat")))
    et = []
    for it in range(warmup + steps):
        flush.fill_(1.0)
        _t.cuda.synchronize()
        t0 = time.perf_counter()
        inflight = []   # (copy finished, what the copy still reads)
        for (kind, sr) in order:
            cp, ir, v = (x.to(dev, non_blocking=True) for x in pinned[sr])
            M = sp.Matrix.csc(ctx, A64.m, A64.n, cp, ir, v, sr)
            C, plan = run_product(kind, sr, M)
            _, _, nz, ccp, cir, cv = C.export()
            done = _t.cuda.Event()
            done.record(st)
            side.wait_event(done)
            copied = _t.cuda.Event()
            with _t.cuda.stream(side):
                out_cp.copy_(ccp, non_blocking=True)
                out_ir[:nz].copy_(cir, non_blocking=True)
                out_v[:nz * SR_WIDTH[sr]].view(sp.TORCH_DTYPE[sr]).copy_(cv, non_blocking=True)
                copied.record(side)
            inflight.append((copied, (C, plan, M, cp, ir, v)))
            del C, plan, M, cp, ir, v
            # results whose copy has finished go back to the allocator
            inflight = [x for x in inflight if not x[0].query()]
        side.synchronize()
        inflight.clear()
        dt = time.perf_counter() - t0
        if it >= warmup:
            et.append(dt)
    value = 2.0 * W["flops1"] * len(products) * len(et) * world / sum(et) / 1e9
    return {"value": value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "steps": len(et), "warmup": warmup, "copy_back": "overlapped with the next product"}


def cpu_leg(A64, scale):
    import oracle
    stride = CPU_STRIDE.get(scale, 4)
    cols = np.arange(0, A64.n, stride)
    lens = np.diff(A64.colptr)
    fl = int(sum(lens[A64.rowidx[A64.colptr[j]:A64.colptr[j + 1]]].sum() for j in cols))
    t0 = time.perf_counter()
    oracle.spgemm_columns(A64, A64, oracle.PT_F64, cols)
    dt = time.perf_counter() - t0
    return {"value": 2.0 * fl / dt / 1e9, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
            "sample": f"every {stride}th output column ({len(cols)} columns, {fl} flops) of the flat "
                      f"plus-times FP64 product, {dt:.2f} s wall on {oracle.max_threads()} threads",
            "single_thread": cpu_single_thread(oracle, A64)}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload != "rmat_square":
        if rank == 0:
            run_sweep(args)
        return
    import torch
    import torch.distributed as dist
    from paper_1006_2183_gb300 import build as _build
    if rank == 0 or world == 1:
        _build.build()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
        dist.barrier()
        _build.build()
    torch.cuda.set_device(local)
    from paper_1006_2183_gb300 import spgemm as sp

    kinds = [k for k in args.products.split(",") if k]
    ctx = sp.Context()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=ctx.device)
    lib_opts = sp.default_opts(**{k: float(v) if k == "predictor_margin" else int(v)
                                  for k, v in (o.split("=", 1) for o in args.opt)})
    W = run_workload(sp, ctx, args.scale, args.grid, args.semirings, kinds, args.steps, args.warmup, lib_opts,
                     flush, world, local)
    roof = slab_roofline(sp, ctx, W, lib_opts, args.scale) if sp.PLUS_TIMES_F64 in W["mats"] and "flat" in kinds \
        else None
    e2e = None
    if not args.no_e2e:
        e2e = e2e_leg(sp, ctx, W, min(args.steps, 5), 3, flush, world)
    cpu = cpu_leg(W["A64"], args.scale) if rank == 0 and world == 1 and not args.no_cpu_baseline else None
    imb = None
    if rank == 0:
        Mimb = W["mats"].get(sp.PLUS_TIMES_F64) or sp.Matrix.from_host(ctx, W["A64"], sp.PLUS_TIMES_F64)
        imb = summa_imbalance(sp, ctx, Mimb, args.grid)
    c5_mats = [(sr, W["mats"][sr]) for sr in (sp.PLUS_TIMES_F64, sp.OR_AND_BOOL) if sr in W["mats"]] \
        if args.scale == 20 else None
    secondary = None
    if not args.no_secondary and (args.scale, args.grid) != SECONDARY[:2]:
        sc2, g2, srs2 = SECONDARY
        del W["run_product"]
        torch.cuda.empty_cache()
        W2 = run_workload(sp, ctx, sc2, g2, srs2, ["flat", "summa"], 10, 3, lib_opts, flush, world, local,
                          sample=False)
        secondary = {"workload": f"rmat{sc2}_AxA", "scale": sc2, "grid": g2, "seed": W2["seed"],
                     "products": [f"{k}_{SR_NAME[s_]}" for k, s_ in W2["products"]], "value": W2["value"],
                     "unit": UNIT, "ms_per_step": W2["ms_per_step"], "steps": 10, "warmup": 3,
                     "flops_per_product": W2["flops1"], "pipeline_hbm_frac": W2["pipeline_frac"],
                     "phase_ms_per_step": W2["phase_tab"]}
        del W2
    lvp = None
    if rank == 0 and world == 1 and not args.no_learned:
        torch.cuda.empty_cache()
        lvp = learned_vs_plain(sp, ctx, steps=10, warmup=3, flush=flush, c5=c5_mats)

    if rank == 0:
        A64, products = W["A64"], W["products"]
        line = {"metric": METRIC, "value": W["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": W["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": f"rmat{args.scale}_AxA", "scale": args.scale, "edge_factor": EF,
                           "abcd": [0.57, 0.19, 0.19, 0.05], "seed": W["seed"], "grid": args.grid,
                           "products": [f"{k}_{SR_NAME[s_]}" for k, s_ in products],
                           "flops_per_product": W["flops1"], "nnz_A": A64.nnz,
                           "l2": "flushed between steps (512 MiB write)",
                           "pipeline_hbm_frac": W["pipeline_frac"], "pipeline": W["pipe"],
                           "phase_ms_per_step": W["phase_tab"],
                           "lib_opts": {k: v for k, v in (o.split("=", 1) for o in args.opt)}},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": W["clocks"],
                "gpu_launches": W["launches"], "secondary": secondary, "learned_batched_vs_plain": lvp,
                "summa_imbalance": imb}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
