#!/usr/bin/env python
"""SpGEMM benchmark on one or more GB300s (one process per GPU).

Workload (default): C = A*A with A an R-MAT matrix of scale 18 (262,144
vertices), edge factor 8, (a, b, c, d) = (0.57, 0.19, 0.19, 0.05), duplicates
merged, self-loops kept, values uniform(0, 1).  One step runs every product
of the workload once: the flat product in plus-times FP64 and in min-plus
FP32, and the same two on a 16 x 16 virtual 2D Sparse SUMMA grid.
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
SCALE, EF, SEED = 18, 8, 0x1802
GRID = 16
# R-MAT seeds of the A*A workloads by scale (scale 20 is the larger flat + 32 x 32 grid configuration)
SEED_OF_SCALE = {18: 0x1802, 20: 0x2005}
# semiring ids of the C ABI: name and value width in bytes
SR_NAME = {0: "pt64", 1: "mp32", 2: "bool", 3: "pti64"}
SR_WIDTH = {0: 8, 1: 4, 2: 1, 3: 8}
L2_FLUSH_BYTES = 512 << 20
CPU_STRIDE = 4   # oracle sample: every 4th output column (~25 core-seconds on the flat scale-18 product)


def _train_predictor(sp, ctx):
    """Predictor trained on exact symbolic counts of R-MAT and ER squares (scales 14-16)
    drawn from seeds disjoint from the measured workloads."""
    import torch
    Xs, ys = [], []
    for M in (gen.rmat(14, 8, 0x7000), gen.erdos_renyi(16384, 16384, 8, 0x7100), gen.rmat(16, 4, 0x7200),
              gen.rmat(15, 16, 0x7300)):
        d = sp.Matrix.from_host(ctx, M, sp.PLUS_TIMES_F64)
        X, y = sp.spgemm_predictor_features(ctx, d, d)
        keep = y > 0
        Xs.append(X[keep])
        ys.append(torch.log1p(y[keep].double()).float())
    X, y = torch.cat(Xs), torch.cat(ys)
    sp.spgemm_predictor_set(ctx, np.random.default_rng(11).normal(0, 0.2, sp.NPARAM).astype(np.float32))
    for _ in range(400):
        loss, _ = sp.spgemm_predictor_train_step(ctx, X, y, 3e-3)
    return loss


def learned_vs_plain(sp, ctx, steps: int, warmup: int) -> dict:
    """The batched workloads, plain (one plan -> symbolic -> numeric per product, in
    sequence) against learned+batched (all products of the workload in one batched
    execution, the predictor sizing the output instead of the symbolic pass, bins from
    the autotuner).  Wall time on the device, synchronised on both sides; outputs
    compared by nnz."""
    import torch
    import oracle
    loss = _train_predictor(sp, ctx)
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
    N = 128
    A, P = gen.grid3d_laplacian(N), gen.aggregation_2x2x2(N)
    R = gen.transpose_host(P)
    dA, dP, dR = (sp.Matrix.from_host(ctx, M, sp.PLUS_TIMES_F64) for M in (A, P, R))
    out = {"predictor_train_loss": loss}

    def timed(fn):
        for _ in range(max(1, warmup)):
            fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            r = fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / steps * 1e3, r

    def nnz_of(Cs):
        return sum(C.shape()[2] for C in Cs)

    for name, (As_, Bs_, sr, flops, desc) in work.items():
        tuned = sp.spgemm_autotune(ctx, As_, Bs_, sr)
        lo = sp.default_opts(use_predictor=1, warp_max_flops=tuned.warp_max_flops,
                             block_max_flops=tuned.block_max_flops, dense_part_flops=tuned.dense_part_flops)
        t_plain, Cp = timed(lambda: [sp.spgemm_multiply(ctx, a, b, sr) for a, b in zip(As_, Bs_)])
        nz_plain = nnz_of(Cp)
        del Cp
        t_lb, Cl = timed(lambda: sp.spgemm_batch(ctx, As_, Bs_, sr, lo))
        nz_lb = nnz_of(Cl)
        del Cl
        out[name] = {"workload": desc, "flops": flops, "plain_ms": t_plain, "learned_batched_ms": t_lb,
                     "speedup": t_plain / t_lb, "plain_gflops": 2 * flops / t_plain / 1e6,
                     "learned_batched_gflops": 2 * flops / t_lb / 1e6, "same_nnz": nz_plain == nz_lb,
                     "tuned": [tuned.warp_max_flops, tuned.block_max_flops, tuned.dense_part_flops]}
        torch.cuda.empty_cache()
    # Galerkin triple product R*(A*P), FP64: plain products vs the learned+autotuned batch form
    tuned = sp.spgemm_autotune(ctx, [dA], [dP], sp.PLUS_TIMES_F64)
    lo = sp.default_opts(use_predictor=1, warp_max_flops=tuned.warp_max_flops,
                         block_max_flops=tuned.block_max_flops, dense_part_flops=tuned.dense_part_flops)

    def rap_plain():
        AP = sp.spgemm_multiply(ctx, dA, dP, sp.PLUS_TIMES_F64)
        return sp.spgemm_multiply(ctx, dR, AP, sp.PLUS_TIMES_F64)

    def rap_learned():
        AP = sp.spgemm_batch(ctx, [dA], [dP], sp.PLUS_TIMES_F64, lo)[0]
        return sp.spgemm_batch(ctx, [dR], [AP], sp.PLUS_TIMES_F64, lo)[0]

    fl = A.nnz + 32 * 64 ** 3 - 24 * 64 ** 2   # flops(A*P) = nnz(A), flops(R*(AP)) = nnz(AP)
    t_plain, C1 = timed(rap_plain)
    t_lb, C2 = timed(rap_learned)
    out["galerkin128_fp64"] = {"workload": "R*(A*P), 7-point Laplacian on 128^3, 2x2x2 aggregation",
                               "flops": fl, "plain_ms": t_plain, "learned_batched_ms": t_lb,
                               "speedup": t_plain / t_lb, "same_nnz": C1.shape()[2] == C2.shape()[2]}
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
    ap.add_argument("--semirings", default="pt64,mp32",
                    help="comma list of pt64 (plus-times FP64), mp32 (min-plus FP32), bool (or-and)")
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
    path = os.path.join(ROOT, "profiles", f"k_range_num_pt64_rmat{scale}.md")
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
    cols = np.arange(0, n, CPU_STRIDE)
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
    sample = (f"every {CPU_STRIDE}th output column ({len(cols)} columns, {flops} flops) of the flat plus-times "
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
    seed = SEED_OF_SCALE.get(args.scale, SEED)
    A64 = gen.rmat(args.scale, EF, seed, gen.PLUS_TIMES_F64)
    flops1 = flops_of(A64)
    ctx = sp.Context()
    dev = ctx.device
    srs = {"pt64": sp.PLUS_TIMES_F64, "mp32": sp.MIN_PLUS_F32, "bool": sp.OR_AND_BOOL}
    wanted = [x for x in args.semirings.split(",") if x]
    # the same pattern in every semiring: FP64 values, their FP32 rounding, boolean ones
    host = {sp.PLUS_TIMES_F64: A64, sp.MIN_PLUS_F32: A64.with_vals(A64.vals.astype(np.float32)),
            sp.OR_AND_BOOL: A64.with_vals(np.ones(A64.nnz, dtype=np.uint8))}
    mats = {srs[nm]: sp.Matrix.from_host(ctx, host[srs[nm]], srs[nm]) for nm in wanted}
    if sp.PLUS_TIMES_F64 not in mats:
        mats[sp.PLUS_TIMES_F64] = sp.Matrix.from_host(ctx, A64, sp.PLUS_TIMES_F64)   # imbalance report
    products = []
    for k in kinds:
        for name in wanted:
            products.append((k, srs[name]))

    lib_opts = sp.default_opts(**{k: float(v) if k == "predictor_margin" else int(v)
                                  for k, v in (o.split("=", 1) for o in args.opt)})

    def run_product(kind, sr, M):
        if kind == "flat":
            ctx.timing_group(0)
            plan = sp.spgemm_plan(ctx, M, M, sr, lib_opts)
            C = sp.spgemm_numeric(plan)
            return C, plan
        ctx.timing_group(1)
        C = sp.spgemm_summa_blocked(ctx, M, M, args.grid, sr, lib_opts)
        return C, None

    # one untimed run of every product first (errors surface here, before any timing)
    for kind, sr in products:
        C, plan = run_product(kind, sr, mats[sr])
        del C, plan
    flops_step = flops1 * len(products)

    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step():
        outs = []
        for kind, sr in products:
            outs.append(run_product(kind, sr, mats[sr]))
        return outs

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    # timed region: per-step CUDA events on the context stream, L2 flushed between steps
    st = ctx.stream
    ctx.timing(True)
    l0 = sp.launch_count()
    times = []
    nnz_seen = {}
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            outs = step()
            e1.record(st)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            for (kind, sr), (C, plan) in zip(products, outs):
                nnz_seen[(kind, sr)] = C.shape()[2]
            del outs
    torch.cuda.synchronize()
    launches = sp.launch_count() - l0
    phases = ctx.phase_ms()
    ctx.timing(False)
    clocks = clk.summary()
    tot_ms, value = aggregate_ranks(sum(times), flops_step, args.steps, world, dev)

    # dominant kernel: numeric dense tier of the flat plus-times FP64 product
    hbm, peak_kind = peaks()
    roof = None
    if ("flat", sp.PLUS_TIMES_F64) in products:
        plan = sp.spgemm_plan(ctx, mats[sp.PLUS_TIMES_F64], mats[sp.PLUS_TIMES_F64], sp.PLUS_TIMES_F64, lib_opts)
        sp.spgemm_symbolic(plan)
        ts = plan.tier_stats()
        ms, cnt = phases[(0, sp.PLUS_TIMES_F64, "numeric_dense")]
        if cnt:
            nnz_d, bnnz_d, cols_d = ts["nnz"][3], ts["bnnz"][3], ts["cols"][3]
            alg = nnz_d * 12 + bnnz_d * 12 + cols_d * 16 + A64.nnz * 12 + 8 * (A64.n + 1)
            per_launch_ms = ms / cnt
            ach = alg / (per_launch_ms / 1e3) / 1e9
            roof = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                    "traffic": profiled_traffic(args.scale), "kernel": "k_range_num<PT64,4096>",
                    "peak_kind": peak_kind, "alg_bytes_per_launch": alg, "ms_per_launch": per_launch_ms,
                    "launches_timed": cnt}
        del plan
    # whole-product roofline on compulsory bytes (A read once, C written once)
    pipe = {}
    for (kind, sr) in products:
        w = SR_WIDTH[sr]
        byt = (A64.n + 1) * 8 + A64.nnz * (4 + w) + (A64.n + 1) * 8 + nnz_seen[(kind, sr)] * (4 + w)
        pipe[f"{kind}_{SR_NAME[sr]}"] = {"compulsory_bytes": byt, "nnz_C": nnz_seen[(kind, sr)]}
    phase_tab = {f"{['flat', 'summa', 'g2', 'g3'][g]}:{SR_NAME[s]}:{p}":
                 round(v[0] / max(1, args.steps), 4) for (g, s, p), v in phases.items() if v[1]}
    byt_step = sum(v["compulsory_bytes"] for v in pipe.values())
    pipeline_frac = byt_step / (tot_ms / args.steps / 1e3) / 1e9 / hbm

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        import torch as _t
        pinned = {}
        for sr in {sr for _, sr in products}:
            H = host[sr]
            pinned[sr] = (_t.from_numpy(H.colptr).pin_memory(), _t.from_numpy(H.rowidx).pin_memory(),
                          _t.from_numpy(np.ascontiguousarray(H.vals)).pin_memory())
        h2d = sum(sum(t.numel() * t.element_size() for t in pinned[sr]) for _, sr in products)
        outbuf = {}
        d2h = 0
        for (kind, sr) in products:
            nz = nnz_seen[(kind, sr)]
            w = SR_WIDTH[sr]
            outbuf[(kind, sr)] = (_t.empty(A64.n + 1, dtype=_t.int64).pin_memory(),
                                  _t.empty(nz, dtype=_t.int32).pin_memory(),
                                  _t.empty(nz, dtype=sp.TORCH_DTYPE[sr]).pin_memory())
            d2h += (A64.n + 1) * 8 + nz * (4 + w)
        et = []
        for it in range(args.warmup + args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for (kind, sr) in products:
                cp, ir, v = (x.to(dev, non_blocking=True) for x in pinned[sr])
                M = sp.Matrix.csc(ctx, A64.m, A64.n, cp, ir, v, sr)
                C, plan = run_product(kind, sr, M)
                _, _, nz, ccp, cir, cv = C.export()
                ob = outbuf[(kind, sr)]
                ob[0].copy_(ccp, non_blocking=True)
                ob[1][:nz].copy_(cir, non_blocking=True)
                ob[2][:nz].copy_(cv, non_blocking=True)
                st.synchronize()
                del C, plan, M
            dt = time.perf_counter() - t0
            if it >= args.warmup:
                et.append(dt)
        e2e_val = 2.0 * flops_step * len(et) * world / sum(et) / 1e9
        e2e = {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        cols = np.arange(0, A64.n, CPU_STRIDE)
        lens = np.diff(A64.colptr)
        fl = int(sum(lens[A64.rowidx[A64.colptr[j]:A64.colptr[j + 1]]].sum() for j in cols))
        t0 = time.perf_counter()
        oracle.spgemm_columns(A64, A64, oracle.PT_F64, cols)
        dt = time.perf_counter() - t0
        cpu = {"value": 2.0 * fl / dt / 1e9, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
               "sample": f"every {CPU_STRIDE}th output column ({len(cols)} columns, {fl} flops) of the flat "
                         f"plus-times FP64 product, {dt:.2f} s wall on {oracle.max_threads()} threads",
               "single_thread": cpu_single_thread(oracle, A64)}

    imb = summa_imbalance(sp, ctx, mats[sp.PLUS_TIMES_F64], args.grid) if rank == 0 else None
    lvp = None
    if rank == 0 and world == 1 and not args.no_learned:
        lvp = learned_vs_plain(sp, ctx, steps=2, warmup=1)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": f"rmat{args.scale}_AxA", "scale": args.scale, "edge_factor": EF,
                           "abcd": [0.57, 0.19, 0.19, 0.05], "seed": seed, "grid": args.grid,
                           "products": [f"{k}_{SR_NAME[s]}" for k, s in products],
                           "flops_per_product": flops1, "nnz_A": A64.nnz, "l2": "flushed between steps (512 MiB write)",
                           "pipeline_hbm_frac": pipeline_frac, "pipeline": pipe, "phase_ms_per_step": phase_tab,
                           "lib_opts": {k: v for k, v in (o.split("=", 1) for o in args.opt)}},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "gpu_launches": launches,
                "learned_batched_vs_plain": lvp, "summa_imbalance": imb}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
