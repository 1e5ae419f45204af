"""Host-side logic of bench.py on the CPU: the replica aggregation over ranks (two
gloo processes) and the load-imbalance measure of Section 7.1."""
import os
import socket
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r took (r + 1) * 100 ms for 3 steps of 10^9 flops
    tot, val = bench.aggregate_ranks((rank + 1) * 100.0, 10 ** 9, 3, world)
    q.put((rank, tot, val))
    dist.destroy_process_group()


def test_replicas_take_the_slowest_rank():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, tot, val in res:
        assert tot == 200.0                                   # max over ranks
        assert abs(val - 2.0 * 1e9 * 3 * world / 0.2 / 1e9) < 1e-9   # all ranks' flops / slowest time


def test_single_rank_aggregation():
    import bench
    tot, val = bench.aggregate_ranks(50.0, 10 ** 9, 2, 1)
    assert tot == 50.0 and abs(val - 80.0) < 1e-9


def test_imbalance_measure():
    """max/mean per stage (SUMMA pairs A(I,s)B(s,J); Cannon pairs A(I,k)B(k,J),
    k = (I+J+s) mod g) and over all stages, on a hand-checked 2 x 2 grid."""
    import bench
    bf = np.zeros((2, 2, 2))        # [s, J, I]
    bf[0, 0, 0] = 4.0               # stage 0: one block product does all the work
    bf[1] = 1.0                     # stage 1: balanced
    r = bench.imbalance(bf)
    assert r["per_stage_max_summa"] == 4.0 and r["per_stage_mean_summa"] == 2.5
    # overall: processor (I=0, J=0) has 5, the others 1 -> mean 2, max 5
    assert r["overall"] == 2.5
    # Cannon stage 0 uses k = (I+J) mod 2: (0,0)->k=0: 4; (1,0)->k=1: 1; (0,1)->k=1: 1; (1,1)->k=0: 0
    assert abs(r["per_stage_max_cannon"] - 4.0 / 1.5) < 1e-12


def test_single_thread_oracle_sample():
    """The single-thread oracle figure: one thread, every 64th column, the flops of
    exactly those columns (checked against the oracle's own flops count)."""
    import bench
    import oracle
    from paper_1006_2183_gb300 import gen
    A = gen.rmat(10, 8, 0x1010, gen.PLUS_TIMES_F64)
    r = bench.cpu_single_thread(oracle, A)
    assert r["cores"] == 1 and r["unit"] == "GFLOPS" and r["value"] > 0
    cols = np.arange(0, A.n, bench.CPU_STRIDE_1T)
    fl = int(oracle.flops_per_col(A, A)[cols].sum())
    assert f"({len(cols)} columns, {fl} flops)" in r["sample"]
