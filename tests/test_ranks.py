"""The multi-rank host logic of bench.py (one independent replica per rank, no data-path
collective): two gloo ranks on the CPU check that the job's time is the slowest rank's, that the
throughput counts every rank's particles, that each rank draws its own seeded inputs, and that the
reference arm does no work beyond rank 0."""
import os
import socket

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    res = {}
    # each rank timed alone; the job lasts as long as the slowest one
    res["max"] = bench.max_over_ranks(1.5 + rank)
    res["rate"] = bench.job_rate(4096, ws, bench.max_over_ranks(2e-3 * (1 + rank)))
    # weak scaling: the same workload shape, a seed of its own per rank
    w = bench.WORKLOADS["uniform_4k_l4_p16"]
    xy, q = bench.make_inputs(w, rank)
    mine = torch.tensor([float(xy.sum()), float(q.sum())], dtype=torch.float64)
    both = [torch.zeros(2, dtype=torch.float64) for _ in range(ws)]
    dist.all_gather(both, mine)
    res["shape"] = list(xy.shape) + list(q.shape)
    res["sums"] = [b.tolist() for b in both]
    # the reference arm: ranks other than 0 exit at once (rank 0 would run the oracle)
    if rank != 0:
        class A:
            steps, warmup, workload = 1, 1, "uniform_4k_l4_p16"
        res["ref"] = bench.run_reference(A())
    dist.barrier()
    dist.destroy_process_group()
    np.save(os.path.join(out_dir, f"rank{rank}.npy"), np.array([res], dtype=object), allow_pickle=True)


def test_two_gloo_ranks(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, str(tmp_path))) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=240)
    for p in procs:
        if p.is_alive():
            p.kill()
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    res = [np.load(tmp_path / f"rank{r}.npy", allow_pickle=True)[0] for r in range(ws)]
    for r in res:
        assert r["max"] == 2.5                       # the slower rank's time on every rank
        assert r["rate"] == pytest.approx(2 * 4096 / 4e-3)
        assert r["shape"] == [4096, 2, 4096]
    s0, s1 = res[0]["sums"]
    assert res[0]["sums"] == res[1]["sums"]          # both ranks saw the same gathered values
    assert s0 != s1                                  # and the two replicas differ
    assert res[1]["ref"] is None
