"""The N > 1 path of bench.py on CPU: two gloo ranks (one process each) run
the replica helpers the GPU runs use with NCCL — barrier, the max over ranks
of the step time and the sum over ranks of the work — and the reference arm,
which only rank 0 runs."""
import json
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port, out_dir):
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": "2",
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    ws, r, local, dist = bench.dist_init(None)
    try:
        bench.barrier(dist)
        t = bench.max_over_ranks(dist, 1.5 + rank)      # per-rank step times 1.5 s and 2.5 s
        work = bench.sum_over_ranks(dist, 2.0)          # 2 solves per rank and step
        ref = bench.run_reference(None, ws, r, dist) if r == 1 else None  # rank 1 returns without work
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"ws": ws, "rank": r, "max_t": t, "work": work, "ref": ref}, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_bench(tmp_path):
    mp.spawn(_rank_main, args=(_free_port(), str(tmp_path)), nprocs=2, join=True)
    res = [json.load(open(tmp_path / f"rank{k}.json")) for k in range(2)]
    for k, r in enumerate(res):
        assert r["ws"] == 2 and r["rank"] == k
        assert r["max_t"] == 2.5          # max over ranks
        assert r["work"] == 4.0           # whole-job work = sum over ranks
    assert res[1]["ref"] == 0             # reference arm: rank 1 exits 0 without work
    # whole-job throughput as the bench reports it: summed work / max time
    assert res[0]["work"] / res[0]["max_t"] == pytest.approx(1.6)
