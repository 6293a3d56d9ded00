"""The multi-rank path on CPU: two gloo ranks shard a batch of independent
instances, solve their shares with the FP64 oracle, and reduce the timing
(MAX) and the work (SUM); the shards together reproduce the one-process
solve bit for bit."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2210_12375_b300.dist import max_over_ranks, shard, sum_over_ranks


def test_shard_partitions_the_batch():
    for n in (0, 1, 7, 256, 1001):
        for world in (1, 2, 3, 8):
            parts = [shard(n, r, world) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(parts[r][1] == parts[r + 1][0] for r in range(world - 1))
            sizes = [b - a for a, b in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard(10, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_2210_12375_b300 import workloads
    w = workloads.make(1, B=40)
    a, b = shard(w["B"], rank, world)
    r = oracle.solve(dict(w["field"], mu=w["field"]["mu"][a:b]),
                     w["y0"][a:b], w["t0"][a:b], w["t1"][a:b], w["t_eval"][a:b],
                     dict(rtol=w["rtol"], atol=w["atol"]), nthreads=1)
    steps = float((r["n_acc"] + r["n_rej"]).sum())
    ms = max_over_ranks(10.0 + rank)
    total = sum_over_ranks(steps)
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), y_eval=r["y_eval"], a=a, b=b, ms=ms,
             total=total, steps=steps)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce(tmp_path):
    world, port = 2, _free_port()
    mp.start_processes(_rank_main, args=(world, port, str(tmp_path)), nprocs=world,
                       start_method="spawn")
    parts = [np.load(tmp_path / f"rank{r}.npz") for r in range(world)]
    assert all(float(p["ms"]) == 11.0 for p in parts)  # MAX over ranks
    assert float(parts[0]["total"]) == sum(float(p["steps"]) for p in parts)
    import oracle
    from paper_2210_12375_b300 import workloads
    w = workloads.make(1, B=40)
    ref = oracle.solve(w["field"], w["y0"], w["t0"], w["t1"], w["t_eval"],
                       dict(rtol=w["rtol"], atol=w["atol"]), nthreads=1)
    got = np.concatenate([p["y_eval"] for p in parts])
    assert np.array_equal(got, ref["y_eval"])
