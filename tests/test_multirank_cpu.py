"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2): every rank gets
its own seeded node batch, the timing is the slowest rank's, and the whole-job value
counts every rank's evaluations.  The path has no data exchange between ranks."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import workloads as W
    w = W.batched()
    u = w.uniforms(seed=bench.rank_seed(w.seed, rank))
    elapsed = 1000.0 * (1 + rank)        # rank 1 is the slow one
    slowest = bench.max_over_ranks(elapsed, dist, "cpu")
    value = bench.weak_scaling_value(world, 3, slowest)
    gathered = [torch.zeros(u.shape, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(gathered, torch.tensor(u))
    out[rank] = (slowest, value, [g.numpy() for g in gathered])
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = dict(out)
    assert set(res) == {0, 1}
    for r in range(world):
        slowest, value, batches = res[r]
        assert slowest == 2000.0                     # max over ranks, on every rank
        assert value == pytest.approx(2 * 3 / 2.0)   # 6 evaluations in 2 s
        assert not np.allclose(batches[0], batches[1])   # independent node batches
    assert np.array_equal(res[0][2][0], res[1][2][0])


def test_single_process_helpers():
    import bench
    assert bench.max_over_ranks(5.0, None, "cpu") == 5.0
    assert bench.rank_seed(2, 0) == 2 and bench.rank_seed(2, 1) != 2
    assert bench.weak_scaling_value(1, 3, 3000.0) == pytest.approx(1.0)
