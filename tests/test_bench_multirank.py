"""The bench's multi-rank host logic on CPU: two gloo ranks (127.0.0.1), each
with its own molecule seed, the timed region reduced to the slowest rank, the
whole-job throughput from every rank's roots."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    try:
        w, r, _ = bench.dist_env()
        slowest = bench.max_over_ranks(10.0 * (rank + 1), "cpu")   # rank r "took" 10 (r + 1) ms
        out[rank] = (w, r, bench.rank_molecule_seed(r), slowest)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_the_slowest():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    assert {v[0] for v in res.values()} == {2}
    assert [res[r][1] for r in (0, 1)] == [0, 1]
    assert res[0][2] != res[1][2]                       # independent molecules
    assert res[0][3] == res[1][3] == 20.0               # every rank sees the slowest time


def test_throughput_and_single_process_fallback():
    import bench
    # 2 ranks x 10 roots x 3 steps over the slowest rank's 1.5 s
    assert bench.throughput(2, 10, 3, 1.5) == pytest.approx(40.0)
    # without a process group the reduction is the identity
    assert bench.max_over_ranks(12.5, "cpu") == 12.5
