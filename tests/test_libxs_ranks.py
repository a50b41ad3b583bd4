"""libxs driven from two gloo ranks on the CPU (127.0.0.1): each rank process
loads the library through the binding, asks for a device that cannot exist,
gets the status back (no crash, no context), sees null-context calls
rejected, and the ranks agree on what the library reports.  This is the
host side of the multi-rank bench (one process per GPU, independent
molecules); nothing here needs a GPU."""
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
    from paper_2505_24807_gb300 import xs
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    try:
        lib = xs.load()
        nparams = xs.xs_mlp_nparams()
        # no device has a negative index: the status comes back, no context is made
        try:
            xs.xs_create(device=-1 - rank)
            status = xs.XS_OK
        except xs.XSError as e:
            status = e.status
        null_rc = lib.xs_set_params(None, None, xs.XS_NELEM)
        null_msg = xs.xs_last_error(None)
        world_seen, rank_seen, _ = bench.dist_env()
        mine = (rank_seen, world_seen, bench.rank_molecule_seed(rank_seen), nparams, status, null_rc, null_msg)
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        out[rank] = gathered
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_load_and_drive_the_library_host_side():
    from paper_2505_24807_gb300 import build
    try:
        build.build()
        import ctypes
        ctypes.CDLL(build.OUT)
    except (OSError, RuntimeError) as e:  # no toolchain or CUDA runtime on this host
        pytest.skip(f"cannot build or load libxs.so here: {e}")
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    assert res[0] == res[1]                                  # every rank saw the same gathered view
    view = res[0]
    assert [v[0] for v in view] == [0, 1] and {v[1] for v in view} == {2}
    assert view[0][2] != view[1][2]                          # independent molecules per rank
    n_mlp = 11 * 256 + 256 + 2 * (256 * 256 + 256) + 256 * 2 + 2
    assert {v[3] for v in view} == {n_mlp}                   # 11-256-256-256-2 weights and biases
    from paper_2505_24807_gb300 import xs
    assert {v[4] for v in view} == {xs.XS_ECUDA}
    assert {v[5] for v in view} == {xs.XS_EINVAL}
    assert {v[6] for v in view} == {"null context"}
