"""The N-GPU benchmark path on CPU ranks (gloo, world size 2): ranks are
replicas that only combine their elapsed time (max) and units done (sum), and
draw disjoint label rows."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import synth
    elapsed = 1.5 + rank            # rank 1 is the slow one
    units = 10.0 * (rank + 1)
    t, u = bench.combine_ranks(elapsed, units)
    obs = synth.observed_labels([5, 4, 3], 1)
    rows = synth.shuffled_rows(obs, 6, bench.rank_seed(77, rank))
    out[rank] = (t, u, rows.tobytes())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_timing_and_disjoint_rows():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    t0, u0, rows0 = out[0]
    t1, u1, rows1 = out[1]
    assert t0 == t1 == 2.5           # max over ranks
    assert u0 == u1 == 30.0          # sum over ranks
    assert rows0 != rows1            # ranks work on different label rows


def test_single_process_is_identity():
    import bench
    assert bench.combine_ranks(3.0, 7.0) == (3.0, 7.0)
