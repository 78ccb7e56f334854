"""The multi-rank logic of bench.py on CPU (gloo, world size 2): each rank
runs its own scene replica (distinct seeds), the whole-job figures are the
slowest rank's time and the sum of all ranks' evals, and the reference arm
runs on rank 0 only."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    secs, evals = bench.reduce_over_ranks(1.0 + rank, 10 * (rank + 1), world, "cpu")
    seed = bench.workload_config("tiny", rank)["spectrum"]["seed"]
    # the reference arm: ranks other than 0 exit at once without work
    ref_rc = bench.run_reference(type("A", (), {"workload": "tiny"})()) if rank != 0 else 0
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, secs, evals, seed, ref_rc))


def test_two_ranks_reduce_and_seed_like_bench():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, s0, e0, seed0, _), (_, s1, e1, seed1, rc1) = res
    assert s0 == s1 == 2.0          # max over ranks
    assert e0 == e1 == 30.0         # sum over ranks
    assert seed0 != seed1           # one independent replica per rank
    assert rc1 == 0


def test_single_rank_passthrough():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(1.5, 7, 1, "cpu") == (1.5, 7.0)
