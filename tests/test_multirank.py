"""The multi-GPU form of the benchmark is independent replicas (one 390-bunch
fill per rank, no collective on the data path; the timing barrier and the
max-over-ranks reduction are the only collectives).  Its host logic, run as
two gloo ranks on the CPU: the slowest rank's time reaches every rank, the
whole-job value counts every rank's units against it, the ranks track
different fills, and the reference arm does its work on rank 0 only."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 10.0 + 5.0 * rank            # rank 1 is the slow one
    t_max = bench.max_over_ranks(local_ms, dist, device="cpu")
    run = bench.replica_run(rank)
    value = bench.weak_scaling_value(run.n_particles, 100, world, t_max)

    class Args:
        steps, warmup, gpus = 1, 1, world
    ref = bench.reference_arm(Args, rank, world) if rank != 0 else None
    out.put((rank, t_max, run.seed, run.n_particles, value, ref))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, s0, n0, v0, _), (r1, t1, s1, n1, v1, ref1) = res
    assert t0 == t1 == 15.0                        # the slowest rank's time everywhere
    assert s0 != s1 and n0 == n1                   # independent fills of the same size
    assert v0 == v1 == pytest.approx(n0 * 100 * 2 / 15e-3)
    assert ref1 == 0                               # the reference arm: rank 0 only
