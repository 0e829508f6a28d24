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


# --------------------------------------------------------------------------
# Bunch-sharded long-range scan (one fill's bunches split over ranks): each
# rank reduces its contiguous range to an affine phasor map, the ranks
# allgather the maps, each composes them with the carried phasor.  Checked on
# gloo ranks against the oracle's direct sum over every earlier passage.
SHARD_TURNS = 25


def _shard_fill():
    import mbt_workloads as W
    ring = W.ring_r0()
    buckets = [0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 200, 201, 202, 350]    # trains with gaps, and the wrap
    currents = [0.5e-3 * (1 + (m % 4)) for m in range(len(buckets))]
    res = [dict(W.HOM), dict(Rs_ohm=3e5, fr_Hz=2.7e9, Q=800.0, range=W.RANGE_LONG)]
    return ring, buckets, currents, res


def _shard_worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch.distributed as dist
    import oracle
    from paper_1809_00391_gb300 import sharded
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ring, buckets, currents, res = _shard_fill()
    nb = len(buckets)
    lo, hi = sharded.split_bounds(nb, world)[rank:rank + 2]
    s = oracle.OracleSim(ring, res, 128, 5.0, buckets, currents, [200] * nb, 11, 0)
    s.init_particles()
    steps = [sharded.phasor_steps(ring, r, buckets) for r in res]
    carry = [0j, 0j]
    worst = 0.0
    for t in range(SHARD_TURNS):
        s.track(1, record=False)
        alr = s.alr()
        for r in range(len(res)):
            E = s.last_emission(r)
            phi, carry[r] = sharded.exchange_turn(steps[r][lo:hi], E[lo:hi], carry[r], dist)
            ref = alr[r, lo:hi]
            # both sides round the phase w t of a delay t to about eps w t (FP64):
            # the scan through its step factors, the direct sum in e^{s t}
            wr = 2 * np.pi * res[r]["fr_Hz"]
            bound = np.finfo(np.float64).eps * wr * (t + 1) * ring["T0_s"]
            err = float(np.max(np.abs(phi - ref)) / np.max(np.abs(alr[r])))
            worst = max(worst, err / bound)
    # every rank ends with the same carry
    import torch
    c = torch.tensor([carry[0].real, carry[0].imag, carry[1].real, carry[1].imag], dtype=torch.float64)
    parts = [torch.empty(4, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(parts, c)
    same = all(bool(torch.equal(p, parts[0])) for p in parts)
    out.put((rank, worst, same))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_phasor_scan_matches_the_direct_history_sum(world):
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, worst, same in res:
        assert worst <= 1.0, (rank, worst)   # within the FP64 phase resolution of the longest delay
        assert same


def test_sharded_phasor_scan_is_one_process_scan_on_one_rank():
    """Splitting changes only the grouping of the same compositions: one range
    (no exchange) and many small ranges give the same phasors to 1e-13."""
    import numpy as np
    sys.path.insert(0, ROOT)
    from paper_1809_00391_gb300 import sharded
    ring, buckets, currents, res = _shard_fill()
    rng = np.random.default_rng(2)
    nb = len(buckets)
    step = sharded.phasor_steps(ring, res[0], buckets)
    E = rng.normal(size=nb) + 1j * rng.normal(size=nb)
    carry = 0.3 - 0.2j
    whole, c1 = sharded.exchange_turn(step, E, carry)
    b = sharded.split_bounds(nb, 5)
    maps = np.stack([sharded.segment_map(step[b[r]:b[r + 1]], E[b[r]:b[r + 1]]) for r in range(5)])
    entry, c2 = sharded.compose(maps, carry)
    parts = np.concatenate([sharded.apply(step[b[r]:b[r + 1]], E[b[r]:b[r + 1]], entry[r]) for r in range(5)])
    assert np.max(np.abs(parts - whole)) <= 1e-13 * np.max(np.abs(whole))
    assert abs(c1 - c2) <= 1e-13 * abs(c1)
    # the definition written out: Phi_m = a_m X_{m-1}, X_m = Phi_m + E_m, X_{-1} = carry
    X, ref = carry, []
    for m in range(nb):
        ref.append(step[m] * X)
        X = ref[-1] + E[m]
    assert np.max(np.abs(np.array(ref) - whole)) <= 1e-14 * np.max(np.abs(whole))
    assert abs(X - c1) <= 1e-14 * abs(X)


def test_phasor_steps_and_empty_ranges():
    """a_m is the resonator's decay and rotation e^{s dt} over the bucket
    distance from the bunch before (the first bunch: from the last bunch of the
    previous turn across the gap), s = -w_r/(2Q) + i w_r sqrt(1 - 1/(4Q^2));
    a rank holding no bunches contributes the identity map and meets its entry
    value unchanged."""
    import math

    import numpy as np
    sys.path.insert(0, ROOT)
    from paper_1809_00391_gb300 import sharded
    ring, buckets, currents, res = _shard_fill()
    r = res[0]
    step = sharded.phasor_steps(ring, r, buckets)
    wr = 2 * math.pi * r["fr_Hz"]
    s = complex(-wr / (2 * r["Q"]), wr * math.sqrt(1 - 1 / (4 * r["Q"] ** 2)))
    T_rf = ring["T0_s"] / ring["h"]
    gaps = np.diff(np.concatenate([[buckets[-1] - ring["h"]], buckets]))
    assert np.all(gaps > 0) and gaps.sum() == ring["h"]
    for m in range(len(buckets)):
        ref = complex(np.exp(s * gaps[m] * T_rf))
        assert abs(step[m] - ref) <= 1e-12 * abs(ref), m
    empty = np.zeros(0, np.complex128)
    A, B = sharded.segment_map(empty, empty)
    assert A == 1 and B == 0
    entry, carry = sharded.compose(np.array([[A, B], [0.5 + 0.5j, 2.0 - 1j]]), 1.0 + 1.0j)
    assert entry[0] == 1.0 + 1.0j and entry[1] == 1.0 + 1.0j
    assert carry == (0.5 + 0.5j) * (1.0 + 1.0j) + (2.0 - 1j)
    assert len(sharded.apply(empty, empty, 3.0 + 0j)) == 0


def test_phasor_calls_refuse_bad_arguments():
    """Buckets out of the ring, not increasing, or a resonator with Q <= 1/2
    (no oscillating wake) are refused with MBT_ERR_ARG, as is a composition of
    no maps; nothing is written on refusal."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import paper_1809_00391_gb300 as p
    from paper_1809_00391_gb300 import sharded
    MBT_ERR_ARG = 1   # include/mbt.h
    ring, buckets, currents, res = _shard_fill()
    r = res[0]
    h = ring["h"]
    for bad in ([3, 2], [0, 0], [-1, 4], [0, h]):
        with pytest.raises(p.MBTError) as ei:
            sharded.phasor_steps(ring, r, bad)
        assert ei.value.status == MBT_ERR_ARG, bad
    with pytest.raises(p.MBTError) as ei:
        sharded.phasor_steps(ring, dict(r, Q=0.5), buckets)
    assert ei.value.status == MBT_ERR_ARG
    with pytest.raises(p.MBTError) as ei:
        sharded.compose(np.zeros((0, 2), np.complex128), 0j)
    assert ei.value.status == MBT_ERR_ARG
