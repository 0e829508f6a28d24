"""Failure detection on the GPU without a fault (GPU test, through the C ABI).

Every device wait of the kernels is bounded by a wall-clock limit after which
the kernel records an error and returns.  Here the cluster-resident kernel's
grid barrier (each cluster waits for the other bunches' emissions of the
turn) is made to wait for a count that nothing reaches, with a 20 ms limit:
every cluster's wait runs out, the launch ends by itself, the next
synchronising call reports MBT_ERR_TIMEOUT, and the context stays usable
(the error word is cleared once reported) and can be destroyed; a fresh
context then tracks the same fill normally.  Before this path runs, every
CTA of a cluster leaves the turn loop together and the clusters' final
barrier keeps each CTA's shared memory alive while its peers read it.
"""
import time

import numpy as np
import pytest

import mbt_workloads as W

pytestmark = pytest.mark.gpu


def _run():
    b, c, n = W._fill([0, 1, 2], 1e-3, 10_000)
    return W.Run(W.ring_r0(), [dict(W.BROADBAND), dict(W.HOM)], b, c, n, seed=6, turns=40,
                 precision=W.PREC_MIXED)


def test_resident_grid_barrier_runs_out_and_reports_timeout():
    import paper_1809_00391_gb300 as pkg
    pkg.build()
    run = _run()
    tr = pkg.tracker_for_run(run, record_turns=64)
    C, per = tr.resident_shape()
    assert C > 0
    tr.init_particles()
    tr.sync()
    tr.set_wait_test(20_000_000, True)
    t0 = time.perf_counter()
    tr.track_resident(5)
    with pytest.raises(pkg.MBTError) as e:
        tr.sync()
    assert e.value.status == 5, str(e.value)   # MBT_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 5.0
    # the error is reported once; the context is usable again
    tr.sync()
    h, out = tr.histograms()
    assert np.array_equal(h.sum(axis=1) + out, run.n_mp)
    tr.set_wait_test(0, False)
    tr.track_resident(3)
    tr.sync()
    tr.close()
    # a fresh context tracks the same fill, resident and streaming alike
    a = pkg.tracker_for_run(run, record_turns=64)
    b = pkg.tracker_for_run(run, record_turns=64)
    a.init_particles()
    b.init_particles()
    a.track_resident(run.turns)
    b.track(run.turns)
    a.sync()
    b.sync()
    ra, rb = a.moments(0, run.turns), b.moments(0, run.turns)
    assert np.max(np.abs(ra[:, :, 0] - rb[:, :, 0]) / rb[:, :, 1]) <= 1e-3
    assert np.max(np.abs(ra[:, :, 1] - rb[:, :, 1]) / rb[:, :, 1]) <= 1e-3
    a.close()
    b.close()
