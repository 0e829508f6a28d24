"""Serving with continuous batching (GPU tests, through the C ABI): requests
submitted while others run are admitted as slots and memory free up, all
active requests advance in the same kernel launches, admission respects the
memory budget, and every request's result equals the same request tracked
alone, bit for bit."""
import dataclasses
import time

import numpy as np
import pytest

import mbt_workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_1809_00391_gb300 as p
    p.build()
    return p


def _requests():
    stream = W.serving_stream(6, rate_hz=20.0, seed=7)
    out = []
    for i, rq in enumerate(stream):
        r = rq.run.scaled(n_mp_per_bunch=int(2000 + 500 * i), nb=min(rq.run.nb, 8 + 7 * i), turns=60 + 20 * i)
        out.append(r)
    return out


def _alone(pkg, run):
    t = pkg.tracker_for_run(run, record_turns=run.turns)
    t.init_particles()
    t.track(run.turns)
    rec = t.moments(0, run.turns)
    t.close()
    nb = rec.shape[1]
    # left-to-right sums over bunches, the server's order (np.mean sums pairwise)
    s2t = np.cumsum(rec[:, :, 0] * rec[:, :, 0], axis=1)[:, -1]
    s2d = np.cumsum(rec[:, :, 2] * rec[:, :, 2], axis=1)[:, -1]
    hist = np.stack([np.sqrt(s2t / nb), np.sqrt(s2d / nb)], axis=1)
    return rec[-1], hist


def _check_against_alone(pkg, srv, ids, runs):
    for rid, r in zip(ids, runs):
        fm, hist = srv.result(rid)
        fm_a, hist_a = _alone(pkg, r)
        assert np.array_equal(fm, fm_a), f"request {rid}: final moments differ"
        assert hist.shape == hist_a.shape
        assert np.array_equal(hist, hist_a), f"request {rid}: centroid history differs"


@pytest.mark.parametrize("lanes", [1, 2], ids=["one_plan", "two_lanes"])
def test_results_are_the_same_alone_and_in_the_mix(pkg, lanes):
    runs = _requests()
    srv = pkg.Server(hbm_budget_bytes=8 << 30, max_active=3, turns_per_step=25, lanes=lanes)
    ids = []
    for i, r in enumerate(runs):
        ids.append(srv.submit(r))
        if i == 2:
            time.sleep(0.05)   # later requests arrive while the first ones run
    for rid in ids:
        srv.wait(rid, timeout_s=300)
    st = srv.stats()
    assert st["completed"] == len(runs) and st["failed"] == 0
    assert 1 < st["max_active_seen"] <= 3
    _check_against_alone(pkg, srv, ids, runs)
    # continuous batching: some request started before an earlier one finished
    stat = [srv.status(i) for i in ids]
    assert any(stat[j]["t_start"] < stat[j - 1]["t_finish"] for j in range(1, len(ids)))
    srv.close()


def test_admission_respects_the_memory_budget(pkg):
    # four requests of the same size (different seeds): a budget of 2.5 of
    # them admits two at a time, never three
    base = _requests()[3]
    runs = [dataclasses.replace(base, seed=base.seed + k) for k in range(4)]
    one = pkg.tracker_for_run(runs[0], record_turns=25).info["device_bytes"]
    srv = pkg.Server(hbm_budget_bytes=int(2.5 * one), max_active=16, turns_per_step=25)
    ids = [srv.submit(r) for r in runs]
    for rid in ids:
        srv.wait(rid, timeout_s=300)
    st = srv.stats()
    assert st["completed"] == 4
    assert st["max_active_seen"] == 2
    assert st["max_bytes_seen"] <= 2.5 * one
    _check_against_alone(pkg, srv, ids, runs)
    big = W.fill_390()
    with pytest.raises(pkg.MBTError):
        srv.submit(big)
    srv.close()


def test_one_at_a_time(pkg):
    """Serial admission: each request replaces a destroyed one (whose host and
    device addresses the allocator may hand out again); every batch must be
    built for its own members."""
    runs = _requests()[:4]
    srv = pkg.Server(hbm_budget_bytes=8 << 30, max_active=1, turns_per_step=25)
    ids = [srv.submit(r) for r in runs]
    for rid in ids:
        srv.wait(rid, timeout_s=300)
    st = srv.stats()
    assert st["completed"] == 4 and st["max_active_seen"] == 1
    _check_against_alone(pkg, srv, ids, runs)
    srv.close()
