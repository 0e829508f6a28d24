"""Cluster-resident tracking (mbt_track_resident) against the streaming path
and the FP64 oracle (GPU tests, through the C ABI): single bunch, three
coupled bunches with the long-range HOM, handover between resident and
streaming turns, and the fill-size limit."""
import numpy as np
import pytest

import mbt_workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_1809_00391_gb300 as p
    p.build()
    return p


def _close(rec_g, rec_o, tol=1e-3):
    st, sd = rec_o[:, :, 1], rec_o[:, :, 3]
    assert np.max(np.abs(rec_g[:, :, 0] - rec_o[:, :, 0]) / st) <= tol
    assert np.max(np.abs(rec_g[:, :, 1] - rec_o[:, :, 1]) / st) <= tol
    assert np.max(np.abs(rec_g[:, :, 2] - rec_o[:, :, 2]) / sd) <= tol
    assert np.max(np.abs(rec_g[:, :, 3] - rec_o[:, :, 3]) / sd) <= tol


def _oracle(oracle_mod, run):
    o = oracle_mod.OracleSim(run.ring, run.resonators, run.nbins, run.half_width_sigmas, run.buckets,
                             run.currents_A, run.n_mp, run.seed, run.flags)
    o.init_particles()
    return o


def test_resident_single_bunch(pkg, oracle_mod):
    run = W.single_bunch(seed=3).scaled(turns=400)
    tr = pkg.tracker_for_run(run, precision=W.PREC_MIXED, record_turns=run.turns)
    C, per = tr.resident_shape()
    assert C >= 1 and per * C >= run.n_mp[0]
    tr.init_particles()
    tr.track_resident(run.turns)
    rec_g = tr.moments(0, run.turns)
    h, out = tr.histograms()
    assert h.sum() + out.sum() == run.n_mp[0]
    rec_o = _oracle(oracle_mod, run).track(run.turns)
    _close(rec_g, rec_o)
    tr.close()


def test_resident_three_bunches_long_range(pkg, oracle_mod):
    run = W.three_bunches(seed=1).scaled(turns=300)
    tr = pkg.tracker_for_run(run, precision=W.PREC_MIXED, record_turns=run.turns)
    C, per = tr.resident_shape()
    assert C >= 1
    tr.init_particles()
    tr.track_resident(run.turns)
    rec_g = tr.moments(0, run.turns)
    rec_o = _oracle(oracle_mod, run).track(run.turns)
    _close(rec_g, rec_o)
    tr.close()


def test_resident_and_streaming_turns_hand_over(pkg, oracle_mod):
    run = W.three_bunches(seed=7).scaled(n_mp_per_bunch=20000, turns=150)
    tr = pkg.tracker_for_run(run, precision=W.PREC_MIXED, record_turns=run.turns)
    tr.init_particles()
    tr.track_resident(50)
    tr.track(50)
    tr.track_resident(50)
    tr.sync()
    assert tr.info["turn"] == 150
    rec_g = tr.moments(0, 150)
    rec_o = _oracle(oracle_mod, run).track(150)
    _close(rec_g, rec_o)
    tr.close()


def test_resident_refuses_fills_that_do_not_fit(pkg):
    run = W.fill_390()
    tr = pkg.tracker_for_run(run, record_turns=16)
    assert tr.resident_shape() == (0, 0)
    with pytest.raises(pkg.MBTError, match="at most 32 bunches"):
        tr.track_resident(1)
    tr.close()


def test_resident_batch_runs_members_concurrently(pkg):
    """mbt_batch_track_resident: each member's resident kernel on a stream of
    its own gives the particles and moments of that member tracked resident
    alone, bit for bit (single bunches of several sizes and currents, and a
    three-bunch fill without long-range coupling); a member whose bunches
    couple over long range is refused before anything runs."""
    base = W.single_bunch(seed=3)
    runs = []
    for k, (n_mp, I) in enumerate([(20_000, 1e-3), (50_000, 3e-3), (8_192, 0.5e-3), (100_000, 2e-3)]):
        b, c, n = W._fill([0], I, n_mp)
        runs.append(W.Run(base.ring, [dict(W.BROADBAND)], b, c, n, seed=40 + k, turns=120,
                          precision=W.PREC_MIXED))
    b, c, n = W._fill([0, 1, 5], 1e-3, 30_000)
    runs.append(W.Run(base.ring, [dict(W.BROADBAND)], b, c, n, seed=50, turns=120, precision=W.PREC_MIXED))
    alone = []
    for r in runs:
        t = pkg.tracker_for_run(r, record_turns=r.turns)
        t.init_particles()
        t.track_resident(60)
        t.track_resident(60)
        t.sync()
        alone.append((t.moments(0, r.turns), [t.particles(m) for m in range(r.nb)]))
        t.close()
    trs = [pkg.tracker_for_run(r, record_turns=r.turns) for r in runs]
    for t in trs:
        t.init_particles()
    bt = pkg.Batch(trs)
    bt.track_resident(60)
    bt.track_resident(60)
    bt.sync()
    for t, r, (rec, parts) in zip(trs, runs, alone):
        assert t.info["turn"] == r.turns
        assert np.array_equal(t.moments(0, r.turns), rec)
        for m in range(r.nb):
            ta, da = t.particles(m)
            assert np.array_equal(ta, parts[m][0]) and np.array_equal(da, parts[m][1])
    bt.close()
    for t in trs:
        t.close()
    # three bunches coupled by the long-range HOM: refused, nothing tracked
    coupled = W.three_bunches(seed=1).scaled(turns=10)
    t1 = pkg.tracker_for_run(runs[0], record_turns=10)
    t2 = pkg.tracker_for_run(coupled, precision=W.PREC_MIXED, record_turns=10)
    t1.init_particles()
    t2.init_particles()
    bt = pkg.Batch([t1, t2])
    with pytest.raises(pkg.MBTError, match="long range") as e:
        bt.track_resident(5)
    assert e.value.status == 6
    bt.sync()
    assert t1.info["turn"] == 0 and t2.info["turn"] == 0
    bt.close()
    t1.close()
    t2.close()
