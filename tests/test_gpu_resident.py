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
