"""Parity of the CUDA path with the FP64 oracle (GPU tests, through the C ABI).

FP64 path: histograms bit-exact, coordinates within 1e-12 relative (to the
largest |coordinate| of the bunch), wakes within 1e-12, over 100 turns, on the
same Philox streams.  Mixed path: bunch centroid and rms within 1e-3 of the
rms (relative), the tensor-core wake within 1e-4 of the exact convolution of
the same histogram, the long-range phasors within 1e-6.
"""
import math

import numpy as np
import pytest

import mbt_workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_1809_00391_gb300 as p
    p.build()
    return p


def _pair(pkg, oracle_mod, run, precision=None):
    tr = pkg.tracker_for_run(run, precision=precision)
    orc = oracle_mod.OracleSim(run.ring, run.resonators, run.nbins, run.half_width_sigmas, run.buckets,
                               run.currents_A, run.n_mp, run.seed, run.flags)
    return tr, orc


def _rel_close(a, b, tol):
    scale = max(np.max(np.abs(b)), 1e-300)
    return np.max(np.abs(a - b)) <= tol * scale


def _compare_f64(tr, orc, nb, check_wake=True):
    h_g, o_g = tr.histograms()
    h_o, o_o = orc.histograms()
    assert np.array_equal(h_g, h_o), f"histograms differ in {np.sum(h_g != h_o)} cells"
    assert np.array_equal(o_g, o_o)
    for m in range(nb):
        tg, dg = tr.particles(m)
        to, do = orc.particles(m)
        assert _rel_close(tg, to, 1e-12), f"bunch {m}: tau max diff {np.max(np.abs(tg - to))}"
        assert _rel_close(dg, do, 1e-12), f"bunch {m}: delta max diff {np.max(np.abs(dg - do))}"
    if check_wake:
        vg, phg = tr.wake()
        vo = orc.vsr()
        assert _rel_close(vg, vo, 1e-12)
        nlong = sum(1 for r in orc.resonators if r["range"] & W.RANGE_LONG)
        if nlong:
            ao = orc.alr()
            long_rows = [i for i, r in enumerate(orc.resonators) if r["range"] & W.RANGE_LONG]
            for li, ri in enumerate(long_rows):
                assert _rel_close(phg[li], ao[ri], 1e-11), f"long-range phasor {li}"


def test_f64_single_bunch_turn_by_turn(pkg, oracle_mod):
    run = W.single_bunch(seed=1)
    tr, orc = _pair(pkg, oracle_mod, run)
    tr.init_particles()
    orc.init_particles()
    for m in range(run.nb):
        tg, dg = tr.particles(m)
        to, do = orc.particles(m)
        assert _rel_close(tg, to, 1e-15) and _rel_close(dg, do, 1e-15)
    for _ in range(5):
        tr.track(1)
        orc.track(1, record=False)
        _compare_f64(tr, orc, run.nb)
    tr.track(95)
    rec_o = orc.track(95)
    _compare_f64(tr, orc, run.nb)
    rec_g = tr.moments(5, 95)
    assert np.allclose(rec_g[:, :, 4:], rec_o[:, :, 4:], rtol=0, atol=0)
    sig = rec_o[:, :, 1:2]
    assert np.max(np.abs(rec_g[:, :, 0] - rec_o[:, :, 0])) <= 1e-11 * np.max(rec_o[:, :, 1])
    assert np.max(np.abs(rec_g[:, :, 1] - rec_o[:, :, 1])) <= 1e-11 * np.max(rec_o[:, :, 1])
    assert np.max(np.abs(rec_g[:, :, 3] - rec_o[:, :, 3])) <= 1e-11 * np.max(rec_o[:, :, 3])
    tr.close()


def test_f64_three_bunches_long_range(pkg, oracle_mod):
    run = W.three_bunches(seed=2).scaled(n_mp_per_bunch=20001, turns=100)
    tr, orc = _pair(pkg, oracle_mod, run)
    tr.init_particles()
    orc.init_particles()
    tr.track(3)
    orc.track(3, record=False)
    _compare_f64(tr, orc, run.nb)
    tr.track(97)
    orc.track(97, record=False)
    _compare_f64(tr, orc, run.nb)
    tr.close()


@pytest.mark.parametrize("case", ["ragged", "ngp-nosr", "noqe-64bins", "wide-gaps"])
def test_f64_edge_cases(pkg, oracle_mod, case):
    ring = W.ring_r0()
    res = [dict(W.BROADBAND), dict(Rs_ohm=2e5, fr_Hz=1.2e9, Q=500.0, range=W.RANGE_BOTH)]
    if case == "ragged":
        run = W.Run(ring, res, np.array([0, 5, 6, 200], np.int32), np.array([1e-3, 0.2e-3, 2e-3, 0.7e-3]),
                    np.array([1, 3, 2049, 5001], np.int64), seed=99, turns=40)
    elif case == "ngp-nosr":
        run = W.Run(ring, res, np.array([10, 11], np.int32), np.array([1e-3, 1e-3]),
                    np.array([4097, 999], np.int64), seed=5, turns=40, flags=W.NO_SR | W.KICK_NGP)
    elif case == "noqe-64bins":
        run = W.Run(ring, res, np.array([0, 240], np.int32), np.array([2e-3, 2e-3]),
                    np.array([3000, 3000], np.int64), seed=6, turns=40, flags=W.NO_QE, nbins=64,
                    half_width_sigmas=4.0)
    else:
        b = np.array([0, 1, 2, 3, 100, 101, 470, 479], np.int32)
        run = W.Run(ring, res, b, np.full(8, 0.8e-3), np.full(8, 1500, np.int64), seed=8, turns=40)
    tr, orc = _pair(pkg, oracle_mod, run, precision=W.PREC_F64)
    tr.init_particles()
    orc.init_particles()
    tr.track(run.turns)
    orc.track(run.turns, record=False)
    _compare_f64(tr, orc, run.nb)
    tr.close()


def test_f64_many_bunches_span_several_tiles(pkg, oracle_mod):
    # 70 bunches -> three post-kernel bunch tiles; long-range scan across tiles
    b = np.arange(0, 140, 2, dtype=np.int32)
    run = W.Run(W.ring_r0(), [dict(W.BROADBAND), dict(W.HOM)], b, np.full(70, 0.5e-3), np.full(70, 600, np.int64),
                seed=12, turns=30)
    tr, orc = _pair(pkg, oracle_mod, run, precision=W.PREC_F64)
    tr.init_particles()
    orc.init_particles()
    tr.track(run.turns)
    orc.track(run.turns, record=False)
    _compare_f64(tr, orc, run.nb)
    tr.close()


# ----------------------------------------------------------------------------- mixed precision
def _mixed_vs_oracle_moments(rec_g, rec_o, tol=1e-3):
    st = rec_o[:, :, 1]
    sd = rec_o[:, :, 3]
    assert np.max(np.abs(rec_g[:, :, 0] - rec_o[:, :, 0]) / st) <= tol
    assert np.max(np.abs(rec_g[:, :, 1] - rec_o[:, :, 1]) / st) <= tol
    assert np.max(np.abs(rec_g[:, :, 2] - rec_o[:, :, 2]) / sd) <= tol
    assert np.max(np.abs(rec_g[:, :, 3] - rec_o[:, :, 3]) / sd) <= tol


def test_mixed_single_bunch_moments(pkg, oracle_mod):
    run = W.single_bunch(seed=3)
    tr, orc = _pair(pkg, oracle_mod, run, precision=W.PREC_MIXED)
    tr.init_particles()
    orc.init_particles()
    tr.track(1000)
    rec_o = orc.track(1000)
    rec_g = tr.moments(0, 1000)
    _mixed_vs_oracle_moments(rec_g, rec_o)
    # particle by particle after the whole run (same Philox streams)
    tg, dg = tr.particles(0)
    to, do = orc.particles(0)
    assert np.median(np.abs(tg - to)) <= 1e-4 * rec_o[-1, 0, 1]
    tr.close()


def test_mixed_three_bunches_moments(pkg, oracle_mod):
    run = W.three_bunches(seed=1).scaled(n_mp_per_bunch=20000, turns=300)
    tr, orc = _pair(pkg, oracle_mod, run, precision=W.PREC_MIXED)
    tr.init_particles()
    orc.init_particles()
    tr.track(run.turns)
    rec_o = orc.track(run.turns)
    rec_g = tr.moments(0, run.turns)
    _mixed_vs_oracle_moments(rec_g, rec_o)
    tr.close()


def test_mixed_tiny_ragged_bunches(pkg, oracle_mod):
    """Per-tile push (a run far too small to stream) with bunch sizes that are
    not multiples of 4, one bunch of a single particle: every particle is pushed
    and deposited exactly once per turn."""
    run = W.Run(W.ring_r0(), [dict(W.BROADBAND), dict(W.HOM)], np.array([0, 3, 7], np.int32), np.full(3, 1e-3),
                np.array([37, 1, 510], np.int64), seed=41, turns=50, precision=W.PREC_MIXED)
    tr, orc = _pair(pkg, oracle_mod, run, precision=W.PREC_MIXED)
    _ragged_vs_oracle(tr, orc, run)
    assert tr.info["push_ctas"] == 0
    tr.close()


def test_streaming_push_ragged_bunches(pkg, oracle_mod):
    """Streaming push (one run large enough for equal per-SM shares) on a fill
    that mixes two bunches of 1.3e6 particles, one not a multiple of 4, with
    bunches of 37, 1 and 1001 particles: shares cut bunches at multiples of 4,
    the tiny bunches sit inside one share, and every particle is pushed and
    deposited exactly once per turn."""
    n_mp = np.array([1_300_000, 37, 1, 1_300_003, 1001], np.int64)
    run = W.Run(W.ring_r0(), [dict(W.BROADBAND), dict(W.HOM)], np.array([0, 3, 7, 12, 20], np.int32),
                np.full(5, 1e-3), n_mp, seed=43, turns=10, precision=W.PREC_MIXED)
    tr, orc = _pair(pkg, oracle_mod, run, precision=W.PREC_MIXED)
    _ragged_vs_oracle(tr, orc, run)
    assert tr.info["push_ctas"] > 0
    tr.close()


def _ragged_vs_oracle(tr, orc, run):
    """Histogram counts exact; per-particle coordinates against the oracle with
    tolerances scaled by the fill's own spreads (a one-particle bunch has none)."""
    tr.init_particles()
    orc.init_particles()
    tr.track(run.turns)
    orc.track(run.turns)
    h, out = tr.histograms()
    assert np.array_equal(h.sum(axis=1) + out, run.n_mp)
    sig = tr.info["sigma_tau0_s"]
    dsig = np.std(np.concatenate([orc.particles(m)[1] for m in range(run.nb)]))   # energy spread of the fill
    for m in range(run.nb):
        tg, dg = tr.particles(m)
        to, do = orc.particles(m)
        assert np.median(np.abs(tg - to)) <= 1e-4 * sig and np.max(np.abs(tg - to)) <= 1e-2 * sig, f"bunch {m}"
        assert np.median(np.abs(dg - do)) <= 1e-4 * dsig and np.max(np.abs(dg - do)) <= 1e-2 * dsig, f"bunch {m}"


@pytest.mark.parametrize("nbins", [128, 256])
def test_tensor_core_wake_matches_direct_convolution(pkg, oracle_mod, nbins):
    """The tcgen05 Toeplitz contraction against the exact FP64 double sum of the
    same histograms (70 bunches: three bunch tiles, a ragged last tile)."""
    b = np.arange(0, 70, dtype=np.int32)
    n = np.array([2000 + 37 * i for i in range(70)], np.int64)
    run = W.Run(W.ring_r0(), [dict(W.BROADBAND), dict(W.HOM)], b, np.linspace(0.1e-3, 3e-3, 70), n, seed=4,
                turns=1, precision=W.PREC_MIXED, nbins=nbins)
    tr, orc = _pair(pkg, oracle_mod, run)
    tr.init_particles()
    tr.track(1)
    h, out = tr.histograms()
    assert np.array_equal(h.sum(axis=1) + out, n)
    v, phi = tr.wake()
    q = run.currents_A * run.ring["T0_s"] / n
    for m in range(run.nb):
        ref = orc.vsr_direct(h[m], q[m])
        assert np.max(np.abs(v[m] - ref)) <= 1e-4 * np.max(np.abs(ref)), f"bunch {m}"
    tr.close()


def test_mixed_long_range_phasor_matches_history_sum(pkg, oracle_mod):
    """Feed the GPU's own histograms of several turns to the oracle's direct
    history sum: the scanned phasors agree."""
    b = np.array([0, 1, 2, 40, 41, 300], np.int32)
    run = W.Run(W.ring_r0(), [dict(W.BROADBAND), dict(W.HOM)], b, np.full(6, 1e-3), np.full(6, 4000, np.int64),
                seed=21, turns=6, precision=W.PREC_MIXED)
    tr, orc = _pair(pkg, oracle_mod, run)
    tr.init_particles()
    for _ in range(run.turns):
        tr.track(1)
        h, _ = tr.histograms()
        orc.feed_histograms(h)
    _, phi = tr.wake()
    ao = orc.alr()[1]
    assert np.max(np.abs(phi[0] - ao)) <= 1e-6 * np.max(np.abs(ao))
    tr.close()


# ----------------------------------------------------------------------------- batch + checkpoint
@pytest.mark.parametrize("prec", [W.PREC_F64, W.PREC_MIXED])
def test_batch_equals_alone(pkg, prec):
    runs = [W.Run(W.ring_r0(), [dict(W.BROADBAND), dict(W.HOM)], np.array([0, 3], np.int32), np.full(2, 1e-3),
                  np.array([5000, 3001], np.int64), seed=31, turns=20, precision=prec),
            W.Run(W.ring_r0(484), [dict(W.BROADBAND), dict(W.HOM, fr_Hz=1.7e9)], np.arange(40, dtype=np.int32),
                  np.full(40, 0.3e-3), np.full(40, 700, np.int64), seed=32, turns=20, precision=prec)]
    alone = []
    for r in runs:
        t = pkg.tracker_for_run(r)
        t.init_particles()
        t.track(r.turns)
        alone.append([t.particles(m) for m in range(r.nb)])
        t.close()
    ts = [pkg.tracker_for_run(r) for r in runs]
    for t in ts:
        t.init_particles()
    bt = pkg.Batch(ts)
    bt.track(20)
    bt.sync()
    for t, r, ref in zip(ts, runs, alone):
        assert t.info["turn"] == 20
        for m in range(r.nb):
            tg, dg = t.particles(m)
            assert np.array_equal(tg, ref[m][0]) and np.array_equal(dg, ref[m][1])
    bt.close()
    for t in ts:
        t.close()


def test_streaming_batch_equals_alone(pkg):
    """Two runs large enough for the streaming push (one with ragged and tiny
    bunches), tracked alone and as one batch in which every CTA takes one
    share of each run: particles, histograms, wakes and moments bit for bit."""
    runs = [W.Run(W.ring_r0(), [dict(W.BROADBAND), dict(W.HOM)], np.arange(30, dtype=np.int32), np.full(30, 0.5e-3),
                  np.full(30, 90_000, np.int64), seed=51, turns=12, precision=W.PREC_MIXED),
            W.Run(W.ring_r0(484), [dict(W.BROADBAND), dict(W.HOM, fr_Hz=1.7e9)], np.arange(100, 127, dtype=np.int32),
                  np.full(27, 0.8e-3), np.array([100_003] * 26 + [37], np.int64), seed=52, turns=12,
                  precision=W.PREC_MIXED)]

    def state(t, r):
        h, out = t.histograms()
        v, phi = t.wake()
        return [t.particles(m) for m in range(r.nb)], h, out, v, phi, t.moments(0, r.turns)

    alone = []
    for r in runs:
        t = pkg.tracker_for_run(r)
        t.init_particles()
        t.track(r.turns)
        assert t.info["push_ctas"] > 0
        alone.append(state(t, r))
        t.close()
    ts = [pkg.tracker_for_run(r) for r in runs]
    for t in ts:
        t.init_particles()
    bt = pkg.Batch(ts)
    bt.track(12)
    bt.sync()
    for t, r, ref in zip(ts, runs, alone):
        got = state(t, r)
        for m in range(r.nb):
            assert np.array_equal(got[0][m][0], ref[0][m][0]) and np.array_equal(got[0][m][1], ref[0][m][1]), m
        for a, b in zip(got[1:], ref[1:]):
            assert np.array_equal(a, b)
    bt.close()
    for t in ts:
        t.close()


@pytest.mark.parametrize("prec", [W.PREC_F64, W.PREC_MIXED])
def test_checkpoint_resume_is_bit_identical(pkg, prec):
    run = W.Run(W.ring_r0(), [dict(W.BROADBAND), dict(W.HOM)], np.array([0, 1, 2], np.int32), np.full(3, 1e-3),
                np.full(3, 3000, np.int64), seed=41, turns=60, precision=prec)
    a = pkg.tracker_for_run(run)
    a.init_particles()
    a.track(30)
    blob = a.save_state()
    a.track(30)
    ref = [a.particles(m) for m in range(run.nb)]
    b = pkg.tracker_for_run(run)
    b.load_state(blob)
    assert b.info["turn"] == 30
    b.track(30)
    for m in range(run.nb):
        tg, dg = b.particles(m)
        assert np.array_equal(tg, ref[m][0]) and np.array_equal(dg, ref[m][1])
    a.close()
    b.close()


def test_graph_replay_equals_plain_launches(pkg):
    run = W.single_bunch(seed=9).scaled(n_mp_per_bunch=20000, turns=64)
    run.precision = W.PREC_MIXED
    a = pkg.tracker_for_run(run)
    a.init_particles()
    a.track(64)
    ref = a.particles(0)
    b = pkg.tracker_for_run(run)
    b.set_graph(16)
    b.init_particles()
    b.track(64)
    t, d = b.particles(0)
    assert np.array_equal(t, ref[0]) and np.array_equal(d, ref[1])
    a.close()
    b.close()
