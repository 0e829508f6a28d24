"""Batched tracking (GPU tests, through the C ABI): the 64-run batch of the
benchmark definitions at full size (3.3e9 macro-particles, 40 GB of state) in
one push + one post launch per turn, replayed from a CUDA graph with the
autotuned push tile; sampled runs agree bit for bit with the same runs
tracked alone, and the smallest run with the oracle."""
import numpy as np
import pytest

import mbt_workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_1809_00391_gb300 as p
    p.build()
    return p


def test_autotune_and_graph_keep_the_physics(pkg):
    run = W.fill_390().scaled(n_mp_per_bunch=20000, nb=40, turns=30)
    a = pkg.tracker_for_run(run, record_turns=64)
    a.init_particles()
    tile = a.autotune(2)
    assert tile in (2048, 4096, 8192, 16384, 32768)
    turns_done = a.info["turn"]
    a.set_graph(8)
    a.track(run.turns)
    b = pkg.tracker_for_run(run, record_turns=64)
    b.init_particles()
    b.track(turns_done + run.turns)
    for m in (0, 17, 39):
        ta, da = a.particles(m)
        tb, db = b.particles(m)
        assert np.array_equal(ta, tb) and np.array_equal(da, db)
    a.close()
    b.close()


def test_batched_64_runs_full_size(pkg, oracle_mod):
    runs = W.batched_runs(64, seed=42, turns=5)
    n_total = sum(r.n_particles for r in runs)
    assert 1e9 < n_total < 1e10
    ts = [pkg.tracker_for_run(r, record_turns=64) for r in runs]
    for t in ts:
        t.init_particles()
    batch = pkg.Batch(ts)
    tile = batch.autotune(2)
    batch.set_graph(5)
    batch.track(5)
    batch.sync()
    turn = ts[0].info["turn"]
    assert all(t.info["turn"] == turn for t in ts)
    for t, r in zip(ts, runs):
        h, out = t.histograms()
        assert np.array_equal(h.sum(axis=1) + out, r.n_mp)
    sizes = [r.n_particles for r in runs]
    small = sorted(range(64), key=lambda i: sizes[i])[:2]
    for i in small:
        r = runs[i]
        alone = pkg.tracker_for_run(r, record_turns=64)
        alone.set_tile(tile)   # same moment summation order as in the batch
        alone.init_particles()
        alone.track(turn)
        for m in range(0, r.nb, max(1, r.nb // 4)):
            ta, da = alone.particles(m)
            tb, db = ts[i].particles(m)
            assert np.array_equal(ta, tb) and np.array_equal(da, db)
        rec_a = alone.moments(turn - 3, 3)
        rec_b = ts[i].moments(turn - 3, 3)
        assert np.array_equal(rec_a, rec_b)
        alone.close()
    # the smallest run against the FP64 oracle
    i = small[0]
    r = runs[i]
    orc = oracle_mod.OracleSim(r.ring, r.resonators, r.nbins, r.half_width_sigmas, r.buckets, r.currents_A, r.n_mp,
                               r.seed, r.flags)
    orc.init_particles()
    rec_o = orc.track(turn)
    rec_g = ts[i].moments(0, turn)
    st, sd = rec_o[:, :, 1], rec_o[:, :, 3]
    assert np.max(np.abs(rec_g[:, :, 0] - rec_o[:, :, 0]) / st) <= 1e-3
    assert np.max(np.abs(rec_g[:, :, 3] - rec_o[:, :, 3]) / sd) <= 1e-3
    batch.close()
    for t in ts:
        t.close()


def test_streaming_batch_of_two_meshes(pkg):
    """A batch of two large runs on the streaming push with meshes of 128 and
    256 cells: each CTA pushes a tile of one run, then of the other, and the
    first run's particles outside its narrow mesh (which count into spill
    cells behind its 128 cells) must not reach the second run's cells 128 and
    up.  Histograms and moments equal the runs tracked alone, bit for bit."""
    ring = W.ring_r0()
    b, c, n = W._fill(range(30), 0.5e-3, 100_000)
    narrow = W.Run(ring, [dict(W.BROADBAND), dict(W.HOM)], b, c, n, seed=61, turns=3, precision=W.PREC_MIXED,
                   nbins=128, half_width_sigmas=2.0, name="128 cells over +-2 sigma")
    wide = W.Run(ring, [dict(W.BROADBAND), dict(W.HOM)], b, c, n, seed=62, turns=3, precision=W.PREC_MIXED,
                 name="256 cells over +-5 sigma")
    alone = []
    for r in (narrow, wide):
        t = pkg.tracker_for_run(r, record_turns=3)
        assert t.info["push_ctas"] > 0
        t.init_particles()
        t.track(3)
        h, out = t.histograms()
        alone.append((h, out, t.moments(0, 3)))
        t.close()
    assert alone[0][1].sum() > 10_000   # the narrow mesh leaves many particles outside
    trs = [pkg.tracker_for_run(r, record_turns=3) for r in (narrow, wide)]
    for t in trs:
        t.init_particles()
    bt = pkg.Batch(trs)
    bt.track(3)
    bt.sync()
    for t, (h, out, rec) in zip(trs, alone):
        h2, out2 = t.histograms()
        assert np.array_equal(h2, h) and np.array_equal(out2, out)
        assert np.array_equal(t.moments(0, 3), rec)
    bt.close()
    for t in trs:
        t.close()


def test_batch_lanes_equal_one_plan(pkg):
    """mbt_batch_set_lanes: the members tracked as 3 groups on streams of
    their own (graph replay, uneven runs: two rings, sizes 5 to 400 bunches)
    give every member's moments, histograms and particles bit for bit as the
    batch in one plan; 8 lanes for 5 members give one member per lane."""
    det = np.linspace(-300e3, 300e3, 3)
    runs = W.l5_scan_runs(det, "uniform", n_mp=2000, turns=40) + \
        W.l5_scan_runs(det[:1], "three_quarter", n_mp=3000, turns=40, seed=5) + \
        [W.fill_390().scaled(n_mp_per_bunch=4000, nb=5, turns=40)]
    turns = 40

    def track(nlanes):
        trs = [pkg.tracker_for_run(r, record_turns=turns) for r in runs]
        for t in trs:
            t.init_particles()
        b = pkg.Batch(trs)
        b.set_graph(10)
        if nlanes > 1:
            b.set_lanes(nlanes)
        b.track(turns - 5)
        b.track(5)
        b.sync()
        out = [(t.moments(0, turns), t.histograms()[0], t.particles(t.nb - 1)) for t in trs]
        b.close()
        for t in trs:
            t.close()
        return out

    ref = track(1)
    for nl in (3, 8):
        got = track(nl)
        for i, ((ma, ha, (ta, da)), (mb, hb, (tb, db))) in enumerate(zip(got, ref)):
            assert np.array_equal(ma, mb), (nl, i)
            assert np.array_equal(ha, hb), (nl, i)
            assert np.array_equal(ta, tb) and np.array_equal(da, db), (nl, i)
    trs = [pkg.tracker_for_run(runs[0], record_turns=4)]
    b = pkg.Batch(trs)
    with pytest.raises(pkg.MBTError):
        b.set_lanes(9)
    with pytest.raises(pkg.MBTError):
        b.set_lanes(0)
    b.close()
    trs[0].close()


def test_autotune_lanes_keeps_the_physics(pkg):
    """mbt_batch_autotune_lanes tracks real turns with 1..3 lanes and keeps the
    fastest: the runs continue bit for bit as one plan tracked as many turns."""
    det = np.linspace(-300e3, 300e3, 4)
    runs = W.l5_scan_runs(det, "uniform", n_mp=1000, turns=60)
    trial, top, more = 6, 3, 10
    total = 2 * trial * top + more
    a = [pkg.tracker_for_run(r, record_turns=total) for r in runs]
    for t in a:
        t.init_particles()
    ba = pkg.Batch(a)
    ba.set_graph(trial)
    k = ba.autotune_lanes(trial, top)
    assert 1 <= k <= top
    assert a[0].info["turn"] == 2 * trial * top
    ba.track(more)
    ba.sync()
    b = [pkg.tracker_for_run(r, record_turns=total) for r in runs]
    for t in b:
        t.init_particles()
    bb = pkg.Batch(b)
    bb.track(total)
    bb.sync()
    for ta, tb in zip(a, b):
        assert np.array_equal(ta.moments(0, total), tb.moments(0, total))
        pa, pb = ta.particles(ta.nb - 1), tb.particles(tb.nb - 1)
        assert np.array_equal(pa[0], pb[0]) and np.array_equal(pa[1], pb[1])
    with pytest.raises(pkg.MBTError):
        ba.autotune_lanes(trial, 9)
    ba.close()
    bb.close()
    for t in a + b:
        t.close()
