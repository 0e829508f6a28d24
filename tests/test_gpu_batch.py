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
