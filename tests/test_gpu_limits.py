"""The stated limits on the GPU (through the C ABI), against the FP64 oracle:
the largest fill (1024 bunches: 32 post-kernel bunch tiles, the most one
warp composes; a ring of h = 1200 with gaps and zero-current bunches) on the
FP64 and mixed paths, and the largest mixed-precision bunch (2^24 - 1
macro-particles, the most the byte-plane split of the tensor-core wake
admits per cell count)."""
import numpy as np
import pytest

import mbt_workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_1809_00391_gb300 as p
    p.build()
    return p


def _oracle(oracle_mod, run):
    return oracle_mod.OracleSim(run.ring, run.resonators, run.nbins, run.half_width_sigmas, run.buckets,
                                run.currents_A, run.n_mp, run.seed, run.flags)


def _max_fill(precision):
    ring = W.ring_r0(h=1200)
    b = np.concatenate([np.arange(0, 600), np.arange(650, 1074)]).astype(np.int32)   # 1024 bunches, two gaps
    cur = np.full(1024, 0.2e-3)
    cur[[5, 600, 1023]] = 0.0
    n = np.full(1024, 64, np.int64)
    n[::7] = 63
    hom = dict(W.HOM, Q=2000.0)   # a short history, so the oracle's direct sum stays fast
    return W.Run(ring, [dict(W.BROADBAND), hom], b, cur, n, seed=31, turns=6, precision=precision)


@pytest.mark.parametrize("prec", [W.PREC_F64, W.PREC_MIXED], ids=["f64", "mixed"])
def test_1024_bunches(pkg, oracle_mod, prec):
    run = _max_fill(prec)
    tr = pkg.tracker_for_run(run, record_turns=16)
    orc = _oracle(oracle_mod, run)
    tr.init_particles()
    orc.init_particles()
    tr.track(run.turns)
    rec_o = orc.track(run.turns)
    rec_g = tr.moments(0, run.turns)
    h_g, o_g = tr.histograms()
    assert np.array_equal(h_g.sum(axis=1) + o_g, run.n_mp)
    v_g, phi_g = tr.wake()
    a_o = orc.alr()[1]
    if prec == W.PREC_F64:
        h_o, o_o = orc.histograms()
        assert np.array_equal(h_g, h_o) and np.array_equal(o_g, o_o)
        assert np.max(np.abs(phi_g[0] - a_o)) <= 1e-11 * np.max(np.abs(a_o))
        tol = 1e-9
    else:
        # the oracle's phasors come from its own histograms, which differ by the
        # few particles FP32 binning moves across cell edges
        assert np.max(np.abs(phi_g[0] - a_o)) <= 1e-3 * np.max(np.abs(a_o))
        tol = 1e-3
    live = run.n_mp > 0
    st, sd = rec_o[:, live, 1], rec_o[:, live, 3]
    for col, scale in ((0, st), (1, st), (2, sd), (3, sd)):
        assert np.max(np.abs(rec_g[:, live, col] - rec_o[:, live, col]) / scale) <= tol, col
    # zero-current bunches leave nothing behind
    assert np.all(np.isfinite(v_g)) and np.all(v_g[[5, 600, 1023]] == 0.0)
    tr.close()


def test_largest_mixed_bunch(pkg, oracle_mod):
    n = (1 << 24) - 1
    b, c, nn = W._fill([0], 3e-3, n)
    run = W.Run(W.ring_r0(), [dict(W.BROADBAND), dict(W.HOM)], b, c, nn, seed=41, turns=3, precision=W.PREC_MIXED)
    tr = pkg.tracker_for_run(run, record_turns=8)
    tr.init_particles()
    tr.track(run.turns)
    h, out = tr.histograms()
    assert int(h.sum() + out[0]) == n
    assert h.max() < (1 << 24)
    v, _ = tr.wake()
    orc = _oracle(oracle_mod, run)
    q = run.currents_A[0] * run.ring["T0_s"] / n
    ref = orc.vsr_direct(h[0], q)
    assert np.max(np.abs(v[0] - ref)) <= 1e-4 * np.max(np.abs(ref))
    orc.init_particles()
    rec_o = orc.track(run.turns)
    rec_g = tr.moments(0, run.turns)
    st, sd = rec_o[:, :, 1], rec_o[:, :, 3]
    assert np.max(np.abs(rec_g[:, :, 0] - rec_o[:, :, 0]) / st) <= 1e-3
    assert np.max(np.abs(rec_g[:, :, 1] - rec_o[:, :, 1]) / st) <= 1e-3
    assert np.max(np.abs(rec_g[:, :, 3] - rec_o[:, :, 3]) / sd) <= 1e-3
    tr.close()
