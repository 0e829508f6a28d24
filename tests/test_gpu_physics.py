"""Physics-level parity of the CUDA path (GPU tests, through the C ABI).

Coupled-bunch growth rates of the mixed-precision and FP64 paths against the
oracle and against Eq. 7 (within 2 %); the 390-bunch fill at full size
(3.9e7 macro-particles) against the oracle for 30 turns: moments, exact
short-range convolution of the GPU's own histograms, conservation of
particles; three bunches at full size over 1000 turns (moments within 1e-3).
"""
import math

import numpy as np
import pytest

import mbt_workloads as W
from physics_helpers import eq7_rate, fit_rate, map_tune, mode_amplitudes, point_bunch_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_1809_00391_gb300 as p
    p.build()
    return p


def _oracle_for(oracle_mod, run):
    return oracle_mod.OracleSim(run.ring, run.resonators, run.nbins, run.half_width_sigmas, run.buckets,
                                run.currents_A, run.n_mp, run.seed, run.flags)


@pytest.mark.parametrize("prec", [W.PREC_MIXED, W.PREC_F64], ids=["mixed", "f64"])
def test_four_bunch_growth_rates_match_oracle_and_eq7(pkg, oracle_mod, prec):
    ring = W.ring_r0()
    nu = map_tune(ring)
    fr = (1441 + nu) / ring["T0_s"]
    Rs, I, turns = 1e7, 1e-3, 2000
    run, parts = point_bunch_run(4, fr, Rs, I, turns, precision=prec)
    tr = pkg.tracker_for_run(run, record_turns=turns)
    orc = _oracle_for(oracle_mod, run)
    for m, (t, d) in enumerate(parts):
        tr.set_particles(m, t, d)
        orc.set_particles(m, t, d)
    tr.track(turns)
    rec_g = tr.moments(0, turns)
    rec_o = orc.track(turns)
    Xg, Xo = mode_amplitudes(rec_g), mode_amplitudes(rec_o)
    pred1 = eq7_rate(4, 1, fr, Rs, 2e4, I, nu)
    g1, o1 = fit_rate(Xg[1], 1000, 2000), fit_rate(Xo[1], 1000, 2000)
    g3, o3 = fit_rate(Xg[3], 0, 600), fit_rate(Xo[3], 0, 600)
    assert g1 == pytest.approx(o1, rel=0.02)
    assert g1 == pytest.approx(pred1, rel=0.02)
    assert g3 == pytest.approx(o3, rel=0.02)
    tr.close()


def test_three_adjacent_bunches_growth_rate_matches_oracle(pkg, oracle_mod):
    """The three-bunch configuration's geometry (buckets 0, 1, 2) with the HOM
    moved onto the upper synchrotron sideband of line 1441 and enlarged so the
    instability grows within 2000 turns; no radiation."""
    ring = W.ring_r0()
    nu = map_tune(ring)
    fr = (1441 + nu) / ring["T0_s"]
    hom = dict(Rs_ohm=2e7, fr_Hz=fr, Q=2e4, range=W.RANGE_LONG)
    n_mp = 400
    run = W.Run(ring, [hom], np.array([0, 1, 2], np.int32), np.full(3, 1e-3), np.full(3, n_mp, np.int64), seed=5,
                turns=2000, precision=W.PREC_MIXED, flags=W.NO_SR)
    rng = np.random.default_rng(9)
    T0, ac = ring["T0_s"], ring["alpha_c"]
    st = 3e-12
    sdl = st * 2 * math.pi * nu / (ac * T0)
    tr = pkg.tracker_for_run(run, record_turns=run.turns)
    orc = _oracle_for(oracle_mod, run)
    for m in range(3):
        ph = rng.uniform(0, 2 * math.pi)
        t = rng.normal(5e-12 * math.cos(ph), st, n_mp)
        d = rng.normal(5e-12 * math.sin(ph) * sdl / st, sdl, n_mp)
        tr.set_particles(m, t, d)
        orc.set_particles(m, t, d)
    tr.track(run.turns)
    rec_g = tr.moments(0, run.turns)
    rec_o = orc.track(run.turns)
    # growth of the centroid envelope summed over the bunches
    def env_rate(rec):
        X = mode_amplitudes(rec)
        amp = np.sqrt(np.sum(np.abs(X) ** 2, axis=0))
        n = np.arange(1000, 2000)
        return np.polyfit(n, np.log(amp[1000:2000]), 1)[0] / T0
    rg, ro = env_rate(rec_g), env_rate(rec_o)
    assert ro > 100.0
    assert rg == pytest.approx(ro, rel=0.02)
    tr.close()


def test_fill390_full_size_against_oracle(pkg, oracle_mod):
    run = W.fill_390(seed=1)
    turns = 30
    tr = pkg.tracker_for_run(run, record_turns=64)
    tr.init_particles()
    tr.track(turns)
    rec_g = tr.moments(0, turns)
    h, out = tr.histograms()
    v, phi = tr.wake()
    assert np.array_equal(h.sum(axis=1) + out, run.n_mp)
    orc = _oracle_for(oracle_mod, run)
    orc.init_particles()
    rec_o = orc.track(turns)
    st, sd = rec_o[:, :, 1], rec_o[:, :, 3]
    assert np.max(np.abs(rec_g[:, :, 0] - rec_o[:, :, 0]) / st) <= 1e-3
    assert np.max(np.abs(rec_g[:, :, 1] - rec_o[:, :, 1]) / st) <= 1e-3
    assert np.max(np.abs(rec_g[:, :, 2] - rec_o[:, :, 2]) / sd) <= 1e-3
    assert np.max(np.abs(rec_g[:, :, 3] - rec_o[:, :, 3]) / sd) <= 1e-3
    h_o, _ = orc.histograms()
    # FP32 binning moves at most a few particles per bunch across cell edges
    assert np.max(np.abs(h - h_o).sum(axis=1)) <= 1e-3 * run.n_mp[0]
    # the tensor-core wake of sampled bunches is the exact convolution of the GPU's own counts
    q = run.currents_A * run.ring["T0_s"] / run.n_mp
    for m in (0, 1, 31, 32, 200, 389):
        ref = orc.vsr_direct(h[m], q[m])
        assert np.max(np.abs(v[m] - ref)) <= 1e-4 * np.max(np.abs(ref)), f"bunch {m}"
    # the oracle's wake of its own (nearly identical) histograms is close to the GPU's
    vo = orc.vsr()
    assert np.max(np.abs(v - vo)) <= 5e-3 * np.max(np.abs(vo))
    tr.close()


def test_three_bunches_full_size_1000_turns(pkg, oracle_mod):
    run = W.three_bunches(seed=2).scaled(turns=1000)
    tr = pkg.tracker_for_run(run, precision=W.PREC_MIXED, record_turns=run.turns)
    tr.init_particles()
    tr.track(run.turns)
    rec_g = tr.moments(0, run.turns)
    orc = _oracle_for(oracle_mod, run)
    orc.init_particles()
    rec_o = orc.track(run.turns)
    st, sd = rec_o[:, :, 1], rec_o[:, :, 3]
    assert np.max(np.abs(rec_g[:, :, 0] - rec_o[:, :, 0]) / st) <= 1e-3
    assert np.max(np.abs(rec_g[:, :, 1] - rec_o[:, :, 1]) / st) <= 1e-3
    assert np.max(np.abs(rec_g[:, :, 2] - rec_o[:, :, 2]) / sd) <= 1e-3
    assert np.max(np.abs(rec_g[:, :, 3] - rec_o[:, :, 3]) / sd) <= 1e-3
    tr.close()
