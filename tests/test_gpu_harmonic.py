"""Active harmonic RF cavity (the paper's RF step with additional harmonic
cavities) on the GPU, through the C ABI: a third-harmonic cavity set for a
flat potential on ring R0 with the broadband wake, against the FP64 oracle
(FP64 path: histograms bit for bit, coordinates to 1e-12; mixed and resident
paths: moments within 1e-3 of the rms), and the analytic double-RF
equilibrium (drawn from it, the bunch stays in it on the mixed path)."""
import numpy as np
import pytest

import mbt_workloads as W
from physics_helpers import double_rf_equilibrium, flat_potential

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_1809_00391_gb300 as p
    p.build()
    return p


def _run(precision, n_mp, turns, I=1e-3, res=(W.BROADBAND,), hw=8.0, seed=9):
    ring = W.ring_r0()
    hc = flat_potential(ring)[0]
    b, c, n = W._fill([0], I, n_mp)
    return W.Run(ring, [dict(r) for r in res], b, c, n, seed=seed, turns=turns, precision=precision,
                 half_width_sigmas=hw, harmonic_cavities=[hc], name="flat third harmonic")


def _oracle(oracle_mod, run):
    return oracle_mod.OracleSim(run.ring, run.resonators, run.nbins, run.half_width_sigmas, run.buckets,
                                run.currents_A, run.n_mp, run.seed, run.flags,
                                harmonic_cavities=run.harmonic_cavities)


def test_f64_harmonic_cavity_matches_oracle(pkg, oracle_mod):
    run = _run(W.PREC_F64, 10_000, 200)
    tr = pkg.tracker_for_run(run, record_turns=run.turns)
    orc = _oracle(oracle_mod, run)
    tr.init_particles()
    orc.init_particles()
    tr.track(run.turns)
    orc.track(run.turns, record=False)
    hg, og = tr.histograms()
    ho, oo = orc.histograms()
    assert np.array_equal(hg, ho) and np.array_equal(og, oo)
    tg, dg = tr.particles(0)
    to, do = orc.particles(0)
    assert np.max(np.abs(tg - to)) <= 1e-12 * np.max(np.abs(to))
    assert np.max(np.abs(dg - do)) <= 1e-12 * np.max(np.abs(do))
    tr.close()


@pytest.mark.parametrize("resident", [False, True], ids=["streaming", "resident"])
def test_mixed_harmonic_cavity_matches_oracle(pkg, oracle_mod, resident):
    run = _run(W.PREC_MIXED, 20_000, 300)
    tr = pkg.tracker_for_run(run, record_turns=run.turns)
    orc = _oracle(oracle_mod, run)
    tr.init_particles()
    orc.init_particles()
    if resident:
        tr.track_resident(run.turns)
    else:
        tr.track(run.turns)
    rec_g = tr.moments(0, run.turns)
    rec_o = orc.track(run.turns)
    st, sd = rec_o[:, :, 1], rec_o[:, :, 3]
    for col, scale in ((0, st), (1, st), (2, sd), (3, sd)):
        assert np.max(np.abs(rec_g[:, :, col] - rec_o[:, :, col]) / scale) <= 1e-3, col
    tr.close()


def test_flat_potential_equilibrium_on_gpu(pkg, oracle_mod):
    """No wake: particles drawn from the analytic double-RF equilibrium keep
    its length (within 1 %) and centre over 3000 turns."""
    run = _run(W.PREC_MIXED, 200_000, 3000, I=0.0, res=(), hw=12.0)
    st0 = oracle_mod.derive(run.ring)["sigma_tau0"]
    tau, lam = double_rf_equilibrium(run.ring, run.harmonic_cavities, 12 * st0)
    mean = np.trapezoid(tau * lam, tau)
    sig = float(np.sqrt(np.trapezoid((tau - mean) ** 2 * lam, tau)))
    g = np.random.default_rng(23)
    cdf = np.cumsum(lam)
    cdf /= cdf[-1]
    n = run.n_mp[0]
    tr = pkg.tracker_for_run(run, record_turns=run.turns)
    tr.set_particles(0, np.interp(g.random(n), cdf, tau), g.normal(0.0, run.ring["sigma_delta"], n))
    tr.track(run.turns)
    rec = tr.moments(0, run.turns)[1000:, 0, :]
    assert rec[:, 1].mean() == pytest.approx(sig, rel=0.01)
    assert abs(rec[:, 0].mean() - mean) < 0.02 * sig
    assert rec[:, 3].mean() == pytest.approx(run.ring["sigma_delta"], rel=0.01)
    tr.close()
