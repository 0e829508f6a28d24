"""Resistive-wall short-range wake (the paper's Sec. 3 benchmark: a copper
pipe of 10 mm radius around the whole 'dc12c' ring) on the GPU, through the C
ABI, against the FP64 oracle, whose resistive-wall wake is its own (pinned)
implementation:

* the short-range voltage of the GPU's own histograms (both precisions) equals
  the oracle's direct double sum with the oracle's cell-averaged wake;
* a generic wake table (the resistive wall sampled by the oracle) gives the
  same voltages as the library's closed-form resistive wall;
* tracking a single bunch agrees with the oracle (moments);
* at low current the equilibrium bunch length follows the potential-well
  (Haissinski) solution on the tracking mesh, shorter than at zero current
  (negative momentum compaction, inductive wake), with the energy spread
  unchanged.
"""
import math

import numpy as np
import pytest

import mbt_workloads as W

pytestmark = pytest.mark.gpu

RW = dict(radius_m=0.01, conductivity_S_per_m=5.8e7, length_m=290.4)


@pytest.fixture(scope="module")
def pkg():
    import paper_1809_00391_gb300 as p
    p.build()
    return p


def _run(I, n_mp, turns, precision, seed=5, hw=5.0):
    b, c, n = W._fill([0], I, n_mp)
    return W.Run(W.ring_dc12c(), [], b, c, n, seed=seed, turns=turns, precision=precision,
                 half_width_sigmas=hw, resistive_wall=[dict(RW)], name="rw single bunch")


def _oracle(oracle_mod, run):
    return oracle_mod.OracleSim(run.ring, run.resonators, run.nbins, run.half_width_sigmas, run.buckets,
                                run.currents_A, run.n_mp, run.seed, run.flags, resistive_wall=run.resistive_wall)


# The FP64 bound is looser than the 1e-12 of the resonator paths because the
# two sides reach the resistive wall's cell averages by different quadratures:
# the library integrates the closed form over each lag cell (analytic head,
# adaptive quadrature for the rest), the oracle integrates samples of its own
# implementation of the form exactly.  Their difference, not the tracking
# arithmetic, sets the 2e-5; the mixed path adds its BF16 wake operands.
@pytest.mark.parametrize("prec,tol", [(W.PREC_F64, 2e-5), (W.PREC_MIXED, 1e-4)], ids=["f64", "mixed"])
def test_rw_voltage_matches_oracle(pkg, oracle_mod, prec, tol):
    run = _run(5e-3, 50_000, 1, prec)
    tr = pkg.tracker_for_run(run)
    tr.init_particles()
    tr.track(1)
    h, _ = tr.histograms()
    v, _ = tr.wake()
    o = _oracle(oracle_mod, run)
    q = run.currents_A[0] * run.ring["T0_s"] / run.n_mp[0]
    ref = o.vsr_direct(h[0], q)
    assert np.max(np.abs(v[0] - ref)) <= tol * np.max(np.abs(ref))
    tr.close()


def test_wake_table_equals_closed_form(pkg, oracle_mod):
    """The oracle's resistive-wall samples fed through mbt_add_wake_table give
    the voltages of mbt_add_resistive_wall (FP64 path)."""
    run = _run(5e-3, 50_000, 1, W.PREC_F64)
    o = _oracle(oracle_mod, run)
    t, w = oracle_mod.resistive_wall_table(RW["radius_m"], RW["conductivity_S_per_m"], RW["length_m"],
                                           (run.nbins + 1) * o.derived["Delta"])
    a = pkg.tracker_for_run(run)
    tab = W.Run(**{**run.__dict__, "resistive_wall": [], "wake_tables": [(t, w)]})
    b = pkg.tracker_for_run(tab)
    for tr in (a, b):
        tr.init_particles()
        tr.track(1)
    ha, _ = a.histograms()
    hb, _ = b.histograms()
    assert np.array_equal(ha, hb)
    va, _ = a.wake()
    vb, _ = b.wake()
    assert np.max(np.abs(va - vb)) <= 2e-5 * np.max(np.abs(va))
    a.close()
    b.close()


# Over 300 turns the 2e-5 difference of the two quadratures' voltages (above)
# moves the particles, and binning turns such shifts into whole-particle count
# changes, so the FP64 moments agree to 1e-4 of the rms, not to rounding.
@pytest.mark.parametrize("prec,tol", [(W.PREC_F64, 1e-4), (W.PREC_MIXED, 1e-3)], ids=["f64", "mixed"])
def test_rw_tracking_matches_oracle(pkg, oracle_mod, prec, tol):
    run = _run(2e-3, 20_000, 300, prec)
    tr = pkg.tracker_for_run(run, record_turns=run.turns)
    o = _oracle(oracle_mod, run)
    tr.init_particles()
    o.init_particles()
    tr.track(run.turns)
    rec_o = o.track(run.turns)
    rec_g = tr.moments(0, run.turns)
    st, sd = rec_o[:, :, 1], rec_o[:, :, 3]
    for col, scale in ((0, st), (1, st), (2, sd), (3, sd)):
        assert np.max(np.abs(rec_g[:, :, col] - rec_o[:, :, col]) / scale) <= tol, col
    tr.close()


def _haissinski_on_mesh(oracle_mod, run):
    """Potential-well equilibrium with the tracking model's wake: the line
    density at the cell centres, the voltage as the causal sum of the lag-cell
    wake, the potential by the trapezoid rule, then lambda ~ exp(-U / (alpha_c
    T0 sigma_E^2)) (alpha_c < 0 flips the well), damped fixed-point iteration."""
    ring = run.ring
    o = _oracle(oracle_mod, run)
    d = o.derived
    wl, D, H = o.wlag(), d["Delta"], d["H"]
    nb = run.nbins
    E0, T0, h, V, ac, sd = (ring[k] for k in ("E0_eV", "T0_s", "h", "V_rf_V", "alpha_c", "sigma_delta"))
    phis = d["phi_s"]
    w = 2 * math.pi * h / T0
    tc = -H + (np.arange(nb) + 0.5) * D
    Urf = -(V / E0) * ((np.cos(phis - w * tc) - math.cos(phis)) / w - math.sin(phis) * tc)
    I = run.currents_A[0]
    lam = np.exp(-tc ** 2 / (2 * d["sigma_tau0"] ** 2))
    lam /= lam.sum() * D
    for _ in range(20000):
        Vw = I * T0 * D * np.array([np.dot(lam[: j + 1], wl[j::-1]) for j in range(nb)])
        U = Urf + np.concatenate([[0.0], np.cumsum(0.5 * (Vw[1:] + Vw[:-1]) * D)]) / E0
        x = U / (ac * T0 * sd * sd)
        new = np.exp(-(x - x.min()))
        new /= new.sum() * D
        done = np.max(np.abs(new - lam)) < 1e-12 * np.max(lam)
        lam = new if done else 0.7 * lam + 0.3 * new
        if done:
            break
    m = np.sum(tc * lam) * D
    return m, math.sqrt(np.sum((tc - m) ** 2 * lam) * D), d["sigma_tau0"]


def test_low_current_equilibrium_follows_haissinski(pkg, oracle_mod):
    runs = [_run(I, 100_000, 16_000, W.PREC_MIXED, seed=40 + k) for k, I in enumerate((1e-4, 1e-3, 2e-3))]
    trs = [pkg.tracker_for_run(r, record_turns=r.turns) for r in runs]
    for t in trs:
        t.init_particles()
    b = pkg.Batch(trs)
    b.track(runs[0].turns)
    b.sync()
    b.close()
    sig = []
    for r, t in zip(runs, trs):
        rec = t.moments(0, r.turns)[-4000:, 0, :]    # the last ~0.9 damping time, after 2.5 of them
        m_h, s_h, st0 = _haissinski_on_mesh(oracle_mod, r)
        assert rec[:, 1].mean() == pytest.approx(s_h, rel=0.015), f"I = {r.currents_A[0]}"
        assert rec[:, 0].mean() == pytest.approx(m_h, abs=0.02 * st0)
        assert rec[:, 3].mean() == pytest.approx(r.ring["sigma_delta"], rel=0.01)
        sig.append(rec[:, 1].mean())
        t.close()
    assert sig[2] < sig[1] < sig[0]   # shortening with current
