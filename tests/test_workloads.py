"""The seeded synthetic inputs follow their stated recipes (ring R0, the
wakes, the fills, the 64-run batch, the Poisson request stream, the L5
detuning scan), and the generators are reproducible: the tests and the
benchmark rely on the same draws."""
import numpy as np
import pytest

import mbt_workloads as W


def test_ring_r0_and_wakes():
    r = W.ring_r0()
    assert (r["E0_eV"], r["h"], r["V_rf_V"], r["alpha_c"], r["U0_eV"], r["sigma_delta"], r["tau_z_s"]) == \
        (2.4e9, 480, 2.1e6, 6e-4, 0.5e6, 9e-4, 4.5e-3)
    assert r["T0_s"] * W.C_LIGHT == pytest.approx(288.0)
    assert W.ring_r0(484)["h"] == 484
    assert W.ring_dc12c()["h"] == 484 and W.ring_dc12c()["alpha_c"] < 0
    assert W.BROADBAND == dict(Rs_ohm=5e3, fr_Hz=10e9, Q=1.0, range=W.RANGE_SHORT)
    assert W.HOM == dict(Rs_ohm=1e6, fr_Hz=1.5e9, Q=2e4, range=W.RANGE_BOTH)


def test_fixed_fills():
    s, t, f = W.single_bunch(), W.three_bunches(), W.fill_390()
    assert (s.nb, s.n_particles, s.turns, s.precision) == (1, 10_000, 1000, W.PREC_F64)
    assert list(t.buckets) == [0, 1, 2] and t.n_particles == 300_000 and t.turns == 10_000
    assert list(f.buckets) == list(range(390)) and np.all(f.n_mp == 100_000) and f.turns == 20_000
    assert np.allclose(f.currents_A, 0.5e-3) and f.precision == W.PREC_MIXED
    assert [r["fr_Hz"] for r in f.resonators] == [10e9, 1.5e9]


def test_batch_of_64_runs():
    runs = W.batched_runs()
    assert len(runs) == 64
    assert runs[0].n_particles == W.batched_runs()[0].n_particles           # reproducible
    assert sum(r.n_particles for r in runs) == 3_350_698_012                  # 3.35e9 particles
    for r in runs:
        assert 1 <= r.nb <= 484 and list(r.buckets) == list(range(r.nb))
        assert r.ring["h"] == (484 if r.nb > 480 else 480)
        assert 1e4 <= r.n_mp[0] <= 1e6 and np.all(r.n_mp == r.n_mp[0])
        assert 0.1e-3 <= r.currents_A[0] <= 3e-3 and r.precision == W.PREC_MIXED
    assert len({r.seed for r in runs}) == 64
    nmp = np.log10([r.n_mp[0] for r in runs])
    assert nmp.min() < 4.5 and nmp.max() > 5.5       # log-uniform over two decades


def test_poisson_request_stream():
    reqs = W.serving_stream()
    assert len(reqs) == 200
    t = np.array([q.arrival_s for q in reqs])
    assert np.all(np.diff(t) > 0)
    assert np.mean(np.diff(t)) == pytest.approx(1 / 20.0, rel=0.2)
    for q in reqs:
        r = q.run
        h = r.ring["h"]
        assert 1 <= r.nb <= h and list(r.buckets) == list(range(r.nb))
        assert 1e4 <= r.n_mp[0] <= 2e5 + 1 and 0.1e-3 <= r.currents_A[0] <= 5e-3
        assert 1e9 <= r.resonators[1]["fr_Hz"] <= 3e9 and 2000 <= r.turns <= 20_000
    work = np.mean([q.run.n_particles * q.run.turns for q in reqs])
    assert 0.5e11 < work < 5e11                      # ~1.7e11 mp-turns per request


def test_l5_scan_fills():
    det = [-500e3, 0.0, 500e3]
    u = W.l5_scan_runs(det, "uniform")
    q = W.l5_scan_runs(det, "three_quarter")
    assert u[0].nb == 484 and q[0].nb == 363
    for runs in (u, q):
        assert runs[0].currents_A.sum() == pytest.approx(0.4)
        assert [r.resonators[0]["fr_Hz"] - W.L5_FR_HZ for r in runs] == pytest.approx(det)
        assert all(len(r.resonators) == 1 and r.resonators[0]["range"] == W.RANGE_BOTH for r in runs)
    with pytest.raises(ValueError):
        W.l5_scan_runs(det, "half")
