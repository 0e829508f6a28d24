"""Host-side analysis of instability scans (paper_1809_00391_gb300.scan),
pinned on the CPU: the linear one-turn map against its closed-form determinant
and the textbook synchrotron tune, the normal form against iteration of the
map, growth fits against planted exponentials, and Eq. 7 against the
independent implementation of the physics tests."""
import math

import numpy as np
import pytest

import mbt_workloads as W
from paper_1809_00391_gb300 import scan as S
from physics_helpers import eq7_rate, textbook_nu_s

RINGS = [W.ring_r0(), W.ring_dc12c()]


@pytest.mark.parametrize("ring", RINGS, ids=["r0", "dc12c"])
@pytest.mark.parametrize("sr", [True, False])
def test_linear_map_determinant_and_tune(ring, sr):
    M = S.linear_map(ring, sr)
    D = 2 * ring["T0_s"] / ring["tau_z_s"] if sr else 0.0
    assert np.linalg.det(M) == pytest.approx(1 - D, rel=1e-12)
    # kick-then-drift tune: cos(2 pi nu) = tr / (2 sqrt(det)); close to the textbook nu_s
    nu = S.synchrotron_tune(ring, sr)
    assert math.cos(2 * math.pi * nu) == pytest.approx(np.trace(M) / (2 * math.sqrt(1 - D)), rel=1e-12)
    assert nu == pytest.approx(textbook_nu_s(ring, sr), rel=1e-3)


@pytest.mark.parametrize("ring", RINGS, ids=["r0", "dc12c"])
def test_normal_form_advances_by_the_eigenvalue(ring):
    M = S.linear_map(ring)
    w, lam = S.normal_form(ring)
    x = np.array([3e-12, -2e-4])
    z0 = w @ x
    for n in range(1, 200):
        x = M @ x
        assert w @ x == pytest.approx(z0 * lam ** n, rel=1e-9)
    assert abs(lam) == pytest.approx(math.sqrt(np.linalg.det(M)), rel=1e-12)


def _planted(ring, M, mu0, gamma, turns, amp=1e-12, noise=0.0, seed=0):
    """Centroids (rec layout) of M bunches carrying one coupled-bunch mode mu0
    growing at gamma [1/s] on top of the free oscillation, plus noise (a
    fraction of the initial amplitude of each coordinate)."""
    Mat = S.linear_map(ring)
    ev, vr = np.linalg.eig(Mat)
    i = int(np.argmax(ev.imag))
    lam, v = ev[i], vr[:, i]
    n = np.arange(turns)[:, None]
    m = np.arange(M)[None, :]
    c = amp * np.exp(gamma * ring["T0_s"] * n) * lam ** n * np.exp(2j * math.pi * mu0 * m / M)
    rec = np.zeros((turns, M, 6))
    rec[:, :, 0] = (c * v[0]).real
    rec[:, :, 2] = (c * v[1]).real
    if noise:
        g = np.random.default_rng(seed)
        rec[:, :, 0] += g.normal(0, noise * amp * abs(v[0]), (turns, M))
        rec[:, :, 2] += g.normal(0, noise * amp * abs(v[1]), (turns, M))
    return rec, abs(lam)


@pytest.mark.parametrize("ring", RINGS, ids=["r0", "dc12c"])
def test_growth_fits_recover_a_planted_mode(ring):
    M, mu0, gamma, turns = 16, 5, 900.0, 1500
    rec, lam_abs = _planted(ring, M, mu0, gamma, turns)
    expect = gamma + math.log(lam_abs) / ring["T0_s"]   # growth plus radiation damping of the map
    lo, hi = 300, turns - 300   # inside the valid range of the one-period moving average
    # a static offset per bunch (a shifted equilibrium) does not change the rates
    rec[:, :, 0] += np.linspace(-3, 3, M)[None, :] * 1e-12
    rates = S.bunch_growth_rates(rec, ring, lo, hi)
    assert np.allclose(rates, expect, rtol=2e-3)
    X = np.fft.fft(S.oscillation(S.centroid_amplitudes(rec, ring), ring), axis=1)
    assert int(np.argmax(np.abs(X[hi]))) == mu0
    mr = S.mode_growth_rates(rec, ring, lo, hi)
    assert mr[mu0] == pytest.approx(expect, rel=2e-3)
    # with noise the fit still finds the rate of a mode well above it
    noisy, _ = _planted(ring, M, mu0, gamma, turns, noise=0.05, seed=1)
    assert S.mode_growth_rates(noisy, ring, lo, hi)[mu0] == pytest.approx(expect, rel=0.02)


@pytest.mark.parametrize("ring", RINGS, ids=["r0", "dc12c"])
def test_oscillation_removes_a_moving_equilibrium(ring):
    """A free damped oscillation about an equilibrium that steps (beam loading
    settles within a few fill times of the HOM) and then drifts linearly is
    recovered by ``oscillation`` up to the residual of a one-period average."""
    turns = 3000
    rec, _ = _planted(ring, 1, 0, 0.0, turns)
    pure = S.centroid_amplitudes(rec, ring)[:, 0]
    w, _ = S.normal_form(ring)
    dtau = 3 * abs(pure[0]) / abs(w[0])   # three oscillation amplitudes
    n = np.arange(turns)
    rec[:, 0, 0] += dtau * (n >= 20) + 0.5 * dtau * n / turns
    osc = S.oscillation(S.centroid_amplitudes(rec, ring), ring)[:, 0]
    P = int(round(1 / S.synchrotron_tune(ring)))
    assert np.isnan(osc[: P // 2]).all() and not np.isnan(osc[P // 2: turns - P]).any()
    ok = (n >= 20 + P) & ~np.isnan(osc)   # averaging windows that no longer contain the step
    assert np.max(np.abs(osc[ok] - pure[ok]) / np.abs(pure[ok])) < 0.05


def test_adaptive_rate_fits_growth_above_noise_only():
    """An oscillation growing out of incoherent noise (random phase each turn,
    as the centroid noise of a finite bunch is) is fitted where it stands
    clear of the noise; pure noise has no measurable growth."""
    T0 = 1e-6
    g = np.random.default_rng(5)
    n = np.arange(6000)
    noise = g.normal(0, 1.0, n.size) + 1j * g.normal(0, 1.0, n.size)
    amp = np.abs(noise + 0.01 * np.exp(2000.0 * T0 * n) * np.exp(0.0148j * n))
    assert S.adaptive_rate(amp, T0, cap=200.0) == pytest.approx(2000.0, rel=0.03)
    assert np.isnan(S.adaptive_rate(np.abs(noise), T0))
    # saturation above the cap is left out of the fit
    assert S.adaptive_rate(np.minimum(amp, 150.0), T0, cap=100.0) == pytest.approx(2000.0, rel=0.03)
