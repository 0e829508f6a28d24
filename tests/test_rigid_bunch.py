"""The rigid-bunch linearised one-turn map (physics_helpers.RigidBunchModel)
and the oracle's coupled-bunch growth on non-uniform fills (CPU).

Eq. 7 of the paper gives coupled-bunch growth rates for M equal bunches
equally spaced around the ring.  For other fills (three adjacent bunches; a
3/4 train with a gap) the rates come from the eigenvalues of the rigid-bunch
map: 2M centroid coordinates plus two per long-range resonator.  The model is
pinned here to closed forms (its derivative, the single-bunch map at zero
current, Eq. 7 on uniform fills), and the oracle's tracked growth is checked
against it on the non-uniform fills.
"""
import math

import numpy as np
import pytest

import mbt_workloads as W
from physics_helpers import RigidBunchModel, eq7_rate, map_tune, projected_rate


def _sideband_hom(Rs, Q=2e4, range_=W.RANGE_LONG):
    ring = W.ring_r0()
    return dict(Rs_ohm=Rs, fr_Hz=(1441 + map_tune(ring)) / ring["T0_s"], Q=Q, range=range_)


def test_jacobian_is_the_derivative_of_the_map():
    ring = W.ring_r0()
    res = [_sideband_hom(1e7), dict(Rs_ohm=3e5, fr_Hz=2.2e9, Q=500.0, range=W.RANGE_BOTH)]
    m = RigidBunchModel(ring, [0, 5, 9, 300], [1e-3, 2e-3, 0.5e-3, 1e-3], res, 10e-12)
    x = m.fixed_point()
    assert np.max(np.abs(m.turn(x) - x) / m._scales(x)) < 1e-6
    # in the variables' own units (ps, 1e-6, kV-ish phasors), element by element
    sc = m._scales(x)
    J = m.jacobian(x) * sc[None, :] / sc[:, None]
    Jf = m.jacobian_fd(x) * sc[None, :] / sc[:, None]
    assert np.max(np.abs(J - Jf)) < 1e-6 * np.max(np.abs(J))


@pytest.mark.parametrize("flags", [0, W.NO_SR])
def test_zero_current_gives_the_single_bunch_map(flags):
    """Without charge every bunch follows the linearised single-particle map
    (kick-then-drift, Eqs. 1, 2, 5): eigenvalues e^{+-i 2 pi nu} sqrt(1 - D),
    cos(2 pi nu) = 1 - (2 pi nu_s)^2 / 2 for a point bunch."""
    ring = W.ring_r0()
    m = RigidBunchModel(ring, [0, 7, 100], [0.0, 0.0, 0.0], [_sideband_hom(1e7)], 1e-15, flags=flags)
    rates, ev, *_ = m.modes()
    D = 0.0 if flags & W.NO_SR else 2 * ring["T0_s"] / ring["tau_z_s"]
    bunch = ev[np.abs(np.abs(ev) - 1) < 0.05]   # the resonator's own mode decays as e^{-a T0} = 0.8
    assert len(bunch) == 6
    assert np.allclose(np.abs(bunch) ** 2, 1 - D, rtol=1e-12, atol=1e-12)
    nu = np.angle(bunch[bunch.imag > 0]) / (2 * math.pi)
    # the tune of the damped map: trace = 2 - (2 pi nu_s)^2 (1 - D) + ... written from its matrix
    if flags & W.NO_SR:
        assert np.allclose(nu, map_tune(ring, sr=False), rtol=1e-9)


@pytest.mark.parametrize("M,mus,Rs,Q", [(1, (0,), 1e6, 1e6), (4, (1, 3), 1e7, 2e4)])
def test_uniform_fills_reproduce_eq7(M, mus, Rs, Q):
    """M equal, equally spaced point bunches, a narrow HOM on the upper
    synchrotron sideband of line 1441: the growth (and damping) rates of the
    map's modes equal Eq. 7 for the coupled-bunch modes mu within 1 %.  (Eq. 7
    is first order in the coupling: the rates must stay well below the
    resonator's bandwidth w_r / 2Q, 4.4e3 /s at Q = 1e6.)"""
    ring = W.ring_r0()
    nu = map_tune(ring)
    I = 1e-3
    hom = _sideband_hom(Rs, Q)
    m = RigidBunchModel(ring, [k * (ring["h"] // M) for k in range(M)], [I] * M, [hom], 1e-13, flags=W.NO_SR)
    rates, ev, *_ = m.modes()
    bunch = rates[np.abs(np.abs(ev) - 1) < 0.05]
    for mu in mus:
        pred = eq7_rate(M, mu, hom["fr_Hz"], Rs, Q, I, nu)
        assert abs(pred) > 20
        assert np.min(np.abs(bunch - pred)) <= 0.01 * abs(pred), (mu, pred, np.sort(bunch))


def _oracle_growth(oracle_mod, ring, buckets, currents, res, sigma, n_mp, turns, flags, window, seed=5):
    """Oracle tracking started at the model's fixed point (Gaussian bunches of
    rms sigma around each centroid), the phasor A_0 read every turn; returns
    (model's dominant rate, tracked rate of that mode over `window`)."""
    m = RigidBunchModel(ring, buckets, currents, res, sigma, flags=flags)
    rates, ev, vr, vl, x0 = m.modes()
    k = int(np.argmax(rates + 1e-9 * np.sign(ev.imag)))
    M = len(buckets)
    s = oracle_mod.OracleSim(ring, res, 256, 5.0, buckets, currents, [n_mp] * M, seed, flags)
    rng = np.random.default_rng(seed)
    sdl = ring["sigma_delta"] if not flags & W.NO_SR else sigma * 2 * math.pi * map_tune(ring) / (
        ring["alpha_c"] * ring["T0_s"])
    for j in range(M):
        s.set_particles(j, x0[j] + rng.normal(0.0, sigma, n_mp), x0[M + j] + rng.normal(0.0, sdl, n_mp))
    states = np.empty((turns, m.n))
    for n in range(turns):
        rec = s.track(1)[0]
        states[n, :M], states[n, M:2 * M] = rec[:, 0], rec[:, 2]
        a = s.alr()
        for r in range(m.nr):
            states[n, 2 * M + 2 * r], states[n, 2 * M + 2 * r + 1] = a[r, 0].real, a[r, 0].imag
    return float(rates[k]), projected_rate(states, vl[:, k], *window, ring["T0_s"])


def test_three_adjacent_bunches_grow_at_the_rigid_bunch_rate(oracle_mod):
    """Buckets 0, 1, 2 (the three-bunch configuration's geometry), the HOM on
    the upper sideband of line 1441, no radiation: not a uniform fill, so Eq. 7
    does not apply; the tracked mode grows at the rigid-bunch rate within 2 %."""
    ring = W.ring_r0()
    pred, got = _oracle_growth(oracle_mod, ring, [0, 1, 2], [1e-3] * 3, [_sideband_hom(2e7)], 3e-12, 400, 1500,
                               W.NO_SR, (300, 1400))
    assert pred > 150
    assert got == pytest.approx(pred, rel=0.02)


@pytest.mark.slow
def test_three_quarter_fill_grows_at_the_rigid_bunch_rate(oracle_mod):
    """The 390-bunch train with a 90-bucket gap at 0.5 mA per bunch, matched
    bunch length, radiation damping on (excitation off, so that the centroids
    carry no noise), a long-range HOM of Q = 2000 (short history, so that the
    oracle runs in seconds): the dominant coupled-bunch mode of the tracked
    fill grows at the rigid-bunch rate within 2 %."""
    ring = W.ring_r0()
    hom = dict(Rs_ohm=1e6, fr_Hz=1.5e9, Q=2000.0, range=W.RANGE_LONG)
    M = 390
    pred, got = _oracle_growth(oracle_mod, ring, list(range(M)), [0.5e-3] * M, [hom], 13.2285e-12, 256, 700,
                               W.NO_QE, (100, 650))
    assert pred > 4000
    assert got == pytest.approx(pred, rel=0.02)
