"""Pins of the FP64 oracle against facts fixed outside it.

Every test here runs on the CPU.  None compares the oracle with itself: each
checks it against a published test vector, a closed form from the textbook
physics of the paper's map (Sec. 2.2, Eqs. 1, 2, 5), a brute-force count, or an
independent definition of the same object (the wake via its impedance).
"""
import math
import os

import numpy as np
import pytest
from scipy import linalg, stats

import mbt_workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _ring(**kw):
    r = W.ring_r0()
    r.update(kw)
    return r


def _sim(oracle_mod, ring=None, res=(), buckets=(0,), currents=(0.0,), n_mp=(2,), seed=1, flags=0,
         nbins=256, hw=5.0):
    ring = ring or W.ring_r0()
    return oracle_mod.OracleSim(ring, list(res), nbins, hw, list(buckets), list(currents), list(n_mp),
                                seed, flags)


def textbook_nu_s(ring, sr=True):
    """Small-amplitude synchrotron tune, nu_s^2 = alpha_c h eV cos(phi_s) / (2 pi E0)."""
    U0 = ring["U0_eV"] if sr else 0.0
    phi = math.asin(U0 / ring["V_rf_V"])
    if ring["alpha_c"] < 0:
        phi = math.pi - phi
    return math.sqrt(ring["alpha_c"] * ring["h"] * ring["V_rf_V"] * math.cos(phi) / (2 * math.pi * ring["E0_eV"]))


# --------------------------------------------------------------------------- RNG
def test_philox_known_answers(oracle_mod):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert oracle_mod.philox4x32_10(v[0:4], v[4:6]) == tuple(v[6:10])


def test_uniform_open_interval(oracle_mod):
    assert oracle_mod.u01(0) == 2.0 ** -33
    assert oracle_mod.u01(0xFFFFFFFF) == 1.0 - 2.0 ** -33
    assert oracle_mod.u01(0x80000000) == 0.5 + 2.0 ** -33
    assert oracle_mod.u01(1) == 1.5 * 2.0 ** -32


def test_box_muller_closed_forms(oracle_mod):
    a, b = oracle_mod.box_muller(math.exp(-0.5), 0.0)
    assert a == pytest.approx(1.0, abs=1e-15) and b == pytest.approx(0.0, abs=1e-15)
    a, b = oracle_mod.box_muller(math.exp(-2.0), 0.25)
    assert a == pytest.approx(0.0, abs=1e-15) and b == pytest.approx(2.0, abs=1e-15)
    a, b = oracle_mod.box_muller(math.exp(-2.0), 0.125)
    assert a == pytest.approx(math.sqrt(2.0), rel=1e-15) and b == pytest.approx(math.sqrt(2.0), rel=1e-15)
    a, b = oracle_mod.box_muller(math.exp(-0.5), 0.5)
    assert a == pytest.approx(-1.0, abs=1e-15)


def test_normals_are_standard_and_independent(oracle_mod):
    n = 10000
    r = np.array([oracle_mod.normal_quad(12345, i, 3, 7, 0) for i in range(n)])
    z = r.ravel()
    assert stats.kstest(z, "norm").pvalue > 1e-3
    assert abs(z.mean()) < 5 / math.sqrt(z.size)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0 / z.size)
    c = np.corrcoef(r.T)
    assert np.max(np.abs(c - np.eye(4))) < 5 / math.sqrt(n)
    # the quad is Box-Muller on the block's four words
    w = oracle_mod.philox4x32_10((17, 3, 7, 0), (12345, 0))
    a = oracle_mod.box_muller(oracle_mod.u01(w[0]), oracle_mod.u01(w[1]))
    b = oracle_mod.box_muller(oracle_mod.u01(w[2]), oracle_mod.u01(w[3]))
    assert oracle_mod.normal_quad(12345, 17, 3, 7, 0) == (a[0], a[1], b[0], b[1])
    # different counters or seeds give different streams
    assert oracle_mod.normal_quad(12345, 0, 3, 7, 0) != oracle_mod.normal_quad(12345, 0, 3, 8, 0)
    assert oracle_mod.normal_quad(12345, 0, 3, 7, 0) != oracle_mod.normal_quad(12346, 0, 3, 7, 0)
    assert oracle_mod.normal_quad(2 ** 32 + 5, 0, 3, 7, 0) != oracle_mod.normal_quad(5, 0, 3, 7, 0)


# --------------------------------------------------------------------------- single-particle map
def _one_turn_jacobian(oracle_mod, ring, flags, tau0=0.0, d0=0.0, ht=1e-15, hd=1e-8):
    s = _sim(oracle_mod, ring=ring, n_mp=(4,), flags=flags)
    t = np.array([tau0, tau0 + ht, tau0, tau0 - ht])
    d = np.array([d0, d0, d0 + hd, d0])
    s.set_particles(0, t, d)
    s.track(1, record=False)
    t1, d1 = s.particles(0)
    J = np.array([[(t1[1] - t1[3]) / (2 * ht), (t1[2] - t1[0]) / hd],
                  [(d1[1] - d1[3]) / (2 * ht), (d1[2] - d1[0]) / hd]])
    return J, (t1[0], d1[0])


def test_synchronous_particle_is_fixed(oracle_mod):
    # Eq. 1: at the synchronous phase the RF gain cancels the radiation loss
    for ring in (W.ring_r0(), W.ring_dc12c()):
        s = _sim(oracle_mod, ring=ring, n_mp=(2,), flags=W.NO_QE)
        s.set_particles(0, [0.0, 0.0], [0.0, 0.0])
        s.track(50, record=False)
        t, d = s.particles(0)
        assert abs(t[0]) < 1e-22 and abs(d[0]) < 1e-17


@pytest.mark.parametrize("ring", [W.ring_r0(), W.ring_dc12c()], ids=["R0", "dc12c"])
def test_linear_map_area_and_tune(oracle_mod, ring):
    # without radiation the one-turn map preserves area; its trace gives the tune
    J, _ = _one_turn_jacobian(oracle_mod, ring, W.NO_SR)
    assert np.linalg.det(J) == pytest.approx(1.0, abs=1e-7)
    nus = textbook_nu_s(ring, sr=False)
    tune_map = math.acos(np.trace(J) / 2) / (2 * math.pi)
    assert tune_map == pytest.approx(math.acos(1 - (2 * math.pi * nus) ** 2 / 2) / (2 * math.pi), rel=1e-6)
    # with damping (no excitation) the area shrinks by 1 - 2 T0 / tau_z per turn
    J, _ = _one_turn_jacobian(oracle_mod, ring, W.NO_QE)
    assert np.linalg.det(J) == pytest.approx(1.0 - 2 * ring["T0_s"] / ring["tau_z_s"], abs=1e-7)


def test_small_amplitude_tune_fft(oracle_mod):
    ring = W.ring_r0()
    nus = textbook_nu_s(ring, sr=False)
    s = _sim(oracle_mod, ring=ring, n_mp=(2,), flags=W.NO_SR)
    s.set_particles(0, [1e-14, 1e-14], [0.0, 0.0])
    n = 8192
    rec = s.track(n)
    x = rec[:, 0, 0]
    win = np.hanning(n)
    sp = np.abs(np.fft.rfft((x - x.mean()) * win))
    k = int(np.argmax(sp[1:])) + 1
    a, b, c = np.log(sp[k - 1]), np.log(sp[k]), np.log(sp[k + 1])
    kk = k + 0.5 * (a - c) / (a - 2 * b + c)
    nu_fft = kk / n
    nu_map = math.acos(1 - (2 * math.pi * nus) ** 2 / 2) / (2 * math.pi)
    assert abs(nu_fft - nu_map) < 1e-5
    # with radiation (phi_s = 0.2404): nu_s = 6.2413e-3, the map's tune 6.2417e-3
    nus_sr = textbook_nu_s(ring, sr=True)
    assert abs(nus_sr - 6.2413e-3) < 1e-7
    assert abs(math.acos(1 - (2 * math.pi * nus_sr) ** 2 / 2) / (2 * math.pi) - 6.2417e-3) < 1e-7


def test_matched_initial_distribution(oracle_mod):
    ring = W.ring_r0()
    nus = textbook_nu_s(ring)
    sig_t = ring["alpha_c"] * ring["sigma_delta"] * ring["T0_s"] / (2 * math.pi * nus)
    s = _sim(oracle_mod, ring=ring, n_mp=(40001,))
    s.init_particles()
    t, d = s.particles(0)
    n = t.size
    assert abs(t.mean()) < 4 * sig_t / math.sqrt(n)
    assert t.std() == pytest.approx(sig_t, rel=4 * math.sqrt(0.5 / n))
    assert d.std() == pytest.approx(ring["sigma_delta"], rel=4 * math.sqrt(0.5 / n))
    assert sig_t == pytest.approx(13.2285e-12, rel=1e-4)


def test_covariance_follows_linear_recursion(oracle_mod):
    """Radiation damping + quantum excitation (Eq. 5): starting from a point, the
    sample covariance follows Sigma' = M Sigma M^T + g g^T of the linearised
    one-turn map, and tends to the discrete Lyapunov solution."""
    ring = W.ring_r0()
    E0, T0, V, ac = ring["E0_eV"], ring["T0_s"], ring["V_rf_V"], ring["alpha_c"]
    phi = math.asin(ring["U0_eV"] / V)
    K = (V / E0) * (2 * math.pi * ring["h"] / T0) * math.cos(phi)
    D = 2 * T0 / ring["tau_z_s"]
    a = ac * T0
    qe = ring["sigma_delta"] * math.sqrt(2 * D)
    M = np.array([[1 - a * K * (1 - D), a * (1 - D)], [-K * (1 - D), 1 - D]])
    g = qe * np.array([a, 1.0])
    N = 20000
    s = _sim(oracle_mod, ring=ring, n_mp=(N,))
    s.set_particles(0, np.zeros(N), np.zeros(N))
    Sig = np.zeros((2, 2))
    done = 0
    for n_check in (200, 800, 3000):
        s.track(n_check - done, record=False)
        for _ in range(n_check - done):
            Sig = M @ Sig @ M.T + np.outer(g, g)
        done = n_check
        t, d = s.particles(0)
        C = np.cov(np.vstack([t, d]), bias=True)
        tol = 5 * math.sqrt(2.0 / N)
        assert C[0, 0] == pytest.approx(Sig[0, 0], rel=tol)
        assert C[1, 1] == pytest.approx(Sig[1, 1], rel=tol)
        assert abs(C[0, 1] / math.sqrt(C[0, 0] * C[1, 1]) - Sig[0, 1] / math.sqrt(Sig[0, 0] * Sig[1, 1])) < 5 / math.sqrt(N)
    # the fixed point: sigma_delta ~ 1.0003 sigma_E and sigma_tau ~ 1.0004 sigma_tau0
    nus = textbook_nu_s(ring)
    st0 = ac * ring["sigma_delta"] * T0 / (2 * math.pi * nus)
    S = np.diag([1.0 / st0, 1.0 / ring["sigma_delta"]])   # solve in units of sigma
    Ms = S @ M @ np.linalg.inv(S)
    gs = S @ g
    Seq = linalg.solve_discrete_lyapunov(Ms, np.outer(gs, gs))
    assert math.sqrt(Seq[1, 1]) == pytest.approx(1.00030, abs=5e-5)
    assert math.sqrt(Seq[0, 0]) == pytest.approx(1.00041, abs=5e-5)


def test_recorded_moments_and_counts(oracle_mod):
    """Per-turn statistics (Sec. 2.4) are the population mean and rms of the
    bunch, and every particle is either binned or counted outside."""
    s = _sim(oracle_mod, res=[dict(W.BROADBAND)], currents=(1e-3,), n_mp=(5001,), hw=2.0)
    s.init_particles()
    rec = s.track(3)
    t, d = s.particles(0)
    hist, out = s.histograms()
    assert rec[-1, 0, 0] == pytest.approx(np.mean(t), rel=1e-12, abs=1e-26)
    assert rec[-1, 0, 1] == pytest.approx(np.std(t), rel=1e-12)
    assert rec[-1, 0, 2] == pytest.approx(np.mean(d), rel=1e-12, abs=1e-20)
    assert rec[-1, 0, 3] == pytest.approx(np.std(d), rel=1e-12)
    assert out[0] > 0 and hist.sum() + out[0] == 5001
    assert rec[-1, 0, 4] == hist.sum() and rec[-1, 0, 5] == out[0]
    dv = s.derived
    expect, _ = np.histogram(t, bins=256, range=(-dv["H"], dv["H"]))
    assert np.abs(expect - hist[0]).sum() <= 2   # numpy's edge rounding may move a boundary particle


# --------------------------------------------------------------------------- binning
def test_binning_brute_force(oracle_mod):
    s = _sim(oracle_mod, nbins=16, hw=5.0)
    H, Dl = s.derived["H"], s.derived["Delta"]
    assert Dl == 2 * H / 16
    e = 1e-3 * Dl
    taus = [-H,                    # lower edge, inside: bin 0
            -H - e, -2 * H,        # below: outside
            H + e, 3 * H,          # above: outside
            H - e,                 # just inside the top: bin 15
            -H + 0.5 * Dl,         # centre of bin 0
            -H + 3.5 * Dl,         # centre of bin 3
            -H + 3.0 * Dl + e,     # just above the 3|4... lower edge of bin 3
            -H + 4.0 * Dl - e,     # just below the top of bin 3
            -H + 4.0 * Dl + e,     # just above: bin 4
            0.0 + e,               # bin 8
            0.0 - e,               # bin 7
            -H + 15.25 * Dl,       # bin 15
            -H + 7.75 * Dl,        # bin 7
            float("nan"),          # not binnable: counted outside
            -H + 11.5 * Dl]        # bin 11
    hist, out = s.bin(taus)
    expect = np.zeros(16, np.int32)
    for k in (0, 15, 0, 3, 3, 3, 4, 8, 7, 15, 7, 11):
        expect[k] += 1
    assert out == 5
    assert np.array_equal(hist, expect)
    assert hist.sum() + out == len(taus)


# --------------------------------------------------------------------------- wakes
@pytest.mark.parametrize("res", [dict(Rs_ohm=5e3, fr_Hz=10e9, Q=1.0, range=1),
                                 dict(Rs_ohm=2e4, fr_Hz=3e9, Q=5.0, range=1),
                                 dict(Rs_ohm=1e5, fr_Hz=1e9, Q=20.0, range=1)])
def test_wake_is_the_resonator_impedance(oracle_mod, res):
    """int_0^inf W(t) e^{-i w t} dt = Rs / (1 + i Q (w/w_r - w_r/w)), and the
    zero-lag value is the loss factor w_r Rs / (2Q) (fundamental theorem of
    beam loading)."""
    wr = 2 * math.pi * res["fr_Hz"]
    a = wr / (2 * res["Q"])
    assert oracle_mod.wake(res, 0.0) == pytest.approx(wr * res["Rs_ohm"] / (2 * res["Q"]), rel=1e-14)
    assert oracle_mod.wake(res, -1e-12) == 0.0
    T = 60.0 / a
    n = 400001
    t = np.linspace(0.0, T, n)
    w = np.array([oracle_mod.wake(res, x) for x in t])
    w[0] = 2 * wr * res["Rs_ohm"] / (2 * res["Q"])  # W(0+)
    for omega in (0.5 * wr, wr, 1.7 * wr):
        f = w * np.exp(-1j * omega * t)
        h = t[1] - t[0]
        Z_num = h / 3 * (f[0] + f[-1] + 4 * f[1:-1:2].sum() + 2 * f[2:-1:2].sum())
        Z = res["Rs_ohm"] / (1 + 1j * res["Q"] * (omega / wr - wr / omega))
        assert abs(Z_num - Z) < 1e-6 * res["Rs_ohm"]


def test_short_range_voltage_is_causal_convolution(oracle_mod):
    bb = dict(W.BROADBAND)
    s = _sim(oracle_mod, res=[bb], nbins=64)
    Dl = s.derived["Delta"]
    q = 3.7e-14
    for k0 in (0, 17, 63):
        hist = np.zeros(64, np.int32)
        hist[k0] = 5
        V = s.vsr_direct(hist, q)
        for j in range(64):
            expect = 0.0 if j < k0 else 5 * q * oracle_mod.wake(bb, (j - k0) * Dl)
            assert V[j] == pytest.approx(expect, rel=1e-14, abs=1e-30)
    # superposition
    h1 = np.zeros(64, np.int32); h1[5] = 2
    h2 = np.zeros(64, np.int32); h2[30] = 7
    np.testing.assert_allclose(s.vsr_direct(h1 + h2, q), s.vsr_direct(h1, q) + s.vsr_direct(h2, q), rtol=1e-13, atol=1e-25)


@pytest.mark.parametrize("ngp", [False, True])
def test_kick_voltage_interpolates_between_cell_centres(oracle_mod, ngp):
    """The short-range voltage a particle is kicked with (Sec. 2.3): the cell
    voltages taken at the cell centres and interpolated linearly between them
    (numpy's interp, which holds the end values beyond the outermost
    centres), or the particle's own cell with the nearest-grid-point option;
    zero outside the mesh."""
    check_kick_interpolation(oracle_mod, ngp)


def check_kick_interpolation(oracle_mod, ngp, lib=None):
    bb = dict(W.BROADBAND)
    s = oracle_mod.OracleSim(W.ring_r0(), [bb], 32, 5.0, [0], [1e-3], [1000], 1,
                             oracle_mod.KICK_NGP if ngp else 0, lib=lib)
    rng = np.random.default_rng(9)
    s.feed_histograms(rng.integers(0, 60, size=(1, 32)).astype(np.int32))
    V = s.vsr()[0]
    assert np.max(np.abs(V)) > 0
    dv = s.derived
    H, D = dv["H"], dv["Delta"]
    centres = -H + (np.arange(32) + 0.5) * D
    taus = np.concatenate([centres, -H + (np.arange(33)) * D * (1 - 1e-12) + 1e-30,
                           rng.uniform(-H, H, 300)])
    for tau in taus:
        x = (tau + H) / D
        if ngp:
            expect = V[min(int(np.floor(x)), 31)]
        else:
            expect = np.interp(tau, centres, V)
        got = s.wake_voltage_at(0, float(tau))
        assert got == pytest.approx(expect, rel=1e-12, abs=1e-12 * np.max(np.abs(V))), tau
    for tau in (-H - 0.25 * D, -H - 3 * D, H + 1e-3 * D, H + 2 * D):
        assert s.wake_voltage_at(0, tau) == 0.0


@pytest.mark.parametrize("ngp", [False, True])
def test_transverse_kick_voltage_interpolates_between_cell_centres(oracle_mod, ngp):
    """The transverse short-range voltage a particle is kicked with (Eq. 6,
    second line): as the longitudinal one, the cell voltages at the cell
    centres interpolated linearly (numpy's interp, end values held), or the
    particle's own cell with the nearest-grid-point option; zero outside the
    mesh.  The cell voltages come from a tracked turn of offset particles, so
    that the voltage a turn builds is the one the check evaluates."""
    check_transverse_kick_interpolation(oracle_mod, ngp)


def check_transverse_kick_interpolation(oracle_mod, ngp, lib=None):
    nb, n = 32, 2000
    s = oracle_mod.OracleSim(W.ring_r0(), [], nb, 5.0, [0], [2e-3], [n], 3,
                             (oracle_mod.KICK_NGP if ngp else 0) | W.NO_QE, lib=lib,
                             transverse=_tplane(resonators=[dict(TRES, range=W.RANGE_SHORT)]))
    rng = np.random.default_rng(21)
    dv = s.derived
    H, D = dv["H"], dv["Delta"]
    s.set_particles(0, rng.normal(0.0, 0.4 * H, n), rng.normal(0.0, 9e-4, n))
    s.set_tparticles(0, rng.normal(2e-4, 1e-4, n), np.zeros(n))
    s.track(1, record=False)
    V = s.vt()[0]
    assert np.max(np.abs(V)) > 0 and np.count_nonzero(V) > nb // 2
    centres = -H + (np.arange(nb) + 0.5) * D
    taus = np.concatenate([centres, -H + (np.arange(nb + 1)) * D * (1 - 1e-12) + 1e-30,
                           rng.uniform(-H, H, 300)])
    for tau in taus:
        x = (tau + H) / D
        expect = V[min(int(np.floor(x)), nb - 1)] if ngp else np.interp(tau, centres, V)
        got = s.tvoltage_at(0, float(tau))
        assert got == pytest.approx(expect, rel=1e-12, abs=1e-12 * np.max(np.abs(V))), tau
    for tau in (-H - 0.25 * D, -H - 3 * D, H + 1e-3 * D, H + 2 * D):
        assert s.tvoltage_at(0, tau) == 0.0


def test_dipole_deposit_brute_force(oracle_mod):
    """The dipole sums of the transverse wake (Eq. 6, second line): every
    particle's offset lands in the cell binning gives it (hand-placed at
    edges, centres and outside, as in the binning check), nothing outside;
    and a tracked turn's sums are exactly this deposit of its particles."""
    check_dipole_deposit(oracle_mod)


def check_dipole_deposit(oracle_mod, lib=None):
    s = oracle_mod.OracleSim(W.ring_r0(), [], 16, 5.0, [0], [1e-3], [64], 5, W.NO_QE, lib=lib,
                             transverse=_tplane(resonators=[dict(TRES, range=W.RANGE_SHORT)]))
    H, Dl = s.derived["H"], s.derived["Delta"]
    e = 1e-3 * Dl
    placed = [(-H, 0), (-H - e, None), (-2 * H, None), (H + e, None), (3 * H, None), (H - e, 15),
              (-H + 0.5 * Dl, 0), (-H + 3.5 * Dl, 3), (-H + 3.0 * Dl + e, 3), (-H + 4.0 * Dl - e, 3),
              (-H + 4.0 * Dl + e, 4), (e, 8), (-e, 7), (-H + 15.25 * Dl, 15), (-H + 7.75 * Dl, 7),
              (float("nan"), None), (-H + 11.5 * Dl, 11)]
    taus = np.array([t for t, _ in placed])
    xs = 1e-4 * (1.0 + np.arange(len(placed))) * (-1.0) ** np.arange(len(placed))
    hist, dip, out = s.deposit(taus, xs)
    expect_h = np.zeros(16, np.int32)
    expect_d = np.zeros(16)
    for (t, k), x in zip(placed, xs):
        if k is not None:
            expect_h[k] += 1
            expect_d[k] += x
    assert out == sum(k is None for _, k in placed)
    assert np.array_equal(hist, expect_h)
    assert np.array_equal(dip, expect_d)
    # a tracked turn deposits its particles the same way
    rng = np.random.default_rng(4)
    s.set_particles(0, rng.normal(0.0, 0.5 * H, 64), rng.normal(0.0, 9e-4, 64))
    s.set_tparticles(0, rng.normal(0.0, 1e-4, 64), rng.normal(0.0, 1e-5, 64))
    s.track(1, record=False)
    t1, _ = s.particles(0)
    x1, _ = s.tparticles(0)
    h1, d1, _ = s.deposit(t1, x1)
    assert np.array_equal(d1, s.dipoles()[0]) and np.array_equal(h1, s.histograms()[0][0])


# Mutants: the source of the oracle with one planted mistake each, compiled
# on the CPU; the check named beside each must fail on it (so that a
# half-cell shift or a wrong cell cannot hide behind the pins).
MUTANTS = [
    ("longitudinal kick half a cell off", "double u = x - 0.5;", "double u = x;",
     lambda o, lib: check_kick_interpolation(o, False, lib)),
    ("transverse kick half a cell off", "double u = xc - 0.5;", "double u = xc;",
     lambda o, lib: check_transverse_kick_interpolation(o, False, lib)),
    ("transverse NGP kick from the next cell", "return V[(int)floor(xc)];",
     "return V[(int)floor(xc) + 1 < nb ? (int)floor(xc) + 1 : nb - 1];",
     lambda o, lib: check_transverse_kick_interpolation(o, True, lib)),
    ("dipole deposit into the cell below", "dip[(int)xc] += x;", "dip[(int)xc > 0 ? (int)xc - 1 : 0] += x;",
     lambda o, lib: check_dipole_deposit(o, lib)),
]


@pytest.mark.parametrize("name,old,new,check", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_fail_on_planted_mistakes(oracle_mod, tmp_path, name, old, new, check):
    src = open(os.path.join(ROOT, "oracle", "mbt_oracle.c")).read()
    assert src.count(old) == 1, name
    mutant = tmp_path / "mutant.c"
    mutant.write_text(src.replace(old, new))
    lib = oracle_mod.load_library(oracle_mod.compile_source(mutant, tmp_path / "libmutant.so"))
    with pytest.raises(AssertionError):
        check(oracle_mod, lib)


def test_long_range_is_the_wake_of_every_earlier_passage(oracle_mod):
    """After feeding histograms for a few turns, the long-range voltage at a
    particle equals the sum over earlier passages of q * count * W(dt + tau -
    tau_k), evaluated with the wake function itself."""
    hom = dict(Rs_ohm=1e6, fr_Hz=1.5e9, Q=300.0, range=W.RANGE_LONG)
    buckets = [0, 3, 10]
    cur = [1e-3, 2e-3, 0.5e-3]
    nmp = [1000, 1000, 1000]
    s = _sim(oracle_mod, res=[hom], buckets=buckets, currents=cur, n_mp=nmp, nbins=32)
    dv = s.derived
    ring = W.ring_r0()
    T0 = ring["T0_s"]
    Trf = T0 / ring["h"]
    rng = np.random.default_rng(5)
    hists = []
    for turn in range(6):
        hh = rng.integers(0, 40, size=(3, 32)).astype(np.int32)
        s.feed_histograms(hh)
        hists.append(hh)
    q = [c * T0 / n for c, n in zip(cur, nmp)]
    tk = -dv["H"] + (np.arange(32) + 0.5) * dv["Delta"]
    n_now = 5
    for m in range(3):
        for tau in (-3e-11, 0.0, 2.2e-11):
            v = 0.0
            for n_p, hh in enumerate(hists):
                for mp in range(3):
                    Dbk = (n_now - n_p) * ring["h"] + buckets[m] - buckets[mp]
                    if Dbk <= 0:
                        continue
                    for k in range(32):
                        if hh[mp, k]:
                            v += q[mp] * hh[mp, k] * oracle_mod.wake(hom, Dbk * Trf + tau - tk[k])
            got = s.wake_voltage_at(m, tau)
            assert got == pytest.approx(v, rel=1e-9)


def test_long_range_single_bunch_geometric_series(oracle_mod):
    """A frozen single bunch seen through a narrow resonator: the amplitude from
    all earlier turns sums to E e^{sT0} / (1 - e^{sT0})."""
    hom = dict(Rs_ohm=1e6, fr_Hz=1.5e9, Q=2e4, range=W.RANGE_LONG)
    s = _sim(oracle_mod, res=[hom], currents=(1e-3,), n_mp=(1000,), nbins=32)
    nh = int(s.derived["nhist"])
    hist = np.zeros((1, 32), np.int32)
    hist[0, 12] = 600
    hist[0, 20] = 400
    for _ in range(nh + 5):
        s.feed_histograms(hist)
    E = s.last_emission(0)[0]
    wr = 2 * math.pi * hom["fr_Hz"]
    a = wr / (2 * hom["Q"])
    sc = -a + 1j * math.sqrt(wr * wr - a * a)
    z = np.exp(sc * W.ring_r0()["T0_s"])
    A = s.alr()[0, 0]
    assert abs(A - E * z / (1 - z)) < 1e-9 * abs(E * z / (1 - z))


# --------------------------------------------------------------------------- collective physics
def _haissinski(ring, res, I, nbins_fine=4001, L=10.0):
    """Potential-well equilibrium of a bunch in the RF + short-range wake, by
    fixed-point iteration of lambda ~ exp(-U / (alpha_c T0 sigma_E^2))."""
    E0, T0, h, V, ac = ring["E0_eV"], ring["T0_s"], ring["h"], ring["V_rf_V"], ring["alpha_c"]
    sd = ring["sigma_delta"]
    phis = math.asin(ring["U0_eV"] / V)
    w = 2 * math.pi * h / T0
    nus = textbook_nu_s(ring)
    st0 = ac * sd * T0 / (2 * math.pi * nus)
    tau = np.linspace(-L * st0, L * st0, nbins_fine)
    dt = tau[1] - tau[0]
    wr = 2 * math.pi * res["fr_Hz"]
    a = wr / (2 * res["Q"])
    wb = math.sqrt(wr * wr - a * a)
    lag = tau - tau[0]
    Wl = 2 * a * res["Rs_ohm"] * np.exp(-a * lag) * (np.cos(wb * lag) - (a / wb) * np.sin(wb * lag))
    Wl[0] *= 0.5
    Urf = -(V / E0) * ((np.cos(phis - w * tau) - math.cos(phis)) / w - math.sin(phis) * tau)
    lam = np.exp(-tau ** 2 / (2 * st0 ** 2))
    lam /= lam.sum() * dt
    for _ in range(5000):
        Vw = I * T0 * np.convolve(lam, Wl)[:nbins_fine] * dt
        Uw = np.concatenate([[0.0], np.cumsum(0.5 * (Vw[1:] + Vw[:-1]) * dt)]) / E0
        U = Urf + Uw
        new = np.exp(-(U - U.min()) / (ac * T0 * sd * sd))
        new /= new.sum() * dt
        if np.max(np.abs(new - lam)) < 1e-13 * np.max(lam):
            lam = new
            break
        lam = 0.5 * lam + 0.5 * new
    return tau, lam, st0


def test_haissinski_equilibrium_is_stationary(oracle_mod):
    """A bunch seeded from the Haissinski solution of the broadband wake stays
    there: centroid shift, length and profile after 600 turns match it, and
    differ clearly from the zero-current Gaussian."""
    ring = W.ring_r0()
    bb = dict(W.BROADBAND)
    I = 1e-3
    tau, lam, st0 = _haissinski(ring, bb, I)
    dt = tau[1] - tau[0]
    mean_h = np.sum(tau * lam) * dt
    sig_h = math.sqrt(np.sum((tau - mean_h) ** 2 * lam) * dt)
    assert mean_h / st0 < -0.4 and sig_h / st0 > 1.03   # a strong distortion
    N = 20000
    rng = np.random.default_rng(11)
    cdf = np.cumsum(lam) * dt
    cdf /= cdf[-1]
    t0 = np.interp(rng.random(N), cdf, tau)
    d0 = rng.normal(0.0, ring["sigma_delta"], N)
    s = _sim(oracle_mod, ring=ring, res=[bb], currents=(I,), n_mp=(N,), nbins=256, hw=5.0)
    s.set_particles(0, t0, d0)
    rec = s.track(600)
    m_tr = rec[200:, 0, 0].mean()
    s_tr = rec[200:, 0, 1].mean()
    assert abs(m_tr - mean_h) < 0.03 * st0
    assert abs(s_tr - sig_h) < 0.012 * st0
    # profile: the tracked histogram is close to Haissinski, far from the Gaussian
    hist, out = s.histograms()
    dv = s.derived
    edges = -dv["H"] + np.arange(257) * dv["Delta"]
    ph = np.diff(np.interp(edges, tau, np.cumsum(lam) * dt))
    g = stats.norm.cdf(edges / st0)
    pg = np.diff(g)
    emp = hist[0] / N
    d_h = np.sqrt(np.sum((emp - ph) ** 2))
    d_g = np.sqrt(np.sum((emp - pg) ** 2))
    assert d_h < 0.35 * d_g


def _coupled_bunch_run(oracle_mod, M, fr, Rs, I_bunch, turns, Q=2e4, amp=5e-12):
    """Point-like bunches (sigma_tau 3 ps) in M equally spaced buckets, no
    radiation, a narrow long-range resonator.  Returns the mode amplitudes
    X_mu(n) = sum_m z_m(n) e^{-2 pi i mu m / M} of the normal-form centroids."""
    ring = W.ring_r0()
    h = ring["h"]
    T0 = ring["T0_s"]
    nus = textbook_nu_s(ring, sr=False)
    nu = math.acos(1 - (2 * math.pi * nus) ** 2 / 2) / (2 * math.pi)
    ac = ring["alpha_c"]
    buckets = [m * (h // M) for m in range(M)]
    hom = dict(Rs_ohm=Rs, fr_Hz=fr, Q=Q, range=W.RANGE_LONG)
    N = 400
    s = _sim(oracle_mod, ring=ring, res=[hom], buckets=buckets, currents=[I_bunch] * M, n_mp=[N] * M,
             flags=W.NO_SR, nbins=256, hw=5.0)
    rng = np.random.default_rng(3)
    st = 3e-12
    sdl = st * 2 * math.pi * nu / (ac * T0)
    for m in range(M):
        ph = rng.uniform(0, 2 * math.pi)
        s.set_particles(m, rng.normal(amp * math.cos(ph), st, N), rng.normal(amp * math.sin(ph) * sdl / st, sdl, N))
    rec = s.track(turns)
    # normal-form coordinate: the left eigenvector of the linear one-turn map
    # for the eigenvalue e^{+i 2 pi nu}, so that free motion is z -> z e^{+i 2 pi nu}
    w_rf = 2 * math.pi * h / T0
    K = (ring["V_rf_V"] / ring["E0_eV"]) * w_rf
    a = ac * T0
    M0 = np.array([[1 - a * K, a], [-K, 1.0]])
    ev, vl = np.linalg.eig(M0.T)
    wl = vl[:, int(np.argmax(ev.imag))]
    z = wl[0] * rec[:, :, 0] + wl[1] * rec[:, :, 2]
    X = np.stack([(z * np.exp(-2j * math.pi * mu * np.arange(M) / M)[None, :]).sum(axis=1) for mu in range(M)])
    return X, nu


def _rate(X, lo, hi):
    n = np.arange(lo, hi)
    return np.polyfit(n, np.log(np.abs(X[lo:hi])), 1)[0] / W.ring_r0()["T0_s"]


def _eq7(M, mu, fr, Rs, Q, I_bunch, nu):
    """Eq. 7 with omega_r in the numerator, summed over the positive-frequency
    upper (q M + mu) w0 + w_s and lower (q' M - mu) w0 - w_s lines."""
    ring = W.ring_r0()
    T0 = ring["T0_s"]
    w0 = 2 * math.pi / T0
    ws = nu * w0
    wr = 2 * math.pi * fr

    def ReZ(w):
        return (Rs / (1 + 1j * Q * (w / wr - wr / w))).real

    p0 = int(round(wr / w0 / M))
    up = sum(ReZ((q * M + mu) * w0 + ws) for q in range(max(0, p0 - 50), p0 + 50) if (q * M + mu) * w0 + ws > 0)
    lo = sum(ReZ((q * M - mu) * w0 - ws) for q in range(max(0, p0 - 50), p0 + 50) if (q * M - mu) * w0 - ws > 0)
    I_tot = M * I_bunch
    return ring["alpha_c"] * I_tot * wr / (2 * ring["E0_eV"] * T0 * ws) * (up - lo)


@pytest.mark.parametrize("side", [+1, -1], ids=["upper-sideband-grows", "lower-sideband-damps"])
def test_single_bunch_resonator_sideband_eq7(oracle_mod, side):
    """One bunch coupled to itself over turns by a narrow HOM on a synchrotron
    sideband of revolution line 1441: Eq. 7 with M = 1 gives the rate and its sign.
    Q = 1e6 keeps the resonance (1.5 kHz wide) on one sideband only, so the
    first-order rate is not a small difference of the two sidebands."""
    ring = W.ring_r0()
    f0 = 1.0 / ring["T0_s"]
    nus = textbook_nu_s(ring, sr=False)
    nu = math.acos(1 - (2 * math.pi * nus) ** 2 / 2) / (2 * math.pi)
    fr = (1441 + side * nu) * f0
    Rs, I, Q = 1e6, 1e-3, 1e6
    X, nu = _coupled_bunch_run(oracle_mod, 1, fr, Rs, I, 3000, Q=Q)
    pred = _eq7(1, 0, fr, Rs, Q, I, nu)
    assert np.sign(pred) == side
    assert _rate(X[0], 1000, 3000) == pytest.approx(pred, rel=0.02)


def test_four_bunch_mode_eq7(oracle_mod):
    """Four equally spaced bunches, HOM on the upper sideband of line 1441 =
    360*4 + 1: coupled-bunch mode 1 grows, mode 3 damps, at the Eq. 7 rates;
    modes 0 and 2 see no resistive impedance."""
    ring = W.ring_r0()
    f0 = 1.0 / ring["T0_s"]
    nus = textbook_nu_s(ring, sr=False)
    nu = math.acos(1 - (2 * math.pi * nus) ** 2 / 2) / (2 * math.pi)
    fr = (1441 + nu) * f0
    Rs, I = 1e7, 1e-3
    X, nu = _coupled_bunch_run(oracle_mod, 4, fr, Rs, I, 2000)
    pred = [_eq7(4, mu, fr, Rs, 2e4, I, nu) for mu in range(4)]
    assert pred[1] > 1000 and pred[3] < -1000
    assert _rate(X[1], 1000, 2000) == pytest.approx(pred[1], rel=0.02)
    # the damped mode is fitted while it still dominates its projection
    assert _rate(X[3], 0, 600) == pytest.approx(pred[3], rel=0.05)
    assert abs(_rate(X[0], 1000, 2000)) < 0.1 * pred[1]
    assert abs(_rate(X[2], 1000, 2000)) < 0.1 * pred[1]


# ----------------------------------------------------------------------------- tabulated wakes, resistive wall
RW = dict(radius_m=0.01, conductivity_S_per_m=5.8e7, length_m=290.4)   # copper, 10 mm, the dc12c circumference


def _rw_consts():
    b, sig, L = RW["radius_m"], RW["conductivity_S_per_m"], RW["length_m"]
    Z0, c = 376.730313668, 299792458.0
    s0 = (2 * b * b / (Z0 * sig)) ** (1 / 3)
    tail = c * L / (4 * math.pi * b) * math.sqrt(Z0 / (math.pi * sig))   # W ~ -tail (c t)^(-3/2)
    return b, sig, L, Z0, c, s0, tail


def test_resistive_wall_head_value(oracle_mod):
    """W(0+) = Z0 c L / (pi b^2), independent of the conductivity."""
    b, sig, L, Z0, c, s0, tail = _rw_consts()
    w0 = oracle_mod.resistive_wall_wake([0.0], b, sig, L)[0]
    assert w0 == pytest.approx(Z0 * c * L / (math.pi * b * b), rel=1e-9)
    w0b = oracle_mod.resistive_wall_wake([0.0], b, 10 * sig, L)[0]
    assert w0b == pytest.approx(w0, rel=1e-9)


def test_resistive_wall_long_range_tail(oracle_mod):
    """Far behind the head (s >> s0) the classic resistive-wall wake
    W = -(c L / (4 pi b)) sqrt(Z0 / (pi sigma)) s^(-3/2)."""
    b, sig, L, Z0, c, s0, tail = _rw_consts()
    for u in (50.0, 200.0):
        t = u * s0 / c
        w = oracle_mod.resistive_wall_wake([t], b, sig, L)[0]
        assert w == pytest.approx(-tail * (c * t) ** -1.5, rel=2e-4)


def test_resistive_wall_wake_integrates_to_zero(oracle_mod):
    """A resistive wall has no impedance at zero frequency, so the wake
    integrates to zero: the integral up to T equals minus the tail beyond T."""
    b, sig, L, Z0, c, s0, tail = _rw_consts()
    T = 500 * s0 / c
    t, w = oracle_mod.resistive_wall_table(b, sig, L, T)
    head = np.trapezoid(w, t)
    beyond = -tail * 2.0 * (c * T) ** -0.5 / c     # integral of -tail (c t)^(-3/2) dt from T to infinity
    scale = np.trapezoid(np.abs(w), t)
    assert abs(head + beyond) < 2e-4 * scale


def test_wake_table_cell_averages_are_exact_for_a_linear_wake(oracle_mod):
    """A linear table A + B t on [0, T]: lag l >= 1 gets its cell average, lag 0
    the integral over the half cell / Delta, lags past T nothing."""
    s = _sim(oracle_mod, nbins=64)
    D = s.derived["Delta"]
    A, B, T = 3.0e12, -2.0e23, 20.5 * D
    t = np.linspace(0.0, T, 7)
    s2 = _sim(oracle_mod, nbins=64)
    base = s2.wlag()
    s3 = oracle_mod.OracleSim(W.ring_r0(), [], 64, 5.0, [0], [0.0], [2], 1, 0, wake_tables=[(t, A + B * t)])
    got = s3.wlag() - base
    for l in range(64):
        lo, hi = (0.0 if l == 0 else (l - 0.5) * D), min((l + 0.5) * D, T)
        exact = 0.0 if hi <= lo else (A * (hi - lo) + 0.5 * B * (hi * hi - lo * lo)) / D
        assert got[l] == pytest.approx(exact, rel=1e-12, abs=1e-3)
    assert got[0] == pytest.approx(A / 2 + B * D / 8, rel=1e-12)
    assert np.all(got[21:] == 0.0)


def test_wake_table_of_a_resonator_differs_by_the_cell_curvature(oracle_mod):
    """The broadband resonator given as a fine table: cell averages differ from
    the resonator's point samples by (Delta^2 / 24) W''(l Delta) (lag 0: W'(0)
    Delta / 8 + W''(0) Delta^2 / 48), to fourth order."""
    res = dict(W.BROADBAND)
    s = _sim(oracle_mod, res=[res], nbins=256)
    point = s.wlag()
    D = s.derived["Delta"]
    wr = 2 * math.pi * res["fr_Hz"]
    a = wr / (2 * res["Q"])
    wb = math.sqrt(wr * wr - a * a)
    Rs = res["Rs_ohm"]
    tt = np.linspace(0.0, 258 * D, 258 * 400 + 1)
    Wt = 2 * a * Rs * np.exp(-a * tt) * (np.cos(wb * tt) - (a / wb) * np.sin(wb * tt))
    tab = oracle_mod.OracleSim(W.ring_r0(), [], 256, 5.0, [0], [0.0], [2], 1, 0, wake_tables=[(tt, Wt)]).wlag()
    # derivatives of W(t) = Re(C e^{s t}), s = -a + i wb, C = 2 a Rs (1 + i a / wb)
    sc = complex(-a, wb)
    C = 2 * a * Rs * complex(1.0, a / wb)
    l = np.arange(1, 256)
    w2 = (C * sc * sc * np.exp(sc * l * D)).real
    assert np.max(np.abs(tab[1:] - point[1:] - D * D / 24 * w2)) < 1e-3 * np.max(np.abs(point))
    w1_0, w2_0 = (C * sc).real, (C * sc * sc).real
    assert tab[0] - point[0] == pytest.approx(w1_0 * D / 8 + w2_0 * D * D / 48, rel=2e-2)


# ----------------------------------------------------------------------------- harmonic cavities
from physics_helpers import double_rf_equilibrium as _double_rf_equilibrium  # noqa: E402
from physics_helpers import flat_potential as _flat_potential  # noqa: E402


def test_flat_potential_phase_and_cubic_energy_change(oracle_mod):
    ring = W.ring_r0()
    hc, sphi, cphi, k = _flat_potential(ring)
    dv = oracle_mod.derive_h(ring, [hc])
    assert dv["sin_phi_s"] == pytest.approx(sphi, rel=1e-12)
    # one turn of particles at rest at small offsets (no wake, no excitation)
    taus = np.array([-4, -3, -2, -1, 0, 1, 2, 3, 4], float) * 1e-12
    s = oracle_mod.OracleSim(ring, [], 64, 5.0, [0], [0.0], [len(taus)], 1, W.NO_QE, harmonic_cavities=[hc])
    s.set_particles(0, taus, np.zeros_like(taus))
    s.track(1, record=False)
    _, d1 = s.particles(0)
    D = 2 * ring["T0_s"] / ring["tau_z_s"]
    w = 2 * math.pi * ring["h"] / ring["T0_s"]
    VoE = ring["V_rf_V"] / ring["E0_eV"]
    assert abs(d1[4]) < 1e-18                  # the synchronous particle gains nothing
    c = np.polyfit(taus / 1e-12, d1 / (1 - D), 5)[::-1]   # c[j]: coefficient of (tau / 1 ps)^j
    K = VoE * w * cphi * 1e-12                 # main cavity alone: first-order change per ps
    assert abs(c[1]) < 1e-7 * K and abs(c[2]) < 1e-7 * K
    assert c[3] == pytest.approx(VoE * w ** 3 * cphi * (1 - 9) / 6 * 1e-36, rel=1e-3)


def test_flat_potential_equilibrium_is_stationary(oracle_mod):
    """Particles drawn from the analytic double-RF equilibrium stay in it (rms
    length within 2.5 % over 2000 turns after 1000), which is far from the
    single-cavity length."""
    ring = W.ring_r0()
    hc = _flat_potential(ring)[0]
    st0 = oracle_mod.derive(ring)["sigma_tau0"]
    tau, lam = _double_rf_equilibrium(ring, [hc], 12 * st0)
    mean = np.trapezoid(tau * lam, tau)
    sig = math.sqrt(np.trapezoid((tau - mean) ** 2 * lam, tau))
    assert sig > 1.8 * st0                       # strongly lengthened
    N = 6000
    g = np.random.default_rng(17)
    cdf = np.cumsum(lam)
    cdf /= cdf[-1]
    t0 = np.interp(g.random(N), cdf, tau)
    d0 = g.normal(0.0, ring["sigma_delta"], N)
    s = oracle_mod.OracleSim(ring, [], 256, 12.0, [0], [0.0], [N], 3, 0, harmonic_cavities=[hc])
    s.set_particles(0, t0, d0)
    rec = s.track(3000)
    assert rec[1000:, 0, 1].mean() == pytest.approx(sig, rel=0.025)
    assert abs(rec[1000:, 0, 0].mean() - mean) < 0.03 * sig


# ----------------------------------------------------------------------------- transverse plane
TRES = dict(Rs_ohm=2e5, fr_Hz=1.5e9, Q=2e4, range=W.RANGE_BOTH)   # Ohm/m


def _tplane(**kw):
    t = dict(beta_m=10.0, alpha=0.0, tune=0.3, chromaticity=0.0, emittance_m=1e-9, resonators=[], resistive_wall=[])
    t.update(kw)
    return t


def test_transverse_wake_transforms_to_resonator_impedance(oracle_mod):
    """i int W(t) e^{-i w t} dt = (wr/w) Rs / (1 + i Q (w/wr - wr/w)) for a
    low-Q transverse resonator, at three frequencies."""
    res = dict(Rs_ohm=1e6, fr_Hz=2e9, Q=3.0, range=W.RANGE_SHORT)
    wr = 2 * math.pi * res["fr_Hz"]
    t = np.linspace(0.0, 60e-9 * 3 / 2e9 * 1e9 / 60 * 40, 400001)
    w_t = np.array([oracle_mod.twake(res, ti) for ti in t])
    for f in (0.5, 1.0, 1.7):
        w = f * wr
        z = 1j * np.trapezoid(w_t * np.exp(-1j * w * t), t)
        ref = (wr / w) * res["Rs_ohm"] / (1 + 1j * res["Q"] * (w / wr - wr / w))
        assert abs(z - ref) < 2e-4 * abs(ref)
    assert oracle_mod.twake(res, 0.0) == 0.0 and oracle_mod.twake(res, -1e-12) == 0.0


def test_transverse_short_range_is_causal_and_linear(oracle_mod):
    s = oracle_mod.OracleSim(W.ring_r0(), [], 128, 5.0, [0], [1e-3], [4], 1, 0,
                             transverse=_tplane(resonators=[dict(TRES, range=W.RANGE_SHORT)]))
    D = s.derived["Delta"]
    dip = np.zeros(128)
    dip[40] = 3e-4
    v = s.vt_direct(dip, 2e-12)
    lags = np.arange(128) - 40
    ref = np.array([2e-12 * 3e-4 * oracle_mod.twake(dict(TRES), l * D) if l > 0 else 0.0 for l in lags])
    assert np.allclose(v, ref, rtol=1e-12, atol=0.0)
    dip2 = dip.copy()
    dip2[70] = -1e-4
    v2 = s.vt_direct(dip2, 2e-12)
    one = np.zeros(128)
    one[70] = -1e-4
    assert np.allclose(v2, v + s.vt_direct(one, 2e-12), rtol=1e-12, atol=1e-30)


@pytest.mark.parametrize("alpha,xi,d0", [(0.0, 0.0, 0.0), (0.7, 0.0, 0.0), (0.0, 2.5, 1e-3), (-0.4, -1.5, -2e-3)])
def test_betatron_map_is_the_twiss_rotation(oracle_mod, alpha, xi, d0):
    """One turn of particles at tau = 0 (no radiation: delta stays) maps (x,
    x') by the Twiss matrix of phase 2 pi nu0 (1 + xi delta): det 1, the
    elements of Eq. 4."""
    beta, nu = 12.0, 0.27
    s = oracle_mod.OracleSim(W.ring_r0(), [], 64, 5.0, [0], [0.0], [4], 1, W.NO_SR,
                             transverse=_tplane(beta_m=beta, alpha=alpha, tune=nu, chromaticity=xi))
    s.set_particles(0, np.zeros(4), np.full(4, d0))
    s.set_tparticles(0, np.array([1e-4, 0.0, 0.0, 0.0]), np.array([0.0, 1e-5, 0.0, 0.0]))
    s.track(1, record=False)
    x, xp = s.tparticles(0)
    M = np.array([[x[0] / 1e-4, x[1] / 1e-5], [xp[0] / 1e-4, xp[1] / 1e-5]])
    psi = 2 * math.pi * nu * (1 + xi * d0)
    g = (1 + alpha * alpha) / beta
    ref = np.array([[math.cos(psi) + alpha * math.sin(psi), beta * math.sin(psi)],
                    [-g * math.sin(psi), math.cos(psi) - alpha * math.sin(psi)]])
    assert np.allclose(M, ref, rtol=0, atol=1e-12)
    assert np.linalg.det(M) == pytest.approx(1.0, abs=1e-12)


def test_transverse_radiation_damping_rate(oracle_mod):
    """A coherent betatron oscillation damps through the momentum ratio across
    the cavity at the rate U0 / (2 E0 T0) (J_x = 1), without excitation."""
    ring = W.ring_r0()
    s = oracle_mod.OracleSim(ring, [], 64, 5.0, [0], [0.0], [400], 2, W.NO_QE, transverse=_tplane())
    s.init_particles()
    x, xp = s.tparticles(0)
    s.set_tparticles(0, x + 5e-4, xp)
    _, trec = s.track2(3000)
    beta = 10.0
    z = trec[:, 0, 0] / math.sqrt(beta) - 1j * math.sqrt(beta) * trec[:, 0, 2]
    n = np.arange(3000)
    rate = np.polyfit(n, np.log(np.abs(z)), 1)[0] / ring["T0_s"]
    assert rate == pytest.approx(-ring["U0_eV"] / (2 * ring["E0_eV"] * ring["T0_s"]), rel=0.02)


def test_transverse_equilibrium_emittance_is_kept(oracle_mod):
    """From the matched start the emittance stays at its equilibrium value
    (damping through the cavity balanced by the excitation of Eq. 5)."""
    ring = W.ring_r0()
    emit = 2e-9
    s = oracle_mod.OracleSim(ring, [], 64, 5.0, [0], [0.0], [4000], 3, 0,
                             transverse=_tplane(emittance_m=emit, alpha=0.3, beta_m=8.0))
    s.init_particles()
    _, trec = s.track2(3000)
    g = (1 + 0.09) / 8.0
    assert np.mean(trec[1000:, 0, 1] ** 2) == pytest.approx(8.0 * emit, rel=0.04)
    assert np.mean(trec[1000:, 0, 3] ** 2) == pytest.approx(g * emit, rel=0.04)


def test_transverse_coupled_bunch_growth_rate(oracle_mod):
    """Four point-like bunches, a narrow long-range transverse resonator on
    the negative-frequency line of mode 3: the mode grows at
    -(I_b M beta / (2 E0 T0)) sum_p Re Z((pM + mu) w0 + w_beta), the result of
    the turn-by-turn kick model summed over lines (Poisson summation)."""
    ring = W.ring_r0()
    T0, h = ring["T0_s"], ring["h"]
    M, nu, beta, Ib, Rs, Q = 4, 0.3, 20.0, 5e-3, 1.2e7, 2e4
    w0 = 2 * math.pi / T0
    fr = (1441 - nu) / T0
    tres = dict(Rs_ohm=Rs, fr_Hz=fr, Q=Q, range=W.RANGE_LONG)
    buckets = [m * (h // M) for m in range(M)]
    n_mp, turns = 200, 3000
    s = oracle_mod.OracleSim(ring, [], 64, 5.0, buckets, [Ib] * M, [n_mp] * M, 4, W.NO_SR,
                             transverse=_tplane(beta_m=beta, tune=nu, resonators=[tres]))
    g = np.random.default_rng(8)
    for m in range(M):
        s.set_particles(m, g.normal(0, 3e-12, n_mp), np.zeros(n_mp))
        ph = g.uniform(0, 2 * math.pi)
        s.set_tparticles(m, np.full(n_mp, 1e-6 * math.cos(ph)), np.full(n_mp, -1e-6 / beta * math.sin(ph)))
    _, trec = s.track2(turns)
    z = trec[:, :, 0] / math.sqrt(beta) - 1j * math.sqrt(beta) * trec[:, :, 2]
    # mode mu: phase (2 pi nu + 2 pi mu) / M from one bunch to the next
    th = (2 * math.pi * nu + 2 * math.pi * 3) / M
    X3 = (z * np.exp(-1j * th * np.arange(M))[None, :]).sum(axis=1)
    rate = np.polyfit(np.arange(1000, turns), np.log(np.abs(X3[1000:])), 1)[0] / T0
    wr = 2 * math.pi * fr

    def re_z(w):
        return ((wr / w) * Rs / (1 + 1j * Q * (w / wr - wr / w))).real

    p = np.arange(-2000, 2000)
    lines = (p * M + 3) * w0 + nu * w0
    pred = -(Ib * M * beta / (2 * ring["E0_eV"] * T0)) * np.sum(re_z(lines[lines != 0]))
    assert pred > 500
    assert rate == pytest.approx(pred, rel=0.02)


def test_transverse_rw_wake_is_the_integral_of_the_longitudinal_one(oracle_mod):
    """Round pipe: Z_x = (2c / (b^2 w)) Z_parallel, i.e. W_x(t) = (2c/b^2) int_0^t
    W_parallel; far behind the head the transverse resistive-wall wake equals
    that integral of the (pinned) longitudinal Bane-Sands wake."""
    b, sig, L, Z0, c, s0, tail = _rw_consts()
    s = oracle_mod.OracleSim(W.ring_r0(), [], 64, 5.0, [0], [0.0], [4], 1, 0,
                             transverse=_tplane(resistive_wall=[dict(radius_m=b, conductivity_S_per_m=sig,
                                                                     length_m=L, history_turns=2)]))
    for u in (2000.0, 8000.0):
        T = u * s0 / c
        t, w = oracle_mod.resistive_wall_table(b, sig, L, T)
        integral = np.trapezoid(w, t)
        assert s.transverse_rw_wake(T) == pytest.approx(2 * c / (b * b) * integral, rel=2e-3)


def test_transverse_rw_kicks_follow_the_centroid_history(oracle_mod):
    """A single offset bunch at integer tune (x frozen, no radiation, no other
    wake): x' grows turn by turn by (Q X0 / E0) sum_k W(k T0) over its earlier
    passages within the history, W(t) = (cL/(pi b^3)) sqrt(Z0/(pi sigma)) / sqrt(c t)."""
    ring = W.ring_r0()
    T0 = ring["T0_s"]
    b, sig, L, nh = 0.01, 5.8e7, 290.4, 3
    Z0, c = 376.730313668, 299792458.0
    A = c * L / (math.pi * b ** 3) * math.sqrt(Z0 / (math.pi * sig)) / math.sqrt(c)
    I, N, X0 = 2e-3, 8, 1e-4
    tp = _tplane(tune=1.0, emittance_m=0.0,
                 resistive_wall=[dict(radius_m=b, conductivity_S_per_m=sig, length_m=L, history_turns=nh)])
    s = oracle_mod.OracleSim(ring, [], 64, 5.0, [0], [I], [N], 1, W.NO_SR, transverse=tp)
    s.set_particles(0, np.zeros(N), np.zeros(N))
    s.set_tparticles(0, np.full(N, X0), np.zeros(N))
    turns = 7
    _, trec = s.track2(turns)
    Q = I * T0
    xp = 0.0
    for n in range(turns):
        # the kick of turn n uses the passages of turns n-1-k, k = 1 .. nh (k = 0 is this passage)
        xp += Q * X0 / ring["E0_eV"] * sum(A / math.sqrt(k * T0) for k in range(1, nh + 1) if n - 1 - k >= 0)
        assert trec[n, 0, 2] == pytest.approx(xp, rel=1e-9, abs=1e-18)   # sin(2 pi) residue ~1e-21
