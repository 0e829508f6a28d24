"""Helpers shared by the physics tests: textbook synchrotron tune, Eq. 7 of the
paper (coupled-bunch growth rates for M equal, equally spaced bunches) and the
normal-form mode projection used to fit growth rates from bunch centroids."""
import math

import numpy as np

import mbt_workloads as W


def textbook_nu_s(ring, sr=True):
    """Small-amplitude synchrotron tune, nu_s^2 = alpha_c h eV cos(phi_s) / (2 pi E0)."""
    U0 = ring["U0_eV"] if sr else 0.0
    phi = math.asin(U0 / ring["V_rf_V"])
    if ring["alpha_c"] < 0:
        phi = math.pi - phi
    return math.sqrt(ring["alpha_c"] * ring["h"] * ring["V_rf_V"] * math.cos(phi) / (2 * math.pi * ring["E0_eV"]))


def map_tune(ring, sr=False):
    """Tune of the linearised kick-then-drift one-turn map."""
    nus = textbook_nu_s(ring, sr=sr)
    return math.acos(1 - (2 * math.pi * nus) ** 2 / 2) / (2 * math.pi)


def eq7_rate(M, mu, fr, Rs, Q, I_bunch, nu, ring=None):
    """Eq. 7 with omega_r in the numerator, summed over the positive-frequency
    upper (q M + mu) w0 + w_s and lower (q' M - mu) w0 - w_s lines [1/s]."""
    ring = ring or W.ring_r0()
    T0 = ring["T0_s"]
    w0 = 2 * math.pi / T0
    ws = nu * w0
    wr = 2 * math.pi * fr

    def ReZ(w):
        return (Rs / (1 + 1j * Q * (w / wr - wr / w))).real

    p0 = int(round(wr / w0 / M))
    up = sum(ReZ((q * M + mu) * w0 + ws) for q in range(max(0, p0 - 50), p0 + 50) if (q * M + mu) * w0 + ws > 0)
    lo = sum(ReZ((q * M - mu) * w0 - ws) for q in range(max(0, p0 - 50), p0 + 50) if (q * M - mu) * w0 - ws > 0)
    return ring["alpha_c"] * M * I_bunch * wr / (2 * ring["E0_eV"] * T0 * ws) * (up - lo)


def point_bunch_run(M, fr, Rs, I_bunch, turns, Q=2e4, amp=5e-12, n_mp=400, precision=W.PREC_F64, seed=3):
    """M point-like bunches (sigma_tau 3 ps, centroid offset amp with random
    phases) equally spaced in the ring, no radiation, a narrow long-range HOM."""
    ring = W.ring_r0()
    h, T0, ac = ring["h"], ring["T0_s"], ring["alpha_c"]
    nu = map_tune(ring)
    buckets = np.array([m * (h // M) for m in range(M)], np.int32)
    hom = dict(Rs_ohm=Rs, fr_Hz=fr, Q=Q, range=W.RANGE_LONG)
    run = W.Run(ring, [hom], buckets, np.full(M, I_bunch), np.full(M, n_mp, np.int64), seed=seed, turns=turns,
                precision=precision, flags=W.NO_SR)
    rng = np.random.default_rng(seed)
    st = 3e-12
    sdl = st * 2 * math.pi * nu / (ac * T0)
    parts = []
    for m in range(M):
        ph = rng.uniform(0, 2 * math.pi)
        parts.append((rng.normal(amp * math.cos(ph), st, n_mp), rng.normal(amp * math.sin(ph) * sdl / st, sdl, n_mp)))
    return run, parts


def mode_amplitudes(rec, ring=None):
    """X_mu(n) = sum_m z_m(n) e^{-2 pi i mu m / M} with z the normal-form
    coordinate (left eigenvector of the linear one-turn map, eigenvalue
    e^{+i 2 pi nu}) of the bunch centroids rec[n][m][0 (tau), 2 (delta)]."""
    ring = ring or W.ring_r0()
    M = rec.shape[1]
    T0, ac, h = ring["T0_s"], ring["alpha_c"], ring["h"]
    K = (ring["V_rf_V"] / ring["E0_eV"]) * 2 * math.pi * h / T0
    a = ac * T0
    M0 = np.array([[1 - a * K, a], [-K, 1.0]])
    ev, vl = np.linalg.eig(M0.T)
    wl = vl[:, int(np.argmax(ev.imag))]
    z = wl[0] * rec[:, :, 0] + wl[1] * rec[:, :, 2]
    return np.stack([(z * np.exp(-2j * math.pi * mu * np.arange(M) / M)[None, :]).sum(axis=1) for mu in range(M)])


def fit_rate(X, lo, hi, ring=None):
    """Exponential rate [1/s] of |X| over turns [lo, hi)."""
    ring = ring or W.ring_r0()
    n = np.arange(lo, hi)
    return np.polyfit(n, np.log(np.abs(X[lo:hi])), 1)[0] / ring["T0_s"]
