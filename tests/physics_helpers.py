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


def flat_potential(ring, n=3):
    """Textbook flat-potential setting of an n-th harmonic cavity: the energy
    change of a turn and its first two derivatives vanish at tau = 0:
      V sin(phi_s) + k V sin(phi_h) = U0,  cos(phi_s) + n k cos(phi_h) = 0,
      sin(phi_s) + n^2 k sin(phi_h) = 0
    => sin(phi_s) = n^2/(n^2-1) U0/V, k = sqrt(1/n^2 - (U0/V)^2/(n^2-1))."""
    u = ring["U0_eV"] / ring["V_rf_V"]
    sphi = n * n / (n * n - 1) * u
    cphi = math.sqrt(1 - sphi * sphi)
    k = math.sqrt(1 / n ** 2 - u * u / (n * n - 1))
    phih = math.atan2(-sphi / (n * n * k), -cphi / (n * k))
    return dict(n=n, V_V=k * ring["V_rf_V"], phi_rad=phih), sphi, cphi, k


def double_rf_equilibrium(ring, hcs, L):
    """Stationary line density exp(-Phi / (alpha_c T0 sigma_E^2)) with Phi the
    exact potential of the main and harmonic cavities and the mean loss."""
    E0, T0, V, ac, sd = ring["E0_eV"], ring["T0_s"], ring["V_rf_V"], ring["alpha_c"], ring["sigma_delta"]
    w = 2 * math.pi * ring["h"] / T0
    Uh = sum(hc["V_V"] * math.sin(hc["phi_rad"]) for hc in hcs)
    phis = math.asin((ring["U0_eV"] - Uh) / V)
    tau = np.linspace(-L, L, 20001)
    Phi = -((V / w) * (np.cos(phis - w * tau) - math.cos(phis)) - ring["U0_eV"] * tau)
    for hc in hcs:
        nw = hc["n"] * w
        Phi -= (hc["V_V"] / nw) * (np.cos(hc["phi_rad"] - nw * tau) - math.cos(hc["phi_rad"]))
    Phi /= E0
    lam = np.exp(-(Phi - Phi.min()) / (ac * T0 * sd * sd))
    lam /= np.trapezoid(lam, tau)
    return tau, lam
