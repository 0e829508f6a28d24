"""Coupled-bunch instability scans (arXiv:1809.00391 Sec. 5): many runs that
differ in one parameter (the HOM frequency of a temperature scan) tracked
together as one batch (one push and one post launch per turn for all runs),
and the growth rates read off the bunch centroids.

Host-side analysis only: the tracking itself runs in libmbt's kernels.

* ``track_scan`` builds one tracker per run, tracks every run for the same
  number of turns in one batch and returns each run's per-turn moments.
* ``normal_form`` gives the left eigenvector of the linearised one-turn map
  (kick, RF, damping, drift: the map of Eqs. 1, 2, 5) so that a bunch's
  centroid (tau, delta) becomes one complex amplitude z with |z| constant for
  a free small oscillation apart from radiation damping.
* ``oscillation`` removes the slowly moving equilibrium (beam loading shifts
  the synchronous phase, differently along a train) from z;
  ``bunch_growth_rates`` and ``mode_growth_rates`` fit exponential rates of
  the oscillation per bunch, or of the fill's Fourier modes for equally
  spaced bunches.
* ``adaptive_rate`` fits only where an amplitude stands clear of its noise
  (a stable bunch reports no growth instead of the slope of its noise);
  ``rms_amplitude`` is the collective amplitude of a fill.
* ``eq7_growth_rates`` is the analytic estimate of Eq. 7 for M equal, equally
  spaced bunches (sums over positive-frequency lines only).
"""
from __future__ import annotations

import math
from typing import List, Sequence

import numpy as np

from . import Batch, tracker_for_run


def _phi_s(ring: dict, sr: bool = True) -> float:
    U0 = ring["U0_eV"] if sr else 0.0
    phi = math.asin(U0 / ring["V_rf_V"])
    return math.pi - phi if ring["alpha_c"] < 0 else phi


def linear_map(ring: dict, sr: bool = True) -> np.ndarray:
    """2x2 one-turn matrix of (tau, delta) about the synchronous particle:
    RF kick delta -= K tau with K = (V/E0) w_rf cos(phi_s), damping by
    (1 - D), D = 2 T0 / tau_z (none without radiation), then the drift
    tau += alpha_c T0 delta with the new delta."""
    T0, h = ring["T0_s"], ring["h"]
    w_rf = 2 * math.pi * h / T0
    K = ring["V_rf_V"] / ring["E0_eV"] * w_rf * math.cos(_phi_s(ring, sr))
    d = 1.0 - (2 * T0 / ring["tau_z_s"] if sr else 0.0)
    a = ring["alpha_c"] * T0
    return np.array([[1 - a * d * K, a * d], [-d * K, d]])


def normal_form(ring: dict, sr: bool = True):
    """(w, lam): left eigenvector w of the linear map with eigenvalue lam,
    Im lam > 0; z = w[0] tau + w[1] delta obeys z' = lam z."""
    ev, vl = np.linalg.eig(linear_map(ring, sr).T)
    i = int(np.argmax(ev.imag))
    return vl[:, i], ev[i]


def centroid_amplitudes(rec: np.ndarray, ring: dict, sr: bool = True) -> np.ndarray:
    """Complex normal-form amplitudes z[n, m] of the bunch centroids
    (rec[n, m, 0] = <tau>, rec[n, m, 2] = <delta>)."""
    w, _ = normal_form(ring, sr)
    return w[0] * rec[:, :, 0] + w[1] * rec[:, :, 2]


def oscillation(z: np.ndarray, ring: dict, sr: bool = True) -> np.ndarray:
    """The oscillating part of normal-form amplitudes z[n, ...]: z minus its
    centred moving average over one synchrotron period (P = round(1 / nu_s)
    turns), which follows the slowly moving equilibrium (the synchronous
    phase shift from beam loading, a transient along a train) and averages
    the oscillation out.  NaN within P/2 turns of either end."""
    P = max(2, int(round(1.0 / synchrotron_tune(ring, sr))))
    c = np.cumsum(np.concatenate([np.zeros((1,) + z.shape[1:], z.dtype), z], axis=0), axis=0)
    ma = (c[P:] - c[:-P]) / P   # ma[k] = mean of z[k : k + P]
    out = np.full(z.shape, np.nan + 0j, dtype=complex)
    h = P // 2
    out[h:h + ma.shape[0]] = z[h:h + ma.shape[0]] - ma
    return out


def oscillation_amplitudes(rec: np.ndarray, ring: dict, sr: bool = True) -> np.ndarray:
    """|oscillation| of every bunch's centroid, [turns][nb] (NaN near the ends)."""
    return np.abs(oscillation(centroid_amplitudes(rec, ring, sr), ring, sr))


def fit_rate(series: np.ndarray, lo: int, hi: int, T0: float) -> float:
    """Exponential rate [1/s] of |series| over turns [lo, hi) (least squares
    on log |series|); NaN if the series vanishes somewhere in the window."""
    a = np.abs(series[lo:hi])
    if not np.all(a > 0):
        return float("nan")
    return float(np.polyfit(np.arange(lo, hi), np.log(a), 1)[0] / T0)


def adaptive_rate(amp: np.ndarray, T0: float, noise_turns=(250, 1100), floor: float = 5.0, cap: float | None = None,
                  min_turns: int = 400) -> float:
    """Growth rate [1/s] of an oscillation amplitude series where it stands
    clear of its noise: from the last turn at or below floor x (median amp
    over noise_turns) up to the first turn that reaches cap (the end of the
    linear regime; the end of the series without a cap).  NaN when that
    stretch is shorter than min_turns (no measurable growth)."""
    noise = np.nanmedian(amp[noise_turns[0]:noise_turns[1]])
    fin = np.flatnonzero(np.isfinite(amp))
    if fin.size == 0:
        return float("nan")
    end = fin[-1] + 1
    if cap is not None:
        over = np.flatnonzero(np.isfinite(amp[:end]) & (amp[:end] >= cap))
        if over.size:
            end = over[0]
    low = np.flatnonzero(~(amp[:end] > floor * noise))   # NaN counts as low
    start = low[-1] + 1 if low.size else 0
    if end - start < min_turns:
        return float("nan")
    return fit_rate(amp, start, end, T0)


def rms_amplitude(rec: np.ndarray, ring: dict, sr: bool = True) -> np.ndarray:
    """Root mean square over bunches of the oscillation amplitudes, per turn."""
    a = oscillation_amplitudes(rec, ring, sr)
    return np.sqrt(np.mean(a * a, axis=1))


def bunch_growth_rates(rec: np.ndarray, ring: dict, lo: int, hi: int, bunches: Sequence[int] | None = None,
                       sr: bool = True) -> np.ndarray:
    """Growth rate [1/s] of each bunch's oscillation amplitude (about its
    moving equilibrium, see ``oscillation``) over turns [lo, hi); negative =
    damped."""
    z = oscillation(centroid_amplitudes(rec, ring, sr), ring, sr)
    idx = range(z.shape[1]) if bunches is None else bunches
    return np.array([fit_rate(z[:, m], lo, hi, ring["T0_s"]) for m in idx])


def mode_growth_rates(rec: np.ndarray, ring: dict, lo: int, hi: int, sr: bool = True) -> np.ndarray:
    """Growth rate [1/s] of every coupled-bunch mode mu of M equally spaced
    bunches: X_mu(n) = sum_m z_m(n) e^{-2 pi i mu m / M} of the oscillating
    parts z_m (see ``oscillation``)."""
    z = oscillation(centroid_amplitudes(rec, ring, sr), ring, sr)
    X = np.fft.fft(z, axis=1)   # e^{-2 pi i mu m / M}
    return np.array([fit_rate(X[:, mu], lo, hi, ring["T0_s"]) for mu in range(X.shape[1])])


def dominant_mode(rec: np.ndarray, ring: dict, lo: int, hi: int, contrast: float = 5.0, sr: bool = True):
    """(mu, rate): the coupled-bunch mode of largest amplitude at turn hi and
    its growth rate [1/s] over [lo, hi); rate is NaN unless that amplitude is
    at least `contrast` times the median over modes (a mode standing out of
    the noise)."""
    z = oscillation(centroid_amplitudes(rec, ring, sr), ring, sr)
    X = np.fft.fft(z, axis=1)
    a = np.abs(X[hi])
    mu = int(np.argmax(a))
    if a[mu] < contrast * np.median(a):
        return mu, float("nan")
    return mu, fit_rate(X[:, mu], lo, hi, ring["T0_s"])


def synchrotron_tune(ring: dict, sr: bool = True) -> float:
    """Tune of the linear map (phase of its eigenvalue / 2 pi)."""
    _, lam = normal_form(ring, sr)
    return float(np.angle(lam) / (2 * math.pi))


def eq7_growth_rates(ring: dict, M: int, I_bunch_A: float, Rs_ohm: float, fr_Hz: float, Q: float,
                     sr: bool = True, harmonics: int = 50) -> np.ndarray:
    """Eq. 7 for every mode mu of M equal bunches equally spaced around the
    ring (one HOM of shunt impedance Rs, frequency fr, quality factor Q):
    alpha_c M I_b w_r / (2 E0 T0 w_s) [sum_q Re Z((qM + mu) w0 + w_s)
    - sum_q' Re Z((q'M - mu) w0 - w_s)], positive-frequency lines only,
    E0 in eV.  Radiation damping is not included."""
    T0 = ring["T0_s"]
    w0 = 2 * math.pi / T0
    ws = synchrotron_tune(ring, sr) * w0
    wr = 2 * math.pi * fr_Hz
    mu = np.arange(M)[:, None]
    p0 = int(round(wr / w0 / M))
    q = np.arange(max(0, p0 - harmonics), p0 + harmonics)[None, :]

    def re_z(w):
        pos = w > 0
        wp = np.where(pos, w, wr)   # placeholder where the line frequency is not positive
        return np.where(pos, (Rs_ohm / (1 + 1j * Q * (wp / wr - wr / wp))).real, 0.0)

    up = re_z((q * M + mu) * w0 + ws).sum(axis=1)
    lo = re_z((q * M - mu) * w0 - ws).sum(axis=1)
    return ring["alpha_c"] * M * I_bunch_A * wr / (2 * ring["E0_eV"] * T0 * ws) * (up - lo)


def track_scan(runs: List, graph_turns: int = 100, stream=None, lanes: int = 1) -> List[np.ndarray]:
    """Track every run (same turn count) in one batch from its matched start;
    returns each run's moments [turns][nb][6].  lanes > 1: the runs in that
    many groups on streams of their own (mbt_batch_set_lanes; the same
    results bit for bit)."""
    turns = runs[0].turns
    if any(r.turns != turns for r in runs):
        raise ValueError("a scan tracks every run for the same number of turns")
    trackers = [tracker_for_run(r, record_turns=turns) for r in runs]
    try:
        for t in trackers:
            t.init_particles(stream)
        b = Batch(trackers)
        try:
            if graph_turns:
                b.set_graph(min(graph_turns, turns))
            if lanes > 1:
                b.set_lanes(lanes)
            b.track(turns, stream)
            b.sync()
        finally:
            b.close()
        return [t.moments(0, turns) for t in trackers]
    finally:
        for t in trackers:
            t.close()
