"""Seeded synthetic workloads shared by the CUDA path's tests/bench and the oracle.

This module holds input definitions only: ring parameters, wake resonators,
fill patterns, currents, macro-particle counts, seeds and turn counts.  It
contains none of the tracking method's arithmetic (no synchronous phase, no
bunch length, no wake function); each side derives those itself.

Rings follow the synthetic SLS-like ring of the benchmark definitions
(E = 2.4 GeV, C = 288 m, h = 480, V = 2.1 MV, alpha_c = 6e-4, U0 = 0.5 MeV,
sigma_delta = 9e-4, tau_z = 4.5 ms).  The revolution period is C/c; the RF
bucket spacing is T0/h (so f_rf = 499.65 MHz rather than the nominal
500 MHz: the bucket grid must be exact).  Runs with more than 480 bunches use
h = 484 (the 'dc12c' harmonic number of Table 1 of the paper) with the other
parameters unchanged.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import List

import numpy as np

C_LIGHT = 299_792_458.0

RANGE_SHORT = 1
RANGE_LONG = 2
RANGE_BOTH = 3

NO_SR = 1
NO_QE = 2
KICK_NGP = 4

PREC_F64 = 0
PREC_MIXED = 1


def ring_r0(h: int = 480) -> dict:
    """The synthetic SLS-like ring (all SI units, energies in eV)."""
    return dict(E0_eV=2.4e9, T0_s=288.0 / C_LIGHT, h=int(h), V_rf_V=2.1e6, alpha_c=6e-4,
                U0_eV=0.5e6, sigma_delta=9e-4, tau_z_s=4.5e-3)


def ring_dc12c() -> dict:
    """Table 1 of the paper ('dc12c'); sigma_delta and tau_z are not printed
    there, so the SLS-like values stand in for them."""
    return dict(E0_eV=2.4e9, T0_s=290.4 / C_LIGHT, h=484, V_rf_V=1.4e6, alpha_c=-1.356e-4,
                U0_eV=569.604e3, sigma_delta=9e-4, tau_z_s=4.5e-3)


BROADBAND = dict(Rs_ohm=5e3, fr_Hz=10e9, Q=1.0, range=RANGE_SHORT)
HOM = dict(Rs_ohm=1e6, fr_Hz=1.5e9, Q=2e4, range=RANGE_BOTH)


@dataclass
class Run:
    """One tracking run: a ring, a wake model, a mesh and a fill."""
    ring: dict
    resonators: List[dict]
    buckets: np.ndarray          # int32 [nb], ascending
    currents_A: np.ndarray       # float64 [nb]
    n_mp: np.ndarray             # int64 [nb]
    seed: int
    turns: int
    precision: int = PREC_F64
    flags: int = 0
    nbins: int = 256
    half_width_sigmas: float = 5.0
    name: str = ""
    wake_tables: list = field(default_factory=list)      # [(t [s], W [V/C])] short range
    resistive_wall: list = field(default_factory=list)   # [dict(radius_m, conductivity_S_per_m, length_m)]
    harmonic_cavities: list = field(default_factory=list)  # [dict(n, V_V, phi_rad)] active harmonic RF
    transverse: dict = None   # dict(beta_m, alpha, tune, chromaticity, emittance_m, resonators=[...]) or None

    @property
    def nb(self) -> int:
        return int(len(self.buckets))

    @property
    def n_particles(self) -> int:
        return int(np.sum(self.n_mp))

    def scaled(self, n_mp_per_bunch=None, turns=None, nb=None):
        """A smaller copy (first ``nb`` bunches, fewer particles or turns)."""
        b = self.buckets if nb is None else self.buckets[:nb]
        c = self.currents_A if nb is None else self.currents_A[:nb]
        n = self.n_mp if nb is None else self.n_mp[:nb]
        if n_mp_per_bunch is not None:
            n = np.full(len(b), int(n_mp_per_bunch), np.int64)
        return replace(self, buckets=np.array(b, np.int32), currents_A=np.array(c, np.float64),
                       n_mp=np.array(n, np.int64), turns=self.turns if turns is None else int(turns))


def _fill(buckets, current_A, n_mp):
    b = np.asarray(buckets, np.int32)
    return b, np.full(len(b), float(current_A)), np.full(len(b), int(n_mp), np.int64)


def single_bunch(seed: int = 1) -> Run:
    """One bunch, 1e4 macro-particles, 1 mA, broadband resonator, FP64, 1000 turns."""
    b, c, n = _fill([0], 1e-3, 10_000)
    return Run(ring_r0(), [dict(BROADBAND)], b, c, n, seed=seed, turns=1000,
               precision=PREC_F64, name="1 bunch x 1e4 mp, BB wake, FP64, 1000 turns")


def three_bunches(seed: int = 1) -> Run:
    """Three adjacent bunches, 1e5 macro-particles each, 1 mA each, broadband +
    narrow-band HOM (long and short range), FP64, 1e4 turns."""
    b, c, n = _fill([0, 1, 2], 1e-3, 100_000)
    return Run(ring_r0(), [dict(BROADBAND), dict(HOM)], b, c, n, seed=seed, turns=10_000,
               precision=PREC_F64, name="3 bunches x 1e5 mp, BB + HOM, FP64, 1e4 turns")


def fill_390(seed: int = 1, precision: int = PREC_MIXED) -> Run:
    """390 bunches in buckets 0..389 of h = 480 (90-bucket ion-cleaning gap),
    1e5 macro-particles and 0.5 mA per bunch, broadband + HOM wake, 2e4 turns."""
    b, c, n = _fill(range(390), 0.5e-3, 100_000)
    return Run(ring_r0(), [dict(BROADBAND), dict(HOM)], b, c, n, seed=seed, turns=20_000,
               precision=precision, name="390-bunch 3/4 fill x 1e5 mp, BB + HOM, 2e4 turns")


def batched_runs(n_runs: int = 64, seed: int = 42, turns: int = 5000) -> List[Run]:
    """Independent runs with seed-drawn sizes: nb ~ U{1..484}, N ~ logU[1e4, 1e6],
    I ~ U[0.1, 3] mA per bunch; runs with nb > 480 use h = 484."""
    g = np.random.default_rng(seed)
    runs = []
    for i in range(n_runs):
        nb = int(g.integers(1, 485))
        nmp = int(round(10 ** g.uniform(4.0, 6.0)))
        cur = float(g.uniform(0.1e-3, 3e-3))
        h = 484 if nb > 480 else 480
        b, c, n = _fill(range(nb), cur, nmp)
        runs.append(Run(ring_r0(h), [dict(BROADBAND), dict(HOM)], b, c, n, seed=1000 + i,
                        turns=turns, precision=PREC_MIXED, name=f"batch run {i}"))
    return runs


# L5 longitudinal HOM of the ELETTRA-type cavity #3 at 45 C (Sec. 5).  Its
# shunt impedance and quality factor are not given: a synthetic pair stands in,
# sized so that the 400 mA uniform fill of the h = 484 ring shows both unstable
# lobes and stable windows within one revolution-harmonic period of detuning.
L5_FR_HZ = 1606.862e6
L5_RS_OHM = 2e5
L5_Q = 3e4


def l5_scan_runs(detunings_Hz, fill: str = "uniform", n_mp: int = 5000, turns: int = 4000, seed: int = 11,
                 total_current_A: float = 0.4, Rs_ohm: float = L5_RS_OHM, Q: float = L5_Q) -> List[Run]:
    """One run per HOM detuning on the 'dc12c' ring (h = 484): the L5 mode
    (short and long range) is the only wake; fill 'uniform' = all 484 buckets,
    'three_quarter' = buckets 0..362; equal bunches sharing total_current_A."""
    ring = ring_dc12c()
    nb = ring["h"] if fill == "uniform" else 363
    if fill not in ("uniform", "three_quarter"):
        raise ValueError("fill must be 'uniform' or 'three_quarter'")
    b, c, n = _fill(range(nb), total_current_A / nb, n_mp)
    runs = []
    for i, df in enumerate(detunings_Hz):
        hom = dict(Rs_ohm=Rs_ohm, fr_Hz=L5_FR_HZ + float(df), Q=Q, range=RANGE_BOTH)
        runs.append(Run(ring, [hom], b, c, n, seed=seed + i, turns=turns, precision=PREC_MIXED,
                        name=f"L5 {fill} fill, detuning {float(df) / 1e3:+.1f} kHz"))
    return runs


@dataclass
class ScanRequest:
    arrival_s: float
    run: Run


def serving_stream(n_requests: int = 200, rate_hz: float = 20.0, seed: int = 7) -> List[ScanRequest]:
    """Poisson stream of instability-scan requests: nb ~ U{1..484}, gap ~ U{0..120}
    (train + gap <= h), N ~ logU[1e4, 2e5], I ~ U[0.1, 5] mA per bunch,
    HOM f_r ~ U[1, 3] GHz, turns ~ U{2000..2e4}."""
    g = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n_requests):
        t += float(g.exponential(1.0 / rate_hz))
        nb = int(g.integers(1, 485))
        gap = int(g.integers(0, 121))
        h = 484 if nb > 480 else 480
        nb = min(nb, h - gap) if gap < h else nb
        nmp = int(round(10 ** g.uniform(4.0, np.log10(2e5))))
        cur = float(g.uniform(0.1e-3, 5e-3))
        fr = float(g.uniform(1e9, 3e9))
        turns = int(g.integers(2000, 20_001))
        b, c, n = _fill(range(nb), cur, nmp)
        hom = dict(HOM, fr_Hz=fr)
        out.append(ScanRequest(t, Run(ring_r0(h), [dict(BROADBAND), hom], b, c, n, seed=5000 + i,
                                      turns=turns, precision=PREC_MIXED, name=f"request {i}")))
    return out
