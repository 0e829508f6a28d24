"""FP64 CPU oracle for longitudinal multi-bunch macro-particle tracking.

TEST INFRASTRUCTURE ONLY.  This package is the plain definition the CUDA
library is checked against (arXiv:1809.00391, Sec. 2.2-2.4, Eqs. 1, 2, 5, 6).
Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference legs of ``bench.py`` may import it.  It shares no code with the
CUDA path: the C source ``mbt_oracle.c`` is compiled here with gcc, with
floating-point contraction disabled so that x86-64 and aarch64 builds round
identically.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "mbt_oracle.c"
_BUILD = _HERE / "_build"
_LIB_PATH = _BUILD / "liboracle.so"
_lock = threading.Lock()
_lib = None

RANGE_SHORT = 1
RANGE_LONG = 2
RANGE_BOTH = 3
NO_SR = 1
NO_QE = 2
KICK_NGP = 4


def compile_source(src: Path, out: Path) -> Path:
    """gcc -O2 without floating-point contraction: the oracle's build flags."""
    tmp = Path(out).with_suffix(f".{os.getpid()}.tmp")
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-o", str(tmp), str(src), "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return Path(out)


def build(force: bool = False) -> Path:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, -O2, no contraction)."""
    _BUILD.mkdir(exist_ok=True)
    if force or not _LIB_PATH.exists() or _LIB_PATH.stat().st_mtime < _SRC.stat().st_mtime:
        compile_source(_SRC, _LIB_PATH)
    return _LIB_PATH


class Ring(ctypes.Structure):
    _fields_ = [("E0_eV", ctypes.c_double), ("T0_s", ctypes.c_double), ("h", ctypes.c_int32),
                ("pad_", ctypes.c_int32), ("V_rf_V", ctypes.c_double), ("alpha_c", ctypes.c_double),
                ("U0_eV", ctypes.c_double), ("sigma_delta", ctypes.c_double), ("tau_z_s", ctypes.c_double)]


class Resonator(ctypes.Structure):
    _fields_ = [("Rs_ohm", ctypes.c_double), ("fr_Hz", ctypes.c_double), ("Q", ctypes.c_double),
                ("range", ctypes.c_int32), ("pad_", ctypes.c_int32)]


class Harmonic(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("pad_", ctypes.c_int32), ("V_V", ctypes.c_double),
                ("phi_rad", ctypes.c_double)]


_P = ctypes.POINTER
_d = ctypes.c_double
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_u32 = ctypes.c_uint32
_u64 = ctypes.c_uint64


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load_library(build())
    return _lib


def load_library(path) -> ctypes.CDLL:
    """A compiled oracle library with its entry points typed (the tests also
    load deliberately mutated builds of the source to show that a pin fails
    on them)."""
    lib = ctypes.CDLL(str(path))
    lib.orc_philox4x32_10.argtypes = [_P(_u32), _P(_u32), _P(_u32)]
    lib.orc_u01.argtypes = [_u32]
    lib.orc_u01.restype = _d
    lib.orc_box_muller.argtypes = [_d, _d, _P(_d), _P(_d)]
    lib.orc_normal_quad.argtypes = [_u64, _u32, _u32, _u32, _u32, _P(_d)]
    lib.orc_derive.argtypes = [_P(Ring), ctypes.c_int, _P(_d)]
    lib.orc_wake.argtypes = [_P(Resonator), _d]
    lib.orc_wake.restype = _d
    lib.orc_create.argtypes = [_P(Ring), ctypes.c_int, _u64, ctypes.c_int, _P(Resonator),
                               ctypes.c_int, _d, ctypes.c_int, _P(_i32), _P(_d), _P(_i64)]
    lib.orc_create.restype = ctypes.c_void_p
    lib.orc_create_h.argtypes = [_P(Ring), ctypes.c_int, _u64, ctypes.c_int, _P(Resonator), ctypes.c_int,
                                 _P(Harmonic), ctypes.c_int, _d, ctypes.c_int, _P(_i32), _P(_d), _P(_i64)]
    lib.orc_create_h.restype = ctypes.c_void_p
    lib.orc_derive_h.argtypes = [_P(Ring), ctypes.c_int, ctypes.c_int, _P(Harmonic), _P(_d)]
    lib.orc_destroy.argtypes = [ctypes.c_void_p]
    lib.orc_get_derived.argtypes = [ctypes.c_void_p, _P(_d)]
    lib.orc_init_particles.argtypes = [ctypes.c_void_p]
    lib.orc_set_particles.argtypes = [ctypes.c_void_p, ctypes.c_int, _P(_d), _P(_d)]
    lib.orc_get_particles.argtypes = [ctypes.c_void_p, ctypes.c_int, _P(_d), _P(_d)]
    lib.orc_cell_coord.argtypes = [ctypes.c_void_p, _d]
    lib.orc_cell_coord.restype = _d
    lib.orc_bin.argtypes = [ctypes.c_void_p, _i64, _P(_d), _P(_i32)]
    lib.orc_bin.restype = _i64
    lib.orc_vsr_direct.argtypes = [ctypes.c_void_p, _P(_i32), _d, _P(_d)]
    lib.orc_track.argtypes = [ctypes.c_void_p, _i64, _P(_d)]
    lib.orc_get_hist.argtypes = [ctypes.c_void_p, _P(_i32), _P(_i64)]
    lib.orc_get_vsr.argtypes = [ctypes.c_void_p, _P(_d)]
    lib.orc_get_alr.argtypes = [ctypes.c_void_p, _P(_d)]
    lib.orc_get_wlag.argtypes = [ctypes.c_void_p, _P(_d)]
    lib.orc_feed_histograms.argtypes = [ctypes.c_void_p, _P(_i32)]
    lib.orc_get_last_emission.argtypes = [ctypes.c_void_p, ctypes.c_int, _P(_d)]
    lib.orc_wake_voltage_at.argtypes = [ctypes.c_void_p, ctypes.c_int, _d]
    lib.orc_wake_voltage_at.restype = _d
    lib.orc_turn.argtypes = [ctypes.c_void_p]
    lib.orc_turn.restype = _i64
    lib.orc_add_wake_table.argtypes = [ctypes.c_void_p, ctypes.c_int, _P(_d), _P(_d)]
    lib.orc_add_wake_table.restype = ctypes.c_int
    lib.orc_twake.argtypes = [_P(Resonator), _d]
    lib.orc_twake.restype = _d
    lib.orc_set_transverse.argtypes = [ctypes.c_void_p, _d, _d, _d, _d, _d, ctypes.c_int, _P(Resonator)]
    lib.orc_set_transverse.restype = ctypes.c_int
    lib.orc_track2.argtypes = [ctypes.c_void_p, _i64, _P(_d), _P(_d)]
    lib.orc_set_tparticles.argtypes = [ctypes.c_void_p, ctypes.c_int, _P(_d), _P(_d)]
    lib.orc_get_tparticles.argtypes = [ctypes.c_void_p, ctypes.c_int, _P(_d), _P(_d)]
    lib.orc_get_dip.argtypes = [ctypes.c_void_p, _P(_d)]
    lib.orc_get_vt.argtypes = [ctypes.c_void_p, _P(_d)]
    lib.orc_get_atlr.argtypes = [ctypes.c_void_p, _P(_d)]
    lib.orc_vt_direct.argtypes = [ctypes.c_void_p, _P(_d), _d, _P(_d)]
    lib.orc_add_transverse_rw.argtypes = [ctypes.c_void_p, _d, _d, _d, ctypes.c_int]
    lib.orc_add_transverse_rw.restype = ctypes.c_int
    lib.orc_transverse_rw_wake.argtypes = [ctypes.c_void_p, _d]
    lib.orc_transverse_rw_wake.restype = _d
    lib.orc_tvoltage_at.argtypes = [ctypes.c_void_p, ctypes.c_int, _d]
    lib.orc_tvoltage_at.restype = _d
    lib.orc_deposit.argtypes = [ctypes.c_void_p, _i64, _P(_d), _P(_d), _P(_i32), _P(_d)]
    lib.orc_deposit.restype = _i64
    return lib


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(_P(ct))


def philox4x32_10(ctr, key):
    """Philox4x32-10 block: 4 counter words, 2 key words -> 4 output words."""
    lib = _load()
    c = (_u32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (_u32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (_u32 * 4)()
    lib.orc_philox4x32_10(c, k, o)
    return tuple(int(x) for x in o)


def u01(w: int) -> float:
    """Uniform on (0,1) from one 32-bit word: (w + 1/2) 2^-32."""
    return _load().orc_u01(w & 0xFFFFFFFF)


def box_muller(u1: float, u2: float):
    a, b = _d(), _d()
    _load().orc_box_muller(u1, u2, ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def normal_quad(seed: int, quad: int, bunch: int, turn: int, tag: int):
    """The four normals of particles 4 quad .. 4 quad + 3."""
    r = (_d * 4)()
    _load().orc_normal_quad(seed, quad, bunch, turn, tag, r)
    return tuple(r)


def make_ring(ring: dict) -> Ring:
    return Ring(E0_eV=ring["E0_eV"], T0_s=ring["T0_s"], h=int(ring["h"]), pad_=0,
                V_rf_V=ring["V_rf_V"], alpha_c=ring["alpha_c"], U0_eV=ring["U0_eV"],
                sigma_delta=ring["sigma_delta"], tau_z_s=ring["tau_z_s"])


def make_resonator(res: dict) -> Resonator:
    return Resonator(Rs_ohm=res["Rs_ohm"], fr_Hz=res["fr_Hz"], Q=res["Q"], range=int(res["range"]), pad_=0)


def derive(ring: dict, flags: int = 0) -> dict:
    """Derived ring quantities (T_rf, omega_rf, phi_s, ...) as the oracle computes them."""
    out = (_d * 12)()
    r = make_ring(ring)
    _load().orc_derive(ctypes.byref(r), flags, out)
    keys = ["T_rf", "omega_rf", "phi_s", "sin_phi_s", "U0_over_E0", "V_over_E0", "D", "qe_amp",
            "nu_s", "sigma_tau0"]
    return {k: out[i] for i, k in enumerate(keys)}


def make_harmonic(hc: dict) -> Harmonic:
    return Harmonic(n=int(hc["n"]), pad_=0, V_V=float(hc["V_V"]), phi_rad=float(hc["phi_rad"]))


def derive_h(ring: dict, harmonic_cavities=(), flags: int = 0) -> dict:
    """Derived quantities with harmonic cavities (the main cavity's phase
    balances U0 against them)."""
    lib = _load()
    r = make_ring(ring)
    hs = list(harmonic_cavities)
    ha = (Harmonic * max(1, len(hs)))(*[make_harmonic(hc) for hc in hs])
    out = (_d * 12)()
    lib.orc_derive_h(ctypes.byref(r), int(flags), len(hs), ha, out)
    keys = ["T_rf", "omega_rf", "phi_s", "sin_phi_s", "U0_over_E0", "V_over_E0", "D", "qe_amp", "nu_s",
            "sigma_tau0"]
    return {k: out[i] for i, k in enumerate(keys)}


def twake(res: dict, t: float) -> float:
    """Transverse resonator wake W(t) [V/(C m)] (Rs_ohm in Ohm/m)."""
    r = make_resonator(res)
    return _load().orc_twake(ctypes.byref(r), float(t))


def wake(res: dict, t: float) -> float:
    r = make_resonator(res)
    return _load().orc_wake(ctypes.byref(r), float(t))


Z0_OHM = 376.730313668          # impedance of free space (mu_0 c)
C_LIGHT = 299_792_458.0


def resistive_wall_wake(t, radius_m: float, conductivity_S_per_m: float, length_m: float) -> np.ndarray:
    """Short-range longitudinal resistive-wall wake W(t) [V/C] of a round pipe
    (radius b, conductivity sigma, length L), t >= 0 the delay behind the
    source: with s = c t, s0 = (2 b^2 / (Z0 sigma))^(1/3), u = s / s0,
      W = (4 Z0 c L / (pi b^2)) [ e^{-u} cos(sqrt(3) u) / 3
                                  - (sqrt(2) / pi) int_0^inf x^2 e^{-x^2 u} / (x^6 + 8) dx ]
    (K. Bane and M. Sands, 'The short-range resistive wall wakefields', 1995,
    written in SI units); each integral by adaptive quadrature.  Positive =
    energy loss, as the resonator wake."""
    from scipy import integrate
    b, sig, L = float(radius_m), float(conductivity_S_per_m), float(length_m)
    s0 = (2.0 * b * b / (Z0_OHM * sig)) ** (1.0 / 3.0)
    pref = 4.0 * Z0_OHM * C_LIGHT * L / (np.pi * b * b)
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    out = np.empty_like(t)
    for i, ti in enumerate(t):
        u = C_LIGHT * ti / s0
        integral = integrate.quad(lambda x: x * x * np.exp(-x * x * u) / (x ** 6 + 8.0), 0.0, np.inf,
                                  epsabs=0.0, epsrel=1e-12, limit=400)[0]
        out[i] = pref * (np.exp(-u) * np.cos(np.sqrt(3.0) * u) / 3.0 - np.sqrt(2.0) / np.pi * integral)
    return out


def resistive_wall_table(radius_m: float, conductivity_S_per_m: float, length_m: float, t_max: float):
    """(t, W) samples of resistive_wall_wake on [0, t_max]: uniform to 20 s0/c
    (the oscillating head, 500 samples per s0/c: the linear interpolant's
    integral over a cell is then within ~1e-6 of the wake's), geometric beyond
    (the t^-3/2 tail)."""
    s0 = (2.0 * radius_m ** 2 / (Z0_OHM * conductivity_S_per_m)) ** (1.0 / 3.0)
    t1 = 20.0 * s0 / C_LIGHT
    t = np.linspace(0.0, t1, 10001)
    if t_max > t1:
        t = np.concatenate([t, np.geomspace(t1, t_max, 3000)[1:]])
    return t, resistive_wall_wake(t, radius_m, conductivity_S_per_m, length_m)


class OracleSim:
    """Plain FP64 multi-bunch tracker (one run).  wake_tables: extra
    short-range wakes as (t, W) samples; resistive_wall: round pipes as dicts
    radius_m, conductivity_S_per_m, length_m (tabulated here with
    resistive_wall_table)."""

    def __init__(self, ring: dict, resonators: list, nbins: int, half_width_sigmas: float,
                 buckets, currents_A, n_mp, seed: int, flags: int = 0, wake_tables=(), resistive_wall=(),
                 harmonic_cavities=(), transverse=None, lib=None):
        self._lib = lib if lib is not None else _load()
        self.nb = len(buckets)
        self.nbins = int(nbins)
        self.nres = len(resonators)
        self.resonators = list(resonators)
        self._ring = make_ring(ring)
        ra = (Resonator * max(1, self.nres))(*[make_resonator(r) for r in resonators])
        self.buckets = np.ascontiguousarray(buckets, dtype=np.int32)
        self.currents = np.ascontiguousarray(currents_A, dtype=np.float64)
        self.n_mp = np.ascontiguousarray(n_mp, dtype=np.int64)
        self.harmonics = list(harmonic_cavities)
        ha = (Harmonic * max(1, len(self.harmonics)))(*[make_harmonic(hc) for hc in self.harmonics])
        self._h = self._lib.orc_create_h(ctypes.byref(self._ring), int(flags), int(seed), self.nres, ra,
                                         len(self.harmonics), ha, self.nbins, float(half_width_sigmas), self.nb,
                                       _ptr(self.buckets, _i32), _ptr(self.currents, _d),
                                       _ptr(self.n_mp, _i64))
        if not self._h:
            raise ValueError("oracle rejected the configuration")
        tables = list(wake_tables)
        if resistive_wall:
            t_max = (self.nbins + 1) * self.derived["Delta"]
            for rw in resistive_wall:
                tables.append(resistive_wall_table(rw["radius_m"], rw["conductivity_S_per_m"], rw["length_m"],
                                                   t_max))
        for t, w in tables:
            t = np.ascontiguousarray(t, np.float64)
            w = np.ascontiguousarray(w, np.float64)
            if self._lib.orc_add_wake_table(self._h, len(t), _ptr(t, _d), _ptr(w, _d)) != 0:
                raise ValueError("wake table needs t[0] = 0 and increasing samples")
        self.transverse = transverse
        self.ntres = 0
        if transverse is not None:
            tres = list(transverse.get("resonators", ()))
            self.ntres = len(tres)
            self.tresonators = tres
            ta = (Resonator * max(1, len(tres)))(*[make_resonator(r) for r in tres])
            if self._lib.orc_set_transverse(self._h, float(transverse["beta_m"]), float(transverse.get("alpha", 0.0)),
                                            float(transverse["tune"]), float(transverse.get("chromaticity", 0.0)),
                                            float(transverse["emittance_m"]), len(tres), ta) != 0:
                raise ValueError("oracle rejected the transverse plane")
            for rw in transverse.get("resistive_wall", ()):
                if self._lib.orc_add_transverse_rw(self._h, float(rw["radius_m"]), float(rw["conductivity_S_per_m"]),
                                                   float(rw["length_m"]), int(rw["history_turns"])) != 0:
                    raise ValueError("oracle rejected the transverse resistive wall")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    @property
    def derived(self) -> dict:
        out = (_d * 12)()
        self._lib.orc_get_derived(self._h, out)
        keys = ["T_rf", "omega_rf", "phi_s", "D", "qe_amp", "nu_s", "sigma_tau0", "H", "Delta",
                "invDelta", "nhist", "turn"]
        return {k: out[i] for i, k in enumerate(keys)}

    def init_particles(self):
        self._lib.orc_init_particles(self._h)

    def set_particles(self, m: int, tau, delta):
        t = np.ascontiguousarray(tau, dtype=np.float64)
        d = np.ascontiguousarray(delta, dtype=np.float64)
        assert t.size == self.n_mp[m] and d.size == self.n_mp[m]
        self._lib.orc_set_particles(self._h, m, _ptr(t, _d), _ptr(d, _d))

    def particles(self, m: int):
        n = int(self.n_mp[m])
        t = np.empty(n, np.float64)
        d = np.empty(n, np.float64)
        self._lib.orc_get_particles(self._h, m, _ptr(t, _d), _ptr(d, _d))
        return t, d

    def cell_coord(self, tau: float) -> float:
        return self._lib.orc_cell_coord(self._h, float(tau))

    def bin(self, tau):
        """Histogram of arrival times on this run's mesh -> (hist, n_outside)."""
        t = np.ascontiguousarray(tau, dtype=np.float64)
        h = np.empty(self.nbins, np.int32)
        out = self._lib.orc_bin(self._h, t.size, _ptr(t, _d), _ptr(h, _i32))
        return h, int(out)

    def track(self, nturns: int, record: bool = True):
        """Track ``nturns``; returns moments [nturns][nb][6] if ``record``."""
        if record:
            rec = np.empty((nturns, self.nb, 6), np.float64)
            self._lib.orc_track(self._h, int(nturns), _ptr(rec, _d))
            return rec
        self._lib.orc_track(self._h, int(nturns), None)
        return None

    def histograms(self):
        h = np.empty((self.nb, self.nbins), np.int32)
        o = np.empty(self.nb, np.int64)
        self._lib.orc_get_hist(self._h, _ptr(h, _i32), _ptr(o, _i64))
        return h, o

    def vsr(self):
        v = np.empty((self.nb, self.nbins), np.float64)
        self._lib.orc_get_vsr(self._h, _ptr(v, _d))
        return v

    def vsr_direct(self, hist, q: float):
        h = np.ascontiguousarray(hist, dtype=np.int32)
        v = np.empty(self.nbins, np.float64)
        self._lib.orc_vsr_direct(self._h, _ptr(h, _i32), float(q), _ptr(v, _d))
        return v

    def alr(self):
        a = np.empty((max(1, self.nres), self.nb, 2), np.float64)
        self._lib.orc_get_alr(self._h, _ptr(a, _d))
        return a[..., 0] + 1j * a[..., 1]

    def wlag(self):
        w = np.empty(self.nbins, np.float64)
        self._lib.orc_get_wlag(self._h, _ptr(w, _d))
        return w

    def feed_histograms(self, hist):
        h = np.ascontiguousarray(hist, dtype=np.int32).reshape(self.nb, self.nbins)
        self._lib.orc_feed_histograms(self._h, _ptr(h, _i32))

    def last_emission(self, r: int):
        e = np.empty((self.nb, 2), np.float64)
        self._lib.orc_get_last_emission(self._h, int(r), _ptr(e, _d))
        return e[:, 0] + 1j * e[:, 1]

    def wake_voltage_at(self, m: int, tau: float) -> float:
        return self._lib.orc_wake_voltage_at(self._h, int(m), float(tau))

    def tvoltage_at(self, m: int, tau: float) -> float:
        """Transverse kick voltage on a particle of bunch m at tau (short range,
        long-range resonators and resistive wall of the previous turn)."""
        return self._lib.orc_tvoltage_at(self._h, int(m), float(tau))

    def deposit(self, tau, x):
        """(counts, dipole sums, outside count) of particles (tau, x) on the mesh."""
        t = np.ascontiguousarray(tau, np.float64)
        xx = np.ascontiguousarray(x, np.float64)
        assert t.shape == xx.shape
        h = np.empty(self.nbins, np.int32)
        d = np.empty(self.nbins, np.float64)
        out = self._lib.orc_deposit(self._h, t.size, _ptr(t, _d), _ptr(xx, _d), _ptr(h, _i32), _ptr(d, _d))
        return h, d, int(out)

    def transverse_rw_wake(self, t: float) -> float:
        return self._lib.orc_transverse_rw_wake(self._h, float(t))

    def track2(self, nturns: int):
        """Track nturns; returns (moments [n][nb][6], transverse moments [n][nb][4])."""
        rec = np.empty((int(nturns), self.nb, 6), np.float64)
        trec = np.empty((int(nturns), self.nb, 4), np.float64)
        self._lib.orc_track2(self._h, int(nturns), _ptr(rec, _d), _ptr(trec, _d))
        return rec, trec

    def set_tparticles(self, m: int, x, xp):
        x = np.ascontiguousarray(x, np.float64)
        xp = np.ascontiguousarray(xp, np.float64)
        assert x.size == self.n_mp[m] and xp.size == self.n_mp[m]
        self._lib.orc_set_tparticles(self._h, int(m), _ptr(x, _d), _ptr(xp, _d))

    def tparticles(self, m: int):
        x = np.empty(int(self.n_mp[m]), np.float64)
        xp = np.empty(int(self.n_mp[m]), np.float64)
        self._lib.orc_get_tparticles(self._h, int(m), _ptr(x, _d), _ptr(xp, _d))
        return x, xp

    def dipoles(self):
        d = np.empty((self.nb, self.nbins), np.float64)
        self._lib.orc_get_dip(self._h, _ptr(d, _d))
        return d

    def vt(self):
        v = np.empty((self.nb, self.nbins), np.float64)
        self._lib.orc_get_vt(self._h, _ptr(v, _d))
        return v

    def atlr(self):
        a = np.empty((max(1, self.ntres), self.nb, 2), np.float64)
        self._lib.orc_get_atlr(self._h, _ptr(a, _d))
        return a[..., 0] + 1j * a[..., 1]

    def vt_direct(self, dip, q: float):
        d = np.ascontiguousarray(dip, np.float64)
        v = np.empty(self.nbins, np.float64)
        self._lib.orc_vt_direct(self._h, _ptr(d, _d), float(q), _ptr(v, _d))
        return v

    @property
    def turn(self) -> int:
        return int(self._lib.orc_turn(self._h))
