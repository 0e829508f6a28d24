"""Python binding of libmbt: GB300-native longitudinal multi-bunch tracking.

A thin ctypes layer over the C ABI in ``include/mbt.h`` (argument marshalling
only; every step of the tracking runs in the library's CUDA kernels).  CUDA
streams may be given as ``None`` (legacy default stream), a raw handle
(``int``) or a ``torch.cuda.Stream``.  The library must have been built
(``paper_1809_00391_gb300.build()``); there is no fallback: using the binding
without it raises ``RuntimeError``.
"""
from __future__ import annotations

import ctypes
import threading
from pathlib import Path

import numpy as np

from ._build import LIB as _LIB_PATH
from ._build import build

__all__ = ["build", "lib", "Tracker", "Batch", "MBTError", "PREC_F64", "PREC_MIXED", "RANGE_SHORT",
           "RANGE_LONG", "RANGE_BOTH", "NO_SR", "NO_QE", "KICK_NGP", "EXPORTS", "tracker_for_run", "wake_noalloc",
           "Server"]

PREC_F64, PREC_MIXED = 0, 1
RANGE_SHORT, RANGE_LONG, RANGE_BOTH = 1, 2, 3
NO_SR, NO_QE, KICK_NGP = 1, 2, 4

# every entry point declared in include/mbt.h
EXPORTS = ["mbt_version", "mbt_status_string", "mbt_create", "mbt_destroy", "mbt_last_error",
           "mbt_add_resonator", "mbt_add_wake_table", "mbt_add_resistive_wall",
           "mbt_add_harmonic_cavity", "mbt_set_transverse", "mbt_add_transverse_resonator",
           "mbt_add_transverse_resistive_wall",
           "mbt_set_transverse_particles", "mbt_get_transverse_particles", "mbt_read_transverse_moments",
           "mbt_read_transverse_wake", "mbt_set_grid", "mbt_set_fill", "mbt_set_record", "mbt_init_particles",
           "mbt_set_particles", "mbt_set_particles_all", "mbt_set_particles_all_f32", "mbt_get_particles", "mbt_track", "mbt_track_resident", "mbt_set_wait_test", "mbt_resident_shape", "mbt_sync", "mbt_read_moments",
           "mbt_read_histograms", "mbt_read_wake", "mbt_get_info", "mbt_set_graph", "mbt_set_tile", "mbt_autotune",
           "mbt_set_timing",
           "mbt_get_timing", "mbt_set_trace", "mbt_read_trace", "mbt_state_size", "mbt_save_state", "mbt_load_state", "mbt_wake_noalloc", "mbt_batch_create",
           "mbt_batch_track", "mbt_batch_sync", "mbt_batch_set_graph", "mbt_batch_set_lanes", "mbt_batch_autotune_lanes", "mbt_batch_autotune",
           "mbt_batch_track_resident",
           "mbt_batch_destroy",
           "mbt_server_create", "mbt_server_submit", "mbt_server_poll", "mbt_server_wait", "mbt_server_get_stats",
           "mbt_server_destroy", "mbt_plan_streams", "mbt_plan_stream_split", "mbt_plan_lanes", "mbt_phasor_steps",
           "mbt_phasor_segment", "mbt_phasor_compose", "mbt_phasor_apply", "mbt_probe_fp64_fma"]


class MBTError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libmbt status {status}: {msg}")
        self.status = status


class Ring(ctypes.Structure):
    _fields_ = [("E0_eV", ctypes.c_double), ("T0_s", ctypes.c_double), ("h", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("V_rf_V", ctypes.c_double), ("alpha_c", ctypes.c_double),
                ("U0_eV", ctypes.c_double), ("sigma_delta", ctypes.c_double), ("tau_z_s", ctypes.c_double)]


class Info(ctypes.Structure):
    _fields_ = [("T_rf_s", ctypes.c_double), ("omega_rf", ctypes.c_double), ("phi_s", ctypes.c_double),
                ("nu_s", ctypes.c_double), ("sigma_tau0_s", ctypes.c_double), ("D", ctypes.c_double),
                ("half_width_s", ctypes.c_double), ("bin_width_s", ctypes.c_double),
                ("n_particles", ctypes.c_int64), ("turn", ctypes.c_int64), ("nb", ctypes.c_int32),
                ("nbins", ctypes.c_int32), ("n_long", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("device_bytes", ctypes.c_int64), ("push_ctas", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_active", ctypes.c_int), ("turns_per_step", ctypes.c_int),
                ("lanes", ctypes.c_int)]


class Request(ctypes.Structure):
    _fields_ = [("ring", Ring), ("precision", ctypes.c_int), ("flags", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("nres", ctypes.c_int), ("Rs_ohm", ctypes.POINTER(ctypes.c_double)),
                ("fr_Hz", ctypes.POINTER(ctypes.c_double)), ("Q", ctypes.POINTER(ctypes.c_double)),
                ("range", ctypes.POINTER(ctypes.c_int32)), ("nbins", ctypes.c_int),
                ("half_width_sigmas", ctypes.c_double), ("nb", ctypes.c_int),
                ("bucket", ctypes.POINTER(ctypes.c_int32)), ("current_A", ctypes.POINTER(ctypes.c_double)),
                ("n_mp", ctypes.POINTER(ctypes.c_int64)), ("turns", ctypes.c_int64)]


class RequestStatus(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int), ("turns_done", ctypes.c_int64), ("t_submit", ctypes.c_double),
                ("t_start", ctypes.c_double), ("t_finish", ctypes.c_double), ("device_bytes", ctypes.c_int64),
                ("error", ctypes.c_char * 128)]


class ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("submitted", "completed", "failed", "queued", "active",
                                              "max_active_seen", "steps", "used_bytes", "max_bytes_seen")] + \
               [("busy_seconds", ctypes.c_double), ("mp_turns", ctypes.c_double), ("now", ctypes.c_double)]


_lock = threading.Lock()
_lib = None
_P = ctypes.POINTER
_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_sz = ctypes.c_size_t


def lib() -> ctypes.CDLL:
    """The loaded libmbt (raises RuntimeError if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not Path(_LIB_PATH).exists():
                raise RuntimeError(f"libmbt is not built ({_LIB_PATH} missing): call paper_1809_00391_gb300.build()")
            L = ctypes.CDLL(str(_LIB_PATH))
            sig = {
                "mbt_version": ([], _i), "mbt_status_string": ([_i], ctypes.c_char_p),
                "mbt_create": ([_P(Ring), _i, _i, ctypes.c_uint64, _P(_vp)], _i),
                "mbt_destroy": ([_vp], None), "mbt_last_error": ([_vp], ctypes.c_char_p),
                "mbt_add_resonator": ([_vp, _d, _d, _d, _i], _i), "mbt_set_grid": ([_vp, _i, _d], _i),
                "mbt_add_wake_table": ([_vp, _i, _P(_d), _P(_d)], _i),
                "mbt_add_resistive_wall": ([_vp, _d, _d, _d], _i),
                "mbt_add_harmonic_cavity": ([_vp, _i, _d, _d], _i),
                "mbt_set_transverse": ([_vp, _d, _d, _d, _d, _d], _i),
                "mbt_add_transverse_resonator": ([_vp, _d, _d, _d, _i], _i),
                "mbt_add_transverse_resistive_wall": ([_vp, _d, _d, _d, _i], _i),
                "mbt_set_transverse_particles": ([_vp, _i, _P(_d), _P(_d)], _i),
                "mbt_get_transverse_particles": ([_vp, _i, _P(_d), _P(_d)], _i),
                "mbt_read_transverse_moments": ([_vp, _i64, _i64, _P(_d)], _i),
                "mbt_read_transverse_wake": ([_vp, _P(_d), _P(_d)], _i),
                "mbt_set_fill": ([_vp, _i, _P(_i32), _P(_d), _P(_i64)], _i),
                "mbt_set_record": ([_vp, _i64], _i), "mbt_init_particles": ([_vp, _vp], _i),
                "mbt_set_particles": ([_vp, _i, _P(_d), _P(_d)], _i),
                "mbt_set_particles_all": ([_vp, _vp, _vp, _vp], _i),
                "mbt_set_particles_all_f32": ([_vp, _vp, _vp, _vp], _i),
                "mbt_get_particles": ([_vp, _i, _P(_d), _P(_d)], _i),
                "mbt_track": ([_vp, _i64, _vp], _i), "mbt_sync": ([_vp], _i),
                "mbt_track_resident": ([_vp, _i64, _vp], _i),
                "mbt_set_wait_test": ([_vp, _i64, _i], _i), "mbt_resident_shape": ([_vp, _P(_i), _P(_i)], _i),
                "mbt_read_moments": ([_vp, _i64, _i64, _P(_d)], _i),
                "mbt_read_histograms": ([_vp, _P(_i32), _P(_i64)], _i),
                "mbt_read_wake": ([_vp, _P(_d), _P(_d)], _i), "mbt_get_info": ([_vp, _P(Info)], _i),
                "mbt_set_graph": ([_vp, _i], _i), "mbt_set_timing": ([_vp, _i], _i),
                "mbt_set_tile": ([_vp, _i], _i), "mbt_autotune": ([_vp, _i, _P(_i)], _i),
                "mbt_batch_set_graph": ([_vp, _i], _i), "mbt_batch_set_lanes": ([_vp, _i], _i), "mbt_batch_autotune_lanes": ([_vp, _i, _i, _P(_i)], _i),
                "mbt_batch_autotune": ([_vp, _i, _P(_i)], _i),
                "mbt_get_timing": ([_vp, _P(_d), _P(_d), _P(_i64)], _i),
                "mbt_set_trace": ([_vp, _i], _i), "mbt_read_trace": ([_vp, _P(_i64), _i, _P(_i)], _i),
                "mbt_state_size": ([_vp, _P(_sz)], _i), "mbt_save_state": ([_vp, _vp, _sz], _i),
                "mbt_load_state": ([_vp, _vp, _sz], _i),
                "mbt_wake_noalloc": ([_P(Ring), _i, _i, _P(_d), _P(_d), _P(_d), _P(_i32), _i, _d, _i, _P(_d), _vp,
                                      _vp, _vp, ctypes.c_char_p, _sz], _i),
                "mbt_batch_create": ([_P(_vp), _i, _P(_vp)], _i), "mbt_batch_track": ([_vp, _i64, _vp], _i),
                "mbt_batch_track_resident": ([_vp, _i64, _vp], _i),
                "mbt_batch_sync": ([_vp], _i), "mbt_batch_destroy": ([_vp], None),
                "mbt_server_create": ([_P(ServerConfig), _P(_vp)], _i),
                "mbt_server_submit": ([_vp, _P(Request), _P(_i64)], _i),
                "mbt_server_poll": ([_vp, _i64, _P(RequestStatus), _P(_d), _P(_d)], _i),
                "mbt_server_wait": ([_vp, _i64, _d], _i), "mbt_server_get_stats": ([_vp, _P(ServerStats)], _i),
                "mbt_server_destroy": ([_vp], None),
                "mbt_plan_streams": ([_i, _P(_i64), _P(_i32), _i, _i, _P(_i)], _i),
                "mbt_plan_stream_split": ([_i, _P(_i32), _P(_i64), _i, _P(_i64), _i64, _P(_i64)], _i),
                "mbt_plan_lanes": ([_i, _P(_i64), _i, _P(_i32)], _i),
                "mbt_phasor_steps": ([_P(Ring), _d, _d, _i, _P(_i32), _P(_d)], _i),
                "mbt_phasor_segment": ([_i, _P(_d), _P(_d), _P(_d)], _i),
                "mbt_phasor_compose": ([_i, _P(_d), _P(_d), _P(_d), _P(_d)], _i),
                "mbt_phasor_apply": ([_i, _P(_d), _P(_d), _P(_d), _P(_d)], _i),
                "mbt_probe_fp64_fma": ([_i, _i, _i, _vp, _P(_d), _P(_i)], _i),
            }
            for name, (args, res) in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def plan_streams(run_n, run_nb, any_transverse: bool, ctas: int) -> bool:
    """Whether runs of run_n[i] macro-particles in run_nb[i] bunches go to the
    streaming push on a device holding `ctas` streaming CTAs (host only)."""
    n = np.ascontiguousarray(run_n, np.int64)
    nb = np.ascontiguousarray(run_nb, np.int32)
    out = _i()
    st = lib().mbt_plan_streams(len(n), _ptr(n, _i64), _ptr(nb, _i32), 1 if any_transverse else 0, ctas,
                                ctypes.byref(out))
    if st != 0:
        raise MBTError(st, "mbt_plan_streams")
    return bool(out.value)


def stream_split(run, n_mp, ctas: int) -> np.ndarray:
    """The streaming push's tiles for bunches (run[i], n_mp[i]) over `ctas`
    CTAs: rows (bunch, first particle, count, CTA) in bunch order (host only)."""
    r = np.ascontiguousarray(run, np.int32)
    n = np.ascontiguousarray(n_mp, np.int64)
    cnt = _i64()
    L = lib()
    st = L.mbt_plan_stream_split(len(n), _ptr(r, _i32), _ptr(n, _i64), ctas, None, 0, ctypes.byref(cnt))
    if st != 0:
        raise MBTError(st, "mbt_plan_stream_split")
    out = np.zeros((cnt.value, 4), np.int64)
    if cnt.value:
        st = L.mbt_plan_stream_split(len(n), _ptr(r, _i32), _ptr(n, _i64), ctas, _ptr(out, _i64), cnt.value,
                                     ctypes.byref(cnt))
        if st != 0:
            raise MBTError(st, "mbt_plan_stream_split")
    return out


def plan_lanes(n_particles, nlanes: int) -> np.ndarray:
    """The lane of each batch member that mbt_batch_set_lanes forms (host only)."""
    n = np.ascontiguousarray(n_particles, np.int64)
    out = np.zeros(len(n), np.int32)
    st = lib().mbt_plan_lanes(len(n), _ptr(n, _i64), int(nlanes), _ptr(out, _i32))
    if st != 0:
        raise MBTError(st, "mbt_plan_lanes")
    return out


def _stream(s) -> ctypes.c_void_p:
    if s is None:
        return ctypes.c_void_p(0)
    if isinstance(s, int):
        return ctypes.c_void_p(s)
    handle = getattr(s, "cuda_stream", None)
    if handle is None:
        raise TypeError("stream must be None, an int handle or a torch.cuda.Stream")
    return ctypes.c_void_p(int(handle))


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(_P(ct))


class Tracker:
    """One run (ring, wakes, mesh, fill) tracked on the GPU through libmbt."""

    def __init__(self, ring: dict, precision: int = PREC_MIXED, flags: int = 0, seed: int = 1,
                 resonators=(), nbins: int = 256, half_width_sigmas: float = 5.0,
                 buckets=(0,), currents_A=(1e-3,), n_mp=(10_000,), record_turns: int = 4096,
                 wake_tables=(), resistive_wall=(), harmonic_cavities=(), transverse=None):
        self._L = lib()
        self._h = ctypes.c_void_p()
        r = Ring(E0_eV=ring["E0_eV"], T0_s=ring["T0_s"], h=int(ring["h"]), reserved=0, V_rf_V=ring["V_rf_V"],
                 alpha_c=ring["alpha_c"], U0_eV=ring["U0_eV"], sigma_delta=ring["sigma_delta"],
                 tau_z_s=ring["tau_z_s"])
        st = self._L.mbt_create(ctypes.byref(r), int(precision), int(flags), int(seed) & (2 ** 64 - 1),
                                ctypes.byref(self._h))
        if st != 0:
            raise MBTError(st, "mbt_create rejected the ring or options")
        self.precision = int(precision)
        for res in resonators:
            self._chk(self._L.mbt_add_resonator(self._h, res["Rs_ohm"], res["fr_Hz"], res["Q"], int(res["range"])))
        for t, w in wake_tables:
            t = np.ascontiguousarray(t, np.float64)
            w = np.ascontiguousarray(w, np.float64)
            if t.shape != w.shape:
                raise ValueError("wake table: t and W differ in length")
            self._chk(self._L.mbt_add_wake_table(self._h, len(t), _ptr(t, _d), _ptr(w, _d)))
        self.transverse = transverse
        if transverse is not None:
            self._chk(self._L.mbt_set_transverse(self._h, float(transverse["beta_m"]), float(transverse.get("alpha", 0.0)),
                                                 float(transverse["tune"]), float(transverse.get("chromaticity", 0.0)),
                                                 float(transverse["emittance_m"])))
            for res in transverse.get("resonators", ()):
                self._chk(self._L.mbt_add_transverse_resonator(self._h, res["Rs_ohm"], res["fr_Hz"], res["Q"],
                                                               int(res["range"])))
            for rw in transverse.get("resistive_wall", ()):
                self._chk(self._L.mbt_add_transverse_resistive_wall(
                    self._h, float(rw["radius_m"]), float(rw["conductivity_S_per_m"]), float(rw["length_m"]),
                    int(rw["history_turns"])))
        for hc in harmonic_cavities:
            self._chk(self._L.mbt_add_harmonic_cavity(self._h, int(hc["n"]), float(hc["V_V"]), float(hc["phi_rad"])))
        for rw in resistive_wall:
            self._chk(self._L.mbt_add_resistive_wall(self._h, float(rw["radius_m"]), float(rw["conductivity_S_per_m"]),
                                                     float(rw["length_m"])))
        self._chk(self._L.mbt_set_grid(self._h, int(nbins), float(half_width_sigmas)))
        self._chk(self._L.mbt_set_record(self._h, int(record_turns)))
        self.buckets = np.ascontiguousarray(buckets, np.int32)
        self.currents = np.ascontiguousarray(currents_A, np.float64)
        self.n_mp = np.ascontiguousarray(n_mp, np.int64)
        self.nb = len(self.buckets)
        self.nbins = int(nbins)
        self._chk(self._L.mbt_set_fill(self._h, self.nb, _ptr(self.buckets, _i32), _ptr(self.currents, _d),
                                       _ptr(self.n_mp, _i64)))

    def _chk(self, st: int):
        if st != 0:
            raise MBTError(st, self._L.mbt_last_error(self._h).decode())

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._L.mbt_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_particles(self, stream=None):
        self._chk(self._L.mbt_init_particles(self._h, _stream(stream)))

    def set_particles(self, bunch: int, tau, delta):
        t = np.ascontiguousarray(tau, np.float64)
        d = np.ascontiguousarray(delta, np.float64)
        if t.size != self.n_mp[bunch] or d.size != self.n_mp[bunch]:
            raise ValueError("array sizes must equal n_mp of the bunch")
        self._chk(self._L.mbt_set_particles(self._h, int(bunch), _ptr(t, _d), _ptr(d, _d)))

    def set_particles_all(self, tau, delta, stream=None):
        """Every bunch's coordinates from back-to-back host arrays (n_particles
        doubles each: bunch 0, then bunch 1, ...).  ``tau`` and ``delta`` are
        numpy arrays or CPU torch tensors; page-locked ones (e.g. torch
        ``pin_memory()``) are read by the device directly."""
        n = int(self.n_mp.sum())
        # tau may be FP32 (mbt_set_particles_all_f32: the mixed path's own precision)
        t32 = str(getattr(tau, "dtype", "")) in ("torch.float32", "float32")
        ptrs = []
        keep = []
        for a, want in ((tau, "float32" if t32 else "float64"), (delta, "float64")):
            if hasattr(a, "data_ptr"):
                if a.dtype.__str__() != "torch." + want or a.numel() != n or not a.is_contiguous() or a.is_cuda:
                    raise ValueError(f"need contiguous CPU {want} tensors of n_particles values")
                ptrs.append(a.data_ptr())
            else:
                arr = np.ascontiguousarray(a, np.dtype(want))
                if arr.size != n:
                    raise ValueError("need n_particles values")
                keep.append(arr)
                ptrs.append(arr.ctypes.data)
        call = self._L.mbt_set_particles_all_f32 if t32 else self._L.mbt_set_particles_all
        self._chk(call(self._h, ctypes.c_void_p(ptrs[0]), ctypes.c_void_p(ptrs[1]), _stream(stream)))

    def particles(self, bunch: int):
        n = int(self.n_mp[bunch])
        t = np.empty(n, np.float64)
        d = np.empty(n, np.float64)
        self._chk(self._L.mbt_get_particles(self._h, int(bunch), _ptr(t, _d), _ptr(d, _d)))
        return t, d

    def track(self, nturns: int, stream=None):
        self._chk(self._L.mbt_track(self._h, int(nturns), _stream(stream)))

    def track_resident(self, nturns: int, stream=None):
        """Track with the bunches' particles resident in cluster shared memory."""
        self._chk(self._L.mbt_track_resident(self._h, int(nturns), _stream(stream)))

    def resident_shape(self):
        """(CTAs per cluster, particles per CTA) of resident tracking; (0, 0) if it does not fit."""
        a, b = _i(), _i()
        self._chk(self._L.mbt_resident_shape(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def sync(self):
        self._chk(self._L.mbt_sync(self._h))

    def set_wait_test(self, limit_ns: int, unreachable: bool):
        """Failure-detection test hook: the resident grid barrier's wait limit,
        and a barrier count nothing reaches (mbt_set_wait_test)."""
        self._chk(self._L.mbt_set_wait_test(self._h, int(limit_ns), 1 if unreachable else 0))

    def moments(self, turn0: int, nturns: int) -> np.ndarray:
        out = np.empty((int(nturns), self.nb, 6), np.float64)
        self._chk(self._L.mbt_read_moments(self._h, int(turn0), int(nturns), _ptr(out, _d)))
        return out

    def histograms(self):
        h = np.empty((self.nb, self.nbins), np.int32)
        o = np.empty(self.nb, np.int64)
        self._chk(self._L.mbt_read_histograms(self._h, _ptr(h, _i32), _ptr(o, _i64)))
        return h, o

    def wake(self):
        info = self.info
        v = np.empty((self.nb, self.nbins), np.float64)
        phi = np.zeros((max(1, info["n_long"]), self.nb, 2), np.float64)
        self._chk(self._L.mbt_read_wake(self._h, _ptr(v, _d), _ptr(phi, _d)))
        return v, phi[..., 0] + 1j * phi[..., 1]

    @property
    def info(self) -> dict:
        i = Info()
        self._chk(self._L.mbt_get_info(self._h, ctypes.byref(i)))
        return {k: getattr(i, k) for k, _ in Info._fields_}

    def set_transverse_particles(self, bunch: int, x, xp):
        x = np.ascontiguousarray(x, np.float64)
        xp = np.ascontiguousarray(xp, np.float64)
        if x.size != self.n_mp[bunch] or xp.size != self.n_mp[bunch]:
            raise ValueError("need n_mp[bunch] coordinates")
        self._chk(self._L.mbt_set_transverse_particles(self._h, int(bunch), _ptr(x, _d), _ptr(xp, _d)))

    def transverse_particles(self, bunch: int):
        n = int(self.n_mp[bunch])
        x = np.empty(n, np.float64)
        xp = np.empty(n, np.float64)
        self._chk(self._L.mbt_get_transverse_particles(self._h, int(bunch), _ptr(x, _d), _ptr(xp, _d)))
        return x, xp

    def transverse_moments(self, turn0: int, nturns: int) -> np.ndarray:
        out = np.empty((int(nturns), self.nb, 4), np.float64)
        self._chk(self._L.mbt_read_transverse_moments(self._h, int(turn0), int(nturns), _ptr(out, _d)))
        return out

    def transverse_wake(self):
        """(dipole sums [nb][nbins] of the last turn, transverse voltage [nb][nbins] for the next kick)."""
        dip = np.empty((self.nb, self.nbins), np.float64)
        v = np.empty((self.nb, self.nbins), np.float64)
        self._chk(self._L.mbt_read_transverse_wake(self._h, _ptr(dip, _d), _ptr(v, _d)))
        return dip, v

    def set_graph(self, turns_per_graph: int):
        self._chk(self._L.mbt_set_graph(self._h, int(turns_per_graph)))

    def set_tile(self, particles: int):
        self._chk(self._L.mbt_set_tile(self._h, int(particles)))

    def autotune(self, turns_per_trial: int = 20) -> int:
        """Pick the fastest push tile by timing real turns; returns it."""
        t = _i()
        self._chk(self._L.mbt_autotune(self._h, int(turns_per_trial), ctypes.byref(t)))
        return t.value

    def set_timing(self, enable: bool):
        self._chk(self._L.mbt_set_timing(self._h, 1 if enable else 0))

    def timing(self):
        a, b, n = _d(), _d(), _i64()
        self._chk(self._L.mbt_get_timing(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(n)))
        return a.value, b.value, n.value

    def set_trace(self, enable: bool):
        self._chk(self._L.mbt_set_trace(self._h, 1 if enable else 0))

    def trace(self) -> np.ndarray:
        """[njobs][5]: job type, bunch tile, start, job done, exit (ns) of the last post launch."""
        n = _i()
        self._chk(self._L.mbt_read_trace(self._h, None, 0, ctypes.byref(n)))
        out = np.zeros((n.value, 5), np.int64)
        self._chk(self._L.mbt_read_trace(self._h, _ptr(out, _i64), n.value, ctypes.byref(n)))
        return out

    def save_state(self) -> bytes:
        n = _sz()
        self._chk(self._L.mbt_state_size(self._h, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        self._chk(self._L.mbt_save_state(self._h, buf, n))
        return buf.raw

    def load_state(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        self._chk(self._L.mbt_load_state(self._h, buf, len(blob)))


class Batch:
    """Several trackers (same precision) advanced by the same kernel launches."""

    def __init__(self, trackers):
        self._L = lib()
        self.trackers = list(trackers)
        arr = (ctypes.c_void_p * len(self.trackers))(*[t.handle.value for t in self.trackers])
        self._h = ctypes.c_void_p()
        st = self._L.mbt_batch_create(arr, len(self.trackers), ctypes.byref(self._h))
        if st != 0:
            raise MBTError(st, "mbt_batch_create failed")

    def track(self, nturns: int, stream=None):
        st = self._L.mbt_batch_track(self._h, int(nturns), _stream(stream))
        if st != 0:
            raise MBTError(st, self._L.mbt_last_error(self.trackers[0].handle).decode())

    def track_resident(self, nturns: int, stream=None):
        """Every member tracked resident at the same time (one stream each,
        forked from and joined into `stream`)."""
        st = self._L.mbt_batch_track_resident(self._h, int(nturns), _stream(stream))
        if st != 0:
            raise MBTError(st, self._L.mbt_last_error(self.trackers[0].handle).decode())

    def set_graph(self, turns_per_graph: int):
        st = self._L.mbt_batch_set_graph(self._h, int(turns_per_graph))
        if st != 0:
            raise MBTError(st, "mbt_batch_set_graph failed")

    def set_lanes(self, nlanes: int):
        """Track the members as nlanes groups on streams of their own (mbt_batch_set_lanes)."""
        st = self._L.mbt_batch_set_lanes(self._h, int(nlanes))
        if st != 0:
            raise MBTError(st, self._L.mbt_last_error(self.trackers[0].handle).decode())

    def autotune_lanes(self, turns_per_trial: int = 20, max_lanes: int = 4) -> int:
        """Choose the lane count by timing 1..max_lanes (mbt_batch_autotune_lanes; real turns)."""
        k = _i()
        st = self._L.mbt_batch_autotune_lanes(self._h, int(turns_per_trial), int(max_lanes), ctypes.byref(k))
        if st != 0:
            raise MBTError(st, self._L.mbt_last_error(self.trackers[0].handle).decode())
        return k.value

    def autotune(self, turns_per_trial: int = 5) -> int:
        t = _i()
        st = self._L.mbt_batch_autotune(self._h, int(turns_per_trial), ctypes.byref(t))
        if st != 0:
            raise MBTError(st, self._L.mbt_last_error(self.trackers[0].handle).decode())
        return t.value

    def sync(self):
        st = self._L.mbt_batch_sync(self._h)
        if st != 0:
            raise MBTError(st, self._L.mbt_last_error(self.trackers[0].handle).decode())

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._L.mbt_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching server for instability-scan requests (mbt_server_*)."""

    STATES = {0: "queued", 1: "running", 2: "done", 3: "failed"}

    def __init__(self, hbm_budget_bytes: int, max_active: int = 64, turns_per_step: int = 100, lanes: int = 1):
        self._L = lib()
        self._h = ctypes.c_void_p()
        cfg = ServerConfig(int(hbm_budget_bytes), int(max_active), int(turns_per_step), int(lanes))
        st = self._L.mbt_server_create(ctypes.byref(cfg), ctypes.byref(self._h))
        if st != 0:
            raise MBTError(st, "mbt_server_create failed")
        self._runs = {}

    def submit(self, run) -> int:
        """Queue an ``mbt_workloads.Run`` (tracked for run.turns turns); returns its id."""
        keep = dict(
            rs=np.ascontiguousarray([r["Rs_ohm"] for r in run.resonators] or [0.0], np.float64),
            fr=np.ascontiguousarray([r["fr_Hz"] for r in run.resonators] or [0.0], np.float64),
            q=np.ascontiguousarray([r["Q"] for r in run.resonators] or [0.0], np.float64),
            rg=np.ascontiguousarray([int(r["range"]) for r in run.resonators] or [0], np.int32),
            b=np.ascontiguousarray(run.buckets, np.int32), c=np.ascontiguousarray(run.currents_A, np.float64),
            n=np.ascontiguousarray(run.n_mp, np.int64))
        req = Request(ring=make_ring(run.ring), precision=int(run.precision), flags=int(run.flags),
                      seed=int(run.seed), nres=len(run.resonators), Rs_ohm=_ptr(keep["rs"], _d),
                      fr_Hz=_ptr(keep["fr"], _d), Q=_ptr(keep["q"], _d), range=_ptr(keep["rg"], _i32),
                      nbins=int(run.nbins), half_width_sigmas=float(run.half_width_sigmas), nb=run.nb,
                      bucket=_ptr(keep["b"], _i32), current_A=_ptr(keep["c"], _d), n_mp=_ptr(keep["n"], _i64),
                      turns=int(run.turns))
        rid = _i64()
        st = self._L.mbt_server_submit(self._h, ctypes.byref(req), ctypes.byref(rid))
        if st != 0:
            raise MBTError(st, "mbt_server_submit rejected the request")
        self._runs[rid.value] = run
        return rid.value

    def wait(self, rid: int, timeout_s: float = 600.0):
        st = self._L.mbt_server_wait(self._h, int(rid), float(timeout_s))
        if st != 0:
            raise MBTError(st, f"request {rid} did not complete: {self.status(rid)['error']}")

    def status(self, rid: int) -> dict:
        s = RequestStatus()
        st = self._L.mbt_server_poll(self._h, int(rid), ctypes.byref(s), None, None)
        if st != 0:
            raise MBTError(st, "unknown request")
        return dict(state=self.STATES[s.state], turns_done=s.turns_done, t_submit=s.t_submit, t_start=s.t_start,
                    t_finish=s.t_finish, device_bytes=s.device_bytes, error=s.error.decode())

    def result(self, rid: int):
        """(final moments [nb][6], history [turns][2]) of a finished request."""
        run = self._runs[rid]
        fm = np.zeros((run.nb, 6), np.float64)
        hist = np.zeros((run.turns, 2), np.float64)
        s = RequestStatus()
        st = self._L.mbt_server_poll(self._h, int(rid), ctypes.byref(s), _ptr(fm, _d), _ptr(hist, _d))
        if st != 0 or s.state != 2:
            raise MBTError(st or 4, f"request {rid} is not done")
        return fm, hist

    def stats(self) -> dict:
        s = ServerStats()
        self._L.mbt_server_get_stats(self._h, ctypes.byref(s))
        return {n: getattr(s, n) for n, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._L.mbt_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_ring(ring: dict) -> Ring:
    return Ring(E0_eV=ring["E0_eV"], T0_s=ring["T0_s"], h=int(ring["h"]), reserved=0, V_rf_V=ring["V_rf_V"],
                alpha_c=ring["alpha_c"], U0_eV=ring["U0_eV"], sigma_delta=ring["sigma_delta"], tau_z_s=ring["tau_z_s"])


def wake_noalloc(ring: dict, resonators, nbins: int, half_width_sigmas: float, charge_per_count, hist_ptr: int,
                 V_ptr: int, flags: int = 0, stream=None) -> None:
    """Short-range wake of device counts ``hist_ptr`` (int32 [nb][nbins]) into
    device ``V_ptr`` (float32 [nb][nbins]) through mbt_wake_noalloc, which
    allocates no device memory."""
    L = lib()
    q = np.ascontiguousarray(charge_per_count, np.float64)
    rs = np.ascontiguousarray([r["Rs_ohm"] for r in resonators] or [0.0], np.float64)
    fr = np.ascontiguousarray([r["fr_Hz"] for r in resonators] or [0.0], np.float64)
    qq = np.ascontiguousarray([r["Q"] for r in resonators] or [0.0], np.float64)
    rg = np.ascontiguousarray([int(r["range"]) for r in resonators] or [0], np.int32)
    r = make_ring(ring)
    err = ctypes.create_string_buffer(256)
    st = L.mbt_wake_noalloc(ctypes.byref(r), int(flags), len(resonators), _ptr(rs, _d), _ptr(fr, _d), _ptr(qq, _d),
                            _ptr(rg, _i32), int(nbins), float(half_width_sigmas), int(q.size), _ptr(q, _d),
                            ctypes.c_void_p(int(hist_ptr)), ctypes.c_void_p(int(V_ptr)), _stream(stream), err, 256)
    if st != 0:
        raise MBTError(st, err.value.decode())


def probe_fp64_fma(blocks_per_sm: int = 8, iters: int = 4096, repeats: int = 5, stream=None):
    """(FP64 DFMA throughput of the GPU [flop/s], SM count), timed with CUDA events."""
    f, n = _d(), _i()
    st = lib().mbt_probe_fp64_fma(int(blocks_per_sm), int(iters), int(repeats), _stream(stream), ctypes.byref(f),
                                  ctypes.byref(n))
    if st != 0:
        raise MBTError(st, "mbt_probe_fp64_fma")
    return f.value, n.value


def tracker_for_run(run, precision=None, record_turns: int = 4096) -> Tracker:
    """A Tracker for an ``mbt_workloads.Run`` description."""
    return Tracker(run.ring, precision=run.precision if precision is None else precision, flags=run.flags,
                   seed=run.seed, resonators=run.resonators, nbins=run.nbins,
                   half_width_sigmas=run.half_width_sigmas, buckets=run.buckets, currents_A=run.currents_A,
                   n_mp=run.n_mp, record_turns=record_turns, wake_tables=run.wake_tables,
                   resistive_wall=run.resistive_wall, harmonic_cavities=run.harmonic_cavities,
                   transverse=run.transverse)
