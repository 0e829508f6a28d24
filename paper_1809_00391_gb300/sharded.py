"""Bunch-sharded long-range scan across ranks (host side; mbt_phasor_* in the
C ABI do the arithmetic, torch.distributed the exchange).

One fill's bunches are split over the ranks of a process group in contiguous
ranges (rank r holds bunches [bounds[r], bounds[r+1])).  Per turn and
long-range resonator each rank reduces its bunches' emissions to one affine
map of the phasor (two complex numbers), the ranks allgather the maps, and
each rank composes them with the carry of the previous turn to obtain the
phasors its own bunches meet (Sec. 2.3, last paragraph: the long-range wake
acts after all bunches).  The only data exchanged per turn is 4 doubles per
resonator per rank.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import MBTError, lib, make_ring

_P = ctypes.POINTER
_d = ctypes.c_double
_i32 = ctypes.c_int32


def _pd(a: np.ndarray):
    return a.ctypes.data_as(_P(_d))


def _c(z: np.ndarray) -> np.ndarray:
    """complex128 array -> contiguous (re, im) float64 pairs."""
    return np.ascontiguousarray(np.asarray(z, np.complex128)).view(np.float64)


def split_bounds(nb: int, world: int) -> np.ndarray:
    """Contiguous bunch ranges, as equal as possible: bounds[r] .. bounds[r+1]."""
    return np.array([(r * nb) // world for r in range(world + 1)], np.int64)


def phasor_steps(ring: dict, resonator: dict, buckets) -> np.ndarray:
    """a_m = e^{s dt_m} of every bunch of the fill for one resonator."""
    b = np.ascontiguousarray(buckets, np.int32)
    out = np.empty(2 * len(b), np.float64)
    r = make_ring(ring)
    st = lib().mbt_phasor_steps(ctypes.byref(r), float(resonator["fr_Hz"]), float(resonator["Q"]), len(b),
                                b.ctypes.data_as(_P(_i32)), _pd(out))
    if st != 0:
        raise MBTError(st, "mbt_phasor_steps")
    return out.view(np.complex128)


def segment_map(step: np.ndarray, E: np.ndarray) -> np.ndarray:
    """(A, B) of this rank's range as complex128[2]."""
    s, e = _c(step), _c(E)
    out = np.empty(4, np.float64)
    st = lib().mbt_phasor_segment(len(s) // 2, _pd(s), _pd(e), _pd(out))
    if st != 0:
        raise MBTError(st, "mbt_phasor_segment")
    return out.view(np.complex128)


def compose(maps: np.ndarray, carry: complex):
    """Values entering every range and the new carry."""
    mp = _c(maps.reshape(-1))
    c = _c(np.array([carry]))
    entry = np.empty(2 * (len(mp) // 4), np.float64)
    out = np.empty(2, np.float64)
    st = lib().mbt_phasor_compose(len(mp) // 4, _pd(mp), _pd(c), _pd(entry), _pd(out))
    if st != 0:
        raise MBTError(st, "mbt_phasor_compose")
    return entry.view(np.complex128), complex(out[0], out[1])


def apply(step: np.ndarray, E: np.ndarray, entry: complex) -> np.ndarray:
    """Phi_m of this rank's bunches."""
    s, e = _c(step), _c(E)
    x = _c(np.array([entry]))
    out = np.empty(len(s), np.float64)
    st = lib().mbt_phasor_apply(len(s) // 2, _pd(s), _pd(e), _pd(x), _pd(out))
    if st != 0:
        raise MBTError(st, "mbt_phasor_apply")
    return out.view(np.complex128)


def exchange_turn(step_local: np.ndarray, E_local: np.ndarray, carry: complex, dist=None, group=None):
    """One turn of the sharded scan for one resonator: this rank's bunches'
    phasors and the carry into the next turn (the same on every rank).
    step_local, E_local: complex128 of this rank's bunches (possibly none)."""
    import torch
    m = segment_map(step_local, E_local)
    if dist is None:
        maps = m[None, :]
    else:
        mine = torch.from_numpy(m.view(np.float64).copy())
        parts = [torch.empty(4, dtype=torch.float64) for _ in range(dist.get_world_size(group))]
        dist.all_gather(parts, mine, group=group)
        maps = np.stack([p.numpy() for p in parts]).view(np.complex128)
    entry, carry_out = compose(maps, carry)
    rank = 0 if dist is None else dist.get_rank(group)
    return apply(step_local, E_local, complex(entry[rank])), carry_out
