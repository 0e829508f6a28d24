"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every entry point that include/mbt.h declares, validates arguments, and
derives the ring quantities from the same definitions as the oracle."""
import math
import os
import re

import numpy as np
import pytest

import mbt_workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    import paper_1809_00391_gb300 as p
    p.build()
    return p


def _declared():
    src = open(os.path.join(ROOT, "include", "mbt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mbt_[a-z0-9_]+)\s*\(", src)))


def test_header_and_binding_agree(pkg):
    assert _declared() == sorted(pkg.EXPORTS)


def test_library_exports_every_declared_symbol(pkg):
    L = pkg.lib()
    for name in _declared():
        assert hasattr(L, name), name
    assert L.mbt_version() == 100
    assert L.mbt_status_string(0) == b"ok"
    assert L.mbt_status_string(5) == b"device wait timed out"


def _create(pkg, ring, prec=0, flags=0):
    import ctypes
    L = pkg.lib()
    r = pkg.Ring(E0_eV=ring["E0_eV"], T0_s=ring["T0_s"], h=ring["h"], reserved=0, V_rf_V=ring["V_rf_V"],
                 alpha_c=ring["alpha_c"], U0_eV=ring["U0_eV"], sigma_delta=ring["sigma_delta"],
                 tau_z_s=ring["tau_z_s"])
    h = ctypes.c_void_p()
    st = L.mbt_create(ctypes.byref(r), prec, flags, 7, ctypes.byref(h))
    return st, h


def test_argument_validation(pkg):
    L = pkg.lib()
    for bad in (dict(E0_eV=0.0), dict(h=0), dict(alpha_c=0.0), dict(U0_eV=3e6), dict(tau_z_s=-1.0)):
        ring = W.ring_r0()
        ring.update(bad)
        st, h = _create(pkg, ring)
        assert st == 1 and not h.value
    st, h = _create(pkg, W.ring_r0(), prec=7)
    assert st == 1
    st, h = _create(pkg, W.ring_r0(), prec=1)
    assert st == 0
    assert L.mbt_add_resonator(h, 1e3, 1e9, 0.4, 1) == 1          # Q <= 1/2
    assert L.mbt_add_resonator(h, 1e3, 1e9, 2.0, 0) == 1          # no range
    for _ in range(4):
        assert L.mbt_add_resonator(h, 1e3, 1e9, 2.0, 3) == 0
    assert L.mbt_add_resonator(h, 1e3, 1e9, 2.0, 2) == 6          # fifth long-range resonator
    assert b"long-range" in L.mbt_last_error(h)
    assert L.mbt_set_grid(h, 200, 5.0) == 6                        # mixed needs 128 or 256
    assert L.mbt_set_grid(h, 128, 5.0) == 0
    assert L.mbt_set_grid(h, 256, -1.0) == 1
    assert L.mbt_track(h, 10, None) == 2                           # no fill yet
    L.mbt_destroy(h)


@pytest.mark.parametrize("ring,flags", [(W.ring_r0(), 0), (W.ring_r0(), W.NO_SR), (W.ring_dc12c(), 0)],
                         ids=["R0", "R0-noSR", "dc12c"])
def test_derived_quantities_match_the_oracle(pkg, oracle_mod, ring, flags):
    import ctypes
    st, h = _create(pkg, ring, prec=0, flags=flags)
    assert st == 0
    L = pkg.lib()
    assert L.mbt_set_grid(h, 256, 5.0) == 0
    info = pkg.Info()
    assert L.mbt_get_info(h, ctypes.byref(info)) == 0
    o = oracle_mod.OracleSim(ring, [], 256, 5.0, [0], [0.0], [2], 7, flags)
    d = o.derived
    assert info.phi_s == pytest.approx(d["phi_s"], rel=1e-15)
    assert info.nu_s == pytest.approx(d["nu_s"], rel=1e-15)
    assert info.sigma_tau0_s == pytest.approx(d["sigma_tau0"], rel=1e-15)
    assert info.half_width_s == pytest.approx(d["H"], rel=1e-15)
    assert info.bin_width_s == pytest.approx(d["Delta"], rel=1e-15)
    assert info.D == pytest.approx(d["D"], rel=1e-15)
    assert info.T_rf_s == pytest.approx(d["T_rf"], rel=1e-15)
    L.mbt_destroy(h)


def test_binding_fails_loudly_without_library(pkg, monkeypatch, tmp_path):
    import paper_1809_00391_gb300 as p
    monkeypatch.setattr(p, "_lib", None)
    monkeypatch.setattr(p, "_LIB_PATH", tmp_path / "missing.so")
    with pytest.raises(RuntimeError, match="not built"):
        p.lib()


def test_tracker_fails_loudly_without_a_gpu(pkg):
    """The Python API has no CPU path either: on a machine without a GPU,
    building a tracker raises MBTError with MBT_ERR_CUDA at mbt_set_fill."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(pkg.MBTError) as e:
        pkg.tracker_for_run(W.single_bunch())
    assert e.value.status == 4 and "CUDA" in str(e.value)


def test_fill_is_validated_before_any_device_work(pkg):
    """mbt_set_fill rejects bad fills on the host (MBT_ERR_ARG, with a message);
    a valid fill needs the GPU and, without one, fails loudly with
    MBT_ERR_CUDA: there is no CPU path behind the boundary."""
    import ctypes
    L = pkg.lib()
    st, h = _create(pkg, W.ring_r0(), prec=1)
    assert st == 0

    def fill(b, c, n):
        b = np.ascontiguousarray(b, np.int32)
        c = np.ascontiguousarray(c, np.float64)
        n = np.ascontiguousarray(n, np.int64)
        return L.mbt_set_fill(h, len(b), pkg._ptr(b, ctypes.c_int32), pkg._ptr(c, ctypes.c_double),
                              pkg._ptr(n, ctypes.c_int64))

    bad = [([0, 0], [1e-3, 1e-3], [10, 10]),      # buckets not strictly increasing
           ([3, 1], [1e-3, 1e-3], [10, 10]),
           ([480], [1e-3], [10]),                 # bucket outside [0, h)
           ([-1], [1e-3], [10]),
           ([0], [-1e-3], [10]),                  # negative current
           ([0], [float("nan")], [10]),
           ([0], [1e-3], [0]),                    # empty bunch
           ([0], [1e-3], [1 << 24])]              # mixed precision: at most 2^24 - 1 per bunch
    for b, c, n in bad:
        assert fill(b, c, n) == 1, (b, c, n)
        assert L.mbt_last_error(h)
    assert L.mbt_set_fill(h, 0, None, None, None) == 1
    import torch
    if not torch.cuda.is_available():
        assert fill([0, 3], [1e-3, 1e-3], [100, 37]) == 4
        assert b"CUDA" in L.mbt_last_error(h)
    L.mbt_destroy(h)


def test_new_entry_points_validate_their_arguments(pkg):
    import ctypes
    L = pkg.lib()
    D = ctypes.c_double
    st, h = _create(pkg, W.ring_r0(), prec=0)
    assert st == 0

    def arr(v):
        a = (D * len(v))(*v)
        return a

    # tabulated wakes: at least 2 samples from t = 0, strictly increasing, finite
    assert L.mbt_add_wake_table(h, 1, arr([0.0]), arr([1.0])) == 1
    assert L.mbt_add_wake_table(h, 2, arr([1e-12, 2e-12]), arr([1.0, 0.5])) == 1
    assert L.mbt_add_wake_table(h, 3, arr([0.0, 2e-12, 1e-12]), arr([1.0, 0.5, 0.2])) == 1
    assert L.mbt_add_wake_table(h, 2, arr([0.0, 1e-12]), arr([float("nan"), 0.5])) == 1
    assert L.mbt_add_wake_table(h, 2, arr([0.0, 1e-12]), arr([1.0, 0.5])) == 0
    # resistive wall: every argument positive
    for bad in ((0.0, 5.8e7, 100.0), (0.01, -1.0, 100.0), (0.01, 5.8e7, 0.0)):
        assert L.mbt_add_resistive_wall(h, *bad) == 1
    assert L.mbt_add_resistive_wall(h, 0.01, 5.8e7, 100.0) == 0
    # harmonic cavities: 1 <= n <= 16, V >= 0, at most two
    assert L.mbt_add_harmonic_cavity(h, 0, 1e5, 0.0) == 1
    assert L.mbt_add_harmonic_cavity(h, 17, 1e5, 0.0) == 1
    assert L.mbt_add_harmonic_cavity(h, 3, -1.0, 0.0) == 1
    assert L.mbt_add_harmonic_cavity(h, 3, 1e5, 0.3) == 0
    assert L.mbt_add_harmonic_cavity(h, 4, 1e4, 0.1) == 0
    assert L.mbt_add_harmonic_cavity(h, 5, 1e4, 0.1) == 6
    # transverse: resonators need the plane first; the long-range limit is shared
    assert L.mbt_add_transverse_resonator(h, 1e5, 1e9, 1e3, 3) == 2
    assert L.mbt_set_transverse(h, -1.0, 0.0, 0.3, 0.0, 1e-9) == 1
    assert L.mbt_set_transverse(h, 10.0, 0.0, 0.3, 0.0, -1e-9) == 1
    assert L.mbt_set_transverse(h, 10.0, 0.0, 0.3, 0.0, 1e-9) == 0
    assert L.mbt_set_transverse(h, 10.0, 0.0, 0.3, 0.0, 1e-9) == 2   # already set
    for _ in range(3):
        assert L.mbt_add_resonator(h, 1e3, 1e9, 2.0, 3) == 0
    assert L.mbt_add_transverse_resonator(h, 1e5, 1e9, 1e3, 2) == 0
    assert L.mbt_add_transverse_resonator(h, 1e5, 1e9, 1e3, 2) == 6   # fifth long-range entry
    assert L.mbt_add_transverse_resonator(h, 1e5, 1e9, 1e3, 1) == 0   # short range only is fine
    assert L.mbt_add_transverse_resonator(h, 1e5, 1e9, 0.2, 1) == 1   # Q <= 1/2
    L.mbt_destroy(h)


def test_harmonic_cavity_derivation_matches_the_oracle(pkg, oracle_mod):
    import ctypes
    ring = W.ring_r0()
    hcs = [dict(n=3, V_V=4e5, phi_rad=-2.9), dict(n=4, V_V=5e4, phi_rad=0.4)]
    st, h = _create(pkg, ring, prec=0)
    L = pkg.lib()
    for hc in hcs:
        assert L.mbt_add_harmonic_cavity(h, hc["n"], hc["V_V"], hc["phi_rad"]) == 0
    assert L.mbt_set_grid(h, 256, 5.0) == 0
    info = pkg.Info()
    assert L.mbt_get_info(h, ctypes.byref(info)) == 0
    d = oracle_mod.derive_h(ring, hcs)
    assert info.phi_s == pytest.approx(math.asin(d["sin_phi_s"]), rel=1e-15)
    assert info.sigma_tau0_s == pytest.approx(d["sigma_tau0"], rel=1e-14)
    L.mbt_destroy(h)


def test_wake_noalloc_refuses_misaligned_pointers_before_device_work(pkg):
    """The allocation-free wake reads the caller's counts 16 bytes at a time
    and stores the voltages as floats: a misaligned pointer (one row of a
    larger buffer, an odd offset) is refused with MBT_ERR_ARG and a message
    before anything reaches the GPU.  The addresses are never dereferenced."""
    run = W.single_bunch()
    q = np.full(2, 1e-13)
    with pytest.raises(pkg.MBTError, match="16-byte aligned") as e:
        pkg.wake_noalloc(run.ring, run.resonators, 256, 5.0, q, 0x10004, 0x20000)
    assert e.value.status == 1
    with pytest.raises(pkg.MBTError, match="4-byte aligned") as e:
        pkg.wake_noalloc(run.ring, run.resonators, 256, 5.0, q, 0x10000, 0x20002)
    assert e.value.status == 1


def test_wait_test_hook_validates_its_arguments(pkg):
    import ctypes
    L = pkg.lib()
    st, h = _create(pkg, W.ring_r0(), prec=1)
    assert st == 0
    try:
        assert L.mbt_set_wait_test(h, -1, 0) == 1
        assert L.mbt_set_wait_test(h, 20_000_000_000, 0) == 1
        assert L.mbt_set_wait_test(h, 1000, 2) == 1
        assert L.mbt_set_wait_test(h, 20_000_000, 1) == 0
        assert L.mbt_set_wait_test(h, 0, 0) == 0
        assert L.mbt_set_wait_test(None, 0, 0) == 1
    finally:
        L.mbt_destroy(h)
    assert ctypes is not None


def test_server_and_lane_arguments_are_validated_before_device_work(pkg):
    """mbt_server_create refuses a bad configuration (lanes outside 0..8
    among them) before it starts a thread or touches a device; the batch
    lane calls refuse a NULL batch."""
    import ctypes
    L = pkg.lib()
    out = ctypes.c_void_p()
    for budget, active, step, lanes in ((1 << 30, 4, 10, 9), (1 << 30, 4, 10, -1), (0, 4, 10, 1),
                                        (1 << 30, 0, 10, 1), (1 << 30, 4, 0, 1)):
        cfg = pkg.ServerConfig(budget, active, step, lanes)
        assert L.mbt_server_create(ctypes.byref(cfg), ctypes.byref(out)) == 1
        assert not out.value
    k = ctypes.c_int()
    assert L.mbt_batch_set_lanes(None, 2) == 1
    assert L.mbt_batch_autotune_lanes(None, 5, 2, ctypes.byref(k)) == 1
