"""Bulk particle upload (mbt_set_particles_all, and mbt_set_particles_all_f32
with tau in FP32) on the GPU: page-locked host arrays read by the device
directly, and pageable arrays through the bunch-by-bunch path, all give the
device state that mbt_set_particles gives bunch by bunch (bit for bit), for
both precisions and ragged bunch sizes."""
import numpy as np
import pytest

import mbt_workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [W.PREC_MIXED, W.PREC_F64])
def test_set_particles_all_equals_per_bunch_copies(prec):
    torch = pytest.importorskip("torch")
    import paper_1809_00391_gb300 as pkg
    pkg.build()
    n_mp = np.array([1, 4, 5, 1023, 40_003, 7], np.int64)
    buckets = np.array([0, 1, 2, 10, 11, 300], np.int32)
    run = W.Run(W.ring_r0(), [dict(W.BROADBAND)], buckets, np.full(len(n_mp), 1e-3), n_mp, seed=5, turns=1,
                precision=prec)
    rng = np.random.default_rng(11)
    tau = rng.normal(0.0, 13e-12, int(n_mp.sum()))
    dl = rng.normal(0.0, 9e-4, int(n_mp.sum()))
    ref = pkg.tracker_for_run(run, record_turns=8)
    off = np.concatenate([[0], np.cumsum(n_mp)])
    for m in range(len(n_mp)):
        ref.set_particles(m, tau[off[m]:off[m + 1]], dl[off[m]:off[m + 1]])
    pinned_t = torch.from_numpy(tau).pin_memory()
    pinned_d = torch.from_numpy(dl).pin_memory()
    tau32 = tau.astype(np.float32)
    pinned_t32 = torch.from_numpy(tau32).pin_memory()
    # the FP32 uploads give what mbt_set_particles gives for the widened FP32 values
    # (the same state as `ref` on the mixed path, which rounds tau to FP32 anyway)
    ref32 = pkg.tracker_for_run(run, record_turns=8)
    for m in range(len(n_mp)):
        ref32.set_particles(m, tau32[off[m]:off[m + 1]].astype(np.float64), dl[off[m]:off[m + 1]])
    if prec == W.PREC_MIXED:
        for m in range(len(n_mp)):
            assert np.array_equal(ref32.particles(m)[0], ref.particles(m)[0])
    hists = {}
    for source in ("pinned", "pageable", "pinned_f32", "pageable_f32"):
        tr = pkg.tracker_for_run(run, record_turns=8)
        if source == "pinned":
            tr.set_particles_all(pinned_t, pinned_d, stream=torch.cuda.current_stream())
        elif source == "pageable":
            tr.set_particles_all(tau, dl)
        elif source == "pinned_f32":
            tr.set_particles_all(pinned_t32, pinned_d, stream=torch.cuda.current_stream())
        else:
            tr.set_particles_all(tau32, dl)
        want = ref32 if source.endswith("f32") else ref
        for m in range(len(n_mp)):
            a_t, a_d = tr.particles(m)
            b_t, b_d = want.particles(m)
            assert np.array_equal(a_t, b_t) and np.array_equal(a_d, b_d), (source, m)
        tr.track(3)
        tr.sync()
        hists[source] = tr.histograms()[0]
        tr.close()
    # and they track identically
    ref.track(3)
    ref32.track(3)
    ref.sync()
    h_ref, h_ref32 = ref.histograms()[0], ref32.histograms()[0]
    for source, h in hists.items():
        assert np.array_equal(h, h_ref32 if source.endswith("f32") else h_ref), source
    ref.close()
    ref32.close()
