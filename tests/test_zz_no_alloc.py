"""The allocation-free wake entry point (mbt_wake_noalloc).

Some callers cannot let a library call cudaMalloc: code that runs inside
another framework's device memory pool or under a fixed device-memory
budget.  mbt_wake_noalloc computes the short-range wake with the same
tensor-core kernel as tracking, keeping its working memory in a static device
array.  This test calls it through the C ABI on two consecutive turns of a
tracked fill and compares its voltages with the ones the tracking context
itself computed (mbt_read_wake) from the same histograms.
"""
import numpy as np
import pytest

import mbt_workloads as W

pytestmark = pytest.mark.gpu


def test_wake_noalloc_matches_tracking_wake_on_two_calls():
    torch = pytest.importorskip("torch")
    import paper_1809_00391_gb300 as pkg
    pkg.build()
    nb, nbins = 70, 256
    run = W.Run(W.ring_r0(), [dict(W.BROADBAND), dict(W.HOM)], np.arange(nb, dtype=np.int32),
                np.linspace(0.1e-3, 3e-3, nb), np.array([2000 + 37 * i for i in range(nb)], np.int64), seed=4,
                turns=2, precision=W.PREC_MIXED, nbins=nbins)
    tr = pkg.tracker_for_run(run)
    tr.init_particles()
    q = run.currents_A * run.ring["T0_s"] / run.n_mp
    V_dev = torch.empty((nb, nbins), dtype=torch.float32, device="cuda")
    for call in range(2):
        tr.track(1)
        h, _ = tr.histograms()
        v_ref, _ = tr.wake()
        hist_dev = torch.from_numpy(h).to("cuda")
        V_dev.fill_(float("nan"))
        torch.cuda.synchronize()
        pkg.wake_noalloc(run.ring, run.resonators, nbins, run.half_width_sigmas, q, hist_dev.data_ptr(),
                         V_dev.data_ptr(), stream=torch.cuda.current_stream())
        v = V_dev.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(v)), f"call {call}: unwritten output"
        assert np.max(np.abs(v - v_ref)) <= 1e-4 * np.max(np.abs(v_ref)), f"call {call}"
    # beyond the stated limits it refuses with a message, before touching the GPU
    with pytest.raises(pkg.MBTError, match="128 or 256"):
        pkg.wake_noalloc(run.ring, run.resonators, 512, 5.0, q, hist_dev.data_ptr(), V_dev.data_ptr())
    with pytest.raises(pkg.MBTError, match="1..1024"):
        pkg.wake_noalloc(run.ring, run.resonators, nbins, 5.0, np.ones(1025), hist_dev.data_ptr(), V_dev.data_ptr())
    tr.close()
