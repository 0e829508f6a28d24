"""The allocation-free wake entry point (mbt_wake_noalloc).

Some callers cannot let a library call cudaMalloc: code that runs inside
another framework's device memory pool or under a fixed device-memory
budget.  mbt_wake_noalloc computes the short-range wake with the same
tensor-core kernel as tracking, keeping its working memory in a static device
array.  These tests call it through the C ABI on two consecutive turns of a
tracked fill (128- and 256-cell meshes) and compare its voltages with the ones
the tracking context itself computed (mbt_read_wake) from the same
histograms; they also check its refusals: counts the kernel cannot split
exactly, and a stream under graph capture.
"""
import numpy as np
import pytest

import mbt_workloads as W

pytestmark = pytest.mark.gpu


def _run(nbins):
    nb = 70
    return W.Run(W.ring_r0(), [dict(W.BROADBAND), dict(W.HOM)], np.arange(nb, dtype=np.int32),
                 np.linspace(0.1e-3, 3e-3, nb), np.array([2000 + 37 * i for i in range(nb)], np.int64), seed=4,
                 turns=2, precision=W.PREC_MIXED, nbins=nbins)


@pytest.mark.parametrize("nbins", [256, 128])
def test_wake_noalloc_matches_tracking_wake_on_two_calls(nbins):
    torch = pytest.importorskip("torch")
    import paper_1809_00391_gb300 as pkg
    pkg.build()
    run = _run(nbins)
    nb = run.nb
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


def test_wake_noalloc_reports_counts_it_cannot_split():
    """A count of 2^24 or a negative count does not fit the kernel's three
    8-bit planes: the call reports MBT_ERR_ARG instead of a silent wrong
    voltage, and the next valid call is unaffected."""
    torch = pytest.importorskip("torch")
    import paper_1809_00391_gb300 as pkg
    pkg.build()
    run = W.single_bunch()
    nb, nbins = 3, 256
    q = np.full(nb, 1e-14)
    V = torch.empty((nb, nbins), dtype=torch.float32, device="cuda")
    for bad in (1 << 24, -1):
        h = np.zeros((nb, nbins), np.int32)
        h[1, 100] = bad
        hd = torch.from_numpy(h).to("cuda")
        with pytest.raises(pkg.MBTError, match=r"outside \[0, 2\^24\)") as e:
            pkg.wake_noalloc(run.ring, run.resonators, nbins, 5.0, q, hd.data_ptr(), V.data_ptr())
        assert e.value.status == 1
    h = np.zeros((nb, nbins), np.int32)
    h[:, 120:136] = (1 << 24) - 1
    hd = torch.from_numpy(h).to("cuda")
    pkg.wake_noalloc(run.ring, run.resonators, nbins, 5.0, q, hd.data_ptr(), V.data_ptr())
    v = V.cpu().numpy()
    assert np.all(np.isfinite(v)) and np.max(np.abs(v)) > 0


def test_wake_noalloc_refuses_a_capturing_stream():
    torch = pytest.importorskip("torch")
    import paper_1809_00391_gb300 as pkg
    pkg.build()
    run = W.single_bunch()
    nb, nbins = 2, 256
    q = np.full(nb, 1e-14)
    hd = torch.zeros((nb, nbins), dtype=torch.int32, device="cuda")
    V = torch.empty((nb, nbins), dtype=torch.float32, device="cuda")
    x = torch.zeros(4, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s):
        x.add_(1.0)
        with pytest.raises(pkg.MBTError, match="captured") as e:
            pkg.wake_noalloc(run.ring, run.resonators, nbins, 5.0, q, hd.data_ptr(), V.data_ptr(), stream=s)
        assert e.value.status == 2
    g.replay()
    torch.cuda.synchronize()
    assert float(x[0]) == 1.0
