"""Precision of the recorded bunch moments on the mixed-precision path (GPU
tests, through the C ABI).

The push sums tau - tau_ref and delta - delta_ref per particle (FP32 over
one warp's share of a tile, FP64 from the tile on; the references are the
tile's first particle before the push), and the post kernel combines the
tiles exactly, so that the variance does not cancel when a bunch's centroid
sits far outside its own length (the
saturated coupled-bunch instability of the 390-bunch fill: centroids of
~100 ps against lengths of 15-80 ps).  The recorded mean and rms of a turn
must equal an FP64 two-pass recomputation from the GPU's own particles of
that turn to 1e-6 (relative to the rms), on every push kernel: the streaming
push (the 390-bunch fill at full size, tracked into saturation, and bunches
started 20 rms lengths off centre), the per-tile push and the cluster-resident
kernel.
"""
import numpy as np
import pytest

import mbt_workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-6


@pytest.fixture(scope="module")
def pkg():
    import paper_1809_00391_gb300 as p
    p.build()
    return p


def _check(tr, bunches, turn):
    """Recorded moments of `turn` against the FP64 two-pass values of the
    GPU's particles.  The push sums delta narrowed to FP32 by truncation
    (the value its drift uses), so the recorded mean delta may sit up to
    2^-23 <|delta|> from the FP64 mean: that bound is added for it."""
    rec = tr.moments(turn, 1)[0]
    worst = 0.0
    for m in bunches:
        t, d = tr.particles(m)
        mt, md = t.mean(), d.mean()
        st, sd = np.sqrt(np.mean((t - mt) ** 2)), np.sqrt(np.mean((d - md) ** 2))
        narrow = 2.0 ** -23 * np.mean(np.abs(d)) / sd
        errs = (abs(rec[m, 0] - mt) / st, abs(rec[m, 1] - st) / st, abs(rec[m, 2] - md) / sd - narrow,
                abs(rec[m, 3] - sd) / sd)
        assert max(errs) <= TOL, (m, errs, mt / st, narrow)
        worst = max(worst, max(errs))
    return worst


def test_saturated_fill390_moments_match_fp64_recomputation(pkg):
    run = W.fill_390(seed=1)
    turns = 1500
    tr = pkg.tracker_for_run(run, record_turns=turns)
    assert tr.info["push_ctas"] > 0   # the streaming push
    tr.init_particles()
    tr.track(turns)
    rec = tr.moments(turns - 1, 1)[0]
    ratio = np.abs(rec[:, 0]) / rec[:, 1]
    assert np.max(ratio) > 2.0, "the instability has not saturated"
    picks = list(np.argsort(ratio)[-6:]) + [0, 389]
    _check(tr, picks, turns - 1)
    tr.close()


def _offset_run(nb, n_mp, nbins=256):
    ring = W.ring_r0()
    return W.Run(ring, [dict(W.BROADBAND)], np.arange(nb, dtype=np.int32), np.full(nb, 0.3e-3),
                 np.full(nb, n_mp, np.int64), seed=8, turns=3, precision=W.PREC_MIXED, nbins=nbins)


def _offset_particles(run, rng, off_sigmas=20.0):
    s_t, s_d = 2e-12, 1.3e-4
    tau, dl = [], []
    for m in range(run.nb):
        n = int(run.n_mp[m])
        tau.append(off_sigmas * s_t * (1 if m % 2 else -1) + rng.normal(0.0, s_t, n))
        dl.append(off_sigmas * s_d * (1 if m % 3 else -1) + rng.normal(0.0, s_d, n))
    return tau, dl


@pytest.mark.parametrize("kind", ["streaming", "per-tile", "resident"])
def test_far_off_centre_bunches_keep_their_moments(pkg, kind):
    """Bunches started 20 rms lengths (and 20 rms energy spreads) off
    centre: each turn's recorded moments equal the FP64 recomputation."""
    rng = np.random.default_rng(3)
    if kind == "streaming":
        run = _offset_run(8, 1_500_000)
    elif kind == "per-tile":
        run = _offset_run(6, 50_003)
    else:
        run = _offset_run(1, 12_000)
    tr = pkg.tracker_for_run(run, record_turns=16)
    if kind == "streaming":
        assert tr.info["push_ctas"] > 0
    elif kind == "per-tile":
        assert tr.info["push_ctas"] == 0
    else:
        C, per = tr.resident_shape()
        assert C > 0
    tau, dl = _offset_particles(run, rng)
    tr.set_particles_all(np.concatenate(tau), np.concatenate(dl))
    for turn in range(3):
        if kind == "resident":
            tr.track_resident(1)
        else:
            tr.track(1)
        tr.sync()
        _check(tr, range(run.nb), turn)
    tr.close()
