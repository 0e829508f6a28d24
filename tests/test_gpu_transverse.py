"""Transverse plane (Eqs. 3-5 x lines, Eq. 6 second line) on the GPU, through
the C ABI, against the FP64 oracle and the transverse coupled-bunch growth
rate -(I_b M beta / (2 E0 T0)) sum_p Re Z((pM + mu) w0 + w_beta)."""
import math

import numpy as np
import pytest

import mbt_workloads as W

pytestmark = pytest.mark.gpu

TRES = dict(Rs_ohm=2e5, fr_Hz=1.5e9, Q=2e4, range=W.RANGE_BOTH)
BBT = dict(Rs_ohm=5e5, fr_Hz=8e9, Q=1.0, range=W.RANGE_SHORT)


@pytest.fixture(scope="module")
def pkg():
    import paper_1809_00391_gb300 as p
    p.build()
    return p


def _plane(**kw):
    t = dict(beta_m=10.0, alpha=0.4, tune=0.31, chromaticity=1.5, emittance_m=1e-9, resonators=[])
    t.update(kw)
    return t


def _run(precision, buckets, n_mp, turns, I=1e-3, tplane=None, res=(W.BROADBAND,), flags=0, seed=5):
    b, c, n = W._fill(buckets, I, n_mp)
    return W.Run(W.ring_r0(), [dict(r) for r in res], b, c, n, seed=seed, turns=turns, precision=precision,
                 flags=flags, transverse=tplane or _plane(), name="transverse")


def _oracle(oracle_mod, run):
    return oracle_mod.OracleSim(run.ring, run.resonators, run.nbins, run.half_width_sigmas, run.buckets,
                                run.currents_A, run.n_mp, run.seed, run.flags, transverse=run.transverse)


def _rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


@pytest.mark.parametrize("wakes", [False, True], ids=["no_wake", "wakes"])
def test_f64_transverse_matches_oracle(pkg, oracle_mod, wakes):
    tplane = _plane(resonators=[dict(TRES), dict(BBT)] if wakes else [])
    run = _run(W.PREC_F64, [0, 1, 7] if wakes else [0], 4000, 150, I=2e-3, tplane=tplane)
    tr = pkg.tracker_for_run(run, record_turns=run.turns)
    orc = _oracle(oracle_mod, run)
    tr.init_particles()
    orc.init_particles()
    for m in range(run.nb):   # the same start on both sides
        assert _rel(tr.transverse_particles(m)[0], orc.tparticles(m)[0]) < 1e-15
    tr.track(run.turns)
    rec_o, trec_o = orc.track2(run.turns)
    trec_g = tr.transverse_moments(0, run.turns)
    h_g, _ = tr.histograms()
    h_o, _ = orc.histograms()
    assert np.array_equal(h_g, h_o)
    # the FP64 path takes the oracle's steps: after 150 turns coordinates and
    # moments agree to ~1e-14 (measured: 3e-15 to 1e-14), well inside 1e-12
    for m in range(run.nb):
        xg, pg = tr.transverse_particles(m)
        xo, po = orc.tparticles(m)
        assert _rel(xg, xo) < 1e-12 and _rel(pg, po) < 1e-12, m
        tg, dg = tr.particles(m)
        to, do = orc.particles(m)
        assert _rel(tg, to) < 1e-12 and _rel(dg, do) < 1e-12, m
    for col in range(4):
        assert _rel(trec_g[:, :, col], trec_o[:, :, col]) < 1e-12, col
    if wakes:
        dip, v = tr.transverse_wake()
        assert _rel(dip, orc.dipoles()) < 1e-12
        q = run.currents_A[0] * run.ring["T0_s"] / run.n_mp[0]
        for m in range(run.nb):
            assert _rel(v[m], orc.vt_direct(dip[m], q)) < 1e-12
    tr.close()


def test_mixed_transverse_matches_oracle(pkg, oracle_mod):
    run = _run(W.PREC_MIXED, [0, 1, 7], 20_000, 300, I=2e-3, tplane=_plane(resonators=[dict(TRES), dict(BBT)]))
    tr = pkg.tracker_for_run(run, record_turns=run.turns)
    orc = _oracle(oracle_mod, run)
    tr.init_particles()
    orc.init_particles()
    tr.track(run.turns)
    rec_o, trec_o = orc.track2(run.turns)
    rec_g = tr.moments(0, run.turns)
    trec_g = tr.transverse_moments(0, run.turns)
    st, sd = rec_o[:, :, 1], rec_o[:, :, 3]
    for col, scale in ((0, st), (1, st), (2, sd), (3, sd)):
        assert np.max(np.abs(rec_g[:, :, col] - rec_o[:, :, col]) / scale) <= 1e-3, col
    sx, sp = trec_o[:, :, 1], trec_o[:, :, 3]
    for col, scale in ((0, sx), (1, sx), (2, sp), (3, sp)):
        assert np.max(np.abs(trec_g[:, :, col] - trec_o[:, :, col]) / scale) <= 1e-3, col
    # the transverse voltage of the GPU's own dipole sums
    dip, v = tr.transverse_wake()
    q = run.currents_A[0] * run.ring["T0_s"] / run.n_mp[0]
    for m in range(run.nb):
        ref = orc.vt_direct(dip[m], q)
        assert np.max(np.abs(v[m] - ref)) <= 1e-5 * np.max(np.abs(ref))
    tr.close()


def test_mixed_transverse_three_long_range_entries(pkg, oracle_mod):
    """Two longitudinal long-range resonators and a transverse one: three of
    the push's four long-range slots in use (the fourth runs with zero
    coefficients), entries of both planes, against the oracle."""
    hom2 = dict(Rs_ohm=5e5, fr_Hz=2.2e9, Q=1e4, range=W.RANGE_LONG)
    run = _run(W.PREC_MIXED, [0, 1, 7], 20_000, 200, I=2e-3, tplane=_plane(resonators=[dict(TRES), dict(BBT)]),
               res=(W.BROADBAND, W.HOM, hom2))
    tr = pkg.tracker_for_run(run, record_turns=run.turns)
    orc = _oracle(oracle_mod, run)
    tr.init_particles()
    orc.init_particles()
    tr.track(run.turns)
    rec_o, trec_o = orc.track2(run.turns)
    rec_g = tr.moments(0, run.turns)
    trec_g = tr.transverse_moments(0, run.turns)
    st, sd = rec_o[:, :, 1], rec_o[:, :, 3]
    for col, scale in ((0, st), (1, st), (2, sd), (3, sd)):
        assert np.max(np.abs(rec_g[:, :, col] - rec_o[:, :, col]) / scale) <= 1e-3, col
    sx, sp = trec_o[:, :, 1], trec_o[:, :, 3]
    for col, scale in ((0, sx), (1, sx), (2, sp), (3, sp)):
        assert np.max(np.abs(trec_g[:, :, col] - trec_o[:, :, col]) / scale) <= 1e-3, col
    tr.close()


@pytest.mark.parametrize("prec", [W.PREC_MIXED, W.PREC_F64], ids=["mixed", "f64"])
def test_transverse_coupled_bunch_growth_rate(pkg, prec):
    ring = W.ring_r0()
    T0, h = ring["T0_s"], ring["h"]
    M, nu, beta, Ib, Rs, Q = 4, 0.3, 20.0, 5e-3, 1.2e7, 2e4
    w0 = 2 * math.pi / T0
    fr = (1441 - nu) / T0
    tplane = dict(beta_m=beta, alpha=0.0, tune=nu, chromaticity=0.0, emittance_m=0.0,
                  resonators=[dict(Rs_ohm=Rs, fr_Hz=fr, Q=Q, range=W.RANGE_LONG)])
    n_mp, turns = 400, 3000
    b, c, n = W._fill([m * (h // M) for m in range(M)], Ib, n_mp)
    run = W.Run(ring, [], b, c, n, seed=4, turns=turns, precision=prec, flags=W.NO_SR, transverse=tplane)
    tr = pkg.tracker_for_run(run, record_turns=turns)
    g = np.random.default_rng(8)
    for m in range(M):
        tr.set_particles(m, g.normal(0, 3e-12, n_mp), np.zeros(n_mp))
        ph = g.uniform(0, 2 * math.pi)
        tr.set_transverse_particles(m, np.full(n_mp, 1e-6 * math.cos(ph)), np.full(n_mp, -1e-6 / beta * math.sin(ph)))
    tr.track(turns)
    trec = tr.transverse_moments(0, turns)
    z = trec[:, :, 0] / math.sqrt(beta) - 1j * math.sqrt(beta) * trec[:, :, 2]
    th = (2 * math.pi * nu + 2 * math.pi * 3) / M
    X3 = (z * np.exp(-1j * th * np.arange(M))[None, :]).sum(axis=1)
    rate = np.polyfit(np.arange(1000, turns), np.log(np.abs(X3[1000:])), 1)[0] / T0
    wr = 2 * math.pi * fr
    p = np.arange(-2000, 2000)
    lines = (p * M + 3 + nu) * w0
    re_z = ((wr / lines) * Rs / (1 + 1j * Q * (lines / wr - wr / lines))).real
    pred = -(Ib * M * beta / (2 * ring["E0_eV"] * T0)) * np.sum(re_z)
    assert rate == pytest.approx(pred, rel=0.02)
    tr.close()


def test_transverse_checkpoint_resume_is_bit_identical(pkg):
    run = _run(W.PREC_F64, [0, 3], 3000, 40, tplane=_plane(resonators=[dict(TRES)]))
    a = pkg.tracker_for_run(run, record_turns=run.turns)
    a.init_particles()
    a.track(20)
    blob = a.save_state()
    a.track(20)
    b = pkg.tracker_for_run(run, record_turns=run.turns)
    b.load_state(blob)
    b.track(20)
    for m in range(run.nb):
        xa, pa = a.transverse_particles(m)
        xb, pb = b.transverse_particles(m)
        assert np.array_equal(xa, xb) and np.array_equal(pa, pb)
    a.close()
    b.close()


def test_transverse_batch_equals_alone_and_resident_refuses(pkg):
    tr_run = _run(W.PREC_MIXED, [0, 5], 8000, 30, tplane=_plane(resonators=[dict(TRES)]))
    lo_run = W.single_bunch(seed=2).scaled(turns=30)
    lo_run = W.Run(**{**lo_run.__dict__, "precision": W.PREC_MIXED})
    alone = pkg.tracker_for_run(tr_run, record_turns=30)
    alone.init_particles()
    alone.track(30)
    t1 = pkg.tracker_for_run(tr_run, record_turns=30)
    t2 = pkg.tracker_for_run(lo_run, record_turns=30)
    t1.init_particles()
    t2.init_particles()
    bt = pkg.Batch([t1, t2])
    bt.track(30)
    bt.sync()
    assert np.array_equal(t1.transverse_moments(0, 30), alone.transverse_moments(0, 30))
    with pytest.raises(pkg.MBTError):
        alone.track_resident(1)
    bt.close()
    for t in (alone, t1, t2):
        t.close()


@pytest.mark.parametrize("prec,tol", [(W.PREC_F64, 1e-12), (W.PREC_MIXED, 1e-3)], ids=["f64", "mixed"])
def test_transverse_resistive_wall_matches_oracle(pkg, oracle_mod, prec, tol):
    """Long-range transverse resistive wall on bunch centroids (a copper pipe
    of 5 mm radius around the ring, 20 turns of history), five offset bunches
    of 5 mA, against the oracle: transverse moments of every turn; the same
    start without the wall moves differently (by ~1.8 sigma_x)."""
    rw = dict(radius_m=0.005, conductivity_S_per_m=5.8e7, length_m=288.0, history_turns=20)
    run = _run(prec, [0, 1, 2, 100, 300], 4000, 120, I=5e-3, tplane=_plane(resistive_wall=[rw]), res=())

    def offsets(sim_set, sim_get):
        g = np.random.default_rng(3)
        for m in range(run.nb):
            x, xp = sim_get(m)
            sim_set(m, x + g.normal(0, 2e-4), xp)

    tr = pkg.tracker_for_run(run, record_turns=run.turns)
    orc = _oracle(oracle_mod, run)
    plain = _oracle(oracle_mod, W.Run(**{**run.__dict__, "transverse": _plane()}))
    tr.init_particles()
    orc.init_particles()
    plain.init_particles()
    offsets(orc.set_tparticles, orc.tparticles)
    offsets(plain.set_tparticles, plain.tparticles)
    for m in range(run.nb):
        tr.set_transverse_particles(m, *orc.tparticles(m))
    tr.track(run.turns)
    _, trec_o = orc.track2(run.turns)
    _, trec_p = plain.track2(run.turns)
    trec_g = tr.transverse_moments(0, run.turns)
    sx, sp = trec_o[:, :, 1], trec_o[:, :, 3]
    assert np.max(np.abs(trec_p[:, :, 0] - trec_o[:, :, 0]) / sx) > 20 * 1e-3   # the wall matters
    if prec == W.PREC_F64:
        for col in range(4):
            assert _rel(trec_g[:, :, col], trec_o[:, :, col]) < tol, col
    else:
        for col, scale in ((0, sx), (2, sp)):
            assert np.max(np.abs(trec_g[:, :, col] - trec_o[:, :, col]) / scale) <= tol, col
    tr.close()


def _dip_unit(tplane):
    """The mixed push's fixed-point dipole unit u = 2^(e - 20) m and accepted
    range 2^(e + 10) m, 2^e the beam size sqrt(beta emit) rounded up to a power
    of two (at least 2^-16 m)."""
    sx = math.sqrt(tplane["beta_m"] * tplane["emittance_m"])
    e = max(-16, math.ceil(math.log2(sx))) if sx > 0 else -16
    return 2.0 ** (e - 20), 2.0 ** (e + 10)


def test_mixed_dipole_deposit_sums_every_cell(pkg):
    """After one turn the dipole sums of the mixed push equal the per-cell sums
    of x of the GPU's own particles, to u/2 per particle (the fixed-point
    quantisation) and one FP32 rounding of the sum: one tile of 65536
    particles, half of them in one cell (the most one cell of a tile can take),
    x of both signs up to half the accepted range, and particles outside the
    mesh, which deposit into no cell."""
    n = 65536
    tplane = _plane(alpha=0.0)   # x1 = cos(mu) x0 + excitation: |x1| stays within the range
    u, rng = _dip_unit(tplane)
    run = _run(W.PREC_MIXED, [0], n, 1, tplane=tplane, res=(), flags=W.NO_SR | W.NO_QE)
    tr = pkg.tracker_for_run(run, record_turns=2)
    tr.set_tile(n)
    info = tr.info
    H, D, nb = info["half_width_s"], info["bin_width_s"], run.nbins
    g = np.random.default_rng(3)
    k = np.where(np.arange(n) < n // 2, 100, g.integers(0, nb, n))
    tau = -H + (k + 0.5) * D   # cell centres: the turn moves tau by far less than a cell
    tau[-64:] = H + 3 * D * (1 + np.arange(64))
    tr.set_particles(0, tau, np.zeros(n))
    tr.set_transverse_particles(0, g.uniform(-0.5 * rng, 0.5 * rng, n), np.zeros(n))
    tr.track(1)
    t1, _ = tr.particles(0)
    x1, _ = tr.transverse_particles(0)
    dip, _ = tr.transverse_wake()
    cell = np.floor((t1 + H) / D).astype(np.int64)
    inside = (cell >= 0) & (cell < nb)
    assert inside.sum() == n - 64
    ref = np.bincount(cell[inside], weights=x1[inside], minlength=nb)
    cnt = np.bincount(cell[inside], minlength=nb)
    assert cnt[100] >= n // 2
    tol = cnt * u / 2 + 2.0 ** -23 * np.abs(ref)
    assert np.all(np.abs(dip[0] - ref) <= tol), np.max(np.abs(dip[0] - ref) / np.maximum(tol, 1e-300))
    tr.close()


def test_mixed_dipole_range_is_reported(pkg):
    """A transverse coordinate beyond the fixed-point dipole range makes the
    mixed push report MBT_ERR_UNSUPPORTED at the next synchronising call; the
    context stays usable."""
    tplane = _plane()
    _, rng = _dip_unit(tplane)
    run = _run(W.PREC_MIXED, [0], 4096, 4, tplane=tplane, res=())
    tr = pkg.tracker_for_run(run, record_turns=4)
    tr.init_particles()
    x, xp = tr.transverse_particles(0)
    tr.track(1)
    tr.sync()
    x, xp = tr.transverse_particles(0)
    # eight particles on the betatron ellipse of amplitude sqrt(beta J) = 4
    # x the range: whatever the phase advance, at least one of them ends the
    # turn beyond the range (|x| >= 4 cos(pi / 8) x the range)
    beta, alpha = tplane["beta_m"], tplane["alpha"]
    a = 4 * rng
    ph = np.arange(8) * (math.pi / 4)
    x0, xp0 = x.copy(), xp.copy()
    x[7:15] = a * np.cos(ph)
    xp[7:15] = -(a / beta) * (np.sin(ph) + alpha * np.cos(ph))
    tr.set_transverse_particles(0, x, xp)
    tr.track(1)
    with pytest.raises(pkg.MBTError) as e:
        tr.sync()
    assert e.value.status == 6
    tr.set_transverse_particles(0, x0, xp0)
    tr.track(1)
    tr.sync()
    tr.close()


def test_mixed_transverse_multi_tile_bunches(pkg, oracle_mod):
    """Bunches that span several push tiles: 24 bunches of ~8e4
    macro-particles (ragged sizes, ten tiles each) with a longitudinal and a
    transverse long-range resonator against the oracle over 30 turns (moments
    of both planes 1e-3 of the rms, counts exact in total); and, since the
    tiles add their dipole sums into the bunch's sums exactly (integers), the
    same run in a batch with another large run gives its particles and
    moments of both planes bit for bit."""
    ring = W.ring_r0()
    buckets = np.array([0, 1, 2, 3, 5, 8, 13, 21, 34, 55, 89, 144, 150, 160, 170, 180, 200, 220, 240, 260, 280, 300,
                        320, 340], np.int32)
    n = np.full(buckets.size, 80_000, np.int64)
    n[3], n[10], n[17] = 80_001, 79_998, 80_003
    c = np.full(buckets.size, 1.5e-3)
    tplane = _plane(resonators=[dict(TRES), dict(BBT)])
    run = W.Run(ring, [dict(W.BROADBAND), dict(W.HOM)], buckets, c, n, seed=23, turns=30, precision=W.PREC_MIXED,
                transverse=tplane, name="transverse, multi-tile bunches")
    tr = pkg.tracker_for_run(run, record_turns=run.turns)
    tr.init_particles()
    tr.track(run.turns)
    rec_g = tr.moments(0, run.turns)
    trec_g = tr.transverse_moments(0, run.turns)
    h, out = tr.histograms()
    assert h.sum() + out.sum() == n.sum()
    orc = _oracle(oracle_mod, run)
    orc.init_particles()
    rec_o, trec_o = orc.track2(run.turns)
    st, sd = rec_o[:, :, 1], rec_o[:, :, 3]
    for col, scale in ((0, st), (1, st), (2, sd), (3, sd)):
        assert np.max(np.abs(rec_g[:, :, col] - rec_o[:, :, col]) / scale) <= 1e-3, col
    sx, sp = trec_o[:, :, 1], trec_o[:, :, 3]
    for col, scale in ((0, sx), (1, sx), (2, sp), (3, sp)):
        assert np.max(np.abs(trec_g[:, :, col] - trec_o[:, :, col]) / scale) <= 1e-3, col
    # alone = in a batch with another large transverse run
    other = W.Run(ring, [dict(W.BROADBAND)], buckets[:20], c[:20], np.full(20, 100_000, np.int64), seed=24,
                  turns=30, precision=W.PREC_MIXED, transverse=_plane(resonators=[dict(TRES)]), name="other")
    t1 = pkg.tracker_for_run(run, record_turns=run.turns)
    t2 = pkg.tracker_for_run(other, record_turns=run.turns)
    t1.init_particles()
    t2.init_particles()
    bt = pkg.Batch([t1, t2])
    bt.track(run.turns)
    bt.sync()
    assert np.array_equal(t1.moments(0, run.turns), rec_g)
    assert np.array_equal(t1.transverse_moments(0, run.turns), trec_g)
    for m in (0, 3, 23):
        assert np.array_equal(t1.transverse_particles(m)[0], tr.transverse_particles(m)[0])
        assert np.array_equal(t1.particles(m)[0], tr.particles(m)[0])
    bt.close()
    for t in (tr, t1, t2):
        t.close()
