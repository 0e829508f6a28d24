"""Host-side planning of the streaming push (no GPU): the work split of a
fill over the push CTAs and the choice between the streaming and the per-tile
push.  The split must give every particle of every bunch to exactly one tile,
start every tile at a multiple of 4 (the push loads particles as aligned
quads), cut each run into equal shares at multiples of 4, and cut a run the
same way alone and in a batch (so its moment sums keep their order)."""
import numpy as np
import pytest

STAGE = 3968   # particles per stage of the streaming push


@pytest.fixture(scope="module")
def pkg():
    import paper_1809_00391_gb300 as p
    p.build()
    return p


def _padded(n):
    return (np.asarray(n, np.int64) + 3) // 4 * 4


def _shares(P, G):
    """Share boundaries of a run of padded length P over G CTAs, from the
    documented definition."""
    q = P // 4
    a = [q * g // G * 4 for g in range(G)]
    e = [q * (g + 1) // G * 4 for g in range(G - 1)] + [P]
    return a, e


def _check_split(run, n_mp, G, tiles):
    run = np.asarray(run)
    n_mp = np.asarray(n_mp, np.int64)
    # bunch order, and each bunch covered exactly once in consecutive tiles
    assert np.all(np.diff(tiles[:, 0]) >= 0)
    for m in range(len(n_mp)):
        t = tiles[tiles[:, 0] == m]
        assert len(t) >= 1, f"bunch {m} has no tile"
        assert t[0, 1] == 0 and t[-1, 1] + t[-1, 2] == n_mp[m], f"bunch {m}"
        assert np.all(t[1:, 1] == t[:-1, 1] + t[:-1, 2]), f"bunch {m}: gap or overlap"
    assert np.all(tiles[:, 1] % 4 == 0)
    assert np.all(tiles[:, 2] >= 1)
    assert np.all((tiles[:, 3] >= 0) & (tiles[:, 3] < G))
    # every tile inside its CTA's share of its run's padded sequence
    for r in np.unique(run):
        idx = np.flatnonzero(run == r)
        pad = _padded(n_mp[idx])
        start = dict(zip(idx, np.concatenate([[0], np.cumsum(pad)[:-1]])))
        a, e = _shares(int(pad.sum()), G)
        sel = np.isin(tiles[:, 0], idx)
        for b, s, c, g in tiles[sel]:
            p0 = start[b] + s
            assert a[g] <= p0 and p0 + c <= e[g], (b, s, c, g)
        # CTAs in order along the run
        assert np.all(np.diff(tiles[sel, 3]) >= 0)
        # shares of the padded sequence differ by at most one quad
        lens = np.array(e) - np.array(a)
        assert lens.max() - lens.min() <= 4


@pytest.mark.parametrize("G", [1, 3, 152])
def test_split_of_a_fill_with_ragged_and_tiny_bunches(pkg, G):
    n = [1_300_000, 37, 1, 1_300_003, 1001, 4, 5, 99_999]
    run = [0] * len(n)
    t = pkg.stream_split(run, n, G)
    _check_split(run, n, G, t)


def test_split_of_seeded_batches(pkg):
    rng = np.random.default_rng(17)
    for _ in range(20):
        nruns = int(rng.integers(1, 5))
        run = np.sort(rng.integers(0, nruns, size=int(rng.integers(1, 60)))).astype(np.int32)
        n = rng.integers(1, 50_000, size=len(run))
        G = int(rng.integers(1, 200))
        _check_split(run, n, G, pkg.stream_split(run, n, G))


def test_a_run_is_cut_the_same_alone_and_in_a_batch(pkg):
    G = 152
    a = np.array([100_000] * 7 + [37, 100_003], np.int64)
    b = np.array([5, 250_000, 1], np.int64)
    alone = pkg.stream_split(np.zeros(len(a), np.int32), a, G)
    batch = pkg.stream_split(np.array([0] * len(b) + [1] * len(a), np.int32), np.concatenate([b, a]), G)
    mine = batch[batch[:, 0] >= len(b)].copy()
    mine[:, 0] -= len(b)
    assert np.array_equal(mine, alone)


def test_one_bunch_one_cta_and_more_ctas_than_quads(pkg):
    t = pkg.stream_split([0], [10], 1)
    assert t.tolist() == [[0, 0, 10, 0]]
    # 3 quads over 8 CTAs: some CTAs get nothing, none gets a partial quad
    t = pkg.stream_split([0], [10], 8)
    _check_split([0], [10], 8, t)
    assert len(t) == 3 and t[:, 2].tolist() == [4, 4, 2]


def test_tiles_are_capped_at_2_pow_28(pkg):
    n = (1 << 29) + 5
    t = pkg.stream_split([0], [n], 1)
    assert t[:, 2].tolist() == [1 << 28, 1 << 28, 5]
    assert t[:, 1].tolist() == [0, 1 << 28, 1 << 29]


def test_invalid_split_arguments(pkg):
    from paper_1809_00391_gb300 import MBTError
    for run, n, G in (([0], [0], 4), ([1, 0], [5, 5], 4), ([0], [5], 0), ([-1], [5], 2)):
        with pytest.raises(MBTError):
            pkg.stream_split(run, n, G)


def test_streaming_choice(pkg):
    G = 152
    big = G * 4 * STAGE   # smallest run with four stages per SM
    assert pkg.plan_streams([big], [big // (2 * STAGE)], False, G)
    assert not pkg.plan_streams([big - 1], [1], False, G)
    # bunches below two stages on average
    assert not pkg.plan_streams([big], [big // (2 * STAGE) + 1], False, G)
    # a transverse plane, or one small run in the batch, selects the per-tile push
    assert not pkg.plan_streams([big], [1], True, G)
    assert not pkg.plan_streams([big, big, 1000], [1, 1, 1], False, G)
    # the 390-bunch fill of 1e5 particles per bunch streams on 152 SMs
    assert pkg.plan_streams([390 * 100_000], [390], False, G)
    from paper_1809_00391_gb300 import MBTError
    with pytest.raises(MBTError):
        pkg.plan_streams([big], [0], False, G)


def _lanes_reference(n, k):
    """Largest first (ties in member order), each into the lane holding the
    fewest particles so far (ties: the lower lane), written from the rule."""
    k = min(k, len(n))
    load = [0] * k
    lane = [None] * len(n)
    for i in sorted(range(len(n)), key=lambda i: (-n[i], i)):
        j = min(range(k), key=lambda j: (load[j], j))
        lane[i] = j
        load[j] += n[i]
    return lane


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_lane_partition_follows_the_rule_and_balances(pkg, seed):
    g = np.random.default_rng(seed)
    n = [int(x) for x in g.integers(1, 10, 37) * 10 ** g.integers(3, 7, 37)]
    for k in (1, 2, 3, 4, 8):
        lane = pkg.plan_lanes(n, k)
        assert lane.tolist() == _lanes_reference(n, k)
        loads = np.bincount(lane, weights=n, minlength=min(k, len(n)))
        assert set(lane.tolist()) == set(range(min(k, len(n))))   # no lane left empty
        # greedy bound: no lane exceeds the mean by more than the largest member
        assert loads.max() <= np.sum(n) / len(loads) + max(n)


def test_lane_partition_edges(pkg):
    assert pkg.plan_lanes([5, 5, 5], 8).tolist() == [0, 1, 2]   # more lanes than members
    assert pkg.plan_lanes([1, 2, 3, 4], 1).tolist() == [0, 0, 0, 0]
    assert pkg.plan_lanes([0, 0, 7], 2).tolist() == [1, 1, 0]
    for bad in (([], 2), ([1, 2], 0), ([1, 2], 9), ([1, -1], 2)):
        with pytest.raises(pkg.MBTError):
            pkg.plan_lanes(*bad)
