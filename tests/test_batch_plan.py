"""rgm_batch_plan, the host-side block plan of a batched cycle launch
(rgm_batch_solve with RGM_BATCH_COOP), on the CPU: waves never exceed the
resident capacity, every system keeps at least one block and never more than
it asked for, systems that all fit keep their own partition, shares follow the
work per Arnoldi step, and the plan is a function of its inputs alone."""
import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def rg():
    from paper_1807_09467_gb300 import build
    build.build()
    import paper_1807_09467_gb300 as rg
    return rg


def _own_blocks(n, nsm=152):
    """The partition a handle uses alone: whole 256-row tiles, at most 4 blocks per SM."""
    ntile = -(-n // 256)
    nb = max(1, min(ntile, 4 * nsm))
    tpb = -(-ntile // nb)
    return -(-n // (tpb * 256))


def _check(rg, n, nnz, nd, cap):
    want = [_own_blocks(x) for x in n]
    blocks, rpb, wave, nw = rg.batch_plan(n, nnz, nd, want, cap)
    k = len(n)
    assert nw == (-(-k // cap) if k else 0)
    for w in range(nw):
        idx = np.nonzero(wave == w)[0]
        assert len(idx) and np.all(np.diff(idx) == 1) and len(idx) <= cap   # consecutive systems
        assert blocks[idx].sum() <= cap
        if sum(want[i] for i in idx) <= cap:
            assert np.all(rpb[idx] == 0) and all(blocks[i] == want[i] for i in idx)
    for i in range(k):
        assert 1 <= blocks[i] <= want[i]
        if rpb[i]:
            assert rpb[i] % 256 == 0 and blocks[i] == -(-n[i] // rpb[i])      # whole tiles, all rows
        else:
            assert blocks[i] == want[i]
    return blocks, rpb, wave


def test_small_systems_keep_their_partition(rg):
    n = [1089, 4225, 16641, 2209]
    _, rpb, _ = _check(rg, n, [9 * x for x in n], [39] * 4, 608)
    assert np.all(rpb == 0)


def test_large_systems_share_in_proportion_to_work(rg):
    n = [300001, 250000, 200003, 320000]
    nnz = [9 * x for x in n]
    nd = [29, 21, 21, 27]
    blocks, rpb, _ = _check(rg, n, nnz, nd, 608)
    assert np.all(rpb > 0) and blocks.sum() <= 608
    w = np.array(nnz, dtype=float) + np.array(n, dtype=float) * np.array(nd)
    # more work, no fewer blocks (up to the rounding to whole tiles)
    order = np.argsort(w)
    assert np.all(np.diff(blocks[order]) >= -1)


def test_more_systems_than_resident_blocks_run_in_waves(rg):
    rng = np.random.default_rng(5)
    n = [int(x) for x in rng.integers(300, 200000, 700)]
    _check(rg, n, [17 * x for x in n], [int(x) for x in rng.integers(3, 98, 700)], 608)
    blocks, rpb, wave = _check(rg, n[:20], [17 * x for x in n[:20]], [30] * 20, 8)
    assert wave.max() == 2


def test_uneven_batch_like_batch64(rg):
    seqs = synth.batch_sequences(64)
    n = [w.n for w, _, _ in seqs]
    nnz = [25 * x for x in n]
    a = _check(rg, n, nnz, [39] * 64, 608)
    b = _check(rg, n, nnz, [39] * 64, 608)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_rejects_bad_input(rg):
    with pytest.raises(rg.RgmError):
        rg.batch_plan([100], [900], [3], [1], 0)
    with pytest.raises(rg.RgmError):
        rg.batch_plan([0], [900], [3], [1], 8)
    with pytest.raises(rg.RgmError):
        rg.batch_plan([100], [900], [3], [0], 8)
    assert rg.batch_plan([], [], [], [], 8)[3] == 0
