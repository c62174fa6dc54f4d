"""Host logic of the launch-shape autotuner (no GPU)."""
import pytest

from paper_1807_09467_gb300 import tune


def test_tiles_per_block_caps_blocks():
    # 1,050,625 rows = 4,104 tiles
    n = 1050625
    assert tune.tiles_per_block(n, None) == 0
    for cap in (1, 76, 152, 304, 608, 4104, 10000):
        tpb = tune.tiles_per_block(n, cap)
        nb = tune.blocks(n, tpb, 608)
        assert nb <= cap and (tpb == 1 or tune.blocks(n, tpb - 1, 608) > cap)
    # the automatic choice: at most 608 blocks of whole tiles
    assert tune.blocks(n, 0, 608) == 587
    assert tune.blocks(1089, 0, 608) == 5 and tune.tiles_per_block(1089, 608) == 1


def test_tune_picks_fastest_and_keeps_order_on_ties():
    calls = []

    def trial(c):
        calls.append(c)
        return {None: 5.0, 304: 3.0, 152: 3.0, 76: 4.0}[c]
    best, times = tune.tune(trial, [None, 304, 152, 76], repeats=2)
    assert best == 304 and times[152] == 3.0 and len(calls) == 8
    best, _ = tune.tune(lambda c: 1.0, [None, 304])
    assert best is None
    with pytest.raises(ValueError):
        tune.tune(lambda c: float("nan"), [None])
    with pytest.raises(ValueError):
        tune.tune(lambda c: 1.0, [])


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("N", [1, 2, 3, 7])
def test_serve_pattern_sizes_match_the_oracle_pattern(orc, p, N):
    # the admission estimate's (n, nnz) of a Q_p Dirichlet pattern, against the
    # oracle's element-connectivity pattern (itself pinned by brute force)
    from paper_1807_09467_gb300 import serve
    rp, col = orc.pattern(p, N, True)
    assert serve.sizes(p, N) == (len(rp) - 1, int(rp[-1]))
