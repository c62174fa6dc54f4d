"""The layout the device row gather of the FE assembly relies on (no GPU).

For p <= 4 and a constant velocity the gather finds an entry's column from
its offset in the row instead of reading it: the columns of an interior row
are the product of its two 1D coupling ranges clipped to the interior nodes,
in y-major order, and k / wx is taken as (k + 1/2) * (1 / wx) in binary32.
Both facts are checked here against the oracle's element-connectivity pattern
(itself pinned by brute force), with the same binary32 arithmetic.
"""
import numpy as np
import pytest


def _crange(I, p, L):
    lo, hi = (I - p, I + p) if I % p == 0 else (I // p * p, I // p * p + p)
    return max(lo, 1), min(hi, L - 2)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("N", [1, 2, 3, 6])
def test_interior_rows_are_clipped_range_products(orc, p, N):
    L = p * N + 1
    rp, col = orc.pattern(p, N, True)
    for row in range(L * L):
        Iy, Ix = divmod(row, L)
        e0, e1 = int(rp[row]), int(rp[row + 1])
        if Ix in (0, L - 1) or Iy in (0, L - 1):
            assert e1 - e0 == 1 and col[e0] == row
            continue
        xl, xh = _crange(Ix, p, L)
        yl, yh = _crange(Iy, p, L)
        wx = xh - xl + 1
        assert e1 - e0 == wx * (yh - yl + 1) <= (2 * p + 1) ** 2
        rwx = np.float32(1.0) / np.float32(wx)
        k = np.arange(e1 - e0, dtype=np.float32)
        dy = ((k + np.float32(0.5)) * rwx).astype(np.int64)
        np.testing.assert_array_equal(dy, np.arange(e1 - e0) // wx)
        jx = xl + np.arange(e1 - e0) - dy * wx
        np.testing.assert_array_equal(col[e0:e1], (yl + dy) * L + jx)
