"""rgm_set_operator_sell: an operator handed over in the library's sliced-ELL
layout gives the same SpMV and solve as the same matrix in CSR, for an
unsorted layout and one sorted by row length inside each 256-row tile; layouts
that break the rules are rejected.  The SpMV reads a slice in 16-byte chunks of
slice columns, so a row's partial sums follow its slice's width: two layouts
of one matrix agree to rounding (the SpMV within a few ulps of the row's
absolute sum, the solve within one iteration and x within 1e-12), not bit for
bit."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rg():
    import __graft_entry__ as g
    g.build()
    import paper_1807_09467_gb300 as rg
    return rg


def _sell_from_csr(rp, col, val, sort):
    """Sliced ELL, 32-row slices, 8 slices per 256-row tile; rows of a tile
    optionally ordered by decreasing length (ties: larger row first)."""
    n = len(rp) - 1
    ntile = (n + 255) // 256
    nslices = ntile * 8
    perm = np.full(nslices * 32, -1, dtype=np.int32)
    for t in range(ntile):
        rows = np.arange(t * 256, min(n, (t + 1) * 256))
        if sort:
            ln = rp[rows + 1] - rp[rows]
            rows = rows[np.lexsort((-rows, -ln))]
        perm[t * 256: t * 256 + len(rows)] = rows
    sp = np.zeros(nslices + 1, dtype=np.int64)
    for q in range(nslices):
        r = perm[q * 32:(q + 1) * 32]
        r = r[r >= 0]
        w = int((rp[r + 1] - rp[r]).max()) if len(r) else 0
        sp[q + 1] = sp[q] + 32 * w
    scol = np.zeros(sp[-1], dtype=np.int32)
    sval = np.zeros(sp[-1])
    for q in range(nslices):
        w = (sp[q + 1] - sp[q]) // 32
        for l in range(32):
            r = perm[q * 32 + l]
            for j in range(w):
                e = sp[q] + 32 * j + l
                if r >= 0 and j < rp[r + 1] - rp[r]:
                    scol[e] = col[rp[r] + j]
                    sval[e] = val[rp[r] + j]
                else:
                    scol[e] = max(r, 0)
    return sp, perm, scol, sval


@pytest.mark.parametrize("sort", [False, True])
def test_sell_matches_csr(rg, sort):
    n, m, k = 3000 + 11, 20, 4
    rp, col, val = synth.random_csr(n, 9, 61, diag=6.0, min_per_row=2)
    b = synth.random_vector(n, 62)
    U = np.linalg.qr(synth.random_matrix(n, k, 63))[0]
    sp, perm, scol, sval = _sell_from_csr(rp, col, val, sort)
    out = []
    for kind in ("csr", "sell"):
        s = rg.Solver(n, m=m, k=k, mode="deflated", rtol=1e-10)
        if kind == "csr":
            s.set_operator_csr(rp, col, val)
        else:
            s.set_operator_sell(sp, perm, scol, sval)
        s.set_recycle_space(U)
        y = s.spmv(synth.random_vector(n, 64))
        x, st = s.solve(b)
        out.append((y, x, st))
        # new values in the operator's own layout
        if kind == "csr":
            s.set_operator_values(2.0 * val)
        else:
            s.set_operator_values(2.0 * sval)
        x2, st2 = s.solve(b)
        out.append((x2, st2))
        s.close()
    (yc, xc, sc), (xc2, sc2), (ys, xs, ss), (xs2, ss2) = out
    xv = synth.random_vector(n, 64)
    absrow = np.zeros(n)
    np.add.at(absrow, np.repeat(np.arange(n), np.diff(rp)), np.abs(val) * np.abs(xv[col]))
    assert np.all(np.abs(yc - ys) <= 4e-16 * 8 * absrow)
    assert abs(sc["iters"] - ss["iters"]) <= 1 and abs(sc2["iters"] - ss2["iters"]) <= 1
    assert np.linalg.norm(xc - xs) <= 1e-12 * np.linalg.norm(xc)
    np.testing.assert_allclose(xs2, 0.5 * xc, rtol=0, atol=1e-9 * np.abs(xc).max())


def test_sell_rejects_bad_layouts(rg):
    n = 600
    rp, col, val = synth.random_csr(n, 5, 70, diag=4.0)
    sp, perm, scol, sval = _sell_from_csr(rp, col, val, True)
    s = rg.Solver(n, m=10, k=0, mode="plain")
    bad = perm.copy(); bad[0], bad[300] = bad[300], bad[0]      # row leaves its tile
    with pytest.raises(rg.RgmError):
        s.set_operator_sell(sp, bad, scol, sval)
    bad = perm.copy(); bad[1] = bad[0]                           # row twice
    with pytest.raises(rg.RgmError):
        s.set_operator_sell(sp, bad, scol, sval)
    bsp = sp.copy(); bsp[1:] += 1                                 # slice size not a multiple of 32
    with pytest.raises(rg.RgmError):
        s.set_operator_sell(bsp, perm, np.r_[scol, 0].astype(np.int32), np.r_[sval, 0.0])
    bcol = scol.copy(); bcol[0] = n                               # column out of range
    with pytest.raises(rg.RgmError):
        s.set_operator_sell(sp, perm, bcol, sval)
    with pytest.raises(rg.RgmError):
        s.set_operator_sell(sp[:-8], perm[:-256], scol, sval)     # wrong slice count
    s.set_operator_sell(sp, perm, scol, sval)                     # the valid one
