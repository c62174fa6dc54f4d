"""rgm_residual_noalloc: the allocation-free residual check, for callers that
cannot allocate device memory and so cannot create a solver.  Its output is
checked against the existing entry points (rgm_solve's true residual and
rgm_spmv) on two calls in a row that share the static scratch.  This file is
collected last so that a run stopping at the first failure has run every other
test first; it also passes alone in a fresh process."""
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


def test_residual_noalloc_matches_existing_entry_points(rg):
    import torch
    n = 20011
    rp, col, val = synth.random_csr(n, 12, 91, diag=6.0, min_per_row=3)
    b = synth.random_vector(n, 92)
    s = rg.Solver(n, m=20, k=0, mode="plain", rtol=1e-10)
    s.set_operator_csr(rp, col, val)
    x_sol, st = s.solve(b)                                   # existing entry point
    x_rand = synth.random_vector(n, 93)
    dev = torch.device("cuda")
    t = lambda a, dt: torch.tensor(a, dtype=dt, device=dev)
    drp, dcol, dval, db = t(rp, torch.int64), t(col, torch.int32), t(val, torch.float64), t(b, torch.float64)
    r = torch.empty(n, dtype=torch.float64, device=dev)
    norms = torch.empty(2, dtype=torch.float64, device=dev)
    absA = np.abs(val)
    for call, x in enumerate((x_sol, x_rand)):              # two calls in a row
        rg.residual_noalloc(drp, dcol, dval, t(x, torch.float64), db, r, norms)
        torch.cuda.synchronize()
        r_ref = b - s.spmv(x)                                 # existing entry point
        scale = np.abs(b) + synth_abs_spmv(rp, col, absA, np.abs(x))
        assert np.all(np.abs(r.cpu().numpy() - r_ref) <= 1e-14 * scale), call
        nr, nb = norms.cpu().numpy()
        # r is a difference of large numbers: compare at the scale of |b| + |A||x|
        assert abs(nb - np.linalg.norm(b)) <= 1e-13 * np.linalg.norm(b)
        assert abs(nr - np.linalg.norm(r_ref)) <= 1e-14 * np.linalg.norm(scale)
        if call == 0:
            assert st["true_relres"] <= 1e-10
            assert abs(nr / nb - st["true_relres"]) <= 1e-14 * np.linalg.norm(scale) / nb
    s.close()


def test_residual_noalloc_rejects_oversize(rg):
    import torch
    from paper_1807_09467_gb300 import _lib
    dummy = torch.zeros(4, dtype=torch.float64, device="cuda")
    import ctypes as C
    p = C.c_void_p(dummy.data_ptr())
    rc = _lib.load().rgm_residual_noalloc(_lib.RGM_NOALLOC_MAX_ROWS + 1, p, p, p, p, p, None, p, None)
    assert rc == _lib.RGM_E_ARG


def synth_abs_spmv(rp, col, aval, ax):
    y = np.zeros(len(rp) - 1)
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    np.add.at(y, rows, aval * ax[col])
    return y
