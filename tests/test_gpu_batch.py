"""rgm_batch_solve: independent systems of different sizes and modes solved
concurrently on their own streams give exactly what each gives alone (same
code path, one launch per pass), and errors are reported per batch.  With
batched cycle launches (coop=True) each system converges as it does alone, to
its solution up to the rounding of its dot-product partition."""
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


def _systems():
    out = []
    for i, (n, mode, k) in enumerate([(1089, "deflated", 4), (5000, "plain", 0), (20001, "augmented", 6),
                                      (66049, "deflated", 8), (3000, "deflated", 3), (777, "plain", 0),
                                      (40000, "deflated", 8), (12345, "augmented", 5)]):
        rp, col, val = synth.random_csr(n, 9, 300 + i, diag=6.0, min_per_row=2)
        b = synth.random_vector(n, 400 + i)
        U = np.linalg.qr(synth.random_matrix(n, k, 500 + i))[0] if k else None
        out.append((n, mode, k, rp, col, val, b, U))
    return out


def _make(rg, torch, sysdef, stream):
    n, mode, k, rp, col, val, b, U = sysdef
    s = rg.Solver(n, m=20, k=max(k, 1), mode=mode, rtol=1e-10, launch_policy="per_pass",
                  stream=stream.cuda_stream if stream is not None else None)
    s.set_operator_csr(rp, col, val)
    if U is not None:
        s.set_recycle_space(U)
    return s


def test_batch_equals_alone(rg):
    import torch
    defs = _systems()
    alone = []
    for d in defs:
        s = _make(rg, torch, d, None)
        x = torch.zeros(d[0], dtype=torch.float64, device="cuda")
        _, st = s.solve(torch.tensor(d[6], device="cuda"), x)
        alone.append((x.cpu().numpy(), st))
        s.close()
    streams = [torch.cuda.Stream() for _ in defs]
    solvers = [_make(rg, torch, d, st) for d, st in zip(defs, streams)]
    bs = [torch.tensor(d[6], device="cuda") for d in defs]
    xs = [torch.zeros(d[0], dtype=torch.float64, device="cuda") for d in defs]
    torch.cuda.synchronize()
    stats = rg.batch_solve(solvers, bs, xs)
    torch.cuda.synchronize()
    for (xa, sa), x, sb in zip(alone, xs, stats):
        assert sb["status"] == 0 and sb["iters"] == sa["iters"] and sb["true_relres"] <= 1e-10
        np.testing.assert_array_equal(x.cpu().numpy(), xa)
    # the same again (handles are reusable after a batch), auto policy inside a batch
    for s in solvers:
        s.close()


def test_batch_rejects_duplicates(rg):
    import torch
    d = _systems()[0]
    s = _make(rg, torch, d, None)
    b = torch.tensor(d[6], device="cuda")
    x = torch.zeros(d[0], dtype=torch.float64, device="cuda")
    with pytest.raises(rg.RgmError):
        rg.batch_solve([s, s], [b, b], [x, x.clone()])
    assert rg.batch_solve([], [], []) == []


# ------------------------------------------------------------ batched cycle launches
def _make_auto(rg, sysdef, stream, precision="fp64"):
    n, mode, k, rp, col, val, b, U = sysdef
    s = rg.Solver(n, m=20, k=max(k, 1), mode=mode, rtol=1e-10, precision=precision,
                  stream=stream.cuda_stream if stream is not None else None)
    s.set_operator_csr(rp, col, val)
    if U is not None:
        s.set_recycle_space(U)
    return s


def _coop_round(rg, torch, defs, coop=True, precisions=None):
    precisions = precisions or ["fp64"] * len(defs)
    streams = [torch.cuda.Stream() for _ in defs]
    solvers = [_make_auto(rg, d, st, p) for d, st, p in zip(defs, streams, precisions)]
    bs = [torch.tensor(d[6], device="cuda") for d in defs]
    xs = [torch.zeros(d[0], dtype=torch.float64, device="cuda") for d in defs]
    torch.cuda.synchronize()
    stats = rg.batch_solve(solvers, bs, xs, coop=coop)
    torch.cuda.synchronize()
    for s in solvers:
        s.close()
    return [x.cpu().numpy() for x in xs], stats


def _alone(rg, torch, defs, precisions=None):
    precisions = precisions or ["fp64"] * len(defs)
    out = []
    for d, p in zip(defs, precisions):
        s = _make_auto(rg, d, None, p)
        x = torch.zeros(d[0], dtype=torch.float64, device="cuda")
        _, st = s.solve(torch.tensor(d[6], device="cuda"), x)
        out.append((x.cpu().numpy(), st))
        s.close()
    return out


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_coop_batch_matches_alone(rg):
    """Uneven systems (sizes, modes, recycle dimensions) whose cycles run as
    batched cooperative launches: each converges as it does alone (its own
    cycle kernel), to the same solution up to rounding, and a repeated batch
    gives the same bits."""
    import torch
    defs = _systems()
    alone = _alone(rg, torch, defs)
    xs1, st1 = _coop_round(rg, torch, defs)
    for (xa, sa), x, sb in zip(alone, xs1, st1):
        assert sb["status"] == 0 and sb["true_relres"] <= 1e-10, sb
        assert abs(sb["iters"] - sa["iters"]) <= 1, (sa, sb)
        assert _rel(x, xa) <= 1e-12
    xs2, st2 = _coop_round(rg, torch, defs)
    for a, b, sa, sb in zip(xs1, xs2, st1, st2):
        assert sa["iters"] == sb["iters"]
        np.testing.assert_array_equal(a, b)


def test_coop_batch_shares_the_resident_grid(rg):
    """Four systems that each want the whole resident grid: each keeps one
    block plus a share of the rest in proportion to its work, and still
    converges to its own solution."""
    import torch
    defs = []
    for i, (n, mode, k) in enumerate([(300001, "deflated", 8), (250000, "plain", 0),
                                      (200003, "augmented", 4), (320000, "deflated", 6)]):
        rp, col, val = synth.random_csr(n, 9, 700 + i, diag=6.0, min_per_row=2)
        b = synth.random_vector(n, 710 + i)
        U = np.linalg.qr(synth.random_matrix(n, k, 720 + i))[0] if k else None
        defs.append((n, mode, k, rp, col, val, b, U))
    alone = _alone(rg, torch, defs)
    xs, st = _coop_round(rg, torch, defs)
    for (xa, sa), x, sb in zip(alone, xs, st):
        assert sb["status"] == 0 and sb["true_relres"] <= 1e-10, sb
        assert abs(sb["iters"] - sa["iters"]) <= 1, (sa, sb)
        assert _rel(x, xa) <= 1e-10


def test_coop_flag_needs_one_precision(rg):
    """Mixed precisions: the flag is ignored and the batch runs per pass on the
    handles' streams, bit for bit as without it."""
    import torch
    defs = _systems()[:4]
    prec = ["fp64", "fp32_ir", "fp64", "fp32_ir"]
    xa, sa = _coop_round(rg, torch, defs, coop=False, precisions=prec)
    xb, sb = _coop_round(rg, torch, defs, coop=True, precisions=prec)
    for a, b, s1, s2 in zip(xa, xb, sa, sb):
        assert s1["iters"] == s2["iters"] and s1["status"] == s2["status"]
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("tpb", [1, 3, 8, 100000])
def test_tiles_per_block_same_solution(rg, tpb):
    """The autotuner's knob (tiles_per_block: rows a block owns) changes only the
    launch shape: a deflated binary64 solve and a deflated GMRES-IR solve reach
    the tolerance with iteration counts within one of the automatic shape's, and
    x within the rounding of the dot-product partition (a count above the tile
    count is clamped: one block)."""
    n = 66049
    rp, col, val = synth.random_csr(n, 9, 321, diag=6.0, min_per_row=2)
    b = synth.random_vector(n, 322)
    U = np.linalg.qr(synth.random_matrix(n, 6, 323))[0]
    for prec, tol in (("fp64", 1e-10), ("fp32_ir", 1e-8)):
        res = []
        for t in (0, tpb):
            s = rg.Solver(n, m=20, k=6, mode="deflated", precision=prec, rtol=tol, tiles_per_block=t)
            s.set_operator_csr(rp, col, val)
            s.set_recycle_space(U)
            x, st = s.solve(b)
            s.close()
            assert st["status"] == 0 and st["true_relres"] <= tol, (t, st)
            res.append((x, st))
        (xa, sa), (xb, sb) = res
        assert abs(sa["iters"] - sb["iters"]) <= 1, (sa, sb)
        assert np.linalg.norm(xa - xb) <= 100 * tol * np.linalg.norm(xa)


def test_tiles_per_block_rejects_negative(rg):
    with pytest.raises(rg.RgmError):
        rg.Solver(1000, tiles_per_block=-1)
