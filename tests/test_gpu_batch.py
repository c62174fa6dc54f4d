"""rgm_batch_solve: independent systems of different sizes and modes solved
concurrently on their own streams give exactly what each gives alone (same
code path, one launch per pass), and errors are reported per batch."""
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
