"""The cooperative cycle kernel (RGM_LAUNCH_AUTO: all Arnoldi steps of a
GMRES cycle in one launch, grid barriers between the fused passes) against
the per-pass launches (RGM_LAUNCH_PER_PASS), and its bounded wait.

Both launch policies run the same device code in the same block-to-row
mapping and reduction order, so iteration counts must be equal and x equal to
rounding; the oracle parity of the default (cooperative) path is covered by
test_gpu_parity.py.  The wait test makes a grid-barrier wait run out on a
generation nothing publishes and checks the status the host reads back.
"""
import time

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


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _system(rg, w, p, N):
    a8, beta = synth.sequence_draws(w, 0)
    fe = rg.FE(p, N, w.eps, w.dt, beta)
    u0 = fe.initial_field(a8)
    val, b = fe.assemble(u0)
    rp, col = fe.pattern()
    return fe.n, rp, col, val, b, u0


def _solve(rg, n, rp, col, val, b, U, policy, **kw):
    s = rg.Solver(n, launch_policy=policy, **kw)
    s.set_operator_csr(rp, col, val)
    if U is not None:
        s.set_recycle_space(U)
    x, st = s.solve(b)
    s.close()
    return x, st


CASES = [
    # (workload, p, N, m, k): one tile per block, many single-tile blocks, multi-tile blocks
    ("q1_32x32_eps0.05_dt0.01", 1, 32, 20, 4),
    ("q2_128x128_eps0.01_dt0.005", 2, 128, 30, 8),
    ("q4_256x256_eps0.002_dt0.002", 4, 256, 40, 12),
]


@pytest.mark.parametrize("wname,p,N,m,k", CASES)
@pytest.mark.parametrize("mode,precision", [("plain", "fp64"), ("deflated", "fp64"),
                                            ("augmented", "fp64"), ("deflated", "fp32_ir")])
def test_cycle_kernel_matches_per_pass(rg, wname, p, N, m, k, mode, precision):
    w = synth.WORKLOADS[wname]
    n, rp, col, val, b, u0 = _system(rg, w, p, N)
    U = None
    if mode != "plain":
        U = np.linalg.qr(np.stack([u0] + [synth.random_vector(n, 70 + i) for i in range(k - 1)], 1))[0]
    rtol = 1e-10 if precision == "fp64" else 1e-8
    kw = dict(m=m, k=k, window=2 * k, mode=mode, precision=precision, rtol=rtol)
    xa, sa = _solve(rg, n, rp, col, val, b, U, "auto", **kw)
    xp, sp = _solve(rg, n, rp, col, val, b, U, "per_pass", **kw)
    assert sa["status"] == 0 and sp["status"] == 0, (sa, sp)
    assert sa["iters"] == sp["iters"] and sa["cycles"] == sp["cycles"], (sa, sp)
    assert sa["true_relres"] <= rtol
    assert _rel(xa, xp) <= 1e-13, _rel(xa, xp)


def test_cycle_kernel_sequence_q2(rg):
    """Ten time steps of the Q2 128x128 sequence through the FE driver (SVD
    update every step): the two policies give the same iterations and field."""
    import torch
    w = synth.Q2_128
    a8, beta = synth.sequence_draws(w, 0)
    out = {}
    for policy in ("auto", "per_pass"):
        fe = rg.FE(w.p, w.N, w.eps, w.dt, beta)
        rp, col = fe.pattern()
        u = torch.tensor(fe.initial_field(a8), dtype=torch.float64, device="cuda")
        s = rg.Solver(fe.n, m=w.m, k=w.k, window=w.window, mode="deflated", rtol=w.rtol,
                      launch_policy=policy)
        s.set_operator_csr(rp, col, np.zeros(len(col)))
        its = []
        for _ in range(10):
            st = fe.time_step(s, u)
            assert st["status"] == 0 and st["true_relres"] <= w.rtol
            its.append((st["iters"], st["k_used"]))
        out[policy] = (its, u.cpu().numpy())
        s.close()
        fe.close()
    assert out["auto"][0] == out["per_pass"][0]
    assert _rel(out["auto"][1], out["per_pass"][1]) <= 1e-12


def test_bounded_wait_gives_up(rg):
    """Two blocks wait at a grid barrier that nothing releases: both waits end
    at the limit (20 ms), the device fault flag is set, and the context stays
    usable (a solve afterwards succeeds)."""
    t0 = time.perf_counter()
    gave_up, fault = rg.wait_selftest(20_000_000)
    dt = time.perf_counter() - t0
    assert (gave_up, fault) == (2, 1)
    assert dt < 5.0
    w = synth.Q1_32
    n, rp, col, val, b, _ = _system(rg, w, w.p, w.N)
    x, st = _solve(rg, n, rp, col, val, b, None, "auto", m=20, k=0, mode="plain", rtol=1e-10)
    assert st["status"] == 0 and st["true_relres"] <= 1e-10
