"""Table 1's orthogonal and least-squares projectors (rgm_config.proj) on the
GPU against the oracle: fixed-step iterates, converged solves (both start
vectors), an FE step, the binary32 refinement, and the cooperative cycle kernel
against per-pass launches.  Bar as in test_gpu_parity.py: iterations within
+-1, x within 1e-9 of the oracle at rtol 1e-10 (1e-11 for fixed-step iterates).
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

PROJ = {"oblique": 0, "orthogonal": 1, "ls": 2}


@pytest.fixture(scope="module")
def rg():
    import __graft_entry__ as g
    g.build()
    import paper_1807_09467_gb300 as rg
    return rg


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _orth(M):
    return np.linalg.qr(M)[0]


def _random_system(n, seed):
    rp, col, val = synth.random_csr(n, 8, seed, diag=6.0, min_per_row=3)
    return rp, col, val, synth.random_vector(n, seed + 1)


@pytest.mark.parametrize("proj", ["orthogonal", "ls"])
@pytest.mark.parametrize("start_r", [False, True])
@pytest.mark.parametrize("maxit", [1, 5, 13])
def test_fixed_steps_iterate(rg, orc, proj, start_r, maxit):
    n, m, k = 300, 8, 3
    rp, col, val, b = _random_system(n, 81)
    U = _orth(synth.random_matrix(n, k, 82))
    s = rg.Solver(n, m=m, k=k, mode="deflated", proj=proj, start_r=start_r, rtol=0.0, maxit=maxit)
    s.set_operator_csr(rp, col, val)
    s.set_recycle_space(U)
    x, st = s.solve(b)
    xo, so, _ = orc.gmres(orc.Csr(rp, col, val), b, U=U, mode=orc.DEFLATED, m=m, rtol=0.0,
                          maxit=maxit, start_r=start_r, proj=PROJ[proj])
    assert st["iters"] == so["iters"] == maxit
    assert _rel(x, xo) <= 1e-11


@pytest.mark.parametrize("proj", ["orthogonal", "ls"])
@pytest.mark.parametrize("start_r", [False, True])
@pytest.mark.parametrize("n,m,k", [(500, 10, 4), (2003, 20, 6), (7001, 30, 12)])
def test_converged_solve(rg, orc, proj, start_r, n, m, k):
    rp, col, val, b = _random_system(n, n + k)
    U = _orth(synth.random_matrix(n, k, n + 9))
    s = rg.Solver(n, m=m, k=k, mode="deflated", proj=proj, start_r=start_r, rtol=1e-10)
    s.set_operator_csr(rp, col, val)
    s.set_recycle_space(U)
    x0 = synth.random_vector(n, 5)
    x, st = s.solve(b, x0)
    xo, so, _ = orc.gmres(orc.Csr(rp, col, val), b, x_in=x0, U=U, mode=orc.DEFLATED, m=m,
                          rtol=1e-10, start_r=start_r, proj=PROJ[proj])
    assert st["status"] == so["status"] == 0 and st["true_relres"] <= 1e-10
    if not (proj == "ls" and start_r):
        assert abs(st["iters"] - so["iters"]) <= 1, (st, so)
    # Table 1's augmented LS method stalls on the in-cycle estimate (its floor is
    # ||(I - P) r0||) and ends cycles only on the true-residual test, so its
    # iteration count follows rounding; it is compared by convergence and x only
    assert _rel(x, xo) <= 1e-9


@pytest.mark.parametrize("proj", ["orthogonal", "ls"])
def test_fe_step(rg, orc, proj):
    """A Q2 32x32 step with U from the initial field and random columns."""
    w = synth.Q2_128
    a8, beta = synth.sequence_draws(w, 0)
    p, N = 2, 32
    fe = rg.FE(p, N, w.eps, w.dt, beta)
    u0 = fe.initial_field(a8)
    val, b = fe.assemble(u0)
    rp, col = fe.pattern()
    orp, ocol, oval, ob = orc.step_system(p, N, w.eps, w.dt, beta, orc.u0_field(p, N, a8))
    U = _orth(np.stack([u0] + [synth.random_vector(fe.n, 90 + i) for i in range(5)], 1))
    s = rg.Solver(fe.n, m=30, k=6, mode="deflated", proj=proj, rtol=1e-10)
    s.set_operator_csr(rp, col, val)
    s.set_recycle_space(U)
    x, st = s.solve(b)
    xo, so, _ = orc.gmres(orc.Csr(orp, ocol, oval), ob, U=U, mode=orc.DEFLATED, m=30, rtol=1e-10,
                          proj=PROJ[proj])
    assert st["status"] == 0 and abs(st["iters"] - so["iters"]) <= 1, (st, so)
    assert _rel(x, xo) <= 1e-9


@pytest.mark.parametrize("proj", ["orthogonal", "ls"])
def test_fp32_ir(rg, orc, proj):
    n, k = 4000, 6
    rp, col, val, b = _random_system(n, 123)
    U = _orth(synth.random_matrix(n, k, 124))
    s = rg.Solver(n, m=20, k=k, mode="deflated", proj=proj, precision="fp32_ir", rtol=1e-8)
    s.set_operator_csr(rp, col, val)
    s.set_recycle_space(U)
    x, st = s.solve(b)
    assert st["status"] == 0 and st["true_relres"] <= 1e-8
    xo, so = orc.gmres_ir(orc.Csr(rp, col, val), b, U=U, mode=orc.DEFLATED, m=20, rtol=1e-8,
                          inner_rtol=1e-4, proj=PROJ[proj])
    assert so["status"] == 0
    assert _rel(x, xo) <= 1e-6


@pytest.mark.parametrize("proj", ["orthogonal", "ls"])
def test_cycle_kernel_matches_per_pass(rg, proj):
    n, k = 66049, 8
    rp, col, val, b = _random_system(n, 200)
    U = _orth(synth.random_matrix(n, k, 201))
    out = []
    for policy in ("auto", "per_pass"):
        s = rg.Solver(n, m=30, k=k, mode="deflated", proj=proj, rtol=1e-10, launch_policy=policy)
        s.set_operator_csr(rp, col, val)
        s.set_recycle_space(U)
        out.append(s.solve(b))
        s.close()
    (xa, sa), (xp, sp) = out
    assert sa["status"] == sp["status"] == 0 and sa["iters"] == sp["iters"]
    assert _rel(xa, xp) <= 1e-13


def test_invalid_projector_rejected(rg):
    with pytest.raises(rg.RgmError):
        rg.Solver(100, proj=3)
