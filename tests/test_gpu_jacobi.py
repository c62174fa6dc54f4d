"""Left Jacobi preconditioning (rgm_config.precond) on the GPU against the
oracle: GMRES on D^{-1} A x = D^{-1} b with D = diag(A), the true residual
||b - A x|| <= rtol ||b|| as the stopping test and the in-cycle estimate
compared with rtol ||D^{-1} b||.  Systems have rows scaled over six decades so
that the preconditioner changes the iteration.  Bar as in test_gpu_parity.py:
iterations within +-1, x within 1e-9 of the oracle at rtol 1e-10 (1e-11 for
fixed-step iterates).
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

MODES = {"plain": 0, "deflated": 1, "augmented": 2}


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


def _mv(rp, col, val, x):
    y = np.zeros(len(rp) - 1)
    np.add.at(y, np.repeat(np.arange(len(rp) - 1), np.diff(rp)), val * x[col])
    return y


def _scaled_system(n, seed, zero_diag_rows=()):
    """Random diagonally dominant CSR with row i multiplied by 10^(3 t_i),
    t_i ~ U(-1, 1); rows in zero_diag_rows get their diagonal entry set to 0."""
    rp, col, val = synth.random_csr(n, 8, seed, diag=6.0, min_per_row=3)
    sc = 10.0 ** (3.0 * synth.random_vector(n, seed + 7))
    rows = np.repeat(np.arange(n), np.diff(rp))
    val = val * sc[rows]
    for r in zero_diag_rows:
        for e in range(rp[r], rp[r + 1]):
            if col[e] == r:
                val[e] = 0.0
    b = synth.random_vector(n, seed + 1) * sc
    return rp, col, val, b


@pytest.mark.parametrize("mode", ["plain", "deflated", "augmented"])
@pytest.mark.parametrize("maxit", [1, 5, 13])
def test_fixed_steps_iterate(rg, orc, mode, maxit):
    n, m, k = 300, 8, 3
    rp, col, val, b = _scaled_system(n, 31)
    U = _orth(synth.random_matrix(n, k, 32)) if mode != "plain" else None
    s = rg.Solver(n, m=m, k=k, mode=mode, rtol=0.0, maxit=maxit, precond="jacobi")
    s.set_operator_csr(rp, col, val)
    if U is not None:
        s.set_recycle_space(U)
    x, st = s.solve(b)
    xo, so, _ = orc.gmres(orc.Csr(rp, col, val), b, U=U, mode=MODES[mode], m=m, rtol=0.0,
                          maxit=maxit, precond=orc.PRECOND_JACOBI)
    assert st["iters"] == so["iters"] == maxit
    assert _rel(x, xo) <= 1e-11
    # rounding floor of a computed residual: eps ||A|| ||x|| / ||b|| (about 1e-14 here)
    assert abs(st["true_relres"] - so["true_relres"]) <= 1e-9 * so["true_relres"] + 1e-14


@pytest.mark.parametrize("mode", ["plain", "deflated", "augmented"])
@pytest.mark.parametrize("n,m,k", [(500, 10, 4), (2003, 20, 6), (7001, 30, 12)])
def test_converged_solve(rg, orc, mode, n, m, k):
    rp, col, val, b = _scaled_system(n, n + 3)
    U = _orth(synth.random_matrix(n, k, n + 9)) if mode != "plain" else None
    s = rg.Solver(n, m=m, k=k, mode=mode, rtol=1e-10, precond="jacobi")
    s.set_operator_csr(rp, col, val)
    if U is not None:
        s.set_recycle_space(U)
    x0 = synth.random_vector(n, 5)
    x, st = s.solve(b, x0)
    xo, so, _ = orc.gmres(orc.Csr(rp, col, val), b, x_in=x0, U=U, mode=MODES[mode], m=m,
                          rtol=1e-10, precond=orc.PRECOND_JACOBI)
    assert st["status"] == so["status"] == 0, (st, so)
    assert st["true_relres"] <= 1e-10
    assert abs(st["iters"] - so["iters"]) <= 1, (st, so)
    assert _rel(x, xo) <= 1e-9
    # the reported residual is the true one of the unscaled system
    true = np.linalg.norm(b - _mv(rp, col, val, x)) / np.linalg.norm(b)
    assert abs(true - st["true_relres"]) <= 1e-13


def test_zero_diagonal_rows(rg, orc):
    """Rows without a (nonzero) diagonal keep d_i = 1."""
    n = 700
    rp, col, val, b = _scaled_system(n, 77, zero_diag_rows=(0, 5, 299, 699))
    s = rg.Solver(n, m=20, k=0, mode="plain", rtol=0.0, maxit=17, precond="jacobi")
    s.set_operator_csr(rp, col, val)
    x, st = s.solve(b)
    xo, so, _ = orc.gmres(orc.Csr(rp, col, val), b, m=20, rtol=0.0, maxit=17,
                          precond=orc.PRECOND_JACOBI)
    assert st["iters"] == so["iters"] == 17
    assert _rel(x, xo) <= 1e-11


def test_fe_step(rg, orc):
    """A Q2 32x32 convection-diffusion step, deflated with U from the initial
    field and random columns."""
    w = synth.Q2_128
    a8, beta = synth.sequence_draws(w, 0)
    p, N = 2, 32
    fe = rg.FE(p, N, w.eps, w.dt, beta)
    u0 = fe.initial_field(a8)
    val, b = fe.assemble(u0)
    rp, col = fe.pattern()
    orp, ocol, oval, ob = orc.step_system(p, N, w.eps, w.dt, beta, orc.u0_field(p, N, a8))
    U = _orth(np.stack([u0] + [synth.random_vector(fe.n, 90 + i) for i in range(5)], 1))
    s = rg.Solver(fe.n, m=30, k=6, mode="deflated", rtol=1e-10, precond="jacobi")
    s.set_operator_csr(rp, col, val)
    s.set_recycle_space(U)
    x, st = s.solve(b)
    xo, so, _ = orc.gmres(orc.Csr(orp, ocol, oval), ob, U=U, mode=orc.DEFLATED, m=30, rtol=1e-10,
                          precond=orc.PRECOND_JACOBI)
    assert st["status"] == so["status"] == 0 and abs(st["iters"] - so["iters"]) <= 1, (st, so)
    assert _rel(x, xo) <= 1e-9


def test_values_update_rescales(rg, orc):
    """New operator values replace D: the second solve matches the oracle on
    the second operator."""
    n = 1500
    rp, col, val, b = _scaled_system(n, 401)
    val2 = val * (1.0 + 0.5 * synth.random_vector(len(val), 9))
    s = rg.Solver(n, m=20, k=0, mode="plain", rtol=1e-10, precond="jacobi")
    s.set_operator_csr(rp, col, val)
    s.solve(b)
    s.set_operator_values(val2)
    x, st = s.solve(b)
    xo, so, _ = orc.gmres(orc.Csr(rp, col, val2), b, m=20, rtol=1e-10, precond=orc.PRECOND_JACOBI)
    assert st["status"] == 0 and abs(st["iters"] - so["iters"]) <= 1, (st, so)
    assert _rel(x, xo) <= 1e-9


def test_spmv_is_unscaled(rg):
    n = 3000
    rp, col, val, _ = _scaled_system(n, 55)
    x = synth.random_vector(n, 56)
    y = _mv(rp, col, val, x)
    s = rg.Solver(n, k=0, mode="plain", precond="jacobi")
    s.set_operator_csr(rp, col, val)
    assert _rel(s.spmv(x), y) <= 1e-14


def test_cycle_kernel_matches_per_pass(rg):
    n, k = 66049, 8
    rp, col, val, b = _scaled_system(n, 210)
    U = _orth(synth.random_matrix(n, k, 211))
    out = []
    for policy in ("auto", "per_pass"):
        s = rg.Solver(n, m=30, k=k, mode="deflated", rtol=1e-10, launch_policy=policy,
                      precond="jacobi")
        s.set_operator_csr(rp, col, val)
        s.set_recycle_space(U)
        out.append(s.solve(b))
        s.close()
    (xa, sa), (xp, sp) = out
    assert sa["status"] == sp["status"] == 0 and sa["iters"] == sp["iters"]
    assert _rel(xa, xp) <= 1e-13


def test_invalid_precond_rejected(rg):
    with pytest.raises(rg.RgmError):
        rg.Solver(100, precond=2)
    with pytest.raises(rg.RgmError):
        rg.Solver(100, precond="jacobi", precision="fp32_ir")
