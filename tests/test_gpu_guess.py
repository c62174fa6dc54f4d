"""Extrapolated initial guesses (rgm_config.guess, Sec. 4.1 Eq. ext2-ext4) on
the GPU against the oracle's sequence driver: per step the same iteration
counts (within 1) and solutions within 1e-9, plain and recycled."""
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


@pytest.mark.parametrize("mode", ["plain", "deflated"])
@pytest.mark.parametrize("guess", [1, 2, 3])
def test_sequence_with_extrapolation(rg, orc, mode, guess):
    import torch
    w = synth.Q1_32
    a8, beta = synth.sequence_draws(w, 0)
    k = w.k if mode != "plain" else 0
    fe = rg.FE(w.p, w.N, w.eps, w.dt, beta)
    rp, col = fe.pattern()
    u = torch.tensor(fe.initial_field(a8), dtype=torch.float64, device="cuda")
    s = rg.Solver(fe.n, m=w.m, k=k, window=w.window, mode=mode, rtol=w.rtol, guess=guess)
    s.set_operator_csr(rp, col, np.zeros(len(col)))
    ref = orc.sequence(w.p, w.N, w.eps, w.dt, beta, w.steps, orc.u0_field(w.p, w.N, a8),
                       mode=rg.MODES[mode], m=w.m, k=k, window=w.window, rtol=w.rtol,
                       keep_all=True, guess=guess)
    for i in range(w.steps):
        st = fe.time_step(s, u)
        assert st["status"] == 0 and st["true_relres"] <= w.rtol
        assert abs(st["iters"] - ref["iters"][i]) <= 1, (i, st, ref["iters"][i])
        assert _rel(u.cpu().numpy(), ref["x_all"][:, i]) <= 1e-9


def test_guess_needs_window(rg):
    with pytest.raises(rg.RgmError):
        rg.Solver(100, k=0, window=2, guess=2)
    with pytest.raises(rg.RgmError):
        rg.Solver(100, guess=4)


# ------------------------------------------------------------------ Sec. 4.2 guess alone
@pytest.mark.parametrize("maxit", [1, 4, 9])
def test_guess_mode_fixed_steps(rg, orc, maxit):
    """RGM_GUESS: the projection initial guess, then GMRES(m) on A."""
    n, k = 3000, 4
    rp, col, val = synth.random_csr(n, 8, 15, diag=6.0, min_per_row=3)
    b, x_in = synth.random_vector(n, 16), synth.random_vector(n, 17)
    U = np.linalg.qr(synth.random_matrix(n, k, 18))[0]
    s = rg.Solver(n, m=5, k=k, mode="guess", rtol=0.0, maxit=maxit)
    s.set_operator_csr(rp, col, val)
    s.set_recycle_space(U)
    x, st = s.solve(b, x_in)
    xo, so, _ = orc.gmres(orc.Csr(rp, col, val), b, x_in=x_in, U=U, mode=orc.GUESS, m=5, rtol=0.0,
                          maxit=maxit)
    assert st["iters"] == so["iters"] == maxit and st["k_used"] == so["k_used"] == k
    assert _rel(x, xo) <= 1e-11


@pytest.mark.parametrize("mode,guess,k", [("guess", 0, 3), ("plain", 2, 0)])
def test_table2_sequences(rg, orc, mode, guess, k):
    """Both columns of Table 2 (projection guess with s = 3 modes, quadratic
    extrapolation from s = 3 solutions) on the paper's nu = 0.1 benchmark."""
    import torch
    w = synth.PAPER_Q1_64[0.1]
    steps, rtol = 25, 1e-10
    forcing = synth.forcing_draws(w, steps)
    fe = rg.FE(w.p, w.N, w.eps, w.dt, (0.0, 0.0))
    fe.set_velocity("cellular")
    rp, col = fe.pattern()
    s = rg.Solver(fe.n, m=30, k=k, window=16, mode=mode, rtol=rtol, guess=guess)
    s.set_operator_csr(rp, col, np.zeros(len(col)))
    u = torch.zeros(fe.n, dtype=torch.float64, device="cuda")
    ref = orc.sequence(w.p, w.N, w.eps, w.dt, (0.0, 0.0), steps, np.zeros(fe.n),
                       mode=rg.MODES[mode], m=30, k=k, window=16, rtol=rtol, velocity=1,
                       forcing=forcing, guess=guess, keep_all=True)
    for i in range(steps):
        fe.set_forcing(forcing[i], w.forcing_C)
        st = fe.time_step(s, u)
        assert st["status"] == 0 and st["true_relres"] <= rtol
        assert st["k_used"] == ref["k_used"][i]
        assert abs(st["iters"] - ref["iters"][i]) <= 1, (i, st, ref["iters"][i])
        assert _rel(u.cpu().numpy(), ref["x_all"][:, i]) <= 1e-9
