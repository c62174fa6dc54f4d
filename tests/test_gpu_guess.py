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
