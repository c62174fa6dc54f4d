"""Sec. 6.1's own benchmark on the GPU against the oracle: assembly with the
cellular velocity and the random forcing (element by element, every p), the
switch back to the constant-velocity workload, and Algorithm 1 over the
Q1 64x64 sequence from a zero initial value (iterations within +-1, k_used
equal, x within 1e-9 at rtol 1e-10)."""
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


@pytest.mark.parametrize("p,N", [(1, 64), (2, 17), (3, 9), (4, 8)])
def test_assembly_parity(rg, orc, p, N):
    w = synth.PAPER_Q1_64[0.01]
    c = synth.forcing_draws(w, 3)[2]
    fe = rg.FE(p, N, w.eps, w.dt, (0.6, 0.8))
    fe.set_velocity("cellular")
    fe.set_forcing(c, w.forcing_C)
    u = orc.u0_field(p, N, synth.random_vector(8, 7) * 0.5)
    val, b = fe.assemble(u)
    rp, col = fe.pattern()
    bx, by = orc.paper_velocity(p, N)
    f = orc.paper_forcing(p, N, c, w.forcing_C)
    orp, ocol, oval, ob = orc.step_system_field(p, N, w.eps, w.dt, bx, by, f, u)
    np.testing.assert_array_equal(rp, orp)
    np.testing.assert_array_equal(col, ocol)
    assert np.max(np.abs(val - oval)) <= 1e-13 * np.max(np.abs(oval))
    assert np.max(np.abs(b - ob)) <= 1e-13 * np.max(np.abs(ob))
    # back to the constant velocity and f = 1
    fe.set_velocity("constant")
    fe.set_forcing(None)
    val, b = fe.assemble(u)
    _, _, oval, ob = orc.step_system(p, N, w.eps, w.dt, (0.6, 0.8), u)
    assert np.max(np.abs(val - oval)) <= 1e-13 * np.max(np.abs(oval))
    assert np.max(np.abs(b - ob)) <= 1e-13 * np.max(np.abs(ob))


def test_forcing_rejects_bad_arguments(rg):
    fe = rg.FE(1, 4, 0.1, 0.5, (0.0, 0.0))
    with pytest.raises(rg.RgmError):
        fe.set_forcing(np.ones(65))
    with pytest.raises(rg.RgmError):
        fe.set_velocity(2)


@pytest.mark.parametrize("mode", ["plain", "deflated", "augmented"])
@pytest.mark.parametrize("nu", [0.1, 0.001])
def test_sequence_paper_q1_64(rg, orc, mode, nu):
    import torch
    w = synth.PAPER_Q1_64[nu]
    steps, rtol = 15, 1e-10
    forcing = synth.forcing_draws(w, steps)
    fe = rg.FE(w.p, w.N, w.eps, w.dt, (0.0, 0.0))
    fe.set_velocity("cellular")
    rp, col = fe.pattern()
    s = rg.Solver(fe.n, m=w.m, k=w.k, window=w.window, mode=mode, rtol=rtol)
    s.set_operator_csr(rp, col, np.zeros(len(col)))
    u = torch.zeros(fe.n, dtype=torch.float64, device="cuda")
    ref = orc.sequence(w.p, w.N, w.eps, w.dt, (0.0, 0.0), steps, np.zeros(fe.n),
                       mode=rg.MODES[mode], m=w.m, k=w.k, window=w.window, rtol=rtol,
                       velocity=1, forcing=forcing, forcing_C=w.forcing_C, keep_all=True)
    for i in range(steps):
        fe.set_forcing(forcing[i], w.forcing_C)
        st = fe.time_step(s, u)
        assert st["status"] == 0 and st["true_relres"] <= rtol
        assert st["k_used"] == ref["k_used"][i]
        assert abs(st["iters"] - ref["iters"][i]) <= 1, (i, st, ref["iters"][i])
        assert _rel(u.cpu().numpy(), ref["x_all"][:, i]) <= 1e-9


# ------------------------------------------------------------------ order-23 spectral elements
def test_sem_assembly_parity(rg, orc):
    """Table 4's discretisation: order 23 on 2 x 2 elements (2,209 dofs),
    cellular velocity, random forcing; nodes through the initial field."""
    w = synth.PAPER_SEM23
    c = synth.forcing_draws(w, 1)[0]
    fe = rg.FE(w.p, w.N, w.eps, w.dt, (0.0, 0.0))
    fe.set_velocity("cellular")
    fe.set_forcing(c, w.forcing_C)
    a8 = synth.random_vector(8, 7) * 0.5
    u = orc.u0_field(w.p, w.N, a8)
    assert np.max(np.abs(fe.initial_field(a8) - u)) <= 1e-13 * np.max(np.abs(u))
    val, b = fe.assemble(u)
    rp, col = fe.pattern()
    bx, by = orc.paper_velocity(w.p, w.N)
    f = orc.paper_forcing(w.p, w.N, c, w.forcing_C)
    orp, ocol, oval, ob = orc.step_system_field(w.p, w.N, w.eps, w.dt, bx, by, f, u)
    np.testing.assert_array_equal(rp, orp)
    np.testing.assert_array_equal(col, ocol)
    assert np.max(np.abs(val - oval)) <= 1e-12 * np.max(np.abs(oval))
    assert np.max(np.abs(b - ob)) <= 1e-12 * np.max(np.abs(ob))


@pytest.mark.parametrize("p,N", [(6, 3), (12, 2)])
def test_high_order_constant_velocity(rg, orc, p, N):
    """Above p = 4 the constant velocity also takes the quadrature path."""
    fe = rg.FE(p, N, 0.01, 0.5, (0.6, 0.8))
    u = orc.u0_field(p, N, synth.random_vector(8, 8) * 0.5)
    val, b = fe.assemble(u)
    _, _, oval, ob = orc.step_system(p, N, 0.01, 0.5, (0.6, 0.8), u)
    assert np.max(np.abs(val - oval)) <= 1e-12 * np.max(np.abs(oval))
    assert np.max(np.abs(b - ob)) <= 1e-12 * np.max(np.abs(ob))


@pytest.mark.parametrize("mode", ["deflated", "augmented"])
def test_sem_sequence_jacobi(rg, orc, mode):
    """Three steps of Algorithm 1 on the order-23 elements with left Jacobi
    (k 4 of a window of 4, SVD every step)."""
    import torch
    w = synth.PAPER_SEM23
    steps, rtol, k, window = 3, 1e-10, 4, 4
    forcing = synth.forcing_draws(w, steps)
    fe = rg.FE(w.p, w.N, w.eps, w.dt, (0.0, 0.0))
    fe.set_velocity("cellular")
    rp, col = fe.pattern()
    s = rg.Solver(fe.n, m=w.m, k=k, window=window, mode=mode, rtol=rtol, precond="jacobi")
    s.set_operator_csr(rp, col, np.zeros(len(col)))
    u = torch.zeros(fe.n, dtype=torch.float64, device="cuda")
    ref = orc.sequence(w.p, w.N, w.eps, w.dt, (0.0, 0.0), steps, np.zeros(fe.n),
                       mode=rg.MODES[mode], m=w.m, k=k, window=window, rtol=rtol, velocity=1,
                       forcing=forcing, forcing_C=w.forcing_C, precond=orc.PRECOND_JACOBI,
                       keep_all=True)
    for i in range(steps):
        fe.set_forcing(forcing[i], w.forcing_C)
        st = fe.time_step(s, u)
        assert st["status"] == 0 and st["true_relres"] <= rtol
        assert st["k_used"] == ref["k_used"][i]
        assert abs(st["iters"] - ref["iters"][i]) <= 1, (i, st, ref["iters"][i])
        assert _rel(u.cpu().numpy(), ref["x_all"][:, i]) <= 1e-9
