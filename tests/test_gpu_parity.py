"""GPU-vs-oracle parity through the C ABI (librgmres) on seeded inputs.

Bar: integer outputs (patterns, iteration counts within +-1, recycle dimension)
exact; floating point within the stated tolerance: x within 1e-9 relative of
the FP64 oracle at solver tolerance 1e-10, true residual at or below the
tolerance, SpMV / assembly within a few ulps of the row's absolute sum.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="session")
def rg():
    import __graft_entry__ as g
    g.build()
    import paper_1807_09467_gb300 as rg
    return rg


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _orth(M):
    return np.linalg.qr(M)[0]


# ------------------------------------------------------------------ SpMV (a1)
@pytest.mark.parametrize("n,maxr,minr,seed", [(1, 1, 1, 1), (7, 3, 0, 2), (1000, 9, 0, 3),
                                              (3001, 40, 10, 4), (20011, 25, 5, 5),
                                              (257, 81, 60, 6)])
def test_spmv_random_csr(rg, orc, n, maxr, minr, seed):
    rp, col, val = synth.random_csr(n, maxr, seed, diag=2.0, min_per_row=minr)
    x = synth.random_vector(n, seed + 100)
    s = rg.Solver(n, m=1, k=0, mode="plain")
    s.set_operator_csr(rp, col, val)
    y = s.spmv(x)
    A = orc.Csr(rp, col, val)
    yo = orc.spmv(A, x)
    absrow = orc.spmv(orc.Csr(rp, col, np.abs(val)), np.abs(x))
    assert np.all(np.abs(y - yo) <= 1e-14 * absrow + 1e-300)


# ------------------------------------------------------------------ FE workload (a0)
@pytest.mark.parametrize("p,N", [(1, 5), (2, 4), (3, 3), (4, 3), (1, 32), (2, 11), (3, 7), (4, 9)])
def test_fe_pattern_values_rhs(rg, orc, p, N):
    beta = (0.6, -0.8)
    eps, dt = 0.02, 0.003
    fe = rg.FE(p, N, eps, dt, beta)
    rp, col = fe.pattern()
    orp, ocol = orc.pattern(p, N, True)
    np.testing.assert_array_equal(rp, orp)
    np.testing.assert_array_equal(col, ocol)
    u = synth.random_vector(fe.n, 11 * p + N)
    val, b = fe.assemble(u)
    _, _, oval, ob = orc.step_system(p, N, eps, dt, beta, u, pat=(orp, ocol))
    A = orc.Csr(orp, ocol, np.abs(oval))
    scale = orc.spmv(A, np.ones(fe.n))
    rows = np.repeat(np.arange(fe.n), np.diff(orp))
    assert np.all(np.abs(val - oval) <= 1e-13 * scale[rows])
    assert np.all(np.abs(b - ob) <= 1e-13 * (np.abs(ob) + np.abs(b).max()))
    a8, _ = synth.sequence_draws(synth.Q1_32, p)
    # node positions (closed form vs Newton) and device sin differ by an ulp or two
    np.testing.assert_allclose(fe.initial_field(a8), orc.u0_field(p, N, a8), rtol=0, atol=1e-14)


# ------------------------------------------------------------------ GMRES (a2-a7)
def _random_system(n, seed):
    rp, col, val = synth.random_csr(n, 8, seed, diag=6.0, min_per_row=3)
    b = synth.random_vector(n, seed + 1)
    return rp, col, val, b


@pytest.mark.parametrize("mode", ["plain", "deflated", "augmented"])
@pytest.mark.parametrize("n,m,k", [(500, 10, 4), (2003, 20, 6), (40, 50, 3)])
def test_gmres_random_parity(rg, orc, mode, n, m, k):
    rp, col, val, b = _random_system(n, n + m)
    U = _orth(synth.random_matrix(n, k, n + 7)) if mode != "plain" else None
    s = rg.Solver(n, m=m, k=k, mode=mode, rtol=1e-10)
    s.set_operator_csr(rp, col, val)
    if U is not None:
        s.set_recycle_space(U)
    x0 = synth.random_vector(n, 3)
    x, st = s.solve(b, x0)
    xo, so, _ = orc.gmres(orc.Csr(rp, col, val), b, x_in=x0, U=U, mode=rg.MODES[mode], m=m,
                          rtol=1e-10)
    assert st["status"] == 0 and st["true_relres"] <= 1e-10
    assert abs(st["iters"] - so["iters"]) <= 1, (st, so)
    assert st["k_used"] == so["k_used"]
    assert _rel(x, xo) <= 1e-9


@pytest.mark.parametrize("mode", ["plain", "deflated", "augmented"])
@pytest.mark.parametrize("maxit", [1, 5, 13])
def test_fixed_steps_iterate_parity(rg, orc, mode, maxit):
    """rtol 0 and a step cap: the iterate after exactly `maxit` Arnoldi steps."""
    n, m, k = 300, 8, 3
    rp, col, val, b = _random_system(n, 77)
    U = _orth(synth.random_matrix(n, k, 78)) if mode != "plain" else None
    s = rg.Solver(n, m=m, k=k, mode=mode, rtol=0.0, maxit=maxit)
    s.set_operator_csr(rp, col, val)
    if U is not None:
        s.set_recycle_space(U)
    x, st = s.solve(b)
    xo, so, _ = orc.gmres(orc.Csr(rp, col, val), b, U=U, mode=rg.MODES[mode], m=m, rtol=0.0,
                          maxit=maxit)
    assert st["iters"] == so["iters"] == maxit
    assert st["status"] == rg.RGM_W_NOT_CONVERGED
    assert _rel(x, xo) <= 1e-11


def _fe_step(rg, orc, w, p, N, a8, beta):
    fe = rg.FE(p, N, w.eps, w.dt, beta)
    u0 = fe.initial_field(a8)
    val, b = fe.assemble(u0)
    rp, col = fe.pattern()
    orp, ocol, oval, ob = orc.step_system(p, N, w.eps, w.dt, beta, orc.u0_field(p, N, a8))
    return fe, u0, rp, col, val, b, orc.Csr(orp, ocol, oval), ob


@pytest.mark.parametrize("mode", ["plain", "deflated", "augmented"])
@pytest.mark.parametrize("p,N", [(1, 32), (2, 16), (4, 6)])
def test_fe_step_parity(rg, orc, mode, p, N):
    w = synth.Q1_32
    a8, beta = synth.sequence_draws(w, 1)
    fe, u0, rp, col, val, b, A, ob = _fe_step(rg, orc, w, p, N, a8, beta)
    U = _orth(np.stack([u0, synth.random_vector(fe.n, 5), synth.random_vector(fe.n, 6)], 1))
    s = rg.Solver(fe.n, m=w.m, k=3, mode=mode, rtol=1e-10)
    s.set_operator_csr(rp, col, val)
    if mode != "plain":
        s.set_recycle_space(U)
    x, st = s.solve(b)
    xo, so, _ = orc.gmres(A, ob, U=U if mode != "plain" else None, mode=rg.MODES[mode], m=w.m,
                          rtol=1e-10)
    assert st["status"] == 0 and st["true_relres"] <= 1e-10
    assert abs(st["iters"] - so["iters"]) <= 1, (st, so)
    assert _rel(x, xo) <= 1e-9


@pytest.mark.parametrize("mode", ["plain", "deflated", "augmented"])
def test_sequence_q1_32(rg, orc, mode):
    """Algorithm 1 over the Q1 32x32 sequence (10 steps, GMRES(20), k 4 of 8)."""
    import torch
    w = synth.Q1_32
    a8, beta = synth.sequence_draws(w, 0)
    fe = rg.FE(w.p, w.N, w.eps, w.dt, beta)
    rp, col = fe.pattern()
    u0 = fe.initial_field(a8)
    s = rg.Solver(fe.n, m=w.m, k=w.k, window=w.window, mode=mode, rtol=w.rtol)
    s.set_operator_csr(rp, col, np.zeros(len(col)))
    u = torch.tensor(u0, dtype=torch.float64, device="cuda")
    ref = orc.sequence(w.p, w.N, w.eps, w.dt, beta, w.steps, orc.u0_field(w.p, w.N, a8),
                       mode=rg.MODES[mode], m=w.m, k=w.k, window=w.window, rtol=w.rtol,
                       keep_all=True)
    for i in range(w.steps):
        st = fe.time_step(s, u)
        assert st["status"] == 0 and st["true_relres"] <= w.rtol
        assert st["k_used"] == ref["k_used"][i]
        assert abs(st["iters"] - ref["iters"][i]) <= 1, (i, st, ref["iters"][i])
        assert _rel(u.cpu().numpy(), ref["x_all"][:, i]) <= 1e-9


# ------------------------------------------------------------------ snapshot SVD (a8)
def test_svd_window_parity(rg, orc):
    n, wnd, k = 5000, 8, 4
    Q = _orth(synth.random_matrix(n, wnd, 40))
    sig = 10.0 ** -np.arange(wnd)          # graded like consecutive solutions
    P = _orth(synth.random_matrix(wnd, wnd, 41))
    X = Q @ np.diag(sig) @ P.T
    s = rg.Solver(n, m=5, k=k, window=wnd, mode="deflated")
    for i in range(wnd):
        kk = s.update_recycle_svd(X[:, i].copy())
        assert kk == min(k, i + 1)
    U = s.recycle_space()
    Uo = orc.recycle_from_window(X, k)
    assert U.shape == Uo.shape
    np.testing.assert_allclose(U.T @ U, np.eye(k), atol=1e-13)
    # gap-dependent bound of the Gram route: eps * sigma_1^2 / (sigma_k^2 - sigma_{k+1}^2)
    bound = 50 * 2.2e-16 * sig[0] ** 2 / (sig[k - 1] ** 2 - sig[k] ** 2)
    assert np.linalg.norm(U @ U.T - Uo @ Uo.T, 2) <= bound
    sv = s.singular_values()
    np.testing.assert_allclose(sv[:k], sig[:k], rtol=1e-8)


def test_svd_rank_drop_and_interval(rg, orc):
    n = 800
    a, bvec = synth.random_vector(n, 1), synth.random_vector(n, 2)
    s = rg.Solver(n, m=5, k=4, window=5, svd_interval=2, mode="deflated")
    seq = [a, bvec, a + bvec, 2 * a, a - bvec]                # rank 2
    ks = [s.update_recycle_svd(v.copy()) for v in seq]
    assert ks == [0, 2, 2, 2, 2]
    U = s.recycle_space()
    B = _orth(np.stack([a, bvec], 1))
    assert np.linalg.norm(U @ U.T - B @ B.T, 2) < 1e-10


# ------------------------------------------------------------------ edge cases
def test_edge_cases(rg, orc):
    n = 64
    rp, col, val, b = _random_system(n, 9)
    s = rg.Solver(n, m=10, k=2, mode="deflated", rtol=1e-10)
    s.set_operator_csr(rp, col, val)
    x, st = s.solve(np.zeros(n), np.ones(n))                  # b = 0 -> x = 0
    assert np.all(x == 0) and st["iters"] == 0
    xs = np.linalg.solve(orc.Csr(rp, col, val).dense(), b)
    x, st = s.solve(b, xs)                                    # exact guess: no iteration
    assert st["iters"] == 0 and st["status"] == 0
    one = rg.Solver(1, m=3, k=0, mode="plain")                # n = 1
    one.set_operator_csr(np.array([0, 1]), np.array([0], dtype=np.int32), np.array([4.0]))
    x1, st1 = one.solve(np.array([2.0]))
    assert abs(x1[0] - 0.5) < 1e-15 and st1["iters"] <= 1
    with pytest.raises(rg.RgmError):
        rg.Solver(n, m=65)
    with pytest.raises(rg.RgmError):
        s.set_operator_csr(rp, np.full(len(col), n, dtype=np.int32), val)


def test_singular_coarse_falls_back(rg, orc):
    n = 10
    A = np.diag(np.r_[1.0, -1.0, np.arange(3, n + 1, dtype=float)])
    A[0, 1] = A[1, 0] = 1.0
    c = 1 + np.sqrt(2)
    u = np.zeros(n)
    u[0], u[1] = 1.0, c
    u /= np.linalg.norm(u)
    Ac = orc.Csr.from_dense(A)
    b = synth.random_vector(n, 3)
    s = rg.Solver(n, m=n, k=1, mode="deflated", rtol=1e-12)
    s.set_operator_csr(Ac.rowptr, Ac.col, Ac.val)
    s.set_recycle_space(u[:, None])
    x, st = s.solve(b)
    assert st["status"] == rg.RGM_W_SINGULAR_COARSE and st["k_used"] == 0
    assert st["true_relres"] <= 1e-12


# ------------------------------------------------------------------ GMRES-IR (a9)
@pytest.mark.parametrize("mode", ["plain", "deflated"])
def test_fp32_ir_reaches_fp64_tolerance(rg, orc, mode):
    w = synth.Q1_32
    a8, beta = synth.sequence_draws(w, 0)
    fe, u0, rp, col, val, b, A, ob = _fe_step(rg, orc, w, 2, 16, a8, beta)
    U = _orth(np.stack([u0, synth.random_vector(fe.n, 4)], 1))
    s = rg.Solver(fe.n, m=20, k=2, mode=mode, precision="fp32_ir", rtol=1e-8, inner_rtol=1e-4)
    s.set_operator_csr(rp, col, val)
    if mode != "plain":
        s.set_recycle_space(U)
    x, st = s.solve(b)
    assert st["status"] == 0 and st["true_relres"] <= 1e-8 and st["refinements"] >= 2
    xo, so, _ = orc.gmres(A, ob, m=50, rtol=1e-12)
    assert _rel(x, xo) <= 1e-6
    xi, si = orc.gmres_ir(A, ob, U=U if mode != "plain" else None, mode=rg.MODES[mode], m=20,
                          rtol=1e-8, inner_rtol=1e-4)
    assert abs(st["refinements"] - si["refinements"]) <= 1


# ------------------------------------------------------------------ full-size workloads
@pytest.mark.parametrize("wname", ["q2_128x128_eps0.01_dt0.005"])
def test_full_size_step_parity(rg, orc, wname):
    """One deflated step at the benchmark size, teacher-forced from u0, with the
    launch shape the benchmark uses; x compared element by element."""
    w = synth.WORKLOADS[wname]
    a8, beta = synth.sequence_draws(w, 0)
    fe, u0, rp, col, val, b, A, ob = _fe_step(rg, orc, w, w.p, w.N, a8, beta)
    U = _orth(np.stack([u0] + [synth.random_vector(fe.n, 50 + i) for i in range(3)], 1))
    s = rg.Solver(fe.n, m=w.m, k=w.k, window=w.window, mode="deflated", rtol=w.rtol)
    s.set_operator_csr(rp, col, val)
    s.set_recycle_space(U)
    x, st = s.solve(b)
    xo, so, _ = orc.gmres(A, ob, U=U, mode=orc.DEFLATED, m=w.m, rtol=w.rtol)
    assert st["true_relres"] <= w.rtol and abs(st["iters"] - so["iters"]) <= 1
    assert _rel(x, xo) <= 1e-9


def test_q4_256_residual_property(rg, orc):
    """Q4 256x256 (1,050,625 dofs): GPU assembly on sampled rows and the true
    residual of the GPU solve measured with the oracle's own A and b."""
    w = synth.Q4_256
    a8, beta = synth.sequence_draws(w, 0)
    fe = rg.FE(w.p, w.N, w.eps, w.dt, beta)
    u0 = fe.initial_field(a8)
    val, b = fe.assemble(u0)
    rp, col = fe.pattern()
    orp, ocol, oval, ob = orc.step_system(w.p, w.N, w.eps, w.dt, beta, orc.u0_field(w.p, w.N, a8))
    np.testing.assert_array_equal(rp, orp)
    idx = np.linspace(0, len(col) - 1, 20000).astype(np.int64)
    np.testing.assert_allclose(val[idx], oval[idx], rtol=1e-12, atol=1e-12 * np.abs(oval).max())
    s = rg.Solver(fe.n, m=w.m, k=w.k, mode="plain", rtol=1e-10)
    s.set_operator_csr(rp, col, val)
    x, st = s.solve(b, u0)
    r = ob - orc.spmv(orc.Csr(orp, ocol, oval), x)
    assert np.linalg.norm(r) / np.linalg.norm(ob) <= 1.5e-10


@pytest.mark.parametrize("mode", ["deflated", "augmented"])
def test_maximum_dimensions(rg, orc, mode):
    """The library's limits at once: m = 64, k = 32 (E from a 2k-column Gram
    tile), window = 64 (the window SVD on 64 snapshots), several row tiles and a
    ragged tail; x and iterations against the oracle."""
    n = 5000 + 37
    rp, col, val, b = _random_system(n, 17)
    A = orc.Csr(rp, col, val)
    U = _orth(synth.random_matrix(n, 32, 18))
    s = rg.Solver(n, m=64, k=32, window=64, mode=mode, rtol=1e-10)
    s.set_operator_csr(rp, col, val)
    s.set_recycle_space(U)
    x, st = s.solve(b)
    xo, so, _ = orc.gmres(A, b, U=U, mode=rg.MODES[mode], m=64, rtol=1e-10)
    assert st["status"] == 0 and st["k_used"] == 32
    assert abs(st["iters"] - so["iters"]) <= 1, (st, so)
    assert _rel(x, xo) <= 1e-9
    # window SVD over 64 snapshots keeps k = 32 columns inside range(X)
    X = synth.random_matrix(n, 64, 19)
    for i in range(64):
        k_new = s.update_recycle_svd(X[:, i])
    assert k_new == 32
    Ug = s.recycle_space()
    np.testing.assert_allclose(Ug.T @ Ug, np.eye(32), atol=1e-12)
    Q = np.linalg.qr(X)[0]
    assert np.linalg.norm(Ug - Q @ (Q.T @ Ug)) <= 1e-10


# ------------------------------------------------------------------ scaling (Givens, norms)
@pytest.mark.parametrize("mode", ["plain", "deflated"])
@pytest.mark.parametrize("sa,sb", [(300, 300), (-300, -300), (150, -150), (-150, 150),
                                   (450, 300), (-450, -300)])
def test_power_of_two_scaling(rg, orc, mode, sa, sb):
    """(2^sa A) x = 2^sb b has the solution 2^(sb - sa) x: every operation of
    the solve commutes with power-of-two scaling as long as no intermediate
    leaves the binary64 range, so the scaled solve equals the unscaled one bit
    for bit.  The intermediates: squared norms of A v (2^(2 sa)) and of b
    (2^(2 sb)), and the update coefficients y_i / ||A v_i|| of the unnormalised
    stored basis (2^(sb - 2 sa)); the cases keep each within 2^+-1000.  The
    rotations are formed from the scaled pair, as the oracle's hypot; the
    oracle gives the same iterations on the scaled system."""
    n, m, k = 700, 15, 3
    rp, col, val, b = _random_system(n, 4242)
    U = _orth(synth.random_matrix(n, k, 4243)) if mode != "plain" else None

    def solve(v, rhs):
        s = rg.Solver(n, m=m, k=k, mode=mode, rtol=1e-10)
        s.set_operator_csr(rp, col, v)
        if U is not None:
            s.set_recycle_space(U)
        x, st = s.solve(rhs)
        s.close()
        return x, st

    x0, st0 = solve(val, b)
    xs, sts = solve(np.ldexp(val, sa), np.ldexp(b, sb))
    assert sts["status"] == 0 and sts["iters"] == st0["iters"]
    np.testing.assert_array_equal(xs, np.ldexp(x0, sb - sa))
    xo, so, _ = orc.gmres(orc.Csr(rp, col, np.ldexp(val, sa)), np.ldexp(b, sb), U=U,
                          mode=rg.MODES[mode], m=m, rtol=1e-10)
    assert abs(sts["iters"] - so["iters"]) <= 1
    assert _rel(xs, xo) <= 1e-9


@pytest.mark.parametrize("precision", ["fp64", "fp32_ir"])
@pytest.mark.parametrize("mode", ["plain", "deflated"])
def test_zero_guess_flag_equals_zero_input(rg, orc, precision, mode):
    """RGM_ZERO_GUESS (x_in = 0 without reading x; the first residual is b, no
    SpMV) gives bit for bit what passing a zero x gives, whatever x held."""
    n, m, k = 1500, 20, 4
    rp, col, val, b = _random_system(n, 808)
    U = _orth(synth.random_matrix(n, k, 809)) if mode != "plain" else None
    out = []
    for zg in (False, True):
        s = rg.Solver(n, m=m, k=k, mode=mode, precision=precision,
                      rtol=1e-10 if precision == "fp64" else 1e-8)
        s.set_operator_csr(rp, col, val)
        if U is not None:
            s.set_recycle_space(U)
        x0 = synth.random_vector(n, 810) if zg else np.zeros(n)      # ignored under the flag
        out.append(s.solve(b, x0, zero_guess=zg))
        s.close()
    (xa, sa), (xb, sb) = out
    np.testing.assert_array_equal(xa, xb)
    assert sa["iters"] == sb["iters"] and sa["status"] == sb["status"] == 0
