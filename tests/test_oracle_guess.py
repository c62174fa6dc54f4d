"""Pins of the oracle's extrapolated initial guess (Sec. 4.1, Eq. ext2 / ext3 /
ext4): the printed coefficients, exactness on vector polynomials in time of
degree below the number of points (and not one degree above), and the
sequence driver using it."""
import numpy as np
import pytest

import synth


@pytest.mark.parametrize("s,coef", [(2, [2, -1]), (3, [3, -3, 1]), (4, [4, -6, 4, -1]), (1, [1])])
def test_printed_coefficients(orc, s, coef):
    # unit columns read the coefficients off directly
    x0 = orc.extrapolate(np.eye(s))
    np.testing.assert_array_equal(x0, np.array(coef, dtype=float))


@pytest.mark.parametrize("s", [1, 2, 3, 4])
def test_exact_on_polynomials(orc, s):
    n = 50
    a = [synth.random_vector(n, 10 + q) for q in range(s + 1)]
    def x(t, deg):
        return sum(a[q] * t ** q for q in range(deg + 1))
    h = 0.37
    for deg in range(s):                            # degree <= s - 1: exact
        P = np.stack([x(-h * j, deg) for j in range(1, s + 1)], 1)
        np.testing.assert_allclose(orc.extrapolate(P), x(0.0, deg), rtol=0, atol=1e-12)
    P = np.stack([x(-h * j, s) for j in range(1, s + 1)], 1)   # degree s: error a_s h^s s!
    err = orc.extrapolate(P) - x(0.0, s)
    fact = float(np.prod(np.arange(1, s + 1)))
    np.testing.assert_allclose(np.abs(err), np.abs(a[s]) * h ** s * fact, rtol=1e-9)


@pytest.mark.parametrize("guess", [1, 2, 3])
def test_sequence_with_extrapolation(orc, guess):
    w = synth.Q1_32
    a8, beta = synth.sequence_draws(w, 0)
    u0 = orc.u0_field(w.p, w.N, a8)
    base = orc.sequence(w.p, w.N, w.eps, w.dt, beta, w.steps, u0, mode=orc.PLAIN, m=w.m, k=0,
                        window=8, rtol=w.rtol, keep_all=True)
    r = orc.sequence(w.p, w.N, w.eps, w.dt, beta, w.steps, u0, mode=orc.PLAIN, m=w.m, k=0,
                     window=8, rtol=w.rtol, keep_all=True, guess=guess)
    assert np.all(r["status"] == 0) and np.all(r["relres"] <= w.rtol)
    # identical until guess + 1 solutions exist, then a better start
    np.testing.assert_array_equal(r["iters"][:guess + 1], base["iters"][:guess + 1])
    assert r["iters"][guess + 1:].sum() < base["iters"][guess + 1:].sum()
    d = np.linalg.norm(r["x_all"] - base["x_all"], axis=0) / np.linalg.norm(base["x_all"], axis=0)
    assert d.max() < 1e-8


def test_table2_qualitative(orc):
    """Table 2's comparison (Sec. 6.1 benchmark, nu = 0.1, without SSOR): the
    projection initial guess (Sec. 4.2, GMRES on A afterwards) needs fewer
    iterations than extrapolation from the same number s of solutions, and
    extrapolation gets worse as s grows.  Means over steps 21..60."""
    w = synth.PAPER_Q1_64[0.1]
    steps = 60
    forcing = synth.forcing_draws(w, steps)
    n = orc.ndofs(w.p, w.N)
    ext, proj = {}, {}
    for s in (2, 3, 4):
        kw = dict(m=30, window=16, rtol=1e-8, velocity=1, forcing=forcing)
        e = orc.sequence(w.p, w.N, w.eps, w.dt, (0.0, 0.0), steps, np.zeros(n), mode=orc.PLAIN,
                         k=0, guess=s - 1, **kw)
        p = orc.sequence(w.p, w.N, w.eps, w.dt, (0.0, 0.0), steps, np.zeros(n), mode=orc.GUESS,
                         k=s, **kw)
        assert np.all(e["status"] == 0) and np.all(p["status"] == 0)
        ext[s], proj[s] = e["iters"][20:].mean(), p["iters"][20:].mean()
    assert all(proj[s] <= ext[s] for s in (2, 3, 4))
    assert proj[3] < ext[3] and proj[4] < ext[4]
    assert ext[2] < ext[3] < ext[4]
    assert proj[4] - proj[2] < ext[4] - ext[2]


def test_guess_mode_is_plain_gmres_from_the_projection_guess(orc):
    """ORC_GUESS = ORC_PLAIN started from x0 = x_in + U E^{-1} U^T (b - A x_in)."""
    n, k = 400, 3
    rp, col, val = synth.random_csr(n, 8, 5, diag=6.0, min_per_row=3)
    A = orc.Csr(rp, col, val)
    b = synth.random_vector(n, 6)
    U = np.linalg.qr(synth.random_matrix(n, k, 7))[0]
    x_in = synth.random_vector(n, 8)
    D = A.dense()
    x0 = x_in + U @ np.linalg.solve(U.T @ D @ U, U.T @ (b - D @ x_in))
    for maxit in (1, 4, 9):
        xg, sg, _ = orc.gmres(A, b, x_in=x_in, U=U, mode=orc.GUESS, m=5, rtol=0.0, maxit=maxit)
        xp, sp, _ = orc.gmres(A, b, x_in=x0, mode=orc.PLAIN, m=5, rtol=0.0, maxit=maxit)
        assert sg["iters"] == sp["iters"] == maxit and sg["k_used"] == k
        np.testing.assert_allclose(xg, xp, rtol=0, atol=1e-12 * np.abs(xp).max())
