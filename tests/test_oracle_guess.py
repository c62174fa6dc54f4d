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
