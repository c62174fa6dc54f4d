"""Pins of the oracle's snapshot SVD (Sec. 5.2) and Algorithm 1 sequence driver.

The SVD is checked against numpy's LAPACK SVD (a library routine), a matrix
built with known singular values, and the Schmidt-Eckart-Young identity
(Eq. best_rank_s / opt_svd).  The sequence driver is checked for the window and
interval bookkeeping of Algorithm 1 and for solving every system of the
sequence it generates.
"""
import numpy as np
import pytest

import synth


def _span_dist(U1, U2):
    return np.linalg.norm(U1 @ U1.T - U2 @ U2.T, 2)


@pytest.mark.parametrize("n,c,seed", [(50, 1, 1), (50, 8, 2), (300, 24, 3), (24, 24, 4)])
def test_svd_matches_lapack(orc, n, c, seed):
    X = synth.random_matrix(n, c, seed)
    s, Psi = orc.svd_left(X)
    Ul, sl, _ = np.linalg.svd(X, full_matrices=False)
    np.testing.assert_allclose(s, sl, rtol=1e-13)
    np.testing.assert_allclose(Psi.T @ Psi, np.eye(c), atol=1e-13)
    for k in range(1, c):
        if sl[k - 1] - sl[k] > 1e-3 * sl[0]:
            assert _span_dist(Psi[:, :k], Ul[:, :k]) < 1e-11
    # each column is a left singular vector: X^T psi_i = sigma_i phi_i, ||X^T psi_i|| = sigma_i
    np.testing.assert_allclose(np.linalg.norm(X.T @ Psi, axis=0), s, rtol=1e-12)


def test_svd_known_singular_values_graded(orc):
    n, c = 200, 10
    Q = np.linalg.qr(synth.random_matrix(n, c, 10))[0]
    P = np.linalg.qr(synth.random_matrix(c, c, 11))[0]
    sig = 10.0 ** -np.arange(c)                       # 1 ... 1e-9
    X = Q @ np.diag(sig) @ P.T
    s, Psi = orc.svd_left(X)
    np.testing.assert_allclose(s, sig, rtol=1e-6)
    np.testing.assert_allclose(s[:5], sig[:5], rtol=1e-12)
    for k in (1, 3, 5):
        assert _span_dist(Psi[:, :k], Q[:, :k]) < 1e-10


@pytest.mark.parametrize("k", [1, 3, 6])
def test_eckart_young(orc, k):
    X = synth.random_matrix(120, 9, 20)
    s, Psi = orc.svd_left(X)
    Uk = Psi[:, :k]
    err = np.linalg.norm(X - Uk @ (Uk.T @ X), "fro") ** 2
    assert abs(err - np.sum(s[k:] ** 2)) <= 1e-12 * np.sum(s ** 2)
    # any other rank-k projection does worse (Eq. opt_svd)
    R = np.linalg.qr(synth.random_matrix(120, k, 21))[0]
    assert np.linalg.norm(X - R @ (R.T @ X), "fro") ** 2 > err


def test_recycle_selection_rank_drop_and_smallest(orc):
    n = 80
    a = synth.random_vector(n, 30)
    bvec = synth.random_vector(n, 31)
    X = np.stack([a, bvec, a + bvec, 2 * a, np.zeros(n)], 1)     # rank 2
    U = orc.recycle_from_window(X, 4)
    assert U.shape[1] == 2
    B = np.linalg.qr(np.stack([a, bvec], 1))[0]
    assert _span_dist(U, B) < 1e-12
    X2 = synth.random_matrix(n, 6, 32)
    s, Psi = orc.svd_left(X2)
    Us = orc.recycle_from_window(X2, 2, select_smallest=True)
    assert _span_dist(Us, Psi[:, 4:6]) < 1e-12
    Ul = orc.recycle_from_window(X2, 2)
    assert _span_dist(Ul, Psi[:, 0:2]) < 1e-12


def _seq(orc, w, steps, mode, ell=1, window=None, keep_all=False):
    a8, beta = synth.sequence_draws(w, 0)
    u0 = orc.u0_field(w.p, w.N, a8)
    r = orc.sequence(w.p, w.N, w.eps, w.dt, beta, steps, u0, mode=mode, m=w.m, k=w.k,
                     window=window or w.window, ell=ell, rtol=w.rtol, keep_all=keep_all)
    return r, u0, beta


@pytest.mark.parametrize("mode", [1, 2])
def test_algorithm1_window_and_interval(orc, mode):
    w = synth.Q1_32          # k = 4
    r, _, _ = _seq(orc, w, 9, mode, ell=1, window=3)
    # step i uses the SVD of the window after step i-1: min(k, window, i-1) columns
    np.testing.assert_array_equal(r["k_used"], [0, 1, 2, 3, 3, 3, 3, 3, 3])
    r, _, _ = _seq(orc, w, 9, mode, ell=2, window=8)
    # SVDs after steps 2, 4, 6, 8 over 2, 4, 6, 8 stored solutions (k = 4)
    np.testing.assert_array_equal(r["k_used"], [0, 0, 2, 2, 4, 4, 4, 4, 4])


def test_sequence_solves_each_system(orc):
    w = synth.Q1_32
    results = {}
    for mode in (0, 1, 2):
        r, u0, beta = _seq(orc, w, w.steps, mode, keep_all=True)
        assert np.all(r["status"] == 0) and np.all(r["relres"] <= w.rtol)
        X = r["x_all"]
        # re-assemble step i from x_{i-1} and check the stored x_i solves it
        prev = u0
        for i in range(w.steps):
            rp, col, val, b = orc.step_system(w.p, w.N, w.eps, w.dt, beta, prev)
            res = np.linalg.norm(b - orc.spmv(orc.Csr(rp, col, val), X[:, i])) / np.linalg.norm(b)
            assert res <= w.rtol * (1 + 1e-6)
            prev = X[:, i]
        results[mode] = X
    # every mode follows the same trajectory up to the solver tolerance
    for mode in (1, 2):
        d = np.linalg.norm(results[mode] - results[0], axis=0) / np.linalg.norm(results[0], axis=0)
        assert d.max() < 1e-8


def test_recycle_space_lies_in_window_range(orc):
    """Algorithm 1 keeps singular modes of X_m, so span U is inside range(X_m):
    with all c modes kept, span U = range(X) even at sigma_c / sigma_1 = 1e-7."""
    n, c = 3000, 6
    B = np.linalg.qr(synth.random_matrix(n, c, 60))[0]
    C = np.linalg.qr(synth.random_matrix(c, c, 61))[0] @ np.diag(np.logspace(0, -7, c))
    X = B @ C
    U = orc.recycle_from_window(X, c, rel_drop=1e-9)
    assert U.shape[1] == c
    assert np.linalg.norm(U - B @ (B.T @ U)) <= 1e-13
    np.testing.assert_allclose(U.T @ U, np.eye(c), atol=1e-14)
