"""Pins of the oracle's GMRES(m), deflation, augmentation and GMRES-IR.

Checks fixed independently of the oracle: exact termination (Sec. 1: GMRES is a
direct method), the minimal-residual definition over an explicit Krylov basis
solved by numpy's least squares (Sec. 3, Eq. x_k_expression with C_k = A S_k),
projector identities (Sec. 3.2, 3.3), the projection guess (Sec. 4.2), the
oblique aug/def equivalence (Eq. equivalence_oblique) and the invariant-space
estimate (Eq. estimate_deflation_vs_augmentation).
"""
import numpy as np
import pytest

import synth


def _rand_system(n, seed, shift=3.0):
    A = synth.random_matrix(n, n, seed) + shift * np.eye(n)
    b = synth.random_vector(n, seed + 1)
    return A, b


def _orth(M):
    q, _ = np.linalg.qr(M)
    return q


@pytest.mark.parametrize("n,seed", [(5, 1), (12, 2), (20, 3)])
def test_full_gmres_is_direct(orc, n, seed):
    A, b = _rand_system(n, seed, shift=0.5)
    x, st, _ = orc.gmres(orc.Csr.from_dense(A), b, m=n, rtol=1e-12, maxit=n)
    assert st["iters"] <= n and st["true_relres"] <= 1e-12
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-9, atol=1e-12)


def _krylov(A, r, j):
    K = np.zeros((len(r), j))
    v = r.copy()
    for i in range(j):
        K[:, i] = v
        v = A @ v
    return K


@pytest.mark.parametrize("j", [1, 2, 4, 7])
def test_fixed_steps_equal_brute_force_minimiser(orc, j):
    n = 15
    A, b = _rand_system(n, 11)
    x0 = synth.random_vector(n, 99)
    x, st, _ = orc.gmres(orc.Csr.from_dense(A), b, x_in=x0, m=30, rtol=0.0, maxit=j)
    assert st["iters"] == j and st["cycles"] == 1
    r0 = b - A @ x0
    K = _krylov(A, r0, j)
    y, *_ = np.linalg.lstsq(A @ K, r0, rcond=None)
    np.testing.assert_allclose(x, x0 + K @ y, rtol=1e-9, atol=1e-11)


def test_distinct_eigenvalues_terminate(orc):
    # A = S D S^-1 with 4 distinct eigenvalues: the minimal polynomial has degree 4
    n = 12
    S = synth.random_matrix(n, n, 5) + 4 * np.eye(n)
    d = np.array([1.0, 2.0, 3.0, 5.0] * 3)
    A = S @ np.diag(d) @ np.linalg.inv(S)
    b = synth.random_vector(n, 6)
    _, _, hist = orc.gmres(orc.Csr.from_dense(A), b, m=n, rtol=0.0, maxit=4, hist_len=8)
    assert hist[3] < 1e-10 and hist[2] > 1e-4


def test_restarted_residuals_monotone(orc):
    n = 60
    rp, col, val = synth.random_csr(n, 6, 21, diag=4.0)
    A = orc.Csr(rp, col, val)
    b = synth.random_vector(n, 22)
    x, st, hist = orc.gmres(A, b, m=5, rtol=1e-10, maxit=2000, hist_len=2000)
    assert st["status"] == 0 and st["cycles"] > 2 and st["true_relres"] <= 1e-10
    assert np.all(np.diff(hist[:5]) <= 1e-15)             # within the first cycle
    # true residual per cycle decreases: re-run with increasing maxit (cycle ends)
    prev = np.inf
    for it in range(5, st["iters"], 5):
        _, s2, _ = orc.gmres(A, b, m=5, rtol=0.0, maxit=it)
        assert s2["true_relres"] <= prev * (1 + 1e-12)
        prev = s2["true_relres"]
    Ad = A.dense()
    np.testing.assert_allclose(x, np.linalg.solve(Ad, b), rtol=1e-8, atol=1e-10)


def test_zero_rhs_and_exact_guess(orc):
    A, b = _rand_system(8, 31)
    Ac = orc.Csr.from_dense(A)
    x, st, _ = orc.gmres(Ac, np.zeros(8), x_in=np.ones(8))
    assert np.all(x == 0) and st["iters"] == 0
    xs = np.linalg.solve(A, b)
    x, st, _ = orc.gmres(Ac, b, x_in=xs, rtol=1e-8)
    assert st["iters"] == 0


# ------------------------------------------------------------------ recycling
def _setup_recycle(n=30, k=4, seed=40):
    A, b = _rand_system(n, seed)
    U = _orth(synth.random_matrix(n, k, seed + 2))
    return A, b, U


def test_oblique_projector_identities(orc):
    A, b, U = _setup_recycle()
    Ac = orc.Csr.from_dense(A)
    W, E = orc.coarse_setup(Ac, U)
    np.testing.assert_allclose(W, A @ U, atol=1e-13)
    np.testing.assert_allclose(E, U.T @ A @ U, atol=1e-13)
    v = synth.random_vector(A.shape[0], 7)
    Pv, rc = orc.apply_oblique(U, W, E, v)
    assert rc == 0
    PPv, _ = orc.apply_oblique(U, W, E, Pv)
    np.testing.assert_allclose(PPv, Pv, atol=1e-12)             # P^2 = P
    for i in range(U.shape[1]):
        PW, _ = orc.apply_oblique(U, W, E, W[:, i])
        assert np.abs(PW).max() < 1e-12                         # P A U = 0
    assert np.abs(U.T @ Pv).max() < 1e-12                       # U^T P = 0
    # against the explicit matrix I - A U E^-1 U^T
    P = np.eye(len(v)) - A @ U @ np.linalg.solve(U.T @ A @ U, U.T)
    np.testing.assert_allclose(Pv, P @ v, atol=1e-12)


@pytest.mark.parametrize("mode", [1, 2])
def test_solution_in_span_U_is_exact(orc, mode):
    A, _, U = _setup_recycle()
    xs = U @ np.array([1.0, -2.0, 0.5, 3.0])
    b = A @ xs
    x, st, _ = orc.gmres(orc.Csr.from_dense(A), b, U=U, mode=mode, rtol=1e-12)
    assert st["iters"] == 0 and st["k_used"] == 4
    np.testing.assert_allclose(x, xs, atol=1e-12)


def test_projection_guess_formula(orc):
    # with maxit = 0 the iterate is x0 = x_in + U E^-1 U^T (b - A x_in)
    A, b, U = _setup_recycle()
    xin = synth.random_vector(len(b), 3)
    x, st, _ = orc.gmres(orc.Csr.from_dense(A), b, x_in=xin, U=U, mode=1, rtol=0.0, maxit=0)
    E = U.T @ A @ U
    np.testing.assert_allclose(x, xin + U @ np.linalg.solve(E, U.T @ (b - A @ xin)), atol=1e-12)


def test_deflated_full_gmres_terminates_in_n_minus_k(orc):
    n, k = 14, 4
    A, b, U = _setup_recycle(n, k, 50)
    x, st, _ = orc.gmres(orc.Csr.from_dense(A), b, U=U, mode=1, m=n, rtol=1e-11, maxit=n - k)
    assert st["iters"] <= n - k and st["true_relres"] <= 1e-11
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-8)


@pytest.mark.parametrize("j", [1, 3, 6])
def test_deflated_fixed_steps_brute_force(orc, j):
    """x = x0 + V y + coarse correction, V spanning K_j(P A, P r0), y minimising
    ||P r0 - P A V y||."""
    A, b, U = _setup_recycle(25, 3, 60)
    x, st, _ = orc.gmres(orc.Csr.from_dense(A), b, U=U, mode=1, m=30, rtol=0.0, maxit=j)
    E = U.T @ A @ U
    Q = U @ np.linalg.solve(E, U.T)
    P = np.eye(len(b)) - A @ Q
    x0 = Q @ b
    r0 = b - A @ x0
    K = _krylov(P @ A, P @ r0, j)
    y, *_ = np.linalg.lstsq(P @ A @ K, P @ r0, rcond=None)
    xk = x0 + K @ y
    xk = xk + Q @ (b - A @ xk)
    np.testing.assert_allclose(x, xk, rtol=1e-9, atol=1e-11)


@pytest.mark.parametrize("j", [1, 3, 6])
def test_augmented_fixed_steps_brute_force(orc, j):
    """Sec. 3.1: x = x0 + z, z minimising ||r0 - A z|| over K_j(A, r0) + span U."""
    A, b, U = _setup_recycle(25, 3, 70)
    x, st, _ = orc.gmres(orc.Csr.from_dense(A), b, U=U, mode=2, m=30, rtol=0.0, maxit=j)
    E = U.T @ A @ U
    x0 = U @ np.linalg.solve(E, U.T @ b)
    r0 = b - A @ x0
    S = np.hstack([_krylov(A, r0, j), U])
    y, *_ = np.linalg.lstsq(A @ S, r0, rcond=None)
    np.testing.assert_allclose(x, x0 + S @ y, rtol=1e-9, atol=1e-11)


def test_oblique_aug_def_equivalence(orc):
    """Eq. equivalence_oblique: Table 1's augmented-oblique (start r0) and
    deflated-oblique (start P r0) coincide without a preconditioner."""
    A, b, U = _setup_recycle(40, 4, 80)
    Ac = orc.Csr.from_dense(A)
    for maxit in (3, 10, 25):
        x1, s1, _ = orc.gmres(Ac, b, U=U, mode=1, m=8, rtol=0.0, maxit=maxit, start_r=False)
        x2, s2, _ = orc.gmres(Ac, b, U=U, mode=1, m=8, rtol=0.0, maxit=maxit, start_r=True)
        np.testing.assert_allclose(x1, x2, rtol=1e-10, atol=1e-12)


def test_invariant_space_estimate(orc):
    """Eq. estimate_deflation_vs_augmentation for an A-invariant span U:
    ||P r_aug|| = 0 <= ||P r_def|| and ||(I-P) r_aug|| <= ||(I-P) r_def||,
    P the orthogonal projector onto span U."""
    n, k = 30, 4
    Q = _orth(synth.random_matrix(n, n, 90))
    T = synth.random_matrix(n, n, 91) + 4 * np.eye(n)
    T[k:, :k] = 0.0                                  # block upper triangular: span Q[:, :k] invariant
    A = Q @ T @ Q.T
    U = Q[:, :k]
    assert np.abs((np.eye(n) - U @ U.T) @ A @ U).max() < 1e-12
    b = synth.random_vector(n, 92)
    Ac = orc.Csr.from_dense(A)
    Pu = U @ U.T
    for j in (2, 5, 9):
        xa, _, _ = orc.gmres(Ac, b, U=U, mode=2, m=30, rtol=0.0, maxit=j)
        xd, _, _ = orc.gmres(Ac, b, U=U, mode=1, m=30, rtol=0.0, maxit=j)
        ra, rd = b - A @ xa, b - A @ xd
        assert np.linalg.norm(Pu @ ra) <= 1e-11 * np.linalg.norm(b)
        assert np.linalg.norm(ra - Pu @ ra) <= np.linalg.norm(rd - Pu @ rd) * (1 + 1e-9)


def test_singular_coarse_falls_back(orc):
    n = 10
    A = np.diag(np.r_[1.0, -1.0, np.arange(3, n + 1, dtype=float)])
    A[0, 1] = 1.0
    A[1, 0] = 1.0                                     # [[1,1],[1,-1]] block
    # u = (1, c)/norm with E = u^T A u = 0: 1 + 2c - c^2 = 0 -> c = 1 + sqrt(2)
    c = 1 + np.sqrt(2)
    u = np.zeros(n)
    u[0], u[1] = 1.0, c
    u /= np.linalg.norm(u)
    b = synth.random_vector(n, 3)
    x, st, _ = orc.gmres(orc.Csr.from_dense(A), b, U=u[:, None], mode=1, m=n, rtol=1e-12)
    assert st["status"] == orc.W_SINGULAR_COARSE and st["k_used"] == 0
    assert st["true_relres"] <= 1e-12


def test_fe_recycled_modes_agree(orc):
    w = synth.Q1_32
    a8, beta = synth.sequence_draws(w, 0)
    u0 = orc.u0_field(w.p, w.N, a8)
    rp, col, val, b = orc.step_system(w.p, w.N, w.eps, w.dt, beta, u0)
    A = orc.Csr(rp, col, val)
    Ad = A.dense()
    xs = np.linalg.solve(Ad, b)
    U = _orth(np.stack([u0, synth.random_vector(len(b), 4)], 1))
    for mode in (0, 1, 2):
        x, st, _ = orc.gmres(A, b, U=U if mode else None, mode=mode, m=w.m, rtol=1e-10)
        assert st["status"] == 0 and st["true_relres"] <= 1e-10
        np.testing.assert_allclose(x, xs, rtol=0, atol=1e-9 * np.abs(xs).max())


@pytest.mark.parametrize("mode", [0, 1])
def test_gmres_ir_reaches_fp64_residual(orc, mode):
    w = synth.Q1_32
    a8, beta = synth.sequence_draws(w, 0)
    u0 = orc.u0_field(w.p, w.N, a8)
    rp, col, val, b = orc.step_system(w.p, w.N, w.eps, w.dt, beta, u0)
    A = orc.Csr(rp, col, val)
    U = _orth(np.stack([u0, synth.random_vector(len(b), 4)], 1)) if mode else None
    x, st = orc.gmres_ir(A, b, U=U, mode=mode, m=20, rtol=1e-8, inner_rtol=1e-4)
    assert st["status"] == 0 and st["true_relres"] <= 1e-8 and st["refinements"] >= 2
    xs = np.linalg.solve(A.dense(), b)
    assert np.linalg.norm(x - xs) <= 1e-6 * np.linalg.norm(xs)


# ------------------------------------------------------------------ Table 1 projector variants
def _explicit_projectors(A, U):
    """The three projectors of Table 1 as dense matrices (Eq. P_A_variant for
    the orthogonal one, so U need not be orthonormal)."""
    n = A.shape[0]
    W = A @ U
    I = np.eye(n)
    return {0: I - W @ np.linalg.solve(U.T @ W, U.T),
            1: I - U @ np.linalg.solve(U.T @ U, U.T),
            2: I - W @ np.linalg.solve(W.T @ W, W.T)}


@pytest.mark.parametrize("proj", [0, 1, 2])
def test_table1_projector_identities(orc, proj):
    A, _, U = _setup_recycle(30, 4, 100)
    U = U @ (np.triu(synth.random_matrix(4, 4, 101)) + 2 * np.eye(4))   # not orthonormal
    W = A @ U
    v = synth.random_vector(30, 102)
    Pv, rc = orc.apply_projector(U, W, proj, v)
    assert rc == 0
    np.testing.assert_allclose(Pv, _explicit_projectors(A, U)[proj] @ v, atol=1e-11)
    PPv, _ = orc.apply_projector(U, W, proj, Pv)
    np.testing.assert_allclose(PPv, Pv, atol=1e-11)                        # P^2 = P
    killed = {0: W, 1: U, 2: W}[proj]                                       # P kills W or U
    for i in range(4):
        Pk, _ = orc.apply_projector(U, W, proj, killed[:, i])
        assert np.abs(Pk).max() < 1e-11 * np.abs(killed[:, i]).max()
    if proj in (1, 2):                                                      # orthogonal projectors
        w2 = synth.random_vector(30, 103)
        Pw2, _ = orc.apply_projector(U, W, proj, w2)
        assert abs(Pv @ w2 - v @ Pw2) < 1e-11 * np.linalg.norm(v) * np.linalg.norm(w2)


@pytest.mark.parametrize("proj", [1, 2])
@pytest.mark.parametrize("start_r", [False, True])
@pytest.mark.parametrize("j", [1, 3, 6])
def test_table1_variant_fixed_steps_brute_force(orc, proj, start_r, j):
    """One cycle of j steps of the Table 1 method: x0 = U E^-1 U^T b, Krylov
    operator P A, start vector P r0 (deflated) or r0 (augmented), y minimising
    ||s - P A K y|| by numpy least squares over the explicit power basis, then
    the cycle-end correction x += Q (b - A x) with Q = U (W^T W)^-1 W^T (LS) or
    U E^-1 U^T (orthogonal)."""
    A, b, U = _setup_recycle(25, 3, 110 + proj)
    x, st, _ = orc.gmres(orc.Csr.from_dense(A), b, U=U, mode=1, m=30, rtol=0.0, maxit=j,
                         start_r=start_r, proj=proj)
    assert st["iters"] == j and st["k_used"] == 3
    W = A @ U
    E = U.T @ W
    P = _explicit_projectors(A, U)[proj]
    Qc = U @ np.linalg.solve(W.T @ W, W.T) if proj == 2 else U @ np.linalg.solve(E, U.T)
    x0 = U @ np.linalg.solve(E, U.T @ b)
    r0 = b - A @ x0
    s = r0 if start_r else P @ r0
    K = _krylov(P @ A, s, j)
    y, *_ = np.linalg.lstsq(P @ A @ K, s, rcond=None)
    xk = x0 + K @ y
    xk = xk + Qc @ (b - A @ xk)
    np.testing.assert_allclose(x, xk, rtol=1e-9, atol=1e-11)


def test_ls_deflated_true_residual_is_the_minimised_one(orc):
    """Deflated LS (the GCRO inner iteration): after the correction with
    Q = U (W^T W)^-1 W^T, I - A Q = P, so the true residual of each cycle equals
    the Givens estimate, as for the oblique projector with Q = U E^-1 U^T."""
    A, b, U = _setup_recycle(40, 4, 120)
    Ac = orc.Csr.from_dense(A)
    for proj in (2, 0):
        for j in (2, 5, 9):
            x, st, hist = orc.gmres(Ac, b, U=U, mode=1, m=30, rtol=0.0, maxit=j, proj=proj,
                                    hist_len=j)
            assert abs(st["true_relres"] - hist[j - 1]) <= 1e-10 * hist[j - 1] + 1e-14


def test_orthogonal_start_vectors_coincide(orc):
    """With the projection guess the first residual is orthogonal to U
    (U^T (I - W E^-1 U^T) = 0), so Table 1's augmented and deflated orthogonal
    methods start from the same vector and give the same iterates."""
    A, b, U = _setup_recycle(40, 4, 130)
    Ac = orc.Csr.from_dense(A)
    for maxit in (3, 10):
        x1, _, _ = orc.gmres(Ac, b, U=U, mode=1, m=8, rtol=0.0, maxit=maxit, proj=1)
        x2, _, _ = orc.gmres(Ac, b, U=U, mode=1, m=8, rtol=0.0, maxit=maxit, proj=1, start_r=True)
        np.testing.assert_allclose(x1, x2, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("proj", [1, 2])
def test_table1_variants_solve_fe_step(orc, proj):
    """Both variants reach the true residual 1e-10 on a Q1 step (restarted)."""
    w = synth.Q1_32
    a8, beta = synth.sequence_draws(w, 0)
    u0 = orc.u0_field(w.p, w.N, a8)
    rp, col, val, b = orc.step_system(w.p, w.N, w.eps, w.dt, beta, u0)
    A = orc.Csr(rp, col, val)
    U = _orth(np.stack([u0, synth.random_vector(len(b), 4), synth.random_vector(len(b), 5)], 1))
    x, st, _ = orc.gmres(A, b, U=U, mode=1, m=w.m, rtol=1e-10, proj=proj)
    assert st["status"] == 0 and st["true_relres"] <= 1e-10
    xs = np.linalg.solve(A.dense(), b)
    np.testing.assert_allclose(x, xs, rtol=0, atol=1e-8 * np.abs(xs).max())


# ------------------------------------------------------------------ left Jacobi preconditioning
def _jacobi(A):
    d = np.diag(A).copy()
    d[d == 0] = 1.0
    return d


def test_jacobi_diagonal_matrix_one_step(orc):
    n = 12
    A = np.diag(np.arange(1.0, n + 1))
    b = synth.random_vector(n, 200)
    x0, s0, _ = orc.gmres(orc.Csr.from_dense(A), b, m=n, rtol=1e-12)
    x1, s1, _ = orc.gmres(orc.Csr.from_dense(A), b, m=n, rtol=1e-12, precond=orc.PRECOND_JACOBI)
    assert s1["iters"] == 1 and s0["iters"] == n               # D^-1 A = I
    np.testing.assert_allclose(x1, b / np.diag(A), rtol=1e-14)


@pytest.mark.parametrize("j", [1, 3, 6])
def test_jacobi_fixed_steps_brute_force(orc, j):
    """x = x0 + K y, K = K_j(D^-1 A, D^-1 r0), y minimising ||D^-1 (r0 - A K y)||."""
    n = 18
    A, b = _rand_system(n, 210)
    A += np.diag(synth.random_vector(n, 211, 1.0, 5.0))          # uneven diagonal
    x0 = synth.random_vector(n, 212)
    x, st, _ = orc.gmres(orc.Csr.from_dense(A), b, x_in=x0, m=30, rtol=0.0, maxit=j,
                         precond=orc.PRECOND_JACOBI)
    assert st["iters"] == j
    Di = np.diag(1.0 / _jacobi(A))
    r0 = Di @ (b - A @ x0)
    K = _krylov(Di @ A, r0, j)
    y, *_ = np.linalg.lstsq(Di @ A @ K, r0, rcond=None)
    np.testing.assert_allclose(x, x0 + K @ y, rtol=1e-9, atol=1e-11)


@pytest.mark.parametrize("j", [1, 4])
def test_jacobi_deflated_fixed_steps_brute_force(orc, j):
    """Deflation on the preconditioned operator: A~ = D^-1 A, W = A~ U,
    P = I - W (U^T W)^-1 U^T, start P r~0 from the projection guess."""
    A, b, U = _setup_recycle(25, 3, 220)
    A += np.diag(synth.random_vector(25, 221, 1.0, 4.0))
    x, st, _ = orc.gmres(orc.Csr.from_dense(A), b, U=U, mode=1, m=30, rtol=0.0, maxit=j,
                         precond=orc.PRECOND_JACOBI)
    Di = np.diag(1.0 / _jacobi(A))
    At, bt = Di @ A, Di @ b
    E = U.T @ At @ U
    Q = U @ np.linalg.solve(E, U.T)
    P = np.eye(25) - At @ Q
    xk0 = Q @ bt
    r0 = bt - At @ xk0
    K = _krylov(P @ At, P @ r0, j)
    y, *_ = np.linalg.lstsq(P @ At @ K, P @ r0, rcond=None)
    xk = xk0 + K @ y
    xk = xk + Q @ (bt - At @ xk)
    np.testing.assert_allclose(x, xk, rtol=1e-9, atol=1e-11)


def test_jacobi_converges_on_true_residual_and_unit_diagonal_is_neutral(orc):
    w = synth.Q1_32
    a8, beta = synth.sequence_draws(w, 0)
    u0 = orc.u0_field(w.p, w.N, a8)
    rp, col, val, b = orc.step_system(w.p, w.N, w.eps, w.dt, beta, u0)
    A = orc.Csr(rp, col, val)
    for mode, U in ((0, None), (1, _orth(np.stack([u0, synth.random_vector(len(b), 4)], 1)))):
        x, st, _ = orc.gmres(A, b, U=U, mode=mode, m=w.m, rtol=1e-10, precond=orc.PRECOND_JACOBI)
        assert st["status"] == 0 and st["true_relres"] <= 1e-10
        r = b - orc.spmv(A, x)
        assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b) * (1 + 1e-9)
    # unit diagonal: scaling by 1 changes nothing, bit for bit
    Ad = A.dense()
    Ad[np.diag_indices_from(Ad)] = 1.0
    Au = orc.Csr.from_dense(Ad)
    xa, sa, _ = orc.gmres(Au, b, m=10, rtol=1e-8, maxit=40)
    xb, sb, _ = orc.gmres(Au, b, m=10, rtol=1e-8, maxit=40, precond=orc.PRECOND_JACOBI)
    np.testing.assert_array_equal(xa, xb)
    assert sa["iters"] == sb["iters"]

