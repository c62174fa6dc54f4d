"""Pins of the oracle's finite-element system (Sec. 2 Eq. def_Axb, Sec. 6.1).

Each check is fixed by mathematics independent of the oracle: textbook quadrature
closed forms, Q1 stencils, exact integrals of polynomial fields, conservation
identities, a brute-force pattern from element connectivity and a manufactured
solution's convergence rate.
"""
import json
import math
import os

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _ev(s):
    return eval(s, {"sqrt": math.sqrt})


def test_gauss_rule_closed_forms(orc):
    g = json.load(open(os.path.join(GOLD, "quadrature.json")))["gauss"]
    for q, d in g.items():
        x, w = orc.gauss_rule(int(q))
        xe = np.array([(_ev(s) + 1) / 2 for s in d["x"]])
        we = np.array([_ev(s) / 2 for s in d["w"]])
        np.testing.assert_allclose(x, xe, rtol=0, atol=1e-15)
        np.testing.assert_allclose(w, we, rtol=0, atol=1e-15)


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5, 6, 9])
def test_gauss_rule_exactness(orc, q):
    x, w = orc.gauss_rule(q)
    for deg in range(2 * q):
        assert abs(np.dot(w, x ** deg) - 1.0 / (deg + 1)) < 1e-14
    # degree 2q is not integrated exactly
    assert abs(np.dot(w, x ** (2 * q)) - 1.0 / (2 * q + 1)) > 1e-12


def test_gll_closed_forms(orc):
    g = json.load(open(os.path.join(GOLD, "quadrature.json")))["gll"]
    for p, d in g.items():
        np.testing.assert_allclose(orc.gll_nodes(int(p)), [(_ev(s) + 1) / 2 for s in d], atol=1e-15)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_lagrange_basis(orc, p):
    nodes = orc.gll_nodes(p)
    for b in range(p + 1):
        phi, _ = orc.lagrange(p, nodes, nodes[b])
        np.testing.assert_allclose(phi, np.eye(p + 1)[b], atol=1e-14)
    for x in [0.0, 0.123, 0.5, 0.77, 1.0]:
        phi, dphi = orc.lagrange(p, nodes, x)
        assert abs(phi.sum() - 1) < 1e-14 and abs(dphi.sum()) < 1e-12
        h = 1e-6
        fp, _ = orc.lagrange(p, nodes, x + h)
        fm, _ = orc.lagrange(p, nodes, x - h)
        np.testing.assert_allclose(dphi, (fp - fm) / (2 * h), atol=1e-7)
        # reproduces x^p exactly
        assert abs(np.dot(phi, nodes ** p) - x ** p) < 1e-13


def _brute_pattern(p, N, dirichlet):
    L = p * N + 1
    rows = [set() for _ in range(L * L)]
    for cy in range(N):
        for cx in range(N):
            dofs = [(cy * p + b) * L + cx * p + a for b in range(p + 1) for a in range(p + 1)]
            for i in dofs:
                rows[i].update(dofs)

    def bnd(d):
        ix, iy = d % L, d // L
        return ix in (0, L - 1) or iy in (0, L - 1)
    rp, col = [0], []
    for r in range(L * L):
        if dirichlet and bnd(r):
            cs = [r]
        else:
            cs = sorted(c for c in rows[r] if not (dirichlet and bnd(c)))
        col.extend(cs)
        rp.append(len(col))
    return np.array(rp), np.array(col)


@pytest.mark.parametrize("p,N", [(1, 3), (2, 2), (3, 2), (4, 3)])
@pytest.mark.parametrize("dirichlet", [False, True])
def test_pattern_brute_force(orc, p, N, dirichlet):
    rp, col = orc.pattern(p, N, dirichlet)
    rpb, colb = _brute_pattern(p, N, dirichlet)
    np.testing.assert_array_equal(rp, rpb)
    np.testing.assert_array_equal(col, colb)


def test_pattern_sizes_of_workloads(orc):
    # dof counts fixed by the workloads' (pN+1)^2; nnz cross-checked with the
    # brute-force pattern on small grids above
    assert orc.ndofs(1, 32) == 1089 and orc.ndofs(2, 128) == 66049 and orc.ndofs(4, 256) == 1050625
    rp, _ = orc.pattern(1, 32)
    assert rp[-1] == 8409 and np.diff(rp).max() == 9


def test_q1_stencils(orc):
    g = json.load(open(os.path.join(GOLD, "q1_stencils.json")))
    N = 8
    h = 1.0 / N
    L = N + 1
    pat = orc.pattern(1, N, False)
    rp, col, M = orc.assemble(1, N, 1, 0, 0, dirichlet=False, pat=pat)
    _, _, K = orc.assemble(1, N, 0, 1, 0, dirichlet=False, pat=pat)
    r = 4 * L + 4                       # an interior node
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            c = r + dy * L + dx
            k = rp[r] + np.searchsorted(col[rp[r]:rp[r + 1]], c)
            assert abs(M[k] - g["mass_over_h2"][dy + 1][dx + 1] * h * h) < 1e-16
            assert abs(K[k] - g["stiffness"][dy + 1][dx + 1]) < 1e-14


def _dense(orc, rp, col, val):
    return orc.Csr(rp, col, val).dense()


@pytest.mark.parametrize("p,N", [(1, 4), (2, 3), (3, 2), (4, 2)])
def test_bilinear_forms_exact_on_polynomials(orc, p, N):
    x, y = orc.node_coords(p, N)
    pat = orc.pattern(p, N, False)
    M = _dense(orc, *orc.assemble(p, N, 1, 0, 0, dirichlet=False, pat=pat))
    K = _dense(orc, *orc.assemble(p, N, 0, 1, 0, dirichlet=False, pat=pat))
    one = np.ones_like(x)
    # mass: integral of 1 = 1, of x*y = 1/4, of x^p * y = 1/(2(p+1))
    assert abs(one @ M @ one - 1) < 1e-13
    assert abs(x @ M @ y - 0.25) < 1e-13
    assert abs((x ** p) @ M @ y - 1 / (2 * (p + 1))) < 1e-13
    # stiffness: K 1 = 0, integral of grad x^p . grad x = integral p x^(p-1) = 1
    assert np.abs(K @ one).max() < 1e-12
    assert abs((x ** p) @ K @ x - 1.0) < 1e-12
    assert abs(x @ K @ y) < 1e-13
    np.testing.assert_allclose(M, M.T, atol=1e-16)
    np.testing.assert_allclose(K, K.T, atol=1e-13)
    assert np.linalg.eigvalsh(K).min() > -1e-12
    # convection N(u; beta)_ij = (u beta.grad phi_j, phi_i)
    beta = (0.3, -0.7)
    Nu = _dense(orc, *orc.assemble(p, N, 0, 0, 1, beta=beta, u=x, dirichlet=False, pat=pat))
    # w=1, u=x, v=y: integral of x * beta_y = beta_y / 2
    assert abs(one @ Nu @ y - beta[1] / 2) < 1e-13
    # w=y, u=x, v=x: integral of y x beta_x = beta_x / 4
    assert abs(y @ Nu @ x - beta[0] / 4) < 1e-13
    # N(u) 1 = 0 (grad of a constant vanishes)
    assert np.abs(Nu @ one).max() < 1e-13


@pytest.mark.parametrize("p,N", [(1, 6), (2, 3), (4, 2)])
def test_convection_skew_on_interior(orc, p, N):
    """For u = 1: v^T N w + w^T N v = integral of beta.grad(v w) = 0 for v, w
    vanishing on the boundary, so the interior block is skew-symmetric."""
    x, y = orc.node_coords(p, N)
    pat = orc.pattern(p, N, False)
    Nd = _dense(orc, *orc.assemble(p, N, 0, 0, 1, beta=(0.6, 0.8), u=np.ones_like(x),
                                   dirichlet=False, pat=pat))
    inner = (x > 0) & (x < 1) & (y > 0) & (y < 1)
    Ni = Nd[np.ix_(inner, inner)]
    np.testing.assert_allclose(Ni + Ni.T, 0, atol=1e-14)
    assert np.abs(Ni).max() > 1e-3


def test_dirichlet_rows_and_interior_block(orc):
    p, N = 2, 3
    x, y = orc.node_coords(p, N)
    u = np.sin(3 * x) * np.cos(2 * y)
    full = _dense(orc, *orc.assemble(p, N, 2.0, 0.1, 1.0, beta=(1, 1), u=u, dirichlet=False))
    dir_ = _dense(orc, *orc.assemble(p, N, 2.0, 0.1, 1.0, beta=(1, 1), u=u, dirichlet=True))
    bnd = (x == 0) | (x == 1) | (y == 0) | (y == 1)
    inner = ~bnd
    np.testing.assert_allclose(dir_[np.ix_(inner, inner)], full[np.ix_(inner, inner)], atol=1e-15)
    np.testing.assert_array_equal(dir_[bnd], np.eye(len(x))[bnd])
    assert np.all(dir_[np.ix_(inner, bnd)] == 0)


def test_step_system_rhs(orc):
    p, N, dt = 2, 4, 0.01
    x, y = orc.node_coords(p, N)
    u = x * (1 - x) * y * (1 - y)
    rp, col, val, b = orc.step_system(p, N, 0.05, dt, (1, 1), u)
    M = _dense(orc, *orc.assemble(p, N, 1, 0, 0, dirichlet=False))
    F = orc.load(p, N)
    assert abs(F.sum() - 1.0) < 1e-13            # integral of f = 1 over the square
    bnd = (x == 0) | (x == 1) | (y == 0) | (y == 1)
    expect = M @ u / dt + F
    np.testing.assert_allclose(b[~bnd], expect[~bnd], rtol=1e-14, atol=1e-14)
    assert np.all(b[bnd] == 0)
    # the matrix is M/dt + eps K + N(u) with identity Dirichlet rows
    A = _dense(orc, rp, col, val)
    A2 = _dense(orc, *orc.assemble(p, N, 1 / dt, 0.05, 1.0, beta=(1, 1), u=u, dirichlet=True))
    np.testing.assert_allclose(A, A2, atol=1e-12)


def test_u0_interpolation(orc):
    p, N = 3, 4
    a8 = np.linspace(-0.5, 0.5, 8)
    x, y = orc.node_coords(p, N)
    u0 = orc.u0_field(p, N, a8)
    ex = sum(a8[j - 1] * np.sin(j * np.pi * x) * np.sin(j * np.pi * y) for j in range(1, 9))
    bnd = (x == 0) | (x == 1) | (y == 0) | (y == 1)
    np.testing.assert_allclose(u0[~bnd], ex[~bnd], atol=1e-15)
    assert np.all(u0[bnd] == 0)


def _manufactured_error(orc, p, N):
    """Stationary manufactured solution u = sin(pi x) sin(pi y) of one implicit
    step with u_prev = I_h u: f = -eps Lap u + u beta.grad u."""
    eps, dt, beta = 0.05, 1.0, (0.8, 0.6)
    x, y = orc.node_coords(p, N)
    uex = np.sin(np.pi * x) * np.sin(np.pi * y)

    def f(X, Y):
        u = math.sin(math.pi * X) * math.sin(math.pi * Y)
        ux = math.pi * math.cos(math.pi * X) * math.sin(math.pi * Y)
        uy = math.pi * math.sin(math.pi * X) * math.cos(math.pi * Y)
        return 2 * eps * math.pi ** 2 * u + u * (beta[0] * ux + beta[1] * uy)
    pat = orc.pattern(p, N, True)
    rp, col, val = orc.assemble(p, N, 1 / dt, eps, 1.0, beta=beta, u=uex, dirichlet=True, pat=pat)
    M = _dense(orc, *orc.assemble(p, N, 1, 0, 0, dirichlet=False))
    b = M @ uex / dt + orc.load(p, N, f)
    bnd = (x == 0) | (x == 1) | (y == 0) | (y == 1)
    b[bnd] = 0
    A = orc.Csr(rp, col, val)
    uh, st, _ = orc.gmres(A, b, m=200, rtol=1e-13)
    assert st["true_relres"] <= 1e-13
    e = uh - uex
    return math.sqrt(e @ M @ e)


@pytest.mark.parametrize("p", [1, 2])
def test_manufactured_solution_rate(orc, p):
    e1 = _manufactured_error(orc, p, 4)
    e2 = _manufactured_error(orc, p, 8)
    rate = math.log2(e1 / e2)
    assert rate > p + 0.7, (e1, e2, rate)
