"""Pins of the oracle's Sec. 6.1 benchmark fields (cellular velocity, random
forcing, nodal-velocity assembly, step system and sequence) against closed
forms, brute force and reductions to the already pinned constant-velocity
routines."""
import numpy as np
import pytest

import synth


def _dense(rp, col, val, n):
    D = np.zeros((n, n))
    for r in range(n):
        for k in range(rp[r], rp[r + 1]):
            D[r, col[k]] += val[k]
    return D


@pytest.mark.parametrize("p,N", [(1, 8), (2, 4), (3, 4)])
def test_paper_velocity_closed_form_and_tangency(orc, p, N):
    x, y = orc.node_coords(p, N)
    bx, by = orc.paper_velocity(p, N)
    # closed form at nodes whose coordinates are exact in binary
    for xv, yv, ex, ey in [(0.5, 0.0, -1.0, 0.0), (0.0, 0.5, 0.0, 1.0),
                           (0.25, 0.25, -0.5, 0.5), (0.5, 0.5, 0.0, 0.0)]:
        i = np.nonzero((x == xv) & (y == yv))[0]
        assert len(i) == 1
        assert abs(bx[i[0]] - ex) <= 1e-15 and abs(by[i[0]] - ey) <= 1e-15
    # the field is tangential on the boundary of the unit square
    assert np.all(np.abs(bx[(x == 0.0) | (x == 1.0)]) <= 1e-15)
    assert np.all(np.abs(by[(y == 0.0) | (y == 1.0)]) <= 1e-15)


def test_paper_forcing_single_modes(orc):
    p, N = 1, 64
    x, y = orc.node_coords(p, N)
    bnd = (x == 0) | (x == 1) | (y == 0) | (y == 1)
    for j in (1, 2, 4, 8, 16):
        c = np.zeros(16)
        c[j - 1] = 1.0
        f = orc.paper_forcing(p, N, c, 0.1)
        # sin(2 j pi x) = 1 at x = 1/(4j)
        i = np.nonzero((x == 1.0 / (4 * j)) & (y == 1.0 / (4 * j)))[0][0]
        assert abs(f[i] - 0.05 * np.exp(-j * j / 20.0)) <= 1e-15
        assert np.all(np.abs(f[bnd]) <= 1e-15)
    # linear in c
    c1, c2 = synth.random_vector(16, 3), synth.random_vector(16, 4)
    f1, f2 = orc.paper_forcing(p, N, c1), orc.paper_forcing(p, N, c2)
    np.testing.assert_allclose(orc.paper_forcing(p, N, c1 + c2), f1 + f2, atol=1e-15)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_constant_nodal_field_reduces_to_constant_beta(orc, p):
    N = 4
    n = orc.ndofs(p, N)
    u = synth.random_vector(n, 11)
    bxn, byn = np.full(n, 0.3), np.full(n, -0.7)
    for dirichlet in (False, True):
        _, _, v1 = orc.assemble(p, N, 2.0, 0.1, 1.0, beta=(0.3, -0.7), u=u, dirichlet=dirichlet)
        _, _, v2 = orc.assemble_field(p, N, 2.0, 0.1, 1.0, bxn, byn, u=u, dirichlet=dirichlet)
        assert np.max(np.abs(v1 - v2)) <= 1e-14 * np.max(np.abs(v1))


def _hat(xs, xi, h):
    """1D Q1 hat function of the node at xi and its derivative at points xs
    (never on a kink)."""
    d = xs - xi
    phi = np.maximum(0.0, 1.0 - np.abs(d) / h)
    dphi = np.where(np.abs(d) < h, -np.sign(d) / h, 0.0)
    return phi, dphi


@pytest.mark.parametrize("N", [2, 3])
def test_linear_field_brute_force_q1(orc, N):
    """Q1 with linear u and b: the 2-point Gauss rule is exact, so the
    convection matrix equals brute-force quadrature over hat functions."""
    p = 1
    n = orc.ndofs(p, N)
    x, y = orc.node_coords(p, N)
    u = x + 2.0 * y
    bxn, byn = x.copy(), -2.0 * y + 0.5
    rp, col, val = orc.assemble_field(p, N, 0.0, 0.0, 1.0, bxn, byn, u=u, dirichlet=False)
    D = _dense(rp, col, val, n)
    h = 1.0 / N
    g, w = np.polynomial.legendre.leggauss(4)
    g, w = 0.5 * (g + 1.0), 0.5 * w
    ref = np.zeros((n, n))
    L = N + 1
    for cy in range(N):
        for cx in range(N):
            qx = (cx + g) * h
            qy = (cy + g) * h
            X, Y = np.meshgrid(qx, qy, indexing="ij")
            W = np.outer(w, w) * h * h
            U = X + 2.0 * Y
            BX, BY = X, -2.0 * Y + 0.5
            nodes = [(cy + b) * L + (cx + a) for b in (0, 1) for a in (0, 1)]
            vals = {}
            for d in nodes:
                px, dpx = _hat(qx, x[d], h)
                py, dpy = _hat(qy, y[d], h)
                vals[d] = (np.outer(px, py), np.outer(dpx, py), np.outer(px, dpy))
            for i in nodes:
                for j in nodes:
                    phi_i = vals[i][0]
                    ref[i, j] += np.sum(W * phi_i * U * (BX * vals[j][1] + BY * vals[j][2]))
    assert np.max(np.abs(D - ref)) <= 1e-14 * np.max(np.abs(ref))


def test_cellular_field_is_nearly_skew(orc):
    """The field is solenoidal and tangential, so N(1; b) is skew-symmetric up
    to the interpolation error of b_h (about h^3 here); a sign error in one
    component (divergence 2 pi cos pi x cos pi y) leaves an O(h) defect."""
    ratios = []
    for N in (16, 32):
        n = orc.ndofs(1, N)
        bx, by = orc.paper_velocity(1, N)
        rp, col, val = orc.assemble_field(1, N, 0.0, 0.0, 1.0, bx, by, u=np.ones(n), dirichlet=False)
        D = _dense(rp, col, val, n)
        ratios.append(np.linalg.norm(D + D.T) / np.linalg.norm(D))
        rp, col, val = orc.assemble_field(1, N, 0.0, 0.0, 1.0, -bx, by, u=np.ones(n), dirichlet=False)
        Dw = _dense(rp, col, val, n)
        assert np.linalg.norm(Dw + Dw.T) / np.linalg.norm(Dw) > 10 * ratios[-1]
    assert ratios[1] < ratios[0] / 3.0 and ratios[1] < 1e-3


def test_step_system_field_reductions(orc):
    p, N, eps, dt = 2, 4, 0.01, 0.5
    n = orc.ndofs(p, N)
    u = orc.u0_field(p, N, synth.random_vector(8, 21) * 0.5)
    beta = (0.6, 0.8)
    rp, col, val0, b0 = orc.step_system(p, N, eps, dt, beta, u)
    bxn, byn = np.full(n, beta[0]), np.full(n, beta[1])
    _, _, val1, b1 = orc.step_system_field(p, N, eps, dt, bxn, byn, None, u)
    assert np.max(np.abs(val1 - val0)) <= 1e-14 * np.max(np.abs(val0))
    assert np.max(np.abs(b1 - b0)) <= 1e-14 * np.max(np.abs(b0))
    # the nodal forcing f = 1 gives M 1 = (v, 1)
    _, _, _, b2 = orc.step_system_field(p, N, eps, dt, bxn, byn, np.ones(n), u)
    assert np.max(np.abs(b2 - b0)) <= 1e-14 * np.max(np.abs(b0))
    # the load of a nodal forcing is M f on interior rows
    f = orc.paper_forcing(p, N, synth.random_vector(16, 22))
    bz = orc.step_system_field(p, N, eps, dt, bxn, byn, np.zeros(n), u)[3]
    bf = orc.step_system_field(p, N, eps, dt, bxn, byn, f, u)[3]
    frp, fcol, mval = orc.assemble(p, N, 1.0, 0.0, 0.0, dirichlet=False)
    Mf = _dense(frp, fcol, mval, n) @ f
    x, y = orc.node_coords(p, N)
    inner = ~((x == 0) | (x == 1) | (y == 0) | (y == 1))
    assert np.max(np.abs((bf - bz)[inner] - Mf[inner])) <= 1e-14 * np.max(np.abs(Mf))
    assert np.all(bf[~inner] == 0.0)


def test_paper_sequence_first_steps_by_dense_solves(orc):
    """Zero initial value: step 1 solves (M/dt + nu K) u = M f_1 (no convection);
    step 2 uses u_1 in the convection and the second row of forcing draws."""
    w = synth.PAPER_Q1_64[0.01]
    p, N = 1, 8
    n = orc.ndofs(p, N)
    forcing = synth.forcing_draws(w, 2)
    out = orc.sequence(p, N, w.eps, w.dt, (0.0, 0.0), 2, np.zeros(n), mode=orc.PLAIN, m=40,
                       rtol=1e-13, velocity=1, forcing=forcing, keep_all=True)
    bx, by = orc.paper_velocity(p, N)
    x, y = orc.node_coords(p, N)
    inner = ~((x == 0) | (x == 1) | (y == 0) | (y == 1))
    frp, fcol, mval = orc.assemble(p, N, 1.0, 0.0, 0.0, dirichlet=False)
    M = _dense(frp, fcol, mval, n)
    _, _, kval = orc.assemble(p, N, 0.0, 1.0, 0.0, dirichlet=False)
    K = _dense(frp, fcol, kval, n)
    u = np.zeros(n)
    for step in range(2):
        _, _, cval = orc.assemble_field(p, N, 0.0, 0.0, 1.0, bx, by, u=u, dirichlet=False)
        A = M / w.dt + w.eps * K + _dense(frp, fcol, cval, n)
        rhs = M @ (u / w.dt + orc.paper_forcing(p, N, forcing[step]))
        # Dirichlet rows: identity, zero data; interior rows drop boundary columns
        A[~inner, :] = 0.0
        A[:, ~inner] = 0.0
        A[~inner, ~inner] = 1.0
        rhs[~inner] = 0.0
        u = np.linalg.solve(A, rhs)
        np.testing.assert_allclose(out["x_all"][:, step], u, rtol=0, atol=1e-11 * np.max(np.abs(u)))
    assert np.max(np.abs(u)) > 0


@pytest.mark.parametrize("p", [8, 23])
def test_high_order_rules_against_numpy(orc, p):
    """Gauss-Lobatto nodes = 0, 1 and the zeros of P_p' (numpy's Legendre
    series routines); the (p+1)-point Gauss rule = numpy's leggauss."""
    leg = np.polynomial.legendre
    roots = np.sort(leg.legroots(leg.legder([0] * p + [1])))
    np.testing.assert_allclose(orc.gll_nodes(p), np.concatenate([[0.0], (roots + 1) / 2, [1.0]]),
                               atol=1e-14)
    x, w = orc.gauss_rule(p + 1)
    xe, we = leg.leggauss(p + 1)
    np.testing.assert_allclose(x, (xe + 1) / 2, atol=1e-14)
    np.testing.assert_allclose(w, we / 2, atol=1e-14)


def test_spectral_element_forms_exact_on_polynomials(orc):
    """Order 23 on one element: the mass and stiffness integrals of
    polynomial fields in the space come out exact."""
    p, N = 23, 1
    x, y = orc.node_coords(p, N)
    pat = orc.pattern(p, N, False)
    n = len(x)
    M = _dense(*orc.assemble(p, N, 1, 0, 0, dirichlet=False, pat=pat), n)
    K = _dense(*orc.assemble(p, N, 0, 1, 0, dirichlet=False, pat=pat), n)
    one = np.ones(n)
    assert abs(one @ M @ one - 1) < 1e-12
    assert abs(x @ M @ y - 0.25) < 1e-12
    assert abs((x ** p) @ M @ y - 1 / (2 * (p + 1))) < 1e-12
    assert np.abs(K @ one).max() < 1e-9 * np.abs(K).max()
    assert abs((x ** p) @ K @ x - 1.0) < 1e-10
    np.testing.assert_allclose(M, M.T, atol=1e-16)
