"""Pins of the oracle's binary32 model in GMRES-IR (orc_gmres_ir).

The mixed-precision form (Carson and Higham's GMRES-IR) stores A's values and every
vector of the inner solve (Krylov basis V, residuals, the recycle columns U and
W = A U, the inner iterate) in binary32, does the arithmetic in binary64 and
rounds on store; W is formed from the binary32 operator and U, E = U^T W is
accumulated in binary64 from the stored columns; the outer residual b - A x,
the update x += d and the projection guess (binary64 U) are binary64.
A plausible mistake is to forget one of those roundings: the inner solve then
becomes more accurate than binary32 storage allows and every FP64 pin still
passes.  These tests catch each omission:

* closed forms on a diagonal operator with entries that binary32 cannot hold:
  the iterate after one and after two refinements, derived by hand from the
  definition (GMRES on a one-dimensional Krylov space);
* a step-by-step numpy restatement of j inner Arnoldi steps (sequential
  summation order, binary32 rounding on store) that must agree bit for bit,
  while each variant that leaves out one rounding must not;
* the accuracy floor of one refinement: an inner solve asked for 1e-12 cannot
  go below the binary32 level, while the refinement loop reaches 1e-12.
"""
import numpy as np
import pytest

import synth


def _f32(v):
    return np.asarray(v, dtype=np.float64).astype(np.float32).astype(np.float64)


# ------------------------------------------------------------------ closed forms
def _diag_csr(orc, a):
    n = len(a)
    return orc.Csr(np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), np.asarray(a, float))


def test_one_refinement_closed_form(orc):
    """A = diag(a), b = e_i: the Krylov space of the inner solve is span{e_i},
    so the inner iterate is (1 / fl32(a_i)) e_i formed in binary64 and stored in
    binary32: x_1 = fl32(1 / fl64(fl32(a_i))).  With A's values left in
    binary64 it would be fl32(1 / a_i), which differs for the a_i chosen."""
    # entries just off a binary32 number (c (1 + t 2^-26)) and two generic ones
    a = np.array([1.0 + 3 * 2.0 ** -26, 0.75 * (1 + 2 * 2.0 ** -26), 0.875 * (1 + 2.0 ** -26),
                  1.0 + 1.0 / 3.0, 11.0 + np.pi * 2.0 ** -25])
    A = _diag_csr(orc, a)
    hit = 0
    for i in range(len(a)):
        b = np.zeros(len(a))
        b[i] = 1.0
        x, st = orc.gmres_ir(A, b, m=5, rtol=1e-30, inner_rtol=1e-4, inner_cycles=1,
                             max_refinements=1)
        expect = np.zeros(len(a))
        expect[i] = _f32(1.0 / _f32(a[i]))
        np.testing.assert_array_equal(x, expect)
        assert st["refinements"] == 1 and st["iters"] == 1
        hit += int(_f32(1.0 / a[i]) != expect[i])
    assert hit >= 2          # the pin separates rounded from unrounded A values


def test_two_refinements_closed_form(orc):
    """Second refinement on the same diagonal system: r_1 = 1 - a_i x_1 in
    binary64, the inner solve returns fl32(fl64(fl32(r_1)) / fl32(a_i)) and the
    binary64 update adds it: x_2 = x_1 + d_2.  A binary32 update would round
    x_2 back to x_1 + O(ulp32)."""
    a = np.array([1.0 + 3 * 2.0 ** -26, 0.75 * (1 + 2 * 2.0 ** -26), 11.0 + np.pi * 2.0 ** -25])
    A = _diag_csr(orc, a)
    for i in range(len(a)):
        b = np.zeros(len(a))
        b[i] = 1.0
        x, st = orc.gmres_ir(A, b, m=5, rtol=1e-30, inner_rtol=1e-4, inner_cycles=1,
                             max_refinements=2)
        x1 = _f32(1.0 / _f32(a[i]))
        r1 = 1.0 - a[i] * x1
        d2 = _f32(_f32(r1) / _f32(a[i]))
        assert st["refinements"] == 2
        assert x[i] == x1 + d2 and x1 + d2 != _f32(x1 + d2)
        np.testing.assert_array_equal(np.delete(x, i), 0.0)


# ------------------------------------------------------------------ numpy restatement
class _Model:
    """j inner Arnoldi steps of one refinement, restated from the algorithm
    with every binary32 store switchable (A values, vectors, U and W)."""

    def __init__(self, rp, col, val, rA=True, rvec=True, rUW=True):
        self.rp, self.col, self.val = rp, col, np.asarray(val, float)
        self.Af = _f32(self.val) if rA else self.val
        self.rvec, self.rUW = rvec, rUW

    def rd(self, v):
        return _f32(v) if self.rvec else np.asarray(v, float)

    @staticmethod
    def dot(a, b):                         # left-to-right sum, as the C loop
        p = np.asarray(a, float) * np.asarray(b, float)
        return float(np.cumsum(p)[-1]) if len(p) else 0.0

    def spmv(self, vals, x):
        y = np.empty(len(self.rp) - 1)
        for r in range(len(y)):
            s, e = self.rp[r], self.rp[r + 1]
            y[r] = self.dot(vals[s:e], x[self.col[s:e]])
        return y

    def solve(self, b, U, m, j, inner_rtol):
        """One refinement from x_in = 0 (plain when U is None, deflated with one
        recycle column otherwise); returns the binary64 iterate."""
        n = len(b)
        x = np.zeros(n)
        if U is not None:
            u = np.asarray(U, float)[:, 0]
            # u and w = A u in binary32 (w formed with the binary32 operator),
            # E = u.w accumulated in binary64 from the stored columns
            uf = _f32(u) if self.rUW else u
            wf = self.spmv(self.Af, uf)
            wf = _f32(wf) if self.rUW else wf
            E = self.dot(uf, wf)
            r = b - self.spmv(self.val, x)             # binary64 projection guess
            cv = self.dot(u, r) / E
            x = x + u * cv
        r = b - self.spmv(self.val, x)                 # outer residual, binary64
        r = _f32(r)                                    # the inner right-hand side
        tol = inner_rtol * np.sqrt(self.dot(r, r))
        d = np.zeros(n)
        if U is not None:                              # inner projection guess
            t = self.rd(r - self.rd(self.spmv(self.Af, d)))
            d = self.rd(d + uf * (self.dot(uf, t) / E))

        def project(w):
            return self.rd(w - wf * (self.dot(uf, w) / E))

        ri = self.rd(r - self.rd(self.spmv(self.Af, d)))
        w = project(ri) if U is not None else ri
        bs = np.sqrt(self.dot(w, w))
        V = [self.rd(w / bs)]
        g = np.zeros(m + 2)
        g[0] = bs
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        J = 0
        for jj in range(min(m, j)):
            w = self.rd(self.spmv(self.Af, V[jj]))
            wn0 = np.sqrt(self.dot(w, w))
            if U is not None:
                w = project(w)
            h = np.array([self.dot(V[i], w) for i in range(jj + 1)])
            s = w.copy()
            for i in range(jj + 1):
                s = s - V[i] * h[i]
            w = self.rd(s)
            h2 = np.array([self.dot(V[i], w) for i in range(jj + 1)])
            s = w.copy()
            for i in range(jj + 1):
                s = s - V[i] * h2[i]
            w = self.rd(s)
            h = h + h2
            hn = np.sqrt(self.dot(w, w))
            col = np.zeros(m + 1)
            col[:jj + 1] = h
            col[jj + 1] = hn
            for i in range(jj):
                a_, b_ = col[i], col[i + 1]
                col[i] = cs[i] * a_ + sn[i] * b_
                col[i + 1] = -sn[i] * a_ + cs[i] * b_
            a_, b_ = col[jj], col[jj + 1]
            rr = np.hypot(a_, b_)
            cs[jj], sn[jj] = (1.0, 0.0) if rr == 0.0 else (a_ / rr, b_ / rr)
            col[jj], col[jj + 1] = rr, 0.0
            g[jj + 1] = -sn[jj] * g[jj]
            g[jj] = cs[jj] * g[jj]
            H[:, jj] = col
            J = jj + 1
            assert hn > 1e-14 * wn0 and abs(g[jj + 1]) > tol    # no early exit in the pin
            V.append(self.rd(w / hn))
        y = np.zeros(J)
        for i in range(J - 1, -1, -1):
            s = g[i]
            for t in range(i + 1, J):
                s -= H[i, t] * y[t]
            y[i] = s / H[i, i]
        s = d.copy()
        for t in range(J):
            s = s + V[t] * y[t]
        d = self.rd(s)
        if U is not None:                              # cycle-end correction
            t = self.rd(r - self.rd(self.spmv(self.Af, d)))
            d = self.rd(d + uf * (self.dot(uf, t) / E))
        return x + d


def _small_system(n, seed):
    rp, col, val = synth.random_csr(n, 6, seed, diag=5.0, min_per_row=3)
    b = synth.random_vector(n, seed + 1)
    U = synth.random_vector(n, seed + 2)[:, None]
    U = U / np.linalg.norm(U)
    return rp, col, val, b, U


@pytest.mark.parametrize("deflated", [False, True])
@pytest.mark.parametrize("j", [1, 3, 6])
def test_inner_steps_match_restatement(orc, deflated, j):
    """j inner steps of one refinement (maxit = j): the oracle equals the
    binary32-store restatement bit for bit; leaving out the rounding of A, of
    the vectors, or of U and W (deflated) changes the iterate."""
    n, m = 48, 10
    rp, col, val, b, U = _small_system(n, 900 + j)
    Uu = U if deflated else None
    x, st = orc.gmres_ir(orc.Csr(rp, col, val), b, U=Uu, mode=1 if deflated else 0, m=m,
                         rtol=1e-30, maxit=j, inner_rtol=1e-30, inner_cycles=1, max_refinements=1)
    assert st["iters"] == j and st["refinements"] == 1
    ref = _Model(rp, col, val).solve(b, Uu, m, j, 1e-30)
    np.testing.assert_array_equal(x, ref)
    variants = [dict(rA=False), dict(rvec=False)] + ([dict(rUW=False)] if deflated else [])
    for kw in variants:
        alt = _Model(rp, col, val, **kw).solve(b, Uu, m, j, 1e-30)
        assert np.max(np.abs(alt - x)) > 1e-12 * np.max(np.abs(x)), kw


def test_one_refinement_accuracy_floor(orc):
    """An inner solve asked for 1e-12 stops near the binary32 level (its
    vectors cannot carry more), while the binary64 refinement loop reaches
    1e-12 on the same system."""
    w = synth.Q1_32
    a8, beta = synth.sequence_draws(w, 0)
    rp, col, val, b = orc.step_system(1, 16, w.eps, w.dt, beta, orc.u0_field(1, 16, a8))
    A = orc.Csr(rp, col, val)
    x1, s1 = orc.gmres_ir(A, b, m=60, rtol=1e-12, inner_rtol=1e-12, inner_cycles=3,
                          max_refinements=1)
    assert s1["refinements"] == 1
    assert 1e-10 < s1["true_relres"] < 1e-5
    x, s = orc.gmres_ir(A, b, m=60, rtol=1e-12, inner_rtol=1e-4, inner_cycles=2)
    assert s["status"] == 0 and s["true_relres"] <= 1e-12 and s["refinements"] >= 3


def test_ir_sequence_matches_step_solves(orc):
    """The sequence driver's GMRES-IR mode (Algorithm 1 with every solve a
    GMRES-IR solve) equals step-by-step calls: each stored x_i reproduces
    gmres_ir on its own re-assembled system with the recycle space of the
    window before it, iterations and refinements included."""
    w = synth.Q1_32
    a8, beta = synth.sequence_draws(w, 0)
    p, N, steps, k, win = 1, 16, 6, 3, 4
    u0 = orc.u0_field(p, N, a8)
    r = orc.sequence(p, N, w.eps, w.dt, beta, steps, u0, mode=1, m=20, k=k, window=win,
                     rtol=1e-8, keep_all=True, precision=1, inner_rtol=1e-4, inner_cycles=2)
    u, X = u0, []
    for i in range(steps):
        rp, col, val, b = orc.step_system(p, N, w.eps, w.dt, beta, u)
        U = None
        if X:
            U = orc.recycle_from_window(np.stack(X[-win:], 1), k)
        x, st = orc.gmres_ir(orc.Csr(rp, col, val), b, x_in=np.zeros_like(b) if U is not None else u,
                             U=U, mode=1, m=20, rtol=1e-8, inner_rtol=1e-4, inner_cycles=2)
        np.testing.assert_array_equal(x, r["x_all"][:, i])
        assert st["iters"] == r["iters"][i] and st["refinements"] == r["refinements"][i]
        assert st["true_relres"] <= 1e-8 and st["refinements"] >= 2
        X.append(x)
        u = x


def test_inner_stop_capped_at_half_the_target(orc):
    """The inner solve stops at max(inner_rtol ||r||, rtol ||b|| / 2): asked for
    an unattainable inner_rtol of 1e-14 with rtol 1e-6, it stops where binary64
    GMRES from the same start reaches rtol / 2 (within one step), and one
    refinement meets the target.  Without the cap it would run all of its
    inner cycles (2 m steps)."""
    w = synth.Q1_32
    a8, beta = synth.sequence_draws(w, 0)
    rp, col, val, b = orc.step_system(1, 16, w.eps, w.dt, beta, orc.u0_field(1, 16, a8))
    A = orc.Csr(rp, col, val)
    m = 30
    x, st = orc.gmres_ir(A, b, m=m, rtol=1e-6, inner_rtol=1e-14, inner_cycles=2)
    _, s64, _ = orc.gmres(A, b, m=m, rtol=0.5e-6)
    assert st["refinements"] == 1 and st["status"] == 0 and st["true_relres"] <= 1e-6
    assert abs(st["iters"] - s64["iters"]) <= 1 and st["iters"] < 2 * m, (st, s64)
