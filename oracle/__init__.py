"""FP64 CPU oracle for recycled GMRES(m) (arXiv 1807.09467) -- TEST INFRASTRUCTURE.

Only the tests, the smoke check and the benchmark's CPU-baseline leg import this
package.  It wraps the plain C sources in this directory (compiled with gcc into
``oracle/_build/liboracle.so``) through ctypes and shares no code with the CUDA
library.  Each wrapper cites the passage its C routine follows; see the headers
of fe.c, gmres.c, svd.c and sequence.c.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = ["fe.c", "gmres.c", "svd.c", "sequence.c"]
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None
_lock = threading.Lock()

PLAIN, DEFLATED, AUGMENTED, GUESS = 0, 1, 2, 3
PROJ_OBLIQUE, PROJ_ORTHOGONAL, PROJ_LS = 0, 1, 2
PRECOND_NONE, PRECOND_JACOBI = 0, 1
OK, W_NOT_CONVERGED, W_SINGULAR_COARSE = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle C sources with gcc (plain -O2, no fast-math, no FMA contraction)."""
    srcs = [os.path.join(_HERE, s) for s in _SRCS]
    hdr = os.path.join(_HERE, "oracle.h")
    if not force and os.path.exists(_LIB_PATH):
        t = os.path.getmtime(_LIB_PATH)
        if all(os.path.getmtime(s) <= t for s in srcs + [hdr]):
            return _LIB_PATH
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    # -ffp-contract=off: every operation rounds as written (no fused multiply-add
    # on targets where the compiler would contract), so results agree across hosts
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off",
           "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Csr(C.Structure):
    _fields_ = [("n", C.c_int64), ("rowptr", C.c_void_p), ("col", C.c_void_p), ("val", C.c_void_p)]


class _Opts(C.Structure):
    _fields_ = [("mode", C.c_int), ("m", C.c_int), ("rtol", C.c_double), ("maxit", C.c_int),
                ("start_r", C.c_int), ("proj", C.c_int), ("precond", C.c_int)]


class _Stats(C.Structure):
    _fields_ = [("iters", C.c_int), ("cycles", C.c_int), ("k_used", C.c_int), ("status", C.c_int),
                ("true_relres", C.c_double)]


class _SeqCfg(C.Structure):
    _fields_ = [("p", C.c_int), ("N", C.c_int), ("eps", C.c_double), ("dt", C.c_double),
                ("bx", C.c_double), ("by", C.c_double), ("steps", C.c_int), ("mode", C.c_int),
                ("m", C.c_int), ("k", C.c_int), ("window", C.c_int), ("ell", C.c_int),
                ("select_smallest", C.c_int), ("rtol", C.c_double), ("maxit", C.c_int),
                ("rel_drop", C.c_double), ("guess", C.c_int), ("velocity", C.c_int),
                ("nmodes", C.c_int), ("fC", C.c_double), ("forcing", C.c_void_p),
                ("proj", C.c_int), ("precond", C.c_int), ("precision", C.c_int),
                ("inner_rtol", C.c_double), ("inner_cycles", C.c_int), ("max_refinements", C.c_int)]


SCALAR_FN = C.CFUNCTYPE(C.c_double, C.c_double, C.c_double, C.c_void_p)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            L = _lib
            L.orc_fe_ndofs.restype = C.c_int64
            L.orc_fe_ndofs.argtypes = [C.c_int, C.c_int]
            L.orc_gll_nodes.argtypes = [C.c_int, C.c_void_p]
            L.orc_gauss_rule.argtypes = [C.c_int, C.c_void_p, C.c_void_p]
            L.orc_lagrange.argtypes = [C.c_int, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p]
            L.orc_fe_node_coords.argtypes = [C.c_int, C.c_int, C.c_void_p, C.c_void_p]
            L.orc_fe_u0.argtypes = [C.c_int, C.c_int, C.c_void_p, C.c_void_p]
            L.orc_spmv.argtypes = [C.POINTER(_Csr), C.c_void_p, C.c_void_p]
            L.orc_fe_pattern.restype = C.c_int64
            L.orc_fe_pattern.argtypes = [C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p]
            L.orc_fe_assemble.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                          C.c_double, C.c_double, C.c_void_p, C.c_int,
                                          C.c_void_p, C.c_void_p, C.c_void_p]
            L.orc_fe_load.argtypes = [C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
            L.orc_fe_step_system.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                             C.c_double, C.c_void_p, C.c_void_p, C.c_void_p,
                                             C.c_void_p, C.c_void_p]
            L.orc_fe_assemble_field.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double,
                                                C.c_double, C.c_void_p, C.c_void_p, C.c_void_p,
                                                C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
            L.orc_fe_step_system_field.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double,
                                                   C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                                   C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
            L.orc_fe_paper_velocity.argtypes = [C.c_int, C.c_int, C.c_void_p, C.c_void_p]
            L.orc_fe_paper_forcing.argtypes = [C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_double,
                                               C.c_void_p]
            L.orc_gmres.argtypes = [C.POINTER(_Csr), C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                    C.POINTER(_Opts), C.POINTER(_Stats), C.c_void_p, C.c_int]
            L.orc_gmres_ir.argtypes = [C.POINTER(_Csr), C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                       C.POINTER(_Opts), C.c_double, C.c_int, C.c_int,
                                       C.POINTER(_Stats), C.POINTER(C.c_int)]
            L.orc_apply_oblique.argtypes = [C.c_int64, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                            C.c_void_p, C.c_void_p]
            L.orc_apply_projector.argtypes = [C.c_int64, C.c_int, C.c_void_p, C.c_void_p, C.c_int,
                                              C.c_void_p, C.c_void_p]
            L.orc_extrapolate.argtypes = [C.c_int64, C.c_int, C.c_void_p, C.c_int64, C.c_void_p]
            L.orc_coarse_setup.argtypes = [C.POINTER(_Csr), C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]
            L.orc_svd_left.argtypes = [C.c_int64, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
            L.orc_recycle_from_window.argtypes = [C.c_int64, C.c_int, C.c_void_p, C.c_int, C.c_int,
                                                  C.c_double, C.c_void_p, C.POINTER(C.c_int)]
            L.orc_sequence.argtypes = [C.POINTER(_SeqCfg), C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
            L.orc_sequence_timed.argtypes = [C.POINTER(_SeqCfg), C.c_void_p, C.c_void_p, C.c_void_p,
                                             C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                             C.c_void_p, C.c_void_p]
        return _lib


def _p(a):
    return a.ctypes.data if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _colmajor(a):
    """(n, k) array -> column-major float64 buffer."""
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


# ---------------------------------------------------------------- FE (fe.c)
def gll_nodes(p):
    out = np.zeros(p + 1)
    assert lib().orc_gll_nodes(p, _p(out)) == 0
    return out


def gauss_rule(q):
    x, w = np.zeros(q), np.zeros(q)
    assert lib().orc_gauss_rule(q, _p(x), _p(w)) == 0
    return x, w


def lagrange(p, nodes, x):
    phi, dphi = np.zeros(p + 1), np.zeros(p + 1)
    nodes = _f64(nodes)
    lib().orc_lagrange(p, _p(nodes), C.c_double(x), _p(phi), _p(dphi))
    return phi, dphi


def ndofs(p, N):
    return int(lib().orc_fe_ndofs(p, N))


def node_coords(p, N):
    n = ndofs(p, N)
    x, y = np.zeros(n), np.zeros(n)
    lib().orc_fe_node_coords(p, N, _p(x), _p(y))
    return x, y


def pattern(p, N, dirichlet=True):
    n = ndofs(p, N)
    nnz = int(lib().orc_fe_pattern(p, N, int(dirichlet), None, None))
    rowptr = np.zeros(n + 1, dtype=np.int64)
    col = np.zeros(nnz, dtype=np.int32)
    lib().orc_fe_pattern(p, N, int(dirichlet), _p(rowptr), _p(col))
    return rowptr, col


def assemble(p, N, cm, ck, cn, beta=(0.0, 0.0), u=None, dirichlet=True, pat=None):
    """val = cm*M + ck*K + cn*N(u; beta) on the (Dirichlet or full) pattern."""
    rowptr, col = pat if pat is not None else pattern(p, N, dirichlet)
    val = np.zeros(len(col))
    uu = _f64(u) if u is not None else None
    rc = lib().orc_fe_assemble(p, N, cm, ck, cn, beta[0], beta[1], _p(uu), int(dirichlet),
                               _p(rowptr), _p(col), _p(val))
    assert rc == 0, rc
    return rowptr, col, val


def load(p, N, f=None):
    n = ndofs(p, N)
    F = np.zeros(n)
    cb = SCALAR_FN(lambda x, y, ctx: float(f(x, y))) if f is not None else None
    lib().orc_fe_load(p, N, C.cast(cb, C.c_void_p) if cb else None, None, _p(F))
    return F


def step_system(p, N, eps, dt, beta, u_prev, pat=None):
    """(rowptr, col, val, b) of one implicit-Euler step (Sec. 6.1, Dirichlet rows)."""
    rowptr, col = pat if pat is not None else pattern(p, N, True)
    val = np.zeros(len(col))
    b = np.zeros(ndofs(p, N))
    u = _f64(u_prev)
    rc = lib().orc_fe_step_system(p, N, eps, dt, beta[0], beta[1], _p(u), _p(rowptr), _p(col),
                                  _p(val), _p(b))
    assert rc == 0, rc
    return rowptr, col, val, b


def assemble_field(p, N, cm, ck, cn, bxn, byn, u=None, dirichlet=True, pat=None):
    """val = cm*M + ck*K + cn*N(u; b_h), b_h the interpolant of nodal (bxn, byn)."""
    rowptr, col = pat if pat is not None else pattern(p, N, dirichlet)
    val = np.zeros(len(col))
    uu = _f64(u) if u is not None else None
    bx, by = _f64(bxn), _f64(byn)
    rc = lib().orc_fe_assemble_field(p, N, cm, ck, cn, _p(bx), _p(by), _p(uu), int(dirichlet),
                                     _p(rowptr), _p(col), _p(val))
    assert rc == 0, rc
    return rowptr, col, val


def paper_velocity(p, N):
    """Sec. 6.1's cellular field at the nodes: (bxn, byn)."""
    n = ndofs(p, N)
    bx, by = np.zeros(n), np.zeros(n)
    assert lib().orc_fe_paper_velocity(p, N, _p(bx), _p(by)) == 0
    return bx, by


def paper_forcing(p, N, c, C_amp=0.1):
    """Sec. 6.1's forcing with mode coefficients c (c[0] = c_1) at the nodes."""
    c = _f64(c)
    out = np.zeros(ndofs(p, N))
    assert lib().orc_fe_paper_forcing(p, N, len(c), _p(c), C_amp, _p(out)) == 0
    return out


def step_system_field(p, N, eps, dt, bxn, byn, fn, u_prev, pat=None):
    """(rowptr, col, val, b) of one step with a nodal velocity and nodal forcing
    (fn None: f = 1)."""
    rowptr, col = pat if pat is not None else pattern(p, N, True)
    val = np.zeros(len(col))
    b = np.zeros(ndofs(p, N))
    bx, by, u = _f64(bxn), _f64(byn), _f64(u_prev)
    f = _f64(fn) if fn is not None else None
    rc = lib().orc_fe_step_system_field(p, N, eps, dt, _p(bx), _p(by), _p(f), _p(u), _p(rowptr),
                                        _p(col), _p(val), _p(b))
    assert rc == 0, rc
    return rowptr, col, val, b


def u0_field(p, N, a8):
    a8 = _f64(a8)
    out = np.zeros(ndofs(p, N))
    lib().orc_fe_u0(p, N, _p(a8), _p(out))
    return out


# ---------------------------------------------------------------- GMRES (gmres.c)
class Csr:
    """Keeps numpy buffers alive for the C struct."""

    def __init__(self, rowptr, col, val):
        self.rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.val = _f64(val)
        self.n = len(self.rowptr) - 1
        self.s = _Csr(self.n, _p(self.rowptr), _p(self.col), _p(self.val))

    @staticmethod
    def from_dense(A):
        A = np.asarray(A, dtype=np.float64)
        rowptr, col, val = [0], [], []
        for r in range(A.shape[0]):
            nz = np.nonzero(A[r])[0]
            col.extend(nz.tolist())
            val.extend(A[r, nz].tolist())
            rowptr.append(len(col))
        return Csr(np.array(rowptr), np.array(col, dtype=np.int32), np.array(val))

    def dense(self):
        D = np.zeros((self.n, self.n))
        for r in range(self.n):
            for k in range(self.rowptr[r], self.rowptr[r + 1]):
                D[r, self.col[k]] += self.val[k]
        return D


def spmv(A: Csr, x):
    x = _f64(x)
    y = np.zeros(A.n)
    lib().orc_spmv(C.byref(A.s), _p(x), _p(y))
    return y


def gmres(A: Csr, b, x_in=None, U=None, mode=PLAIN, m=30, rtol=1e-10, maxit=10000,
          start_r=False, hist_len=0, proj=PROJ_OBLIQUE, precond=0):
    """Returns (x, stats dict, hist)."""
    b = _f64(b)
    x = _f64(x_in).copy() if x_in is not None else np.zeros(A.n)
    k = 0
    Uc = None
    if U is not None and np.asarray(U).size:
        Uc = _colmajor(U)
        k = Uc.shape[1]
    o = _Opts(mode, m, rtol, maxit, int(start_r), int(proj), int(precond))
    st = _Stats()
    hist = np.zeros(hist_len) if hist_len else None
    rc = lib().orc_gmres(C.byref(A.s), _p(b), _p(x), _p(Uc), k, C.byref(o), C.byref(st),
                         _p(hist), hist_len)
    assert rc >= 0, rc
    stats = dict(iters=st.iters, cycles=st.cycles, k_used=st.k_used, status=st.status,
                 true_relres=st.true_relres)
    if hist is not None:
        hist = hist[: st.iters] if st.iters <= hist_len else hist
    return x, stats, hist


def gmres_ir(A: Csr, b, x_in=None, U=None, mode=PLAIN, m=30, rtol=1e-8, maxit=20000,
             inner_rtol=1e-4, inner_cycles=2, max_refinements=50, proj=PROJ_OBLIQUE):
    b = _f64(b)
    x = _f64(x_in).copy() if x_in is not None else np.zeros(A.n)
    k, Uc = 0, None
    if U is not None and np.asarray(U).size:
        Uc = _colmajor(U)
        k = Uc.shape[1]
    o = _Opts(mode, m, rtol, maxit, 0, int(proj), 0)
    st = _Stats()
    nref = C.c_int(0)
    rc = lib().orc_gmres_ir(C.byref(A.s), _p(b), _p(x), _p(Uc), k, C.byref(o), inner_rtol,
                            inner_cycles, max_refinements, C.byref(st), C.byref(nref))
    assert rc >= 0, rc
    return x, dict(iters=st.iters, cycles=st.cycles, k_used=st.k_used, status=st.status,
                   true_relres=st.true_relres, refinements=nref.value)


def coarse_setup(A: Csr, U):
    Uc = _colmajor(U)
    k = Uc.shape[1]
    W = np.zeros((A.n, k), order="F")
    E = np.zeros((k, k), order="F")
    lib().orc_coarse_setup(C.byref(A.s), _p(Uc), k, _p(W), _p(E))
    return W, E


def apply_oblique(U, W, E, v):
    Uc, Wc, Ec = _colmajor(U), _colmajor(W), _colmajor(E)
    v = _f64(v)
    out = np.zeros_like(v)
    rc = lib().orc_apply_oblique(Uc.shape[0], Uc.shape[1], _p(Uc), _p(Wc), _p(Ec), _p(v), _p(out))
    return out, rc


def extrapolate(P):
    """Eq. ext2-ext4: column j of P is x_{i-1-j}; returns x0 (order P.shape[1]-1)."""
    Pc = _colmajor(P)
    n, s = Pc.shape
    out = np.zeros(n)
    rc = lib().orc_extrapolate(n, s, _p(Pc), n, _p(out))
    assert rc == 0, rc
    return out


def apply_projector(U, W, proj, v):
    """P v for the projector proj (PROJ_*) of Table 1, W = A U."""
    Uc, Wc = _colmajor(U), _colmajor(W)
    v = _f64(v)
    out = np.zeros_like(v)
    rc = lib().orc_apply_projector(Uc.shape[0], Uc.shape[1], _p(Uc), _p(Wc), int(proj), _p(v),
                                   _p(out))
    return out, rc


# ---------------------------------------------------------------- SVD (svd.c)
def svd_left(X):
    Xc = _colmajor(X)
    n, c = Xc.shape
    sigma = np.zeros(c)
    Psi = np.zeros((n, c), order="F")
    rc = lib().orc_svd_left(n, c, _p(Xc), _p(sigma), _p(Psi))
    assert rc == 0, rc
    return sigma, Psi


def recycle_from_window(X, k, select_smallest=False, rel_drop=1e-7):
    Xc = _colmajor(X)
    n, c = Xc.shape
    U = np.zeros((n, max(k, 1)), order="F")
    ke = C.c_int(0)
    rc = lib().orc_recycle_from_window(n, c, _p(Xc), k, int(select_smallest), rel_drop, _p(U),
                                       C.byref(ke))
    assert rc == 0, rc
    return U[:, : ke.value].copy(order="F")


# ---------------------------------------------------------------- Algorithm 1 (sequence.c)
def sequence(p, N, eps, dt, beta, steps, u0, mode=PLAIN, m=30, k=8, window=16, ell=1,
             rtol=1e-10, maxit=20000, select_smallest=False, rel_drop=1e-7, keep_all=False,
             guess=0, velocity=0, forcing=None, forcing_C=0.1, proj=PROJ_OBLIQUE, precond=0,
             precision=0, inner_rtol=1e-4, inner_cycles=2, max_refinements=50):
    """velocity 1 / forcing (steps x nmodes coefficients): Sec. 6.1's benchmark.
    precision 1: every solve is GMRES-IR (gmres_ir) with the inner parameters given."""
    n = ndofs(p, N)
    fc = np.ascontiguousarray(forcing, dtype=np.float64) if forcing is not None else None
    nmodes = fc.shape[1] if fc is not None else 0
    if fc is not None:
        assert fc.shape[0] >= steps
    cfg = _SeqCfg(p, N, eps, dt, beta[0], beta[1], steps, mode, m, k, window, ell,
                  int(select_smallest), rtol, maxit, rel_drop, int(guess), int(velocity), nmodes,
                  forcing_C, _p(fc), int(proj), int(precond), int(precision), inner_rtol,
                  int(inner_cycles), int(max_refinements))
    u0 = _f64(u0)
    x_all = np.zeros((n, steps), order="F") if keep_all else None
    x_final = np.zeros(n)
    iters = np.zeros(steps, dtype=np.int32)
    k_used = np.zeros(steps, dtype=np.int32)
    relres = np.zeros(steps)
    status = np.zeros(steps, dtype=np.int32)
    secs = np.zeros(steps)
    nref = np.zeros(steps, dtype=np.int32)
    rc = lib().orc_sequence_timed(C.byref(cfg), _p(u0), _p(x_all), _p(x_final), _p(iters),
                                  _p(k_used), _p(relres), _p(status), _p(secs), _p(nref))
    assert rc == 0, rc
    return dict(x_final=x_final, x_all=x_all, iters=iters, k_used=k_used, relres=relres,
                status=status, step_seconds=secs, refinements=nref)
