"""GB300-native recycled GMRES(m) for sequences of convection-diffusion systems.

Thin binding over librgmres (include/rgmres.h).  Every step of the solve runs in
the library's CUDA kernels; this module only marshals arguments.  Arrays are
numpy arrays (host; the library copies) or CUDA torch tensors (device pointers,
used in place on the solver's stream).

Method: Pitton & Heltai, arXiv 1807.09467 -- restarted GMRES (Sec. 3) with a
recycle space from a thin SVD of previous solutions (Sec. 5.2, Algorithm 1) used
for deflation (Sec. 3.2, Table 1) or augmentation (Sec. 3.1).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import (AUGMENTED, DEFLATED, FP32_IR, FP64, GUESS, PLAIN, RGM_BATCH_COOP, RGM_DEVICE_PTRS,
                   RGM_ZERO_GUESS, RGM_W_NOT_CONVERGED, RGM_W_SINGULAR_COARSE, RgmConfig, RgmError,
                   RgmStats, check)

MODES = {"plain": PLAIN, "deflated": DEFLATED, "augmented": AUGMENTED, "guess": GUESS}
PRECISIONS = {"fp64": FP64, "fp32_ir": FP32_IR}
LAUNCH_POLICIES = {"auto": 0, "per_pass": 1}
PROJECTORS = {"oblique": 0, "orthogonal": 1, "ls": 2}
PRECONDS = {"none": 0, "jacobi": 1}

__all__ = ["Solver", "FE", "residual_noalloc", "RgmError", "MODES", "PRECISIONS", "PLAIN", "DEFLATED", "AUGMENTED",
           "FP64", "FP32_IR", "RGM_W_NOT_CONVERGED", "RGM_W_SINGULAR_COARSE"]


def _is_dev(a):
    return hasattr(a, "is_cuda") and a.is_cuda


def _ptr(a, dtype):
    """(pointer, flags, keepalive) for a numpy array or a CUDA torch tensor."""
    if _is_dev(a):
        assert a.is_contiguous(), "device tensors must be contiguous"
        return C.c_void_p(a.data_ptr()), RGM_DEVICE_PTRS, a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return C.c_void_p(arr.ctypes.data), 0, arr


def _stats(st: RgmStats):
    return dict(iters=st.iters, cycles=st.cycles, refinements=st.refinements, k_used=st.k_used,
                status=st.status, true_relres=st.true_relres)


class Solver:
    """One handle = one sequence of systems of size n (rgm_solver_create)."""

    def __init__(self, n, m=30, k=8, window=16, svd_interval=1, select_smallest=False,
                 mode="deflated", precision="fp64", start_r=False, maxit=20000, inner_cycles=2,
                 max_refinements=50, rtol=1e-10, inner_rtol=1e-4, rel_drop=1e-7, stream=None,
                 launch_policy="auto", proj="oblique", guess=0, precond="none", tiles_per_block=0):
        L = _lib.load()
        cfg = RgmConfig()
        L.rgm_config_default(C.byref(cfg))
        cfg.n, cfg.m, cfg.k, cfg.window = n, m, k, window
        cfg.svd_interval, cfg.select_smallest = svd_interval, int(select_smallest)
        cfg.mode = MODES[mode] if isinstance(mode, str) else int(mode)
        cfg.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        cfg.start_r, cfg.maxit, cfg.inner_cycles = int(start_r), maxit, inner_cycles
        cfg.max_refinements, cfg.rtol, cfg.inner_rtol, cfg.rel_drop = (
            max_refinements, rtol, inner_rtol, rel_drop)
        cfg.launch_policy = LAUNCH_POLICIES[launch_policy] if isinstance(launch_policy, str) \
            else int(launch_policy)
        cfg.proj = PROJECTORS[proj] if isinstance(proj, str) else int(proj)
        cfg.guess = int(guess)
        cfg.precond = PRECONDS[precond] if isinstance(precond, str) else int(precond)
        cfg.tiles_per_block = int(tiles_per_block)
        cfg.cuda_stream = stream
        self.cfg = cfg
        self.n = n
        h = C.c_void_p()
        check(L.rgm_solver_create(C.byref(h), C.byref(cfg)), "rgm_solver_create")
        self._h = h
        self._L = L
        self.nnz = 0

    def close(self):
        if getattr(self, "_h", None):
            self._L.rgm_solver_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_operator_csr(self, rowptr, col, val):
        rp, f1, k1 = _ptr(rowptr, np.int64)
        cl, f2, k2 = _ptr(col, np.int32)
        vl, f3, k3 = _ptr(val, np.float64)
        assert f1 == f2 == f3, "mix of host and device arrays"
        nnz = int(len(col))
        check(self._L.rgm_set_operator_csr(self._h, self.n, nnz, rp, cl, vl, f1),
              "rgm_set_operator_csr")
        self.nnz = nnz

    def set_operator_sell(self, slice_ptr, perm, col, val):
        """rgm_set_operator_sell: the operator in the library's sliced-ELL layout
        (see include/rgmres.h); later set_operator_values calls take values in
        that layout."""
        sp, f1, k1 = _ptr(slice_ptr, np.int64)
        pm, f2, k2 = _ptr(perm, np.int32)
        cl, f3, k3 = _ptr(col, np.int32)
        vl, f4, k4 = _ptr(val, np.float64)
        assert f1 == f2 == f3 == f4, "mix of host and device arrays"
        nslices = int(len(slice_ptr)) - 1
        check(self._L.rgm_set_operator_sell(self._h, self.n, nslices, sp, pm, cl, vl, f1),
              "rgm_set_operator_sell")
        self.nnz = int(len(col))

    def set_operator_values(self, val):
        vl, f, k = _ptr(val, np.float64)
        check(self._L.rgm_set_operator_values(self._h, vl, f), "rgm_set_operator_values")

    def set_recycle_space(self, U):
        if U is None or np.asarray(U).size == 0:
            check(self._L.rgm_set_recycle_space(self._h, None, 0, self.n, 0), "set_recycle_space")
            return
        Uf = np.asfortranarray(np.asarray(U, dtype=np.float64))
        check(self._L.rgm_set_recycle_space(self._h, C.c_void_p(Uf.ctypes.data), Uf.shape[1],
                                            Uf.shape[0], 0), "rgm_set_recycle_space")

    def device_bytes(self):
        """rgm_solver_device_bytes: device memory the handle holds now."""
        v = C.c_int64(0)
        check(self._L.rgm_solver_device_bytes(self._h, C.byref(v)), "rgm_solver_device_bytes")
        return v.value

    def recycle_dim(self):
        """Number of recycle vectors currently held."""
        k = C.c_int(0)
        check(self._L.rgm_get_recycle_space(self._h, None, self.n, C.byref(k), 0), "get_recycle")
        return k.value

    def recycle_space(self):
        k = C.c_int(0)
        check(self._L.rgm_get_recycle_space(self._h, None, self.n, C.byref(k), 0), "get_recycle")
        U = np.zeros((self.n, k.value), order="F")
        if k.value:
            check(self._L.rgm_get_recycle_space(self._h, C.c_void_p(U.ctypes.data), self.n,
                                                C.byref(k), 0), "rgm_get_recycle_space")
        return U

    def solve(self, b, x=None, zero_guess=False):
        """Returns (x, stats).  Host arrays: a new numpy x.  Device tensors: x in place.
        zero_guess: x_in = 0 whatever x holds (RGM_ZERO_GUESS; x is output only)."""
        st = RgmStats()
        zf = RGM_ZERO_GUESS if zero_guess else 0
        if _is_dev(b):
            assert x is not None and _is_dev(x)
            rc = self._L.rgm_solve(self._h, C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()),
                                   RGM_DEVICE_PTRS | zf, C.byref(st))
            check(rc, "rgm_solve")
            return x, _stats(st)
        bb = np.ascontiguousarray(b, dtype=np.float64)
        xx = np.zeros(self.n) if x is None else np.array(x, dtype=np.float64, copy=True)
        rc = self._L.rgm_solve(self._h, C.c_void_p(bb.ctypes.data), C.c_void_p(xx.ctypes.data), zf,
                               C.byref(st))
        check(rc, "rgm_solve")
        return xx, _stats(st)

    def update_recycle_svd(self, x, want_k=True):
        """Algorithm 1 window update; returns the new recycle dimension (with
        want_k=False the call does not wait for the device and returns None)."""
        xp, f, keep = _ptr(x, np.float64)
        k = C.c_int(0)
        check(self._L.rgm_update_recycle_svd(self._h, xp, f, C.byref(k) if want_k else None),
              "rgm_update_recycle_svd")
        return k.value if want_k else None

    def singular_values(self):
        out = np.zeros(64)
        c = C.c_int(0)
        check(self._L.rgm_get_singular_values(self._h, C.c_void_p(out.ctypes.data), C.byref(c)),
              "rgm_get_singular_values")
        return out[: c.value].copy()

    def reset_recycling(self):
        check(self._L.rgm_reset_recycling(self._h), "rgm_reset_recycling")

    def export_state(self):
        """rgm_export_state: the recycling state (window, U) as bytes."""
        n = C.c_size_t()
        check(self._L.rgm_export_state(self._h, None, C.byref(n)), "rgm_export_state")
        buf = C.create_string_buffer(n.value)
        check(self._L.rgm_export_state(self._h, buf, C.byref(n)), "rgm_export_state")
        return buf.raw[:n.value]

    def import_state(self, data):
        """rgm_import_state: resume from bytes written by export_state."""
        buf = C.create_string_buffer(bytes(data), len(data))
        check(self._L.rgm_import_state(self._h, buf, C.c_size_t(len(data))), "rgm_import_state")

    def profile(self, enable=True):
        """Reset and switch per-launch CUDA-event timing on or off."""
        check(self._L.rgm_profile(self._h, int(enable)), "rgm_profile")

    def profile_read(self):
        """{kind: dict(ms, launches, flops, bytes, units, step_bytes)}, total launches."""
        n = len(_lib.PROF_KINDS)
        arr = (_lib.RgmKernelProf * n)()
        tot = C.c_int64(0)
        check(self._L.rgm_profile_read(self._h, arr, n, C.byref(tot)), "rgm_profile_read")
        out = {k: dict(ms=a.ms, launches=a.launches, flops=a.flops, bytes=a.bytes, units=a.units,
                       step_bytes=a.step_bytes)
               for k, a in zip(_lib.PROF_KINDS, arr)}
        return out, tot.value

    def spmv(self, x):
        if _is_dev(x):
            import torch
            y = torch.empty_like(x)
            check(self._L.rgm_spmv(self._h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                   RGM_DEVICE_PTRS), "rgm_spmv")
            return y
        xx = np.ascontiguousarray(x, dtype=np.float64)
        y = np.zeros(self.n)
        check(self._L.rgm_spmv(self._h, C.c_void_p(xx.ctypes.data), C.c_void_p(y.ctypes.data), 0),
              "rgm_spmv")
        return y


def batch_solve(solvers, bs, xs, coop=False, zero_guess=False):
    """rgm_batch_solve: solves system i on solvers[i] with right-hand side bs[i]
    and initial guess / result xs[i] (CUDA tensors, updated in place),
    concurrently.  coop: the systems' GMRES cycles run together as batched
    cooperative launches (RGM_BATCH_COOP) instead of per-pass launches on the
    handles' streams.  Returns the list of stats dicts."""
    L = _lib.load()
    n = len(solvers)
    assert len(bs) == n and len(xs) == n
    for b, x in zip(bs, xs):
        assert _is_dev(b) and _is_dev(x) and b.is_contiguous() and x.is_contiguous()
    H = (C.c_void_p * n)(*[s._h.value for s in solvers])
    B = (C.c_void_p * n)(*[b.data_ptr() for b in bs])
    X = (C.c_void_p * n)(*[x.data_ptr() for x in xs])
    st = (RgmStats * n)()
    flags = RGM_DEVICE_PTRS | (RGM_BATCH_COOP if coop else 0) | (RGM_ZERO_GUESS if zero_guess else 0)
    check(L.rgm_batch_solve(H, n, B, X, flags, st), "rgm_batch_solve")
    return [_stats(st[i]) for i in range(n)]


def batch_plan(n, nnz, nd, want, cap):
    """rgm_batch_plan: the block plan of one batched cycle launch (host only).
    Returns (blocks, rows per block (0: own partition), wave) per system and the
    number of waves."""
    L = _lib.load()
    k = len(n)
    assert len(nnz) == k and len(nd) == k and len(want) == k
    n_ = np.ascontiguousarray(n, dtype=np.int64)
    z_ = np.ascontiguousarray(nnz, dtype=np.int64)
    d_ = np.ascontiguousarray(nd, dtype=np.int32)
    w_ = np.ascontiguousarray(want, dtype=np.int32)
    blocks, rpb, wave = (np.zeros(k, dtype=np.int32) for _ in range(3))
    nw = L.rgm_batch_plan(k, n_.ctypes.data, z_.ctypes.data, d_.ctypes.data, w_.ctypes.data, int(cap),
                          blocks.ctypes.data, rpb.ctypes.data, wave.ctypes.data)
    check(min(nw, 0), "rgm_batch_plan")
    return blocks, rpb, wave, nw


def wait_selftest(limit_ns):
    """rgm_wait_selftest: two blocks wait at a grid barrier that is never
    released, with the given wait limit.  Returns (blocks that gave up, device
    fault flag); (2, 1) when the bounded wait works."""
    L = _lib.load()
    g, f = C.c_int(), C.c_int()
    check(L.rgm_wait_selftest(int(limit_ns), C.byref(g), C.byref(f)), "rgm_wait_selftest")
    return g.value, f.value


def residual_noalloc(rowptr, col, val, x, b, r, norms, stream=None):
    """rgm_residual_noalloc: r = b - A x and norms = [||b - A x||, ||b||] with no
    device allocation, for callers that cannot allocate (see include/rgmres.h).
    All arguments are contiguous tensors on the current CUDA device (int64
    rowptr, int32 col, float64 others; x, b, r of n = rowptr.numel() - 1
    elements, norms of 2); r may be None and must not alias x or b.  Queued on
    `stream` (a torch.cuda.Stream or a raw cudaStream_t handle, None for the
    legacy default stream); the call does not wait.  Arguments that break these
    rules raise ValueError before anything reaches the device."""
    import torch
    L = _lib.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    n = rowptr.numel() - 1

    def need(t, name, dtype, numel=None):
        if not (isinstance(t, torch.Tensor) and t.device == dev):
            raise ValueError(f"{name}: a tensor on the current CUDA device {dev} is required")
        if t.dtype != dtype:
            raise ValueError(f"{name}: dtype {dtype} required, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name}: must be contiguous")
        if numel is not None and t.numel() != numel:
            raise ValueError(f"{name}: {numel} elements required, got {t.numel()}")

    need(rowptr, "rowptr", torch.int64)
    if n < 0:
        raise ValueError("rowptr: at least one element required")
    need(col, "col", torch.int32)
    need(val, "val", torch.float64, col.numel())
    need(x, "x", torch.float64, n)
    need(b, "b", torch.float64, n)
    need(norms, "norms", torch.float64, 2)
    if r is not None:
        need(r, "r", torch.float64, n)
        for other, name in ((x, "x"), (b, "b")):
            if r.data_ptr() == other.data_ptr():
                raise ValueError(f"r must not alias {name}")
    if isinstance(stream, torch.cuda.Stream):
        stream = stream.cuda_stream
    rp = C.c_void_p(r.data_ptr()) if r is not None else None
    check(L.rgm_residual_noalloc(n, C.c_void_p(rowptr.data_ptr()), C.c_void_p(col.data_ptr()),
                                 C.c_void_p(val.data_ptr()), C.c_void_p(x.data_ptr()),
                                 C.c_void_p(b.data_ptr()), rp, C.c_void_p(norms.data_ptr()),
                                 C.c_void_p(stream) if stream else None),
          "rgm_residual_noalloc")


class FE:
    """The Sec. 6.1 time-step systems built on the device (rgm_fe_*)."""

    def __init__(self, p, N, eps, dt, beta, stream=None):
        L = _lib.load()
        h = C.c_void_p()
        check(L.rgm_fe_create(C.byref(h), p, N, eps, dt, float(beta[0]), float(beta[1]), stream),
              "rgm_fe_create")
        self._h, self._L = h, L
        n, nnz = C.c_int64(), C.c_int64()
        L.rgm_fe_sizes(h, C.byref(n), C.byref(nnz))
        self.n, self.nnz = n.value, nnz.value
        self.p, self.N = p, N

    def device_bytes(self):
        """rgm_fe_device_bytes: device memory the workload holds now."""
        v = C.c_int64(0)
        check(self._L.rgm_fe_device_bytes(self._h, C.byref(v)), "rgm_fe_device_bytes")
        return v.value

    def close(self):
        if getattr(self, "_h", None):
            self._L.rgm_fe_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def pattern(self):
        rp = np.zeros(self.n + 1, dtype=np.int64)
        cl = np.zeros(self.nnz, dtype=np.int32)
        check(self._L.rgm_fe_pattern(self._h, C.c_void_p(rp.ctypes.data),
                                     C.c_void_p(cl.ctypes.data), 0), "rgm_fe_pattern")
        return rp, cl

    def assemble(self, u_prev):
        if _is_dev(u_prev):
            import torch
            val = torch.empty(self.nnz, dtype=torch.float64, device=u_prev.device)
            b = torch.empty(self.n, dtype=torch.float64, device=u_prev.device)
            check(self._L.rgm_fe_assemble(self._h, C.c_void_p(u_prev.data_ptr()),
                                          C.c_void_p(val.data_ptr()), C.c_void_p(b.data_ptr()),
                                          RGM_DEVICE_PTRS), "rgm_fe_assemble")
            return val, b
        u = np.ascontiguousarray(u_prev, dtype=np.float64)
        val, b = np.zeros(self.nnz), np.zeros(self.n)
        check(self._L.rgm_fe_assemble(self._h, C.c_void_p(u.ctypes.data), C.c_void_p(val.ctypes.data),
                                      C.c_void_p(b.ctypes.data), 0), "rgm_fe_assemble")
        return val, b

    VELOCITIES = {"constant": 0, "cellular": 1}

    def set_velocity(self, kind="cellular"):
        """'constant' (beta of the constructor) or 'cellular' (Sec. 6.1's field)."""
        k = self.VELOCITIES[kind] if isinstance(kind, str) else int(kind)
        check(self._L.rgm_fe_set_velocity(self._h, k), "rgm_fe_set_velocity")

    def set_forcing(self, c=None, C_amp=0.1):
        """Sec. 6.1's forcing with mode coefficients c (c[0] = c_1); None: f = 1."""
        if c is None:
            check(self._L.rgm_fe_set_forcing(self._h, 0, None, 0.0, 0), "rgm_fe_set_forcing")
            return
        a = np.ascontiguousarray(c, dtype=np.float64)
        check(self._L.rgm_fe_set_forcing(self._h, len(a), C.c_void_p(a.ctypes.data), float(C_amp), 0),
              "rgm_fe_set_forcing")

    def initial_field(self, a8):
        a = np.ascontiguousarray(a8, dtype=np.float64)
        u0 = np.zeros(self.n)
        check(self._L.rgm_fe_initial_field(self._h, C.c_void_p(a.ctypes.data),
                                           C.c_void_p(u0.ctypes.data), 0), "rgm_fe_initial_field")
        return u0

    def time_step(self, solver: Solver, u_dev):
        """One step of Algorithm 1 on the device; u_dev (CUDA float64 tensor) is updated."""
        st = RgmStats()
        rc = self._L.rgm_fe_time_step(self._h, solver._h, C.c_void_p(u_dev.data_ptr()), C.byref(st))
        check(rc, "rgm_fe_time_step")
        return _stats(st)
