"""Served form: a request loop over time-step sequences with continuous batching.

Each request is one convection-diffusion sequence (its FE workload, seeded
initial field and number of time steps).  Requests arrive over time.  The loop
admits a waiting request as soon as it has arrived, a slot is free and its
device footprint fits the free HBM read at that moment; each admitted sequence
keeps its operator, snapshot window and recycle space U / A U resident on the
device for its whole life and advances on a stream of its own, driven by a
host thread of its own: assemble the next system, solve, update the window,
again.  Sequences therefore progress independently -- their kernels overlap
on the device, a short sequence is not held back by a long one, and a request
that arrives while others run is admitted the moment a sequence ends (a slot
frees) instead of at the end of a lockstep tick.  Every solve's latency runs
from the moment its system could start (the request's arrival for the first
step, the end of the sequence's previous step otherwise) to the end of its
solve and window update.

Host-side orchestration only: assembly, solves and window updates all run in
librgmres's kernels.  The solves use the per-pass launches (launch_policy
"per_pass"): cooperative grids of different sequences are not guaranteed to be
resident together, so a cooperative cycle launch is left to single-sequence
use.
"""
from __future__ import annotations

import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import FE, Solver, tune


@dataclass
class Request:
    """One sequence to serve.  a8 / beta: the seeded initial-field amplitudes
    and velocity direction; steps: time steps to take."""
    rid: int
    arrival_s: float
    p: int
    N: int
    eps: float
    dt: float
    steps: int
    a8: np.ndarray
    beta: tuple
    m: int = 30
    k: int = 8
    window: int = 16
    rtol: float = 1e-8


@dataclass
class Result:
    rid: int
    iters: list = field(default_factory=list)
    latencies_ms: list = field(default_factory=list)
    final: np.ndarray | None = None
    admitted_s: float = 0.0
    finished_s: float = 0.0
    device_bytes: int = 0        # what its solver and workload held on the device
    error: str | None = None


def sizes(p: int, N: int) -> tuple[int, int]:
    """(n, nnz) of the Q_p Dirichlet pattern on N x N quads: two nodes couple
    when they share an element, i.e. in each direction their 1D indices share
    a 1D element (a vertex index i couples to [i - p, i + p], an index inside
    an element to that element's p + 1 indices); boundary rows are identity
    rows and boundary columns are dropped from interior rows."""
    L = p * N + 1
    inner = np.zeros(L, dtype=np.int64)      # interior neighbours of each 1D index
    for i in range(1, L - 1):
        lo, hi = (max(i - p, 0), min(i + p, L - 1)) if i % p == 0 else (i // p * p, i // p * p + p)
        inner[i] = min(hi, L - 2) - max(lo, 1) + 1
    n = L * L
    return n, int(inner.sum()) ** 2 + (n - (L - 2) ** 2)


def device_bytes(req: Request, precision: str = "fp32_ir") -> int:
    """Upper estimate of the device memory one admitted sequence holds: the
    solver (Krylov basis, recycle space, window, operator in sliced ELL with
    its CSR map, binary32 copies in GMRES-IR, scratch) and the FE workload
    (pattern, values, element tables, per-cell matrices).  Checked against the library's own
    count (rgm_solver_device_bytes + rgm_fe_device_bytes) by the tests."""
    n, nnz = sizes(req.p, req.N)
    ld = (n + 31) // 32 * 32
    ncolV = req.m + req.k + 1
    kmax = max(req.k, 1)
    ir = precision == "fp32_ir"
    vec = 8 * ld * (ncolV + 3 * kmax + 1 + 4 + req.window) + (4 * ld * (ncolV + 2 * kmax + 4) if ir else 0)
    nsell = int(1.6 * nnz) + 32 * 256          # sliced-ELL padding (at most ~1.5x on FE patterns)
    op = nsell * (4 + 8 + (4 if ir else 0)) + nnz * (4 + 8) + 8 * (n // 8 + 2) + 4 * (n + 256)
    nblocks = min((n + 255) // 256, 4 * 152)  # grid of the fused kernels (<= 4 blocks per SM)
    scratch = 8 * 3200 * nblocks + 8 * 3200 * (nblocks // 32 + 1) + 16 * 3200 + (320 << 10)
    fe = 8 * (n + 1) + 12 * nnz + 16 * n + 8 * (req.p + 1) ** 6 * 4 + (1 << 16)
    if req.p <= 4:                              # per-cell matrices (constant velocity)
        fe += 8 * req.N * req.N * (req.p + 1) ** 4
    return int(vec + op + scratch + fe)


class _Live:
    def __init__(self, req: Request, precision: str, mode: str, max_blocks: int | None = None):
        import torch
        self.req = req
        self.stream = torch.cuda.Stream()
        self.fe = FE(req.p, req.N, req.eps, req.dt, req.beta, stream=self.stream.cuda_stream)
        rp, col = self.fe.pattern()
        self.sol = Solver(self.fe.n, m=req.m, k=req.k, window=req.window, mode=mode,
                          precision=precision, rtol=req.rtol, stream=self.stream.cuda_stream,
                          launch_policy="per_pass",
                          tiles_per_block=tune.tiles_per_block(self.fe.n, max_blocks))
        self.sol.set_operator_csr(rp, col, np.zeros(len(col)))
        with torch.cuda.stream(self.stream):
            self.u = torch.tensor(self.fe.initial_field(req.a8), dtype=torch.float64, device="cuda")
        self.stream.synchronize()

    def device_bytes(self) -> int:
        return self.sol.device_bytes() + self.fe.device_bytes()

    def close(self):
        self.sol.close()
        self.fe.close()


class Server:
    """Continuous-batching loop.  max_slots bounds the sequences in flight;
    each admission also needs its estimated footprint to fit hbm_fraction of
    the device memory free at that moment.  max_blocks caps the blocks of any
    one sequence's passes (tiles_per_block of its handle; None: the library's
    automatic shape), the knob of the launch-shape autotuner (tune.py)."""

    def __init__(self, max_slots: int = 64, hbm_fraction: float = 0.8, precision: str = "fp32_ir",
                 mode: str = "deflated", max_blocks: int | None = None):
        self.max_slots = max_slots
        self.hbm_fraction = hbm_fraction
        self.precision = precision
        self.mode = mode
        self.max_blocks = max_blocks

    def _drive(self, lv: _Live, res: Result, t0: float, done):
        """One sequence, step after step on its own stream (a host thread)."""
        import torch
        try:
            ready = max(lv.req.arrival_s, 0.0)
            with torch.cuda.stream(lv.stream):
                for _ in range(lv.req.steps):
                    val, b = lv.fe.assemble(lv.u)
                    lv.sol.set_operator_values(val)
                    zg = lv.sol.recycle_dim() > 0 and self.mode != "plain"
                    x = torch.empty_like(lv.u) if zg else lv.u.clone()
                    _, st = lv.sol.solve(b, x, zero_guess=zg)
                    lv.sol.update_recycle_svd(x, want_k=False)
                    lv.stream.synchronize()
                    t_end = time.perf_counter() - t0
                    if st["status"] < 0 or st["true_relres"] > lv.req.rtol:
                        raise RuntimeError(f"request {lv.req.rid}: solve failed {st}")
                    lv.u.copy_(x)
                    res.iters.append(st["iters"])
                    res.latencies_ms.append(1e3 * (t_end - ready))
                    ready = t_end
                res.final = lv.u.cpu().numpy()
            res.finished_s = time.perf_counter() - t0
        except Exception as e:          # reported by run(); the slot is freed either way
            res.error = repr(e)
        finally:
            lv.close()
            done(lv)

    def run(self, requests: list[Request], realtime: bool = True) -> tuple[list[Result], dict]:
        """Serve the requests (arrival_s relative to the call).  realtime: wait
        for arrivals on the wall clock; else admit in arrival order as fast as
        slots free up.  Returns per-request results and totals."""
        import torch
        pending = sorted(requests, key=lambda r: (r.arrival_s, r.rid))
        results = {r.rid: Result(r.rid) for r in requests}
        cv = threading.Condition()
        live: set = set()
        threads = []
        est_over = []           # estimate / measured footprint of each admitted sequence

        def done(lv):
            with cv:
                live.discard(lv)
                cv.notify_all()

        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0
        while pending:
            req = pending[0]
            with cv:
                # a free slot (or an empty device) and the request's arrival
                while len(live) >= self.max_slots:
                    cv.wait(0.05)
                if realtime and req.arrival_s > now():
                    cv.wait(min(req.arrival_s - now(), 0.05))
                    continue
                need = device_bytes(req, self.precision)
                free, _ = torch.cuda.mem_get_info()
                if live and need > self.hbm_fraction * free:
                    cv.wait(0.05)        # wait for a sequence to end and free its memory
                    continue
            pending.pop(0)
            res = results[req.rid]
            res.admitted_s = now()
            lv = _Live(req, self.precision, self.mode, self.max_blocks)
            res.device_bytes = lv.device_bytes()
            est_over.append(need / max(res.device_bytes, 1))
            if not realtime:
                req_ready = res.admitted_s
                lv.req = Request(**{**lv.req.__dict__, "arrival_s": req_ready})
            with cv:
                live.add(lv)
            th = threading.Thread(target=self._drive, args=(lv, res, t0, done), daemon=True)
            threads.append(th)
            th.start()
        for th in threads:
            th.join()
        torch.cuda.synchronize()
        wall = now()
        errors = [r.error for r in results.values() if r.error]
        if errors:
            raise RuntimeError(errors[0])
        solves = sum(len(r.iters) for r in results.values())
        lat = np.concatenate([np.asarray(r.latencies_ms) for r in results.values()]) if solves else np.zeros(1)
        totals = dict(solves=solves, wall_s=wall, solves_per_s=solves / wall,
                      p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)),
                      footprint_estimate_over_measured=(min(est_over), max(est_over)) if est_over else None)
        return [results[r.rid] for r in requests], totals
