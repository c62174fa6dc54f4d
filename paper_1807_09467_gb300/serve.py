"""Served form: a request loop over time-step sequences with continuous batching.

Each request is one convection-diffusion sequence (its FE workload, seeded
initial field and number of time steps).  Requests arrive over time; the loop
admits a waiting request as soon as a slot is free and its device memory fits
the free HBM, keeps each admitted sequence's operator, snapshot window and
recycle space resident on the device for its whole life, and advances all
admitted sequences together: every tick assembles each sequence's next
system on its own stream, solves all of them with one rgm_batch_solve, and
updates their windows.  A sequence that finishes frees its slot and memory for
the next arrival; a request that arrives while others run joins at the next
tick.  Every solve's latency (from the moment its system could start -- the
request's arrival for the first step, the end of the previous tick otherwise
-- to the end of the tick that solved it) is recorded.

Host-side orchestration only: assembly, solves and window updates all run in
librgmres's kernels.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import FE, Solver, batch_solve


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


def device_bytes(req: Request) -> int:
    """Estimate of the device memory one admitted sequence holds (solver basis,
    recycle space, window, operator in binary64 + binary32, FE pattern)."""
    n = (req.p * req.N + 1) ** 2
    nnz_row = (2 * req.p + 1) ** 2
    nnz = n * nnz_row
    vecs = (req.m + req.k + 1) * 12 + 2 * req.k * 12 + req.window * 8 + 32 * 8
    return int(n * vecs + nnz * (8 + 4 + 4 + 8 + 4 + 4) + (1 << 20))


class _Live:
    def __init__(self, req: Request, precision: str, mode: str, stream):
        import torch
        self.req = req
        self.stream = stream
        self.fe = FE(req.p, req.N, req.eps, req.dt, req.beta, stream=stream.cuda_stream)
        rp, col = self.fe.pattern()
        self.sol = Solver(self.fe.n, m=req.m, k=req.k, window=req.window, mode=mode,
                          precision=precision, rtol=req.rtol, stream=stream.cuda_stream)
        self.sol.set_operator_csr(rp, col, np.zeros(len(col)))
        self.u = torch.tensor(self.fe.initial_field(req.a8), dtype=torch.float64, device="cuda")
        self.done_steps = 0
        self.ready_s = req.arrival_s

    def close(self):
        self.sol.close()
        self.fe.close()


class Server:
    """Continuous-batching loop.  max_slots bounds the sequences in flight;
    hbm_fraction of the free device memory at start bounds their estimated
    footprint."""

    def __init__(self, max_slots: int = 64, hbm_fraction: float = 0.8, precision: str = "fp32_ir",
                 mode: str = "deflated", coop: bool = False):
        import torch
        self.max_slots = max_slots
        self.coop = coop
        free, _ = torch.cuda.mem_get_info()
        self.budget = int(hbm_fraction * free)
        self.precision = precision
        self.mode = mode

    def run(self, requests: list[Request], realtime: bool = True) -> tuple[list[Result], dict]:
        """Serve the requests (arrival_s relative to the call).  realtime: wait
        for arrivals on the wall clock; else admit in arrival order as fast as
        slots free up.  Returns per-request results and totals."""
        import torch
        pending = sorted(requests, key=lambda r: (r.arrival_s, r.rid))
        results = {r.rid: Result(r.rid) for r in requests}
        live: list[_Live] = []
        used = 0
        t_start = time.perf_counter()
        now = lambda: time.perf_counter() - t_start
        ticks = 0
        solves = 0
        while pending or live:
            # admission: arrived, a free slot, and memory for its footprint
            while pending and len(live) < self.max_slots and (not realtime or pending[0].arrival_s <= now()):
                need = device_bytes(pending[0])
                if used + need > self.budget and live:
                    break
                req = pending.pop(0)
                lv = _Live(req, self.precision, self.mode, torch.cuda.Stream())
                lv.ready_s = max(req.arrival_s, now()) if realtime else now()
                results[req.rid].admitted_s = now()
                live.append(lv)
                used += need
            if not live:
                if pending and realtime:
                    time.sleep(max(0.0, min(pending[0].arrival_s - now(), 0.01)))
                continue
            # one tick: the next system of every live sequence, solved together
            xs, bs = [], []
            for lv in live:
                val, b = lv.fe.assemble(lv.u)
                lv.sol.set_operator_values(val)
                x = torch.zeros_like(lv.u) if lv.sol.recycle_dim() else lv.u.clone()
                xs.append(x)
                bs.append(b)
            torch.cuda.synchronize()
            stats = batch_solve([lv.sol for lv in live], bs, xs, coop=self.coop)
            for lv, x in zip(live, xs):
                lv.sol.update_recycle_svd(x, want_k=False)
            torch.cuda.synchronize()
            t_end = now()
            ticks += 1
            still = []
            for lv, x, st in zip(live, xs, stats):
                res = results[lv.req.rid]
                if st["status"] < 0 or st["true_relres"] > lv.req.rtol:
                    raise RuntimeError(f"request {lv.req.rid}: solve failed {st}")
                lv.u.copy_(x)
                res.iters.append(st["iters"])
                res.latencies_ms.append(1e3 * (t_end - lv.ready_s))
                lv.ready_s = t_end
                lv.done_steps += 1
                solves += 1
                if lv.done_steps == lv.req.steps:
                    res.final = lv.u.cpu().numpy()
                    res.finished_s = t_end
                    used -= device_bytes(lv.req)
                    lv.close()
                else:
                    still.append(lv)
            live = still
        wall = now()
        lat = np.concatenate([np.asarray(r.latencies_ms) for r in results.values()]) if solves else np.zeros(1)
        totals = dict(solves=solves, ticks=ticks, wall_s=wall, solves_per_s=solves / wall,
                      p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)))
        return [results[r.rid] for r in requests], totals
