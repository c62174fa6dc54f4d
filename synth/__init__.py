"""Seeded synthetic inputs shared by the oracle tests, the CUDA-path tests and the benchmark.

This module holds no arithmetic of the method: it draws random numbers
(SplitMix64, Steele, Lea & Flood 2014, "Fast splittable pseudorandom number
generators") and names the workloads.  Both sides receive these numbers and build
everything else themselves.

Workloads (the paper's benchmark of Sec. 6.1 re-parameterised; see the tables
below): the 2D problem -div(eps grad u) + u beta.grad u = f on the unit square,
f = 1, u = 0 on the boundary, u0 = sum_{j=1..8} a_j sin(j pi x) sin(j pi y) with
a_j ~ U(-0.5, 0.5), implicit Euler with the convection coefficient lagged one step.
PAPER_Q1_64 is the paper's own configuration (cellular velocity, random forcing,
zero initial value).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1
BASE_SEED = 0x1807


class SplitMix64:
    """SplitMix64 as published: golden-gamma increment, then the mix13 finaliser."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi]."""
        return lo + int(self.uniform() * (hi - lo + 1))


@dataclass(frozen=True)
class Workload:
    name: str
    p: int              # Q_p elements
    N: int              # N x N quads
    eps: float
    dt: float
    steps: int
    m: int              # GMRES restart
    k: int              # recycle dimension
    window: int         # snapshot window
    rtol: float
    fixed_beta: tuple | None = None   # None: (cos t, sin t) with t ~ U(0, 2 pi)
    ell: int = 1        # SVD interval
    modes: tuple = field(default=("plain", "deflated", "augmented"))
    velocity: str = "constant"   # or "cellular": Sec. 6.1's b = (-sin pi x cos pi y, cos pi x sin pi y)
    forcing_modes: int = 0       # > 0: Sec. 6.1's random forcing with this many modes (else f = 1)
    forcing_C: float = 0.1
    u0: str = "sines"            # or "zero"
    precond: str = "none"        # or "jacobi" (left Jacobi in place of the paper's SSOR)

    @property
    def n(self) -> int:
        return (self.p * self.N + 1) ** 2


# Q1 32^2: 1089 dofs, eps 0.05, velocity (u, u), dt 0.01, 10 steps, GMRES(20), k 4 of 8.
Q1_32 = Workload("q1_32x32_eps0.05_dt0.01", 1, 32, 0.05, 0.01, 10, 20, 4, 8, 1e-10,
                 fixed_beta=(1.0, 1.0))
# Q2 128^2: 66,049 dofs, eps 0.01, velocity (cos t, sin t) u, dt 0.005, 40 steps,
# GMRES(30), k 8 of 16.
Q2_128 = Workload("q2_128x128_eps0.01_dt0.005", 2, 128, 0.01, 0.005, 40, 30, 8, 16, 1e-10)
# Q4 256^2: 1,050,625 dofs, eps 0.002, dt 0.002, 50 steps, GMRES(40), k 12 of 24,
# FP64 and FP32-inner iterative refinement to a true residual of 1e-8.
Q4_256 = Workload("q4_256x256_eps0.002_dt0.002", 4, 256, 0.002, 0.002, 50, 40, 12, 24, 1e-8,
                  modes=("plain", "deflated", "augmented", "ir"))

# Sec. 6.1's own benchmark: Q1 64^2 (4225 dofs), the cellular velocity, forcing of
# 16 Laplace modes with C = 0.1, c_1 = 1 and c_2..c_16 ~ U[-1, 1] drawn at every step,
# zero initial value, dt 0.5, 1000 steps, true residual 1e-8, nu in {1e-1, 1e-2,
# 1e-3}.  The paper sweeps the restart and the window; GMRES(30), k 8 of 16 here.
PAPER_Q1_64 = {nu: Workload(f"paper_q1_64x64_nu{nu:g}", 1, 64, nu, 0.5, 1000, 30, 8, 16, 1e-8,
                            fixed_beta=(0.0, 0.0), velocity="cellular", forcing_modes=16,
                            u0="zero")
               for nu in (1e-1, 1e-2, 1e-3)}

# Table 4's spectral elements: order 23 on a 2 x 2 grid (2,209 dofs, about 1.1 M
# nonzeros), nu = 1e-2, the same fields; the paper's runs recycle 20 modes with
# the SVD every 20..80 steps over as many solutions, GMRES(30).  High-order
# operators need a preconditioner: left Jacobi here (the paper: SSOR).
PAPER_SEM23 = Workload("paper_sem23_2x2_nu0.01", 23, 2, 1e-2, 0.5, 1000, 30, 20, 20, 1e-8,
                       fixed_beta=(0.0, 0.0), velocity="cellular", forcing_modes=16, u0="zero",
                       ell=20, precond="jacobi")

WORKLOADS = {w.name: w for w in (Q1_32, Q2_128, Q4_256, *PAPER_Q1_64.values(), PAPER_SEM23)}


def sequence_draws(w: Workload, seq_index: int = 0):
    """(a8, beta) for one sequence: a_j ~ U(-0.5, 0.5), then theta ~ U(0, 2 pi)."""
    g = SplitMix64(BASE_SEED + seq_index)
    a8 = np.array([g.uniform(-0.5, 0.5) for _ in range(8)])
    theta = g.uniform(0.0, 2.0 * math.pi)
    beta = w.fixed_beta if w.fixed_beta is not None else (math.cos(theta), math.sin(theta))
    return a8, beta


def forcing_draws(w: Workload, steps: int, seq_index: int = 0) -> np.ndarray:
    """(steps, forcing_modes) coefficients of Sec. 6.1's forcing, one row per time
    step: c_1 = 1, c_2..c_m ~ U(-1, 1) in order."""
    g = SplitMix64(BASE_SEED + 0x6000 + seq_index)
    out = np.ones((steps, w.forcing_modes))
    for i in range(steps):
        for j in range(1, w.forcing_modes):
            out[i, j] = g.uniform(-1.0, 1.0)
    return out


def batch_sequences(count: int = 64, steps: int = 20, seed_index: int = 0, n_lo: int = 32,
                    n_hi: int = 192):
    """Independent sequences of uneven size for the batched form: per sequence
    p ~ U{1..4}, N ~ U{n_lo..n_hi}, eps = 10^U(-3, -1), then the u0 amplitudes
    a_1..a_8 ~ U(-0.5, 0.5) and theta ~ U(0, 2 pi) of that sequence; dt 0.005,
    GMRES(30), k 8 from a window of 16, true residual 1e-8.  Returns a list of
    (Workload, a8, beta)."""
    g = SplitMix64(BASE_SEED + 0x4000 + seed_index)
    out = []
    for i in range(count):
        p = g.randint(1, 4)
        N = g.randint(n_lo, n_hi)
        eps = 10.0 ** g.uniform(-3.0, -1.0)
        a8 = np.array([g.uniform(-0.5, 0.5) for _ in range(8)])
        theta = g.uniform(0.0, 2.0 * math.pi)
        w = Workload(f"batch{i}_q{p}_{N}x{N}", p, N, eps, 0.005, steps, 30, 8, 16, 1e-8)
        out.append((w, a8, (math.cos(theta), math.sin(theta))))
    return out


def serve_stream(count: int = 512, rate_per_s: float = 100.0, n_lo: int = 16, n_hi: int = 256,
                 steps_lo: int = 10, steps_hi: int = 100, seed_index: int = 0):
    """A seeded arrival stream for the served form: inter-arrival gaps
    Exp(rate_per_s) (inverse transform of a uniform draw), then per sequence
    p ~ U{1..4}, N ~ U{n_lo..n_hi}, eps = 10^U(-3, -1), steps ~ U{steps_lo..
    steps_hi}, the u0 amplitudes and theta.  dt 0.005, GMRES(30), k 8 of 16,
    true residual 1e-8.  Returns dicts (keys of serve.Request)."""
    g = SplitMix64(BASE_SEED + 0x5000 + seed_index)
    t = 0.0
    out = []
    for i in range(count):
        t += -math.log(1.0 - g.uniform()) / rate_per_s
        p = g.randint(1, 4)
        N = g.randint(n_lo, n_hi)
        eps = 10.0 ** g.uniform(-3.0, -1.0)
        steps = g.randint(steps_lo, steps_hi)
        a8 = np.array([g.uniform(-0.5, 0.5) for _ in range(8)])
        theta = g.uniform(0.0, 2.0 * math.pi)
        out.append(dict(rid=i, arrival_s=t, p=p, N=N, eps=eps, dt=0.005, steps=steps, a8=a8,
                        beta=(math.cos(theta), math.sin(theta))))
    return out


def random_vector(n: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    g = SplitMix64(seed)
    return np.array([g.uniform(lo, hi) for _ in range(n)])


def random_matrix(rows: int, cols: int, seed: int) -> np.ndarray:
    """Dense matrix of U(-1, 1) entries, filled column by column."""
    return random_vector(rows * cols, seed).reshape(cols, rows).T.copy()


def random_csr(n: int, max_per_row: int, seed: int, diag: float = 0.0, min_per_row: int = 0,
               n_cols: int | None = None):
    """Random CSR: row r gets U{min..max} off-diagonal entries at distinct random
    columns, values U(-1, 1); if diag != 0 the diagonal entry diag*(1 + U(0,1)) is
    added.  Returns (rowptr int64, col int32, val float64), columns ascending."""
    g = SplitMix64(seed)
    nc = n if n_cols is None else n_cols
    rowptr = [0]
    cols, vals = [], []
    for r in range(n):
        cnt = g.randint(min_per_row, max_per_row)
        row = {}
        for _ in range(cnt):
            c = g.randint(0, nc - 1)
            row[c] = row.get(c, 0.0) + g.uniform(-1.0, 1.0)
        if diag != 0.0 and r < nc:
            row[r] = row.get(r, 0.0) + diag * (1.0 + g.uniform())
        for c in sorted(row):
            cols.append(c)
            vals.append(row[c])
        rowptr.append(len(cols))
    return (np.array(rowptr, dtype=np.int64), np.array(cols, dtype=np.int32),
            np.array(vals, dtype=np.float64))
