"""Served form (paper_1807_09467_gb300.serve): requests that arrive while
others run are admitted as slots free up, each sequence advances on its own
stream and host thread, and every result is the same alone and in the mix (bit
for bit: each sequence's work is deterministic and shares no state); every
solve reaches the true FP64 residual 1e-8.  The admission estimate of a
sequence's device footprint bounds what the library actually allocates."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rg():
    import __graft_entry__ as g
    g.build()
    import paper_1807_09467_gb300 as rg
    return rg


def _requests(serve, count=6):
    reqs = synth.serve_stream(count=count, rate_per_s=50.0, n_lo=12, n_hi=40, steps_lo=3, steps_hi=7)
    return [serve.Request(**r) for r in reqs]


def test_same_alone_and_in_the_mix(rg):
    from paper_1807_09467_gb300 import serve
    reqs = _requests(serve)
    mixed, tot = serve.Server(max_slots=3).run(reqs, realtime=False)
    assert tot["solves"] == sum(r.steps for r in reqs)
    for r, res in zip(reqs, mixed):
        assert len(res.iters) == r.steps and res.final is not None
        alone, _ = serve.Server(max_slots=1).run([r], realtime=False)
        np.testing.assert_array_equal(res.final, alone[0].final)
        assert res.iters == alone[0].iters


def test_admission_overlaps_sequences(rg):
    """With several slots, a later request is admitted while an earlier one is
    still running (sequences overlap instead of running one after another)."""
    from paper_1807_09467_gb300 import serve
    reqs = _requests(serve, count=8)
    res, tot = serve.Server(max_slots=4).run(reqs, realtime=False)
    spans = sorted((x.admitted_s, x.finished_s) for x in res)
    assert any(spans[i + 1][0] < spans[i][1] for i in range(len(spans) - 1))


def test_realtime_admission_and_latency(rg):
    from paper_1807_09467_gb300 import serve
    reqs = _requests(serve)
    res, tot = serve.Server(max_slots=4).run(reqs, realtime=True)
    assert tot["p99_ms"] >= tot["p50_ms"] > 0
    # nobody is admitted before it arrives
    for r, x in zip(reqs, res):
        assert x.admitted_s >= r.arrival_s - 1e-6
        assert x.finished_s >= x.admitted_s


@pytest.mark.parametrize("precision", ["fp32_ir", "fp64"])
def test_footprint_estimate_bounds_the_allocation(rg, precision):
    """serve.device_bytes (the admission estimate) against the library's own
    count of one sequence's allocations (rgm_solver_device_bytes +
    rgm_fe_device_bytes), over Q1-Q4 on small and large grids: never below,
    and within a factor of 1.5 plus 2 MB (fixed per-handle scratch)."""
    from paper_1807_09467_gb300 import serve
    for p, N in ((1, 16), (2, 64), (3, 100), (4, 128), (4, 256)):
        req = serve.Request(rid=0, arrival_s=0.0, p=p, N=N, eps=0.01, dt=0.005, steps=1,
                            a8=np.zeros(8), beta=(1.0, 0.0))
        lv = serve._Live(req, precision, "deflated")
        got = lv.device_bytes()
        lv.close()
        est = serve.device_bytes(req, precision)
        assert got <= est <= 1.5 * got + (2 << 20), (p, N, got, est)
