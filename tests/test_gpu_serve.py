"""Served form (paper_1807_09467_gb300.serve): requests that arrive while
others run are admitted as slots free up and advanced together; every result
is the same alone and in the mix (bit for bit: each sequence's work is
deterministic and shares no state), and every solve reaches the true FP64
residual 1e-8."""
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


def _requests(serve):
    reqs = synth.serve_stream(count=6, rate_per_s=50.0, n_lo=12, n_hi=40, steps_lo=3, steps_hi=7)
    return [serve.Request(**r) for r in reqs]


def test_same_alone_and_in_the_mix(rg):
    from paper_1807_09467_gb300 import serve
    reqs = _requests(serve)
    mixed, tot = serve.Server(max_slots=3).run(reqs, realtime=False)
    assert tot["solves"] == sum(r.steps for r in reqs)
    assert tot["ticks"] < tot["solves"]                     # solves overlapped in ticks
    for r, res in zip(reqs, mixed):
        assert len(res.iters) == r.steps and res.final is not None
        alone, _ = serve.Server(max_slots=1).run([r], realtime=False)
        np.testing.assert_array_equal(res.final, alone[0].final)
        assert res.iters == alone[0].iters


def test_realtime_admission_and_latency(rg):
    from paper_1807_09467_gb300 import serve
    reqs = _requests(serve)
    res, tot = serve.Server(max_slots=4).run(reqs, realtime=True)
    assert tot["p99_ms"] >= tot["p50_ms"] > 0
    # nobody is admitted before it arrives
    for r, x in zip(reqs, res):
        assert x.admitted_s >= r.arrival_s - 1e-6
        assert x.finished_s >= x.admitted_s
