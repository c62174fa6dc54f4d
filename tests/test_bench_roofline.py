"""Host arithmetic of bench.py's roofline object (no GPU): the achieved rate is
the steps' algorithmic bytes over the steps' event time, the fraction is that
rate over the peak, and a traffic record only counts on the sources it was
captured from."""
from types import SimpleNamespace

import pytest


def _prof():
    # three passes over 10 Arnoldi steps: 1.0 + 0.5 + 0.25 ms, 4.5 GB of
    # algorithmic bytes, 6 GB moved by the passes
    def kind(ms, units, step_bytes, byts, flops):
        return {"ms": ms, "launches": 10, "units": units, "step_bytes": step_bytes, "bytes": byts,
                "flops": flops}
    return {"arnoldi_spmv_dots": kind(1.0, 10, 4.5e9, 3e9, 1e9),
            "arnoldi_cgs1_axpy_dots": kind(0.5, 0, 0.0, 2e9, 5e8),
            "arnoldi_cgs2_axpy_norm": kind(0.25, 0, 0.0, 1e9, 5e8),
            "gram": kind(9.0, 3, 1e9, 1e9, 1e9)}


def test_arnoldi_step_roofline_arithmetic():
    import bench
    w = SimpleNamespace(name="no_such_workload")
    r, _ = bench.cycle_roofline(_prof(), w, "fp32_ir", hbm_peak=6000.0, fp64_peak=1.1, fp32_peak=80.0)
    t = 1.75e-3 / 10                                # seconds per step
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["steps"] == 10
    assert r["achieved"] == pytest.approx(4.5e9 / 10 / t / 1e9, abs=0.1)
    assert r["frac"] == pytest.approx(r["achieved"] / 6000.0, abs=1e-4)
    assert r["pass_gbs"] == pytest.approx(6e9 / 10 / t / 1e9, abs=0.1)
    assert r["second_bound"]["achieved"] == pytest.approx(2e9 / 10 / t / 1e12, abs=1e-4)
    assert r["traffic"] is None                     # no record for this workload
    # binary64: the FP64 pipe leads, HBM second
    r64, _ = bench.cycle_roofline(_prof(), w, "fp64", hbm_peak=6000.0, fp64_peak=1.1)
    assert r64["bound"] == "alu" and r64["second_bound"]["bound"] == "hbm"


def test_cooperative_cycle_is_the_unit_when_present():
    import bench
    prof = _prof()
    prof["arnoldi_cycle"] = {"ms": 2.0, "launches": 2, "units": 20, "step_bytes": 9e9, "bytes": 9e9,
                             "flops": 2e9}
    r, _ = bench.cycle_roofline(prof, SimpleNamespace(name="x"), "fp32_ir", 6000.0, 1.1, 80.0)
    assert r["kernel"].startswith("arnoldi_cycle") and r["steps"] == 20
    assert r["achieved"] == pytest.approx(9e9 / 20 / (2e-3 / 20) / 1e9, abs=0.1)


def test_traffic_record_follows_the_source_digest(monkeypatch):
    import bench
    key = ("q4_256x256_eps0.002_dt0.002", "fp32_ir", "arnoldi_step")
    rec = bench.traffic_record(*key)
    assert rec is None or rec > 0
    monkeypatch.setattr(bench, "src_digest", lambda: "0000000000000000")
    assert bench.traffic_record(*key) is None
