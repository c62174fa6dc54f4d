"""Checkpoint / resume of the recycling state (rgm_export_state /
rgm_import_state): a sequence resumed in a new handle from a checkpoint
continues exactly as the uninterrupted run (same recycle dimension and
iteration counts per step, same field)."""
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


def _run(rg, w, beta, u, steps, s, fe):
    out = []
    for _ in range(steps):
        st = fe.time_step(s, u)
        assert st["status"] == 0 and st["true_relres"] <= w.rtol
        out.append((st["iters"], st["k_used"]))
    return out


@pytest.mark.parametrize("wname,mode,steps,cut", [("q1_32x32_eps0.05_dt0.01", "deflated", 10, 4),
                                                  ("q1_32x32_eps0.05_dt0.01", "augmented", 10, 7),
                                                  ("q2_128x128_eps0.01_dt0.005", "deflated", 20, 17)])
def test_resume_matches_uninterrupted(rg, wname, mode, steps, cut):
    import torch
    w = synth.WORKLOADS[wname]
    a8, beta = synth.sequence_draws(w, 0)

    def new_handles():
        fe = rg.FE(w.p, w.N, w.eps, w.dt, beta)
        rp, col = fe.pattern()
        s = rg.Solver(fe.n, m=w.m, k=w.k, window=w.window, mode=mode, rtol=w.rtol)
        s.set_operator_csr(rp, col, np.zeros(len(col)))
        return fe, s

    fe, s = new_handles()
    u = torch.tensor(fe.initial_field(a8), dtype=torch.float64, device="cuda")
    full = _run(rg, w, beta, u, steps, s, fe)
    u_full = u.cpu().numpy()

    fe, s = new_handles()
    u = torch.tensor(fe.initial_field(a8), dtype=torch.float64, device="cuda")
    first = _run(rg, w, beta, u, cut, s, fe)
    blob = s.export_state()
    s.close()
    fe2, s2 = new_handles()
    s2.import_state(blob)
    rest = _run(rg, w, beta, u, steps - cut, s2, fe2)
    assert first + rest == full
    np.testing.assert_array_equal(u.cpu().numpy(), u_full)


def test_import_rejects_mismatch(rg):
    s = rg.Solver(100, k=4, window=8)
    blob = s.export_state()
    t = rg.Solver(101, k=4, window=8)
    with pytest.raises(rg.RgmError):
        t.import_state(blob)
    u = rg.Solver(100, k=4, window=9)
    with pytest.raises(rg.RgmError):
        u.import_state(blob)
    with pytest.raises(rg.RgmError):
        s.import_state(blob[:-1] if len(blob) > 8 else b"x")
    s.import_state(blob)           # empty state round trip
    assert s.recycle_dim() == 0


@pytest.mark.parametrize("smallest", [True, False])
def test_state_without_eigenvectors_is_accepted(rg, smallest):
    """A checkpoint written before the eigenvectors of the last window SVD were
    part of the state (version 2: no trailing eigenvector block) is accepted and
    the sequence goes on converging; a version-3 header whose eigenvector count
    exceeds the window count is refused and leaves the handle usable.  The
    eigenvectors are stored by the warm-started eigen-solve of the trailing
    modes (select_smallest); the leading-mode solve stores none (count 0)."""
    import struct
    import torch
    w = synth.WORKLOADS["q1_32x32_eps0.05_dt0.01"]
    a8, beta = synth.sequence_draws(w, 0)
    fe = rg.FE(w.p, w.N, w.eps, w.dt, beta)
    rp, col = fe.pattern()
    s = rg.Solver(fe.n, m=w.m, k=w.k, window=w.window, mode="deflated", rtol=w.rtol,
                  select_smallest=smallest)
    s.set_operator_csr(rp, col, np.zeros(len(col)))
    u = torch.tensor(fe.initial_field(a8), dtype=torch.float64, device="cuda")
    _run(rg, w, beta, u, 6, s, fe)
    blob = s.export_state()
    fmt = "<IIqiiiiqii"
    hdr = list(struct.unpack_from(fmt, blob))
    magic, version, n, window, k_cur, win_count, win_head, updates, gram, phi_c = hdr
    assert version == 3 and (0 < phi_c <= win_count if smallest else phi_c == 0)
    body = blob[struct.calcsize(fmt):]
    assert len(body) == 8 * (n * (win_count + k_cur) + gram * win_count ** 2 + phi_c ** 2)
    v2 = struct.pack(fmt, magic, 2, n, window, k_cur, win_count, win_head, updates, gram, 0) + \
        body[:len(body) - 8 * phi_c ** 2]
    bad = struct.pack(fmt, magic, 3, n, window, k_cur, win_count, win_head, updates, gram, win_count + 1) + \
        body + bytes(8 * ((win_count + 1) ** 2 - phi_c ** 2))
    s2 = rg.Solver(fe.n, m=w.m, k=w.k, window=w.window, mode="deflated", rtol=w.rtol,
                   select_smallest=smallest)
    s2.set_operator_csr(rp, col, np.zeros(len(col)))
    with pytest.raises(rg.RgmError):
        s2.import_state(bad)
    s2.import_state(v2)
    rest = _run(rg, w, beta, u, 4, s2, fe)
    assert all(kk > 0 for _, kk in rest)
    s.close()
    s2.close()
    fe.close()
