"""The multi-GPU path is replicas only (sequences are independent, no data-path
collective): two gloo ranks on CPU check the host logic bench.py uses for
N > 1 -- each rank solves its own seeded sequence, the job time is the slowest
rank's (max over ranks), every rank's solves count, and only rank 0 reports."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, outdir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import bench
    import synth
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    w = synth.Q2_128                                   # seeded u0 amplitudes and velocity angle
    seq = synth.sequence_draws(w, bench.replica_sequence(rank))
    my_sec = 1.0 + 0.5 * rank                          # rank 1 is the slow one

    def reduce_max(x):
        t = torch.tensor([x], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    value, tot = bench.aggregate_replicas(my_sec, 10, ws, reduce_max)
    dist.barrier()
    with open(os.path.join(outdir, f"r{rank}.txt"), "w") as f:
        f.write(f"{float(seq[0][0])!r} {float(seq[1][0])!r} {value!r} {tot!r} {int(rank == 0)}\n")
    dist.destroy_process_group()


def test_two_replicas_gloo(tmp_path):
    ws = 2
    mp.spawn(_rank_main, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, join=True)
    rows = [open(tmp_path / f"r{r}.txt").read().split() for r in range(ws)]
    a0 = [float(r[0]) for r in rows]
    th = [float(r[1]) for r in rows]
    assert a0[0] != a0[1] and th[0] != th[1]             # distinct problems per rank
    for r in rows:
        assert float(r[3]) == 1.5                        # job time = slowest rank
        assert float(r[2]) == pytest.approx(10 * ws / 1.5)
    assert [int(r[4]) for r in rows] == [1, 0]           # rank 0 alone reports


def test_single_rank_aggregate_is_local():
    import bench
    value, tot = bench.aggregate_replicas(2.0, 30, 1, reduce_max=None)
    assert (value, tot) == (15.0, 2.0)
