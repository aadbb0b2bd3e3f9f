"""The multi-rank host logic of bench.py on CPU (gloo, world size 2): the
timed region is the maximum over ranks, every rank receives it, the job's
throughput counts every rank's replica, and the reference arm runs on rank 0
only (the other ranks exit without work or output).  The GPU data path is
replicas only: no collective besides this reduction and the barriers."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    w, r, local = bench.dist_setup()
    ms = bench.job_time_ms(100.0 + 50.0 * rank, dist, "cpu")
    out[rank] = (w, r, local, ms, bench.job_throughput(1000, 5, w, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput():
    ws = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    for rank in range(ws):
        w, r, local, ms, value = res[rank]
        assert (w, r, local) == (ws, rank, rank)
        assert ms == 150.0
        assert value == pytest.approx(1000 * 5 * ws / 0.150)


def test_single_process_time_is_local():
    assert bench.job_time_ms(12.5, None, "cpu") == 12.5
    assert bench.job_throughput(2097152, 5, 1, 120.0) == pytest.approx(2097152 * 5 / 0.12)


def test_reference_arm_other_ranks_exit_quietly(capsys):
    class Args:
        size = "8,8,8"
        steps = 1
        warmup = 0
        gpus = 2
        integrator = "rk3"
    assert bench.run_reference(Args(), 2, 1) == 0
    assert capsys.readouterr().out == ""


def test_reference_arm_line(capsys):
    """Rank 0 of the reference arm times the oracle on the given torus and
    prints one JSON line with the contract's keys."""
    import json

    class Args:
        size = "16,8,4"
        steps = 1
        warmup = 0
        gpus = 1
        integrator = "rk3"
    assert bench.run_reference(Args(), 1, 0) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    for k in ("metric", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "config", "cpu_baseline", "e2e"):
        assert k in line
    assert line["e2e"]["h2d_bytes_per_step"] == 0
