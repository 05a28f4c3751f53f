"""The multi-rank bookkeeping of bench.py (replicas: one process per GPU, no data-path
collective) on two gloo ranks on the CPU: the whole-job value is the units all ranks
processed divided by the slowest rank's time, the same on every rank."""
import importlib.util
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _load_bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    bench = _load_bench()
    assert bench._dist()[:2] == (ws, rank)
    # rank r processed 1000 (r + 1) units in 100 (r + 1) ms
    value, ms = bench.whole_job(1000.0 * (rank + 1), 100.0 * (rank + 1), ws)
    out[rank] = (value, ms)
    dist.barrier()
    dist.destroy_process_group()


def test_whole_job_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ws = 2
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_rank_main, args=(ws, port, out), nprocs=ws, join=True)
    expected = (1000.0 + 2000.0) / 0.2      # 3000 units over the slowest rank's 200 ms
    for r in range(ws):
        value, ms = out[r]
        assert ms == 200.0
        assert value == pytest.approx(expected, rel=1e-15)


def test_whole_job_single_rank_needs_no_group():
    bench = _load_bench()
    value, ms = bench.whole_job(500.0, 250.0, 1)
    assert (value, ms) == (2000.0, 250.0)
