"""The multi-GPU path of bench.py is replicas only: each rank transforms its
own signal, the only collective is the max of the per-rank times, and the
reported value is the whole-job throughput.  These checks run that host logic
with the gloo backend on CPU, world size 2."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    sig = bench.rank_signal("multitone_n4096_gdw_s32", rank, world)
    t = bench.max_over_ranks(10.0 + 5.0 * rank)          # per-rank "times" 10 and 15 ms
    v = bench.weak_scaling_value(1000.0, 4, world, t)
    out[rank] = (float(sig[:8].sum()), t, v)
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_max_time_and_weak_value():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    (s0, t0, v0), (s1, t1, v1) = out[0], out[1]
    assert t0 == t1 == 15.0                     # max over ranks
    assert v0 == v1 == pytest.approx(2 * 1000.0 * 4 / 0.015)
    assert s0 != s1                             # independent replica signals


def test_single_rank_defaults():
    import bench
    import synth
    sig = bench.rank_signal("multitone_n4096_gdw_s32", 0, 1)
    assert np.array_equal(sig, synth.workload_signal("multitone_n4096_gdw_s32"))
    assert bench.max_over_ranks(3.5) == 3.5
