"""The multi-GPU path of bench.py on CPU: two gloo ranks.

Each rank runs its own batch (weak scaling, no collective on the data path); the only
collectives are the barrier and the max over ranks of the timed duration.  This checks the
host logic that combines the ranks and that the ranks draw different seeded inputs.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2510_26313_gb300 import synth
    ms = 10.0 + 5.0 * rank                      # rank 1 is the slower one
    job_ms = bench.max_over_ranks(ms, "cpu")
    value = bench.weak_scaling_value(1e12, job_ms, world)
    phi = synth.random_phi(2, 3, T=1, instance=rank, orthonormal=False)
    dist.barrier()
    out[rank] = (job_ms, value, complex(phi.ravel()[0]))
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_rank_and_draw_their_own_inputs():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    assert out[0][0] == out[1][0] == 15.0
    # two ranks, 1e12 flops each, in 15 ms -> 2e12 / 0.015 s = 133.3 TFLOP/s
    assert abs(out[0][1] - 2e12 / 0.015 / 1e12) < 1e-9
    assert out[0][2] != out[1][2]


def test_single_rank_is_a_no_op():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5, "cpu") == 7.5
    assert bench.weak_scaling_value(2e12, 10.0, 1) == pytest.approx(200.0)
