"""The replicas path of bench.py on CPU: two gloo ranks agree on the slowest
rank's time, and only rank 0 runs the reference arm."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, values, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = bench.max_over_ranks(values[rank], dist, "cpu")
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("values", [[3.25, 7.5], [9.0, 1.0]])
def test_max_over_two_gloo_ranks(values):
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank_main, args=(2, _free_port(), values, out), nprocs=2, join=True,
                           start_method="spawn")
        assert dict(out) == {0: max(values), 1: max(values)}


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(4.5, None, "cpu") == 4.5


def test_reference_arm_other_ranks_do_no_work(capsys):
    sys.path.insert(0, ROOT)
    import bench
    # a rank other than 0 returns before reading its arguments, generating the
    # workload or printing
    assert bench.reference_arm(None, 1, 2) is None
    assert capsys.readouterr().out == ""
