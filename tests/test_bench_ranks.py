"""The replica path of bench.py (one rank per GPU under torchrun) on gloo
ranks on the CPU: rank discovery from the launcher's environment, the
max-over-ranks time, and the whole-job value derived from it."""
import os
import socket

import pytest

import bench

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    w, r, local = bench.dist_setup()
    assert (w, r, local) == (world, rank, rank)
    dist.init_process_group("gloo", rank=r, world_size=w)
    try:
        total = bench.max_over_ranks(10.0 + 5.0 * rank, "cpu")   # rank k took 10 + 5k ms
        with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
            f.write(repr(total))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_max_over_ranks_on_gloo(tmp_path, world):
    import torch.multiprocessing as mp
    mp.spawn(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    seen = {float((tmp_path / f"r{k}.txt").read_text()) for k in range(world)}
    assert seen == {10.0 + 5.0 * (world - 1)}


def test_job_value_is_slowest_time_over_all_solves():
    # 2 ranks x 4 steps in 40 ms (slowest rank): 8 solves, 5 ms each
    assert bench.job_ms_per_solve(40.0, 4, 2) == 5.0
    assert bench.job_ms_per_solve(40.0, 4, 1) == 10.0


def test_dist_setup_defaults(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_setup() == (1, 0, 0)
