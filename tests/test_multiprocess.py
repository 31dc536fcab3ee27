"""The multi-process (replicas) path of bench.py on CPU ranks with the gloo backend:
the step time is the maximum over ranks and the value counts every rank's work."""
import importlib.util
import os
import subprocess
import sys

import pytest

from conftest import ROOT


def _load_bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench = _load_bench()
    ms = bench.max_over_ranks(1.0 + 2.0 * rank)  # rank 1 is the slow one
    value = bench.whole_job_gflops(4e9, world, ms)
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
        f.write(f"{ms} {value}\n")
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value_with_gloo(tmp_path):
    import socket

    import torch.multiprocessing as mp

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    for r in range(2):
        ms, value = map(float, open(tmp_path / f"r{r}.txt").read().split())
        assert ms == 3.0  # max over ranks, seen by every rank
        assert value == pytest.approx(2 * 4e9 / 3e-3 / 1e9)


def test_single_process_is_identity():
    bench = _load_bench()
    assert bench.max_over_ranks(2.5) == 2.5
    assert bench.whole_job_gflops(1e9, 1, 1.0) == pytest.approx(1000.0)


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
