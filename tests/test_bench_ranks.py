"""The N > 1 path of bench.py on CPU: replicas only, so the one collective is the
whole-job reduction (slowest rank's time, sum of converged pairs), run here over two
gloo ranks; and the reference arm's other ranks exit without work."""
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [100.0, 120.0][rank]
    e2e = [0.11, 0.13][rank]
    conv = [49, 48][rank]
    out.put((rank, bench.whole_job(ms, e2e, conv, conv, dist, "cpu")))
    dist.barrier()
    dist.destroy_process_group()


def test_whole_job_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        ms_max, e2e_max, value, e2e_value = res[r]
        assert ms_max == 120.0 and e2e_max == 0.13
        assert value == pytest.approx(97 / 0.120) and e2e_value == pytest.approx(97 / 0.13)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job(50.0, 0.06, 49, 49) == (50.0, 0.06, pytest.approx(980.0), pytest.approx(49 / 0.06))


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
