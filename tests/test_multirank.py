"""The multi-process path of bench.py on CPU: two gloo ranks, the timing is the
max over ranks and the value is the whole job's work over that time; the
reference arm runs on rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    elapsed = [2.0, 3.5][rank]
    m = bench.max_over_ranks(elapsed, dist)
    rate = bench.whole_job_rate(1000, world, m)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, m, rate))


def test_two_gloo_ranks_take_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, rate in out:
        assert m == 3.5
        assert rate == pytest.approx(2000 / 3.5)


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(1.25) == 1.25
    assert bench.whole_job_rate(10, 1, 2.0) == 5.0


def test_report_helpers_describe_the_workload_they_measure():
    """The JSON line's traffic figure belongs to the captured particle count only,
    and its L2 note tells a streamed state from an L2-resident one."""
    sys.path.insert(0, ROOT)
    import bench
    import workloads as W
    big, small = W.lorenz96_large(), W.windkessel()
    for tag in ("k_propagate<L96,40,f32>", "k_resample"):
        assert bench.read_traffic(tag, small.P) is None
        t = bench.read_traffic(tag, big.P)
        assert t is None or t > 0  # None once the kernels change after the capture
    assert bench.l2_note(big).startswith("inputs larger than L2")
    assert bench.l2_note(small).startswith("L2-resident")
