"""The N > 1 path of bench.py on CPU: two gloo ranks on 127.0.0.1.

The path does not shard (each rank runs an independent replica); what the
ranks share is the timing: a barrier before the timed region, the maximum
of the times over the ranks, and the whole-job value (updates of all ranks
over the slowest rank's time).  The reference arm runs on rank 0 only.
"""
import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist

    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    bench.barrier(world)
    ms = bench.max_over_ranks(10.0 + 3.0 * rank, world)  # rank 1 is the slower one
    value = bench.whole_job_mlups(2_000_000, world, ms * 1e-3)
    bench.barrier(world)
    q.put((rank, ms, value))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_sum_the_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [13.0, 13.0]
    assert all(abs(o[2] - 2 * 2_000_000 / 13e-3 / 1e6) < 1e-9 for o in out)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        steps, warmup, gpus, precision = 1, 3, 2, "fp32"

    bench.run_reference(Args(), rank=1, world=2)  # returns at once, no output, no oracle run
    assert capsys.readouterr().out == ""
