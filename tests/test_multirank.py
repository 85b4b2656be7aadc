"""The benchmark's multi-rank bookkeeping on CPU with two gloo processes: every rank runs
its own seeded replica, the job's time is the slowest rank's, the whole-job rate counts
all ranks' units, and the reference arm does its work on rank 0 only."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, queue):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seconds = 1.0 + 0.5 * rank                     # rank 1 is the slower one
    t_max = bench.max_over_ranks(seconds, world, torch.device("cpu"))
    rate = bench.job_throughput(1000.0, 4, world, t_max)
    dist.barrier()
    dist.destroy_process_group()
    queue.put((rank, bench.replica_seed(rank), t_max, rate))


def test_two_rank_replicas_take_the_slowest_time():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    seeds = {g[1] for g in got}
    assert len(seeds) == 2                          # independent replicas
    for _, _, t_max, rate in got:
        assert t_max == 1.5                          # max over ranks
        assert rate == pytest.approx(1000.0 * 4 * 2 / 1.5)


def test_single_rank_is_its_own_time():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.0, 1, None) == 2.0
    assert bench.job_throughput(10.0, 3, 1, 2.0) == 15.0


def test_reference_arm_skips_other_ranks():
    sys.path.insert(0, ROOT)
    import bench

    class A:
        workload = "cfg1"
        steps = 1
        warmup = 0

    assert bench.run_reference(A(), 1, 2) == 0     # rank 1 exits at once, without work


def test_phase_times_serial_and_concurrent():
    """The bench's per-phase arithmetic on synthetic event times (ms from each iteration's
    first event): serial phases follow one another; under the concurrent schedule the
    prior's span starts at e0 and the MACE pass waits for the later branch."""
    import bench
    # serial: agents 0.4, prior 1.2, MACE 0.15 ms
    a, p, c = bench.phase_times([0.4, 0.4], [1.6, 1.6], [1.75, 1.75], False)
    assert (round(a * 1e3, 9), round(p * 1e3, 9), round(c * 1e3, 9)) == (0.4, 1.2, 0.15)
    # concurrent: agents end at 1.5, the prior at 1.54, MACE ends at 1.69 -> 0.15 after the prior
    a, p, c = bench.phase_times([1.5], [1.54], [1.69], True)
    assert (round(a * 1e3, 9), round(p * 1e3, 9), round(c * 1e3, 9)) == (1.5, 1.54, 0.15)
    # concurrent with the agents finishing last: the MACE pass is timed from them
    a, p, c = bench.phase_times([1.2], [0.9], [1.3], True)
    assert round(c * 1e3, 9) == 0.1
