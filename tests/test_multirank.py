"""The N > 1 path of the bench on CPU: two gloo ranks on 127.0.0.1.  Each rank
takes its own box (seed + rank) and no particle data is exchanged; the timing
every rank reports is the slowest rank's, and the whole-job value counts the
particles of both boxes (weak scaling)."""
import os
import queue
import socket

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        spec = bench.rank_spec(synth.SMALL_32, rank, world)
        pos, _ = synth.generate(spec, device="cpu", velocities=False)
        # the only collective: a checksum per rank, to show the boxes differ
        mine = torch.tensor([float(pos.double().sum())], dtype=torch.float64)
        sums = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(sums, mine)
        ms = bench.slowest_rank_ms(10.0 * (rank + 1), dist, "cpu")
        q.put((rank, spec.seed, [float(t.item()) for t in sums], ms, bench.job_value(world, spec.N, ms)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_boxes_and_report_the_slowest():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        res = sorted(q.get(timeout=180) for _ in range(world))
    except queue.Empty:
        for p in procs:
            p.kill()
        raise
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    base = synth.SMALL_32
    assert [r[1] for r in res] == [base.seed, base.seed + 1]
    sums = res[0][2]
    assert sums == res[1][2] and sums[0] != sums[1]          # two different boxes
    assert all(r[3] == 20.0 for r in res)                     # the slower rank's time on both
    assert all(r[4] == 2 * base.N / 20.0e-3 for r in res)     # both boxes' particles


def test_single_rank_uses_the_workload_itself():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.rank_spec(synth.BOX_1024, 0, 1) is synth.BOX_1024
    assert bench.slowest_rank_ms(7.5, None, "cpu") == 7.5
    assert bench.job_value(1, synth.BOX_1024.N, 1000.0) == synth.BOX_1024.N
