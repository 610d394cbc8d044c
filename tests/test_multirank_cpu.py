"""The N > 1 path of the benchmark on CPU ranks (gloo, world size 2): each rank
simulates its own events (disjoint ids, weak scaling) and the whole-job
numbers are the slowest rank's time and the summed counts."""
import os
import socket

import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    evs = bench.shard_events("batch_20keV_320um", 5, rank)
    ids = [e["event_id"] for e in evs]
    # rank r "takes" 100 * (r + 1) ms and did 10 * (r + 1) interactions
    t, inter, nev = bench.aggregate(dist, "cpu", 100.0 * (rank + 1), 10.0 * (rank + 1), 5.0)
    q.put((rank, ids, t, inter, nev))
    dist.barrier()
    dist.destroy_process_group()


def test_two_cpu_ranks_shard_events_and_aggregate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    (r0, ids0, t0, i0, n0), (r1, ids1, t1, i1, n1) = out
    assert ids0 == list(range(0, 5)) and ids1 == list(range(5, 10))
    assert t0 == t1 == 200.0            # max over ranks
    assert i0 == i1 == 30.0 and n0 == n1 == 10.0   # sums


def test_single_rank_aggregate_is_identity():
    import bench
    assert bench.aggregate(None, "cpu", 12.5, 3.0, 4.0) == (12.5, 3.0, 4.0)
