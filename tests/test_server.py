"""Host logic of the continuous-batching server and of the replica sharding (no GPU).

The server is driven with a fake runner that only sleeps, so admission by slot and HBM
footprint, first-come-first-served order and completion are checked without a device.
The replica helpers run as two gloo ranks on the CPU.
"""
import os
import threading
import time

import pytest

from paper_2209_07969_gb300 import replicas, server


class _Spec:
    def __init__(self, size):
        self.size = size
        self.increments = [0.0] * 3


def test_admission_respects_slots_budget_and_order():
    budget, slots = 100, 3
    running = {"fp": 0, "n": 0, "max_fp": 0, "max_n": 0}
    lock = threading.Lock()

    def runner(req):
        with lock:
            running["fp"] += req.spec.size
            running["n"] += 1
            running["max_fp"] = max(running["max_fp"], running["fp"])
            running["max_n"] = max(running["max_n"], running["n"])
        time.sleep(0.01 * (1 + req.rid % 3))
        with lock:
            running["fp"] -= req.spec.size
            running["n"] -= 1
        return server.Result(req.rid, ok=True, reactions=[float(req.rid)])

    srv = server.Server(budget, slots, runner=runner, footprint=lambda r: r.spec.size)
    sizes = [40, 30, 50, 10, 60, 20, 35, 45, 5, 90]
    ids = [srv.submit(server.Request(_Spec(s))) for s in sizes]
    assert srv.drain(timeout=30)
    srv.close()
    assert sorted(srv.results) == ids
    assert all(r.ok for r in srv.results.values())
    assert running["max_fp"] <= budget and srv.peak_in_use <= budget
    assert running["max_n"] <= slots and srv.peak_running <= slots
    assert srv.admitted_order == ids            # first come, first served
    assert srv.peak_running >= 2                # requests overlapped


def test_oversized_request_is_rejected_and_failures_are_reported():
    def runner(req):
        if req.spec.size == 7:
            raise RuntimeError("injected failure")
        return server.Result(req.rid, ok=True)

    srv = server.Server(50, 2, runner=runner, footprint=lambda r: r.spec.size)
    with pytest.raises(ValueError):
        srv.submit(server.Request(_Spec(51)))
    a = srv.submit(server.Request(_Spec(7)))
    b = srv.submit(server.Request(_Spec(8)))
    assert srv.drain(timeout=10)
    srv.close()
    assert not srv.results[a].ok and "injected failure" in srv.results[a].error
    assert srv.results[b].ok


def test_served_batch_generator_is_seeded():
    from paper_2209_07969_gb300 import specimens as S
    a = S.served_batch(8, seed=0, grids=(16, 32))
    b = S.served_batch(8, seed=0, grids=(16, 32))
    assert [x[0] for x in a] == [x[0] for x in b]
    assert [(x[1].nx, x[1].E, x[2]) for x in a] == [(x[1].nx, x[1].E, x[2]) for x in b]
    for t, sp, scheme in a:
        h = 1.0 / sp.nx
        assert 2 * h <= sp.l <= 4 * h and 20 <= sp.E <= 210 and scheme in (0, 1, 2)


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = replicas.shard(list(range(10)), rank, world)
    t = replicas.max_over_ranks(1.0 + rank)
    n = replicas.sum_over_ranks(len(mine))
    out.put((rank, mine, t, n))
    dist.destroy_process_group()


def test_replicas_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    got = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
    assert got[0][1] == [0, 2, 4, 6, 8] and got[1][1] == [1, 3, 5, 7, 9]
    assert got[0][2] == got[1][2] == 2.0          # max over ranks of the timing
    assert got[0][3] == got[1][3] == 10.0         # every request ran exactly once
