"""Domain sharding across ranks (host logic, CPU, gloo with two ranks): longest-processing-
time assignment covers every domain once with balanced loads, and the counter gather and
the max-over-ranks timing give every rank the whole job's view."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2406_16786_gb300 import sharding


def test_lpt_assignment_is_a_balanced_partition():
    rng = np.random.default_rng(3)
    work = np.exp(rng.uniform(np.log(1e4), np.log(5e5), 64))
    for n in (1, 2, 3, 4, 8):
        parts = sharding.assign_lpt(work, n)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(64))
        loads = [work[p].sum() for p in parts]
        # LPT bound: no rank exceeds the average by more than the largest single domain
        assert max(loads) <= work.sum() / n + work.max() + 1e-9
    assert sharding.assign_lpt([5, 1, 4, 2, 3], 2) == [[0, 1, 3], [2, 4]]  # 5->0, 4->1, 3->1, 2->0, 1->0 (tie)
    with pytest.raises(ValueError):
        sharding.assign_lpt([1.0], 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, work, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = sharding.assign_lpt(work, world)[rank]
    local = {q: {"injected": 10 * q, "rank": rank} for q in mine}
    merged = sharding.gather_counters(local)
    t = sharding.max_over_ranks(1.5 + rank)
    out.put((rank, sorted(merged), [merged[q]["injected"] for q in sorted(merged)], t))
    dist.barrier()
    dist.destroy_process_group()


def test_gather_and_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    work = [float(x) for x in range(1, 21)]
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, work, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, keys, inj, t in res:
        assert keys == list(range(20))
        assert inj == [10 * k for k in range(20)]
        assert t == 2.5
