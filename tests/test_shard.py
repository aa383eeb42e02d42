"""Host-side logic of the multi-GPU path, on CPU: balanced disjoint shards of
a sweep, and the gather / max-over-ranks helpers over a two-rank gloo group
(the same calls the benchmark makes over NCCL)."""
import os
import socket

import numpy as np
import pytest

from paper_1003_0282_gb300 import inputs as I
from paper_1003_0282_gb300 import shard as S


def test_balanced_shards_cover_disjoint_and_balance():
    doms = I.batch_sweep()
    cells = [p.cells for p in doms]
    for world in (1, 2, 3, 4, 8):
        parts = S.balanced_shards(cells, world)
        flat = sorted(d for p in parts for d in p)
        assert flat == list(range(len(doms)))
        loads = [sum(cells[d] for d in p) for p in parts]
        assert max(loads) - min(loads) <= max(cells)
        assert all(p == sorted(p) for p in parts)
    assert S.balanced_shards(cells, 2) == S.balanced_shards(cells, 2)


def test_rank_problems_modes():
    kw = dict(scale=0.25)
    weak0 = S.rank_problems(I.batch_sweep, 2, 0, "weak", **kw)
    weak1 = S.rank_problems(I.batch_sweep, 2, 1, "weak", **kw)
    assert len(weak0) == len(weak1) == 320
    assert [p.name for p in weak0] != [p.name for p in weak1]  # own seeds
    strong = [S.rank_problems(I.batch_sweep, 3, r, "strong", **kw) for r in range(3)]
    assert sum(len(x) for x in strong) == 320
    full = I.batch_sweep(scale=0.25)
    assert sorted(p.name for x in strong for p in x) == sorted(p.name for p in full)
    with pytest.raises(ValueError):
        S.rank_problems(I.batch_sweep, 2, 0, "diagonal")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        full = I.batch_sweep(scale=0.25)
        parts = S.balanced_shards([p.cells for p in full], world)
        mine = parts[rank]
        # per-domain rows as a solver would report them: (residual, mass, budget)
        local = np.array([[1e-3 * d, float(full[d].cells), -0.5 * d] for d in mine])
        got = S.gather_per_domain(local, mine, len(full))
        t = S.max_over_ranks(10.0 + rank)
        total = S.sum_over_ranks(float(sum(full[d].cells for d in mine)))
        q.put((rank, got, t, total))
    finally:
        dist.destroy_process_group()


def test_gather_and_max_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    full = I.batch_sweep(scale=0.25)
    want = np.array([[1e-3 * d, float(full[d].cells), -0.5 * d] for d in range(len(full))])
    for rank, got, t, total in out:
        assert np.array_equal(got, want), rank
        assert t == 11.0
        assert total == float(sum(p.cells for p in full))


def test_gather_rejects_overlap_and_gaps():
    rows = np.zeros((2, 3))
    with pytest.raises(ValueError):
        S.gather_per_domain(rows, [0, 0], 3)
    with pytest.raises(ValueError):
        S.gather_per_domain(rows, [0, 1], 3)
    assert np.array_equal(S.gather_per_domain(rows, [1, 0], 2), rows)


def _say(q, msg):
    """Put msg and wait for the queue's feeder thread to write it (os._exit follows)."""
    q.put(msg)
    q.close()
    q.join_thread()


def _leaving_worker(rank, world, port, q):
    import datetime
    import time

    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    try:
        dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
        S.max_over_ranks(float(rank))  # one whole step together: the group is fully connected
    except Exception as e:
        _say(q, (f"setup failed on rank {rank}: {type(e).__name__}", -1.0))
        os._exit(4)
    if rank == 1:
        os._exit(3)  # leaves between steps, with nothing in flight and without a word
    time.sleep(0.5)
    t0 = time.time()
    try:
        S.max_over_ranks(1.0)
        _say(q, ("no error", time.time() - t0))
    except Exception as e:  # the collective must end with an error, not wait forever
        _say(q, (type(e).__name__, time.time() - t0))
    os._exit(0)


def test_a_rank_that_leaves_ends_the_next_collective_with_an_error():
    """Failure detection on the host: a rank that exits between steps makes
    the survivors' next reduction raise within the process group's timeout."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_leaving_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    what, waited = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
    assert what != "no error" and not what.startswith("setup failed"), what
    assert 0.0 <= waited < 60.0
    assert procs[1].exitcode == 3 and procs[0].exitcode == 0
