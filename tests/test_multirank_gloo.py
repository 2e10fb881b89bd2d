"""The multi-rank host logic on CPU: two gloo ranks agree on the max-over-ranks timing
and the element slabs cover every element once (no GPU involved)."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world_size, port, out):
    import torch.distributed as dist
    from paper_1808_05066_gb300.multirank import max_over_ranks, partition, sum_over_ranks
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world_size)
    m = max_over_ranks(10.0 + rank)
    n = sum_over_ranks(partition(82944 + 1, rank, world_size)[1])
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, m, n))


def test_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [11.0, 11.0]
    assert [r[2] for r in res] == [82945.0, 82945.0]


def test_partition_covers_units():
    from paper_1808_05066_gb300.multirank import partition
    for n in (0, 1, 7, 82944):
        for w in (1, 2, 3, 8):
            spans = [partition(n, r, w) for r in range(w)]
            assert sum(c for _, c in spans) == n
            pos = 0
            for s, c in spans:
                assert s == pos
                pos += c
