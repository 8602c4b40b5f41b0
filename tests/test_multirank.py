"""The N > 1 path of bench.py on CPU: two gloo ranks (no GPU).

Ranks draw disjoint Philox round ranges and report one whole-job line: the
slowest rank's time, the sum of their valid counts and the union of their
distinct keys (all-gathered once after the timed region).
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        t, u, v = bench.merge_ranks(10.0 + 5.0 * rank, 100 * (rank + 1), 7 + rank, device="cpu")
        # distinct keys: rank 0 holds keys 0..99, rank 1 keys 50..179 (50 shared) -> 180 distinct
        import numpy as np
        ids = np.arange(0, 100) if rank == 0 else np.arange(50, 180)
        keys = np.zeros((len(ids), 3), np.uint32)
        keys[:, 0], keys[:, 2] = ids, ids * 7 + 1
        d = bench.distinct_keys_across_ranks(keys, device="cpu")
        q.put((rank, t, u, v, bench.round_base_of(rank), d))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_merge_and_disjoint_streams():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    for rank, t, u, v, base, d in out:
        assert t == 15.0            # slowest rank
        assert u == 300 and v == 15  # summed over ranks
        assert d == 180              # union of the ranks' distinct keys, on every rank
    bases = [o[4] for o in out]
    # the rounds one rank can use (2^20) never reach the next rank's range
    assert bases[1] - bases[0] >= 1 << 20


def test_single_process_merge_is_identity():
    import numpy as np
    import bench
    assert bench.merge_ranks(3.0, 5, 7, device="cpu") == (3.0, 5, 7)
    keys = np.array([[1, 2], [3, 4], [1, 2], [0, 0]], np.uint32)
    assert bench.distinct_keys_across_ranks(keys, device="cpu") == 3
    assert bench.distinct_keys_across_ranks(np.zeros((0, 2), np.uint32), device="cpu") == 0
