"""Replica path on CPU: two gloo ranks hold MLMC sums of disjoint sample sets
(as replicas with disjoint Philox counter ranges do), gather them, and merge
with Chan's formula; the result must equal the two-pass moments of the union
(oracle).  Also checks bench.py's max/sum reductions over ranks."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as tmp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _chan_table(y):
    """(count, mean, M2) per QoI of y[n][q] built by repeated pairwise merges
    of single samples (the same update the device uses), [2][q][3] with the
    second slot a copy."""
    n, q = y.shape
    t = np.zeros((2, q, 3))
    for i in range(n):
        for w in range(2):
            na, ma, m2a = t[w, :, 0], t[w, :, 1], t[w, :, 2]
            nn = na + 1
            d = y[i] - ma
            t[w, :, 1] = ma + d / nn
            t[w, :, 2] = m2a + d * d * na / nn
            t[w, :, 0] = nn
    return t


def _worker(rank, world, port, ys, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2302_07804_gb300 import mlmc
    import bench
    local = torch.tensor(_chan_table(ys[rank]), dtype=torch.float64)
    parts = [torch.zeros_like(local) for _ in range(world)]
    dist.all_gather(parts, local)
    merged = mlmc.merge_sums(parts)
    mx = bench.reduce_max(float(rank + 1), world)
    sm = bench.reduce_sum(float(rank + 1), world)
    if rank == 0:
        out.put((merged.numpy(), mx, sm))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_merge_equals_two_pass_of_union():
    from oracle import mlmc as omlmc
    from paper_2302_07804_gb300 import inputs
    gen = inputs.rng(77)
    ys = [gen.normal(0.5, 0.1, size=(37, 2)), gen.normal(0.52, 0.12, size=(53, 2))]
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, ys, q)) for r in range(2)]
    for p in procs:
        p.start()
    merged, mx, sm = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    n, mean, m2 = omlmc.two_pass_moments(np.concatenate(ys))
    assert merged[0, 0, 0] == n
    np.testing.assert_allclose(merged[0, :, 1], mean, rtol=1e-13)
    np.testing.assert_allclose(merged[0, :, 2], m2, rtol=1e-11)
    assert mx == 2.0 and sm == 3.0
