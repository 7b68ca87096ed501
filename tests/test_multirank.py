"""Host logic of the multi-GPU path on CPU with two gloo ranks (no GPU): the
view split of an uplift, the merge of the ranks' partial sums (Eq. 3 / Eq. 5
are additive over views) and the max-over-ranks step time.  Each rank computes
its views' partial num / den with the oracle; the merged result must equal
the single-process oracle uplift."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2410_14462_gb300 import inputs, shard


def _workload():
    return inputs.small_field_workload(n=3000, views=5, d=6, width=48, height=40)


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl = _workload()
        n, d = wl.scene.n, wl.d
        v0, v1 = shard.view_range(wl.cams.v, world, rank)
        num = np.zeros((n, d))
        den = np.zeros(n)
        for v in range(v0, v1):
            oracle.view_uplift(wl.scene, wl.cams.params[v], wl.cams.width, wl.cams.height,
                               wl.features(v).numpy(), num, den, nthreads=2)
        tn, td = torch.from_numpy(num), torch.from_numpy(den)
        shard.merge_partials(tn, td)
        slowest = shard.max_over_ranks(10.0 + rank)
        q.put((rank, (v0, v1), oracle.normalise(tn.numpy(), td.numpy()), td.numpy(), slowest))
    finally:
        dist.destroy_process_group()


def test_view_range_partitions():
    for V in (0, 1, 5, 150):
        for world in (1, 2, 3, 8):
            ranges = [shard.view_range(V, world, r) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == V
            assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.view_range(5, 2, 2)


def test_view_sharded_uplift_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    # read the results before joining (a worker's put blocks until it is read);
    # every wait is bounded, and a worker's exception surfaces through join
    procs = mp.spawn(_worker, args=(2, _free_port(), q), nprocs=2, join=False)
    got = []
    try:
        for _ in range(2):
            got.append(q.get(timeout=180))
    except Exception:
        procs.join(timeout=30)
        raise
    for _ in range(6):
        if procs.join(timeout=30):
            break
    else:
        for p in procs.processes:
            p.kill()
        pytest.fail("a gloo rank did not exit")
    got.sort(key=lambda t: t[0])
    assert [g[1] for g in got] == [(0, 3), (3, 5)]
    wl = _workload()
    f_ref, b_ref = oracle.uplift(wl.scene, wl.cams, lambda v: wl.features(v), nthreads=2)
    for rank, _, f, beta, slowest in got:
        np.testing.assert_allclose(beta, b_ref, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(f, f_ref, rtol=1e-11, atol=1e-13)
        assert slowest == 11.0
