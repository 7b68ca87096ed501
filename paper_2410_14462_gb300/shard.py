"""Host logic of runs on several GPUs (one process per GPU, torch.distributed).

The uplift is a sum over views (Eq. 3 / Eq. 5: num = W^T F and den = W^T 1
are additive over any partition of the views), so one uplift can be split
across ranks by views and merged by summing the partial (num, den) before the
division.  The benchmark itself runs independent replicas of the whole step
(no data-path collective) and only reduces its timing.

* ``view_range``   the contiguous views a rank takes;
* ``merge_partials`` sums the ranks' partial num and den in place (the one
                   exchange step a view-sharded uplift has);
* ``sharded_uplift`` a view-sharded uplift on the GPUs through the C ABI;
* ``max_over_ranks`` the step time that counts: the slowest rank's.
"""
from __future__ import annotations


def view_range(n_views: int, world: int, rank: int) -> tuple[int, int]:
    """Views [v0, v1) of ``rank``: contiguous, sizes differing by at most one,
    every view in exactly one range."""
    if world < 1 or not 0 <= rank < world or n_views < 0:
        raise ValueError(f"bad split: {n_views} views, rank {rank} of {world}")
    base, extra = divmod(n_views, world)
    v0 = rank * base + min(rank, extra)
    return v0, v0 + base + (1 if rank < extra else 0)


def merge_partials(num, den, group=None):
    """Sum the ranks' partial numerators [n, d] and denominators [n] in place
    (torch tensors on the process group's device)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(num, op=dist.ReduceOp.SUM, group=group)
        dist.all_reduce(den, op=dist.ReduceOp.SUM, group=group)
    return num, den


def max_over_ranks(value: float, device="cpu", group=None) -> float:
    """The largest of the ranks' values (the step time of a synchronised job)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def sharded_uplift(scene, cams_params, width: int, height: int, feats, out=None, beta=None, stream=None):
    """Uplift with the views split across the ranks of the default process
    group: each rank accumulates its views (``feats`` [V, H, W, D] on this
    rank's GPU holds all V views or just this rank's, see below), the partial
    sums are added across ranks, and every rank normalises the total.

    ``feats`` may hold all views (the rank slices its range) or exactly the
    rank's range (shape[0] == v1 - v0)."""
    import torch
    import torch.distributed as dist
    from . import ludvig
    world = dist.get_world_size() if dist.is_initialized() else 1
    rank = dist.get_rank() if dist.is_initialized() else 0
    n_views = len(cams_params)
    v0, v1 = view_range(n_views, world, rank)
    local = feats if feats.shape[0] == v1 - v0 and world > 1 else feats[v0:v1]
    d = int(feats.shape[-1])
    num = torch.zeros((scene.n, d), dtype=torch.float32, device="cuda")
    den = torch.zeros((scene.n,), dtype=torch.float32, device="cuda")
    if v1 > v0:
        ludvig.uplift_accumulate(scene, cams_params[v0:v1], width, height, local.contiguous(), num, den,
                                 stream=stream)
    merge_partials(num, den)
    out = ludvig.uplift_finalize(num, den, out=out, beta=beta, stream=stream)
    return out, den
