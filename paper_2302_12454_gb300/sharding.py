"""Trial sharding across ranks (one process per GPU).

Trials are independent and every random draw of a trial is keyed by its
global index (ssqa_params.trial_offset + local index), so a run split into
contiguous trial ranges over ranks is identical to one run over all trials.
No collective is needed on the data path; results are gathered at the end.
"""
from __future__ import annotations


def trial_range(rank: int, world: int, total: int):
    """Contiguous [start, stop) share of `total` trials for `rank` of `world`
    (the first total % world ranks get one extra trial)."""
    if world < 1 or not 0 <= rank < world or total < 0:
        raise ValueError("bad rank/world/total")
    base, extra = divmod(total, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def gather_trials(local: dict, dist=None):
    """Concatenate per-rank result dicts (arrays with a leading trial axis) in
    rank order on every rank (torch.distributed all_gather_object)."""
    import numpy as np

    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return local
    parts = [None] * dist.get_world_size()
    dist.all_gather_object(parts, local)
    return {k: np.concatenate([p[k] for p in parts if p[k].shape[0]]) for k in local}
