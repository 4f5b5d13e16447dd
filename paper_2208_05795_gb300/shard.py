"""Several GPUs: independent problems per rank, or one code's canonical
candidate list split into ranges.

Candidates are independent, so ranks share nothing while they decode.  When
one code is split, the per-range trapping-set lists meet in one exchange
step: every rank contributes its (key -> record) map and the maps are merged
by key -- counts add, the threshold is the minimum, the sieve flags are
OR-ed -- which does not depend on the order of the ranks.  The timing of a
multi-rank run is the maximum over ranks and the work is summed.
"""
from __future__ import annotations


def shard_bounds(n_total: int, rank: int, world: int) -> tuple[int, int]:
    """Candidate range [begin, end) of `rank`: contiguous, sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world or n_total < 0:
        raise ValueError("bad shard")
    q, r = divmod(n_total, world)
    begin = rank * q + min(rank, r)
    return begin, begin + q + (1 if rank < r else 0)


def ts_records(view: dict) -> dict:
    """key -> (a, b, orbit, flags, count, thr, thr_f) of a ts_list_view() result."""
    out = {}
    for i, k in enumerate(view["keys"]):
        out[tuple(k)] = (int(view["a"][i]), int(view["b"][i]), int(view["orbit"][i]), int(view["flags"][i]),
                         int(view["count"][i]), int(view["thr"][i]), float(view["thr_f"][i]))
    return out


def _min_set(x, y):
    # thresholds: -1 (or negative) = none
    if x < 0:
        return y
    if y < 0:
        return x
    return min(x, y)


def merge_records(parts) -> dict:
    """Merges per-range maps; raises if two ranges disagree on a set's (a, b, orbit)."""
    out = {}
    for part in parts:
        for k, (a, b, orbit, flags, count, thr, thr_f) in part.items():
            if k not in out:
                out[k] = (a, b, orbit, flags, count, thr, thr_f)
                continue
            a0, b0, o0, f0, c0, t0, tf0 = out[k]
            if (a0, b0, o0) != (a, b, orbit) or (f0 & 1) != (flags & 1):
                raise ValueError(f"shards disagree on {k}")
            out[k] = (a0, b0, o0, f0 | flags, c0 + count, _min_set(t0, thr), _min_set(tf0, thr_f))
    return out


def exchange(records: dict, group=None) -> dict:
    """The exchange step: all ranks' maps, merged, on every rank."""
    import torch.distributed as dist
    parts = [None] * dist.get_world_size(group)
    dist.all_gather_object(parts, records, group=group)
    return merge_records(parts)


def reduce_time_and_work(ms: float, work, group=None, device="cpu"):
    """Max over ranks of the timed milliseconds and the sum of each work count."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    w = torch.tensor([float(x) for x in work], dtype=torch.float64, device=device)
    dist.all_reduce(w, group=group)
    return float(t.item()), [float(x) for x in w.tolist()]
