"""Shot-range sharding across processes (one process per GPU).

Shots are independent and the sampler is counter-based (the Philox counter is the global
shot index), so a run split into disjoint global shot ranges over several ranks decodes
exactly the same shots as one rank decoding them all.  The only exchange is the sum of the
per-rank counters (u64 counts), done once per run.
"""

COUNT_KEYS = ("shots", "fail", "unconverged", "forced_output", "conv_fail", "iterations",
              "msg_updates", "defects", "forced_runs", "forced_rounds", "unconverged_any", "conv_fail_any")


def shot_range(rank, world, step, shots_per_rank, first=0):
    """Global [start, start + shots_per_rank) of `rank` at `step`: steps are interleaved so
    that the union over ranks of steps 0..k-1 is the contiguous range [first, first +
    k * world * shots_per_rank)."""
    if not (0 <= rank < world):
        raise ValueError("rank out of range")
    start = first + (step * world + rank) * shots_per_rank
    return start, start + shots_per_rank


def flatten(counts):
    out = []
    for k in COUNT_KEYS:
        v = counts.get(k, 0)
        out.extend(v if isinstance(v, (list, tuple)) else [v])
    return out


def unflatten(values, template):
    out = {}
    pos = 0
    for k in COUNT_KEYS:
        v = template.get(k, 0)
        n = len(v) if isinstance(v, (list, tuple)) else 1
        chunk = [int(x) for x in values[pos:pos + n]]
        out[k] = chunk if isinstance(v, (list, tuple)) else chunk[0]
        pos += n
    return out


def allreduce_counts(counts, device="cpu"):
    """Sums a counts dict over the default torch.distributed group (gloo or nccl)."""
    import torch
    import torch.distributed as dist
    flat = torch.tensor(flatten(counts), dtype=torch.int64, device=device)
    dist.all_reduce(flat, op=dist.ReduceOp.SUM)
    return unflatten(flat.tolist(), counts)


def add_counts(a, b):
    return unflatten([x + y for x, y in zip(flatten(a), flatten(b))], a)
