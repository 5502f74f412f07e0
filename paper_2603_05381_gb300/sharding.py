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


# ---------------------------------------------------------------- failure handling
#
# A run split over ranks survives a rank that leaves between steps: every rank publishes
# the counts of each (step, rank) range it decodes and a heartbeat in a key-value store
# (torch.distributed.TCPStore or any object with set/get/add/check); when the ranks finish,
# a survivor re-issues every range whose owner stopped beating before publishing it, and
# the counts are summed from the store.  Because a range's counts depend only on its
# global shot indices, the result equals the uninterrupted run's.

import json
import threading
import time


class ShardedRun:
    """Shot-range sharding with host-side failure handling.

    run_range(first_shot, shots) -> counts dict (for example a closure over
    Graph.sample_and_decode) decodes one range.  Every rank calls step(k, run_range) for
    its steps, then finish(steps, run_range); finish returns the counts of all
    world x steps ranges, re-issuing those of ranks that left."""

    def __init__(self, store, rank, world, shots_per_rank, first=0, heartbeat_s=0.25, dead_after_s=2.0,
                 prefix="bp4m"):
        self.store, self.rank, self.world = store, rank, world
        self.per, self.first = shots_per_rank, first
        self.dead_after = dead_after_s
        self.prefix = prefix
        self.reissued = []
        self._stop = threading.Event()
        self._beat()
        self._hb = threading.Thread(target=self._beat_loop, args=(heartbeat_s,), daemon=True)
        self._hb.start()

    def _key(self, *parts):
        return "/".join([self.prefix] + [str(p) for p in parts])

    def _beat(self):
        self.store.set(self._key("hb", self.rank), repr(time.time()))

    def _beat_loop(self, period):
        while not self._stop.wait(period):
            try:
                self._beat()
            except Exception:
                return

    def _publish(self, k, r, counts):
        self.store.set(self._key("c", k, r), json.dumps(counts))

    def step(self, k, run_range):
        lo, hi = shot_range(self.rank, self.world, k, self.per, self.first)
        counts = run_range(lo, hi - lo)
        self._publish(k, self.rank, counts)
        return counts

    def leave(self):
        """Stops this rank's heartbeat (a rank that exits between steps)."""
        self._stop.set()

    def _alive(self, r):
        try:
            t = float(self.store.get(self._key("hb", r)))
        except Exception:
            return False
        return time.time() - t < self.dead_after

    def finish(self, steps, run_range, timeout_s=600.0):
        self.store.set(self._key("finished", self.rank), "1")
        t_end = time.time() + timeout_s
        total = None
        pending = [(k, r) for k in range(steps) for r in range(self.world)]
        while pending:
            left = []
            for k, r in pending:
                if self.store.check([self._key("c", k, r)]):
                    c = json.loads(self.store.get(self._key("c", k, r)))
                    total = c if total is None else add_counts(total, c)
                elif not self._alive(r) and not self.store.check([self._key("finished", r)]):
                    # the owner left before publishing: the first survivor to claim the range
                    # decodes it
                    if self.store.add(self._key("claim", k, r), 1) == 1:
                        lo, hi = shot_range(r, self.world, k, self.per, self.first)
                        self._publish(k, r, run_range(lo, hi - lo))
                        self.reissued.append((k, r))
                    left.append((k, r))
                else:
                    left.append((k, r))
            pending = left
            if pending:
                if time.time() > t_end:
                    raise TimeoutError("ranges %r were never published" % (pending[:4],))
                time.sleep(0.05)
        self._stop.set()
        return total
