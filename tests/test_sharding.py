"""Multi-process shot sharding on the CPU (gloo, world size 2): the union of the ranks'
shot ranges is the single-rank range, and the all-reduced counts equal the counts of one
process decoding every shot.  The per-shot decoder here is the oracle, so no GPU is needed;
the library's sample_and_decode_range takes the same global ranges."""
import os

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2603_05381_gb300 import sharding

D, P, T, SHOTS, STEPS, SEED = 3, 0.06, 20, 64, 3, 5


def _counts_for_range(start, stop):
    from oracle.decoders import decode_shot
    from oracle.graph import code_capacity_tables
    from oracle.sampler import code_capacity_sample
    from oracle.surface import code_capacity_graph, rotated_code
    code = rotated_code(D)
    samp = code_capacity_sample(code, P, np.arange(start, stop), seed=SEED)
    c = {"shots": stop - start, "fail": [0, 0, 0], "unconverged": [0, 0], "forced_output": [0, 0],
         "conv_fail": [0, 0], "iterations": 0, "msg_updates": 0, "defects": 0, "forced_runs": 0,
         "forced_rounds": 0, "unconverged_any": 0, "conv_fail_any": 0}
    anyf = np.zeros(stop - start, dtype=bool)
    allconv = np.ones(stop - start, dtype=bool)
    for ty, kind in ((0, "X"), (1, "Z")):
        tb = code_capacity_tables(code_capacity_graph(code, kind), P)
        synd, obs = samp[kind]
        for k in range(stop - start):
            r = decode_shot(tb, np.flatnonzero(synd[k]), T)
            f = r.obs_pred != obs[k]
            anyf[k] |= f
            c["fail"][ty] += int(f)
            c["unconverged"][ty] += int(not r.converged)
            allconv[k] &= bool(r.converged)
            c["iterations"] += r.iters
            c["msg_updates"] += r.msg_updates
            c["defects"] += int(synd[k].sum())
    c["fail"][2] = int(anyf.sum())
    c["unconverged_any"] = int((~allconv).sum())
    c["conv_fail_any"] = int((allconv & anyf).sum())
    return c


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    total = None
    ranges = []
    for step in range(STEPS):
        a, b = sharding.shot_range(rank, world, step, SHOTS)
        ranges.append((a, b))
        c = _counts_for_range(a, b)
        total = c if total is None else sharding.add_counts(total, c)
    red = sharding.allreduce_counts(total)
    q.put((rank, ranges, red))
    dist.destroy_process_group()


def test_two_rank_sharding_matches_single_process():
    world = 2
    port = 29500 + (os.getpid() % 2000)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    covered = sorted(r for _, ranges, _ in res for r in ranges)
    assert covered[0][0] == 0 and all(covered[i][1] == covered[i + 1][0] for i in range(len(covered) - 1))
    assert covered[-1][1] == world * STEPS * SHOTS
    single = _counts_for_range(0, world * STEPS * SHOTS)
    assert res[0][2] == res[1][2] == single


def test_shot_range_rejects_bad_rank():
    with pytest.raises(ValueError):
        sharding.shot_range(2, 2, 0, 10)


# ---------------------------------------------------------------- a rank that leaves


def _worker_leaving(rank, world, port, q, leave_after):
    import torch.distributed as dist
    store = dist.TCPStore("127.0.0.1", port, world, rank == 0, timeout=__import__("datetime").timedelta(seconds=120))
    dist.init_process_group("gloo", store=store, rank=rank, world_size=world)
    run = sharding.ShardedRun(store, rank, world, SHOTS, heartbeat_s=0.1, dead_after_s=1.0)
    for step in range(STEPS):
        if rank == 1 and step == leave_after:
            # leaves between steps: no kernel or collective in flight, the heartbeat stops
            run.leave()
            q.put((rank, None, []))
            return
        run.step(step, lambda lo, n: _counts_for_range(lo, lo + n))
    total = run.finish(STEPS, lambda lo, n: _counts_for_range(lo, lo + n), timeout_s=240)
    q.put((rank, total, run.reissued))


def test_rank_that_leaves_between_steps_has_its_ranges_reissued():
    world = 2
    port = 31500 + (os.getpid() % 2000)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker_leaving, args=(r, world, port, q, 1)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict((r, (t, ri)) for r, t, ri in (q.get(timeout=300) for _ in range(world)))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    total, reissued = res[0]
    # rank 1 decoded step 0 only; its steps 1 and 2 were re-issued on rank 0
    assert sorted(reissued) == [(1, 1), (2, 1)]
    assert total == _counts_for_range(0, world * STEPS * SHOTS)
