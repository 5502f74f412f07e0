"""The sample-and-decode boundary through the C ABI: the physical error rate argument and
shot-range sharding.

  * bp4m_sample_and_decode with a p other than the graph's re-derives the tables for p, so
    its counts equal, bit for bit, those of a graph built at p (code capacity: only the
    priors change; circuit: the merged edge probabilities, shortest paths, priors and
    parities all change).
  * Shots are independent and the Philox counter is the global shot index, so
    bp4m_sample_and_decode_range over [0, a) and [a, N) adds up to the counts of one call
    over [0, N), for any split point (across the library's internal batch boundary too) and
    any Philox stream id.  This is what the multi-GPU path relies on: each rank decodes its
    own range and only the counts are summed.
"""
import pytest

import paper_2603_05381_gb300 as pkg
from paper_2603_05381_gb300 import sharding

from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


@pytest.mark.parametrize("model,d,p_built,p_run,T", [("code_capacity", 7, 0.08, 0.13, 14),
                                                      ("circuit", 5, 0.004, 0.007, 50)])
def test_sample_and_decode_rederives_tables_for_p(torch, model, d, p_built, p_run, T):
    n, seed = 40000, 17
    opts = pkg.make_opts(precision="fp32", early_exit=True)
    g = pkg.Graph(d, model, p_built)
    ref = pkg.Graph(d, model, p_run)
    want = ref.sample_and_decode(n, seed=seed, iters=T, opts=opts, p=p_run)
    got = g.sample_and_decode(n, seed=seed, iters=T, opts=opts, p=p_run)
    assert got == want
    # the cached tables serve a second call; the graph's own p is unaffected
    assert g.sample_and_decode(n, seed=seed, iters=T, opts=opts, p=p_run) == want
    own = g.sample_and_decode(n, seed=seed, iters=T, opts=opts, p=p_built)
    assert own == pkg.Graph(d, model, p_built).sample_and_decode(n, seed=seed, iters=T, opts=opts)
    assert own != want
    # profiling sees the launches made through the re-derived tables
    g.profile_enable(True)
    g.sample_and_decode(1000, seed=seed, iters=T, opts=opts, p=p_run)
    prof = g.profile_read()
    g.profile_enable(False)
    assert prof["sample"]["launches"] >= 1 and prof["count"]["launches"] >= 1
    for bad_p in (0.0, 0.5, -0.1):
        with pytest.raises(pkg.Bp4mError):
            g.sample_and_decode(10, seed=seed, iters=T, opts=opts, p=bad_p)


@pytest.mark.parametrize("model,d,p,T,stream_id", [("circuit", 5, 0.006, 50, 0), ("circuit", 5, 0.006, 50, 7),
                                                    ("code_capacity", 9, 0.1, 18, 3)])
def test_range_sharding_adds_up_to_one_call(torch, model, d, p, T, stream_id):
    # N spans the library's internal 2^20-shot batch and ends in a ragged tail
    n = (1 << 20) + 12345
    seed = 99
    opts = pkg.make_opts(precision="fp32", early_exit=True)
    g = pkg.Graph(d, model, p)
    whole = g.sample_and_decode(n, seed=seed, iters=T, opts=opts, stream_id=stream_id)
    assert whole["shots"] == n
    for split in (n // 2, 300001, 1 << 20):
        a = g.sample_and_decode(split, seed=seed, iters=T, opts=opts, stream_id=stream_id)
        b = g.sample_and_decode(n - split, seed=seed, iters=T, opts=opts, first_shot=split, stream_id=stream_id)
        assert sharding.add_counts(a, b) == whole, split
    # the interleaved per-rank ranges of the benchmark (two ranks, three steps) cover the
    # same shots as one rank
    per = 100000
    total = None
    for step in range(3):
        for rank in range(2):
            lo, hi = sharding.shot_range(rank, 2, step, per)
            c = g.sample_and_decode(hi - lo, seed=seed, iters=T, opts=opts, first_shot=lo, stream_id=stream_id)
            total = c if total is None else sharding.add_counts(total, c)
    assert total == g.sample_and_decode(6 * per, seed=seed, iters=T, opts=opts, stream_id=stream_id)
