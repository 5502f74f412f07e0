"""Fused decode of several graphs (bp4m_multi_*): one launch per decode tier over the shots of
circuit and code-capacity graphs of different distances with uneven shot counts.  Every
run (the autotuning first run, the run that captures the CUDA graph, the replays, and a
recapture for a new shot vector) must give, graph by graph, exactly what
bp4m_decode_batch gives each graph alone."""
import numpy as np
import pytest

import paper_2603_05381_gb300 as pkg

from gpu_util import gpu_sample, torch_cuda

pytestmark = pytest.mark.gpu

T = 40


@pytest.fixture(scope="module")
def setup():
    torch_cuda()
    specs = [("circuit", 5, 0.005, 0, 3000), ("circuit", 9, 0.005, 0, 1500), ("circuit", 13, 0.005, 0, 700),
             ("code_capacity", 9, 0.10, 0, 2500), ("code_capacity", 9, 0.10, 1, 2500)]
    graphs, entries = {}, []
    for model, d, p, ty, n in specs:
        key = (model, d, p)
        if key not in graphs:
            graphs[key] = pkg.Graph(d, model, p)
        g = graphs[key]
        synds, _ = gpu_sample(g, 0, n, seed=d + 31 * ty)
        entries.append((g, ty, synds[ty].cpu().numpy().view(np.uint32).copy()))
    yield entries
    for g in graphs.values():
        g.close()


def _alone(g, ty, synd, prec):
    n = synd.shape[0]
    pred = np.empty(n, dtype=np.uint8)
    conv = np.empty(n, dtype=np.uint8)
    g.decode_batch(synd, T, pkg.make_opts(precision=prec, type=ty), pred, conv)
    return pred, conv


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_fused_runs_match_decode_alone(setup, prec):
    entries = setup
    graphs = [g for g, _, _ in entries]
    types = [ty for _, ty, _ in entries]
    caps = [s.shape[0] for _, _, s in entries]
    want = [_alone(g, ty, s, prec) for g, ty, s in entries]
    m = pkg.Multi(graphs, caps, T, pkg.make_opts(precision=prec), types=types, max_defects=256)
    for rep in range(3):
        outs = [np.full(c, 9, dtype=np.uint8) for c in caps]
        convs = [np.full(c, 9, dtype=np.uint8) for c in caps]
        m.run([s for _, _, s in entries], outs, convs)
        for (p0, c0), o, c in zip(want, outs, convs):
            assert np.array_equal(o, p0) and np.array_equal(c, c0)
    info = m.info()
    print("%s fused: plan %d (%s ms), runs %d, replays %d" % (prec, info["plan"], [round(x, 2) for x in info["plan_ms"]],
                                                              info["runs"], info["graph_replays"]))
    assert info["runs"] == 3 and info["graph_replays"] == 2 and min(info["plan_ms"]) > 0
    # the autotuner also timed the streaming tier's cluster form (max_defects is above the
    # shared-memory tiers) and kept the faster block shape
    assert min(info["stream_ms"]) > 0 and info["stream_cluster"] in (1, 16)
    # a new shot vector: the graph is captured again
    half = [c // 2 for c in caps]
    outs = [np.empty(h, dtype=np.uint8) for h in half]
    m.run([np.ascontiguousarray(s[:h]) for (_, _, s), h in zip(entries, half)], outs)
    for (p0, _), o, h in zip(want, outs, half):
        assert np.array_equal(o, p0[:h])
    assert m.info()["graph_replays"] == 3
    m.close()


def test_fused_cluster_form_as_asked(setup):
    # a requested streaming cluster size is used as is (no timing of the alternative); outputs
    # equal decode alone
    entries = setup
    graphs = [g for g, _, _ in entries]
    types = [ty for _, ty, _ in entries]
    caps = [s.shape[0] for _, _, s in entries]
    want = [_alone(g, ty, s, "fp32") for g, ty, s in entries]
    m = pkg.Multi(graphs, caps, T, pkg.make_opts(precision="fp32", stream_cluster=4), types=types, max_defects=256)
    for rep in range(2):
        outs = [np.full(c, 9, dtype=np.uint8) for c in caps]
        m.run([s for _, _, s in entries], outs)
        for (p0, _), o in zip(want, outs):
            assert np.array_equal(o, p0)
    info = m.info()
    assert info["stream_cluster"] == 4 and info["stream_ms"] == [0.0, 0.0]
    m.close()


def test_fused_rejects_shots_beyond_max_defects(setup):
    g = setup[2][0]   # d = 13 circuit
    nw = g.info()["n_words"][0]
    n_det = g.info()["n_det"][0]
    synd = np.zeros((4, nw), dtype=np.uint32)
    rng = np.random.default_rng(5)
    for r in range(4):
        for k in rng.choice(n_det, size=300 if r == 1 else 20, replace=False):
            synd[r, k // 32] |= np.uint32(1 << (k % 32))
    m = pkg.Multi([g], [4], T, pkg.make_opts(), max_defects=256, cuda_graph=False)
    with pytest.raises(pkg.Bp4mError) as e:
        m.run([synd], [np.empty(4, dtype=np.uint8)])
    assert e.value.code == -3
    m.close()
