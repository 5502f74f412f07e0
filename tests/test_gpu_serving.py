"""The decoding service (bp4m_server_*): requests of mixed graphs submitted together give,
request by request, exactly what bp4m_decode_batch gives each of them alone; compatible
pending requests are merged into batches; the slots' batches overlap; the device budget
evicts workspaces or refuses a batch that cannot fit."""
import numpy as np
import pytest

import paper_2603_05381_gb300 as pkg

from gpu_util import gpu_sample, torch_cuda

pytestmark = pytest.mark.gpu

T = 30


def _host_syndromes(g, shots, seed, ty=0):
    (synds), obs = gpu_sample(g, 0, shots, seed=seed)
    return synds[ty].cpu().numpy().view(np.uint32).copy()


def _alone(g, synd, opts):
    n = synd.shape[0]
    pred = np.empty(n, dtype=np.uint8)
    conv = np.empty(n, dtype=np.uint8)
    its = np.empty(n, dtype=np.int16)
    g.decode_batch(synd, T, opts, pred, conv, its)
    return pred, conv


@pytest.fixture(scope="module")
def graphs():
    torch_cuda()
    # d = 25 at p = 0.005 (about 900 defects a shot) runs in the streaming tier
    gs = [pkg.Graph(5, "circuit", 0.006), pkg.Graph(9, "circuit", 0.005), pkg.Graph(7, "code_capacity", 0.08),
          pkg.Graph(25, "circuit", 0.005)]
    yield gs
    for g in gs:
        g.close()


def test_mixed_requests_match_decode_alone(graphs):
    rng = np.random.default_rng(3)
    pools = []
    for k, g in enumerate(graphs):
        ty = 1 if k == 2 else 0
        synd = _host_syndromes(g, 6000, seed=20 + k, ty=ty)
        opts = pkg.make_opts(precision="fp32" if k != 1 else "fp16", early_exit=True, type=ty)
        pools.append((g, synd, opts))
    srv = pkg.Server(slots=3, max_batch_shots=4096)
    ids = [srv.add_graph(g) for g, _, _ in pools]
    reqs = []
    # three large requests occupy the slots, then many small ones queue up behind them
    for k in range(3):
        g, synd, opts = pools[1]
        a = 2000 * k
        reqs.append((1, a, 2000))
    for _ in range(60):
        k = int(rng.integers(0, 4))
        n = int(rng.integers(1, 300 if k < 3 else 64))
        a = int(rng.integers(0, 6000 - n))
        reqs.append((k, a, n))
    outs = []
    rids = []
    for k, a, n in reqs:
        g, synd, opts = pools[k]
        sub = np.ascontiguousarray(synd[a:a + n])
        pred = np.full(n, 7, dtype=np.uint8)
        conv = np.full(n, 7, dtype=np.uint8)
        rids.append(srv.submit(ids[k], sub, T, opts, pred, conv))
        outs.append((k, sub, pred, conv))
    infos = [srv.wait(r) for r in rids]
    st = srv.stats()
    srv.close()
    for (k, sub, pred, conv), info in zip(outs, infos):
        g, _, opts = pools[k]
        p0, c0 = _alone(g, sub, opts)
        assert np.array_equal(pred, p0) and np.array_equal(conv, c0)
        assert info["t_submit"] <= info["t_start"] <= info["t_done"]
    lat = np.array([i["latency_s"] for i in infos])
    print("service: %d requests, %d batches, %d merged, max %d batches in flight, latency p50 %.2f ms p99 %.2f ms"
          % (len(reqs), st["batches"], st["merged_requests"], st["max_inflight_batches"],
             1e3 * np.percentile(lat, 50), 1e3 * np.percentile(lat, 99)))
    assert st["shots"] == sum(n for _, _, n in reqs)
    assert st["merged_requests"] >= 1
    assert st["max_inflight_batches"] >= 2


def test_budget_evicts_and_refuses(graphs):
    g5, g9 = graphs[0], graphs[1]
    s5 = _host_syndromes(g5, 2048, seed=41)
    s9 = _host_syndromes(g9, 2048, seed=42)
    opts = pkg.make_opts(precision="fp32")
    # per-shot buffers of one 2048-shot workspace of the d = 9 graph: a budget of 1.5 of
    # them holds one graph at a time, so alternating graphs evicts
    w9 = 2048 * (s9.shape[1] * 4 + 5 + 9 * 4)
    srv = pkg.Server(slots=1, max_batch_shots=2048, device_budget_bytes=int(1.5 * w9))
    a, b = srv.add_graph(g5), srv.add_graph(g9)
    for rep in range(3):
        for gid, g, synd in ((a, g5, s5), (b, g9, s9)):
            pred = np.empty(2048, dtype=np.uint8)
            srv.wait(srv.submit(gid, synd, T, opts, pred))
            assert np.array_equal(pred, _alone(g, synd, opts)[0])
    st = srv.stats()
    srv.close()
    print("budget: %d evictions" % st["evictions"])
    assert st["evictions"] >= 3
    # a budget below one workspace refuses the batch
    srv = pkg.Server(slots=1, max_batch_shots=2048, device_budget_bytes=1024)
    gid = srv.add_graph(g9)
    pred = np.empty(2048, dtype=np.uint8)
    rid = srv.submit(gid, s9, T, opts, pred)
    with pytest.raises(pkg.Bp4mError) as e:
        srv.wait(rid)
    assert e.value.code == -2
    srv.close()


def test_heavy_scratch_is_outside_the_budget(graphs):
    # the budget covers per-shot buffers only; the streaming tier's scratch of a heavy graph
    # (hundreds of MB here) is outside it, so a budget that holds the per-shot buffers of the
    # d = 25 and d = 5 workspaces serves both graphs without evicting or refusing either
    g25, g5 = graphs[3], graphs[0]
    s25 = _host_syndromes(g25, 300, seed=51)
    s5 = _host_syndromes(g5, 300, seed=52)
    opts = pkg.make_opts(precision="fp32")
    cap = 1024
    w = sum(cap * (s.shape[1] * 4 + 5 + 9 * 4) for s in (s25, s5))
    srv = pkg.Server(slots=1, max_batch_shots=cap, device_budget_bytes=int(1.1 * w))
    a, b = srv.add_graph(g25), srv.add_graph(g5)
    for rep in range(2):
        for gid, g, synd in ((a, g25, s25), (b, g5, s5)):
            pred = np.empty(synd.shape[0], dtype=np.uint8)
            srv.wait(srv.submit(gid, synd, T, opts, pred))
            assert np.array_equal(pred, _alone(g, synd, opts)[0])
    st = srv.stats()
    srv.close()
    assert st["evictions"] == 0


def test_rejects_device_buffers_and_bbp4mf(graphs):
    torch = torch_cuda()
    g = graphs[0]
    srv = pkg.Server(slots=1)
    gid = srv.add_graph(g)
    nw = g.info()["n_words"][0]
    dev = torch.zeros((4, nw), dtype=torch.int32, device="cuda")
    pred = np.empty(4, dtype=np.uint8)
    with pytest.raises(pkg.Bp4mError):
        srv.submit(gid, dev, T, pkg.make_opts(), pred)
    host = np.zeros((4, nw), dtype=np.uint32)
    with pytest.raises(pkg.Bp4mError):
        srv.submit(gid, host, T, pkg.make_opts(decoder="bbp4mf"), pred)
    srv.close()


def test_heavy_request_is_served_in_pieces(graphs):
    # a 3072-shot request of the d = 25 circuit (a heavy graph, streaming tier) is decoded in
    # pieces of at most 1024 shots; small requests submitted right after it are served
    # between its pieces, and every result equals decode alone
    g_heavy, g_light = graphs[3], graphs[0]
    heavy = _host_syndromes(g_heavy, 3072, seed=41)
    light = _host_syndromes(g_light, 400, seed=42)
    opts = pkg.make_opts(precision="fp32", early_exit=True)
    srv = pkg.Server(slots=2, max_batch_shots=4096)
    gid_h, gid_l = srv.add_graph(g_heavy), srv.add_graph(g_light)
    out_h = np.empty(3072, dtype=np.uint8)
    conv_h = np.empty(3072, dtype=np.uint8)
    rid_h = srv.submit(gid_h, heavy, T, opts, out_h, conv_h)
    small = []
    for k in range(4):
        o = np.empty(100, dtype=np.uint8)
        small.append((srv.submit(gid_l, np.ascontiguousarray(light[100 * k:100 * (k + 1)]), T, opts, o), k, o))
    info_h = srv.wait(rid_h)
    infos = [(srv.wait(rid), k, o) for rid, k, o in small]
    st = srv.stats()
    srv.close()
    want_h, want_c = _alone(g_heavy, heavy, opts)
    assert np.array_equal(out_h, want_h) and np.array_equal(conv_h, want_c)
    want_l, _ = _alone(g_light, light, opts)
    for info, k, o in infos:
        assert np.array_equal(o, want_l[100 * k:100 * (k + 1)])
    # at least three pieces for the heavy request, and the small requests did not wait for
    # all of it
    assert st["batches"] >= 3 + 1
    assert info_h["batch_shots"] <= 1024
    assert min(info["t_done"] for info, _, _ in infos) < info_h["t_done"]
