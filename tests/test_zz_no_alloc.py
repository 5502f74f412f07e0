"""bp4m_decode_noalloc: decoding for callers that cannot allocate device memory.

Such callers (for example a decoding service that fixes its device-memory footprint at
start-up) get an entry point whose scratch is a file-scope device array.  These tests call
it through the C ABI and check that it returns what bp4m_decode_batch returns on the same
syndromes, on two calls in a row, within the tolerance of the other parity tests: results
must agree exactly unless the oracle's decision margin on the shot is below tau (1e-9 for
FP64 messages, 1e-2 for FP32), where two correct roundings may decide differently.  The
file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import paper_2603_05381_gb300 as pkg
from paper_2603_05381_gb300 import _capi

pytestmark = pytest.mark.gpu

TAU = {"fp64": 1e-9, "fp32": 1e-2}


def _noalloc_fn():
    lib = _capi.load()
    fn = lib.bp4m_decode_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.POINTER(_capi.Opts),
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    return fn


def _call_noalloc(g, synd, T, opts, torch):
    n = synd.shape[0]
    obs = torch.full((n,), 0xAB, dtype=torch.uint8, device="cuda")
    conv = torch.full((n,), 0xAB, dtype=torch.uint8, device="cuda")
    its = torch.full((n,), -7, dtype=torch.int16, device="cuda")
    rc = _noalloc_fn()(g._h, synd.data_ptr(), n, T, ctypes.byref(opts), obs.data_ptr(), conv.data_ptr(),
                       its.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return rc, obs.cpu().numpy(), conv.cpu().numpy(), its.cpu().numpy()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_matches_decode_batch_twice(prec):
    import torch
    from oracle.circuit import Noise, circuit_graph
    from oracle.decoders import decode_shot
    from oracle.graph import circuit_tables
    from oracle.sampler import unpack_syndromes

    assert torch.cuda.is_available()
    d, p, n, T = 5, 0.008, 3000, 30
    g = pkg.Graph(d, "circuit", p)
    nw = g.info()["n_words"][0]
    synd = torch.empty((n * nw,), dtype=torch.int32, device="cuda")
    obs_true = torch.empty((1, n), dtype=torch.uint8, device="cuda")
    g.sample(synd, obs_true, first_shot=0, seed=21)
    synd = synd.view(n, nw)
    opts = pkg.make_opts(precision=prec, early_exit=True)
    # the existing entry point (its first call also puts the graph's tables on the device)
    ref_obs = torch.empty((n,), dtype=torch.uint8, device="cuda")
    ref_conv = torch.empty((n,), dtype=torch.uint8, device="cuda")
    ref_its = torch.empty((n,), dtype=torch.int16, device="cuda")
    g.decode_batch(synd, T, opts, ref_obs, ref_conv, ref_its)
    torch.cuda.synchronize()
    ref = (ref_obs.cpu().numpy(), ref_conv.cpu().numpy(), ref_its.cpu().numpy())
    og, _, _ = circuit_graph(d, Noise(p))
    ot = circuit_tables(og)
    sb = unpack_syndromes(synd.cpu().numpy().view(np.uint32), og.n_det)
    for call in range(2):
        rc, o, c, it = _call_noalloc(g, synd, T, opts, torch)
        assert rc == 0, _capi.load().bp4m_last_error().decode()
        diff = np.flatnonzero((o != ref[0]) | (c != ref[1]) | (it != ref[2]))
        for k in diff:
            r = decode_shot(ot, np.flatnonzero(sb[k]), T)
            assert r.margin < TAU[prec], (call, int(k), r.margin)
        assert len(diff) <= n // 100
    g.close()


def test_noalloc_rejects_shots_beyond_its_limit():
    import torch
    assert torch.cuda.is_available()
    g = pkg.Graph(13, "circuit", 0.005)
    info = g.info()
    n_det, nw = info["n_det"][0], info["n_words"][0]
    rng = np.random.default_rng(3)
    rows = np.zeros((2, nw), dtype=np.uint32)
    for r, s in ((0, 40), (1, 193)):
        for j in rng.choice(n_det, size=s, replace=False):
            rows[r, j >> 5] |= np.uint32(1) << np.uint32(j & 31)
    synd = torch.as_tensor(rows.view(np.int32), device="cuda")
    opts = pkg.make_opts(precision="fp32")
    g.decode_batch(synd[:1].contiguous(), 8, opts)  # set-up: tables on the device
    rc, o, c, it = _call_noalloc(g, synd, 8, opts, torch)
    assert rc == _capi.BP4M_OK - 1  # BP4M_EINVAL
    assert "192" in _capi.load().bp4m_last_error().decode()
    assert o[1] == 0 and c[1] == 0 and it[1] == 0
    # the array keeps no stale state: the valid shot alone decodes
    rc, o, c, it = _call_noalloc(g, synd[:1].contiguous(), 8, opts, torch)
    assert rc == 0 and it[0] > 0
    g.close()
