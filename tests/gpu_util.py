"""Helpers shared by the GPU parity tests: run the library through the C ABI with device
buffers, and compare its per-shot results with the oracle's."""
import numpy as np

import paper_2603_05381_gb300 as pkg
from oracle.decoders import decode_shot


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def gpu_sample(g, first_shot, shots, seed, stream_id=0):
    """Device-resident sample: returns (syndromes uint32 [types][shots][words], obs uint8 [types][shots])
    as numpy arrays plus the device tensors."""
    torch = torch_cuda()
    info = g.info()
    nt = info["n_types"]
    words = sum(info["n_words"])
    synd = torch.empty((shots * words,), dtype=torch.int32, device="cuda")
    obs = torch.empty((nt, shots), dtype=torch.uint8, device="cuda")
    g.sample(synd, obs, first_shot=first_shot, seed=seed, stream_id=stream_id)
    torch.cuda.synchronize()
    out = []
    off = 0
    for ty in range(nt):
        nw = info["n_words"][ty]
        out.append(synd[off:off + shots * nw].view(shots, nw))
        off += shots * nw
    return out, obs


def gpu_decode(g, synd_dev, T, opts, s_cap=0, lam_dtype=None):
    """decode_trace on device buffers; returns numpy dict."""
    torch = torch_cuda()
    n = synd_dev.shape[0]
    pred = torch.empty((n,), dtype=torch.uint8, device="cuda")
    flags = torch.empty((n,), dtype=torch.uint8, device="cuda")
    defects = torch.empty((n,), dtype=torch.int32, device="cuda")
    lam = partner = None
    if s_cap:
        dt = torch.float64 if opts.precision == pkg.FP64 else torch.float32
        lam = torch.full((n, s_cap, s_cap), float("nan"), dtype=dt, device="cuda")
        partner = torch.full((n, s_cap), -7, dtype=torch.int16, device="cuda")
    g.decode_trace(synd_dev, T, opts, pred, lam=lam, partner=partner, defects=defects, flags=flags,
                   s_cap=max(s_cap, 1))
    torch.cuda.synchronize()
    its = torch.empty((n,), dtype=torch.int16, device="cuda")
    conv = torch.empty((n,), dtype=torch.uint8, device="cuda")
    pred2 = torch.empty((n,), dtype=torch.uint8, device="cuda")
    g.decode_batch(synd_dev, T, opts, pred2, conv, its)
    torch.cuda.synchronize()
    out = {"obs": pred.cpu().numpy(), "flags": flags.cpu().numpy(), "s": defects.cpu().numpy(),
           "iters": its.cpu().numpy(), "conv": conv.cpu().numpy(), "obs2": pred2.cpu().numpy()}
    if s_cap:
        out["lam"] = lam.cpu().numpy()
        out["partner"] = partner.cpu().numpy()
    return out


def oracle_partner(matching, s):
    p = np.full(s, -1, dtype=np.int64)
    for i, j in matching:
        p[i] = j
        p[j] = i
    return p


def compare_shots(tables, synd_bool, gpu, T, idx, tau, decoder="bp4m", early_exit=True, alpha=1.0,
                  check_partner=True, pool=None, oracle=None, forced="greedy"):
    """Decodes shots `idx` with the oracle (in this process, or over `pool`, an
    oracle_pool.OraclePool of the same tables) and compares with the GPU.  Returns
    (n_compared, list of mismatching (shot, margin)).  `oracle`, if given, holds the oracle's
    results of every shot (indexed like synd_bool).  A mismatch with oracle margin >= tau
    is an error."""
    idx = list(idx)
    if oracle is not None:
        results = [oracle[k] for k in idx]
    elif pool is not None:
        results = pool.decode([np.flatnonzero(synd_bool[k]) for k in idx], T, decoder=decoder,
                              early_exit=early_exit, alpha=alpha, forced=forced)
    else:
        results = None
    bad = []
    for pos, k in enumerate(idx):
        dets = np.flatnonzero(synd_bool[k])
        if results is not None:
            r = results[pos]
        else:
            r = decode_shot(tables, dets, T, decoder=decoder, early_exit=early_exit, alpha=alpha, forced=forced)
        same = (r.obs_pred == int(gpu["obs"][k]) and int(r.converged) == int(gpu["flags"][k] & 1)
                and r.iters == int(gpu["iters"][k]) and int(r.from_forced) == int((gpu["flags"][k] >> 2) & 1))
        if same and check_partner and "partner" in gpu and len(dets) <= gpu["partner"].shape[1] and len(dets):
            same = np.array_equal(gpu["partner"][k][:len(dets)], oracle_partner(r.matching, len(dets)))
        if not same:
            bad.append((int(k), r.margin))
    return len(idx), bad
