"""16-bit message storage (FP16 or BF16 messages; FP32 priors and arithmetic) against the
FP32 path on the same shots and against the FP64 oracle.

The bar for reduced precision is statistical: the logical error rate on the benchmark's
d = 13 circuit workload must lie within one Monte Carlo standard error of the FP32 rate on
the same shots.  The posterior LLRs after T iterations are compared with the oracle's
(error relative to |l| + 1, reported per format), and so is the per-shot output."""
import numpy as np
import pytest

import paper_2603_05381_gb300 as pkg
from oracle.bp import run_bp
from oracle.circuit import Noise, circuit_graph
from oracle.graph import circuit_tables
from oracle.sampler import unpack_syndromes

from gpu_util import compare_shots, gpu_decode, gpu_sample, torch_cuda

pytestmark = pytest.mark.gpu

_cache = {}


def _pair(d, p):
    key = (d, p)
    if key not in _cache:
        og, _, _ = circuit_graph(d, Noise(p))
        _cache[key] = (pkg.Graph(d, "circuit", p), og, circuit_tables(og))
    return _cache[key]


def _decode(g, synd, T, prec):
    torch = torch_cuda()
    n = synd.shape[0]
    pred = torch.empty((n,), dtype=torch.uint8, device="cuda")
    conv = torch.empty((n,), dtype=torch.uint8, device="cuda")
    its = torch.empty((n,), dtype=torch.int16, device="cuda")
    g.decode_batch(synd, T, pkg.make_opts(precision=prec, early_exit=True), pred, conv, its)
    torch.cuda.synchronize()
    return pred.cpu().numpy(), its.cpu().numpy()


# minimum fraction of shots whose output equals the FP32 output (measured on a GB300:
# 0.9998 for FP16, 0.9979 for BF16)
AGREE = {"fp16": 0.999, "bf16": 0.99}
# largest fraction of the oracle comparison's shots allowed to differ (measured: 1 and 2 of
# 400)
ORACLE_DIFF = {"fp16": 0.01, "bf16": 0.02}


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_reduced_precision_ler_within_one_standard_error(prec):
    g = pkg.Graph(13, "circuit", 0.005)
    n, T = 1 << 18, 50
    (synd,), obs = gpu_sample(g, 0, n, seed=11)
    obs = obs[0].cpu().numpy()
    p32, _ = _decode(g, synd, T, "fp32")
    p16, _ = _decode(g, synd, T, prec)
    ler32 = float((p32 != obs).mean())
    ler16 = float((p16 != obs).mean())
    sigma = np.sqrt(ler32 * (1 - ler32) / n)
    agree = float((p16 == p32).mean())
    print("%s: LER %.5f vs FP32 %.5f (sigma %.5f, diff %.2f sigma), outputs equal on %.4f of shots"
          % (prec, ler16, ler32, sigma, (ler16 - ler32) / sigma, agree))
    assert abs(ler16 - ler32) <= sigma
    assert agree >= AGREE[prec]


# bound on max |lambda - lambda_oracle| / (|l| + 1) after T iterations (measured: 0.0014
# for FP16, 0.0106 for BF16)
LAM_TOL = {"fp16": 0.005, "bf16": 0.04}


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_reduced_precision_posteriors_vs_oracle(prec):
    g, og, ot = _pair(5, 0.008)
    n = 48
    (synd,), _ = gpu_sample(g, 5000, n, seed=9)
    sb = unpack_syndromes(synd.cpu().numpy().view(np.uint32), og.n_det)
    worst, errs = 0.0, []
    for T in (1, 2, 5, 12):
        res = gpu_decode(g, synd, T, pkg.make_opts(precision=prec, early_exit=False), s_cap=64)
        for k in range(n):
            dets = np.flatnonzero(sb[k])
            s = len(dets)
            if s < 2:
                continue
            L = ot.L[np.ix_(dets, dets)]
            lam = run_bp(L, T)[-1][1]
            got = res["lam"][k][:s, :s].astype(np.float64)
            e = np.abs(got - lam) / (np.abs(L) + 1.0)
            errs.append(float(np.median(e)))
            worst = max(worst, float(e.max()))
    print("%s: |dlambda|/(|l|+1) worst %.3g, median of per-shot medians %.3g" % (prec, worst, np.median(errs)))
    assert worst < LAM_TOL[prec]


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_reduced_precision_outputs_vs_oracle(prec):
    g, og, ot = _pair(5, 0.008)
    n, T = 400, 30
    (synd,), _ = gpu_sample(g, 1000, n, seed=5)
    res = gpu_decode(g, synd, T, pkg.make_opts(precision=prec, early_exit=True), s_cap=64)
    sb = unpack_syndromes(synd.cpu().numpy().view(np.uint32), og.n_det)
    cnt, bad = compare_shots(ot, sb, res, T, range(n), 1e9)
    print("%s d5: %d/%d shots differ from the FP64 oracle (output, convergence, iterations)" % (prec, len(bad), cnt))
    assert len(bad) <= cnt * ORACLE_DIFF[prec]


def test_reduced_precision_rejected_where_unsupported():
    g = pkg.Graph(3, "code_capacity", 0.05)
    torch = torch_cuda()
    synd = torch.zeros((2 * 4,), dtype=torch.int32, device="cuda")
    pred = torch.empty((2, 4), dtype=torch.uint8, device="cuda")
    with pytest.raises(pkg.Bp4mError):
        g.decode_bbp4mf(synd, 5, pkg.make_opts(precision="fp16"), pred)
