"""Statistical agreement with the paper's printed BP4M data (unrotated code, code capacity).

The paper reports, for BP4M with T = 25 on the unrotated surface code under depolarizing
code-capacity noise, the fraction of shots whose marginalization never converged (the
calls to matching of BP4M+M) and logical error rates at d = 9 and 11
(tests/golden/paper_code_capacity.json).  These are Monte Carlo estimates from another
implementation whose prior convention and shot counts the paper does not state, so the
check is a band rather than an equality: the ratio ours / paper must lie in [0.85, 1.2]
for the non-convergence ratio (a shot counts as unconverged when either Pauli type never
converged) and in [0.6, 1.25] for the logical error rate.  The observed ratios are
printed.
"""
import json
import os

import pytest

import paper_2603_05381_gb300 as pkg

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_code_capacity.json")


def _run(d, p, shots, T):
    g = pkg.Graph(d, "code_capacity", p, family="unrotated")
    c = g.sample_and_decode(shots, seed=2026, iters=T, opts=pkg.make_opts(precision="fp32", early_exit=False))
    g.close()
    return c


def test_nonconvergence_ratio_and_ler_match_paper():
    import torch
    assert torch.cuda.is_available()
    ref = json.load(open(GOLDEN))
    T = ref["T"]
    shots = 1_000_000
    lines = []
    for p_s, per_d in ref["rnc"].items():
        for d_s, want in per_d.items():
            c = _run(int(d_s), float(p_s), shots, T)
            got = c["unconverged_any"] / c["shots"]
            lines.append(("rnc", int(d_s), float(p_s), got, want, got / want))
    for d_s, per_p in ref["ler"].items():
        for p_s, want in per_p.items():
            c = _run(int(d_s), float(p_s), shots, T)
            got = c["fail"][2] / c["shots"]
            lines.append(("ler", int(d_s), float(p_s), got, want, got / want))
    for kind, d, p, got, want, ratio in lines:
        print("%s d=%2d p=%.2f ours %.4g paper %.4g ratio %.3f" % (kind, d, p, got, want, ratio))
    for kind, d, p, got, want, ratio in lines:
        lo, hi = (0.85, 1.2) if kind == "rnc" else (0.6, 1.25)
        assert lo <= ratio <= hi, (kind, d, p, got, want)


def test_bbp4mf_ler_matches_paper():
    # B-BP4MF (quaternary BP, then BP4MF on reweighted priors) against the paper's printed
    # curve data.  At d = 5 the ratio ours / paper must lie in [0.75, 1.25] at every p, and
    # above the threshold (p = 0.18) in [0.6, 1.25] at every d.  Below the threshold at
    # d = 9 and 13 the paper's curves depend on how it treats posteriors above one half
    # (non-positive Dijkstra weights), which it does not state; the reading here takes such
    # edges as present (flipped), as matching decoders with negative weights do, and this
    # decoder is then stronger than the paper's curves there, so it must only be no worse
    # than the paper (ratio <= 1.25).  The threshold behaviour must reproduce: at p = 0.10
    # the logical error rate falls with d, at p = 0.18 it rises.
    import torch
    assert torch.cuda.is_available()
    ref = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_bbp4mf.json")))
    T = ref["T"]
    got = {}
    rows = []
    for d_s, per_p in ref["ler"].items():
        for p_s, want in per_p.items():
            g = pkg.Graph(int(d_s), "code_capacity", float(p_s), family="unrotated")
            c = g.sample_and_decode(1 << 20, seed=77, iters=T, opts=pkg.make_opts(precision="fp32", decoder="bbp4mf"))
            g.close()
            ler = c["fail"][2] / c["shots"]
            got[(int(d_s), float(p_s))] = ler
            rows.append((int(d_s), float(p_s), ler, want, ler / want))
    for d, p, ler, want, ratio in rows:
        print("bbp4mf ler d=%2d p=%.2f ours %.4g paper %.4g ratio %.3f" % (d, p, ler, want, ratio))
    for d, p, ler, want, ratio in rows:
        if d == 5:
            lo = 0.75
        elif p > ref["threshold"]:
            lo = 0.6
        else:
            lo = 0.0
        assert lo <= ratio <= 1.25, (d, p, ler, want)
    assert got[(5, 0.1)] > got[(9, 0.1)] > got[(13, 0.1)]
    assert got[(5, 0.18)] < got[(9, 0.18)] < got[(13, 0.18)]
