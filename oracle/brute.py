"""Brute-force enumeration of P0 on small factor graphs (oracle side).

Test infrastructure only: nothing in the product path imports this module.

The valid configurations of Eq. (prob fg) are exactly the perfect matchings of the s
unsatisfied detectors in which a detector may also be matched to the boundary; each
has probability proportional to prod over its kept variables of rho(1)/rho(0) =
exp(l_v).  Enumerating them gives exact marginals, the maximiser of P0 and the
minimum-weight matching, for s up to about 10.
"""
import math

import numpy as np


def matchings(s, valid=None):
    """All involutions of range(s) restricted to valid variables, as lists of (i, j), i <= j."""
    if valid is None:
        valid = np.ones((s, s), dtype=bool)

    def rec(rem):
        if not rem:
            yield []
            return
        a = rem[0]
        rest = rem[1:]
        if valid[a, a]:
            for tail in rec(rest):
                yield [(a, a)] + tail
        for idx, b in enumerate(rest):
            if valid[a, b]:
                for tail in rec(rest[:idx] + rest[idx + 1:]):
                    yield [(a, b)] + tail

    return list(rec(list(range(s))))


def exact_marginal_llrs(L, valid=None):
    """ln P(v=1)/P(v=0) for every variable (s x s, symmetric); -inf/+inf where exact."""
    s = L.shape[0]
    ms = matchings(s, valid)
    logw = np.array([sum(float(L[i, j]) for i, j in m) for m in ms])
    top = logw.max()
    w = np.exp(logw - top)
    total = w.sum()
    on = np.zeros((s, s))
    for wk, m in zip(w, ms):
        for i, j in m:
            on[i, j] += wk
            if i != j:
                on[j, i] += wk
    off = total - on
    with np.errstate(divide="ignore"):
        out = np.log(on) - np.log(off)
    return out


def map_matching(L, valid=None):
    """The configuration maximising P0."""
    s = L.shape[0]
    best, arg = -math.inf, None
    for m in matchings(s, valid):
        v = sum(float(L[i, j]) for i, j in m)
        if v > best:
            best, arg = v, m
    return arg


def min_weight(W, valid=None):
    s = W.shape[0]
    return min(sum(float(W[i, j]) for i, j in m) for m in matchings(s, valid))
