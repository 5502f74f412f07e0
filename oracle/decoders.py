"""BP4M and its variants on one shot, plus per-shot logical failure (oracle side).

Test infrastructure only: nothing in the product path imports this module.

BP4M (Sec. "Belief Propagation for Matching"): T iterations of message passing with a
marginalization after each.
  * full-T mode (the paper's text): every converged iteration yields a candidate, the
    lightest is kept (ties: the earliest).  If the last iteration did not converge,
    forced convergence runs once on its posteriors and the lighter of the two candidates
    is output (ties: the marginalization candidate).
  * early-exit mode (Sec. "Checking convergence" motivates checking early): the first
    converged iteration is output; if none converges in T iterations, the forced
    candidate of iteration T is output.
BP4MF (Sec. "BP4M Forced"): every iteration yields a candidate (the marginalization one if
it converged, else the forced one); the lightest over all T iterations is output (ties:
the earliest).  Memory-BP4MF is BP4MF with alpha != 1 (Sec. "BP Improvements").

The weight of a candidate is the sum of W_ij over its variables, added in ascending
(i, j) order.  The predicted observable flip is the XOR of the parity table over its
variables; a shot fails iff it differs from the true flip.
"""
import math

import numpy as np

from . import bp


class ShotResult:
    __slots__ = ("matching", "converged", "from_forced", "fallback", "iters",
                 "msg_updates", "lam", "margin", "weight", "obs_pred", "lam_hist")

    def __init__(self):
        self.matching = []
        self.converged = True
        self.from_forced = False
        self.fallback = False
        self.iters = 0
        self.msg_updates = 0
        self.lam = None
        self.margin = math.inf
        self.weight = 0.0
        self.obs_pred = 0
        self.lam_hist = None


def candidate_weight(W, matching):
    acc = 0.0
    for i, j in sorted(matching):
        acc += float(W[i, j])
    return acc


def _forced(lam, forced):
    """(matching in pick order, decisive margin) of forced convergence: the global greedy
    (default reading) or the paper's static partition."""
    if forced == "static":
        return bp.forced_convergence_static(lam), bp.static_margin(lam)
    return bp.forced_convergence(lam), bp.greedy_margin(lam)


def bp4m(L, W, T, early_exit=True, alpha=1.0, keep_hist=False, forced="greedy"):
    """BP4M on one shot's prior matrix L (s x s, diagonal = boundary) and weights W."""
    s = L.shape[0]
    r = ShotResult()
    if s == 0:
        return r
    M = np.zeros((s, s))
    best = None
    lam = None
    hist = [] if keep_hist else None
    conv = False
    for t in range(1, T + 1):
        M = bp.factor_update(L, M, alpha)
        lam = bp.posterior(L, M)
        if keep_hist:
            hist.append(lam.copy())
        r.msg_updates += s * s
        r.margin = min(r.margin, bp.decision_margin(lam))
        V, conv = bp.decide(lam)
        r.iters = t
        if conv:
            match = bp.matching_from(V)
            if early_exit:
                r.matching, r.converged, r.lam, r.lam_hist = match, True, lam, hist
                r.weight = candidate_weight(W, match)
                return r
            w = candidate_weight(W, match)
            if best is None or w < best[0]:
                best = (w, match)
    r.lam = lam
    r.lam_hist = hist
    r.converged = best is not None
    if not early_exit and conv:
        r.weight, r.matching = best
        return r
    r.fallback = True
    fmatch, fmargin = _forced(lam, forced)
    r.margin = min(r.margin, fmargin)
    wf = candidate_weight(W, fmatch)
    if best is not None and best[0] <= wf:
        r.weight, r.matching = best
    else:
        r.weight, r.matching, r.from_forced = wf, fmatch, True
    return r


def bp4mf(L, W, T, alpha=1.0, keep_hist=False, forced="greedy"):
    """BP4MF (alpha = 1) and Memory-BP4MF (alpha != 1) on one shot."""
    s = L.shape[0]
    r = ShotResult()
    if s == 0:
        return r
    M = np.zeros((s, s))
    best = None
    hist = [] if keep_hist else None
    any_conv = False
    for t in range(1, T + 1):
        M = bp.factor_update(L, M, alpha)
        lam = bp.posterior(L, M)
        if keep_hist:
            hist.append(lam.copy())
        r.msg_updates += s * s
        r.margin = min(r.margin, bp.decision_margin(lam))
        V, conv = bp.decide(lam)
        if conv:
            any_conv = True
            match, from_forced = bp.matching_from(V), False
        else:
            match, fmargin = _forced(lam, forced)
            r.margin = min(r.margin, fmargin)
            from_forced = True
            r.fallback = True
        w = candidate_weight(W, match)
        if best is None or w < best[0]:
            best = (w, match, from_forced)
        r.lam = lam
    r.iters = T
    r.lam_hist = hist
    r.converged = any_conv
    r.weight, r.matching, r.from_forced = best
    return r


def decode_shot(tables, dets, T, decoder="bp4m", early_exit=True, alpha=1.0, keep_hist=False, forced="greedy"):
    """Decode one shot given its sorted unsatisfied detectors; fills obs_pred.  forced:
    "greedy" (global greedy forced convergence, the default reading) or "static" (the
    paper's static partition)."""
    dets = np.asarray(dets, dtype=np.int64)
    L = tables.L[np.ix_(dets, dets)]
    W = tables.W[np.ix_(dets, dets)]
    if decoder == "bp4m":
        r = bp4m(L, W, T, early_exit=early_exit, alpha=alpha, keep_hist=keep_hist, forced=forced)
    elif decoder == "bp4mf":
        r = bp4mf(L, W, T, alpha=alpha, keep_hist=keep_hist, forced=forced)
    else:
        raise ValueError(decoder)
    par = 0
    for i, j in r.matching:
        par ^= int(tables.P[dets[i], dets[j]])
    r.obs_pred = par
    return r


def decode_syndromes(tables, synd, T, **kw):
    """Decode a bool [shots, n_det] syndrome matrix; returns a list of ShotResult."""
    out = []
    for row in np.asarray(synd, dtype=bool):
        out.append(decode_shot(tables, np.flatnonzero(row), T, **kw))
    return out
