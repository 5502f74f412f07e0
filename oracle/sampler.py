"""Error samplers and syndrome extraction (oracle side).

Test infrastructure only: nothing in the product path imports this module.

Each (shot, unit) pair draws one 32-bit Philox word (see `philox.unit_words`).
  * Code capacity (Sec. "Numerical Results", depolarizing channel): unit = data qubit;
    with t_k = floor(k * p / 3 * 2**32) the qubit suffers X if u < t1, Y if u < t2,
    Z if u < t3, nothing otherwise.
  * Circuit level: unit = edge of the merged detector graph in canonical order (sorted by
    (u, v, obs)); the edge fires iff u < floor(q_e * 2**32).
The syndrome is the XOR of the endpoints of the fired edges (boundary excluded); the
true observable flip is the XOR of their observable bits.
"""
import math

import numpy as np

from .philox import unit_words
from .surface import parity_check_matrices


def pauli_thresholds(p):
    return [math.floor(k * p / 3.0 * 4294967296.0) for k in (1, 2, 3)]


def edge_threshold(q):
    return math.floor(q * 4294967296.0)


def code_capacity_sample(code, p, shots, seed, stream=0):
    """Returns dict with 'X' and 'Z' entries of (syndrome bool [shots, n_det], obs [shots])."""
    u = unit_words(shots, code.n, seed, stream)
    t1, t2, t3 = pauli_thresholds(p)
    xcomp = (u < t2)                    # X or Y
    zcomp = (u >= t1) & (u < t3)        # Y or Z
    hz, hx = parity_check_matrices(code)
    out = {}
    for kind, comp, h, logical in (("X", xcomp, hz, code.zl), ("Z", zcomp, hx, code.xl)):
        synd = (comp.astype(np.int64) @ h.T.astype(np.int64)) % 2
        obs = comp[:, logical].sum(axis=1) % 2
        out[kind] = (synd.astype(bool), obs.astype(np.uint8))
    return out


def graph_sample(g, shots, seed, stream=0):
    """Circuit-level sampler on a merged detector graph (edges with q)."""
    n_e = len(g.edges)
    u = unit_words(shots, n_e, seed, stream)
    thr = np.array([edge_threshold(q) for (_, _, _, q) in g.edges], dtype=np.uint64)
    fired = u < thr[None, :]
    synd = np.zeros((len(np.atleast_1d(shots)), g.n_det), dtype=bool)
    obs = np.zeros(len(np.atleast_1d(shots)), dtype=np.uint8)
    for e, (a, b, ob, _) in enumerate(g.edges):
        col = fired[:, e]
        if not col.any():
            continue
        synd[:, a] ^= col
        if b < g.n_det:
            synd[:, b] ^= col
        if ob:
            obs ^= col.astype(np.uint8)
    return synd, obs


def pack_syndromes(synd):
    """Bool [shots, n_det] -> uint32 [shots, ceil(n_det/32)], detector j at word j>>5 bit j&31."""
    synd = np.asarray(synd, dtype=bool)
    shots, n = synd.shape
    words = (n + 31) // 32
    out = np.zeros((shots, words), dtype=np.uint32)
    for j in range(n):
        out[:, j >> 5] |= synd[:, j].astype(np.uint32) << np.uint32(j & 31)
    return out


def unpack_syndromes(packed, n_det):
    packed = np.asarray(packed, dtype=np.uint32)
    out = np.zeros((packed.shape[0], n_det), dtype=bool)
    for j in range(n_det):
        out[:, j] = (packed[:, j >> 5] >> np.uint32(j & 31)) & 1
    return out
