"""Pins for the rotated surface code geometry (code-capacity graphs)."""
import itertools
from collections import deque

import numpy as np
import pytest

from oracle.surface import code_capacity_graph, parity_check_matrices, rotated_code


@pytest.mark.parametrize("d", [3, 5, 7, 9])
def test_check_counts_and_commutation(d):
    code = rotated_code(d)
    assert len(code.z_checks) == (d * d - 1) // 2
    assert len(code.x_checks) == (d * d - 1) // 2
    hz, hx = parity_check_matrices(code)
    assert not ((hx.astype(int) @ hz.T.astype(int)) % 2).any()
    for h in (hz, hx):
        deg = h.sum(axis=0)
        assert deg.min() >= 1 and deg.max() <= 2
        assert set(h.sum(axis=1)) <= {2, 4}
    zl = np.zeros(d * d, dtype=int)
    zl[code.zl] = 1
    xl = np.zeros(d * d, dtype=int)
    xl[code.xl] = 1
    assert not ((hx @ zl) % 2).any()      # Z_L commutes with X-checks
    assert not ((hz @ xl) % 2).any()      # X_L commutes with Z-checks
    assert (zl @ xl) % 2 == 1             # and they anticommute


def _gf2_rank(m):
    m = m.copy() % 2
    r = 0
    for c in range(m.shape[1]):
        piv = [i for i in range(r, m.shape[0]) if m[i, c]]
        if not piv:
            continue
        m[[r, piv[0]]] = m[[piv[0], r]]
        for i in range(m.shape[0]):
            if i != r and m[i, c]:
                m[i] ^= m[r]
        r += 1
    return r


def test_logicals_are_not_stabilizers():
    code = rotated_code(5)
    hz, hx = parity_check_matrices(code)
    zl = np.zeros((1, 25), dtype=np.uint8)
    zl[0, code.zl] = 1
    assert _gf2_rank(np.vstack([hz, zl])) == _gf2_rank(hz) + 1


def test_min_weight_logical_d3_brute_force():
    # Every X error of weight < 3 with trivial Z-syndrome commutes with Z_L; a weight-3 one
    # that does not exists.
    code = rotated_code(3)
    hz, _ = parity_check_matrices(code)
    zl = np.zeros(9, dtype=int)
    zl[code.zl] = 1
    best = None
    for w in range(1, 4):
        for sup in itertools.combinations(range(9), w):
            e = np.zeros(9, dtype=int)
            e[list(sup)] = 1
            if not ((hz @ e) % 2).any() and (e @ zl) % 2 == 1:
                best = w
                break
        if best:
            break
    assert best == 3


def _odd_cycle_through_boundary(g):
    """Hops of the shortest boundary-to-boundary path with odd observable parity."""
    adj = [[] for _ in range(g.n_det + 1)]
    for (u, v, ob, _) in g.edges:
        adj[u].append((v, ob))
        adj[v].append((u, ob))
    B = g.n_det
    dist = {}
    dq = deque()
    for v, ob in adj[B]:
        if (v, ob) not in dist:
            dist[(v, ob)] = 1
            dq.append((v, ob))
    while dq:
        u, par = dq.popleft()
        for v, ob in adj[u]:
            st = (v, par ^ ob)
            if v == B:
                if par ^ ob == 1:
                    return dist[(u, par)] + 1
                continue
            if st not in dist:
                dist[st] = dist[(u, par)] + 1
                dq.append(st)
    return None


@pytest.mark.parametrize("d", [3, 5, 7])
@pytest.mark.parametrize("kind", ["X", "Z"])
def test_graph_distance_equals_d(d, kind):
    g = code_capacity_graph(rotated_code(d), kind)
    assert g.n_det == (d * d - 1) // 2
    assert len(g.edges) == d * d
    assert _odd_cycle_through_boundary(g) == d


@pytest.mark.parametrize("d", [2, 3, 5, 7])
def test_unrotated_counts_commutation_distance(d):
    from oracle.surface import unrotated_code
    code = unrotated_code(d)
    assert code.n == d * d + (d - 1) ** 2
    assert len(code.z_checks) == d * (d - 1) and len(code.x_checks) == d * (d - 1)
    hz, hx = parity_check_matrices(code)
    assert not ((hx.astype(int) @ hz.T.astype(int)) % 2).any()
    for h in (hz, hx):
        deg = h.sum(axis=0)
        assert deg.min() >= 1 and deg.max() <= 2
        assert set(h.sum(axis=1)) <= {3, 4} or d == 2
    zl = np.zeros(code.n, dtype=int)
    zl[code.zl] = 1
    xl = np.zeros(code.n, dtype=int)
    xl[code.xl] = 1
    assert not ((hx @ zl) % 2).any() and not ((hz @ xl) % 2).any() and (zl @ xl) % 2 == 1
    for kind in ("X", "Z"):
        g = code_capacity_graph(code, kind)
        assert _odd_cycle_through_boundary(g) == d
