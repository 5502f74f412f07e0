"""CPU check of the leave-one-out formula the register-tile decode form evaluates for every
column of a row with no branch on the row's argmax (FP32 emulated in numpy, base-2 units):

    u_k = 2^max(x, 2^126 x), x = Q_k - m2;   S = sum_k min(u_k, 1)
    M'_k = min(-(m1 + lg2(1 + c (S - 1 - u_k))), -(m2 + lg2(S - 1))),  c = 2^(m2 - m1)

against the exact leave-one-out -max*_{j != k} Q_j of the oracle (Sec. "Belief Propagation":
the factor update is minus the Jacobian logarithm over the other variables of the factor),
on rows with exact ties, near-ties, very large gaps between the two largest entries and
padded (-inf) columns."""
import math

import numpy as np
import pytest

from oracle.bp import loo_lse

F = np.float32


def _register_tile_row(q):
    q = q.astype(F)
    srt = np.sort(q)[::-1]
    m1, m2 = srt[0], srt[1]
    x = (q - m2).astype(F)
    with np.errstate(over="ignore", invalid="ignore"):
        w = np.maximum(x, (x * F(2.0 ** 126)).astype(F))
        u = np.exp2(w.astype(np.float64)).astype(F)
    s = F(0)
    for v in np.minimum(u, F(1)):
        s = F(s + v)
    s1 = F(s - F(1))
    c = F(np.exp2(np.float64(m2 - m1)))
    a = F(np.float64(c) * np.float64(s1) + 1.0)
    sp = F(-(m2 + F(np.log2(np.float64(s1)))))
    with np.errstate(invalid="ignore", divide="ignore", over="ignore"):
        y = (np.float64(a) - np.float64(c) * u.astype(np.float64)).astype(F)
        out = (-(np.log2(y.astype(np.float64)).astype(F)) - m1).astype(F)
    return np.fmin(out, sp)


def _rows(seed, n):
    rng = np.random.default_rng(seed)
    for t in range(n):
        s = int(rng.integers(2, 40))
        kind = t % 5
        if kind == 0:
            q = rng.normal(-30, 20, s)
        elif kind == 1:
            q = rng.integers(-20, 0, s).astype(float)          # many exact ties
        elif kind == 2:
            q = np.concatenate([[rng.normal(0, 1)], rng.normal(-150, 5, s - 1)])  # gap ~150
        elif kind == 3:
            q = rng.normal(-5, 1e-6, s)                        # near-ties
        else:
            q = rng.normal(-30, 20, s)
            if s >= 3:
                q[rng.integers(0, s)] = -np.inf                 # a padded column
        yield q.astype(F).astype(np.float64)


@pytest.mark.parametrize("seed", [1, 2])
def test_register_tile_formula_is_the_exact_leave_one_out(seed):
    worst = 0.0
    for q in _rows(seed, 5000):
        got = _register_tile_row(q)
        # the oracle works in natural-log units: scale base-2 entries by ln 2 and back
        exact = -loo_lse(q * math.log(2.0), np.ones(q.shape[0], dtype=bool)) / math.log(2.0)
        ok = np.isfinite(exact)
        assert np.all(np.isfinite(got[ok]))
        err = float(np.max(np.abs(got[ok] - exact[ok]) / (np.abs(exact[ok]) + 1.0)))
        worst = max(worst, err)
    assert worst < 2e-6, worst


def test_argmax_of_a_row_gets_the_second_term():
    # a unique maximum: only its column takes the second term, the others the first
    q = np.array([-3.0, -1.0, -7.5, -2.0], dtype=np.float64)
    got = _register_tile_row(q)
    exact = -loo_lse(q * math.log(2.0), np.ones(4, dtype=bool)) / math.log(2.0)
    assert np.allclose(got, exact, rtol=0, atol=1e-5)
    # column 1 (the maximum) leaves out -1.0: -log2(2^-3 + 2^-7.5 + 2^-2)
    assert abs(got[1] + math.log2(2 ** -3 + 2 ** -7.5 + 2 ** -2)) < 1e-5
