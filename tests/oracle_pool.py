"""A process pool that decodes shots with the FP64 oracle on every host core (test helper).

Started with the `spawn` method, so that it is safe to create after the parent process has
initialised CUDA.  Each worker receives the per-pair tables once (initializer) and decodes
one shot per task with `oracle.decoders.decode_shot`; results come back as plain tuples.
"""
import multiprocessing as mp
import os

import numpy as np

_TB = {}


def _init(L, W, P):
    _TB["tb"] = type("Tables", (), {"L": L, "W": W, "P": P})()


def _decode(task):
    from oracle.decoders import decode_shot
    dets, T, decoder, early_exit, alpha, forced = task
    r = decode_shot(_TB["tb"], np.asarray(dets, dtype=np.int64), T, decoder=decoder, early_exit=early_exit,
                    alpha=alpha, forced=forced)
    return (int(r.obs_pred), bool(r.converged), int(r.iters), bool(r.from_forced),
            [(int(i), int(j)) for i, j in r.matching], float(r.margin))


class OracleResult:
    __slots__ = ("obs_pred", "converged", "iters", "from_forced", "matching", "margin")

    def __init__(self, t):
        self.obs_pred, self.converged, self.iters, self.from_forced, self.matching, self.margin = t


class OraclePool:
    """with OraclePool(tables) as pool: results = pool.decode(list_of_detector_arrays, T, ...)"""

    def __init__(self, tables, procs=None):
        self.procs = procs or max(1, os.cpu_count() or 1)
        ctx = mp.get_context("spawn")
        self.pool = ctx.Pool(self.procs, initializer=_init,
                             initargs=(np.asarray(tables.L), np.asarray(tables.W), np.asarray(tables.P)))

    def decode(self, dets_list, T, decoder="bp4m", early_exit=True, alpha=1.0, forced="greedy"):
        tasks = [(np.asarray(d, dtype=np.int64), T, decoder, early_exit, alpha, forced) for d in dets_list]
        # large shots first so that the pool's tail is short
        order = sorted(range(len(tasks)), key=lambda k: -len(tasks[k][0]))
        out = self.pool.map(_decode, [tasks[k] for k in order], chunksize=1)
        res = [None] * len(tasks)
        for k, r in zip(order, out):
            res[k] = OracleResult(r)
        return res

    def close(self):
        self.pool.close()
        self.pool.join()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.pool.terminate()
        self.pool.join()


# ---------------------------------------------------------------- B-BP4MF shots

_BB = {}


def _init_bbp(d, family):
    from oracle.surface import code_capacity_graph, make_code
    code = make_code(d, family)
    _BB["code"] = code
    _BB["graphs"] = {k: code_capacity_graph(code, k) for k in ("X", "Z")}


def _bbp(task):
    from oracle.bbp4mf import bbp4mf_shot
    sx, sz, p, T = task
    out = bbp4mf_shot(_BB["code"], _BB["graphs"], sx, sz, p, T, T)
    return {k: out[k] for k in ("X", "Z", "qbp_converged", "margin", "margin_qbp", "margin_flip", "margin_bp")}


def bbp4mf_pool(d, family, shots, p, T, procs=None):
    """Oracle B-BP4MF of every (X-check syndrome, Z-check syndrome) pair in `shots` over a
    spawn process pool; returns the per-shot output dicts."""
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs or max(1, os.cpu_count() or 1), initializer=_init_bbp, initargs=(d, family)) as pool:
        return pool.map(_bbp, [(np.asarray(sx, dtype=int), np.asarray(sz, dtype=int), p, T) for sx, sz in shots],
                        chunksize=1)
