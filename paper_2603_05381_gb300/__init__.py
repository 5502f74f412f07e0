"""BP4M decoding on GB300: Python binding of libbp4m (include/bp4m.h).

Every call below marshals arguments and forwards to the C ABI; all decoding work runs in
the library's CUDA kernels.  Buffers may be torch tensors (CUDA or CPU) or numpy arrays.
There is no CPU fallback: a missing or unloadable libbp4m.so raises.

    g = Graph(d=13, model="circuit", p=0.005)
    counts = g.sample_and_decode(shots=10**6, seed=1, iters=50)
"""
import ctypes

import numpy as np

from . import _capi
from ._capi import (CIRCUIT, CODE_CAPACITY, DEC_BBP4MF, DEC_BP4M, DEC_BP4MF, BF16, FP16, FP32, FP64, PRIOR_2P3,
                    PRIOR_P, Bp4mError, check, load)

__all__ = ["Graph", "Bp4mError", "load", "version", "FP32", "FP64", "DEC_BP4M", "DEC_BP4MF"]


def version():
    return load().bp4m_version().decode()


def probe_mufu(steps=4096, stream=None):
    """Special-function unit throughput of the current GPU (bp4m_probe_mufu): results per SM
    per clock of ex2, lg2 and the two alternating, and the SM count."""
    out = (ctypes.c_double * 4)()
    check(load().bp4m_probe_mufu(int(steps), out, _stream(stream)))
    return {"ex2": out[0], "lg2": out[1], "ex2_lg2_alternating": out[2], "sms": int(out[3])}


def _ptr(buf):
    """Raw address of a torch tensor or numpy array (None -> NULL)."""
    if buf is None:
        return None
    if hasattr(buf, "data_ptr"):
        if not buf.is_contiguous():
            raise ValueError("buffers must be contiguous")
        return buf.data_ptr()
    if isinstance(buf, np.ndarray):
        if not buf.flags["C_CONTIGUOUS"]:
            raise ValueError("buffers must be C-contiguous")
        return buf.ctypes.data
    raise TypeError("expected a torch tensor or a numpy array, got %r" % type(buf))


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def make_opts(precision=FP32, early_exit=True, decoder="bp4m", alpha=1.0, type=0, forced="greedy",
              stream_cluster=0, tile_form=0):
    """Decoder options (bp4m_opts).  forced: "greedy" (global greedy forced convergence) or
    "static" (the paper's static partition of the variables into per-factor blocks).
    stream_cluster: thread blocks sharing one shot in the streaming tier (0 = by width,
    1 = one block per shot, 2/4/8/16 = that size where available); outputs do not depend on it.
    tile_form: FP32 tiers of 113..144 defects, 0 = library default, 1 = row form, 2 = register tiles."""
    dec = ({"bp4m": DEC_BP4M, "bp4mf": DEC_BP4MF, "bbp4mf": DEC_BBP4MF}[decoder] if isinstance(decoder, str)
           else int(decoder))
    prec = {"fp32": FP32, "fp64": FP64, "fp16": FP16, "bf16": BF16}[precision] if isinstance(precision, str) else int(precision)
    fc = {"greedy": 0, "static": 1}[forced] if isinstance(forced, str) else int(forced)
    return _capi.Opts(prec, 1 if early_exit else 0, dec, float(alpha), int(type), fc, int(stream_cluster),
                      int(tile_form))


class Graph:
    """A static detector graph with its per-pair tables (bp4m_build_graph)."""

    def __init__(self, d, model="circuit", p=0.005, rounds=0, prior="p", pair_through_boundary=False,
                 family="rotated"):
        lib = load()
        m = {"code_capacity": CODE_CAPACITY, "circuit": CIRCUIT}[model] if isinstance(model, str) else model
        fam = {"rotated": _capi.ROTATED, "unrotated": _capi.UNROTATED}[family]
        code = _capi.Code(fam, int(d), int(rounds), _capi.MEMORY_Z)
        noise = _capi.Noise(m, float(p), {"p": PRIOR_P, "2p/3": PRIOR_2P3}[prior],
                            1 if pair_through_boundary else 0)
        h = ctypes.c_void_p()
        check(lib.bp4m_build_graph(ctypes.byref(code), ctypes.byref(noise), ctypes.byref(h)))
        self._h = h
        self.d, self.model, self.p = int(d), m, float(p)

    def close(self):
        if getattr(self, "_h", None):
            load().bp4m_free_graph(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        gi = _capi.GraphInfo()
        check(load().bp4m_graph_info(self._h, ctypes.byref(gi)))
        return {"n_types": gi.n_types, "n_det": list(gi.n_det)[:gi.n_types],
                "n_words": list(gi.n_words)[:gi.n_types], "n_edges": list(gi.n_edges)[:gi.n_types],
                "n_units": gi.n_units, "model": gi.model, "d": gi.d, "rounds": gi.rounds, "p": gi.p,
                "table_bytes": gi.table_bytes, "mean_defects": list(gi.mean_defects)[:gi.n_types]}

    def export(self, what, type=0):
        """Host copy of a table: 'W', 'L', 'parity', 'edges', 'thresholds'."""
        info = self.info()
        n = info["n_det"][type]
        if what == "W" or what == "L":
            out = np.empty((n, n), dtype=np.float64)
            code = _capi.EXPORT_W if what == "W" else _capi.EXPORT_L
        elif what == "parity":
            out = np.empty((n, n), dtype=np.uint8)
            code = _capi.EXPORT_PARITY
        elif what == "edges":
            arr = (_capi.Edge * info["n_edges"][type])()
            check(load().bp4m_graph_export(self._h, type, _capi.EXPORT_EDGES, ctypes.addressof(arr),
                                           ctypes.sizeof(arr)))
            return [(e.u, e.v, e.obs, e.q) for e in arr]
        elif what == "thresholds":
            k = info["n_units"] if info["model"] == CIRCUIT else 3
            out = np.empty(k, dtype=np.uint32)
            code = _capi.EXPORT_THRESH
        else:
            raise ValueError(what)
        check(load().bp4m_graph_export(self._h, type, code, out.ctypes.data, out.nbytes))
        return out

    def sample(self, syndromes, obs_true, first_shot=0, seed=1, stream_id=0, stream=None):
        """bp4m_sample into caller buffers: syndromes uint32 [types][shots][words], obs uint8 [types][shots]."""
        shots = obs_true.shape[-1]
        check(load().bp4m_sample(self._h, int(first_shot), int(shots), int(seed), int(stream_id),
                                 _ptr(syndromes), _ptr(obs_true), _stream(stream)))

    def decode_batch(self, syndromes, iters, opts, obs_pred=None, converged=None, iters_used=None,
                     stream=None):
        shots = syndromes.shape[0]
        check(load().bp4m_decode_batch(self._h, _ptr(syndromes), int(shots), int(iters), ctypes.byref(opts),
                                       _ptr(obs_pred), _ptr(converged), _ptr(iters_used), _stream(stream)))

    def decode_trace(self, syndromes, iters, opts, obs_pred, lam=None, partner=None, defects=None,
                     flags=None, s_cap=0, stream=None):
        tr = _capi.Trace(_ptr(lam), _ptr(partner), _ptr(defects), _ptr(flags), int(s_cap))
        check(load().bp4m_decode_trace(self._h, _ptr(syndromes), int(syndromes.shape[0]), int(iters),
                                       ctypes.byref(opts), _ptr(obs_pred), ctypes.byref(tr), _stream(stream)))

    def decode_bbp4mf(self, syndromes, iters, opts, obs_pred, flags=None, stream=None):
        """B-BP4MF on both types: syndromes uint32 [2][shots][words] (flat), outputs uint8 [2][shots]."""
        shots = obs_pred.shape[-1]
        check(load().bp4m_decode_bbp4mf(self._h, _ptr(syndromes), int(shots), int(iters), ctypes.byref(opts),
                                        _ptr(obs_pred), _ptr(flags), _stream(stream)))

    def profile_enable(self, on=True):
        """Start (and reset) or stop event timing of every kernel launch of this graph."""
        check(load().bp4m_profile_enable(self._h, 1 if on else 0))

    def profile_read(self):
        """Per slot (classify, tier1..7, global, sample, count): launches, ms, msg updates, shots."""
        pr = _capi.Profile()
        check(load().bp4m_profile_read(self._h, ctypes.byref(pr)))
        return {name: {"launches": pr.launches[k], "ms": pr.ms[k], "msg_updates": pr.msg_updates[k],
                       "shots": pr.shots[k]} for k, name in enumerate(_capi.PROFILE_SLOTS)}

    def sample_and_decode(self, shots, seed, iters, opts, first_shot=0, stream_id=0, stream=None, p=None):
        """Counts of the global shot range [first_shot, first_shot + shots) (bp4m_sample_and_decode_range),
        or with `p` given, of shots 0..shots-1 at physical error rate p (bp4m_sample_and_decode: a p
        other than the graph's re-derives the tables, cached per p)."""
        c = _capi.Counts()
        if p is not None:
            if first_shot or stream_id:
                raise ValueError("p is taken with the shot range starting at 0 on stream 0")
            check(load().bp4m_sample_and_decode(self._h, float(p), int(shots), int(seed), int(iters),
                                                ctypes.byref(opts), ctypes.byref(c), _stream(stream)))
        else:
            check(load().bp4m_sample_and_decode_range(self._h, int(first_shot), int(shots), int(seed),
                                                      int(stream_id), int(iters), ctypes.byref(opts),
                                                      ctypes.byref(c), _stream(stream)))
        return {"shots": c.shots, "fail": list(c.fail), "unconverged": list(c.unconverged),
                "forced_output": list(c.forced_output), "conv_fail": list(c.conv_fail),
                "iterations": c.iterations, "msg_updates": c.msg_updates, "defects": c.defects,
                "forced_runs": c.forced_runs, "forced_rounds": c.forced_rounds,
                "unconverged_any": c.unconverged_any, "conv_fail_any": c.conv_fail_any}


class Server:
    """Decoding service (bp4m_server_*): worker slots with their own streams decode queued
    requests of any registered graph, merging compatible pending requests into one batch.
    Host numpy buffers only."""

    def __init__(self, slots=4, max_batch_shots=4096, device_budget_bytes=0):
        lib = load()
        h = lib.bp4m_server_create(int(slots), int(max_batch_shots), int(device_budget_bytes))
        if not h:
            raise Bp4mError(-1, lib.bp4m_last_error().decode(errors="replace"))
        self._h = ctypes.c_void_p(h)
        self._keep = {}

    def add_graph(self, graph):
        gid = load().bp4m_server_add_graph(self._h, graph._h)
        if gid < 0:
            check(gid)
        return gid

    def submit(self, graph_id, syndromes, iters, opts, obs_pred, converged=None):
        """syndromes: uint32 [shots, n_words] (numpy); obs_pred / converged: uint8 [shots]
        numpy arrays filled when the request completes.  Returns the request id."""
        shots = obs_pred.shape[0]
        rid = load().bp4m_server_submit(self._h, int(graph_id), _ptr(syndromes), int(shots), int(iters),
                                        ctypes.byref(opts), _ptr(obs_pred), _ptr(converged))
        if rid < 0:
            check(int(rid))
        self._keep[rid] = (obs_pred, converged)
        return rid

    def wait(self, request, timeout=-1.0):
        """Blocks until the request finished; returns its timing dict."""
        info = _capi.RequestInfo()
        rc = load().bp4m_server_wait(self._h, int(request), float(timeout), ctypes.byref(info))
        if rc != _capi.BP4M_ETIMEOUT:
            self._keep.pop(request, None)  # finished (or failed): the service forgot it
        check(rc)
        return {"t_submit": info.t_submit, "t_start": info.t_start, "t_done": info.t_done,
                "latency_s": info.latency_s, "batch_shots": info.batch_shots, "slot": info.slot}

    def stats(self):
        st = _capi.ServerStats()
        check(load().bp4m_server_stats(self._h, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in _capi.ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            load().bp4m_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Multi:
    """Fused decode of several graphs (bp4m_multi_*): one launch per decode tier over the
    shots of all graphs, autotuned tier plan, CUDA-graph replay.  Host numpy buffers."""

    def __init__(self, graphs, max_shots, iters, opts, types=None, max_defects=256, cuda_graph=True):
        lib = load()
        n = len(graphs)
        hs = (ctypes.c_void_p * n)(*[g._h.value for g in graphs])
        caps = (ctypes.c_int64 * n)(*[int(x) for x in max_shots])
        tys = (ctypes.c_int * n)(*[int(t) for t in (types or [0] * n)])
        h = lib.bp4m_multi_create(n, hs, tys, caps, int(iters), ctypes.byref(opts), int(max_defects),
                                  1 if cuda_graph else 0)
        if not h:
            raise Bp4mError(-1, lib.bp4m_last_error().decode(errors="replace"))
        self._h = ctypes.c_void_p(h)
        self.n = n

    def run(self, syndromes, obs_pred, converged=None):
        """syndromes[k]: uint32 [shots_k, n_words]; obs_pred[k] (and converged[k]): uint8 [shots_k]."""
        n = self.n
        sy = (ctypes.c_void_p * n)(*[_ptr(x) for x in syndromes])
        sh = (ctypes.c_int64 * n)(*[int(o.shape[0]) for o in obs_pred])
        ob = (ctypes.c_void_p * n)(*[_ptr(x) for x in obs_pred])
        cv = (ctypes.c_void_p * n)(*[_ptr(x) for x in converged]) if converged is not None else None
        check(load().bp4m_multi_run(self._h, sy, sh, ob, cv))

    def info(self):
        mi = _capi.MultiInfo()
        check(load().bp4m_multi_info(self._h, ctypes.byref(mi)))
        return {"plan": mi.plan, "plan_ms": list(mi.plan_ms), "runs": mi.runs, "graph_replays": mi.graph_replays,
                "msg_updates": mi.msg_updates, "stream_cluster": mi.stream_cluster, "stream_ms": list(mi.stream_ms)}

    def close(self):
        if getattr(self, "_h", None):
            load().bp4m_multi_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

