"""Threshold sweeps over (distance, physical error rate) points with checkpoint/resume.

Two sweeps of the paper's experiments (Sec. "Numerical Results") on the rotated code:

  * code capacity: d in {5, 7, 9, 11, 13, 15, 17, 21} x p in {0.05, 0.06, ..., 0.20},
    BP4M with FP32 messages, at most 2d iterations with early exit, X and Z decoded
    separately (a shot fails if either type fails);
  * circuit level: the memory-Z experiment with d rounds, d in {3, 5, ..., 15} x p in
    {0.001, ..., 0.010}, BP4M with FP32 messages, T = 50 with early exit.

Every point runs through the C ABI (bp4m_sample_and_decode_range) in chunks of global shot
ranges; after each chunk the point's cumulative counts are appended to a JSON-lines state
file as {"key", "shots_done", "counts", ...}.  A run that is stopped and started again with
the same state file continues every point at its last recorded shot: the sampler is
counter-based (a shot's errors depend only on its global index and the seed), so the
resumed counts are bit-identical to an uninterrupted run's.

Per point the result has the logical error rate and its standard error, the
non-convergence ratio r_nc (shots where some type never converged; the paper's "fraction
of calls to MWPM"), the logical error rate among converged shots, mean iterations,
shots/s and message updates/s, and the dominant decode tier with its roofline fraction.

    python -m paper_2603_05381_gb300.sweep --config code_capacity --shots 1000000 --state cc.jsonl
"""
import argparse
import json
import math
import os
import sys
import time

CODE_CAPACITY_D = (5, 7, 9, 11, 13, 15, 17, 21)
CODE_CAPACITY_P = tuple(round(0.05 + 0.01 * k, 2) for k in range(16))
CIRCUIT_D = (3, 5, 7, 9, 11, 13, 15)
CIRCUIT_P = tuple(round(0.001 * k, 3) for k in range(1, 11))
TIER_SLOTS = ["tier%d" % k for k in range(1, 8)] + ["global"]


def config_points(name, ds=None, ps=None):
    """The points of a sweep: dicts with model, d, p, T (iterations) and a key."""
    if name == "code_capacity":
        ds, ps = ds or CODE_CAPACITY_D, ps or CODE_CAPACITY_P
        pts = [{"model": "code_capacity", "d": d, "p": p, "T": 2 * d} for d in ds for p in ps]
    elif name == "circuit":
        ds, ps = ds or CIRCUIT_D, ps or CIRCUIT_P
        pts = [{"model": "circuit", "d": d, "p": p, "T": 50} for d in ds for p in ps]
    else:
        raise ValueError("unknown sweep %r" % name)
    for pt in pts:
        pt["key"] = point_key(pt)
    return pts


def point_key(pt):
    return "%s:d=%d:p=%.6g:T=%d" % (pt["model"], pt["d"], pt["p"], pt["T"])


def load_state(path):
    """Last recorded line of every point in a JSON-lines state file (missing file: empty).
    A torn last line (a run killed while writing) is ignored."""
    state = {}
    if not path or not os.path.exists(path):
        return state
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line:
                continue
            try:
                rec = json.loads(line)
            except json.JSONDecodeError:
                continue
            prev = state.get(rec["key"])
            if prev is None or rec["shots_done"] >= prev["shots_done"]:
                state[rec["key"]] = rec
    return state


def _append(path, rec):
    if not path:
        return
    with open(path, "a") as f:
        f.write(json.dumps(rec, sort_keys=True) + "\n")
        f.flush()
        os.fsync(f.fileno())


def _add(a, b):
    if a is None:
        return json.loads(json.dumps(b))
    out = {}
    for k, v in a.items():
        out[k] = [x + y for x, y in zip(v, b[k])] if isinstance(v, list) else v + b[k]
    return out


def summarize(pt, counts, seconds, prof=None, peak=None):
    """Point statistics from cumulative counts (and optionally the profile of its launches)."""
    n = max(int(counts["shots"]), 1)
    fails = int(counts["fail"][2])
    ler = fails / n
    unconv = int(counts["unconverged_any"])
    conv = n - unconv
    res = {"key": pt["key"], "model": pt["model"], "d": pt["d"], "p": pt["p"], "T": pt["T"], "shots": n,
           "ler": ler, "ler_sigma": math.sqrt(max(ler * (1 - ler), 0.0) / n),
           "r_nc": unconv / n, "converged_ler": (int(counts["conv_fail_any"]) / conv) if conv else None,
           "mean_iters": int(counts["iterations"]) / n, "mean_defects": int(counts["defects"]) / n,
           "shots_per_s": n / seconds if seconds > 0 else None,
           "msg_updates_per_s": int(counts["msg_updates"]) / seconds if seconds > 0 else None}
    if prof:
        dom = max(TIER_SLOTS, key=lambda k: prof[k]["ms"])
        dp = prof[dom]
        if dp["ms"] > 0:
            g = dp["msg_updates"] / (dp["ms"] / 1e3) / 1e9
            res["dominant_tier"] = dom
            res["dominant_share"] = dp["ms"] / max(sum(prof[k]["ms"] for k in TIER_SLOTS), 1e-12)
            res["dominant_gmsg_per_s"] = g
            if peak:
                # shared-memory tiers: the special-function roof; the streaming tier: HBM at
                # 8 bytes per FP32 message update (read M[k][i], write M'[i][j])
                if dom == "global":
                    res["roofline"] = {"bound": "hbm", "frac": g * 8.0 / peak["hbm_gbs"], "peak_gbs": peak["hbm_gbs"]}
                else:
                    res["roofline"] = {"bound": "alu", "frac": g / peak["mufu_gmsg"], "peak_gmsg": peak["mufu_gmsg"]}
    return res


def sweep(points, shots, state_path=None, chunk=1 << 20, seed=1, precision="fp32", run_range=None,
          profile=False, peak=None, on_point=None, log=None):
    """Runs every point to `shots` shots, resuming from state_path.  run_range(pt, first,
    n) -> counts dict decodes one global shot range (default: the library, one graph per
    point).  Returns the per-point summaries."""
    state = load_state(state_path)
    if state_path and os.path.exists(state_path) and os.path.getsize(state_path):
        with open(state_path, "rb+") as f:
            f.seek(-1, os.SEEK_END)
            if f.read(1) != b"\n":
                f.write(b"\n")   # end a line torn by a killed writer before appending
    graphs = {}

    def lib_range(pt, first, n):
        import paper_2603_05381_gb300 as pkg
        g = graphs.get(pt["key"])
        if g is None:
            for old in list(graphs.values()):
                old.close()
            graphs.clear()
            g = graphs[pt["key"]] = pkg.Graph(pt["d"], pt["model"], pt["p"])
            if profile:
                g.profile_enable(True)
        opts = pkg.make_opts(precision=precision, early_exit=True)
        return g.sample_and_decode(n, seed=seed, iters=pt["T"], opts=opts, first_shot=first)

    run = run_range or lib_range
    out = []
    for pt in points:
        rec = state.get(pt["key"])
        done = rec["shots_done"] if rec else 0
        counts = rec["counts"] if rec else None
        seconds = rec["seconds"] if rec else 0.0
        while done < shots:
            n = min(chunk, shots - done)
            t0 = time.perf_counter()
            c = run(pt, done, n)
            seconds += time.perf_counter() - t0
            counts = _add(counts, c)
            done += n
            _append(state_path, {"key": pt["key"], "shots_done": done, "counts": counts, "seconds": seconds,
                                 "seed": seed, "precision": precision})
        prof = None
        if profile and run_range is None and pt["key"] in graphs:
            prof = graphs[pt["key"]].profile_read()
        res = summarize(pt, counts, seconds, prof, peak)
        out.append(res)
        if on_point:
            on_point(res)
        if log:
            print(json.dumps(res), file=log, flush=True)
    for g in graphs.values():
        g.close()
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--config", choices=["code_capacity", "circuit"], required=True)
    ap.add_argument("--shots", type=int, default=1000000)
    ap.add_argument("--chunk", type=int, default=1 << 20)
    ap.add_argument("--state", default=None, help="JSON-lines checkpoint file (resumed if it exists)")
    ap.add_argument("--d", default=None, help="comma-separated distances (default: the sweep's)")
    ap.add_argument("--p", default=None, help="comma-separated error rates (default: the sweep's)")
    ap.add_argument("--seed", type=int, default=1)
    args = ap.parse_args(argv)
    ds = tuple(int(x) for x in args.d.split(",")) if args.d else None
    ps = tuple(float(x) for x in args.p.split(",")) if args.p else None
    sweep(config_points(args.config, ds, ps), args.shots, state_path=args.state, chunk=args.chunk, seed=args.seed,
          log=sys.stdout)


if __name__ == "__main__":
    main()
