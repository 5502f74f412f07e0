"""Benchmark: Monte Carlo BP4M decoding of the rotated memory-Z circuit at d = 13.

One step = sample 10^6 shots (Philox), extract their syndromes, decode them with BP4M
(FP32 messages, at most 50 iterations, early exit, forced convergence when never
converged) and count logical failures: every step of the hot path, through the C ABI
call bp4m_sample_and_decode_range, with the shot range advancing every step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  N > 1 is launched by torchrun, one process per GPU; each
rank decodes its own shot range (no data-path collective).
"""
import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

D, P, T = 13, 0.005, 50
SHOTS = 1_000_000
SEED = 1
# FP32 decode kernel of each profile slot (rows per shot, columns per thread CH, threads per row G)
KERNEL_OF = {"tier1": "decode_smem_kernel<float, CH=32, G=1> (s <= 32)",
             "tier2": "decode_smem_kernel<float, CH=32, G=2> (s <= 64)",
             "tier3": "decode_smem_kernel<float, CH=24, G=4> (s <= 96)",
             "tier4": "decode_smem_kernel<float, CH=28, G=4> (s <= 112)",
             "tier5": "decode_smem_kernel<float, CH=32, G=4> (s <= 128)",
             "tier6": "decode_smem_kernel<float, CH=36, G=4> (s <= 144)",
             "tier7": "decode_smem_kernel<float, CH=40, G=4> (s <= 160)",
             "global": "decode_stream_kernel<float> (s > 160)"}
# the 113..144-defect tiers in the register-tile form (--tile-form 2)
KERNEL_OF_REG = {"tier5": "decode_reg_kernel<NB=32, B=4> (s <= 128)",
                 "tier6": "decode_reg_kernel<NB=24, B=6> (s <= 144)"}
# DRAM bytes (read + write) per decoded shot of each FP32 tier kernel, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum) of the 65,536-shot case of this workload,
# divided by the shots the launch decoded; a full launch's traffic is this times its shots.
DRAM_BYTES_PER_SHOT = {"tier4": 8.536e6 / 10172, "tier5": 12.013e6 / 26656, "tier6": 11.048e6 / 21645,
                       "tier7": 7.452e6 / 5503}
# the same with the register-tile form of tiers 5 and 6 (not yet captured for those two)
DRAM_BYTES_PER_SHOT_REG = {"tier4": DRAM_BYTES_PER_SHOT["tier4"], "tier7": DRAM_BYTES_PER_SHOT["tier7"]}
METRIC = "decoded shots/s & msg-updates/s vs HBM roofline (d=13 circuit); p50/p99 latency"
WORKLOAD = "rotated surface code memory-Z circuit, d=13, 13 rounds, uniform depolarizing p=0.005 " \
           "(gates, idles, data before rounds, reset/measure flips); 10^6 shots per step; BP4M, " \
           "FP32 messages, T=50 with early exit and forced-convergence fallback"
# The roofline denominator of the shared-memory tiers is measured in the same run by
# bp4m_probe_mufu (profiles/mufu_peak.md): ex2 and lg2 results per SM per clock, and the
# SM count of the device.  A message update needs one ex2 and one lg2, so it costs
# 1/ex2 + 1/lg2 SM-cycles of the special-function unit.


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--shots", type=int, default=SHOTS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    # message storage: fp32 (the configuration's, default) or the 16-bit forms (FP32 math)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp16", "bf16"])
    # FP32 tiers of 113..144 defects, passed explicitly: 1 = row form (the library's default),
    # 2 = register tiles
    ap.add_argument("--tile-form", type=int, default=1, choices=[1, 2])
    # decoding-service measurement: circuit graphs of these distances (p = 0.005; the
    # default is every odd distance 5..25), requests of 1..4096 shots arriving as a Poisson
    # process at a fraction of the measured capacity
    ap.add_argument("--serve-d", default="5,7,9,11,13,15,17,19,21,23,25")
    # a second mix of small distances only, where every batch fits the shared-memory tiers
    ap.add_argument("--serve-d-low", default="5,9,13")
    ap.add_argument("--serve-requests", type=int, default=200)
    # offered loads as fractions of the measured capacity (comma-separated), one Poisson
    # stream of --serve-requests requests each
    ap.add_argument("--serve-load", default="0.5")
    ap.add_argument("--serve-slots", type=int, default=4)
    # message storage of the service's requests (the plain per-request form it is compared with
    # is always FP32): the reduced-precision serving form by default
    ap.add_argument("--serve-precision", default="fp16", choices=["fp32", "fp16", "bf16"])
    ap.add_argument("--no-serve", action="store_true")
    # fused multi-graph decode of circuit and code-capacity graphs (d = 5, 9, 13, 17) with
    # uneven shot counts, FP16/BF16/FP32 messages against the plain per-graph FP32 form
    ap.add_argument("--fused", default=True, action=argparse.BooleanOptionalAction)
    ap.add_argument("--fused-scale", type=float, default=0.1)
    # only measure the special-function unit (the shared-memory tiers' roofline
    # denominator) with the SM clocks sampled meanwhile, print it and exit
    ap.add_argument("--mufu-probe", action="store_true")
    # threshold sweeps (code-capacity and circuit-level grids of the paper's experiments):
    # one JSON line per (d, p) point instead of the benchmark line
    ap.add_argument("--sweep", choices=["code_capacity", "circuit"], default=None)
    ap.add_argument("--sweep-shots", type=int, default=1000000)
    ap.add_argument("--sweep-state", default=None, help="JSON-lines checkpoint (resumed if present)")
    ap.add_argument("--sweep-d", default=None)
    ap.add_argument("--sweep-p", default=None)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


# ---------------------------------------------------------------- CPU baseline (oracle)

_W = {}


def _oracle_init(L, W, P):
    _W["tb"] = type("T", (), {"L": L, "W": W, "P": P})()


def _oracle_decode(dets):
    from oracle.decoders import decode_shot
    import numpy as np
    r = decode_shot(_W["tb"], np.asarray(dets), T)
    return r.obs_pred, r.msg_updates


def cpu_baseline(n_shots=None, seed=SEED, first_shot=0):
    """Times the FP64 oracle (as it stands) on a bounded sample of the same workload, on all
    host cores through a spawn-started process pool."""
    import numpy as np
    from oracle.circuit import Noise, circuit_graph
    from oracle.graph import all_pairs, edge_weights_circuit, prior_llr
    from oracle.sampler import graph_sample
    cores = os.cpu_count() or 1
    n = n_shots or max(16, min(10 * cores, 400))
    og, _, _ = circuit_graph(D, Noise(P))
    synd, _ = graph_sample(og, np.arange(first_shot, first_shot + n, dtype=np.uint64), seed=seed)
    dets = [np.flatnonzero(r) for r in synd]
    srcs = sorted(set(int(x) for dd in dets for x in dd))
    Wt, Pt = all_pairs(og, edge_weights_circuit(og), sources=srcs)
    Lt = prior_llr(Wt)
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores, initializer=_oracle_init, initargs=(Lt, Wt, Pt)) as pool:
        pool.map(_oracle_decode, [dets[0]] * cores)  # warm the workers
        t0 = time.perf_counter()
        out = pool.map(_oracle_decode, dets, chunksize=1)
        dt = time.perf_counter() - t0
    msgs = sum(m for _, m in out)
    return {"value": n / dt, "unit": "shots/s", "cores": cores, "kind": "oracle",
            "sample": "%d shots (global indices %d..%d, seed %d) of the same d=13 p=0.005 workload, FP64 "
                      "oracle BP4M, T=50 early exit; %.1f s wall on %d processes" % (n, first_shot, first_shot + n - 1,
                                                                                      seed, dt, cores),
            "msg_updates_per_s": msgs / dt, "seconds": dt}


# ---------------------------------------------------------------- our arm

def run_serving(args, dev, serve_d):
    """p50/p99 request latency and sustained shots/s of the decoding service (Server) on a
    Poisson stream of requests of mixed distance: each request a uniform 1..4096-shot slice
    of pre-sampled syndromes of one of the graphs.  Capacity is measured first by a closed
    burst of requests; arrivals then run at serve_load x capacity."""
    import numpy as np
    import torch
    import paper_2603_05381_gb300 as pkg

    ds = [int(x) for x in serve_d.split(",") if x]
    rng = np.random.default_rng(SEED)
    opts = pkg.make_opts(precision=args.serve_precision, early_exit=True)
    graphs, pools = [], []
    for d in ds:
        g = pkg.Graph(d, "circuit", P)
        nw = g.info()["n_words"][0]
        pool = 8192
        synd = torch.empty((pool * nw,), dtype=torch.int32, device=dev)
        obs = torch.empty((1, pool), dtype=torch.uint8, device=dev)
        g.sample(synd, obs, first_shot=10**9, seed=SEED)
        torch.cuda.synchronize()
        graphs.append(g)
        pools.append(synd.view(pool, nw).cpu().numpy().view(np.uint32).copy())
    srv = pkg.Server(slots=args.serve_slots, max_batch_shots=4096)
    gids = [srv.add_graph(g) for g in graphs]

    def make_request():
        k = int(rng.integers(0, len(graphs)))
        n = int(rng.integers(1, 4097))
        a = int(rng.integers(0, 8192 - n + 1))
        return k, np.ascontiguousarray(pools[k][a:a + n]), np.empty(n, dtype=np.uint8)

    # warm-up: workspaces of every graph in the slots (two random requests per graph and slot)
    warm = [make_request() for _ in range(2 * len(graphs) * args.serve_slots)]
    for r in [srv.submit(gids[k], s, T, opts, o) for k, s, o in warm]:
        srv.wait(r)
    # capacity: a closed burst
    burst = [make_request() for _ in range(64)]
    t0 = time.perf_counter()
    ids = [srv.submit(gids[k], s, T, opts, o) for k, s, o in burst]
    for r in ids:
        srv.wait(r)
    cap_shots = sum(o.shape[0] for _, _, o in burst) / (time.perf_counter() - t0)
    # the plain form on the same requests: one FP32 bp4m_decode_batch call per request, in order
    opts32 = pkg.make_opts(precision="fp32", early_exit=True)
    t0 = time.perf_counter()
    for k, sy, o in burst:
        graphs[k].decode_batch(sy, T, opts32, o)
    plain_shots = sum(o.shape[0] for _, _, o in burst) / (time.perf_counter() - t0)
    mean_req = 2048.5
    loads = []
    # every load replays the same requests with the same arrival pattern, its gaps scaled by
    # the load's rate, so that the loads differ only in the offered rate
    reqs = [make_request() for _ in range(args.serve_requests)]
    unit_gaps = rng.exponential(1.0, size=len(reqs))
    for load in [float(x) for x in str(args.serve_load).split(",") if x]:
        rate = load * cap_shots / mean_req
        gaps = unit_gaps / rate
        st0 = srv.stats()
        t0 = time.perf_counter()
        t_next = t0
        ids = []
        for (k, s, o), gap in zip(reqs, gaps):
            t_next += gap
            while time.perf_counter() < t_next:
                pass
            ids.append(srv.submit(gids[k], s, T, opts, o))
        infos = [srv.wait(r) for r in ids]
        wall = time.perf_counter() - t0
        st = srv.stats()
        lat = np.array([i["latency_s"] for i in infos]) * 1e3
        shots = sum(o.shape[0] for _, _, o in reqs)
        loads.append({"offered_load": load, "requests": len(reqs), "p50_ms": float(np.percentile(lat, 50)),
                      "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
                      "sustained_shots_per_s": shots / wall, "batches": st["batches"] - st0["batches"],
                      "merged_requests": st["merged_requests"] - st0["merged_requests"]})
    st = srv.stats()
    srv.close()
    # few-shot latency of the heaviest graphs through bp4m_decode_batch from host buffers: one
    # block per shot against the automatic choice, which spreads a class too small to fill the
    # device over thread-block clusters (best of 5 calls)
    few = {}
    for k in sorted(range(len(ds)), key=lambda k: -ds[k])[:3]:
        row = {}
        for n in (1, 8, 64):
            sy = np.ascontiguousarray(pools[k][:n])
            o = np.empty(n, dtype=np.uint8)
            ms = {}
            for name, cl in (("one_block_ms", 1), ("cluster_ms", 0)):
                op = pkg.make_opts(precision="fp32", early_exit=True, stream_cluster=cl)
                graphs[k].decode_batch(sy, T, op, o)
                best = 1e9
                for _ in range(5):
                    t1 = time.perf_counter()
                    graphs[k].decode_batch(sy, T, op, o)
                    best = min(best, time.perf_counter() - t1)
                ms[name] = 1e3 * best
            ms["speedup"] = ms["one_block_ms"] / ms["cluster_ms"]
            row["%d_shots" % n] = ms
        few["d=%d" % ds[k]] = row
    for g in graphs:
        g.close()
    first = loads[0]
    return {"graphs": "rotated memory-Z circuit, d in {%s}, p=%g" % (",".join(map(str, ds)), P),
            "requests": first["requests"], "request_shots": "uniform 1..4096", "iters": T, "slots": args.serve_slots,
            "precision": args.serve_precision, "plain_precision": "fp32",
            "admission": "free device memory (no caller budget)",
            "capacity_shots_per_s": cap_shots, "plain_fp32_per_request_shots_per_s": plain_shots,
            "capacity_vs_plain": cap_shots / plain_shots, "offered_load": first["offered_load"],
            "p50_ms": first["p50_ms"], "p99_ms": first["p99_ms"], "mean_ms": first["mean_ms"],
            "sustained_shots_per_s": first["sustained_shots_per_s"], "loads": loads,
            "max_inflight_batches": st["max_inflight_batches"], "few_shot_latency_fp32": few}


def run_fused(args, dev):
    """Fused decode (Multi) over circuit (p = 0.005) and code-capacity (p = 0.10, X type)
    graphs of d = 5, 9, 13, 17 with uneven shot counts drawn from {1e5, 2.5e5, 5e5, 1e6}
    (seed 7, scaled by --fused-scale), T = 50, against one bp4m_decode_batch call per graph
    in FP32.  Shots/s of each form; outputs must agree with the FP32 plain form on the
    recorded fraction of shots."""
    import numpy as np
    import torch
    import paper_2603_05381_gb300 as pkg

    rng = np.random.default_rng(7)
    specs = [(m, d) for d in (5, 9, 13, 17) for m in ("circuit", "code_capacity")]
    counts = [int(args.fused_scale * rng.choice([100000, 250000, 500000, 1000000])) for _ in specs]
    graphs, synds = [], []
    for (model, d), n in zip(specs, counts):
        g = pkg.Graph(d, model, 0.005 if model == "circuit" else 0.10)
        info = g.info()
        words = sum(info["n_words"])
        sy = torch.empty((n * words,), dtype=torch.int32, device=dev)
        ob = torch.empty((info["n_types"], n), dtype=torch.uint8, device=dev)
        g.sample(sy, ob, first_shot=0, seed=SEED)
        nw = info["n_words"][0]
        synds.append(sy[:n * nw].view(n, nw).cpu().numpy().view(np.uint32).copy())
        graphs.append(g)
        del sy, ob
    torch.cuda.synchronize()
    total = sum(counts)
    out = {"graphs": "rotated circuit p=0.005 and code-capacity p=0.10 (X), d in {5,9,13,17}", "shots": counts,
           "iters": T}
    # plain: one FP32 decode_batch per graph
    opts32 = pkg.make_opts(precision="fp32")
    plain = []
    for g, sy in zip(graphs, synds):   # warm
        g.decode_batch(sy[:1024], T, opts32, np.empty(1024, dtype=np.uint8))
    t0 = time.perf_counter()
    per_graph = []
    for (model, d), g, sy in zip(specs, graphs, synds):
        o = np.empty(sy.shape[0], dtype=np.uint8)
        t1 = time.perf_counter()
        g.decode_batch(sy, T, opts32, o)
        per_graph.append({"graph": "%s d=%d" % (model, d), "shots": int(sy.shape[0]),
                          "ms": 1e3 * (time.perf_counter() - t1)})
        plain.append(o)
    out["plain_fp32_shots_per_s"] = total / (time.perf_counter() - t0)
    out["plain_fp32_per_graph"] = per_graph
    # the largest defect count of the batch sizes the streaming tier (64-column steps)
    max_s = max(int(np.unpackbits(sy.view(np.uint8), axis=1).sum(axis=1).max()) for sy in synds)
    out["max_defects"] = max(161, min(1024, max_s))
    for prec in ("fp32", "fp16", "bf16"):
        m = pkg.Multi(graphs, counts, T, pkg.make_opts(precision=prec), max_defects=out["max_defects"])
        outs = [np.empty(n, dtype=np.uint8) for n in counts]
        m.run(synds, outs)          # autotuner
        m.run(synds, outs)          # capture
        t0 = time.perf_counter()
        m.run(synds, outs)          # replay
        dt = time.perf_counter() - t0
        info = m.info()
        m.close()
        agree = sum(int((o == p).sum()) for o, p in zip(outs, plain)) / total
        out[prec] = {"shots_per_s": total / dt, "vs_plain_fp32": total / dt / out["plain_fp32_shots_per_s"],
                     "outputs_equal_to_fp32_plain": agree, "tier_plan": info["plan"],
                     "plan_ms": info["plan_ms"], "stream_cluster": info["stream_cluster"],
                     "stream_ms": info["stream_ms"]}
    for g in graphs:
        g.close()
    return out


def run_ours(args, rank, world, local):
    import numpy as np
    import torch
    import paper_2603_05381_gb300 as pkg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    mufu = pkg.probe_mufu()
    g = pkg.Graph(D, "circuit", P)
    info = g.info()
    opts = pkg.make_opts(precision=args.precision, early_exit=True, decoder="bp4m", tile_form=args.tile_form)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    shots = args.shots
    from paper_2603_05381_gb300.sharding import shot_range

    def step(k):
        first, _ = shot_range(rank, world, k, shots)
        return g.sample_and_decode(shots, seed=SEED, iters=T, opts=opts, first_shot=first, stream=stream)

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    totals = {"shots": 0, "msg": 0, "fail": 0, "unconv": 0, "iters": 0, "defects": 0, "fc": 0, "fcr": 0}
    ms = 0.0
    barrier()
    clocks.start()
    g.profile_enable(True)
    for k in range(args.steps):
        flush.zero_()  # evict L2 between timed steps (kept outside the timed events)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        c = step(args.warmup + k)
        e1.record(stream)
        e1.synchronize()
        ms += e0.elapsed_time(e1)
        totals["shots"] += c["shots"]
        totals["msg"] += c["msg_updates"]
        totals["fail"] += c["fail"][0]
        totals["unconv"] += c["unconverged"][0]
        totals["iters"] += c["iterations"]
        totals["defects"] += c["defects"]
        totals["fc"] += c["forced_runs"]
        totals["fcr"] += c["forced_rounds"]
    barrier()
    prof = g.profile_read()
    g.profile_enable(False)
    clk = clocks.stop()
    t_max = ms
    if world > 1:
        tt = torch.tensor([ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        t_max = float(tt.item())
        agg = torch.tensor([totals["shots"], totals["msg"]], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(agg)
        all_shots, all_msg = float(agg[0]), float(agg[1])
    else:
        all_shots, all_msg = float(totals["shots"]), float(totals["msg"])
    value = all_shots / (t_max / 1e3)

    # ---- roofline of the dominant kernel (largest share of event-timed decode time)
    kernel_of = dict(KERNEL_OF)
    reg_form = args.precision == "fp32" and args.tile_form == 2
    if reg_form:
        kernel_of.update(KERNEL_OF_REG)
    traffic_of = DRAM_BYTES_PER_SHOT_REG if reg_form else DRAM_BYTES_PER_SHOT
    slots = ["tier%d" % k for k in range(1, 8)] + ["global"]
    dom = max(slots, key=lambda s: prof[s]["ms"])
    dp = prof[dom]
    per_launch_ms = dp["ms"] / max(dp["launches"], 1)
    msgs_per_launch = dp["msg_updates"] / max(dp["launches"], 1)
    sm_mhz = clk["sm_mhz"] or 2070.0
    achieved = msgs_per_launch / (per_launch_ms / 1e3) / 1e9
    msg_per_sm_clk = 1.0 / (1.0 / mufu["ex2"] + 1.0 / mufu["lg2"])
    peak = msg_per_sm_clk * mufu["sms"] * sm_mhz * 1e6 / 1e9
    launches = sum(v["launches"] for v in prof.values())
    decode_ms = sum(prof[s]["ms"] for s in slots)
    decode_msgs = sum(prof[s]["msg_updates"] for s in slots)

    # ---- end to end: decode_batch from pinned host syndromes to host outputs
    nw = info["n_words"][0]
    e2e_shots = shots
    synd_dev = torch.empty((e2e_shots * nw,), dtype=torch.int32, device=dev)
    obs_dev = torch.empty((1, e2e_shots), dtype=torch.uint8, device=dev)
    g.sample(synd_dev, obs_dev, first_shot=shot_range(rank, world, 10**4, shots)[0], seed=SEED, stream=stream)
    synd_host = synd_dev.view(e2e_shots, nw).cpu().pin_memory()
    pred_h = torch.empty((e2e_shots,), dtype=torch.uint8).pin_memory()
    conv_h = torch.empty((e2e_shots,), dtype=torch.uint8).pin_memory()
    its_h = torch.empty((e2e_shots,), dtype=torch.int16).pin_memory()
    g.decode_batch(synd_host, T, opts, pred_h, conv_h, its_h, stream=stream)  # warm
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        g.decode_batch(synd_host, T, opts, pred_h, conv_h, its_h, stream=stream)
    torch.cuda.synchronize()
    e2e_dt = time.perf_counter() - t0
    e2e_val = e2e_steps * e2e_shots / e2e_dt
    if world > 1:
        tt = torch.tensor([e2e_val], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(tt)
        e2e_val = float(tt.item())

    line = {
        "metric": METRIC, "value": value, "unit": "shots/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": {"fp32": "f32", "fp16": "f16 messages, f32 math", "bf16": "bf16 messages, f32 math"}[args.precision], "data": "synthetic (Philox-sampled circuit noise)",
        "config": {"workload": WORKLOAD.replace("FP32 messages", {"fp32": "FP32 messages", "fp16": "FP16 messages (FP32 arithmetic)", "bf16": "BF16 messages (FP32 arithmetic)"}[args.precision]), "d": D, "p": P, "rounds": D, "detectors": info["n_det"][0],
                   "graph_edges": info["n_edges"][0], "shots_per_step": shots, "iters": T,
                   "decoder": "BP4M early exit", "precision": args.precision,
                   "tiles_113_144": "register tiles" if reg_form else "rows",
                   "l2": "256 MB buffer written between timed steps; per-step syndromes (148 MB) exceed L2",
                   "parallelism": "shots sharded across ranks, no collective on the data path"},
        "msg_updates_per_s": all_msg / (t_max / 1e3),
        "mean_defects": totals["defects"] / max(totals["shots"], 1),
        "forced_rounds_per_run": totals["fcr"] / max(totals["fc"], 1),
        "unconverged_fraction": totals["unconv"] / max(totals["shots"], 1),
        "ler": totals["fail"] / max(totals["shots"], 1),
        "mean_iters": totals["iters"] / max(totals["shots"], 1),
        "roofline": {"bound": "alu", "kernel": kernel_of.get(dom, dom), "achieved": achieved,
                     "peak": peak, "unit": "Gmsg/s", "frac": achieved / peak,
                     "traffic": (traffic_of[dom] * dp["shots"] / max(dp["launches"], 1)
                                 if dom in traffic_of and args.precision == "fp32" else None),
                     "traffic_unit": "bytes per launch (ncu DRAM read + write, 65,536-shot capture scaled by shots)",
                     "peak_basis": "MUFU, measured in this run by bp4m_probe_mufu: one ex2 (%.2f/clk/SM) + one "
                                   "lg2 (%.2f/clk/SM) per message update = %.4f SM-cycles; x %d SMs x %.0f MHz "
                                   "(median SM clock in the timed region)"
                                   % (mufu["ex2"], mufu["lg2"], 1.0 / msg_per_sm_clk, mufu["sms"], sm_mhz),
                     "mufu_probe": mufu,
                     "launches": dp["launches"], "ms_per_launch": per_launch_ms,
                     "msg_updates_per_launch": msgs_per_launch,
                     "share_of_decode_time": dp["ms"] / max(decode_ms, 1e-9),
                     "all_decode_tiers": {"achieved": decode_msgs / max(decode_ms, 1e-9) / 1e6,
                                          "frac": decode_msgs / max(decode_ms, 1e-9) / 1e6 / peak}},
        "kernel_ms": {k: round(v["ms"], 3) for k, v in prof.items()},
        "tier_shots": {k: v["shots"] for k, v in prof.items() if v["shots"]},
        "tier_msg_updates": {k: v["msg_updates"] for k, v in prof.items() if v["msg_updates"]},
        "clocks": clk,
        "e2e": {"value": e2e_val, "unit": "shots/s", "h2d_bytes_per_step": e2e_shots * nw * 4,
                "d2h_bytes_per_step": e2e_shots * 4, "path": "bp4m_decode_batch, pinned host syndromes in, "
                                                             "host outputs (obs, converged, iters) out"},
        "gpu_launches": launches,
    }
    if rank == 0 and not args.no_serve:
        if args.serve_d:
            line["serving"] = run_serving(args, dev, args.serve_d)
        if args.serve_d_low:
            line["serving_low_d"] = run_serving(args, dev, args.serve_d_low)
    if rank == 0 and args.fused:
        line["fused"] = run_fused(args, dev)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if world > 1:
        torch.distributed.destroy_process_group()
    return line


def run_reference(args, rank, world):
    """Reference arm: the FP64 oracle on the host cores, same workload, metric and unit."""
    if rank != 0:
        return None
    cores = os.cpu_count() or 1
    n_step = max(8, min(2 * cores, 64))
    for k in range(args.warmup):
        cpu_baseline(n_shots=max(cores, 8), first_shot=k * n_step)
    tot_shots, tot_s = 0, 0.0
    last = None
    for k in range(args.steps):
        r = cpu_baseline(n_shots=n_step, first_shot=(args.warmup + k) * n_step)
        tot_shots += n_step
        tot_s += r["seconds"]
        last = r
    val = tot_shots / tot_s
    return {"impl": "reference", "metric": METRIC, "value": val, "unit": "shots/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (Philox-sampled circuit noise)",
            "config": {"workload": WORKLOAD + " (each step a bounded sample of %d shots)" % n_step, "d": D, "p": P},
            "cpu_baseline": {"kind": "oracle", "cores": cores, "value": val, "unit": "shots/s",
                             "sample": "%d steps x %d shots; %s" % (args.steps, n_step, last["sample"] if last else "")},
            "e2e": {"value": val, "unit": "shots/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_mufu_probe(local):
    """bp4m_probe_mufu repeated for about a second with the SM clocks sampled meanwhile."""
    import torch
    import paper_2603_05381_gb300 as pkg
    torch.cuda.set_device(local)
    pkg.probe_mufu(256)  # load the kernels
    clocks = ClockSampler(local)
    clocks.start()
    t0 = time.perf_counter()
    runs = []
    while time.perf_counter() - t0 < 1.5 or len(runs) < 3:
        runs.append(pkg.probe_mufu(16384))
    clk = clocks.stop()
    med = {k: statistics.median(r[k] for r in runs) for k in ("ex2", "lg2", "ex2_lg2_alternating")}
    upd = 1.0 / (1.0 / med["ex2"] + 1.0 / med["lg2"])
    return {"mufu_per_sm_per_clk": med, "runs": len(runs), "sms": runs[0]["sms"],
            "msg_updates_per_sm_per_clk": upd, "clocks": clk,
            "peak_gmsg_per_s_at_median_clock": (upd * runs[0]["sms"] * clk["sm_mhz"] / 1e3
                                                if clk["sm_mhz"] else None)}


def measured_hbm_gbs():
    """The machine's measured copy bandwidth (MEASURED_PEAKS.json), else the stated fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def run_sweep(args, local):
    """Every point of a sweep through the library, with per-point statistics and the
    dominant tier's roofline fraction (special-function roof measured in this run; HBM
    roof from the measured copy bandwidth)."""
    import torch
    import paper_2603_05381_gb300 as pkg
    from paper_2603_05381_gb300 import sweep as sw
    torch.cuda.set_device(local)
    probe = run_mufu_probe(local)
    hbm, hbm_kind = measured_hbm_gbs()
    sm_mhz = probe["clocks"]["sm_mhz"] or 2070.0
    peak = {"hbm_gbs": hbm, "mufu_gmsg": probe["msg_updates_per_sm_per_clk"] * probe["sms"] * sm_mhz / 1e3}
    ds = tuple(int(x) for x in args.sweep_d.split(",")) if args.sweep_d else None
    ps = tuple(float(x) for x in args.sweep_p.split(",")) if args.sweep_p else None
    pts = sw.config_points(args.sweep, ds, ps)
    print(json.dumps({"sweep": args.sweep, "points": len(pts), "shots_per_point": args.sweep_shots,
                      "peaks": dict(peak, hbm_kind=hbm_kind, sm_mhz=sm_mhz), "mufu_probe": probe}), flush=True)
    clocks = ClockSampler(local)
    clocks.start()
    sw.sweep(pts, args.sweep_shots, state_path=args.sweep_state, seed=SEED, profile=True, peak=peak, log=sys.stdout)
    print(json.dumps({"sweep_done": args.sweep, "clocks": clocks.stop()}), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.mufu_probe:
        print(json.dumps(run_mufu_probe(local)), flush=True)
        return
    if args.sweep:
        if rank == 0:
            run_sweep(args, local)
        return
    if args.impl == "reference":
        line = run_reference(args, rank, world)
    else:
        line = run_ours(args, rank, world, local)
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
