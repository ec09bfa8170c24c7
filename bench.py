#!/usr/bin/env python3
"""Benchmark: IMIN solve time on the 1M-node Chung-Lu workload (k=100, eps=0.1,
delta=1/n, |S|=50 seeds from the top-1% out-degree nodes, weighted-cascade p),
with samples/s, GTEPS and the roofline of the dominant kernel.

A step is one imin_solve through the C ABI: the spread estimate, LSBM (lower
bound sampling + greedy), GSBM (upper bound sampling + greedy), LHGA and the
three final estimates of Algorithm 1.  ``value`` is the device time of one
step with the graph resident in HBM; ``e2e`` times the same call sequence a
user makes from host buffers (graph upload + solve + free).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (single-threaded C) on a bounded sample
of the same workload and projects the solve time from it.  For N > 1 (one
process per GPU under torchrun) every rank runs an independent replica of the
query (its own instance id): the path has no exchange step.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "IMIN solve time at k=100 on the 1M-node Chung-Lu graph"
UNIT = "s"
WORKLOAD = {"workload": "chung-lu-1M", "nodes": 1_000_000, "edge_draws": 10_000_000,
            "degree_exponent": 2.1, "p": "weighted cascade 1/indeg (fp32)", "seeds": 50,
            "seed_pool": "top-1% out-degree", "k": 100, "eps": 0.1, "delta": "1/n",
            "beta": 0.1, "gamma": 0.1, "variant": "SandIMIN (LSBM+GSBM+LHGA)",
            "l2": "flushed (256 MB write) before every timed step"}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks/throttle sampling while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        if not self.proc:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if sm:
            out = {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(smax),
                   "reasons": sorted(reasons), "samples": len(sm)}
        return out


# ---------------------------------------------------------------------------
def cpu_oracle_projection(g, S, cfg, counts, worlds=(1000, 500, 300), seed_tag=11):
    """Time the oracle (as it stands, single-threaded) on a fixed sample of the workload's
    worlds per sampling mode and project the solve time from the solve's own world
    counts: reach-only worlds (spread estimates), CP worlds (LSBM), LRR worlds (GSBM)."""
    import oracle
    og = oracle.OracleGraph.from_graph(g)
    per = {}
    desc = []
    for (name, mode), nw in zip((("reach", 1), ("lower", 2), ("upper", 4)), worlds):
        t0 = time.perf_counter()
        og.sample(S, theta=nw, first=1_000_000, key=7, tag=seed_tag, mode=mode)
        per[name] = (time.perf_counter() - t0) / nw
        desc.append(f"{nw} {name} worlds")
    proj = (per["reach"] * counts["reach_worlds"] + per["lower"] * counts["cp_worlds"] +
            per["upper"] * counts["lrr_worlds"])
    sample = ("oracle (single-threaded C, as committed) timed on " + ", ".join(desc) +
              " of the same graph and seeds; solve time projected as per-world time x the "
              f"solve's world counts (reach {counts['reach_worlds']}, CP {counts['cp_worlds']}, "
              f"LRR {counts['lrr_worlds']}); greedy and host math not included")
    return proj, sample, sum(per.values())


_ORACLE_G = None


def _oracle_init(n, row_ptr, col, prob, S):
    """Pool initializer: each worker process builds its own oracle graph once."""
    global _ORACLE_G
    import oracle
    from paper_2405_12871_gb300 import synth
    g = synth.Graph(n, row_ptr, col, prob)
    _ORACLE_G = (oracle.OracleGraph.from_graph(g), S)


def _oracle_task(job):
    mode, first, theta, tag = job
    og, S = _ORACLE_G
    og.sample(S, theta=theta, first=first, key=7, tag=tag, mode=mode)
    return theta


class OraclePool:
    """The same oracle, unchanged, with its world loop split over every host core: each
    worker process holds its own copy of the graph and samples its own world range
    (worlds are index-addressed, so the ranges are independent)."""

    def __init__(self, g, S, procs=None):
        import multiprocessing as mp
        self.procs = procs or os.cpu_count() or 1
        ctxp = mp.get_context("spawn")        # never fork a process that holds a CUDA context
        self.pool = ctxp.Pool(self.procs, initializer=_oracle_init,
                              initargs=(g.n, g.row_ptr, g.col, g.prob, np.asarray(S, np.int32)))
        self.pool.map(_oracle_task, [(1, 5_000_000 + 2 * i, 2, 3) for i in range(self.procs)])   # warm

    def rates(self, worlds, seed_tag, first=2_000_000):
        """worlds per mode (reach, lower, upper), split evenly over the processes;
        returns wall-clock worlds per second per mode."""
        rates = {}
        for (name, mode), total in zip((("reach", 1), ("lower", 2), ("upper", 4)), worlds):
            per = max(1, -(-int(total) // self.procs))
            jobs = [(mode, first + i * per, per, seed_tag) for i in range(self.procs)]
            t0 = time.perf_counter()
            done = sum(self.pool.map(_oracle_task, jobs))
            rates[name] = done / (time.perf_counter() - t0)
        return rates

    def close(self):
        self.pool.close()
        self.pool.join()


def project(counts, rates):
    return (counts["reach_worlds"] / rates["reach"] + counts["cp_worlds"] / rates["lower"] +
            counts["lrr_worlds"] / rates["upper"])


def cpu_oracle_parallel(g, S, counts, worlds=(10_000, 10_000, 10_000), seed_tag=12):
    pool = OraclePool(g, S)
    try:
        rates = pool.rates(worlds, seed_tag)
    finally:
        pool.close()
    sample = (f"the oracle's world loop split over {pool.procs} processes, each on its own world range: "
              f"{worlds[0]} reach, {worlds[1]} lower and {worlds[2]} upper worlds in all, wall-clock rates "
              "per mode; solve time projected from the solve's world counts; greedy and host math not "
              "included")
    return project(counts, rates), sample, pool.procs


def solve_counts(r):
    return {"reach_worlds": int(r["n_spread"] + sum(r["n_final"])),
            "cp_worlds": int(r["theta_C1"] + r["theta_C2"]),
            "lrr_worlds": int(r["theta_L1"] + r["theta_L2"])}


# ---------------------------------------------------------------------------
def run_reference(args, rank, world):
    if rank != 0:
        return 0
    from paper_2405_12871_gb300 import synth
    g, S, cfg = synth.workload_cl1m()
    # the solve's world counts are not known without running it: the reference arm uses
    # the counts the GPU arm measured (committed in profiles/) when present
    counts = {"reach_worlds": 900_000, "cp_worlds": 12_000, "lrr_worlds": 200_000}
    pth = os.path.join(ROOT, "profiles", "solve_counts_cl1m.json")
    if os.path.exists(pth):
        counts = json.load(open(pth))
    pool = OraclePool(g, S)
    per_step = (1600, 800, 640)
    vals = []
    try:
        for step in range(args.warmup + args.steps):
            v = project(counts, pool.rates(per_step, seed_tag=20 + step, first=3_000_000 + step * 10_000))
            if step >= args.warmup:
                vals.append(v)
    finally:
        pool.close()
    v = float(np.mean(vals))
    sample = (f"oracle (C, as committed) with its world loop split over {pool.procs} host processes; each "
              f"step times {per_step[0]} reach, {per_step[1]} lower and {per_step[2]} upper worlds of the "
              f"CL-1M workload and projects the solve time from the solve's world counts "
              f"(reach {counts['reach_worlds']}, CP {counts['cp_worlds']}, LRR {counts['lrr_worlds']}); "
              "greedy and host math not included")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "config": dict(WORKLOAD, parallelism=f"replicas x{world}"),
            "projected": True,
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": pool.procs, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
def run_batch(args):
    """Batched vs plain on the same instances (identical results are checked)."""
    import torch
    from paper_2405_12871_gb300 import _lib, synth
    t0 = time.time()
    items = synth.workload_batch(args.batch)
    gen_s = time.time() - t0
    ctx = _lib.Context(0, stream=torch.cuda.current_stream().cuda_stream)
    Gs = [ctx.load_graph(g) for g, _, _ in items]
    qs = [(G, S, c["k"], c["eps"], c["delta"], dict(key=c["key"], inst=c["inst"]))
          for G, (g, S, c) in zip(Gs, items)]
    # warm-up: every graph's launch shape is tuned before either path is timed (the
    # autotuner otherwise runs inside the first solve that reaches a graph), and a
    # small instance loads the kernels and sizes the slot arenas
    for (G, S, k, eps, delta, kw) in qs:
        G.autotune(S)
    small = min(range(len(items)), key=lambda i: items[i][0].n)
    G, S, k, eps, delta, kw = qs[small]
    G.solve(S, k, eps, delta, **kw)
    torch.cuda.synchronize()
    a = time.perf_counter()
    plain = [] if args.batch_only else [G.solve(S, k, eps, delta, **kw) for (G, S, k, eps, delta, kw) in qs]
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - a
    a = time.perf_counter()
    batched = ctx.solve_batch(qs)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - a
    if args.batch_only:
        print(json.dumps({"mode": "batch-only", "instances": len(items), "batched_s": t_batch,
                          "batched_kernel_launches": int(batched[0]["kernel_launches"]),
                          "batched_stage_ms": [round(x, 1) for x in batched[0]["ms_stage"]]}), flush=True)
        return 0
    diff = [i for i, (x, y) in enumerate(zip(plain, batched))
            if not (list(x["blockers"]) == list(y["blockers"]) and x["I_after"] == y["I_after"])]
    same = not diff
    for i in diff[:8]:
        print(json.dumps({"batch_mismatch": i, "n": items[i][0].n, "plain_I_after": plain[i]["I_after"],
                          "batched_I_after": batched[i]["I_after"]}), file=sys.stderr, flush=True)
    line = {"mode": "batch", "instances": len(items), "plain_s": t_plain, "batched_s": t_batch,
            "speedup": t_plain / t_batch, "plain_inst_per_s": len(items) / t_plain,
            "batched_inst_per_s": len(items) / t_batch, "identical_results": same,
            "total_nodes": int(sum(g.n for g, _, _ in items)),
            "total_edges": int(sum(g.m for g, _, _ in items)),
            "batched_kernel_launches": int(batched[0]["kernel_launches"]),
            "batched_stage_ms": [round(x, 1) for x in batched[0]["ms_stage"]],
            "batched_kernel_ms": [round(x, 1) for x in batched[0]["kernel_ms"]],
            "plain_stage_ms_sum": [round(sum(x["ms_stage"][i] for x in plain), 1) for i in range(8)],
            "plain_kernel_launches": int(sum(x["kernel_launches"] for x in plain)),
            "config": {"workload": "batch of Chung-Lu instances", "n": "log-uniform 1e3..1e6",
                       "avg_degree": 10, "exponent": 2.1, "seeds": "U{5..100} from top-1% out-degree",
                       "k": "U{10..200}", "eps": 0.2, "delta": "1/n"}, "graph_gen_s": gen_s}
    print(json.dumps(line), flush=True)
    for G in Gs:
        G.free()
    ctx.close()
    return 0 if same else 1


def run_baselines(args):
    """SandIMIN against the dominator-tree baselines AG and GR on the CL-1M query: solve
    time, blockers, and the spread left by each blocker set, re-estimated on the same
    independent worlds (stream tag 9, which no solve uses)."""
    import torch
    from paper_2405_12871_gb300 import _lib, baselines, synth
    g, S, cfg = synth.workload_cl1m()
    ctx = _lib.Context(0, stream=torch.cuda.current_stream().cuda_stream)
    G = ctx.load_graph(g)
    kw = dict(k=cfg["k"], eps=cfg["eps"], delta=cfg["delta"], key=cfg["key"])
    G.solve(S, **kw)                              # warm-up (autotuner, arenas)
    torch.cuda.synchronize()
    out = {"mode": "baselines", "workload": "chung-lu-1M", "k": cfg["k"], "theta_per_estimate": args.baseline_theta,
           "eval_worlds": args.baseline_eval}
    t = time.perf_counter()
    r = G.solve(S, **kw)
    torch.cuda.synchronize()
    sets = {"sandimin": ([int(x) for x in r["blockers"]], time.perf_counter() - t, None)}
    for name, fn in (("ag", lambda: baselines.advanced_greedy(G.sample, g.n, S, cfg["k"], args.baseline_theta)),
                     ("gr", lambda: baselines.greedy_replace(G.sample, g, S, cfg["k"], args.baseline_theta))):
        t = time.perf_counter()
        B, calls, worlds = fn()
        torch.cuda.synchronize()
        sets[name] = (B, time.perf_counter() - t, {"estimates": calls, "worlds": worlds})
    for name, (B, sec, extra) in sets.items():
        ev = G.sample(S, B, theta=args.baseline_eval, key=1, tag=9, mode=0, per_world=True)
        ws = ev["world_spread"].astype(np.float64)
        out[name] = {"seconds": sec, "blockers": len(B), "spread": float(ws.mean()),
                     "spread_stderr": float(ws.std(ddof=1) / np.sqrt(len(ws)))}
        if extra:
            out[name].update(extra)
    ev0 = G.sample(S, (), theta=args.baseline_eval, key=1, tag=9, mode=0)
    out["spread_without_blockers"] = ev0["total_spread"] / args.baseline_eval
    print(json.dumps(out), flush=True)
    G.free()
    ctx.close()
    return 0


def run_sweep(args):
    """Effectiveness sweeps on the CL-1M stand-in (analogues of the paper's eps, |S| and
    k sweeps): for each setting, solve time, the estimated spread before and after each
    candidate's blockers, the chosen candidate and the approximation-ratio lower bound."""
    import torch
    from paper_2405_12871_gb300 import _lib, synth
    g, S50, cfg = synth.workload_cl1m()
    ctx = _lib.Context(0, stream=torch.cuda.current_stream().cuda_stream)
    G = ctx.load_graph(g)
    G.solve(S50, k=cfg["k"], eps=cfg["eps"], delta=cfg["delta"])     # warm-up
    settings = [("eps", e, 50, 100) for e in (0.1, 0.2, 0.3)]
    settings += [("k", e, 50, k) for e, k in ((0.1, 25), (0.1, 50), (0.1, 200))]
    settings += [("seeds", 0.1, s, 100) for s in (10, 100)]
    rows = []
    for what, eps, ns, k in settings:
        S = S50 if ns == 50 else synth.seeds_top_outdeg(g, ns, 0.01, seed=2)
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = G.solve(S, k=k, eps=eps, delta=cfg["delta"])
        torch.cuda.synchronize()
        rows.append({"sweep": what, "eps": eps, "seeds": ns, "k": k, "seconds": time.perf_counter() - t,
                     "I_hat": r["I_hat"], "I_after": list(r["I_after"]), "chosen": "LUR"[r["chosen"]],
                     "ratio_lb": r["ratio_lb"], "worlds": int(r["worlds_sampled"])})
    print(json.dumps({"mode": "sweep", "workload": "chung-lu-1M", "delta": "1/n", "rows": rows}), flush=True)
    G.free()
    ctx.close()
    return 0


def run_serve(args):
    """Poisson stream through the server; the same stream replayed one query at a time
    (first come, first served) gives the plain latency and throughput."""
    import torch
    from paper_2405_12871_gb300 import _lib, synth
    rng = np.random.Generator(np.random.Philox(77))
    sizes = (100_000, 300_000, 1_000_000)
    graphs = [synth.chung_lu_poisson(n, 10.0, 2.1, seed=21 + i) for i, n in enumerate(sizes)]
    ctx = _lib.Context(0, stream=torch.cuda.current_stream().cuda_stream)
    Gs = [ctx.load_graph(g) for g in graphs]
    nq = int(rng.poisson(args.serve_rate * args.serve_seconds))
    arrivals = np.sort(rng.uniform(0.0, args.serve_seconds, size=nq))
    if args.serve_burst:            # every query arrives at once: throughput at saturation
        arrivals = np.zeros(nq)
    qs = []
    for i in range(nq):
        gi = int(rng.integers(0, len(graphs)))
        g = graphs[gi]
        nS = int(rng.integers(10, 201))
        S = np.sort(rng.choice(g.n, nS, replace=False)).astype(np.int32)
        k = int(min(rng.integers(10, 501), g.n - nS - 1))
        qs.append((Gs[gi], S, k, 0.2, 1.0 / g.n, dict(key=i, inst=i)))
    # warm-up: the three graphs' launch shapes are tuned before either path is timed
    for G in Gs:
        seeds = next((q[1] for q in qs if q[0] is G), np.arange(10, dtype=np.int32))
        G.autotune(seeds)
    G, S, k, eps, delta, kw = qs[0]
    G.solve(S, k, eps, delta, **kw)
    srv = _lib.Server(ctx, max_active=args.serve_active)
    t0 = time.perf_counter()
    tickets = []
    for (G, S, k, eps, delta, kw), at in zip(qs, arrivals):
        now = time.perf_counter() - t0
        if at > now:
            time.sleep(at - now)
        tickets.append(srv.submit(G, S, k, eps, delta, **kw))
    served = [srv.poll(t, wait_ms=-1) for t in tickets]
    t_served = time.perf_counter() - t0
    srv.stop()
    lat_s = np.array([r["latency_ms"] for r in served]) / 1e3
    # plain replay
    service = []
    plain = []
    for (G, S, k, eps, delta, kw) in qs:
        a = time.perf_counter()
        plain.append(G.solve(S, k, eps, delta, **kw))
        service.append(time.perf_counter() - a)
    free_at, lat_p = 0.0, []
    for at, sv in zip(arrivals, service):
        start = max(at, free_at)
        free_at = start + sv
        lat_p.append(free_at - at)
    lat_p = np.array(lat_p)
    same = all(list(x["blockers"]) == list(y["blockers"]) for x, y in zip(plain, served))
    line = {"mode": "serve", "queries": nq, "rate_per_s": args.serve_rate, "burst": bool(args.serve_burst),
            "duration_s": args.serve_seconds, "served_qps": nq / t_served,
            "served_p50_s": float(np.percentile(lat_s, 50)), "served_p99_s": float(np.percentile(lat_s, 99)),
            "plain_qps": nq / float(np.sum(service)), "plain_p50_s": float(np.percentile(lat_p, 50)),
            "plain_p99_s": float(np.percentile(lat_p, 99)), "identical_results": same,
            "config": {"graphs": "Chung-Lu (Poisson model) 1e5 / 3e5 / 1e6 nodes, degree 10, WC p",
                       "arrivals": "Poisson", "seeds": "U{10..200} uniform nodes", "k": "U{10..500}",
                       "eps": 0.2, "delta": "1/n", "max_active": args.serve_active}}
    print(json.dumps(line), flush=True)
    for G in Gs:
        G.free()
    ctx.close()
    return 0 if same else 1


# ---------------------------------------------------------------------------
def run_rmat(args):
    """The R-MAT-4M configuration (4,194,304 nodes, 2^26 edge draws, trivalency p,
    |S| = 100 uniform seeds, k = 200, eps = 0.1, delta = 1/n): reach-only sampling
    throughput with its roofline (a world reaches about half a million nodes, so the
    graph and the visited maps do not fit in L2), then timed solves."""
    import torch
    from paper_2405_12871_gb300 import _lib, synth
    t0 = time.time()
    g, S, cfg = synth.workload_rmat4m()
    gen_s = time.time() - t0
    stream = torch.cuda.current_stream()
    ctx = _lib.Context(0, stream=stream.cuda_stream)
    G = ctx.load_graph(g)
    pk = peaks()
    peak = float(pk.get("hbm_gbs", 6800.0))
    out = {"mode": "rmat", "config": {"workload": "rmat-4M", "nodes": g.n, "edges": g.m, "a_b_c": [0.57, 0.19, 0.19],
                                      "p": "uniform from {0.1, 0.01, 0.001}", "seeds": 100, "k": cfg["k"],
                                      "eps": cfg["eps"], "delta": "1/n"}, "graph_gen_s": round(gen_s, 1)}
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    theta = args.rmat_worlds
    G.sample(S, theta=64, key=0, tag=0, first=10_000_000, mode=0)
    ev0.record(stream)
    r = G.sample(S, theta=theta, key=0, tag=0, first=0, mode=0)
    ev1.record(stream)
    torch.cuda.synchronize()
    dt = ev0.elapsed_time(ev1) / 1e3
    alg = 16.0 * r["total_spread"] + 8.0 * r["edges_scanned"]
    out["reach_sampling"] = {"worlds": theta, "s": dt, "samples_per_s": theta / dt,
                             "gteps": r["edges_scanned"] / dt / 1e9, "nodes_per_world": r["total_spread"] / theta,
                             "edges_per_world": r["edges_scanned"] / theta,
                             "roofline": {"bound": "hbm", "achieved": alg / dt / 1e9, "peak": peak, "unit": "GB/s",
                                          "frac": alg / dt / 1e9 / peak, "kernel": "cta_world_kernel<reach-only>",
                                          "launch_shape": G.tuning(),
                                          "algorithmic_bytes": "16 B per reached node + 8 B per scanned edge"}}
    print(json.dumps(out), flush=True)
    if args.rmat_solves:
        kw = dict(k=cfg["k"], eps=cfg["eps"], delta=cfg["delta"], key=cfg["key"])
        sol = []
        for i in range(args.rmat_solves):
            torch.cuda.synchronize()
            ev0.record(stream)
            rs = G.solve(S, **kw)
            ev1.record(stream)
            torch.cuda.synchronize()
            sol.append({"s": ev0.elapsed_time(ev1) / 1e3, "stage_ms": [round(x, 1) for x in rs["ms_stage"]],
                        "kernel_ms": [round(x, 1) for x in rs["kernel_ms"]],
                        "final_kernel_ms": round(rs["final_kernel_ms"], 1), "worlds": int(rs["worlds_sampled"]),
                        "edges": int(rs["edges_scanned"]), "I_hat": rs["I_hat"], "I_after": rs["I_after"],
                        "chosen": rs["chosen"], "counts": solve_counts(rs)})
        out["solves"] = sol
        print(json.dumps(out), flush=True)
    G.free()
    ctx.close()
    return 0


# ---------------------------------------------------------------------------
def run_final_only(args):
    """Profiling case for the fused final-estimate kernel: the final estimates
    (Algorithm 1, line 4) of three blocker sets on the CL-1M workload through
    imin_final_estimates alone, so that the process holds only the graph and the fused
    kernel's slots.  The sets: the top 100 of the seeds' out-neighbours by
    q(v) * outdeg(v) (LHGA's rule), by q(v), and the 100 largest out-degrees."""
    import torch
    from paper_2405_12871_gb300 import _lib, synth
    g, S, cfg = synth.workload_cl1m()
    ctx = _lib.Context(0, stream=torch.cuda.current_stream().cuda_stream)
    G = ctx.load_graph(g)
    Sset = set(int(s) for s in S)
    pq = np.ceil(g.prob.astype(np.float64) * 16777216.0) / 16777216.0
    prod = {}
    for s in S:
        for e in range(int(g.row_ptr[s]), int(g.row_ptr[s + 1])):
            v = int(g.col[e])
            if pq[e] > 0 and v not in Sset:
                prod[v] = prod.get(v, 1.0) * (1.0 - pq[e])
    outdeg = np.diff(g.row_ptr)
    on = sorted(prod)
    by_score = sorted(on, key=lambda v: (-(1.0 - prod[v]) * outdeg[v], v))[:cfg["k"]]
    by_q = sorted(on, key=lambda v: (-(1.0 - prod[v]), v))[:cfg["k"]]
    order = np.lexsort((np.arange(g.n), -outdeg))
    by_deg = [int(v) for v in order if int(v) not in Sset][:cfg["k"]]
    cands = [sorted(by_score), sorted(by_q), sorted(by_deg)]
    for it in range(2):
        torch.cuda.synchronize()
        a = time.perf_counter()
        I, N = G.final_estimates(S, cands, gamma=0.1, delta=cfg["delta"], key=cfg["key"], spread_hint=18314.0)
        torch.cuda.synchronize()
        print(json.dumps({"mode": "final-only", "s": time.perf_counter() - a, "I_after": I, "n_worlds": N}),
              flush=True)
    G.free()
    ctx.close()
    return 0


# ---------------------------------------------------------------------------
def run_useq(args):
    """The LRR-sequence estimator of D^U (Sec. 4.2, Discussion; every reached node's
    LRR set per world) against Global Sampling (Algorithm 3; one LRR set per world) on
    the CL-1M query, for the blocker set B_U of a solve: time per world and per-world
    variance of each estimate of D^U(B_U), and the time each needs for the same
    standard error.  GS's per-world estimate is |V'_s| times a Bernoulli(D^U/|V'_s|)
    indicator, so its variance is D^U (|V'_s| - D^U); D^U is taken from the sequence
    estimate, which is far tighter."""
    import torch
    from paper_2405_12871_gb300 import _lib, synth
    g, S, cfg = synth.workload_cl1m()
    ctx = _lib.Context(0, stream=torch.cuda.current_stream().cuda_stream)
    G = ctx.load_graph(g)
    kw = dict(k=cfg["k"], eps=cfg["eps"], delta=cfg["delta"], key=cfg["key"])
    G.solve(S, **kw)
    r = G.solve(S, **kw)
    BU = [int(x) for x in r["B_U"]]
    theta = args.useq_worlds
    G.lrr_sequences(S, query=BU, theta=64, key=1, tag=11, first=10_000_000)
    torch.cuda.synchronize()
    a = time.perf_counter()
    q = G.lrr_sequences(S, query=BU, theta=theta, key=1, tag=11)
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - a
    cw = q["cov_world"].astype(np.float64)
    du = float(cw.mean())
    var_seq = float(cw.var(ddof=1))
    nvs = int(r["nVs"])
    var_gs = du * (nvs - du)
    gs_worlds = int(r["theta_L1"] + r["theta_L2"])
    t_gs = r["kernel_ms"][2] / 1e3 / max(gs_worlds, 1)
    out = {"mode": "lrr-sequences", "workload": "chung-lu-1M", "query": "B_U of the solve (k = 100)",
           "worlds": theta, "seq_s_per_world": t_seq / theta, "seq_elements_per_world": q["elements"] / theta,
           "seq_nodes_per_world": q["total_spread"] / theta, "DU_seq": du, "DU_seq_rel_stderr":
           float(np.sqrt(var_seq / theta) / du), "DU_gs_solve": r["DU_hat"], "nVs": nvs,
           "var_per_world_seq": var_seq, "var_per_world_gs": var_gs,
           "gs_s_per_world": t_gs, "gs_worlds_in_solve": gs_worlds,
           "time_for_equal_stderr_gs_over_seq": (var_gs * t_gs) / (var_seq * (t_seq / theta))}
    print(json.dumps(out), flush=True)
    G.free()
    ctx.close()
    return 0


# ---------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-mc-check", action="store_true")
    ap.add_argument("--batch-only", action="store_true", help="time the batched path alone (no plain replay)")
    ap.add_argument("--batch", type=int, default=0,
                    help="batched vs plain: the first N instances of the 512-instance Chung-Lu "
                         "batch recipe, solved one by one and as one imin_solve_batch")
    ap.add_argument("--serve", action="store_true",
                    help="serving: Poisson query stream over resident graphs through the "
                         "continuous-batching server vs a plain one-at-a-time replay")
    ap.add_argument("--serve-rate", type=float, default=4.0)
    ap.add_argument("--serve-seconds", type=float, default=15.0)
    ap.add_argument("--serve-active", type=int, default=32)
    ap.add_argument("--serve-burst", action="store_true",
                    help="all queries of the stream arrive at time 0 (throughput at saturation)")
    ap.add_argument("--sweep", action="store_true",
                    help="eps / |S| / k sweeps of the solve on the CL-1M stand-in")
    ap.add_argument("--baselines", action="store_true",
                    help="SandIMIN vs the AG and GR baselines on the CL-1M query")
    ap.add_argument("--baseline-theta", type=int, default=10_000,
                    help="worlds per AG / GR estimate")
    ap.add_argument("--baseline-eval", type=int, default=100_000,
                    help="worlds of the final spread re-estimate")
    ap.add_argument("--useq", action="store_true",
                    help="the LRR-sequence estimator against Global Sampling on the CL-1M query")
    ap.add_argument("--useq-worlds", type=int, default=2000)
    ap.add_argument("--final-only", action="store_true",
                    help="profiling case: the fused final estimates of three blocker sets on CL-1M alone")
    ap.add_argument("--rmat", action="store_true",
                    help="the R-MAT-4M configuration: reach-only sampling roofline and timed solves")
    ap.add_argument("--rmat-worlds", type=int, default=2000)
    ap.add_argument("--rmat-solves", type=int, default=1)
    ap.add_argument("--reach-only-worlds", type=int, default=0,
                    help="profiling case: run two imin_sample launches of this many reach-only "
                         "worlds on the same workload (the stopping rule's kernel) and exit")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus)))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.batch:
        return run_batch(args)
    if args.serve:
        return run_serve(args)
    if args.baselines:
        return run_baselines(args)
    if args.sweep:
        return run_sweep(args)
    if args.rmat:
        return run_rmat(args)
    if args.final_only:
        return run_final_only(args)
    if args.useq:
        return run_useq(args)

    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    from paper_2405_12871_gb300 import _lib, synth

    t0 = time.time()
    g, S, cfg = synth.workload_cl1m()
    gen_s = time.time() - t0
    stream = torch.cuda.current_stream()
    ctx = _lib.Context(local, stream=stream.cuda_stream)
    G = ctx.load_graph(g)
    if args.reach_only_worlds:
        th = args.reach_only_worlds
        for it in range(2):
            torch.cuda.synchronize()
            a = time.perf_counter()
            r = G.sample(S, theta=th, key=0, tag=0, first=it * th, mode=0)
            torch.cuda.synchronize()
            dt = time.perf_counter() - a
            print(json.dumps({"reach_only_worlds": th, "s": dt, "nodes": r["total_spread"],
                              "edges": r["edges_scanned"], "gteps": r["edges_scanned"] / dt / 1e9}))
        G.free()
        ctx.close()
        return 0
    inst = rank                                   # independent replica per rank
    kw = dict(k=cfg["k"], eps=cfg["eps"], delta=cfg["delta"], key=cfg["key"], inst=inst)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        r = G.solve(S, **kw)
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    times, results = [], []
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        ev0.record(stream)
        r = G.solve(S, **kw)
        ev1.record(stream)
        torch.cuda.synchronize()
        times.append(ev0.elapsed_time(ev1) / 1e3)
        results.append(r)
    barrier()
    clk = clocks.stop()
    shape = G.tuning()          # the autotuner's launch shape for reach-only worlds
    step_s = float(np.mean(times))
    if world > 1:
        t = torch.tensor([step_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        step_s = float(t.item())

    # ---- independent Monte Carlo re-estimate of the chosen blockers' spread ----
    mc = None
    if rank == 0 and not args.no_mc_check:
        torch.cuda.synchronize()
        a = time.perf_counter()
        ev = G.sample(S, results[-1]["blockers"], theta=1_000_000, key=1, tag=9, mode=0, per_world=True)
        torch.cuda.synchronize()
        ws = ev["world_spread"].astype(np.float64)
        m = float(ws.mean())
        est = float(results[-1]["I_after"][results[-1]["chosen"]])
        mc = {"worlds": 1_000_000, "stream": "key 1, tag 9 (no solve draws it)", "estimate": est, "mc_mean": m,
              "rel_diff": abs(est - m) / m, "mc_rel_stderr": float(ws.std(ddof=1) / np.sqrt(len(ws)) / m),
              "tolerance": 0.01, "within_tolerance": abs(est - m) / m <= 0.01,
              "seconds": time.perf_counter() - a}

    # ---- end to end: upload the graph from host buffers, solve, read back, free ----
    e2e = None
    if not args.no_e2e:
        G.free()
        # the inputs sit in page-locked host buffers, as a serving process keeps them;
        # filling those buffers is outside the timed region (pageable memory if pinning
        # is not available)
        host, pinned, keep = g, False, []
        try:
            keep = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (g.row_ptr, g.col, g.prob)]
            host = synth.Graph(g.n, keep[0].numpy(), keep[1].numpy(), keep[2].numpy(), g.name)
            pinned = True
        except Exception:
            host = g
        e2e_t = []
        for i in range(max(1, min(args.steps, 2)) + 1):
            flush.zero_()
            torch.cuda.synchronize()
            a = time.perf_counter()
            G2 = ctx.load_graph(host)
            r2 = G2.solve(S, **kw)
            G2.free()
            torch.cuda.synchronize()
            if i > 0:
                e2e_t.append(time.perf_counter() - a)
        h2d = int(g.row_ptr.nbytes + g.col.nbytes + g.prob.nbytes + S.nbytes)
        d2h = int(4 * 4 * cfg["k"] + 512)
        e2e = {"value": float(np.mean(e2e_t)), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h,
               "what": "imin_load_graph from host CSR + imin_solve + imin_free_graph",
               "host_buffers": ("pinned caller buffers; prob is copied to the device from them, row_ptr "
                                "and col through the library's own host copies (kept for the host controller)")
               if pinned else "pageable"}
        assert list(r2["blockers"]) == list(results[-1]["blockers"])

    # ---- throughput and roofline of the two stopping-rule kernels ----
    rr = results[-1]
    worlds = np.mean([x["worlds_sampled"] for x in results])
    edges = np.mean([x["edges_scanned"] for x in results])
    pk = peaks()
    peak = float(pk.get("hbm_gbs", 6800.0))
    peak_src = ("MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in pk else "fallback 6.8 TB/s")

    def roofline(kms, nodes, redges, launches, kernel, shape, traffic_file):
        alg_bytes = 16.0 * nodes + 8.0 * redges
        achieved = alg_bytes / kms / 1e9 if kms > 0 else 0.0
        # DRAM traffic per launch: bytes per algorithmic byte from one ncu capture of the
        # same kernel and launch shape on a smaller case, times this launch's algorithmic
        # bytes (traffic grows with the nodes and edges a launch processes)
        traffic = None
        tp = os.path.join(ROOT, "profiles", traffic_file)
        if os.path.exists(tp):
            try:
                tj = json.load(open(tp))
                if tj.get("shape") == shape:
                    traffic = tj["dram_bytes_per_alg_byte"] * alg_bytes / max(launches, 1)
            except Exception:
                traffic = None
        return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": kernel, "launch_shape": shape,
                "per_launch_ms": kms * 1e3 / max(launches, 1), "launches_per_solve": launches,
                "algorithmic_bytes": "16 B per queue entry (row_ptr pair, queue write + read, visited "
                                     "word) + 8 B per scanned edge",
                "peak_source": peak_src}

    f_kms = np.mean([x["final_kernel_ms"] for x in results]) / 1e3
    f_nodes = np.mean([x["final_entries"] for x in results])
    f_edges = np.mean([x["final_edges"] for x in results])
    f_launch = np.mean([x["final_launches"] for x in results])
    r_kms = np.mean([x["kernel_ms"][0] for x in results]) / 1e3 - f_kms
    r_nodes = np.mean([x["reach_nodes"] for x in results]) - f_nodes
    r_edges = np.mean([x["reach_edges"] for x in results]) - f_edges
    r_launch = np.mean([x["reach_launches"] for x in results]) - f_launch
    fshape = {"threads": 512 if shape.get("threads", 256) >= 512 else 256,
              "ctas_per_sm": 4 if shape.get("threads", 256) >= 512 else 8, "map": "4-bit candidate field per node"}
    roof_final = roofline(f_kms, f_nodes, f_edges, f_launch,
                          "cta_final_kernel (the three final estimates in one traversal per world)", fshape,
                          "final_kernel_traffic.json")
    roof_reach = roofline(r_kms, r_nodes, r_edges, r_launch,
                          "cta_world_kernel<reach-only, stopping rule> (the spread estimate I_hat)", shape,
                          "reach_kernel_traffic.json")
    # the roofline reported is that of the kernel with the larger device time
    roof, roof_other = (roof_final, roof_reach) if f_kms >= r_kms else (roof_reach, roof_final)

    # ---- the parity configuration: one full GPU solve next to one full oracle solve ----
    er = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        ge, Se, ce = synth.workload_er1k()
        Ge = ctx.load_graph(ge)
        kwe = dict(k=ce["k"], eps=0.2, delta=1.0 / ge.n, key=ce["key"])
        Ge.solve(Se, **kwe)
        torch.cuda.synchronize()
        a = time.perf_counter()
        re_ = Ge.solve(Se, **kwe)
        torch.cuda.synchronize()
        t_gpu = time.perf_counter() - a
        Ge.free()
        a = time.perf_counter()
        ro = oracle.OracleGraph.from_graph(ge).solve(Se, **kwe)
        t_or = time.perf_counter() - a
        er = {"workload": "erdos-renyi-1K (1,000 nodes, 5,000 edges, |S| = 10, k = 5, eps = 0.2, delta = 1/n)",
              "gpu_s": t_gpu, "oracle_s": t_or, "oracle_cores": 1, "projected": False,
              "identical": list(re_["blockers"]) == list(ro["blockers"]) and re_["I_after"] == ro["I_after"],
              "worlds": int(re_["n_spread"] + sum(re_["n_final"]) + re_["theta_C1"] + re_["theta_C2"] +
                            re_["theta_L1"] + re_["theta_L2"])}

    line = {"metric": METRIC, "value": step_s, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": dict(WORKLOAD, parallelism=f"replicas x{world}"),
            "samples_per_s": worlds / step_s, "gteps": edges / step_s / 1e9,
            "solves_per_s": world / step_s,
            "stage_ms": [round(x, 2) for x in rr["ms_stage"]],
            "kernel_ms": [round(x, 2) for x in rr["kernel_ms"]],
            "final_kernel_ms": round(rr["final_kernel_ms"], 2),
            "counts": solve_counts(rr), "I_hat": rr["I_hat"], "I_after": rr["I_after"],
            "chosen": rr["chosen"], "gpu_launches": int(np.mean([x["kernel_launches"] for x in results])),
            "roofline": roof, "roofline_other": roof_other, "clocks": clk, "graph_gen_s": round(gen_s, 1)}
    if e2e:
        line["e2e"] = e2e
    if mc:
        line["mc_check"] = mc
    if er:
        line["er1k_full_solve"] = er
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        proj, sample, _ = cpu_oracle_projection(g, S, cfg, solve_counts(rr))
        line["cpu_baseline"] = {"value": proj, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": sample}
        try:
            pproj, psample, pcores = cpu_oracle_parallel(g, S, solve_counts(rr))
            line["cpu_baseline_parallel"] = {"value": pproj, "unit": UNIT, "cores": pcores,
                                             "kind": "oracle", "sample": psample}
        except Exception as exc:          # the one-core line stands on its own
            line["cpu_baseline_parallel"] = {"unavailable": f"{type(exc).__name__}: {exc}"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if G.h:
        G.free()
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
