"""Benchmark of the refinement hot path: edges refined per second.

One step = one upr_refine call (all rounds of the workload: gain table,
selection, rebalancing, interleaving, exact gains, best prefix) on the R-MAT
scale-22 workload (4,194,304 nodes, 128.3M adjacency entries after
symmetrisation and deduplication, unit weights, k = 64, eps = 0.03, seeded
random balanced initial partition, 8 rounds).  value = rounds * |E| / step
time, with the graph and the initial partition resident in HBM; e2e = the
same metric through the C ABI from pinned host buffers (graph upload and
checks, refinement, partition read-back) per step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]

N > 1 runs under torch.distributed.run: every rank refines its own replica
(the single-graph path does not shard), scaling "weak".  --impl reference
times the CPU oracle on one round of the same workload per step.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOAD = "plain_large"
METRIC = "edges refined/s"
UNIT = "edges/s"


def _config(w):
    E = w.m // 2
    return {"workload": f"{w.name}: R-MAT scale 22 (a=0.57, b=c=0.19), edge factor 16, symmetrised + dedup, "
                        f"unit weights, k={w.k}, eps={w.eps}, seeded random balanced initial partition, "
                        f"{w.rounds} rounds",
            "n": w.n, "m": w.m, "edges": E, "k": w.k, "rounds": w.rounds,
            "l2": "inputs larger than L2 (CSR 0.55 GB, gain table 1.07 GB per build)"}


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = max(smax, float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax or None,
                "reasons": sorted(reasons), "samples": len(sm)}


HBM_NOMINAL_GBS = 7900.0      # GB300 HBM3e, nominal


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def code_digest(path: str) -> str:
    """First 16 hex digits of the sha256 of a C/CUDA source with its comments
    removed and its blank space normalised: edits of comments keep the
    digest, any change of the code changes it."""
    src = open(path, encoding="utf-8").read()
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    src = " ".join(src.split())
    src = re.sub(r"\s*([^\w\s])\s*", r"\1", src)     # no blank next to punctuation
    return hashlib.sha256(src.encode()).hexdigest()[:16]


def _dominant_kernel(profile: str):
    """The first row of a committed ncu launch-list summary (kernels by total
    device time in one step): name, launches and share of the step's kernel
    time."""
    try:
        txt = open(os.path.join(ROOT, "profiles", profile)).read()
    except OSError:
        return None
    m = re.search(r"^\| `([^`]+)` \| (\d+) \| (\d+) \| ([\d.]+)%", txt, flags=re.M)
    if not m:
        return None
    return {"kernel": m.group(1), "launches": int(m.group(2)), "us_total": int(m.group(3)),
            "share": float(m.group(4)) / 100, "source": f"profiles/{profile}"}


def _traffic(kernel_src: str, profile: str):
    """Per-launch DRAM bytes of the dominant kernel from a committed ncu summary,
    only if it was taken on the current kernel source (same code digest)."""
    try:
        txt = open(os.path.join(ROOT, "profiles", profile)).read()
    except OSError:
        return None
    sha = code_digest(os.path.join(ROOT, kernel_src))
    m1 = re.search(r"code_sha256_16:\s*([0-9a-f]+)", txt)
    m2 = re.search(r"traffic_bytes_per_launch:\s*([0-9]+)", txt)
    if not m1 or not m2 or m1.group(1) != sha:
        return None
    return int(m2.group(1))


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---- multi-rank host logic (one process per GPU; gloo on CPU in the tests)
def rank_graph_range(rank: int, per_rank: int):
    """Graphs of the batch owned by a rank: ids [rank * per_rank, (rank + 1) * per_rank)
    (each rank refines its own graphs: weak scaling, no collective on the data path)."""
    return rank * per_rank, per_rank


def allreduce_max(x: float, ws: int, device: str = "cuda") -> float:
    """Maximum of x over the ranks (x itself when running alone)."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank: float, ws: int, seconds_max: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return ws * units_per_rank / seconds_max


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    w = synth.cached(getattr(synth, WORKLOAD))
    oracle.build()
    E = w.m // 2
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        rc, p, c, tr = oracle.run_round(w, w.part, 1, w.rounds)
        t = time.perf_counter() - t0
        assert rc == oracle.OK
        if i >= args.warmup:
            times.append(t)
    per = sum(times) / len(times)
    value = E / per
    sample = f"one round (round 1 of {w.rounds}) of the full workload per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic", "config": _config(w),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def cpu_baseline(w):
    """The oracle as it stands, single-threaded, on one round of the same workload."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    rc, p, c, tr = oracle.run_round(w, w.part, 1, w.rounds)
    t = time.perf_counter() - t0
    return {"value": (w.m // 2) / t, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"round 1 of {w.rounds} on the full workload, {t:.1f} s, 1 of {os.cpu_count()} host cores"}


def batched_leg(args, upr, rank, ws, local, graphs):
    """The 4096-graph Chung-Lu batch refined by one context
    (upr_batch_create_mixed: the graphs of each k form one batch, the batches
    run concurrently, and from the second call on each batch's rounds are one
    CUDA graph launch, params.graphs = 2), every graph for its 4 rounds per
    step; against the plain one-graph-per-call form (upr_refine per graph,
    graph resident) on a sample of the same graphs, whose cuts must be
    identical; end to end from pinned host arrays."""
    import torch
    rounds = graphs[0].rounds
    ng = len(graphs)
    ks = [w.k for w in graphs]
    prm = upr.upr_params_default()
    prm.graphs = 2
    main = torch.cuda.current_stream()
    ctx = upr.upr_batch_create_mixed([(w.xadj, w.adj, w.vwgt, w.adjw) for w in graphs], ks,
                                     [w.eps for w in graphs], params=prm)
    init = torch.from_numpy(np.concatenate([w.part for w in graphs]).astype(np.int32)).cuda()
    part = torch.empty_like(init)

    def step():
        part.copy_(init)
        return upr.upr_batch_refine(ctx, part, rounds)

    for _ in range(max(2, min(args.warmup, 3))):        # the second call builds the batches' step graphs
        res = step()
    torch.cuda.synchronize()
    steps = max(1, min(args.steps, 5))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(main)
    for _ in range(steps):
        res = step()
    e1.record(main)
    torch.cuda.synchronize()
    t_batch = e0.elapsed_time(e1) / 1e3 / steps
    stat_b, _, cut_b, st_b = res
    cut_b = np.asarray(cut_b).copy()
    E = sum(w.m // 2 for w in graphs)
    n_batches = len(set(ks))

    # the plain form on a sample: one context and one upr_refine per graph
    sample = list(range(0, ng, max(1, ng // args.plain_sample)))[: args.plain_sample]
    plain = []
    for i in sample:
        w = graphs[i]
        c = upr.create_from_workload(w, device=True)
        plain.append((i, c, torch.from_numpy(w.part.copy()).cuda()))
    work = [torch.empty_like(p) for _, _, p in plain]
    for (i, c, p), q in zip(plain, work):       # warm-up
        q.copy_(p)
        upr.upr_refine(c, q, rounds)
    torch.cuda.synchronize()
    e0.record(main)
    cut_p = {}
    for (i, c, p), q in zip(plain, work):
        q.copy_(p)
        cut_p[i] = upr.upr_refine(c, q, rounds).cut_out
    e1.record(main)
    torch.cuda.synchronize()
    t_plain = e0.elapsed_time(e1) / 1e3
    identical = all(cut_p[i] == cut_b[i] for i in sample)
    del plain, work

    # end to end from pinned host arrays: one context created (upload and
    # checks), refined, partition read back
    def _pinned_views(arrays):
        # one pinned buffer per array kind, one view per graph
        buf = torch.from_numpy(np.concatenate(arrays)).pin_memory().numpy()
        ends = np.cumsum([len(a) for a in arrays])
        return [buf[e - len(a):e] for e, a in zip(ends, arrays)]

    xs = _pinned_views([w.xadj for w in graphs])
    adjs = _pinned_views([w.adj for w in graphs])
    assert all(w.vwgt is None and w.adjw is None for w in graphs)       # unit weights
    pinned = [(x, a, None, None) for x, a in zip(xs, adjs)]
    part_t = torch.from_numpy(np.concatenate([w.part for w in graphs]).astype(np.int32)).pin_memory()
    work_t = torch.empty(len(part_t), dtype=torch.int32).pin_memory()
    part_h, work_h = part_t.numpy(), work_t.numpy()
    prm1 = upr.upr_params_default()
    prm1.graphs = 2
    eps_all = [w.eps for w in graphs]
    # a context kept across steps (as a service refining batch after batch):
    # every step binds the step's graphs to it (upload from pinned host
    # memory and checks, its device memory reused), refines, reads back
    c_e2e = upr.upr_batch_create_mixed(pinned, ks, eps_all, params=prm1)

    def e2e_step():
        upr.upr_batch_rebind(c_e2e, pinned, ks, eps_all)
        work_t.copy_(part_t)         # the step's input partition (a host copy on several threads)
        return upr.upr_batch_refine(c_e2e, work_h, rounds)

    for _ in range(2):          # the second call captures the batches' step graphs
        e2e_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_steps = 3
    for _ in range(e2e_steps):
        e2e_step()
    torch.cuda.synchronize()
    t_e2e = (time.perf_counter() - t0) / e2e_steps
    upr.upr_destroy(c_e2e)
    # the same with the context created and destroyed inside the step
    t0 = time.perf_counter()
    c1 = upr.upr_batch_create_mixed(pinned, ks, eps_all, params=prm1)
    work_t.copy_(part_t)
    upr.upr_batch_refine(c1, work_h, rounds)
    upr.upr_destroy(c1)
    torch.cuda.synchronize()
    t_e2e_create = time.perf_counter() - t0
    h2d = sum(sum(x.nbytes for x in t if x is not None) for t in pinned) + part_h.nbytes
    d2h = part_h.nbytes
    upr.upr_destroy(ctx)
    return {
        "workload": f"{ng} Chung-Lu graphs, n log-uniform in [2^10, 2^16], avg degree U[4,32], exponent U[2.0,2.8], "
                    f"k from {{2,4,8,16,32}}, eps 0.03, unit weights, {rounds} rounds; one context "
                    f"(upr_batch_create_mixed: {n_batches} batches by k, run concurrently)",
        "graphs": ng, "nodes": int(sum(w.n for w in graphs)), "edges": int(E),
        "graphs_per_s": ng / t_batch, "edges_per_s": rounds * E / t_batch, "ms_per_step": t_batch * 1e3,
        "steps": steps, "gpu_launches_per_step": int(st_b.kernel_launches),
        "graph_launches_per_step": n_batches if st_b.rebalance_graphs == n_batches * rounds else None,
        "rounds_in_graphs_per_step": int(st_b.rebalance_graphs),
        "infeasible_graphs": int((stat_b != 0).sum()),
        "plain": {"form": "one upr_refine per graph, graph resident on the device", "graphs": len(sample),
                  "graphs_per_s": len(sample) / t_plain, "ms_per_graph": t_plain * 1e3 / len(sample)},
        "speedup_vs_plain": (ng / t_batch) / (len(sample) / t_plain),
        "identical_cuts_on_sample": bool(identical),
        "e2e": {"graphs_per_s": ng / t_e2e, "ms": t_e2e * 1e3, "h2d_bytes": int(h2d), "d2h_bytes": int(d2h),
                "includes": "upr_batch_rebind of the step's graphs from pinned host arrays to a context kept "
                            "across steps (upload, checks), refinement, partition read-back; the graphs have "
                            "the shape of the previous step's, so each batch's captured step graph is kept",
                "with_context_creation": {"graphs_per_s": ng / t_e2e_create, "ms": t_e2e_create * 1e3,
                                          "includes": "upr_batch_create_mixed, refinement, read-back, "
                                                      "upr_destroy (one step)"}},
        "_cuts": cut_b,
    }


def other_configs_leg(args, upr):
    """The two other single-graph workloads, timed like the main one (graph and
    partition resident, CUDA events around upr_refine): the Chung-Lu graph
    with 16,384 nodes (k = 8, 4 rounds) and the weighted random geometric
    graph with 2^22 nodes (k = 256, 8 rounds; also with each table layout
    forced), and the R-MAT workload under the round drivers of Sec. 4.4 / 6.2
    (the paper's final configuration also with the paper's ten rounds) and
    the variants of Sec. 7.2."""
    import torch
    peak, _ = _peaks()
    out = {}
    legs = (("chung_lu_n16384_k8", "plain_tiny", 20, {}), ("rgg_2^22_weighted_k256", "plain_weighted", 3, {}),
            ("rgg_2^22_weighted_k256_dense_table", "plain_weighted", 3, {"table": 1}),
            ("rgg_2^22_weighted_k256_hashed_table", "plain_weighted", 3, {"table": 2}),
            ("rgg_2^22_weighted_k256_gain_priority", "plain_weighted", 3, {"gain_priority": 1}),
            ("rmat_s22_k64_final_configuration_10_rounds", "plain_large", 3, {"schedule": 6, "rounds": 10}),
            ("rmat_s22_k64_final_configuration", "plain_large", 3, {"schedule": 6}),
            ("rmat_s22_k64_dynamic_activation", "plain_large", 3, {"schedule": 1}),
            ("rmat_s22_k64_constant_tau_half", "plain_large", 3, {"schedule": 3, "tau1_num": 1, "tau1_den": 2}),
            ("rmat_s22_k64_fully_unconstrained", "plain_large", 3, {"schedule": 4}),
            ("rmat_s22_k64_limited_imbalance", "plain_large", 3, {"schedule": 5}),
            ("rmat_s22_k64_appended_sequence", "plain_large", 3, {"append": 1}),
            ("rmat_s22_k64_label_propagation", "plain_large", 3, {"lp_rounds": 5}),
            ("rmat_s22_k64_label_propagation_final_configuration_10_rounds", "plain_large", 3,
             {"lp_rounds": 5, "schedule": 6, "rounds": 10}))
    for name, builder, steps, over in legs:
        w = synth.cached(getattr(synth, builder))
        prm = upr.upr_params_default()
        prm.graphs = 2              # as the headline: the rounds of a call as one graph where the schedule allows
        over = dict(over)
        rounds = over.pop("rounds", w.rounds)
        for key, val in over.items():
            setattr(prm, key, val)
        table, schedule = prm.table, prm.schedule
        ctx = upr.create_from_workload(w, params=prm, device=True)
        init = torch.from_numpy(w.part.copy()).cuda()
        part = torch.empty_like(init)
        for _ in range(2):
            part.copy_(init)
            upr.upr_refine(ctx, part, rounds)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        sts = []
        e0.record()
        for _ in range(steps):
            part.copy_(init)
            sts.append(upr.upr_refine(ctx, part, rounds))
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        st = sts[-1]
        t_build = sum(x.ms_gain_table for x in sts) / max(1, sum(x.gain_table_builds for x in sts))
        out[name] = {"n": w.n, "m": w.m, "k": w.k, "rounds": rounds, "weighted": w.adjw is not None,
                     "ms_per_refine": ms, "edges_per_s": rounds * (w.m // 2) / (ms / 1e3),
                     "cut_in": st.cut_in, "cut_out": st.cut_out,
                     "table": ("hashed rows" if st.sparse_table else "dense n x k")
                              + (" (chosen by size)" if table == 0 else ""),
                     "schedule": ["every round unconstrained",
                                  "dynamic activation (Sec. 4.4; not in the paper's final configuration)",
                                  "every round constrained", "constant penalty tau = 0.5 (Sec. 7.2)",
                                  "fully unconstrained (Sec. 7.2)", "limited imbalance 2 -> 1.1 (Sec. 7.2)",
                                  "the paper's final configuration (Sec. 4.4, Sec. 7.2)"][schedule],
                     "rebalancing_priority": "gain alone (Sec. 7.2)" if prm.gain_priority else "g/c, g*c (Sec. 6.1)",
                     "sequence": "appended (Sec. 7.2)" if prm.append else "interleaved (Sec. 4.4)",
                     "label_propagation_rounds_kept": st.lp_rounds,
                     "rounds_as_one_graph": st.ms_select == 0 and rounds > 0,
                     "constrained_rounds": st.constrained_rounds,
                     "gain_table_ms": t_build or None,
                     "gain_table_gbs": st.gain_table_bytes / (t_build / 1e3) / 1e9 if t_build else None,
                     "gain_table_frac": st.gain_table_bytes / (t_build / 1e3) / 1e9 / peak if t_build else None}
        del ctx
    return out


def _served_pool_cached(spec):
    synth.cached(synth.served_rmat, *spec)


SERVED_RMAT = [(18, 8, i) for i in range(4)] + [(18, 64, i) for i in range(4, 8)] + [(21, 8, 0), (21, 64, 1)]


def served_inputs(small):
    """Input pools of the served mix: the first Chung-Lu batch graphs, and
    R-MAT scale-18 / scale-21 graphs with k from {8, 64} (generated in a
    spawned pool before CUDA starts)."""
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(min(len(SERVED_RMAT), os.cpu_count() or 1)) as pool:
        pool.map(_served_pool_cached, SERVED_RMAT)
    rm = [synth.cached(synth.served_rmat, *spec) for spec in SERVED_RMAT]
    return {"small": small, "s18": [w for w in rm if w.info["scale"] == 18],
            "s21": [w for w in rm if w.info["scale"] == 21]}


def served_leg(args, upr, pools, batched_cuts):
    """Poisson stream of requests (50% Chung-Lu batch graphs, 40% R-MAT scale
    18, 10% R-MAT scale 21) into the continuous-batching server at a fixed
    arrival rate; latency is arrival (scheduled submit time) to result.  The
    capacity of a closed-loop burst of the same mix is measured before and
    reported beside it (a burst batches far more of the small graphs than a
    stream does, so it is an upper bound, not a sustainable rate)."""
    import concurrent.futures as cf
    rng = np.random.default_rng(20230815)
    kinds = ["small", "s18", "s21"]
    probs = [0.5, 0.4, 0.1]

    def draw():
        kind = kinds[int(rng.choice(3, p=probs))]
        pool = pools[kind]
        return kind, int(rng.integers(len(pool)))

    srv = upr.Server(max_jobs=args.serve_slots)
    ex = cf.ThreadPoolExecutor(256)
    results = []
    lock = threading.Lock()

    def request(kind, j, t_arrive, record):
        w = pools[kind][j]
        t = srv.submit(w)
        part, cut, st = srv.wait(t, timeout_ms=600000)
        t_done = time.perf_counter()
        if record:
            with lock:
                results.append((kind, j, t_arrive, t_done, cut, st.batch_graphs))

    # warm-up and closed-loop capacity: a burst of the mix submitted at once
    burst = [draw() for _ in range(args.serve_burst)]
    list(ex.map(lambda kj: request(kj[0], kj[1], 0.0, False), burst[:32]))
    t0 = time.perf_counter()
    list(ex.map(lambda kj: request(kj[0], kj[1], 0.0, False), burst))
    capacity = len(burst) / (time.perf_counter() - t0)
    lam = args.serve_rate
    # open loop: Poisson arrivals for serve_seconds
    futs = []
    start = time.perf_counter()
    t_next = start
    while t_next - start < args.serve_seconds:
        now = time.perf_counter()
        if t_next > now:
            time.sleep(t_next - now)
        kind, j = draw()
        futs.append(ex.submit(request, kind, j, t_next, True))
        t_next += rng.exponential(1.0 / lam)
    for f in futs:
        f.result()
    end = max(r[3] for r in results)
    ex.shutdown()
    srv.close()
    lat = np.array([(r[3] - r[2]) * 1e3 for r in results])
    # every request of one input must give one cut; Chung-Lu inputs also the batched leg's
    cuts = {}
    same = True
    for kind, j, _, _, cut, _ in results:
        same &= cuts.setdefault((kind, j), cut) == cut
        if kind == "small" and batched_cuts is not None:
            same &= int(batched_cuts[j]) == cut
    by_kind = {k: int(sum(r[0] == k for r in results)) for k in kinds}
    return {
        "workload": "Poisson arrivals; 50% Chung-Lu batch graphs (their own k, 4 rounds), 40% R-MAT scale 18, "
                    "10% R-MAT scale 21 (edge factor 16, k from {8, 64}, 8 rounds), eps 0.03; inputs drawn from "
                    f"pools of {len(pools['small'])} / {len(pools['s18'])} / {len(pools['s21'])} graphs",
        "slots": args.serve_slots, "seconds": args.serve_seconds, "requests": len(results), "by_kind": by_kind,
        "capacity_closed_loop_burst_per_s": capacity, "arrival_rate_per_s": lam,
        "graphs_per_s": len(results) / (end - start),
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "mean": float(lat.mean()), "max": float(lat.max())},
        "batched_requests": int(sum(r[5] > 1 for r in results)),
        "identical_results": bool(same),
    }


def run_gpu(args):
    import torch
    ws, rank, local = _dist()
    graphs = pools = None
    if args.batch_graphs > 0 and not args.profile:
        # generated before CUDA starts (a spawned pool); rank r owns its own graphs
        start, count = rank_graph_range(rank, args.batch_graphs)
        graphs = synth.batch_graphs(count, start=start)
        if args.serve_seconds > 0:
            pools = served_inputs(graphs[:512])
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2308_15494_gb300 import build as cuda_build
    cuda_build.build()
    import paper_2308_15494_gb300 as upr
    upr.load()

    w = synth.cached(getattr(synth, WORKLOAD), args.shrink)
    E = w.m // 2
    stream = torch.cuda.current_stream()
    prm = upr.upr_params_default()
    prm.graphs = 0 if args.no_graphs else args.graphs
    if args.profile and args.lp_rounds > 0:
        prm.lp_rounds = args.lp_rounds
    ctx = upr.create_from_workload(w, params=prm, device=True)
    part_init = torch.from_numpy(w.part.copy()).cuda()
    part = torch.empty_like(part_init)

    def step():
        part.copy_(part_init)
        return upr.upr_refine(ctx, part, w.rounds)

    # the context's first call runs its rounds from the host (phase times);
    # with graphs = 2 the later calls run them as one graph launch
    first_call = None
    for _ in range(args.warmup):
        st_w = step()
        first_call = first_call or st_w
    torch.cuda.synchronize()

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    stats = []
    barrier()
    with Clocks(local) as clk:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("timed")
        e0.record(stream)
        for _ in range(args.steps):
            stats.append(step())
        e1.record(stream)
        torch.cuda.nvtx.range_pop()
        barrier()
    ms = e0.elapsed_time(e1)
    if args.profile:
        if rank == 0:
            st = stats[-1]
            print(json.dumps({"profile": True, "ms_per_step": ms / args.steps,
                              "launches_per_step": st.kernel_launches,
                              "rebalance_graph_rounds": st.rebalance_graphs, "subrounds": st.subrounds,
                              "cut_out": st.cut_out,
                              "phases_ms": {"gain_table": st.ms_gain_table, "select": st.ms_select,
                                            "rebalance": st.ms_rebalance, "sequence": st.ms_sequence}}))
        return 0
    ms = allreduce_max(ms, ws)
    ms_step = ms / args.steps
    value = job_value(w.rounds * E, ws, ms_step / 1e3)

    # roofline of the dominant kernel: the gain-table build (device time from
    # CUDA events on the context's stream around every build)
    builds = sum(s.gain_table_builds for s in stats)
    t_build = sum(s.ms_gain_table for s in stats) / max(builds, 1) / 1e3
    bytes_build = stats[0].gain_table_bytes
    peak, peak_kind = _peaks()
    achieved = bytes_build / t_build / 1e9
    roofline = {"bound": "hbm", "kernel": "gain table build (k_table_tiles + k_table_hub_chunks)",
                "achieved": achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                "frac": achieved / peak, "peak_nominal": HBM_NOMINAL_GBS, "frac_nominal": achieved / HBM_NOMINAL_GBS,
                "bytes_per_launch": bytes_build, "ms_per_launch": t_build * 1e3,
                "traffic": _traffic("paper_2308_15494_gb300/csrc/graph.cu", "gain_table_rmat_s22_k64.md")}

    # the whole step against the same peak: the rounds' algorithmic bytes
    # (the per-round byte formula, counted by the library) over the call's
    # device time, and the same per round
    s_last = stats[-1]
    step_bytes = s_last.bytes_algorithmic
    step_ms = statistics.median(x.ms_device for x in stats)
    roofline["step"] = {"bytes_algorithmic": step_bytes, "ms_device": step_ms,
                        "achieved_gbs": step_bytes / (step_ms / 1e3) / 1e9,
                        "frac": step_bytes / (step_ms / 1e3) / 1e9 / peak,
                        "seq_degree_sum": s_last.seq_degree_sum,
                        "gain_table_builds": s_last.gain_table_builds,
                        "kernel_launches": s_last.kernel_launches}
    roofline["per_round"] = {"rounds": w.rounds, "bytes": step_bytes / w.rounds, "ms": step_ms / w.rounds,
                             "achieved_gbs": step_bytes / (step_ms / 1e3) / 1e9,
                             "frac": step_bytes / (step_ms / 1e3) / 1e9 / peak,
                             "phases_ms": None}
    roofline["dominant_kernel_by_time"] = _dominant_kernel("launches_rmat_s22_k64.md")

    # end to end through the C ABI from pinned host buffers
    pinned = {k: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
              for k, a in (("xadj", w.xadj), ("adj", w.adj), ("part", w.part), ("work", w.part))}
    pin = {k: t.numpy() for k, t in pinned.items()}
    h2d = pin["xadj"].nbytes + pin["adj"].nbytes + pin["part"].nbytes
    d2h = pin["part"].nbytes + 8
    e2e_steps = max(1, min(args.steps, 5))

    # a context kept across steps (as a service refining graph after graph):
    # every step binds the step's graph to it (upload from pinned host memory
    # and checks, its device memory reused), refines, reads the partition back
    c_e2e = upr.upr_create(pin["xadj"], pin["adj"], w.k, w.eps, params=prm)

    def e2e_step():
        upr.upr_rebind(c_e2e, pin["xadj"], pin["adj"], w.k, w.eps)
        pinned["work"].copy_(pinned["part"])     # the step's input partition (a host copy)
        return upr.upr_refine(c_e2e, pin["work"], w.rounds)

    def e2e_step_create():
        c = upr.upr_create(pin["xadj"], pin["adj"], w.k, w.eps)
        pinned["work"].copy_(pinned["part"])
        st = upr.upr_refine(c, pin["work"], w.rounds)
        upr.upr_destroy(c)
        return st

    for _ in range(2):          # with graphs = 2 the second call captures the step graph
        e2e_step()
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    barrier()
    t_e2e = (time.perf_counter() - t0) / e2e_steps
    t_e2e = allreduce_max(t_e2e, ws)
    upr.upr_destroy(c_e2e)
    e2e_step_create()
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step_create()
    barrier()
    t_e2e_c = allreduce_max((time.perf_counter() - t0) / e2e_steps, ws)
    e2e = {"value": job_value(w.rounds * E, ws, t_e2e), "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "ms_per_step": t_e2e * 1e3, "steps": e2e_steps,
           "includes": "upr_batch_rebind of the graph from pinned host buffers to a context kept across steps "
                       "(upload, checks), upr_refine from and to a pinned host partition; the graph has the "
                       "shape of the previous step's, so the captured step graph is kept",
           "with_context_creation": {"value": job_value(w.rounds * E, ws, t_e2e_c), "ms_per_step": t_e2e_c * 1e3,
                                     "includes": "upr_create, upr_refine, upr_destroy every step"}}

    # phase times: the timed calls run their rounds as one graph launch, so a
    # second context (graphs = 1, the lane schedules already tuned) refines
    # once with its rounds launched from the host
    phase_call = None
    if prm.graphs == 2 and rank == 0:
        prm_ph = upr.upr_params_default()
        prm_ph.graphs = 1
        ctx_ph = upr.create_from_workload(w, params=prm_ph, device=True)
        for _ in range(2):
            part.copy_(part_init)
            phase_call = upr.upr_refine(ctx_ph, part, w.rounds)
        upr.upr_destroy(ctx_ph)

    others = other_configs_leg(args, upr) if rank == 0 and not args.profile and args.other_configs else None
    batched = batched_leg(args, upr, rank, ws, local, graphs) if graphs else None
    served = served_leg(args, upr, pools, batched.get("_cuts") if batched else None) if pools else None
    if batched is not None:
        batched.pop("_cuts", None)
    if batched is not None and ws > 1:
        batched["ms_per_step"] = allreduce_max(batched["ms_per_step"], ws)
        batched["graphs_per_s"] = job_value(batched["graphs"], ws, batched["ms_per_step"] / 1e3)
    if rank == 0:
        cb = cpu_baseline(w) if ws == 1 and not args.no_cpu_baseline else None
        s0 = stats[-1]
        ph = s0 if (s0.ms_select > 0 or first_call is None or phase_call is None) else phase_call
        roofline["per_round"]["phases_ms"] = {"gain_table": s0.ms_gain_table / w.rounds,
                                              "select": ph.ms_select / w.rounds,
                                              "rebalance": ph.ms_rebalance / w.rounds,
                                              "sequence": ph.ms_sequence / w.rounds}
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "int64", "data": "synthetic", "config": _config(w),
                "e2e": e2e, "gpu_launches": int(sum(s.kernel_launches for s in stats)),
                "roofline": roofline, "cpu_baseline": cb, "clocks": clk.summary(),
                "phases_ms_per_step": {"gain_table": s0.ms_gain_table, "select": ph.ms_select,
                                       "rebalance": ph.ms_rebalance, "sequence": ph.ms_sequence,
                                       "host_wall": s0.ms_host,
                                       "phases_from": "the timed calls" if ph is s0 else
                                       "a second context with graphs = 1 (rounds launched from the host), "
                                       "second call; the timed calls run the rounds as one CUDA graph"},
                "result": {"cut_in": s0.cut_in, "cut_out": s0.cut_out, "moves": s0.n_moves,
                           "rebalance_moves": s0.n_rebalance_moves, "applied": s0.n_applied,
                           "subrounds": s0.subrounds, "table_builds_per_step": s0.gain_table_builds,
                           "rebalance_graph_rounds_per_step": s0.rebalance_graphs,
                           "lanes_per_node": {"select": s0.select_lanes, "propose": s0.propose_lanes}},
                "other_configs": others, "batched": batched, "served": served}
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-graphs", type=int, default=4096,
                    help="graphs of the Chung-Lu batch per GPU (0: skip the batched leg)")
    ap.add_argument("--plain-sample", type=int, default=256,
                    help="graphs of the batch timed in the one-graph-per-call form")
    ap.add_argument("--no-other-configs", dest="other_configs", action="store_false",
                    help="skip timing the 16k Chung-Lu and weighted RGG workloads")
    ap.add_argument("--serve-rate", type=float, default=200.0,
                    help="arrival rate of the served Poisson stream (requests/s)")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="length of the Poisson arrival window of the served leg (0: skip it)")
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--serve-burst", type=int, default=400,
                    help="requests of the closed-loop burst that measures capacity")
    ap.add_argument("--shrink", type=int, default=0,
                    help="profiling only: the same workload family with 2^-shrink of the nodes")
    ap.add_argument("--no-graphs", action="store_true",
                    help="launch every rebalancing sub-round from the host instead of one CUDA graph per round "
                         "(same kernels; ncu's NVTX filter does not see kernels launched by a graph)")
    ap.add_argument("--graphs", type=int, default=2, choices=[1, 2],
                    help="params.graphs of the headline workload: 1 each rebalancing loop as a CUDA graph, 2 also "
                         "all rounds of a call as one graph (from the context's second call on)")
    ap.add_argument("--lp-rounds", type=int, default=0,
                    help="with --profile: label propagation rounds before the FM rounds of the headline workload")
    ap.add_argument("--profile", action="store_true",
                    help="device loop only (for ncu launch lists): no e2e, no CPU baseline")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
