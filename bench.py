"""Benchmark of the exact minimum-cut solve (one JSON line on rank 0).

Default workload (the largest single-GPU configuration): the planted cut --
two G(2^21, average degree 42) blocks, each reduced to its 30-core, joined by
25 unit cross edges, ids permuted (seed 3): n = 4,071,044, m = 84,682,111,
lambda = 25.  A step is one full exact solve (every contraction-round kernel:
degree bound, label-propagation bound, PR1-PR4, CAPFOREST passes, union-find,
relabel/sort/segment-sum contraction, until lambda is proven) on the graph
already resident in HBM.

  value  = input edges m / device time of one solve (CUDA events on the
           graph's stream), whole job (sum over ranks / max time)
  e2e    = the same metric through the public API with host buffers: per
           step mincut_graph_from_csr from pinned host arrays (H2D copy,
           validation, canonicalisation), the solve and the D2H read of the
           value and the side bitmap
  roofline of the dominant kernel from the library's live CUDA-event profile
  cpu_baseline = the CPU oracle (sequential NOI) on a bounded sample of the
           workload: the same construction at 2^17 vertices per block
  rmat20 = the R-MAT scale-20 10-core (n = 247,314, m = 14,515,608) measured
           the same way, with its own roofline
  batched = 4096 small graphs in one packed batch solve vs one at a time
  serving = open-loop Poisson request stream through the continuous-batching
            server at 0.5x and 2x the sequential throughput: solves/s,
            p50/p99 latency
  small_config = connected G(2000, 16000) single solve against the CPU
            oracle's Stoer-Wagner and NOI

--workload picks the single-graph workload of the main line: planted21 (the
default above), planted18 / planted17 (the same construction at 2^18 / 2^17
vertices per block, for profiling), rmat20, rmat18 or er2000 (the small
configuration).
--impl reference times the CPU oracle as the reference arm (on the bounded
sample for planted21).  Multi-GPU runs (torchrun) are independent replicas:
the solve does not shard.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "exact min-cut edges/s & contraction HBM GB/s; batched solves/s, p50/p99 latency"

# Algorithmic bytes per unit (directed CSR entry) of each kernel category,
# int32 weights: what the step must move, not what an implementation re-reads.
ALG_BYTES = {
    "degree": 4,            # read w
    "pr_marks": 8,          # read col + w (PR1/PR2; PR3/PR4 row reads are extra)
    "lp_sweep": 12,         # read col + w, gather one label
    "lp_bound": 12,         # read col + w, gather one label
    "capforest_passes": 8,  # read col + w once
    "capforest_seq": 8,
    "emit": 20,             # read col + w (8), write key + value (12)
    "sort_pass": 24,        # read key + value (12), write key + value (12)
    "sort_hist": 8,         # read key
    "build_csr": 20,        # read key + value (12), write col + w (8)
    "contract_rows": 8,     # row-wise contraction, two scopes per round over the
                            # round's entries: together read col + w once (8)
                            # and write col + w of the contracted graph (<= 8)
}

# DRAM bytes per unit measured by ncu (dram__bytes_read.sum +
# dram__bytes_write.sum of one launch on the R-MAT core's first round, the
# capture summarised under profiles/), scaled to a launch by its units.  A
# kernel changed since its capture has no entry here (traffic: null).
TRAFFIC_PER_UNIT = {
    "pr_marks": (422.862080e6 + 3.253248e6) / 29031216,
}


CONTRACTION = ("contract_rows", "emit", "sort_hist", "sort_pass", "build_csr")

# Kernel categories bound by one dependent chain of memory accesses rather
# than by bandwidth: their HBM fraction is reported, with this note.
LATENCY_BOUND = {
    "capforest_seq": "latency-bound: one chain of dependent visits per pass (each visit a row "
                     "load and a gather of its neighbours' keys); the HBM fraction is tiny by "
                     "construction",
    "capforest_passes": "latency-bound: one chain of dependent pops per warp",
}

# Timed steps and end-to-end steps of each main-line workload by default
# (a planted-cut solve takes seconds; keep the timed work near a minute).
DEFAULT_STEPS = {"planted21": 3}
E2E_STEPS = {"planted21": 2}


def contraction_gbs(prof, peak, peak_kind):
    """The metric's contraction HBM GB/s: algorithmic bytes of the contraction
    kernels (ALG_BYTES per unit) over their CUDA-event time in the timed
    steps, per category and together, with the fraction of the HBM peak."""
    out, tot_b, tot_ms = {}, 0.0, 0.0
    for k in CONTRACTION:
        d = prof.get(k)
        if not d or d["ms"] <= 0:
            continue
        b = d["units"] * ALG_BYTES[k]
        out[k] = {"gbs": b / (d["ms"] / 1e3) / 1e9, "ms": d["ms"], "alg_bytes": b}
        tot_b += b
        tot_ms += d["ms"]
    if tot_ms > 0:
        gbs = tot_b / (tot_ms / 1e3) / 1e9
        out["total"] = {"gbs": gbs, "frac": gbs / peak, "peak": peak, "peak_kind": peak_kind}
    return out


def kernel_table(prof, steps, peak):
    """Per kernel category of the live profile: launches, CUDA-event time
    per step, share of the profiled time and, for the categories with an
    algorithmic byte count, the achieved algorithmic GB/s and its fraction
    of the HBM peak."""
    total = sum(v["ms"] for v in prof.values())
    out = {}
    for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"]):
        d = {"launches": v["launches"], "ms_per_step": v["ms"] / steps,
             "share": v["ms"] / total if total else None}
        if k in ALG_BYTES and v["ms"] > 0:
            gbs = v["units"] * ALG_BYTES[k] / (v["ms"] / 1e3) / 1e9
            d["alg_gbs"] = gbs
            d["frac"] = gbs / peak
        out[k] = d
    return out


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        return parse_clock_lines(self.lines)


def parse_clock_lines(lines):
    """Median SM clock, maximum SM clock and the throttle reasons seen active
    in nvidia-smi CSV lines of ClockSampler.Q (noheader, nounits); None when
    no line parses."""
    sm, mx, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for ln in lines:
        f = [x.strip() for x in ln.split(",")]
        if len(f) < 9:
            continue
        try:
            cur, top = float(f[1]), float(f[2])
        except ValueError:
            continue
        sm.append(cur)
        mx = top
        for nm, v in zip(names, f[5:9]):
            if v.lower().startswith("active"):
                reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
            "samples": len(sm)}


def make_workload(name: str):
    import synth
    if name == "rmat20":
        return synth.workload_rmat_core(20, 10, 2)
    if name == "rmat18":
        return synth.workload_rmat_core(18, 10, 2)
    if name == "er2000":
        return synth.workload_er2000()
    if name == "planted21":
        return synth.workload_planted(21, 42, 30, 25, 3)
    if name == "planted17":
        return synth.workload_planted(17, 42, 30, 25, 3)
    if name == "planted18":
        return synth.workload_planted(18, 42, 30, 25, 3)
    raise SystemExit(f"unknown workload {name}")


# The bounded CPU sample of each workload: the same construction at a size
# the single-core oracle solves in seconds (the full planted cut takes the
# oracle's NOI about two minutes on one core).
CPU_SAMPLE = {"planted21": "planted17"}
FULL_DESC = {"planted21": "planted_2x2^21_deg42_30core_cross25 (n=4071044, m=84682111, seed=3)"}
FULL_ORACLE_NOTE = {
    "planted21": "oracle NOI on the full workload: 130.9 s on one x86 core "
                 "(tests/golden/planted21_noi.json, lambda = 25)",
}


def arithmetic_desc(g) -> str:
    """The path's arithmetic for this workload: exact integers, with the sum
    width the library picks from the total weight of the directed entries."""
    wide = int(np.asarray(g.w, dtype=np.int64).sum()) > 0x7FFFFFFF
    return ("int32 weights, exact integer sums (" + ("64-bit" if wide else "32-bit") +
            " here; 32-bit when the total weight < 2^31, else 64-bit)")


def workload_desc(g) -> str:
    return f"{g.meta.get('workload')} (n={g.n}, m={g.m}, seed={g.meta.get('seed')})"


def cpu_oracle_time(name, g, budget_s: float = 30.0):
    """Time the CPU oracle (sequential NOI, one core) on the workload, or on
    its bounded sample (CPU_SAMPLE) for workloads too large for a few seconds
    of CPU; returns the baseline object and the value the oracle found on the
    graph it ran on (the workload's own lambda when it ran on the workload)."""
    import oracle
    sample = CPU_SAMPLE.get(name)
    gs = make_workload(sample) if sample else g
    t0 = time.perf_counter()
    lam, _, _ = oracle.noi(gs.n, gs.row_ptr, gs.col, gs.w)
    dt = time.perf_counter() - t0
    what = (f"one sequential NOI solve of {workload_desc(gs)}, the same construction as the "
            f"workload at a size one core solves in seconds ({dt:.2f} s, lambda={lam})"
            if sample else f"one sequential NOI solve of the full workload ({dt:.2f} s, "
            f"lambda={lam})")
    out = {"value": gs.m / dt, "unit": "edges/s", "cores": 1, "kind": "oracle", "sample": what}
    if name in FULL_ORACLE_NOTE:
        out["full_workload"] = FULL_ORACLE_NOTE[name]
    return out, (None if sample else lam)


def measure_batched(mc, n_graphs: int = 4096, alone: int = 256, reps: int = 3):
    """Batched workload: n_graphs graphs (n log-uniform in [20, 2000], average
    degree uniform in [3, 12], weights in [1, 100], seed 4) solved by one
    packed batch solve, against solving them one at a time on the device."""
    import synth
    import torch
    graphs = []
    for i in range(n_graphs):
        s = synth.batch_graph(4, i)
        graphs.append((s.n, s.row_ptr, s.col, s.w))
    vo, rp, col, w = mc.pack_graphs(graphs)
    B = mc.mincut_batch_from_csr(vo, rp, col, w)
    mc.mincut_batch_solve(B, bitmap=False)  # first solve: times the warp-solver thresholds
    small_n, small_graphs = mc.mincut_batch_info(B)
    paths = {}
    for name, t in (("round_kernels_only", -1), ("one_warp_per_graph_only", 2048)):
        o = mc.default_options(batch_small_n=t)
        mc.mincut_batch_solve(B, o, bitmap=False)
        tp = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            mc.mincut_batch_solve(B, o)
            torch.cuda.synchronize()
            tp.append(time.perf_counter() - t0)
        paths[name] = {"ms_per_batch": statistics.median(tp) * 1e3}
    ts = []
    launches = 0
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        vals, _, st = mc.mincut_batch_solve(B)
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
        launches += st["kernel_launches"]
    B.destroy()
    t_batch = statistics.median(ts)
    Gs = [mc.mincut_graph_from_csr(*g) for g in graphs[:alone]]
    for Gi in Gs[:8]:
        mc.mincut_solve(Gi, bitmap=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    one = [mc.mincut_solve(Gi)[0] for Gi in Gs]
    torch.cuda.synchronize()
    t_one = (time.perf_counter() - t0) / alone
    for Gi in Gs:
        Gi.destroy()
    assert one == [int(v) for v in vals[:alone]]
    rate = n_graphs / t_batch
    return {"workload": f"{n_graphs} graphs, n log-uniform [20,2000], avg deg U[3,12], w U[1,100], seed 4",
            "solves_per_s": rate, "ms_per_batch": t_batch * 1e3, "rounds": st["rounds"],
            "one_at_a_time_solves_per_s": 1.0 / t_one,
            "speedup_vs_one_at_a_time": rate * t_one, "gpu_launches_per_batch": launches // reps,
            "one_at_a_time_sample": alone,
            "warp_solver": {"threshold_n": small_n, "graphs": small_graphs,
                            "chosen_by": "timing candidate thresholds on the first solve"},
            "paths": paths}


def measure_variants(mc, g, val=None, reps: int = 3):
    """The paper's variants on the same workload: concurrent CAPFOREST passes
    with private visit arrays, the shared/private settings alternated over
    the first rounds, and the coarsening heuristic for the first bound.
    Host wall time of one solve (median of reps after one warm-up)."""
    import torch
    G = mc.mincut_graph_from_csr(g.n, g.row_ptr, g.col, g.w)
    out = {}
    for name, kw in [("default", {}), ("private_visit", {"cf_visit": 1}),
                     ("alternate_visit", {"cf_visit": 2}), ("coarsening_bound", {"init_bound": 1})]:
        o = mc.default_options(**kw)
        mc.mincut_solve(G, o, bitmap=False)
        ts, rounds = [], 0
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            v, _, st = mc.mincut_solve(G, o, bitmap=False)
            torch.cuda.synchronize()
            ts.append((time.perf_counter() - t0) * 1e3)
            rounds = st["rounds"]
            if val is None:
                val = v
            assert v == val, (name, v, val)
        out[name] = {"ms": statistics.median(ts), "rounds": rounds,
                     "lambda_source": st["lambda_source"]}
    G.destroy()
    return out


def measure_small_config(mc, reps: int = 5):
    """The small single-graph configuration: connected G(n=2000, m=16000),
    weights in [1, 10], seed 1.  GPU solve (host wall time, median of reps
    after a warm-up, graph resident) against the CPU oracle's Stoer-Wagner
    and sequential NOI on one host core."""
    import torch

    import oracle
    import synth
    g = synth.workload_er2000()
    G = mc.mincut_graph_from_csr(g.n, g.row_ptr, g.col, g.w)
    mc.mincut_solve(G, bitmap=False)
    ts = []
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        v, _, st = mc.mincut_solve(G, bitmap=False)
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
    G.destroy()
    c = (g.row_ptr, g.col, g.w.astype(np.int64))
    t0 = time.perf_counter()
    sw = oracle.stoer_wagner(g.n, *c)[0]
    t_sw = time.perf_counter() - t0
    t0 = time.perf_counter()
    noi = oracle.noi(g.n, *c)[0]
    t_noi = time.perf_counter() - t0
    assert v == sw == noi, (v, sw, noi)
    t = statistics.median(ts)
    return {"workload": workload_desc(g), "lambda": int(v), "ms": t * 1e3,
            "edges_per_s": g.m / t, "rounds": st["rounds"],
            "cpu_oracle": {"stoer_wagner_ms": t_sw * 1e3, "noi_ms": t_noi * 1e3, "cores": 1}}


def measure_adversarial(mc, reps: int = 2):
    """Families that defeat the PR tests: a wheel whose n trivial cuts are all
    minimum, and two interleaved cycles hiding one minimum cut (Theta(n)
    rounds).  Solve time and rounds with one sequential pass per round
    (Algorithm 2 as written) and with several whole passes at once (default);
    the CPU oracle's sequential NOI on the same graphs for context."""
    import synth
    import torch
    out = {}
    for name, gg in [("wheel_4097", synth.wheel(4097, seed=1)),
                     ("dblcyc_1026", synth.dblcyc(1026, 1000, 3, seed=2))]:
        G = mc.mincut_graph_from_csr(gg.n, gg.row_ptr, gg.col, gg.w)
        rec = {"n": gg.n, "m": int(gg.row_ptr[-1]) // 2, "lambda": gg.meta["lambda"]}
        for mode, kw in [("seq_passes_1", {"seq_passes": 1}), ("default", {})]:
            o = mc.default_options(**kw)
            ts = []
            for _ in range(reps):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                v, _, st = mc.mincut_solve(G, o, bitmap=False)
                torch.cuda.synchronize()
                ts.append((time.perf_counter() - t0) * 1e3)
                assert v == gg.meta["lambda"], (name, mode, v)
            ms = min(ts)
            rec[mode] = {"ms": ms, "rounds": st["rounds"],
                         "ms_per_round": ms / max(st["rounds"], 1),
                         "gpu_launches": st["kernel_launches"]}
        G.destroy()
        import oracle
        t0 = time.perf_counter()
        v, _, r = oracle.noi(gg.n, gg.row_ptr, gg.col, gg.w.astype(np.int64))
        rec["cpu_oracle_noi"] = {"ms": (time.perf_counter() - t0) * 1e3, "rounds": r, "cores": 1}
        assert v == gg.meta["lambda"]
        out[name] = rec
    return out


def _gen_request(args):
    import synth
    seed, i, nlo, nhi = args
    g = synth.serving_request(seed, i, nlo, nhi)
    return g.n, g.row_ptr, g.col, g.w, g.meta.get("kind")


def measure_serving(mc, n_req: int = 20000, nhi: int = 1 << 20, pool: int = 48, seed: int = 5,
                    workers: int = 16, window: int = 64, seq_sample: int = 1000,
                    low_sample: int = 4000):
    """Serving workload: a stream of n_req solve requests, n log-uniform in
    [100, nhi], R-MAT (scale ceil(log2 n), edge factor 16, truncated) or
    G(n, 8n) with probability 1/2 each, weights in [1, 100], largest
    component (seed 5), under the server's 60 GB device-memory admission cap.
    Host generation of 2^20-vertex R-MAT graphs takes seconds each, so the
    stream draws its requests from a pool of `pool` distinct seeded requests
    (generated in parallel processes; request j of the stream is pool entry
    mix(seed, j) mod pool).  Measured: sequential submission (create + solve +
    read back, one at a time) on the first seq_sample requests; a closed loop
    of `window` outstanding requests over the whole stream (saturation);
    open-loop Poisson arrivals at 2x the sequential rate over the whole stream
    and at 0.5x over its first low_sample requests.  The pool is in pinned
    host memory, read in place by the device on every path; the server
    borrows the arrays (mincut_server_submit_borrowed).  Latency = submission
    to completion.  Every served value equals its graph's value solved
    alone."""
    import multiprocessing as mp
    import threading
    from concurrent.futures import ProcessPoolExecutor

    import torch

    import synth
    t0 = time.perf_counter()
    with ProcessPoolExecutor(max_workers=min(16, os.cpu_count() or 4),
                             mp_context=mp.get_context("spawn")) as ex:
        reqs = list(ex.map(_gen_request, [(seed, i, 100, nhi) for i in range(pool)]))
    t_gen = time.perf_counter() - t0
    # the pool lives in pinned host memory: the device reads each request in
    # place, and the server borrows the arrays instead of copying them
    reqs = [(n, torch.from_numpy(rp).pin_memory().numpy(), torch.from_numpy(col).pin_memory().numpy(),
             torch.from_numpy(w).pin_memory().numpy(), kind) for (n, rp, col, w, kind) in reqs]
    # the value of every pool graph, solved alone
    expected = []
    for (n, rp, col, w, _) in reqs:
        Gi = mc.mincut_graph_from_csr(n, rp, col, w)
        expected.append(mc.mincut_solve(Gi, bitmap=False)[0])
        Gi.destroy()
    stream = [synth.splitmix64(seed ^ (0x9E3779B97F4A7C15 * (j + 1) & ((1 << 64) - 1)))[0] % pool
              for j in range(n_req)]
    sizes = [reqs[k][0] for k in stream]
    edges = [int(reqs[k][1][-1]) // 2 for k in stream]
    # ---- sequential submission on the first seq_sample requests
    lat_seq = []
    t0 = time.perf_counter()
    for k in stream[:seq_sample]:
        n, rp, col, w, _ = reqs[k]
        t1 = time.perf_counter()
        Gi = mc.mincut_graph_from_csr(n, rp, col, w)
        v, _, _ = mc.mincut_solve(Gi)
        Gi.destroy()
        lat_seq.append((time.perf_counter() - t1) * 1e3)
        assert v == expected[k]
    seq_rate = seq_sample / (time.perf_counter() - t0)
    out = {"workload": (f"{n_req} requests, n log-uniform [100,{nhi}], R-MAT/ER 50/50, "
                        f"w U[1,100], largest component, seed {seed}; drawn from a pool of "
                        f"{pool} distinct seeded requests (host generation of 2^20-vertex "
                        f"R-MAT graphs takes seconds each; pool generated in {t_gen:.1f} s)"),
           "requests": n_req, "n_max_drawn": max(sizes), "n_median": int(np.median(sizes)),
           "edges_total": int(sum(edges)), "workers": workers,
           "admission_cap_bytes": int(60 << 30),
           "sequential": {"sample": seq_sample, "solves_per_s": seq_rate,
                          "p50_ms": float(np.percentile(lat_seq, 50)),
                          "p99_ms": float(np.percentile(lat_seq, 99))}}

    def run(order, gaps=None):
        """Serve `order` (pool indices): with gaps, open-loop arrivals at those
        inter-arrival times; else a closed loop of `window` outstanding."""
        S = mc.Server(workers=workers)
        ids = [None] * len(order)
        lats = [0.0] * len(order)
        vals = [None] * len(order)
        start = time.perf_counter()
        if gaps is None:
            nxt = 0
            for i in range(len(order)):
                while nxt < len(order) and nxt - i < window:
                    n, rp, col, w, _ = reqs[order[nxt]]
                    ids[nxt] = S.submit(n, rp, col, w, borrow=True)
                    nxt += 1
                vals[i], lats[i], _ = S.wait(ids[i], bitmap=False)
        else:
            def submitter():
                t_next = start
                for i, k in enumerate(order):
                    t_next += gaps[i]
                    d = t_next - time.perf_counter()
                    if d > 0:
                        time.sleep(d)
                    n, rp, col, w, _ = reqs[k]
                    ids[i] = S.submit(n, rp, col, w, borrow=True)
            th = threading.Thread(target=submitter)
            th.start()
            for i in range(len(order)):
                while ids[i] is None:
                    time.sleep(0.0002)
                vals[i], lats[i], _ = S.wait(ids[i], bitmap=False)
            th.join()
        wall = time.perf_counter() - start
        st = S.stats()
        S.close()
        assert all(v == expected[k] for v, k in zip(vals, order))
        return {"solves_per_s": len(order) / wall, "wall_s": wall,
                "p50_ms": float(np.percentile(lats, 50)),
                "p99_ms": float(np.percentile(lats, 99)),
                "packed_batches": st["packed_batches"], "peak_inflight": st["peak_inflight"],
                "all_equal_alone": True}

    rng = np.random.default_rng(seed)
    out["closed_loop"] = dict(run(stream), window=window)
    out["closed_loop"]["speedup_vs_sequential"] = out["closed_loop"]["solves_per_s"] / seq_rate
    out["load_2.0x"] = dict(run(stream, rng.exponential(1.0 / (2 * seq_rate), size=n_req)),
                            offered_per_s=2 * seq_rate)
    low = stream[:low_sample]
    out["load_0.5x"] = dict(run(low, rng.exponential(1.0 / (0.5 * seq_rate), size=len(low))),
                            offered_per_s=0.5 * seq_rate, requests=len(low))
    return out


def reduce_max_over_ranks(vals, device):
    """Element-wise maximum of vals over all ranks: each replica times its
    own copy of the workload, and the job's step time is the slowest rank's."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(vals, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t]


def job_rate(world, units_per_rank, ms_max):
    """Whole-job throughput: every rank processed units_per_rank in at most
    ms_max milliseconds."""
    return world * units_per_rank / (ms_max / 1e3)


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle's sequential NOI (one host core) on the
    main line's workload -- on its bounded sample (CPU_SAMPLE) where the full
    workload takes the oracle minutes -- for the same metric and unit."""
    if rank != 0:
        return
    import oracle
    name = args.workload
    sample = CPU_SAMPLE.get(name)
    g = make_workload(sample or name)
    steps = args.steps if args.steps > 0 else DEFAULT_STEPS.get(name, 5)
    for _ in range(args.warmup):
        pass  # the oracle has no warm state; warm-up steps are not repeated solves
    times = []
    lam = None
    for _ in range(steps):
        t0 = time.perf_counter()
        lam, _, _ = oracle.noi(g.n, g.row_ptr, g.col, g.w)
        times.append(time.perf_counter() - t0)
    t = statistics.mean(times)
    v = g.m / t
    what = (f"{steps} sequential NOI solves of {workload_desc(g)}, the bounded sample of "
            f"{name} (same construction, one core)" if sample else
            f"{steps} sequential NOI solves of the full workload")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "edges/s",
            "n_gpus": world, "steps": steps, "warmup": args.warmup,
            "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": FULL_DESC.get(name, name) if sample else workload_desc(g),
                       "sample": workload_desc(g) if sample else None, "lambda": lam,
                       "parallelism": "single host thread"},
            "cpu_baseline": {"value": v, "unit": "edges/s", "cores": 1, "kind": "oracle",
                             "sample": what},
            "e2e": {"value": v, "unit": "edges/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    if name in FULL_ORACLE_NOTE:
        line["cpu_baseline"]["full_workload"] = FULL_ORACLE_NOTE[name]
    print(json.dumps(line), flush=True)


def measure_single(mc, g, steps, warmup, dev, stream, e2e_steps):
    """One single-graph workload: warm-up solves, then `steps` timed solves on
    the resident graph (CUDA events on the graph's stream, a 256 MB buffer
    written between steps to flush L2, nvidia-smi clocks sampled during the
    timed region), the live per-kernel profile of the timed solves, and the
    end-to-end time through the public API from pinned host arrays."""
    import torch
    G = mc.mincut_graph_from_csr(g.n, g.row_ptr, g.col, g.w, stream=stream.cuda_stream)
    opts = mc.default_options(profile=1)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=f"cuda:{dev}")
    for _ in range(max(warmup, 3)):
        val, _, _ = mc.mincut_solve(G, opts, bitmap=False)
    mc.mincut_profile_read(G, reset=True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    clocks = ClockSampler(dev)
    launches = 0
    rounds = []
    torch.cuda.synchronize()
    clocks.start()
    for i in range(steps):
        flush.fill_(i)  # write 256 MB (> L2) between steps, outside the timed events
        with torch.cuda.stream(stream):
            stream.wait_stream(torch.cuda.current_stream())
            ev[i][0].record(stream)
            val, bm, st = mc.mincut_solve(G, opts)
            ev[i][1].record(stream)
        launches += st["kernel_launches"]
        rounds.append(st["rounds"])
    torch.cuda.synchronize()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    prof = mc.mincut_profile_read(G, reset=True)
    G.destroy()
    # ---- end to end through the public API with host buffers
    rp_h = torch.from_numpy(g.row_ptr).pin_memory()
    col_h = torch.from_numpy(g.col).pin_memory()
    w_h = torch.from_numpy(g.w).pin_memory()
    e2e_ms = []
    for i in range(e2e_steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        G2 = mc.mincut_graph_from_csr(g.n, rp_h.numpy(), col_h.numpy(), w_h.numpy(),
                                      stream=stream.cuda_stream)
        v2, bm2, _ = mc.mincut_solve(G2, mc.default_options())
        G2.destroy()
        torch.cuda.synchronize()
        if i > 0:  # first call warms the allocator pool
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
        assert v2 == val
    return {"val": val, "ms": statistics.mean(step_ms), "step_ms": step_ms,
            "e2e_ms": statistics.mean(e2e_ms), "prof": prof, "launches": launches,
            "rounds": statistics.median(rounds), "clocks": clk,
            "h2d": int(g.row_ptr.nbytes + g.col.nbytes + g.w.nbytes),
            "d2h": int(8 * ((g.n + 63) // 64) + 8)}


def roofline_of(prof, peak, peak_kind):
    """Roofline object of the dominant kernel category (longest CUDA-event
    time among those with an algorithmic byte count): algorithmic bytes per
    launch over its average launch time, against the measured HBM peak."""
    kern = {k: v for k, v in prof.items() if k in ALG_BYTES and v["launches"] > 0}
    if not kern:
        return None
    dom = max(kern, key=lambda k: kern[k]["ms"])
    d = kern[dom]
    alg_bytes = d["units"] * ALG_BYTES[dom] / d["launches"]
    avg_s = d["ms"] / d["launches"] / 1e3
    ach = alg_bytes / avg_s / 1e9
    tpu = TRAFFIC_PER_UNIT.get(dom)
    out = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": peak, "unit": "GB/s",
           "frac": ach / peak, "peak_kind": peak_kind,
           "traffic": (tpu * d["units"] / d["launches"]) if tpu else None,
           "alg_bytes_per_launch": alg_bytes, "avg_launch_ms": d["ms"] / d["launches"]}
    if dom in LATENCY_BOUND:
        out["note"] = LATENCY_BOUND[dom]
    return out


def run_gpu(args, rank, world):
    import torch

    import paper_2609_07204_gb300 as mc
    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream()
    g = make_workload(args.workload)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    barrier()
    steps = args.steps if args.steps > 0 else DEFAULT_STEPS.get(args.workload, 5)
    e2e_steps = max(1, min(steps, E2E_STEPS.get(args.workload, steps)))
    r = measure_single(mc, g, steps, args.warmup, dev, stream, e2e_steps)
    barrier()
    t_max, e_max = r["ms"], r["e2e_ms"]
    if world > 1:
        t_max, e_max = reduce_max_over_ranks([r["ms"], r["e2e_ms"]], f"cuda:{dev}")
    if rank != 0:
        return
    val = r["val"]
    value = job_rate(world, g.m, t_max)
    peak, peak_kind = load_peaks()
    prof = r["prof"]
    line = {
        "metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": world,
        "steps": steps, "warmup": max(args.warmup, 3), "ms_per_step": t_max,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": arithmetic_desc(g),
        "data": "synthetic",
        "config": {"workload": workload_desc(g), "lambda": val,
                   "rounds": r["rounds"], "parallelism": "replicas",
                   "l2": "256 MB buffer written between steps, outside the timed events; "
                         f"input CSR {(g.col.nbytes + g.w.nbytes) >> 20} MB > L2"},
        "e2e": {"value": job_rate(world, g.m, e_max), "unit": "edges/s",
                "h2d_bytes_per_step": r["h2d"], "d2h_bytes_per_step": r["d2h"],
                "ms_per_step": e_max, "steps": e2e_steps},
        "gpu_launches": int(r["launches"]),
        "roofline": roofline_of(prof, peak, peak_kind),
        "kernels": kernel_table(prof, steps, peak),
        "contraction": contraction_gbs(prof, peak, peak_kind),
        "clocks": r["clocks"],
    }
    if not args.no_extra and args.workload != "rmat20":
        g2 = make_workload("rmat20")
        r2 = measure_single(mc, g2, 5, 3, dev, stream, 3)
        line["rmat20"] = {
            "workload": workload_desc(g2), "lambda": r2["val"],
            "value": g2.m / (r2["ms"] / 1e3), "unit": "edges/s", "ms_per_step": r2["ms"],
            "steps": 5, "rounds": r2["rounds"],
            "e2e": {"value": g2.m / (r2["e2e_ms"] / 1e3), "ms_per_step": r2["e2e_ms"],
                    "h2d_bytes_per_step": r2["h2d"], "d2h_bytes_per_step": r2["d2h"]},
            "roofline": roofline_of(r2["prof"], peak, peak_kind),
            "kernels": kernel_table(r2["prof"], 5, peak),
            "contraction": contraction_gbs(r2["prof"], peak, peak_kind),
            "clocks": r2["clocks"]}
    if not args.no_extra:
        line["batched"] = measure_batched(mc)
        line["serving"] = measure_serving(mc)
        line["variants"] = measure_variants(mc, make_workload("rmat20"))
        line["small_config"] = measure_small_config(mc)
        if not args.no_cpu_baseline:
            line["adversarial"] = measure_adversarial(mc)
    if not args.no_cpu_baseline:
        cb, lam = cpu_oracle_time(args.workload, g)
        assert lam is None or lam == val, (lam, val)
        line["cpu_baseline"] = cb
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=0,
                    help="timed steps (0: 3 for planted21, 5 otherwise)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="planted21")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the batched and serving measurements")
    ap.add_argument("--batched-only", action="store_true",
                    help="only the batched measurement, printed as one JSON object "
                         "(a short command to profile the batched kernels)")
    ap.add_argument("--serving-only", action="store_true",
                    help="only the serving measurement, printed as one JSON object")
    ap.add_argument("--small-only", action="store_true",
                    help="only the small single-graph measurement, printed as one JSON "
                         "object (a short command to profile the sequential pass)")
    args = ap.parse_args()
    if args.batched_only or args.small_only or args.serving_only:
        import torch

        import paper_2609_07204_gb300 as mc
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        mc.load_library()
        if args.batched_only:
            print(json.dumps({"batched": measure_batched(mc)}), flush=True)
        elif args.serving_only:
            print(json.dumps({"serving": measure_serving(mc)}), flush=True)
        else:
            print(json.dumps({"small_config": measure_small_config(mc)}), flush=True)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and args.impl == "gpu":
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_gpu(args, rank, world)
    if world > 1 and args.impl == "gpu":
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
