#!/usr/bin/env python
"""ε-graph benchmark: one step = cover-tree build + exact ε query (count ->
scan -> emit -> row sort) of one synthetic input resident in HBM.

Default workload: 1,000,000 points, 128-D, 100-component Gaussian mixture in
8-D embedded in 128-D, eps calibrated for ~70 mean neighbours (the paper's
sift eps=175 shape).  Prints ONE JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
                  [--workload gmm_1m_k70|gmm_1m_k500|dna_50k|clouds_64|small_3d]
                  [--form tc+learned+upper|tc+learned|tc|learned|plain|auto|auto+learned|...+upper]
                  [--no-compare] [--no-cpu-baseline] [--no-e2e]

The default form is the tensor-core-filtered, learned, upper-triangle one
for L2 points and the learned, upper-triangle one for edit distance and
Hamming codes.  Every other form is timed beside it on the
same input ("forms" in the JSON line), and its whole CSR is compared with the
default form's, entry for entry.

With N > 1 (torchrun) every rank runs an independent replica of the workload
(nothing is sharded; weak scaling) and the time is the max over ranks.
``--impl reference`` times the CPU oracle (plain cover tree, FP64, OpenMP) on
a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import re
import shutil
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2510_14147_gb300 import inputs as I  # noqa: E402

METRIC = "ε-graph edges/s"
UNIT = "edges/s"
SMS, FP32_LANES, INT32_LANES = 152, 128, 64   # GB300: 152 SMs; FP32 and INT32 lanes per SM
PROFILES = os.path.join(ROOT, "profiles")


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def combine_ranks(t_ms: float, units: float, dist, device="cuda"):
    """Whole-job figures of a timed region: the time is the slowest rank's,
    the units (edges) are summed over the ranks (each rank runs its own
    replica).  Without a process group the rank's own figures."""
    if not dist:
        return t_ms, units
    import torch
    tt = torch.tensor([float(t_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    uu = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(uu, op=dist.ReduceOp.SUM)
    return float(tt.item()), int(round(uu.item()))


# ------------------------------------------------------------------ inputs

def load_points(wl: dict) -> np.ndarray:
    if wl["kind"] == "gmm":
        return I.gmm_embedded(wl["n"], dim=wl["dim"], seed=wl["seed"])
    if wl["kind"] == "uniform":
        return I.uniform_cube(wl["n"], wl["dim"], seed=wl["seed"])
    raise ValueError("workload %s has no point cloud" % wl)


def load_input(wl: dict):
    """("points", x) for L2 workloads, ("strings", (data, offsets)) for edit
    distance, ("bits", (rows, bits)) for Hamming."""
    if wl["kind"] == "bits":
        return "bits", (I.binary_codes(wl["n"], wl["bits"], n_centres=wl["n_centres"], flip=wl["flip"],
                                       seed=wl["seed"]), wl["bits"])
    if wl["kind"] == "dna":
        return "strings", I.dna_strings(n_seeds=wl["n_seeds"], per_seed=wl["per_seed"],
                                        seed_len=wl["seed_len"], seed=wl["seed"])
    return "points", load_points(wl)


def n_of(kind, host) -> int:
    if kind == "bits":
        return host[0].shape[0]
    return host.shape[0] if kind == "points" else host[1].size - 1


def oracle_space(kind, host):
    import oracle
    if kind == "bits":
        return oracle.Space(bits=host)
    return oracle.Space(points=host) if kind == "points" else oracle.Space(strings=host)


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clock/throttle sampling while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.lines = []
        self.proc = None
        self.t0 = self.t1 = None

    def start(self):
        exe = shutil.which("nvidia-smi")
        if not exe:
            return
        self.proc = subprocess.Popen([exe, "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                      "-lms", "100", "-i", self.gpu_id],
                                     stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        self._th = threading.Thread(target=self._read, daemon=True)
        self._th.start()
        time.sleep(0.3)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self, which):
        setattr(self, which, time.time())

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for ts, line in self.lines:
            if self.t0 and self.t1 and not (self.t0 - 0.05 <= ts <= self.t1 + 0.15):
                continue
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append({"sm": float(parts[1]), "max": float(parts[2]),
                             "power": float(parts[3]) if parts[3] not in ("[N/A]", "N/A") else 0.0,
                             "hw": parts[5], "hwt": parts[6], "swt": parts[7], "pcap": parts[8]})
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("pcap", "sw_power_cap")):
                if r[key].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median([r["sm"] for r in rows])),
                "sm_max_mhz": max(r["max"] for r in rows), "reasons": sorted(reasons),
                "samples": len(rows), "power_w_max": max(r["power"] for r in rows)}


def gpu_identifier(torch, dev: int) -> str:
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        if vis:
            return vis.split(",")[dev]
        return str(dev)


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {}


def profile_value(kernel: str, workload: str, key: str):
    """A figure (e.g. dram_bytes_per_launch) from a committed ncu summary, or None."""
    path = os.path.join(PROFILES, "%s__%s.txt" % (kernel, workload))
    if not os.path.exists(path):
        return None
    for line in open(path):
        m = re.match(r"\s*%s\s*[:=]\s*([0-9.eE+]+)" % re.escape(key), line)
        if m:
            return float(m.group(1))
    return None


# --------------------------------------------------------------- CPU oracle

def oracle_sample(kind, host, wl: dict, n_queries: int, seed: int = 7):
    """Oracle cover tree (Algorithms 1-3, FP64) built on every point, queried
    for a random sample of points; extrapolated to all n queries."""
    import oracle
    oracle.build()
    sp = oracle_space(kind, host)
    n = n_of(kind, host)
    t0 = time.perf_counter()
    tree = oracle.build_tree(sp, zeta=wl.get("zeta", 32))
    t_build = time.perf_counter() - t0
    rng = np.random.default_rng(seed)
    rows = np.sort(rng.choice(n, size=min(n_queries, n), replace=False))
    t0 = time.perf_counter()
    res = oracle.tree_query_rows(sp, tree, wl["eps"], rows)
    t_query = time.perf_counter() - t0
    scale = n / rows.size
    edges = float(res["row_ptr"][-1]) * scale
    t_total = t_build + t_query * scale
    evals = (tree.dist_evals + res["dist_evals"] * scale)
    return {"value": edges / t_total, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": "oracle tree built on all %d points (%.1f s); %d random queries (%.1f s) "
                      "extrapolated to %d queries" % (n, t_build, rows.size, t_query, n),
            "dist_evals_per_s": evals / t_total, "wall_s": t_build + t_query,
            "extrapolated_s": t_total}


def oracle_rows_sample(kind, host, wl: dict, n_queries: int, seed: int = 7):
    """The oracle's brute force (the Sec. III definition) for a random sample
    of query rows, extrapolated to all n rows (used where the oracle's cover
    tree would take the CPU too long to build: Hamming rows are compared bit
    by bit, and farthest-first splits of 1000 clusters need 1000 centres per
    pass over a million points)."""
    import oracle
    oracle.build()
    sp = oracle_space(kind, host)
    n = n_of(kind, host)
    rng = np.random.default_rng(seed)
    rows = np.sort(rng.choice(n, size=min(n_queries, n), replace=False))
    t0 = time.perf_counter()
    res = oracle.brute_rows(sp, wl["eps"], rows)
    dt = time.perf_counter() - t0
    scale = n / rows.size
    return {"value": float(res["row_ptr"][-1]) * scale / (dt * scale), "unit": UNIT, "cores": oracle.num_threads(),
            "kind": "oracle", "sample": "oracle brute force on %d random rows of %d (%.1f s), extrapolated to all "
                                        "rows" % (rows.size, n, dt),
            "wall_s": dt, "extrapolated_s": dt * scale}


def oracle_clouds_sample(specs, per_cloud: int, seed: int = 7):
    """Many clouds: the oracle's brute force (the ε-graph definition, FP64)
    for a random sample of query rows of every cloud, each cloud extrapolated
    to all its rows (a cover tree of the uniform 64-D clouds would take the
    CPU minutes to build: their farthest-first levels are quadratic)."""
    import oracle
    oracle.build()
    rng = np.random.default_rng(seed)
    edges = t_total = wall = 0.0
    for sp in specs:
        x = I.cloud_points(sp)
        s = oracle.Space(points=x)
        rows = np.sort(rng.choice(x.shape[0], size=min(per_cloud, x.shape[0]), replace=False))
        t0 = time.perf_counter()
        res = oracle.brute_rows(s, sp["eps"], rows)
        dt = time.perf_counter() - t0
        scale = x.shape[0] / rows.size
        edges += float(res["row_ptr"][-1]) * scale
        t_total += dt * scale
        wall += dt
    return {"value": edges / t_total, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": "oracle brute force (FP64) on %d random rows of each of %d clouds (%.1f s), each cloud "
                      "extrapolated to all its rows" % (per_cloud, len(specs), wall),
            "wall_s": wall, "extrapolated_s": t_total}


def run_reference(args, wl):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    if wl["kind"] == "clouds":
        samp = lambda seed: oracle_clouds_sample(wl["specs"], args.ref_queries // 40, seed=seed)
        cfg = clouds_config(args, wl, world)
    elif wl["kind"] == "bits":
        kind, host = load_input(wl)
        samp = lambda seed: oracle_rows_sample(kind, host, wl, args.ref_queries // 20, seed=seed)
        cfg = config_of(args, wl, world)
    else:
        kind, host = load_input(wl)
        samp = lambda seed: oracle_sample(kind, host, wl, args.ref_queries, seed=seed)
        cfg = config_of(args, wl, world)
    for _ in range(args.warmup):
        samp(11)
    vals, walls, ext = [], [], []
    for k in range(args.steps):
        r = samp(100 + k)
        vals.append(r["value"] * r["extrapolated_s"])
        walls.append(r["wall_s"])
        ext.append(r["extrapolated_s"])
        last = r
    value = sum(vals) / sum(ext)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(walls) / len(walls),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32" if wl["kind"] in ("dna", "bits") else "f64", "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": last["cores"], "kind": "oracle",
                             "sample": last["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# the three radii of a sweep over one tree (sift's eps = 125, 175, 225 shapes)
SWEEPS = {"gmm_1m_k70": ["gmm_1m_k10", "gmm_1m_k70", "gmm_1m_k500"],
          "gmm_1m_k500": ["gmm_1m_k10", "gmm_1m_k70", "gmm_1m_k500"]}

FORMS = {"plain": (0, False), "tc": (1, False), "learned": (0, True), "tc+learned": (1, True),
         "auto": (2, False), "auto+learned": (2, True)}
# any form with "+upper": the upper-triangle query (each pair of two query
# groups evaluated once, mirrored into both rows)
FORMS.update({k + "+upper": v for k, v in list(FORMS.items())})


def form_opts(name):
    prec, learned = FORMS[name]
    return prec, learned, name.endswith("+upper")


def default_form(wl) -> str:
    return "learned+upper" if wl["kind"] in ("dna", "bits") else "tc+learned+upper"


def config_of(args, wl, world):
    prec, learned, upper = form_opts(args.form)
    if wl["kind"] == "bits":
        return {"workload": args.workload, "n": wl["n"], "bits": wl["bits"], "metric": "hamming", "eps": wl["eps"],
                "zeta": wl.get("zeta", 32), "target_degree": wl.get("target_degree"), "form": args.form,
                "precision": prec, "learned": learned, "upper_triangle": upper,
                "codes": "%d centres, bits flipped with probability %g" % (wl["n_centres"], wl["flip"]),
                "parallelism": "replicas%d" % world if world > 1 else "single",
                "l2": "inputs (%.0f MB) smaller than L2 (129 MB): a 256 MB buffer is written before every "
                      "timed step" % (wl["n"] * wl["bits"] / 8e6),
                "step": "ct_build + eps_graph_query + csr_free"}
    if wl["kind"] == "dna":
        n = wl["n_seeds"] * wl["per_seed"]
        return {"workload": args.workload, "n": n, "metric": "levenshtein", "eps": wl["eps"],
                "zeta": wl.get("zeta", 32), "form": args.form, "precision": prec, "learned": learned,
                "upper_triangle": upper, "strings": "%d seeds of length %d, %d mutants each" % (wl["n_seeds"], wl["seed_len"],
                                                                       wl["per_seed"]),
                "parallelism": "replicas%d" % world if world > 1 else "single",
                "l2": "inputs (strings, 5 MB) smaller than L2 (129 MB): a 256 MB buffer is written before every "
                      "timed step",
                "step": "ct_build + eps_graph_query + csr_free"}
    return {"workload": args.workload, "n": wl["n"], "dim": wl["dim"], "eps": wl["eps"],
            "zeta": wl.get("zeta", 32), "target_degree": wl.get("target_degree"),
            "form": args.form, "precision": prec, "learned": learned, "upper_triangle": upper,
            "parallelism": "replicas%d" % world if world > 1 else "single",
            "l2": "inputs (%.0f MB) larger than L2 (129 MB); no flush" % (wl["n"] * wl["dim"] * 4 / 1e6)
            if wl["n"] * wl["dim"] * 4 > 129e6 else "inputs smaller than L2; no flush",
            "step": "ct_build + eps_graph_query + csr_free"}


def clouds_config(args, wl, world):
    prec, learned, upper = form_opts(args.form)
    specs = wl["specs"]
    return {"workload": args.workload, "clouds": len(specs), "points": sum(sp["n"] for sp in specs),
            "dims": sorted(set(sp["dim"] for sp in specs)), "form": args.form,
            "precision": prec, "learned": learned, "upper_triangle": upper, "zeta": wl.get("zeta", 32),
            "parallelism": "replicas%d" % world if world > 1 else "single",
            "l2": "inputs (%.0f MB) larger than L2 (129 MB); no flush"
                  % (sum(sp["n"] * sp["dim"] * 4 for sp in specs) / 1e6),
            "step": "ct_build of every cloud + eps_graph_query_batched + csr_free"}


# ------------------------------------------------------------------ roofline

def roofline(prof: dict, st: dict, wl: dict, workload: str, peaks: dict, dim: int, mean_len=None):
    """Roofline of the count pass's leaf kernel, by the rules of each path:
    tensor-core tiles: 2 D flops per candidate pair against the dense f16/bf16
    tensor peak (sustained: the kernel runs inside a long step); FP32 tiles:
    3 D flops per pair against the FP32 lanes; edit distance: 17 64-bit word
    operations per pattern word per text character against the INT32 lanes
    (two 32-bit operations per word operation)."""
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    stage = {k: v for k, v in prof.items() if k not in ("build",)}
    dom = max(stage, key=lambda k: stage[k][0]) if stage else None
    if "leaf_count_tc" in prof:
        t = prof["leaf_count_tc"][0] / prof["leaf_count_tc"][1] / 1e3
        flops = st["leaf_pairs"] * 2.0 * dim
        peak = peaks.get("bf16_tflops_sustained", 1700.0)
        ach = flops / t / 1e12
        traffic = profile_value("k_leaf_tc", workload, "dram_bytes_per_launch")
        kp = 64 * ((((dim + 3) // 4) * 4 + 63) // 64)
        nbytes = st["leaf_rows"] * (2.0 * kp + 4.0) + st["recheck_fp32"] * 4.0 * dim
        return {"kernel": "k_leaf_tc", "bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": traffic,
                "peak_note": ("measured cuBLAS bf16 sustained (MEASURED_PEAKS.json); fp16 operands run at the "
                              "same dense rate" if peaks else "fallback 1.7 PFLOP/s sustained"),
                "flops_rule": "leaf_pairs x 2 x dim (every (query, candidate point) pair of the MMA tiles)",
                "flops_per_launch": flops, "ms_per_launch": t * 1e3,
                "dram_gbs": traffic / t / 1e9 if traffic else None,
                "dram_frac": traffic / t / 1e9 / peaks.get("hbm_gbs", 6800.0) if traffic else None,
                "l2_served_bytes_per_launch": nbytes,
                "l2_served_rule": "leaf_rows x (2 kp + 4) B (fp16 rows and norms) + recheck_fp32 x 4 dim B",
                "recheck_fp32_pairs": st["recheck_fp32"], "dominant_stage": dom}
    if "leaf_count" in prof and wl.get("kind") == "bits":
        t = prof["leaf_count"][0] / prof["leaf_count"][1] / 1e3
        words = 4 * ((wl["bits"] + 127) // 128)                   # 32-bit words per row (padded)
        ops = st["leaf_pairs"] * float(words)                       # one population count per word
        peak = SMS * 16 * sm_max * 1e6 / 1e12                      # T popc/s
        ach = ops / t / 1e12
        return {"kernel": "k_leaf_ham<count>", "bound": "alu", "achieved": ach, "peak": peak,
                "unit": "Tpopc/s", "frac": ach / peak,
                "traffic": profile_value("k_leaf_ham_count", workload, "dram_bytes_per_launch"),
                "peak_note": "derived: 152 SMs x 16 32-bit population counts per clock x %.0f MHz (the "
                             "population-count rate of the SM's integer pipe, 16 per clock)" % sm_max,
                "ops_rule": "leaf_pairs x 32-bit words per row (%d)" % words,
                "ops_per_launch": ops, "ms_per_launch": t * 1e3, "dominant_stage": dom}
    if "leaf_count" in prof and wl.get("kind") != "dna":
        t = prof["leaf_count"][0] / prof["leaf_count"][1] / 1e3
        peak = 2.0 * SMS * FP32_LANES * sm_max * 1e6 / 1e12
        flops = st["leaf_pairs"] * 3.0 * dim
        ach = flops / t / 1e12
        return {"kernel": "k_leaf_l2<count>", "bound": "alu", "achieved": ach, "peak": peak,
                "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": profile_value("k_leaf_l2_count", workload, "dram_bytes_per_launch"),
                "peak_note": "derived: 152 SMs x 128 FP32 lanes x 2 flop x %.0f MHz; direct differences "
                             "(sub+mul+add) can reach at most 0.75 of it" % sm_max,
                "flops_rule": "leaf_pairs x 3 x dim", "flops_per_launch": flops, "ms_per_launch": t * 1e3,
                "dominant_stage": dom}
    if "leaf_count" in prof:
        t = prof["leaf_count"][0] / prof["leaf_count"][1] / 1e3
        ops = st["lev_columns"] * 17.0                              # 64-bit word operations
        peak = SMS * INT32_LANES * sm_max * 1e6 / 2.0 / 1e12       # T word-ops/s
        ach = ops / t / 1e12
        return {"kernel": "k_leaf_lev<count>", "bound": "alu", "achieved": ach, "peak": peak,
                "unit": "Tword-op/s", "frac": ach / peak,
                "traffic": profile_value("k_leaf_lev_count", workload, "dram_bytes_per_launch"),
                "peak_note": "derived: 152 SMs x 64 INT32 lanes x %.0f MHz / 2 (a 64-bit word operation is "
                             "two 32-bit ones)" % sm_max,
                "ops_rule": "lev_columns (text characters processed x pattern words, counted by the kernel: "
                            "pairs that stop early count what they ran) x 17 word-ops per column",
                "full_recurrence_ops_per_launch": st["leaf_pairs"] * 17.0 * math.ceil(mean_len / 64.0) * mean_len,
                "ops_per_launch": ops, "ms_per_launch": t * 1e3, "dominant_stage": dom}
    return None


def traversal_roofline(prof: dict, st: dict, n: int, dim: int, workload: str, peaks: dict):
    """The walk's algorithmic bytes (per vertex test: 4 D of centre + 16 B of
    vertex record; per query: 4 D to read it) per unit time, and its DRAM
    bytes from the committed ncu summary, against the measured HBM copy
    bandwidth."""
    if "traverse" not in prof:
        return None
    t = prof["traverse"][0] / prof["traverse"][1] / 1e3
    nbytes = st["traversal_evals"] * (4.0 * dim + 16.0) + n * 4.0 * dim
    hbm = peaks.get("hbm_gbs", 6800.0)
    dram = profile_value("k_traverse_l2", workload, "dram_bytes_per_query")
    return {"kernel": "k_traverse_l2", "bound": "hbm", "ms_per_query": t * 1e3,
            "algorithmic_gbs": nbytes / t / 1e9, "algorithmic_frac": nbytes / t / 1e9 / hbm,
            "dram_gbs": dram / t / 1e9 if dram else None, "dram_frac": dram / t / 1e9 / hbm if dram else None,
            "peak": hbm, "unit": "GB/s", "bytes_rule": "traversal_evals x (4 dim + 16) B + n x 4 dim B"}


# ------------------------------------------------------------------ native

def csr_equal(a, b) -> bool:
    """Exact equality of two device CSRs: row_ptr, col and dist bit for bit."""
    import torch
    return (a.nnz == b.nnz and torch.equal(a.row_ptr, b.row_ptr) and torch.equal(a.col, b.col)
            and torch.equal(a.dist.view(torch.int32), b.dist.view(torch.int32)))


def run_single(args, wl, world, rank, dist):
    import torch
    from paper_2510_14147_gb300 import ctgraph as cg
    kind, host = load_input(wl)
    n = n_of(kind, host)
    dim = host.shape[1] if kind == "points" else 0
    mean_len = float(np.diff(host[1]).mean()) if kind == "strings" else None
    if kind == "points":
        dev = torch.from_numpy(host).cuda()
        build = lambda stream, d=None: cg.ct_build(points=dev if d is None else d, leaf_size=zeta, stream=stream)
    elif kind == "bits":
        dev = torch.from_numpy(host[0]).cuda()
        build = lambda stream, d=None: cg.ct_build(bits=(dev if d is None else d, host[1]), leaf_size=zeta,
                                                   stream=stream)
    else:
        dev = (torch.from_numpy(host[0]).cuda(), torch.from_numpy(host[1]).cuda())
        build = lambda stream, d=None: cg.ct_build(strings=dev if d is None else d, leaf_size=zeta, stream=stream)
    stream = torch.cuda.Stream()
    eps, zeta = wl["eps"], wl.get("zeta", 32)
    precision, learned, upper = form_opts(args.form)

    last = {}
    pred = None
    fit_info = None
    need_pred = learned or (not args.no_compare)
    if need_pred:
        # fitted once, outside the timed region, on another draw of the recipe
        kf, hf = load_input(dict(wl, seed=wl["seed"] + 1))
        if kf == "points":
            df = torch.from_numpy(hf).cuda()
            mk = lambda: cg.ct_build(points=df, leaf_size=zeta, stream=stream)
        elif kf == "bits":
            df = torch.from_numpy(hf[0]).cuda()
            mk = lambda: cg.ct_build(bits=(df, hf[1]), leaf_size=zeta, stream=stream)
        else:
            df = (torch.from_numpy(hf[0]).cuda(), torch.from_numpy(hf[1]).cuda())
            mk = lambda: cg.ct_build(strings=df, leaf_size=zeta, stream=stream)
        with torch.cuda.stream(stream):
            tf = mk()
            pred = cg.ct_predictor_create(seed=1)
            t0 = time.perf_counter()
            loss = cg.ct_predictor_fit(pred, tf, eps, steps=args.fit_steps, seed=2, stream=stream)
            fit_s = time.perf_counter() - t0
            tf.free()
            if args.order_radius:
                cg.ct_predictor_set_order(pred, False)
        del df
        fit_info = {"fit_on": "another draw of the recipe (seed %d)" % (wl["seed"] + 1),
                    "fit_steps": args.fit_steps, "final_loss": loss, "fit_s": fit_s,
                    "walk_order": "radius" if args.order_radius else "predicted walk length"}

    flush = None
    if kind in ("strings", "bits"):   # inputs smaller than L2: written over before every timed step
        flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")

    def step(prec=precision, use_pred=learned, keep=False, up=upper):
        if flush is not None:
            flush.fill_(1.0)
        t = build(stream)
        c = cg.eps_graph_query(t, eps, precision=prec, stream=stream, use_predictor=use_pred,
                               predictor=pred if use_pred else None, upper_triangle=up)
        last["nnz"] = c.nnz
        last["stats"] = c.stats()
        t.free()
        if keep:
            return c
        c.free()
        return c.nnz

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    barrier()

    sampler = ClockSampler(gpu_identifier(torch, torch.cuda.current_device()))
    if rank == 0:
        sampler.start()
    cg.ct_profile_reset()
    cg.ct_profile_enable(True)
    l0 = cg.ct_kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    sampler.mark("t0")
    e0.record(stream)
    nnz_total = 0
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            nnz_total += step()
    e1.record(stream)
    barrier()
    sampler.mark("t1")
    launches = cg.ct_kernel_launches() - l0
    cg.ct_profile_enable(False)
    prof = cg.ct_profile_read()
    clocks = sampler.stop() if rank == 0 else None
    t_ms, nnz_total = combine_ranks(e0.elapsed_time(e1), nnz_total, dist)
    value = nnz_total / (t_ms / 1e3)
    st = last["stats"]
    nnz = last["nnz"]

    # the other forms on the same input: time, stage times, and their whole
    # CSR against the default form's
    forms = None
    if not args.no_compare:
        forms = {}
        with torch.cuda.stream(stream):
            ref = step(keep=True)
        names = ["plain", "learned"] if kind in ("strings", "bits") else ["plain", "tc", "learned", "tc+learned"]
        names = names + [nm + "+upper" for nm in names]
        for name in names:
            if name == args.form:
                continue
            pf, lf, uf = form_opts(name)
            with torch.cuda.stream(stream):
                c = step(pf, lf, keep=True, up=uf)
                same = csr_equal(c, ref)
                c.free()
                step(pf, lf, up=uf)
            barrier()
            cg.ct_profile_reset()
            cg.ct_profile_enable(True)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            tot = 0
            with torch.cuda.stream(stream):
                for _ in range(args.steps):
                    tot += step(pf, lf, up=uf)
            b.record(stream)
            barrier()
            cg.ct_profile_enable(False)
            fp = cg.ct_profile_read()
            tp, tot = combine_ranks(a.elapsed_time(b), tot, dist)
            forms[name] = {"value": tot / (tp / 1e3), "ms_per_step": tp / args.steps,
                           "csr_identical_to_default_form": bool(same),
                           "stage_ms": {k: v[0] / max(v[1], 1) for k, v in fp.items()},
                           "speedup_of_default_form": value / (tot / (tp / 1e3))}
            if not same:
                raise RuntimeError("form %s produced a different CSR than %s" % (name, args.form))
        ref.free()

    # several radii over one tree (Table I's three radii per dataset): three
    # independent queries against one eps_graph_query_sweep, tree built once
    sweep = None
    radii = SWEEPS.get(args.workload)
    if radii and not args.no_sweep:
        wls = I.load_workloads()
        reps = [wls[k]["eps"] for k in radii]
        with torch.cuda.stream(stream):
            t = build(stream)
            ind = [cg.eps_graph_query(t, e, precision=precision, stream=stream, use_predictor=learned,
                                      predictor=pred, upper_triangle=upper) for e in reps]
            sw = cg.eps_graph_query_sweep(t, reps, precision=precision, stream=stream, use_predictor=learned,
                                          predictor=pred, upper_triangle=upper)
            same = all(csr_equal(a, b) for a, b in zip(ind, sw))
            sw_nnz = [c.nnz for c in sw]
            for c in ind + sw:
                c.free()
        if not same:
            raise RuntimeError("the radius sweep differs from independent queries")
        times = {}
        for mode in ("independent", "sweep"):
            barrier()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            with torch.cuda.stream(stream):
                for _ in range(args.steps):
                    if mode == "sweep":
                        cs = cg.eps_graph_query_sweep(t, reps, precision=precision, stream=stream,
                                                      use_predictor=learned, predictor=pred, upper_triangle=upper)
                    else:
                        cs = [cg.eps_graph_query(t, e, precision=precision, stream=stream, use_predictor=learned,
                                                 predictor=pred, upper_triangle=upper) for e in reps]
                    for c in cs:
                        c.free()
            b.record(stream)
            barrier()
            times[mode] = a.elapsed_time(b) / args.steps
        t.free()
        sweep = {"radii": dict(zip(radii, reps)), "nnz": dict(zip(radii, sw_nnz)),
                 "csr_identical_to_independent_queries": bool(same),
                 "ms_independent": times["independent"], "ms_sweep": times["sweep"],
                 "edges_per_s_sweep": sum(sw_nnz) / (times["sweep"] / 1e3),
                 "speedup": times["independent"] / times["sweep"],
                 "note": "one tree, built once outside the timed region; queries of the form above"}

    # the landmark form (Voronoi cells of m random centres, Lemma 1 ghosts, a
    # tree per cell, one batched query) against the step above, same form
    landmark = None
    if kind == "points" and not args.no_landmark:
        m = args.landmark_m
        centres = np.random.default_rng(60).choice(n, size=m, replace=False)
        lm_kw = dict(points=dev, leaf_size=zeta, precision=precision, use_predictor=learned,
                     predictor=pred if learned else None, upper_triangle=upper, stream=stream)
        with torch.cuda.stream(stream):
            ref = step(keep=True)
            c, info = cg.eps_graph_query_landmark(centres, eps, **lm_kw)
            same = csr_equal(c, ref)
            c.free()
            ref.free()
        if not same:
            raise RuntimeError("the landmark form's CSR differs from the query's")
        barrier()
        cg.ct_profile_reset()
        cg.ct_profile_enable(True)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        with torch.cuda.stream(stream):
            for _ in range(args.steps):
                cg.eps_graph_query_landmark(centres, eps, **lm_kw)[0].free()
        b.record(stream)
        barrier()
        cg.ct_profile_enable(False)
        lp = cg.ct_profile_read()
        tl = a.elapsed_time(b) / args.steps
        landmark = {"m": m, "centres": "uniform random points (seed 60)", "ms_per_step": tl,
                    "value": nnz / (tl / 1e3), "csr_identical_to_default_form": bool(same),
                    "stage_ms": {k: v[0] / max(v[1], 1) for k, v in lp.items()}, "partition": info,
                    "speedup_over_one_tree": (t_ms / args.steps) / tl}

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        if kind == "points":
            hin = [torch.from_numpy(host).pin_memory()]
        elif kind == "bits":
            hin = [torch.from_numpy(host[0]).pin_memory()]
        else:
            hin = [torch.from_numpy(host[0]).pin_memory(), torch.from_numpy(host[1]).pin_memory()]
        din = [torch.empty_like(h, device="cuda") for h in hin]
        rp_h = torch.empty(n + 1, dtype=torch.int64).pin_memory()
        col_h = torch.empty(max(nnz, 1), dtype=torch.int32).pin_memory()
        dist_h = torch.empty(max(nnz, 1), dtype=torch.float32).pin_memory()

        def e2e_step():
            for d, h in zip(din, hin):
                d.copy_(h, non_blocking=True)
            t = build(stream, din[0] if kind in ("points", "bits") else (din[0], din[1]))
            c = cg.eps_graph_query(t, eps, precision=precision, stream=stream,
                                   use_predictor=learned, predictor=pred, upper_triangle=upper)
            rp_h.copy_(c.row_ptr, non_blocking=True)
            col_h[:c.nnz].copy_(c.col, non_blocking=True)
            dist_h[:c.nnz].copy_(c.dist, non_blocking=True)
            stream.synchronize()
            k = c.nnz
            c.free()
            t.free()
            return k

        with torch.cuda.stream(stream):
            for _ in range(args.warmup):   # fresh pinned buffers copy slowly at first
                e2e_step()
            barrier()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            tot = 0
            for _ in range(args.steps):
                tot += e2e_step()
            b.record(stream)
        barrier()
        te, tot = combine_ranks(a.elapsed_time(b), tot, dist)
        e2e = {"value": tot / (te / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": int(sum(h.numel() * h.element_size() for h in hin)),
               "d2h_bytes_per_step": int((n + 1) * 8 + nnz * 8), "ms_per_step": te / args.steps}

    stage_ms = {k: v[0] / max(v[1], 1) for k, v in prof.items()}
    peaks = measured_peaks()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32" if kind in ("strings", "bits") else "f32",
            "data": "synthetic", "config": config_of(args, wl, world), "nnz": nnz, "edges_undirected": nnz // 2,
            "dist_evals_per_s": (st["traversal_evals"] + st["leaf_pairs"]) * world * args.steps / (t_ms / 1e3),
            "query_stats": st, "stage_ms": stage_ms,
            "roofline": roofline(prof, st, wl, args.workload, peaks, dim, mean_len),
            "traversal": traversal_roofline(prof, st, n, dim, args.workload, peaks) if kind == "points" else None,
            "e2e": e2e, "gpu_launches": launches, "clocks": clocks, "library": cg.library_path(),
            "forms": forms, "sweep": sweep, "landmark": landmark}
    if fit_info:
        line["learned"] = fit_info
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            if kind == "bits":
                line["cpu_baseline"] = oracle_rows_sample(kind, host, wl, args.ref_queries // 20)
            else:
                line["cpu_baseline"] = oracle_sample(kind, host, wl, args.ref_queries)
        except Exception as e:  # reported, never silently replaced
            line["cpu_baseline"] = {"error": str(e)}
    if rank == 0:
        print(json.dumps(line))
    return 0


def run_clouds(args, wl, world, rank, dist):
    """Many clouds per step: every cloud's tree is built, then one batched
    query over all of them; value = all clouds' edges / step time."""
    import torch
    from paper_2510_14147_gb300 import ctgraph as cg
    precision, learned, upper = form_opts(args.form)
    specs = wl["specs"]
    hosts = [I.cloud_points(sp) for sp in specs]
    xs = [torch.from_numpy(x).cuda() for x in hosts]
    eps = [sp["eps"] for sp in specs]
    zeta = wl.get("zeta", 32)
    stream = torch.cuda.Stream()
    pred = None
    fit_info = None
    if learned:
        # one predictor for every cloud, fitted outside the timed region on
        # another draw of three clouds of the recipe (a uniform and two mixtures)
        fit_specs = [dict(sp, seed=sp["seed"] + 100000) for sp in specs[:3]]
        with torch.cuda.stream(stream):
            pred = cg.ct_predictor_create(seed=1)
            t0 = time.perf_counter()
            loss = None
            for sp in fit_specs:
                tf = cg.ct_build(points=torch.from_numpy(I.cloud_points(sp)).cuda(), leaf_size=zeta, stream=stream)
                loss = cg.ct_predictor_fit(pred, tf, sp["eps"], steps=args.fit_steps // len(fit_specs) or 1,
                                           seed=2, stream=stream)
                tf.free()
            fit_info = {"fit_on": "another draw of clouds 0-2 of the recipe", "final_loss": loss,
                        "fit_s": time.perf_counter() - t0}
    last = {}

    def step(prec, use_pred, keep=False, src=None, up=upper):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        trees = [cg.ct_build(points=x, leaf_size=zeta, stream=stream) for x in (src or xs)]
        e[1].record(stream)
        csrs = cg.eps_graph_query_batched(trees, eps, precision=prec, stream=stream,
                                          use_predictor=use_pred, predictor=pred if use_pred else None,
                                          upper_triangle=up)
        e[2].record(stream)
        nnz = sum(c.nnz for c in csrs)
        last["stats"] = [c.stats() for c in csrs]
        last["events"] = e
        for t in trees:
            t.free()
        if keep:
            return csrs
        for c in csrs:
            c.free()
        return nnz

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    tuned = None
    if precision == 2:  # autotune the count kernels on these clouds, outside the timed region
        with torch.cuda.stream(stream):
            trees = [cg.ct_build(points=x, leaf_size=zeta, stream=stream) for x in xs]
            t0 = time.perf_counter()
            ch = cg.ct_autotune(trees, eps, stream=stream)
            tuned = {"tc_clouds": int(sum(ch)), "fp32_clouds": len(ch) - int(sum(ch)),
                     "tune_s": time.perf_counter() - t0}
            for t in trees:
                t.free()
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step(precision, learned)
    barrier()
    sampler = ClockSampler(gpu_identifier(torch, torch.cuda.current_device()))
    if rank == 0:
        sampler.start()
    cg.ct_profile_reset()
    cg.ct_profile_enable(True)
    l0 = cg.ct_kernel_launches()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    build_ms = query_ms = 0.0
    barrier()
    sampler.mark("t0")
    a.record(stream)
    tot = 0
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            tot += step(precision, learned)
    b.record(stream)
    barrier()
    sampler.mark("t1")
    launches = cg.ct_kernel_launches() - l0
    cg.ct_profile_enable(False)
    prof = cg.ct_profile_read()
    clocks = sampler.stop() if rank == 0 else None
    t_ms, tot = combine_ranks(a.elapsed_time(b), tot, dist)
    value = tot / (t_ms / 1e3)
    st = last["stats"][0]          # a batch reports its counters once, for all its clouds
    ev = last["events"]
    build_ms, query_ms = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])

    forms = None
    if not args.no_compare:
        forms = {}
        with torch.cuda.stream(stream):
            ref = step(precision, learned, keep=True)
        for name in ("plain",):
            if name == args.form:
                continue
            pf, lf, uf = form_opts(name)
            with torch.cuda.stream(stream):
                cs = step(pf, lf, keep=True, up=uf)
                same = all(csr_equal(x, y) for x, y in zip(cs, ref))
                for c in cs:
                    c.free()
            barrier()
            a2, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a2.record(stream)
            tp = 0
            with torch.cuda.stream(stream):
                for _ in range(args.steps):
                    tp += step(pf, lf, up=uf)
            b2.record(stream)
            barrier()
            tpm, tp = combine_ranks(a2.elapsed_time(b2), tp, dist)
            forms[name] = {"value": tp / (tpm / 1e3), "ms_per_step": tpm / args.steps,
                           "csr_identical_to_default_form": bool(same),
                           "speedup_of_default_form": value / (tp / (tpm / 1e3))}
            if not same:
                raise RuntimeError("form %s produced a different CSR than %s" % (name, args.form))
        for c in ref:
            c.free()

    # the same batch as a plan (buffers sized once, one persistent leaf launch
    # over a device work queue, replayed from a CUDA graph) against the batched
    # query and the sum of the single-cloud queries, on the same trees
    plan_info = None
    if not args.no_plan:
        with torch.cuda.stream(stream):
            trees = [cg.ct_build(points=x, leaf_size=zeta, stream=stream) for x in xs]
        opts = dict(precision=precision, use_predictor=learned, predictor=pred if learned else None, stream=stream,
                    upper_triangle=upper)

        def timed(fn, reps):
            barrier()
            a4, b4 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a4.record(stream)
            with torch.cuda.stream(stream):
                for _ in range(reps):
                    fn()
            b4.record(stream)
            barrier()
            return a4.elapsed_time(b4) / reps

        def singles():
            for t, e in zip(trees, eps):
                cg.eps_graph_query(t, e, **opts).free()

        def batched():
            for c in cg.eps_graph_query_batched(trees, eps, **opts):
                c.free()

        t0 = time.perf_counter()
        plan = cg.ct_plan_create(trees, eps, margin=0.05, use_graph=True, **opts)
        t_plan = time.perf_counter() - t0
        with torch.cuda.stream(stream):
            ref = cg.eps_graph_query_batched(trees, eps, **opts)
            cg.ct_plan_launch(plan, stream=stream)
            outs = cg.ct_plan_result(plan, stream=stream)
            same = all(csr_equal(x, y) for x, y in zip(outs, ref))
            for c in ref:
                c.free()
        if not same:
            raise RuntimeError("the plan's CSRs differ from the batched query's")
        reps = max(1, min(args.steps, 3))
        l1 = cg.ct_kernel_launches()
        ms_plan = timed(lambda: cg.ct_plan_launch(plan, stream=stream), reps)
        with torch.cuda.stream(stream):
            cg.ct_plan_result(plan, stream=stream)
        plan_launches = (cg.ct_kernel_launches() - l1) // reps
        ms_batched = timed(batched, reps)
        ms_singles = timed(singles, 1)
        plan_info = {"ms_graph_replay": ms_plan, "ms_batched_query": ms_batched,
                     "ms_sum_of_single_cloud_queries": ms_singles, "create_s": t_plan,
                     "csr_identical_to_batched_query": bool(same),
                     "host_launch_calls_per_replay": plan_launches,
                     "note": "query only (trees built once outside); the plan's leaf tiles are the FP32 ones"}
        plan.free()
        for t in trees:
            t.free()

    e2e = None
    if not args.no_e2e:
        hin = [torch.from_numpy(x).pin_memory() for x in hosts]
        din = [torch.empty_like(h, device="cuda") for h in hin]
        nn = [x.shape[0] for x in hosts]
        caps = {}

        def e2e_step():
            for d, h in zip(din, hin):
                d.copy_(h, non_blocking=True)
            cs = step(precision, learned, keep=True, src=din)
            outs = []
            for i, c in enumerate(cs):
                need = (c.nnz, nn[i])
                if caps.get(i, (-1, -1))[0] < c.nnz:
                    caps[i] = (c.nnz, torch.empty(max(c.nnz, 1), dtype=torch.int32).pin_memory(),
                               torch.empty(max(c.nnz, 1), dtype=torch.float32).pin_memory(),
                               torch.empty(nn[i] + 1, dtype=torch.int64).pin_memory())
                _, ch, dh, rh = caps[i]
                rh.copy_(c.row_ptr, non_blocking=True)
                ch[:c.nnz].copy_(c.col, non_blocking=True)
                dh[:c.nnz].copy_(c.dist, non_blocking=True)
                outs.append(need)
            stream.synchronize()
            k = sum(c.nnz for c in cs)
            for c in cs:
                c.free()
            return k

        with torch.cuda.stream(stream):
            for _ in range(args.warmup):   # fresh pinned buffers copy slowly at first
                e2e_step()
            barrier()
            a3, b3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a3.record(stream)
            te_tot = 0
            for _ in range(args.steps):
                te_tot += e2e_step()
            b3.record(stream)
        barrier()
        te, te_tot = combine_ranks(a3.elapsed_time(b3), te_tot, dist)
        nnz_step = te_tot // max(args.steps, 1) // max(world, 1)
        e2e = {"value": te_tot / (te / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": int(sum(x.nbytes for x in hosts)),
               "d2h_bytes_per_step": int(sum((m + 1) * 8 for m in nn) + nnz_step * 8),
               "ms_per_step": te / args.steps}

    peaks = measured_peaks()
    roof = roofline(prof, st, wl, args.workload, peaks, max(sp["dim"] for sp in specs))
    if roof:
        roof["note"] = ("a batch mixes dims 3/16/64: the flop count takes the largest dim for every pair of the "
                        "launch (an upper bound on the work)")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": clouds_config(args, wl, world),
            "nnz": tot // max(args.steps, 1) // world, "query_stats": st,
            "stage_ms": dict({k: v[0] / max(v[1], 1) for k, v in prof.items()},
                             build_all=build_ms, query_batched=query_ms),
            "roofline": roof, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
            "library": cg.library_path(), "forms": forms, "autotune": tuned, "plan": plan_info}
    if fit_info:
        line["learned"] = fit_info
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            line["cpu_baseline"] = oracle_clouds_sample(specs, args.ref_queries // 40)
        except Exception as e:
            line["cpu_baseline"] = {"error": str(e)}
    if rank == 0:
        print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="gmm_1m_k70")
    ap.add_argument("--form", default=None, choices=sorted(FORMS),
                    help="plain: FP32 two-pass; tc: tensor-core filter (fp16 rows); learned: one-pass emit "
                         "sized by the predictor; tc+learned: both; auto: the autotuned count kernel")
    ap.add_argument("--no-compare", action="store_true", help="skip timing the other forms beside it")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-queries", type=int, default=4000)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-sweep", action="store_true", help="skip timing the three-radius sweep")
    ap.add_argument("--no-plan", action="store_true", help="clouds: skip timing the plan (graph replay)")
    ap.add_argument("--no-landmark", action="store_true", help="skip timing the landmark form")
    ap.add_argument("--landmark-m", type=int, default=60, help="landmark centres (the paper's m = 60)")
    ap.add_argument("--fit-steps", type=int, default=1500)
    ap.add_argument("--order-radius", action="store_true",
                    help="learned forms: walk groups by radius instead of predicted walk length")
    args = ap.parse_args()
    wl = I.load_workloads()[args.workload]
    if args.form is None:
        args.form = "auto+learned+upper" if wl["kind"] == "clouds" else default_form(wl)

    if args.impl == "reference":
        return run_reference(args, wl)

    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2510_14147_gb300 import build as libbuild
    if rank == 0 or world == 1:
        libbuild.build()
    if dist:
        dist.barrier()

    if wl["kind"] == "clouds":
        rc = run_clouds(args, wl, world, rank, dist)
    else:
        rc = run_single(args, wl, world, rank, dist)
    if dist:
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
