#!/usr/bin/env python
"""ε-graph benchmark: one step = cover-tree build + exact ε query (count ->
scan -> emit -> row sort) of one synthetic point cloud, resident in HBM.

Default workload: 1,000,000 points, 128-D, 100-component Gaussian mixture in
8-D embedded in 128-D, eps calibrated for ~70 mean neighbours (the paper's
sift eps=175 shape).  Prints ONE JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
                  [--workload gmm_1m_k70] [--form tc+learned|tc|learned|plain]
                  [--no-compare] [--no-cpu-baseline] [--no-e2e]

The default form is the tensor-core-filtered, learned one; the plain FP32 two-pass
form is timed beside it on the same input ("plain" in the JSON line).

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
SMS, FP32_LANES = 152, 128          # GB300: 152 SMs x 128 FP32 lanes
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


def load_points(wl: dict) -> np.ndarray:
    if wl["kind"] == "gmm":
        return I.gmm_embedded(wl["n"], dim=wl["dim"], seed=wl["seed"])
    if wl["kind"] == "uniform":
        return I.uniform_cube(wl["n"], wl["dim"], seed=wl["seed"])
    raise ValueError("workload %s has no point cloud" % wl)


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


def profile_traffic(kernel: str, workload: str):
    """DRAM bytes per launch of `kernel` from a committed ncu summary, or None."""
    path = os.path.join(PROFILES, "%s__%s.txt" % (kernel, workload))
    if not os.path.exists(path):
        return None
    for line in open(path):
        m = re.match(r"\s*dram_bytes_per_launch\s*[:=]\s*([0-9.eE+]+)", line)
        if m:
            return float(m.group(1))
    return None


# --------------------------------------------------------------- CPU oracle

def oracle_sample(x: np.ndarray, wl: dict, n_queries: int, seed: int = 7):
    """Oracle cover tree (Algorithms 1-3, FP64) built on every point, queried
    for a random sample of points; extrapolated to all n queries."""
    import oracle
    oracle.build()
    sp = oracle.Space(points=x)
    t0 = time.perf_counter()
    tree = oracle.build_tree(sp, zeta=wl.get("zeta", 32))
    t_build = time.perf_counter() - t0
    rng = np.random.default_rng(seed)
    rows = np.sort(rng.choice(x.shape[0], size=min(n_queries, x.shape[0]), replace=False))
    t0 = time.perf_counter()
    res = oracle.tree_query_rows(sp, tree, wl["eps"], rows)
    t_query = time.perf_counter() - t0
    scale = x.shape[0] / rows.size
    edges = float(res["row_ptr"][-1]) * scale
    t_total = t_build + t_query * scale
    evals = (tree.dist_evals + res["dist_evals"] * scale)
    return {"value": edges / t_total, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": "oracle tree built on all %d points (%.1f s); %d random queries (%.1f s) "
                      "extrapolated to %d queries" % (x.shape[0], t_build, rows.size, t_query, x.shape[0]),
            "dist_evals_per_s": evals / t_total, "wall_s": t_build + t_query,
            "extrapolated_s": t_total}


def run_reference(args, wl):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    x = load_points(wl)
    nq = args.ref_queries
    for _ in range(args.warmup):
        oracle_sample(x, wl, nq, seed=11)
    vals, walls, ext = [], [], []
    for k in range(args.steps):
        r = oracle_sample(x, wl, nq, seed=100 + k)
        vals.append(r["value"] * r["extrapolated_s"])
        walls.append(r["wall_s"])
        ext.append(r["extrapolated_s"])
        last = r
    value = sum(vals) / sum(ext)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(walls) / len(walls),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(args, wl, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": last["cores"], "kind": "oracle",
                             "sample": last["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


FORMS = {"plain": (0, False), "tc": (1, False), "learned": (0, True), "tc+learned": (1, True),
         "auto": (2, False), "auto+learned": (2, True)}


def run_clouds(args, wl, world, rank, dist):
    """Many clouds per step: every cloud's tree is built, then one batched
    query over all of them; value = all clouds' edges / step time."""
    import torch
    from paper_2510_14147_gb300 import ctgraph as cg
    precision, learned = FORMS[args.form]
    specs = wl["specs"]
    xs = [torch.from_numpy(I.cloud_points(sp)).cuda() for sp in specs]
    eps = [sp["eps"] for sp in specs]
    zeta = wl.get("zeta", 32)
    stream = torch.cuda.Stream()
    pred = None
    if learned:
        raise SystemExit("the learned form of the many-cloud batch is not available yet")
    last = {}

    def step(prec):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        trees = [cg.ct_build(points=x, leaf_size=zeta, stream=stream) for x in xs]
        e[1].record(stream)
        csrs = cg.eps_graph_query_batched(trees, eps, precision=prec, stream=stream,
                                          use_predictor=pred is not None, predictor=pred)
        e[2].record(stream)
        nnz = sum(c.nnz for c in csrs)
        last["stats"] = [c.stats() for c in csrs]
        last["events"] = e
        for c in csrs:
            c.free()
        for t in trees:
            t.free()
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
            step(precision)
    barrier()
    sampler = ClockSampler(gpu_identifier(torch, torch.cuda.current_device()))
    if rank == 0:
        sampler.start()
    l0 = cg.ct_kernel_launches()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    build_ms = query_ms = 0.0
    barrier()
    a.record(stream)
    tot = 0
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            tot += step(precision)
            ev = last["events"]
            ev[2].synchronize()
            build_ms += ev[0].elapsed_time(ev[1])
            query_ms += ev[1].elapsed_time(ev[2])
    b.record(stream)
    barrier()
    launches = cg.ct_kernel_launches() - l0
    clocks = sampler.stop() if rank == 0 else None
    t_ms, tot = combine_ranks(a.elapsed_time(b), tot, dist)
    value = tot / (t_ms / 1e3)
    st = last["stats"]
    plain = None
    if args.form != "plain" and not args.no_compare:
        with torch.cuda.stream(stream):
            step(0)
        barrier()
        a2, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a2.record(stream)
        tp = 0
        with torch.cuda.stream(stream):
            for _ in range(args.steps):
                tp += step(0)
        b2.record(stream)
        barrier()
        tpm = a2.elapsed_time(b2)
        plain = {"form": "plain", "value": tp * world / (tpm / 1e3), "ms_per_step": tpm / args.steps,
                 "speedup_of_form": value / (tp * world / (tpm / 1e3))}
    agg = {k: sum(x[k] for x in st) for k in st[0]}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "clouds": len(specs), "points": sum(sp["n"] for sp in specs),
                       "dims": sorted(set(sp["dim"] for sp in specs)), "form": args.form,
                       "precision": precision, "learned": learned, "zeta": zeta,
                       "parallelism": "replicas%d" % world if world > 1 else "single",
                       "step": "ct_build of every cloud + eps_graph_query_batched + csr_free"},
            "nnz": tot // max(args.steps, 1) // world, "query_stats": agg,
            "stage_ms": {"build_all": build_ms / args.steps, "query_batched": query_ms / args.steps},
            "gpu_launches": launches, "clocks": clocks, "plain": plain, "roofline": None, "e2e": None,
            "autotune": tuned}
    if rank == 0:
        print(json.dumps(line))
    return 0



def config_of(args, wl, world):
    prec, learned = FORMS[args.form]
    return {"workload": args.workload, "n": wl["n"], "dim": wl["dim"], "eps": wl["eps"],
            "zeta": wl.get("zeta", 32), "target_degree": wl.get("target_degree"),
            "form": args.form, "precision": prec, "learned": learned,
            "parallelism": "replicas%d" % world if world > 1 else "single",
            "l2": "inputs (%.0f MB) larger than L2 (129 MB); no flush" % (wl["n"] * wl["dim"] * 4 / 1e6),
            "step": "ct_build + eps_graph_query + csr_free"}


# ------------------------------------------------------------------ native

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="gmm_1m_k70")
    ap.add_argument("--form", default="tc+learned", choices=sorted(FORMS),
                    help="plain: FP32 two-pass; tc: tensor-core filter (fp16 rows); learned: one-pass emit "
                         "sized by the predictor; tc+learned: both")
    ap.add_argument("--no-compare", action="store_true", help="skip timing the plain form beside it")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-queries", type=int, default=4000)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--fit-steps", type=int, default=1500)
    ap.add_argument("--order-radius", action="store_true",
                    help="learned forms: walk groups by radius instead of predicted walk length")
    args = ap.parse_args()
    wl = I.load_workloads()[args.workload]
    precision, learned = FORMS[args.form]

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
    from paper_2510_14147_gb300 import ctgraph as cg

    if wl["kind"] == "clouds":
        rc = run_clouds(args, wl, world, rank, dist)
        if dist:
            dist.destroy_process_group()
        return rc

    x = load_points(wl)
    xd = torch.from_numpy(x).cuda()
    stream = torch.cuda.Stream()
    eps, zeta = wl["eps"], wl.get("zeta", 32)

    last = {}
    pred = None
    fit_info = None
    if learned:
        # fitted once, outside the timed region, on another draw of the recipe
        wl_fit = dict(wl, seed=wl["seed"] + 1)
        xf = torch.from_numpy(load_points(wl_fit)).cuda()
        with torch.cuda.stream(stream):
            tf = cg.ct_build(points=xf, leaf_size=zeta, stream=stream)
            pred = cg.ct_predictor_create(seed=1)
            t0 = time.perf_counter()
            loss = cg.ct_predictor_fit(pred, tf, eps, steps=args.fit_steps, seed=2, stream=stream)
            fit_s = time.perf_counter() - t0
            tf.free()
            if args.order_radius:
                cg.ct_predictor_set_order(pred, False)
        del xf
        fit_info = {"fit_on": "another draw of the recipe (seed %d)" % wl_fit["seed"],
                    "fit_steps": args.fit_steps, "final_loss": loss, "fit_s": fit_s,
                    "walk_order": "radius" if args.order_radius else "predicted walk length"}

    def step(points, prec=precision, use_pred=learned):
        t = cg.ct_build(points=points, leaf_size=zeta, stream=stream)
        c = cg.eps_graph_query(t, eps, precision=prec, stream=stream, use_predictor=use_pred,
                               predictor=pred if use_pred else None)
        last["nnz"] = c.nnz
        last["stats"] = c.stats()
        c.free()
        t.free()
        return c.nnz

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step(xd)
    barrier()

    sampler = ClockSampler(gpu_identifier(torch, local))
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
            nnz_total += step(xd)
    e1.record(stream)
    barrier()
    sampler.mark("t1")
    launches = cg.ct_kernel_launches() - l0
    cg.ct_profile_enable(False)
    prof = cg.ct_profile_read()
    clocks = sampler.stop() if rank == 0 else None
    rank_nnz = nnz_total
    t_ms, nnz_total = combine_ranks(e0.elapsed_time(e1), nnz_total, dist)
    value = nnz_total / (t_ms / 1e3)
    st = last["stats"]
    nnz = last["nnz"]

    # the plain form on the same input, for the comparison
    plain = None
    if args.form != "plain" and not args.no_compare:
        with torch.cuda.stream(stream):
            step(xd, 0, False)
        barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        tot = 0
        with torch.cuda.stream(stream):
            for _ in range(args.steps):
                tot += step(xd, 0, False)
        b.record(stream)
        barrier()
        if tot != rank_nnz:
            raise RuntimeError("plain form produced a different edge count")
        tp, tot = combine_ranks(a.elapsed_time(b), tot, dist)
        plain = {"form": "plain", "value": tot / (tp / 1e3), "ms_per_step": tp / args.steps,
                 "speedup_of_form": value / (tot / (tp / 1e3))}

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        xh = torch.from_numpy(x).pin_memory()
        xdev = torch.empty_like(xd)
        rp_h = torch.empty(wl["n"] + 1, dtype=torch.int64).pin_memory()
        col_h = torch.empty(max(nnz, 1), dtype=torch.int32).pin_memory()
        dist_h = torch.empty(max(nnz, 1), dtype=torch.float32).pin_memory()

        def e2e_step():
            xdev.copy_(xh, non_blocking=True)
            t = cg.ct_build(points=xdev, leaf_size=zeta, stream=stream)
            c = cg.eps_graph_query(t, eps, precision=precision, stream=stream,
                                   use_predictor=learned, predictor=pred)
            rp_h.copy_(c.row_ptr, non_blocking=True)
            col_h[:c.nnz].copy_(c.col, non_blocking=True)
            dist_h[:c.nnz].copy_(c.dist, non_blocking=True)
            stream.synchronize()
            k = c.nnz
            c.free()
            t.free()
            return k

        with torch.cuda.stream(stream):
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
               "h2d_bytes_per_step": int(x.nbytes),
               "d2h_bytes_per_step": int((wl["n"] + 1) * 8 + nnz * 8),
               "ms_per_step": te / args.steps}

    # roofline of the dominant kernel
    stage_ms = {k: v[0] / max(v[1], 1) for k, v in prof.items()}
    peaks = measured_peaks()
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    fp32_peak = 2.0 * SMS * FP32_LANES * sm_max * 1e6 / 1e12   # TFLOP/s, FMA = 2 flops
    kernel_stages = {k: v for k, v in prof.items() if k not in ("build",)}
    dom = max(kernel_stages, key=lambda k: kernel_stages[k][0]) if kernel_stages else None
    roof = None
    if "leaf_count_tc" in prof:
        # tensor-core form: 32 queries x 128 dims x 2 flops per 260-byte fp16
        # candidate row (+ norm) is 32 flop/B, far below the tensor ridge
        # (~250 flop/B): the tiles are bound by streaming the candidate rows
        # (and the original rows of the kept pairs), so the roofline is HBM
        t_launch = prof["leaf_count_tc"][0] / prof["leaf_count_tc"][1] / 1e3
        kp = 64 * ((((wl["dim"] + 3) // 4) * 4 + 63) // 64)  # fp16 row length (dp rounded up to 64)
        nbytes = st["leaf_rows"] * (2.0 * kp + 4.0) + st["recheck_fp32"] * 4.0 * wl["dim"]
        hbm = peaks.get("hbm_gbs", 6800.0)
        ach = nbytes / t_launch / 1e9
        roof = {"kernel": "k_leaf_tc", "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                "frac": ach / hbm, "traffic": profile_traffic("k_leaf_tc", args.workload),
                "peak_note": "measured copy bandwidth (MEASURED_PEAKS.json)" if peaks else "fallback 6.8 TB/s",
                "bytes_per_launch": nbytes,
                "bytes_rule": "leaf_rows x (2 kp + 4) B (fp16 candidate rows and norms, kp = dim rounded "
                              "up to 64) + recheck_fp32 x dim x 4 B (original candidate rows of kept pairs)",
                "ms_per_launch": t_launch * 1e3, "tensor_flops_per_launch": st["leaf_pairs"] * 2.0 * kp,
                "tensor_frac_of_sustained_f16": st["leaf_pairs"] * 2.0 * kp / t_launch / 1e12
                / peaks.get("bf16_tflops_sustained", 1700.0),
                "recheck_fp32_pairs": st["recheck_fp32"], "dominant_stage": dom}
    elif "leaf_count" in prof:
        t_launch = prof["leaf_count"][0] / prof["leaf_count"][1] / 1e3
        flops = st["leaf_pairs"] * 3.0 * wl["dim"]
        ach = flops / t_launch / 1e12
        roof = {"kernel": "k_leaf_l2<count>", "bound": "alu", "achieved": ach, "peak": fp32_peak,
                "unit": "TFLOP/s", "frac": ach / fp32_peak,
                "traffic": profile_traffic("k_leaf_l2_count", args.workload),
                "peak_note": "derived: 152 SMs x 128 FP32 lanes x 2 flop x %.0f MHz; direct "
                             "differences (sub+mul+add) can reach at most 0.75 of it" % sm_max,
                "flops_per_launch": flops, "ms_per_launch": t_launch * 1e3,
                "dominant_stage": dom}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config_of(args, wl, world), "nnz": nnz, "edges_undirected": nnz // 2,
            "dist_evals_per_s": (st["traversal_evals"] + st["leaf_pairs"]) * world * args.steps / (t_ms / 1e3),
            "query_stats": st, "stage_ms": stage_ms, "roofline": roof, "e2e": e2e,
            "gpu_launches": launches, "clocks": clocks, "library": cg.library_path(), "plain": plain}
    if fit_info:
        line["learned"] = fit_info
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            line["cpu_baseline"] = oracle_sample(x, wl, args.ref_queries)
        except Exception as e:  # reported, never silently replaced
            line["cpu_baseline"] = {"error": str(e)}
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
