"""Writes ``paper_2510_14147_gb300/workloads.json``: the workload table with the
radius ε of every L2 workload calibrated for a target mean degree.

Calibration (a reading of "ε tuned for ≈k mean neighbours"): draw Q query ids
with a seeded generator, take their FP64 distances to all n points, and set ε
to the ceil(k*Q)-th smallest non-self distance, rounded to fp32.  The squared
distances of the calibration sample are computed block-wise in FP64; ε is an
input parameter, so no result of the CUDA library enters it.

Run:  python -m oracle.calibrate_eps   (from the repository root; minutes)
"""
from __future__ import annotations

import json
import math
import os
import sys

import numpy as np

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, _ROOT)
from paper_2510_14147_gb300 import inputs as I  # noqa: E402

OUT = os.path.join(_ROOT, "paper_2510_14147_gb300", "workloads.json")


PROFILE_SIZE = {"kind": "gmm", "n": 300_000, "dim": 128, "seed": 0, "target_degree": 70.0, "zeta": 32,
                "note": "profiling size of the 1M generator (154 MB of points, above the 129 MB L2)"}


BASE = {
    "small_3d": {"kind": "uniform", "n": 2000, "dim": 3, "seed": 0, "eps": 0.08,
                 "zeta": 32, "note": "uniform [0,1]^3, eps=0.08"},
    "gmm_1m_k10": {"kind": "gmm", "n": 1_000_000, "dim": 128, "seed": 0,
                   "target_degree": 10.0, "zeta": 32,
                   "note": "same generator; sift eps=125 stand-in (the smallest radius of the sweep)"},
    "gmm_1m_k70": {"kind": "gmm", "n": 1_000_000, "dim": 128, "seed": 0,
                   "target_degree": 70.0, "zeta": 32,
                   "note": "100-component 8-D GMM embedded in 128-D; sift eps=175 stand-in"},
    "gmm_1m_k500": {"kind": "gmm", "n": 1_000_000, "dim": 128, "seed": 0,
                    "target_degree": 500.0, "zeta": 32,
                    "note": "same generator; sift eps=225 stand-in"},
    "ham_1m_256": {"kind": "bits", "n": 1_000_000, "bits": 256, "n_centres": 1000, "flip": 0.05, "seed": 0,
                   "target_degree": 70.0, "zeta": 32,
                   "note": "1M clustered 256-bit codes (1000 centres, 5% bit flips); sift-hamming stand-in"},
    "dna_50k": {"kind": "dna", "n_seeds": 500, "per_seed": 100, "seed_len": 96,
                "seed": 0, "eps": 8, "zeta": 32,
                "note": "Levenshtein; 4% substitution, 0.5% insertion, 0.5% deletion per site"},
}


def calibrate(x: np.ndarray, target_degree: float, n_queries: int = 4096, seed: int = 12345) -> float:
    n = x.shape[0]
    rng = np.random.Generator(np.random.PCG64(seed))
    q = np.sort(rng.choice(n, size=min(n_queries, n), replace=False))
    nq = q.size
    rank = int(math.ceil(target_degree * nq))
    keep = min(n - 1, max(256, 40 * int(math.ceil(target_degree))))
    x64 = x.astype(np.float64)
    sq = np.einsum("ij,ij->i", x64, x64)
    best = []
    exhausted = []
    for s in range(0, nq, 64):
        qb = q[s:s + 64]
        d2 = sq[qb][:, None] + sq[None, :] - 2.0 * (x64[qb] @ x64.T)
        d2[np.arange(qb.size), qb] = np.inf            # drop self pairs
        np.maximum(d2, 0.0, out=d2)
        part = np.partition(d2, keep - 1, axis=1)[:, :keep]
        best.append(part)
        exhausted.append(part.max(axis=1))
    allv = np.sort(np.concatenate([b.ravel() for b in best]))
    thr2 = allv[rank - 1]
    if np.any(np.concatenate(exhausted) <= thr2):
        raise RuntimeError("calibration sample truncated; raise `keep`")
    return float(np.float32(math.sqrt(thr2)))


def calibrate_bits(rows: np.ndarray, target_degree: float, n_queries: int = 1024, seed: int = 12345) -> int:
    """Hamming workloads: the same rule on integer distances (exact popcounts
    of the XOR of 64-bit words): eps = the ceil(k*Q)-th smallest non-self
    distance of Q sampled queries."""
    n = rows.shape[0]
    rng = np.random.Generator(np.random.PCG64(seed))
    q = np.sort(rng.choice(n, size=min(n_queries, n), replace=False))
    pad = (-rows.shape[1]) % 8
    w = np.ascontiguousarray(np.pad(rows, ((0, 0), (0, pad)))).view(np.uint64)
    rank = int(math.ceil(target_degree * q.size))
    hist = np.zeros(rows.shape[1] * 8 + 1, np.int64)
    for s in range(0, q.size, 16):
        qb = q[s:s + 16]
        d = np.bitwise_count(w[qb][:, None, :] ^ w[None, :, :]).sum(axis=2, dtype=np.int64)
        d[np.arange(qb.size), qb] = -1                 # drop self pairs
        hist += np.bincount(d[d >= 0].ravel(), minlength=hist.size)[:hist.size]
    return int(np.searchsorted(np.cumsum(hist), rank))


def main():
    import argparse
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", default=None, help="recompute one workload and keep the others")
    args = ap.parse_args()
    if args.only:
        with open(OUT) as f:
            wl = json.load(f)
        key = args.only
        spec = dict(PROFILE_SIZE) if key == "gmm_300k_k70" else wl.get(key) or BASE[key]
        if spec["kind"] == "bits":
            rows = I.binary_codes(spec["n"], spec["bits"], n_centres=spec["n_centres"], flip=spec["flip"],
                                  seed=spec["seed"])
            spec["eps"] = calibrate_bits(rows, spec["target_degree"])
        else:
            x = I.gmm_embedded(spec["n"], dim=spec["dim"], seed=spec["seed"])
            spec["eps"] = calibrate(x, spec["target_degree"])
        wl[key] = spec
        print(key, spec["eps"])
        with open(OUT, "w") as f:
            json.dump(wl, f, indent=1)
        return
    wl = {k: dict(v) for k, v in BASE.items()}
    wl["gmm_300k_k70"] = dict(PROFILE_SIZE)
    x3 = I.gmm_embedded(300_000, seed=0)
    wl["gmm_300k_k70"]["eps"] = calibrate(x3, 70.0)
    del x3
    hb = wl["ham_1m_256"]
    hb["eps"] = calibrate_bits(I.binary_codes(hb["n"], hb["bits"], n_centres=hb["n_centres"], flip=hb["flip"],
                                              seed=hb["seed"]), hb["target_degree"])
    x = I.gmm_embedded(1_000_000, seed=0)
    for key in ("gmm_1m_k10", "gmm_1m_k70", "gmm_1m_k500"):
        wl[key]["eps"] = calibrate(x, wl[key]["target_degree"])
        print(key, wl[key]["eps"], flush=True)
    del x
    specs = I.cloud_specs()
    for sp in specs:
        pts = I.cloud_points(sp)
        sp["eps"] = calibrate(pts, sp["target_degree"], n_queries=1024)
        print("cloud", sp["cloud"], sp["n"], sp["dim"], sp["kind"], sp["eps"], flush=True)
    wl["clouds_64"] = {"kind": "clouds", "zeta": 32, "specs": specs,
                       "note": "64 clouds, sizes log-uniform 1e4..5e5, dims {3,16,64}"}
    with open(OUT, "w") as f:
        json.dump(wl, f, indent=1)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
