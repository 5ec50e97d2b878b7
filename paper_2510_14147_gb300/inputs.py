"""Seeded synthetic inputs for the ε-graph workloads.

This module only draws random inputs; it holds none of the ε-graph method's
arithmetic (no distances, no predicates).  It is shared by the CUDA path, the
benchmarks and the tests, and imports nothing else from this package.

Every generator uses numpy ``Generator(PCG64(seed))`` and avoids BLAS/LAPACK so
that the same seed gives bit-identical arrays on x86-64 and on aarch64 hosts.

Workload shapes follow the paper's datasets (Table I): 1M x 128-D points with
~70 and ~500 mean neighbours stand in for ``sift`` (eps=175 and eps=225); DNA
strings under edit distance stand in for the paper's non-Euclidean workloads.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_cube(n: int, dim: int, seed: int = 0) -> np.ndarray:
    """n points uniform in [0,1]^dim, fp32, row-major (n, dim)."""
    rng = _rng(seed)
    return rng.random((n, dim), dtype=np.float64).astype(np.float32)


def _orthonormal_columns(rng: np.random.Generator, dim: int, k: int) -> np.ndarray:
    """dim x k matrix with orthonormal columns: modified Gram-Schmidt of a seeded
    Gaussian, with every inner product taken by ``math.fsum`` (exactly rounded),
    so the result does not depend on the host's BLAS."""
    g = rng.normal(0.0, 1.0, size=(dim, k))
    q = np.empty_like(g)
    for j in range(k):
        v = g[:, j].copy()
        for i in range(j):
            proj = math.fsum((q[:, i] * v).tolist())
            v = v - proj * q[:, i]
        nrm = math.sqrt(math.fsum((v * v).tolist()))
        q[:, j] = v / nrm
    return q


def gmm_embedded(n: int, dim: int = 128, n_centres: int = 100, intrinsic: int = 8,
                 centre_sd: float = 5.0, cluster_sd: float = 1.0,
                 noise_sd: float = 0.01, seed: int = 0,
                 chunk: int = 1 << 17) -> np.ndarray:
    """Gaussian mixture in an ``intrinsic``-D space, embedded in ``dim``-D.

    centres ~ N(0, centre_sd^2 I); each point picks a centre uniformly at random;
    z = centre + N(0, cluster_sd^2 I); x = Q z + N(0, noise_sd^2 I_dim) with Q a
    dim x intrinsic matrix of orthonormal columns.  Returned as fp32 (n, dim).
    The embedding product is written out column by column (no BLAS)."""
    rng = _rng(seed)
    k = min(intrinsic, dim)
    centres = rng.normal(0.0, centre_sd, size=(n_centres, k))
    q = _orthonormal_columns(rng, dim, k) if k < dim else np.eye(dim)
    labels = rng.integers(0, n_centres, size=n)
    out = np.empty((n, dim), dtype=np.float32)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        z = centres[labels[s:e]] + rng.normal(0.0, cluster_sd, size=(e - s, k))
        x = rng.normal(0.0, noise_sd, size=(e - s, dim))
        acc = np.zeros((e - s, dim))
        for j in range(k):
            acc = acc + z[:, j:j + 1] * q[:, j][None, :]
        out[s:e] = (acc + x).astype(np.float32)
    return out


_BASES = np.frombuffer(b"ACGT", dtype=np.uint8)


def _mutate(rng: np.random.Generator, seq: np.ndarray, p_sub: float,
            p_ins: float, p_del: float) -> np.ndarray:
    """One mutant of ``seq``.  Per site: with probability p_ins a random base is
    inserted before it; then the site is deleted with probability p_del, else
    substituted by a uniformly chosen *different* base with probability p_sub."""
    m = seq.size
    ins = rng.random(m) < p_ins
    ins_base = _BASES[rng.integers(0, 4, size=m)]
    u = rng.random(m)
    shift = rng.integers(1, 4, size=m)
    code = np.searchsorted(_BASES, seq)                # ACGT is sorted
    sub = (u >= p_del) & (u < p_del + p_sub)
    kept = _BASES[np.where(sub, (code + shift) % 4, code)]
    keep = u >= p_del
    pieces = np.empty(2 * m, dtype=np.uint8)
    mask = np.zeros(2 * m, dtype=bool)
    pieces[0::2] = ins_base
    mask[0::2] = ins
    pieces[1::2] = kept
    mask[1::2] = keep
    return pieces[mask]


def dna_strings(n_seeds: int = 500, per_seed: int = 100, seed_len: int = 96,
                p_sub: float = 0.04, p_ins: float = 0.005, p_del: float = 0.005,
                min_len: int = 80, max_len: int = 112, seed: int = 0):
    """DNA strings (ASCII 'ACGT', uint8): ``n_seeds`` uniform random seeds of length
    ``seed_len``, each mutated ``per_seed`` times with per-site substitution
    (to a different base), insertion and deletion probabilities.  Mutants whose
    length falls outside [min_len, max_len] are redrawn.

    Returns (data uint8[total], offsets int64[n+1]) with string i occupying
    data[offsets[i]:offsets[i+1]]."""
    rng = _rng(seed)
    strings = []
    for _ in range(n_seeds):
        base = _BASES[rng.integers(0, 4, size=seed_len)]
        for _ in range(per_seed):
            while True:
                m = _mutate(rng, base, p_sub, p_ins, p_del)
                if min_len <= m.size <= max_len:
                    break
            strings.append(m)
    offsets = np.zeros(len(strings) + 1, dtype=np.int64)
    offsets[1:] = np.cumsum([s.size for s in strings])
    data = np.concatenate(strings) if strings else np.zeros(0, dtype=np.uint8)
    return data, offsets


def random_strings(n: int, min_len: int, max_len: int, alphabet: bytes = b"ACGT",
                   seed: int = 0):
    """Independent random strings (uint8) with lengths uniform in [min_len, max_len]."""
    rng = _rng(seed)
    alpha = np.frombuffer(alphabet, dtype=np.uint8)
    lens = rng.integers(min_len, max_len + 1, size=n)
    offsets = np.zeros(n + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(lens)
    data = alpha[rng.integers(0, alpha.size, size=int(offsets[-1]))] if n else np.zeros(0, np.uint8)
    return data.astype(np.uint8), offsets


def binary_codes(n: int, bits: int = 256, n_centres: int = 1000, flip: float = 0.05, seed: int = 0,
                 chunk: int = 1 << 16) -> np.ndarray:
    """Bit strings clustered around random centres: ``n_centres`` uniform
    random codes of ``bits`` bits; each point picks a centre uniformly at
    random and flips each of its bits independently with probability
    ``flip``.  Returned as uint8 rows of ceil(bits/8) bytes, bit j of a row =
    bit j % 8 of byte j // 8, bits past ``bits`` zero."""
    rng = _rng(seed)
    centres = rng.random((n_centres, bits)) < 0.5
    labels = rng.integers(0, n_centres, size=n)
    nb = (bits + 7) // 8
    out = np.empty((n, nb), dtype=np.uint8)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        x = centres[labels[s:e]] ^ (rng.random((e - s, bits)) < flip)
        out[s:e] = np.packbits(x, axis=1, bitorder="little")
    return out


def cloud_specs(n_clouds: int = 64, seed: int = 0, min_n: int = 10_000,
                max_n: int = 500_000, dims=(3, 16, 64), min_deg: float = 20.0,
                max_deg: float = 300.0):
    """Per-cloud recipe for the many-cloud batch: size log-uniform in
    [min_n, max_n], dim uniform over ``dims``, generator uniform-cube or the
    embedded Gaussian mixture (intrinsic dim min(8, dim)), and a target mean
    degree log-uniform in [min_deg, max_deg]."""
    rng = _rng(seed)
    specs = []
    for c in range(n_clouds):
        n = int(round(math.exp(rng.uniform(math.log(min_n), math.log(max_n)))))
        dim = int(dims[rng.integers(0, len(dims))])
        kind = "uniform" if rng.random() < 0.5 else "gmm"
        deg = float(math.exp(rng.uniform(math.log(min_deg), math.log(max_deg))))
        specs.append({"cloud": c, "n": n, "dim": dim, "kind": kind,
                      "target_degree": deg, "seed": 1000 + c})
    return specs


def cloud_points(spec: dict) -> np.ndarray:
    if spec["kind"] == "uniform":
        return uniform_cube(spec["n"], spec["dim"], seed=spec["seed"])
    return gmm_embedded(spec["n"], dim=spec["dim"], intrinsic=min(8, spec["dim"]),
                        n_centres=max(1, spec["n"] // 10_000), seed=spec["seed"])


def load_workloads() -> dict:
    """Workload table (sizes, seeds and calibrated ε values)."""
    with open(os.path.join(_HERE, "workloads.json")) as f:
        return json.load(f)
