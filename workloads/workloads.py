"""ctypes wrapper over libworkloads.so plus the few pure-numpy generators.

Seeds and shapes of the standard workloads are chosen by the callers
(tests, bench.py); this module only draws the numbers.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "gen.c")
LIB = os.path.join(HERE, "libworkloads.so")

# Share of queries by term count on ClueWeb09 (Table 4a of the paper), in
# tenths of a percent; used only as distribution parameters.
CLUEWEB_TERM_WEIGHTS_2_5 = (198, 325, 263, 132)          # 2..5 terms
CLUEWEB_TERM_WEIGHTS_2_8 = (198, 325, 263, 132, 49, 17, 16)  # 2..8 terms

_lib = None


def build_workloads(force: bool = False) -> str:
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-std=gnu11", "-O2", "-Wall", "-fPIC",
                           "-shared", "-pthread", "-o", tmp, SRC])
    os.replace(tmp, LIB)
    return LIB


def _L():
    global _lib
    if _lib is None:
        lib = C.CDLL(build_workloads())
        u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
        u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
        u64 = C.c_uint64
        lib.wl_uniform.argtypes = [u64, u64, u64, u64, u32p]
        lib.wl_clustered.argtypes = [u64, u64, u64, u64, u32p]
        lib.wl_many.argtypes = [C.c_int, u64, u64p, u64p, u64, u64, u64,
                                C.c_int, u32p]
        lib.wl_pair_short.argtypes = [u32p, u64, u64, u64, u64, u64, u32p]
        lib.wl_queries.argtypes = [u64, u64p, u64, C.c_uint32, u32p,
                                   C.c_uint32, u64, u32p, u64p]
        for f in ("wl_uniform", "wl_clustered", "wl_many", "wl_pair_short",
                  "wl_queries"):
            getattr(lib, f).restype = C.c_int
        _lib = lib
    return _lib


def _check(rc: int, what: str):
    if rc:
        raise ValueError(f"{what}: generator error {rc}")


def uniform(n: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """n distinct values drawn uniformly from [lo, hi), ascending."""
    out = np.empty(max(n, 1), np.uint32)
    _check(_L().wl_uniform(n, lo, hi, seed, out), "uniform")
    return out[:n]


def clustered(n: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """n distinct values from [lo, hi) by recursive interval splitting."""
    out = np.empty(max(n, 1), np.uint32)
    _check(_L().wl_clustered(n, lo, hi, seed, out), "clustered")
    return out[:n]


def many(kind: str, lens, lo: int, hi: int, seed_base: int,
         nthreads: int | None = None):
    """Lists i = 0..len(lens)-1 with seed seed_base + i, drawn in parallel.
    Returns (values concatenated, offsets with len(lens)+1 entries)."""
    lens = np.ascontiguousarray(lens, np.uint64)
    offs = np.zeros(lens.size + 1, np.uint64)
    np.cumsum(lens, out=offs[1:])
    out = np.empty(max(int(offs[-1]), 1), np.uint32)
    nthreads = nthreads or min(32, os.cpu_count() or 1)
    k = {"uniform": 0, "clustered": 1}[kind]
    _check(_L().wl_many(k, lens.size, lens, offs[:-1].copy(), lo, hi,
                        seed_base, nthreads, out), "many")
    return out[: int(offs[-1])], offs


def pair_short(f: np.ndarray, m: int, k: int, U: int, seed: int) -> np.ndarray:
    """Short list of a pair: k values of f plus m-k values of [0,U) not in f."""
    f = np.ascontiguousarray(f, np.uint32)
    out = np.empty(max(m, 1), np.uint32)
    _check(_L().wl_pair_short(f, f.size, m, k, U, seed, out), "pair_short")
    return out[:m]


def zipf_lengths(terms: int, total: int, cap: int) -> np.ndarray:
    """Lengths min(floor(C/r), cap), r = 1..terms, with C the smallest
    integer whose sum reaches `total` (Zipf with s = 1)."""
    r = np.arange(1, terms + 1, dtype=np.float64)

    def tot(c):
        return int(np.minimum(np.floor(c / r), cap).sum())

    lo, hi = 1, total
    while lo < hi:
        mid = (lo + hi) // 2
        if tot(mid) >= total:
            hi = mid
        else:
            lo = mid + 1
    return np.minimum(np.floor(lo / r), cap).astype(np.uint64)


def queries(lens, nq: int, weights, tmin: int, seed: int):
    """nq conjunctive queries; term count tmin + i with weight weights[i];
    distinct terms drawn with probability proportional to list length.
    Returns (terms uint32, term_off uint64 with nq+1 entries)."""
    lens = np.ascontiguousarray(lens, np.uint64)
    cum = np.cumsum(lens).astype(np.uint64)
    w = np.ascontiguousarray(weights, np.uint32)
    terms = np.empty(max(1, nq * (tmin + w.size - 1)), np.uint32)
    off = np.empty(nq + 1, np.uint64)
    _check(_L().wl_queries(nq, cum, lens.size, tmin, w, w.size, seed, terms,
                           off), "queries")
    return terms[: int(off[-1])], off


def stepped_walk(n: int, b: int, seed: int, every: int = 4) -> np.ndarray:
    """A random walk modulo 2^32 that moves only at positions i = 0 mod
    `every`, by a step drawn uniformly from [0, 2^b); it stays put
    elsewhere.  Any `every` consecutive steps contain one move, so every
    difference x[i] - x[i-k] for 1 <= k <= `every` is below 2^b.  Not
    strictly increasing (equal neighbours, wrap-around)."""
    rng = np.random.default_rng(seed)
    steps = np.zeros(n, np.uint64)
    m = (n + every - 1) // every
    steps[::every] = rng.integers(0, 1 << b, m, dtype=np.uint64) if b else 0
    return (np.cumsum(steps, dtype=np.uint64) & np.uint64(0xFFFFFFFF)).astype(np.uint32)


def poisson_arrivals(rate: float, count: int, seed: int) -> np.ndarray:
    """Arrival times in seconds of an open-loop Poisson process."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, count))
