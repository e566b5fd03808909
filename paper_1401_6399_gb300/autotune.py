"""Autotuner for the intersection and query kernels.

Measures every candidate of the tuning space (skew threshold between the
dense and sparse regimes, blocks of the shortest list per work item, warps
per CTA of the persistent query kernel, span limit of the merge regime) on
a sample of the caller's own workload, installs the fastest with
bp_set_tuning, and records the choice in a JSON file keyed by GPU name.  Every candidate gives the same answers (the
tests check this); only speed differs.
"""
from __future__ import annotations

import itertools
import json
import os
import time

import numpy as np
import torch

from . import capi

SPACE = {
    "dense_blocks": (1, 2, 4, 8),
    "query_chunk_blocks": (1, 2, 4, 8),
    "query_warps": (4, 8),
    "merge_span": (0, 2, 4, 16),
}

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "tuning.json")


def gpu_key() -> str:
    return torch.cuda.get_device_name().replace(" ", "_")


def _time_ms(fn, reps: int, stream) -> float:
    fn()
    stream.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def tune_queries(index, terms: np.ndarray, term_off: np.ndarray, reps: int = 3,
                 space: dict | None = None, save_cache: bool = True) -> dict:
    """Tune bp_query_batch on a sample batch (terms, term_off) of `index`.
    Returns {"best": params, "ms": {params: ms}} and installs the best (and
    records it for this GPU unless save_cache is False)."""
    space = space or SPACE
    dev = index.device
    terms = np.ascontiguousarray(terms, np.uint32)
    term_off = np.ascontiguousarray(term_off, np.uint64)
    nq = term_off.size - 1
    # size the output once, exactly
    _, o, _ = index.query_batch(terms, term_off, out_cap=1 << 26, on_device=True)
    cap = max(1, int(o[-1]))
    d_terms = torch.from_numpy(terms.view(np.int32).copy()).to(dev)
    d_off = torch.from_numpy(term_off.view(np.int64).copy()).to(dev)
    out = torch.empty(cap, dtype=torch.int32, device=dev)
    out_off = torch.empty(nq + 1, dtype=torch.int64, device=dev)
    counts = torch.empty(nq, dtype=torch.int32, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    stream = torch.cuda.Stream()
    old = capi.bp_get_tuning()
    results = {}
    keys = list(space)
    for combo in itertools.product(*(space[k] for k in keys)):
        capi.bp_set_tuning(**dict(zip(keys, combo)))
        sb = capi.bp_query_batch_scratch_bytes(index.h_lists, terms, term_off, cap)
        scratch = torch.empty(sb, dtype=torch.uint8, device=dev)

        def run():
            index.query_batch_async(d_terms, d_off, nq, int(term_off[-1]), out, out_off, counts,
                                    scratch, st, stream)

        results[combo] = _time_ms(run, reps, stream)
        del scratch
    stream.synchronize()
    if int(st.item()) != 0:
        capi.bp_set_tuning(**old)
        raise capi.BPError(int(st.item()), "autotune")
    best = min(results, key=results.get)
    params = dict(zip(keys, best))
    capi.bp_set_tuning(**params)
    if save_cache:
        save(params, results)
    return {"best": params, "ms": {",".join(str(x) for x in k): round(v, 4)
                                   for k, v in results.items()}}


def save(params: dict, results: dict) -> None:
    try:
        data = json.load(open(CACHE)) if os.path.exists(CACHE) else {}
    except (OSError, ValueError):
        data = {}
    data[gpu_key()] = {"params": params, "when": time.strftime("%Y-%m-%dT%H:%M:%S"),
                       "candidates": len(results)}
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    with open(CACHE, "w") as fh:
        json.dump(data, fh, indent=1)


def load_installed() -> dict | None:
    """Install the tuned parameters recorded for this GPU, if any."""
    try:
        params = json.load(open(CACHE))[gpu_key()]["params"]
    except (OSError, ValueError, KeyError):
        return None
    capi.bp_set_tuning(**params)
    return params
