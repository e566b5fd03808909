#!/usr/bin/env python3
"""Benchmark of the S4-BP128-D4 decode hot path on GB300.

Workload (one step): decode 32 lists of 2^26 sorted distinct uint32 drawn
uniformly without replacement from [0, 2^29), S4-BP128-D4 encoded in the GPU
layout, in one bp_decode_batch launch (8 GiB of decoded output per step).
Inputs (1.9 GB compressed) and outputs (8 GiB) are far larger than L2, so no
flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--layout gpu|paper|pfor] [--lists L] [--no-extra]
                  [--pairs-only] [--queries-only --query-scale S]

Prints one JSON line.  Besides the timed step it measures (unless
--no-extra): decode+sum, clustered lists, the paper layout, the DM/D2/D1
kinds, S4-FastPFOR, a per-bit-width unpack sweep with the two-pass prefix
ablation, fused vs unfused pair intersections, 64 pairs per launch, batched
conjunctive queries (with and without bitmaps), open-loop serving, the end
to end call from host memory, and the oracle on the host cores.  With N > 1 (torchrun) every rank decodes its own 32
lists (weak scaling, no collective on the data path); the reported value is
all ranks' integers over the slowest rank's time.
"""
from __future__ import annotations

import argparse
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

METRIC = "S4-BP128-D4 decoded Gint/s"
UNIT = "Gint/s"
N_PER_LIST = 1 << 26
UNIVERSE = 1 << 29
SEED_BASE = 0x2000


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=300)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--lists", type=int, default=32)
    p.add_argument("--layout", choices=["gpu", "paper", "pfor"], default="gpu",
                   help="stream layout of the timed decode (paper: the Section 4.3 layout; "
                        "pfor: S4-FastPFOR-D4 in the GPU page layout)")
    p.add_argument("--log2n", type=int, default=26)
    p.add_argument("--no-extra", action="store_true", help="skip secondary measurements")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--pairs-only", action="store_true",
                   help="run only the pair sweep (for profiling)")
    p.add_argument("--queries-only", action="store_true",
                   help="run only the batched-query measurement (for profiling)")
    p.add_argument("--query-scale", type=int, default=1,
                   help="with --queries-only: index and batch this many times smaller")
    p.add_argument("--profile-queries", type=int, default=0,
                   help="with --profile-case queries: only the first N queries of the batch")
    p.add_argument("--profile-tuning", default="",
                   help="with --profile-case queries: dense_blocks,query_chunk_blocks,"
                        "query_warps,merge_span to install first (the autotuner's choice)")
    p.add_argument("--serving-only", action="store_true",
                   help="only the serving measurements on the batched-query index")
    p.add_argument("--serving-sweep", action="store_true",
                   help="only the serving engine at 1M queries/s offered over slot counts "
                        "and batch sizes")
    p.add_argument("--profile-case",
                   choices=["decode", "decode_sum", "gp_decode", "pl_decode", "pair", "queries"],
                   help="time one case of one kernel alone (for ncu): the decodes on 4 lists "
                        "of 2^26, the fused pair on m = n = 2^22, the batched queries on the "
                        "index --query-scale times smaller")
    return p.parse_args()


# ---- distributed plumbing -----------------------------------------------------------

def dist_setup(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def dist_init(world, local):
    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend="nccl", device_id=torch.device("cuda", local))
    return dist if world > 1 else None


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, value: float) -> float:
    """The largest of the ranks' values (the slowest rank's time), on the
    GPU under NCCL, on the host under gloo."""
    if dist is None:
        return value
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_seed(rank: int) -> int:
    """Seed base of a rank's lists: every rank decodes lists of its own
    (weak scaling, no data exchanged)."""
    return SEED_BASE + 4096 * rank


def whole_job_rate(world: int, ints_per_rank: int, ms_max: float) -> float:
    """Gint/s of the whole job: all ranks' integers over the slowest rank's
    time per step."""
    return world * ints_per_rank / (ms_max * 1e-3) / 1e9


# ---- clocks --------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons (read only)."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None
        self.thread = None
        self.marks = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.time(), [x.strip() for x in line.split(",")]))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0: float, t1: float) -> dict:
        rows = [r for (t, r) in self.samples if t0 <= t <= t1 and len(r) >= 8]
        if not rows:  # timed region shorter than one sample: take the nearest ones
            rows = [r for (t, r) in self.samples if t0 - 0.3 <= t <= t1 + 0.3 and len(r) >= 8]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[0]) for r in rows if num(r[0]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4)
                          if r[4 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": num(rows[0][1]), "reasons": reasons, "samples": len(rows),
                "power_w_max": max((num(r[2]) or 0) for r in rows)}


# ---- workload --------------------------------------------------------------------------

def make_lists(kind: str, count: int, n: int, U: int, seed_base: int):
    import workloads as W
    vals, offs = W.many(kind, [n] * count, 0, U, seed_base)
    return [vals[int(offs[i]):int(offs[i + 1])] for i in range(count)]


def encode_all(lists, layout: int):
    from concurrent.futures import ThreadPoolExecutor
    from paper_1401_6399_gb300 import capi
    nt = max(1, min(8, (os.cpu_count() or 8) // 2))
    with ThreadPoolExecutor(max_workers=min(len(lists), 8)) as ex:
        return list(ex.map(lambda x: capi.bp_encode(x, layout, nthreads=nt), lists))


def encode_all_kind(lists, layout: int, kind: int):
    from concurrent.futures import ThreadPoolExecutor
    from paper_1401_6399_gb300 import capi
    nt = max(1, min(8, (os.cpu_count() or 8) // 2))
    with ThreadPoolExecutor(max_workers=min(len(lists), 8)) as ex:
        return list(ex.map(lambda x: capi.bp_encode(x, layout, nthreads=nt, delta=kind), lists))


def kernel_sha() -> str:
    h = hashlib.sha256()
    for f in ("common.cuh", "bulk.cuh", "gl_block.cuh", "decode_gl.cu", "format.h", "decode.h"):
        with open(os.path.join(ROOT, "paper_1401_6399_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(sha: str):
    """DRAM bytes per full launch of the headline decode kernel from the
    committed ncu summary, if it was taken on this kernel source."""
    path = os.path.join(ROOT, "profiles", "gl_decode_uniform_32x2p26.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    m_sha = re.search(r"kernel_source_sha:\s*([0-9a-f]+)", text)
    m_b = re.search(r"dram_bytes_per_full_launch:\s*([0-9.eE+]+)", text)
    if not m_sha or not m_b or m_sha.group(1) != sha:
        return None
    return float(m_b.group(1))


# source files of each kernel with a counted instruction cost (profiles/issue_counts.md)
KERNEL_SOURCES = {
    "gl_decode": ["common.cuh", "bulk.cuh", "gl_block.cuh", "decode_gl.cu", "format.h", "decode.h"],
    "gl_decode_sum": ["common.cuh", "bulk.cuh", "gl_block.cuh", "decode_gl.cu", "format.h",
                      "decode.h"],
    "gp_decode": ["common.cuh", "bulk.cuh", "gl_block.cuh", "decode_pfor.cu", "format.h",
                  "decode.h"],
    "fused_pair": ["common.cuh", "gl_block.cuh", "intersect.cuh", "lookback.cuh", "intersect.cu",
                   "tuning.h"],
    "q_main": ["common.cuh", "gl_block.cuh", "intersect.cuh", "lookback.cuh", "query.cu",
               "tuning.h"],
    "pl_tiles": ["common.cuh", "bulk.cuh", "gl_block.cuh", "pl_block.cuh", "decode_pl.cu",
                 "format.h", "decode.h"],
}


def source_sha(files) -> str:
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_1401_6399_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def issue_counts() -> dict:
    """Warp-instructions per unit of work from profiles/issue_counts.md, for
    the kernels whose sources are unchanged since the capture."""
    out = {}
    try:
        text = open(os.path.join(ROOT, "profiles", "issue_counts.md")).read()
    except OSError:
        return out
    for m in re.finditer(r"^\| (\w+) \| ([^|]+) \| (\d+) \| (\d+) \| ([0-9.]+) \| (\w+) \| "
                         r"([0-9a-f]+) \|$", text, flags=re.M):
        key = m.group(1)
        src = "q_main" if key.startswith("q_main") else key  # q_main_t<tuning>
        if src in KERNEL_SOURCES and source_sha(KERNEL_SOURCES[src]) == m.group(7):
            out[key] = {"case": m.group(2).strip(), "per_unit": float(m.group(5)),
                        "unit": m.group(6)}
    return out


def issue_roof(key: str, units: float, ms: float, sm_mhz) -> dict | None:
    """Issue roofline of one launch: counted warp-instructions (per unit x
    units) over its time, against SMs x 4 schedulers x 1 warp-instruction
    per cycle at the sampled SM clock."""
    e = issue_counts().get(key)
    if e is None or not ms or not sm_mhz:
        return None
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    inst = e["per_unit"] * units
    achieved = inst / (ms * 1e-3) / 1e9
    peak = sms * 4 * sm_mhz * 1e6 / 1e9
    return {"bound": "issue", "achieved": round(achieved, 1), "peak": round(peak, 1),
            "unit": "G warp-instructions/s", "frac": round(achieved / peak, 4),
            "warp_instructions_per_launch": int(inst),
            "per_unit": f"{e['per_unit']} per {e['unit']} (ncu smsp__inst_executed.sum, "
                        f"{e['case']}; profiles/issue_counts.md)",
            "clock_mhz": sm_mhz}


def load_sm_max():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["sm_max_mhz"])
    except (OSError, KeyError, ValueError):
        return 2070.0


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ---- the oracle as a CPU baseline --------------------------------------------------------

def oracle_decode_rate(encs, ns, threads: int, layout: int = 1):
    """Decode the given streams (GL, PL if layout is 0, GP if 3) with the
    scalar oracle on `threads` host threads; returns (Gint/s, seconds,
    threads)."""
    from concurrent.futures import ThreadPoolExecutor
    from oracle import Oracle
    orc = Oracle()
    dec = {0: orc.pl_decode, 1: orc.gl_decode, 3: orc.gp_decode}[layout]
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        outs = list(ex.map(dec, encs))
    dt = time.perf_counter() - t0
    assert [o.size for o in outs] == list(ns)
    return sum(ns) / dt / 1e9, dt, threads


def oracle_query_rates(data, h_lists, terms, toff, qids, threads: int):
    """The oracle answering queries from the compressed index, as a CPU
    system would: every term's GL stream decoded by the scalar oracle, then
    Set-vs-Set by merging (orc.svs).  Each query runs on one thread, queries
    spread over `threads` threads (closed loop).  Returns (queries/s, per-
    query service times in s, answer counts)."""
    from concurrent.futures import ThreadPoolExecutor
    from oracle import Oracle
    orc = Oracle()
    eo = h_lists["enc_offset"].astype(np.int64)
    eb = h_lists["enc_bytes"].astype(np.int64)

    def one(q):
        t0 = time.perf_counter()
        t = terms[int(toff[q]):int(toff[q + 1])]
        lists = [orc.gl_decode(data[eo[u]:eo[u] + eb[u]]) for u in t]
        k = orc.svs(lists).size
        return time.perf_counter() - t0, k

    w0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        res = list(ex.map(one, [int(q) for q in qids]))
    wall = time.perf_counter() - w0
    return len(qids) / wall, np.array([r[0] for r in res]), np.array([r[1] for r in res])


def run_reference(args, rank, world):
    """Reference arm: the scalar C oracle on the host cores, on the headline
    decode workload itself: 32 lists of 2^26 uniform integers of [0, 2^29)
    in the GPU layout, written by the oracle's own encoder; every step
    decodes all of them, lists spread over the host threads."""
    if rank != 0:
        return
    from concurrent.futures import ThreadPoolExecutor
    from oracle import Oracle, build_oracle
    from workloads.workloads import build_workloads
    build_oracle()
    build_workloads()
    orc = Oracle()
    threads = min(16, os.cpu_count() or 1)
    n = 1 << args.log2n
    L = args.lists
    lists = make_lists("uniform", L, n, UNIVERSE, SEED_BASE)
    with ThreadPoolExecutor(max_workers=threads) as ex:
        encs = list(ex.map(lambda x: np.frombuffer(orc.gl_encode(x), np.uint8), lists))
    assert np.array_equal(orc.gl_decode(encs[0]), lists[0])
    del lists
    comp = sum(e.size for e in encs)

    def step():
        with ThreadPoolExecutor(max_workers=threads) as ex:
            outs = list(ex.map(lambda e: orc.gl_decode(e).size, encs))
        assert outs == [n] * L

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    val = n * L * args.steps / dt / 1e9
    sample = (f"the whole workload every step: {L} GL streams of 2^{args.log2n} ints "
              f"(oracle-encoded, {comp} bytes) decoded by the scalar C oracle on {threads} threads")
    line = {"metric": METRIC, "value": round(val, 4), "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * dt / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": f"decode {L} lists x 2^{args.log2n} uniform uint32 of "
                                   "[0,2^29) per GPU, S4-BP128-D4 GPU layout",
                       "lists_per_gpu": L, "ints_per_list": n, "compressed_bytes_per_gpu": comp,
                       "l2": "inputs (compressed) and outputs larger than L2; no flush"},
            "cpu_baseline": {"value": round(val, 4), "unit": UNIT, "cores": threads,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(val, 4), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---- our arm -------------------------------------------------------------------------------

def time_launches(stream, fn, steps: int, warmup: int):
    """Run fn() warmup + steps times on `stream`; return ms per step from CUDA
    events recorded on that stream."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / steps


def time_graph(stream, fn, reps: int):
    """Capture `reps` back-to-back calls of fn() in one CUDA graph, replay it
    (after one warm-up replay) and return ms per call from CUDA events: the
    per-launch CPU overhead drops out, which matters for launches of a few
    microseconds."""
    import torch
    with torch.cuda.stream(stream):
        fn()
    stream.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        for _ in range(reps):
            fn()
    with torch.cuda.stream(stream):
        g.replay()
        stream.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.replay()
        e1.record(stream)
        e1.synchronize()
    return e0.elapsed_time(e1) / reps


def gl_widths(enc: np.ndarray) -> np.ndarray:
    """Bit widths of the blocks of a GL stream (from its header fields)."""
    h = enc[:64].view(np.uint32)
    nb, off_bw = int(h[3]), int(h[8])
    return enc[off_bw:off_bw + nb]


def unpack_sweep(stream, reps: int = 20, lists: int = 12, n: int = 1 << 20):
    """Unpacking speed per bit width (Section 7.4, Figure 6) on the GPU: for
    b = 0..32 and each kind, `lists` GL lists of n integers whose blocks all
    have width b (stepped walks modulo 2^32, BP_ENCODE_ANY_ORDER), decoded
    by one bp_decode_batch (the product kernels) and by bp_decode_ablation
    with the prefix integrated (one pass) or applied as a separate pass over
    a block buffer in shared memory (two pass, Figure 6a).  12 x 2^20 integers: 48 MiB out plus at most
    48 MiB in, so repeated launches run from L2 and time the unpacking, not
    HBM.  Gint/s, CUDA events over `reps` launches captured in one CUDA
    graph."""
    import torch
    import workloads as W
    from paper_1401_6399_gb300 import api, capi
    GL = capi.BP_LAYOUT_GPU
    total = lists * n
    out = torch.empty(total, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    res = {}
    for kname, kind in (("D4", 0), ("DM", 1), ("D2", 2), ("D1", 3)):
        rows = {"batch": [], "one_pass": [], "two_pass": []}
        for b in range(33):
            xs = [W.stepped_walk(n, b, 0x7000 + 64 * b + 8 * kind + i) for i in range(lists)]
            encs = encode_all_kind(xs, GL, kind | capi.BP_ENCODE_ANY_ORDER)
            batch = api.ListBatch(encs, [n] * lists, GL)
            want = torch.from_numpy(np.concatenate(xs).view(np.int32)).to("cuda")
            for mode, fn in (("batch", lambda: batch.decode_into(out, status, stream)),
                             ("one_pass", lambda: batch.ablation_into(out, status, 0, stream)),
                             ("two_pass", lambda: batch.ablation_into(out, status, 1, stream))):
                with torch.cuda.stream(stream):  # the fill must land before the decode
                    out.fill_(-1)
                    fn()
                stream.synchronize()
                assert int(status.item()) == 0 and torch.equal(out, want), (kname, b, mode)
                ms = time_graph(stream, fn, reps)
                rows[mode].append(round(total / (ms * 1e-3) / 1e9, 1))
            del batch, want, encs, xs
        gain = [round(o / t, 3) for o, t in zip(rows["one_pass"], rows["two_pass"])]
        res[kname] = {**rows, "integration_gain": gain,
                      "gain_range": [min(gain[1:32]), max(gain[1:32])]}
    del out
    torch.cuda.empty_cache()
    return {"widths": "0..32", "ints_per_launch": total, "gints": res}


def pair_sweep(stream, reps: int, cpu_threads: int = 0, sm_mhz=None):
    """Longer list 2^22 uniform values of [0,2^26); shorter lists of 2^22 .. 2^8
    values sharing 10% of theirs; fused vs unfused bp_intersect_pair, L2
    flushed before every call (one pair fits in L2).  cpu_threads > 0: the
    oracle beside it (decode both streams, merge), one pair on one thread and
    one pair per thread on cpu_threads threads."""
    import torch
    import workloads as W
    from paper_1401_6399_gb300 import api, capi
    GL = capi.BP_LAYOUT_GPU
    f = W.uniform(1 << 22, 0, 1 << 26, 0x3000)
    encf = capi.bp_encode(f, GL, nthreads=8)
    ef = api.to_device(encf)
    first = f[::128].astype(np.int64)
    bw = gl_widths(encf).astype(np.int64)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    out = {}
    for m in (1 << 22, 1 << 18, 1 << 14, 1 << 10, 1 << 8):
        k = round(0.1 * m)
        r = W.pair_short(f, m, k, 1 << 26, 0x3000 + m)
        encr = capi.bp_encode(r, GL, nthreads=8)
        er = api.to_device(encr)
        row = {}
        answers = {}
        for name, mode in (("fused", capi.BP_MODE_FUSED), ("unfused", capi.BP_MODE_UNFUSED)):
            cap = m
            res = torch.empty(cap, dtype=torch.int32, device="cuda")
            cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
            sb = capi.bp_intersect_scratch_bytes(m, f.size, GL, mode)
            scratch = torch.empty(max(sb, 16), dtype=torch.uint8, device="cuda")
            st = torch.zeros(1, dtype=torch.int32, device="cuda")

            def call():
                capi.check(capi.bp_intersect_pair(er.data_ptr(), er.numel(), m, ef.data_ptr(),
                                                  ef.numel(), f.size, GL, mode, res.data_ptr(),
                                                  cap, cnt.data_ptr(), scratch.data_ptr(), sb,
                                                  st.data_ptr(), stream.cuda_stream), "pair")
            with torch.cuda.stream(stream):
                call()
            stream.synchronize()
            assert int(st.item()) == 0 and int(cnt.item()) == k
            answers[name] = res[:k].clone()
            tot = 0.0
            for _ in range(reps):
                with torch.cuda.stream(stream):
                    flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                call()
                e1.record(stream)
                e1.synchronize()
                tot += e0.elapsed_time(e1)
            row[name + "_us"] = round(1e3 * tot / reps, 2)
            if mode == capi.BP_MODE_FUSED:  # the same call with the merge regime off
                saved = capi.bp_get_tuning()
                capi.bp_set_tuning(merge_span=0)
                try:
                    call()
                    tot = 0.0
                    for _ in range(reps):
                        with torch.cuda.stream(stream):
                            flush.zero_()
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        call()
                        e1.record(stream)
                        e1.synchronize()
                        tot += e0.elapsed_time(e1)
                    assert int(st.item()) == 0 and torch.equal(res[:k], answers["fused"])
                finally:
                    capi.bp_set_tuning(**saved)
                row["fused_no_merge_us"] = round(1e3 * tot / reps, 2)
        assert torch.equal(answers["fused"], answers["unfused"])
        cand = np.unique(np.searchsorted(first, r.astype(np.int64), side="right") - 1)
        cand = cand[cand >= 0]
        alg = encr.size + 4 * first.size + int(16 * bw[cand].sum()) + 4 * k
        row["speedup_fused"] = round(row["unfused_us"] / row["fused_us"], 2)
        row["fused_alg_bytes"] = alg
        row["fused_gbs"] = round(alg / (row["fused_us"] * 1e-6) / 1e9, 1)
        row["candidate_blocks"] = int(cand.size)
        if m == f.size:  # the counted launch: m = n = 2^22
            row["roofline"] = issue_roof("fused_pair", 1, row["fused_us"] * 1e-3,
                                         sm_mhz or load_sm_max())
        if cpu_threads:
            row.update(cpu_pair_rates(encr, encf, k, cpu_threads))
            row["gpu_vs_cpu_1t"] = round(row["cpu_us_1t"] / row["fused_us"], 1)
        out[f"m=2^{int(np.log2(m))}"] = row
    return out


def cpu_pair_rates(encr, encf, k: int, threads: int) -> dict:
    """The oracle on one pair of GL streams: decode both, intersect by merge
    (Section 6), on one thread (best of 3) and as `threads` concurrent pairs."""
    from concurrent.futures import ThreadPoolExecutor
    from oracle import Oracle
    orc = Oracle()

    def pair():
        return orc.intersect(orc.gl_decode(encr), orc.gl_decode(encf)).size
    best = float("inf")
    for _ in range(3):
        t0 = time.perf_counter()
        assert pair() == k
        best = min(best, time.perf_counter() - t0)
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        assert list(ex.map(lambda _: pair(), range(threads))) == [k] * threads
    wall = time.perf_counter() - t0
    return {"cpu_us_1t": round(1e6 * best, 1), "cpu_pairs_per_s": round(threads / wall, 1),
            "cpu_threads": threads}


def pair_batch(stream, reps: int, pairs: int = 64):
    """The pair sweep as independent pairs per launch: 64 longer lists of 2^22
    uniform values of [0,2^26) (seeds 0x3100+i) and, per length ratio, 64
    shorter lists sharing 10% of their values with their partner, all in one
    resident index (together far larger than L2); one bp_query_batch of 64
    two-term queries per launch, autotuned per length ratio."""
    import torch
    import workloads as W
    from paper_1401_6399_gb300 import api, autotune, capi
    ms = (1 << 22, 1 << 18, 1 << 14, 1 << 10, 1 << 8)
    fv, fo = W.many("uniform", [1 << 22] * pairs, 0, 1 << 26, 0x3100)
    parts, lens = [fv], [np.diff(fo).astype(np.uint64)]
    for m in ms:
        k = round(0.1 * m)
        parts += [W.pair_short(fv[int(fo[i]):int(fo[i + 1])], m, k, 1 << 26, 0x3200 + 131 * i + m)
                  for i in range(pairs)]
        lens.append(np.full(pairs, m, np.uint64))
    lens = np.concatenate(lens)
    offs = np.zeros(lens.size + 1, np.uint64)
    np.cumsum(lens, out=offs[1:])
    idx = api.Index(np.concatenate(parts), offs)
    del parts, fv
    dev = "cuda"
    out = {}
    saved = capi.bp_get_tuning()
    for j, m in enumerate(ms):
        k = round(0.1 * m)
        terms = np.empty(2 * pairs, np.uint32)
        terms[0::2] = pairs * (j + 1) + np.arange(pairs)
        terms[1::2] = np.arange(pairs)
        toff = np.arange(0, 2 * pairs + 1, 2, dtype=np.uint64)
        tuned = autotune.tune_queries(idx, terms, toff, reps=2, save_cache=False)["best"]
        total = pairs * k
        d_terms = torch.from_numpy(terms.view(np.int32).copy()).to(dev)
        d_off = torch.from_numpy(toff.view(np.int64).copy()).to(dev)
        res = torch.empty(total, dtype=torch.int32, device=dev)
        out_off = torch.empty(pairs + 1, dtype=torch.int64, device=dev)
        counts = torch.empty(pairs, dtype=torch.int32, device=dev)
        sb = capi.bp_query_batch_scratch_bytes(idx.h_lists, terms, toff, total)
        scratch = torch.empty(sb, dtype=torch.uint8, device=dev)
        st = torch.zeros(1, dtype=torch.int32, device=dev)

        def call():
            idx.query_batch_async(d_terms, d_off, pairs, terms.size, res, out_off, counts,
                                  scratch, st, stream)
        with torch.cuda.stream(stream):
            call()
        stream.synchronize()
        assert int(st.item()) == 0
        assert (counts.cpu().numpy() == k).all()  # exact by construction
        ms_b = time_launches(stream, call, reps, 2)
        out[f"m=2^{int(np.log2(m))}"] = {
            "batch_us": round(1e3 * ms_b, 2), "us_per_pair": round(1e3 * ms_b / pairs, 3),
            "pairs_per_s": round(pairs / (ms_b * 1e-3), 1),
            "short_gints": round(pairs * m / (ms_b * 1e-3) / 1e9, 2), "tuned": tuned}
        del scratch, res
    capi.bp_set_tuning(**saved)
    return out


def graph_batch(idx, terms, toff, total, stream, reps, out_pinned: bool = False):
    """bp_query_batch over idx captured in a CUDA graph and replayed `reps`
    times; returns (ms per batch, answers, offsets, counts).  out_pinned:
    the answers go to pinned host memory (written by the kernels over the
    host link, as the serving engine delivers them) instead of HBM."""
    import torch
    from paper_1401_6399_gb300 import capi
    nq = toff.size - 1
    dev = "cuda"
    d_terms = torch.from_numpy(terms.view(np.int32).copy()).to(dev)
    d_off = torch.from_numpy(toff.view(np.int64).copy()).to(dev)
    out = (torch.empty(max(total, 1), dtype=torch.int32).pin_memory() if out_pinned else
           torch.empty(max(total, 1), dtype=torch.int32, device=dev))
    out_off = torch.empty(nq + 1, dtype=torch.int64, device=dev)
    counts = torch.empty(nq, dtype=torch.int32, device=dev)
    sb = capi.bp_query_batch_scratch_bytes(idx.h_lists, terms, toff, total)
    scratch = torch.empty(sb, dtype=torch.uint8, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    with torch.cuda.stream(stream):
        idx.query_batch_async(d_terms, d_off, nq, terms.size, out, out_off, counts, scratch, st,
                              stream)
    stream.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        idx.query_batch_async(d_terms, d_off, nq, terms.size, out, out_off, counts, scratch, st,
                              torch.cuda.current_stream())
    with torch.cuda.stream(stream):  # replays run on the current stream
        g.replay()
        stream.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            g.replay()
        e1.record(stream)
        e1.synchronize()
    assert int(st.item()) == 0, f"bp_query_batch status {int(st.item())}"
    return e0.elapsed_time(e1) / reps, out[:total], out_off, counts


def query_alg_bytes(idx, vals, offs, terms, toff, sample: int, seed: int) -> float:
    """Algorithmic bytes of one fused query, averaged over `sample` queries
    of the batch, computed on the host by Set-vs-Set in the kernel's order:
    the shortest list's whole stream; for every other list, the payload and
    skip-header entry (first value, width byte) of each block that holds a
    still-alive candidate; 4 bytes per answer value."""
    rng = np.random.default_rng(seed)
    nq = toff.size - 1
    L = idx.h_lists
    data = idx.host_data
    total = 0
    for q in rng.choice(nq, min(sample, nq), replace=False):
        t = [int(u) for u in terms[int(toff[q]):int(toff[q + 1])]]
        order = sorted(t, key=lambda u: (int(L["n"][u]), u))
        drv = order[0]
        total += int(L["enc_bytes"][drv])
        cand = vals[int(offs[drv]):int(offs[drv + 1])]
        for u in order[1:]:
            if cand.size == 0:
                break
            f = vals[int(offs[u]):int(offs[u + 1])]
            blk = np.unique(np.searchsorted(f[::128], cand, side="right") - 1)
            blk = blk[blk >= 0]
            eo = int(L["enc_offset"][u])
            off_bw = int(data[eo + 32:eo + 36].view(np.uint32)[0])
            bw = data[eo + off_bw + blk].astype(np.int64)
            total += int(16 * bw.sum()) + 5 * int(blk.size)
            pos = np.minimum(np.searchsorted(f, cand), max(f.size - 1, 0))
            cand = cand[f[pos] == cand] if f.size else cand[:0]
        total += 4 * int(cand.size)
    return total / min(sample, nq)


def batched_queries(stream, reps: int, plain_queries: int, scale: int = 1,
                    hybrid_bs=(8, 16, 32), cpu_threads: int = 0, sm_mhz=None):
    """Synthetic index of 2^19 terms over [0,2^25), Zipf(1) lengths capped at
    2^24 (1.5e9 postings, clustered lists, GL with skip headers, resident);
    100,000 queries of 2-5 terms drawn in proportion to list length.  One
    autotuned, CUDA-graph-captured bp_query_batch vs bp_query_one per query.
    scale > 1 divides the terms, postings, cap and queries by it (a small
    case of the same shape, for profiling)."""
    import torch
    import workloads as W
    from paper_1401_6399_gb300 import api, autotune, capi
    t0 = time.time()
    lens = W.zipf_lengths((1 << 19) // scale, 1_500_000_000 // scale, (1 << 24) // scale)
    vals, offs = W.many("clustered", lens, 0, 1 << 25, 0x4000)
    idx = api.Index(vals, offs)
    terms, toff = W.queries(lens, 100_000 // scale, W.CLUEWEB_TERM_WEIGHTS_2_5, 2, 0x4A00)
    setup_s = time.time() - t0
    # autotune on a 5,000-query sample of the batch
    sample_n = min(5000, toff.size - 1)
    tuned = autotune.tune_queries(idx, terms[: int(toff[sample_n])], toff[: sample_n + 1],
                                  reps=2)
    # exact output size, then a graph-captured batch
    _, o, _ = idx.query_batch(terms, toff, out_cap=1 << 30, on_device=True)
    total = int(o[-1])
    nq = toff.size - 1
    dev = "cuda"
    ms, out, out_off, counts = graph_batch(idx, terms, toff, total, stream, reps)
    o = out_off.cpu().numpy().view(np.uint64)
    c = counts.cpu().numpy().view(np.uint32)
    # the same batch over hybrid indexes (hyb+m2): lists with average gap <= B
    # stored as bitmaps of 2^25 bits; the answers must be the same
    hybrid = {}
    for B in hybrid_bs:
        h0 = time.time()
        hidx = api.Index(vals, offs, hybrid_B=B, universe=1 << 25)
        enc_s = time.time() - h0
        hms, hout, hoff, hcnt = graph_batch(hidx, terms, toff, total, stream, reps)
        assert torch.equal(hoff, out_off) and torch.equal(hcnt, counts)
        assert torch.equal(hout, out), f"hybrid B={B} answers differ"
        nbm = int((hidx.h_lists["layout"] == capi.BP_LAYOUT_BITMAP).sum())
        hybrid[f"B{B}"] = {"bitmap_lists": nbm,
                           "bitmap_postings": int(lens[hidx.h_lists["layout"] ==
                                                       capi.BP_LAYOUT_BITMAP].sum()),
                           "ms_per_batch": round(hms, 3), "queries_per_s": round(nq / (hms * 1e-3), 1),
                           "index_bytes": hidx.compressed_bytes,
                           "bits_per_posting": round(8 * hidx.compressed_bytes / int(lens.sum()), 3),
                           "encode_s": round(enc_s, 1)}
        del hidx, hout, hoff, hcnt
        torch.cuda.empty_cache()
    # plain per-query path on the first queries (decode every list, then
    # intersect pairwise), launched back to back; same answers required
    qn = min(plain_queries, nq)
    lens_np = idx.h_lists["n"].astype(np.int64)
    qterms = [terms[int(toff[q]):int(toff[q + 1])] for q in range(qn)]
    caps = np.array([max(1, int(lens_np[t].min())) for t in qterms], np.int64)
    pos = np.concatenate([[0], np.cumsum(caps)])
    pout = torch.empty(int(pos[-1]), dtype=torch.int32, device=dev)
    pcnt = torch.zeros(qn, dtype=torch.int32, device=dev)
    psb = max(capi.bp_query_one_scratch_bytes(idx.h_lists, t) for t in qterms)
    pscr = torch.empty(psb, dtype=torch.uint8, device=dev)
    pst = torch.zeros(1, dtype=torch.int32, device=dev)

    def plain_all():
        for q in range(qn):
            capi.check(capi.bp_query_one(idx.data.data_ptr(), idx.h_lists, qterms[q],
                                         pout.data_ptr() + 4 * int(pos[q]), int(caps[q]),
                                         pcnt.data_ptr() + 4 * q, pscr.data_ptr(), psb,
                                         pst.data_ptr(), stream.cuda_stream), "bp_query_one")
    plain_all()  # warm-up
    stream.synchronize()
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    plain_all()
    p1.record(stream)
    p1.synchronize()
    ms_plain = p0.elapsed_time(p1)
    assert int(pst.item()) == 0
    pc = pcnt.cpu().numpy()
    for q in range(qn):
        got = out[int(o[q]):int(o[q]) + int(c[q])]
        want = pout[int(pos[q]):int(pos[q]) + int(pc[q])]
        assert torch.equal(got, want), f"batched and plain answers differ for query {q}"
    qps = nq / (ms * 1e-3)
    qps_plain = qn / (ms_plain * 1e-3)
    # algorithmic bytes per query on a sample of 300 queries -> HBM fraction
    apq = query_alg_bytes(idx, vals, offs, terms, toff, 300, 0x4A10)
    peak, peak_kind = load_peaks()
    alg_gbs = apq * nq / (ms * 1e-3) / 1e9
    batched_queries.index = (idx, lens)  # reused by the serving measurement
    cpu = None
    if cpu_threads:
        # the oracle on the first queries of the batch: decode every term's
        # stream, merge (Set-vs-Set); answer sizes must match the GPU's
        qids = np.arange(min(800, nq))
        qps_c, svc, kc = oracle_query_rates(idx.host_data, idx.h_lists, terms, toff, qids,
                                            cpu_threads)
        assert np.array_equal(kc, c[qids].astype(np.int64))
        qps_1, _, _ = oracle_query_rates(idx.host_data, idx.h_lists, terms, toff, qids[:100], 1)
        cpu = {"value": round(qps_c, 1), "unit": "queries/s", "cores": cpu_threads,
               "kind": "oracle", "value_single_thread": round(qps_1, 1),
               "sample": f"the first {qids.size} queries of the batch ({cpu_threads} threads; "
                         "100 on one thread): every term's GL stream decoded by the scalar "
                         "oracle, then Set-vs-Set by merging",
               "gpu_vs_cpu": round(qps / qps_c, 1)}
    # counted for one tuning: reported when the autotuner chose the same
    tkey = "q_main_t{dense_blocks}_{query_chunk_blocks}_{query_warps}_{merge_span}".format(
        **tuned["best"])
    roof = (issue_roof(tkey, nq, ms, sm_mhz or load_sm_max()) if scale == 1 else None)
    return {"queries": nq, "cpu_baseline": cpu, "roofline": roof, "ms_per_batch": round(ms, 3), "queries_per_s": round(qps, 1),
            "plain_queries_timed": qn, "plain_queries_per_s": round(qps_plain, 1),
            "speedup_vs_plain": round(qps / qps_plain, 1), "answer_values": total,
            "index_postings": int(lens.sum()), "index_bytes": idx.compressed_bytes,
            "bits_per_posting": round(8 * idx.compressed_bytes / int(lens.sum()), 3),
            "tuned": tuned["best"], "setup_s": round(setup_s, 1),
            "alg_bytes_per_query_sampled": round(apq, 1),
            "alg_gbs": round(alg_gbs, 1), "hbm_frac": round(alg_gbs / peak, 4),
            "hbm_peak": f"{peak} GB/s ({peak_kind})", "hybrid": hybrid}


def serving_warmup(srv, lens):
    """An unmeasured replay that launches every kernel the engine uses, so
    that module loading and first-launch set-up stay out of the runs."""
    import workloads as W
    wt, wo = W.queries(lens, 4000, W.CLUEWEB_TERM_WEIGHTS_2_8, 2, 0x50FF)
    srv.replay(np.arange(4000, dtype=np.uint64), wt, wo, W.poisson_arrivals(2e4, 4000, 0x51FF))
    srv.drain(600.0)
    srv.poll(with_answers=False)
    srv.batches()


def timeline_summary(recs, res) -> dict:
    """Where the time of the slowest queries went, from the engine's batch
    records: for the batch that held the slowest query, its wait before
    admission, enqueue time and device time; and the largest of each over
    all batches."""
    if recs.size == 0:
        return {}
    lat = np.array([r[5] - r[3] for r in res])
    worst = res[int(np.argmax(lat))]
    # the batch that finished at the worst query's completion time
    k = int(np.argmin(np.abs(recs["done_s"] - worst[5])))
    b = recs[k]
    gap = np.diff(np.sort(recs["done_s"]))

    def ms(x):
        return round(1e3 * float(x), 3)
    return {"batches": int(recs.size),
            "mean_queries_per_batch": round(float(recs["queries"].mean()), 1),
            "worst_query_ms": ms(lat.max()),
            "worst_batch": {"queries": int(b["queries"]), "slot": int(b["slot"]),
                            "wait_before_admit_ms": ms(b["admit_s"] - b["first_arrival_s"]),
                            "enqueue_ms": ms(b["launched_s"] - b["admit_s"]),
                            "device_ms": ms(b["done_s"] - b["launched_s"])},
            "max_wait_before_admit_ms": ms((recs["admit_s"] - recs["first_arrival_s"]).max()),
            "max_enqueue_ms": ms((recs["launched_s"] - recs["admit_s"]).max()),
            "max_device_ms": ms((recs["done_s"] - recs["launched_s"]).max()),
            "max_gap_between_completions_ms": ms(gap.max()) if gap.size else 0.0}


def serve_rate(srv, lens, rate: float, n: int, seed: int) -> dict:
    """One open-loop run of n Poisson arrivals at `rate` queries/s.  Latency
    = completion - scheduled arrival; lag = queued - scheduled arrival."""
    import workloads as W
    terms, toff = W.queries(lens, n, W.CLUEWEB_TERM_WEIGHTS_2_8, 2, seed)
    arrivals = W.poisson_arrivals(rate, n, seed + 0x100)
    srv.batches()  # drop earlier records
    srv.replay(np.arange(n, dtype=np.uint64), terms, toff, arrivals)
    srv.drain(900.0)
    res = srv.poll(with_answers=False)
    recs = srv.batches()
    assert len(res) == n and all(r[2] == 0 for r in res)
    arr = np.array([r[3] for r in res])
    sub = np.array([r[4] for r in res])
    done = np.array([r[5] for r in res])
    lat_ms = (done - arr) * 1e3
    lag_ms = (sub - arr) * 1e3
    span = done.max() - arr.min()
    return {"queries": n, "offered_qps": rate, "offered_s": round(float(arrivals[-1]), 2),
            "achieved_qps": round(n / span, 1),
            "p50_ms": round(float(np.percentile(lat_ms, 50)), 3),
            "p99_ms": round(float(np.percentile(lat_ms, 99)), 3),
            "p999_ms": round(float(np.percentile(lat_ms, 99.9)), 3),
            "submit_lag_p99_ms": round(float(np.percentile(lag_ms, 99)), 4),
            "submit_lag_max_ms": round(float(lag_ms.max()), 4),
            "answer_values": int(sum(r[1] for r in res)),
            "timeline": timeline_summary(recs, res)}


def serving_cpu(idx, lens, threads: int, n: int = 1600) -> dict:
    """The oracle as a closed-loop server on the serving mix (2-8 terms):
    `threads` workers each take the next query when done with the last, so
    a query's latency is its service time (decode every term's stream,
    merge)."""
    import workloads as W
    terms, toff = W.queries(lens, n, W.CLUEWEB_TERM_WEIGHTS_2_8, 2, 0x5000 + 100_000)
    qps, svc, _ = oracle_query_rates(idx.host_data, idx.h_lists, terms, toff, np.arange(n),
                                     threads)
    ms = svc * 1e3
    return {"value": round(qps, 1), "unit": "queries/s", "cores": threads, "kind": "oracle",
            "p50_ms": round(float(np.percentile(ms, 50)), 3),
            "p99_ms": round(float(np.percentile(ms, 99)), 3),
            "sample": f"{n} queries of the 2-8-term serving mix, closed loop on {threads} "
                      "threads (latency = service time: decode every term, merge)"}


def serving(idx, lens, rates=(1e4, 1e5, 1e6)):
    """Open-loop Poisson arrivals of 2-8-term queries against the resident
    index; the engine batches continuously over 4 slots of 1 GiB (at most
    4 GiB of scratch and answers in flight).  Each rate runs for 10 s of
    arrivals or 1e6 queries, whichever is fewer.  Latency = completion -
    scheduled arrival."""
    from paper_1401_6399_gb300 import api
    out = {}
    srv = api.Server(idx, slots=4, max_batch_queries=8192, max_terms=8, slot_bytes=1 << 30,
                     deliver_answers=False)
    try:
        serving_warmup(srv, lens)
        for rate in rates:
            n = int(min(1_000_000, 10 * rate))
            out[f"{int(rate)}/s"] = serve_rate(srv, lens, rate, n, 0x5000 + int(rate))
        out["engine"] = srv.stats()
    finally:
        srv.close()
    # the offline rate on the same 2-8-term mix (first 50,000 queries of the
    # 1M/s run), answers on the device: what the engine saturates against
    import torch
    import workloads as W
    terms, toff = W.queries(lens, 1_000_000, W.CLUEWEB_TERM_WEIGHTS_2_8, 2, 0x5000 + 1_000_000)
    nq = 50_000
    terms, toff = terms[: int(toff[nq])], toff[: nq + 1]
    _, o, _ = idx.query_batch(terms, toff, out_cap=1 << 31, on_device=True)
    stream = torch.cuda.Stream()
    ms, res, _, _ = graph_batch(idx, terms, toff, int(o[-1]), stream, 3)
    del res
    torch.cuda.empty_cache()
    # the same batch with its answers written to pinned host memory, as the
    # engine delivers them: the host link's share of the saturation rate
    ms_h, res, _, _ = graph_batch(idx, terms, toff, int(o[-1]), stream, 3, out_pinned=True)
    del res
    out["offline_same_mix"] = {"queries": nq, "ms_per_batch": round(ms, 3),
                               "queries_per_s": round(nq / (ms * 1e-3), 1),
                               "answer_values": int(o[-1]),
                               "answers_to_host_queries_per_s": round(nq / (ms_h * 1e-3), 1),
                               "answers_to_host_gbs": round(4 * int(o[-1]) / (ms_h * 1e-3) / 1e9,
                                                            1)}
    return out


def serving_sweep(idx, lens, rate=1e6, n=1_000_000):
    """Saturation of the engine at `rate` offered queries/s for several slot
    counts and batch sizes, with 4 GiB in flight in total: is the achieved
    rate set by the slots or by the device?"""
    from paper_1401_6399_gb300 import api
    rows = []
    for slots in (2, 4, 8, 16):
        for mbq in (1024, 8192, 65536):
            srv = api.Server(idx, slots=slots, max_batch_queries=mbq, max_terms=8,
                             slot_bytes=(4 << 30) // slots, deliver_answers=False)
            try:
                serving_warmup(srv, lens)
                r = serve_rate(srv, lens, rate, n, 0x5000 + int(rate))
                st = srv.stats()
            finally:
                srv.close()
            rows.append({"slots": slots, "max_batch_queries": mbq,
                         "achieved_qps": r["achieved_qps"], "p50_ms": r["p50_ms"],
                         "p99_ms": r["p99_ms"], "max_busy_slots": st["max_busy_slots"],
                         "mean_queries_per_batch": r["timeline"].get("mean_queries_per_batch"),
                         "max_device_ms": r["timeline"].get("max_device_ms")})
    return rows


def run_ours(args, rank, world, local):
    import torch
    dist = dist_init(world, local)
    sys.path.insert(0, ROOT)
    import __graft_entry__ as ge
    if rank == 0:
        ge.build()
    barrier(dist)
    ge.build()
    from paper_1401_6399_gb300 import api, capi

    n = 1 << args.log2n
    L = args.lists
    seed = rank_seed(rank)
    lists = make_lists("uniform", L, n, UNIVERSE, seed)
    layout = {"paper": capi.BP_LAYOUT_PAPER, "gpu": capi.BP_LAYOUT_GPU,
              "pfor": capi.BP_LAYOUT_PFOR}[args.layout]
    lay_name = {capi.BP_LAYOUT_PAPER: "pl", capi.BP_LAYOUT_GPU: "gl",
             capi.BP_LAYOUT_PFOR: "gp"}[layout]
    encs = encode_all(lists, layout)
    batch = api.ListBatch(encs, [n] * L, layout)
    # kernels of one bp_decode_batch call: GL the D4 kernel and the one for
    # other kinds (it leaves at once on D4 lists); PL plan, parse, resolve,
    # emit, leftover, four pl_tiles instances (D4 and other kinds, narrow and
    # wide stage; the three not chosen leave at once), tail
    launches_per_step = {capi.BP_LAYOUT_GPU: 2, capi.BP_LAYOUT_PAPER: 10,
                         capi.BP_LAYOUT_PFOR: 1}[layout]
    total_n = n * L
    out = torch.empty(total_n, dtype=torch.int32, device="cuda")
    status = api.status_tensor()
    stream = torch.cuda.Stream()

    # correctness gate before timing: the decoded lists are the input lists
    with torch.cuda.stream(stream):
        batch.decode_into(out, status, stream)
    stream.synchronize()
    assert int(status.item()) == 0, "decode reported an error"
    want = torch.from_numpy(np.concatenate(lists).view(np.int32)).to("cuda")
    assert torch.equal(out, want), "decoded output differs from the input lists"
    del want

    def step():
        batch.decode_into(out, status, stream)

    gpu_index = int((os.environ.get("CUDA_VISIBLE_DEVICES") or str(local)).split(",")[0]) \
        if (os.environ.get("CUDA_VISIBLE_DEVICES") or "").split(",")[0].isdigit() else local
    clocks = ClockSampler(gpu_index)
    clocks.start()
    time.sleep(0.3)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(dist)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    w0 = time.time()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    e1.synchronize()
    w1 = time.time()
    barrier(dist)
    torch.cuda.synchronize()
    ms_local = e0.elapsed_time(e1) / args.steps
    ms = max_over_ranks(dist, ms_local)
    clk = clocks.summary(w0, w1)
    assert int(status.item()) == 0

    value = whole_job_rate(world, total_n, ms)  # Gint/s over all ranks
    comp_bytes = batch.compressed_bytes
    alg_bytes = comp_bytes + 4 * total_n  # per launch (one launch per step)
    peak, peak_kind = load_peaks()
    achieved = alg_bytes / (ms_local * 1e-3) / 1e9
    sha = kernel_sha()
    traffic = profiled_traffic(sha) if layout == capi.BP_LAYOUT_GPU else None

    result = {
        "metric": METRIC if layout != capi.BP_LAYOUT_PFOR else "S4-FastPFOR-D4 decoded Gint/s",
        "value": round(value, 3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": f"decode {L} lists x 2^{args.log2n} uniform uint32 of [0,2^29) "
                               f"per GPU, "
                               f"{ {'gl': 'S4-BP128-D4 GPU', 'pl': 'S4-BP128-D4 paper', 'gp': 'S4-FastPFOR-D4 GPU page'}[lay_name]} layout, "
                               "one bp_decode_batch call",
                   "lists_per_gpu": L, "ints_per_list": n,
                   "compressed_bytes_per_gpu": comp_bytes,
                   "bits_per_int": round(8 * comp_bytes / total_n, 3),
                   "l2": "inputs (compressed) and outputs larger than L2; no flush",
                   "parallelism": f"weak x{world}"},
        "gpu_launches": args.steps * launches_per_step,
        "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"],
                   "reasons": clk["reasons"], "samples": clk["samples"]},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": traffic,
                     "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                     "kernel": {"gl": "gl_decode_kernel<false> (+ gl_decode_other_kernel, "
                                      "empty for D4 lists; both timed)",
                                "pl": "PL decode call (all its kernels)",
                                "gp": "gp_decode_kernel<false>"}[lay_name],
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "frac_of_nominal_8TBs": round(achieved / 8000.0, 4)},
    }

    if layout == capi.BP_LAYOUT_GPU:
        result["roofline_issue"] = issue_roof("gl_decode", total_n / 128, ms_local,
                                              clk["sm_mhz"] or load_sm_max())
        # context for the HBM fraction: the decode is write-dominated (1.9 GB in,
        # 8.6 GB out) while the measured peak is a half-read, half-write copy;
        # a pure write of the same output (torch's fill of 8 GiB) on this GPU
        def fill():
            with torch.cuda.stream(stream):  # on the stream the events are recorded on
                out.fill_(0)
        ms_fill = time_launches(stream, fill, 5, 2)
        result["roofline"]["write_only_fill_gbs"] = round(4 * total_n / (ms_fill * 1e-3) / 1e9, 1)

    # end to end through the host-buffer C-ABI call (pinned host memory),
    # before the other measurements allocate host memory (8 GiB of pinned
    # output taken after them ran at half the rate on some boxes)
    if not args.no_e2e:
        h_data = torch.from_numpy(batch.host_data).pin_memory()
        h_lists = torch.from_numpy(batch.lists.view(np.uint8).copy()).pin_memory()
        h_out = torch.empty(total_n, dtype=torch.int32).pin_memory()
        h_status = torch.zeros(1, dtype=torch.int32).pin_memory()
        d_data = torch.empty_like(batch.data)
        d_lists = torch.empty_like(batch.d_lists)

        def e2e_step():
            capi.check(capi.bp_decode_batch_host(
                h_data.data_ptr(), h_data.numel(), h_lists.data_ptr(), L, batch.total_units,
                layout, d_data.data_ptr(), d_lists.data_ptr(), out.data_ptr(),
                total_n, h_out.data_ptr(), batch.scratch.data_ptr(), batch.scratch_bytes,
                status.data_ptr(), h_status.data_ptr(), stream.cuda_stream), "e2e")

        e2e_steps = max(3, min(20, args.steps // 10))
        barrier(dist)
        ms_e = time_launches(stream, e2e_step, e2e_steps, 2)
        ms_e = max_over_ranks(dist, ms_e)
        assert int(h_status.item()) == 0
        assert np.array_equal(h_out[:1000].numpy().view(np.uint32), lists[0][:1000])
        result["e2e"] = {"value": round(world * total_n / (ms_e * 1e-3) / 1e9, 3), "unit": UNIT,
                         "h2d_bytes_per_step": int(h_data.numel() + h_lists.numel()),
                         "d2h_bytes_per_step": int(4 * total_n + 4),
                         "ms_per_step": round(ms_e, 3), "steps": e2e_steps,
                         "call": "bp_decode_batch_host"}
        del h_data, h_lists, h_out, d_data, d_lists

    extra = {}
    if not args.no_extra:
        reps = max(5, min(50, args.steps // 4))
        sm_mhz = clk["sm_mhz"] or load_sm_max()
        # decode + sum (compressed bytes only)
        sums = torch.zeros(L, dtype=torch.int64, device="cuda")
        ms_sum = time_launches(stream, lambda: batch.sum_into(sums, status, stream), reps, 2)
        extra[f"{lay_name}_decode_sum_uniform"] = {
            "gints": round(total_n / (ms_sum * 1e-3) / 1e9, 2), "ms": round(ms_sum, 4),
            "gbs_compressed": round(comp_bytes / (ms_sum * 1e-3) / 1e9, 1),
            "roofline": (issue_roof("gl_decode_sum", total_n / 128, ms_sum, sm_mhz)
                         if lay_name == "gl" else None)}
        # clustered lists
        cl = make_lists("clustered", L, n, UNIVERSE, seed + 1000)
        cbatch = api.ListBatch(encode_all(cl, capi.BP_LAYOUT_GPU), [n] * L, capi.BP_LAYOUT_GPU)
        with torch.cuda.stream(stream):
            cbatch.decode_into(out, status, stream)
        stream.synchronize()
        assert torch.equal(out, torch.from_numpy(np.concatenate(cl).view(np.int32)).to("cuda"))
        ms_c = time_launches(stream, lambda: cbatch.decode_into(out, status, stream), reps, 2)
        extra["gl_decode_clustered"] = {
            "gints": round(total_n / (ms_c * 1e-3) / 1e9, 2), "ms": round(ms_c, 4),
            "bits_per_int": round(8 * cbatch.compressed_bytes / total_n, 3),
            "hbm_gbs": round((cbatch.compressed_bytes + 4 * total_n) / (ms_c * 1e-3) / 1e9, 1)}
        del cbatch
        # S4-FastPFOR (GP layout, Section 4.4) on the same uniform and
        # clustered lists, D4 and D1 (the paper's query experiments use D1)
        pfor = {}
        for dname, data_lists in (("uniform", lists), ("clustered", cl)):
            want = torch.from_numpy(np.concatenate(data_lists).view(np.int32)).to("cuda")
            for kname, kind in (("D4", capi.BP_DELTA_D4), ("D1", capi.BP_DELTA_D1)):
                gb = api.ListBatch(encode_all_kind(data_lists, capi.BP_LAYOUT_PFOR, kind),
                                   [n] * L, capi.BP_LAYOUT_PFOR)
                with torch.cuda.stream(stream):
                    gb.decode_into(out, status, stream)
                stream.synchronize()
                assert int(status.item()) == 0 and torch.equal(out, want)
                ms_g = time_launches(stream, lambda: gb.decode_into(out, status, stream),
                                     max(3, reps // 5), 1)
                gl_bytes = sum(e.size for e in encode_all_kind(data_lists, capi.BP_LAYOUT_GPU,
                                                                kind))
                pfor[f"{dname}_{kname}"] = {
                    "gints": round(total_n / (ms_g * 1e-3) / 1e9, 2), "ms": round(ms_g, 4),
                    "bits_per_int": round(8 * gb.compressed_bytes / total_n, 3),
                    "gl_bits_per_int": round(8 * gl_bytes / total_n, 3),
                    "hbm_gbs": round((gb.compressed_bytes + 4 * total_n) / (ms_g * 1e-3) / 1e9,
                                     1)}
                if dname == "uniform" and kname == "D4":
                    pfor[f"{dname}_{kname}"]["roofline"] = issue_roof(
                        "gp_decode", total_n / 128, ms_g, sm_mhz)
                del gb
            del want
        extra["gp_decode_s4fastpfor"] = pfor
        del cl
        # paper layout
        pbatch = api.ListBatch(encode_all(lists, capi.BP_LAYOUT_PAPER), [n] * L,
                               capi.BP_LAYOUT_PAPER)
        with torch.cuda.stream(stream):
            pbatch.decode_into(out, status, stream)
        stream.synchronize()
        assert int(status.item()) == 0
        assert torch.equal(out, torch.from_numpy(np.concatenate(lists).view(np.int32)).to("cuda"))
        ms_p = time_launches(stream, lambda: pbatch.decode_into(out, status, stream),
                             max(3, reps // 5), 1)
        pl_gbs = (pbatch.compressed_bytes + 4 * total_n) / (ms_p * 1e-3) / 1e9
        extra["pl_decode_uniform"] = {
            "gints": round(total_n / (ms_p * 1e-3) / 1e9, 2), "ms": round(ms_p, 4),
            "bits_per_int": round(8 * pbatch.compressed_bytes / total_n, 3),
            "roofline": {"bound": "hbm", "achieved": round(pl_gbs, 1), "peak": peak,
                         "unit": "GB/s", "frac": round(pl_gbs / peak, 4),
                         "scope": "the whole bp_decode_batch call (parse, offsets, decode); "
                                  "algorithmic bytes = compressed + 4 B per integer, the "
                                  "stream being read twice (parse and decode) not counted"}}
        del pbatch
        # sparser lists (about 9 bits/int): paper-layout chunks wider than
        # the shared-memory stage, read from global memory after an L2 prefetch
        sp = make_lists("uniform", 8, n, 1 << 31, SEED_BASE + 0x100)
        sn = 8 * n
        sout = out[:sn]
        swant = torch.from_numpy(np.concatenate(sp).view(np.int32)).to("cuda")
        sparse = {"lists": 8, "ints_per_list": n, "universe": "[0,2^31)"}
        for lname, lay in (("paper", capi.BP_LAYOUT_PAPER), ("gpu", capi.BP_LAYOUT_GPU)):
            sb = api.ListBatch(encode_all(sp, lay), [n] * 8, lay)
            with torch.cuda.stream(stream):
                sb.decode_into(sout, status, stream)
            stream.synchronize()
            assert int(status.item()) == 0
            assert torch.equal(sout, swant)
            ms_s = time_launches(stream, lambda: sb.decode_into(sout, status, stream),
                                 max(3, reps // 5), 1)
            sparse[lname] = {"gints": round(sn / (ms_s * 1e-3) / 1e9, 2), "ms": round(ms_s, 4),
                             "bits_per_int": round(8 * sb.compressed_bytes / sn, 3)}
            del sb
        extra["decode_sparse_uniform"] = sparse
        del sp, swant, sout
        # the other kinds of differential coding (Section 5), both layouts
        kinds = {}
        for kname, kind in (("DM", capi.BP_DELTA_DM), ("D2", capi.BP_DELTA_D2),
                            ("D1", capi.BP_DELTA_D1)):
            for lname, lay in (("gl", capi.BP_LAYOUT_GPU), ("pl", capi.BP_LAYOUT_PAPER)):
                encs_k = encode_all_kind(lists, lay, kind)
                kb = api.ListBatch(encs_k, [n] * L, lay)
                with torch.cuda.stream(stream):
                    kb.decode_into(out, status, stream)
                stream.synchronize()
                assert int(status.item()) == 0
                assert torch.equal(out, torch.from_numpy(np.concatenate(lists).view(np.int32))
                                   .to("cuda"))
                ms_k = time_launches(stream, lambda: kb.decode_into(out, status, stream),
                                     max(3, reps // 5), 1)
                kinds[f"{lname}_{kname}"] = {
                    "gints": round(total_n / (ms_k * 1e-3) / 1e9, 2), "ms": round(ms_k, 4),
                    "bits_per_int": round(8 * kb.compressed_bytes / total_n, 3)}
                del kb, encs_k
        extra["decode_kinds_uniform"] = kinds
        del out
        torch.cuda.empty_cache()
        try:
            extra["unpack_sweep"] = unpack_sweep(stream)
        except Exception as e:
            extra["unpack_sweep"] = {"error": repr(e)[:300]}
        cpu_t = 0 if (args.no_cpu or world > 1 or rank != 0) else min(16, os.cpu_count() or 1)
        try:
            extra["pair_sweep"] = pair_sweep(stream, reps=20, cpu_threads=cpu_t, sm_mhz=sm_mhz)
        except Exception as e:  # report, do not hide the headline
            extra["pair_sweep"] = {"error": repr(e)[:300]}
        try:
            extra["pair_batch_64"] = pair_batch(stream, reps=10)
        except Exception as e:
            extra["pair_batch_64"] = {"error": repr(e)[:300]}
        torch.cuda.empty_cache()
        try:
            extra["batched_queries"] = batched_queries(stream, reps=5, plain_queries=2000,
                                                       cpu_threads=cpu_t, sm_mhz=sm_mhz)
        except Exception as e:
            extra["batched_queries"] = {"error": repr(e)[:300]}
        try:
            if hasattr(batched_queries, "index"):
                extra["serving"] = serving(*batched_queries.index)
                if cpu_t:
                    extra["serving"]["cpu_baseline"] = serving_cpu(*batched_queries.index, cpu_t)
                del batched_queries.index
        except Exception as e:
            extra["serving"] = {"error": repr(e)[:300]}
        torch.cuda.empty_cache()
        out = torch.empty(total_n, dtype=torch.int32, device="cuda")
    clocks.stop()
    if extra:
        result["secondary"] = extra

    # the oracle on the host cores, rank 0 at N = 1 only
    if world == 1 and rank == 0 and not args.no_cpu:
        threads = min(16, os.cpu_count() or 1)
        k = L
        val, dt, used = oracle_decode_rate(encs[:k], [n] * k, threads, layout)
        val1, dt1, _ = oracle_decode_rate(encs[:1], [n], 1, layout)
        result["cpu_baseline"] = {
            "value": round(val, 4), "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": f"all {k} {lay_name.upper()}-encoded lists "
                      f"(2^{args.log2n} ints each) decoded by "
                      f"the scalar C oracle on {used} threads, {dt:.1f} s wall",
            "value_single_thread": round(val1, 4),
            "sample_single_thread": f"1 list on 1 thread, {dt1:.1f} s"}
    if rank == 0:
        print(json.dumps(result), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def profile_case(args) -> dict:
    """One kernel's case, launched warmup + steps times on its own (the
    command ncu captures).  Decodes: 4 lists of 2^26 uniform integers, more
    than L2 in and out.  pair: the fused intersection of the m = n = 2^22
    pair of the sweep, L2 flushed before each call.  queries: the batched
    queries (default tuning) on the index --query-scale times smaller."""
    import torch
    import __graft_entry__ as ge
    ge.build()
    from paper_1401_6399_gb300 import api, capi
    if args.profile_case == "pair":
        import workloads as W
        f = W.uniform(1 << 22, 0, 1 << 26, 0x3000)
        r = W.pair_short(f, 1 << 22, round(0.1 * (1 << 22)), 1 << 26, 0x3000 + (1 << 22))
        er = api.to_device(capi.bp_encode(r, capi.BP_LAYOUT_GPU, nthreads=8))
        ef = api.to_device(capi.bp_encode(f, capi.BP_LAYOUT_GPU, nthreads=8))
        flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
        stream = torch.cuda.Stream()
        tot = 0.0
        for i in range(args.warmup + args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = api.intersect_pair(er, r.size, ef, f.size, capi.BP_LAYOUT_GPU,
                                     capi.BP_MODE_FUSED, stream=stream)
            e1.record(stream)
            e1.synchronize()
            if i >= args.warmup:
                tot += e0.elapsed_time(e1)
        assert res.numel() == round(0.1 * (1 << 22))
        return {"profile_case": "pair", "us": round(1e3 * tot / args.steps, 2)}
    if args.profile_case == "queries":
        import workloads as W
        sc = args.query_scale
        lens = W.zipf_lengths((1 << 19) // sc, 1_500_000_000 // sc, (1 << 24) // sc)
        vals, offs = W.many("clustered", lens, 0, 1 << 25, 0x4000)
        idx = api.Index(vals, offs)
        if args.profile_tuning:
            d, c, wp, mg = (int(x) for x in args.profile_tuning.split(","))
            capi.bp_set_tuning(dense_blocks=d, query_chunk_blocks=c, query_warps=wp,
                               merge_span=mg)
        terms, toff = W.queries(lens, 100_000 // sc, W.CLUEWEB_TERM_WEIGHTS_2_5, 2, 0x4A00)
        if args.profile_queries:  # a sample: the first N queries of the batch
            nq = min(args.profile_queries, toff.size - 1)
            terms, toff = terms[: int(toff[nq])], toff[: nq + 1]
        _, o, _ = idx.query_batch(terms, toff, out_cap=1 << 31, on_device=True)
        stream = torch.cuda.Stream()
        ms, _, _, _ = graph_batch(idx, terms, toff, int(o[-1]), stream, args.steps)
        return {"profile_case": "queries", "scale": sc, "queries": int(toff.size - 1),
                "tuning": capi.bp_get_tuning(),
                "ms": round(ms, 4), "queries_per_s": round((toff.size - 1) / (ms * 1e-3), 1)}
    n, L = 1 << args.log2n, 4
    lists = make_lists("uniform", L, n, UNIVERSE, SEED_BASE)
    layout = {"decode": capi.BP_LAYOUT_GPU, "decode_sum": capi.BP_LAYOUT_GPU,
              "gp_decode": capi.BP_LAYOUT_PFOR, "pl_decode": capi.BP_LAYOUT_PAPER}[args.profile_case]
    batch = api.ListBatch(encode_all(lists, layout), [n] * L, layout)
    stream = torch.cuda.Stream()
    status = api.status_tensor()
    if args.profile_case == "decode_sum":
        sums = torch.zeros(L, dtype=torch.int64, device="cuda")
        fn = lambda: batch.sum_into(sums, status, stream)  # noqa: E731
    else:
        out = torch.empty(n * L, dtype=torch.int32, device="cuda")
        fn = lambda: batch.decode_into(out, status, stream)  # noqa: E731
    ms = time_launches(stream, fn, args.steps, args.warmup)
    assert int(status.item()) == 0
    return {"profile_case": args.profile_case, "lists": L, "ints_per_list": n,
            "ms": round(ms, 4), "gints": round(n * L / (ms * 1e-3) / 1e9, 2),
            "compressed_bytes": batch.compressed_bytes}


def main():
    args = parse_args()
    rank, world, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.pairs_only:
        # the pair sweep alone (for profiling the pair kernels); one JSON line
        import torch
        import __graft_entry__ as ge
        ge.build()
        stream = torch.cuda.Stream()
        print(json.dumps({"pair_sweep": pair_sweep(stream, reps=args.steps),
                          "pair_batch_64": pair_batch(stream, reps=max(3, args.steps))}),
              flush=True)
        return
    if args.serving_only:
        import torch
        import __graft_entry__ as ge
        ge.build()
        stream = torch.cuda.Stream()
        batched_queries(stream, reps=2, plain_queries=10, hybrid_bs=())
        print(json.dumps({"serving": serving(*batched_queries.index)}), flush=True)
        return
    if args.serving_sweep:
        import torch
        import __graft_entry__ as ge
        ge.build()
        stream = torch.cuda.Stream()
        batched_queries(stream, reps=2, plain_queries=10, hybrid_bs=())
        idx, lens = batched_queries.index
        print(json.dumps({"serving_sweep": serving_sweep(idx, lens)}), flush=True)
        return
    if args.profile_case:
        print(json.dumps(profile_case(args)), flush=True)
        return
    if args.queries_only:
        # the batched-query measurement alone, on an index `--query-scale`
        # times smaller (for profiling its kernels); one JSON line
        import torch
        import __graft_entry__ as ge
        ge.build()
        stream = torch.cuda.Stream()
        res = batched_queries(stream, reps=args.steps, plain_queries=100,
                              scale=args.query_scale, hybrid_bs=())
        print(json.dumps({"batched_queries": res, "scale": args.query_scale}), flush=True)
        return
    run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
