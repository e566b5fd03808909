"""PyTorch-facing helpers over the C ABI.  PyTorch only allocates device
memory and supplies streams; every step of decoding and intersection runs in
libbp128.so's kernels.  The helpers that return results synchronise the
stream to read the device status word and raise BPError on a data error."""
from __future__ import annotations

import numpy as np
import torch

from . import capi
from .capi import BP_LIST, BP_LAYOUT_GPU, BP_LAYOUT_PAPER, check  # noqa: F401


def _stream(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def status_tensor(device="cuda") -> torch.Tensor:
    return torch.zeros(1, dtype=torch.int32, device=device)


def check_status(status: torch.Tensor, what: str) -> None:
    code = int(status.item())
    if code != capi.BP_OK:
        raise capi.BPError(code, what)


def to_device(enc: np.ndarray, device="cuda") -> torch.Tensor:
    """Copy an encoded stream (uint8) to the device (torch allocations are
    256-byte aligned, which meets the 16-byte rule of the ABI)."""
    a = np.ascontiguousarray(enc, np.uint8)
    t = torch.from_numpy(a if a.flags.writeable else a.copy())
    return t.to(device, non_blocking=False)


def as_u32(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)


def decode(enc_dev: torch.Tensor, layout: int, n: int, stream=None) -> torch.Tensor:
    if stream is not None:
        with torch.cuda.stream(stream):
            return decode(enc_dev, layout, n)
    out = torch.empty(max(n, 1), dtype=torch.int32, device=enc_dev.device)
    sb = capi.bp_decode_scratch_bytes(n, layout)
    scratch = torch.empty(max(sb, 1), dtype=torch.uint8, device=enc_dev.device)
    st = status_tensor(enc_dev.device)
    check(capi.bp_decode(enc_dev.data_ptr(), enc_dev.numel(), layout, n, out.data_ptr(), n,
                         scratch.data_ptr(), sb, st.data_ptr(), _stream(stream)), "bp_decode")
    check_status(st, "bp_decode")
    return out[:n]


def decode_sum(enc_dev: torch.Tensor, layout: int, n: int, stream=None) -> int:
    if stream is not None:
        with torch.cuda.stream(stream):
            return decode_sum(enc_dev, layout, n)
    acc = torch.zeros(1, dtype=torch.int64, device=enc_dev.device)
    sb = capi.bp_decode_scratch_bytes(n, layout)
    scratch = torch.empty(max(sb, 1), dtype=torch.uint8, device=enc_dev.device)
    st = status_tensor(enc_dev.device)
    check(capi.bp_decode_sum(enc_dev.data_ptr(), enc_dev.numel(), layout, n, acc.data_ptr(),
                             scratch.data_ptr(), sb, st.data_ptr(), _stream(stream)),
          "bp_decode_sum")
    check_status(st, "bp_decode_sum")
    return int(acc.item()) & ((1 << 64) - 1)


class ListBatch:
    """Several encoded lists of one layout packed into one device buffer
    (each stream 16-byte aligned) with planned descriptors."""

    def __init__(self, encs: list[np.ndarray], counts: list[int], layout: int, device="cuda"):
        self.layout = layout
        self.count = len(encs)
        offs, pos = [], 0
        for e in encs:
            offs.append(pos)
            pos += (e.size + 15) // 16 * 16
        host = np.zeros(max(pos, 16), np.uint8)
        for o, e in zip(offs, encs):
            host[o:o + e.size] = e
        lists = np.zeros(self.count, BP_LIST)
        out_off = 0
        for i, (o, e, n) in enumerate(zip(offs, encs, counts)):
            lists[i] = (o, e.size, out_off, 0, n, layout, 0)
            out_off += n
        self.total_units = capi.bp_plan_lists(lists)
        self.lists = lists
        self.total_n = out_off
        self.host_data = host
        self.data = to_device(host, device)
        self.d_lists = torch.from_numpy(lists.view(np.uint8).copy()).to(device)
        self.scratch_bytes = capi.bp_decode_batch_scratch_bytes(lists)
        self.scratch = torch.empty(max(self.scratch_bytes, 1), dtype=torch.uint8, device=device)
        self.compressed_bytes = int(sum(e.size for e in encs))

    def decode_into(self, out: torch.Tensor, status: torch.Tensor, stream=None) -> None:
        check(capi.bp_decode_batch(self.data.data_ptr(), self.d_lists.data_ptr(), self.count,
                                   self.total_units, self.layout, out.data_ptr(), out.numel(),
                                   None, self.scratch.data_ptr(), self.scratch_bytes,
                                   status.data_ptr(), _stream(stream)), "bp_decode_batch")

    def sum_into(self, sums: torch.Tensor, status: torch.Tensor, stream=None) -> None:
        check(capi.bp_decode_batch(self.data.data_ptr(), self.d_lists.data_ptr(), self.count,
                                   self.total_units, self.layout, None, 0, sums.data_ptr(),
                                   self.scratch.data_ptr(), self.scratch_bytes,
                                   status.data_ptr(), _stream(stream)), "bp_decode_batch")

    def ablation_into(self, out: torch.Tensor, status: torch.Tensor, mode: int,
                      stream=None) -> None:
        """GL only: the list-major decoder with the prefix integrated (mode
        0) or as a separate pass through shared memory (1)
        (bp_decode_ablation)."""
        check(capi.bp_decode_ablation(self.data.data_ptr(), self.d_lists.data_ptr(), self.count,
                                      out.data_ptr(), out.numel(), status.data_ptr(), int(mode),
                                      _stream(stream)),
              "bp_decode_ablation")

    def decode(self) -> torch.Tensor:
        out = torch.empty(max(self.total_n, 1), dtype=torch.int32, device=self.data.device)
        st = status_tensor(self.data.device)
        self.decode_into(out, st)
        check_status(st, "bp_decode_batch")
        return out[: self.total_n]

    def sums(self) -> np.ndarray:
        s = torch.zeros(self.count, dtype=torch.int64, device=self.data.device)
        st = status_tensor(self.data.device)
        self.sum_into(s, st)
        check_status(st, "bp_decode_batch")
        return s.cpu().numpy().view(np.uint64)


def intersect_pair(a_dev: torch.Tensor, n_a: int, b_dev: torch.Tensor, n_b: int,
                   layout: int = capi.BP_LAYOUT_GPU, mode: int = capi.BP_MODE_AUTO,
                   stream=None) -> torch.Tensor:
    """Sorted intersection of two device-resident compressed lists."""
    if stream is not None:
        with torch.cuda.stream(stream):
            return intersect_pair(a_dev, n_a, b_dev, n_b, layout, mode)
    dev = a_dev.device
    cap = max(1, min(n_a, n_b))
    out = torch.empty(cap, dtype=torch.int32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)
    sb = capi.bp_intersect_scratch_bytes(n_a, n_b, layout, mode)
    scratch = torch.empty(max(sb, 16), dtype=torch.uint8, device=dev)
    st = status_tensor(dev)
    check(capi.bp_intersect_pair(a_dev.data_ptr(), a_dev.numel(), n_a, b_dev.data_ptr(),
                                 b_dev.numel(), n_b, layout, mode, out.data_ptr(), cap,
                                 cnt.data_ptr(), scratch.data_ptr(), sb, st.data_ptr(),
                                 _stream(None)), "bp_intersect_pair")
    check_status(st, "bp_intersect_pair")
    return out[: int(cnt.item())]


class Index:
    """A resident index: one GL stream per term in one device buffer, the
    descriptors on host and device, and the query calls over it."""

    def __init__(self, values: np.ndarray, offs: np.ndarray, device="cuda", nthreads: int = 16,
                 hybrid_B: int = 0, universe: int = 0):
        """hybrid_B > 0: lists whose average gap is at most hybrid_B are stored
        as bitmaps of `universe` bits (hyb+m2)."""
        if hybrid_B:
            host, lists = capi.bp_index_encode_hybrid(values, offs, universe, hybrid_B, nthreads)
        else:
            host, lists = capi.bp_index_encode(values, offs, nthreads)
        self.h_lists = lists
        self.n_terms = lists.size
        self.host_data = host
        self.data = to_device(host, device)
        self.d_lists = torch.from_numpy(lists.view(np.uint8).copy()).to(device)
        self.compressed_bytes = int(host.size)
        self.device = device

    def lengths(self) -> np.ndarray:
        return self.h_lists["n"].astype(np.uint64)

    def query_batch_async(self, d_terms: torch.Tensor, d_term_off: torch.Tensor, nq: int,
                          total_terms: int, out: torch.Tensor, out_off: torch.Tensor,
                          counts: torch.Tensor, scratch: torch.Tensor, status: torch.Tensor,
                          stream=None) -> None:
        check(capi.bp_query_batch(self.data.data_ptr(), self.d_lists.data_ptr(), self.n_terms,
                                  d_terms.data_ptr() if total_terms else None,
                                  d_term_off.data_ptr(), total_terms, nq, out.data_ptr(),
                                  out.numel(), out_off.data_ptr(), counts.data_ptr(),
                                  scratch.data_ptr(), scratch.numel(), status.data_ptr(),
                                  _stream(stream)), "bp_query_batch")

    def query_batch(self, terms: np.ndarray, term_off: np.ndarray, out_cap: int | None = None,
                    retry: bool = True, on_device: bool = False):
        """Answer all queries; returns a list of uint32 arrays.  If the
        answers overflow out_cap the call is repeated once with the exact
        total (the counts of a call that ran out of room are still exact)."""
        terms = np.ascontiguousarray(terms, np.uint32)
        term_off = np.ascontiguousarray(term_off, np.uint64)
        nq = term_off.size - 1
        if out_cap is None:
            lens = self.h_lists["n"]
            out_cap = 0
            for q in range(nq):
                t = terms[term_off[q]:term_off[q + 1]]
                out_cap += int(lens[t].min()) if t.size else 0
        out_cap = max(int(out_cap), 1)
        dev = self.device
        d_terms = torch.from_numpy(terms.view(np.int32).copy() if terms.size else
                                   np.zeros(1, np.int32)).to(dev)
        d_off = torch.from_numpy(term_off.view(np.int64).copy()).to(dev)
        out_off = torch.empty(nq + 1, dtype=torch.int64, device=dev)
        counts = torch.empty(max(nq, 1), dtype=torch.int32, device=dev)
        for attempt in range(2):
            sb = capi.bp_query_batch_scratch_bytes(self.h_lists, terms, term_off, out_cap)
            out = torch.empty(out_cap, dtype=torch.int32, device=dev)
            scratch = torch.empty(max(sb, 16), dtype=torch.uint8, device=dev)
            st = status_tensor(dev)
            self.query_batch_async(d_terms, d_off, nq, int(term_off[-1]), out, out_off, counts,
                                   scratch, st)
            code = int(st.item())
            total = int(out_off[nq].item()) if nq else 0
            del scratch
            if code == capi.BP_ERR_CAPACITY and retry and attempt == 0 and total > out_cap:
                out_cap = total
                del out
                continue
            if code != capi.BP_OK:
                raise capi.BPError(code, "bp_query_batch")
            break
        self.last_total = total
        o = out_off.cpu().numpy().view(np.uint64)
        c = counts.cpu().numpy().view(np.uint32)
        if on_device:  # (device answers, offsets, counts)
            return out[:total], o, c[:nq]
        flat = as_u32(out[:total]) if nq else np.zeros(0, np.uint32)
        return [flat[int(o[q]):int(o[q]) + int(c[q])] for q in range(nq)]

    def query_one(self, terms, stream=None) -> torch.Tensor:
        terms = np.ascontiguousarray(terms, np.uint32)
        dev = self.device
        cap = max(1, int(self.h_lists["n"][terms].min()) if terms.size else 1)
        out = torch.empty(cap, dtype=torch.int32, device=dev)
        cnt = torch.zeros(1, dtype=torch.int32, device=dev)
        sb = capi.bp_query_one_scratch_bytes(self.h_lists, terms)
        scratch = torch.empty(max(sb, 16), dtype=torch.uint8, device=dev)
        st = status_tensor(dev)
        check(capi.bp_query_one(self.data.data_ptr(), self.h_lists, terms, out.data_ptr(), cap,
                                cnt.data_ptr(), scratch.data_ptr(), sb, st.data_ptr(),
                                _stream(stream)), "bp_query_one")
        check_status(st, "bp_query_one")
        return out[: int(cnt.item())]


class Server:
    """The serving engine (bp_server_*) over a resident Index: PyTorch
    allocates its device memory, pinned host memory and streams."""

    def __init__(self, index: Index, slots: int = 4, max_batch_queries: int = 4096,
                 max_terms: int = 8, slot_bytes: int = 1 << 30, deliver_answers: bool = True):
        import ctypes as C
        self.index = index
        self.cfg = capi.bp_server_config(slots, max_batch_queries, max_terms,
                                         1 if deliver_answers else 0, slot_bytes)
        self.d_mem = torch.empty(capi.lib.bp_server_device_bytes(C.byref(self.cfg)),
                                 dtype=torch.uint8, device=index.device)
        self.h_mem = torch.empty(capi.lib.bp_server_host_bytes(C.byref(self.cfg)),
                                 dtype=torch.uint8).pin_memory()
        self.streams = [torch.cuda.Stream(device=index.device) for _ in range(slots)]
        sp = (C.c_void_p * slots)(*[s.cuda_stream for s in self.streams])
        err = C.c_int(0)
        self.h_lists = np.ascontiguousarray(index.h_lists)
        self.ptr = capi.lib.bp_server_create(
            index.data.data_ptr(), index.d_lists.data_ptr(), self.h_lists.ctypes.data,
            index.n_terms, C.byref(self.cfg), self.d_mem.data_ptr(), self.h_mem.data_ptr(), sp,
            C.byref(err))
        if not self.ptr:
            raise capi.BPError(err.value, "bp_server_create")
        self._res = (capi.bp_server_result * 65536)()

    def submit(self, tag: int, terms) -> None:
        t = np.ascontiguousarray(terms, np.uint32)
        check(capi.lib.bp_server_submit(self.ptr, tag, t.ctypes.data if t.size else None,
                                        t.size), "bp_server_submit")

    def replay(self, tags, terms, term_off, arrival_s) -> None:
        tags = np.ascontiguousarray(tags, np.uint64)
        terms = np.ascontiguousarray(terms, np.uint32)
        term_off = np.ascontiguousarray(term_off, np.uint64)
        arrival_s = np.ascontiguousarray(arrival_s, np.float64)
        check(capi.lib.bp_server_replay(self.ptr, tags.ctypes.data, terms.ctypes.data,
                                        term_off.ctypes.data, tags.size,
                                        arrival_s.ctypes.data), "bp_server_replay")

    def poll(self, with_answers: bool = True) -> list:
        """Finished queries as (tag, count, status, arrival_s, submit_s,
        done_s, answer) tuples; latency is done_s - arrival_s."""
        out = []
        while True:
            n = capi.lib.bp_server_poll(self.ptr, self._res, len(self._res))
            for i in range(n):
                r = self._res[i]
                ans = None
                if with_answers and r.answer:
                    ans = np.ctypeslib.as_array(r.answer, shape=(r.count,)).copy()
                elif with_answers and r.status == capi.BP_OK:
                    ans = np.zeros(0, np.uint32)
                out.append((int(r.tag), int(r.count), int(r.status), float(r.arrival_s),
                            float(r.submit_s), float(r.done_s), ans))
            if n < len(self._res):
                return out

    def batches(self) -> np.ndarray:
        """Records of the retired batches (oldest first) as a structured
        array: slot, queries, answer_values, first_arrival_s, admit_s,
        launched_s, done_s, retired_s."""
        buf = (capi.bp_server_batch * 65536)()
        parts = []
        while True:
            n = capi.lib.bp_server_batches(self.ptr, buf, len(buf))
            if n:
                parts.append(np.ctypeslib.as_array(buf)[:n].copy())
            if n < len(buf):
                break
        if not parts:
            return np.ctypeslib.as_array(buf)[:0].copy()
        return np.concatenate(parts)

    def drain(self, timeout_s: float = 120.0) -> None:
        check(capi.lib.bp_server_drain(self.ptr, timeout_s), "bp_server_drain")

    def stats(self) -> dict:
        import ctypes as C
        a = (C.c_uint64 * 6)()
        check(capi.lib.bp_server_stats(self.ptr, a), "bp_server_stats")
        keys = ("submitted", "completed", "batches", "rejected", "max_busy_slots", "waiting")
        return dict(zip(keys, [int(x) for x in a]))

    def close(self) -> None:
        if self.ptr:
            capi.lib.bp_server_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
