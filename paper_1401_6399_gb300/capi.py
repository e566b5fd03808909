"""ctypes binding of libbp128.so (include/bp128.h): same names, argument
marshalling only.  Device pointers are plain ints (e.g. tensor.data_ptr()),
streams are cudaStream_t handles as ints (torch.cuda.Stream.cuda_stream).

The library must have been built (paper_1401_6399_gb300.build.build());
importing this module without it raises at once -- there is no fallback."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import LIB

BP_OK, BP_ERR_ARG, BP_ERR_UNSORTED, BP_ERR_CORRUPT = 0, 1, 2, 3
BP_ERR_CAPACITY, BP_ERR_CUDA, BP_ERR_TIMEOUT, BP_ERR_SCRATCH = 4, 5, 6, 7
BP_LAYOUT_PAPER, BP_LAYOUT_GPU = 0, 1
BP_MODE_AUTO, BP_MODE_UNFUSED, BP_MODE_FUSED = 0, 1, 2


class bp_tuning(C.Structure):
    _fields_ = [("dense_blocks", C.c_uint32), ("query_chunk_blocks", C.c_uint32),
                ("query_warps", C.c_uint32), ("lookback_spin_limit", C.c_uint32),
                ("withhold_tile", C.c_uint32), ("merge_span", C.c_uint32),
                ("reserved", C.c_uint32 * 2)]

class bp_server_config(C.Structure):
    _fields_ = [("slots", C.c_uint32), ("max_batch_queries", C.c_uint32),
                ("max_terms", C.c_uint32), ("deliver_answers", C.c_uint32),
                ("slot_bytes", C.c_uint64), ("reserved", C.c_uint64 * 4)]


class bp_server_result(C.Structure):
    _fields_ = [("tag", C.c_uint64), ("count", C.c_uint32), ("status", C.c_int32),
                ("arrival_s", C.c_double), ("submit_s", C.c_double), ("done_s", C.c_double),
                ("answer", C.POINTER(C.c_uint32))]


class bp_server_batch(C.Structure):
    _fields_ = [("slot", C.c_uint32), ("queries", C.c_uint32), ("answer_values", C.c_uint64),
                ("first_arrival_s", C.c_double), ("admit_s", C.c_double),
                ("launched_s", C.c_double), ("done_s", C.c_double), ("retired_s", C.c_double)]


# struct bp_list (48 bytes)
BP_LIST = np.dtype([("enc_offset", "<u8"), ("enc_bytes", "<u8"), ("out_offset", "<u8"),
                    ("unit_base", "<u8"), ("n", "<u4"), ("layout", "<u4"),
                    ("reserved", "<u8")])
assert BP_LIST.itemsize == 48

if not os.path.exists(LIB):
    raise ImportError(f"{LIB} is missing: build it with paper_1401_6399_gb300.build.build()")

lib = C.CDLL(LIB)

_vp, _sz, _u64, _u32, _int = C.c_void_p, C.c_size_t, C.c_uint64, C.c_uint32, C.c_int


def _decl(name, restype, *argtypes):
    f = getattr(lib, name)
    f.restype = restype
    f.argtypes = list(argtypes)
    return f


_decl("bp_status_string", C.c_char_p, _int)
_decl("bp_encode_bound", _sz, _sz, _int)
_decl("bp_encode", _int, _vp, _sz, _int, _vp, _sz, C.POINTER(_sz), _int)
_decl("bp_encode_kind", _int, _vp, _sz, _int, _int, _vp, _sz, C.POINTER(_sz), _int)
_decl("bp_stream_info", _int, _vp, _sz, C.POINTER(_u32), C.POINTER(_int))
_decl("bp_stream_kind", _int, _vp, _sz, C.POINTER(_int))
_decl("bp_plan_lists", _u64, _vp, _u32)
_decl("bp_index_bound", _sz, _vp, _u32)
_decl("bp_index_encode", _int, _vp, _vp, _u32, _vp, _sz, _vp, C.POINTER(_sz), _int)
_decl("bp_index_hybrid_bound", _sz, _vp, _u32, _u32, _u32)
_decl("bp_index_encode_hybrid", _int, _vp, _vp, _u32, _u32, _u32, _vp, _sz, _vp, C.POINTER(_sz),
      _int)
_decl("bp_decode_scratch_bytes", _sz, _sz, _int)
_decl("bp_decode", _int, _vp, _sz, _int, _sz, _vp, _sz, _vp, _sz, _vp, _vp)
_decl("bp_decode_sum", _int, _vp, _sz, _int, _sz, _vp, _vp, _sz, _vp, _vp)
_decl("bp_decode_batch_scratch_bytes", _sz, _vp, _u32)
_decl("bp_decode_batch", _int, _vp, _vp, _u32, _u64, _int, _vp, _u64, _vp, _vp, _sz, _vp, _vp)
_decl("bp_decode_ablation", _int, _vp, _vp, _u32, _vp, _u64, _vp, _int, _vp)
_decl("bp_decode_batch_host", _int, _vp, _sz, _vp, _u32, _u64, _int, _vp, _vp, _vp, _u64, _vp,
      _vp, _sz, _vp, _vp, _vp)
_decl("bp_query_batch_scratch_bytes", _sz, _vp, _u32, _vp, _vp, _u32, _u64)
_decl("bp_query_batch", _int, _vp, _vp, _u32, _vp, _vp, _u64, _u32, _vp, _u64, _vp, _vp, _vp,
      _sz, _vp, _vp)
_decl("bp_query_one_scratch_bytes", _sz, _vp, _u32, _vp, _u32)
_decl("bp_query_one", _int, _vp, _vp, _u32, _vp, _u32, _vp, _sz, _vp, _vp, _sz, _vp, _vp)
_decl("bp_server_device_bytes", _sz, C.POINTER(bp_server_config))
_decl("bp_server_host_bytes", _sz, C.POINTER(bp_server_config))
_decl("bp_server_create", _vp, _vp, _vp, _vp, _u32, C.POINTER(bp_server_config), _vp, _vp,
      C.POINTER(_vp), C.POINTER(_int))
_decl("bp_server_submit", _int, _vp, _u64, _vp, _u32)
_decl("bp_server_replay", _int, _vp, _vp, _vp, _vp, _u32, _vp)
_decl("bp_server_poll", _u32, _vp, C.POINTER(bp_server_result), _u32)
_decl("bp_server_drain", _int, _vp, C.c_double)
_decl("bp_server_stats", _int, _vp, C.POINTER(C.c_uint64))
_decl("bp_server_batches", _u32, _vp, C.POINTER(bp_server_batch), _u32)
_decl("bp_server_destroy", None, _vp)
_decl("bp_get_tuning", _int, C.POINTER(bp_tuning))
_decl("bp_set_tuning", _int, C.POINTER(bp_tuning))
_decl("bp_intersect_scratch_bytes", _sz, _sz, _sz, _int, _int)
_decl("bp_intersect_pair", _int, _vp, _sz, _sz, _vp, _sz, _sz, _int, _int, _vp, _sz, _vp, _vp,
      _sz, _vp, _vp)


class BPError(RuntimeError):
    def __init__(self, code: int, what: str):
        msg = lib.bp_status_string(code).decode()
        super().__init__(f"{what}: {msg} ({code})")
        self.code = code


def check(code: int, what: str) -> None:
    if code != BP_OK:
        raise BPError(code, what)


def bp_status_string(code: int) -> str:
    return lib.bp_status_string(code).decode()


# ---- host -----------------------------------------------------------------------

def bp_encode_bound(n: int, layout: int) -> int:
    return int(lib.bp_encode_bound(n, layout))


# kinds of differential coding (bp_delta)
BP_DELTA_D4, BP_DELTA_DM, BP_DELTA_D2, BP_DELTA_D1 = 0, 1, 2, 3


BP_ENCODE_ANY_ORDER = 0x100


def bp_encode(x, layout: int, nthreads: int = 1, delta: int = BP_DELTA_D4) -> np.ndarray:
    """Encode a sorted distinct uint32 array (any uint32 array if delta has
    BP_ENCODE_ANY_ORDER set); returns the stream as uint8."""
    x = np.ascontiguousarray(x, np.uint32)
    cap = bp_encode_bound(x.size, layout)
    out = np.empty(max(cap, 16), np.uint8)
    nbytes = _sz(0)
    if delta == BP_DELTA_D4:
        rc = lib.bp_encode(x.ctypes.data if x.size else None, x.size, layout, out.ctypes.data,
                           cap, C.byref(nbytes), nthreads)
    else:
        rc = lib.bp_encode_kind(x.ctypes.data if x.size else None, x.size, layout, delta,
                                out.ctypes.data, cap, C.byref(nbytes), nthreads)
    check(rc, "bp_encode")
    return out[: nbytes.value]


def bp_stream_kind(enc) -> int:
    enc = np.ascontiguousarray(enc, np.uint8)
    k = _int(0)
    check(lib.bp_stream_kind(enc.ctypes.data, enc.size, C.byref(k)), "bp_stream_kind")
    return int(k.value)


def bp_stream_info(enc) -> tuple[int, int]:
    enc = np.ascontiguousarray(np.frombuffer(bytes(enc), np.uint8) if isinstance(enc, (bytes, bytearray)) else enc, np.uint8)
    n, layout = _u32(0), _int(0)
    check(lib.bp_stream_info(enc.ctypes.data, enc.size, C.byref(n), C.byref(layout)),
          "bp_stream_info")
    return int(n.value), int(layout.value)


def bp_plan_lists(lists: np.ndarray) -> int:
    assert lists.dtype == BP_LIST and lists.flags.c_contiguous
    return int(lib.bp_plan_lists(lists.ctypes.data, lists.size))


def bp_index_encode(values: np.ndarray, offs: np.ndarray, nthreads: int = 8):
    """Encode many lists into one GL buffer; returns (uint8 buffer, BP_LIST array)."""
    values = np.ascontiguousarray(values, np.uint32)
    offs = np.ascontiguousarray(offs, np.uint64)
    count = offs.size - 1
    cap = int(lib.bp_index_bound(offs.ctypes.data, count))
    out = np.empty(max(cap, 16), np.uint8)
    lists = np.zeros(count, BP_LIST)
    used = _sz(0)
    check(lib.bp_index_encode(values.ctypes.data if values.size else None, offs.ctypes.data,
                              count, out.ctypes.data, cap, lists.ctypes.data, C.byref(used),
                              nthreads), "bp_index_encode")
    return out[: max(used.value, 16)], lists


BP_LAYOUT_BITMAP = 2
BP_LAYOUT_PFOR = 3


def bp_index_encode_hybrid(values: np.ndarray, offs: np.ndarray, universe: int, B: int,
                           nthreads: int = 8):
    """Hybrid (hyb+m2) index: lists with average gap <= B become bitmaps of
    `universe` bits, the others GL streams; returns (uint8 buffer, BP_LIST array)."""
    values = np.ascontiguousarray(values, np.uint32)
    offs = np.ascontiguousarray(offs, np.uint64)
    count = offs.size - 1
    cap = int(lib.bp_index_hybrid_bound(offs.ctypes.data, count, universe, B))
    out = np.empty(max(cap, 16), np.uint8)
    lists = np.zeros(count, BP_LIST)
    used = _sz(0)
    check(lib.bp_index_encode_hybrid(values.ctypes.data if values.size else None,
                                     offs.ctypes.data, count, universe, B, out.ctypes.data, cap,
                                     lists.ctypes.data, C.byref(used), nthreads),
          "bp_index_encode_hybrid")
    return out[: max(used.value, 16)], lists


# ---- device (raw pointers) ---------------------------------------------------------

def bp_decode_scratch_bytes(n: int, layout: int) -> int:
    return int(lib.bp_decode_scratch_bytes(n, layout))


def bp_decode(d_enc, enc_bytes, layout, n, d_out, out_cap, d_scratch, scratch_bytes,
              d_status, stream) -> int:
    return lib.bp_decode(d_enc, enc_bytes, layout, n, d_out, out_cap, d_scratch,
                         scratch_bytes, d_status, stream)


def bp_decode_sum(d_enc, enc_bytes, layout, n, d_sum, d_scratch, scratch_bytes, d_status,
                  stream) -> int:
    return lib.bp_decode_sum(d_enc, enc_bytes, layout, n, d_sum, d_scratch, scratch_bytes,
                             d_status, stream)


def bp_decode_batch_scratch_bytes(lists: np.ndarray) -> int:
    assert lists.dtype == BP_LIST and lists.flags.c_contiguous
    return int(lib.bp_decode_batch_scratch_bytes(lists.ctypes.data, lists.size))


def bp_decode_batch(d_data, d_lists, count, total_units, layout, d_out, out_cap, d_sums,
                    d_scratch, scratch_bytes, d_status, stream) -> int:
    return lib.bp_decode_batch(d_data, d_lists, count, total_units, layout, d_out, out_cap,
                               d_sums, d_scratch, scratch_bytes, d_status, stream)


def bp_decode_ablation(d_data, d_lists, count, d_out, out_cap, d_status, two_pass, stream) -> int:
    return lib.bp_decode_ablation(d_data, d_lists, count, d_out, out_cap, d_status, two_pass,
                                  stream)


def bp_get_tuning() -> dict:
    t = bp_tuning()
    check(lib.bp_get_tuning(C.byref(t)), "bp_get_tuning")
    return {"dense_blocks": t.dense_blocks, "query_chunk_blocks": t.query_chunk_blocks,
            "query_warps": t.query_warps, "lookback_spin_limit": t.lookback_spin_limit,
            "withhold_tile": t.withhold_tile, "merge_span": t.merge_span}


def bp_set_tuning(**kw) -> None:
    cur = bp_get_tuning()
    cur.update(kw)
    t = bp_tuning(cur["dense_blocks"], cur["query_chunk_blocks"], cur["query_warps"],
                  cur["lookback_spin_limit"], cur["withhold_tile"], cur["merge_span"])
    check(lib.bp_set_tuning(C.byref(t)), "bp_set_tuning")


def bp_intersect_scratch_bytes(n_a: int, n_b: int, layout: int, mode: int) -> int:
    return int(lib.bp_intersect_scratch_bytes(n_a, n_b, layout, mode))


def bp_intersect_pair(d_a, a_bytes, n_a, d_b, b_bytes, n_b, layout, mode, d_out, out_cap,
                      d_count, d_scratch, scratch_bytes, d_status, stream) -> int:
    return lib.bp_intersect_pair(d_a, a_bytes, n_a, d_b, b_bytes, n_b, layout, mode, d_out,
                                 out_cap, d_count, d_scratch, scratch_bytes, d_status, stream)


def bp_decode_batch_host(h_data, data_bytes, h_lists, count, total_units, layout, d_data, d_lists,
                         d_out, out_cap, h_out, d_scratch, scratch_bytes, d_status, h_status,
                         stream) -> int:
    return lib.bp_decode_batch_host(h_data, data_bytes, h_lists, count, total_units, layout,
                                    d_data, d_lists, d_out, out_cap, h_out, d_scratch,
                                    scratch_bytes, d_status, h_status, stream)


def bp_query_batch_scratch_bytes(h_lists: np.ndarray, h_terms: np.ndarray,
                                 h_term_off: np.ndarray, out_cap: int) -> int:
    assert h_lists.dtype == BP_LIST
    h_terms = np.ascontiguousarray(h_terms, np.uint32)
    h_term_off = np.ascontiguousarray(h_term_off, np.uint64)
    return int(lib.bp_query_batch_scratch_bytes(
        h_lists.ctypes.data, h_lists.size, h_terms.ctypes.data if h_terms.size else None,
        h_term_off.ctypes.data, h_term_off.size - 1, out_cap))


def bp_query_batch(d_data, d_lists, n_terms, d_terms, d_term_off, total_terms, n_queries, d_out,
                   out_cap, d_out_off, d_counts, d_scratch, scratch_bytes, d_status,
                   stream) -> int:
    return lib.bp_query_batch(d_data, d_lists, n_terms, d_terms, d_term_off, total_terms,
                              n_queries, d_out, out_cap, d_out_off, d_counts, d_scratch,
                              scratch_bytes, d_status, stream)


def bp_query_one_scratch_bytes(h_lists: np.ndarray, terms) -> int:
    t = np.ascontiguousarray(terms, np.uint32)
    return int(lib.bp_query_one_scratch_bytes(h_lists.ctypes.data, h_lists.size,
                                              t.ctypes.data if t.size else None, t.size))


def bp_query_one(d_data, h_lists: np.ndarray, terms, d_out, out_cap, d_count, d_scratch,
                 scratch_bytes, d_status, stream) -> int:
    t = np.ascontiguousarray(terms, np.uint32)
    return lib.bp_query_one(d_data, h_lists.ctypes.data, h_lists.size,
                            t.ctypes.data if t.size else None, t.size, d_out, out_cap, d_count,
                            d_scratch, scratch_bytes, d_status, stream)
