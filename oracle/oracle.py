"""ctypes wrapper around liboracle.so (the scalar C oracle).

TEST INFRASTRUCTURE ONLY.  Arrays are numpy uint32/uint8; every call copies
nothing beyond what the C functions need.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "bp_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

ORC_OK, ORC_EARG, ORC_ECORRUPT, ORC_ECAPACITY = 0, 1, 3, 4


def build_oracle(force: bool = False) -> str:
    """Compile bp_oracle.c into liboracle.so with gcc (no GPU needed)."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC[:-1] + "h")):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-std=c11", "-O2", "-Wall", "-Wextra",
                           "-fPIC", "-shared", "-o", tmp, SRC])
    os.replace(tmp, LIB)
    return LIB


_u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
_sz = C.c_size_t


def _u32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint32)


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: oracle error {code}")
        self.code = code


class Oracle:
    """Thin typed access to the oracle's C functions."""

    def __init__(self, path: str | None = None):
        self.lib = C.CDLL(path or build_oracle())
        L = self.lib
        L.orc_bits.argtypes = [C.c_uint32]
        L.orc_bits.restype = C.c_uint
        L.orc_max_bits.argtypes = [_u32p, _sz]
        L.orc_max_bits.restype = C.c_uint
        L.orc_pack_scalar.argtypes = [_u32p, _sz, C.c_uint, _u8p]
        L.orc_unpack_scalar.argtypes = [_u8p, _sz, C.c_uint, _u32p]
        L.orc_s4_pack128.argtypes = [_u32p, C.c_uint, _u32p]
        L.orc_s4_unpack128.argtypes = [_u32p, C.c_uint, C.c_int, _u32p, _u32p]
        L.orc_d4_deltas.argtypes = [_u32p, _sz, _u32p]
        L.orc_d4_prefix.argtypes = [_u32p, _sz, _u32p]
        L.orc_deltas.argtypes = [C.c_int, _u32p, _sz, C.c_uint32, _u32p]
        L.orc_prefix.argtypes = [C.c_int, _u32p, _sz, C.c_uint32, _u32p]
        L.orc_varint_encode.argtypes = [_u32p, _sz, _u8p]
        L.orc_varint_encode.restype = _sz
        L.orc_varint_decode.argtypes = [_u8p, _sz, _sz, _u32p, C.POINTER(_sz)]
        L.orc_varint_decode.restype = C.c_int
        L.orc_pfor_choose.argtypes = [_u32p, C.POINTER(C.c_uint), C.POINTER(C.c_uint),
                                      C.POINTER(C.c_uint)]
        for f in ("orc_pl_bound", "orc_gl_bound", "orc_gp_bound"):
            getattr(L, f).argtypes = [_sz]
            getattr(L, f).restype = _sz
        for f in ("orc_pl_encode", "orc_gl_encode"):
            getattr(L, f).argtypes = [_u32p, _sz, _u8p, _sz, C.POINTER(_sz)]
            getattr(L, f).restype = C.c_int
        for f in ("orc_pl_encode_kind", "orc_gl_encode_kind", "orc_gp_encode_kind"):
            getattr(L, f).argtypes = [_u32p, _sz, C.c_int, _u8p, _sz, C.POINTER(_sz)]
            getattr(L, f).restype = C.c_int
        for f in ("orc_pl_decode", "orc_gl_decode", "orc_gp_decode"):
            getattr(L, f).argtypes = [_u8p, _sz, _u32p, _sz, C.POINTER(_sz)]
            getattr(L, f).restype = C.c_int
        L.orc_stream_count.argtypes = [_u8p, _sz, C.POINTER(_sz)]
        L.orc_stream_count.restype = C.c_int
        L.orc_gl_info.argtypes = [_u8p, _sz, _u32p]
        L.orc_gl_info.restype = C.c_int
        for f in ("orc_intersect_merge", "orc_intersect_gallop",
                  "orc_intersect_hybrid"):
            getattr(L, f).argtypes = [_u32p, _sz, _u32p, _sz, _u32p]
            getattr(L, f).restype = _sz
        for f in ("orc_intersect_v1", "orc_intersect_v3",
                  "orc_intersect_simd_gallop"):
            getattr(L, f).argtypes = [_u32p, _sz, _u32p, _sz, C.c_uint, _u32p]
            getattr(L, f).restype = _sz
        L.orc_svs.argtypes = [C.POINTER(C.c_void_p), C.POINTER(_sz), _sz, _u32p]
        L.orc_svs.restype = _sz

    # -- widths and packing ---------------------------------------------------
    def bits(self, v: int) -> int:
        return int(self.lib.orc_bits(v))

    def max_bits(self, v) -> int:
        v = _u32(v)
        return int(self.lib.orc_max_bits(v, v.size))

    def pack_scalar(self, v, b: int) -> bytes:
        v = _u32(v)
        out = np.zeros(max(1, (v.size * b + 7) // 8), np.uint8)
        self.lib.orc_pack_scalar(v, v.size, b, out)
        return out[: (v.size * b + 7) // 8].tobytes()

    def unpack_scalar(self, data: bytes, n: int, b: int) -> np.ndarray:
        buf = np.frombuffer(bytes(data) + b"\0", np.uint8).copy()
        out = np.zeros(max(1, n), np.uint32)
        self.lib.orc_unpack_scalar(buf, n, b, out)
        return out[:n]

    def s4_pack128(self, v, b: int) -> np.ndarray:
        v = _u32(v)
        assert v.size == 128
        out = np.zeros(max(1, 4 * b), np.uint32)
        self.lib.orc_s4_pack128(v, b, out)
        return out[: 4 * b]

    # prefix functions of Algorithm 1 (ORC_P_*)
    P_NONE, P_D4, P_DM, P_D2, P_D1 = 0, 1, 2, 3, 4

    def s4_unpack128(self, words, b: int, d4: bool = True, seed=(0, 0, 0, 0),
                     kind: int | None = None):
        """Algorithm 1; kind (P_*) overrides d4 (True: P_D4, False: P_NONE)."""
        w = np.zeros(max(1, 4 * b + 4), np.uint32)
        w[: 4 * b] = _u32(words)[: 4 * b]
        v = _u32(seed).copy()
        out = np.zeros(128, np.uint32)
        k = kind if kind is not None else (1 if d4 else 0)
        self.lib.orc_s4_unpack128(w, b, k, v, out)
        return out, v

    # -- differential coding ---------------------------------------------------
    def d4_deltas(self, x) -> np.ndarray:
        x = _u32(x)
        d = np.zeros(max(1, x.size), np.uint32)
        self.lib.orc_d4_deltas(x, x.size, d)
        return d[: x.size]

    def d4_prefix(self, d) -> np.ndarray:
        d = _u32(d)
        x = np.zeros(max(1, d.size), np.uint32)
        self.lib.orc_d4_prefix(d, d.size, x)
        return x[: d.size]

    # kinds of differential coding (Section 5), as stored in stream headers
    D4, DM, D2, D1 = 0, 1, 2, 3

    def deltas(self, kind: int, x, seed: int = 0) -> np.ndarray:
        x = _u32(x)
        d = np.zeros(max(1, x.size), np.uint32)
        self.lib.orc_deltas(kind, x, x.size, seed, d)
        return d[: x.size]

    def prefix(self, kind: int, d, seed: int = 0) -> np.ndarray:
        d = _u32(d)
        x = np.zeros(max(1, d.size), np.uint32)
        self.lib.orc_prefix(kind, d, d.size, seed, x)
        return x[: d.size]

    # -- varint ---------------------------------------------------------------
    def varint_encode(self, v) -> bytes:
        v = _u32(v)
        out = np.zeros(max(1, 5 * v.size), np.uint8)
        k = self.lib.orc_varint_encode(v, v.size, out)
        return out[:k].tobytes()

    def varint_decode(self, data: bytes, n: int):
        buf = np.frombuffer(bytes(data) + b"\0", np.uint8).copy()
        out = np.zeros(max(1, n), np.uint32)
        used = _sz(0)
        rc = self.lib.orc_varint_decode(buf, len(data), n, out, C.byref(used))
        if rc:
            raise OracleError(rc, "varint_decode")
        return out[:n], used.value

    # -- containers -------------------------------------------------------------
    def _encode(self, fn, bound, x) -> bytes:
        x = _u32(x)
        cap = int(bound(x.size))
        out = np.zeros(cap, np.uint8)
        nbytes = _sz(0)
        rc = fn(x, x.size, out, cap, C.byref(nbytes))
        if rc:
            raise OracleError(rc, fn.__name__)
        return out[: nbytes.value].tobytes()

    def _decode(self, fn, data) -> np.ndarray:
        """data: bytes, or a C-contiguous uint8 array (read in place)."""
        if (isinstance(data, np.ndarray) and data.dtype == np.uint8
                and data.flags.c_contiguous and data.size):
            buf, nbytes = data, data.size
        else:
            buf = np.frombuffer(bytes(data), np.uint8)
            nbytes = buf.size
            buf = buf.copy() if buf.size else np.zeros(1, np.uint8)
        n = _sz(0)
        rc = self.lib.orc_stream_count(buf, nbytes, C.byref(n))
        if rc:
            raise OracleError(rc, "stream_count")
        out = np.empty(max(1, n.value), np.uint32)
        got = _sz(0)
        rc = fn(buf, nbytes, out, out.size, C.byref(got))
        if rc:
            raise OracleError(rc, fn.__name__)
        return out[: got.value]

    def _encode_kind(self, fn, bound, x, kind: int) -> bytes:
        x = _u32(x)
        cap = int(bound(x.size))
        out = np.zeros(cap, np.uint8)
        nbytes = _sz(0)
        rc = fn(x, x.size, kind, out, cap, C.byref(nbytes))
        if rc:
            raise OracleError(rc, fn.__name__)
        return out[: nbytes.value].tobytes()

    def pl_encode(self, x, kind: int = 0) -> bytes:
        if kind:
            return self._encode_kind(self.lib.orc_pl_encode_kind, self.lib.orc_pl_bound, x, kind)
        return self._encode(self.lib.orc_pl_encode, self.lib.orc_pl_bound, x)

    def pl_decode(self, data: bytes) -> np.ndarray:
        return self._decode(self.lib.orc_pl_decode, data)

    def gl_encode(self, x, kind: int = 0) -> bytes:
        if kind:
            return self._encode_kind(self.lib.orc_gl_encode_kind, self.lib.orc_gl_bound, x, kind)
        return self._encode(self.lib.orc_gl_encode, self.lib.orc_gl_bound, x)

    def gl_decode(self, data: bytes) -> np.ndarray:
        return self._decode(self.lib.orc_gl_decode, data)

    def gp_encode(self, x, kind: int = 0) -> bytes:
        """S4-FastPFOR in the GPU layout (GP)."""
        return self._encode_kind(self.lib.orc_gp_encode_kind, self.lib.orc_gp_bound, x, kind)

    def gp_decode(self, data: bytes) -> np.ndarray:
        return self._decode(self.lib.orc_gp_decode, data)

    def pfor_choose(self, d) -> tuple:
        """(b, b', c) of one block of 128 deltas (Section 4.4)."""
        d = _u32(d)
        assert d.size == 128
        b, bp, c = C.c_uint(0), C.c_uint(0), C.c_uint(0)
        self.lib.orc_pfor_choose(d, C.byref(b), C.byref(bp), C.byref(c))
        return int(b.value), int(bp.value), int(c.value)

    def gl_info(self, data: bytes) -> dict:
        buf = np.frombuffer(bytes(data), np.uint8).copy()
        info = np.zeros(8, np.uint32)
        rc = self.lib.orc_gl_info(buf, len(data), info)
        if rc:
            raise OracleError(rc, "gl_info")
        keys = ("n", "nblocks", "nsuper", "payload_words", "off_first",
                "off_sbo", "off_bw", "off_payload")
        return {k: int(v) for k, v in zip(keys, info)}

    # -- intersections ----------------------------------------------------------
    def _pair(self, fn, a, b, *extra) -> np.ndarray:
        a, b = _u32(a), _u32(b)
        out = np.zeros(max(1, min(a.size, b.size)), np.uint32)
        pa = a if a.size else np.zeros(1, np.uint32)
        pb = b if b.size else np.zeros(1, np.uint32)
        k = fn(pa, a.size, pb, b.size, *extra, out)
        return out[:k]

    def intersect(self, a, b):
        return self._pair(self.lib.orc_intersect_merge, a, b)

    def intersect_gallop(self, a, b):
        return self._pair(self.lib.orc_intersect_gallop, a, b)

    def intersect_hybrid(self, a, b):
        return self._pair(self.lib.orc_intersect_hybrid, a, b)

    def intersect_v1(self, r, f, T=8):
        return self._pair(self.lib.orc_intersect_v1, r, f, T)

    def intersect_v3(self, r, f, T=32):
        return self._pair(self.lib.orc_intersect_v3, r, f, T)

    def intersect_simd_gallop(self, r, f, T=32):
        return self._pair(self.lib.orc_intersect_simd_gallop, r, f, T)

    def svs(self, lists) -> np.ndarray:
        arrs = [_u32(x) if len(x) else np.zeros(1, np.uint32) for x in lists]
        lens = (_sz * len(lists))(*[len(x) for x in lists])
        ptrs = (C.c_void_p * len(lists))(*[a.ctypes.data for a in arrs])
        out = np.zeros(max(1, min([len(x) for x in lists] or [0])), np.uint32)
        k = self.lib.orc_svs(ptrs, lens, len(lists), out)
        return out[:k]

    def svs_gallop(self, lists) -> np.ndarray:
        """Set-vs-Set (Section 6) with every step done by galloping: the
        lists in increasing order of length (ties in the given order), the
        candidates start as the shortest list and are intersected with each
        longer list in turn by orc_intersect_gallop; stops once no candidate
        is left.  Same result as svs (the intersection is unique); the cost
        is O(m log n) per step instead of O(m + n), which makes sets with
        lists of 2^24 values affordable."""
        if not len(lists):
            return np.zeros(0, np.uint32)
        order = sorted(range(len(lists)), key=lambda i: len(lists[i]))
        cur = _u32(lists[order[0]])
        for i in order[1:]:
            if cur.size == 0:
                break
            cur = self.intersect_gallop(cur, lists[i])
        return cur.copy() if cur.base is not None else cur
