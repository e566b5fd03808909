"""CPU checks of the boundary: the C-ABI library loads and exports every
function declared in include/*.h, and its host-side logic (encoder, header
parsing, batch planning) agrees byte for byte with the oracle."""
import glob
import os
import re

import numpy as np
import pytest

import workloads as W
from conftest import ROOT

from paper_1401_6399_gb300.build import build

build()
from paper_1401_6399_gb300 import capi  # noqa: E402


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(bp_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for need in ("bp_encode", "bp_decode", "bp_decode_sum", "bp_decode_batch"):
        assert need in names


@pytest.mark.parametrize("name", declared_functions())
def test_library_exports_symbol(name):
    assert hasattr(capi.lib, name), f"{name} declared in include/ but not exported"


def _lists(rng):
    out = []
    for n in [0, 1, 3, 4, 5, 127, 128, 129, 2047, 2048, 2049, 4096 + 128 * 5 + 7, 70001]:
        for U in (n + 1, 8 * n + 16, 1 << 32):
            out.append(np.sort(rng.choice(U, n, replace=False)).astype(np.uint32))
    return out


@pytest.mark.parametrize("layout", [0, 1])
def test_encoder_matches_oracle_bytes(orc, layout):
    rng = np.random.default_rng(42)
    for x in _lists(rng):
        want = orc.pl_encode(x) if layout == 0 else orc.gl_encode(x)
        for nt in (1, 4):
            got = capi.bp_encode(x, layout, nthreads=nt).tobytes()
            assert got == want, (layout, x.size, nt)
        assert capi.bp_encode_bound(x.size, layout) >= len(want)
        assert capi.bp_stream_info(np.frombuffer(want, np.uint8)) == (x.size, layout)


@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("kind", [1, 2, 3])
def test_encoder_kinds_match_oracle_bytes(orc, layout, kind):
    """DM, D2 and D1 streams (Section 5) byte for byte as the oracle writes
    them, with the kind readable from the header."""
    rng = np.random.default_rng(43 + kind)
    for x in _lists(rng)[::2]:
        want = orc.pl_encode(x, kind) if layout == 0 else orc.gl_encode(x, kind)
        for nt in (1, 4):
            got = capi.bp_encode(x, layout, nthreads=nt, delta=kind).tobytes()
            assert got == want, (layout, kind, x.size, nt)
        enc = np.frombuffer(want, np.uint8)
        assert capi.bp_stream_info(enc) == (x.size, layout)
        assert capi.bp_stream_kind(enc) == kind


def test_encoder_any_order_fixed_widths(orc):
    """BP_ENCODE_ANY_ORDER: any uint32 sequence (here stepped walks modulo
    2^32 whose differences over 1..4 positions are below 2^b) encodes, with
    every GL block of width exactly b, and the oracle decodes it back in both
    layouts; without the flag the encoder rejects it."""
    for b in (0, 1, 2, 3, 9, 16, 31, 32):
        for kind in range(4):
            x = W.stepped_walk(4096 * 2 + 200, b, 77 + b)
            g = capi.bp_encode(x, capi.BP_LAYOUT_GPU, 1, kind | capi.BP_ENCODE_ANY_ORDER)
            assert np.array_equal(orc.gl_decode(g.tobytes()), x)
            info = orc.gl_info(g.tobytes())
            assert info["payload_words"] == 4 * b * info["nblocks"]
            p = capi.bp_encode(x, capi.BP_LAYOUT_PAPER, 1, kind | capi.BP_ENCODE_ANY_ORDER)
            assert np.array_equal(orc.pl_decode(p.tobytes()), x)
            assert capi.bp_stream_kind(g) == capi.bp_stream_kind(p) == kind
            if b > 0:
                with pytest.raises(capi.BPError) as e:
                    capi.bp_encode(x, capi.BP_LAYOUT_GPU, 1, kind)
                assert e.value.code == capi.BP_ERR_UNSORTED


def test_pfor_encoder_matches_oracle_bytes(orc):
    """S4-FastPFOR in the GP layout: the library's encoder writes the oracle's
    bytes for every kind (lists with outliers, so blocks have exceptions),
    and bp_stream_info / bp_stream_kind read the header."""
    rng = np.random.default_rng(62)
    for kind in range(4):
        for n in (0, 1, 300, 4096 * 3 + 5, 70_000):
            gaps = rng.geometric(0.25, n).astype(np.uint64)
            jumps = rng.random(n) < 0.02
            gaps[jumps] = rng.integers(1 << 8, 1 << 16, int(jumps.sum()))
            x = np.cumsum(gaps).astype(np.uint32)
            e = capi.bp_encode(x, capi.BP_LAYOUT_PFOR, 3, kind)
            assert e.tobytes() == orc.gp_encode(x, kind)
            assert capi.bp_stream_info(e) == (n, capi.BP_LAYOUT_PFOR)
            assert capi.bp_stream_kind(e) == kind
            assert e.size <= capi.bp_encode_bound(n, capi.BP_LAYOUT_PFOR)


def test_pfor_stream_info_rejects_bad_headers_and_bound_holds():
    """The host header parser rejects GP headers whose geometry, length or
    kind do not add up; the encoder never exceeds bp_encode_bound, also for
    blocks of width 32 and blocks full of exceptions."""
    rng = np.random.default_rng(63)
    for x in (rng.integers(0, 1 << 32, 9000, dtype=np.uint64).astype(np.uint32),
              W.stepped_walk(4096 * 3 + 1, 32, 64), W.stepped_walk(777, 0, 65)):
        for kind in range(4):
            e = capi.bp_encode(x, capi.BP_LAYOUT_PFOR, 2, kind | capi.BP_ENCODE_ANY_ORDER)
            assert e.size <= capi.bp_encode_bound(x.size, capi.BP_LAYOUT_PFOR)
    x = np.arange(5, 5 + 3 * 20000, 3, dtype=np.uint32)
    e = capi.bp_encode(x, capi.BP_LAYOUT_PFOR, 1)
    assert capi.bp_stream_info(e) == (x.size, capi.BP_LAYOUT_PFOR)
    for word, value in ((0, 0x12345678), (3, 7), (4, 99), (8, 12), (12, 4)):
        bad = e.copy()
        bad[4 * word:4 * word + 4] = np.array([value], np.uint32).view(np.uint8)
        with pytest.raises(capi.BPError) as err:
            capi.bp_stream_info(bad)
        assert err.value.code == capi.BP_ERR_CORRUPT
    with pytest.raises(capi.BPError):
        capi.bp_stream_info(e[:-4])  # shorter than the header's total


def test_hybrid_index_bitmaps():
    """hyb+m2 index: a list whose average gap is at most B becomes a bitmap
    (bit v set iff v is in the list; header {magic, 2, n, words}), the others
    GL streams byte for byte as bp_encode writes them."""
    rng = np.random.default_rng(5)
    U = 1 << 16
    lens = [0, 3, 100, U // 8 - 1, U // 8, U // 2, 4000]
    xs = [np.sort(rng.choice(U, n, replace=False)).astype(np.uint32) for n in lens]
    offs = np.zeros(len(xs) + 1, np.uint64)
    np.cumsum([x.size for x in xs], out=offs[1:])
    data, lists = capi.bp_index_encode_hybrid(np.concatenate(xs), offs, U, 8, nthreads=3)
    for x, L in zip(xs, lists):
        s = data[int(L["enc_offset"]):int(L["enc_offset"]) + int(L["enc_bytes"])]
        if x.size * 8 >= U:
            assert L["layout"] == capi.BP_LAYOUT_BITMAP
            h = s[:16].view(np.uint32)
            assert h[0] == 0x314D5042 and h[1] == 2 and h[2] == x.size
            words = s[16:16 + 4 * int(h[3])].view(np.uint32)
            bits = np.unpackbits(words.view(np.uint8), bitorder="little")
            assert int(h[3]) * 32 >= U and int(h[3]) % 4 == 0
            assert np.array_equal(np.flatnonzero(bits), x)
        else:
            assert L["layout"] == capi.BP_LAYOUT_GPU
            assert s.tobytes() == capi.bp_encode(x, 1).tobytes()
    with pytest.raises(capi.BPError):  # a value beyond the universe
        bad = np.array([1, U + 5], np.uint32)
        capi.bp_index_encode_hybrid(bad, np.array([0, 2], np.uint64), 16, 8)


def test_encoder_rejects_unsorted_and_small_buffers():
    with pytest.raises(capi.BPError) as e:
        capi.bp_encode(np.array([5, 4], np.uint32), 0)
    assert e.value.code == capi.BP_ERR_UNSORTED
    with pytest.raises(capi.BPError):
        capi.bp_encode(np.array([5, 5], np.uint32), 1)
    with pytest.raises(capi.BPError):
        capi.bp_encode(np.array([1, 2], np.uint32), 7)


def test_stream_info_rejects_garbage():
    with pytest.raises(capi.BPError):
        capi.bp_stream_info(np.full(64, 0xAB, np.uint8))


def test_plan_lists_units():
    lists = np.zeros(4, capi.BP_LIST)
    lists["n"] = [0, 128 * 32, 128 * 32 + 1, 5000]
    lists["layout"] = 1
    total = capi.bp_plan_lists(lists)
    per = [0, 1, 2, 2]  # superblocks of 32 blocks
    assert lists["unit_base"].tolist() == [0, 0, 1, 3] and total == sum(per)
    lists["layout"] = 0
    total = capi.bp_plan_lists(lists)
    per = [0 + 1, 32 + 1, 32 + 1, 39 + 1]  # blocks + a tail unit
    assert total == sum(per) and lists["unit_base"].tolist() == [0, 1, 34, 67]


def test_scratch_sizes():
    assert capi.bp_decode_scratch_bytes(10**6, capi.BP_LAYOUT_GPU) == 0
    a = capi.bp_decode_scratch_bytes(10**6, capi.BP_LAYOUT_PAPER)
    b = capi.bp_decode_scratch_bytes(2 * 10**6, capi.BP_LAYOUT_PAPER)
    assert 8 * (10**6 // 128) < a < b


def test_tuning_round_trip_and_wait_limit_range():
    old = capi.bp_get_tuning()
    try:
        capi.bp_set_tuning(lookback_spin_limit=1 << 10, withhold_tile=3)
        t = capi.bp_get_tuning()
        assert t["lookback_spin_limit"] == 1 << 10 and t["withhold_tile"] == 3
        with pytest.raises(capi.BPError) as e:  # above the default limit
            capi.bp_set_tuning(lookback_spin_limit=(1 << 22) + 1)
        assert e.value.code == capi.BP_ERR_ARG
    finally:
        capi.bp_set_tuning(**old)
    assert capi.bp_get_tuning() == old
