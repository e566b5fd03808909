"""CPU checks of the boundary: the C-ABI library loads and exports every
function declared in include/*.h, and its host-side logic (encoder, header
parsing, batch planning) agrees byte for byte with the oracle."""
import glob
import os
import re

import numpy as np
import pytest

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
