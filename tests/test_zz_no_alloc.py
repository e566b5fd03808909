"""bp_intersect_pair_noalloc: the fused intersection for callers that cannot
allocate device memory (a plug-in limited to the buffers it is given, a
server whose pool already holds all device memory, latency-bound code that
must not call cudaMalloc).  It keeps its scratch in a fixed array of device
memory owned by the library.  Its answers must equal the oracle's
intersection and those of bp_intersect_pair, value for value, on consecutive
calls (which reuse that array and must each clear it).  The file name makes
pytest collect it last."""
import ctypes as C

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1401_6399_gb300.build import build  # noqa: E402

build()
from paper_1401_6399_gb300 import api, capi  # noqa: E402

lib = capi.lib
lib.bp_intersect_pair_noalloc.restype = C.c_int
lib.bp_intersect_pair_noalloc.argtypes = [C.c_void_p, C.c_size_t, C.c_size_t, C.c_void_p,
                                          C.c_size_t, C.c_size_t, C.c_void_p, C.c_size_t,
                                          C.c_void_p, C.c_void_p, C.c_void_p]
MAX_SHORT = 33552384  # BP_NOALLOC_MAX_SHORT_LIST


def noalloc(ea, na, eb, nb, stream):
    cap = max(1, min(na, nb))
    out = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = api.status_tensor()
    rc = lib.bp_intersect_pair_noalloc(ea.data_ptr(), ea.numel(), na, eb.data_ptr(), eb.numel(),
                                       nb, out.data_ptr(), cap, cnt.data_ptr(), st.data_ptr(),
                                       stream.cuda_stream)
    return rc, out, cnt, st


def pairs():
    f = W.uniform(1 << 22, 0, 1 << 26, 0x3000)
    out = []
    for m, seed in ((1 << 18, 0x3000 + (1 << 18)), (1 << 10, 0x3000 + (1 << 10))):
        out.append((W.pair_short(f, m, round(0.1 * m), 1 << 26, seed), f))
    g = W.clustered(300_000, 0, 1 << 25, 0x4004)
    out.append((W.clustered(200_000, 0, 1 << 25, 0x4005), g))
    return out


def test_matches_intersect_pair_on_consecutive_calls(orc):
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for r, f in pairs():
            er = api.to_device(capi.bp_encode(r, capi.BP_LAYOUT_GPU, nthreads=8))
            ef = api.to_device(capi.bp_encode(f, capi.BP_LAYOUT_GPU, nthreads=8))
            want = orc.intersect(r, f)
            fused = api.as_u32(api.intersect_pair(er, r.size, ef, f.size, capi.BP_LAYOUT_GPU,
                                                  capi.BP_MODE_FUSED, stream=s))
            assert np.array_equal(fused, want)
            for _ in range(2):  # two calls in a row share the library's array
                rc, out, cnt, st = noalloc(er, r.size, ef, f.size, s)
                assert rc == capi.BP_OK
                s.synchronize()
                assert int(st.item()) == capi.BP_OK
                n = int(cnt.item())
                assert np.array_equal(api.as_u32(out[:n]), want)
            # arguments in the other order give the same answer
            rc, out, cnt, st = noalloc(ef, f.size, er, r.size, s)
            s.synchronize()
            assert rc == capi.BP_OK and int(st.item()) == capi.BP_OK
            assert np.array_equal(api.as_u32(out[: int(cnt.item())]), want)


def test_empty_list_and_empty_intersection(orc):
    """An empty list in either argument gives an empty answer; disjoint lists
    with the shorter one second give an empty answer too."""
    s = torch.cuda.Stream()
    f = W.uniform(50_000, 0, 1 << 20, 0x6200)
    ef = api.to_device(capi.bp_encode(f, capi.BP_LAYOUT_GPU, nthreads=8))
    empty = np.zeros(0, np.uint32)
    ee = api.to_device(capi.bp_encode(empty, capi.BP_LAYOUT_GPU))
    for a, b in ((ee, ef), (ef, ee)):
        na = 0 if a is ee else f.size
        nb = 0 if b is ee else f.size
        rc, out, cnt, st = noalloc(a, na, b, nb, s)
        s.synchronize()
        assert rc == capi.BP_OK and int(st.item()) == capi.BP_OK and int(cnt.item()) == 0
    f_even = np.unique(f & ~np.uint32(1))  # even values only
    g = np.unique(f[:3000] | np.uint32(1))   # odd values only: disjoint from f_even
    assert orc.intersect(g, f_even).size == 0
    ev = api.to_device(capi.bp_encode(f_even, capi.BP_LAYOUT_GPU, nthreads=8))
    eg = api.to_device(capi.bp_encode(g, capi.BP_LAYOUT_GPU, nthreads=8))
    rc, out, cnt, st = noalloc(ev, f_even.size, eg, g.size, s)  # shorter list second
    s.synchronize()
    assert rc == capi.BP_OK and int(st.item()) == capi.BP_OK and int(cnt.item()) == 0


def test_rejects_a_shorter_list_beyond_the_limit():
    x = api.to_device(capi.bp_encode(np.arange(16, dtype=np.uint32), capi.BP_LAYOUT_GPU))
    s = torch.cuda.Stream()
    rc, out, cnt, st = noalloc(x, MAX_SHORT + 1, x, MAX_SHORT + 1, s)
    assert rc == capi.BP_ERR_SCRATCH
