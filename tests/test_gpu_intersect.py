"""GPU parity of bp_intersect_pair (fused GL x GL, unfused GL and PL) against
the oracle's merge intersection, bit-exact: the tiny pair, the full-size
length-ratio sweep (2^22 against 2^22 .. 2^8), clustered pairs, edge cases,
every regime threshold, capacity overflow."""
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

MODES = [(capi.BP_LAYOUT_GPU, capi.BP_MODE_FUSED), (capi.BP_LAYOUT_GPU, capi.BP_MODE_UNFUSED),
         (capi.BP_LAYOUT_PAPER, capi.BP_MODE_UNFUSED)]


def gpu_intersect(a, b, layout, mode):
    ea = api.to_device(capi.bp_encode(a, layout, nthreads=8))
    eb = api.to_device(capi.bp_encode(b, layout, nthreads=8))
    return api.as_u32(api.intersect_pair(ea, a.size, eb, b.size, layout, mode))


@pytest.mark.parametrize("layout,mode", MODES)
def test_tiny_pair(orc, layout, mode):
    a = W.uniform(65536, 0, 1 << 20, 0x1001)
    b = W.uniform(4096, 0, 1 << 20, 0x1002)
    want = orc.intersect(a, b)
    assert np.array_equal(gpu_intersect(a, b, layout, mode), want)
    assert np.array_equal(gpu_intersect(b, a, layout, mode), want)


@pytest.fixture(scope="module")
def long_list():
    return W.uniform(1 << 22, 0, 1 << 26, 0x3000)


@pytest.mark.parametrize("m", [1 << 22, 1 << 18, 1 << 14, 1 << 10, 1 << 8])
@pytest.mark.parametrize("layout,mode", MODES)
def test_ratio_sweep_full_size(orc, long_list, m, layout, mode):
    """Longer list 2^22 values of [0, 2^26); shorter list m values sharing
    round(0.1 m) of them."""
    f = long_list
    k = round(0.1 * m)
    r = W.pair_short(f, m, k, 1 << 26, 0x3000 + m)
    want = orc.intersect(r, f)
    assert want.size == k
    assert np.array_equal(gpu_intersect(r, f, layout, mode), want)


@pytest.mark.parametrize("m", [1 << 22, 1 << 18, 1 << 14])
@pytest.mark.parametrize("merge_span", [0, 1, 64])
def test_ratio_sweep_merge_regime_on_and_off(orc, long_list, m, merge_span):
    """The fused path of the ratio sweep with the merge regime off (0), only
    for runs of equal density (1), and for every run within 64 blocks of f
    per block of r."""
    f = long_list
    k = round(0.1 * m)
    r = W.pair_short(f, m, k, 1 << 26, 0x3000 + m)
    want = orc.intersect(r, f)
    old = capi.bp_get_tuning()
    try:
        capi.bp_set_tuning(merge_span=merge_span)
        got = gpu_intersect(r, f, capi.BP_LAYOUT_GPU, capi.BP_MODE_FUSED)
    finally:
        capi.bp_set_tuning(**old)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("dense,merge_span", [(1, 0), (2, 4), (4, 0), (4, 4), (8, 64), (8, 1)])
def test_every_regime_threshold_gives_the_same_result(orc, dense, merge_span):
    old = capi.bp_get_tuning()
    try:
        capi.bp_set_tuning(dense_blocks=dense, merge_span=merge_span)
        f = W.clustered(300_000, 0, 1 << 26, 0x77)
        for m in (300_000, 30_000, 3_000, 300, 30):
            r = W.pair_short(f, m, m // 3, 1 << 26, m)
            want = orc.intersect(r, f)
            for layout, mode in MODES[:2]:
                assert np.array_equal(gpu_intersect(r, f, layout, mode), want)
    finally:
        capi.bp_set_tuning(**old)


@pytest.mark.parametrize("layout,mode", MODES)
def test_clustered_pairs(orc, layout, mode):
    for i, (n, m) in enumerate([(1 << 20, 1 << 20), (1 << 20, 5000), (200_000, 199_999)]):
        f = W.clustered(n, 0, 1 << 25, 0x4000 + i)
        g = W.clustered(m, 0, 1 << 25, 0x5000 + i)
        assert np.array_equal(gpu_intersect(g, f, layout, mode), orc.intersect(g, f))


@pytest.mark.parametrize("layout,mode", MODES)
def test_edge_cases(orc, layout, mode):
    rng = np.random.default_rng(5)
    f = np.sort(rng.choice(1 << 20, 5000, replace=False)).astype(np.uint32)
    cases = [
        (np.zeros(0, np.uint32), f),
        (f, np.zeros(0, np.uint32)),
        (np.zeros(0, np.uint32), np.zeros(0, np.uint32)),
        (f, f),                                             # identical
        (f[::7].copy(), f),                                 # subset
        (f * 2 + 1 if f.max() < 2**30 else f, f * 2),       # disjoint
        (np.array([f[0]], np.uint32), f),                   # single, first
        (np.array([f[-1]], np.uint32), f),                  # single, last
        (np.array([0], np.uint32), f + 1),                  # below everything
        (np.array([2**32 - 1], np.uint32), f),              # above everything
        (np.arange(0, 1 << 20, 3, dtype=np.uint32), f),     # dense r
        (f[:129].copy(), f[:131].copy()),                   # ragged tails
    ]
    for a, b in cases:
        a = np.ascontiguousarray(a, np.uint32)
        b = np.ascontiguousarray(b, np.uint32)
        want = orc.intersect(a, b)
        assert np.array_equal(gpu_intersect(a, b, layout, mode), want)


def test_fused_requires_gpu_layout():
    a = api.to_device(capi.bp_encode(np.arange(10, dtype=np.uint32), 0))
    with pytest.raises(capi.BPError) as e:
        api.intersect_pair(a, 10, a, 10, capi.BP_LAYOUT_PAPER, capi.BP_MODE_FUSED)
    assert e.value.code == capi.BP_ERR_ARG


def test_capacity_overflow_reports_count():
    x = np.arange(0, 40_000, dtype=np.uint32)
    ea = api.to_device(capi.bp_encode(x, 1))
    out = torch.empty(100, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    sb = capi.bp_intersect_scratch_bytes(x.size, x.size, 1, 2)
    scratch = torch.empty(max(sb, 16), dtype=torch.uint8, device="cuda")
    st = api.status_tensor()
    rc = capi.bp_intersect_pair(ea.data_ptr(), ea.numel(), x.size, ea.data_ptr(), ea.numel(),
                                x.size, 1, 2, out.data_ptr(), 100, cnt.data_ptr(),
                                scratch.data_ptr(), sb, st.data_ptr(),
                                torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert rc == capi.BP_OK
    assert int(st.item()) == capi.BP_ERR_CAPACITY
    assert int(cnt.item()) == x.size
    assert np.array_equal(api.as_u32(out), x[:100])


@pytest.mark.parametrize("kind", [1, 2, 3])
def test_kinds_unfused_and_fused_rejection(orc, kind):
    """Lists coded with DM, D2 or D1 (Section 5): the unfused intersection
    (decode both, then intersect) is exact in both layouts; the fused path,
    whose probes use D4 columns, records BP_ERR_ARG instead of an answer."""
    f = W.uniform(1 << 18, 0, 1 << 22, 0x7100 + kind)
    r = W.pair_short(f, 1 << 12, 400, 1 << 22, 0x7200 + kind)
    want = orc.intersect(r, f)
    for layout in (capi.BP_LAYOUT_PAPER, capi.BP_LAYOUT_GPU):
        er = api.to_device(capi.bp_encode(r, layout, delta=kind))
        ef = api.to_device(capi.bp_encode(f, layout, delta=kind))
        got = api.intersect_pair(er, r.size, ef, f.size, layout, capi.BP_MODE_UNFUSED)
        assert np.array_equal(api.as_u32(got), want), (kind, layout)
    er = api.to_device(capi.bp_encode(r, capi.BP_LAYOUT_GPU, delta=kind))
    ef = api.to_device(capi.bp_encode(f, capi.BP_LAYOUT_GPU, delta=kind))
    with pytest.raises(capi.BPError) as e:
        api.intersect_pair(er, r.size, ef, f.size, capi.BP_LAYOUT_GPU, capi.BP_MODE_FUSED)
    assert e.value.code == capi.BP_ERR_ARG
