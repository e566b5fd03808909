"""Bounded device waits end and are reported.  The ordered output of
bp_intersect_pair makes every CTA wait, by polling, for the output counts of
the CTAs before it (a decoupled look-back).  Here one tile is told to publish
nothing (bp_tuning.withhold_tile) and the poll limit is made short
(bp_tuning.lookback_spin_limit), so the tiles after it run out of polls: the
call must still complete, report BP_ERR_TIMEOUT in its status word, and leave
the stream usable: the next normal call on it gives the exact answer."""
import time

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


def fused_call(er, nr, ef, nf, stream):
    cap = max(1, min(nr, nf))
    out = torch.empty(cap, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    sb = capi.bp_intersect_scratch_bytes(nr, nf, capi.BP_LAYOUT_GPU, capi.BP_MODE_FUSED)
    scratch = torch.empty(max(sb, 16), dtype=torch.uint8, device="cuda")
    st = api.status_tensor()
    capi.check(capi.bp_intersect_pair(er.data_ptr(), er.numel(), nr, ef.data_ptr(), ef.numel(),
                                      nf, capi.BP_LAYOUT_GPU, capi.BP_MODE_FUSED,
                                      out.data_ptr(), cap, cnt.data_ptr(), scratch.data_ptr(), sb,
                                      st.data_ptr(), stream.cuda_stream), "bp_intersect_pair")
    return out, cnt, st


@pytest.mark.parametrize("withhold", [1, 7])
def test_lookback_wait_runs_out_and_is_reported(orc, withhold):
    # 2^18 against 2^18: 256 tiles of 8 warps (one block of r per warp)
    f = W.uniform(1 << 18, 0, 1 << 22, 0x6100)
    r = W.pair_short(f, 1 << 18, 1 << 14, 1 << 22, 0x6101)
    want = orc.intersect(r, f)
    er = api.to_device(capi.bp_encode(r, capi.BP_LAYOUT_GPU, nthreads=8))
    ef = api.to_device(capi.bp_encode(f, capi.BP_LAYOUT_GPU, nthreads=8))
    s = torch.cuda.Stream()
    old = capi.bp_get_tuning()
    try:
        capi.bp_set_tuning(lookback_spin_limit=1 << 10, withhold_tile=withhold)
        t0 = time.time()
        out, cnt, st = fused_call(er, r.size, ef, f.size, s)
        s.synchronize()
        dt = time.time() - t0
    finally:
        capi.bp_set_tuning(**old)
    assert int(st.item()) == capi.BP_ERR_TIMEOUT
    assert dt < 30.0  # 1,024 polls per wait: milliseconds, not the default's seconds
    # the same stream, normal limits: exact
    out, cnt, st = fused_call(er, r.size, ef, f.size, s)
    s.synchronize()
    assert int(st.item()) == capi.BP_OK
    assert np.array_equal(api.as_u32(out[: int(cnt.item())]), want)
