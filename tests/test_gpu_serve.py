"""The serving engine: continuous batching of conjunctive queries over a
resident index.  Every answer must be the same when its query runs alone and
when it runs in an open-loop mix with others (and equal to the oracle's
Set-vs-Set), batches must overlap on the device, and queries too large for a
slot must be rejected without disturbing the others."""
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


@pytest.fixture(scope="module")
def index():
    lens = W.zipf_lengths(1 << 13, 20_000_000, 1 << 20)
    vals, offs = W.many("clustered", lens, 0, 1 << 22, 0x4100)
    return api.Index(vals, offs), vals, offs


def svs(orc, vals, offs, terms):
    return orc.svs([vals[int(offs[t]):int(offs[t + 1])] for t in terms])


def test_alone_equals_mixed_equals_oracle(orc, index):
    idx, vals, offs = index
    terms, toff = W.queries(np.diff(offs), 400, W.CLUEWEB_TERM_WEIGHTS_2_8, 2, 0x5001)
    n = toff.size - 1
    srv = api.Server(idx, slots=4, max_batch_queries=64, max_terms=8, slot_bytes=256 << 20)
    try:
        alone = {}
        for q in range(n):  # one query at a time
            srv.submit(q, terms[int(toff[q]):int(toff[q + 1])])
            srv.drain()
            (tag, cnt, st, ta, t0, t1, ans), = srv.poll()
            assert ta == t0 <= t1  # a direct submission arrives when it is queued
            assert tag == q and st == capi.BP_OK and ans.size == cnt
            alone[q] = ans
        # the same queries in an open-loop mix at 200,000 queries/s
        arrivals = W.poisson_arrivals(200_000.0, n, 0x5002)
        srv.replay(np.arange(n) + 1000, terms, toff, arrivals)
        srv.drain()
        res = srv.poll()
        mixed = {r[0] - 1000: r[6] for r in res}
        st = srv.stats()
        recs = srv.batches()
    finally:
        srv.close()
    assert sorted(mixed) == list(range(n))
    for q in range(n):
        want = svs(orc, vals, offs, terms[int(toff[q]):int(toff[q + 1])])
        assert np.array_equal(alone[q], want), q
        assert np.array_equal(mixed[q], want), q
    assert st["completed"] == st["submitted"] == 2 * n
    assert st["batches"] > n  # alone: one batch each; mixed: several batches
    assert st["max_busy_slots"] >= 2  # batches overlapped on the device
    # replayed queries are stamped with their scheduled arrival: queued no
    # earlier than due, answered after both
    arr = np.array([r[3] for r in res])
    sub = np.array([r[4] for r in res])
    done = np.array([r[5] for r in res])
    assert np.all(sub >= arr) and np.all(done >= sub)
    order = np.argsort([r[0] for r in res])
    assert np.all(np.abs(arr[order] - arr[order][0] - (arrivals - arrivals[0])) < 1e-6)
    # the timeline holds every batch of both phases, in a consistent order
    assert recs.size == st["batches"]
    assert int(recs["queries"].sum()) == 2 * n
    assert np.all(recs["admit_s"] <= recs["launched_s"])
    assert np.all(recs["launched_s"] <= recs["done_s"])
    assert np.all(recs["done_s"] <= recs["retired_s"])


def test_oversized_query_is_rejected_alone(orc, index):
    idx, vals, offs = index
    lens = np.diff(offs)
    big = int(np.argmax(lens))           # longest list: its answer bound is huge
    small = [int(np.argsort(lens)[10]), int(np.argsort(lens)[20])]
    srv = api.Server(idx, slots=2, max_batch_queries=16, max_terms=8, slot_bytes=1 << 20)
    try:
        srv.submit(1, [big])
        srv.submit(2, small)
        srv.drain()
        res = {r[0]: r for r in srv.poll()}
    finally:
        srv.close()
    assert res[1][2] == capi.BP_ERR_SCRATCH
    assert res[2][2] == capi.BP_OK
    assert np.array_equal(res[2][6], svs(orc, vals, offs, small))


def test_hybrid_index_served(orc):
    """The engine over a hybrid (hyb+m2) index: lists with average gap <= 16
    are bitmaps; answers of an open-loop mix equal the oracle's."""
    lens = W.zipf_lengths(1 << 12, 8_000_000, 1 << 20)
    vals, offs = W.many("clustered", lens, 0, 1 << 22, 0x5100)
    idx = api.Index(vals, offs, hybrid_B=16, universe=1 << 22)
    assert (idx.h_lists["layout"] == capi.BP_LAYOUT_BITMAP).any()
    terms, toff = W.queries(np.diff(offs), 300, W.CLUEWEB_TERM_WEIGHTS_2_8, 2, 0x5101)
    n = toff.size - 1
    srv = api.Server(idx, slots=4, max_batch_queries=64, max_terms=8, slot_bytes=256 << 20)
    try:
        srv.replay(np.arange(n), terms, toff, W.poisson_arrivals(100_000.0, n, 0x5102))
        srv.drain()
        got = {r[0]: (r[2], r[6]) for r in srv.poll()}
    finally:
        srv.close()
    assert sorted(got) == list(range(n))
    for q in range(n):
        st, ans = got[q]
        assert st == capi.BP_OK
        assert np.array_equal(ans, svs(orc, vals, offs, terms[int(toff[q]):int(toff[q + 1])])), q
