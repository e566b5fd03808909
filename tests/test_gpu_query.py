"""GPU parity of conjunctive queries (bp_query_batch, bp_query_one) against
the oracle's Set-vs-Set, bit-exact: a Zipf index with clustered lists,
queries of 1..8 terms, every tuning choice, CUDA-graph replay with new
queries, capacity and bad-term handling.  The full-size workload is in
test_gpu_full_size.py."""
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
def small_index():
    lens = W.zipf_lengths(1 << 13, 20_000_000, 1 << 20).astype(np.int64)
    lens[5] = 0      # an empty list
    lens[17] = 1     # a single value
    vals, offs = W.many("clustered", lens, 0, 1 << 22, 0x4100)
    idx = api.Index(vals, offs)
    return idx, vals, offs


def lists_of(vals, offs, terms):
    return [vals[int(offs[t]):int(offs[t + 1])] for t in terms]


def queries(lens, nq, seed, weights=W.CLUEWEB_TERM_WEIGHTS_2_8):
    return W.queries(lens, nq, weights, 2, seed)


def check_all(orc, idx, vals, offs, terms, toff, results):
    for q in range(toff.size - 1):
        t = terms[int(toff[q]):int(toff[q + 1])]
        want = orc.svs(lists_of(vals, offs, t)) if t.size else np.zeros(0, np.uint32)
        assert np.array_equal(results[q], want), f"query {q} terms {t.tolist()}"


def test_batch_matches_svs(orc, small_index):
    idx, vals, offs = small_index
    terms, toff = queries(np.diff(offs), 3000, 0x4A01)
    res = idx.query_batch(terms, toff)
    check_all(orc, idx, vals, offs, terms, toff, res)


def test_batch_single_and_degenerate_queries(orc, small_index):
    idx, vals, offs = small_index
    qs = [[3], [5], [17], [5, 3], [17, 0, 1], [0, 0], [1, 1, 2], [], [2, 9, 33, 70, 101, 500,
                                                                       1000, 4000]]
    terms = np.array([t for q in qs for t in q], np.uint32)
    toff = np.cumsum([0] + [len(q) for q in qs]).astype(np.uint64)
    res = idx.query_batch(terms, toff)
    check_all(orc, idx, vals, offs, terms, toff, res)


@pytest.mark.parametrize("dense,chunk,warps,merge", [(1, 1, 8, 0), (8, 8, 4, 4), (2, 3, 8, 64),
                                                     (4, 1, 4, 1), (4, 8, 8, 0), (8, 8, 8, 64)])
def test_every_tuning_gives_the_same_answers(orc, small_index, dense, chunk, warps, merge):
    idx, vals, offs = small_index
    old = capi.bp_get_tuning()
    try:
        capi.bp_set_tuning(dense_blocks=dense, query_chunk_blocks=chunk, query_warps=warps,
                           merge_span=merge)
        terms, toff = queries(np.diff(offs), 800, 0x4A02 + dense)
        res = idx.query_batch(terms, toff)
        check_all(orc, idx, vals, offs, terms, toff, res)
    finally:
        capi.bp_set_tuning(**old)


def test_plain_path_matches(orc, small_index):
    idx, vals, offs = small_index
    terms, toff = queries(np.diff(offs), 150, 0x4A03)
    for q in range(150):
        t = terms[int(toff[q]):int(toff[q + 1])]
        got = api.as_u32(idx.query_one(t))
        assert np.array_equal(got, orc.svs(lists_of(vals, offs, t)))


def test_graph_replay_with_new_queries(orc, small_index):
    """Capture bp_query_batch once, then refill the same device arrays with
    other queries of the same shape and replay."""
    idx, vals, offs = small_index
    nq, k = 500, 3
    lens = np.diff(offs)
    batches = []
    for s in range(3):
        terms, toff = W.queries(lens, nq, (1,), 3, 0x4B00 + s)  # exactly 3 terms each
        assert np.all(np.diff(toff) == k)
        batches.append(terms)
    toff = np.arange(0, nq * k + 1, k, dtype=np.uint64)
    cap = int(sum(min(int(lens[t]) for t in b.reshape(nq, k)[i]) for b in batches
                  for i in range(nq)))
    sb = max(capi.bp_query_batch_scratch_bytes(idx.h_lists, b, toff, cap) for b in batches)
    dev = "cuda"
    d_terms = torch.zeros(nq * k, dtype=torch.int32, device=dev)
    d_off = torch.from_numpy(toff.view(np.int64).copy()).to(dev)
    out = torch.empty(cap, dtype=torch.int32, device=dev)
    out_off = torch.empty(nq + 1, dtype=torch.int64, device=dev)
    counts = torch.empty(nq, dtype=torch.int32, device=dev)
    scratch = torch.empty(sb, dtype=torch.uint8, device=dev)
    st = api.status_tensor()
    d_terms.copy_(torch.from_numpy(batches[0].view(np.int32)))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):  # warm-up (sets kernel attributes) outside capture
        idx.query_batch_async(d_terms, d_off, nq, nq * k, out, out_off, counts, scratch, st, s)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        idx.query_batch_async(d_terms, d_off, nq, nq * k, out, out_off, counts, scratch, st,
                              torch.cuda.current_stream())
    for b in batches:
        d_terms.copy_(torch.from_numpy(b.view(np.int32)))
        st.zero_()
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        o = out_off.cpu().numpy().view(np.uint64)
        c = counts.cpu().numpy().view(np.uint32)
        flat = api.as_u32(out)
        res = [flat[int(o[q]):int(o[q]) + int(c[q])] for q in range(nq)]
        check_all(orc, idx, vals, offs, b, toff, res)


def test_capacity_and_bad_terms(small_index):
    idx, vals, offs = small_index
    terms = np.array([3, 3], np.uint32)
    toff = np.array([0, 1, 2], np.uint64)
    with pytest.raises(capi.BPError) as e:
        idx.query_batch(terms, toff, out_cap=10, retry=False)
    assert e.value.code == capi.BP_ERR_CAPACITY
    res = idx.query_batch(terms, toff, out_cap=10)  # sized exactly on the second call
    assert idx.last_total == 2 * int(idx.h_lists["n"][3])
    assert np.array_equal(res[0], vals[int(offs[3]):int(offs[4])])
    with pytest.raises(capi.BPError) as e:
        idx.query_batch(np.array([idx.n_terms + 5], np.uint32), np.array([0, 1], np.uint64),
                        out_cap=10)
    assert e.value.code == capi.BP_ERR_ARG


@pytest.fixture(scope="module")
def zipf_data():
    lens = W.zipf_lengths(1 << 13, 20_000_000, 1 << 20).astype(np.int64)
    lens[5] = 0
    lens[17] = 1
    vals, offs = W.many("clustered", lens, 0, 1 << 22, 0x4100)
    return vals, offs


@pytest.mark.parametrize("B", [8, 32, 1 << 22])
def test_hybrid_index_matches_svs(orc, zipf_data, B):
    """hyb+m2: lists with average gap <= B are bitmaps over [0, 2^22); the
    answers are the oracle's Set-vs-Set whatever mix of bitmaps and GL lists a
    query has (B = 2^22: every non-empty list is a bitmap)."""
    vals, offs = zipf_data
    U = 1 << 22
    idx = api.Index(vals, offs, hybrid_B=B, universe=U)
    lens = np.diff(offs)
    is_bm = idx.h_lists["layout"] == capi.BP_LAYOUT_BITMAP
    assert np.array_equal(is_bm, lens.astype(np.uint64) * B >= U)
    assert is_bm.any()
    terms, toff = queries(lens, 1500, 0x4C00 + B)
    nbm = [int(is_bm[terms[int(toff[q]):int(toff[q + 1])]].sum()) for q in range(toff.size - 1)]
    kq = np.diff(toff)
    if B < U:
        assert any(0 < m < k for m, k in zip(nbm, kq))  # mixed queries
    assert any(m == k and k > 1 for m, k in zip(nbm, kq))  # all-bitmap queries
    res = idx.query_batch(terms, toff)
    check_all(orc, idx, vals, offs, terms, toff, res)
    # hand-picked: bitmap alone, bitmap twice, bitmap with the empty list and
    # the single-value list, the longest lists together
    big = np.argsort(lens)[::-1][:4].astype(np.uint32)
    qs = [[big[0]], [big[0], big[0]], [big[0], 5], [17, big[1]], list(big), [big[3], 3, big[2]]]
    terms = np.array([t for q in qs for t in q], np.uint32)
    toff = np.cumsum([0] + [len(q) for q in qs]).astype(np.uint64)
    check_all(orc, idx, vals, offs, terms, toff, idx.query_batch(terms, toff))
    if is_bm[big[0]]:
        with pytest.raises(capi.BPError) as e:  # the plain path takes GL lists only
            idx.query_one(np.array([big[0], 3], np.uint32))
        assert e.value.code == capi.BP_ERR_ARG
