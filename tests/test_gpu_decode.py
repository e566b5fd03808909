"""GPU parity of decoding (bp_decode, bp_decode_sum, bp_decode_batch) against
the scalar oracle, bit-exact, for both layouts: edge lengths, ragged tails,
many tiles, mixed widths, full-size lists, corrupt streams."""
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

LAYOUTS = [capi.BP_LAYOUT_PAPER, capi.BP_LAYOUT_GPU]


def oracle_decode(orc, x, layout):
    return orc.pl_decode(orc.pl_encode(x)) if layout == 0 else orc.gl_decode(orc.gl_encode(x))


def gpu_decode(x, layout):
    enc = capi.bp_encode(x, layout, nthreads=8)
    return api.as_u32(api.decode(api.to_device(enc), layout, x.size))


EDGE = [0, 1, 2, 4, 5, 127, 128, 129, 255, 2047, 2048, 2049, 4095, 4096, 4097,
        3 * 4096 + 129, 16 * 2048 + 15 * 128 + 127, 65536, 65549]


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("n", EDGE)
def test_decode_edge_lengths(orc, layout, n):
    rng = np.random.default_rng(n * 3 + layout)
    for U in (n + 1, 16 * n + 16, 1 << 32):
        x = np.sort(rng.choice(U, n, replace=False)).astype(np.uint32)
        got = gpu_decode(x, layout)
        ref = oracle_decode(orc, x, layout)
        assert np.array_equal(ref, x)
        assert np.array_equal(got, ref)


@pytest.mark.parametrize("layout", LAYOUTS)
def test_decode_tiny_config(orc, layout):
    """A = 65,536 and B = 4,096 distinct values of [0, 2^20)."""
    for n, seed in ((65536, 0x1001), (4096, 0x1002)):
        x = W.uniform(n, 0, 1 << 20, seed)
        assert np.array_equal(gpu_decode(x, layout), oracle_decode(orc, x, layout))


@pytest.mark.parametrize("layout", LAYOUTS)
def test_decode_clustered_many_tiles(orc, layout):
    """Clustered values mix widths 3..25 inside one list; 2^20+77 integers
    span thousands of tiles and end in a ragged tail."""
    x = W.clustered((1 << 20) + 77, 0, 1 << 29, 0x2100)
    enc = capi.bp_encode(x, layout, nthreads=8)
    got = api.as_u32(api.decode(api.to_device(enc), layout, x.size))
    ref = orc.pl_decode(enc.tobytes()) if layout == 0 else orc.gl_decode(enc.tobytes())
    assert np.array_equal(got, ref)
    assert np.array_equal(got, x)


@pytest.mark.parametrize("layout", LAYOUTS)
def test_decode_all_widths(orc, layout):
    """One block of every width 0..32: D4 deltas drawn below 2^w per block
    (the codec is exact modulo 2^32 for any sequence), streams built bit by
    bit from the format definition, decoded on the GPU and by the oracle."""
    import brute
    rng = np.random.default_rng(7)
    widths = list(range(33)) + [7, 0, 32]
    d = []
    for w in widths:
        blk = rng.integers(0, 1 << max(w - 1, 0), 128, dtype=np.uint64) if w else \
            np.zeros(128, np.uint64)
        if w:
            blk[rng.integers(1, 128)] = (1 << w) - 1
        d.append(blk)
    if layout == 0:  # D4 carried across blocks from (0,0,0,0)
        d = np.concatenate(d)
        x = np.zeros(d.size + 37, np.uint64)
        for i in range(d.size):
            x[i] = (d[i] + (x[i - 4] if i >= 4 else 0)) % (1 << 32)
        x[d.size:] = (x[d.size - 1] + np.arange(1, 38)) % (1 << 32)
    else:  # D4 restarted at every block from its first value F
        parts = []
        for blk in d:
            blk[0] = 0
            F = int(rng.integers(0, 1 << 32))
            xb = np.zeros(128, np.uint64)
            for i in range(128):
                xb[i] = (int(blk[i]) + (int(xb[i - 4]) if i >= 4 else F)) % (1 << 32)
            parts.append(xb)
        x = np.concatenate(parts + [np.arange(5, dtype=np.uint64)])
    x = x.astype(np.uint32)
    stream = brute.pl_stream(x) if layout == 0 else brute.gl_stream(x)
    enc = np.frombuffer(stream, np.uint8)
    got = api.as_u32(api.decode(api.to_device(enc), layout, x.size))
    ref = orc.pl_decode(stream) if layout == 0 else orc.gl_decode(stream)
    assert np.array_equal(ref, x)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("layout", LAYOUTS)
def test_decode_sum(orc, layout):
    for n, seed in ((0, 1), (100, 2), (65536 + 99, 3), (1 << 20, 4)):
        x = W.clustered(n, 0, 1 << 31, seed) if n else np.zeros(0, np.uint32)
        enc = capi.bp_encode(x, layout)
        got = api.decode_sum(api.to_device(enc), layout, n)
        ref = oracle_decode(orc, x, layout)
        assert got == int(ref.astype(np.uint64).sum()) % (1 << 64)


@pytest.mark.parametrize("layout", LAYOUTS)
def test_decode_batch(orc, layout):
    rng = np.random.default_rng(99)
    sizes = [0, 1, 130, 4096, 5000, 2048 * 16 + 3, 777, 128 * 33]
    xs = [np.sort(rng.choice(1 << 30, n, replace=False)).astype(np.uint32) for n in sizes]
    encs = [capi.bp_encode(x, layout) for x in xs]
    batch = api.ListBatch(encs, sizes, layout)
    got = api.as_u32(batch.decode())
    ref = np.concatenate([oracle_decode(orc, x, layout) for x in xs])
    assert np.array_equal(got, ref)
    sums = batch.sums()
    assert sums.tolist() == [int(x.astype(np.uint64).sum()) for x in xs]


KINDS = [1, 2, 3]  # DM, D2, D1 (Section 5); D4 is every other test here


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("kind", KINDS)
def test_decode_kinds(orc, layout, kind):
    """DM, D2 and D1 streams decode bit-exactly (both layouts): edge lengths,
    ragged tails, widths from 1 to 32 and every width dispatch path."""
    rng = np.random.default_rng(10 * kind + layout)
    for n in (0, 1, 5, 127, 128, 129, 2047, 2049, 4097, 3 * 2048 + 15 * 128 + 127, 300_001):
        for U in (n + 1, 64 * n + 64, 1 << 32):
            x = np.sort(rng.choice(U, n, replace=False)).astype(np.uint32)
            enc = capi.bp_encode(x, layout, delta=kind)
            want = orc.pl_decode(enc.tobytes()) if layout == 0 else orc.gl_decode(enc.tobytes())
            assert np.array_equal(want, x)
            got = api.as_u32(api.decode(api.to_device(enc), layout, x.size))
            assert np.array_equal(got, want), (layout, kind, n, U)
            assert api.decode_sum(api.to_device(enc), layout, x.size) == int(x.astype(np.uint64).sum()) % (1 << 64)


@pytest.mark.parametrize("layout", LAYOUTS)
def test_decode_batch_mixed_kinds(orc, layout):
    """One batch of lists of all four kinds, clustered and uniform: every
    list decodes with its own kind (read from its header)."""
    xs, encs = [], []
    for i in range(12):
        n = [70_000, 128 * 40 + 3, 2048 * 5, 99][i % 4]
        x = (W.clustered(n, 0, 1 << 30, 7000 + i) if i % 2 else
             W.uniform(n, 0, 1 << 30, 7000 + i))
        xs.append(x)
        encs.append(capi.bp_encode(x, layout, delta=i % 4))
    batch = api.ListBatch(encs, [x.size for x in xs], layout)
    got = api.as_u32(batch.decode())
    assert np.array_equal(got, np.concatenate(xs))
    assert batch.sums().tolist() == [int(x.astype(np.uint64).sum()) for x in xs]


@pytest.mark.parametrize("kind", [0, 1, 2, 3])
def test_paper_layout_stage_regimes(orc, kind):
    """Paper layout at densities on both sides of its two shared-memory
    stages (chunks of 32 blocks up to about 7.3 and 9.9 bits/int) and far
    beyond them (chunks read from global memory after an L2 prefetch): each
    list alone (its own density picks the stage), then all of them in one
    batch (the average picks it, wider chunks go to global memory); decode
    and decode+sum, bit-exact against the oracle and the input."""
    n = 3 * 2048 * 16 + 2048 + 77  # many chunks and tiles, a ragged tail
    xs, encs = [], []
    for k, shift in enumerate((2, 3, 4, 5, 6, 9, 14)):  # about shift + 4 bits per integer
        x = W.uniform(n, 0, n << shift, 0x5100 + 16 * kind + k)
        enc = capi.bp_encode(x, capi.BP_LAYOUT_PAPER, delta=kind)
        want = orc.pl_decode(enc.tobytes())
        assert np.array_equal(want, x)
        got = api.as_u32(api.decode(api.to_device(enc), capi.BP_LAYOUT_PAPER, n))
        assert np.array_equal(got, want), (kind, shift)
        assert api.decode_sum(api.to_device(enc), capi.BP_LAYOUT_PAPER, n) == \
            int(x.astype(np.uint64).sum()) % (1 << 64)
        xs.append(x)
        encs.append(enc)
    for order in (xs, xs[::-1]):
        oe = encs if order is xs else encs[::-1]
        batch = api.ListBatch(oe, [n] * len(oe), capi.BP_LAYOUT_PAPER)
        assert np.array_equal(api.as_u32(batch.decode()), np.concatenate(order))
        assert batch.sums().tolist() == [int(x.astype(np.uint64).sum()) for x in order]


def _outlier_list(rng, n):
    """Sorted distinct values: small gaps with rare large jumps, so that
    S4-FastPFOR blocks carry exceptions of several widths."""
    gaps = rng.geometric(0.2, n).astype(np.uint64)
    jumps = rng.random(n) < 0.02
    gaps[jumps] = rng.integers(1 << 8, 1 << 22, int(jumps.sum()))
    return (np.cumsum(gaps) % (1 << 32)).astype(np.uint32) if n else np.zeros(0, np.uint32)


@pytest.mark.parametrize("kind", [0, 1, 2, 3])
def test_decode_pfor(orc, kind):
    """S4-FastPFOR (GP layout) decodes bit-exactly against the oracle: edge
    lengths, ragged tails, exceptions of many widths, the stream of the
    library encoder equal to the oracle's byte for byte, decode and sum."""
    rng = np.random.default_rng(60 + kind)
    for n in (0, 1, 5, 127, 128, 129, 4095, 4096, 4097, 3 * 4096 + 200, 300_001):
        x = np.unique(_outlier_list(rng, n))
        enc = capi.bp_encode(x, capi.BP_LAYOUT_PFOR, 4, kind)
        assert enc.tobytes() == orc.gp_encode(x, kind)
        want = orc.gp_decode(enc.tobytes())
        assert np.array_equal(want, x)
        got = api.as_u32(api.decode(api.to_device(enc), capi.BP_LAYOUT_PFOR, x.size))
        assert np.array_equal(got, want), (kind, n)
        assert (api.decode_sum(api.to_device(enc), capi.BP_LAYOUT_PFOR, x.size) ==
                int(x.astype(np.uint64).sum()) % (1 << 64))


def test_decode_pfor_batch_widths_and_order(orc):
    """One batch of GP lists: every width 0..32 (stepped walks modulo 2^32 with
    planted outliers, BP_ENCODE_ANY_ORDER), all kinds, ragged lengths; pages
    too large for the shared-memory stage take the global-memory path."""
    xs, encs = [], []
    rng = np.random.default_rng(61)
    for b in range(33):
        kind = b % 4
        n = [4096, 4096 * 2 + 77, 129, 1, 0, 6000][b % 6]
        x = W.stepped_walk(n, b, 1200 + b)
        if n > 10:  # outliers: a few values moved far away
            idx = rng.choice(n, max(1, n // 100), replace=False)
            x[idx] = rng.integers(0, 1 << 32, idx.size, dtype=np.uint64).astype(np.uint32)
        e = capi.bp_encode(x, capi.BP_LAYOUT_PFOR, 1, kind | capi.BP_ENCODE_ANY_ORDER)
        assert np.array_equal(orc.gp_decode(e.tobytes()), x)
        xs.append(x)
        encs.append(e)
    batch = api.ListBatch(encs, [x.size for x in xs], capi.BP_LAYOUT_PFOR)
    assert np.array_equal(api.as_u32(batch.decode()), np.concatenate(xs))
    assert batch.sums().tolist() == [int(x.astype(np.uint64).sum()) % (1 << 64) for x in xs]


@pytest.mark.parametrize("mode", [0, 1])
def test_decode_ablation_any_width_and_order(orc, mode):
    """bp_decode_ablation (prefix integrated or as a separate pass) and
    bp_decode_batch agree with the oracle on GL streams of every kind whose
    blocks all have width b (stepped walks modulo 2^32, encoded with
    BP_ENCODE_ANY_ORDER), ragged lengths, one batch of lists."""
    xs, encs = [], []
    for b in (0, 1, 2, 3, 7, 8, 13, 16, 24, 31, 32):
        for kind in range(4):
            n = [4096, 4096 * 3 + 77, 129, 1, 0][(b + kind) % 5]
            x = W.stepped_walk(n, b, 900 + 4 * b + kind)
            e = capi.bp_encode(x, capi.BP_LAYOUT_GPU, 1, kind | capi.BP_ENCODE_ANY_ORDER)
            assert np.array_equal(orc.gl_decode(e.tobytes()), x)
            xs.append(x)
            encs.append(e)
    batch = api.ListBatch(encs, [x.size for x in xs], capi.BP_LAYOUT_GPU)
    want = np.concatenate(xs)
    out = torch.full((max(batch.total_n, 1),), -1, dtype=torch.int32, device="cuda")
    st = api.status_tensor()
    batch.ablation_into(out, st, mode)
    api.check_status(st, "bp_decode_ablation")
    assert np.array_equal(api.as_u32(out[:batch.total_n]), want)
    assert np.array_equal(api.as_u32(batch.decode()), want)


def test_decode_batch_kinds_short_output():
    """A batch whose last list (DM) does not fit the output records
    BP_ERR_CAPACITY; the lists that fit are decoded."""
    xs = [W.uniform(5000 + 1000 * i, 0, 1 << 28, 7100 + i) for i in range(3)]
    encs = [capi.bp_encode(x, capi.BP_LAYOUT_GPU, delta=k) for x, k in zip(xs, (0, 2, 1))]
    batch = api.ListBatch(encs, [x.size for x in xs], capi.BP_LAYOUT_GPU)
    short = xs[0].size + xs[1].size + 10
    out = torch.full((short,), -1, dtype=torch.int32, device="cuda")
    st = api.status_tensor()
    batch.decode_into(out, st)
    torch.cuda.synchronize()
    assert int(st.item()) == capi.BP_ERR_CAPACITY
    assert np.array_equal(api.as_u32(out[:short - 10]), np.concatenate(xs[:2]))


@pytest.mark.parametrize("layout", LAYOUTS)
def test_decode_batch_host(orc, layout):
    """bp_decode_batch_host from pinned host memory to pinned host memory.
    Streams packed in list order take the pipelined path (groups of lists
    copied in, decoded and copied out on library streams); streams packed in
    reverse order take the one-shot path.  Both must give the oracle's lists,
    and work enqueued afterwards on the caller's stream must see the output."""
    rng = np.random.default_rng(7)
    sizes = [0, 1, 130, 4096, 5000, 2048 * 16 + 3, 777, 128 * 33, 300000, 65536, 2, 1 << 20]
    xs = [np.sort(rng.choice(1 << 31, n, replace=False)).astype(np.uint32) for n in sizes]
    encs = [capi.bp_encode(x, layout) for x in xs]
    ref = np.concatenate([oracle_decode(orc, x, layout) for x in xs])
    total_n = ref.size
    for order in ("ascending", "reversed"):
        place = list(range(len(xs))) if order == "ascending" else list(reversed(range(len(xs))))
        enc_off, pos = {}, 0
        for i in place:
            enc_off[i] = pos
            pos += (encs[i].size + 15) // 16 * 16
        host = np.zeros(max(pos, 16), np.uint8)
        lists = np.zeros(len(xs), capi.BP_LIST)
        out_off = 0
        for i, (e, n) in enumerate(zip(encs, sizes)):
            host[enc_off[i]:enc_off[i] + e.size] = e
            lists[i] = (enc_off[i], e.size, out_off, 0, n, layout, 0)
            out_off += n
        total_units = capi.bp_plan_lists(lists)
        h_data = torch.from_numpy(host).pin_memory()
        h_lists = torch.from_numpy(lists.view(np.uint8).copy()).pin_memory()
        h_out = torch.zeros(total_n, dtype=torch.int32).pin_memory()
        h_status = torch.full((1,), -1, dtype=torch.int32).pin_memory()
        d_data = torch.empty(host.size, dtype=torch.uint8, device="cuda")
        d_lists = torch.empty(h_lists.numel(), dtype=torch.uint8, device="cuda")
        d_out = torch.empty(total_n, dtype=torch.int32, device="cuda")
        d_status = torch.zeros(1, dtype=torch.int32, device="cuda")
        sb = capi.bp_decode_batch_scratch_bytes(lists)
        scratch = torch.empty(max(sb, 16), dtype=torch.uint8, device="cuda")
        s = torch.cuda.Stream()
        for _ in range(2):  # a second call reuses the library's streams and events
            capi.check(capi.bp_decode_batch_host(
                h_data.data_ptr(), host.size, h_lists.data_ptr(), len(xs), total_units, layout,
                d_data.data_ptr(), d_lists.data_ptr(), d_out.data_ptr(), total_n,
                h_out.data_ptr(), scratch.data_ptr(), sb, d_status.data_ptr(),
                h_status.data_ptr(), s.cuda_stream), "bp_decode_batch_host")
            with torch.cuda.stream(s):
                after = d_out.clone()  # ordered after the call on the caller's stream
            s.synchronize()
            assert int(h_status.item()) == 0, order
            assert np.array_equal(h_out.numpy().view(np.uint32), ref), order
            assert np.array_equal(api.as_u32(after), ref), order
            h_out.zero_()


@pytest.mark.parametrize("layout", LAYOUTS)
def test_decode_full_size_batch(layout):
    """Four lists of 2^26 integers in [0, 2^29) (two uniform, two clustered),
    decoded in one batch launch as the benchmark does; a decoded list must be
    the encoded list (round trip), and the sums must match."""
    xs, _ = W.many("uniform", [1 << 26] * 2, 0, 1 << 29, 0x2000)
    xc, _ = W.many("clustered", [1 << 26] * 2, 0, 1 << 29, 0x2000)
    lists = [xs[:1 << 26], xs[1 << 26:], xc[:1 << 26], xc[1 << 26:]]
    encs = [capi.bp_encode(x, layout, nthreads=16) for x in lists]
    batch = api.ListBatch(encs, [x.size for x in lists], layout)
    got = batch.decode()
    want = torch.from_numpy(np.concatenate(lists).view(np.int32)).to(got.device)
    assert torch.equal(got, want)
    assert batch.sums().tolist() == [int(x.astype(np.uint64).sum()) for x in lists]


def _status_of(enc, layout, n, cap=None):
    d = api.to_device(enc)
    out = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    sb = capi.bp_decode_scratch_bytes(n, layout)
    scratch = torch.empty(max(sb, 1), dtype=torch.uint8, device="cuda")
    st = api.status_tensor()
    rc = capi.bp_decode(d.data_ptr(), d.numel(), layout, n, out.data_ptr(),
                        cap if cap is not None else n, scratch.data_ptr(), sb, st.data_ptr(),
                        torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return rc, int(st.item())


def test_corrupt_streams_record_status():
    x = np.arange(3, 3 + 5 * 9000, 5, dtype=np.uint32)
    pl = capi.bp_encode(x, 0).copy()
    bad = pl.copy()
    bad[16] = 33  # a width byte beyond 32
    assert _status_of(bad, 0, x.size) == (capi.BP_OK, capi.BP_ERR_CORRUPT)
    assert _status_of(pl[:-5], 0, x.size)[1] == capi.BP_ERR_CORRUPT  # truncated
    assert _status_of(pl, 0, x.size - 1)[1] == capi.BP_ERR_CORRUPT   # wrong n
    gl = capi.bp_encode(x, 1).copy()
    off_bw = int(gl[32:36].view(np.uint32)[0])
    bad = gl.copy()
    bad[off_bw + 3] = 40
    assert _status_of(bad, 1, x.size)[1] == capi.BP_ERR_CORRUPT
    bad = gl.copy()
    bad[0] ^= 1  # magic
    assert _status_of(bad, 1, x.size)[1] == capi.BP_ERR_CORRUPT
    assert _status_of(gl, 1, x.size)[1] == capi.BP_OK
    assert _status_of(gl, 1, x.size, cap=x.size - 1)[0] == capi.BP_ERR_CAPACITY


def test_corrupt_pfor_streams_record_status():
    """GP streams with an inconsistent meta entry, page offset, position byte,
    magic or length record BP_ERR_CORRUPT (every access stays inside the
    stream: the page's words are checked against its meta entries first)."""
    rng = np.random.default_rng(70)
    x = np.unique(_outlier_list(rng, 20_000))
    gp = capi.bp_encode(x, capi.BP_LAYOUT_PFOR, 1).copy()
    L = capi.BP_LAYOUT_PFOR
    assert _status_of(gp, L, x.size) == (capi.BP_OK, capi.BP_OK)
    h = gp[:64].view(np.uint32)
    off_spo, off_meta, off_payload = int(h[7]), int(h[8]), int(h[9])
    meta = gp[off_meta:off_meta + 4 * int(h[3])].reshape(-1, 4)
    k = int(np.flatnonzero(meta[:, 2])[0])        # a block with exceptions
    bad = gp.copy()
    bad[off_meta + 4 * k + 1] = 40                # b' + (b - b') > 32
    assert _status_of(bad, L, x.size)[1] == capi.BP_ERR_CORRUPT
    bad = gp.copy()
    bad[off_meta + 4 * k + 0] += 1                # page words no longer match
    assert _status_of(bad, L, x.size)[1] == capi.BP_ERR_CORRUPT
    bad = gp.copy()
    bad[off_spo + 4:off_spo + 8] = np.array([0xFFFFFF00], np.uint32).view(np.uint8)
    assert _status_of(bad, L, x.size)[1] == capi.BP_ERR_CORRUPT
    # the first exception position byte of page 0 set beyond the block
    low = 4 * int(meta[:32, 0].astype(np.int64).sum())
    bad = gp.copy()
    bad[off_payload + 4 * low] = 200
    assert _status_of(bad, L, x.size)[1] == capi.BP_ERR_CORRUPT
    bad = gp.copy()
    bad[0] ^= 1
    assert _status_of(bad, L, x.size)[1] == capi.BP_ERR_CORRUPT
    assert _status_of(gp[:-16], L, x.size)[1] == capi.BP_ERR_CORRUPT
    assert _status_of(gp, L, x.size - 1)[1] == capi.BP_ERR_CORRUPT


def test_decode_is_deterministic_across_streams():
    x = W.clustered(300_000, 0, 1 << 28, 5)
    for layout in LAYOUTS:
        enc = api.to_device(capi.bp_encode(x, layout))
        s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
        a = api.decode(enc, layout, x.size, stream=s1)
        b = api.decode(enc, layout, x.size, stream=s2)
        torch.cuda.synchronize()
        assert torch.equal(a, b)
