"""Pins of the scalar oracle to things other than itself: the paper's worked
examples (Figs. 1b, 1c, 2, 4), closed forms, invariants, bit-at-a-time brute
force on tiny inputs and Python set intersection.  CPU only."""
import itertools

import numpy as np
import pytest

import brute
from conftest import read_golden
from oracle.oracle import ORC_ECORRUPT, OracleError

M32 = 0xFFFFFFFF


def _sorted_distinct(rng, n, U):
    return np.sort(rng.choice(U, n, replace=False)).astype(np.uint32)


# ---- worked examples printed in the paper ---------------------------------

def test_fig1b_varint_bytes(orc):
    g = read_golden("fig1b_varint.txt")
    vals = [int(v) for v in g["values"]]
    want = bytes(int(b, 16) for b in g["bytes"])
    assert orc.varint_encode(vals) == want
    got, used = orc.varint_decode(want, len(vals))
    assert got.tolist() == vals and used == len(want)


def test_fig1c_packed_bytes(orc):
    g = read_golden("fig1c_packed.txt")
    vals = [int(v) for v in g["values"]]
    b = int(g["bits"][0])
    want = bytes(int(x, 16) for x in g["bytes"])
    assert orc.pack_scalar(vals, b) == want
    assert orc.unpack_scalar(want, len(vals), b).tolist() == vals
    # the largest value needs exactly 18 bits (Section 4.2)
    assert orc.max_bits(vals) == b


def test_fig2_interleave_b18(orc):
    """Fig. 2 / Section 4.2: x1..x4 fill the first 18 bits of four
    consecutive words, the first 14 bits of x5..x8 the next 14 bits, and
    their remaining 4 bits start the next four words, followed by x9.., x13.."""
    rng = np.random.default_rng(18)
    x = rng.integers(0, 1 << 18, 128, dtype=np.uint32)
    y = orc.s4_pack128(x, 18).astype(np.uint64)
    X = [None] + [int(v) for v in x]  # 1-based as in the figure
    for s in range(4):
        assert int(y[s]) == (X[1 + s] | (X[5 + s] << 18)) & M32
        assert int(y[4 + s]) == ((X[5 + s] >> 14) | (X[9 + s] << 4)
                                 | (X[13 + s] << 22)) & M32
    out, _ = orc.s4_unpack128(y.astype(np.uint32), 18, d4=False)
    assert np.array_equal(out, x)


def test_fig4_v1_example(orc):
    g = read_golden("fig4_v1.txt")
    r = [int(v) for v in g["r"]]
    f = [int(v) for v in g["f"]]
    T = int(g["T"][0])
    assert orc.intersect_v1(r, f, T).tolist() == [int(v) for v in g["expect"]]


# ---- bit widths -----------------------------------------------------------

def test_bit_width_definition(orc):
    """Section 4.3: b is the smallest value with all integers < 2^b."""
    edge = [0, 1, 2, 3, 4, 7, 8, M32, 1 << 31, (1 << 31) - 1]
    edge += [(1 << k) - 1 for k in range(1, 33)] + [1 << k for k in range(32)]
    for v in edge:
        b = orc.bits(v)
        assert b == int(v).bit_length()
        assert v < 2 ** b and (b == 0 or v >= 2 ** (b - 1))


# ---- Algorithm 1 ------------------------------------------------------------

@pytest.mark.parametrize("b", list(range(0, 33)))
def test_alg1_roundtrip_every_width(orc, b):
    rng = np.random.default_rng(100 + b)
    hi = 1 << b
    x = rng.integers(0, hi, 128, dtype=np.uint64).astype(np.uint32) if b else \
        np.zeros(128, np.uint32)
    if b:
        x[rng.integers(0, 128)] = hi - 1  # make sure the width is used
    words = orc.s4_pack128(x, b)
    assert words.tolist() == brute.s4_block_words(x.tolist(), b)
    plain, _ = orc.s4_unpack128(words, b, d4=False)
    assert np.array_equal(plain, x)
    seed = rng.integers(0, 1 << 32, 4, dtype=np.uint64).astype(np.uint32)
    got, v = orc.s4_unpack128(words, b, d4=True, seed=seed)
    want = np.zeros(128, np.uint64)
    for n in range(128):
        prev = int(seed[n]) if n < 4 else int(want[n - 4])
        want[n] = (prev + int(x[n])) & M32
    assert np.array_equal(got, want.astype(np.uint32))
    assert v.tolist() == want[-4:].astype(np.uint32).tolist()


# ---- D4 differential coding (Section 5) -----------------------------------

@pytest.mark.parametrize("c", [1, 3, 1000, 77777])
def test_d4_arithmetic_progression_closed_form(orc, c):
    """x_i = c*i (i = 1..n) has D4 deltas (c, 2c, 3c, 4c, 4c, 4c, ...)."""
    n = 1000
    x = (c * np.arange(1, n + 1, dtype=np.uint64)).astype(np.uint32)
    d = orc.d4_deltas(x)
    want = [c, 2 * c, 3 * c] + [4 * c] * (n - 3)
    assert d.tolist() == [w & M32 for w in want]
    assert np.array_equal(orc.d4_prefix(d), x)


def test_pl_arithmetic_progression_widths_and_size(orc):
    """For x_i = c*i every block has width bits(4c) and the stream size is
    16 + 16*meta + leftover + sum(16 b) + tail bytes."""
    c, n = 5, 128 * 37 + 9
    x = (c * np.arange(1, n + 1, dtype=np.uint64)).astype(np.uint32)
    data = orc.pl_encode(x)
    nb = n // 128
    b = (4 * c).bit_length()
    tail = brute.varint([c] * (n - 128 * nb))
    assert len(data) == 16 + 16 * (nb // 16) + nb % 16 + nb * 16 * b + len(tail)
    assert data.endswith(tail)
    assert data[16:32] == bytes([b] * 16)


# ---- DM, D2, D1 (Section 5) ---------------------------------------------------

KINDS = [0, 1, 2, 3]  # D4, DM, D2, D1 as stored in stream headers


@pytest.mark.parametrize("c", [1, 3, 77777])
def test_variant_arithmetic_progression_closed_forms(orc, c):
    """x_i = c*i (i = 1..n): D1 deltas are all c; D2 (c, 2c, 2c, ...); DM
    (c, 2c, 3c, 4c) repeated (every 4-vector minus the last value of the
    previous one); D4 (c, 2c, 3c, 4c, 4c, ...)."""
    n = 1000
    x = (c * np.arange(1, n + 1, dtype=np.uint64)).astype(np.uint32)
    want = {
        orc.D1: [c] * n,
        orc.D2: [c] + [2 * c] * (n - 1),
        orc.DM: [c, 2 * c, 3 * c, 4 * c] * (n // 4),
        orc.D4: [c, 2 * c, 3 * c] + [4 * c] * (n - 3),
    }
    for kind, w in want.items():
        d = orc.deltas(kind, x)
        assert d.tolist() == [v & M32 for v in w], kind
        assert np.array_equal(orc.prefix(kind, d), x), kind


def test_variant_mean_delta_ratios(orc):
    """Section 5 expects deltas 4x (D4), 2.5x (DM) and 2x (D2) larger than
    D1's on average: exactly so in expectation for independent gaps."""
    rng = np.random.default_rng(11)
    gaps = rng.integers(1, 64, 400_000, dtype=np.uint64)
    x = np.cumsum(gaps).astype(np.uint32)
    m1 = orc.deltas(orc.D1, x)[4:].astype(np.float64).mean()
    for kind, ratio in ((orc.D4, 4.0), (orc.DM, 2.5), (orc.D2, 2.0)):
        m = orc.deltas(kind, x)[4:].astype(np.float64).mean()
        assert abs(m / m1 - ratio) < 0.02 * ratio, (kind, m / m1)


@pytest.mark.parametrize("kind", [1, 2, 3])
def test_variant_integrated_unpack(orc, kind):
    """Algorithm 1 with the vector prefix steps of Section 5 (DM: add the
    last value of the previous vector; D2: shift by two and add, then add
    (v2, v3, v2, v3); D1: the D2 steps, a shift by one and add, then the last
    value) equals the prefix of the definition, from any seed vector."""
    rng = np.random.default_rng(100 + kind)
    for b in (0, 1, 7, 18, 31, 32):
        for _ in range(4):
            d = [int(v) for v in rng.integers(0, 1 << b, 128, dtype=np.uint64)] if b else [0] * 128
            prev = [int(v) for v in rng.integers(0, 1 << 32, 4, dtype=np.uint64)]
            words = brute.s4_block_words(d, b)
            got, last = orc.s4_unpack128(words, b, kind=kind + 1, seed=prev)
            x = list(prev)
            for p in range(128):  # the definition, on prev followed by the block
                x.append((d[p] + brute.reference(kind, x, 4 + p, 0)) % 2**32)
            assert got.tolist() == x[4:], (kind, b)
            assert last.tolist() == x[-4:], (kind, b)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("n", [0, 1, 129, 2047, 2048 + 128 + 5, 2 * 2048 + 15 * 128 + 127])
def test_variant_streams_match_bitwise_construction(orc, kind, n):
    rng = np.random.default_rng(50 * kind + n)
    x = _sorted_distinct(rng, n, 1 << 28)
    pl = orc.pl_encode(x, kind)
    gl = orc.gl_encode(x, kind)
    assert pl == brute.pl_stream(x, kind)
    assert gl == brute.gl_stream(x, kind)
    assert np.array_equal(orc.pl_decode(pl), x)
    assert np.array_equal(orc.gl_decode(gl), x)


def test_variant_sizes_order(orc):
    """Smaller deltas, fewer bits: on the same list D1 <= D2 <= DM <= D4."""
    rng = np.random.default_rng(3)
    x = np.sort(rng.choice(1 << 26, 200_000, replace=False)).astype(np.uint32)
    sizes = [len(orc.pl_encode(x, k)) for k in (orc.D1, orc.D2, orc.DM, orc.D4)]
    assert sizes == sorted(sizes)


# ---- S4-FastPFOR (Section 4.4) ------------------------------------------------

def test_fig3_fastpfor_block(orc):
    g = read_golden("fig3_fastpfor.txt")
    d = [int(v) for v in g["prefix"]] + [i % 4 for i in range(5, 128)]
    b, bp, c = orc.pfor_choose(d)
    assert (b, bp, c) == (int(g["b"][0]), int(g["b_prime"][0]), int(g["exceptions"][0]))
    assert brute.pfor_widths(d) == (b, bp, c)
    exc = [i for i, v in enumerate(d) if v >> bp]
    assert exc == [int(g["position"][0])]
    assert d[exc[0]] >> bp == int(g["high"][0])
    assert (int(g["high"][0]) << bp) | (d[exc[0]] & ((1 << bp) - 1)) == d[exc[0]]


def test_pfor_choose_against_exhaustive_search(orc):
    rng = np.random.default_rng(44)
    for trial in range(300):
        kind = trial % 3
        if kind == 0:    # small values with a few large outliers
            d = rng.geometric(0.3, 128).astype(np.uint64)
            d[rng.choice(128, rng.integers(0, 12), replace=False)] = rng.integers(
                1 << 10, 1 << 32, 1)
        elif kind == 1:  # one width everywhere
            d = rng.integers(0, 1 << int(rng.integers(0, 33)), 128, dtype=np.uint64)
        else:            # ties are likely: values 0/1 and one large value
            d = rng.integers(0, 2, 128).astype(np.uint64)
            d[int(rng.integers(0, 128))] = 1 << int(rng.integers(1, 32))
        d = (d & 0xFFFFFFFF).astype(np.uint32)
        assert orc.pfor_choose(d) == brute.pfor_widths(d.tolist()), d.tolist()


@pytest.mark.parametrize("kind", [0, 1, 2, 3])
@pytest.mark.parametrize("n", [0, 1, 5, 127, 128, 129, 4096, 4097, 2 * 4096 + 15 * 128 + 3])
def test_gp_stream_matches_bitwise_construction(orc, kind, n):
    """GP streams byte for byte against the bit-at-a-time construction, on
    lists with outliers (clustered runs with large jumps) so that blocks have
    exceptions of several widths."""
    rng = np.random.default_rng(700 + 10 * n + kind)
    gaps = rng.geometric(0.2, n).astype(np.uint64)
    jumps = rng.random(n) < 0.03
    gaps[jumps] = rng.integers(1 << 8, 1 << 20, int(jumps.sum()))
    x = np.cumsum(gaps).astype(np.uint32)
    data = orc.gp_encode(x, kind)
    assert data == brute.gp_stream(x, kind)
    assert np.array_equal(orc.gp_decode(data), x)
    if n >= 128 and kind == 0:
        meta = np.frombuffer(data, np.uint8)
        hdr = meta[:64].view(np.uint32)
        c = meta[int(hdr[8]) + 2:int(hdr[8]) + 4 * int(hdr[3]):4]
        assert c.sum() > 0  # the outliers became exceptions


def test_gp_roundtrip_every_width(orc):
    """Lists whose deltas reach every width 0..32, in the GP layout; patching
    never makes a list longer than GL (b' = b is always a candidate)."""
    rng = np.random.default_rng(45)
    for b in range(0, 33):
        n = 3000
        top = (1 << 32) - 1
        step = max(1, min(top // n, (1 << b) // 4 if b >= 2 else 1))
        x = np.unique(np.cumsum(rng.integers(1, step + 1, n, dtype=np.uint64)) & top)
        x = x.astype(np.uint32)
        for kind in range(4):
            gp = orc.gp_encode(x, kind)
            assert np.array_equal(orc.gp_decode(gp), x)
            gl = orc.gl_encode(x, kind)
            # per block: 4 B of meta vs 1 B width; payload never larger
            assert len(gp) <= len(gl) + 3 * ((x.size + 127) // 128) + 16 * (x.size // 4096 + 2)


# ---- containers -------------------------------------------------------------

EDGE_N = [0, 1, 2, 3, 4, 5, 127, 128, 129, 255, 256, 257, 2047, 2048, 2049,
          2048 + 128 + 5, 2 * 2048 + 15 * 128 + 127]


@pytest.mark.parametrize("n", EDGE_N)
def test_pl_stream_matches_bitwise_construction(orc, n):
    rng = np.random.default_rng(n)
    x = _sorted_distinct(rng, n, 1 << 24)
    data = orc.pl_encode(x)
    assert data == brute.pl_stream(x)
    assert np.array_equal(orc.pl_decode(data), x)


@pytest.mark.parametrize("n", EDGE_N)
def test_gl_stream_matches_bitwise_construction(orc, n):
    rng = np.random.default_rng(1000 + n)
    x = _sorted_distinct(rng, n, 1 << 30)
    data = orc.gl_encode(x)
    assert data == brute.gl_stream(x)
    assert np.array_equal(orc.gl_decode(data), x)


def test_pl_widths_are_ceil_log2_of_max_delta(orc):
    rng = np.random.default_rng(7)
    n = 2048 * 3 + 128 * 5 + 17
    x = np.sort(rng.choice(1 << 27, n, replace=False)).astype(np.uint32)
    data = orc.pl_encode(x)
    xs = [int(v) for v in x]
    d = [(xs[i] - (xs[i - 4] if i >= 4 else 0)) % 2**32 for i in range(n)]
    nb = n // 128
    pos, widths = 16, []
    for m in range(nb // 16):
        ws = list(data[pos:pos + 16])
        widths += ws
        pos += 16 + 16 * sum(ws)
    for _ in range(nb % 16):
        widths.append(data[pos])
        pos += 1 + 16 * data[pos]
    for k, w in enumerate(widths):
        mx = max(d[128 * k:128 * k + 128])
        assert w == int(np.ceil(np.log2(mx + 1))) == mx.bit_length()
    tail_bytes = int.from_bytes(data[8:12], "little")
    assert pos + tail_bytes == len(data)
    # size = header + width bytes + sum over blocks of 4b words + tail
    assert len(data) == 16 + nb + sum(16 * w for w in widths) + tail_bytes


@pytest.mark.parametrize("n", [0, 1, 5, 128, 3000, 4097, 100_000])
def test_pl_gl_roundtrip_and_agreement(orc, n):
    rng = np.random.default_rng(n + 5)
    for U in (n + 1, 4 * n + 8, 1 << 32):
        x = np.sort(rng.choice(U, n, replace=False)).astype(np.uint32)
        a = orc.pl_decode(orc.pl_encode(x))
        b = orc.gl_decode(orc.gl_encode(x))
        assert np.array_equal(a, x) and np.array_equal(b, x)


def test_gl_info_fields(orc):
    x = np.arange(0, 3 * 40 * 128 + 3, 3, dtype=np.uint32)
    data = orc.gl_encode(x)
    info = orc.gl_info(data)
    assert info["n"] == x.size
    assert info["nblocks"] == (x.size + 127) // 128
    assert info["nsuper"] == (info["nblocks"] + 31) // 32
    assert info["off_payload"] % 16 == 0
    assert len(data) == info["off_payload"] + 4 * info["payload_words"]
    first = np.frombuffer(data, np.uint32, info["nblocks"], info["off_first"])
    assert np.array_equal(first, x[::128])


def test_encode_rejects_unsorted(orc):
    with pytest.raises(OracleError):
        orc.pl_encode([3, 2])
    with pytest.raises(OracleError):
        orc.gl_encode([5, 5])


def test_corrupt_streams_are_rejected(orc):
    x = np.arange(10, 10 + 7 * 4000, 7, dtype=np.uint32)
    pl = bytearray(orc.pl_encode(x))
    bad = bytearray(pl)
    bad[16] = 33  # width byte beyond 32
    with pytest.raises(OracleError) as e:
        orc.pl_decode(bytes(bad))
    assert e.value.code == ORC_ECORRUPT
    with pytest.raises(OracleError):
        orc.pl_decode(bytes(pl[:-3]))
    gl = bytearray(orc.gl_encode(x))
    info = orc.gl_info(bytes(gl))
    bad = bytearray(gl)
    bad[info["off_bw"]] = 40
    with pytest.raises(OracleError):
        orc.gl_decode(bytes(bad))
    with pytest.raises(OracleError):
        orc.varint_decode(bytes([0, 0, 0, 0, 0, 0x81]), 1)  # overlong


# ---- intersections (Section 6) --------------------------------------------

ALGOS = ["intersect", "intersect_gallop", "intersect_hybrid"]
TALGOS = [("intersect_v1", 8), ("intersect_v1", 4), ("intersect_v3", 32),
          ("intersect_v3", 2), ("intersect_simd_gallop", 32),
          ("intersect_simd_gallop", 4)]


def _all_algos(orc, r, f):
    outs = [getattr(orc, a)(r, f) for a in ALGOS]
    outs += [getattr(orc, a)(r, f, T) for a, T in TALGOS]
    return outs


def test_intersections_all_subsets_tiny_universe(orc):
    U = 6
    subsets = [np.array(c, np.uint32) for k in range(U + 1)
               for c in itertools.combinations(range(U), k)]
    for a in subsets:
        for b in subsets:
            want = sorted(set(a.tolist()) & set(b.tolist()))
            r, f = (a, b) if a.size <= b.size else (b, a)
            for got in _all_algos(orc, r, f):
                assert got.tolist() == want


@pytest.mark.parametrize("m,n", [(0, 0), (0, 50), (1, 1), (1, 1000), (37, 37),
                                 (100, 5000), (300, 300_000), (2000, 2100),
                                 (5, 200_000)])
def test_intersections_random(orc, m, n):
    rng = np.random.default_rng(m * 7 + n)
    U = max(4 * n, 64)
    f = _sorted_distinct(rng, n, U)
    k = min(m // 3, n)
    r = np.union1d(rng.choice(f, k, replace=False) if k else [],
                   _sorted_distinct(rng, m - k, U)).astype(np.uint32)[:m]
    want = sorted(set(r.tolist()) & set(f.tolist()))
    for got in _all_algos(orc, r, f):
        assert got.tolist() == want
    # edge cases: identical, disjoint, subset
    assert orc.intersect(f, f).tolist() == f.tolist()
    assert orc.intersect(f * 2 + 1, f * 2).size == 0 if n < 2**30 else True
    assert orc.intersect(f[::3], f).tolist() == f[::3].tolist()


def test_output_to_input_property(orc):
    """Section 6.2: the result may overwrite the shorter input."""
    rng = np.random.default_rng(3)
    f = _sorted_distinct(rng, 5000, 1 << 16)
    r = _sorted_distinct(rng, 800, 1 << 16)
    want = sorted(set(r.tolist()) & set(f.tolist()))
    assert orc.svs([r, f]).tolist() == want


def test_svs_against_python_sets(orc):
    rng = np.random.default_rng(11)
    for trial in range(30):
        k = int(rng.integers(1, 6))
        lists = [_sorted_distinct(rng, int(rng.integers(0, 3000)), 1 << 13)
                 for _ in range(k)]
        want = set(lists[0].tolist())
        for L in lists[1:]:
            want &= set(L.tolist())
        assert orc.svs(lists).tolist() == sorted(want)


def test_svs_gallop_against_python_sets(orc):
    """The galloping Set-vs-Set used on sets with very long lists: the same
    unique answer as Python's set intersection, including skewed sets (one
    list 1000x longer), empty lists and a single list."""
    rng = np.random.default_rng(12)
    for trial in range(40):
        k = int(rng.integers(1, 7))
        sizes = [int(rng.integers(0, 400)) for _ in range(k)]
        if trial % 3 == 0:
            sizes[int(rng.integers(0, k))] = 200_000
        lists = [_sorted_distinct(rng, s, 1 << 18) for s in sizes]
        want = set(lists[0].tolist())
        for L in lists[1:]:
            want &= set(L.tolist())
        assert orc.svs_gallop(lists).tolist() == sorted(want)
        assert orc.svs_gallop(lists).tolist() == orc.svs(lists).tolist()
    assert orc.svs_gallop([]).size == 0
