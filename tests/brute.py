"""Brute-force restatements of the formats, one bit at a time, for tiny inputs.

These build the expected byte strings directly from the prose definitions
(Python integers used as bit strings), with none of the word-level logic of
Algorithm 1.  They exist to pin the oracle to something other than itself.
"""
from __future__ import annotations


def bitstring_put(acc: int, pos: int, value: int, b: int) -> int:
    for k in range(b):
        if (value >> k) & 1:
            acc |= 1 << (pos + k)
    return acc


def bits_of(v: int) -> int:
    return v.bit_length()  # smallest b with v < 2**b


def s4_block_words(deltas, b: int):
    """Fig. 2: integer n -> lane n % 4, slot n // 4; each lane is an LSB-first
    b-bit stream; lane word k is block word 4k + lane."""
    lanes = [0, 0, 0, 0]
    for n, v in enumerate(deltas):
        lanes[n % 4] = bitstring_put(lanes[n % 4], b * (n // 4), v, b)
    words = [0] * (4 * b)
    for k in range(b):
        for s in range(4):
            words[4 * k + s] = (lanes[s] >> (32 * k)) & 0xFFFFFFFF
    return words


def gl_block_words(deltas, b: int):
    """GL: delta of in-block position 4t+s at bit b*(32s+t)."""
    acc = 0
    for t in range(32):
        for s in range(4):
            acc = bitstring_put(acc, b * (32 * s + t), deltas[4 * t + s], b)
    return [(acc >> (32 * k)) & 0xFFFFFFFF for k in range(4 * b)]


def le32(words) -> bytes:
    return b"".join(int(w).to_bytes(4, "little") for w in words)


def varint(values) -> bytes:
    out = bytearray()
    for v in values:
        while True:
            if v < 128:
                out.append(v | 128)
                break
            out.append(v & 127)
            v >>= 7
    return bytes(out)


# kinds of differential coding (Section 5) as stored in stream headers
D4, DM, D2, D1 = 0, 1, 2, 3


def reference(kind: int, x, i: int, seed: int) -> int:
    """The earlier value that x[i] is coded against (Section 5): D4 x[i-4],
    DM the last value of the previous 4-vector, D2 x[i-2], D1 x[i-1];
    positions before the list hold `seed`."""
    j = {D4: i - 4, DM: 4 * (i // 4) - 1, D2: i - 2, D1: i - 1}[kind]
    return x[j] if j >= 0 else seed


def deltas(kind: int, x, seed: int = 0):
    return [(x[i] - reference(kind, x, i, seed)) % 2**32 for i in range(len(x))]


def pl_stream(x, kind: int = D4) -> bytes:
    """The S4-BP128 paper layout of Section 4.3 with our header/tail
    reading, built from the prose: deltas of the given kind against a zero
    seed, meta-blocks of 16 widths + 16 blocks, leftover blocks with a width
    byte each, varint of D1 gaps for the last n mod 128 integers; header
    {n, 0, tail bytes, kind}."""
    x = [int(v) for v in x]
    n = len(x)
    nb = n // 128
    np_ = 128 * nb
    d = deltas(kind, x[:np_])
    widths = [bits_of(max(d[128 * k:128 * k + 128])) for k in range(nb)]
    body = bytearray()
    for m in range(nb // 16):
        ks = range(16 * m, 16 * m + 16)
        body += bytes(widths[k] for k in ks)
        for k in ks:
            body += le32(s4_block_words(d[128 * k:128 * k + 128], widths[k]))
    for k in range(16 * (nb // 16), nb):
        body.append(widths[k])
        body += le32(s4_block_words(d[128 * k:128 * k + 128], widths[k]))
    prev = x[np_ - 1] if np_ else 0
    gaps = []
    for v in x[np_:]:
        gaps.append((v - prev) % 2**32)
        prev = v
    tail = varint(gaps)
    hdr = le32([n, 0, len(tail), kind])
    return hdr + bytes(body) + tail


def gl_stream(x, kind: int = D4) -> bytes:
    """GL layout (ours): see the oracle header for the field list."""
    x = [int(v) for v in x]
    n = len(x)
    nb = (n + 127) // 128
    ns = (nb + 31) // 32

    def up16(v):
        return (v + 15) // 16 * 16

    off_first = 64
    off_sbo = off_first + up16(4 * nb)
    off_bw = off_sbo + up16(4 * (ns + 1))
    off_payload = off_bw + up16(nb)
    first, widths, payload, sbo = [], [], [], []
    for k in range(nb):
        blk = x[128 * k:128 * k + 128]
        F = blk[0]
        full = list(blk)
        for i in range(len(blk), 128):  # padding: every missing delta is zero
            full.append(reference(kind, full, i, F))
        d = deltas(kind, full, F)
        b = bits_of(max(d))
        if k % 32 == 0:
            sbo.append(len(payload))
        first.append(F)
        widths.append(b)
        payload += gl_block_words(d, b)
    sbo.append(len(payload))
    total = off_payload + 4 * len(payload)
    out = bytearray(total)
    hdr = [0x344C4742, 1, n, nb, ns, len(payload), off_first, off_sbo, off_bw,
           off_payload, total & 0xFFFFFFFF, total >> 32, kind, 0, 0, 0]
    out[0:64] = le32(hdr)
    out[off_first:off_first + 4 * nb] = le32(first)
    out[off_sbo:off_sbo + 4 * (ns + 1)] = le32(sbo)
    out[off_bw:off_bw + nb] = bytes(widths)
    out[off_payload:] = le32(payload)
    return bytes(out)


def pfor_widths(d):
    """Section 4.4 by exhaustive search: b, and the b' of [0, b] with the
    lowest 128 b' + c(b') (b - b' + 8), the largest on a tie; c(b') counts
    the deltas that need more than b' bits."""
    b = bits_of(max(d))
    best = None
    for bp in range(b + 1):
        c = sum(1 for v in d if bits_of(v) > bp)
        cost = 128 * bp + c * (b - bp + 8)
        if best is None or cost <= best[0]:
            best = (cost, bp, c)
    return b, best[1], best[2]


def gp_stream(x, kind: int = D4) -> bytes:
    """GP layout (S4-FastPFOR, ours): see the oracle header for the fields."""
    x = [int(v) for v in x]
    n = len(x)
    nb = (n + 127) // 128
    npg = (nb + 31) // 32

    def up16(v):
        return (v + 15) // 16 * 16

    off_first = 64
    off_spo = off_first + up16(4 * nb)
    off_meta = off_spo + up16(4 * (npg + 1))
    off_payload = off_meta + up16(4 * nb)
    first, meta, payload, spo = [], [], [], []
    for p in range(npg):
        spo.append(len(payload))
        positions, highs = [], []
        for k in range(32 * p, min(nb, 32 * p + 32)):
            blk = x[128 * k:128 * k + 128]
            F = blk[0]
            full = list(blk)
            for i in range(len(blk), 128):
                full.append(reference(kind, full, i, F))
            d = deltas(kind, full, F)
            b, bp, c = pfor_widths(d)
            first.append(F)
            meta += [bp, b - bp, c, 0]
            payload += gl_block_words([v % 2**bp for v in d], bp)
            for i, v in enumerate(d):
                if bits_of(v) > bp:
                    positions.append(i)
                    highs.append((v >> bp, b - bp))
        pos_bytes = bytes(positions) + bytes(-len(positions) % 4)
        payload += [int.from_bytes(pos_bytes[i:i + 4], "little")
                    for i in range(0, len(pos_bytes), 4)]
        acc, pos = 0, 0
        for v, w in highs:
            acc = bitstring_put(acc, pos, v, w)
            pos += w
        payload += [(acc >> (32 * k)) & 0xFFFFFFFF for k in range((pos + 31) // 32)]
        payload += [0] * (-len(payload) % 4)
    spo.append(len(payload))
    total = off_payload + 4 * len(payload)
    out = bytearray(total)
    hdr = [0x34504742, 3, n, nb, npg, len(payload), off_first, off_spo, off_meta,
           off_payload, total & 0xFFFFFFFF, total >> 32, kind, 0, 0, 0]
    out[0:64] = le32(hdr)
    out[off_first:off_first + 4 * nb] = le32(first)
    out[off_spo:off_spo + 4 * (npg + 1)] = le32(spo)
    out[off_meta:off_meta + 4 * nb] = bytes(meta)
    out[off_payload:] = le32(payload)
    return bytes(out)
