"""Mutation check of the oracle pins: each plausible mistake below is planted
in a copy of the oracle source (on the CPU, in a temporary directory), the
copy is compiled, and the pin suite must fail against it.  A mutant that
survives means a pin is missing."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "bp_oracle.c")

# (name, text in the source, replacement); each text must occur in the source
MUTANTS = [
    ("d4 index x[i-3]", "d[i] = x[i] - (i >= 4 ? x[i - 4] : 0u);",
     "d[i] = x[i] - (i >= 3 ? x[i - 3] : 0u);"),
    ("d4 prefix sign", "x[i] = d[i] + (i >= 4 ? x[i - 4] : 0u);",
     "x[i] = d[i] - (i >= 4 ? x[i - 4] : 0u);"),
    ("alg1 straddle shift", "(y[4 * (k + 1) + s] << (32 - i))",
     "(y[4 * (k + 1) + s] << (31 - i))"),
    ("alg1 offset update", "i = i + b - 32;", "i = i + b - 31;"),
    ("alg1 prefix uses last lane", "t[s] += v[s];", "t[s] += v[3];"),
    ("pack transposed word", "out[4 * k + s] |= v << o;",
     "out[4 * s + k] |= v << o;"),
    ("lane/slot swapped", "const unsigned s = n % 4, j = n / 4;",
     "const unsigned s = n / 32, j = n % 32;"),
    ("varint continuation bit", "out[k++] = (uint8_t)(v | 128u);",
     "out[k++] = (uint8_t)(v & 127u);"),
    ("bit width off by one", "while (b < 32 && (v >> b) != 0) b++;",
     "while (b < 32 && (v >> b) > 1) b++;"),
    ("meta-block of 8", "const size_t nb = n / 128, np = nb * 128, meta = nb / 16;\n"
     "  uint32_t *d", "const size_t nb = n / 128, np = nb * 128, meta = nb / 8;\n"
     "  uint32_t *d"),
    ("tail gaps not chained", "gaps[i] = x[np + i] - prev;\n    prev = x[np + i];",
     "gaps[i] = x[np + i] - prev;"),
    ("gl row-major bits", "put_bits(words, (size_t)b * (32 * s + t), d[4 * t + s], b);",
     "put_bits(words, (size_t)b * (4 * t + s), d[4 * t + s], b);"),
    ("gl seed zero", "d[i] = xx[i] - (i >= 4 ? xx[i - 4] : F);",
     "d[i] = xx[i] - (i >= 4 ? xx[i - 4] : 0u);"),
    ("merge skips on equal", "if (a[i] < b[j]) i++;", "if (a[i] <= b[j]) i++;"),
    ("gallop bsearch bound", "if (f[mid] < ri) L = mid + 1;",
     "if (f[mid] <= ri) L = mid + 1;"),
    ("v3 wrong quarter", "F = (f[j + T - 1] >= ri) ? f + j : f + j + T;",
     "F = (f[j + T - 1] >= ri) ? f + j : f + j + 2 * T;"),
    ("simd gallop skips bsearch", "j += lo * T;", "j += delta;"),
    ("dm against x[4t-2]", "case ORC_DELTA_DM: j = 4 * (long long)(i / 4) - 1; break;",
     "case ORC_DELTA_DM: j = 4 * (long long)(i / 4) - 2; break;"),
    ("d2 prefix takes v3 for lane 0", "t[0] = u[0] + v[2];", "t[0] = u[0] + v[3];"),
    ("d1 second shift by two", "const uint32_t w[4] = {u[0], u[0] + u[1], u[1] + u[2], u[2] + u[3]};",
     "const uint32_t w[4] = {u[0], u[1], u[0] + u[2], u[1] + u[3]};"),
    ("dm prefix adds lane-wise", "for (int s = 0; s < 4; s++) t[s] += last;",
     "for (int s = 0; s < 4; s++) t[s] += v[s];"),
    ("gl kind not in header", "                      (uint32_t)kind,\n", "                      0u,\n"),
    ("pl decode ignores kind", "const int pkind = prefix_kind(kind);", "const int pkind = ORC_P_D4;"),
    ("pfor cost without the position byte",
     "const uint64_t cost = 128ull * bp + (uint64_t)c * (b - bp + 8);",
     "const uint64_t cost = 128ull * bp + (uint64_t)c * (b - bp);"),
    ("pfor tie to the smaller width", "    if (128ull * bp + (uint64_t)c * (b - bp + 8) == best_cost) {",
     "    if (0) {"),
    ("pfor exception test off by one", "      if (orc_bits(d[i]) > bp) c++;\n    const uint64_t cost",
     "      if (orc_bits(d[i]) > bp + 1) c++;\n    const uint64_t cost"),
    ("pfor high bits not shifted", "high[ne] = d[i] >> bp;", "high[ne] = d[i];"),
    ("pfor patch before the low bits", "d[q] |= get_bits(payload + high_w, bit, w) << bp;",
     "d[q] |= get_bits(payload + high_w, bit, w);"),
    ("pfor positions not padded to a word", "    wpos += (ne + 3) / 4;", "    wpos += ne / 4;"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_mutant(tmp_path, name, old, new):
    src = open(SRC).read()
    assert old in src, f"mutation site for '{name}' no longer in the oracle"
    mutated = src.replace(old, new, 1)
    cfile = tmp_path / "bp_oracle.c"
    cfile.write_text(mutated)
    hdr = os.path.join(ROOT, "oracle", "bp_oracle.h")
    (tmp_path / "bp_oracle.h").write_text(open(hdr).read())
    lib = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-std=c11", "-O1", "-fPIC", "-shared", "-o",
                           str(lib), str(cfile)])
    env = dict(os.environ, BP_ORACLE_LIB=str(lib))
    res = subprocess.run(
        [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
         os.path.join(ROOT, "tests", "test_oracle_pins.py")],
        env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert res.returncode != 0, f"mutant '{name}' survived the pins"
