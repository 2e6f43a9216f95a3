"""Pins for the oracle's block codec (Sec. II: SZ-style error-bounded lossy compression,
restated as absolute-bound linear quantization, a 1-D Lorenzo predictor on the integer
codes, 16-bit symbols and canonical Huffman coding).

What pins it: the pointwise error bound |x - x'| <= eb evaluated in FP64, losslessness of
the entropy-coding layers (round trip, idempotence), an independent heap-based textbook
Huffman (optimal total cost is unique), the Kraft equality, the Fibonacci depth bound and
a structural parse of the documented byte layout."""
import heapq
import math
import struct

import numpy as np
import pytest

import oracle
from blockgen import KINDS, gen_block

B_LOG2 = [5, 8, 12]




def reconstruct(x, eb, dtype):
    """Elementwise reconstruction the codec must reproduce after its lossless layers:
    x' = fl(rint(fl(x r)) * 2eb) (complex64: rounded to float), or x itself (verbatim)."""
    xd = np.asarray(x, dtype=np.float64)
    two = 2.0 * eb
    r = 1.0 / two
    t = xd * r
    ok = np.abs(t) < 2.0 ** 29
    q = np.where(ok, np.rint(np.where(ok, t, 0.0)), 0.0)
    xr = q * two
    if dtype == oracle.C64:
        xr = xr.astype(np.float32).astype(np.float64)
    with np.errstate(invalid="ignore"):
        ok &= np.abs(xd - xr) <= eb
    return np.where(ok, xr, xd), ~ok


def as_real(v):
    return np.stack([v.real, v.imag], axis=-1).reshape(-1)


@pytest.mark.parametrize("dtype", [oracle.C128, oracle.C64])
@pytest.mark.parametrize("b", B_LOG2)
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("eb", [1e-4, 1e-6, 1e-8])
def test_pointwise_bound_and_roundtrip(dtype, b, kind, eb):
    rng = np.random.default_rng(hash((dtype, b, kind)) % 2**32)
    v = gen_block(kind, b, rng, dtype)
    stream, info = oracle.compress_block(v, b, dtype, eb)
    d = oracle.decompress_block(stream, b, dtype, eb)
    x = as_real(v).astype(np.float64)
    xd = as_real(d).astype(np.float64)
    # pointwise error bound, evaluated in FP64
    assert np.all(np.abs(x - xd) <= eb)
    # the entropy-coding layers are lossless
    ref, verb = reconstruct(as_real(v), eb, dtype)
    assert np.array_equal(xd, ref)
    assert info["n_verbatim"] == int(verb.sum())
    assert len(stream) % 16 == 0
    # compressing the reconstruction again gives the same stream (idempotence), where
    # the float grid is fine enough for the quantization grid (always for complex128)
    if dtype == oracle.C128 or np.abs(x).max() * 2.0 ** -23 < eb:
        stream2, _ = oracle.compress_block(d, b, dtype, eb)
        assert stream2 == stream


def test_zero_block_is_const_header_only():
    for dtype in (oracle.C64, oracle.C128):
        for b in B_LOG2:
            z = np.zeros(1 << b, dtype=np.complex128)
            s, info = oracle.compress_block(z, b, dtype, 1e-6)
            assert info["mode"] == oracle.MODE_CONST and len(s) == 16
            assert np.array_equal(oracle.decompress_block(s, b, dtype, 1e-6), z)


def test_modes_selected_by_rule():
    rng = np.random.default_rng(0)
    s, info = oracle.compress_block(gen_block("const", 8, rng, oracle.C128), 8, oracle.C128, 1e-6)
    assert info["mode"] == oracle.MODE_CONST
    # peaked (Gaussian) deltas with few distinct symbols: Huffman beats fixed width
    v = gen_block("normal", 12, rng, oracle.C128)
    s, info = oracle.compress_block(v, 12, oracle.C128, 1e-4)
    assert info["mode"] == oracle.MODE_HUFF and info["n_distinct"] <= 256
    # more than 256 distinct symbols: PACK
    s, info = oracle.compress_block(gen_block("wide", 12, rng, oracle.C128), 12, oracle.C128, 1e-6)
    assert info["n_distinct"] > 256 and info["mode"] == oracle.MODE_PACK


def test_escapes_roundtrip():
    rng = np.random.default_rng(1)
    v = gen_block("walsh", 8, rng, oracle.C128)
    s, info = oracle.compress_block(v, 8, oracle.C128, 1e-8)
    assert info["n_escape"] > 0
    d = oracle.decompress_block(s, 8, oracle.C128, 1e-8)
    assert np.all(np.abs(as_real(d) - as_real(v)) <= 1e-8)


def test_verbatim_values_exact():
    b = 6
    v = np.zeros(1 << b, dtype=np.complex128)
    v[3] = 1e6 + 0j            # |x r| >= 2^29: out of the quantizer's range
    v[7] = complex(np.inf, 1.0)
    v[9] = complex(0.5, np.nan)
    s, info = oracle.compress_block(v, b, oracle.C128, 1e-6)
    assert info["n_verbatim"] == 3
    d = oracle.decompress_block(s, b, oracle.C128, 1e-6)
    assert as_real(d).tobytes() == as_real(v).tobytes()


def textbook_huffman_cost(freqs):
    """Classic heap construction; its total cost sum(f * depth) is the optimum."""
    if len(freqs) == 1:
        return freqs[0]
    h = list(freqs)
    heapq.heapify(h)
    cost = 0
    while len(h) > 1:
        a = heapq.heappop(h)
        b = heapq.heappop(h)
        cost += a + b
        heapq.heappush(h, a + b)
    return cost


@pytest.mark.parametrize("seed", range(40))
def test_huffman_optimal_and_complete(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 600))
    f = rng.integers(1, [2, 10, 1000, 100000][seed % 4], size=n).astype(np.uint32)
    syms = rng.choice(65536, size=n, replace=False).astype(np.uint32)
    L = oracle.huffman_lengths(f, syms)
    assert int((f.astype(np.int64) * L).sum()) == textbook_huffman_cost([int(x) for x in f])
    # a full binary tree: Kraft sum exactly 1
    assert sum(2.0 ** -int(l) for l in L) == 1.0


def test_huffman_fibonacci_depth_bound():
    fib = [1, 1]
    while len(fib) < 19:
        fib.append(fib[-1] + fib[-2])
    L = oracle.huffman_lengths(np.array(fib, dtype=np.uint32))
    assert L.max() == len(fib) - 1  # the classic worst case: a chain
    # total weight 2B <= 8192 symbols per block: F(20) = 6765 <= 8192 < F(21), so <= 18
    assert sum(fib[:18]) <= 8192


def test_huffman_tie_break_leaf_first():
    # equal weights: leaf queue first; (1,1,2): merge leaves 1+1 -> 2; then leaf 2 first.
    L = oracle.huffman_lengths(np.array([1, 1, 2], dtype=np.uint32), np.array([5, 6, 7], dtype=np.uint32))
    assert list(L) == [2, 2, 1]
    L = oracle.huffman_lengths(np.array([2, 2, 2, 2], dtype=np.uint32))
    assert list(L) == [2, 2, 2, 2]


def parse_stream(s, b, dtype, chunk=32):
    mode, dt, bl, param, nverb, D = struct.unpack_from("<BBBBHH", s, 0)
    assert dt == dtype and bl == b
    out = dict(mode=mode, param=param, nverb=nverb, D=D)
    if mode == oracle.MODE_HUFF:
        pbits, total = struct.unpack_from("<II", s, 8)
        assert total == len(s)
        off = 16
        counts = struct.unpack_from("<%dH" % param, s, off)
        off += (2 * param + 3) // 4 * 4
        syms = struct.unpack_from("<%dH" % D, s, off)
        off += (2 * D + 3) // 4 * 4
        C = (2 << b) // chunk
        chunks = struct.unpack_from("<%dH" % C, s, off)
        off += (2 * C + 3) // 4 * 4
        assert sum(chunks) == pbits
        out.update(counts=counts, syms=syms, pbits=pbits, chunks=chunks, payload_off=off)
    return out


def test_canonical_code_structure():
    rng = np.random.default_rng(5)
    for kind in ["normal", "qft", "walsh"]:
        v = gen_block(kind, 12, rng, oracle.C128)
        s, info = oracle.compress_block(v, 12, oracle.C128, 1e-6)
        p = parse_stream(s, 12, oracle.C128)
        if p["mode"] != oracle.MODE_HUFF:
            continue
        counts, syms = p["counts"], p["syms"]
        assert sum(counts) == p["D"] == info["n_distinct"]
        # symbols ascending within each length (canonical order)
        i = 0
        codes = []
        code = 0
        prev = None
        for L, c in enumerate(counts, start=1):
            assert list(syms[i:i + c]) == sorted(syms[i:i + c])
            for _ in range(c):
                if prev is not None:
                    code = (code + 1) << (L - prev)
                codes.append((code, L))
                prev = L
            i += c
        # prefix-free, and a complete code when D >= 2
        for a in range(len(codes)):
            for bb in range(len(codes)):
                if a != bb and codes[a][1] <= codes[bb][1]:
                    assert codes[bb][0] >> (codes[bb][1] - codes[a][1]) != codes[a][0]
        if len(codes) >= 2:
            assert sum(2.0 ** -L for _, L in codes) == 1.0


def test_const_header_fields():
    # eb = 2^-11: 2eb = 2^-10 and r = 2^10 exactly, so the codes are exact integers
    eb = 2.0 ** -11
    v = np.full(1 << 8, 0.125 - 0.25j)
    s, _ = oracle.compress_block(v, 8, oracle.C128, eb)
    mode, dt, bl, param, nverb, D, qre, qim = struct.unpack("<BBBBHHii", s)
    assert (mode, dt, bl, nverb) == (oracle.MODE_CONST, oracle.C128, 8, 0)
    assert (qre, qim) == (128, -256)


def test_round_half_even_ties():
    eb = 2.0 ** -11
    two = 2.0 ** -10
    v = np.array([2.5 * two + 3.5j * two, -2.5 * two - 0.5j * two] * 16)
    s, info = oracle.compress_block(v, 5, oracle.C128, eb)
    d = oracle.decompress_block(s, 5, oracle.C128, eb)
    # ties go to the even code, and |x - x'| == eb exactly is within the bound
    assert info["n_verbatim"] == 0
    assert d[0] == 2 * two + 4j * two and d[1] == -2 * two - 0j


@pytest.mark.parametrize("chunk", [16, 32, 64])
@pytest.mark.parametrize("kind,eb", [("qft", 1e-4), ("walsh", 1e-6), ("normal", 1e-4), ("grover", 1e-6)])
def test_chunk_table_matches_an_independent_decode(chunk, kind, eb):
    # the Huffman chunk size only changes the table of per-chunk bit counts: decode the payload
    # bit by bit with the canonical code (written here from the stored counts and symbols) and
    # check every stored count is the bits its `chunk` symbols take (32 more per escape), and
    # the reconstruction is the same for every chunk size
    b = 10
    rng = np.random.default_rng(11)
    v = gen_block(kind, b, rng, oracle.C128)
    v[::97] += 0.5  # a few large jumps: escapes
    s, info = oracle.compress_block(v, b, oracle.C128, eb, chunk=chunk)
    p = parse_stream(s, b, oracle.C128, chunk=chunk)
    assert p["mode"] == oracle.MODE_HUFF
    code_of = {}
    code, prev, i = 0, None, 0
    for L, c in enumerate(p["counts"], start=1):
        for _ in range(c):
            if prev is not None:
                code = (code + 1) << (L - prev)
            code_of[(code, L)] = p["syms"][i]
            prev = L
            i += 1
    words = struct.unpack_from("<%dI" % ((p["pbits"] + 31) // 32), s, p["payload_off"])
    bits = "".join(format(w, "032b") for w in words)
    pos = 0
    deltas = []
    for ci, stored in enumerate(p["chunks"]):
        start = pos
        for _ in range(chunk):
            L = 1
            while (int(bits[pos:pos + L], 2), L) not in code_of:
                L += 1
                assert L <= 24
            sym = code_of[(int(bits[pos:pos + L], 2), L)]
            pos += L
            if sym == 0:  # escape: the 32-bit delta follows
                d = int(bits[pos:pos + 32], 2)
                deltas.append(d - (1 << 32) if d >= 1 << 31 else d)
                pos += 32
            else:
                deltas.append(sym - 32768)
        assert pos - start == stored, ci
    assert pos == p["pbits"]
    # the values from the decoded deltas by the format's own rule: Lorenzo per plane
    # (q_j = q_{j-2} + delta_j over interleaved re/im, q_{-2} = q_{-1} = 0), x' = q * fl(2 eb)
    assert p["nverb"] == 0 and len(deltas) == 2 << b
    q = np.zeros(2 << b, dtype=np.int64)
    for j, d in enumerate(deltas):
        q[j] = (q[j - 2] if j >= 2 else 0) + d
    xr = q.astype(np.float64) * (2 * eb)
    mine = oracle.decompress_block(s, b, oracle.C128, eb, chunk=chunk)
    assert np.array_equal(xr[0::2], mine.real) and np.array_equal(xr[1::2], mine.imag)
    base = oracle.decompress_block(oracle.compress_block(v, b, oracle.C128, eb)[0], b, oracle.C128, eb)
    got = oracle.decompress_block(s, b, oracle.C128, eb, chunk=chunk)
    assert got.tobytes() == base.tobytes()


@pytest.mark.parametrize("dtype", [oracle.C128, oracle.C64])
def test_pack_mode_matches_an_independent_decode(dtype):
    # PACK: every delta as a zigzag code (0, -1, 1, -2, 2, ... -> 0, 1, 2, 3, 4, ...) of
    # `width` bits, MSB-first in little-endian u32 words; values by the per-plane Lorenzo rule
    b = 8
    eb = 1e-8 if dtype == oracle.C128 else 1e-5  # complex64: float rounding stays inside eb
    rng = np.random.default_rng(23)
    v = gen_block("wide", b, rng, dtype)
    s, info = oracle.compress_block(v, b, dtype, eb)
    mode, dt, bl, width, nverb, D = struct.unpack_from("<BBBBHH", s, 0)
    assert mode == oracle.MODE_PACK and nverb == 0
    pbits, total = struct.unpack_from("<II", s, 8)
    nv = 2 << b
    assert pbits == nv * width and total == len(s) and 1 <= width <= 32
    words = struct.unpack_from("<%dI" % ((pbits + 31) // 32), s, 16)
    bits = "".join(format(w, "032b") for w in words)
    q = np.zeros(nv, dtype=np.int64)
    for j in range(nv):
        z = int(bits[j * width:(j + 1) * width], 2)
        d = (z >> 1) if z % 2 == 0 else -((z + 1) >> 1)
        q[j] = (q[j - 2] if j >= 2 else 0) + d
    x = q.astype(np.float64) * (2 * eb)
    if dtype == oracle.C64:
        x = x.astype(np.float32)
    mine = oracle.decompress_block(s, b, dtype, eb)
    assert np.array_equal(x[0::2], mine.real) and np.array_equal(x[1::2], mine.imag)
    # and the width is the smallest that holds the largest zigzag code
    zmax = max(int(bits[j * width:(j + 1) * width], 2) for j in range(nv))
    assert zmax.bit_length() == width


@pytest.mark.parametrize("dtype", [oracle.C128, oracle.C64])
def test_verbatim_section_layout(dtype):
    # verbatim section after the body: u16 value positions ascending (value j = 2 * amplitude
    # + 0 for re, + 1 for im), then the raw values at the next multiple of the value size;
    # the verbatim values enter the prediction as code 0
    b, eb = 6, 1e-6
    rng = np.random.default_rng(4)
    v = (rng.standard_normal(1 << b) + 1j * rng.standard_normal(1 << b)) * 1e-3
    big = {5: 3e6 + 0j, 17: complex(0.0, -4e6), 40: complex(5e6, 6e6)}
    for k, x in big.items():
        v[k] = x
    v = v.astype(np.complex64 if dtype == oracle.C64 else np.complex128)
    s, info = oracle.compress_block(v, b, dtype, eb)
    mode, dt, bl, param, nverb, D = struct.unpack_from("<BBBBHH", s, 0)
    pos_want = sorted([2 * 5, 2 * 17 + 1, 2 * 40, 2 * 40 + 1])
    assert nverb == len(pos_want) == info["n_verbatim"]
    # the body ends where the chunk table, codebook and payload end; the section is the
    # stream's tail: positions, padding to the value size, values, zero padding to 16 bytes
    vs = np.dtype(np.float32 if dtype == oracle.C64 else np.float64).itemsize
    raw = np.frombuffer(v.view(np.float32 if dtype == oracle.C64 else np.float64).tobytes(),
                        dtype=np.float32 if dtype == oracle.C64 else np.float64)
    want_vals = b"".join(raw[j:j + 1].tobytes() for j in pos_want)
    want_pos = struct.pack("<%dH" % nverb, *pos_want)
    i = s.find(want_pos)
    assert i >= 16 and i % 4 == 0
    voff = (i + 2 * nverb + vs - 1) // vs * vs
    assert s[voff:voff + vs * nverb] == want_vals
    assert len(s) % 16 == 0 and set(s[voff + vs * nverb:]) <= {0}
    # prediction treats them as 0: the same block with those values replaced by 0 gives the
    # same mode, symbol count, payload bits and body; only the verbatim count, the total
    # length and the section differ
    z = v.copy()
    for k in big:
        z[k] = 0
    s0, _ = oracle.compress_block(z, b, dtype, eb)
    assert s0[0:4] == s[0:4] and s0[6:12] == s[6:12] and s0[16:i] == s[16:i]
    assert struct.unpack_from("<H", s0, 4)[0] == 0 and len(s0) == (i + 15) // 16 * 16


@pytest.mark.parametrize("dtype", [oracle.C128, oracle.C64])
def test_quantizer_range_boundary(dtype):
    # a value is quantized while |x r| < 2^29 (codes and their deltas then fit 32-bit
    # integers) and stored raw from 2^29 on; eb = 2^-11 makes r = 2^10 exact
    b, eb = 5, 2.0 ** -11
    lim = 2.0 ** 29 / 2.0 ** 10  # |x| at which |x r| reaches 2^29
    below = np.nextafter(np.float32(lim), np.float32(0)) if dtype == oracle.C64 else np.nextafter(lim, 0)
    for x, verb in [(lim, True), (-lim, True), (float(below), False), (-float(below), False)]:
        v = np.zeros(1 << b, dtype=np.complex64 if dtype == oracle.C64 else np.complex128)
        v[3] = x
        s, info = oracle.compress_block(v, b, dtype, eb)
        assert info["n_verbatim"] == (1 if verb else 0), x
        d = oracle.decompress_block(s, b, dtype, eb)
        assert abs(float(d[3].real) - x) <= eb
