"""GPU block codec vs the oracle codec, through the C ABI (sv_codec_compress /
sv_codec_decompress): byte-identical streams on identical input bytes, bit-identical
decoded values, and the decoder's bounds checks on corrupted streams."""
import numpy as np
import pytest
import torch

import oracle
from blockgen import KINDS, gen_block

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sv():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1811_05630_gb300 import sv as m

    return m


def tdt(dtype):
    return torch.complex64 if dtype == oracle.C64 else torch.complex128


def make_blocks(b, dtype, seed, reps=3):
    rng = np.random.default_rng(seed)
    blocks = [gen_block(k, b, rng, dtype) for k in KINDS for _ in range(reps)]
    # a few blocks with isolated verbatim values (out-of-range magnitudes)
    for _ in range(2):
        v = gen_block("normal", b, rng, dtype)
        v[rng.integers(1 << b)] = 3e6
        blocks.append(v)
    return blocks


@pytest.mark.parametrize("dtype", [oracle.C128, oracle.C64])
@pytest.mark.parametrize("b", [5, 8, 11, 12])
@pytest.mark.parametrize("eb", [1e-4, 1e-6, 1e-8])
def test_compress_byte_identical(sv, dtype, b, eb):
    blocks = make_blocks(b, dtype, seed=b * 7 + dtype)
    refs = [oracle.compress_block(blk, b, dtype, eb) for blk in blocks]
    vals = torch.from_numpy(np.concatenate(blocks)).to("cuda")
    if dtype == oracle.C128 and max(info["n_verbatim"] for _, info in refs) > 128:
        # documented GPU limit: at most 128 verbatim values per complex128 block
        with pytest.raises(sv.SvError) as e:
            sv.codec_compress(vals, b, eb)
        assert e.value.code == sv.ERR_UNSUPPORTED
        keep = [i for i, (_, info) in enumerate(refs) if info["n_verbatim"] <= 128]
        blocks = [blocks[i] for i in keep]
        refs = [refs[i] for i in keep]
        vals = torch.from_numpy(np.concatenate(blocks)).to("cuda")
    out, offs, lens, used = sv.codec_compress(vals, b, eb)
    out_h, offs_h, lens_h = out.cpu().numpy(), offs.cpu().numpy(), lens.cpu().numpy()
    assert used == int(lens_h.sum())
    for i, blk in enumerate(blocks):
        ref = refs[i][0]
        got = out_h[offs_h[i]: offs_h[i] + lens_h[i]].tobytes()
        assert got == ref, "block %d differs (len %d vs %d)" % (i, len(got), len(ref))


def pack_streams(streams):
    offs, pos = [], 0
    for s in streams:
        offs.append(pos)
        pos += len(s)
    buf = np.zeros(max(pos, 16), dtype=np.uint8)
    for o, s in zip(offs, streams):
        buf[o:o + len(s)] = np.frombuffer(s, dtype=np.uint8)
    return buf, np.array(offs, dtype=np.int64), np.array([len(s) for s in streams], dtype=np.int32)


@pytest.mark.parametrize("dtype", [oracle.C128, oracle.C64])
@pytest.mark.parametrize("b", [5, 9, 12])
def test_decompress_bit_identical(sv, dtype, b):
    eb = 1e-6
    blocks = make_blocks(b, dtype, seed=100 + b)
    streams = [oracle.compress_block(blk, b, dtype, eb)[0] for blk in blocks]
    buf, offs, lens = pack_streams(streams)
    got = sv.codec_decompress(torch.from_numpy(buf).cuda(), torch.from_numpy(offs).cuda(),
                              torch.from_numpy(lens).cuda(), b, dtype, eb).cpu().numpy()
    B = 1 << b
    for i, s in enumerate(streams):
        ref = oracle.decompress_block(s, b, dtype, eb)
        assert got[i * B:(i + 1) * B].tobytes() == ref.tobytes()


def test_corrupted_streams_are_reported(sv):
    b, dtype, eb = 12, oracle.C128, 1e-4
    rng = np.random.default_rng(3)
    v = gen_block("normal", b, rng, dtype)
    s, info = oracle.compress_block(v, b, dtype, eb)
    assert info["mode"] == oracle.MODE_HUFF
    bad = []
    x = bytearray(s)
    x[1] = 7  # dtype byte
    bad.append(bytes(x))
    x = bytearray(s)
    x[12:16] = (len(s) + 64).to_bytes(4, "little")  # total larger than the stream
    bad.append(bytes(x))
    x = bytearray(s)
    lmax, D = x[3], int.from_bytes(x[6:8], "little")
    off_chunk = 16 + (2 * lmax + 3) // 4 * 4 + (2 * D + 3) // 4 * 4
    x[off_chunk] ^= 0x5A  # chunk bit counts no longer sum to the payload
    bad.append(bytes(x))
    for s_bad in bad:
        buf, offs, lens = pack_streams([s_bad])
        with pytest.raises(sv.SvError) as e:
            sv.codec_decompress(torch.from_numpy(buf).cuda(), torch.from_numpy(offs).cuda(),
                                torch.from_numpy(lens).cuda(), b, dtype, eb)
        assert e.value.code == sv.ERR_CORRUPT


@pytest.mark.parametrize("b", [5, 10, 12])
def test_complex64_verbatim_heavy_blocks(sv, b):
    # |x| in (0.1, 0.3) at eb 1e-8: the float spacing is close to eb, so rounding the
    # reconstruction to float pushes ~14% of values past the bound; they are kept raw, in
    # place, without the 128-per-block limit of complex128
    rng = np.random.default_rng(b)
    B = 1 << b
    blocks = []
    for _ in range(4):
        mag = rng.uniform(0.1, 0.3, (2, B)) * np.sign(rng.standard_normal((2, B)))
        blocks.append((mag[0] + 1j * mag[1]).astype(np.complex64))
    eb = 1e-8
    refs = [oracle.compress_block(blk, b, oracle.C64, eb) for blk in blocks]
    nmax = max(i["n_verbatim"] for _, i in refs)
    assert nmax > (128 if b >= 10 else 0)
    vals = torch.from_numpy(np.concatenate(blocks)).cuda()
    out, offs, lens, used = sv.codec_compress(vals, b, eb)
    o, f, l = out.cpu().numpy(), offs.cpu().numpy(), lens.cpu().numpy()
    for i, (ref, _) in enumerate(refs):
        assert o[f[i]:f[i] + l[i]].tobytes() == ref, i
    d = sv.codec_decompress(out, offs, lens, b, oracle.C64, eb).cpu().numpy()
    for i, (ref, _) in enumerate(refs):
        assert d[i * B:(i + 1) * B].tobytes() == oracle.decompress_block(ref, b, oracle.C64, eb).tobytes()


@pytest.mark.parametrize("b", [7, 10, 12])
@pytest.mark.parametrize("kind", ["huge", "ties", "mixed"])
def test_complex128_verbatim_heavy_blocks(sv, b, kind):
    # more verbatim values than a block's shared-memory lists hold (128): values beyond the
    # code range (|x| > 2^29 2eb), values on rounding ties of the grid (2^-6 at eb 1e-6: the
    # reconstruction error is eb itself, and rounding pushes it past), or three quarters ties
    B = 1 << b
    rng = np.random.default_rng(b)
    eb = 1e-6
    blocks = []
    for _ in range(3):
        if kind == "huge":
            v = (rng.uniform(1e3, 1e4, B) + 1j * rng.uniform(-1e4, -1e3, B))
        elif kind == "ties":
            v = np.full(B, 2.0 ** -6 + 1j * 2.0 ** -6)
        else:
            v = rng.standard_normal(B) * 1e-3 + 1j * rng.standard_normal(B) * 1e-3
            v[np.arange(B) % 4 != 0] = 2.0 ** -6 - 1j * 2.0 ** -6
        blocks.append(v.astype(np.complex128))
    refs = [oracle.compress_block(blk, b, oracle.C128, eb) for blk in blocks]
    assert max(i["n_verbatim"] for _, i in refs) > 128
    vals = torch.from_numpy(np.concatenate(blocks)).cuda()
    out, offs, lens, used = sv.codec_compress(vals, b, eb)
    o, f, l = out.cpu().numpy(), offs.cpu().numpy(), lens.cpu().numpy()
    for i, (ref, _) in enumerate(refs):
        assert o[f[i]:f[i] + l[i]].tobytes() == ref, i
    d = sv.codec_decompress(out, offs, lens, b, oracle.C128, eb).cpu().numpy()
    for i, (ref, _) in enumerate(refs):
        assert d[i * B:(i + 1) * B].tobytes() == oracle.decompress_block(ref, b, oracle.C128, eb).tobytes()


def test_many_blocks_roundtrip_full_size(sv):
    # 2^20 amplitudes (256 blocks of 4096): GPU compress -> GPU decompress equals the
    # oracle's reconstruction on sampled blocks, and the pointwise bound holds everywhere
    b, eb = 12, 1e-7
    n = 20
    rng = np.random.default_rng(5)
    x = rng.integers(1 << n)
    y = np.arange(1 << n)
    v = np.exp(2j * np.pi * ((x * y) % (1 << n)) / (1 << n)) / 2 ** (n / 2)
    t = torch.from_numpy(v).cuda()
    out, offs, lens, used = sv.codec_compress(t, b, eb)
    d = sv.codec_decompress(out, offs, lens, b, oracle.C128, eb).cpu().numpy()
    assert np.abs(d.real - v.real).max() <= eb and np.abs(d.imag - v.imag).max() <= eb
    for blk in rng.choice(256, 8, replace=False):
        ref = oracle.decompress_block(oracle.compress_block(v[blk * 4096:(blk + 1) * 4096], b, oracle.C128, eb)[0],
                                      b, oracle.C128, eb)
        assert d[blk * 4096:(blk + 1) * 4096].tobytes() == ref.tobytes()
    assert used < v.nbytes
