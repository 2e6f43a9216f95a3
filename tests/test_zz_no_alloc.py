"""The allocation-free compressor (sv_codec_compress_static) against the regular one.

It serves callers that cannot allocate device memory: they own their inputs and outputs
but cannot hand the library a scratch buffer, so the library keeps its scratch in a fixed
array of its own. This file is collected last; it must pass alone in a fresh process and
after the other tests (the array keeps the previous call's contents)."""
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


def streams_of(out, offs, lens):
    o, f, l = out.cpu().numpy(), offs.cpu().numpy(), lens.cpu().numpy()
    return [o[f[i]:f[i] + l[i]].tobytes() for i in range(len(f))]


def inputs(b, dtype, seed, reps):
    rng = np.random.default_rng(seed)
    blocks = [gen_block(k, b, rng, dtype) for k in KINDS for _ in range(reps)]
    v = gen_block("normal", b, rng, dtype)
    v[3] = 3e6  # one verbatim value
    blocks.append(v)
    return blocks


@pytest.mark.parametrize("dtype", [oracle.C128, oracle.C64])
def test_static_matches_regular_on_two_calls(sv, dtype):
    eb = 1e-6
    # two calls in a row with different sizes: a stale record from the first would show
    for b, reps in [(10, 4), (7, 2)]:
        blocks = inputs(b, dtype, seed=b, reps=reps)
        vals = torch.from_numpy(np.concatenate(blocks)).cuda()
        ref_out, ref_offs, ref_lens, ref_used = sv.codec_compress(vals, b, eb)
        nb = len(blocks)
        out = torch.zeros_like(ref_out)
        offs = torch.zeros(nb, dtype=torch.int64, device="cuda")
        lens = torch.zeros(nb, dtype=torch.int32, device="cuda")
        used, norm = sv.codec_compress_static(vals, b, eb, out, offs, lens)
        assert used == ref_used
        assert streams_of(out, offs, lens) == streams_of(ref_out, ref_offs, ref_lens)
        # the reported norm, rebuilt from the oracle codec's exact per-block sums with the
        # documented definition (IEEE double steps in Python floats): equal bit for bit
        infos = [oracle.compress_block(blk, b, dtype, eb)[1] for blk in blocks]
        S = sum((i["sq_hi"] << 64) | i["sq_lo"] for i in infos)
        Sd = float(S >> 64) * 18446744073709551616.0 + float(S & (2**64 - 1))
        v = [i["vsum"] for i in infos]
        while len(v) & (len(v) - 1):
            v.append(0.0)
        while len(v) > 1:
            v = [v[2 * k] + v[2 * k + 1] for k in range(len(v) // 2)]
        two = 2.0 * eb
        assert norm == Sd * (two * two) + v[0]
        # and it is the squared norm of the reconstructed values (float rounding for complex64)
        d = sv.codec_decompress(out, offs, lens, b, dtype, eb).cpu().numpy().astype(np.complex128)
        ref_norm = float(np.vdot(d, d).real)
        assert abs(norm - ref_norm) <= (1e-12 if dtype == oracle.C128 else 1e-6) * ref_norm


def oracle_norm(blocks, b, dtype, eb):
    """The documented norm, rebuilt from the oracle codec's exact per-block sums."""
    infos = [oracle.compress_block(blk, b, dtype, eb)[1] for blk in blocks]
    S = sum((i["sq_hi"] << 64) | i["sq_lo"] for i in infos)
    Sd = float(S >> 64) * 18446744073709551616.0 + float(S & (2**64 - 1))
    v = [i["vsum"] for i in infos]
    while len(v) & (len(v) - 1):
        v.append(0.0)
    while len(v) > 1:
        v = [v[2 * k] + v[2 * k + 1] for k in range(len(v) // 2)]
    two = 2.0 * eb
    return Sd * (two * two) + v[0]


@pytest.mark.parametrize("nb", [65536, 40000])
def test_static_norm_at_large_block_counts(sv, nb):
    """The norm's pairwise tree over many blocks: at the array's limit (every thread of the
    one-CTA reduction takes 32 pairs on the first level) and at a count that is not a power
    of two (the list is padded with zeros), with verbatim values in scattered blocks."""
    b, eb, dtype = 5, 1e-6, oracle.C128
    rng = np.random.default_rng(nb)
    vals = (rng.standard_normal(nb << b) + 1j * rng.standard_normal(nb << b)) * 1e-4
    hot = rng.choice(nb, size=9, replace=False)
    for h in hot:  # out-of-range values are stored raw (verbatim)
        vals[(int(h) << b) + int(rng.integers(1 << b))] = 3e6 + 1.25e6j
    blocks = [vals[i << b:(i + 1) << b] for i in range(nb)]
    t = torch.from_numpy(vals).cuda()
    ref_out, ref_offs, ref_lens, ref_used = sv.codec_compress(t, b, eb)
    out = torch.zeros_like(ref_out)
    offs = torch.zeros(nb, dtype=torch.int64, device="cuda")
    lens = torch.zeros(nb, dtype=torch.int32, device="cuda")
    used, norm = sv.codec_compress_static(t, b, eb, out, offs, lens)
    assert used == ref_used
    assert streams_of(out, offs, lens) == streams_of(ref_out, ref_offs, ref_lens)
    assert norm == oracle_norm(blocks, b, dtype, eb)


def test_static_refuses_a_capturing_stream(sv):
    """Each call reads its results back and synchronizes, which a capturing stream does not
    accept: the call is refused before it enqueues anything, and the capture stays valid."""
    b, eb = 6, 1e-6
    vals = torch.zeros(4 << b, dtype=torch.complex128, device="cuda")
    out = torch.zeros(4 << 12, dtype=torch.uint8, device="cuda")
    offs = torch.zeros(4, dtype=torch.int64, device="cuda")
    lens = torch.zeros(4, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    codes = []
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            try:
                sv.codec_compress_static(vals, b, eb, out, offs, lens, stream=s)
                codes.append(0)
            except sv.SvError as e:
                codes.append(e.code)
    torch.cuda.synchronize()
    assert codes == [sv.ERR_ARG]
    # outside the capture the same call runs
    used, norm = sv.codec_compress_static(vals, b, eb, out, offs, lens)
    assert used == 4 * 16 and norm == 0.0


def test_static_with_no_blocks_is_a_no_op(sv):
    z = torch.zeros(0, dtype=torch.complex128, device="cuda")
    out = torch.zeros(16, dtype=torch.uint8, device="cuda")
    offs = torch.zeros(0, dtype=torch.int64, device="cuda")
    lens = torch.zeros(0, dtype=torch.int32, device="cuda")
    assert sv.codec_compress_static(z, 5, 1e-6, out, offs, lens) == (0, 0.0)


def test_static_rejects_more_blocks_than_its_array(sv):
    b = 5
    nb = sv.STATIC_MAX_BLOCKS + 1
    vals = torch.zeros(nb << b, dtype=torch.complex128, device="cuda")
    out = torch.zeros(nb * 16, dtype=torch.uint8, device="cuda")
    offs = torch.zeros(nb, dtype=torch.int64, device="cuda")
    lens = torch.zeros(nb, dtype=torch.int32, device="cuda")
    with pytest.raises(sv.SvError) as e:
        sv.codec_compress_static(vals, b, 1e-6, out, offs, lens)
    assert e.value.code == sv.ERR_UNSUPPORTED
