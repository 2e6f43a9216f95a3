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
