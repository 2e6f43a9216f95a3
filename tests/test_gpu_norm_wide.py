"""GPU stored norm when the exact sum of squared codes passes 2^64 (the high word of the
128-bit accumulator and its carries), against the oracle bit for bit.

At eb = 1e-10 a unit-norm state whose amplitudes are all below the quantizer's limit
(2^29 * 2eb = 0.107) has Σq² = N / (2eb)² = 2.5e19 > 2^64 = 1.8e19.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1811_05630_gb300 import circuits as C

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("b", [6, 9])
def test_norm_with_codes_summing_past_64_bits(b):
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1811_05630_gb300 import sv

    n, eb = 9, 1e-10
    gates = [C.Gate(C.H, (q,), (), "H") for q in range(n)] + C.random_brickwork(n, 2, seed=4)
    pool = sv.Pool(1 << 28)
    st = sv.State(pool, n, n, eb, sv.C128, block_log2=b)
    cs = oracle.CompressedSim(n, n, b, oracle.C128, eb, 0)
    try:
        st.reset_basis(0)
        wide = 0
        for i, g in enumerate(gates):
            st.apply(g.matrix, g.targets, g.controls)
            cs.apply(g.matrix, g.targets, g.controls)
            for blk in range(cs.nblocks):
                assert st.block_stream(blk) == cs.block_stream(blk), "gate %d block %d" % (i, blk)
            assert st.norm() == cs.norm, "gate %d" % i
            # codes of the quantized (not verbatim) components
            c = np.concatenate([cs.read().real, cs.read().imag]) / (2 * eb)
            c = np.round(c[np.abs(c) < 2.0 ** 29])
            if np.sum(c * c) > 2.0 ** 64:
                wide += 1
        assert wide >= len(gates) // 2  # most passes ran with the high word in use
    finally:
        st.close()
        pool.close()
