"""Failure detection on the GPU without a fault: the bounded mbarrier wait that the tensor-core
pass uses gives up on a barrier nothing arrives on, reports it, and leaves the context usable."""
import numpy as np
import pytest
import torch

import oracle
from paper_1811_05630_gb300 import circuits as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sv():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1811_05630_gb300 import sv as m

    return m


@pytest.mark.parametrize("polls", [1, 1000, 20000])
def test_bounded_wait_gives_up(sv, polls):
    assert sv.check_bounded_wait(polls) is True
    # the context still runs work: a small compressed QFT equals the oracle's byte for byte
    pool = sv.Pool(8 << 20)
    st = sv.State(pool, 8, 8, 1e-6, oracle.C128, block_log2=6)
    try:
        st.reset_basis(5)
        st.run(C.qft(8))
        cs = oracle.CompressedSim(8, 8, 6, oracle.C128, 1e-6, 5).run(C.qft(8))
        assert st.norm() == cs.norm
        for b in range(cs.nblocks):
            assert st.block_stream(b) == cs.block_stream(b)
    finally:
        st.close()
        pool.close()


def test_bounded_wait_arguments(sv):
    for polls in (0, -1, (1 << 24) + 1):
        with pytest.raises(sv.SvError) as e:
            sv.check_bounded_wait(polls)
        assert e.value.code == sv.ERR_ARG
