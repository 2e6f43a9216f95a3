"""Host spill: a state whose device pool holds its metadata and its first arenas keeps its
grown compressed streams in a pinned host-memory pool (reached by the kernels over
NVLink-C2C); every pass equals the oracle's byte for byte."""
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


@pytest.mark.parametrize("dtype", [oracle.C128, oracle.C64])
def test_arenas_in_host_memory_bit_exact(sv, dtype):
    # the device pool holds the metadata run and the two initial arenas (one 2 MiB page each).
    # The dense state of this circuit reaches about 1.29 MB of streams in either dtype, and the
    # arena the next pass writes is then sized for twice that: two pages, which the device pool
    # no longer has in one run, so the grown arenas come from the host pool
    n, sl, b, eb = 18, 12, 8, 1e-8
    dev = sv.Pool(6 << 20)
    host = sv.Pool(64 << 20, "host")
    gates = C.random_brickwork(n, 3, seed=5) + C.qft(n)[:40]
    st = sv.State(dev, n, sl, eb, dtype, block_log2=b)
    try:
        st.set_spill(host)
        st.reset_basis(0)
        cs = oracle.CompressedSim(n, sl, b, dtype, eb, 0)
        for i, g in enumerate(gates):
            st.apply(g.matrix, g.targets, g.controls)
            cs.apply(g.matrix, g.targets, g.controls)
            if i % 16 == 15 or i == len(gates) - 1:
                for blk in range(cs.nblocks):
                    assert st.block_stream(blk) == cs.block_stream(blk), (i, blk)
                assert st.norm() == cs.norm
        assert st.stats()["spill_arena_bytes"] > 0
        assert host.usage()[0] > 0
        assert st.read().tobytes() == cs.read().astype(np.complex128).tobytes()
    finally:
        st.close()
    assert host.usage()[0] == 0  # every spilled page is back
    host.close()
    dev.close()


def test_spill_pool_arguments(sv):
    dev = sv.Pool(16 << 20)  # pages for a compressed state and a plain one
    st = sv.State(dev, 10, 10, 1e-6, oracle.C128, block_log2=6)
    try:
        with pytest.raises(sv.SvError) as e:
            st.set_spill(dev)  # the state's own pool
        assert e.value.code == sv.ERR_ARG
        plain = sv.State(dev, 8, 8, 0.0, oracle.C128)
        host = sv.Pool(4 << 20, "host")
        with pytest.raises(sv.SvError):
            plain.set_spill(host)
        plain.close()
        host.close()
    finally:
        st.close()
        dev.close()
