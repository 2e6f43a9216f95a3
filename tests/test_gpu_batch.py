"""Batched passes (sv_batch_apply): many states advanced one gate each per launch give the
same bytes as advancing each state alone with sv_apply_gate, and as the oracle, with and
without CUDA-graph replay."""
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


def circuits_mix():
    # uneven sizes and kinds sharing one block size (b = 7)
    return [
        (10, 8, 1e-6, C.seeded_index(1, 10), C.qft(10)),
        (12, 9, 1e-8, 0, C.grover(12, C.seeded_index(2, 12), 2)),
        (11, 11, 1e-5, 0, C.random_brickwork(11, 3, seed=3)),
        (9, 9, 1e-6, 0, C.random_brickwork(9, 4, seed=4)),
    ]


def streams(st, nb):
    return [st.block_stream(i) for i in range(nb)]


@pytest.mark.parametrize("graphs", [False, True])
@pytest.mark.parametrize("dtype", [oracle.C128, oracle.C64])
def test_batch_equals_single_and_oracle(sv, dtype, graphs):
    b = 7
    pool = sv.Pool(1 << 30)
    mix = circuits_mix()
    stream = torch.cuda.Stream()  # graph capture needs a stream other than the legacy default
    batched = [sv.State(pool, n, sl, eb, dtype, block_log2=b, stream=stream) for n, sl, eb, x, _ in mix]
    single = [sv.State(pool, n, sl, eb, dtype, block_log2=b, stream=stream) for n, sl, eb, x, _ in mix]
    for st, (n, sl, eb, x, _) in zip(batched + single, mix + mix):
        st.reset_basis(x)
    batch = sv.Batch(pool, len(mix), stream=stream, graphs=graphs)
    steps = max(len(c[4]) for c in mix)
    for t in range(steps):
        act = [i for i, c in enumerate(mix) if t < len(c[4])]  # continuous: finished ones leave
        batch.apply([batched[i] for i in act], [mix[i][4][t] for i in act])
        for i in act:
            g = mix[i][4][t]
            single[i].apply(g.matrix, g.targets, g.controls)
    for i, (n, sl, eb, x, gates) in enumerate(mix):
        nb = 1 << (n - b)
        sb = streams(batched[i], nb)
        assert sb == streams(single[i], nb), i
        assert batched[i].norm() == single[i].norm()
        cs = oracle.CompressedSim(n, sl, b, dtype, eb, x).run(gates)
        assert sb == [cs.block_stream(k) for k in range(nb)], i
    batch.close()
    for st in batched + single:
        st.close()
