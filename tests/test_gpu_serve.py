"""Serving loop: requests of uneven size, kind, dtype and error bound arrive while others
run; every result equals (byte for byte) the same request simulated alone."""
import numpy as np
import pytest
import torch

from paper_1811_05630_gb300 import circuits as C

pytestmark = pytest.mark.gpu


def test_each_result_is_the_same_alone_and_in_the_mix():
    from paper_1811_05630_gb300 import sv
    from paper_1811_05630_gb300.serve import Server

    reqs = C.serving_requests(count=14, rate=200.0, seed=3, nmin=8, nmax=13)
    srv = Server(pool_bytes=2 << 30, budget_bytes=1 << 30, block_log2=7, max_batch=8, graphs=True,
                 keep_results=True)
    out = srv.run(reqs)
    assert out["completed"] == len(reqs)
    pool = sv.Pool(1 << 30)
    for res in out["results"]:
        req = reqs[res.rid]
        b = min(7, req.n)
        st = sv.State(pool, req.n, req.n, req.eb, req.dtype, block_log2=b)
        st.reset_basis(req.basis)
        st.run(req.gates)
        alone = [st.block_stream(i) for i in range(1 << (req.n - b))]
        assert alone == res.streams, req.rid
        assert st.norm() == res.norm
        st.close()
    assert out["p99_s"] >= out["p50_s"] > 0
    srv.close()
