"""Seeded random parity cases: circuits of mixed gate kinds on random sizes, precisions,
bounds and launch shapes, every stream and the stored norm equal to the oracle's at the end
and midway (GPU)."""
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


@pytest.fixture(scope="module")
def pool(sv):
    return sv.Pool(2 << 30)


def random_unitary(rng, d):
    z = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def random_circuit(rng, n, b, count):
    kinds = ["H", "X", "Z", "phase", "su2", "cnot", "swap", "u2", "u3", "diag2"]
    gates = []
    while len(gates) < count:
        kind = kinds[int(rng.integers(len(kinds)))]
        qs = [int(q) for q in rng.permutation(n)]
        nc = int(rng.integers(0, 3))
        if kind in ("H", "X", "Z", "phase", "su2"):
            m = {"H": C.H, "X": C.X, "Z": C.Z, "phase": C.phase(int(rng.integers(1, 6))),
                 "su2": C.haar_su2(rng)}[kind]
            t = qs[:1]
        elif kind == "cnot":
            m, t = np.eye(4, dtype=np.complex128)[[0, 3, 2, 1]], qs[:2]
        elif kind == "swap":
            m, t = C.SWAP, qs[:2]
        elif kind == "diag2":
            m, t = np.diag(np.exp(1j * rng.uniform(0, 2 * np.pi, 4))), qs[:2]
        else:
            k = 2 if kind == "u2" else 3
            m, t = random_unitary(rng, 1 << k), qs[:k]
        if sum(q >= b for q in t) > 2:
            continue
        gates.append(C.Gate(np.asarray(m, dtype=np.complex128), tuple(t), tuple(qs[len(t):len(t) + nc]), kind))
    return gates


def shape_for(rng, b):
    nv = 2 << b
    threads = [t for t in (32, 64, 128, 256) if 2 <= nv // t <= 32]
    t = threads[int(rng.integers(len(threads)))]
    chunks = [k for k in (16, 32, 64) if nv // k <= t]
    return t, bool(rng.integers(2)), chunks[int(rng.integers(len(chunks)))]


@pytest.mark.parametrize("seed", range(16))
def test_random_circuits_bit_exact(sv, pool, seed):
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(8, 15))
    b = int(rng.integers(5, min(n, 12) + 1))
    dtype = [oracle.C64, oracle.C128][int(rng.integers(2))]
    eb = [1e-4, 1e-6, 1e-8][int(rng.integers(3))]
    threads, compact, chunk = shape_for(rng, b)
    x = int(rng.integers(0, 1 << n))
    gates = random_circuit(rng, n, b, 40)
    st = sv.State(pool, n, n, eb, dtype, block_log2=b)
    try:
        st.set_threads(threads)
        st.set_compact(compact)
        st.set_chunk(chunk)
        st.reset_basis(x)
        cs = oracle.CompressedSim(n, n, b, dtype, eb, x, chunk=chunk)
        tag = "n=%d b=%d dtype=%d eb=%g T=%d compact=%d chunk=%d" % (n, b, dtype, eb, threads, compact, chunk)
        for i, g in enumerate(gates):
            st.apply(g.matrix, g.targets, g.controls)
            try:
                cs.apply(g.matrix, g.targets, g.controls)
            except RuntimeError:  # the oracle's norm collapsed: the GPU must report it too
                with pytest.raises(sv.SvError):
                    st.sync()
                return
            if i in (19, len(gates) - 1):
                for blk in range(cs.nblocks):
                    assert st.block_stream(blk) == cs.block_stream(blk), "%s gate %d block %d" % (tag, i, blk)
                assert st.norm() == cs.norm, tag
    finally:
        st.close()
