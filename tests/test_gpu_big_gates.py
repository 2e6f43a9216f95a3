"""4- and 5-qubit gates (Algorithm 1's GateComputation with a dense 2^k x 2^k matrix, k <= 5):
Haar-random dense gates and fused brickwork circuits through sv_apply_gate, compared with the
oracle's Algorithm 1 byte for byte after every pass (streams and stored norm), and the plain
GPU path with the plain oracle (O1) within 1e-12 (FP64) / 1e-5 (FP32) per component."""
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
    return sv.Pool(1 << 30)


def assert_same_state(st, cs, tag=""):
    for b in range(cs.nblocks):
        assert st.block_stream(b) == cs.block_stream(b), "%s block %d" % (tag, b)
    assert st.norm() == cs.norm, tag


def dense_gates(n, rng):
    """An H layer (dense state), then Haar 4- and 5-qubit gates on target sets inside the
    block, spanning one or two high qubits, and under controls inside and above the block
    (block_log2 6 in the tests)."""
    gates = [C.Gate(C.H, (q,), (), "H") for q in range(n)]
    sets = [((0, 1, 2, 3, 4), ()), ((1, 3, 5, 0), ()), ((0, 2, 4, 7, 9), ()), ((8, 1, 3, 5), (10,)),
            ((2, 6, 4, 0, 11), (1,)), ((5, 4, 3, 2), (0, 9)), ((0, 1, 2, 3, 4), (6, 7))]
    for t, c in sets:
        gates.append(C.Gate(C.haar_unitary(len(t), rng), t, c, "U%d" % len(t)))
    return gates


@pytest.mark.parametrize("dtype", [oracle.C128, oracle.C64])
@pytest.mark.parametrize("eb", [1e-5, 1e-7])
def test_dense_4_and_5_qubit_gates_bit_exact(sv, pool, dtype, eb):
    n, sl, b = 12, 9, 6
    rng = np.random.default_rng(int(eb * 1e9) + dtype)
    gates = dense_gates(n, rng)
    st = sv.State(pool, n, sl, eb, dtype, block_log2=b)
    try:
        st.reset_basis(0)
        cs = oracle.CompressedSim(n, sl, b, dtype, eb, 0)
        for i, g in enumerate(gates):
            st.apply(g.matrix, g.targets, g.controls)
            cs.apply(g.matrix, g.targets, g.controls)
            if g.k >= 4 or i == n - 1:
                assert_same_state(st, cs, "gate %d %s %s %s" % (i, g.name, g.targets, g.controls))
        assert st.read().tobytes() == cs.read().astype(np.complex128).tobytes()
    finally:
        st.close()


@pytest.mark.parametrize("dtype", [oracle.C128, oracle.C64])
def test_fused_brickwork_bit_exact(sv, pool, dtype):
    # a brickwork circuit fused into gates of up to 5 qubits (at most 2 at or above the block):
    # both simulators run the same fused list
    n, sl, b, eb = 14, 10, 8, 1e-6
    fused = C.fuse(C.random_brickwork(n, 6, seed=4), 5, block_log2=b)
    assert max(g.k for g in fused) == 5
    st = sv.State(pool, n, sl, eb, dtype, block_log2=b)
    try:
        st.reset_basis(0)
        cs = oracle.CompressedSim(n, sl, b, dtype, eb, 0)
        for i, g in enumerate(fused):
            st.apply(g.matrix, g.targets, g.controls)
            cs.apply(g.matrix, g.targets, g.controls)
            assert_same_state(st, cs, "pass %d %s %s" % (i, g.name, g.targets))
    finally:
        st.close()


@pytest.mark.parametrize("block_log2,threads", [(5, 32), (8, 64), (8, 256), (11, 256)])
def test_big_gates_at_every_block_size(sv, pool, block_log2, threads):
    # the round structure (whole tuples per round of CTA rows) at the smallest and the largest
    # blocks, with few and many rows per round
    n, eb, dtype = 13, 1e-6, oracle.C128
    rng = np.random.default_rng(block_log2 * 31 + threads)
    gates = [C.Gate(C.H, (q,), (), "H") for q in range(n)]
    gates.append(C.Gate(C.haar_unitary(5, rng), (0, 1, 2, 3, 4), (), "U5"))
    gates.append(C.Gate(C.haar_unitary(5, rng), (1, 3, block_log2, 0, block_log2 + 1), (), "U5h"))
    gates.append(C.Gate(C.haar_unitary(4, rng), (4, 2, 0, block_log2 + 1), (3,), "U4c"))
    st = sv.State(pool, n, n, eb, dtype, block_log2=block_log2)
    try:
        st.set_threads(threads)
        st.reset_basis(0)
        cs = oracle.CompressedSim(n, n, block_log2, dtype, eb, 0)
        for i, g in enumerate(gates):
            st.apply(g.matrix, g.targets, g.controls)
            cs.apply(g.matrix, g.targets, g.controls)
        assert_same_state(st, cs, "end")
    finally:
        st.close()


def test_unit_and_diagonal_5_qubit_gates_bit_exact(sv, pool):
    # a 5-qubit permutation (unit rows) and a diagonal phase gate take the single-term and
    # diagonal forms of the fixed-point path
    n, sl, b, eb = 12, 9, 6, 1e-6
    rng = np.random.default_rng(7)
    perm = np.eye(32, dtype=np.complex128)[rng.permutation(32)]
    perm[3] *= -1j
    diag = np.diag(np.exp(2j * np.pi * rng.random(32)))
    gates = [C.Gate(C.H, (q,), (), "H") for q in range(n)] + [
        C.Gate(perm, (0, 2, 4, 6, 8), (), "P5"), C.Gate(diag, (1, 3, 5, 7, 9), (), "D5")]
    st = sv.State(pool, n, sl, eb, oracle.C128, block_log2=b)
    try:
        st.reset_basis(0)
        cs = oracle.CompressedSim(n, sl, b, oracle.C128, eb, 0)
        for g in gates:
            st.apply(g.matrix, g.targets, g.controls)
            cs.apply(g.matrix, g.targets, g.controls)
        assert_same_state(st, cs, "end")
    finally:
        st.close()


@pytest.mark.parametrize("dtype,tol", [(oracle.C128, 1e-12), (oracle.C64, 1e-5)])
def test_plain_path_4_and_5_qubit_gates(sv, pool, dtype, tol):
    n = 12
    rng = np.random.default_rng(11)
    gates = dense_gates(n, rng)
    st = sv.State(pool, n, n, 0.0, dtype)
    try:
        st.reset_basis(0)
        st.run(gates)
        ref = oracle.PlainSim(n, dtype, 0).run(gates).state.astype(np.complex128)
        got = st.read()
        assert np.max(np.abs(got.real - ref.real)) <= tol and np.max(np.abs(got.imag - ref.imag)) <= tol
    finally:
        st.close()


def test_batches_refuse_gates_above_3_qubits(sv, pool):
    st = sv.State(pool, 10, 10, 1e-6, oracle.C128, block_log2=6)
    bt = sv.Batch(pool, 2)
    try:
        with pytest.raises(sv.SvError) as e:
            bt.apply([st], [C.Gate(C.haar_unitary(4, np.random.default_rng(0)), (0, 1, 2, 3))])
        assert e.value.code == sv.ERR_UNSUPPORTED
    finally:
        bt.close()
        st.close()


def tc_gates(n, b, rng):
    """Dense gates at 2048-amplitude blocks: inside the block, with two high targets (four blocks
    per group: two chunks of 128 tuples), a 4-qubit gate under a control, a control above the
    block, and unit / diagonal 5-qubit gates."""
    perm = np.eye(32, dtype=np.complex128)[rng.permutation(32)]
    perm[5] *= 1j
    diag = np.diag(np.exp(2j * np.pi * rng.random(32)))
    gates = [C.Gate(C.H, (q,), (), "H") for q in range(n)]
    for t, c in [((0, 1, 2, 3, 4), ()), ((1, 3, b, 0, b + 1), ()), ((4, 2, 0, b + 2), (3,)),
                 ((5, 6, 7, 8, 9), (b + 1,)), ((2, 9, 4, 10), ()), ((0, 1, 2, 3, 4), (5, 6))]:
        gates.append(C.Gate(C.haar_unitary(len(t), rng), t, c, "U%d" % len(t)))
    gates += [C.Gate(perm, (0, 2, 4, 6, 8), (), "P5"), C.Gate(diag, (1, 3, 5, 7, 9), (), "D5")]
    return gates


@pytest.mark.parametrize("eb", [1e-4, 1e-6, 1e-8])
@pytest.mark.parametrize("tensor_cores", [True, False])
def test_tensor_core_gate_bit_exact(sv, pool, eb, tensor_cores):
    # eb 1e-4: every |code| < 256 (one code digit); 1e-6: two code digits; 1e-8: codes beyond
    # the digit form (the CUDA-core rounds); each pass byte for byte against the oracle
    n, sl, b = 14, 14, 11
    gates = tc_gates(n, b, np.random.default_rng(int(-np.log10(eb))))
    st = sv.State(pool, n, sl, eb, oracle.C128, block_log2=b)
    try:
        st.set_tensor_cores(tensor_cores)
        st.reset_basis(0)
        cs = oracle.CompressedSim(n, sl, b, oracle.C128, eb, 0)
        for i, g in enumerate(gates):
            st.apply(g.matrix, g.targets, g.controls)
            cs.apply(g.matrix, g.targets, g.controls)
            if g.k >= 4:
                assert_same_state(st, cs, "gate %d %s %s %s" % (i, g.name, g.targets, g.controls))
    finally:
        st.close()


def test_tensor_cores_do_not_change_fused_brickwork(sv, pool):
    # a fused brickwork circuit at 2048-amplitude blocks, tensor cores on and off: equal streams
    n, b, eb = 15, 11, 1e-6
    fused = C.fuse(C.random_brickwork(n, 5, seed=9), 5, block_log2=b)
    out = []
    for tc in (True, False):
        st = sv.State(pool, n, n, eb, oracle.C128, block_log2=b)
        st.set_tensor_cores(tc)
        st.reset_basis(0)
        st.run(fused)
        out.append(([st.block_stream(i) for i in range(1 << (n - b))], st.norm()))
        st.close()
    assert out[0] == out[1]
    cs = oracle.CompressedSim(n, n, b, oracle.C128, eb, 0).run(fused)
    assert out[0][0] == [cs.block_stream(i) for i in range(cs.nblocks)] and out[0][1] == cs.norm
