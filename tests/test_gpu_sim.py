"""GPU Algorithm 1 (sv_apply_gate through the C ABI) vs the oracle's Algorithm 1.

Every FP step of the pass (dequantize, normalize by sigma, gate, quantize) is an IEEE
operation in the oracle's order on both sides, so the compressed streams, the stored norm
and the decoded amplitudes must be identical bit for bit after every checked gate. The plain
(uncompressed) GPU path is compared with O1 within 1e-12 (FP64) / 1e-5 (FP32) per component.
"""
import math

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
    p = sv.Pool(1 << 30)
    yield p


def assert_same_state(st, cs, tag=""):
    nb = cs.nblocks
    for b in range(nb):
        assert st.block_stream(b) == cs.block_stream(b), "%s block %d" % (tag, b)
    assert st.norm() == cs.norm, tag


def run_compare(sv, pool, n, sl, b, dtype, eb, x, gates, every=1, arena_bytes=0):
    st = sv.State(pool, n, sl, eb, dtype, block_log2=b, arena_bytes=arena_bytes)
    try:
        st.reset_basis(x)
        cs = oracle.CompressedSim(n, sl, b, dtype, eb, x)
        assert_same_state(st, cs, "init")
        for i, g in enumerate(gates):
            st.apply(g.matrix, g.targets, g.controls)
            cs.apply(g.matrix, g.targets, g.controls)
            if (i + 1) % every == 0 or i == len(gates) - 1:
                assert_same_state(st, cs, "gate %d %s" % (i, g.name))
        got = st.read()
        ref = cs.read().astype(np.complex128)
        assert got.tobytes() == ref.tobytes()
        return st.stats(), got
    finally:
        st.close()


def test_qft12_config_bit_exact(sv, pool):
    # 12 qubits, 16 slices of 256 amplitudes, eb = 1e-6, complex128 (one block per slice)
    n = 12
    x = C.seeded_index(0, n)
    stats, got = run_compare(sv, pool, n, 8, 8, oracle.C128, 1e-6, x, C.qft(n))
    ref = np.exp(2j * np.pi * ((x * np.arange(1 << n)) % (1 << n)) / (1 << n)) / 2 ** (n / 2)
    F = abs(np.vdot(ref, got)) ** 2 / np.vdot(got, got).real
    print("QFT12 fidelity vs closed form: 1 - F = %.3e, bytes %d" % (1 - F, stats["compressed_bytes"]))
    assert 1 - F < 1e-6


def test_qft_overlap_matches_host(sv, pool):
    # sv_overlap_qft streams the state against the closed form on the GPU
    n = 14
    x = C.seeded_index(5, n)
    st = sv.State(pool, n, 10, 1e-6, oracle.C128, block_log2=8)
    try:
        st.reset_basis(x)
        st.run(C.qft(n))
        got = st.read()
        ref = np.exp(2j * np.pi * ((x * np.arange(1 << n)) % (1 << n)) / (1 << n)) / 2 ** (n / 2)
        F = abs(np.vdot(ref, got)) ** 2 / np.vdot(got, got).real
        assert abs(st.fidelity_qft(x) - F) < 1e-12
    finally:
        st.close()


@pytest.mark.parametrize("dtype", [oracle.C128, oracle.C64])
def test_qft_cross_block_pairing_bit_exact(sv, pool, dtype):
    # small blocks (32 amplitudes) so that most targets, SWAP pairs and controls are high
    n = 12
    stats, _ = run_compare(sv, pool, n, 7, 5, dtype, 1e-6, C.seeded_index(1, n), C.qft(n), every=7)


@pytest.mark.parametrize("dtype", [oracle.C128, oracle.C64])
@pytest.mark.parametrize("eb", [1e-4, 1e-6])
def test_random_brickwork_bit_exact(sv, pool, dtype, eb):
    n = 12
    run_compare(sv, pool, n, 9, 6, dtype, eb, 0, C.random_brickwork(n, 4, seed=21), every=5)


def test_complex64_fine_bound_verbatim_heavy(sv, pool):
    # complex64 at eb 1e-8: the float grid is about as coarse as the quantization grid, so
    # many values are stored verbatim in place; every pass must still match the oracle
    n = 10
    gates = C.qft(n)[:30] + C.random_brickwork(n, 2, seed=6)
    stats, _ = run_compare(sv, pool, n, 9, 7, oracle.C64, 1e-8, C.seeded_index(4, n), gates, every=3)
    assert stats["n_verbatim"] > 0


def test_grover_bit_exact_and_success_probability(sv, pool):
    n, eb = 10, 1e-8
    marked = C.seeded_index(2, n)
    k = 3
    gates = C.grover(n, marked, k)
    st = sv.State(pool, n, 8, eb, oracle.C128, block_log2=6)
    try:
        st.reset_basis(0)
        st.run(gates)
        cs = oracle.CompressedSim(n, 8, 6, oracle.C128, eb, 0).run(gates)
        assert_same_state(st, cs, "grover")
        p = st.probs(list(range(n)))
        theta = math.asin(2.0 ** (-n / 2))
        bound = len(gates) * math.sqrt(2.0 ** (n + 1)) * eb * 1.01
        assert abs(p[marked] - math.sin((2 * k + 1) * theta) ** 2) <= 2 * bound + bound ** 2
    finally:
        st.close()


def random_unitary(rng, d):
    z = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


@pytest.mark.parametrize("dtype", [oracle.C128, oracle.C64])
def test_multi_target_controlled_gates_bit_exact(sv, pool, dtype):
    n, b = 11, 5
    rng = np.random.default_rng(77)
    gates = []
    for _ in range(24):
        k = int(rng.integers(1, 4))
        while True:
            qs = [int(q) for q in rng.permutation(n)]
            t = qs[:k]
            if sum(q >= b for q in t) <= 2:
                break
        nc = int(rng.integers(0, 3))
        gates.append(C.Gate(random_unitary(rng, 1 << k), tuple(t), tuple(qs[k:k + nc]), "U%d" % k))
    run_compare(sv, pool, n, 8, b, dtype, 1e-5, C.seeded_index(9, n), gates, every=4)


def _gate(m, targets, controls=(), name=""):
    return C.Gate(np.asarray(m, dtype=np.complex128), tuple(targets), tuple(controls), name)


def run_compare_reuse(sv, pool, n, b, dtype, eb, x, gates, threads=0, compact=False, chunk=32):
    """run_compare, gate by gate, summing the blocks each pass re-emitted unchanged."""
    st = sv.State(pool, n, n, eb, dtype, block_log2=b)
    reused = 0
    try:
        if threads:
            st.set_threads(threads)
        st.set_compact(compact)
        if chunk != 32:
            st.set_chunk(chunk)
        st.reset_basis(x)
        cs = oracle.CompressedSim(n, n, b, dtype, eb, x, chunk=chunk)
        for i, g in enumerate(gates):
            st.apply(g.matrix, g.targets, g.controls)
            cs.apply(g.matrix, g.targets, g.controls)
            reused += st.stats()["blocks_reused"]
            assert_same_state(st, cs, "gate %d %s" % (i, g.name))
        return reused
    finally:
        st.close()


def test_stream_pass_through_bit_exact(sv, pool):
    # complex128 blocks whose codes a pass provably reproduces (controls above the block not
    # all 1, unit rows, +1 permutations across blocks) re-emit their stream; every pass
    # must still equal the oracle's full recode byte for byte
    n, b = 11, 5
    X = [[0, 1], [1, 0]]
    CNOT_like = [[1, 0, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0], [0, 1, 0, 0]]  # X on t1 when t0 = 1
    gates = C.qft(n)[:40] + [
        _gate(X, (9,), (), "X_high"),
        _gate(X, (7,), (8, 10), "CCX_high"),
        _gate(X, (8,), (2,), "CX_lowctrl"),
        _gate(C.SWAP, (6, 10), (), "SWAP_hh"),
        _gate(C.SWAP, (1, 9), (), "SWAP_lh"),
        _gate(CNOT_like, (7, 9), (), "CX_hh"),
        _gate(CNOT_like, (3, 8), (), "CX_lh"),
        _gate(np.diag([1, 1j]), (10,), (), "S_high"),
        _gate(np.diag([-1, 1]), (6,), (), "Zneg_high"),
        _gate(C.H, (9,), (), "H_high"),
    ] + C.qft(n)[40:80]
    reused = run_compare_reuse(sv, pool, n, b, oracle.C128, 1e-6, C.seeded_index(3, n), gates)
    assert reused > 0


@pytest.mark.parametrize("dtype", [oracle.C128, oracle.C64])
def test_zero_blocks_pass_through_bit_exact(sv, pool, dtype):
    # QFT of a basis state: the early stages leave most blocks all zero, which every gate
    # maps to zero; both precisions re-emit them and still match the oracle
    n, b = 12, 5
    reused = run_compare_reuse(sv, pool, n, b, dtype, 1e-6, C.seeded_index(7, n), C.qft(n)[:30])
    assert reused > 0


def test_pass_through_rejects_verbatim_and_rescaled_blocks(sv, pool):
    # Grover at eb 4e-10 stores the large marked amplitude verbatim (|x| > 2^29 * 2eb), and
    # a non-unitary gate moves sigma far from 1: blocks with a verbatim value or a code
    # beyond the safe range must be recoded, and the result still equals the oracle's
    n, b = 10, 5
    marked = C.seeded_index(12, n)
    gates = C.grover(n, marked, 8)  # marked amplitude sin(17 asin(2^-5)) = 0.51 > 0.43
    gates += [_gate(np.diag([1.0, 0.8]), (9,), (), "shrink"), _gate(np.diag([1, -1]), (2,), (8,), "CZ_hc"),
              _gate([[0, 1], [1, 0]], (7,), (), "X_high")]
    reused = run_compare_reuse(sv, pool, n, b, oracle.C128, 4e-10, 0, gates)
    assert reused > 0


@pytest.mark.parametrize("b", [8, 10])
def test_grover_on_rounding_ties_bit_exact(sv, pool, b):
    # Grover on 12 qubits at eb 1e-6: the uniform superposition 2^-6 sits on rounding ties of
    # the 2e-6 grid, so every value is stored verbatim -- far more than the 128 a complex128
    # block keeps in shared memory. At block_log2 8 the H gates on qubits 8..11 also pair
    # blocks. Every pass must match the oracle byte for byte.
    n = 12
    gates = C.grover(n, C.seeded_index(13, n), 2)
    run_compare_reuse(sv, pool, n, b, oracle.C128, 1e-6, 0, gates)


@pytest.mark.parametrize("threads,compact", [(64, False), (128, False), (256, False), (256, True), (128, True)])
@pytest.mark.parametrize("dtype", [oracle.C128, oracle.C64])
def test_launch_shape_does_not_change_results(sv, pool, threads, compact, dtype):
    # default CTA size 64 at block_log2 10; 128 and 256 idle part of the CTA while decoding;
    # the register-capped build spills but must compute the same bytes
    n, b = 12, 10
    gates = C.qft(n)[:20] + C.random_brickwork(n, 1, seed=8)
    run_compare_reuse(sv, pool, n, b, dtype, 1e-7, C.seeded_index(6, n), gates, threads=threads, compact=compact)


@pytest.mark.parametrize("chunk,b,threads", [(16, 10, 128), (16, 9, 64), (64, 10, 64), (64, 6, 32)])
@pytest.mark.parametrize("dtype", [oracle.C128, oracle.C64])
def test_huffman_chunk_size_bit_exact(sv, pool, chunk, b, threads, dtype):
    # the chunk size changes the stream bytes (its chunk table) but not the decoded values;
    # every pass must equal the oracle run with the same chunk size
    n = 12
    gates = C.qft(n)[:30] + C.random_brickwork(n, 1, seed=3)
    run_compare_reuse(sv, pool, n, b, dtype, 1e-6, C.seeded_index(8, n), gates, threads=threads, chunk=chunk)


def test_huffman_chunk_size_checked(sv, pool):
    st = sv.State(pool, 14, 14, 1e-6, oracle.C128, block_log2=12)  # default CTA: 256 threads
    try:
        for bad in (8, 24, 128, 16):  # 16: 8192 / 16 = 512 chunks > 256 threads
            with pytest.raises(sv.SvError):
                st.set_chunk(bad)
        st.set_chunk(64)
        st.set_chunk(32)
    finally:
        st.close()


def test_cta_size_checked(sv, pool):
    st = sv.State(pool, 12, 12, 1e-6, oracle.C128, block_log2=10)
    try:
        for bad in (16, 32, 48, 512, 1024):
            with pytest.raises(sv.SvError):
                st.set_threads(bad)
        st.set_threads(0)
    finally:
        st.close()


def test_arena_overflow_is_replayed(sv, pool):
    # 20 qubits starting from 2 MiB arenas: the random circuit's streams (about 3.5 MB)
    # outgrow them; sv_sync grows the arena to what the pass asked for and replays, and the
    # result equals the oracle's
    n, b = 20, 12
    gates = C.random_brickwork(n, 2, seed=4)
    stats, _ = run_compare(sv, pool, n, 14, b, oracle.C128, 1e-7, 0, gates, every=len(gates),
                           arena_bytes=2 << 20)
    assert stats["compressed_bytes"] > 2 << 20
    assert stats["replayed_passes"] > 0


@pytest.mark.parametrize("dtype,tol", [(oracle.C128, 1e-12), (oracle.C64, 1e-5)])
def test_plain_path_matches_o1(sv, pool, dtype, tol):
    n = 12
    rng = np.random.default_rng(5)
    gates = C.random_brickwork(n, 3, seed=8) + C.qft(n)
    for _ in range(6):
        qs = [int(q) for q in rng.permutation(n)]
        gates.append(C.Gate(random_unitary(rng, 8), tuple(qs[:3]), (qs[3],), "U3"))
    # the plain kernel's diagonal and permutation forms, with and without controls
    gates += C.grover(n, 1234, 1)
    P3 = np.eye(8, dtype=np.complex128)[[3, 0, 6, 1, 2, 7, 4, 5]]
    D3 = np.diag(np.exp(1j * rng.uniform(0, 2 * np.pi, 8)))
    D3[0, 0] = D3[5, 5] = 1.0
    gates += [C.Gate(P3, (2, 9, 5), (0,), "P3"), C.Gate(P3, (11, 1, 4), (), "P3"),
              C.Gate(D3, (3, 10, 6), (7, 8), "D3"), C.Gate(np.eye(2, dtype=np.complex128), (4,), (), "I"),
              C.Gate(-np.eye(4, dtype=np.complex128), (0, 1), (2,), "-I")]
    st = sv.State(pool, n, n, 0.0, dtype)
    try:
        st.run(gates)
        got = st.read()
        ref = oracle.PlainSim(n, dtype, 0).run(gates).state.astype(np.complex128)
        assert np.abs(got.real - ref.real).max() <= tol and np.abs(got.imag - ref.imag).max() <= tol
        p = st.probs([0, 3, 7])
        pr = np.zeros(8)
        idx = np.arange(1 << n)
        v = ((idx >> 0) & 1) | (((idx >> 3) & 1) << 1) | (((idx >> 7) & 1) << 2)
        np.add.at(pr, v, np.abs(ref) ** 2)
        assert np.abs(p - pr / pr.sum()).max() < 10 * tol
    finally:
        st.close()


def test_fidelity_and_probs_of_compressed_state(sv, pool):
    n = 12
    x = C.seeded_index(3, n)
    gates = C.qft(n)
    a = sv.State(pool, n, 8, 1e-6, oracle.C128)
    p = sv.State(pool, n, n, 0.0, oracle.C128)
    try:
        a.reset_basis(x)
        p.reset_basis(x)
        a.run(gates)
        p.run(gates)
        va, vp = a.read(), p.read()
        F_ref = abs(np.vdot(va, vp)) ** 2 / (np.vdot(va, va).real * np.vdot(vp, vp).real)
        assert abs(a.fidelity(p) - F_ref) < 1e-12
        assert 1 - a.fidelity(p) < 1e-6
        pr = a.probs([0, 1, 11])
        idx = np.arange(1 << n)
        v = (idx & 1) | (((idx >> 1) & 1) << 1) | (((idx >> 11) & 1) << 2)
        ref = np.zeros(8)
        np.add.at(ref, v, np.abs(va) ** 2)
        assert np.abs(pr - ref / ref.sum()).max() < 1e-12
        amps = a.amplitudes([0, 5, 4095])
        assert np.array_equal(amps, va[[0, 5, 4095]])
    finally:
        a.close()
        p.close()


@pytest.mark.parametrize("b,compact", [(10, True), (11, True), (10, False)])
def test_grover20_bench_shape_bit_exact(sv, pool, b, compact):
    # the bench workload at full size (20 qubits, eb 1e-8, complex128) in the launch shapes the
    # autotuner picks: every block stream and the stored norm equal the oracle's after the H
    # layer and after 60 more gates of the dense stage
    n = 20
    gates = C.grover(n, C.seeded_index(11, n))[:80]
    st = sv.State(pool, n, 14, 1e-8, oracle.C128, block_log2=b)
    try:
        st.set_threads(256)
        st.set_compact(compact)
        st.reset_basis(0)
        cs = oracle.CompressedSim(n, 14, b, oracle.C128, 1e-8, 0)
        for i, g in enumerate(gates):
            st.apply(g.matrix, g.targets, g.controls)
            cs.apply(g.matrix, g.targets, g.controls)
            if i + 1 in (20, 50, 80):
                assert_same_state(st, cs, "gate %d" % i)
    finally:
        st.close()


def test_qft30_full_size_properties(sv):
    # 30 qubits (16 GiB uncompressed), the QFT34 path at a size the test box holds: the oracle
    # cannot run it, so properties that hold at any size are checked -- the fidelity against
    # the closed form within the first-order error model (fresh quantization adds about
    # (2/3) eb^2 per value over ~2.5 2^n values; 4x margin), |psi|^2 of sampled amplitudes at
    # 2^-n, a stored norm of 1 within the same error
    n, eb = 30, 1e-7
    x = C.seeded_index(0, n)
    pool = sv.Pool(24 << 30)
    st = sv.State(pool, n, 24, eb, oracle.C128, block_log2=11)
    try:
        st.set_threads(256)
        st.set_compact(True)
        st.reset_basis(x)
        st.run(C.qft(n))
        f = st.fidelity_qft(x)
        model = 2.5 * 2.0 ** n * (2.0 / 3.0) * eb * eb
        assert 1.0 - f < 4 * model, (1.0 - f, model)
        idx = np.random.default_rng(3).integers(0, 1 << n, size=4000, dtype=np.uint64)
        amps = st.amplitudes(idx)
        ratio = np.abs(amps) ** 2 / st.norm() * 2.0 ** n
        assert abs(ratio.mean() - 1.0) < 0.01 and ratio.std() < 0.1
        assert abs(st.norm() - 1.0) < 1e-3
        assert st.stats()["replayed_passes"] < 16
    finally:
        st.close()
        pool.close()


def test_qft22_at_the_qft34_block_shape_bit_exact(sv, pool):
    """The whole QFT22 circuit with the launch shape of the QFT34 workload (2048-amplitude blocks,
    2^20-amplitude slices, complex128, eb 1e-7, 256 threads, register-capped build): targets and
    SWAP partners above the block, controls above the block and the slice, at full block size.
    Streams are compared every 24 passes and at the end, the stored norm after every pass."""
    n, sl, b, eb = 22, 20, 11, 1e-7
    x = C.seeded_index(0, n)
    gates = C.qft(n)
    st = sv.State(pool, n, sl, eb, oracle.C128, block_log2=b)
    try:
        st.set_threads(256)
        st.set_compact(True)
        st.reset_basis(x)
        cs = oracle.CompressedSim(n, sl, b, oracle.C128, eb, x)
        for i, g in enumerate(gates):
            st.apply(g.matrix, g.targets, g.controls)
            cs.apply(g.matrix, g.targets, g.controls)
            assert st.norm() == cs.norm, "gate %d" % i
            if i % 24 == 23 or i == len(gates) - 1:
                assert_same_state(st, cs, "gate %d %s %s %s" % (i, g.name, g.targets, g.controls))
        F = st.fidelity_qft(x)
        print("QFT22 at the QFT34 block shape: 1 - F = %.3e" % (1 - F))
    finally:
        st.close()


@pytest.mark.parametrize("kind", ["qft", "random"])
def test_complex64_fidelity_against_the_fp64_plain_oracle(sv, pool, kind):
    """The FP32 variant's error against FP64: the complex64 compressed state (byte-exact with
    the oracle's complex64 Algorithm 1) compared with the FP64 plain oracle (O1 in complex128)."""
    n, sl, b, eb = 12, 10, 8, 1e-6
    x = C.seeded_index(3, n) if kind == "qft" else 0
    gates = C.qft(n) if kind == "qft" else C.random_brickwork(n, 6, seed=2)
    st = sv.State(pool, n, sl, eb, oracle.C64, block_log2=b)
    try:
        st.reset_basis(x)
        st.run(gates)
        cs = oracle.CompressedSim(n, sl, b, oracle.C64, eb, x).run(gates)
        assert_same_state(st, cs, "end")
        ref = oracle.PlainSim(n, oracle.C128, x).run(gates).state
        got = st.read()
        F = abs(np.vdot(ref, got)) ** 2 / (np.vdot(got, got).real * np.vdot(ref, ref).real)
        # the complex128 run at the same bound, for scale
        st2 = sv.State(pool, n, sl, eb, oracle.C128, block_log2=b)
        st2.reset_basis(x)
        st2.run(gates)
        got2 = st2.read()
        st2.close()
        F2 = abs(np.vdot(ref, got2)) ** 2 / (np.vdot(got2, got2).real * np.vdot(ref, ref).real)
        print("%s%d eb %g: 1 - F complex64 vs FP64 = %.3e, complex128 vs FP64 = %.3e" % (kind, n, eb, 1 - F, 1 - F2))
        # FP32 rounding (2^-24 relative) stays below the bound's quantization error here
        assert 1 - F < 1e-6 and 1 - F < 10 * (1 - F2) + 1e-9
    finally:
        st.close()
