"""Pins for O1, the plain FP64/FP32 state-vector oracle (Sec. I: full amplitude-vector
update). Each check compares against something the oracle does not compute itself:
closed forms (QFT, Grover), an independent tensor-contraction construction of the gate,
and unitarity."""
import math

import numpy as np
import pytest

import oracle
from paper_1811_05630_gb300 import circuits as C


def qft_closed_form(n, x):
    # 2^{-n/2} exp(2 pi i (x y mod 2^n) / 2^n), with the product taken in exact integers
    N = 1 << n
    y = np.arange(N, dtype=object)
    ph = np.array([(int(x) * int(v)) % N for v in y], dtype=np.float64) / N
    return np.exp(2j * np.pi * ph) / math.sqrt(N)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 11, 12])
def test_qft_closed_form(n):
    for seed in range(3):
        x = C.seeded_index(seed, n)
        s = oracle.PlainSim(n, oracle.C128, x).run(C.qft(n)).state
        ref = qft_closed_form(n, x)
        assert np.abs(s - ref).max() < 1e-13
        assert np.allclose(np.abs(s), 2.0 ** (-n / 2), atol=1e-14, rtol=0)


def test_qft_gate_count():
    assert len(C.qft(12)) == 12 + 66 + 6
    assert len(C.qft(34)) == 34 + 34 * 33 // 2 + 17


@pytest.mark.parametrize("n", [4, 6, 8, 10])
def test_grover_success_probability(n):
    marked = C.seeded_index(7 + n, n)
    theta = math.asin(2.0 ** (-n / 2))
    kopt = C.grover_iterations(n)
    for k in sorted({1, 2, kopt}):
        s = oracle.PlainSim(n, oracle.C128, 0).run(C.grover(n, marked, k)).state
        p = abs(s[marked]) ** 2
        assert abs(p - math.sin((2 * k + 1) * theta) ** 2) < 1e-12
        assert abs(np.vdot(s, s).real - 1.0) < 1e-12


def apply_by_tensordot(state, n, G, targets, controls):
    """Independent construction: view the state as an n-axis tensor (axis n-1-q is qubit q),
    select the sub-tensor where every control is 1 and contract G over the target axes."""
    psi = state.reshape((2,) * n).copy()
    k = len(targets)
    Gt = G.reshape((2,) * (2 * k))  # axes: out bits k-1..0, in bits k-1..0
    sl = [slice(None)] * n
    for c in controls:
        sl[n - 1 - c] = 1
    sub = psi[tuple(sl)]
    # axes of `sub`: the remaining qubits in decreasing order
    rem = [q for q in range(n - 1, -1, -1) if q not in controls]
    tax = [rem.index(targets[l]) for l in range(k - 1, -1, -1)]  # target t_{k-1} .. t_0
    out = np.tensordot(Gt, sub, axes=(list(range(k, 2 * k)), tax))
    # out axes: k output target axes (t_{k-1}..t_0) then the rest of `sub` in order
    rest = [a for a in range(sub.ndim) if a not in tax]
    perm = [0] * sub.ndim
    for i, a in enumerate(tax):
        perm[a] = i
    for i, a in enumerate(rest):
        perm[a] = k + i
    psi[tuple(sl)] = np.transpose(out, perm)
    return psi.reshape(-1)


def random_unitary(rng, d):
    z = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


@pytest.mark.parametrize("n", [3, 5, 6, 7])
def test_dense_bruteforce(n):
    # gates on up to five targets (2^k x 2^k matrices, k <= 5), with controls
    rng = np.random.default_rng(100 + n)
    v = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    v /= np.linalg.norm(v)
    sim = oracle.PlainSim(n, oracle.C128, state=v)
    ref = v.copy()
    for _ in range(25):
        k = int(rng.integers(1, min(5, n - 1) + 1))
        qs = rng.permutation(n)
        targets = tuple(int(q) for q in qs[:k])
        nc = int(rng.integers(0, n - k + 1))
        controls = tuple(int(q) for q in qs[k:k + nc])
        G = random_unitary(rng, 1 << k)
        sim.apply(G, targets, controls)
        ref = apply_by_tensordot(ref, n, G, targets, controls)
        assert np.abs(sim.state - ref).max() < 1e-13


def test_single_qubit_kron():
    # U = I_{2^{n-1-t}} (x) G (x) I_{2^t} for an uncontrolled single-qubit gate
    n = 5
    rng = np.random.default_rng(3)
    for t in range(n):
        G = random_unitary(rng, 2)
        U = np.kron(np.kron(np.eye(1 << (n - 1 - t)), G), np.eye(1 << t))
        v = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
        sim = oracle.PlainSim(n, oracle.C128, state=v)
        sim.apply(G, (t,))
        assert np.abs(sim.state - U @ v).max() < 1e-13


def test_unit_norm_random_circuit():
    n = 10
    s = oracle.PlainSim(n, oracle.C128, 0).run(C.random_brickwork(n, 8, seed=5)).state
    assert abs(np.vdot(s, s).real - 1.0) < 1e-13


def test_complex64_within_fp32_tolerance():
    n = 10
    g = C.random_brickwork(n, 6, seed=9)
    s128 = oracle.PlainSim(n, oracle.C128, 0).run(g).state
    s64 = oracle.PlainSim(n, oracle.C64, 0).run(g).state
    assert s64.dtype == np.complex64
    assert np.abs(s64.astype(np.complex128) - s128).max() < 1e-5


# ---- gate fusion (host-side circuit transformation) ----------------------------------------

def test_expand_places_controls_and_targets():
    from paper_1811_05630_gb300 import circuits as C

    # CZ as a controlled Z on (target 3, control 1) inside qubits (1, 3): diag(1, 1, 1, -1)
    M = C.expand(C.Z, (3,), (1,), (1, 3))
    assert np.array_equal(M, np.diag([1, 1, 1, -1]).astype(complex))
    # X on qubit 5 embedded as the high bit of (2, 5): swaps index pairs differing in bit 1
    M = C.expand(C.X, (5,), (), (2, 5))
    assert np.array_equal(M, np.kron(C.X, np.eye(2)))


@pytest.mark.parametrize("seed", [0, 1])
def test_fused_circuit_equals_the_original_on_the_plain_oracle(seed):
    from paper_1811_05630_gb300 import circuits as C

    n = 10
    gates = C.random_brickwork(n, 5, seed=seed) + C.qft(n)
    fused = C.fuse(gates, 5, block_log2=6)
    assert len(fused) < len(gates) / 3 and C.unfused_count(fused) == len(gates)
    for g in fused:
        assert g.k + len(g.controls) <= 5 and sum(1 for q in g.targets + g.controls if q >= 6) <= 2
        U = g.matrix
        assert np.allclose(U.conj().T @ U, np.eye(U.shape[0]), atol=1e-12)
    a = oracle.PlainSim(n, oracle.C128, 3).run(gates).state
    b = oracle.PlainSim(n, oracle.C128, 3).run(fused).state
    assert np.max(np.abs(a - b)) < 1e-12


def test_haar_unitary_is_unitary_and_seeded():
    from paper_1811_05630_gb300 import circuits as C

    U = C.haar_unitary(5, np.random.default_rng(1))
    assert U.shape == (32, 32) and np.allclose(U.conj().T @ U, np.eye(32), atol=1e-12)
    assert np.array_equal(U, C.haar_unitary(5, np.random.default_rng(1)))
