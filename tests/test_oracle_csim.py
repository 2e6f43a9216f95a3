"""Pins for O2, the oracle's Algorithm 1 (for each gate, for each slice: Decompress,
Normalize, GateComputation, Compress).

The paper prints no worked example, so O2 is pinned by what the method implies:
  * on circuits that map the quantization grid onto itself (permutations and sign flips,
    with a state whose stored norm is exactly 1) every pass is exact: the result equals
    the exact state;
  * its results do not depend on how the amplitudes are grouped into slices;
  * the angle between O2's state and O1's grows by at most the norm of each pass's
    quantization error (<= sqrt(2^{n+1}) eb), because unitaries and the global rescale do
    not change angles: 1 - F <= (L sqrt(2^{n+1}) eb (1 + 1e-2))^2;
  * the stored norm stays within that error of 1;
  * QFT of a basis state meets the closed form and Grover meets sin^2((2k+1) theta)."""
import math

import numpy as np
import pytest

import oracle
from paper_1811_05630_gb300 import circuits as C


def fidelity(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return abs(np.vdot(a, b)) ** 2 / (np.vdot(a, a).real * np.vdot(b, b).real)


def test_grid_preserving_circuit_is_exact():
    # eb = 2^-11: the grid is multiples of 2^-10. 256 amplitudes of +-64 * 2^-10 (=1/16):
    # sum q^2 = 2^20 so the stored norm is exactly 1 and sigma = 1.
    n, eb = 10, 2.0 ** -11
    rng = np.random.default_rng(11)
    v = np.zeros(1 << n, dtype=np.complex128)
    idx = rng.choice(1 << n, 256, replace=False)
    signs = rng.choice([-1.0, 1.0], 256)
    v[idx] = np.where(rng.random(256) < 0.5, signs, 1j * signs) / 16
    gates = []
    for _ in range(40):
        kind = rng.integers(5)
        qs = [int(q) for q in rng.permutation(n)]
        if kind == 0:
            gates.append(C.Gate(C.X, (qs[0],), ()))
        elif kind == 1:
            gates.append(C.Gate(C.SWAP, (qs[0], qs[1]), ()))
        elif kind == 2:
            gates.append(C.Gate(C.X, (qs[0],), (qs[1], qs[2])))  # Toffoli
        elif kind == 3:
            gates.append(C.Gate(C.Z, (qs[0],), (qs[1],)))
        else:
            gates.append(C.Gate(np.array([[0, 1j], [1j, 0]]), (qs[0],), ()))  # iX
    for sl in (5, 7, 10):
        cs = oracle.CompressedSim(n, sl, 5, oracle.C128, eb)
        cs.load(v)
        assert cs.norm == 1.0
        ps = oracle.PlainSim(n, oracle.C128, state=v)
        for g in gates:
            cs.apply(g.matrix, g.targets, g.controls)
            ps.apply(g.matrix, g.targets, g.controls)
            assert cs.norm == 1.0
        assert np.array_equal(cs.read(), ps.state)


@pytest.mark.parametrize("dtype", [oracle.C128, oracle.C64])
def test_slice_grouping_does_not_change_streams(dtype):
    n, b = 10, 5
    gates = C.random_brickwork(n, 3, seed=3) + C.qft(n)[:20]
    sims = [oracle.CompressedSim(n, sl, b, dtype, 1e-5, 37) for sl in (5, 6, 8, 10)]
    for g in gates:
        for s in sims:
            s.apply(g.matrix, g.targets, g.controls)
    ref = [sims[0].block_stream(i) for i in range(sims[0].nblocks)]
    for s in sims[1:]:
        assert [s.block_stream(i) for i in range(s.nblocks)] == ref
        assert s.norm == sims[0].norm


@pytest.mark.parametrize("eb", [1e-4, 1e-6])
@pytest.mark.parametrize("circuit", ["qft", "brick"])
def test_fidelity_within_error_propagation_bound(eb, circuit):
    n = 10
    x = C.seeded_index(3, n)
    gates = C.qft(n) if circuit == "qft" else C.random_brickwork(n, 4, seed=1)
    cs = oracle.CompressedSim(n, 8, 6, oracle.C128, eb, x)
    ps = oracle.PlainSim(n, oracle.C128, x)
    per_pass = math.sqrt(2.0 ** (n + 1)) * eb
    for L, g in enumerate(gates, start=1):
        cs.apply(g.matrix, g.targets, g.controls)
        ps.apply(g.matrix, g.targets, g.controls)
        # stored norm within the accumulated error of 1
        assert abs(math.sqrt(cs.norm) - 1.0) <= 2 * per_pass * 1.01
    F = fidelity(cs.read(), ps.state)
    assert 1.0 - F <= (len(gates) * per_pass * 1.01) ** 2


def test_qft12_config_fidelity():
    # 12 qubits, 16 slices of 256 amplitudes, eb = 1e-6
    n = 12
    x = C.seeded_index(0, n)
    cs = oracle.CompressedSim(n, 8, 8, oracle.C128, 1e-6, x).run(C.qft(n))
    ref = np.exp(2j * np.pi * ((x * np.arange(1 << n)) % (1 << n)) / (1 << n)) / 2 ** (n / 2)
    F = fidelity(cs.read(), ref)
    assert 1.0 - F < 1e-6
    assert cs.total_bytes() < 16 * (1 << n)


def test_grover_compressed_success_probability():
    n, eb = 8, 1e-8
    marked = C.seeded_index(4, n)
    k = C.grover_iterations(n)
    gates = C.grover(n, marked, k)
    cs = oracle.CompressedSim(n, 6, 5, oracle.C128, eb, 0).run(gates)
    v = cs.read()
    p = abs(v[marked]) ** 2 / np.vdot(v, v).real
    theta = math.asin(2.0 ** (-n / 2))
    bound = len(gates) * math.sqrt(2.0 ** (n + 1)) * eb * 1.01
    assert abs(p - math.sin((2 * k + 1) * theta) ** 2) <= 2 * bound + bound ** 2


def test_complex64_variant_close_to_fp64():
    n = 10
    gates = C.qft(n)
    x = C.seeded_index(8, n)
    c128 = oracle.CompressedSim(n, 8, 6, oracle.C128, 1e-6, x).run(gates).read()
    c64 = oracle.CompressedSim(n, 8, 6, oracle.C64, 1e-6, x).run(gates).read()
    ps = oracle.PlainSim(n, oracle.C128, x).run(gates).state
    assert 1 - fidelity(c64, ps) < 1e-6
    assert 1 - fidelity(c128, ps) < 1e-6
