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
from test_oracle_plain import apply_by_tensordot, random_unitary


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


@pytest.mark.parametrize("scale,sigma", [(2.0, 0.5), (0.5, 2.0)])
def test_normalize_rescales_by_inverse_sqrt_of_stored_norm(scale, sigma):
    # Alg. 1 Normalize: y = x' / sqrt(N) with N the stored norm. On the grid of eb = 2^-11
    # (multiples of 2^-10), 256 amplitudes of +-scale/16 store N = scale^2 exactly; sigma is
    # then a power of two and the pass after an X gate is exact: every value scales by sigma.
    n, eb = 10, 2.0 ** -11
    rng = np.random.default_rng(5)
    v = np.zeros(1 << n, dtype=np.complex128)
    idx = rng.choice(1 << n, 256, replace=False)
    signs = rng.choice([-1.0, 1.0], 256)
    v[idx] = np.where(rng.random(256) < 0.5, signs, 1j * signs) * scale / 16
    cs = oracle.CompressedSim(n, 7, 5, oracle.C128, eb)
    cs.load(v)
    assert cs.norm == scale * scale
    for t in (2, 8):  # a target inside a slice, then one above the slice
        cs.apply(C.X, (t,))
        v = apply_by_tensordot(v, n, C.X, (t,), ())
        assert np.array_equal(cs.read(), v * sigma)
        assert cs.norm == 1.0
        v = v * sigma
        sigma = 1.0


SINGLE_PASS_GATES = [
    ("1q low target", 1, (2,), ()),
    ("1q target above the slice", 1, (7,), ()),
    ("2q across slices", 2, (1, 8), ()),
    ("controlled, control above the slice", 1, (3,), (8,)),
    ("two controls", 1, (0,), (4, 6)),
    ("3q", 3, (5, 0, 7), ()),
]


@pytest.mark.parametrize("dtype", [oracle.C128, oracle.C64])
@pytest.mark.parametrize("case", SINGLE_PASS_GATES, ids=[c[0] for c in SINGLE_PASS_GATES])
def test_single_pass_is_normalized_gate_within_bound(dtype, case):
    # One pass of Alg. 1 on a state whose stored norm N is not 1: every amplitude after the
    # pass lies within eb (per component) of (G y)_i, y = x' / sqrt(N), x' the decompressed
    # values before the pass, computed here by an independent tensor contraction; amplitudes
    # the gate leaves alone (controls unset) are rescaled too, since every slice goes through
    # the cycle. The new stored norm is the squared norm of the stored values.
    _, k, targets, controls = case
    n, sl, b = 9, 6, 5
    eb = 1e-6 if dtype == oracle.C128 else 1e-4
    rng = np.random.default_rng(40 + k + len(controls))
    v = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    v *= 1.7 / np.linalg.norm(v)
    G = random_unitary(rng, 1 << k)
    cs = oracle.CompressedSim(n, sl, b, dtype, eb)
    cs.load(v)
    x = cs.read().astype(np.complex128)
    N = cs.norm
    # N is the norm of the stored grid values q 2eb; complex64 decodes them rounded to float
    rel = 1e-12 if dtype == oracle.C128 else 2.0 ** -22
    assert abs(N - np.vdot(x, x).real) <= rel * N
    assert abs(N - 1.7 ** 2) < 1e-3
    cs.apply(G, targets, controls)
    y = apply_by_tensordot(x / math.sqrt(N), n, G, targets, controls)
    got = cs.read().astype(np.complex128)
    # FP arithmetic of the pass (FP64, or FP32 for complex64) on top of the quantization bound
    fp = (1e-15 if dtype == oracle.C128 else 6e-7) * (2 ** k) * np.abs(x).max() / math.sqrt(N)
    assert np.abs(got.real - y.real).max() <= eb + fp
    assert np.abs(got.imag - y.imag).max() <= eb + fp
    assert abs(cs.norm - np.vdot(got, got).real) <= rel * cs.norm
    # the bound is tight enough to see a wrong scale: 1/N instead of 1/sqrt(N) misses by far more
    wrong = apply_by_tensordot(x / N, n, G, targets, controls)
    assert np.abs(got - wrong).max() > 100 * eb


@pytest.mark.parametrize("dtype", [oracle.C128, oracle.C64])
def test_stored_norm_counts_verbatim_values(dtype):
    # Values with |x r| >= 2^29 are stored raw (verbatim). The stored norm N must still be the
    # squared norm of every stored value, the raw ones included; and a pass over such a state
    # rescales them like the rest.
    n, sl, b = 8, 6, 5
    eb = 1e-10 if dtype == oracle.C128 else 2e-8
    lim = 2.0 ** 29 * 2 * eb  # the largest magnitude the quantizer takes
    rng = np.random.default_rng(17)
    v = (rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)) * lim / 8
    big = rng.choice(1 << n, 12, replace=False)
    v[big] = (3 + rng.random(12)) * lim * np.exp(2j * np.pi * rng.random(12))
    cs = oracle.CompressedSim(n, sl, b, dtype, eb)
    cs.load(v)
    x = cs.read().astype(np.complex128)
    rel = 1e-12 if dtype == oracle.C128 else 2.0 ** -22
    if dtype == oracle.C128:
        assert np.array_equal(x[big], v[big])  # raw values come back exactly
    N = cs.norm
    assert abs(N - np.vdot(x, x).real) <= rel * N
    # the raw values carry most of the norm, so dropping them would miss by far more than rel
    assert np.vdot(x[big], x[big]).real > 0.5 * N
    cs.apply(C.X, (1,))
    y = apply_by_tensordot(x / math.sqrt(N), n, C.X, (1,), ())
    got = cs.read().astype(np.complex128)
    fp = (1e-15 if dtype == oracle.C128 else 6e-7) * np.abs(y).max()
    assert np.abs(got - y).max() <= math.sqrt(2) * eb + fp
    assert abs(cs.norm - np.vdot(got, got).real) <= rel * cs.norm


@pytest.mark.parametrize("n,eb", [(10, 1e-5), (12, 1e-6), (13, 1e-7)])
def test_qft_infidelity_matches_the_first_order_model(n, eb):
    # Rounding to the 2eb grid adds a uniform error in [-eb, eb] to each component of every
    # freshly quantized value: eb^2/3 per component, (2/3) eb^2 per complex value, almost all
    # of it orthogonal to the state. QFT of a basis state freshly quantizes about 2.5 * 2^n
    # values over the circuit (each stage's H, and the controlled phases where the control is
    # set; SWAPs and identities stay on the grid), so 1 - F ~ 2.5 * 2^n * (2/3) eb^2. O2 must
    # land within 20 % of it (truncating instead of rounding would quadruple it).
    x = C.seeded_index(0, n)
    cs = oracle.CompressedSim(n, 8, 8, oracle.C128, eb, x).run(C.qft(n))
    ref = np.exp(2j * np.pi * ((x * np.arange(1 << n)) % (1 << n)) / (1 << n)) / 2 ** (n / 2)
    measured = 1.0 - fidelity(cs.read(), ref)
    model = 2.5 * (1 << n) * (2.0 / 3.0) * eb * eb
    assert 0.8 < measured / model < 1.2, (measured, model)


def test_stored_norm_beyond_64_bits():
    # codes near the quantizer's limit (|q| ~ 2^28): Σq² over 2^10 values exceeds 2^64, so the
    # exact integer sum needs its high word; N must still be the squared norm of the values
    n, sl, b = 9, 9, 8
    eb = 2.0 ** -11
    lim = 2.0 ** 29 / 2.0 ** 10
    rng = np.random.default_rng(29)
    v = (rng.uniform(0.4, 0.9, 1 << n) * np.exp(2j * np.pi * rng.random(1 << n))) * lim
    cs = oracle.CompressedSim(n, sl, b, oracle.C128, eb)
    cs.load(v)
    x = cs.read()
    q2 = np.sum(np.round(x.real * 2 ** 10) ** 2 + np.round(x.imag * 2 ** 10) ** 2)
    assert q2 > 2.0 ** 64
    N = cs.norm
    assert abs(N - np.vdot(x, x).real) <= 1e-12 * N
