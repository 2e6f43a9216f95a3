"""Pins for O2L, the oracle's second mode of Algorithm 1: lazy normalization with slice
skipping. A slice the gate leaves unchanged (controls above the slice not all 1, or a
diagonal gate whose entries for the slice are exactly 1) keeps its stream, and the pass's
normalization sigma = 1/sqrt(N) accumulates in a per-slice scale c_s; the state it stands for
is c_s x'. The pins:
  * with nothing skipped, or with sigma exactly 1, O2L is O2 byte for byte;
  * a skipped slice's stream is unchanged and its scale is c_s sigma, rounded once;
  * one pass equals the normalized gate applied to the represented state, within eb on the
    slices it recodes and to rounding on the slices it skips (an independent tensor
    contraction);
  * the stored norm is the squared norm of the represented state;
  * skipping never costs fidelity against O1 on the paper's workloads."""
import math

import numpy as np
import pytest

import oracle
from paper_1811_05630_gb300 import circuits as C
from test_oracle_plain import apply_by_tensordot


def fidelity(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return abs(np.vdot(a, b)) ** 2 / (np.vdot(a, a).real * np.vdot(b, b).real)


def streams(cs):
    return [cs.block_stream(b) for b in range(cs.nblocks)]


@pytest.mark.parametrize("dtype", [oracle.C128, oracle.C64])
@pytest.mark.parametrize("circuit", ["qft", "brickwork"])
def test_one_slice_is_algorithm_1(dtype, circuit):
    # a single slice: no gate of these circuits is the identity on it, nothing is skipped
    n = 10
    gates = C.qft(n) if circuit == "qft" else C.random_brickwork(n, 4, seed=3)
    a = oracle.CompressedSim(n, n, 6, dtype, 1e-6, 5)
    b = oracle.CompressedSim(n, n, 6, dtype, 1e-6, 5, lazy=True)
    for g in gates:
        a.apply(g.matrix, g.targets, g.controls)
        b.apply(g.matrix, g.targets, g.controls)
        assert b.norm == a.norm
    assert b.skipped == 0
    assert streams(a) == streams(b)
    assert np.all(b.scales() == 1.0)


def test_sigma_one_skips_without_changing_a_byte():
    # eb = 2^-20: the basis state's 1.0 is the code 2^19 on the grid, N = 1 exactly, sigma = 1,
    # and permutations keep the grid: every scale stays 1 while slices are skipped
    n, sl, eb = 10, 6, 2.0 ** -20
    rng = np.random.default_rng(4)
    gates = []
    for _ in range(60):
        qs = [int(q) for q in rng.permutation(n)]
        kind = rng.integers(4)
        if kind == 0:
            gates.append(C.Gate(C.X, (qs[0],), (qs[1],)))
        elif kind == 1:
            gates.append(C.Gate(C.SWAP, (qs[0], qs[1]), (qs[2],)))
        elif kind == 2:
            gates.append(C.Gate(C.Z, (qs[0],), (qs[1],)))
        else:
            gates.append(C.Gate(C.X, (qs[0],), ()))
    a = oracle.CompressedSim(n, sl, 5, oracle.C128, eb, 37)
    b = oracle.CompressedSim(n, sl, 5, oracle.C128, eb, 37, lazy=True)
    for g in gates:
        a.apply(g.matrix, g.targets, g.controls)
        b.apply(g.matrix, g.targets, g.controls)
        assert a.norm == 1.0 and b.norm == 1.0
    assert b.skipped > 0
    assert np.all(b.scales() == 1.0)
    assert streams(a) == streams(b)


def superposition(n, sl, eb, lazy=True, dtype=oracle.C128):
    cs = oracle.CompressedSim(n, sl, 5, dtype, eb, 0, lazy=lazy)
    for q in range(n):
        cs.apply(C.H, (q,), ())
    return cs


@pytest.mark.parametrize("dtype", [oracle.C128, oracle.C64])
def test_skipped_slice_keeps_its_stream_and_takes_sigma(dtype):
    n, sl, eb = 10, 6, 1e-6
    cs = superposition(n, sl, eb, dtype=dtype)
    # a phase controlled by qubit 8 (above the slice): the slices whose bit 2 is 0 are skipped
    for g in [C.Gate(np.diag([1, np.exp(0.3j)]), (2,), (8,)),
              C.Gate(C.H, (0,), (9,)), C.Gate(np.diag([1, 1j]), (7,), ())]:
        before = streams(cs)
        sc = cs.scales()
        N = cs.norm
        sigma = 1.0 / math.sqrt(N)
        skipped = cs.skipped
        cs.apply(g.matrix, g.targets, g.controls)
        after = streams(cs)
        sc2 = cs.scales()
        per = 1 << (sl - 5)
        ctrl_hi = [c for c in g.controls if c >= sl]
        diag_unit_hi = g.matrix.shape == (2, 2) and g.matrix[0, 1] == 0 and g.matrix[1, 0] == 0
        nskip = 0
        for s in range(1 << (n - sl)):
            left = any(not (s >> (c - sl)) & 1 for c in ctrl_hi)
            if not left and diag_unit_hi and g.targets[0] >= sl:
                # a diagonal gate on a qubit above the slice: the slices of the row with entry 1
                bit = (s >> (g.targets[0] - sl)) & 1
                left = g.matrix[bit, bit] == 1
            if left:
                nskip += 1
                assert after[s * per:(s + 1) * per] == before[s * per:(s + 1) * per]
                assert sc2[s] == sc[s] * sigma  # one rounding, in this order
            else:
                assert sc2[s] == 1.0
        assert nskip > 0 and cs.skipped == skipped + nskip


def pending_state(dtype=oracle.C128):
    """A state whose slices carry different pending scales (some skipped once or twice; at
    eb 1.3e-6 the uniform superposition's stored norm is not exactly 1)."""
    n, sl, eb = 10, 6, 1.3e-6
    cs = superposition(n, sl, eb, dtype=dtype)
    cs.apply(np.diag([1, np.exp(0.4j)]), (3,), (8,))
    cs.apply(C.H, (1,), (9,))
    sc = cs.scales()
    assert np.any(sc != 1.0) and np.any(sc == 1.0) and len(set(sc.tolist())) >= 3
    return cs, n, eb


@pytest.mark.parametrize("dtype", [oracle.C128, oracle.C64])
@pytest.mark.parametrize("case", ["dense_low", "controlled_high", "diag_high", "two_high"])
def test_single_pass_is_the_normalized_gate_on_the_represented_state(dtype, case):
    cs, n, eb = pending_state(dtype)
    rng = np.random.default_rng(8)
    if case == "dense_low":
        G, targets, controls = C.haar_unitary(2, rng), (0, 4), ()
    elif case == "controlled_high":
        G, targets, controls = C.haar_unitary(1, rng), (2,), (7,)
    elif case == "diag_high":
        G, targets, controls = np.diag([1, np.exp(1.1j)]), (8,), (1,)
    else:
        G, targets, controls = C.haar_unitary(2, rng), (6, 9), ()
    v = cs.read_values()
    N = cs.norm
    sc = cs.scales()
    ref = apply_by_tensordot(v / math.sqrt(N), n, G, targets, controls)
    cs.apply(G, targets, controls)
    w = cs.read_values()
    sc2 = cs.scales()
    S = 1 << 6
    tol_fp = 1e-6 if dtype == oracle.C64 else 1e-13  # FP32 gate arithmetic on complex64
    for s in range(1 << (n - 6)):
        a, b = w[s * S:(s + 1) * S], ref[s * S:(s + 1) * S]
        if sc2[s] == 1.0:  # recoded: within eb per component (plus the gate's rounding)
            assert np.max(np.abs(a.real - b.real)) <= eb * (1 + 1e-9) + tol_fp
            assert np.max(np.abs(a.imag - b.imag)) <= eb * (1 + 1e-9) + tol_fp
        else:  # skipped: the same values, rescaled
            assert np.max(np.abs(a - b)) <= 1e-14 * max(1.0, np.max(np.abs(b)))
    # the gates on qubits above the slice skip slices; the others recode every slice
    assert np.any(sc2 != 1.0) == (case in ("controlled_high", "diag_high"))


@pytest.mark.parametrize("dtype", [oracle.C128, oracle.C64])
def test_stored_norm_is_the_norm_of_the_represented_state(dtype):
    n, sl = 11, 6
    rng = np.random.default_rng(2)
    cs = oracle.CompressedSim(n, sl, 5, dtype, 1e-6, 3, lazy=True)
    gates = C.random_brickwork(n, 3, seed=7)
    for i in range(30):  # controlled gates with controls above the slice
        t, c = (int(q) for q in rng.choice(n, 2, replace=False))
        gates.append(C.Gate(C.haar_unitary(1, rng), (t,), (max(c, sl),) if max(c, sl) != t else ()))
    # complex64: the stored norm counts the exact codes, the values are their FP32 roundings
    tol = 1e-12 if dtype == oracle.C128 else 1e-6
    for g in gates:
        cs.apply(g.matrix, g.targets, g.controls)
        v = cs.read_values()
        assert abs(cs.norm - np.vdot(v, v).real) <= tol * cs.norm
    assert cs.skipped > 0


@pytest.mark.parametrize("workload", ["qft", "grover"])
def test_skipping_costs_no_fidelity(workload):
    n, sl, b, eb = 12, 8, 6, 1e-6
    if workload == "qft":
        x = C.seeded_index(0, n)
        gates, basis = C.qft(n), x
        ref = np.exp(2j * np.pi * ((x * np.arange(1 << n)) % (1 << n)) / (1 << n)) / 2 ** (n / 2)
    else:
        m = C.seeded_index(11, n)
        gates, basis = C.grover(n, m)[:400], 0
        ref = oracle.PlainSim(n, oracle.C128, 0).run(gates).state
    a = oracle.CompressedSim(n, sl, b, oracle.C128, eb, basis).run(gates)
    z = oracle.CompressedSim(n, sl, b, oracle.C128, eb, basis, lazy=True).run(gates)
    assert z.skipped > 0
    Fa = fidelity(ref, a.read())
    Fz = fidelity(ref, z.read_values())
    assert 1 - Fz <= (1 - Fa) * 1.05 + 1e-12, (1 - Fa, 1 - Fz)


def test_mode_switch_refused_while_a_scale_is_pending():
    cs = superposition(8, 5, 1.3e-6)  # a stored norm other than 1: sigma != 1
    cs.apply(C.H, (0,), (7,))
    assert np.any(cs.scales() != 1.0)
    assert cs._L.orc_csim_set_lazy(cs._h, 0) == -1
