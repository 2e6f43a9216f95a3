"""Seeded synthetic circuits: the workloads the simulator is measured on.

This module generates inputs only. It holds none of the simulator's arithmetic (no
quantization, coding, normalization or gate application): it emits lists of gates
(FP64 matrices computed on the host, target and control qubits) that the CUDA path and
the CPU oracle consume identically.

Workload shapes follow the paper's evaluation (Sec. III): the Quantum Fourier Transform
and Grover's search, plus random brickwork circuits as a poorly compressible stress case.
Qubit q is bit q of the amplitude index (little-endian). A gate's targets[0] is the least
significant bit of its matrix's basis index.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np


@dataclass(frozen=True)
class Gate:
    matrix: np.ndarray            # complex128, shape (2^k, 2^k)
    targets: Tuple[int, ...]
    controls: Tuple[int, ...] = ()
    name: str = ""

    @property
    def k(self) -> int:
        return len(self.targets)


S2 = 1.0 / math.sqrt(2.0)
H = np.array([[S2, S2], [S2, -S2]], dtype=np.complex128)
X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
SWAP = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=np.complex128)


def phase(m: int) -> np.ndarray:
    """R_m = diag(1, exp(2 pi i / 2^m))."""
    a = 2.0 * math.pi / float(1 << m)
    return np.array([[1, 0], [0, complex(math.cos(a), math.sin(a))]], dtype=np.complex128)


def splitmix64(x: int) -> int:
    """SplitMix64 output for state x (published constants of the SplitMix64 generator)."""
    x = (x + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
    z = x
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
    return z ^ (z >> 31)


def seeded_index(seed: int, n: int) -> int:
    """A seeded uniformly random n-bit basis index."""
    return splitmix64(seed) & ((1 << n) - 1)


def qft(n: int) -> List[Gate]:
    """QFT on n qubits: H, then controlled R_m from every less significant qubit, for each
    qubit from the most significant down; then the bit-reversal SWAPs.
    On |x> it produces 2^{-n/2} sum_y exp(2 pi i x y / 2^n) |y>.
    Gate count: n + n(n-1)/2 + floor(n/2)."""
    gates: List[Gate] = []
    for j in range(n - 1, -1, -1):
        gates.append(Gate(H, (j,), (), "H"))
        for k in range(j - 1, -1, -1):
            gates.append(Gate(phase(j - k + 1), (j,), (k,), "CR%d" % (j - k + 1)))
    for i in range(n // 2):
        gates.append(Gate(SWAP, (i, n - 1 - i), (), "SWAP"))
    return gates


def grover_iterations(n: int) -> int:
    return int(math.floor(math.pi / 4.0 * math.sqrt(float(1 << n))))


def _mcz(n: int) -> Gate:
    """Z on qubit 0 controlled by qubits 1..n-1: a phase flip of |1...1>."""
    return Gate(Z, (0,), tuple(range(1, n)), "MCZ")


def grover(n: int, marked: int, iterations: int | None = None) -> List[Gate]:
    """Grover search: H on every qubit, then `iterations` rounds of
    oracle (X on the zero bits of `marked`, MCZ, X) and diffusion (H^n X^n MCZ X^n H^n)."""
    if iterations is None:
        iterations = grover_iterations(n)
    zeros = [q for q in range(n) if not (marked >> q) & 1]
    gates: List[Gate] = [Gate(H, (q,), (), "H") for q in range(n)]
    for _ in range(iterations):
        gates += [Gate(X, (q,), (), "X") for q in zeros]
        gates.append(_mcz(n))
        gates += [Gate(X, (q,), (), "X") for q in zeros]
        gates += [Gate(H, (q,), (), "H") for q in range(n)]
        gates += [Gate(X, (q,), (), "X") for q in range(n)]
        gates.append(_mcz(n))
        gates += [Gate(X, (q,), (), "X") for q in range(n)]
        gates += [Gate(H, (q,), (), "H") for q in range(n)]
    return gates


def haar_su2(rng: np.random.Generator) -> np.ndarray:
    """Haar-random SU(2) from a normalized 4-Gaussian quaternion (a, b, c, d):
    [[a + ib, c + id], [-c + id, a - ib]]."""
    v = rng.standard_normal(4)
    a, b, c, d = v / np.linalg.norm(v)
    return np.array([[complex(a, b), complex(c, d)], [complex(-c, d), complex(a, -b)]], dtype=np.complex128)


def random_brickwork(n: int, depth: int, seed: int) -> List[Gate]:
    """Each layer: a Haar SU(2) on every qubit, then CZ on nearest-neighbour pairs starting
    at qubit 0 on even layers and at qubit 1 on odd layers."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gates: List[Gate] = []
    for layer in range(depth):
        for q in range(n):
            gates.append(Gate(haar_su2(rng), (q,), (), "U"))
        for q in range(layer % 2, n - 1, 2):
            gates.append(Gate(Z, (q + 1,), (q,), "CZ"))
    return gates


def expand(matrix: np.ndarray, targets: Sequence[int], controls: Sequence[int], qubits: Sequence[int]) -> np.ndarray:
    """The gate (matrix on `targets`, applied where every control is 1) as a dense matrix on
    `qubits` (a superset of targets and controls; qubits[0] is the least significant bit of
    the result's basis index)."""
    k = len(qubits)
    pos = {q: i for i, q in enumerate(qubits)}
    tb = [pos[t] for t in targets]
    cmask = sum(1 << pos[c] for c in controls)
    tmask = sum(1 << b for b in tb)
    M = np.zeros((1 << k, 1 << k), dtype=np.complex128)
    for x in range(1 << k):
        if (x & cmask) != cmask:
            M[x, x] = 1.0
            continue
        xt = sum(((x >> b) & 1) << i for i, b in enumerate(tb))
        rest = x & ~tmask
        for yt in range(1 << len(tb)):
            y = rest | sum(((yt >> i) & 1) << b for i, b in enumerate(tb))
            M[y, x] = matrix[yt, xt]
    return M


def fuse(gates: Sequence[Gate], max_qubits: int = 5, block_log2: int | None = None,
         max_high: int = 2) -> List[Gate]:
    """Gate fusion: consecutive gates merged into dense unitaries on at most `max_qubits`
    qubits (with at most `max_high` of them at or above `block_log2`, the number of coupled
    blocks a pass can hold). A gate joins the latest group it shares a qubit with when the union
    fits, else a later group (it commutes with every group after the last one it shares a qubit
    with), else it starts a group. A group of one gate is emitted unchanged; others become one
    gate on the sorted union of their qubits, named FUSED<count>, with the matrix product
    computed here once in FP64 (the simulators consume the resulting matrices as given)."""
    groups: List[dict] = []

    def high(qs):
        return 0 if block_log2 is None else sum(1 for q in qs if q >= block_log2)

    for g in gates:
        Q = set(g.targets) | set(g.controls)
        last = -1
        for i in range(len(groups) - 1, -1, -1):
            if groups[i]["qubits"] & Q:
                last = i
                break
        choice = -1
        for i in [last] + list(range(len(groups) - 1, last, -1)) if last >= 0 else range(len(groups) - 1, -1, -1):
            u = groups[i]["qubits"] | Q
            if len(u) <= max_qubits and high(u) <= max_high:
                choice = i
                break
        if choice < 0:
            groups.append({"qubits": set(Q), "gates": [g]})
        else:
            groups[choice]["qubits"] |= Q
            groups[choice]["gates"].append(g)
    out: List[Gate] = []
    for grp in groups:
        if len(grp["gates"]) == 1:
            out.append(grp["gates"][0])
            continue
        qs = sorted(grp["qubits"])
        U = np.eye(1 << len(qs), dtype=np.complex128)
        for g in grp["gates"]:
            U = expand(g.matrix, g.targets, g.controls, qs) @ U
        out.append(Gate(U, tuple(qs), (), "FUSED%d" % len(grp["gates"])))
    return out


def unfused_count(gates: Sequence[Gate]) -> int:
    """Gates of the original circuit a (possibly fused) gate list stands for."""
    return sum(int(g.name[5:]) if g.name.startswith("FUSED") else 1 for g in gates)


def haar_unitary(k: int, rng: np.random.Generator) -> np.ndarray:
    """A Haar-random 2^k x 2^k unitary: QR of a complex Gaussian matrix with the phases of R's
    diagonal moved into Q."""
    d = 1 << k
    z = (rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    ph = np.diag(r) / np.abs(np.diag(r))
    return np.ascontiguousarray(q * ph[None, :])


def count_amplitude_updates(n: int, gates: Sequence[Gate]) -> int:
    """Amplitude-updates of a circuit: 2^n per (unfused) gate."""
    return (1 << n) * len(gates)


@dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the stream
    kind: str               # "qft" | "grover" | "random"
    n: int
    dtype: int              # 1 complex64, 2 complex128
    eb: float
    basis: int
    gates: List[Gate] = field(default_factory=list)

    @property
    def amp_updates(self) -> int:
        return (1 << self.n) * len(self.gates)


def serving_requests(count: int = 2000, rate: float = 20.0, seed: int = 0, nmin: int = 10,
                     nmax: int = 28) -> List[Request]:
    """Seeded Poisson arrivals (mean `rate` per second); each request uniformly one of QFT on
    a random basis state, Grover with a random marked item and 1-8 iterations, or a random
    brickwork circuit of depth 4-16; qubits uniform in [nmin, nmax]; complex64 or complex128
    at equal odds; absolute error bound from {1e-4, 1e-6, 1e-8}."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out: List[Request] = []
    for rid in range(count):
        t += float(rng.exponential(1.0 / rate))
        kind = ["qft", "grover", "random"][int(rng.integers(3))]
        n = int(rng.integers(nmin, nmax + 1))
        dtype = 1 if rng.random() < 0.5 else 2
        eb = [1e-4, 1e-6, 1e-8][int(rng.integers(3))]
        sub = int(rng.integers(1 << 62))
        if kind == "qft":
            basis = sub & ((1 << n) - 1)
            gates = qft(n)
        elif kind == "grover":
            basis = 0
            gates = grover(n, sub & ((1 << n) - 1), int(rng.integers(1, 9)))
        else:
            basis = 0
            gates = random_brickwork(n, int(rng.integers(4, 17)), seed=sub)
        out.append(Request(rid, t, kind, n, dtype, eb, basis, gates))
    return out
