"""Memory accounting the paper reports its results in (host arithmetic only).

Sec. I sizes a full state vector of n qubits at 16 bytes per amplitude (complex double),
2^(n+4) bytes; complex64 amplitudes take half. Sec. IV and V express a compression ratio as
the fraction of that memory the compressed state needs (the abstract's 16.5 % and 2.24e-06)
and as the number of extra qubits the same memory then holds (6x: 2 qubits; 445144x: 18).
"""
from __future__ import annotations

import math

C64 = 1
C128 = 2


def raw_state_bytes(n: int, dtype: int = C128) -> int:
    """Bytes of the uncompressed state: 2^n amplitudes at 16 (complex128) or 8 (complex64)
    bytes each (Sec. I)."""
    if dtype not in (C64, C128):
        raise ValueError("dtype must be C64 (1) or C128 (2)")
    return (16 if dtype == C128 else 8) << n


def compression_ratio(n: int, dtype: int, compressed_bytes: int) -> float:
    """Uncompressed over compressed bytes (every stream byte, metadata included)."""
    if compressed_bytes <= 0:
        raise ValueError("compressed_bytes must be positive")
    return raw_state_bytes(n, dtype) / compressed_bytes


def memory_fraction(ratio: float) -> float:
    """Fraction of the uncompressed memory the compressed state takes (abstract)."""
    if ratio <= 0:
        raise ValueError("ratio must be positive")
    return 1.0 / ratio


def extra_qubits(ratio: float) -> int:
    """Qubits a memory that held the uncompressed state can add at this ratio: every qubit
    doubles the state, so floor(log2(ratio)) (Sec. IV and V)."""
    if ratio < 1:
        return 0
    k = int(math.floor(math.log2(ratio)))
    # guard the floor against log2 rounding at exact powers of two
    while (1 << (k + 1)) <= ratio:
        k += 1
    while k > 0 and (1 << k) > ratio:
        k -= 1
    return k
