"""Seeded synthetic codec blocks shaped like the simulator's data (shared by the oracle pins
and the GPU parity tests; generates inputs only)."""
import numpy as np

import oracle


def gen_block(kind, b, rng, dtype):
    B = 1 << b
    if kind == "normal":
        v = (rng.standard_normal(B) + 1j * rng.standard_normal(B)) * 1e-3
    elif kind == "qft":  # unit-modulus phases scaled like a 2^-n/2 amplitude
        ph = rng.uniform(0, 2 * np.pi) + np.arange(B) * rng.uniform(0, 2 * np.pi)
        v = np.exp(1j * ph) * 2.0 ** -8
    elif kind == "grover":  # one value almost everywhere, a spike
        v = np.full(B, 2.0 ** -10 + 0j)
        v[rng.integers(B)] = 0.7
    elif kind == "walsh":  # +-c sign patterns: large Lorenzo deltas (escapes)
        v = 0.01 * (1 - 2 * (np.arange(B) & 1)) + 0j
    elif kind == "zeros":
        v = np.zeros(B, dtype=np.complex128)
    elif kind == "const":
        v = np.full(B, 0.125 - 0.25j)
    elif kind == "wide":  # many distinct symbols: forces PACK
        v = (rng.standard_normal(B) + 1j * rng.standard_normal(B)) * 0.05
    else:
        raise ValueError(kind)
    return v.astype(np.complex64 if dtype == oracle.C64 else np.complex128)


KINDS = ["normal", "qft", "grover", "walsh", "zeros", "const", "wide"]
