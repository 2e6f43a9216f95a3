"""GB300-native compressed state-vector simulator (per-gate slice update of Algorithm 1 of
Wu et al., "Memory-Efficient Quantum Circuit Simulation by Using Lossy Data Compression").

The compute path is the CUDA library ``libsv.so`` (built from ``csrc/``); ``sv`` is its thin
ctypes binding. Importing this package does not load the library; ``paper_1811_05630_gb300.sv``
does, and fails loudly when it is missing.
"""
__all__ = ["circuits", "sv"]
