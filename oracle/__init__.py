"""CPU oracle for the compressed state-vector simulator — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package. The product (``paper_1811_05630_gb300``) never imports it, and the two
share no code: this package wraps ``sv_oracle.c`` (plain C, FP64/FP32 IEEE operations in
the written order, ``-ffp-contract=off``) through ctypes.

Paper: Wu et al., "Memory-Efficient Quantum Circuit Simulation by Using Lossy Data
Compression" (PMES 2018).
  * ``PlainSim``       — O1, the "original simulator": full amplitude-vector update (Sec. I).
  * ``compress_block`` / ``decompress_block`` — the SZ-style block codec (Sec. II).
  * ``CompressedSim``  — O2, Algorithm 1 (Decompress, Normalize, GateComputation,
    Compress for every slice, gate by gate); with ``lazy=True`` the second mode O2L: slices
    a gate leaves unchanged keep their streams and hold their pending normalization as a
    per-slice scale (see sv_oracle.h).
  * ``huffman_lengths`` — the two-queue Huffman code lengths the codec uses.

Parity pins (tests/test_oracle_*.py) check every function here against closed forms,
invariants, brute force and an independent textbook Huffman. The paper prints no value of
O2's output; a single O2 pass is pinned element by element against the normalized gate
(G x' / sqrt(N), by an independent tensor contraction) within eb, exactly on power-of-two
norms, and whole circuits by exactness on grid-preserving circuits, grouping invariance and
a fidelity bound against O1.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sv_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

C64 = 1
C128 = 2
MODE_CONST, MODE_HUFF, MODE_PACK = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile sv_oracle.c into liboracle.so next to it (plain gcc, no FMA contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "sv_oracle.h"))
    ):
        tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
        cmd = [
            "gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
            "-shared", "-o", tmp, _SRC, "-lm",
        ]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _BlockInfo(ctypes.Structure):
    _fields_ = [
        ("mode", ctypes.c_int),
        ("n_verbatim", ctypes.c_int),
        ("n_escape", ctypes.c_int),
        ("n_distinct", ctypes.c_int),
        ("sq_lo", ctypes.c_uint64),
        ("sq_hi", ctypes.c_uint64),
        ("vsum", ctypes.c_double),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        L = ctypes.CDLL(_LIB_PATH)
        vp, i, d, u64, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_uint64, ctypes.c_size_t
        L.orc_block_bound.argtypes = [i, i]
        L.orc_block_bound.restype = sz
        L.orc_compress_block.argtypes = [vp, i, i, d, vp, ctypes.POINTER(_BlockInfo)]
        L.orc_compress_block.restype = sz
        L.orc_decompress_block.argtypes = [vp, sz, i, i, d, vp]
        L.orc_decompress_block.restype = i
        L.orc_compress_block_k.argtypes = [vp, i, i, d, i, vp, ctypes.POINTER(_BlockInfo)]
        L.orc_compress_block_k.restype = sz
        L.orc_decompress_block_k.argtypes = [vp, sz, i, i, d, i, vp]
        L.orc_decompress_block_k.restype = i
        L.orc_csim_create_k.argtypes = [i, i, i, i, d, u64, i]
        L.orc_csim_create_k.restype = vp
        L.orc_huffman_lengths.argtypes = [vp, vp, i, vp]
        L.orc_huffman_lengths.restype = i
        L.orc_plain_apply.argtypes = [vp, i, i, vp, vp, i, vp, i]
        L.orc_plain_apply.restype = None
        L.orc_csim_create.argtypes = [i, i, i, i, d, u64]
        L.orc_csim_create.restype = vp
        L.orc_csim_destroy.argtypes = [vp]
        L.orc_csim_apply.argtypes = [vp, vp, vp, i, vp, i]
        L.orc_csim_apply.restype = i
        L.orc_csim_read.argtypes = [vp, vp]
        L.orc_csim_norm.argtypes = [vp]
        L.orc_csim_norm.restype = d
        L.orc_csim_nblocks.argtypes = [vp]
        L.orc_csim_nblocks.restype = u64
        L.orc_csim_block_stream.argtypes = [vp, u64, ctypes.POINTER(ctypes.c_void_p)]
        L.orc_csim_block_stream.restype = sz
        L.orc_csim_total_bytes.argtypes = [vp]
        L.orc_csim_total_bytes.restype = u64
        L.orc_csim_load.argtypes = [vp, vp]
        L.orc_csim_set_lazy.argtypes = [vp, i]
        L.orc_csim_set_lazy.restype = i
        L.orc_csim_scales.argtypes = [vp, vp]
        L.orc_csim_skipped.argtypes = [vp]
        L.orc_csim_skipped.restype = u64
        L.orc_csim_read_values.argtypes = [vp, vp]
        _lib = L
        return L


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _cdtype(dtype: int):
    return np.complex64 if dtype == C64 else np.complex128


def block_bound(block_log2: int, dtype: int) -> int:
    return int(_load().orc_block_bound(block_log2, dtype))


def compress_block(values: np.ndarray, block_log2: int, dtype: int, eb: float, chunk: int = 32):
    """Compress 2^block_log2 complex amplitudes; returns (stream bytes, info dict). `chunk`:
    Huffman symbols per stored chunk bit count (16, 32 or 64)."""
    L = _load()
    v = np.ascontiguousarray(values, dtype=_cdtype(dtype))
    assert v.size == 1 << block_log2
    out = np.zeros(block_bound(block_log2, dtype), dtype=np.uint8)
    info = _BlockInfo()
    n = L.orc_compress_block_k(_ptr(v), block_log2, dtype, eb, chunk, _ptr(out), ctypes.byref(info))
    if n == 0:
        raise ValueError("orc_compress_block rejected its arguments")
    d = {f: getattr(info, f) for f, _ in _BlockInfo._fields_}
    return out[:n].tobytes(), d


def decompress_block(stream: bytes, block_log2: int, dtype: int, eb: float, chunk: int = 32) -> np.ndarray:
    L = _load()
    buf = np.frombuffer(stream, dtype=np.uint8).copy()
    out = np.zeros(1 << block_log2, dtype=_cdtype(dtype))
    rc = L.orc_decompress_block_k(_ptr(buf), buf.size, block_log2, dtype, eb, chunk, _ptr(out))
    if rc != 0:
        raise ValueError("malformed block stream (%d)" % rc)
    return out


def huffman_lengths(freqs, syms=None) -> np.ndarray:
    L = _load()
    f = np.ascontiguousarray(freqs, dtype=np.uint32)
    s = np.arange(f.size, dtype=np.uint32) if syms is None else np.ascontiguousarray(syms, dtype=np.uint32)
    out = np.zeros(f.size, dtype=np.int32)
    L.orc_huffman_lengths(_ptr(f), _ptr(s), f.size, _ptr(out))
    return out


def _gate_arrays(G, targets, controls):
    G = np.ascontiguousarray(np.asarray(G, dtype=np.complex128))
    t = np.ascontiguousarray(np.asarray(targets, dtype=np.int32))
    c = np.ascontiguousarray(np.asarray(list(controls) if controls else [0], dtype=np.int32))
    nc = len(controls) if controls else 0
    assert G.shape == (1 << t.size, 1 << t.size)
    return G, t, c, nc


class PlainSim:
    """O1: plain state vector (complex128 with FP64 gates, or complex64 with FP32 gates)."""

    def __init__(self, n: int, dtype: int = C128, basis_index: int = 0, state=None):
        self.n, self.dtype = n, dtype
        if state is not None:
            self.state = np.ascontiguousarray(state, dtype=_cdtype(dtype)).copy()
        else:
            self.state = np.zeros(1 << n, dtype=_cdtype(dtype))
            self.state[basis_index] = 1.0

    def apply(self, G, targets, controls=()):
        G, t, c, nc = _gate_arrays(G, targets, controls)
        _load().orc_plain_apply(_ptr(self.state), self.n, self.dtype, _ptr(G), _ptr(t), t.size, _ptr(c), nc)

    def run(self, gates):
        for g in gates:
            self.apply(g.matrix, g.targets, g.controls)
        return self


class CompressedSim:
    """O2: Algorithm 1 over a block-compressed state (see sv_oracle.c); ``lazy``: the second
    mode O2L (lazy normalization with slice skipping, see sv_oracle.h)."""

    def __init__(self, n: int, slice_log2: int, block_log2: int, dtype: int, eb: float, basis_index: int = 0,
                 chunk: int = 32, lazy: bool = False):
        self.n, self.slice_log2, self.block_log2, self.dtype, self.eb = n, slice_log2, block_log2, dtype, eb
        self.chunk = chunk
        self._L = _load()
        self._h = self._L.orc_csim_create_k(n, slice_log2, block_log2, dtype, eb, basis_index, chunk)
        if not self._h:
            raise ValueError("orc_csim_create rejected its arguments")
        if lazy and self._L.orc_csim_set_lazy(self._h, 1) != 0:
            raise ValueError("orc_csim_set_lazy refused")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.orc_csim_destroy(h)
            self._h = None

    def apply(self, G, targets, controls=()):
        G, t, c, nc = _gate_arrays(G, targets, controls)
        rc = self._L.orc_csim_apply(self._h, _ptr(G), _ptr(t), t.size, _ptr(c), nc)
        if rc != 0:
            raise RuntimeError("orc_csim_apply failed (%d)" % rc)

    def run(self, gates):
        for g in gates:
            self.apply(g.matrix, g.targets, g.controls)
        return self

    def read(self) -> np.ndarray:
        out = np.zeros(1 << self.n, dtype=_cdtype(self.dtype))
        self._L.orc_csim_read(self._h, _ptr(out))
        return out

    def load(self, values) -> None:
        v = np.ascontiguousarray(values, dtype=_cdtype(self.dtype))
        assert v.size == 1 << self.n
        self._L.orc_csim_load(self._h, _ptr(v))

    @property
    def norm(self) -> float:
        return float(self._L.orc_csim_norm(self._h))

    @property
    def nblocks(self) -> int:
        return int(self._L.orc_csim_nblocks(self._h))

    def block_stream(self, b: int) -> bytes:
        p = ctypes.c_void_p()
        n = self._L.orc_csim_block_stream(self._h, b, ctypes.byref(p))
        return ctypes.string_at(p.value, n)

    def total_bytes(self) -> int:
        return int(self._L.orc_csim_total_bytes(self._h))

    def scales(self) -> np.ndarray:
        """Pending normalization c_s per slice (all 1 outside the second mode)."""
        out = np.zeros(1 << (self.n - self.slice_log2), dtype=np.float64)
        self._L.orc_csim_scales(self._h, _ptr(out))
        return out

    @property
    def skipped(self) -> int:
        return int(self._L.orc_csim_skipped(self._h))

    def read_values(self) -> np.ndarray:
        """The represented amplitudes c_s x' (complex128 for either dtype)."""
        out = np.zeros(1 << self.n, dtype=np.complex128)
        self._L.orc_csim_read_values(self._h, _ptr(out))
        return out
