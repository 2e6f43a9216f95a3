"""Thin ctypes binding of libsv.so (include/sv.h): argument marshalling only.

PyTorch supplies the device memory (one uint8 tensor per pool) and the CUDA streams; every
step of the simulation runs in the library's CUDA kernels. Importing this module loads
libsv.so and raises ImportError when it has not been built (``python -m
paper_1811_05630_gb300.build``) — there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Iterable, Sequence

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("SV_LIBRARY") or os.path.join(_HERE, "libsv.so")
if not os.path.exists(LIB_PATH):
    raise ImportError("libsv.so is not built; run `python -m paper_1811_05630_gb300.build`")
_L = ctypes.CDLL(LIB_PATH)

C64, C128 = 1, 2
OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_NORM, ERR_CORRUPT, ERR_UNSUPPORTED, ERR_TIMEOUT, ERR_INTERNAL = (
    0, -1, -2, -3, -4, -5, -6, -7, -8)
_ERR_NAMES = {-1: "SV_ERR_ARG", -2: "SV_ERR_OOM", -3: "SV_ERR_CUDA", -4: "SV_ERR_NORM",
              -5: "SV_ERR_CORRUPT", -6: "SV_ERR_UNSUPPORTED", -7: "SV_ERR_TIMEOUT", -8: "SV_ERR_INTERNAL"}


class SvError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__("%s failed: %s (%d)" % (what, _ERR_NAMES.get(code, "?"), code))
        self.code = code


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise SvError(rc, what)


class Stats(ctypes.Structure):
    _fields_ = [
        ("pass_index", ctypes.c_uint64), ("compressed_bytes", ctypes.c_uint64),
        ("table_bytes", ctypes.c_uint64), ("n_blocks", ctypes.c_uint64),
        ("blocks_const", ctypes.c_uint64), ("blocks_huff", ctypes.c_uint64),
        ("blocks_pack", ctypes.c_uint64), ("n_verbatim", ctypes.c_uint64),
        ("n_escape", ctypes.c_uint64), ("norm", ctypes.c_double), ("sigma", ctypes.c_double),
        ("blocks_reused", ctypes.c_uint64), ("replayed_passes", ctypes.c_uint64),
        ("peak_compressed_bytes", ctypes.c_uint64), ("spill_arena_bytes", ctypes.c_uint64),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class GateT(ctypes.Structure):
    _fields_ = [("G", ctypes.c_void_p), ("targets", ctypes.c_void_p), ("k", ctypes.c_int),
                ("controls", ctypes.c_void_p), ("n_controls", ctypes.c_int)]


_vp, _i, _d, _sz, _u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t, ctypes.c_uint64
_P = ctypes.POINTER
_SIGS = {
    "sv_pool_create": ([_vp, _sz, _P(_vp)], _i),
    "sv_pool_destroy": ([_vp], _i),
    "sv_pool_usage": ([_vp, _P(_sz), _P(_sz)], _i),
    "sv_create": ([_vp, _i, _i, _d, _i, _vp, _P(_vp)], _i),
    "sv_create_ex": ([_vp, _i, _i, _i, _d, _i, _sz, _vp, _P(_vp)], _i),
    "sv_destroy": ([_vp], _i),
    "sv_reset_basis": ([_vp, _u64], _i),
    "sv_apply_gate": ([_vp, _vp, _vp, _i, _vp, _i], _i),
    "sv_sync": ([_vp], _i),
    "sv_set_threads": ([_vp, _i], _i),
    "sv_set_compact": ([_vp, _i], _i),
    "sv_set_tensor_cores": ([_vp, _i], _i),
    "sv_set_spill_pool": ([_vp, _vp], _i),
    "sv_set_chunk": ([_vp, _i], _i),
    "sv_measure_probs": ([_vp, _vp, _i, _vp], _i),
    "sv_amplitudes": ([_vp, _vp, _sz, _vp], _i),
    "sv_read_amplitudes": ([_vp, _u64, _u64, _vp], _i),
    "sv_fidelity": ([_vp, _vp, _P(_d)], _i),
    "sv_compressed_bytes": ([_vp, _P(_u64)], _i),
    "sv_stats": ([_vp, _P(Stats)], _i),
    "sv_norm": ([_vp, _P(_d)], _i),
    "sv_block_stream": ([_vp, _u64, _vp, _sz, _P(_sz)], _i),
    "sv_codec_scratch_bytes": ([], _sz),
    "sv_codec_compress": ([_vp, _u64, _i, _i, _d, _vp, _u64, _vp, _vp, _vp, _vp, _P(_u64)], _i),
    "sv_codec_decompress": ([_vp, _vp, _vp, _u64, _i, _i, _d, _vp, _vp, _vp], _i),
    "sv_codec_compress_static": ([_vp, _u64, _i, _i, _d, _vp, _u64, _vp, _vp, _vp, _P(_u64), _P(_d)], _i),
    "sv_overlap_qft": ([_vp, _u64, _vp], _i),
    "sv_batch_create": ([_vp, _i, _vp, _P(_vp)], _i),
    "sv_batch_destroy": ([_vp], _i),
    "sv_batch_use_graphs": ([_vp, _i], _i),
    "sv_batch_ready": ([_vp], _i),
    "sv_batch_apply": ([_vp, _vp, _vp, _i], _i),
    "sv_set_pass_timing": ([_vp, _i], _i),
    "sv_get_pass_timing": ([_vp, _P(_d), _P(_u64), _P(_u64)], _i),
    "sv_check_bounded_wait": ([ctypes.c_longlong, _vp, _P(_i)], _i),
    "sv_version": ([], ctypes.c_char_p),
}
_OPTIONAL = {"sv_set_tensor_cores", "sv_set_spill_pool"}  # absent from builds that predate them
for _name, (_args, _res) in _SIGS.items():
    if _name in _OPTIONAL and not hasattr(_L, _name):
        continue
    _f = getattr(_L, _name)
    _f.argtypes = _args
    _f.restype = _res


def _stream_handle(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _np_ptr(a: np.ndarray) -> int:
    return a.ctypes.data


class Pool:
    """One caller-owned device buffer (a torch uint8 tensor) the library sub-allocates."""

    def __init__(self, nbytes: int, device="cuda"):
        if device == "host":  # pinned host memory the device addresses: a spill pool
            self.buf = torch.empty(int(nbytes), dtype=torch.uint8).pin_memory()
        else:
            self.buf = torch.empty(int(nbytes), dtype=torch.uint8, device=device)
        h = ctypes.c_void_p()
        _check(_L.sv_pool_create(self.buf.data_ptr(), self.buf.numel(), ctypes.byref(h)), "sv_pool_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    def usage(self):
        u, c = ctypes.c_size_t(), ctypes.c_size_t()
        _check(_L.sv_pool_usage(self._h, ctypes.byref(u), ctypes.byref(c)), "sv_pool_usage")
        return u.value, c.value

    def close(self):
        if self._h:
            _check(_L.sv_pool_destroy(self._h), "sv_pool_destroy")
            self._h = None


class State:
    """A state vector of n qubits kept compressed (error_bound > 0) or plain (0)."""

    def __init__(self, pool: Pool, n: int, slice_log2: int, error_bound: float, dtype: int = C128,
                 block_log2: int = -1, arena_bytes: int = 0, stream=None):
        self.pool, self.n, self.dtype, self.eb = pool, n, dtype, error_bound
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        _check(_L.sv_create_ex(pool.handle, n, slice_log2, block_log2, float(error_bound), dtype,
                               int(arena_bytes), _stream_handle(self.stream), ctypes.byref(h)), "sv_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _check(_L.sv_destroy(self._h), "sv_destroy")
            self._h = None

    def reset_basis(self, index: int):
        _check(_L.sv_reset_basis(self._h, int(index)), "sv_reset_basis")

    def apply(self, G, targets: Sequence[int], controls: Sequence[int] = ()):
        g = np.ascontiguousarray(G, dtype=np.complex128)
        t = np.ascontiguousarray(targets, dtype=np.int32)
        c = np.ascontiguousarray(controls if len(controls) else [0], dtype=np.int32)
        _check(_L.sv_apply_gate(self._h, _np_ptr(g), _np_ptr(t), t.size, _np_ptr(c), len(controls)),
               "sv_apply_gate")

    def run(self, gates: Iterable) -> "State":
        for gt in gates:
            self.apply(gt.matrix, gt.targets, gt.controls)
        return self

    def sync(self):
        _check(_L.sv_sync(self._h), "sv_sync")

    def norm(self) -> float:
        v = ctypes.c_double()
        _check(_L.sv_norm(self._h, ctypes.byref(v)), "sv_norm")
        return v.value

    def set_threads(self, threads: int) -> None:
        """CTA size of the fused pass (0: default); results do not depend on it."""
        _check(_L.sv_set_threads(self._h, int(threads)), "sv_set_threads")

    def set_chunk(self, chunk: int) -> None:
        """Huffman chunk size of the block format (16, 32, 64); resets the state to |0...0>."""
        _check(_L.sv_set_chunk(self._h, int(chunk)), "sv_set_chunk")

    def set_spill(self, pool: "Pool | None") -> None:
        """Arenas that do not fit in the state's pool go to `pool` (e.g. Pool(n, "host"))."""
        _check(_L.sv_set_spill_pool(self._h, pool.handle if pool is not None else None), "sv_set_spill_pool")
        self.spill_pool = pool

    def set_tensor_cores(self, on: bool) -> None:
        """4- and 5-qubit complex128 gates on the tensor cores (default) or the CUDA cores
        (results unchanged)."""
        _check(_L.sv_set_tensor_cores(self._h, 1 if on else 0), "sv_set_tensor_cores")

    def set_compact(self, on: bool) -> None:
        """Register-capped build of the fused pass for 1- and 2-qubit gates (results unchanged)."""
        _check(_L.sv_set_compact(self._h, 1 if on else 0), "sv_set_compact")

    def stats(self) -> dict:
        st = Stats()
        _check(_L.sv_stats(self._h, ctypes.byref(st)), "sv_stats")
        return st.as_dict()

    def compressed_bytes(self) -> int:
        v = ctypes.c_uint64()
        _check(_L.sv_compressed_bytes(self._h, ctypes.byref(v)), "sv_compressed_bytes")
        return v.value

    def probs(self, qubits: Sequence[int]) -> np.ndarray:
        q = np.ascontiguousarray(qubits, dtype=np.int32)
        out = np.zeros(1 << q.size, dtype=np.float64)
        _check(_L.sv_measure_probs(self._h, _np_ptr(q), q.size, _np_ptr(out)), "sv_measure_probs")
        return out

    def amplitudes(self, idx) -> np.ndarray:
        ix = np.ascontiguousarray(idx, dtype=np.uint64)
        out = np.zeros(ix.size, dtype=np.complex128)
        _check(_L.sv_amplitudes(self._h, _np_ptr(ix), ix.size, _np_ptr(out)), "sv_amplitudes")
        return out

    def read(self, start: int = 0, count: int | None = None) -> np.ndarray:
        if count is None:
            count = (1 << self.n) - start
        out = np.zeros(count, dtype=np.complex128)
        _check(_L.sv_read_amplitudes(self._h, start, count, _np_ptr(out)), "sv_read_amplitudes")
        return out

    def fidelity(self, other: "State") -> float:
        v = ctypes.c_double()
        _check(_L.sv_fidelity(self._h, other._h, ctypes.byref(v)), "sv_fidelity")
        return v.value

    def fidelity_qft(self, x: int) -> float:
        """Fidelity with the exact QFT of |x> (closed form), computed on the GPU."""
        out = np.zeros(3, dtype=np.float64)
        _check(_L.sv_overlap_qft(self._h, int(x), _np_ptr(out)), "sv_overlap_qft")
        return float((out[0] ** 2 + out[1] ** 2) / out[2])

    def set_pass_timing(self, on: bool = True):
        _check(_L.sv_set_pass_timing(self._h, 1 if on else 0), "sv_set_pass_timing")

    def pass_timing(self):
        """(summed fused-kernel ms, passes, algorithmic bytes) since set_pass_timing."""
        ms, n, by = ctypes.c_double(), ctypes.c_uint64(), ctypes.c_uint64()
        _check(_L.sv_get_pass_timing(self._h, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(by)),
               "sv_get_pass_timing")
        return ms.value, n.value, by.value

    def block_stream(self, b: int) -> bytes:
        ln = ctypes.c_size_t()
        _check(_L.sv_block_stream(self._h, b, None, 0, ctypes.byref(ln)), "sv_block_stream")
        buf = np.zeros(max(ln.value, 1), dtype=np.uint8)
        _check(_L.sv_block_stream(self._h, b, _np_ptr(buf), buf.size, ctypes.byref(ln)), "sv_block_stream")
        return buf[: ln.value].tobytes()


class Batch:
    """Advance many states by one gate each per step, in one launch (optionally replayed
    from captured CUDA graphs). States must share dtype, block size and this stream."""

    def __init__(self, pool: Pool, max_states: int, stream=None, graphs: bool = False):
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        _check(_L.sv_batch_create(pool.handle, max_states, _stream_handle(self.stream), ctypes.byref(h)),
               "sv_batch_create")
        self._h = h
        self.use_graphs(graphs)

    def use_graphs(self, on: bool):
        _check(_L.sv_batch_use_graphs(self._h, 1 if on else 0), "sv_batch_use_graphs")

    def ready(self) -> bool:
        r = _L.sv_batch_ready(self._h)
        if r < 0:
            _check(r, "sv_batch_ready")
        return r == 1

    def apply(self, states, gates):
        n = len(states)
        keep = []
        arr = (GateT * n)()
        for i, g in enumerate(gates):
            m = np.ascontiguousarray(g.matrix, dtype=np.complex128)
            t = np.ascontiguousarray(g.targets, dtype=np.int32)
            c = np.ascontiguousarray(g.controls if len(g.controls) else [0], dtype=np.int32)
            keep += [m, t, c]
            arr[i] = GateT(m.ctypes.data, t.ctypes.data, t.size, c.ctypes.data, len(g.controls))
        hs = (ctypes.c_void_p * n)(*[s._h.value for s in states])
        _check(_L.sv_batch_apply(self._h, hs, arr, n), "sv_batch_apply")

    def close(self):
        if getattr(self, "_h", None):
            _check(_L.sv_batch_destroy(self._h), "sv_batch_destroy")
            self._h = None


def codec_scratch_bytes() -> int:
    return int(_L.sv_codec_scratch_bytes())


def codec_compress(values: torch.Tensor, block_log2: int, error_bound: float, cap: int | None = None,
                   stream=None):
    """Compress device complex values (complex128/complex64, length a multiple of
    2^block_log2). Returns (out uint8 tensor, offsets u64 tensor, lengths i32 tensor, used)."""
    assert values.is_cuda and values.is_contiguous()
    dtype = C64 if values.dtype == torch.complex64 else C128
    B = 1 << block_log2
    nblocks = values.numel() // B
    assert nblocks * B == values.numel()
    if cap is None:  # largest stream: PACK at 32 bits plus every value verbatim
        cap = nblocks * (16 + 4 * 2 * B + 2 * 2 * B + 8 * 2 * B + 32)
    out = torch.zeros(cap, dtype=torch.uint8, device=values.device)
    offs = torch.zeros(nblocks, dtype=torch.int64, device=values.device)
    lens = torch.zeros(nblocks, dtype=torch.int32, device=values.device)
    scratch = torch.zeros(codec_scratch_bytes(), dtype=torch.uint8, device=values.device)
    used = ctypes.c_uint64()
    _check(_L.sv_codec_compress(values.data_ptr(), nblocks, block_log2, dtype, float(error_bound),
                                out.data_ptr(), cap, offs.data_ptr(), lens.data_ptr(), scratch.data_ptr(),
                                _stream_handle(stream), ctypes.byref(used)), "sv_codec_compress")
    return out, offs, lens, used.value


STATIC_MAX_BLOCKS = 65536


def codec_compress_static(values: torch.Tensor, block_log2: int, error_bound: float, out: torch.Tensor,
                          offsets: torch.Tensor, lengths: torch.Tensor, stream=None):
    """Like codec_compress, for callers that cannot allocate device memory: the caller owns
    every buffer passed here and the library uses its own fixed scratch array (no scratch
    argument, nothing allocated). Returns (used bytes, stored norm of the compressed values)."""
    assert values.is_cuda and values.is_contiguous()
    assert values.dtype in (torch.complex64, torch.complex128)
    dtype = C64 if values.dtype == torch.complex64 else C128
    nblocks = values.numel() >> block_log2
    # the C side takes no buffer lengths and its scratch is per device: check here what it
    # cannot (every buffer on the values' device, long enough, of the declared type)
    assert nblocks << block_log2 == values.numel(), "length must be a multiple of 2^block_log2"
    assert out.dtype == torch.uint8 and out.is_contiguous()
    assert offsets.dtype == torch.int64 and offsets.is_contiguous() and offsets.numel() >= nblocks
    assert lengths.dtype == torch.int32 and lengths.is_contiguous() and lengths.numel() >= nblocks
    for t in (out, offsets, lengths):
        assert t.device == values.device, "every buffer must be on the device of `values`"
    used, norm = ctypes.c_uint64(), ctypes.c_double()
    with torch.cuda.device(values.device):
        _check(_L.sv_codec_compress_static(values.data_ptr(), nblocks, block_log2, dtype, float(error_bound),
                                           out.data_ptr(), out.numel(), offsets.data_ptr(), lengths.data_ptr(),
                                           _stream_handle(stream), ctypes.byref(used), ctypes.byref(norm)),
               "sv_codec_compress_static")
    return used.value, norm.value


def codec_decompress(data: torch.Tensor, offsets: torch.Tensor, lengths: torch.Tensor, block_log2: int,
                     dtype: int, error_bound: float, stream=None) -> torch.Tensor:
    nblocks = offsets.numel()
    tdt = torch.complex64 if dtype == C64 else torch.complex128
    vals = torch.zeros(nblocks << block_log2, dtype=tdt, device=data.device)
    scratch = torch.zeros(codec_scratch_bytes(), dtype=torch.uint8, device=data.device)
    _check(_L.sv_codec_decompress(data.data_ptr(), offsets.data_ptr(), lengths.data_ptr(), nblocks, block_log2,
                                  dtype, float(error_bound), vals.data_ptr(), scratch.data_ptr(),
                                  _stream_handle(stream)), "sv_codec_decompress")
    return vals


def check_bounded_wait(polls: int = 1000, stream=None) -> bool:
    """Run the tensor-core pass's bounded mbarrier wait on a barrier nothing arrives on;
    True when the wait gave up after `polls` polls (the expected result)."""
    out = ctypes.c_int(-1)
    _check(_L.sv_check_bounded_wait(int(polls), _stream_handle(stream), ctypes.byref(out)), "sv_check_bounded_wait")
    return out.value == 1


def version() -> str:
    return _L.sv_version().decode()
