"""Autotuner for the block size (block_log2), the CTA size, the register budget of the
fused pass and the Huffman chunk size of the block format.

The block size sets the codec's parallel unit: small blocks give more CTAs per pass and
more CTAs per SM (less shared memory each), large blocks amortize the per-block codebook
and headers. The CTA size (threads per block-group) trades per-block latency against CTAs
resident per SM; the register-capped build (64 registers per thread, spilling) fits four
256-thread CTAs on an SM. The best pair depends on the state size, dtype, error bound and
circuit, so the tuner times a few gate passes of a representative circuit for each candidate
on the GPU (fused-kernel CUDA events) and keeps the fastest. No knob changes results.
Results are cached in a JSON file keyed by (GPU name, dtype, qubits, error bound, circuit
kind).
"""
from __future__ import annotations

import json
import os
from typing import Dict, Iterable, List, Optional, Sequence

import torch

from . import sv
from .circuits import Gate

CACHE = os.environ.get("SV_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "sv_tune.json"))


def _key(n: int, dtype: int, eb: float, kind: str) -> str:
    return "%s|%d|%d|%.3g|%s" % (torch.cuda.get_device_name(), dtype, n, eb, kind)


def _load() -> Dict[str, dict]:
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(d: Dict[str, dict]) -> None:
    try:
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        with open(CACHE + ".tmp", "w") as f:
            json.dump(d, f, indent=1)
        os.replace(CACHE + ".tmp", CACHE)
    except OSError:
        pass


def thread_candidates(b: int) -> List[int]:
    """CTA sizes the fused pass accepts for block size b (powers of two, 32..256, 2 to 32
    values per thread)."""
    nv = 2 << b
    return [t for t in (32, 64, 128, 256) if 2 <= nv // t <= 32]


def probe(pool: sv.Pool, n: int, dtype: int, eb: float, b: int, prefix: Sequence[Gate], timed: Sequence[Gate],
          basis: int = 0, threads: int = 0, compact: bool = False, chunk: int = 32) -> float:
    """Fused-kernel milliseconds per pass for `timed` after `prefix`, at block size b, CTA
    size `threads` (0: the default), with or without the register-capped build, and Huffman
    chunk size `chunk`."""
    st = sv.State(pool, n, n, eb, dtype, block_log2=b)
    try:
        st.set_threads(threads)
        st.set_compact(compact)
        if chunk != 32:
            st.set_chunk(chunk)
        st.reset_basis(basis)
        st.run(prefix)
        st.sync()
        st.set_pass_timing(True)
        st.run(timed)
        ms, npass, _ = st.pass_timing()
        return ms / max(npass, 1)
    finally:
        st.close()


def best_config(n: int, dtype: int, eb: float, kind: str, prefix: Sequence[Gate], timed: Sequence[Gate],
                basis: int = 0, candidates: Iterable[int] = (8, 9, 10, 11, 12), pool: Optional[sv.Pool] = None,
                use_cache: bool = True, chunks: Iterable[int] = (32,)) -> dict:
    """Tune (block_log2, threads, register-capped build, Huffman chunk size) for a workload;
    returns {"block_log2": b, "threads": T, "compact": c, "chunk": k, "ms_per_pass":
    {"b/T/c/k": ms}}. The chunk size also changes the compressed size (16 more bits per
    chunk), so `chunks` limits the sizes tried (the default: 32 only, the format default)."""
    key = _key(n, dtype, eb, kind)
    cache = _load() if use_cache else {}
    if key in cache and "chunk" in cache[key]:
        return cache[key]
    own = pool is None
    if own:
        pool = sv.Pool(max(1 << 30, (24 if dtype == 2 else 12) << n))
    times: Dict[tuple, float] = {}
    try:
        for b in candidates:
            if b > n:
                continue
            for t in thread_candidates(b):
                for c in ((0, 1) if t >= 128 else (0,)):
                    for k in chunks:
                        if (2 << b) // k > t:
                            continue
                        times[(b, t, c, k)] = probe(pool, n, dtype, eb, b, prefix, timed, basis, threads=t,
                                                    compact=bool(c), chunk=k)
    finally:
        if own:
            pool.close()
    best = min(times, key=times.get)
    res = {"block_log2": best[0], "threads": best[1], "compact": bool(best[2]), "chunk": best[3],
           "ms_per_pass": {"%d/%d/%d/%d" % k: v for k, v in sorted(times.items())}}
    if use_cache:
        cache[key] = res
        _store(cache)
    return res
