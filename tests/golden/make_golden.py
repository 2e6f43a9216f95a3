"""Write the oracle-derived golden files of this folder.

Every value written here comes from the CPU oracle (``oracle/``) on seeded inputs; nothing
comes from the CUDA path. The files freeze the oracle's output so that a change to its
arithmetic shows up as a diff of these files (a change of that kind names the passage of
the paper that justifies it). Run from the repository root:

    python tests/golden/make_golden.py

Files:
  qft12_oracle.txt   QFT on 12 qubits from a seeded basis state, eb 1e-6, complex128,
                     slices and blocks of 256 amplitudes (Algorithm 1, gate by gate): the
                     stored bytes and the stored norm N_g after every gate, and a SHA-256 of
                     the final block streams.
  codec_streams.txt  one seeded block per (kind, block_log2, dtype, eb, chunk) through the
                     block codec (Sec. II): stream length, mode and SHA-256.
"""
from __future__ import annotations

import hashlib
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
if os.path.dirname(HERE) not in sys.path:
    sys.path.insert(0, os.path.dirname(HERE))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from blockgen import KINDS, gen_block  # noqa: E402
from paper_1811_05630_gb300 import circuits as C  # noqa: E402

QFT12 = dict(n=12, slice_log2=8, block_log2=8, dtype=oracle.C128, eb=1e-6, seed=0)
CODEC_CASES = [(kind, b, dtype, eb, chunk)
               for kind in KINDS
               for b in (5, 8, 11)
               for dtype in (oracle.C128, oracle.C64)
               for eb in (1e-4, 1e-8)
               for chunk in (16, 32, 64)
               if (2 << b) >= chunk]


def qft12_rows():
    """(gate index, gate name, stored bytes, stored norm as a hex float) after each gate;
    index -1 is the compressed initial state. Also returns the final streams' SHA-256."""
    c = QFT12
    x = C.seeded_index(c["seed"], c["n"])
    cs = oracle.CompressedSim(c["n"], c["slice_log2"], c["block_log2"], c["dtype"], c["eb"], x)
    rows = [(-1, "init", cs.total_bytes(), float(cs.norm).hex())]
    for i, g in enumerate(C.qft(c["n"])):
        cs.apply(g.matrix, g.targets, g.controls)
        rows.append((i, g.name, cs.total_bytes(), float(cs.norm).hex()))
    h = hashlib.sha256()
    for blk in range(cs.nblocks):
        h.update(cs.block_stream(blk))
    return x, rows, h.hexdigest()


def codec_block(kind, b, dtype, eb, seed):
    rng = np.random.default_rng(seed)
    return gen_block(kind, b, rng, dtype)


def codec_rows():
    rows = []
    for i, (kind, b, dtype, eb, chunk) in enumerate(CODEC_CASES):
        v = codec_block(kind, b, dtype, eb, 1000 + i)
        stream, info = oracle.compress_block(v, b, dtype, eb, chunk=chunk)
        rows.append((kind, b, dtype, eb, chunk, 1000 + i, len(stream), info["mode"],
                     hashlib.sha256(stream).hexdigest()))
    return rows


def write_qft12(path):
    x, rows, digest = qft12_rows()
    c = QFT12
    with open(path, "w") as f:
        f.write("# Written by tests/golden/make_golden.py from the CPU oracle (Algorithm 1).\n")
        f.write("# QFT n=%d from basis index %d (SplitMix64 seed %d), eb %g, complex128, slice_log2 %d, "
                "block_log2 %d.\n" % (c["n"], x, c["seed"], c["eb"], c["slice_log2"], c["block_log2"]))
        f.write("# columns: gate index (-1 = initial state), gate, stored bytes, stored norm N_g (hex)\n")
        for r in rows:
            f.write("%d %s %d %s\n" % r)
        f.write("final_streams_sha256 %s\n" % digest)


def write_codec(path):
    with open(path, "w") as f:
        f.write("# Written by tests/golden/make_golden.py from the CPU oracle's block codec.\n")
        f.write("# Block values: tests/blockgen.py gen_block(kind, block_log2, numpy default_rng(seed), dtype).\n")
        f.write("# columns: kind block_log2 dtype eb chunk seed stream_bytes mode sha256\n")
        for r in codec_rows():
            f.write("%s %d %d %r %d %d %d %d %s\n" % r)


def main():
    write_qft12(os.path.join(HERE, "qft12_oracle.txt"))
    write_codec(os.path.join(HERE, "codec_streams.txt"))


if __name__ == "__main__":
    main()
