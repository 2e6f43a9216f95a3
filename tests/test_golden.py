"""Golden files under tests/golden/.

* paper_printed.txt — numbers the paper prints (cited per line); they pin the memory
  accounting in which results are reported (state size, ratio, memory fraction, extra
  qubits).
* qft12_oracle.txt, codec_streams.txt — the oracle's own output on seeded inputs, written by
  tests/golden/make_golden.py (which calls only the oracle). The CPU tests re-run the oracle
  and require the same values, so a change to its arithmetic shows up here; the GPU tests
  require the CUDA path to reproduce the stored values through the C ABI.
"""
import hashlib
import math
import os

import numpy as np
import pytest

import oracle
from blockgen import gen_block
from paper_1811_05630_gb300 import circuits as C
from paper_1811_05630_gb300 import report

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [line.split() for line in f if line.strip() and not line.startswith("#")]


def paper():
    return {r[0]: float(r[1]) for r in read_rows("paper_printed.txt")}


def qft12():
    rows, digest = [], None
    for r in read_rows("qft12_oracle.txt"):
        if r[0] == "final_streams_sha256":
            digest = r[1]
        else:
            rows.append((int(r[0]), r[1], int(r[2]), float.fromhex(r[3])))
    return rows, digest


def codec_cases():
    out = []
    for r in read_rows("codec_streams.txt"):
        out.append(dict(kind=r[0], b=int(r[1]), dtype=int(r[2]), eb=float(r[3]), chunk=int(r[4]),
                        seed=int(r[5]), nbytes=int(r[6]), mode=int(r[7]), sha=r[8]))
    return out


# ---- values the paper prints ---------------------------------------------------------------

def test_state_size_is_two_to_the_n_plus_4_bytes():
    P = paper()
    k = int(P["state_bytes_log2_offset"])
    for n in range(1, 60):
        assert report.raw_state_bytes(n, report.C128) == 2 ** (n + k)
        assert report.raw_state_bytes(n, report.C64) == 2 ** (n + k - 1)
    # Sec. I: 45 qubits need 0.5 PB (petabyte read as 2^50 bytes)
    assert report.raw_state_bytes(45) / 2.0 ** 50 == P["state_45_qubits_petabytes"]


def test_grover_ratio_memory_fraction_and_extra_qubits():
    P = paper()
    r = P["grover30_min_ratio"]
    # the abstract's 2.24E-06 is 1/445144 = 2.2465E-06 cut (not rounded) to the digits printed
    f = report.memory_fraction(r)
    assert P["grover_memory_fraction"] <= f < P["grover_memory_fraction"] + 0.01e-6
    assert report.extra_qubits(r) == int(P["grover_extra_qubits"])


def test_qft_ratio_memory_fraction_and_extra_qubits():
    P = paper()
    lo = P["qft30_min_ratio_lower"]
    assert report.extra_qubits(lo) == int(P["qft30_extra_qubits"])
    # the abstract's 16.5 % is a ratio of 6.06, consistent with "greater than 6x"
    r = 1.0 / P["qft_memory_fraction"]
    assert r > lo and report.extra_qubits(r) == int(P["qft30_extra_qubits"])


def test_extra_qubits_at_powers_of_two():
    for k in range(0, 62):
        assert report.extra_qubits(2.0 ** k) == k
        if k >= 1:
            assert report.extra_qubits(2.0 ** k * (1 - 1e-12)) == k - 1
    assert report.extra_qubits(0.5) == 0


def test_compression_ratio_per_dtype():
    assert report.compression_ratio(20, report.C128, 1 << 20) == 16.0
    assert report.compression_ratio(20, report.C64, 1 << 20) == 8.0
    with pytest.raises(ValueError):
        report.compression_ratio(20, 3, 1)
    with pytest.raises(ValueError):
        report.compression_ratio(20, report.C128, 0)


# ---- the oracle reproduces its stored output -----------------------------------------------

def test_oracle_qft12_matches_golden():
    rows, digest = qft12()
    n, x = 12, C.seeded_index(0, 12)
    gates = C.qft(n)
    assert len(rows) == len(gates) + 1
    cs = oracle.CompressedSim(n, 8, 8, oracle.C128, 1e-6, x)
    assert (cs.total_bytes(), cs.norm) == (rows[0][2], rows[0][3])
    for (i, name, nbytes, norm), g in zip(rows[1:], gates):
        cs.apply(g.matrix, g.targets, g.controls)
        assert name == g.name
        assert (cs.total_bytes(), cs.norm) == (nbytes, norm), "gate %d %s" % (i, name)
    h = hashlib.sha256()
    for blk in range(cs.nblocks):
        h.update(cs.block_stream(blk))
    assert h.hexdigest() == digest


def test_oracle_codec_matches_golden():
    cases = codec_cases()
    assert len(cases) > 200
    assert {c["mode"] for c in cases} == {oracle.MODE_CONST, oracle.MODE_HUFF, oracle.MODE_PACK}
    for c in cases:
        v = gen_block(c["kind"], c["b"], np.random.default_rng(c["seed"]), c["dtype"])
        s, info = oracle.compress_block(v, c["b"], c["dtype"], c["eb"], chunk=c["chunk"])
        assert (len(s), info["mode"], hashlib.sha256(s).hexdigest()) == (c["nbytes"], c["mode"], c["sha"]), c


def test_golden_norms_stay_near_one():
    # every stored norm of the QFT12 run is within the accumulated quantization error of 1
    rows, _ = qft12()
    eb, B = 1e-6, 1 << 12
    per_pass = math.sqrt(2 * B) * eb
    for i, _, _, N in rows:
        assert abs(math.sqrt(N) - 1.0) <= 2 * per_pass * 1.01, i


# ---- the CUDA path reproduces the stored oracle output -------------------------------------

@pytest.mark.gpu
def test_gpu_qft12_matches_golden():
    import torch

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1811_05630_gb300 import sv

    rows, digest = qft12()
    n, x = 12, C.seeded_index(0, 12)
    pool = sv.Pool(1 << 28)
    st = sv.State(pool, n, 8, 1e-6, sv.C128, block_log2=8)
    try:
        st.reset_basis(x)
        assert (st.compressed_bytes(), st.norm()) == (rows[0][2], rows[0][3])
        for (i, name, nbytes, norm), g in zip(rows[1:], C.qft(n)):
            st.apply(g.matrix, g.targets, g.controls)
            assert (st.compressed_bytes(), st.norm()) == (nbytes, norm), "gate %d %s" % (i, name)
        h = hashlib.sha256()
        for blk in range(1 << (n - 8)):
            h.update(st.block_stream(blk))
        assert h.hexdigest() == digest
    finally:
        st.close()
        pool.close()


@pytest.mark.gpu
def test_gpu_codec_matches_golden():
    import torch

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1811_05630_gb300 import sv

    groups = {}
    for c in codec_cases():
        if c["chunk"] == 32:  # the device codec writes the format's default chunk size
            groups.setdefault((c["b"], c["dtype"], c["eb"]), []).append(c)
    assert groups
    for (b, dtype, eb), cases in sorted(groups.items()):
        vals = np.concatenate([gen_block(c["kind"], b, np.random.default_rng(c["seed"]), dtype) for c in cases])
        t = torch.from_numpy(vals).cuda()
        out, offs, lens, _ = sv.codec_compress(t, b, eb)
        torch.cuda.synchronize()
        out, offs, lens = out.cpu().numpy(), offs.cpu().numpy(), lens.cpu().numpy()
        for k, c in enumerate(cases):
            s = out[int(offs[k]):int(offs[k]) + int(lens[k])].tobytes()
            assert (len(s), hashlib.sha256(s).hexdigest()) == (c["nbytes"], c["sha"]), c
