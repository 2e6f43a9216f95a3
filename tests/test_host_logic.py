"""Host-side logic on the CPU: the serving scheduler (against a fake device backend), the
tuner's candidate rules, the seeded circuit generators and the bench's traffic records.

The fake backend stands in for the C ABI only to drive the scheduler's bookkeeping
(admission under the byte budget, batching by bucket, completion, failure reporting); it
computes nothing of the method.
"""
import math
import types

import numpy as np
import pytest

from paper_1811_05630_gb300 import circuits as C


@pytest.fixture(scope="module")
def lib():
    """serve.py and tune.py import the ctypes binding, which loads libsv.so (built here by nvcc
    if missing; nothing in it is called)."""
    from paper_1811_05630_gb300 import build

    return build.build()


# ---- serving scheduler ----------------------------------------------------------------------

class FakeSvError(RuntimeError):
    pass


class FakeBackend:
    """Records what the scheduler asks of the library."""

    def __init__(self, budget, block_log2, max_batch, fail_eb=None):
        self.budget, self.block_log2, self.max_batch, self.fail_eb = budget, block_log2, max_batch, fail_eb
        self.live = {}       # id(state) -> footprint
        self.peak = 0
        self.created = []
        self.batch_sizes = []
        self.errors = []
        backend = self

        class Pool:
            def __init__(self, nbytes, device="cuda"):
                self.nbytes = nbytes

            def usage(self):
                return sum(backend.live.values()), self.nbytes

            def close(self):
                pass

        class State:
            def __init__(self, pool, n, slice_log2, eb, dtype, block_log2=0, stream=None, **kw):
                from paper_1811_05630_gb300 import serve

                self.n, self.eb, self.dtype, self.b, self.stream = n, eb, dtype, block_log2, stream
                self.applied = 0
                self.closed = False
                self.threads = 0
                # the fake state holds metadata and two arenas sized for its peak (1 byte per
                # amplitude, what stats() reports): at most what admission reserves, before
                # (prior) and after (learned, with its margin) a request of the class finished
                req = types.SimpleNamespace(n=n, dtype=dtype, eb=eb)
                fp = serve.footprint(req, block_log2, 1.0)
                backend.live[id(self)] = fp
                backend.peak = max(backend.peak, sum(backend.live.values()))
                backend.created.append(self)

            def set_threads(self, t):
                self.threads = t

            def reset_basis(self, x):
                self.basis = x

            def sync(self):
                if backend.fail_eb is not None and self.eb == backend.fail_eb:
                    raise FakeSvError("SV_ERR_NORM_COLLAPSE")

            def block_stream(self, i):
                return b"%d" % i

            def norm(self):
                return 1.0

            def stats(self):  # a compressed state of 1 byte per amplitude at its peak
                return {"peak_compressed_bytes": 1 << self.n}

            def close(self):
                assert not self.closed
                self.closed = True
                backend.live.pop(id(self))

        class Batch:
            def __init__(self, pool, max_states, stream=None, graphs=False):
                self.max_states, self.stream = max_states, stream

            def ready(self):
                return True

            def apply(self, states, gates):
                if len(states) > self.max_states:
                    backend.errors.append("batch of %d over %d" % (len(states), self.max_states))
                keys = {(s.dtype, s.b, s.stream) for s in states}
                if len(keys) != 1:
                    backend.errors.append("mixed bucket %s" % keys)
                if len(states) != len(gates):
                    backend.errors.append("states and gates differ")
                for s in states:
                    s.applied += 1
                backend.batch_sizes.append(len(states))

            def close(self):
                pass

        self.sv = types.SimpleNamespace(Pool=Pool, State=State, Batch=Batch, SvError=FakeSvError)

        class Stream:
            pass

        class Event:
            def record(self, stream):
                self.stream = stream

            def query(self):
                return True

        self.torch = types.SimpleNamespace(cuda=types.SimpleNamespace(Stream=Stream, Event=Event))


def small_requests(count=40, seed=3):
    rng = np.random.default_rng(seed)
    out, t = [], 0.0
    for rid in range(count):
        t += float(rng.exponential(0.002))
        n = int(rng.integers(10, 21))
        dtype = 1 if rng.random() < 0.5 else 2
        eb = [1e-4, 1e-6][int(rng.integers(2))]
        gates = C.qft(n)[: int(rng.integers(1, 12))]
        out.append(C.Request(rid, t, "qft", n, dtype, eb, 0, gates))
    return out


def run_server(monkeypatch, reqs, budget, max_batch=4, fail_eb=None, block_log2=10, time_limit=30.0):
    from paper_1811_05630_gb300 import serve

    fb = FakeBackend(budget, block_log2, max_batch, fail_eb)
    monkeypatch.setattr(serve, "sv", fb.sv)
    monkeypatch.setattr(serve, "torch", fb.torch)
    srv = serve.Server(1 << 30, budget, block_log2=block_log2, max_batch=max_batch, graphs=False)
    try:
        out = srv.run(reqs, time_limit=time_limit)
    finally:
        srv.close()
    return fb, out


def test_server_completes_every_request_within_budget(lib, monkeypatch):
    from paper_1811_05630_gb300 import serve

    reqs = small_requests()
    biggest = max(serve.footprint(r, min(10, r.n)) for r in reqs)
    budget = 3 * biggest
    fb, out = run_server(monkeypatch, reqs, budget)
    assert not fb.errors, fb.errors
    assert out["completed"] == len(reqs) and out["failed"] == 0
    assert out["waiting_at_end"] == 0 and out["active_at_end"] == 0
    # every state advanced by exactly its gate count and was released
    by_rid = {r.rid: r for r in reqs}
    assert len(fb.created) == len(reqs)
    assert all(st.closed for st in fb.created)
    assert sorted(s.applied for s in fb.created) == sorted(len(r.gates) for r in reqs)
    assert fb.peak <= budget
    assert max(fb.batch_sizes) <= 4
    # latencies: admission after arrival, completion after admission
    for res in out["results"]:
        assert res.admitted >= by_rid[res.rid].arrival - 1e-9
        assert res.done >= res.admitted
        assert res.amp_updates == by_rid[res.rid].amp_updates
    lat = sorted(r.latency for r in out["results"])
    assert out["p50_s"] == pytest.approx(float(np.percentile(lat, 50)))
    assert out["p99_s"] == pytest.approx(float(np.percentile(lat, 99)))


def test_server_sets_cta_size_only_where_valid(lib, monkeypatch):
    reqs = [C.Request(0, 0.0, "qft", 5, 2, 1e-6, 0, C.qft(5)[:2]),
            C.Request(1, 0.0, "qft", 12, 2, 1e-6, 0, C.qft(12)[:2])]
    fb, out = run_server(monkeypatch, reqs, 1 << 30)
    t = {s.n: s.threads for s in fb.created}
    assert t[12] == 128      # 2^(10+1) values / 128 threads = 16 per thread
    assert t[5] == 0         # 64 values: 128 threads would leave less than 2 per thread


def test_server_reports_failed_requests_and_frees_them(lib, monkeypatch):
    reqs = small_requests(24, seed=5)
    fb, out = run_server(monkeypatch, reqs, 1 << 40, fail_eb=1e-4)
    nfail = sum(1 for r in reqs if r.eb == 1e-4)
    assert 0 < nfail < len(reqs)
    assert out["failed"] == nfail and out["completed"] == len(reqs) - nfail
    assert out["failure_reasons"] == ["SV_ERR_NORM_COLLAPSE"]
    assert all(s.closed for s in fb.created)


def test_server_admits_in_arrival_order_under_a_tight_budget(lib, monkeypatch):
    from paper_1811_05630_gb300 import serve

    reqs = small_requests(16, seed=9)
    budget = max(serve.footprint(r, min(10, r.n)) for r in reqs)  # one request at a time fits
    fb, out = run_server(monkeypatch, reqs, budget)
    assert out["completed"] == len(reqs)
    assert fb.peak <= budget
    adm = [r.admitted for r in sorted(out["results"], key=lambda r: r.rid)]
    assert adm == sorted(adm)


def test_size_classes_and_footprint(lib):
    from paper_1811_05630_gb300 import serve

    assert [serve.size_class(n) for n in (10, 16, 17, 22, 23, 28)] == [0, 0, 1, 1, 2, 2]
    MB = 1 << 20
    # metadata of 2^10 blocks (2 x 8 + 2 x 4 + 2 x 16 + 8 bytes each, plus scalars and tree
    # scratch) fits one 2 MiB page; two arenas at twice the expected compressed state
    assert serve.meta_bytes(20, 10) == 2 * MB
    r = types.SimpleNamespace(n=20, dtype=2, eb=1e-6)  # prior: 8 bytes per amplitude
    assert serve.footprint(r, 10) == 2 * MB + 2 * (2 * 8 * MB)
    r = types.SimpleNamespace(n=20, dtype=1, eb=1e-4)  # prior: 2 bytes per amplitude
    assert serve.footprint(r, 10) == 2 * MB + 2 * (2 * 2 * MB)
    # far below the uncompressed vector once the class is known to compress well
    assert serve.footprint(r, 10, bytes_per_amp=0.1) == 2 * MB + 2 * (2 * MB)
    assert serve.footprint(types.SimpleNamespace(n=28, dtype=2, eb=1e-8), 10, 0.5) < (16 << 28) // 2


def test_footprint_model_follows_the_largest_peak_of_a_class(lib):
    from paper_1811_05630_gb300 import serve

    m = serve.FootprintModel()
    a = C.Request(0, 0.0, "qft", 20, 2, 1e-6, 0, [])
    b = C.Request(1, 0.0, "qft", 22, 2, 1e-6, 0, [])
    other = C.Request(2, 0.0, "random", 20, 2, 1e-6, 0, [])
    assert m.bytes_per_amp(a) == serve.prior_bytes_per_amp(a) == 8.0
    m.observe(a, 2 << 20)  # peak 2 bytes per amplitude
    assert m.bytes_per_amp(b) == 2.5  # 25 % margin, shared by the class
    m.observe(b, 1 << 22)  # a smaller peak does not lower it
    assert m.bytes_per_amp(a) == 2.5
    m.observe(b, 3 << 22)
    assert m.bytes_per_amp(a) == 3.75
    assert m.bytes_per_amp(other) == 8.0


def test_server_counts_unfinished_requests_as_censored(lib, monkeypatch):
    reqs = small_requests(12, seed=4)
    # a budget below every footprint admits nothing: every arrived request is censored, and the
    # percentiles are lower bounds (end of the run minus arrival)
    fb, out = run_server(monkeypatch, reqs, budget=1, time_limit=0.5)
    assert out["completed"] == 0 and out["censored"] == len(reqs)
    assert out["latency_is_lower_bound"] and out["p99_s"] >= out["p50_s"] > 0
    assert out["p50_s_completed"] is None


# ---- tuner candidates ----------------------------------------------------------------------

def test_thread_candidates_follow_the_launch_rule(lib):
    from paper_1811_05630_gb300 import tune

    for b in range(5, 13):
        nv = 2 << b
        want = [t for t in (32, 64, 128, 256) if 2 <= nv // t <= 32]
        assert tune.thread_candidates(b) == want
        assert want, b


def test_best_config_picks_the_fastest_and_caches(lib, monkeypatch, tmp_path):
    from paper_1811_05630_gb300 import tune

    calls = []

    def fake_probe(pool, n, dtype, eb, b, prefix, timed, basis=0, threads=0, compact=False, chunk=32):
        calls.append((b, threads, compact, chunk))
        return 1.0 + abs(b - 10) + (0.0 if compact else 0.5) + (0.0 if threads == 256 else 0.25)

    monkeypatch.setattr(tune, "probe", fake_probe)
    monkeypatch.setattr(tune, "CACHE", str(tmp_path / "tune.json"))
    monkeypatch.setattr(tune, "_key", lambda n, dtype, eb, kind: "k|%d|%d|%g|%s" % (dtype, n, eb, kind))
    pool = types.SimpleNamespace(close=lambda: None)
    res = tune.best_config(20, 2, 1e-8, "grover", [], [], pool=pool, candidates=(9, 10, 11), chunks=(16, 32))
    assert (res["block_log2"], res["threads"], res["compact"]) == (10, 256, True)
    # only valid shapes were probed: chunk count per block within the CTA, compact from 128 threads
    for b, t, c, k in calls:
        assert (2 << b) // k <= t and (not c or t >= 128) and t in tune.thread_candidates(b)
    n1 = len(calls)
    again = tune.best_config(20, 2, 1e-8, "grover", [], [], pool=pool, candidates=(9, 10, 11), chunks=(16, 32))
    assert again["block_log2"] == 10 and len(calls) == n1  # served from the cache file


# ---- seeded circuit generators -------------------------------------------------------------

def test_splitmix64_published_sequence():
    # SplitMix64 (Steele, Lea, Flood 2014) from state 1234567: the state advances by the golden
    # gamma before each output; these are the generator's first five outputs
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423,
            4593380528125082431, 16408922859458223821]
    x = 1234567
    got = []
    for _ in range(5):
        got.append(C.splitmix64(x))
        x = (x + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
    assert got == want


def test_haar_su2_is_special_unitary():
    rng = np.random.Generator(np.random.PCG64(1))
    for _ in range(50):
        U = C.haar_su2(rng)
        assert np.allclose(U.conj().T @ U, np.eye(2), atol=1e-14)
        assert abs(np.linalg.det(U) - 1.0) < 1e-14


def test_brickwork_structure():
    n, depth = 7, 5
    g = C.random_brickwork(n, depth, seed=2)
    per_layer = [n + len(range(layer % 2, n - 1, 2)) for layer in range(depth)]
    assert len(g) == sum(per_layer)
    i = 0
    for layer in range(depth):
        assert [x.targets for x in g[i:i + n]] == [(q,) for q in range(n)]
        cz = g[i + n:i + per_layer[layer]]
        assert [(x.targets, x.controls) for x in cz] == [((q + 1,), (q,)) for q in range(layer % 2, n - 1, 2)]
        i += per_layer[layer]
    assert C.random_brickwork(n, depth, seed=2)[3].matrix.tobytes() == g[3].matrix.tobytes()


def test_grover_gate_list():
    n, marked = 6, 0b101001
    k = C.grover_iterations(n)
    assert k == int(math.floor(math.pi / 4 * math.sqrt(2 ** n)))
    g = C.grover(n, marked)
    zeros = sum(1 for q in range(n) if not (marked >> q) & 1)
    assert len(g) == n + k * (2 * zeros + 1 + 4 * n + 1)
    assert sum(1 for x in g if x.name == "MCZ") == 2 * k


def test_serving_stream_recipe():
    reqs = C.serving_requests(300, rate=20.0, seed=0)
    gaps = np.diff([0.0] + [r.arrival for r in reqs])
    assert np.all(gaps > 0)
    assert abs(gaps.mean() - 1 / 20.0) < 0.25 / 20.0
    assert {r.kind for r in reqs} == {"qft", "grover", "random"}
    assert min(r.n for r in reqs) >= 10 and max(r.n for r in reqs) <= 28
    assert {r.dtype for r in reqs} == {1, 2} and {r.eb for r in reqs} == {1e-4, 1e-6, 1e-8}
    assert [r.rid for r in reqs] == list(range(300))
    again = C.serving_requests(300, rate=20.0, seed=0)
    assert [(r.arrival, r.n, r.basis, len(r.gates)) for r in again] == [(r.arrival, r.n, r.basis, len(r.gates)) for r in reqs]


# ---- bench traffic records -----------------------------------------------------------------

def test_traffic_record_needs_matching_sources_and_shape(monkeypatch, tmp_path):
    import bench

    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "k_pass_demo.md").write_text(
        "text\nTRAFFIC digest=abc block_log2=11 threads=256 compact=1 window=586-606 bytes_per_launch=123 "
        "launches=x_y\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "source_digest", lambda: "abc")
    assert bench.recorded_traffic("demo", 11, 256, True, window="586-606") == (123.0, "x y")
    assert bench.recorded_traffic("demo", 10, 256, True, window="586-606")[0] is None
    assert bench.recorded_traffic("demo", 11, 256, False, window="586-606")[0] is None
    # a line without a chunk size describes the default 32-symbol chunks only
    assert bench.recorded_traffic("demo", 11, 256, True, window="586-606", chunk=16)[0] is None
    # a capture of another window of passes does not describe this run's launches
    assert bench.recorded_traffic("demo", 11, 256, True, window="25-45") == (
        None, "no ncu capture of this window of passes")
    monkeypatch.setattr(bench, "source_digest", lambda: "def")
    assert bench.recorded_traffic("demo", 11, 256, True, window="586-606") == (
        None, "kernel sources changed since the ncu capture")
    assert bench.recorded_traffic("other", 11, 256, True, window="586-606")[0] is None
    (prof / "k_pass_demo16.md").write_text(
        "TRAFFIC digest=def block_log2=11 threads=256 compact=1 chunk=16 window=586-606 bytes_per_launch=7 "
        "launches=z\n")
    assert bench.recorded_traffic("demo16", 11, 256, True, window="586-606", chunk=16) == (7.0, "z")
    assert bench.recorded_traffic("demo16", 11, 256, True, window="586-606")[0] is None


def test_clock_summary_reads_throttle_reasons():
    import bench

    cs = bench.ClockSampler(0)
    cs.rows = [
        ["0", "2070", "2070", "812.3", "0x0000000000000000", "Not Active", "Not Active", "Not Active", "Not Active"],
        ["0", "2055", "2070", "1390.1", "0x0000000000000004", "Not Active", "Not Active", "Not Active", "Active"],
        ["0", "1980", "2070", "1402.0", "0x0000000000000008", "Active", "Not Active", "Not Active", "Active"],
        ["0", "[N/A]", "2070"],  # a malformed line is skipped
    ]
    s = cs.summary()
    assert s["samples"] == 3 and s["sm_mhz"] == 2055.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert bench.ClockSampler(0).summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_dense_stage_start():
    import bench

    # QFT: every gate of the stages of qubits n-1 .. block_log2 (H plus one controlled phase
    # per lower qubit) comes before the first stage that mixes values inside a block
    wl = {"name": "qft34", "n": 34, "block_log2": 11}
    assert bench.start_of_dense_stage(wl) == sum(1 + j for j in range(33, 10, -1))
    gates = C.qft(34)
    i0 = bench.start_of_dense_stage(wl)
    assert gates[i0].name == "H" and gates[i0].targets == (10,)
    # Grover: the first H of the first diffusion, after the initial H layer and the oracle
    # (X on the marked item's zero bits, MCZ, X again): before it every block is constant
    marked = C.seeded_index(11, 20)
    g20 = C.grover(20, marked)
    i0 = bench.start_of_dense_stage({"name": "grover20", "n": 20, "block_log2": 10, "marked": marked})
    zeros = [q for q in range(20) if not (marked >> q) & 1]
    assert i0 == 20 + 2 * len(zeros) + 1
    assert [g.name for g in g20[i0:i0 + 20]] == ["H"] * 20 and g20[i0 - 1].name == "X"
    assert g20[i0 - len(zeros) - 1].name == "MCZ"


def test_qft_window_ends_at_the_last_recoding_pass():
    import bench

    wl = bench.workload("qft34")
    b = wl["block_log2"]
    w0, t0, t1 = bench.timed_window(wl, 20, 5)
    g = wl["gates"]
    assert (t0 - w0, t1 - t0) == (5, 20)
    # the passes after the window are SWAPs of two qubits at or above the block (they move whole
    # blocks and re-emit every stream); every pass of the window recodes blocks
    assert all(x.name == "SWAP" and min(x.targets) >= b for x in g[t1:])
    assert all(bench.recodes_every_block(x, b) for x in g[w0:t1])
    assert g[t1 - 1].name == "SWAP" and g[t1 - 1].targets == (b - 1, 34 - b)
    # the window lies in the dense stage (every block holds more than one nonzero value)
    assert w0 >= bench.start_of_dense_stage(wl)
    assert {x.name for x in g[t0:t1]} >= {"H", "SWAP"}
    with pytest.raises(ValueError):
        bench.timed_window(wl, 700, 5)
