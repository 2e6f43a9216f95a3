"""Benchmark: amplitude-updates/s of the compressed gate pass (Algorithm 1 of Wu et al.,
PMES 2018) on one GB300, with the plain (uncompressed) GPU path and the CPU oracle beside it.

A step is one gate pass over the whole compressed state: every block is decoded,
normalized, has the gate applied and is re-encoded (plus the norm finalization). The
default workload is the QFT on 34 qubits applied to a seeded random basis state (complex128,
eb = 1e-7, slice_log2 = 24, 2048-amplitude blocks, 150 GB pool; 256 GiB uncompressed, beyond
what the plain path can keep beside anything else): the circuit runs untimed up to its dense
stage, the timed steps are its last passes that recode every block (the H and controlled-phase
gates of the low qubits and the SWAPs that couple a low and a high qubit), the rest of the
circuit runs untimed, and the final state's fidelity is taken against the closed form.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
       [--workload qft34|grover20|qft12|random30]
Under torchrun each rank runs an independent replica on its own GPU (the method does not
shard; "replicas only"), rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import re
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1811_05630_gb300 import circuits as C  # noqa: E402
from paper_1811_05630_gb300 import report  # noqa: E402

METRIC = "amplitude-updates/s compressed vs plain at fidelity>=1-1e-6; ratio; p99 latency"
UNIT = "amp-updates/s"


def workload(name: str):
    if name == "grover20":
        n = 20
        marked = C.seeded_index(11, n)
        return dict(name="grover20", n=n, eb=1e-8, slice_log2=14, block_log2=10, dtype=2,
                    gates=C.grover(n, marked), basis=0, marked=marked, pool_gb=8.0,
                    desc="Grover search, 20 qubits, 804 iterations, complex128, eb 1e-8 abs, slice_log2 14")
    if name == "qft34":
        n = 34
        x = C.seeded_index(0, n)
        # the launch shape the tuner picked on QFT dense stages (tuning at 34 qubits would take
        # minutes per candidate): 2048-amplitude blocks, 256 threads, register-capped build;
        # 16-symbol Huffman chunks (every thread decodes: 3.03 ms against 3.33 ms per pass of
        # chunk 32 on the 26-qubit stand-in's window, whose final size is the same)
        return dict(name="qft34", n=n, eb=1e-7, slice_log2=24, block_log2=11, dtype=2, gates=C.qft(n),
                    basis=x, pool_gb=150.0, threads=256, compact=True, chunk=16,
                    desc="QFT on a random basis state, 34 qubits, complex128, eb 1e-7 abs, slice_log2 24, "
                         "compressed pool capped at 150 GB")
    if name in ("qft26p", "qft28p", "qft30p"):
        # the 34-qubit workload's codec work on a state ncu can capture: amplitudes 2^-n/2 at
        # eb 1e-7 2^((34 - n) / 2) have the codes of amplitudes 2^-17 at eb 1e-7 (|q| about 38),
        # same launch shape; two sizes show how a launch's DRAM traffic grows with the state
        n = int(name[3:5])
        eb = 1e-7 * 2.0 ** ((34 - n) / 2)
        return dict(name=name, n=n, eb=eb, slice_log2=24, block_log2=11, dtype=2, gates=C.qft(n),
                    basis=C.seeded_index(0, n), pool_gb=8.0, threads=256, compact=True, chunk=16,
                    desc="QFT on a random basis state, %d qubits, complex128, eb %.3g abs (the codes of the "
                         "34-qubit workload), slice_log2 24" % (n, eb))
    if name == "qft12":
        n = 12
        return dict(name="qft12", n=n, eb=1e-6, slice_log2=8, block_log2=8, dtype=2, gates=C.qft(n),
                    basis=C.seeded_index(0, n), desc="QFT 12 qubits, complex128, eb 1e-6, 16 slices of 256")
    if name == "random30":
        n = 30
        return dict(name="random30", n=n, eb=1e-6, slice_log2=20, block_log2=12, dtype=2,
                    gates=C.random_brickwork(n, 20, seed=0), basis=0,
                    desc="random brickwork, 30 qubits, depth 20, complex128, eb 1e-6, slice_log2 20")
    raise ValueError(name)


def start_of_dense_stage(wl):
    """First pass that recodes every block with values that mix inside the block.
    QFT: the stage of qubit block_log2 - 1 (before it every block holds one nonzero value and
    most passes re-emit blocks unchanged). Grover: the first H layer of the first diffusion
    (before it the state is the uniform superposition, every block constant, and the oracle's
    X gates only permute blocks). Random brickwork: after the first layer of single-qubit
    gates the product state is dense."""
    n = wl["n"]
    if wl["name"].startswith("qft"):
        b = wl["block_log2"]
        return sum(1 + j for j in range(n - 1, b - 1, -1))
    if wl["name"].startswith("grover"):
        zeros = sum(1 for q in range(n) if not (wl["marked"] >> q) & 1)
        return n + 2 * zeros + 1  # initial H layer, oracle (X, MCZ, X), then the diffusion's H layer
    return n


def recodes_every_block(g, b: int) -> bool:
    """Whether a pass of gate g recodes blocks, as opposed to re-emitting every stream (a
    permutation with unit entries whose targets all lie at or above the block, e.g. a SWAP of
    two high qubits, moves whole blocks)."""
    m = np.asarray(g.matrix)
    unit_perm = all(np.count_nonzero(r) == 1 for r in m) and np.all((m == 0) | (m == 1))
    return not (unit_perm and min(g.targets) >= b)


def timed_window(wl, steps: int, warmup: int):
    """(first warm-up pass, first timed pass, end) of the bench's window of consecutive passes.
    QFT: the window ends with the circuit's last pass that recodes blocks (the SWAPs of two
    high qubits after it re-emit every stream) and reaches back as far as the steps need;
    other circuits: the window starts at the dense stage."""
    gates = wl["gates"]
    if wl["name"].startswith("qft"):
        end = max(i for i, g in enumerate(gates) if recodes_every_block(g, wl["block_log2"])) + 1
        t0 = end - steps
        w0 = t0 - warmup
        if w0 < 0:
            raise ValueError("the circuit has %d passes before its last recoding pass; %d requested"
                             % (end, steps + warmup))
        return w0, t0, end
    w0 = start_of_dense_stage(wl)
    if w0 + warmup + steps > len(gates):
        raise ValueError("not enough gates for the requested steps")
    return w0, w0 + warmup, w0 + warmup + steps


class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock and throttle reasons)."""

    def __init__(self, gpu: int):
        self.gpu, self.rows, self.proc = gpu, [], None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except FileNotFoundError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for k, nm in enumerate(names):
                    if r[5 + k].lower().startswith("active"):
                        reasons.add(nm)
            except (ValueError, IndexError):
                pass
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# the device-code sources of the fused pass (host-side files do not change what it moves)
KERNEL_SOURCES = ("sv_block.cuh", "sv_device.cuh", "sv_pass.cuh", "sv_pass_big.cuh", "sv_pass_tc.cuh", "sv_tc.cuh",
                  "sv_pass_compact.cu", "sv_kernels.cu")


def source_digest() -> str:
    """Digest of the fused pass's device sources, to tie an ncu traffic figure to the code it
    measured."""
    import hashlib

    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1811_05630_gb300", "csrc")
    for f in KERNEL_SOURCES:
        h.update(f.encode())
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(workload: str, block_log2: int, threads: int, compact: bool, window: str = "",
                     chunk: int = 32):
    """DRAM bytes per fused-pass launch from the committed ncu summary of this workload, when
    it was taken on these exact kernel sources, this launch configuration (block size, CTA
    size, build, Huffman chunk) and the same window of passes: (bytes, description of the
    captured launches), else (None, why not)."""
    path = os.path.join(ROOT, "profiles", "k_pass_%s.md" % workload)
    why = "no ncu capture recorded for this workload"
    try:
        with open(path) as f:
            for line in f:
                if line.startswith("TRAFFIC "):
                    kv = dict(x.split("=", 1) for x in line.split()[1:])
                    if kv.get("digest") != source_digest():
                        why = "kernel sources changed since the ncu capture"
                        continue
                    if (int(kv["block_log2"]), int(kv["threads"]), bool(int(kv["compact"])),
                            int(kv.get("chunk", "32"))) != (block_log2, threads, bool(compact), chunk):
                        why = "no ncu capture at this launch configuration"
                        continue
                    if kv.get("window", "") != window:
                        why = "no ncu capture of this window of passes"
                        continue
                    return float(kv["bytes_per_launch"]), kv.get("launches", "").replace("_", " ")
    except (OSError, ValueError, KeyError):
        pass
    return None, why


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {"hbm_gbs": 6800.0, "fallback": True}


def grover_fidelity(st, wl, iters):
    """Fidelity of the GPU state with the exact Grover state a|m> + b sum_{x != m}|x>."""
    n, m = wl["n"], wl["marked"]
    th = math.asin(2.0 ** (-n / 2))
    N = 1 << n
    a = math.sin((2 * iters + 1) * th)
    b = math.cos((2 * iters + 1) * th) / math.sqrt(N - 1)
    v = st.read()
    ov = a * v[m] + b * (v.sum() - v[m])
    return abs(ov) ** 2 / np.vdot(v, v).real, abs(v[m]) ** 2 / np.vdot(v, v).real


def log(msg: str) -> None:
    """Progress on stderr (the JSON line is the only stdout output)."""
    print("[bench %.0f s] %s" % (time.time() - T_START, msg), file=sys.stderr, flush=True)


T_START = time.time()


def max_over_ranks(x: float, dist) -> float:
    """The largest x over the ranks of the process group (x itself without one): replicas are
    timed each on its own GPU and the job takes as long as the slowest."""
    if not dist:
        return x
    import torch

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _oracle_sample(wl, steps: int, warmup: int, nmax: int = 20):
    """The oracle's share of the workload: the same circuit family and parameters on
    n = min(n, nmax) qubits, at the same place of its circuit as the GPU's timed window (the
    window of that smaller circuit). Returns (n, first pass, gates of the window)."""
    n = min(wl["n"], nmax)
    b = min(wl["block_log2"], n)
    sw = dict(wl, n=n, block_log2=b)
    if n < wl["n"]:
        if wl["name"].startswith("grover"):
            sw["marked"] = C.seeded_index(11, n)
            sw["gates"] = C.grover(n, sw["marked"])
        elif wl["name"].startswith("qft"):
            sw["gates"] = C.qft(n)
        else:
            sw["gates"] = C.random_brickwork(n, 20, seed=0)
    sw["basis"] = wl["basis"] & ((1 << n) - 1)
    end = len(sw["gates"])
    want = min(steps + warmup, end)
    try:
        w0, _, end = timed_window(sw, want - min(warmup, want - 1), min(warmup, want - 1))
    except ValueError:
        w0 = max(0, end - want)
    return sw, w0, sw["gates"][w0:end]


def _oracle_at(sw, w0):
    """The oracle's Algorithm 1 state at pass w0 of the sample circuit: the exact state there
    (the plain oracle runs the passes before it, untimed) compressed by the oracle codec."""
    import oracle

    n = sw["n"]
    ps = oracle.PlainSim(n, sw["dtype"], sw["basis"]).run(sw["gates"][:w0])
    cs = oracle.CompressedSim(n, min(sw["slice_log2"], n), sw["block_log2"], sw["dtype"], sw["eb"], 0,
                              chunk=sw.get("chunk", 32))
    cs.load(ps.state)
    return cs


def _oracle_worker(sw, w0, gates, warmup, budget_s, barrier, out):
    """One host process: warm-up passes, then timed passes of the window until the CPU-time
    budget runs out or the window ends (a sample of the workload, not the whole of it)."""
    cs = _oracle_at(sw, w0)
    for g in gates[:warmup]:
        cs.apply(g.matrix, g.targets, g.controls)
    if barrier is not None:
        barrier.wait()
    t0 = time.process_time()
    w = time.time()
    done = 0
    for g in gates[warmup:]:
        cs.apply(g.matrix, g.targets, g.controls)
        done += 1
        if budget_s and time.process_time() - t0 > budget_s:
            break
    out.put((done, time.time() - w))


def oracle_throughput(sw, w0, gates, warmup, budget_s, procs: int):
    """Amplitude-updates/s of the oracle (as it stands, single-threaded C) on `procs` host
    processes at once, each running the same sample (processes started with spawn)."""
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    bar = ctx.Barrier(procs) if procs > 1 else None
    ps = [ctx.Process(target=_oracle_worker, args=(sw, w0, gates, warmup, budget_s, bar, out))
          for _ in range(procs)]
    for p in ps:
        p.start()
    res = [out.get() for _ in ps]
    for p in ps:
        p.join()
    done = sum(r[0] for r in res)
    wall = max(r[1] for r in res)
    return (1 << sw["n"]) * done / wall, done, wall


def cpu_oracle_sample(wl, steps, warmup, budget_s=15.0):
    """The oracle (Algorithm 1 in plain C, as it stands) on the host cores: one thread, and one
    process per core, on the same circuit family at the place of the GPU's window."""
    sw, w0, gates = _oracle_sample(wl, steps, warmup)
    wu = min(warmup, max(0, len(gates) - 1))
    cores = os.cpu_count() or 1
    v1, d1, t1 = oracle_throughput(sw, w0, gates, wu, budget_s, 1)
    vn, dn, tn = oracle_throughput(sw, w0, gates, wu, budget_s, cores)
    what = ("passes %d..%d of the %s circuit on %d qubits (the same place of its circuit as the GPU "
            "window; exact state there compressed by the oracle codec), oracle Algorithm 1 in plain C"
            % (w0 + wu, w0 + len(gates) - 1, wl["name"].rstrip("0123456789"), sw["n"]))
    return dict(value=vn, unit=UNIT, cores=cores, kind="oracle",
                sample="%s; %d independent processes (one per host core), %d passes in %.1f s"
                       % (what, cores, dn, tn),
                one_thread={"value": v1, "cores": 1, "passes": d1, "wall_s": t1}, nproc=cores)


def run_reference(args, rank, world):
    """The oracle as the reference arm, on the host cores of rank 0: every step is one
    Algorithm 1 pass over the 20-qubit instance of the workload's circuit (a bounded sample of
    one pass of the workload), run by one process per core at once."""
    wl = workload(args.workload)
    if rank != 0:
        return None
    sw, w0, gates = _oracle_sample(wl, args.steps, args.warmup)
    wu = min(args.warmup, max(0, len(gates) - 1))
    # every process runs exactly the warm-up and timed passes (no time budget)
    gates = gates[: wu + args.steps]
    cores = os.cpu_count() or 1
    val, done, wall = oracle_throughput(sw, w0, gates, wu, 0.0, cores)
    steps = done // cores
    sample = ("one Algorithm 1 pass per step over 2^%d amplitudes of the %s circuit (passes %d..%d of its "
              "%d-qubit instance, the place of the GPU window), oracle in plain C, %d processes (one per core)"
              % (sw["n"], wl["name"].rstrip("0123456789"), w0 + wu, w0 + wu + steps - 1, sw["n"], cores))
    return {"metric": METRIC, "value": val, "unit": UNIT, "impl": "reference", "n_gpus": world,
            "steps": steps, "warmup": wu, "ms_per_step": wall * 1e3 / max(steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if wl["dtype"] == 2 else "f32", "data": "synthetic",
            "config": {"workload": wl["desc"], "sample": sample},
            "cpu_baseline": {"kind": "oracle", "cores": cores, "value": val, "unit": UNIT, "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_ours(args, rank, world, dist):
    import torch

    from paper_1811_05630_gb300 import sv

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    wl = workload(args.workload)
    n = wl["n"]
    gates = wl["gates"]
    tuned = None
    if args.block_log2:
        wl["block_log2"] = args.block_log2
    elif args.autotune and n <= 30 and not wl.get("threads"):
        from paper_1811_05630_gb300 import tune

        i0t = start_of_dense_stage(wl)
        tuned = tune.best_config(n, wl["dtype"], wl["eb"], wl["name"], gates[:i0t], gates[i0t:i0t + 200],
                                 basis=wl["basis"], use_cache=False, chunks=(16, 32))
        wl["block_log2"] = tuned["block_log2"]
        wl["threads"] = tuned["threads"]
        wl["compact"] = tuned["compact"]
        wl["chunk"] = tuned["chunk"]
    w0, t0, t1 = timed_window(wl, args.steps, args.warmup)
    if args.threads:
        wl["threads"] = args.threads
    if args.compact:
        wl["compact"] = True
    if args.chunk:
        wl["chunk"] = args.chunk
    pool_bytes = int((args.pool_gb or wl.get("pool_gb", 8.0)) * (1 << 30))
    pool = sv.Pool(pool_bytes)
    arena = args.arena_mb << 20
    if not arena:
        # arenas sized for the largest possible streams (every block PACK at 32 bits plus its
        # verbatim section) when that is small, so no pass can overflow and be replayed
        nv = 2 << wl["block_log2"]
        verb = 10 * min(nv, 128) if wl["dtype"] == 2 else 6 * nv
        worst = (1 << (n - wl["block_log2"])) * (16 + 4 * nv + verb + 32)
        arena = worst if worst <= (512 << 20) else 0
    st = sv.State(pool, n, wl["slice_log2"], wl["eb"], wl["dtype"], block_log2=wl["block_log2"],
                  arena_bytes=arena)
    if wl.get("threads"):
        st.set_threads(wl["threads"])
    st.set_compact(bool(wl.get("compact")))
    if wl.get("chunk", 32) != 32:
        st.set_chunk(wl["chunk"])
    t_setup = time.time()
    st.reset_basis(wl["basis"])
    st.run(gates[:t0])  # untimed: the circuit up to the window, then the warm-up passes
    st.sync()
    t_setup = time.time() - t_setup
    log("reached pass %d in %.1f s (compressed %d bytes)" % (t0, t_setup, st.compressed_bytes()))
    timed = gates[t0:t1]
    b = wl["block_log2"]
    st.set_pass_timing(True)
    stream = torch.cuda.current_stream()
    # L2 (126 MiB) is flushed between timed steps by writing a 512 MiB buffer on the same
    # stream, outside every step's timed interval
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in timed]
    stats0 = st.stats()
    replays0 = stats0["replayed_passes"]
    bytes_before = stats0["compressed_bytes"]
    # every step goes through the public API with host buffers: its gate is written to pinned
    # host memory and handed to sv_apply_gate (which copies it to the device with the launch),
    # and the step's result, the stored norm, is read back to the host. The CUDA events give
    # the device time of the step's kernels (`value`), the host clock the end-to-end time.
    pin = torch.empty(16 * 32 * 32, dtype=torch.uint8).pin_memory()
    h2d = d2h = 0
    e2e_s = 0.0
    reused = 0
    per_step_bytes = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if args.profile_window:  # ncu --profile-from-start off captures exactly the timed passes
        torch.cuda.cudart().cudaProfilerStart()
    with ClockSampler(dev) as clk:
        for i, g in enumerate(timed):
            flush.fill_(i & 0xFF)
            torch.cuda.synchronize()
            h0 = time.perf_counter()
            gm = np.ascontiguousarray(g.matrix, dtype=np.complex128)
            pin_view = pin.numpy()[: gm.nbytes]
            pin_view[:] = gm.view(np.uint8).reshape(-1)
            ev[i][0].record(stream)
            st.apply(pin_view.view(np.complex128).reshape(gm.shape), g.targets, g.controls)
            ev[i][1].record(stream)
            st.norm()
            e2e_s += time.perf_counter() - h0
            h2d += gm.nbytes + 4 * (len(g.targets) + len(g.controls))
            d2h += 8
            sti = st.stats()  # already synchronized: the pinned copy of the scalars
            reused += sti["blocks_reused"]
            per_step_bytes.append(sti["compressed_bytes"])
        st.sync()
        torch.cuda.synchronize()
    if args.profile_window:
        torch.cuda.cudart().cudaProfilerStop()
    ms = sum(a.elapsed_time(c) for a, c in ev)
    kern_ms, npass, alg_bytes = st.pass_timing()
    stats = st.stats()
    replays = stats["replayed_passes"] - replays0
    nblocks = stats["n_blocks"]
    ms = max_over_ranks(ms, dist)
    e2e_s = max_over_ranks(e2e_s, dist)
    value = (1 << n) * len(timed) * world / (ms * 1e-3)
    e2e = {"value": (1 << n) * len(timed) * world / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": h2d // len(timed), "d2h_bytes_per_step": d2h // len(timed),
           "what": "the timed passes through sv_apply_gate with the gate copied from pinned host memory and "
                   "the stored norm read back after every step (host clock)"}
    # the rest of the circuit, untimed, and the final state's fidelity
    fid = None
    t_rest = time.time()
    if wl["name"].startswith("qft") and args.fidelity:
        st.run(gates[t1:])
        st.sync()
        F = st.fidelity_qft(wl["basis"])
        fid = {"fidelity_vs_closed_form": F, "one_minus_F": 1.0 - F, "gates": len(gates),
               "final_compressed_bytes": st.compressed_bytes(),
               "what": "whole circuit; overlap with 2^{-n/2} sum_y exp(2 pi i x y / 2^n) computed on the GPU "
                       "from the decoded state"}
    t_rest = time.time() - t_rest
    pool_used = pool.usage()[0]
    # release the compressed state's pool before the plain vector and the serving run
    st.close()
    pool.close()
    del st, pool
    import gc

    gc.collect()
    torch.cuda.empty_cache()
    log("timed window done: %.3g amp-updates/s, setup %.0f s, rest %.0f s, fidelity %s"
        % (value, t_setup, t_rest, fid and fid.get("one_minus_F")))

    result = None
    if rank == 0:
        pk = peaks()
        kern_s = kern_ms * 1e-3
        achieved = alg_bytes / kern_s / 1e9 if kern_s > 0 else 0.0
        # the default CTA size is one thread per 32-value decode chunk, 32 to 256 threads
        eff_threads = int(wl.get("threads") or min(256, max(32, (2 << b) // 32)))
        traffic, traffic_src = recorded_traffic(wl["name"], b, eff_threads, bool(wl.get("compact")),
                                                window="%d-%d" % (t0, t1), chunk=wl.get("chunk", 32))
        roof = {"bound": "hbm", "achieved": achieved, "peak": pk.get("hbm_gbs"), "unit": "GB/s",
                "frac": achieved / pk.get("hbm_gbs", 1.0), "traffic": traffic,
                "traffic_source": traffic_src, "source_digest": source_digest(),
                "kernel": "k_pass_c / k_pass_c3 (fused pass, register-capped builds for 1- and 2-qubit "
                          "gates)" if wl.get("compact") else "k_pass (fused pass)", "kernel_ms_per_launch": kern_ms / max(npass, 1),
                "alg_bytes_per_launch": alg_bytes / max(npass, 1), "launches": npass,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured copy bandwidth)"
                if "fallback" not in pk else "fallback 6.8 TB/s"}
        # the oracle on the host cores: at N = 1 only (under torchrun the host's cores serve
        # every rank's replica)
        cpu = (cpu_oracle_sample(wl, args.steps, args.warmup, budget_s=args.cpu_budget)
               if args.cpu_budget > 0 and world == 1 else None)
        log("cpu baseline: %s" % (cpu and cpu["value"]))
        # plain GPU path on the same gates, where its vector fits: its time does not depend on
        # the amplitudes' values, so it runs from the basis state
        plain = None
        if args.plain:
            try:
                ppool = sv.Pool(((16 if wl["dtype"] == 2 else 8) << n) + (64 << 20))
                ps = sv.State(ppool, n, n, 0.0, wl["dtype"])
                ps.reset_basis(wl["basis"])
                ps.sync()
                for g in gates[w0:t0]:
                    ps.apply(g.matrix, g.targets, g.controls)
                torch.cuda.synchronize()
                for i, g in enumerate(timed):
                    flush.fill_(i & 0xFF)
                    ev[i][0].record(stream)
                    ps.apply(g.matrix, g.targets, g.controls)
                    ev[i][1].record(stream)
                torch.cuda.synchronize()
                pms = sum(a.elapsed_time(c) for a, c in ev)
                plain = (1 << n) * len(timed) / (pms * 1e-3)
                ps.close()
                ppool.close()
                del ps, ppool
            except Exception as ex:  # noqa: BLE001
                plain = "unavailable: %s" % ex
            log("plain path: %s" % plain)
        del flush
        if fid is None and args.fidelity and wl["name"] == "grover20":
            fid = full_grover_fidelity(sv, wl)
        serving = None
        if args.serve_in_bench > 0:
            gc.collect()
            torch.cuda.empty_cache()
            try:
                serving = serving_run(args.serve_in_bench, args.serve_rate, args.serve_in_bench_limit,
                                      args.pool_gb or 150.0, args.serve_budget_gb)
                log("serving: p50 %s p99 %s completed %d censored %d" % (
                    serving["p50_s"], serving["p99_s"], serving["completed"], serving["censored"]))
            except Exception as ex:  # noqa: BLE001
                serving = {"error": "%s: %s" % (type(ex).__name__, ex)}
        launches_per_pass = 2  # the fused pass and the one-CTA norm kernel
        raw = report.raw_state_bytes(n, wl["dtype"])
        result = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": len(timed),
            "warmup": t0 - w0, "ms_per_step": ms / len(timed), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if wl["dtype"] == 2 else "f32",
            "data": "synthetic",
            "config": {"workload": wl["desc"], "block_log2": b,
                       "threads_per_cta": wl.get("threads") or "default",
                       "register_capped_build": bool(wl.get("compact")), "huffman_chunk": wl.get("chunk", 32),
                       "autotune": tuned if tuned else "not run above 30 qubits (fixed shape)",
                       "timed_passes": [t0, t1], "warmup_passes": [w0, t0],
                       "timed_gates": sorted({g.name for g in timed}),
                       "blocks_reused_fraction": reused / (len(timed) * nblocks),
                       "untimed_setup_s": t_setup, "untimed_rest_s": t_rest,
                       "arena_bytes": arena, "replayed_passes_in_timed_region": replays,
                       "parallelism": "replicas",
                       "l2": "flushed between timed steps (512 MiB write, untimed)",
                       "compressed_bytes_before_window": bytes_before,
                       "compressed_bytes_per_step": per_step_bytes,
                       "compression_ratio_min_in_window": raw / max(per_step_bytes),
                       "pool_used_bytes": pool_used,
                       "plain_amp_updates_per_s": plain,
                       "ratio_plain_over_compressed": (plain / (value / world)) if isinstance(plain, float) else None,
                       "fidelity": fid},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk.summary(),
            "gpu_launches": launches_per_pass * len(timed),
            "serving": serving,
        }
    return result


def full_grover_fidelity(sv, wl):
    """Run the whole Grover circuit (outside the timed region) and report its fidelity."""
    import torch

    pool = sv.Pool(1 << 30)
    st = sv.State(pool, wl["n"], wl["slice_log2"], wl["eb"], wl["dtype"], block_log2=wl["block_log2"])
    st.reset_basis(0)
    st.run(wl["gates"])
    st.sync()
    iters = C.grover_iterations(wl["n"])
    F, p = grover_fidelity(st, wl, iters)
    st.close()
    pool.close()
    torch.cuda.synchronize()
    return {"fidelity_vs_exact": F, "p_marked": p, "iterations": iters, "passes": len(wl["gates"])}


def run_full_circuit(args):
    """Whole-circuit run (QFT34 is the target configuration): every pass, compressed bytes
    after every gate, exact fidelity against the closed form, marginal probabilities, and
    the plain GPU path timed on the same dense-stage gates where its vector fits."""
    import torch

    from paper_1811_05630_gb300 import sv

    wl = workload(args.workload)
    if args.n and args.n != wl["n"]:  # the same circuit family on another qubit count
        n2 = args.n
        if wl["name"].startswith("qft"):
            wl.update(gates=C.qft(n2), basis=C.seeded_index(0, n2))
        elif wl["name"].startswith("random"):
            wl.update(gates=C.random_brickwork(n2, 20, seed=0))
        else:
            raise ValueError("--n applies to the QFT and random workloads")
        wl["desc"] = wl["desc"].replace("%d qubits" % wl["n"], "%d qubits" % n2)
        wl.update(n=n2, slice_log2=min(wl["slice_log2"], n2))
    if args.block_log2:
        wl["block_log2"] = args.block_log2
    if args.eb:
        wl["desc"] = re.sub(r"eb [0-9.eE+-]+", "eb %.3g" % args.eb, wl["desc"], count=1)
        wl["eb"] = args.eb
    if args.dtype:
        wl["dtype"] = {"c128": 2, "c64": 1}[args.dtype]
        if args.dtype == "c64":
            wl["desc"] = wl["desc"].replace("complex128", "complex64")
    n, gates = wl["n"], wl["gates"]
    unfused = len(gates)
    if args.fuse:
        # gates fused into dense unitaries of up to 5 qubits (at most 2 at or above the block);
        # amplitude-updates still count the original circuit's gates
        gates = C.fuse(gates, 5, block_log2=wl["block_log2"])
    pool = sv.Pool(int((args.pool_gb or wl.get("pool_gb", 8.0)) * (1 << 30)))
    st = sv.State(pool, n, wl["slice_log2"], wl["eb"], wl["dtype"], block_log2=wl["block_log2"],
                  arena_bytes=args.arena_mb << 20)
    host = None
    if args.spill_gb:  # arenas beyond the device pool go to pinned host memory
        host = sv.Pool(int(args.spill_gb * (1 << 30)), "host")
        st.set_spill(host)
    if args.threads:
        st.set_threads(args.threads)
    st.set_compact(args.compact)
    if not args.tensor_cores:
        st.set_tensor_cores(False)
    if args.chunk and args.chunk != 32:
        st.set_chunk(args.chunk)
    st.reset_basis(wl["basis"])
    st.sync()
    raw = report.raw_state_bytes(n, wl["dtype"])
    per_gate = []
    reused = 0
    stream = torch.cuda.current_stream()
    t_all = time.time()
    kern_total = 0.0
    st.set_pass_timing(True)
    with ClockSampler(0) as clk:
        for i, g in enumerate(gates):
            try:
                st.apply(g.matrix, g.targets, g.controls)
                stt = st.stats()  # synchronizes: per-gate compressed size
            except sv.SvError as ex:
                # e.g. every amplitude quantized to zero (a bound far above the amplitudes)
                return {"workload": wl["desc"], "dtype": wl["dtype"], "eb": wl["eb"], "gates_done": i,
                        "error": str(ex), "bytes_per_gate": per_gate}
            per_gate.append(stt["compressed_bytes"])
            reused += stt["blocks_reused"]
    wall = time.time() - t_all
    kern_ms, npass, alg_bytes = st.pass_timing()
    x = wl["basis"]
    fid = st.fidelity_qft(x) if wl["name"].startswith("qft") else None
    m = min(10, n)
    p = st.probs(list(range(m)))
    pool_used, pool_cap = pool.usage()
    rng = np.random.default_rng(1)
    idx = rng.integers(0, 1 << n, size=2000, dtype=np.uint64)
    amps = st.amplitudes(idx)
    norm = st.norm()
    samp = np.abs(amps) ** 2 / norm * (1 << n)
    res = {
        "workload": wl["desc"], "dtype": wl["dtype"], "eb": wl["eb"],
        "block_log2": wl["block_log2"], "threads_per_cta": args.threads or "default",
        "register_capped_build": args.compact, "huffman_chunk": args.chunk or 32,
        "gates": unfused, "passes": len(gates), "fused": bool(args.fuse),
        "tensor_cores": bool(args.tensor_cores) and wl["dtype"] == 2,
        "blocks_reused_fraction": reused / (len(gates) * stt["n_blocks"]),
        "replayed_passes": stt["replayed_passes"],
        "amp_updates_per_s_wall": (1 << n) * unfused / wall,
        "amp_updates_per_s_kernel": (1 << n) * unfused / (kern_ms * 1e-3) if kern_ms else None,
        "passes_per_s_kernel": npass / (kern_ms * 1e-3) if kern_ms else None,
        "kernel_ms_total": kern_ms, "wall_s": wall, "fused_kernel_gbs": alg_bytes / (kern_ms * 1e-3) / 1e9,
        "fidelity_vs_closed_form": fid,
        "compression_ratio_final": raw / per_gate[-1], "compression_ratio_min": raw / max(per_gate),
        "memory_fraction_max": report.memory_fraction(raw / max(per_gate)),
        "extra_qubits_at_min_ratio": report.extra_qubits(raw / max(per_gate)),
        "compressed_bytes_max": max(per_gate), "compressed_bytes_final": per_gate[-1],
        "marginal_probs_max_abs_dev_from_uniform": float(np.abs(p - 2.0 ** -m).max()),
        "sampled_prob_ratio_mean": float(samp.mean()), "sampled_prob_ratio_std": float(samp.std()),
        "pool_used_bytes": pool_used, "clocks": clk.summary(),
        "spill_pool_gb": args.spill_gb or None,
        "spill_used_bytes_end": host.usage()[0] if host is not None else None,
        "spill_arena_bytes_end": stt.get("spill_arena_bytes"),
        "bytes_per_gate": per_gate,
    }
    if fid is None and args.plain:
        # no closed form: the plain GPU path runs the whole circuit beside the compressed
        # state. The fidelity reference is the FP64 (complex128) plain state whatever the
        # compressed dtype, so a complex64 run states its error against FP64; the plain path of
        # the compressed run's own dtype is what the speed is compared with.
        try:
            raw128 = report.raw_state_bytes(n, 2)
            ppool = sv.Pool(raw128 + (wl["dtype"] == 1) * raw + (256 << 20))
            ref = sv.State(ppool, n, n, 0.0, 2)
            ref.reset_basis(x)
            ref.sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ref.run(gates)
            e1.record(stream)
            torch.cuda.synchronize()
            res["fidelity_vs_fp64_plain"] = st.fidelity(ref)
            t_plain = e0.elapsed_time(e1)
            if wl["dtype"] == 1:
                ps = sv.State(ppool, n, n, 0.0, 1)
                ps.reset_basis(x)
                ps.sync()
                e0.record(stream)
                ps.run(gates)
                e1.record(stream)
                torch.cuda.synchronize()
                t_plain = e0.elapsed_time(e1)
                res["fidelity_complex64_plain_vs_fp64_plain"] = ps.fidelity(ref)
                ps.close()
            res["plain_amp_updates_per_s_whole_circuit"] = (1 << n) * unfused / (t_plain * 1e-3)
            ref.close()
            ppool.close()
        except Exception as ex:  # noqa: BLE001
            res["plain_amp_updates_per_s_whole_circuit"] = "unavailable: %s" % ex
        st.close()
        pool.close()
        return res
    st.close()
    pool.close()
    del st, pool
    import gc

    gc.collect()
    torch.cuda.empty_cache()
    if args.plain:
        try:
            i0 = start_of_dense_stage(wl)
            sel = gates[i0:i0 + args.steps]
            ppool = sv.Pool(raw + (64 << 20))
            ps = sv.State(ppool, n, n, 0.0, wl["dtype"])
            ps.reset_basis(x)
            ps.sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ps.run(sel)
            e1.record(stream)
            torch.cuda.synchronize()
            res["plain_amp_updates_per_s_dense_stage"] = (1 << n) * len(sel) / (e0.elapsed_time(e1) * 1e-3)
            ps.close()
            ppool.close()
        except Exception as ex:  # noqa: BLE001
            res["plain_amp_updates_per_s_dense_stage"] = "unavailable: %s" % ex
    return res


def serving_run(count: int, rate: float, time_limit: float, pool_gb: float, budget_gb: float):
    """The mixed request stream through the continuous-batching loop: the first `count`
    requests of the seeded stream (Poisson arrivals at `rate` per second; QFT / Grover /
    brickwork, 10-28 qubits, both dtypes, three bounds), until every one is done or the time
    limit; requests still queued or running at the limit are counted as censored."""
    from paper_1811_05630_gb300.serve import Server, size_class

    reqs = C.serving_requests(count=count, rate=rate, seed=0)
    srv = Server(pool_bytes=int(pool_gb * (1 << 30)), budget_bytes=int(budget_gb * 1e9),
                 block_log2=10, max_batch=64, graphs=True)
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        out = srv.run(reqs, time_limit=time_limit)
    res = out.pop("results")
    out["failed_requests"] = [{"rid": r.rid, "kind": reqs[r.rid].kind, "n": reqs[r.rid].n,
                               "dtype": reqs[r.rid].dtype, "eb": reqs[r.rid].eb, "error": r.error}
                              for r in res if r.error]
    by = {}
    for r in res:
        if r.error:
            continue
        by.setdefault(size_class(reqs[r.rid].n), []).append(r.latency)
    names = ["n<=16", "17-22", "23-28"]
    out["completed_by_size_class"] = {names[c]: len(v) for c, v in sorted(by.items())}
    out["p50_s_by_size_class"] = {names[c]: float(np.percentile(v, 50)) for c, v in sorted(by.items())}
    out["p99_s_by_size_class"] = {names[c]: float(np.percentile(v, 99)) for c, v in sorted(by.items())}
    arrived = [r for r in reqs if r.arrival <= out["wall_s"]]
    out["arrived_within_limit"] = len(arrived)
    out["offered_within_limit_amp_updates_per_s"] = sum(r.amp_updates for r in arrived) / out["wall_s"]
    out["config"] = {"requests": count, "rate_per_s": rate, "budget_gb": budget_gb, "pool_gb": pool_gb,
                     "time_limit_s": time_limit, "block_log2": 10, "threads_per_cta": 128, "max_batch": 64,
                     "graphs": True, "admission": "estimated compressed footprint (learned per class) and "
                                                   "actual pool usage under the budget"}
    out["clocks"] = clk.summary()
    srv.close()
    return out


def run_serving(args):
    """The serving stream on its own (2000 requests at 20/s by default) for --serve-seconds."""
    return serving_run(args.serve_count, args.serve_rate, args.serve_seconds, args.pool_gb or 150.0,
                       args.serve_budget_gb)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="qft34", choices=["qft34", "qft26p", "qft28p", "qft30p", "grover20", "qft12", "random30"])
    ap.add_argument("--block-log2", type=int, default=0)
    ap.add_argument("--threads", type=int, default=0, help="CTA size of the fused pass (0: tuned/default)")
    ap.add_argument("--compact", action="store_true", help="register-capped build of the fused pass")
    ap.add_argument("--chunk", type=int, default=0, help="Huffman chunk size (16, 32, 64; 0: tuned/32)")
    ap.add_argument("--eb", type=float, default=0.0, help="override the workload's error bound (full-circuit mode)")
    ap.add_argument("--dtype", choices=["c128", "c64"], default=None, help="override the workload's dtype (full-circuit mode)")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="use the workload's fixed block size instead of tuning it")
    ap.add_argument("--pool-gb", type=float, default=0.0, help="device pool (GB; 0: the workload's default)")
    ap.add_argument("--arena-mb", type=int, default=0)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-plain", dest="plain", action="store_false")
    ap.add_argument("--no-fidelity", dest="fidelity", action="store_false")
    ap.add_argument("--full-circuit", action="store_true",
                    help="run the whole circuit once (per-gate sizes, closed-form fidelity)")
    ap.add_argument("--n", type=int, default=0, help="full-circuit mode: the workload's circuit on n qubits")
    ap.add_argument("--spill-gb", type=float, default=0.0,
                    help="full-circuit mode: a pinned host-memory spill pool (GB) for arenas beyond the device pool")
    ap.add_argument("--profile-window", action="store_true",
                    help="bracket the timed passes with cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    ap.add_argument("--no-tensor-cores", dest="tensor_cores", action="store_false",
                    help="full-circuit mode: 4- and 5-qubit gates on the CUDA cores only")
    ap.add_argument("--fuse", action="store_true",
                    help="full-circuit mode: fuse the circuit into dense gates of up to 5 qubits")
    ap.add_argument("--serve", action="store_true", help="serve the mixed request stream")
    ap.add_argument("--serve-count", type=int, default=2000)
    ap.add_argument("--serve-rate", type=float, default=20.0)
    ap.add_argument("--serve-seconds", type=float, default=90.0)
    ap.add_argument("--serve-budget-gb", type=float, default=120.0)
    ap.add_argument("--serve-in-bench", type=int, default=100,
                    help="requests of the serving stream run after the timed passes (0: none)")
    ap.add_argument("--serve-in-bench-limit", type=float, default=120.0,
                    help="wall-time limit of that serving run (unfinished requests are censored)")
    args = ap.parse_args()
    if args.full_circuit:
        print(json.dumps(run_full_circuit(args)))
        return
    if args.serve:
        print(json.dumps(run_serving(args)))
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if args.impl == "reference":
        res = run_reference(args, rank, world)
    else:
        if world > 1:
            import torch.distributed as dist_mod

            dist_mod.init_process_group("nccl")
            dist = dist_mod
        res = run_ours(args, rank, world, dist)
        if dist:
            dist.barrier()
            dist.destroy_process_group()
    if rank == 0 and res is not None:
        print(json.dumps(res))


if __name__ == "__main__":
    main()
