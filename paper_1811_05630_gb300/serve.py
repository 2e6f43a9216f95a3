"""Continuous-batching request loop over compressed state vectors.

Requests (circuit simulations of uneven size, dtype and error bound) arrive over time; each is
admitted when its estimated compressed pool footprint fits the budget, gets a compressed state
on the device, and from then on advances by one gate per step, batched with every other active
request of the same (dtype, block size) in one fused pass launch (sv_batch_apply, optionally
replayed from CUDA graphs). Requests that finish leave the batch and free their memory;
waiting ones are admitted as room appears. The loop records each request's latency
(completion - arrival) and the served amplitude-updates.

The footprint estimate is the compressed size, not the uncompressed vector: a state holds its
metadata and two arenas, each reserved at about twice the live compressed state, so the
estimate is the metadata plus four times the expected compressed bytes. The expected bytes per
amplitude start from a conservative prior per (circuit kind, dtype, error bound) and follow the
largest compressed size the requests of that class have reached; admission also checks the
pool's actual usage, since arenas grow on overflow while a request runs.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field
from typing import Dict, List, Optional

import numpy as np
import torch

from . import sv
from .circuits import Request


@dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    done: float
    amp_updates: int
    streams: Optional[List[bytes]] = None
    norm: Optional[float] = None
    error: Optional[str] = None  # e.g. SV_ERR_NORM: every amplitude quantized to zero

    @property
    def latency(self) -> float:
        return self.done - self.arrival


PAGE = 2 << 20


def meta_bytes(n: int, block_log2: int) -> int:
    """Pool bytes of a compressed state's metadata run (scalars, two offset and length tables,
    two block-summary tables, per-block verbatim sums, tree scratch), page-rounded."""
    nb = 1 << (n - block_log2)
    m = 256 + 2 * 8 * nb + 2 * 4 * nb + 2 * 16 * nb + 8 * nb + 16 * (nb // 256 + 1) + 8 * 256
    return -(-m // PAGE) * PAGE


def prior_bytes_per_amp(req: Request) -> float:
    """Conservative compressed bytes per amplitude before any request of the class finished:
    half the uncompressed size (the codec's verbatim and escape paths can approach it at tight
    bounds on small states), a quarter at the loose bound."""
    raw = 16.0 if req.dtype == 2 else 8.0
    return raw * (0.25 if req.eb >= 1e-4 else 0.5)


def footprint(req: Request, block_log2: int, bytes_per_amp: float | None = None) -> int:
    """Pool bytes reserved at admission: metadata plus two arenas, each reserved at about twice
    the expected compressed state (arenas still grow on overflow while the request runs)."""
    bpa = prior_bytes_per_amp(req) if bytes_per_amp is None else bytes_per_amp
    live = int(bpa * (1 << req.n))
    arena = max(PAGE, -(-2 * live // PAGE) * PAGE)
    return meta_bytes(req.n, block_log2) + 2 * arena


class FootprintModel:
    """Expected compressed bytes per amplitude per request class (kind, dtype, error bound):
    the prior until a request of the class completes, then the largest peak seen in the class
    (the compressed size reached by any pass) with a 25 % margin."""

    def __init__(self):
        self.seen = {}

    @staticmethod
    def key(req: Request):
        return (req.kind, req.dtype, req.eb)

    def bytes_per_amp(self, req: Request) -> float:
        return self.seen.get(self.key(req), prior_bytes_per_amp(req))

    def observe(self, req: Request, peak_bytes: int) -> None:
        v = 1.25 * peak_bytes / float(1 << req.n)
        k = self.key(req)
        self.seen[k] = max(v, self.seen.get(k, 0.0)) if k in self.seen else v


def size_class(n: int) -> int:
    """Requests of similar size share a batch (a step lasts as long as its largest pass)."""
    return 0 if n <= 16 else (1 if n <= 22 else 2)


class Server:
    def __init__(self, pool_bytes: int, budget_bytes: int, block_log2: int = 10, max_batch: int = 64,
                 graphs: bool = True, keep_results: bool = False, threads: int = 128):
        self.pool = sv.Pool(pool_bytes)
        self.threads = threads  # CTA size of the fused pass where the block size allows it
        self.budget = budget_bytes
        self.block_log2 = block_log2
        self.max_batch = max_batch
        self.graphs = graphs
        self.keep = keep_results
        self.streams: Dict[tuple, torch.cuda.Stream] = {}
        self.batches: Dict[tuple, sv.Batch] = {}
        self.model = FootprintModel()

    def key(self, req: Request) -> tuple:
        return (req.dtype, min(self.block_log2, req.n), size_class(req.n))

    def _bucket(self, key: tuple):
        if key not in self.batches:
            self.streams[key] = torch.cuda.Stream()
            self.batches[key] = sv.Batch(self.pool, self.max_batch, stream=self.streams[key], graphs=self.graphs)

    def run(self, requests: List[Request], time_limit: Optional[float] = None) -> dict:
        """Serve `requests` (arrival times relative to the start of this call). Each bucket
        steps on its own stream whenever its staging ring has room, so small requests are not
        held to the pace of large ones; completions are seen through CUDA events."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        waiting: collections.deque = collections.deque()
        active: Dict[tuple, list] = collections.defaultdict(list)  # key -> [req, state, next, t_admit, fp]
        finishing: list = []  # [req, state, event, t_admit, fp, key]
        used = 0
        results: List[Result] = []
        served = 0
        steps = 0
        t0 = time.time()
        while pending or waiting or finishing or any(active.values()):
            now = time.time() - t0
            if time_limit is not None and now > time_limit:
                break
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            while waiting:  # admission in arrival order while the footprint fits
                req = waiting[0]
                key = self.key(req)
                fp = footprint(req, key[1], self.model.bytes_per_amp(req))
                in_pool = self.pool.usage()[0]  # what the live states hold now (arenas grow)
                if max(used, in_pool) + fp > self.budget or len(active[key]) >= self.max_batch:
                    break
                waiting.popleft()
                self._bucket(key)
                st = sv.State(self.pool, req.n, req.n, req.eb, req.dtype, block_log2=key[1],
                              stream=self.streams[key])
                nv = 2 << key[1]
                if 32 <= self.threads <= 256 and 2 <= nv // self.threads <= 32:
                    st.set_threads(self.threads)
                st.reset_basis(req.basis)
                used += fp
                active[key].append([req, st, 0, now, fp])
            progressed = False
            for key, lst in active.items():
                if not lst or not self.batches[key].ready():
                    continue
                self.batches[key].apply([e[1] for e in lst], [e[0].gates[e[2]] for e in lst])
                progressed = True
                steps += 1
                keep = []
                for e in lst:
                    e[2] += 1
                    served += 1 << e[0].n
                    if e[2] == len(e[0].gates):
                        ev = torch.cuda.Event()
                        ev.record(self.streams[key])
                        finishing.append([e[0], e[1], ev, e[3], e[4], key])
                    else:
                        keep.append(e)
                lst[:] = keep
            still = []
            for f in finishing:
                req, st, ev, tadm, fp, key = f
                if not ev.query():
                    still.append(f)
                    continue
                tdone = time.time() - t0
                res = Result(req.rid, req.arrival, tadm, tdone, req.amp_updates)
                try:
                    st.sync()
                    self.model.observe(req, st.stats()["peak_compressed_bytes"])
                except sv.SvError as ex:
                    res.error = str(ex)
                if self.keep and res.error is None:
                    res.streams = [st.block_stream(i) for i in range(1 << (req.n - key[1]))]
                    res.norm = st.norm()
                st.close()
                used -= fp
                results.append(res)
                progressed = True
            finishing = still
            if not progressed:
                time.sleep(0.0002)
        wall = time.time() - t0
        for lst in active.values():
            for e in lst:
                e[1].close()
        for f in finishing:
            f[1].close()
        ok = [r for r in results if r.error is None]
        lat = np.array([r.latency for r in ok]) if ok else np.zeros(0)
        # requests that arrived but did not finish before the time limit are censored: their
        # latency is at least (end of the run - arrival); the percentiles over every arrived
        # request take them at that bound, so with censored requests they are lower bounds
        unfinished = [e[0] for lst in active.values() for e in lst] + [f[0] for f in finishing] + \
            [r for r in waiting] + [r for r in pending if r.arrival <= wall]
        cens = np.array([wall - r.arrival for r in unfinished])
        every = np.concatenate([lat, cens]) if lat.size + cens.size else np.zeros(0)
        offered = sum(r.amp_updates for r in requests)
        span = max((r.arrival for r in requests), default=0.0)
        return {
            "requests": len(requests), "completed": len(ok), "failed": len(results) - len(ok),
            "failure_reasons": sorted({r.error for r in results if r.error}),
            "censored": len(unfinished),
            "waiting_at_end": len(waiting) + len(pending),
            "active_at_end": sum(len(v) for v in active.values()) + len(finishing),
            "steps": steps, "wall_s": wall,
            "p50_s": float(np.percentile(every, 50)) if every.size else None,
            "p99_s": float(np.percentile(every, 99)) if every.size else None,
            "latency_is_lower_bound": bool(cens.size),
            "p50_s_completed": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_s_completed": float(np.percentile(lat, 99)) if lat.size else None,
            "served_amp_updates_per_s": served / wall if wall > 0 else 0.0,
            "offered_amp_updates_per_s": offered / span if span > 0 else None,
            "results": results,
        }

    def close(self):
        for b in self.batches.values():
            b.close()
        self.batches.clear()
        self.pool.close()
