"""Serving: a request loop that sorts arrays of different sizes and key
types as they arrive, with continuous admission.

Requests arrive over time (`Request.arrival`, seconds from the start). The
loop admits a request as soon as it has arrived, a slot (a CUDA stream with
its own resident workspace) is free, and the device-memory budget covers the
request's key buffer; admitted requests run concurrently on their slots'
streams, so a request that arrives while others are on the GPU starts
without waiting for them to finish. Each request sorts its own device buffer
(filled from a resident source array); its latency is measured from its
arrival to the completion event of its sort on the GPU clock.

`run_plain` is the comparison: the same arrival stream served one request at
a time on one stream.

Nothing here changes what a sort computes: every request's result is the
unique sorted order of its keys, alone or in the mix.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np

from . import KEY_BYTES, alloc_workspace, sort_ws_


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float            # seconds after the start of the run
    dtype: str
    n: int
    source: object            # CUDA tensor holding at least n keys (resident)
    offset: int = 0           # first key of this request in `source`
    descending: bool = False
    # filled in by the server
    out: object = None
    start_ms: float = 0.0
    done_ms: float = 0.0
    latency_ms: float = 0.0


def key_buffer_bytes(r: Request) -> int:
    return r.n * KEY_BYTES[r.dtype]


class Server:
    """Continuous batching over `slots` streams under `budget_bytes` of device
    memory (workspaces included)."""

    def __init__(self, slots: int = 8, budget_bytes: int = 40 * 10**9, max_keys: int = 10**7,
                 keep_outputs: bool = False, device=None):
        import torch
        self.torch = torch
        self.device = device or torch.device("cuda")
        self.slots = slots
        self.budget = budget_bytes
        self.keep_outputs = keep_outputs
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(slots)]
        # one resident workspace per slot, large enough for the biggest request
        self.ws = [alloc_workspace("kv64", max_keys, 1, device=self.device) for _ in range(slots)]
        self.ws_bytes = sum(w.numel() for w in self.ws)
        if self.ws_bytes >= budget_bytes:
            raise ValueError("budget does not cover the slot workspaces")
        self.max_keys = max_keys

    def _launch(self, r: Request, slot: int, t0_event):
        torch = self.torch
        s = self.streams[slot]
        with torch.cuda.stream(s):
            if KEY_BYTES[r.dtype] == 16:
                buf = r.source[r.offset:r.offset + r.n].clone()
            else:
                buf = r.source[r.offset:r.offset + r.n].clone()
            start = torch.cuda.Event(enable_timing=True)
            done = torch.cuda.Event(enable_timing=True)
            start.record(s)
            sort_ws_(buf, self.ws[slot], r.dtype, r.descending, s)
            done.record(s)
        return buf, start, done

    def run(self, requests: list[Request], poll_sleep: float = 20e-6) -> dict:
        """Serves `requests` (sorted by arrival) and returns latency and
        throughput statistics. Wall-clock arrival times are honoured."""
        torch = self.torch
        reqs = sorted(requests, key=lambda r: r.arrival)
        for r in reqs:
            if r.n > self.max_keys:
                raise ValueError(f"request {r.rid} exceeds max_keys")
        pending = collections.deque()
        free_slots = list(range(self.slots))
        inflight = {}   # slot -> (request, buf, start_event, done_event, bytes)
        used = self.ws_bytes
        nxt = 0
        torch.cuda.synchronize(self.device)
        t0_event = torch.cuda.Event(enable_timing=True)
        t0_event.record(torch.cuda.current_stream(self.device))
        t_start = time.perf_counter()
        finished = []
        while len(finished) < len(reqs):
            now = time.perf_counter() - t_start
            while nxt < len(reqs) and reqs[nxt].arrival <= now:
                pending.append(reqs[nxt])
                nxt += 1
            # admit while a slot is free and memory allows
            while pending and free_slots and used + key_buffer_bytes(pending[0]) <= self.budget:
                r = pending.popleft()
                slot = free_slots.pop()
                buf, st, dn = self._launch(r, slot, t0_event)
                used += key_buffer_bytes(r)
                inflight[slot] = (r, buf, st, dn, key_buffer_bytes(r))
            # retire finished work
            progressed = False
            for slot in list(inflight):
                r, buf, st, dn, nbytes = inflight[slot]
                if dn.query():
                    r.start_ms = t0_event.elapsed_time(st)
                    r.done_ms = t0_event.elapsed_time(dn)
                    r.latency_ms = r.done_ms - r.arrival * 1e3
                    if self.keep_outputs:
                        r.out = buf
                    used -= nbytes
                    free_slots.append(slot)
                    del inflight[slot]
                    finished.append(r)
                    progressed = True
            if not progressed and (not pending or not free_slots):
                if nxt < len(reqs) and not inflight and not pending:
                    wait = reqs[nxt].arrival - (time.perf_counter() - t_start)
                    if wait > 0:
                        time.sleep(min(wait, 1e-3))
                else:
                    time.sleep(poll_sleep)
        torch.cuda.synchronize(self.device)
        return summarize(finished)


def run_plain(requests: list[Request], max_keys: int = 10**7, keep_outputs: bool = False) -> dict:
    """The same requests served one at a time on one stream, in arrival order."""
    server = Server(slots=1, max_keys=max_keys, keep_outputs=keep_outputs)
    return server.run(requests)


def summarize(done: list[Request]) -> dict:
    lat = np.array([r.latency_ms for r in done])
    keys = sum(r.n for r in done)
    first = min(r.arrival * 1e3 for r in done)
    last = max(r.done_ms for r in done)
    span_ms = max(1e-9, last - first)
    return {
        "requests": len(done), "keys": int(keys),
        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
        "mean_ms": float(lat.mean()), "span_ms": float(span_ms),
        "gkeys_per_s": keys / (span_ms * 1e-3) / 1e9,
    }


def poisson_requests(num: int, rate_per_s: float, sources: dict, seed: int = 1, lo: int = 1000,
                     hi: int = 10**7, dtypes=("i16", "u32", "f32", "u64", "kv64")) -> list[Request]:
    """Poisson arrivals with log-uniform sizes in [lo, hi] and a key type drawn
    uniformly from `dtypes`; each request reads a seeded slice of the resident
    source array of its type (`sources[dtype]`, at least `hi` keys)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=num)
    arrivals = np.cumsum(gaps) - gaps[0]
    sizes = np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi), size=num))).astype(np.int64)
    kinds = rng.integers(0, len(dtypes), size=num)
    out = []
    for i in range(num):
        dt = dtypes[kinds[i]]
        src = sources[dt]
        total = src.shape[0]
        n = int(min(sizes[i], total))
        off = int(rng.integers(0, total - n + 1))
        out.append(Request(i, float(arrivals[i]), dt, n, src, off))
    return out
