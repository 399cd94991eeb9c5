"""Serving: continuous batching of RANMAR stream requests on one GPU.

A request (seed, k, J, count, dtype) asks for the next `count` outputs of
stream k of (seed, J), i.e. of the block that starts k*J transitions after the
LAMMPS-seeded state (Sec. 1).  Later requests for the same stream resume
where earlier ARRIVALS of that stream stopped: the offset of a request is the
sum of the counts of earlier arrivals with the same (seed, k, J), fixed when
it arrives, so results never depend on how requests are batched.

The scheduler itself is native (ranmar_serve_* in libranmar): admission by
output and state-pool memory, segmenting, resident stream states with
least-recently-used eviction, one packed staging copy per iteration,
pipelined iterations and retirement all run in C++ on the host, and every
step of the generator in the library's kernels.  This module marshals
requests (numpy records of ranmar_request_t) and summarises latencies.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import binding as bd


@dataclasses.dataclass
class Request:
    rid: int
    t: float                # arrival time, seconds from the start of the run
    seed: int
    k: int
    J: int
    count: int
    f32: bool
    offset: int = -1        # outputs of this stream taken by earlier arrivals
    done: float = -1.0      # completion time (GPU clock, seconds from start)
    host_done: float = -1.0  # when the host saw the completion (host clock, same origin)
    checksum: int = -1      # device checksum of the outputs
    rejected: bool = False  # could never be served: refused on arrival
    iteration: int = -1     # scheduler iteration that served it

    @property
    def key(self):
        return (self.seed, self.k, self.J)

    @property
    def overlaps(self) -> bool:
        """The request runs past the end (k+1)J of its stream (Sec. 1): its
        outputs are still served, but they are no longer disjoint from
        stream k+1's."""
        return self.offset + self.count > self.J


def assign_offsets(reqs) -> None:
    """Resume semantics: offset = sum of counts of earlier arrivals of the stream."""
    pos: dict = {}
    for r in reqs:
        r.offset = pos.get(r.key, 0)
        pos[r.key] = r.offset + r.count


def make_requests(t, seeds, ks, counts, f32, J) -> list[Request]:
    reqs = [Request(i, float(t[i]), int(seeds[i]), int(ks[i]), int(J), int(counts[i]),
                    bool(f32[i])) for i in range(len(t))]
    assign_offsets(reqs)
    return reqs


def assign_offsets_array(a: np.ndarray) -> None:
    """assign_offsets for REQUEST_DTYPE records (vectorised): group by
    (seed, k, J), exclusive prefix sums of the counts in arrival order."""
    n = a.size
    if n == 0:
        return
    order = np.lexsort((np.arange(n), a["J"][:, 1], a["J"][:, 0], a["k"], a["seed"]))
    s = a[order]
    cnt = s["count"]
    excl = np.cumsum(cnt, dtype=np.uint64) - cnt
    new = np.ones(n, dtype=bool)
    new[1:] = ((s["seed"][1:] != s["seed"][:-1]) | (s["k"][1:] != s["k"][:-1]) |
               (s["J"][1:, 0] != s["J"][:-1, 0]) | (s["J"][1:, 1] != s["J"][:-1, 1]))
    first = np.maximum.accumulate(np.where(new, np.arange(n), 0))
    a["offset"][order] = excl - excl[first]


def requests_array(t, seeds, ks, counts, f32, J: int) -> np.ndarray:
    """REQUEST_DTYPE records for arrival arrays, offsets assigned."""
    n = len(t)
    a = np.zeros(n, dtype=bd.REQUEST_DTYPE)
    a["t"] = t
    a["seed"] = seeds
    a["k"] = np.asarray(ks, dtype=np.uint64)
    a["J"][:, 0] = J & ((1 << 64) - 1)
    a["J"][:, 1] = J >> 64
    a["count"] = np.asarray(counts, dtype=np.uint64)
    a["f32"] = np.asarray(f32, dtype=bool)
    a["status"] = bd.REQ_PENDING
    a["done"] = -1.0
    a["host_done"] = -1.0
    assign_offsets_array(a)
    return a


def _to_array(reqs) -> np.ndarray:
    a = np.zeros(len(reqs), dtype=bd.REQUEST_DTYPE)
    for i, r in enumerate(reqs):
        if r.J >= 1 << 128 or r.k >= 1 << 64 or r.offset >= 1 << 64 or r.count >= 1 << 64:
            raise ValueError(f"request {r.rid}: k, J, offset or count out of range")
        a[i] = (r.t, r.seed, int(r.f32), r.k, (r.J & ((1 << 64) - 1), r.J >> 64), r.offset,
                r.count, r.done, r.host_done, max(r.checksum, 0),
                bd.REQ_TOO_LARGE if r.rejected else
                (bd.REQ_DONE if r.done >= 0 else bd.REQ_PENDING), 0)
    return a


def _from_array(reqs, a: np.ndarray) -> None:
    for r, rec in zip(reqs, a.tolist()):
        r.done, r.host_done, r.checksum = rec[7], rec[8], int(rec[9])
        r.rejected = rec[10] in (bd.REQ_TOO_LARGE, bd.REQ_BAD)
        r.iteration = int(rec[11]) if rec[10] == bd.REQ_DONE else -1


def summarize_array(a: np.ndarray) -> dict:
    """Latency percentiles over the served requests.  `p50_ms`/`p99_ms`: the
    GPU event that ends the request's iteration minus its arrival (the device
    is done; the host has not looked yet).  `host_p50_ms`/`host_p99_ms`: the
    moment the host's scheduler loop saw that event complete, minus arrival
    (what a caller polling the engine observes)."""
    served = a[a["status"] == bd.REQ_DONE]
    lat = served["done"] - served["t"]
    hs = served[served["host_done"] >= 0]
    hlat = hs["host_done"] - hs["t"]
    outs = int(served["count"].sum(dtype=np.uint64)) if served.size else 0
    span = float(served["done"].max() - served["t"].min()) if served.size else 0.0
    pct = lambda x, q: float(np.percentile(x, q) * 1e3) if x.size else None
    J0, J1 = a["J"][:, 0], a["J"][:, 1]
    over = (J1 == 0) & ((a["offset"] > J0) | (a["count"] > J0 - np.minimum(a["offset"], J0)))
    rejected = (a["status"] == bd.REQ_TOO_LARGE) | (a["status"] == bd.REQ_BAD)
    return {"requests": int(a.size), "served": int(served.size),
            "rejected": int(rejected.sum()), "outputs": outs,
            "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99),
            "mean_ms": float(lat.mean() * 1e3) if lat.size else None,
            "host_p50_ms": pct(hlat, 50), "host_p99_ms": pct(hlat, 99),
            "span_s": span, "outputs_per_s": outs / span if span > 0 else None,
            "overlapping_requests": int(over.sum())}


def summarize(reqs) -> dict:
    """summarize_array for Request objects."""
    return summarize_array(_to_array(reqs))


class Engine:
    """Continuous-batching request server on one GPU (ranmar_serve_t).

    use_table: segment start states by the fixed-base table jump
    (bit-identical to square-and-multiply, far fewer multiply-adds);
    False keeps square-and-multiply.  host_only: the scheduler alone, with
    no device (it records its plan; see trace())."""

    def __init__(self, budget_bytes: int = 40 << 30, seg: int = 4096,
                 state_entries: int = 1 << 18, max_seeds: int = 10**4 + 1,
                 max_segments_per_iter: int = 8192, max_inflight: int = 4, device="cuda",
                 use_table: bool = True, host_only: bool = False):
        flags = (0 if use_table else bd.SERVE_SQUARE) | (bd.SERVE_HOST_ONLY if host_only else 0)
        args = (budget_bytes, seg, state_entries, max_seeds, max_segments_per_iter,
                max_inflight, flags)
        self.host_only = host_only
        self.dev = None if host_only else torch.device(device)
        if host_only:
            self.h = bd.Serve(*args)
        else:
            with torch.cuda.device(self.dev):
                self.h = bd.Serve(*args)

    def _stream(self):
        return None if self.host_only else torch.cuda.current_stream(self.dev)

    @property
    def stats(self) -> dict:
        s = self.h.stats()
        s["max_loop_ms"] = s["max_loop_ns"] / 1e6
        s["jumps"] = s["base_jumps"] + s["pool_jumps"]
        return s

    def preload_seeds(self, seeds) -> None:
        """Seed a known range of seeds up front (engine set-up)."""
        self.h.preload(np.asarray(list(seeds), dtype=np.int32), stream=self._stream())

    def _serve(self, fn, reqs, realtime, max_wait) -> dict:
        if isinstance(reqs, np.ndarray):
            fn(reqs, realtime=realtime, max_wait=max_wait, stream=self._stream())
            return summarize_array(reqs)
        a = _to_array(reqs)
        try:
            fn(a, realtime=realtime, max_wait=max_wait, stream=self._stream())
        finally:
            _from_array(reqs, a)
        return summarize_array(a)

    def run(self, reqs, realtime: bool = True, max_wait: float = 120.0) -> dict:
        """Serve `reqs` (Request objects or REQUEST_DTYPE records, sorted by
        arrival time).  realtime=True replays the arrival times against the
        host clock; False makes every request available at once."""
        return self._serve(self.h.run, reqs, realtime, max_wait)

    def run_plain(self, reqs, realtime: bool = True, max_wait: float = 120.0) -> dict:
        """Comparator: every request alone, in arrival order -- one jump
        launch and one plain one-warp generation launch per request (no
        batching, no segments, no resident states), checksum as above."""
        return self._serve(self.h.run_plain, reqs, realtime, max_wait)

    def trace(self) -> np.ndarray:
        """The segments a host-only engine planned (SEG_DTYPE records)."""
        return self.h.trace()

    def close(self):
        if self.host_only:
            self.h.close()
        else:
            with torch.cuda.device(self.dev):
                self.h.close()
