"""Serving engine: continuous batching of RANMAR stream requests on one GPU.

A request (seed, k, J, count, dtype) asks for the next `count` outputs of
stream k of (seed, J), i.e. of the block that starts k*J transitions after the
LAMMPS-seeded state (Sec. 1).  Later requests for the same stream resume
where earlier ARRIVALS of that stream stopped: the offset of a request is the
sum of the counts of earlier arrivals with the same (seed, k, J), fixed when
it arrives, so results never depend on how requests are batched.

The engine keeps stream states resident in a device state pool, so a request
that resumes a resident stream needs no jump.  It admits arrived requests in
order while the output memory (and state pool) budget allows, and every
scheduler iteration enqueues on the GPU, for all newly admitted requests at
once:
  * jumps of the segment start states (ranmar_jump_scatter; from the seed's
    base state by k*J + offset + j*seg, or from the resident state by j*seg);
  * one batched generation of all segments (persistent kernel), each segment
    at most `seg` outputs with its own state, so a long request runs on many
    warps at once instead of one;
  * the on-device checksum of every segment into its request's result slot,
    which is how outputs are consumed before their memory is recycled.
Iterations are pipelined: the host builds and enqueues the next one while the
GPU runs the previous ones; a request is done when the event of its
iteration completes, and its latency is that GPU time minus its arrival time.
Host-side scheduling only -- every step of the generator runs in libranmar.
"""
from __future__ import annotations

import bisect
import collections
import dataclasses
import gc
import time

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
    rejected: bool = False  # larger than the engine could ever hold: refused on arrival

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


def exp_rows(base: int, ns: int, seg: int) -> np.ndarray:
    """Exponents base + q*seg for q < ns as (ns, 5) little-endian uint32 rows."""
    out = np.zeros((ns, bd.MAX_EXP_WORDS), dtype=np.uint32)
    lo = base & ((1 << 64) - 1)
    hi = base >> 64
    q = np.arange(ns, dtype=np.uint64) * np.uint64(seg)
    with np.errstate(over="ignore"):
        lo_q = np.uint64(lo) + q
    carry = lo_q < np.uint64(lo)
    out[:, 0] = (lo_q & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    out[:, 1] = (lo_q >> np.uint64(32)).astype(np.uint32)
    for c in (False, True):
        rows = carry == c
        if rows.any():
            h = hi + int(c)
            for w in range(2, bd.MAX_EXP_WORDS):
                out[rows, w] = (h >> (32 * (w - 2))) & 0xFFFFFFFF
    return out


def add_rows(out: np.ndarray, base: np.ndarray, add: np.ndarray) -> None:
    """out[i] = base[i] + add[i] as 5-word little-endian integers (add < 2^64)."""
    lo = base[:, 0].astype(np.uint64) | (base[:, 1].astype(np.uint64) << np.uint64(32))
    with np.errstate(over="ignore"):
        s = lo + add
    carry = (s < lo).astype(np.uint64)
    out[:, 0] = (s & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    out[:, 1] = (s >> np.uint64(32)).astype(np.uint32)
    c = carry
    for w in range(2, base.shape[1]):
        v = base[:, w].astype(np.uint64) + c
        out[:, w] = (v & np.uint64(0xFFFFFFFF)).astype(np.uint32)
        c = v >> np.uint64(32)


class FirstFit:
    """First-fit allocator over [0, size) units with coalescing (host side)."""

    def __init__(self, size: int, align: int = 32):
        self.size = size
        self.align = align
        self.starts = [0]          # free blocks, sorted by start
        self.lens = [size]
        self.used = 0

    def alloc(self, n: int):
        n = max(self.align, (n + self.align - 1) // self.align * self.align)
        for i, ln in enumerate(self.lens):
            if ln >= n:
                st = self.starts[i]
                if ln == n:
                    del self.starts[i]
                    del self.lens[i]
                else:
                    self.starts[i] = st + n
                    self.lens[i] = ln - n
                self.used += n
                return st, n
        return None

    def free(self, st: int, n: int) -> None:
        i = bisect.bisect_left(self.starts, st)
        self.starts.insert(i, st)
        self.lens.insert(i, n)
        self.used -= n
        # coalesce with the next and the previous block
        if i + 1 < len(self.starts) and self.starts[i] + self.lens[i] == self.starts[i + 1]:
            self.lens[i] += self.lens[i + 1]
            del self.starts[i + 1]
            del self.lens[i + 1]
        if i > 0 and self.starts[i - 1] + self.lens[i - 1] == self.starts[i]:
            self.lens[i - 1] += self.lens[i]
            del self.starts[i]
            del self.lens[i]


class _Staging:
    """Pinned host + device arrays for one iteration's small inputs."""

    def __init__(self, dev, cap: int):
        self.dev = dev
        self.cap = 0
        self._grow(cap)

    def _grow(self, cap):
        self.cap = cap
        mk = lambda shape, dt: (torch.empty(shape, dtype=dt).pin_memory(),
                                torch.empty(shape, dtype=dt, device=self.dev))
        self.exps = mk((cap, bd.MAX_EXP_WORDS), torch.int32)
        self.base_idx = mk((cap,), torch.int32)
        self.dst_idx = mk((cap,), torch.int32)
        self.pexps = mk((cap, bd.MAX_EXP_WORDS), torch.int32)
        self.pbase_idx = mk((cap,), torch.int32)
        self.pdst_idx = mk((cap,), torch.int32)
        self.desc_u = mk((cap, 3), torch.int64)
        self.desc_f = mk((cap, 3), torch.int64)
        self.items = mk((cap, 4), torch.int64)
        self.seeds = mk((cap,), torch.int32)

    def ensure(self, n):
        if n > self.cap:
            self._grow(max(n, 2 * self.cap))


class Engine:
    """Continuous-batching request server over libranmar (one GPU)."""

    def __init__(self, budget_bytes: int = 40 << 30, seg: int = 1 << 16,
                 state_entries: int = 1 << 18, max_seeds: int = 10**4 + 1,
                 result_slots: int = 1 << 17, max_segments_per_iter: int = 8192,
                 max_inflight: int = 4, device="cuda", use_table: bool = True):
        self.dev = torch.device(device)
        # fixed-base table jump (bit-identical to square-and-multiply, far fewer
        # multiply-adds per segment start); use_table=False keeps the latter
        self.table = bd.Table() if use_table else None
        self.seg = seg
        self.max_segs = max_segments_per_iter
        self.max_inflight = max_inflight
        state_bytes = state_entries * 400
        out_words = (budget_bytes - state_bytes) // 4
        if out_words <= 0:
            raise ValueError("budget too small for the state pool")
        self.pool = torch.empty((state_entries, bd.STATE_WORDS), dtype=torch.int32,
                                device=self.dev)
        self.out = torch.empty(out_words, dtype=torch.int32, device=self.dev)
        self.outf = self.out.view(torch.float32)
        self.alloc = FirstFit(out_words)
        self.state_entries = state_entries
        self.free_entries = list(range(state_entries - 1, -1, -1))
        self.resident: collections.OrderedDict = collections.OrderedDict()  # key -> (entry, end)
        self.base = torch.empty((max_seeds, bd.STATE_WORDS), dtype=torch.int32, device=self.dev)
        self.seed_row: dict = {}
        self.results = torch.zeros(result_slots, dtype=torch.int64, device=self.dev)
        self.results_host = torch.zeros(result_slots, dtype=torch.int64).pin_memory()
        self.res_next = 0
        self.batch = bd.Batch(max(self.max_segs, 1024))
        # one staging set per possible in-flight iteration: pinned buffers are
        # read by asynchronous copies, so a set is reused only after the event
        # of the iteration that last used it has completed
        cap = max(4096, max_segments_per_iter)   # never grown (pinned allocation) mid-run
        self.stages = [_Staging(self.dev, cap) for _ in range(max_inflight + 1)]
        self.stage_ev = [None] * (max_inflight + 1)
        self.stream = torch.cuda.current_stream(self.dev)
        self.status = torch.zeros(1, dtype=torch.int32, device=self.dev)
        self.stats = collections.Counter()

    # --- admission ---------------------------------------------------------
    def _nseg(self, r: Request) -> int:
        return max(1, (r.count + self.seg - 1) // self.seg)

    def fits_ever(self, r: Request) -> bool:
        """Whether `r` fits the engine when nothing else is held: its output
        region in the output pool and its segments' states in the state pool.
        A request that does not is refused when it reaches the queue head
        instead of blocking every request behind it."""
        need = max(self.alloc.align, -(-max(1, r.count) // self.alloc.align) * self.alloc.align)
        return need <= self.alloc.size and self._nseg(r) <= self.state_entries

    def _take_entries(self, n: int):
        while len(self.free_entries) < n and self.resident:
            _, (e, _) = self.resident.popitem(last=False)      # evict least recently used
            self.free_entries.append(e)
            self.stats["evicted"] += 1
        if len(self.free_entries) < n:
            return None
        return [self.free_entries.pop() for _ in range(n)]

    def admit(self, waiting: collections.deque) -> list:
        out = []
        nsegs = 0
        while waiting:
            r = waiting[0]
            if not self.fits_ever(r):
                waiting.popleft()
                r.rejected = True
                self.stats["rejected"] += 1
                continue
            ns = self._nseg(r)
            if out and nsegs + ns > self.max_segs:
                break
            res = self.resident.get(r.key)
            resume = res is not None and res[1] == r.offset
            region = self.alloc.alloc(max(1, r.count))
            if region is None:
                break
            # take the resumed state out of the resident map first, so that the
            # eviction below cannot pick it
            e0 = self.resident.pop(r.key)[0] if resume else None
            need = ns - 1 if resume else ns
            ents = self._take_entries(need) if need else []
            if ents is None:
                self.alloc.free(*region)
                if resume:
                    self.resident[r.key] = (e0, r.offset)
                break
            if resume:
                ents = [e0] + ents
                self.stats["resumed"] += 1
            waiting.popleft()
            r._region, r._ents, r._resume = region, ents, resume
            out.append(r)
            nsegs += ns
        return out

    # --- one iteration -------------------------------------------------------
    def _seed_rows(self, reqs, st=None):
        """Rows of the base-state table for the seeds of `reqs`; new seeds are
        seeded on the device (Algorithm 3, one launch for all of them)."""
        new = list(dict.fromkeys(r.seed for r in reqs if r.seed not in self.seed_row))
        if not new:
            return
        r0 = len(self.seed_row)
        if r0 + len(new) > self.base.shape[0]:
            raise ValueError(f"more than {self.base.shape[0]} distinct seeds (max_seeds)")
        for i, sd in enumerate(new):
            self.seed_row[sd] = r0 + i
        m = len(new)
        if st is None:
            sd_dev = torch.tensor(new, dtype=torch.int32, device=self.dev)
        else:
            st.seeds[0][:m] = torch.tensor(new, dtype=torch.int32)
            st.seeds[1][:m].copy_(st.seeds[0][:m], non_blocking=True)
            sd_dev = st.seeds[1][:m]
        bd.seed_batch(sd_dev, out=self.base[r0:r0 + m], status=self.status, stream=self.stream)

    def preload_seeds(self, seeds) -> None:
        """Seed a known range of seeds up front (engine set-up)."""
        self._seed_rows([Request(0, 0.0, int(sd), 0, 1, 1, False) for sd in seeds])
        torch.cuda.synchronize(self.dev)

    def _slots(self, n: int) -> int:
        """n consecutive result slots (never wrapping inside one iteration)."""
        size = self.results.numel()
        if self.res_next % size + n > size:
            self.res_next += size - self.res_next % size
        lo = self.res_next % size
        self.res_next += n
        return lo

    def enqueue(self, reqs: list, t0_event) -> dict:
        # one NVTX range per iteration (timeline tools show it beside the
        # library's own ranges)
        with torch.cuda.nvtx.range(f"serve.enqueue[{len(reqs)}]"):
            return self._enqueue(reqs, t0_event)

    def _enqueue(self, reqs: list, t0_event) -> dict:
        nreq = len(reqs)
        seg = self.seg
        counts = np.fromiter((r.count for r in reqs), dtype=np.int64, count=nreq)
        nseg = np.maximum(1, (counts + seg - 1) // seg)
        ntot = int(nseg.sum())
        si = self.stats["iterations"] % len(self.stages)
        if self.stage_ev[si] is not None:
            self.stage_ev[si].synchronize()
        st = self.stages[si]
        st.ensure(max(ntot, nreq))
        self._seed_rows(reqs, st)
        lo_s = self._slots(nreq)
        for q, r in enumerate(reqs):
            r._slot = lo_s + q
        # per-segment arrays
        sreq = np.repeat(np.arange(nreq), nseg)
        starts = np.cumsum(nseg) - nseg
        j = np.arange(ntot, dtype=np.int64) - np.repeat(starts, nseg)
        cnt = np.maximum(0, np.minimum(seg, counts[sreq] - j * seg))
        region = np.fromiter((r._region[0] for r in reqs), dtype=np.int64, count=nreq)
        offs = region[sreq] + j * seg
        ents = np.fromiter((e for r in reqs for e in r._ents), dtype=np.int64, count=ntot)
        last = j == nseg[sreq] - 1
        f32 = np.fromiter((r.f32 for r in reqs), dtype=bool, count=nreq)[sreq]
        resume = np.fromiter((r._resume for r in reqs), dtype=bool, count=nreq)[sreq]
        # jumps from the seed's base state: E = k J + offset + j seg
        sj = ~resume
        nj = int(sj.sum())
        if nj:
            rq = sreq[sj]
            basew = np.zeros((nreq, bd.MAX_EXP_WORDS), dtype=np.uint32)
            for q, r in enumerate(reqs):
                if not r._resume:
                    e = r.k * r.J + r.offset
                    basew[q] = [(e >> (32 * w)) & 0xFFFFFFFF for w in range(bd.MAX_EXP_WORDS)]
            add_rows(st.exps[0].numpy()[:nj].view(np.uint32), basew[rq],
                     (j[sj] * seg).astype(np.uint64))
            st.base_idx[0].numpy()[:nj] = np.fromiter((self.seed_row[reqs[q].seed] for q in rq),
                                                      dtype=np.int32, count=nj)
            st.dst_idx[0].numpy()[:nj] = ents[sj]
        # jumps from a resumed resident state by j seg (segments j >= 1)
        pj = resume & (j > 0)
        npj = int(pj.sum())
        if npj:
            e = (j[pj] * seg).astype(np.uint64)
            pe = st.pexps[0].numpy()[:npj].view(np.uint32)
            pe[:] = 0
            pe[:, 0] = (e & np.uint64(0xFFFFFFFF)).astype(np.uint32)
            pe[:, 1] = (e >> np.uint64(32)).astype(np.uint32)
            first_ent = ents[starts]                      # segment 0 of each request
            st.pbase_idx[0].numpy()[:npj] = first_ent[sreq[pj]]
            st.pdst_idx[0].numpy()[:npj] = ents[pj]
        # generation descriptors (write back only the last segment's state)
        flags = last.astype(np.int64) * bd.DESC_WRITE_BACK
        d_all = np.stack([ents | (flags << 32), offs, cnt], axis=1)
        nu = int((~f32).sum())
        nf = ntot - nu
        if nu:
            st.desc_u[0].numpy()[:nu] = d_all[~f32]
        if nf:
            st.desc_f[0].numpy()[:nf] = d_all[f32]
        it = st.items[0].numpy()
        it[:ntot, 0] = offs
        it[:ntot, 1] = cnt
        it[:ntot, 2] = j * seg
        it[:ntot, 3] = lo_s + sreq
        s = self.stream
        for pair, n in ((st.exps, nj), (st.base_idx, nj), (st.dst_idx, nj), (st.pexps, npj),
                        (st.pbase_idx, npj), (st.pdst_idx, npj), (st.desc_u, nu),
                        (st.desc_f, nf), (st.items, ntot)):
            if n:
                pair[1][:n].copy_(pair[0][:n], non_blocking=True)
        if nj:
            self._jump(self.base, st.exps[1], st.dst_idx[1], st.base_idx[1], nj)
        if npj:
            self._jump(self.pool, st.pexps[1], st.pdst_idx[1], st.pbase_idx[1], npj)
        if nu:
            self.batch.generate_u24(self.pool, st.desc_u[1][:nu], self.out, status=self.status,
                                    stream=s)
        if nf:
            self.batch.generate_f32(self.pool, st.desc_f[1][:nf], self.outf, status=self.status,
                                    stream=s)
        hi_s = lo_s + nreq
        self.results[lo_s:hi_s].zero_()
        bd.checksum(self.out, st.items[1][:ntot], self.results, status=self.status, stream=s,
                    n=ntot)
        self.results_host[lo_s:hi_s].copy_(self.results[lo_s:hi_s], non_blocking=True)
        ev = torch.cuda.Event(enable_timing=True)
        ev.record(s)
        self.stage_ev[si] = ev
        self.stats["iterations"] += 1
        self.stats["segments"] += ntot
        self.stats["jumps"] += nj + npj
        return {"event": ev, "reqs": reqs, "t0": t0_event, "slots": (lo_s, hi_s)}

    def _jump(self, base, exps, dst_idx, base_idx, n):
        if self.table is not None:
            self.table.jump(base, exps, base_idx=base_idx, out=self.pool, dst_idx=dst_idx,
                            status=self.status, stream=self.stream, n=n)
        else:
            bd.jump_scatter(base, exps, self.pool, dst_idx, base_idx=base_idx,
                            status=self.status, stream=self.stream, n=n)

    def retire(self, it: dict) -> None:
        with torch.cuda.nvtx.range("serve.retire"):
            self._retire(it)

    def _retire(self, it: dict) -> None:
        it["event"].synchronize()
        done = it["t0"].elapsed_time(it["event"]) * 1e-3
        host_done = time.perf_counter() - self._h0
        lo_s, hi_s = it["slots"]
        host = self.results_host[lo_s:hi_s].numpy().view(np.uint64)
        for r in it["reqs"]:
            r.done = done
            r.host_done = host_done
            r.checksum = int(host[r._slot - lo_s])
            self.alloc.free(*r._region)
            ents = r._ents
            self.free_entries.extend(ents[:-1])
            last, end = ents[-1], r.offset + r.count
            cur = self.resident.get(r.key)
            if cur is None or cur[1] < end:
                if cur is not None:
                    self.free_entries.append(cur[0])
                self.resident[r.key] = (last, end)
                self.resident.move_to_end(r.key)
            else:
                self.free_entries.append(last)
            self.stats["outputs"] += r.count

    # --- drivers ---------------------------------------------------------------
    def run(self, reqs: list, realtime: bool = True, max_wait: float = 120.0) -> dict:
        """Serve `reqs` (sorted by arrival time).  realtime=True replays the
        arrival times against the wall clock; False makes every request
        available at once."""
        waiting: collections.deque = collections.deque()
        inflight: collections.deque = collections.deque()
        i = 0
        # no collector pauses inside the latency-measured loop
        gc_was = gc.isenabled()
        gc.disable()
        try:
            return self._run(reqs, realtime, max_wait, waiting, inflight)
        finally:
            if gc_was:
                gc.enable()

    def _run(self, reqs, realtime, max_wait, waiting, inflight) -> dict:
        i = 0
        torch.cuda.synchronize(self.dev)
        t0 = torch.cuda.Event(enable_timing=True)
        t0.record(self.stream)
        h0 = time.perf_counter()
        self._h0 = h0
        n = len(reqs)
        t_prev = time.perf_counter()
        max_loop = 0.0
        while i < n or waiting or inflight:
            t_now = time.perf_counter()
            max_loop = max(max_loop, t_now - t_prev)   # host time of one loop turn
            if t_now - t_prev > 0.01:
                self.stats["slow_loops"] += 1
            t_prev = t_now
            now = t_now - h0
            if now > max_wait:
                raise RuntimeError("serving run exceeded its time limit")
            while i < n and (not realtime or reqs[i].t <= now):
                waiting.append(reqs[i])
                i += 1
            admitted = self.admit(waiting) if len(inflight) < self.max_inflight else []
            if admitted:
                inflight.append(self.enqueue(admitted, t0))
            progressed = bool(admitted)
            while inflight and (inflight[0]["event"].query() or
                                (not admitted and (waiting or i >= n))):
                self.retire(inflight.popleft())
                progressed = True
                if inflight and not inflight[0]["event"].query():
                    break
            if not progressed and realtime and i < n and not waiting:
                wait = reqs[i].t - (time.perf_counter() - h0)
                if wait > 0:
                    time.sleep(min(wait, 2e-4))
        torch.cuda.synchronize(self.dev)
        self.stats["max_loop_ms"] = max(self.stats["max_loop_ms"], int(max_loop * 1e3))
        st = int(self.status.item())
        if st:
            raise RuntimeError(f"device status bits {st}")
        return summarize(reqs)

    def run_plain(self, reqs: list, realtime: bool = True, max_wait: float = 120.0) -> dict:
        """Comparator: every request alone, in arrival order -- one jump launch
        and one plain one-warp generation launch per request (no batching, no
        segments, no resident states), checksum as above."""
        torch.cuda.synchronize(self.dev)
        t0 = torch.cuda.Event(enable_timing=True)
        t0.record(self.stream)
        h0 = time.perf_counter()
        self._h0 = h0
        s = self.stream
        st_d = torch.empty((1, bd.STATE_WORDS), dtype=torch.int32, device=self.dev)
        one = torch.zeros(1, dtype=torch.int32, device=self.dev)
        pending = collections.deque()
        for r in reqs:
            if realtime:
                wait = r.t - (time.perf_counter() - h0)
                if wait > 0:
                    time.sleep(wait)
            if time.perf_counter() - h0 > max_wait:
                raise RuntimeError("plain run exceeded its time limit")
            if not self.fits_ever(r):
                r.rejected = True
                continue
            self._seed_rows([r])
            region = self.alloc.alloc(max(1, r.count))
            while region is None and pending:
                self._retire_plain(pending.popleft(), t0)
                region = self.alloc.alloc(max(1, r.count))
            r._region = region
            ex = bd.exps_tensor([r.k * r.J + r.offset], bd.MAX_EXP_WORDS, device=self.dev)
            bi = torch.full((1,), self.seed_row[r.seed], dtype=torch.int32, device=self.dev)
            bd.jump_scatter(self.base, ex, st_d, one, base_idx=bi, stream=s)
            view = (self.outf if r.f32 else self.out)[region[0]:region[0] + r.count]
            (bd.generate_plain_f32 if r.f32 else bd.generate_plain_u24)(st_d, r.count, view,
                                                                         write_back=False,
                                                                         stream=s)
            r._slot = self._slots(1)
            self.results[r._slot] = 0
            items = torch.tensor([[region[0], r.count, 0, r._slot]], dtype=torch.int64,
                                 device=self.dev)
            bd.checksum(self.out, items, self.results, stream=s)
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(s)
            pending.append((r, ev))
            while pending and pending[0][1].query():
                self._retire_plain(pending.popleft(), t0)
        while pending:
            self._retire_plain(pending.popleft(), t0)
        return summarize(reqs)

    def _retire_plain(self, item, t0):
        r, ev = item
        ev.synchronize()
        r.done = t0.elapsed_time(ev) * 1e-3
        r.host_done = time.perf_counter() - self._h0
        r.checksum = int(np.int64(self.results[r._slot].item()).astype(np.uint64))
        self.alloc.free(*r._region)

    def close(self):
        self.batch.close()
        if self.table is not None:
            self.table.close()


def summarize(reqs) -> dict:
    """Latency percentiles over the served requests.  `p50_ms`/`p99_ms`: the
    GPU event that ends the request's iteration minus its arrival (the device
    is done; the host has not looked yet).  `host_p50_ms`/`host_p99_ms`: the
    moment the host's scheduler loop saw that event complete, minus arrival
    (what a caller polling the engine observes)."""
    served = [r for r in reqs if r.done >= 0 and not r.rejected]
    lat = np.array([r.done - r.t for r in served])
    hlat = np.array([r.host_done - r.t for r in served if r.host_done >= 0])
    outs = sum(r.count for r in served)
    span = max(r.done for r in served) - min(r.t for r in served) if served else 0.0
    pct = lambda a, q: float(np.percentile(a, q) * 1e3) if a.size else None
    return {"requests": len(reqs), "served": len(served),
            "rejected": sum(1 for r in reqs if r.rejected), "outputs": outs,
            "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99),
            "mean_ms": float(lat.mean() * 1e3) if lat.size else None,
            "host_p50_ms": pct(hlat, 50), "host_p99_ms": pct(hlat, 99),
            "span_s": span, "outputs_per_s": outs / span if span > 0 else None,
            "overlapping_requests": sum(1 for r in reqs if r.overlaps)}
