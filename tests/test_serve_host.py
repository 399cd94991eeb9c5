"""Host side of the serving engine (no GPU): resume offsets, the request
recipe, and the native scheduler run with RANMAR_SERVE_HOST_ONLY, whose
recorded plan (jumps, segments, write-backs, regions) is executed here with
the oracle and must give every request exactly its stream's outputs."""
import collections

import numpy as np
import pytest

from paper_2512_00093_gb300 import serve
from paper_2512_00093_gb300.serve import Request, assign_offsets
from paper_2512_00093_gb300.workloads import Serving


@pytest.fixture(scope="module")
def bd():
    from paper_2512_00093_gb300.build import build_library
    build_library()
    from paper_2512_00093_gb300 import binding
    return binding


def host_engine(**kw):
    args = dict(budget_bytes=64 << 20, seg=16, state_entries=64, max_seeds=64,
                max_segments_per_iter=24, max_inflight=3, host_only=True)
    args.update(kw)
    return serve.Engine(**args)


def test_offsets_follow_arrival_order():
    reqs = [Request(i, 0.1 * i, s, k, 1 << 48, c, False)
            for i, (s, k, c) in enumerate([(1, 0, 10), (1, 1, 5), (1, 0, 7), (2, 0, 3),
                                           (1, 0, 1), (1, 1, 2)])]
    assign_offsets(reqs)
    assert [r.offset for r in reqs] == [0, 0, 10, 0, 17, 5]


def test_offsets_array_match_the_list_rule(bd):
    rng = np.random.default_rng(3)
    n = 3000
    t = np.sort(rng.random(n))
    sd, k = rng.integers(1, 6, n), rng.integers(0, 7, n)
    c = rng.integers(0, 1000, n)
    f32 = rng.random(n) < 0.5
    a = serve.requests_array(t, sd, k, c, f32, 1 << 48)
    reqs = serve.make_requests(t, sd, k, c, f32, 1 << 48)
    assert [int(x) for x in a["offset"]] == [r.offset for r in reqs]
    assert a.dtype.itemsize == 88 and (a["status"] == bd.REQ_PENDING).all()


def test_serving_recipe():
    t, seeds, ks, counts, f32 = Serving().requests(duration=2.0)
    assert abs(len(t) / 2.0 / 20000 - 1) < 0.02
    assert np.all(np.diff(t) >= 0) and t.min() >= 0 and t.max() <= 2.0
    assert seeds.min() >= 1 and seeds.max() <= 10**4 and ks.max() <= 1 << 20
    assert counts.min() >= 1000 and counts.max() <= 10**7
    # log-uniform 10^3..10^7: mean (10^7 - 10^3) / (4 ln 10) ~ 1.09e6
    assert abs(counts.mean() / 1.085e6 - 1) < 0.1
    assert abs(f32.mean() - 0.5) < 0.02


def test_overlap_flag_in_summary():
    """A request that runs past (k+1)J of its stream is served and counted as
    overlapping (Sec. 1); the requests before it are not."""
    J = 100
    reqs = serve.make_requests(np.array([0.0, 0.1, 0.2, 0.3]), np.array([7, 7, 7, 8]),
                               np.array([3, 3, 3, 3]), np.array([60, 40, 1, 101]),
                               np.array([False] * 4), J)
    assert [r.offset for r in reqs] == [0, 60, 100, 0]
    assert [r.overlaps for r in reqs] == [False, False, True, True]
    for r in reqs:
        r.done = r.t + 0.001
    assert serve.summarize(reqs)["overlapping_requests"] == 2


def test_create_argument_checks(bd):
    ok = dict(budget_bytes=1 << 20, seg=16, state_entries=8, max_seeds=4,
              max_segments=16, max_inflight=2, flags=bd.SERVE_HOST_ONLY)
    bd.Serve(**ok).close()
    for bad, code in [(dict(seg=0), bd.EINVAL), (dict(state_entries=0), bd.EINVAL),
                      (dict(max_inflight=0), bd.EINVAL), (dict(flags=8), bd.EINVAL),
                      (dict(max_segments=0), bd.EINVAL),
                      (dict(budget_bytes=8 * 400), bd.ERANGE)]:     # no room for outputs
        with pytest.raises(bd.RanmarError) as ei:
            bd.Serve(**{**ok, **bad})
        assert ei.value.code == code, bad
    e = bd.Serve(**ok)
    a = serve.requests_array([0.2, 0.1], [1, 1], [0, 1], [5, 5], [False, False], 100)
    with pytest.raises(bd.RanmarError) as ei:              # arrivals out of order
        e.run(a, realtime=False)
    assert ei.value.code == bd.EINVAL
    with pytest.raises(bd.RanmarError):
        e.run_plain(a[:1].copy(), realtime=False)          # no device: no plain mode
    e.close()


def test_admission_refuses_requests_that_can_never_fit(bd):
    """A request larger than the output pool, or with more segments than the
    state pool has entries, is refused where it stands and the requests
    behind it are served; a bad seed or an exponent past 2^160 is refused."""
    eng = host_engine(budget_bytes=4 * 400 + 1024 * 4, state_entries=4, seg=16)
    reqs = serve.make_requests(np.array([0.0, 0.1, 0.2, 0.3]), np.array([1, 2, 3, 4]),
                               np.array([0, 0, 0, 0]), np.array([2000, 100, 30, 64]),
                               np.array([False] * 4), 1 << 48)
    bad = [Request(4, 0.4, 0, 0, 1 << 48, 10, False, offset=0),
           Request(5, 0.5, 900000001, 0, 1 << 48, 10, False, offset=0),
           Request(6, 0.6, 5, (1 << 64) - 1, (1 << 97), 10, False, offset=0),
           Request(7, 0.7, 5, 1, (1 << 128) - 1, 10, False, offset=0)]
    s = eng.run(reqs + bad, realtime=False)
    # 2000 > 1024 output words; 100 outputs = 7 segments > 4 state entries
    assert [r.rejected for r in reqs + bad] == [True, True, False, False, True, True, True, False]
    assert (s["requests"], s["served"], s["rejected"]) == (8, 3, 5)
    assert eng.stats["rejected"] == 5
    eng.close()


def exponent(rec) -> int:
    return sum(int(w) << (32 * q) for q, w in enumerate(rec["exp"]))


def execute_plan(orc, bd, a, tr):
    """Runs a host-only engine's plan with the oracle in iteration order, as
    the device would: an iteration's jumps, then its generations (with their
    write-backs).  Returns each request's outputs and checks the plan's
    invariants on the way."""
    pool, row_seed, outs = {}, {}, {}
    iters = np.unique(tr["iteration"])
    assert (iters == np.arange(iters.size)).all()
    for it in iters:
        segs = tr[tr["iteration"] == it]
        assert len(set(segs["entry"].tolist())) == segs.size, "an entry twice in one iteration"
        jumped = {}
        resident = {int(x["entry"]) for x in segs if x["kind"] == bd.SEG_RESIDENT}
        for s in segs:
            r = a[s["request"]]
            if s["kind"] == bd.SEG_FROM_SEED:
                assert row_seed.setdefault(int(s["src"]), int(r["seed"])) == int(r["seed"])
                jumped[int(s["entry"])] = orc.jump(*orc.seeded_state(int(r["seed"])),
                                                   exponent(s))
            elif s["kind"] == bd.SEG_FROM_POOL:
                assert int(s["src"]) in resident     # read, and written by no jump here
                jumped[int(s["entry"])] = orc.jump(*pool[int(s["src"])], exponent(s))
            else:
                assert s["kind"] == bd.SEG_RESIDENT and int(s["entry"]) in pool
        pool.update(jumped)
        for s in segs:
            y, x2, c2 = orc.generate(*pool[int(s["entry"])], int(s["count"]))
            outs.setdefault(int(s["request"]), {})[int(s["index0"])] = y
            if s["flags"] & bd.DESC_WRITE_BACK:
                pool[int(s["entry"])] = (x2, c2)
    return {q: np.concatenate([d[i] for i in sorted(d)]) for q, d in outs.items()}


def check_regions(tr, out_words):
    """Output regions are 32-word aligned, inside the pool, and no two
    segments that are on the device at the same time overlap."""
    assert (tr[tr["index0"] == 0]["out_offset"] % 32 == 0).all()
    for s in tr:
        assert int(s["out_offset"]) + int(s["count"]) <= out_words
    for i, s in enumerate(tr):
        live = tr[(tr["iteration"] >= s["iteration"]) & (tr["iteration"] < s["live_until"])]
        for t in live:
            if t["iteration"] == s["iteration"] and t["request"] == s["request"] and \
                    t["index0"] == s["index0"]:
                continue
            a0, a1 = int(s["out_offset"]), int(s["out_offset"]) + int(s["count"])
            b0, b1 = int(t["out_offset"]), int(t["out_offset"]) + int(t["count"])
            assert a1 <= b0 or b1 <= a0 or a0 == a1 or b0 == b1, (s, t)


@pytest.mark.parametrize("state_entries,max_inflight", [(40, 3), (12, 2), (200, 4)])
def test_host_plan_gives_every_request_its_stream(bd, orc, state_entries, max_inflight):
    """Few distinct streams, small segments and a small state pool: resumes
    (no jump), pool jumps, seed jumps and evictions all occur, with several
    iterations in flight; the oracle run of the plan equals each request's
    outputs offset .. offset + count of its stream."""
    rng = np.random.default_rng(state_entries)
    n = 160
    t = np.sort(rng.random(n))
    sd, k = rng.integers(1, 5, n), rng.integers(0, 6, n)
    c = np.minimum(150, np.floor(10.0 ** (2.3 * rng.random(n)))).astype(np.int64)
    c[:6] = [0, 1, 15, 16, 17, 33]
    f32 = rng.random(n) < 0.5
    J = (1 << 70) + 12345
    a = serve.requests_array(t, sd, k, c, f32, J)
    budget = state_entries * 400 + 2000 * 4
    eng = host_engine(budget_bytes=budget, state_entries=state_entries,
                      max_inflight=max_inflight)
    s = eng.run(a, realtime=False)
    st = eng.stats
    assert s["served"] == n and st["iterations"] > 5
    assert st["resumed"] > 0 and st["pool_jumps"] > 0 and st["base_jumps"] > 0
    if state_entries <= 40:
        assert st["evicted"] > 0
    assert st["max_inflight"] <= max_inflight
    if state_entries >= 40:     # 12 entries: one iteration takes them all
        assert st["max_inflight"] >= 2
    tr = eng.trace()
    eng.close()
    assert tr.size == st["segments"]
    check_regions(tr, (budget - state_entries * 400) // 4)
    got = execute_plan(orc, bd, a, tr)
    for q in range(n):
        r = a[q]
        want = orc.stream(int(r["seed"]), int(r["k"]) * J + int(r["offset"]), int(r["count"]))
        assert np.array_equal(got[q], want), q
        segs = tr[tr["request"] == q]
        assert int(r["iteration"]) == int(segs["iteration"][0])
        if segs["kind"][0] == bd.SEG_FROM_SEED:
            assert exponent(segs[0]) == int(r["k"]) * J + int(r["offset"])


def test_host_plan_exponents_span_words(bd, orc):
    """Start exponents k J + offset + j seg with J up to 2^127 carry across
    all five words; the plan's exponents equal the integers."""
    J = (1 << 127) - 3
    reqs = [Request(i, 0.0, 11, kk, J, 40, False) for i, kk in
            enumerate([0, 1, 2, (1 << 32) - 1, 1 << 32, 0, 1])]
    assign_offsets(reqs)
    eng = host_engine(seg=16)
    eng.run(reqs, realtime=False)
    tr = eng.trace()
    eng.close()
    for s in tr:
        r = reqs[int(s["request"])]
        if s["kind"] == bd.SEG_FROM_SEED:
            assert exponent(s) == r.k * J + r.offset + int(s["index0"])
        elif s["kind"] == bd.SEG_FROM_POOL:
            assert exponent(s) == int(s["index0"])
    assert all(not r.rejected for r in reqs)


def test_host_pool_coalesces_after_retirement(bd):
    """After many small requests have come and gone, one request the size of
    the whole output pool is served: the freed regions coalesced."""
    out_words = 4096
    eng = host_engine(budget_bytes=16 * 400 + out_words * 4, state_entries=16, seg=4096,
                      max_inflight=3)
    rng = np.random.default_rng(5)
    n = 200
    c = rng.integers(1, 700, n).tolist() + [out_words]
    reqs = serve.make_requests(np.arange(n + 1) * 1e-3, rng.integers(1, 4, n + 1),
                               np.arange(n + 1), np.array(c), np.zeros(n + 1, bool), 1 << 40)
    s = eng.run(reqs, realtime=False)
    assert s["served"] == n + 1 and not reqs[-1].rejected
    tr = eng.trace()
    eng.close()
    assert int(tr[tr["request"] == n]["out_offset"][0]) == 0
    check_regions(tr, out_words)


def test_host_realtime_replays_arrivals(bd):
    """realtime=True: no request is served before it arrives."""
    t = np.linspace(0.0, 0.05, 40)
    a = serve.requests_array(t, np.full(40, 3), np.arange(40), np.full(40, 50),
                             np.zeros(40, bool), 1 << 48)
    eng = host_engine()
    s = eng.run(a, realtime=True)
    eng.close()
    assert s["served"] == 40
    assert (a["host_done"] >= a["t"]).all()


def test_hot_stream_recipe():
    """The hot-stream serving variant: 1,024 streams revisited, so nearly every
    stream has many requests and later ones resume at the earlier ones' end."""
    from paper_2512_00093_gb300.workloads import ServingHot
    w = ServingHot()
    t, seeds, ks, counts, f32 = w.requests(duration=1.0)
    assert abs(len(t) / 20000 - 1) < 0.03
    assert seeds.min() >= 1 and seeds.max() <= 64 and ks.min() >= 0 and ks.max() <= 15
    assert counts.min() >= 1000 and counts.max() < 10**6
    reqs = serve.make_requests(t, seeds, ks, counts, f32, w.J)
    assert len({r.key for r in reqs}) <= 1024
    assert sum(r.offset > 0 for r in reqs) > 0.9 * len(reqs)


def test_host_preload_fills_the_seed_table(bd):
    """Preloading exactly max_seeds seeds works (repeats are free); one more
    distinct seed is refused."""
    eng = host_engine(max_seeds=8)
    eng.preload_seeds([1, 2, 3, 3, 4, 5, 6, 7, 8, 1])
    with pytest.raises(bd.RanmarError) as ei:
        eng.preload_seeds([9])
    assert ei.value.code == bd.ERANGE
    eng.close()


class SchedulerModel:
    """The scheduler's rules written out in Python for a host-only engine
    run with every request available at once (no timing involved): FIFO
    admission while the iteration's segments, a first-fit output region and
    the state entries allow (least recently used resident states evicted
    first), resume when the stream's resident state stands at the request's
    offset, iterations retired oldest first when the loop must wait, the
    last state of each request kept resident.  Produces the plan the native
    engine must record."""

    def __init__(self, out_words, entries, seg, max_segs, max_inflight, max_seeds):
        self.free_blocks = {0: out_words}          # start -> length
        self.out_words, self.entries, self.seg = out_words, entries, seg
        self.max_segs, self.max_inflight, self.max_seeds = max_segs, max_inflight, max_seeds
        self.free = list(range(entries - 1, -1, -1))
        self.resident = collections.OrderedDict()  # key -> (entry, end), LRU first
        self.seed_row = {}
        self.evicted = self.resumed = 0

    @staticmethod
    def rounded(n):
        return (max(n, 1) + 31) // 32 * 32

    def alloc(self, n):
        n = self.rounded(n)
        for st in sorted(self.free_blocks):
            ln = self.free_blocks[st]
            if ln >= n:
                del self.free_blocks[st]
                if ln > n:
                    self.free_blocks[st + n] = ln - n
                return st
        return None

    def release(self, st, n):
        n = self.rounded(n)
        self.free_blocks[st] = n
        nxt = st + n
        if nxt in self.free_blocks:
            self.free_blocks[st] += self.free_blocks.pop(nxt)
        prev = [s for s in self.free_blocks if s < st]
        if prev and max(prev) + self.free_blocks[max(prev)] == st:
            p = max(prev)
            self.free_blocks[p] += self.free_blocks.pop(st)

    def nseg(self, count):
        return max(1, -(-count // self.seg))

    def take(self, n):
        while len(self.free) < n and self.resident:
            _, (e, _) = self.resident.popitem(last=False)
            self.free.append(e)
            self.evicted += 1
        if len(self.free) < n:
            return None
        got = self.free[len(self.free) - n:]
        del self.free[len(self.free) - n:]
        return got

    def run(self, reqs):
        waiting = collections.deque(range(len(reqs)))
        inflight, plan, live, n_iter = collections.deque(), [], {}, 0
        while waiting or inflight:
            it, nsegs = [], 0
            if len(inflight) < self.max_inflight:
                while waiting:
                    r = reqs[waiting[0]]
                    ns = self.nseg(r.count)
                    if self.rounded(r.count) > self.out_words or ns > self.entries:
                        waiting.popleft()
                        continue
                    if it and nsegs + ns > self.max_segs:
                        break
                    res = self.resident.get(r.key)
                    resume = res is not None and res[1] == r.offset
                    region = self.alloc(r.count)
                    if region is None:
                        break
                    ents = []
                    if resume:
                        ents.append(self.resident.pop(r.key)[0])
                    got = self.take(ns - 1 if resume else ns)
                    if got is None:
                        self.release(region, r.count)
                        if resume:
                            self.resident[r.key] = (ents[0], r.offset)
                        break
                    self.resumed += resume
                    it.append((waiting.popleft(), region, ents + got, resume))
                    nsegs += ns
            if it:
                for q, _, _, _ in it:
                    if reqs[q].seed not in self.seed_row:
                        self.seed_row[reqs[q].seed] = len(self.seed_row)
                for q, region, ents, resume in it:
                    r = reqs[q]
                    for j, ent in enumerate(ents):
                        js = j * self.seg
                        if not resume:
                            kind, src, e = 0, self.seed_row[r.seed], r.k * r.J + r.offset + js
                        elif j:
                            kind, src, e = 1, ents[0], js
                        else:
                            kind, src, e = 2, ent, 0
                        plan.append((n_iter, q, kind, ent, src, int(j == len(ents) - 1), e,
                                     region + js, max(0, min(self.seg, r.count - js)), js))
                inflight.append((n_iter, it))
                n_iter += 1
                continue
            num, old = inflight.popleft()
            live[num] = n_iter
            for q, region, ents, _ in old:
                r = reqs[q]
                self.release(region, r.count)
                self.free.extend(ents[:-1])
                cur = self.resident.get(r.key)
                end = r.offset + r.count
                if cur is None:
                    self.resident[r.key] = (ents[-1], end)
                elif cur[1] < end:
                    self.free.append(cur[0])
                    del self.resident[r.key]
                    self.resident[r.key] = (ents[-1], end)
                else:
                    self.free.append(ents[-1])
        return plan, live


@pytest.mark.parametrize("entries,max_inflight,max_segs", [(40, 3, 24), (12, 2, 24),
                                                           (300, 4, 7), (64, 1, 100)])
def test_native_scheduler_follows_the_model(bd, entries, max_inflight, max_segs):
    """The native scheduler's plan (iterations, entries, eviction and resume
    choices, regions, exponents) equals the Python model's, record for
    record, on request mixes with many repeats of few streams."""
    rng = np.random.default_rng(entries + max_segs)
    n = 400
    t = np.sort(rng.random(n))
    sd, k = rng.integers(1, 4, n), rng.integers(0, 7, n)
    c = np.minimum(10 * 16, np.floor(10.0 ** (2.3 * rng.random(n)))).astype(np.int64)
    c[:5] = [0, 1, 16, 17, 160]
    J = (1 << 64) + 5
    reqs = serve.make_requests(t, sd, k, c, np.zeros(n, bool), J)
    out_words = 3000
    eng = host_engine(budget_bytes=entries * 400 + out_words * 4, state_entries=entries,
                      max_inflight=max_inflight, max_segments_per_iter=max_segs)
    eng.run(reqs, realtime=False)
    tr = eng.trace()
    st = eng.stats
    eng.close()
    model = SchedulerModel(out_words, entries, 16, max_segs, max_inflight, 64)
    plan, live = model.run(reqs)
    got = [(int(x["iteration"]), int(x["request"]), int(x["kind"]), int(x["entry"]),
            int(x["src"]), int(x["flags"]), exponent(x) if x["kind"] != 2 else 0,
            int(x["out_offset"]), int(x["count"]), int(x["index0"])) for x in tr]
    assert len(got) == len(plan)
    for a, b in zip(got, plan):
        assert a == b, (a, b)
    assert [int(x["live_until"]) for x in tr] == [live[p[0]] for p in plan]
    assert (st["evicted"], st["resumed"]) == (model.evicted, model.resumed)
    assert st["resumed"] > 0
    if entries <= 64:
        assert st["evicted"] > 0


def test_request_records_with_long_streams(bd):
    """J of 2^64 and more splits over the record's two words; offsets group
    by the whole key; a request is overlapping only when it runs past J."""
    J = (1 << 100) + 3
    a = serve.requests_array([0.0, 0.1, 0.2], [5, 5, 5], [(1 << 63) + 1, (1 << 63) + 1, 2],
                             [10, 20, 30], [False, True, False], J)
    assert [int(x) for x in a["J"][:, 0]] == [3] * 3 and [int(x) for x in a["J"][:, 1]] == [1 << 36] * 3
    assert [int(x) for x in a["offset"]] == [0, 10, 0]
    a["status"] = bd.REQ_DONE
    a["done"] = a["t"] + 1e-3
    assert serve.summarize_array(a)["overlapping_requests"] == 0
    b = serve.requests_array([0.0, 0.1], [5, 5], [0, 0], [60, 50], [False, False], 100)
    b["status"] = bd.REQ_DONE
    b["done"] = b["t"] + 1e-3
    assert serve.summarize_array(b)["overlapping_requests"] == 1     # 60 + 50 > 100
