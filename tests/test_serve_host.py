"""Host side of the serving engine (no GPU): resume offsets, the request
recipe, and the native scheduler run with RANMAR_SERVE_HOST_ONLY, whose
recorded plan (jumps, segments, write-backs, regions) is executed here with
the oracle and must give every request exactly its stream's outputs."""
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
