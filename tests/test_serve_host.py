"""Host-side logic of the serving engine (no GPU): resume offsets, exponent
rows, the output allocator, admission, and the request recipe."""
import collections

import numpy as np

from paper_2512_00093_gb300 import serve
from paper_2512_00093_gb300.serve import FirstFit, Request, assign_offsets, exp_rows
from paper_2512_00093_gb300.workloads import Serving


def test_offsets_follow_arrival_order():
    reqs = [Request(i, 0.1 * i, s, k, 1 << 48, c, False)
            for i, (s, k, c) in enumerate([(1, 0, 10), (1, 1, 5), (1, 0, 7), (2, 0, 3),
                                           (1, 0, 1), (1, 1, 2)])]
    assign_offsets(reqs)
    assert [r.offset for r in reqs] == [0, 0, 10, 0, 17, 5]


def test_exp_rows_multiword_and_carry():
    seg = 1 << 16
    for base in [0, 1, (1 << 64) - 5, (1 << 96) - 1, ((1 << 20) - 1) * (1 << 48) + 10**7,
                 (1 << 159) + 3]:
        rows = exp_rows(base, 9, seg)
        for q in range(9):
            e = base + q * seg
            assert [int(x) for x in rows[q]] == [(e >> (32 * w)) & 0xFFFFFFFF for w in range(5)]


def test_firstfit_alignment_reuse_and_coalescing():
    rng = np.random.default_rng(0)
    f = FirstFit(1 << 20, align=32)
    live = []
    for step in range(2000):
        if live and rng.random() < 0.45:
            f.free(*live.pop(int(rng.integers(len(live)))))
        else:
            r = f.alloc(int(rng.integers(1, 5000)))
            if r is not None:
                assert r[0] % 32 == 0 and r[1] % 32 == 0
                for a, n in live:
                    assert r[0] + r[1] <= a or a + n <= r[0], "overlap"
                live.append(r)
    for r in live:
        f.free(*r)
    assert f.starts == [0] and f.lens == [1 << 20] and f.used == 0


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


def _bare_engine(out_words, state_entries, seg):
    """An Engine with only its host-side admission state (no device memory)."""
    eng = serve.Engine.__new__(serve.Engine)
    eng.seg, eng.max_segs = seg, 1000
    eng.alloc = FirstFit(out_words)
    eng.state_entries = state_entries
    eng.free_entries = list(range(state_entries - 1, -1, -1))
    eng.resident = collections.OrderedDict()
    eng.stats = collections.Counter()
    return eng


def test_admit_refuses_requests_that_can_never_fit():
    """A request larger than the output pool, or with more segments than the
    state pool has entries, is refused when it reaches the head of the queue;
    the requests behind it are admitted instead of waiting behind it."""
    eng = _bare_engine(out_words=1024, state_entries=4, seg=16)
    reqs = serve.make_requests(np.array([0.0, 0.1, 0.2, 0.3]), np.array([1, 2, 3, 4]),
                               np.array([0, 0, 0, 0]), np.array([2000, 100, 30, 64]),
                               np.array([False] * 4), 1 << 48)
    waiting = collections.deque(reqs)
    got = eng.admit(waiting)
    # 2000 > 1024 output words; 100 outputs = 7 segments > 4 state entries
    assert [r.rid for r in got] == [2] and [r.rejected for r in reqs] == [True, True, False, False]
    assert eng.stats["rejected"] == 2
    assert [r.rid for r in waiting] == [3]          # 64 outputs = 4 segments: waits for entries
    for r in reqs[2:]:
        r.done = r.host_done = r.t + 0.001
    s = serve.summarize(reqs)
    assert (s["requests"], s["served"], s["rejected"]) == (4, 2, 2)


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
