"""GPU serving tests: every request's outputs (through the device checksum)
equal the oracle's, and each result is the same alone and in the mix.
Tolerance 0."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

J48 = 1 << 48


@pytest.fixture(scope="module")
def rm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_00093_gb300 as rm
    return rm


def mixed_requests(n, seed, seeds=5, ks=6, cmax=120_000, duration=0.2):
    """A Poisson-like request list with few distinct streams, so that many
    requests resume a stream that earlier requests consumed."""
    from paper_2512_00093_gb300.serve import make_requests
    rng = np.random.default_rng(seed)
    t = np.sort(rng.random(n) * duration)
    sd = rng.integers(1, seeds + 1, n)
    k = rng.integers(0, ks, n)
    c = np.floor(10.0 ** (1 + np.log10(cmax / 10) * rng.random(n))).astype(np.int64)
    c[:8] = [1, 31, 32, 33, 4095, 4096, 4097, 8192 + 5]
    f32 = rng.random(n) < 0.5
    return make_requests(t, sd, k, c, f32, J48)


def expected_checksum(orc, rm, r):
    y = orc.stream(r.seed, r.k * r.J + r.offset, r.count)
    if r.f32:
        y = (y.astype(np.float64) / 16777216.0).astype(np.float32).view(np.uint32)
    return rm.checksum_np(y)


def check_all(orc, rm, reqs):
    bad = [r.rid for r in reqs if r.checksum != expected_checksum(orc, rm, r)]
    assert not bad, f"checksum mismatch for requests {bad[:10]}"


def test_checksum_kernel_matches_host(rm):
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(1)
    data = torch.as_tensor(rng.integers(0, 1 << 24, 100_000).astype(np.int32), device=dev)
    items = torch.tensor([[0, 40_000, 0, 0], [40_000, 60_000, 40_000, 0], [5, 7, 3, 1]],
                         dtype=torch.int64, device=dev)
    res = torch.zeros(2, dtype=torch.int64, device=dev)
    rm.checksum(data, items, res)
    torch.cuda.synchronize()
    h = data.cpu().numpy()
    got = res.cpu().numpy().astype(np.uint64)
    assert int(got[0]) == rm.checksum_np(h)                 # split items sum to the whole
    assert int(got[1]) == rm.checksum_np(h[5:12], index0=3)


def test_checksum_kernel_ragged_items(rm):
    """Items at every alignment, of lengths 0..9 and across several passes of
    the kernel's vector loop, some sharing a result slot: each slot equals
    the host sum of its items."""
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(2)
    data_h = rng.integers(0, 1 << 32, 300_000, dtype=np.uint64).astype(np.uint32)
    data = torch.as_tensor(data_h.view(np.int32), device=dev)
    items, want = [], {}
    for q in range(400):
        off = int(rng.integers(0, 200_000))
        cnt = int(rng.integers(0, 10)) if q % 2 else int(rng.integers(0, 90_000))
        idx0 = int(rng.integers(0, 1 << 40))
        slot = q % 37
        items.append([off, cnt, idx0, slot])
        want[slot] = (want.get(slot, 0) + rm.checksum_np(data_h[off:off + cnt], index0=idx0)) \
            % (1 << 64)
    res = torch.zeros(37, dtype=torch.int64, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    rm.checksum(data, torch.tensor(items, dtype=torch.int64, device=dev), res, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    got = res.cpu().numpy().astype(np.uint64)
    assert [int(got[s]) for s in range(37)] == [want[s] for s in range(37)]


def test_serving_mix_matches_oracle_and_alone(rm, orc):
    from paper_2512_00093_gb300.serve import Engine, Request
    reqs = mixed_requests(260, 7)
    # small segments, few segments per iteration and a tiny state pool: many
    # iterations, multi-segment requests, pool jumps, resumes and evictions.
    # 40 entries: the 30 distinct streams stay resident once seen, so every
    # admission of a request of more than 10 segments must evict, however
    # many iterations happen to be in flight
    eng = Engine(budget_bytes=64 << 20, seg=4096, state_entries=40,
                 max_segments_per_iter=48, max_inflight=3, use_table=False)
    summary = eng.run(reqs, realtime=False)
    assert summary["requests"] == len(reqs)
    assert eng.stats["resumed"] > 0 and eng.stats["evicted"] > 0
    check_all(orc, rm, reqs)
    eng.close()
    # each of a sample, alone in a fresh engine, with its offset as admitted
    for r in [reqs[i] for i in (0, 3, 7, 40, 100, 200, 259)]:
        solo = Request(0, 0.0, r.seed, r.k, r.J, r.count, r.f32, offset=r.offset)
        e2 = Engine(budget_bytes=64 << 20, seg=4096, state_entries=96, use_table=True)
        e2.run([solo], realtime=False)
        e2.close()
        assert solo.checksum == r.checksum, r.rid


def test_serving_realtime_and_plain(rm, orc):
    from paper_2512_00093_gb300.serve import Engine
    reqs = mixed_requests(150, 9, seeds=40, ks=1000, duration=0.15)
    eng = Engine(budget_bytes=256 << 20, seg=1 << 14, state_entries=4096)
    s = eng.run(reqs, realtime=True)
    assert s["p50_ms"] is not None and s["p99_ms"] >= s["p50_ms"]
    check_all(orc, rm, reqs)
    got = [r.checksum for r in reqs]
    for r in reqs:
        r.checksum, r.done = -1, -1.0
    eng.run_plain(reqs, realtime=True)
    assert [r.checksum for r in reqs] == got
    eng.close()


def test_serving_injected_failure_then_recovers(rm, orc):
    """Failure detection on the host: a library call that fails in the middle
    of a serving run (injected with ranmar_debug_fail_next) ends the run with
    an exception instead of a hang; the context stays usable and a new
    engine serves the same requests correctly."""
    from paper_2512_00093_gb300.serve import Engine, assign_offsets
    reqs = mixed_requests(60, 21, seeds=3, ks=4, cmax=50_000, duration=0.05)
    eng = Engine(budget_bytes=64 << 20, seg=4096, state_entries=256)
    rm.debug_fail_next(rm.binding.ECUDA)
    with pytest.raises(rm.RanmarError) as ei:
        eng.run(reqs, realtime=False)
    assert ei.value.code == rm.binding.ECUDA
    torch.cuda.synchronize()
    eng.close()
    for r in reqs:
        r.checksum, r.done = -1, -1.0
    assign_offsets(reqs)
    eng = Engine(budget_bytes=64 << 20, seg=4096, state_entries=256)
    eng.run(reqs, realtime=False)
    check_all(orc, rm, reqs)
    eng.close()


def test_serving_multiword_J_empty_requests_and_arrays(rm, orc):
    """Streams of length J = 2^120 + 12345 (start exponents k J + offset
    across four words), requests of 0 and 1 outputs, and the same requests
    as REQUEST_DTYPE records give the same checksums as the oracle."""
    from paper_2512_00093_gb300.serve import Engine, make_requests, requests_array
    J = (1 << 120) + 12345
    rng = np.random.default_rng(31)
    n = 40
    t = np.sort(rng.random(n) * 0.01)
    sd, k = rng.integers(1, 4, n), rng.integers(0, 5, n)
    c = rng.integers(0, 20_000, n)
    c[:4] = [0, 1, 0, 4097]
    f32 = rng.random(n) < 0.5
    reqs = make_requests(t, sd, k, c, f32, J)
    eng = Engine(budget_bytes=64 << 20, seg=4096, state_entries=128, max_segments_per_iter=16)
    eng.run(reqs, realtime=False)
    check_all(orc, rm, reqs)
    assert reqs[0].checksum == 0 and reqs[2].checksum == 0
    a = requests_array(t, sd, k, c, f32, J)
    e2 = Engine(budget_bytes=64 << 20, seg=1000, state_entries=128, use_table=False)
    s = e2.run(a, realtime=False)
    assert s["served"] == n
    assert [int(x) for x in a["checksum"]] == [r.checksum for r in reqs]
    eng.close()
    e2.close()


def test_serving_iterations_overlap_on_the_device(rm, orc):
    """Continuous batching: with requests arriving while earlier iterations
    run, more than one iteration is on the device at once, and the results
    still equal the oracle's."""
    from paper_2512_00093_gb300.serve import Engine
    reqs = mixed_requests(300, 17, seeds=20, ks=50, cmax=400_000, duration=0.05)
    eng = Engine(budget_bytes=512 << 20, seg=1 << 14, state_entries=4096, max_inflight=4)
    eng.run(reqs, realtime=True)
    st = eng.stats
    assert st["max_inflight"] >= 2 and st["iterations"] > 10
    check_all(orc, rm, reqs)
    eng.close()


def test_serving_large_iterations_sum_separately(rm, orc):
    """Iterations of more than 4,096 segments take the separate checksum
    kernel instead of the sums inside the generation: checksums still equal
    the oracle's."""
    from paper_2512_00093_gb300.serve import Engine, make_requests
    rng = np.random.default_rng(41)
    n = 12
    t = np.zeros(n)
    sd, k = rng.integers(1, 4, n), rng.integers(0, 50, n)
    c = rng.integers(150_000, 250_000, n)
    reqs = make_requests(t, sd, k, c, rng.random(n) < 0.5, J48)
    eng = Engine(budget_bytes=64 << 20, seg=64, state_entries=16384, max_segments_per_iter=8192)
    eng.run(reqs, realtime=False)
    st = eng.stats
    eng.close()
    assert st["segments"] / st["iterations"] > 4096
    check_all(orc, rm, reqs)
