"""GPU parity of the partition plan (256 streams by the table jump, then
levels of jump matrices of radix 256, 16, ...): the states equal the table
partition's and the oracle's, bit for bit, for stream counts that end
inside every level, and the plan's host checks."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_00093_gb300 as rm
    return rm


@pytest.fixture(scope="module")
def table(rm):
    t = rm.Table()
    yield t
    t.close()


METHODS = {"tensor": 0, "imad": 1, "tensor_pipelined": 2}


@pytest.mark.parametrize("method", list(METHODS))
@pytest.mark.parametrize("J", [1 << 40, (1 << 64) + 12345, (1 << 120) + 12345])
def test_plan_equals_table_partition(rm, table, orc, J, method):
    dev = torch.device("cuda:0")
    base = rm.seed(12345).to(dev)
    plan = rm.Plan(table, J, 70000)
    plan.set_method(METHODS[method])
    for n, k0 in [(1, 0), (255, 3), (256, 0), (257, 9), (511, 1), (512, 0), (513, 4),
                  (4097, 7), (65535, 0), (65536, 123), (65537, 5), (70000, 1 << 20)]:
        a = plan.partition(base, k0, n)
        b = table.partition(base, J, k0, n)
        torch.cuda.synchronize()
        assert torch.equal(a, b), (n, k0)
    # a sample against the oracle directly
    st = rm.state_words_np(a)
    x0, c0 = orc.seeded_state(12345)
    for i in [0, 255, 256, 511, 512, 4095, 4096, 65535, 65536, 69999]:
        xr, cr = orc.jump(x0, c0, ((1 << 20) + i) * J)
        assert np.array_equal(st[i, :97], xr) and st[i, 97] == cr, i
        pos = int(st[i, 98]) | (int(st[i, 99]) << 32)
        assert pos == (((1 << 20) + i) * J) % (1 << 64), i
    assert plan.status() == 0
    plan.close()


def test_plan_other_seeds_and_resume(rm, table, orc):
    dev = torch.device("cuda:0")
    J = 1 << 48
    plan = rm.Plan(table, J, 300)
    for s in (1, 54217138, 900000000):
        base = rm.seed(s).to(dev)
        a = plan.partition(base, 77, 300)
        b = table.partition(base, J, 77, 300)
        torch.cuda.synchronize()
        assert torch.equal(a, b), s
    # a non-seeded base (an advanced state with its own c and pos)
    base = table.partition(rm.seed(5).to(dev), 12345, 9, 1)
    a = plan.partition(base, 2, 300)
    b = table.partition(base, J, 2, 300)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    plan.close()


def test_plan_host_checks(rm, table):
    dev = torch.device("cuda:0")
    base = rm.seed(3).to(dev)
    plan = rm.Plan(table, 1 << 40, 1000)
    with pytest.raises(rm.RanmarError):
        plan.partition(base, 0, 1001)                # n > max_n
    with pytest.raises(rm.RanmarError):
        plan.partition(base, (1 << 64) - 1, 2)       # k0 + n - 1 overflows
    with pytest.raises(rm.RanmarError):
        rm.Plan(table, (1 << 159), 1 << 20)          # 15 * 65536 * J >= 2^160
    out = torch.empty((4, 100), dtype=torch.int32, device=dev)
    with pytest.raises(rm.RanmarError):
        plan.partition(out[0:1], 0, 4, out=out)      # output overlaps the base
    with pytest.raises(rm.RanmarError):
        plan.set_method(7)
    plan.close()


@pytest.mark.parametrize("ctas", [1, 3, 7, 32, 151, 600])
def test_plan_ctas(rm, table, ctas):
    """A tensor-core level on fewer (or more) CTAs than SMs: every CTA takes a
    balanced range of (tile, matrix) items; the states do not change."""
    dev = torch.device("cuda:0")
    J = 1 << 40
    base = rm.seed(12345).to(dev)
    plan = rm.Plan(table, J, 70000)
    ref = table.partition(base, J, 7, 70000)
    plan.set_ctas(ctas)
    got = plan.partition(base, 7, 70000)
    torch.cuda.synchronize()
    assert torch.equal(got, ref)
    assert plan.status() == 0
    with pytest.raises(rm.RanmarError):
        plan.set_ctas(70000)
    plan.close()


@pytest.mark.parametrize("method", ["tensor", "tensor_pipelined"])
def test_plan_timeout_path(rm, table, method):
    """Failure detection without a fault: with the first wait of every CTA of
    the tensor-core level made on a barrier that nothing completes (one
    non-blocking probe), the level gives up, flags
    RANMAR_ST_TIMEOUT and returns (its CTAs drain their own copies and MMAs
    first); the context stays usable and a fresh plan gives the right
    states."""
    dev = torch.device("cuda:0")
    J = 1 << 40
    base = rm.seed(3).to(dev)
    plan = rm.Plan(table, J, 5000)
    plan.set_method(METHODS[method])
    torch.cuda.synchronize()
    rm.debug_set_wait_limit(1)
    try:
        plan.partition(base, 0, 5000)
        torch.cuda.synchronize()
        assert plan.status() & rm.ST_TIMEOUT
    finally:
        rm.debug_set_wait_limit(0)
    plan.close()
    plan = rm.Plan(table, J, 5000)
    plan.set_method(METHODS[method])
    got = plan.partition(base, 0, 5000)
    ref = table.partition(base, J, 0, 5000)
    torch.cuda.synchronize()
    assert torch.equal(got, ref)
    assert plan.status() == 0
    plan.close()


def test_plan_expand_from_table_rows(rm, table):
    """expand() from the first 256 rows computed elsewhere (the table
    partition on another stream) gives the same states as one partition_plan
    call."""
    dev = torch.device("cuda:0")
    J = 1 << 40
    base = rm.seed(12345).to(dev)
    plan = rm.Plan(table, J, 5000)
    side = torch.cuda.Stream(dev)
    st = torch.empty((5000, 100), dtype=torch.int32, device=dev)
    table.partition(base, J, 99, 256, out=st[:256], stream=side)
    ev = torch.cuda.Event()
    ev.record(side)
    torch.cuda.current_stream().wait_event(ev)
    plan.expand(st, 5000)
    ref = plan.partition(base, 99, 5000)
    torch.cuda.synchronize()
    assert torch.equal(st, ref)
    assert plan.status() == 0
    plan.close()


def test_plan_million_streams_equals_table(rm, table):
    """10^6 streams (the batched-uneven shape, J = 2^64): the radix-256 level
    and a radix-16 level, both methods, against the per-stream table jump."""
    dev = torch.device("cuda:0")
    J = 1 << 64
    n = 1_000_000
    base = rm.seed(12345).to(dev)
    plan = rm.Plan(table, J, n)
    ref = table.partition(base, J, 3, n)
    for method in (rm.Plan.TENSOR, rm.Plan.IMAD):
        plan.set_method(method)
        got = plan.partition(base, 3, n)
        torch.cuda.synchronize()
        assert torch.equal(got, ref), method
        del got
    assert plan.status() == 0
    plan.close()


def test_partitioned_full_size_bench_path(rm, table, orc):
    """The benchmark's step at full size (65,536 streams x 4,096 u24 outputs,
    J = 2^40, a batch that starts at k0 = 5 * 65,536): the first 256 streams
    by the table jump on a side stream, the tensor-core level for the rest,
    then generation with write-back; 256 sampled rows and their advanced
    states against the oracle."""
    from paper_2512_00093_gb300.workloads import Partitioned
    w = Partitioned()
    dev = torch.device("cuda:0")
    n, count, k0 = w.n_streams, w.count, 5 * w.n_streams
    base = rm.seed(w.seed).to(dev)
    plan = rm.Plan(table, w.J, n)
    states = torch.empty((n, rm.STATE_WORDS), dtype=torch.int32, device=dev)
    out = torch.empty((n, count), dtype=torch.int32, device=dev)
    desc = rm.make_desc(np.arange(n), np.arange(n) * count, count, rm.DESC_WRITE_BACK,
                        device=dev)
    side, main = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    table.partition(base, w.J, k0, 256, out=states[:256], stream=side)
    ev = torch.cuda.Event()
    ev.record(side)
    main.wait_event(ev)
    plan.expand(states, n, stream=main)
    rm.generate_u24(states, desc, out, stream=main)
    torch.cuda.synchronize()
    assert plan.status() == 0
    rows = w.verify_rows()
    got = out[torch.as_tensor(rows, device=dev)].cpu().numpy().view(np.uint32)
    after = rm.state_words_np(states)
    x0, c0 = orc.seeded_state(w.seed)
    for q, (r, row) in enumerate(zip(rows, got)):
        E = (k0 + int(r)) * w.J
        assert np.array_equal(row, orc.stream(w.seed, E, count)), int(r)
        if q % 32 == 0:
            xs, cs = orc.jump(x0, c0, E + count)
            assert np.array_equal(after[r, :97], xs) and after[r, 97] == cs, int(r)
    plan.close()


@pytest.mark.parametrize("J", [3, 10**6, 1 << 40, (1 << 64) + 12345, (1 << 120) + 12345,
                               (1 << 140) + 7])
def test_plan_jump_by_powers_of_tJ(rm, table, orc, J):
    """ranmar_plan_jump (P_{kJ} over the base-256 digits of k, from the plan's
    table of the powers of t^J) gives the fixed-base table's states, and the
    oracle's on a sample; streams past the table's windows are refused."""
    dev = torch.device("cuda:0")
    base = rm.seed(12345).to(dev)
    plan = rm.Plan(table, J, 300)
    W = min(8, (160 - J.bit_length()) // 8)
    x0, c0 = orc.seeded_state(12345)
    for k0, n in [(0, 1), (0, 300), (255, 3), (12345, 700), ((1 << 31) + 5, 33),
                  ((1 << 63) - 40, 40)]:
        kmax = k0 + n - 1
        if kmax.bit_length() + J.bit_length() > 160:
            continue
        if kmax.bit_length() > 8 * W:
            with pytest.raises(rm.RanmarError):
                plan.jump(base, k0, n)
            continue
        got = plan.jump(base, k0, n)
        ref = table.partition(base, J, k0, n)
        torch.cuda.synchronize()
        assert torch.equal(got, ref), (J, k0, n)
        st = rm.state_words_np(got)
        for i in {0, n - 1}:
            xs, cs = orc.jump(x0, c0, (k0 + i) * J)
            assert np.array_equal(st[i, :97], xs) and st[i, 97] == cs
    plan.close()


def test_plan_base_falls_back_to_fixed_table(rm, table):
    """J = 2^140: the table of the powers of t^J has two windows (k < 2^16),
    so the first streams of a batch at k0 = 65,500 (k up to 65,799) come
    from the fixed-base table; the states are the same, and ranmar_plan_jump
    refuses those k."""
    dev = torch.device("cuda:0")
    J = 1 << 140
    base = rm.seed(9).to(dev)
    plan = rm.Plan(table, J, 300)
    got = plan.partition(base, 65500, 300)
    ref = table.partition(base, J, 65500, 300)
    torch.cuda.synchronize()
    assert torch.equal(got, ref)
    with pytest.raises(rm.RanmarError):
        plan.jump(base, 65500, 300)
    assert torch.equal(plan.jump(base, 0, 256), table.partition(base, J, 0, 256))
    plan.close()
