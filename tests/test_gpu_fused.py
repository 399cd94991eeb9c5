"""GPU parity of the fused partition + generation kernel
(ranmar_partition_generate_*): every output and every resumed state equals
the oracle's, and the same as the two-call path (table partition, then
generation with write-back), bit for bit.  Tolerance 0."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

F = 1.0 / 16777216.0


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


@pytest.fixture(scope="module")
def dev(rm):
    return torch.device("cuda:0")


@pytest.mark.parametrize("f32", [False, True])
@pytest.mark.parametrize("n,count,k0,J", [
    (37, 1000, 0, 1 << 40),            # ragged group (37 = 2*16 + 5) and ragged count
    (16, 4096, 7, 1 << 40),            # one whole group, whole ring turns
    (5, 97, 123456, (1 << 48) + 1),    # fewer streams than an interleaved set
    (21, 1, 3, 12345),                 # one output each
    (18, 0, 11, 1 << 64),              # no outputs: only the jump (state written)
    (33, 3 * 96 + 31, 0, (1 << 120) + 12345),
])
def test_fused_matches_oracle(rm, table, dev, orc, f32, n, count, k0, J):
    seed = 12345
    base = rm.seed(seed).to(dev)
    states, out = table.partition_generate(base, J, k0, n, count, f32=f32)
    torch.cuda.synchronize()
    st = rm.state_words_np(states)
    o = out.cpu().numpy()
    x0, c0 = orc.seeded_state(seed)
    for i in range(n):
        E = (k0 + i) * J
        if count:
            ref = orc.stream(seed, E, count)
            if f32:
                assert np.array_equal(o[i], (ref.astype(np.float64) * F).astype(np.float32)), i
            else:
                assert np.array_equal(o[i].view(np.uint32), ref), i
        xs, cs = orc.jump(x0, c0, E + count)
        assert np.array_equal(st[i, :97], xs) and st[i, 97] == cs, i
        pos = int(st[i, 98]) | (int(st[i, 99]) << 32)
        assert pos == (E + count) % (1 << 64), i


def test_fused_full_size_equals_two_calls(rm, table, dev, orc):
    from paper_2512_00093_gb300.workloads import Partitioned
    w = Partitioned()
    base = rm.seed(w.seed).to(dev)
    n, count = w.n_streams, w.count
    s1, o1 = table.partition_generate(base, w.J, w.k0, n, count)
    s2 = table.partition(base, w.J, w.k0, n)
    o2 = torch.empty((n, count), dtype=torch.int32, device=dev)
    desc = rm.make_desc(np.arange(n), np.arange(n) * count, count, rm.DESC_WRITE_BACK, device=dev)
    rm.generate_u24(s2, desc, o2)
    torch.cuda.synchronize()
    assert torch.equal(o1, o2)
    assert torch.equal(s1, s2)
    rows = w.verify_rows()[:32]
    got = o1[torch.as_tensor(rows, device=dev)].cpu().numpy().view(np.uint32)
    for r, row in zip(rows, got):
        assert np.array_equal(row, orc.stream(w.seed, (w.k0 + int(r)) * w.J, count)), int(r)


def test_fused_period_reduction_same_results(rm, table, dev):
    base = rm.seed(2).to(dev)
    J = (1 << 130) + 7
    a = table.partition_generate(base, J, 1000, 40, 500, flags=rm.JUMP_REDUCE_PERIOD)
    b = table.partition_generate(base, J, 1000, 40, 500, flags=0)
    torch.cuda.synchronize()
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


def test_fused_host_errors(rm, table, dev):
    base = rm.seed(3).to(dev)
    lib = rm.binding._lib()
    states = torch.empty((8, 100), dtype=torch.int32, device=dev)
    out = torch.empty(8 * 64, dtype=torch.int32, device=dev)
    J = np.array([0, 1], dtype=np.uint32)   # 2^32
    call = lib.ranmar_partition_generate_u24
    # unknown flag
    assert call(table._h, base.data_ptr(), J.ctypes.data, 2, 0, 8, 64, 4, states.data_ptr(),
                out.data_ptr(), None) == rm.binding.EINVAL
    # output overlapping the states
    assert call(table._h, base.data_ptr(), J.ctypes.data, 2, 0, 8, 64, 0, states.data_ptr(),
                states.data_ptr() + 64, None) == rm.binding.EINVAL
    # misaligned states
    assert call(table._h, base.data_ptr(), J.ctypes.data, 2, 0, 8, 64, 0,
                states.data_ptr() + 4, out.data_ptr(), None) == rm.binding.EINVAL
    # exponent beyond 160 bits
    Jbig = np.array([0, 0, 0, 0, 0x80000000], dtype=np.uint32)
    assert call(table._h, base.data_ptr(), Jbig.ctypes.data, 5, 2, 8, 64, 0, states.data_ptr(),
                out.data_ptr(), None) == rm.binding.ERANGE
    # n = 0 is a no-op
    assert call(table._h, base.data_ptr(), J.ctypes.data, 2, 0, 0, 64, 0, states.data_ptr(),
                out.data_ptr(), None) == 0
