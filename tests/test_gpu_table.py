"""GPU parity of the fixed-base table jump: the table rows are t^{d 2^{8j}}
mod phi (oracle), and every jumped state equals the square-and-multiply
kernel's and the oracle's, bit for bit."""
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


def test_table_rows_are_fixed_base_powers(rm, table, orc):
    rows = table.rows_tensor().cpu().numpy().view(np.uint32)
    rng = np.random.default_rng(0)
    picks = [(0, 0), (0, 1), (0, 255), (1, 1), (19, 255), (19, 1), (12, 128)]
    picks += [(int(j), int(d)) for j, d in zip(rng.integers(0, 20, 40), rng.integers(0, 256, 40))]
    for j, d in picks:
        ref = orc.poly_pow_t(d << (8 * j))
        assert np.array_equal(rows[j * 256 + d, :97], ref), (j, d)
        assert not rows[j * 256 + d, 97:].any()


def test_table_jump_equals_square_and_multiply_and_oracle(rm, table, orc):
    from paper_2512_00093_gb300.workloads import random_exponents
    dev = torch.device("cuda:0")
    exps = random_exponents(170, 160, seed=21)
    seeds = [12345, 2, 54217138]
    bases = torch.stack([rm.seed(s).to(dev) for s in seeds])
    idx = torch.tensor([i % 3 for i in range(len(exps))], dtype=torch.int32, device=dev)
    ex = rm.exps_tensor(exps, 5, device=dev)
    a = table.jump(bases, ex, base_idx=idx)
    b = rm.jump(bases, ex, base_idx=idx)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    got = rm.state_words_np(a)
    for i in range(0, len(exps), 7):
        x, c = orc.seeded_state(seeds[i % 3])
        xr, cr = orc.jump(x, c, exps[i])
        assert np.array_equal(got[i, :97], xr) and got[i, 97] == cr, i


def test_table_jump_scatter_into_pool(rm, table):
    dev = torch.device("cuda:0")
    pool = torch.zeros((64, 100), dtype=torch.int32, device=dev)
    pool[5] = rm.seed(77).to(dev)
    exps = [0, 1, 1 << 70, (1 << 159) + 3, 12345678901]
    dst = torch.tensor([9, 40, 2, 63, 11], dtype=torch.int32, device=dev)
    bi = torch.full((5,), 5, dtype=torch.int32, device=dev)
    ex = rm.exps_tensor(exps, 5, device=dev)
    table.jump(pool, ex, base_idx=bi, out=pool, dst_idx=dst)
    ref = rm.jump(pool[5:6].clone(), ex)
    torch.cuda.synchronize()
    assert torch.equal(pool[dst.long()], ref)


@pytest.mark.parametrize("which", ["partitioned", "large"])
def test_partition_tab_full_size_equals_square_and_multiply(rm, table, which):
    from paper_2512_00093_gb300.workloads import LargeJumps, Partitioned
    w = Partitioned() if which == "partitioned" else LargeJumps()
    dev = torch.device("cuda:0")
    base = rm.seed(w.seed).to(dev)
    a = table.partition(base, w.J, 0, w.n_streams)
    b = rm.partition(base, w.J, 0, w.n_streams)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


@pytest.mark.parametrize("use_table", [True, False])
def test_period_reduction_gives_identical_states(rm, table, use_table):
    """E mod T (T = (2^97 - 1) 2^23, the order of t) for the polynomial part:
    same states as the unreduced jump, for J around and beyond 2^120."""
    from paper_2512_00093_gb300.workloads import LargeJumps
    dev = torch.device("cuda:0")
    t = table if use_table else None
    w = LargeJumps()
    base = rm.seed(w.seed).to(dev)
    n = w.n_streams if use_table else 2048
    a = rm.partition_ex(base, w.J, 0, n, table=t, flags=rm.JUMP_REDUCE_PERIOD)
    b = rm.partition_ex(base, w.J, 0, n, table=t, flags=0)
    T = ((1 << 97) - 1) << 23
    for J, k0, cnt in [(T, 0, 64), (T - 1, 5, 64), ((1 << 159) - 1, 0, 2),
                       ((1 << 130) + 7, 1000, 64), (12345, 3, 64)]:
        x = rm.partition_ex(base, J, k0, cnt, table=t, flags=rm.JUMP_REDUCE_PERIOD)
        y = rm.partition_ex(base, J, k0, cnt, table=t, flags=0)
        torch.cuda.synchronize()
        assert torch.equal(x, y), (J, k0)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
