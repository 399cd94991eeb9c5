"""GPU parity of the warp-per-stream table jump (RANMAR_JUMP_MAP_WARP)
against the two-lanes-per-stream kernels and the oracle: the same P_E
(Sec. 3.1, a product of table rows over the digits of the exponent) and the
same application and c jump (Sec. 3.2), so every state must be bit-identical
whichever mapping runs."""
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
def tables(rm):
    """One table per mapping (the mapping is a property of the handle)."""
    out = {}
    for name, m in [("pair", rm.JUMP_MAP_PAIR), ("warp", rm.JUMP_MAP_WARP),
                    ("auto", rm.JUMP_MAP_AUTO)]:
        t = rm.Table()
        t.set_jump_mapping(m)
        out[name] = t
    yield out
    for t in out.values():
        t.close()


EDGE_EXPS = [0, 1, 2, 96, 97, 98, 255, 256, 257, 1 << 8, (1 << 16) - 1, 1 << 40,
             (1 << 64) + 12345, (1 << 120) + 12345, ((1 << 97) - 1) << 23,
             (1 << 159) + 3, (1 << 160) - 1, int("5a" * 20, 16)]


def test_warp_jump_equals_pair_and_oracle(rm, tables, orc):
    from paper_2512_00093_gb300.workloads import random_exponents
    dev = torch.device("cuda:0")
    exps = EDGE_EXPS + random_exponents(150, 160, seed=33)
    seeds = [12345, 2, 54217138]
    bases = torch.stack([rm.seed(s).to(dev) for s in seeds])
    idx = torch.tensor([i % 3 for i in range(len(exps))], dtype=torch.int32, device=dev)
    ex = rm.exps_tensor(exps, 5, device=dev)
    w = tables["warp"].jump(bases, ex, base_idx=idx)
    p = tables["pair"].jump(bases, ex, base_idx=idx)
    torch.cuda.synchronize()
    assert torch.equal(w, p)
    got = rm.state_words_np(w)
    for i in list(range(len(EDGE_EXPS))) + list(range(len(EDGE_EXPS), len(exps), 11)):
        x, c = orc.seeded_state(seeds[i % 3])
        xr, cr = orc.jump(x, c, exps[i])
        assert np.array_equal(got[i, :97], xr) and got[i, 97] == cr, (i, exps[i])
        assert int(got[i, 98]) | int(got[i, 99]) << 32 == exps[i] % (1 << 64), i


@pytest.mark.parametrize("J", [1 << 40, (1 << 64) + 12345, (1 << 120) + 12345])
def test_warp_partition_equals_pair(rm, tables, J):
    """Mode 1 (E = (k0 + i) J), batch sizes around the warp count of a CTA
    and the automatic switch, with the exponent-period reduction on and off."""
    dev = torch.device("cuda:0")
    base = rm.seed(12345).to(dev)
    for k0, n in [(0, 1), (3, 5), (0, 255), (7, 256), (1 << 20, 257),
                  (99, rm.JUMP_WARP_AUTO_MAX), (5, rm.JUMP_WARP_AUTO_MAX + 1), (0, 5000)]:
        if (k0 + n - 1).bit_length() + J.bit_length() > 160:
            continue
        for flags in (0, rm.JUMP_REDUCE_PERIOD):
            a = rm.partition_ex(base, J, k0, n, table=tables["warp"], flags=flags)
            b = rm.partition_ex(base, J, k0, n, table=tables["pair"], flags=flags)
            c = rm.partition_ex(base, J, k0, n, table=tables["auto"], flags=flags)
            torch.cuda.synchronize()
            assert torch.equal(a, b), (J, k0, n, flags)
            assert torch.equal(c, b), (J, k0, n, flags)


def test_warp_jump_scatter_and_bad_indices(rm, tables):
    """Destination indices, base indices past the end (flagged, skipped) and a
    capped grid (the kernel strides over the remaining streams)."""
    dev = torch.device("cuda:0")
    t = tables["warp"]
    pool = torch.zeros((64, 100), dtype=torch.int32, device=dev)
    pool[5] = rm.seed(77).to(dev)
    exps = [0, 1, 1 << 70, (1 << 159) + 3, 12345678901]
    dst = torch.tensor([9, 40, 2, 63, 11], dtype=torch.int32, device=dev)
    bi = torch.full((5,), 5, dtype=torch.int32, device=dev)
    ex = rm.exps_tensor(exps, 5, device=dev)
    t.jump(pool, ex, base_idx=bi, out=pool, dst_idx=dst)
    ref = rm.jump(pool[5:6].clone(), ex)
    torch.cuda.synchronize()
    assert torch.equal(pool[dst.long()], ref)

    st = torch.zeros(1, dtype=torch.int32, device=dev)
    base = rm.seed(9).to(dev).reshape(1, -1)
    bad = torch.tensor([0, 1, 0], dtype=torch.int32, device=dev)   # 1 >= n_base
    out = torch.zeros((3, 100), dtype=torch.int32, device=dev)
    t.jump(base, rm.exps_tensor([5, 6, 7], 5, device=dev), base_idx=bad, out=out, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) & rm.ST_BAD_INDEX
    assert not out[1].any()
    assert torch.equal(out[[0, 2]], rm.jump(base, rm.exps_tensor([5, 7], 5, device=dev)))

    t.set_ctas_per_sm(1)
    try:
        n = 3000
        a = rm.partition_ex(rm.seed(1).to(dev), 1 << 48, 11, n, table=t)
        b = rm.partition_ex(rm.seed(1).to(dev), 1 << 48, 11, n, table=tables["pair"])
        torch.cuda.synchronize()
        assert torch.equal(a, b)
    finally:
        t.set_ctas_per_sm(0)


@pytest.mark.parametrize("J", [1 << 40, (1 << 120) + 12345])
def test_plan_jump_warp_equals_pair(rm, tables, orc, J):
    """The plan's jumps by the powers of t^J under both mappings, and the
    plan's partition (its first 256 streams by those jumps)."""
    dev = torch.device("cuda:0")
    base = rm.seed(12345).to(dev)
    plan = rm.Plan(tables["auto"], J, 20000)
    x0, c0 = orc.seeded_state(12345)
    for k0, n in [(0, 1), (0, 256), (255, 300), (12345, 2100)]:
        plan.set_jump_mapping(rm.JUMP_MAP_WARP)
        a = plan.jump(base, k0, n)
        plan.set_jump_mapping(rm.JUMP_MAP_PAIR)
        b = plan.jump(base, k0, n)
        torch.cuda.synchronize()
        assert torch.equal(a, b), (k0, n)
        st = rm.state_words_np(a)
        for i in {0, n - 1}:
            xs, cs = orc.jump(x0, c0, (k0 + i) * J)
            assert np.array_equal(st[i, :97], xs) and st[i, 97] == cs
    plan.set_jump_mapping(rm.JUMP_MAP_WARP)
    got = plan.partition(base, 0, 20000)
    ref = tables["pair"].partition(base, J, 0, 20000)
    torch.cuda.synchronize()
    assert torch.equal(got, ref)
    with pytest.raises(rm.RanmarError):
        plan.set_jump_mapping(3)
    plan.close()
