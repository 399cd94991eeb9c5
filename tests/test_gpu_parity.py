"""GPU parity: every output of libranmar equals the CPU oracle, bit for bit.

The results of the method are unique (integers mod 2^24, and floats that
are those integers times 2^-24), so the tolerance is zero everywhere.
All calls go through the C ABI via the binding.
"""
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
def dev(rm):
    return torch.device("cuda:0")


def st_np(t):
    return t.reshape(-1, 100).cpu().numpy().view(np.uint32)


def pos_of(row):
    return int(row[98]) | (int(row[99]) << 32)


def seeded(rm, seed, dev):
    return rm.seed(seed).to(dev)


# --------------------------------------------------------------------------
# Tiny: one stream, 10^6 outputs, u24 and f32; one jump of 10^6.
# --------------------------------------------------------------------------
def test_tiny_plain_u24_f32(rm, dev, orc):
    from paper_2512_00093_gb300.workloads import Tiny
    w = Tiny()
    x, c = orc.seeded_state(w.seed)
    ref, xa, ca = orc.generate(x, c, w.count)
    ref_f = orc.generate_alg1(x, c, w.count)           # Algorithm 1, double
    st = seeded(rm, w.seed, dev).clone()
    out = torch.empty(w.count, dtype=torch.int32, device=dev)
    rm.generate_plain_u24(st, w.count, out, write_back=True)
    st2 = seeded(rm, w.seed, dev).clone()
    outf = torch.empty(w.count, dtype=torch.float32, device=dev)
    rm.generate_plain_f32(st2, w.count, outf, write_back=False)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().view(np.uint32), ref)
    gf = outf.cpu().numpy()
    assert np.array_equal(gf.astype(np.float64), ref_f)  # f32 is exact: equals Alg. 1
    s = st_np(st)[0]
    assert np.array_equal(s[:97], xa) and s[97] == ca and pos_of(s) == w.count
    assert np.array_equal(st_np(st2)[0], st_np(seeded(rm, w.seed, dev))[0])  # no write-back


def test_tiny_desc_path_equals_plain(rm, dev, orc):
    from paper_2512_00093_gb300.workloads import Tiny
    w = Tiny()
    x, c = orc.seeded_state(w.seed)
    ref, _, _ = orc.generate(x, c, w.count)
    st = seeded(rm, w.seed, dev).reshape(1, 100).clone()
    out = torch.empty(w.count, dtype=torch.int32, device=dev)
    desc = rm.make_desc([0], [0], [w.count], 0, device=dev)
    rm.generate_u24(st, desc, out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().view(np.uint32), ref)


def test_tiny_jump_vs_brute_force(rm, dev, orc):
    from paper_2512_00093_gb300.workloads import Tiny
    w = Tiny()
    x, c = orc.seeded_state(w.seed)
    xb, cb = orc.brute_jump(x, c, w.jump)
    base = seeded(rm, w.seed, dev)
    out = rm.jump(base, rm.exps_tensor([w.jump], 1, device=dev))
    torch.cuda.synchronize()
    s = st_np(out)[0]
    assert np.array_equal(s[:97], xb) and s[97] == cb and pos_of(s) == w.jump


# --------------------------------------------------------------------------
# Jump: many exponents (edge cases, 0..160 bits), several bases.
# --------------------------------------------------------------------------
def test_jump_many_exponents(rm, dev, orc):
    from paper_2512_00093_gb300.workloads import random_exponents
    exps = random_exponents(100, 160, seed=3)       # not a multiple of 32 streams
    seeds = [12345, 1, 54217138]
    bases = torch.stack([seeded(rm, s, dev) for s in seeds])
    idx = torch.tensor([i % 3 for i in range(len(exps))], dtype=torch.int32, device=dev)
    out = rm.jump(bases, rm.exps_tensor(exps, 5, device=dev), base_idx=idx)
    torch.cuda.synchronize()
    got = st_np(out)
    for i, e in enumerate(exps):
        x, c = orc.seeded_state(seeds[i % 3])
        xr, cr = orc.jump(x, c, e)
        assert np.array_equal(got[i, :97], xr), (i, e)
        assert got[i, 97] == cr and pos_of(got[i]) == e % (1 << 64), (i, e)


def test_jump_small_exponents_vs_brute(rm, dev, orc):
    Js = list(range(0, 200)) + [1000, 4096, 10**5 + 3]
    base = seeded(rm, 777, dev)
    out = rm.jump(base, rm.exps_tensor(Js, 1, device=dev))
    torch.cuda.synchronize()
    got = st_np(out)
    x, c = orc.seeded_state(777)
    for i, J in enumerate(Js):
        xb, cb = orc.brute_jump(x, c, J)
        assert np.array_equal(got[i, :97], xb) and got[i, 97] == cb, J


def test_jump_composition_on_device(rm, dev, orc):
    """jump(jump(s, a), b) == jump(s, a + b) entirely on the GPU."""
    rng = np.random.default_rng(9)
    a = [int(rng.integers(1, 1 << 62)) << 60 for _ in range(40)]
    b = [int(rng.integers(1, 1 << 62)) << 30 for _ in range(40)]
    base = seeded(rm, 4242, dev)
    s_a = rm.jump(base, rm.exps_tensor(a, 5, device=dev))
    s_ab = rm.jump(s_a, rm.exps_tensor(b, 5, device=dev),
                   base_idx=torch.arange(40, dtype=torch.int32, device=dev))
    s_d = rm.jump(base, rm.exps_tensor([x + y for x, y in zip(a, b)], 5, device=dev))
    torch.cuda.synchronize()
    assert np.array_equal(st_np(s_ab)[:, :98], st_np(s_d)[:, :98])


def test_jump_bad_base_index_flags_status(rm, dev):
    base = seeded(rm, 5, dev)
    out = torch.full((3, 100), -7, dtype=torch.int32, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    idx = torch.tensor([0, 5, 0], dtype=torch.int32, device=dev)
    rm.jump(base, rm.exps_tensor([1, 2, 3], 1, device=dev), base_idx=idx, out=out, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) & rm.ST_BAD_INDEX
    assert (out[1] == -7).all()                   # skipped
    assert not (out[0] == -7).all() and not (out[2] == -7).all()


# --------------------------------------------------------------------------
# Generation: ragged counts, unaligned offsets, write-back and resume.
# --------------------------------------------------------------------------
RAGGED = [0, 1, 2, 31, 32, 33, 63, 64, 65, 95, 96, 97, 98, 127, 128, 129, 1000, 1013, 4096, 5000]


@pytest.mark.parametrize("f32", [False, True])
def test_generate_ragged_batch(rm, dev, orc, f32):
    n = len(RAGGED)
    exps = [(i * 7919) << 20 for i in range(n)]
    states = rm.jump(seeded(rm, 31337, dev), rm.exps_tensor(exps, 2, device=dev))
    offs = np.concatenate([[3], 3 + np.cumsum(RAGGED)[:-1] + np.arange(1, n)])  # gaps, unaligned
    total = int(offs[-1] + RAGGED[-1] + 5)
    dt = torch.float32 if f32 else torch.int32
    out = torch.full((total,), -1, dtype=dt, device=dev)
    desc = rm.make_desc(np.arange(n), offs, RAGGED, rm.DESC_WRITE_BACK, device=dev)
    before = st_np(states).copy()
    (rm.generate_f32 if f32 else rm.generate_u24)(states, desc, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    after = st_np(states)
    x0, c0 = orc.seeded_state(31337)
    for i, cnt in enumerate(RAGGED):
        xs, cs = orc.jump(x0, c0, exps[i])
        ref, xa, ca = orc.generate(xs, cs, cnt)
        g = got[offs[i]:offs[i] + cnt]
        if f32:
            assert np.array_equal(g, (ref.astype(np.float64) * F).astype(np.float32)), cnt
        else:
            assert np.array_equal(g.view(np.uint32), ref), cnt
        assert np.array_equal(after[i, :97], xa) and after[i, 97] == ca, cnt
        assert pos_of(after[i]) == pos_of(before[i]) + cnt
    # gaps untouched
    mask = np.ones(total, bool)
    for i, cnt in enumerate(RAGGED):
        mask[offs[i]:offs[i] + cnt] = False
    assert np.all(got[mask] == -1)


def test_resume_equals_one_call(rm, dev, orc):
    """generate(a) then generate(b) with write-back == generate(a + b)."""
    st = seeded(rm, 99, dev).reshape(1, 100).clone()
    parts = [37, 1, 96, 97, 500, 31, 4096 + 3]
    outs = []
    for p in parts:
        o = torch.empty(p, dtype=torch.int32, device=dev)
        rm.generate_u24(st, rm.make_desc([0], [0], [p], rm.DESC_WRITE_BACK, device=dev), o)
        outs.append(o)
    torch.cuda.synchronize()
    got = torch.cat(outs).cpu().numpy().view(np.uint32)
    x, c = orc.seeded_state(99)
    ref, _, _ = orc.generate(x, c, sum(parts))
    assert np.array_equal(got, ref)


def test_generate_status_bits(rm, dev):
    st = seeded(rm, 3, dev).reshape(1, 100).clone()
    out = torch.full((100,), -1, dtype=torch.int32, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    desc = rm.make_desc([0, 1, 0, 0], [0, 0, 90, 50], [10, 10, 11, 10], 0, device=dev)
    rm.generate_u24(st, desc, out, status)
    torch.cuda.synchronize()
    s = int(status.item())
    assert s & rm.ST_BAD_INDEX and s & rm.ST_OUT_RANGE
    got = out.cpu().numpy()
    assert np.all(got[:10] >= 0) and np.all(got[50:60] >= 0)
    assert np.all(got[10:50] == -1) and np.all(got[60:] == -1)


# --------------------------------------------------------------------------
# Full-size configurations, sampled against the oracle.
# --------------------------------------------------------------------------
def test_partitioned_full_size_sampled(rm, dev, orc):
    from paper_2512_00093_gb300.workloads import Partitioned
    w = Partitioned()
    base = seeded(rm, w.seed, dev)
    states = rm.partition(base, w.J, w.k0, w.n_streams)
    out = torch.empty((w.n_streams, w.count), dtype=torch.int32, device=dev)
    desc = rm.make_desc(np.arange(w.n_streams), np.arange(w.n_streams) * w.count, w.count,
                        rm.DESC_WRITE_BACK, device=dev)
    rm.generate_u24(states, desc, out)
    torch.cuda.synchronize()
    rows = w.verify_rows()
    got = out[torch.as_tensor(rows, device=dev)].cpu().numpy().view(np.uint32)
    for r, row in zip(rows, got):
        ref = orc.stream(w.seed, (w.k0 + int(r)) * w.J, w.count)
        assert np.array_equal(row, ref), int(r)
    # non-overlap structure: the write-back state of stream k advanced by
    # J - count more steps is the start state of stream k + 1
    after = rm.state_words_np(states)
    x0, c0 = orc.seeded_state(w.seed)
    for r in rows[:8]:
        xs, cs = orc.jump(x0, c0, (int(r)) * w.J + w.count)
        assert np.array_equal(after[r, :97], xs) and after[r, 97] == cs


def test_large_jumps_sampled(rm, dev, orc):
    from paper_2512_00093_gb300.workloads import LargeJumps
    w = LargeJumps()
    base = seeded(rm, w.seed, dev)
    states = rm.partition(base, w.J, 0, w.n_streams)
    out = torch.empty((w.n_streams, w.count), dtype=torch.int32, device=dev)
    desc = rm.make_desc(np.arange(w.n_streams), np.arange(w.n_streams) * w.count, w.count, 0,
                        device=dev)
    rm.generate_u24(states, desc, out)
    torch.cuda.synchronize()
    rng = np.random.default_rng(4)
    rows = np.concatenate([[0, 1, w.n_streams - 1], rng.choice(w.n_streams, 29, replace=False)])
    st = rm.state_words_np(states)
    x0, c0 = orc.seeded_state(w.seed)
    got = out.cpu().numpy().view(np.uint32)
    for r in rows:
        E = int(r) * w.J
        xr, cr = orc.jump(x0, c0, E)
        assert np.array_equal(st[r, :97], xr) and st[r, 97] == cr, int(r)
        ref, _, _ = orc.generate(xr, cr, w.count)
        assert np.array_equal(got[r], ref), int(r)


def test_device_seeding_matches_oracle(rm, dev, orc):
    rng = np.random.default_rng(17)
    seeds = np.concatenate([[1, 2, 12345, 54217138, 900000000, 30082, 30083],
                            rng.integers(1, 900000001, 300)]).astype(np.int32)
    out = rm.seed_batch(torch.as_tensor(seeds, device=dev))
    torch.cuda.synchronize()
    got = st_np(out)
    for i, sd in enumerate(seeds):
        x, c = orc.seeded_state(int(sd))
        assert np.array_equal(got[i, :97], x) and got[i, 97] == c and pos_of(got[i]) == 0, sd
    bad = torch.tensor([5, 0, -3, 900000001, 7], dtype=torch.int32, device=dev)
    o2 = torch.full((5, 100), -9, dtype=torch.int32, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    rm.seed_batch(bad, out=o2, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) & rm.ST_BAD_SEED
    assert (o2[1:4] == -9).all() and not (o2[0] == -9).all() and not (o2[4] == -9).all()


def test_generate_into_pinned_host_memory(rm, dev, orc):
    """Outputs stored straight into pinned host memory over the CPU-GPU link
    (ranmar_host_device_pointer) equal the device-memory outputs."""
    states = rm.partition(seeded(rm, 12345, dev), 1 << 40, 7, 64)
    count = 1000 + 7
    desc = rm.make_desc(np.arange(64), np.arange(64) * count, count, 0, device=dev)
    h = torch.full((64 * count,), -1, dtype=torch.int32).pin_memory()
    d = torch.empty(64 * count, dtype=torch.int32, device=dev)
    rm.generate_u24(states, desc, h)
    rm.generate_u24(states, desc, d)
    torch.cuda.synchronize()
    assert torch.equal(h, d.cpu())
    ref = orc.stream(12345, 9 * (1 << 40), count)
    assert np.array_equal(h[2 * count:3 * count].numpy().view(np.uint32), ref)


def test_injected_launch_failure(rm, dev):
    """ranmar_debug_fail_next makes the next launching call return its code
    once (RanmarError in the binding); the call after it succeeds."""
    st = rm.partition(seeded(rm, 3, dev), 1000, 0, 2)
    out = torch.empty(100, dtype=torch.int32, device=dev)
    desc = rm.make_desc(np.array([0]), np.array([0]), 100, 0, device=dev)
    rm.debug_fail_next(rm.binding.ECUDA)
    with pytest.raises(rm.RanmarError) as ei:
        rm.generate_u24(st, desc, out)
    assert ei.value.code == rm.binding.ECUDA
    rm.generate_u24(st, desc, out)
    torch.cuda.synchronize()

