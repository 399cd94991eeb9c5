"""GPU parity of the general-lag jump and generation (lagged Fibonacci
recurrences x_n = x_{n-r} - x_{n-s} mod 2^e, the concluding remarks): every
jumped window and every generated word equals the oracle's, bit for bit,
with the classical and the Karatsuba squaring.  Tolerance 0."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

# r <= 128 with the classical squaring runs a warp per stream, above a CTA
# per stream: (128, 100, 32) and (129, 5, 24) sit on either side
LAGS = [(97, 33, 24), (55, 24, 32), (17, 5, 16), (607, 273, 24), (1279, 418, 32), (33, 32, 8),
        (2, 1, 24), (2048, 1029, 24), (128, 100, 32), (129, 5, 24)]


@pytest.fixture(scope="module")
def rm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_00093_gb300 as rm
    return rm


def windows(rng, k, r, e):
    return rng.integers(0, 1 << e, (k, r), dtype=np.uint64).astype(np.uint32)


@pytest.mark.parametrize("r,s,e", LAGS)
def test_lfg_jump_matches_oracle(rm, orc, r, s, e):
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(r * 131 + s)
    base = windows(rng, 3, r, e)
    exps = [0, 1, r - 1, r, r + 1, 2 * r + 5, 12345, (1 << 40) + 7, (1 << 64) - 1,
            (1 << 120) + 12345, (1 << 159) + 3]
    if r > 1000:
        exps = exps[:1] + exps[3:8]   # keep the CPU oracle's time bounded
    ex = rm.exps_tensor(exps, 5, device=dev)
    idx = torch.tensor([i % 3 for i in range(len(exps))], dtype=torch.int32, device=dev)
    xb = torch.as_tensor(base.view(np.int32), device=dev)
    methods = [rm.LFG_CLASSICAL, rm.LFG_KARATSUBA]
    methods += [rm.LFG_KARATSUBA_LEVELS(L) for L in range(1, 7)
                if (r + (1 << L) - 1) >> L >= 8 and L <= 4 + (r > 1000)]
    for method in methods:
        try:
            got = rm.lfg_jump(r, s, e, xb, ex, base_idx=idx, method=method)
        except rm.RanmarError:
            assert method >= 16   # an explicit depth that does not fit
            continue
        torch.cuda.synchronize()
        g = got.cpu().numpy().view(np.uint32)
        for i, E in enumerate(exps):
            want = orc.lfg_jump(base[i % 3], E, r, s, e, karatsuba=True)
            assert np.array_equal(g[i], want), (r, s, e, E, method)


def test_lfg_karatsuba_levels(rm):
    # the automatic depth: classical below r = 512, 1 level below 1024, else 2
    assert rm.lfg_karatsuba_levels(97, 33, 24) == 0
    assert rm.lfg_karatsuba_levels(17, 5, 16) == 0
    assert rm.lfg_karatsuba_levels(607, 273, 24) == 1
    assert rm.lfg_karatsuba_levels(1279, 418, 32) == 2
    assert rm.lfg_karatsuba_levels(1279, 418, 32, rm.LFG_CLASSICAL) == 0
    assert rm.lfg_karatsuba_levels(1279, 418, 32, rm.LFG_KARATSUBA_LEVELS(5)) == 5
    with pytest.raises(rm.RanmarError):
        rm.lfg_karatsuba_levels(17, 5, 16, rm.LFG_KARATSUBA_LEVELS(3))   # leaves of 3
    with pytest.raises(rm.RanmarError):
        rm.lfg_karatsuba_levels(97, 97, 24)
    with pytest.raises(rm.RanmarError):
        rm.lfg_karatsuba_levels(4096, 33, 24)


@pytest.mark.parametrize("r,s,e", [(97, 33, 24), (55, 24, 32), (33, 32, 8), (17, 5, 16),
                                   (1279, 418, 32), (2, 1, 24)])
def test_lfg_generate_matches_oracle(rm, orc, r, s, e):
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(7 + r)
    base = windows(rng, 37, r, e)
    count = 3 * 32 + 7 + r
    x = torch.as_tensor(base.view(np.int32).copy(), device=dev)
    out = rm.lfg_generate(r, s, e, x, count)
    torch.cuda.synchronize()
    o = out.cpu().numpy().view(np.uint32)
    xa = x.cpu().numpy().view(np.uint32)
    for i in range(37):
        words, after = orc.lfg_generate(base[i], r, s, e, count)
        assert np.array_equal(o[i], words), (r, s, i)
        assert np.array_equal(xa[i], after), (r, s, i)


def test_lfg_jump_then_generate_is_the_sequence(rm, orc):
    """Jump by E then generate = the words E .. E + count of one sequence."""
    dev = torch.device("cuda:0")
    r, s, e = 607, 273, 24
    rng = np.random.default_rng(99)
    base = windows(rng, 1, r, e)
    E, count = 5000, 700
    ex = rm.exps_tensor([E], 2, device=dev)
    x = rm.lfg_jump(r, s, e, torch.as_tensor(base.view(np.int32), device=dev), ex)
    out = rm.lfg_generate(r, s, e, x, count)
    torch.cuda.synchronize()
    words, _ = orc.lfg_generate(base[0], r, s, e, E + count)
    assert np.array_equal(out.cpu().numpy().view(np.uint32)[0], words[E:])


def test_lfg_host_errors(rm):
    dev = torch.device("cuda:0")
    x = torch.zeros((1, 4096), dtype=torch.int32, device=dev)
    ex = torch.zeros((1, 1), dtype=torch.int32, device=dev)
    for bad in [(97, 0, 24), (97, 97, 24), (1, 1, 24), (97, 33, 0), (97, 33, 33), (4096, 33, 24)]:
        r = bad[0]
        with pytest.raises(rm.RanmarError):
            rm.lfg_jump(*bad, x.view(-1)[: 4096 // r * r], ex)
    with pytest.raises(rm.RanmarError):
        rm.lfg_jump(97, 33, 24, x.view(-1)[:97], ex, method=5)
