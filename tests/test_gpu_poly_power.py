"""GPU parity of ranmar_poly_power (Sec. 3.1, the polynomial part of a jump,
what the paper's Table 2 times): t^E mod (t^97 + t^64 - 1) over Z/2^24 equals
the oracle's for edge and random exponents up to 2^160 - 1, bit for bit."""
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


def test_poly_power_matches_oracle(rm, orc):
    from paper_2512_00093_gb300.workloads import random_exponents
    dev = torch.device("cuda:0")
    edge = [0, 1, 2, 63, 64, 96, 97, 98, 193, (1 << 64) - 1, (1 << 120) - 1,
            ((1 << 97) - 1) << 23, (1 << 159) + 3, (1 << 160) - 1]
    exps = edge + random_exponents(45, 160, seed=8)
    got = rm.poly_power(rm.exps_tensor(exps, 5, device=dev))
    torch.cuda.synchronize()
    g = got.cpu().numpy().view(np.uint32)
    assert not g[:, 97:].any()
    for i, e in enumerate(exps):
        assert np.array_equal(g[i, :97], orc.poly_pow_t(e)), (i, e)


def test_poly_power_is_the_jumps_polynomial(rm, orc):
    """x P_E(A) from the returned coefficients is the jumped state."""
    dev = torch.device("cuda:0")
    exps = [5, 10**6, (1 << 64) - 1, (1 << 120) + 12345]
    p = rm.poly_power(rm.exps_tensor(exps, 5, device=dev)).cpu().numpy().view(np.uint32)
    x, c = orc.seeded_state(12345)
    for i, e in enumerate(exps):
        assert np.array_equal(orc.apply_dot(x, p[i, :97]), orc.jump(x, c, e)[0])


def test_poly_power_ragged_batch_and_errors(rm, orc):
    dev = torch.device("cuda:0")
    for n in (1, 15, 16, 17, 33):
        exps = [(1 << 64) - 1 - i for i in range(n)]
        got = rm.poly_power(rm.exps_tensor(exps, 3, device=dev)).cpu().numpy().view(np.uint32)
        for i in {0, n - 1}:
            assert np.array_equal(got[i, :97], orc.poly_pow_t(exps[i]))
    with pytest.raises(rm.RanmarError):
        rm.poly_power(torch.zeros((2, 6), dtype=torch.int32, device=dev))   # 6 words


def test_poly_power_warp_and_pair_mappings_agree(rm):
    """Batches up to SQUARE_WARP_AUTO_MAX take a warp per exponent, larger ones
    two lanes: the same exponents through both give the same polynomials."""
    from paper_2512_00093_gb300.workloads import random_exponents
    dev = torch.device("cuda:0")
    n = rm.SQUARE_WARP_AUTO_MAX + 1
    exps = random_exponents(n, 134, seed=12)
    ex = rm.exps_tensor(exps, 5, device=dev)
    pair = rm.poly_power(ex)                     # n > the switch: two lanes each
    warp = rm.poly_power(ex[: n - 1])            # the first n - 1: a warp each
    torch.cuda.synchronize()
    assert torch.equal(pair[: n - 1], warp)


def test_square_multiply_jump_warp_and_pair_agree(rm):
    dev = torch.device("cuda:0")
    base = rm.seed(77).to(dev)
    n = rm.SQUARE_WARP_AUTO_MAX + 1
    for J, flags in [((1 << 120) + 12345, 0), ((1 << 64) - 1, rm.JUMP_REDUCE_PERIOD)]:
        pair = rm.partition_ex(base, J, 3, n, flags=flags)          # square-and-multiply
        warp = rm.partition_ex(base, J, 3, n - 1, flags=flags)
        torch.cuda.synchronize()
        assert torch.equal(pair[: n - 1], warp), (J, flags)


def test_poly_power_every_ten_bit_start(rm, orc):
    """Both kernels start from the leading ten bits v0 = 97 q + r of E as
    t^r (1 - t^64)^q mod phi.  Every E < 1,024 (the start alone, no
    squaring) and, for every v0, an exponent v0 2^40 + tail (the start
    followed by 40 squarings), through the warp mapping (1,024 exponents)
    and the lane pairs (all 2,048 at once, so that a CTA's 16 streams mix
    different q and, for the small ones, different bit lengths)."""
    dev = torch.device("cuda:0")
    small = list(range(1024))
    large = [(v << 40) + (v * 2654435761) % (1 << 40) for v in range(1024)]
    want = {e: orc.poly_pow_t(e) for e in small + large}
    assert len(small) <= rm.SQUARE_WARP_AUTO_MAX < len(small) + len(large)
    for exps in (small, large, small + large):
        got = rm.poly_power(rm.exps_tensor(exps, 2, device=dev)).cpu().numpy().view(np.uint32)
        for i, e in enumerate(exps):
            assert np.array_equal(got[i, :97], want[e]), (len(exps), e)
