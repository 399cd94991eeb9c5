"""Pins for the CPU oracle: facts fixed by the paper and by mathematics.

None of these re-types the oracle's own formula.  Each pin compares the
oracle with something independent of the code under test:
  * the published RANMAR check values (James 1990, cited by the paper);
  * Algorithm 1 (floating point) against Algorithm 2 (modular integer),
    which Sec. 4 states are equivalent;
  * the integer and floating forms of Algorithm 3 (Appendix A states they
    agree);
  * the polynomial jump against brute-force stepping of the recurrence;
  * Cayley-Hamilton on the companion matrix A built as printed in Sec. 3.1;
  * the composition law t^a t^b = t^(a+b) and f^a o f^b = f^(a+b);
  * the exact multiplicative order of t modulo phi over Z/2^24, which is
    (2^97 - 1) 2^23 (so the combined period is about 2^144, Sec. 2);
  * the closed form of c (Sec. 3.2) against stepping, and its period m.
A mutation test plants one known mistake at a time in the oracle (compile
switch ORC_MUTANT) and checks that some pin fails for each.
"""
import os
import random

import numpy as np
import pytest

from oracle import Oracle, R, M_C, D_C, C0
from oracle import matrix as omat

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

T_ORDER = ((1 << 97) - 1) << 23          # order of t mod phi over Z/2^24
Q97 = 13842607235828485645766393          # 2^97 - 1 = 11447 * Q97


def _read_golden(name):
    vals, meta = [], {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            if len(parts) == 2:
                meta[parts[0]] = int(parts[1])
            else:
                vals.append(int(parts[0]))
    return meta, vals


def tpow(e):
    b = np.zeros(R, np.uint32)
    b[e] = 1
    return b


# ----------------------------------------------------------------------------
# pins as plain functions, so the mutation test can run them on mutants
# ----------------------------------------------------------------------------
def pin_james(o):
    meta, vals = _read_golden("james1990_ranmar.txt")
    x, c = o.seeded_state(meta["seed"])
    out, _, _ = o.generate(x, c, meta["skip"] + len(vals))
    assert out[meta["skip"]:].tolist() == vals


def pin_seed_int_float(o):
    for seed in [1, 2, 12345, 54217138, 899999999, 900000000, 31415926]:
        ui = o.seed_int(seed)
        uf = o.seed_float(seed)
        assert np.all(ui < (1 << 24))
        assert np.array_equal(ui.astype(np.float64), uf * 16777216.0), seed


def pin_alg1_alg2(o, n=200_000, seeds=(12345, 1, 54217138, 777)):
    for seed in seeds:
        x, c = o.seeded_state(seed)
        u24, xa, ca = o.generate(x, c, n)
        f = o.generate_alg1(x, c, n)
        assert np.all((f >= 0.0) & (f < 1.0))
        assert np.array_equal(f, u24.astype(np.float64) / 16777216.0), seed


def pin_brute(o, Js=(0, 1, 2, 31, 32, 33, 64, 96, 97, 98, 193, 1000, 12345, 10**6)):
    x, c = o.seeded_state(12345)
    for J in Js:
        xj, cj = o.jump(x, c, J)
        xb, cb = o.brute_jump(x, c, J)
        assert np.array_equal(xj, xb), J
        assert cj == cb, J


def pin_special(o):
    assert np.array_equal(o.poly_pow_t(0), tpow(0))
    for J in [1, 2, 33, 64, 95, 96]:
        assert np.array_equal(o.poly_pow_t(J), tpow(J)), J
    p97 = tpow(0)
    p97[64] = (1 << 24) - 1              # t^97 = 1 - t^64 (phi = t^97 + t^64 - 1)
    assert np.array_equal(o.poly_pow_t(97), p97)


def pin_cayley_hamilton(o, Js=(0, 1, 5, 64, 96, 97, 98, 131, 149)):
    A = omat.companion()
    assert not omat.char_poly_check(A).any()
    P = np.eye(R, dtype=np.int64)
    x, c = o.seeded_state(54217138)
    done = 0
    for J in sorted(Js):
        while done < J:
            P = omat.matmul(P, A)
            done += 1
        b = o.poly_pow_t(J)
        assert np.array_equal(omat.poly_of_matrix(b, A), P), J
        # the jumped state is the row vector x times A^J
        xj, _ = o.jump(x, c, J)
        assert np.array_equal(omat.row_times(x, P).astype(np.uint32), xj), J


def pin_horner_dot(o):
    rng = np.random.default_rng(5)
    for _ in range(5):
        x = rng.integers(0, 1 << 24, R, dtype=np.uint32)
        b = rng.integers(0, 1 << 24, R, dtype=np.uint32)
        assert np.array_equal(o.apply_dot(x, b), o.apply_horner(x, b))


def pin_composition(o):
    rnd = random.Random(11)
    x, c = o.seeded_state(12345)
    for bits_a, bits_b in [(40, 57), (100, 90), (121, 134), (64, 64), (150, 10)]:
        a = rnd.getrandbits(bits_a) | (1 << (bits_a - 1))
        b = rnd.getrandbits(bits_b) | (1 << (bits_b - 1))
        pa, pb, pab = o.poly_pow_t(a), o.poly_pow_t(b), o.poly_pow_t(a + b)
        assert np.array_equal(o.poly_mulmod(pa, pb), pab), (a, b)
        xa, ca = o.jump(x, c, a)
        xab, cab = o.jump(xa, ca, b)
        xd, cd = o.jump(x, c, a + b)
        assert np.array_equal(xab, xd) and cab == cd, (a, b)


def pin_order(o):
    one = tpow(0)
    assert np.array_equal(o.poly_pow_t(T_ORDER), one)
    for p in (2, 11447, Q97):
        assert not np.array_equal(o.poly_pow_t(T_ORDER // p), one), p


def pin_large_jump_brute(o):
    """P_{2^120+12345} = P_{2^23+12345} since t^(2^120 - 2^23) = 1; the x part
    is then checked by 2^23 + 12345 brute-force steps, and the c part by
    (2^120 + 12345) mod m steps."""
    E = (1 << 120) + 12345
    assert E - T_ORDER == (1 << 23) + 12345
    x, c = o.seeded_state(12345)
    xj, cj = o.jump(x, c, E)
    xb, _ = o.brute_jump(x, c, (1 << 23) + 12345)
    assert np.array_equal(xj, xb)
    assert cj == o.c_step(c, E % M_C)


def pin_c_closed_form(o):
    for c in (C0, 0, M_C - 1, 5):
        for n in (0, 1, 2, 3, 100, 4097, 10**6):
            assert o.c_jump(c, n) == o.c_step(c, n), (c, n)
        assert o.c_step(c, M_C) == c                   # period divides m
        assert o.c_step(c, 1) != c
        huge = (1 << 134) + 987654321
        assert o.c_jump(c, huge) == o.c_step(c, huge % M_C)
        assert o.c_jump(c, M_C * 12345) == c


def pin_stream_blocks(o):
    """Stream k of (seed, J) is outputs kJ+1 .. kJ+count of one sequence."""
    J, K, cnt = 1000, 5, 300
    x, c = o.seeded_state(4242)
    whole, _, _ = o.generate(x, c, J * K + cnt)
    for k in range(K + 1):
        s = o.stream(4242, k * J, cnt)
        assert np.array_equal(s, whole[k * J:k * J + cnt]), k


def pin_first_step_is_F1(o):
    """The first Algorithm 2 step computes x_1 - x_65 (F1 in Sec. 3.1), and
    the state read back in sequence order is F1 applied to x."""
    x, c = o.seeded_state(2024)
    out, xa, ca = o.generate(x, c, 1)
    new = (int(x[0]) - int(x[64])) & 0xFFFFFF
    assert np.array_equal(xa[:-1], x[1:]) and int(xa[-1]) == new
    assert ca == (c - D_C) % M_C
    assert int(out[0]) == (new - ca) & 0xFFFFFF


def pin_jump_linear_brute(o):
    """The x part of f^E is linear over Z/2^24 (x' = x A^E, Sec. 3.1): by
    brute-force stepping alone, the jumped x of any state is the sum of the
    jumped unit states weighted by its words, mod 2^24.  (A jump of a block
    of states by one fixed E is therefore one matrix product.)"""
    rng = np.random.default_rng(17)
    for E in (1, 64, 150, 1000):
        M = np.zeros((R, R), np.uint64)
        for i in range(R):
            e = np.zeros(R, np.uint32)
            e[i] = 1
            M[i] = o.brute_jump(e, 0, E)[0]
        for _ in range(2):
            x = rng.integers(0, 1 << 24, R).astype(np.uint32)
            xb, _ = o.brute_jump(x, 5, E)
            xs = [int(v) for v in x]
            lin = [sum(xs[i] * int(M[i, w]) for i in range(R)) & 0xFFFFFF for w in range(R)]
            assert xb.tolist() == lin, E


PINS = [pin_james, pin_seed_int_float, pin_alg1_alg2, pin_brute, pin_special,
        pin_cayley_hamilton, pin_horner_dot, pin_composition, pin_order,
        pin_large_jump_brute, pin_c_closed_form, pin_stream_blocks,
        pin_first_step_is_F1, pin_jump_linear_brute]


@pytest.mark.parametrize("pin", PINS, ids=lambda f: f.__name__)
def test_pin(orc, pin):
    pin(orc)


def test_seed_domain(orc):
    for bad in (0, -1, 900000001, -2147483648):
        with pytest.raises(ValueError):
            orc.seeded_state(bad)


def test_brute_force_to_1e7(orc):
    """Jumps up to 10^7 agree with brute-force stepping."""
    x, c = orc.seeded_state(12345)
    rnd = random.Random(3)
    for J in [10**7, rnd.randrange(10**6, 10**7), rnd.randrange(10**5, 10**6)]:
        xj, cj = orc.jump(x, c, J)
        xb, cb = orc.brute_jump(x, c, J)
        assert np.array_equal(xj, xb) and cj == cb, J


def test_radix_blocks_by_jump_matrices(orc):
    """Stream k + rR of (seed, J) = stream k times the matrix of the jump by
    rRJ (rows: unit states jumped by the oracle's polynomial method); the
    composition the GPU partition plan uses level by level."""
    J = 1 << 40
    x0, c0 = orc.seeded_state(12345)
    for r, Rr, k in [(1, 16, 777), (15, 16, 0), (3, 256, 5)]:
        E = r * Rr * J
        M = np.zeros((R, R), np.uint64)
        for i in range(R):
            e = np.zeros(R, np.uint32)
            e[i] = 1
            M[i] = orc.jump(e, 0, E)[0]
        xs, cs = orc.jump(x0, c0, k * J)
        xd, cd = orc.jump(x0, c0, (k + r * Rr) * J)
        v = [int(a) for a in xs]
        lin = [sum(v[i] * int(M[i, w]) for i in range(R)) & 0xFFFFFF for w in range(R)]
        assert xd.tolist() == lin
        assert cd == orc.c_jump(cs, E)


def test_regression_values(orc):
    """Values the oracle produced when first pinned (regenerated by
    tests/golden/make_regression.py); guards against later drift."""
    meta, vals = _read_golden("regression_seed12345.txt")
    x, c = orc.seeded_state(12345)
    out, _, _ = orc.generate(x, c, 8)
    assert out.tolist() == vals[:8]
    xj, cj = orc.jump(x, c, meta["jump"])
    assert int(xj.astype(np.uint64).sum()) == meta["xsum"] and cj == meta["cjump"]


# Mutants planted in oracle/ranmar_oracle.c under ORC_MUTANT=n.
MUTANTS = {
    1: "reduction sign of the t^(k-33) term",
    2: "reduction lag 32 instead of 33",
    3: "Algorithm 3 with the printed Quotient",
    4: "Algorithm 2 adds d instead of m - d",
    5: "application with a reversed coefficient index",
    6: "exponent bits scanned in the wrong order",
    7: "c jump with the wrong sign",
    8: "top exponent word dropped",
    9: "Algorithm 3 integer conversion shift 7",
    11: "Horner with the coefficients in the wrong order",
}


@pytest.mark.parametrize("mutant", sorted(MUTANTS), ids=lambda m: f"m{m}")
def test_pins_catch_mutant(mutant):
    o = Oracle(mutant)
    failed = []
    for pin in PINS:
        try:
            pin(o)
        except AssertionError:
            failed.append(pin.__name__)
    assert failed, f"no pin caught mutant {mutant}: {MUTANTS[mutant]}"
