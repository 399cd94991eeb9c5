"""Pins for the oracle's general-lag jump (the concluding remarks: lagged
Fibonacci recurrences x_n = x_{n-r} - x_{n-s} mod 2^e of any order, jumped
by t^E mod phi_{r,s}, phi_{r,s} = t^r + t^{r-s} - 1, with the classical or
Karatsuba product).  Each pin compares with something independent of the
code under test: brute-force stepping of the recurrence, the RANMAR oracle
(pinned by the published check values) at r = 97, s = 33, e = 24, the
classical product against Karatsuba's, the composition law, and the
special cases t^E (E < r) and t^r = 1 - t^{r-s}."""
import numpy as np
import pytest

from oracle import Oracle

# (r, s, e): RANMAR's lags, Knuth's (55, 24) and (607, 273) and (1279, 418)
# lag pairs, and small or odd shapes.
LAGS = [(97, 33, 24), (55, 24, 32), (17, 5, 16), (607, 273, 24), (1279, 418, 32), (33, 32, 8),
        (2, 1, 24)]


def rand_window(rng, r, e):
    return rng.integers(0, 1 << e, r, dtype=np.uint64).astype(np.uint32)


def pin_lfg_brute(o):
    rng = np.random.default_rng(5)
    for r, s, e in LAGS:
        x = rand_window(rng, r, e)
        for E in sorted({0, 1, r - 1, r, r + 1, 2 * r + 7, int(rng.integers(1, 20000))}):
            for kara in (False, True):
                assert np.array_equal(o.lfg_jump(x, E, r, s, e, kara), o.lfg_step(x, r, s, e, E)), \
                    (r, s, e, E, kara)


def pin_lfg_ranmar(o):
    """At RANMAR's (97, 33, 24) the general jump is the x part of the RANMAR
    oracle's jump (its Algorithm 3 and Algorithm 2 pinned by James's values)."""
    for seed, E in [(12345, 10**6), (54217138, (1 << 120) + 12345), (7, (1 << 40) * 3)]:
        x, c = o.seeded_state(seed)
        xr, _ = o.jump(x, c, E)
        assert np.array_equal(o.lfg_jump(x, E, 97, 33, 24), xr)
        assert np.array_equal(o.lfg_jump(x, E, 97, 33, 24, karatsuba=True), xr)


def pin_lfg_karatsuba(o):
    rng = np.random.default_rng(9)
    for r, s, e in LAGS + [(1000, 333, 24), (129, 7, 20)]:
        for _ in range(2):
            a, b = rand_window(rng, r, e), rand_window(rng, r, e)
            assert np.array_equal(o.lfg_mulmod(a, b, r, s, e, False),
                                  o.lfg_mulmod(a, b, r, s, e, True)), (r, s, e)


def pin_lfg_special(o):
    for r, s, e in LAGS:
        for E in (0, 1, r // 2, r - 1):
            want = np.zeros(r, np.uint32)
            want[E] = 1
            assert np.array_equal(o.lfg_pow_t(E, r, s, e), want), (r, s, E)
        want = np.zeros(r, np.uint32)
        want[0] = 1
        want[r - s] = (1 << e) - 1 if e < 32 else 0xFFFFFFFF     # t^r = 1 - t^{r-s}
        assert np.array_equal(o.lfg_pow_t(r, r, s, e), want), (r, s)


def pin_lfg_composition(o):
    rng = np.random.default_rng(13)
    for r, s, e in [(55, 24, 32), (607, 273, 24)]:
        x = rand_window(rng, r, e)
        a, b = (1 << 100) + 3, (1 << 77) + 12345
        assert np.array_equal(o.lfg_jump(o.lfg_jump(x, a, r, s, e), b, r, s, e),
                              o.lfg_jump(x, a + b, r, s, e, karatsuba=True))


def pin_lfg_generate_ranmar(o):
    """At RANMAR's lags the generated words are Algorithm 2's LFG words: its
    outputs plus c_n mod 2^24 (Algorithm 2 outputs x_{96+n} - c_n)."""
    x, c = o.seeded_state(12345)
    words, after = o.lfg_generate(x, 97, 33, 24, 500)
    out, xa, _ = o.generate(x, c, 500)
    cs = np.array([o.c_step(c, n + 1) for n in range(500)], np.int64)
    assert np.array_equal((out.astype(np.int64) + cs) & 0xFFFFFF, words.astype(np.int64))
    assert np.array_equal(after, xa)


PINS = [pin_lfg_brute, pin_lfg_ranmar, pin_lfg_karatsuba, pin_lfg_special, pin_lfg_composition,
        pin_lfg_generate_ranmar]


@pytest.mark.parametrize("pin", PINS, ids=lambda f: f.__name__)
def test_lfg_pin(orc, pin):
    pin(orc)


MUTANTS = {12: "Karatsuba middle term without - a1 b1", 13: "general reduction sign"}


@pytest.mark.parametrize("mutant", sorted(MUTANTS), ids=lambda m: f"m{m}")
def test_lfg_pins_catch_mutant(mutant):
    o = Oracle(mutant)
    failed = []
    for pin in PINS:
        try:
            pin(o)
        except AssertionError:
            failed.append(pin.__name__)
    assert failed, f"no pin caught mutant {mutant}: {MUTANTS[mutant]}"
