"""CPU emulations of GPU schedules, checked against the oracle.

These tests replay, in numpy, the exact index arithmetic the kernels use, so
that a wrong offset, block order or fold step in the design fails on the CPU
(the GPU parity tests then check the kernels themselves):

* the warp-per-stream table jump (one warp per stream): the product of two
  polynomials mod phi = t^97 + t^64 - 1 over Z/2^24 (Sec. 3.1) with lane l
  forming coefficients 6l .. 6l+5 through a sliding window over a
  zero-padded copy of b, the fold in three blocks of distinct targets, and
  the application x P(A) (Sec. 3.1, the linear combination of the window)
  with lane l forming outputs 3l .. 3l+2;
* the lane-pair general product (table jump): 16 x 16 tiles along
  descending anti-diagonals, the pair's partial-sum exchange, the
  closed-form gather of the folded high half, and the ring application;
* the mirrored lane-pair square of the square-and-multiply: lane 0 forms
  the low half of x^2 from x, lane 1 the high half from x reversed (the
  same instructions), output-stationary over symmetric block triangles,
  then the gather, the shift by t on a 1 bit and both copies written;
* the tensor-core plan level: x' = x M mod 2^24 from balanced 8-bit limbs
  in fp16, with A = [A0 | A1 | A2 | 0] and B = [B2 | B1 | B0 | 0] along
  K = 320 (limb blocks of 104), D2 over all of K, D1 = A[0, 208) B[104, 312),
  D0 = A[0, 112) B[208, 320), each accumulator inside the range where fp32
  sums of integers are exact, and x' = D0 + 2^8 D1 + 2^16 D2 mod 2^24.
"""
import numpy as np

R, S = 97, 33
M32 = (1 << 32) - 1
MASK = (1 << 24) - 1


def u32(v):
    return int(v) & M32


# --- warp-per-stream jump --------------------------------------------------
def warp_mulmod(a, b):
    """a b mod phi as the warp kernel schedules it (arithmetic mod 2^32)."""
    a = [int(v) for v in a] + [0, 0, 0]          # a[97..99]: the row padding
    bz = [0] * 288                               # b_0 at 96, zeros either side
    for i in range(R):
        bz[96 + i] = int(b[i])
    c = [0] * 193
    for lane in range(32):
        n0 = 6 * lane
        win = [bz[96 + n0 + j] for j in range(6)]
        acc = [0] * 6
        for i in range(R):
            for j in range(6):
                acc[j] = u32(acc[j] + a[i] * win[j])
            if i + 1 < R:
                win = [bz[96 + n0 - i - 1]] + win[:5]
        for j in range(6):
            c[n0 + j] = acc[j]
    c[192] = u32(a[96] * int(b[96]))
    # fold blocks [160, 192], [127, 159], [97, 126]: all reads of a block
    # before its writes, targets distinct and below the block
    for hi, lo in ((192, 160), (159, 127), (126, 97)):
        ks = list(range(hi, lo - 1, -1))
        vals = {k: c[k] for k in ks}
        targets = [k - R for k in ks] + [k - S for k in ks]
        assert len(set(targets)) == len(targets) and max(targets) < lo
        for k in ks:
            c[k - R] = u32(c[k - R] + vals[k])
            c[k - S] = u32(c[k - S] - vals[k])
    return np.array([v & MASK for v in c[:R]], dtype=np.uint32)


def warp_apply(x, p):
    """New state words k = sum_i p_i X_{i+k} as the warp kernel schedules it."""
    X = [int(v) for v in x] + [0] * 96
    for r in range(3):
        q0 = R + S * r
        q1 = min(R + S * (r + 1), 2 * R - 1)
        src = [(X[q - R], X[q - S]) for q in range(q0, q1)]   # reads first
        assert all(q - S < q0 for q in range(q0, q1))
        for q, (u, v) in zip(range(q0, q1), src):
            X[q] = u32(u - v)
    p = [int(v) for v in p]
    out = [0] * R
    for lane in range(32):
        k0 = 3 * lane
        win = [X[k0 + j] for j in range(3)]
        acc = [0] * 3
        for i in range(R):
            for j in range(3):
                acc[j] = u32(acc[j] + p[i] * win[j])
            if i + 1 < R:
                win = win[1:] + [X[k0 + 3 + i]]
        for j in range(3):
            out[k0 + j] = acc[j]
    out[96] = u32(sum(p[i] * X[96 + i] for i in range(R)))
    return np.array([v & MASK for v in out], dtype=np.uint32)


def test_warp_product_schedule_matches_oracle(orc):
    rng = np.random.default_rng(5)
    cases = [(1, 1), (96, 1), (97, 0), (12345, 2**40), (2**64 + 7, 2**100 + 3)]
    cases += [(int(a), int(b)) for a, b in rng.integers(0, 2**62, (4, 2))]
    for ea, eb in cases:
        pa, pb = orc.poly_pow_t(ea), orc.poly_pow_t(eb)
        got = warp_mulmod(pa, pb)
        assert np.array_equal(got, orc.poly_mulmod(pa, pb)), (ea, eb)
        assert np.array_equal(got, orc.poly_pow_t(ea + eb)), (ea, eb)   # P_a P_b = P_{a+b}
    # dense random operands (not powers of t)
    for _ in range(3):
        a = rng.integers(0, 1 << 24, R, dtype=np.uint32)
        b = rng.integers(0, 1 << 24, R, dtype=np.uint32)
        assert np.array_equal(warp_mulmod(a, b), orc.poly_mulmod(a, b))


LEAD_BITS = 10


def mul_one_minus_t64(a, plant=0):
    """a (1 - t^64) mod phi as the kernels form it: t^64 a folded in closed
    form (t^97 = 1 - t^64): coefficient n of t^64 a is a_{n+33} - [n <= 30]
    a_{n+66} for n <= 63 and a_{n-64} - a_{n-31} + [n <= 94] a_{n+2} above."""
    b = []
    for n in range(R):
        if n <= 63:
            t64 = a[n + 33] - (a[n + 66] if n <= 30 and plant != 1 else 0)
        else:
            t64 = a[n - 64] - a[n - 31] + (a[n + 2] if n <= 94 and plant != 2 else 0)
        b.append(a[n] - t64)
    return b


def lead(e, bits=LEAD_BITS, plant=0):
    """The kernels' start: the leading (up to) ten bits v0 = 97 q + r of e,
    the bit below them (-1 when none), and t^v0 mod phi = t^r (1 - t^64)^q
    (exact integers, before any reduction mod 2^24)."""
    L = e.bit_length()
    v0, p = (e & ((1 << bits) - 1), -1) if L <= bits else ((e >> (L - bits)) & ((1 << bits) - 1),
                                                          L - bits - 1)
    q, r = divmod(v0, R)
    a = [0] * R
    a[r] = 1
    for _ in range(q):
        a = mul_one_minus_t64(a, plant)
    return v0, p, a


def warp_poly_power(e):
    """t^e mod phi as the warp square-and-multiply schedules it: the leading
    ten bits as t^r (1 - t^64)^q, then per bit a warp square and, on a 1 bit,
    the shift by t with the fold t^97 = 1 - t^64."""
    _, p, start = lead(e)
    a = np.array([v & MASK for v in start], dtype=np.uint32)
    while p >= 0:
        a = warp_mulmod(a, a.copy())
        if (e >> p) & 1:
            top = int(a[R - 1])
            v = [top] + [int(a[q - 1]) for q in range(1, R)]
            v[R - S] = u32(v[R - S] - top)
            a = np.array([x & MASK for x in v], dtype=np.uint32)
        p -= 1
    return a


def test_lead_start_matches_oracle(orc):
    # every start the kernels can take (v0 < 1024) against the oracle's t^v0
    for v0 in range(1 << LEAD_BITS):
        _, p, a = lead(v0)
        assert p == -1
        assert np.array_equal(np.array([v % (1 << 24) for v in a], dtype=np.uint32),
                              orc.poly_pow_t(v0)), v0
    assert lead((1 << 120) + 12345)[:2] == (512, 110)
    assert lead(1000)[:2] == (1000, -1)
    assert lead(5000)[:2] == (625, 2)
    # each dropped fold term (a_{n+66} below 31, a_{n+2} above 63) fails it
    for pl in (1, 2):
        assert any(np.any(np.array([v % (1 << 24) for v in lead(v0, plant=pl)[2]], dtype=np.uint32)
                          != orc.poly_pow_t(v0)) for v0 in range(1 << LEAD_BITS)), pl


def test_warp_square_multiply_schedule_matches_oracle(orc):
    for e in (0, 1, 63, 64, 65, 96, 97, 1000, 2**40 + 5, 2**64 - 1):
        assert np.array_equal(warp_poly_power(e), orc.poly_pow_t(e)), e


def test_warp_apply_schedule_matches_oracle(orc):
    x, c = orc.seeded_state(12345)
    for e in (0, 1, 33, 96, 97, 10**6, 2**40 + 5):
        p = orc.poly_pow_t(e)
        xe, _ = orc.jump(x, c, e)
        got = warp_apply(x, p)
        assert np.array_equal(got, xe), e
        assert np.array_equal(got, orc.apply_dot(x, p)), e


# --- lane-pair jump (two lanes per stream) ---------------------------------
W32 = 1 << 32


def gather_low(c, h, n):
    """Coefficient n < 97 after folding the high half (h_j = c_{97+j}): the
    closed form the pair kernel applies to a completed low block,
    a_n = c_n + h_n - h_{n+33} + h_{n+66} - h_{n-64} + h_{n-31} - h_{n+2}
    over the ranges in which each term exists."""
    v = c
    if n <= 95:
        v += h(n)
    if n <= 62:
        v -= h(n + 33)
    if n <= 29:
        v += h(n + 66)
    if n >= 64:
        v += h(n - 31) - h(n - 64)
        if n <= 93:
            v -= h(n + 2)
    return v


def pair_product(a_in, b_in):
    """a b mod phi in the pair kernel's order (the general product of the
    table jump): anti-diagonals s = I + J of 16 x 16 tiles walked from 10
    down to 0, lane g taking rows 8g .. 8g+7 of each tile, the pair
    exchanging partial sums, each completed block written at once: high
    blocks (with the rank-1 a_96 term) to a 128-word region, low blocks
    through the closed-form gather straight into a."""
    a = [int(v) for v in a_in] + [0] * 15
    b = [int(v) for v in b_in] + [0] * 15
    a96, b96 = a[96], b[96]
    reg = [0] * 128                               # reg[k - 96] = c_k
    reg[96] = (a96 * b96) % W32                   # c_192
    out_a = list(a)

    def h(j):
        return reg[j + 1]

    def complete(B, outs):
        for g in range(2):
            for jj in range(8):
                k = 16 * B + 8 * g + jj
                v = outs[g][jj]
                if B >= 6 and k <= 191:
                    i = k - 96
                    v += a96 * b[i] + b96 * a[i]
                v %= W32
                if B >= 6:
                    reg[k - 96] = v
                if B <= 6 and k <= 96:
                    out_a[k] = gather_low(v, h, k) % W32

    pend = [[0] * 8, [0] * 8]
    for s_ in range(10, -1, -1):
        acc = [[0] * 23, [0] * 23]
        ilo, ihi = max(0, s_ - 5), min(s_, 5)
        for g in range(2):
            for I, J in [(I, s_ - I) for I in range(ilo, ihi + 1)]:
                for p in range(8):
                    for q in range(16):
                        acc[g][p + q] += a[16 * I + 8 * g + p] * b[16 * J + q]
        recv = [[acc[1][8 + j] for j in range(8)], [acc[0][8 + j] for j in range(8)]]
        outs, newp = [[0] * 8, [0] * 8], [[0] * 8, [0] * 8]
        for g in range(2):
            for j in range(8):
                outs[g][j] = pend[g][j] + (acc[g][16 + j] if j <= 6 else 0) + \
                    (recv[g][j] if g == 0 else 0)
                newp[g][j] = acc[g][j] + (recv[g][j] if g == 1 else 0)
        pend = newp
        complete(s_ + 1, outs)
    complete(0, pend)
    return np.array([v % (1 << 24) for v in out_a[:R]], dtype=np.uint32)


def pair_apply(p, x):
    """x P(A) in the pair kernel's order: the window through a 128-word ring,
    output blocks of 16 as six 16 x 16 tiles plus the a_96 column, 32 new
    window words per round, output 96 as a plain dot product."""
    p = [int(v) for v in p] + [0] * 15
    ring = [0] * 128
    for q in range(R):
        ring[q] = int(x[q])
    for q in range(R, 128):
        ring[q] = (ring[q - R] - ring[q - S]) % W32
    out = [0] * R
    for m in range(3):
        for g in range(2):
            K = 2 * m + g
            acc = [0] * 16
            for I in range(6):
                for q in range(16):
                    for r in range(16):
                        acc[r] += p[16 * I + q] * ring[(16 * (I + K) + q + r) % 128]
            for r in range(16):
                acc[r] += p[96] * ring[(96 + 16 * K + r) % 128]
                out[16 * K + r] = acc[r] % (1 << 24)
        if m < 2:
            for q in range(32 * m + 128, 32 * m + 160):
                ring[q % 128] = (ring[(q - R) % 128] - ring[(q - S) % 128]) % W32
    x192 = (ring[(192 - R) % 128] - ring[(192 - S) % 128]) % W32
    out[96] = (sum(p[i] * ring[(96 + i) % 128] for i in range(96)) + p[96] * x192) % (1 << 24)
    return np.array(out, dtype=np.uint32)


def test_pair_schedule_matches_oracle(orc):
    rng = np.random.default_rng(11)
    for _ in range(3):
        a = rng.integers(0, 1 << 24, R).astype(np.uint32)
        b = rng.integers(0, 1 << 24, R).astype(np.uint32)
        assert np.array_equal(pair_product(a, b), orc.poly_mulmod(a, b))
        assert np.array_equal(pair_product(a, a), orc.poly_mulmod(a, a))
        x = rng.integers(0, 1 << 24, R).astype(np.uint32)
        assert np.array_equal(pair_apply(a, x), orc.apply_dot(x, a))


# --- tensor-core plan level ------------------------------------------------
LIMB_K, KTOT, NPAD = 104, 320, 112


def test_limb_values():
    for v, want in [(0x7F7F7F, [127] * 3), (0x7F7F80, [-128] * 3), (0, [0] * 3),
                    ((1 << 24) - 1, [-1, 0, 0]), (0x123456, None)]:
        l = [int(x[0]) for x in limbs(np.array([v]))]
        if want is not None:
            assert l == want, hex(v)
        assert (l[0] + 256 * l[1] + 65536 * l[2]) % (1 << 24) == v


def limbs(v):
    """Balanced 8-bit limbs l_0..l_2 of 24-bit words: the bytes of
    (v + 0x808080) mod 2^24, minus 128; v = sum 2^(8k) l_k mod 2^24."""
    w = (v.astype(np.int64) + 0x808080) & MASK
    return [((w >> (8 * k)) & 0xFF) - 128 for k in range(3)]


def plan_level_emulated(X, M):
    """x' = x M mod 2^24 (rows of X: source states; M: 97 x 97 words) through
    the K = 320 limb layout and the three accumulators."""
    n = X.shape[0]
    A = np.zeros((n, KTOT), np.int64)
    for k, l in enumerate(limbs(X)):              # A = [A0 | A1 | A2 | 0]
        A[:, LIMB_K * k: LIMB_K * k + R] = l
    B = np.zeros((KTOT, NPAD), np.int64)
    ml = limbs(M)                                 # B = [B2 | B1 | B0 | 0]
    for blk, k in enumerate((2, 1, 0)):
        B[LIMB_K * blk: LIMB_K * blk + R, :R] = ml[k]
    D2 = A @ B                                    # A0 B2 + A1 B1 + A2 B0
    D1 = A[:, :2 * LIMB_K] @ B[LIMB_K:3 * LIMB_K]  # A0 B1 + A1 B0
    D0 = A[:, :NPAD] @ B[2 * LIMB_K:]             # A0 B0
    # fp32 accumulation of these integer products is exact below 2^24
    assert np.abs(D2).max() < 2**23 and np.abs(D1).max() < 2**22 and np.abs(D0).max() < 2**22
    out = (D0 + (D1 << 8) + (D2 << 16)) & MASK
    return out[:, :R].astype(np.uint32)


def test_plan_limb_layout_matches_modular_product():
    rng = np.random.default_rng(9)
    X = rng.integers(0, 1 << 24, (37, R), dtype=np.int64)
    M = rng.integers(0, 1 << 24, (R, R), dtype=np.int64)
    X[0] = 0x7F7F7F                               # limbs (127, 127, 127)
    X[1] = 0x7F7F80                               # limbs (-128, -128, -128)
    X[2] = 0                                      # limbs (0, 0, 0)
    X[3] = MASK                                   # limbs (-1, 0, 0): -1 mod 2^24
    M[:, 0] = 0x7F7F80                            # with X[1]: every product +2^14,
    M[:, 1] = 0x7F7F7F                            # the accumulators' largest sums
    want = np.zeros((X.shape[0], R), np.int64)
    for j in range(R):                            # exact, then mod 2^24
        want[:, j] = (X * M[:, j]).sum(axis=1) & MASK
    assert np.array_equal(plan_level_emulated(X, M), want.astype(np.uint32))


def test_plan_limb_layout_is_the_jump(orc):
    """Rows of M_E = the unit states jumped by E: x M_E is x jumped by E."""
    E = 2**40 + 77
    M = np.stack([orc.jump(np.eye(R, dtype=np.uint32)[i], 0, E)[0] for i in range(R)])
    xs = [orc.seeded_state(s)[0] for s in (12345, 2, 54217138)]
    X = np.stack(xs).astype(np.int64)
    got = plan_level_emulated(X, M.astype(np.int64))
    for i, s in enumerate((12345, 2, 54217138)):
        x, c = orc.seeded_state(s)
        assert np.array_equal(got[i], orc.jump(x, c, E)[0])


# --- mirrored lane-pair square (symmetric triangles) ------------------------
def mirror_block_ops(m):
    """The 16 x 16 block terms that land in output block m (coefficients
    16m .. 16m+15) of x^2 for blocks X_0 .. X_5 of x: full blocks products
    X_I X_J (I < J) contribute their low triangle (p + q <= 15) when
    I + J = m and their high triangle (p + q >= 16) when I + J = m - 1; the
    square X_I^2 of one block contributes its cross terms p < q likewise."""
    low = [(I, m - I) for I in range(6) if I < m - I <= 5]
    high = [(I, m - 1 - I) for I in range(6) if I < m - 1 - I <= 5]
    low_sym = [m // 2] if m % 2 == 0 else []
    high_sym = [(m - 1) // 2] if m % 2 == 1 else []
    return low, high, low_sym, high_sym


def mirror_lane_block(X, m, plant=0):
    """One lane's output block m of x^2 (x = X_0 .. X_5, 96 coefficients) by
    16 x 16 block triangles: cross terms once, doubled, then the squares
    x_p^2 at the even outputs."""
    low, high, low_sym, high_sym = mirror_block_ops(m)
    acc = [0] * 16
    for I, J in low:
        for p in range(16):
            for q in range(16 - p):
                acc[p + q] += X[16 * I + p] * X[16 * J + q]
    for I, J in high:
        for p in range(1, 16):
            for q in range(16 - p, 16):
                acc[p + q - 16] += X[16 * I + p] * X[16 * J + q]
    for I in low_sym:
        for p in range(16):
            for q in range(p + 1, 16 - p):
                acc[p + q] += X[16 * I + p] * X[16 * I + q]
    hs_lo = 15 if plant == 1 else 16               # planted: a wrong triangle edge
    for I in high_sym:
        for p in range(16):
            for q in range(max(p + 1, hs_lo - p), 16):
                if p + q >= 16:
                    acc[p + q - 16] += X[16 * I + p] * X[16 * I + q]
                elif plant == 1:
                    acc[p + q] += X[16 * I + p] * X[16 * I + q]
    acc = [2 * v for v in acc]
    for r in range(0, 16, 2):
        acc[r] += X[8 * m + r // 2] ** 2
    return [v % W32 for v in acc]


def mirror_lane_block_chunks(X, m, plant=0):
    """The same block m as the kernel's loop forms it: m full chunks, each
    acc[r] += sum_{u<8} x_{8c+u} x_{16m+r-8c-u} (an 8 x 16 parallelogram of
    the product, i < j throughout), then the chunk at 8m, whose terms with
    i < j are u < r/2, then doubling and the squares x_{8m+r/2}^2 at even r."""
    acc = [0] * 16
    for c in range(m):
        w = X[16 * m - 8 * c - 8: 16 * m - 8 * c + 16]           # 24 words, w[k] = x_{base+k}
        for u in range(8):
            for r in range(16):
                acc[r] += X[8 * c + u] * w[r - u + 8 - (plant == 1)]
    t = X[8 * m: 8 * m + 16]
    for u in range(8):
        for r in range(2 * u + 1 + (plant == 2), 16):
            acc[r] += t[u] * t[r - u]
    acc = [2 * v for v in acc]
    for r in range(0, 16, 2):
        acc[r] += t[r // 2] ** 2
    return [v % W32 for v in acc]


def mirror_square(A, Bv, shift, plant=0):
    """x^2 t^shift mod phi as the mirrored pair schedules it.  A holds x
    (coefficients 0..96), Bv the same polynomial reversed (Bv[i] = x_{96-i}).
    Lane 0 forms c_0..c_95 of c = x^2 from A; lane 1 runs the same
    instructions on Bv, which gives the reversed top half c_192..c_97
    (written as Hr[k] = c_{192-k}); c_96 is split between the lanes.  The
    gather folds the top half in closed form, each lane's 8 outputs per
    block are rotated by one position for a 1 bit (the missing word from the
    partner by shuffle), t^97 = 1 - t^64 adds the old a_96 at 0 and
    subtracts it at 64, and both copies are written."""
    X = [list(map(int, A)), list(map(int, Bv))]
    C, Hr = [0] * 96, [0] * 96
    for g, dst in ((0, C), (1, Hr)):
        for m in range(6):
            blk = mirror_lane_block_chunks(X[g], m, plant)
            assert plant or blk == mirror_lane_block(X[g], m)
            dst[16 * m: 16 * m + 16] = blk
    part = [sum(X[g][24 * g + i] * X[g][96 - 24 * g - i] for i in range(24)) for g in (0, 1)]
    c96 = (2 * (part[0] + part[1]) + X[0][48] ** 2) % W32
    assert X[1][48] == X[0][48]

    def h(k):
        return Hr[95 - k]

    a96 = (c96 + h(65) - h(32)) % W32
    newA, newB = [0] * 100, [0] * 100
    prev7 = [0, 0]                                # lane 1's v[7] of the previous block
    v = [[0] * 8, [0] * 8]
    for kB in range(6):
        for g in (0, 1):
            for j in range(8):
                n = 16 * kB + 8 * g + j
                v[g][j] = gather_low(C[n], h, n) % W32
        recv = [prev7[1], v[0][7]]                # what each lane gets from its partner
        for g in (0, 1):
            for j in range(8):
                pos = 16 * kB + 8 * g + j
                w = (recv[g] if j == 0 else v[g][j - 1]) if shift else v[g][j]
                if shift and pos == 0:
                    w += a96
                if shift and pos == 64:
                    w -= a96
                newA[pos] = w % W32
                newB[96 - pos] = w % W32
        prev7 = [v[0][7], v[1][7]]
    w96 = prev7[1] if shift else a96
    newA[96] = newB[0] = w96
    return newA, newB


def mirror_poly_power(e, plant=0):
    _, p, start = lead(e)
    A, Bv = [0] * 100, [0] * 100
    for d, cf in enumerate(start):
        A[d] = cf % W32
        Bv[96 - d] = cf % W32
    while p >= 0:
        A, Bv = mirror_square(A, Bv, (e >> p) & 1, plant)
        p -= 1
    return np.array([v & MASK for v in A[:R]], dtype=np.uint32), Bv


def test_mirror_square_multiply_schedule_matches_oracle(orc):
    for e in (0, 1, 63, 64, 65, 96, 97, 127, 128, 1000, 2**40 + 5, (1 << 64) - 1,
              (1 << 120) + 12345):
        a, Bv = mirror_poly_power(e)
        assert np.array_equal(a, orc.poly_pow_t(e)), e
        assert [v & MASK for v in Bv[:R]] == [int(x) for x in a[::-1]], e


def test_mirror_square_dense_and_planted_edge(orc):
    rng = np.random.default_rng(13)
    t = np.zeros(R, np.uint32)
    t[1] = 1
    for _ in range(3):
        a = rng.integers(0, 1 << 24, R).astype(np.uint32)
        A = [int(v) for v in a] + [0, 0, 0]
        Bv = [int(v) for v in a[::-1]] + [0, 0, 0]
        sq = orc.poly_mulmod(a, a)
        for shift, want in ((0, sq), (1, orc.poly_mulmod(sq, t))):
            nA, nB = mirror_square(A, Bv, shift)
            assert [v & MASK for v in nA[:R]] == [int(x) for x in want]
            assert [v & MASK for v in nB[:R]] == [int(x) for x in want[::-1]]
        # the same schedule with the window of the full chunks one word off,
        # or with the i < j edge of the last chunk off by one
        for pl in (1, 2):
            bad, _ = mirror_square(A, Bv, 0, plant=pl)
            assert [v & MASK for v in bad[:R]] != [int(x) for x in sq]
    # the six blocks' terms add up to the symmetric count 97 * 98 / 2 - 1 - 48
    # (everything but c_96's 49 products), split evenly between the lanes
    n = 0
    for m in range(6):
        low, high, ls, hs = mirror_block_ops(m)
        n += 136 * len(low) + 120 * len(high) + 64 * len(ls) + 56 * len(hs) + 8
    assert 2 * n + 49 == 97 * 98 // 2


def mirror_apply(p, x, plant=0):
    """x P(A) as the four-worker application forms it: the window X(0..192)
    (the recurrence in three rounds, each reading only earlier rounds), worker
    t forming 8-output blocks t, t+4, t+8 from twelve chunks of 8 coefficients
    (each against two window octets) plus the p_96 term, and output 96 as four
    quarters (i = 24t .. 24t+23, and 96 by worker 3)."""
    P = [int(v) for v in p]
    W = [int(v) for v in x] + [0] * 96
    for lo, hi in ((97, 129), (130, 162), (163, 192)):
        for q in range(lo, hi + 1):
            assert q - S < lo                     # inputs from the rounds before
            W[q] = (W[q - R] - W[q - S]) % W32
    out = [0] * R
    for t in range(4):
        for B in (t, t + 4, t + 8):
            acc = [0] * 8
            for c in range(12):
                win = W[8 * (B + c): 8 * (B + c) + 16]
                for u in range(8):
                    for r in range(8):
                        acc[r] += P[8 * c + u] * win[r + u + (plant == 1)]
            for r in range(8):
                acc[r] += P[96] * W[8 * B + 96 + r]
            out[8 * B: 8 * B + 8] = [v % (1 << 24) for v in acc]
    parts = [sum(P[24 * t + i] * W[96 + 24 * t + i] for i in range(24)) for t in range(4)]
    parts[3] += P[96] * W[192]
    out[96] = sum(parts) % (1 << 24)
    return np.array(out, dtype=np.uint32)


def test_mirror_apply_schedule_matches_oracle(orc):
    x, c = orc.seeded_state(12345)
    rng = np.random.default_rng(19)
    for e in (0, 1, 96, 97, 10**6, 2**40 + 5, (1 << 120) + 12345):
        p = orc.poly_pow_t(e)
        assert np.array_equal(mirror_apply(p, x), orc.jump(x, c, e)[0]), e
    p = rng.integers(0, 1 << 24, R).astype(np.uint32)
    assert np.array_equal(mirror_apply(p, x), orc.apply_dot(x, p))
    assert not np.array_equal(mirror_apply(p, x, plant=1), orc.apply_dot(x, p))
