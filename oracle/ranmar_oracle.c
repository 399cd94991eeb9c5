/*
 * ranmar_oracle.c -- plain, slow, obviously-correct CPU reference for the
 * RANMAR generator of Haramoto & Suzuki, "Making the RANMAR pseudorandom
 * number generator in LAMMPS up to four times faster, with an implementation
 * of jump-ahead" (arXiv 2512.00093).
 *
 * THIS IS TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant with the CUDA library; the library never calls it.
 *
 * Every routine follows one passage of the paper, in its order and notation:
 *   - Algorithm 3 (Appendix A): seeding, integer form; plus the floating
 *     accumulator form it is stated to reproduce.
 *   - Algorithm 1 (Sec. 4): the floating-point generator used by LAMMPS.
 *   - Algorithm 2 (Sec. 4): the 24-bit modular-integer generator.
 *   - Sec. 2: the automaton f = (f1, f2); Sec. 3.1: F1, the companion matrix A,
 *     phi(t) = t^97 + t^64 - 1, t^J mod phi, Cayley-Hamilton, Horner.
 *   - Sec. 3.2: c_J = (c'_0 - J d') mod m.
 * Residues mod 2^24 are kept in uint32_t and reduced by masking (Sec. 4: w-bit
 * unsigned arithmetic wraps mod 2^w, and (u - v) mod 2^e depends only on
 * u, v mod 2^e).
 *
 * Readings of the paper that this file takes (each is listed with its reason
 * in the design notes):
 *   R1  Algorithm 3's update of m reads Remainder(Remainder(i*j,179)*k,179)
 *       (the Marsaglia-Zaman procedure the appendix says it reproduces); the
 *       printed "Quotient" is taken as a typo.
 *   R2  Seeds are 1 <= s <= 900000000 (s = 0 would make s - 1 negative).
 *   R3  Sequence order of the state: after seeding with i = 97, j = 33 the
 *       oldest word is u[97]; x_1..x_97 = u[97], u[96], ..., u[1].  In
 *       general x_oldest = u[i], then u[i-1], wrapping 1 -> 97.
 *   R4  The c carried in the state is the value after the last transition:
 *       output n uses c_n = (c_0 - n d) mod m with c_0 = 362436 as seeded.
 *   R5  "mod m" is the non-negative residue.
 *
 * Compile-time switch ORC_MUTANT=n plants one known mistake (tests only use
 * it to show that the pins catch each one); the default build has none.
 */
#include <stdint.h>
#include <string.h>
#include <stdlib.h>

#ifndef ORC_MUTANT
#define ORC_MUTANT 0
#endif

/* Parameters (Sec. 2): (r, s) = (97, 33); M = 2^24; m = 2^24 - 3;
 * d' = 7654321; c'_0 = 362436 (Algorithm 3, last lines). */
enum { ORC_R = 97, ORC_S = 33 };
static const uint32_t ORC_MASK = 0x00FFFFFFu;     /* 2^24 - 1 */
static const uint32_t ORC_m = 16777213u;          /* 2^24 - 3 */
static const uint32_t ORC_d = 7654321u;
static const uint32_t ORC_c0 = 362436u;

/* ------------------------------------------------------------------------ */
/* Algorithm 3 (Appendix A): seed -> u_1..u_97, integer form with w = 32.    */
/* u[ii-1] receives u_ii.  Returns 0, or -1 for a seed outside R2.           */
/* ------------------------------------------------------------------------ */
int orc_seed_int(int32_t seed, uint32_t *u)
{
    if (seed < 1 || seed > 900000000) return -1;
    int32_t ij = (seed - 1) / 30082;
    int32_t kl = (seed - 1) - 30082 * ij;
    int32_t i = (ij / 177) % 177 + 2;
    int32_t j = ij % 177 + 2;
    int32_t k = (kl / 169) % 178 + 1;
    int32_t l = kl % 169;
    for (int ii = 1; ii <= 97; ii++) {
        uint32_t s = 0;
        uint32_t t = 0x80000000u;               /* 2^(w-1): "0.5" */
        for (int jj = 1; jj <= 24; jj++) {
#if ORC_MUTANT == 3
            int32_t m = (((i * j) / 179) * k) % 179;   /* printed Quotient */
#else
            int32_t m = (((i * j) % 179) * k) % 179;   /* reading R1 */
#endif
            i = j;
            j = k;
            k = m;
            l = (53 * l + 1) % 169;
            if ((l * m) % 64 >= 32) s += t;
            t /= 2;
        }
#if ORC_MUTANT == 9
        u[ii - 1] = s >> 7;
#else
        u[ii - 1] = s >> 8;                     /* Quotient(s, 2^(w-24)) */
#endif
    }
    return 0;
}

/* The same procedure with a floating accumulator: t starts at 0.5 and is
 * halved, s accumulates t (the form LAMMPS uses and Algorithm 3 restates). */
int orc_seed_float(int32_t seed, double *u)
{
    if (seed < 1 || seed > 900000000) return -1;
    int32_t ij = (seed - 1) / 30082;
    int32_t kl = (seed - 1) - 30082 * ij;
    int32_t i = (ij / 177) % 177 + 2;
    int32_t j = ij % 177 + 2;
    int32_t k = (kl / 169) % 178 + 1;
    int32_t l = kl % 169;
    for (int ii = 1; ii <= 97; ii++) {
        double s = 0.0, t = 0.5;
        for (int jj = 1; jj <= 24; jj++) {
            int32_t m = (((i * j) % 179) * k) % 179;
            i = j;
            j = k;
            k = m;
            l = (53 * l + 1) % 169;
            if ((l * m) % 64 >= 32) s = s + t;
            t = 0.5 * t;
        }
        u[ii - 1] = s;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 (Sec. 4): LAMMPS floating-point RANMAR, in double.           */
/* u[0..96] holds u_1..u_97; *i, *j are the 1-based ring indices; *c is the  */
/* arithmetic-sequence value in [0, m/M).  Writes n outputs y in [0, 1).     */
/* ------------------------------------------------------------------------ */
void orc_alg1(double *u, int32_t *pi, int32_t *pj, double *pc, uint64_t n,
              double *out)
{
    const double cd = 7654321.0 / 16777216.0;
    const double cm = 16777213.0 / 16777216.0;
    int32_t i = *pi, j = *pj;
    double c = *pc;
    for (uint64_t t = 0; t < n; t++) {
        double y = u[i - 1] - u[j - 1];
        if (y < 0.0) y = y + 1.0;
        u[i - 1] = y;
        i = i - 1;
        if (i == 0) i = 97;
        j = j - 1;
        if (j == 0) j = 97;
        c = c - cd;
        if (c < 0.0) c = c + cm;
        y = y - c;
        if (y < 0.0) y = y + 1.0;
        out[t] = y;
    }
    *pi = i;
    *pj = j;
    *pc = c;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 2 (Sec. 4): the modular-integer form.  Same layout as above,    */
/* v is the numerator c' in [0, m).  out may be NULL (stepping only).       */
/* Outputs are the 24-bit integers (u - v) mod 2^24; y = out * 2^-24.        */
/* ------------------------------------------------------------------------ */
void orc_alg2(uint32_t *u, int32_t *pi, int32_t *pj, uint32_t *pv, uint64_t n,
              uint32_t *out)
{
    int32_t i = *pi, j = *pj;
    uint32_t v = *pv;
    for (uint64_t t = 0; t < n; t++) {
        uint32_t w = u[i - 1] - u[j - 1];      /* wraps mod 2^32 */
        u[i - 1] = w;
        i = i - 1;
        if (i == 0) i = 97;
        j = j - 1;
        if (j == 0) j = 97;
#if ORC_MUTANT == 4
        v = v + ORC_d;
#else
        v = v + (ORC_m - ORC_d);
#endif
        if (v >= ORC_m) v = v - ORC_m;
        if (out) out[t] = (w - v) & ORC_MASK;
    }
    *pi = i;
    *pj = j;
    *pv = v;
}

/* ------------------------------------------------------------------------ */
/* Reading R3: LAMMPS ring (u_1..u_97, i) <-> sequence order x_1..x_97.      */
/* ------------------------------------------------------------------------ */
void orc_lammps_to_seq(const uint32_t *u, int32_t i, uint32_t *x)
{
    int32_t p = i;
    for (int q = 0; q < ORC_R; q++) {
        x[q] = u[p - 1] & ORC_MASK;
        p = p - 1;
        if (p == 0) p = 97;
    }
}

/* x_1..x_97 -> u[98-q] = x_q, with i = 97 and j = 33 (j = i - 64 mod 97). */
void orc_seq_to_lammps(const uint32_t *x, uint32_t *u, int32_t *pi, int32_t *pj)
{
    for (int q = 1; q <= ORC_R; q++) u[(98 - q) - 1] = x[q - 1] & ORC_MASK;
    *pi = 97;
    *pj = 33;
}

/* Seeded state in sequence order: x_1..x_97 and c'_0 (Algorithm 3). */
int orc_seeded_state(int32_t seed, uint32_t *x, uint32_t *c)
{
    uint32_t u[ORC_R];
    if (orc_seed_int(seed, u) != 0) return -1;
    orc_lammps_to_seq(u, 97, x);
    *c = ORC_c0;
    return 0;
}

/* Generate n outputs (24-bit) from a sequence-order state by Algorithm 2.
 * x_after / c_after (may be NULL) receive the advanced state. */
void orc_generate(const uint32_t *x, uint32_t c, uint64_t n, uint32_t *out,
                  uint32_t *x_after, uint32_t *c_after)
{
    uint32_t u[ORC_R];
    int32_t i, j;
    uint32_t v = c;
    orc_seq_to_lammps(x, u, &i, &j);
    orc_alg2(u, &i, &j, &v, n, out);
    if (x_after) orc_lammps_to_seq(u, i, x_after);
    if (c_after) *c_after = v;
}

/* Same stream through Algorithm 1 in double, the state mapped by the
 * isomorphism sigma^{-1} (Sec. 3.1): u_i = x * 2^-24, c = c' * 2^-24. */
void orc_generate_alg1(const uint32_t *x, uint32_t c, uint64_t n, double *out)
{
    uint32_t ui[ORC_R];
    double u[ORC_R];
    int32_t i, j;
    orc_seq_to_lammps(x, ui, &i, &j);
    for (int q = 0; q < ORC_R; q++) u[q] = (double)ui[q] / 16777216.0;
    double cc = (double)c / 16777216.0;
    orc_alg1(u, &i, &j, &cc, n, out);
}

/* Brute-force jump: J transitions of f (Sec. 2) by stepping Algorithm 2. */
void orc_brute_jump(uint32_t *x, uint32_t *c, uint64_t J)
{
    orc_generate(x, *c, J, NULL, x, c);
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.1: polynomials over Z/2^24 of degree < 97, reduced mod             */
/* phi(t) = t^97 + t^64 - 1, i.e. t^97 = 1 - t^64.                           */
/* ------------------------------------------------------------------------ */
void orc_poly_mulmod(const uint32_t *a, const uint32_t *b, uint32_t *out)
{
    uint32_t prod[2 * ORC_R - 1];
    memset(prod, 0, sizeof(prod));
    for (int i = 0; i < ORC_R; i++)
        for (int j = 0; j < ORC_R; j++) prod[i + j] += a[i] * b[j];
    /* Reduce from the top: t^k = t^(k-97) t^97 = t^(k-97) - t^(k-33). */
    for (int k = 2 * ORC_R - 2; k >= ORC_R; k--) {
        uint32_t h = prod[k];
        prod[k] = 0;
        prod[k - ORC_R] += h;
#if ORC_MUTANT == 1
        prod[k - (ORC_R - 64)] += h;
#elif ORC_MUTANT == 2
        prod[k - (ORC_R - 65)] -= h;
#else
        prod[k - (ORC_R - 64)] -= h;           /* k - 33 */
#endif
    }
    for (int i = 0; i < ORC_R; i++) out[i] = prod[i] & ORC_MASK;
}

/* P_E(t) = t^E mod phi(t) by left-to-right binary exponentiation (Sec. 4):
 * for each bit of E from the top, square, then multiply by t on a 1 bit.
 * E is little-endian in nw 32-bit words. */
void orc_poly_pow_t(const uint32_t *E, int nw, uint32_t *out)
{
    uint32_t p[ORC_R], t1[ORC_R];
    memset(p, 0, sizeof(p));
    memset(t1, 0, sizeof(t1));
    p[0] = 1;
    t1[1] = 1;
#if ORC_MUTANT == 8
    nw = nw - 1;
#endif
    for (int w = nw - 1; w >= 0; w--) {
        for (int bit = 31; bit >= 0; bit--) {
#if ORC_MUTANT == 6
            int b = (E[w] >> (31 - bit)) & 1u;
#else
            int b = (E[w] >> bit) & 1u;
#endif
            orc_poly_mulmod(p, p, p);
            if (b) orc_poly_mulmod(p, t1, p);
        }
    }
    memcpy(out, p, sizeof(p));
}

/* u P(A) as a linear combination (Sec. 3.1): u A^i is the state after i
 * transitions, so word k of u P(A) is sum_i b_i x_{i+k+1} (1-based x).
 * The window x_1..x_193 is extended by the recurrence x_n = x_{n-97} -
 * x_{n-33}. */
void orc_apply_dot(const uint32_t *x, const uint32_t *b, uint32_t *out)
{
    uint32_t X[2 * ORC_R - 1];
    for (int q = 0; q < ORC_R; q++) X[q] = x[q];
    for (int q = ORC_R; q < 2 * ORC_R - 1; q++)
        X[q] = X[q - ORC_R] - X[q - ORC_S];
    for (int k = 0; k < ORC_R; k++) {
        uint32_t acc = 0;
        for (int i = 0; i < ORC_R; i++) {
#if ORC_MUTANT == 5
            acc += b[i] * X[(ORC_R - 1 - i) + k];
#else
            acc += b[i] * X[i + k];
#endif
        }
        out[k] = acc & ORC_MASK;
    }
}

/* The same by Horner's rule exactly as printed in Sec. 3.1:
 * u P(A) = (...((b_96 u A + b_95 u) A + b_94 u) A + ... + b_1 u) A + b_0 u,
 * with vA = F1(v) = (v_2, ..., v_97, v_1 - v_65). */
void orc_apply_horner(const uint32_t *x, const uint32_t *b, uint32_t *out)
{
    uint32_t v[ORC_R], nv[ORC_R];
    for (int q = 0; q < ORC_R; q++) v[q] = b[ORC_R - 1] * x[q];
    for (int i = ORC_R - 2; i >= 0; i--) {
#if ORC_MUTANT == 11
        int bi = ORC_R - 2 - i;
#else
        int bi = i;
#endif
        for (int q = 0; q < ORC_R - 1; q++) nv[q] = v[q + 1];
        nv[ORC_R - 1] = v[0] - v[ORC_R - ORC_S];   /* v_1 - v_{r-s+1} */
        for (int q = 0; q < ORC_R; q++) v[q] = nv[q] + b[bi] * x[q];
    }
    for (int q = 0; q < ORC_R; q++) out[q] = v[q] & ORC_MASK;
}

/* E mod m for a multi-word E (Horner over 32-bit digits). */
uint32_t orc_exp_mod_m(const uint32_t *E, int nw)
{
    uint64_t r = 0;
    for (int w = nw - 1; w >= 0; w--) r = ((r << 32) | E[w]) % ORC_m;
    return (uint32_t)r;
}

/* Sec. 3.2: c_J = (c'_0 - J d') mod m, needing only J mod m (reading R5). */
uint32_t orc_c_jump(uint32_t c, const uint32_t *E, int nw)
{
    uint64_t e = orc_exp_mod_m(E, nw);
#if ORC_MUTANT == 7
    return (uint32_t)(((uint64_t)c + e * ORC_d) % ORC_m);
#else
    return (uint32_t)(((uint64_t)c + (uint64_t)(ORC_m - e) * ORC_d) % ORC_m);
#endif
}

/* c stepped n times by f2 (Sec. 2): c <- c - d mod m. */
uint32_t orc_c_step(uint32_t c, uint64_t n)
{
    for (uint64_t t = 0; t < n; t++) c = (c >= ORC_d) ? c - ORC_d : c + ORC_m - ORC_d;
    return c;
}

/* Full jump of a sequence-order state by E transitions (Sec. 2: f^E =
 * (f1^E, f2^E)): P_E = t^E mod phi, x' = x P_E(A), c' = c_E. */
void orc_jump(const uint32_t *x, uint32_t c, const uint32_t *E, int nw,
              uint32_t *x_out, uint32_t *c_out)
{
    uint32_t b[ORC_R], xo[ORC_R];
    orc_poly_pow_t(E, nw, b);
    orc_apply_dot(x, b, xo);
    memcpy(x_out, xo, sizeof(xo));
    *c_out = orc_c_jump(c, E, nw);
}

/* Stream k of (seed, J) (Sec. 1): the block that starts E = kJ transitions
 * after the seeded state; writes its first `count` 24-bit outputs. */
int orc_stream(int32_t seed, const uint32_t *E, int nw, uint64_t count,
               uint32_t *out)
{
    uint32_t x[ORC_R], c;
    if (orc_seeded_state(seed, x, &c) != 0) return -1;
    orc_jump(x, c, E, nw, x, &c);
    orc_generate(x, c, count, out, NULL, NULL);
    return 0;
}

/* ======================================================================== */
/* Concluding remarks: the jump for lagged Fibonacci recurrences of general */
/* order.  x_n = x_{n-r} - x_{n-s} mod 2^e (r > s >= 1, 1 <= e <= 32) has    */
/* the transition matrix of Sec. 3.1 with characteristic polynomial          */
/*     phi_{r,s}(t) = t^r + t^{r-s} - 1,   i.e. t^k = t^{k-r} - t^{k-s},     */
/* and the jump by E is x' = x P_E(A) with P_E = t^E mod phi_{r,s} (for      */
/* r = 97, s = 33, e = 24 it is the lagged Fibonacci part of RANMAR).  The   */
/* cost of P_E is one polynomial product per exponent bit: r^2 multiply-adds */
/* with the classical product, about r^{log2 3} with Karatsuba's (the        */
/* concluding remarks).  The window x[0..r) is kept oldest first.            */
/* ======================================================================== */
static uint32_t lfg_mask(int e) { return e >= 32 ? 0xFFFFFFFFu : ((1u << e) - 1u); }

/* n transitions of the window by the recurrence (brute force). */
void orc_lfg_step(uint32_t *x, int r, int s, int e, uint64_t n)
{
    uint32_t mask = lfg_mask(e);
    uint32_t *ring = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)r);
    memcpy(ring, x, sizeof(uint32_t) * (size_t)r);
    int h = 0;                                   /* ring[h] = oldest word */
    int q = r - s;                               /* ring[q] = x_{n-s}     */
    for (uint64_t t = 0; t < n; t++) {
        uint32_t w = (ring[h] - ring[q]) & mask;
        ring[h] = w;
        h = (h + 1 == r) ? 0 : h + 1;
        q = (q + 1 == r) ? 0 : q + 1;
    }
    for (int i = 0; i < r; i++) x[i] = ring[(h + i) % r];
    free(ring);
}

/* c[0 .. 2r-1) reduced mod phi_{r,s} from the top: t^k = t^{k-r} - t^{k-s}. */
static void lfg_reduce(uint32_t *c, int r, int s)
{
    for (int k = 2 * r - 2; k >= r; k--) {
        uint32_t h = c[k];
        c[k] = 0;
        c[k - r] += h;
#if ORC_MUTANT == 13
        c[k - s] += h;
#else
        c[k - s] -= h;
#endif
    }
}

/* Classical product c[0 .. 2n-1) = a b of two n-coefficient polynomials. */
static void lfg_school(const uint32_t *a, const uint32_t *b, uint32_t *c, int n)
{
    memset(c, 0, sizeof(uint32_t) * (size_t)(2 * n));
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) c[i + j] += a[i] * b[j];
}

/* Karatsuba's product c[0 .. 2n-1) = a b: with a = a0 + t^h a1, b likewise
 * (h = n/2), a b = z0 + t^h (z1 - z0 - z2) + t^{2h} z2 for z0 = a0 b0,
 * z2 = a1 b1, z1 = (a0 + a1)(b0 + b1); classical below 16 coefficients. */
static void lfg_kara(const uint32_t *a, const uint32_t *b, uint32_t *c, int n)
{
    if (n <= 16) {
        lfg_school(a, b, c, n);
        return;
    }
    int h = n / 2, hh = n - h;                   /* a0: h coefficients, a1: hh >= h */
    uint32_t *sa = (uint32_t *)calloc((size_t)hh, sizeof(uint32_t));
    uint32_t *sb = (uint32_t *)calloc((size_t)hh, sizeof(uint32_t));
    uint32_t *a0 = (uint32_t *)calloc((size_t)hh, sizeof(uint32_t));
    uint32_t *b0 = (uint32_t *)calloc((size_t)hh, sizeof(uint32_t));
    uint32_t *z0 = (uint32_t *)calloc((size_t)(2 * hh), sizeof(uint32_t));
    uint32_t *z1 = (uint32_t *)calloc((size_t)(2 * hh), sizeof(uint32_t));
    uint32_t *z2 = (uint32_t *)calloc((size_t)(2 * hh), sizeof(uint32_t));
    memcpy(a0, a, sizeof(uint32_t) * (size_t)h);
    memcpy(b0, b, sizeof(uint32_t) * (size_t)h);
    for (int i = 0; i < hh; i++) {
        sa[i] = a0[i] + a[h + i];
        sb[i] = b0[i] + b[h + i];
    }
    lfg_kara(a0, b0, z0, hh);                    /* a0, b0 zero padded to hh */
    lfg_kara(a + h, b + h, z2, hh);
    lfg_kara(sa, sb, z1, hh);
    memset(c, 0, sizeof(uint32_t) * (size_t)(2 * n));
    for (int i = 0; i < 2 * hh; i++) {
#if ORC_MUTANT == 12
        uint32_t mid = z1[i] - z0[i];
#else
        uint32_t mid = z1[i] - z0[i] - z2[i];
#endif
        if (i < 2 * h) c[i] += z0[i];
        c[h + i] += mid;
        if (2 * h + i < 2 * n) c[2 * h + i] += z2[i];
    }
    free(sa); free(sb); free(a0); free(b0); free(z0); free(z1); free(z2);
}

/* out = a b mod phi_{r,s}, classical (karatsuba = 0) or Karatsuba product. */
void orc_lfg_mulmod(const uint32_t *a, const uint32_t *b, uint32_t *out, int r, int s, int e,
                    int karatsuba)
{
    uint32_t *c = (uint32_t *)calloc((size_t)(2 * r), sizeof(uint32_t));
    if (karatsuba) lfg_kara(a, b, c, r);
    else lfg_school(a, b, c, r);
    lfg_reduce(c, r, s);
    uint32_t mask = lfg_mask(e);
    for (int i = 0; i < r; i++) out[i] = c[i] & mask;
    free(c);
}

/* P_E = t^E mod phi_{r,s} by left-to-right binary exponentiation (square,
 * then multiply by t on a 1 bit); E little-endian in nw 32-bit words. */
void orc_lfg_pow_t(const uint32_t *E, int nw, uint32_t *out, int r, int s, int e, int karatsuba)
{
    uint32_t *p = (uint32_t *)calloc((size_t)r, sizeof(uint32_t));
    uint32_t *t1 = (uint32_t *)calloc((size_t)r, sizeof(uint32_t));
    uint32_t mask = lfg_mask(e);
    p[0] = 1;
    if (r > 1) t1[1] = 1;
    else t1[0] = 1;
    for (int w = nw - 1; w >= 0; w--) {
        for (int bit = 31; bit >= 0; bit--) {
            int b = (E[w] >> bit) & 1u;
            orc_lfg_mulmod(p, p, p, r, s, e, karatsuba);
            if (b) {
                /* p t: shift up, the word on t^r becomes 1 - t^{r-s} */
                uint32_t top = p[r - 1];
                memmove(p + 1, p, sizeof(uint32_t) * (size_t)(r - 1));
                p[0] = top;
                p[r - s] = (p[r - s] - top) & mask;
            }
        }
    }
    memcpy(out, p, sizeof(uint32_t) * (size_t)r);
    free(p);
    free(t1);
}

/* x' = x P(A): new word k = sum_i p_i X_{i+k}, X the window extended by the
 * recurrence to 2r-1 words (the dot-product form of Sec. 3.1). */
void orc_lfg_apply(const uint32_t *x, const uint32_t *p, uint32_t *out, int r, int s, int e)
{
    uint32_t *X = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(2 * r));
    memcpy(X, x, sizeof(uint32_t) * (size_t)r);
    for (int q = r; q < 2 * r - 1; q++) X[q] = X[q - r] - X[q - s];
    uint32_t mask = lfg_mask(e);
    for (int k = 0; k < r; k++) {
        uint32_t acc = 0;
        for (int i = 0; i < r; i++) acc += p[i] * X[i + k];
        out[k] = acc & mask;
    }
    free(X);
}

/* The jump by E of the window x (out may alias x). */
void orc_lfg_jump(const uint32_t *x, const uint32_t *E, int nw, uint32_t *out, int r, int s,
                  int e, int karatsuba)
{
    uint32_t *p = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)r);
    uint32_t *o = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)r);
    orc_lfg_pow_t(E, nw, p, r, s, e, karatsuba);
    orc_lfg_apply(x, p, o, r, s, e);
    memcpy(out, o, sizeof(uint32_t) * (size_t)r);
    free(p);
    free(o);
}

/* The next n words of the recurrence after the window x (brute force); x is
 * advanced by n transitions. */
void orc_lfg_generate(uint32_t *x, int r, int s, int e, uint64_t n, uint32_t *out)
{
    uint32_t mask = lfg_mask(e);
    uint32_t *ring = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)r);
    memcpy(ring, x, sizeof(uint32_t) * (size_t)r);
    int h = 0, q = r - s;
    for (uint64_t t = 0; t < n; t++) {
        uint32_t w = (ring[h] - ring[q]) & mask;
        out[t] = w;
        ring[h] = w;
        h = (h + 1 == r) ? 0 : h + 1;
        q = (q + 1 == r) ? 0 : q + 1;
    }
    for (int i = 0; i < r; i++) x[i] = ring[(h + i) % r];
    free(ring);
}
