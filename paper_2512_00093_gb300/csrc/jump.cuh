// jump.cuh -- batched jump-ahead (Sec. 3.1, Sec. 3.2).
//
// For each stream: P_E(t) = t^E mod phi(t), phi = t^97 + t^64 - 1 over
// Z/2^24, by left-to-right square-and-multiply (a 1 bit multiplies by t: a
// shift plus the fold t^97 = 1 - t^64); then the new state word k =
// sum_i b_i x_{i+k+1} (x extended by the recurrence), which is the Horner
// form u P_E(A) of Sec. 3.1; then c_E = (c - E d) mod m (Sec. 3.2).
//
// Mapping: TWO lanes per stream, 16 streams per warp, one warp per CTA.  Every
// pair runs the same instruction stream on its own polynomial, so the 97x97
// products are register-blocked 8x8 tiles of 32-bit multiply-adds (mul.lo
// wraps mod 2^32, exact mod 2^24; masks only at the end).  Within a tile the
// pair splits the rows: lane g takes rows 4g..4g+3 against all 8 columns
// (32 multiply-adds into 11 accumulators).
//
// Squaring a(t)^2, in place: tiles (I, J), I <= J, of 8-coefficient blocks
// are summed along the anti-diagonal s = I + J (outputs 8s .. 8s+14), walking
// s DOWN from 24 to 0.  Off-diagonal tiles are summed and doubled; the
// diagonal tile (I = J) is then added as a full 8x8 product (its off-diagonal
// pairs twice, its squares once).  After anti-diagonal s the product block
// s+1 (coefficients 8s+8 .. 8s+15) is complete, and block s+1 of `a` is no
// longer read (anti-diagonals <= s use blocks <= s), so:
//   * blocks >= 12 (degree >= 96) go to a 128-word region R (R[k-96] = c_k);
//   * blocks <= 12 are reduced at once and written into `a` itself:
//       a_n = c_n + h_n[n<=95] - h_{n+33}[n<=62] + h_{n+66}[n<=29]
//             - h_{n-64}[n>=64] + h_{n-31}[n>=64] - h_{n+2}[64<=n<=93]
//     with h_j = c_{97+j} (t^k = t^{k-97} - t^{k-33} applied until the
//     degree is below 97; every high block is complete before the first low
//     one, because s walks down).
// A multiplication by t shifts the written index by one; the word that lands
// on t^97 is folded back at the end.  After each anti-diagonal the pair
// swaps 4 partial sums by shuffle.
//
// Application: the extended window X(0..207) is consumed through the same
// 128-word region used as a ring (window X[8K .. 8K+111] for output block K,
// 16 new words per round computed by the recurrence).
//
// Shared memory per stream: a (104 words, 13 zero-padded blocks of 8) + R
// (128 words); stride 232 = 8 mod 32, so that the 16-byte loads of a quarter
// warp (4 streams x 2 lanes) fall in 8 distinct bank groups.  14,848 B per
// CTA.
#pragma once

#include "ranmar_device.cuh"

namespace ranmar {

constexpr int kPolyWords = 104;    // 13 blocks of 8 >= 97
constexpr int kRingWords = 128;    // high product words / application ring
constexpr int kStreamWords = 232;  // per-stream slice stride (8 mod 32)
constexpr int kJumpStreamsPerWarp = 16;
constexpr size_t kJumpSmemBytes = sizeof(uint32_t) * kStreamWords * kJumpStreamsPerWarp;
static_assert(kPolyWords + kRingWords <= kStreamWords, "slice");
static_assert(kStreamWords % 32 == 8, "bank spread");

struct ExpParams {
  uint32_t J[kMaxExpWords];  // partition mode: E = (k0 + i) * J
  uint32_t J_words;
  uint32_t flags;            // RANMAR_JUMP_REDUCE_PERIOD
  uint64_t k0;
};

struct Quad {
  uint32_t v[4];
};
struct Oct {
  uint32_t v[8];
};

__device__ __forceinline__ Quad lds4(const uint32_t* p) {
  const uint4 t = *reinterpret_cast<const uint4*>(p);
  return Quad{{t.x, t.y, t.z, t.w}};
}
__device__ __forceinline__ Oct lds8(const uint32_t* p) {
  const uint4 lo = *reinterpret_cast<const uint4*>(p);
  const uint4 hi = *reinterpret_cast<const uint4*>(p + 4);
  return Oct{{lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w}};
}

// acc[p + q] += r[p] * col[q]: rows of this lane (4) x columns (8).
__device__ __forceinline__ void tile_mac(uint32_t (&acc)[11], const Quad& r, const Oct& col) {
#pragma unroll
  for (int p = 0; p < 4; ++p) {
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[p + q] += r.v[p] * col.v[q];
  }
}

// Reduced coefficients n = 8b + 4g + k (k < 4, n <= 96) of a completed
// product block, written to a[n + shift].  Blocks 0-2, 4-6 and 8-10 have one
// fixed set of terms for all their coefficients; the four blocks that
// straddle a range boundary (3, 7, 11, 12) test each coefficient.
enum ReduceTerms { kLow3 = 0, kLow2 = 1, kHigh4 = 2, kGeneric = 3 };

template <int kTerms>
__device__ __forceinline__ void reduce_block_t(uint32_t* __restrict__ a,
                                               const uint32_t* __restrict__ R, int b,
                                               unsigned g, const uint32_t (&cv)[4],
                                               uint32_t shift) {
  const uint32_t* h = R + 1;  // h_j = c_{97+j}
  const int n0 = 8 * b + 4 * static_cast<int>(g);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int n = n0 + k;
    uint32_t v = cv[k];
    if (kTerms == kLow3) {          // n <= 23
      v += h[n] - h[n + 33] + h[n + 66];
    } else if (kTerms == kLow2) {   // 32 <= n <= 55
      v += h[n] - h[n + 33];
    } else if (kTerms == kHigh4) {  // 64 <= n <= 87
      v += h[n] - h[n - 64] + h[n - 31] - h[n + 2];
    } else {
      if (n > 96) continue;
      if (n <= 95) v += h[n];
      if (n <= 62) v -= h[n + 33];
      if (n <= 29) v += h[n + 66];
      if (n >= 64) {
        v += h[n - 31] - h[n - 64];
        if (n <= 93) v -= h[n + 2];
      }
    }
    a[n + shift] = v;
  }
}

__device__ __forceinline__ void reduce_block(uint32_t* __restrict__ a,
                                             const uint32_t* __restrict__ R, int b, unsigned g,
                                             const uint32_t (&cv)[4], uint32_t shift) {
  if (b <= 2)
    reduce_block_t<kLow3>(a, R, b, g, cv, shift);
  else if (b >= 4 && b <= 6)
    reduce_block_t<kLow2>(a, R, b, g, cv, shift);
  else if (b >= 8 && b <= 10)
    reduce_block_t<kHigh4>(a, R, b, g, cv, shift);
  else
    reduce_block_t<kGeneric>(a, R, b, g, cv, shift);
}

// In place, with the lanes g = 0, 1 of the pair cooperating:
//   kSquare:  a = a^2 t^shift mod phi          (b unused)
//   !kSquare: a = a b mod phi (shift must be 0; b is not modified)
// `mask` holds the lanes taking part (both lanes of every participating pair).
template <bool kSquare>
__device__ __forceinline__ void product_reduce_pair(uint32_t* __restrict__ a,
                                                    const uint32_t* __restrict__ b,
                                                    uint32_t* __restrict__ R, uint32_t shift,
                                                    unsigned g, unsigned mask) {
  uint32_t pend[4] = {0u, 0u, 0u, 0u};  // low half of the previous anti-diagonal
  const uint32_t* arow = a + 4 * g;
  const uint32_t* bcol = kSquare ? a : b;
  const uint32_t keep0 = g ? 0u : ~0u;
#pragma unroll 1
  for (int s = 24; s >= 0; --s) {
    uint32_t acc[11];
#pragma unroll
    for (int r = 0; r < 11; ++r) acc[r] = 0;
    const int ilo = s > 12 ? s - 12 : 0;
    // squaring: off-diagonal tiles I < J, i.e. I in [ilo, iend); general: all I
    const int iend = kSquare ? ((s & 1) ? (s >> 1) + 1 : (s >> 1)) : (s < 12 ? s : 12) + 1;
    if (ilo < iend) {
      Quad r0 = lds4(arow + 8 * ilo), r1;
      Oct c0 = lds8(bcol + 8 * (s - ilo)), c1;
      int I = ilo;
#pragma unroll 1
      for (; I + 1 < iend; I += 2) {  // operands one tile ahead, ping-pong
        r1 = lds4(arow + 8 * (I + 1));
        c1 = lds8(bcol + 8 * (s - I - 1));
        tile_mac(acc, r0, c0);
        if (I + 2 < iend) {
          r0 = lds4(arow + 8 * (I + 2));
          c0 = lds8(bcol + 8 * (s - I - 2));
        }
        tile_mac(acc, r1, c1);
      }
      if (I < iend) tile_mac(acc, r0, c0);
      if (kSquare) {
#pragma unroll
        for (int k = 0; k < 11; ++k) acc[k] += acc[k];
      }
    }
    if (kSquare && (s & 1) == 0) tile_mac(acc, lds4(arow + 4 * s), lds8(a + 4 * s));

    // Lane 0 holds outputs 0..10 of this anti-diagonal, lane 1 outputs 4..14.
    // Block s+1 = outputs 8..14 here + the low half of anti-diagonal s+1.
    uint32_t out[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t recv = __shfl_xor_sync(mask, acc[4 + k], 1);
      out[k] = (k < 3 ? acc[8 + k] : 0u) + pend[k] + (recv & keep0);
      pend[k] = acc[k] + (recv & ~keep0);
    }
    const int bb = s + 1;
    if (bb <= 24) {
      if (bb >= 12)
        *reinterpret_cast<uint4*>(R + 8 * bb - 96 + 4 * g) = make_uint4(out[0], out[1], out[2], out[3]);
      if (bb <= 12) reduce_block(a, R, bb, g, out, shift);
    }
    __syncwarp(mask);
  }
  reduce_block(a, R, 0, g, pend, shift);
  __syncwarp(mask);
  if (kSquare && shift && g == 0) {  // fold t^97 = 1 - t^64
    const uint32_t top = a[kR];
    a[0] = top;
    a[64] -= top;
    a[kR] = 0;
  }
  __syncwarp(mask);
}

__device__ __forceinline__ void square_reduce_pair(uint32_t* __restrict__ a,
                                                   uint32_t* __restrict__ R, uint32_t shift,
                                                   unsigned g) {
  product_reduce_pair<true>(a, a, R, shift, g, kFull);
}

__device__ __forceinline__ uint32_t exp_word(const uint32_t (&E)[kMaxExpWords], int w) {
  uint32_t v = E[0];
#pragma unroll
  for (int i = 1; i < kMaxExpWords; ++i) v = (w == i) ? E[i] : v;
  return v;
}

__device__ __forceinline__ uint32_t exp_bit(const uint32_t (&E)[kMaxExpWords], int p) {
  return (exp_word(E, p >> 5) >> (p & 31)) & 1u;
}

// Six bits of E starting at bit p (p >= 0).
__device__ __forceinline__ uint32_t exp_bits6(const uint32_t (&E)[kMaxExpWords], int p) {
  const int w = p >> 5, sh = p & 31;
  const uint32_t lo = exp_word(E, w);
  const uint32_t hi = (w + 1 < kMaxExpWords) ? exp_word(E, w + 1) : 0u;
  return __funnelshift_r(lo, hi, sh) & 63u;
}

__device__ __forceinline__ int exp_bitlen(const uint32_t (&E)[kMaxExpWords]) {
  int n = 0;
#pragma unroll
  for (int w = 0; w < kMaxExpWords; ++w)
    if (E[w] != 0) n = 32 * w + 32 - __clz(E[w]);
  return n;
}

// E mod m by Horner over 32-bit digits.
__device__ __forceinline__ uint32_t exp_mod_m(const uint32_t (&E)[kMaxExpWords]) {
  uint64_t r = 0;
#pragma unroll
  for (int w = kMaxExpWords - 1; w >= 0; --w) r = ((r << 32) | E[w]) % kModM;
  return static_cast<uint32_t>(r);
}

// E += J * m * 2^(32 shift) (multi-word), truncated to kMaxExpWords.
__device__ __forceinline__ void exp_mul_add(uint32_t (&E)[kMaxExpWords], const uint32_t* J,
                                            uint32_t m, int shift) {
  uint64_t carry = 0;
#pragma unroll
  for (int w = 0; w < kMaxExpWords; ++w) {
    if (w + shift < kMaxExpWords) {
      const uint64_t t = static_cast<uint64_t>(J[w]) * m + E[w + shift] + carry;
      E[w + shift] = static_cast<uint32_t>(t);
      carry = t >> 32;
    }
  }
}

// E mod T for T = (2^97 - 1) 2^23 = 2^120 - 2^23, the multiplicative order of
// t modulo phi over Z/2^24 (so t^E = t^(E mod T) and the polynomial part of a
// jump may use the reduced exponent; c needs E mod m instead).  Two folds of
// 2^120 = 2^23 (mod T) bring E below 2^120, then one conditional
// subtraction of T.
__device__ __forceinline__ void reduce_period(uint32_t (&E)[kMaxExpWords]) {
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const uint64_t hi = (static_cast<uint64_t>(E[4]) << 8) | (E[3] >> 24);  // bits 120..159
    if (hi != 0) {
      E[3] &= 0x00FFFFFFu;
      E[4] = 0;
      const uint64_t add = hi << 23;  // < 2^63
      uint64_t t = static_cast<uint64_t>(E[0]) + static_cast<uint32_t>(add);
      E[0] = static_cast<uint32_t>(t);
      t = (t >> 32) + E[1] + static_cast<uint32_t>(add >> 32);
      E[1] = static_cast<uint32_t>(t);
      t = (t >> 32) + E[2];
      E[2] = static_cast<uint32_t>(t);
      t = (t >> 32) + E[3];
      E[3] = static_cast<uint32_t>(t);
    }
  }
  if (E[3] == 0x00FFFFFFu && E[2] == 0xFFFFFFFFu && E[1] == 0xFFFFFFFFu &&
      E[0] >= 0xFF800000u) {  // T <= E < 2^120
    E[0] -= 0xFF800000u;
    E[1] = E[2] = E[3] = 0;
  }
}

// a = t^E mod phi for the stream of this lane pair by left-to-right
// square-and-multiply; all 32 lanes of the warp call it together (the bit
// loop is warp-uniform: it runs over the longest exponent of the warp).
__device__ __forceinline__ void poly_power_pair(const uint32_t (&E)[kMaxExpWords], bool active,
                                                uint32_t* __restrict__ a,
                                                uint32_t* __restrict__ R, unsigned g) {
  const int nb = active ? exp_bitlen(E) : 0;
  const int L = static_cast<int>(__reduce_max_sync(kFull, static_cast<unsigned>(nb)));

  // Leading (up to) six bits: P = t^v0 with v0 < 64 < 97 is a monomial.
  uint32_t v0;
  int p;
  if (L <= 6) {
    v0 = E[0] & 63u;
    p = -1;
  } else {
    v0 = exp_bits6(E, L - 6);
    p = L - 7;
  }
  if (!active) v0 = 0;
  for (int q = static_cast<int>(g); q < kPolyWords / 4; q += 2)
    reinterpret_cast<uint4*>(a)[q] = make_uint4(0u, 0u, 0u, 0u);
  __syncwarp();
  if (g == 0) a[v0] = 1u;
  __syncwarp();

#pragma unroll 1
  for (; p >= 0; --p) {
    const uint32_t bit = active ? exp_bit(E, p) : 0u;
    square_reduce_pair(a, R, bit, g);
  }
}

// dst = x P(A) with P = a (97 coefficients, zero padded), and the c / pos
// jump by E.  The extended window X is consumed through the 128-word region
// R used as a ring: X(0..96) is the base state, X(q) = X(q-97) - X(q-33)
// beyond.  Round m handles output blocks K = 2m + g, whose windows are
// X[8K .. 8K+111]; between rounds 16 new words replace the 16 oldest (each
// depends only on words still in the ring).
__device__ __forceinline__ void apply_pair(const ranmar_state_t* __restrict__ base,
                                           const uint32_t (&E)[kMaxExpWords], bool active,
                                           ranmar_state_t* __restrict__ dst,
                                           const uint32_t* __restrict__ a,
                                           uint32_t* __restrict__ R, unsigned g) {
  uint32_t* ring = R;
  const uint32_t* bx = base->x;
  for (int q = static_cast<int>(g); q < kR; q += 2) ring[q] = bx[q];
  __syncwarp();
  for (int q = kR + static_cast<int>(g); q < kRingWords; q += 2) ring[q] = ring[q - kR] - ring[q - kS];
  __syncwarp();

  uint32_t* ox = dst->x;
#pragma unroll 1
  for (int m = 0; m < 7; ++m) {
    const int K = 2 * m + static_cast<int>(g);
    if (K < 13) {
      uint32_t acc[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) acc[r] = 0;
      // 13 tiles, fully unrolled so that the sliding window (blocks I+K and
      // I+K+1 of X) and the coefficient blocks are renamed, not moved.
      Oct w[14];
      w[0] = lds8(ring + ((8 * K) & (kRingWords - 1)));
#pragma unroll
      for (int I = 0; I < 13; ++I) {
        const Oct b = lds8(a + 8 * I);
        w[I + 1] = lds8(ring + ((8 * (I + 1 + K)) & (kRingWords - 1)));
#pragma unroll
        for (int p2 = 0; p2 < 8; ++p2) {
#pragma unroll
          for (int r = 0; r < 8; ++r) {
            const int idx = p2 + r;
            acc[r] += b.v[p2] * (idx < 8 ? w[I].v[idx & 7] : w[I + 1].v[idx & 7]);
          }
        }
      }
      if (active) {
        if (K < 12) {
          uint4* o4 = reinterpret_cast<uint4*>(ox + 8 * K);
          o4[0] = make_uint4(acc[0] & kMask24, acc[1] & kMask24, acc[2] & kMask24,
                             acc[3] & kMask24);
          o4[1] = make_uint4(acc[4] & kMask24, acc[5] & kMask24, acc[6] & kMask24,
                             acc[7] & kMask24);
        } else {
          ox[96] = acc[0] & kMask24;
        }
      }
    }
    __syncwarp();
    if (m < 6) {
      for (int j = static_cast<int>(g); j < 16; j += 2) {
        const int q = 16 * m + kRingWords + j;
        ring[q & (kRingWords - 1)] =
            ring[(q - kR) & (kRingWords - 1)] - ring[(q - kS) & (kRingWords - 1)];
      }
      __syncwarp();
    }
  }

  if (active && g == 0) {
    const uint32_t e = exp_mod_m(E);
    // (c - e d) mod m = (c + (m - e) d) mod m, non-negative residue.
    const uint64_t cn =
        (static_cast<uint64_t>(base->c) + static_cast<uint64_t>(kModM - e) * kD) % kModM;
    dst->c = static_cast<uint32_t>(cn);
    dst->pos = base->pos + (static_cast<uint64_t>(E[1]) << 32 | E[0]);
  }
}

// dst = f^E(base) for the stream of this lane pair.
// Ep is the exponent of the polynomial part (E itself, or E mod T), E the
// full exponent (for c and pos).
__device__ __forceinline__ void jump_pair(const ranmar_state_t* __restrict__ base,
                                          const uint32_t (&Ep)[kMaxExpWords],
                                          const uint32_t (&E)[kMaxExpWords], bool active,
                                          ranmar_state_t* __restrict__ dst,
                                          uint32_t* __restrict__ a, uint32_t* __restrict__ R,
                                          unsigned g) {
  poly_power_pair(Ep, active, a, R, g);
  apply_pair(base, E, active, dst, a, R, g);
}

// Exponent of stream i: mode 0 reads it from d_exp, mode 1 forms (k0 + i) J.
__device__ __forceinline__ void load_exponent(uint32_t (&E)[kMaxExpWords], int mode,
                                              const uint32_t* __restrict__ d_exp,
                                              uint32_t exp_words, const ExpParams& part,
                                              uint64_t i) {
#pragma unroll
  for (int w = 0; w < kMaxExpWords; ++w) E[w] = 0;
  if (mode == 0) {
    const uint32_t* ew = d_exp + i * exp_words;
#pragma unroll
    for (int w = 0; w < kMaxExpWords; ++w)
      if (w < static_cast<int>(exp_words)) E[w] = ew[w];
  } else {
    const uint64_t k = part.k0 + i;
    exp_mul_add(E, part.J, static_cast<uint32_t>(k), 0);
    exp_mul_add(E, part.J, static_cast<uint32_t>(k >> 32), 1);
  }
}

// mode 0: E_i from d_exp (exp_words per stream), base d_base[base_idx[i]].
// mode 1: E_i = (k0 + i) * J, base d_base[0].
// d_dst_idx (mode 0 only, may be null): stream i is written to
// d_out[d_dst_idx[i]] (index < n_dst) instead of d_out[i].
__global__ void __launch_bounds__(32) jump_kernel(
    const ranmar_state_t* __restrict__ d_base, uint64_t n_base,
    const uint32_t* __restrict__ d_base_idx, const uint32_t* __restrict__ d_exp,
    uint32_t exp_words, ExpParams part, int mode, ranmar_state_t* __restrict__ d_out,
    uint64_t n, uint32_t* status, const uint32_t* __restrict__ d_dst_idx, uint64_t n_dst) {
  extern __shared__ __align__(16) uint32_t smem[];
  const unsigned lane = threadIdx.x & 31;
  const unsigned g = lane & 1;
  const unsigned slot = lane >> 1;
  const uint64_t i = static_cast<uint64_t>(blockIdx.x) * kJumpStreamsPerWarp + slot;
  uint32_t* a = smem + slot * kStreamWords;
  uint32_t* R = a + kPolyWords;

  bool active = i < n;
  uint32_t E[kMaxExpWords];
  load_exponent(E, active ? mode : 0, d_exp, active ? exp_words : 0, part, i);
  const ranmar_state_t* base = d_base;
  if (active && mode == 0) {
    const uint32_t bi = d_base_idx ? d_base_idx[i] : 0u;
    if (bi >= n_base) {
      if (g == 0) flag_status(status, RANMAR_ST_BAD_INDEX);
      active = false;
    } else {
      base = d_base + bi;
    }
  }
  uint64_t di = i;
  if (active && d_dst_idx) {
    di = d_dst_idx[i];
    if (di >= n_dst) {
      if (g == 0) flag_status(status, RANMAR_ST_BAD_INDEX);
      active = false;
    }
  }
  uint32_t Ep[kMaxExpWords];
#pragma unroll
  for (int w = 0; w < kMaxExpWords; ++w) Ep[w] = E[w];
  if (part.flags & RANMAR_JUMP_REDUCE_PERIOD) reduce_period(Ep);
  jump_pair(base, Ep, E, active, d_out + (active ? di : 0), a, R, g);
}

}  // namespace ranmar
