// jump.cuh -- building blocks of the jump-ahead (Sec. 3.1, Sec. 3.2), a
// lane pair per stream (lanes L and L + 16 of the warp, 16 streams per
// warp): the exponent arithmetic, the general product a b mod phi(t) of two
// polynomials (phi = t^97 + t^64 - 1 over Z/2^24), and the application of a
// jump polynomial to a state.  The squaring of the paper's square-and-
// multiply and its kernels are in square_mirror.cuh.
//
// General product: a polynomial is held as six 16-coefficient blocks
// (coefficients 0..95) plus coefficient 96 alone:
//     a = a' + a_96 t^96,  a b = a'b' + t^96 (a_96 b' + b_96 a') + a_96 b_96 t^192,
// so the 97x97 product is 6x6 register-blocked 16x16 tiles of 32-bit
// multiply-adds (mul.lo wraps mod 2^32, exact mod 2^24; masks only at the
// end) plus a rank-1 correction of the coefficients 96..192.  Within a tile
// the pair splits the rows: lane g takes rows 8g..8g+7 against all 16
// columns (128 multiply-adds into 23 accumulators).
//
// In place, anti-diagonal by anti-diagonal: tiles (I, J) with I + J = s
// produce the outputs 16s .. 16s+30; s walks DOWN from 10 to 0.  After
// anti-diagonal s the product block s+1 (coefficients 16s+16 .. 16s+31) is
// complete, and block s+1 of `a` is no longer read (anti-diagonals <= s use
// blocks <= s), so:
//   * blocks >= 6 (degree >= 96) get the rank-1 correction and go to a
//     128-word region R (R[k-96] = c_k; R[96] = c_192 = a_96 b_96);
//   * blocks <= 5 and coefficient 96 are reduced at once and written into
//     `a` itself:
//       a_n = c_n + h_n[n<=95] - h_{n+33}[n<=62] + h_{n+66}[n<=29]
//             - h_{n-64}[n>=64] + h_{n-31}[n>=64] - h_{n+2}[64<=n<=93]
//     with h_j = c_{97+j} (t^k = t^{k-97} - t^{k-33} applied until the
//     degree is below 97; every high block is complete before the first low
//     one, because s walks down).
// After each anti-diagonal the pair swaps 8 partial sums by shuffle.
//
// Application: the extended window X(0..192) is consumed through the same
// 128-word region used as a ring (window X(16K .. 16K+111) for output block
// K, 32 new words per round computed by the recurrence).
//
// Shared memory per stream: a (100 words: blocks, coefficient 96, padding)
// + R (128 words); stride 228 = 4 mod 32, so that the 16-byte loads of a
// quarter warp (8 streams, same half) fall in 8 distinct bank groups.
#pragma once

#include "ranmar_device.cuh"

namespace ranmar {

constexpr int kPolyWords = 100;    // 6 x 16 coefficients, a_96, 3 pad
constexpr int kRingWords = 128;    // high product words / application ring
constexpr int kStreamWords = 228;  // per-stream slice stride (4 mod 32)
constexpr int kJumpStreamsPerWarp = 16;
constexpr int kPairXor = 16;       // the two lanes of a stream: L and L + 16
constexpr size_t kJumpSmemBytes = sizeof(uint32_t) * kStreamWords * kJumpStreamsPerWarp;
static_assert(kPolyWords + kRingWords <= kStreamWords, "slice");
static_assert(kStreamWords % 32 == 4, "bank spread");

struct ExpParams {
  uint32_t J[kMaxExpWords];  // partition mode: E = (k0 + i) * J
  uint32_t J_words;
  uint32_t flags;            // RANMAR_JUMP_REDUCE_PERIOD
  uint64_t k0;
};

struct Oct {
  uint32_t v[8];
};
struct Hex {
  uint32_t v[16];
};

__device__ __forceinline__ void lds4_to(uint32_t* d, const uint32_t* p) {
  const uint4 t = *reinterpret_cast<const uint4*>(p);
  d[0] = t.x;
  d[1] = t.y;
  d[2] = t.z;
  d[3] = t.w;
}
__device__ __forceinline__ Oct lds8(const uint32_t* p) {
  Oct o;
  lds4_to(o.v, p);
  lds4_to(o.v + 4, p + 4);
  return o;
}
__device__ __forceinline__ Hex lds16(const uint32_t* p) {
  Hex h;
#pragma unroll
  for (int q = 0; q < 4; ++q) lds4_to(h.v + 4 * q, p + 4 * q);
  return h;
}
__device__ __forceinline__ void st4(uint32_t* p, uint32_t x, uint32_t y, uint32_t z, uint32_t w) {
  *reinterpret_cast<uint4*>(p) = make_uint4(x, y, z, w);
}

// acc[p + q] += r[p] * col[q]: this lane's 8 rows x the block's 16 columns.
__device__ __forceinline__ void tile_mac(uint32_t (&acc)[23], const Oct& r, const Hex& col) {
#pragma unroll
  for (int p = 0; p < 8; ++p) {
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[p + q] += r.v[p] * col.v[q];
  }
}

// v[j] += h_{n+kOff} (kAdd) or -= (otherwise) for the lane's coefficients
// n = 16 kB + 8g + j, j < 8, with kLo <= n <= kHi; h_i = c_{97+i} = R[i+1].
// The 8 words come from 16-byte loads of R at the rounded-down index (Rg =
// R + 8g) and are selected at compile time.
template <int kB, int kOff, int kLo, int kHi, bool kAdd>
__device__ __forceinline__ void add_term(uint32_t (&v)[8], const uint32_t* __restrict__ Rg,
                                         unsigned g) {
  constexpr int n_first = 16 * kB, n_last = 16 * kB + 15;
  if constexpr (kHi >= n_first && kLo <= n_last) {
    constexpr int w = 16 * kB + kOff + 1;  // R index of j = 0 for g = 0
    constexpr int d = w & 3;
    static_assert(w - d >= 0 && w - d + 8 + 12 <= kRingWords, "R window");
    const uint32_t* p = Rg + (w - d);
    uint32_t t[12];
    lds4_to(t, p);
    lds4_to(t + 4, p + 4);
    if constexpr (d != 0) lds4_to(t + 8, p + 8);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int n0 = 16 * kB + j, n1 = n0 + 8;
      const bool ok0 = kLo <= n0 && n0 <= kHi;
      const bool ok1 = kLo <= n1 && n1 <= kHi;
      if (!ok0 && !ok1) continue;
      uint32_t x = t[d + j];
      if (ok0 != ok1) x = ((g != 0) ? ok1 : ok0) ? x : 0u;
      v[j] = kAdd ? v[j] + x : v[j] - x;
    }
  }
}

// Reduces the lane's 8 coefficients of the completed low product block kB
// (n = 16 kB + 8g + j) and writes them to a[n].
template <int kB>
__device__ __forceinline__ void reduce_low(uint32_t* __restrict__ a,
                                           const uint32_t* __restrict__ R, unsigned g,
                                           uint32_t (&v)[8]) {
  const uint32_t* Rg = R + 8 * g;
  add_term<kB, 0, 0, 95, true>(v, Rg, g);
  add_term<kB, 33, 0, 62, false>(v, Rg, g);
  add_term<kB, 66, 0, 29, true>(v, Rg, g);
  add_term<kB, -64, 64, 96, false>(v, Rg, g);
  add_term<kB, -31, 64, 96, true>(v, Rg, g);
  add_term<kB, 2, 64, 93, false>(v, Rg, g);
  uint32_t* dst = a + 16 * kB + 8 * g;
  st4(dst, v[0], v[1], v[2], v[3]);
  st4(dst + 4, v[4], v[5], v[6], v[7]);
}

__device__ __forceinline__ void reduce_low_dispatch(int B, uint32_t* __restrict__ a,
                                                    const uint32_t* __restrict__ R, unsigned g,
                                                    uint32_t (&v)[8]) {
  switch (B) {
    case 0: reduce_low<0>(a, R, g, v); break;
    case 1: reduce_low<1>(a, R, g, v); break;
    case 2: reduce_low<2>(a, R, g, v); break;
    case 3: reduce_low<3>(a, R, g, v); break;
    case 4: reduce_low<4>(a, R, g, v); break;
    default: reduce_low<5>(a, R, g, v); break;
  }
}

// a = a b mod phi in place (b is not modified), with the lanes g = 0, 1 of
// the pair cooperating.  `mask` holds the lanes taking part (both lanes of
// every participating pair).
__device__ __forceinline__ void product_reduce_pair(uint32_t* __restrict__ a,
                                                    const uint32_t* __restrict__ b,
                                                    uint32_t* __restrict__ R, unsigned g,
                                                    unsigned mask) {
  const uint32_t* arow = a + 8 * g;
  const uint32_t a96 = a[96];
  const uint32_t b96 = b[96];
  if (g == 0) R[96] = a96 * b96;  // c_192
  uint32_t pend[8];  // low half of the previous anti-diagonal
#pragma unroll
  for (int k = 0; k < 8; ++k) pend[k] = 0;
#pragma unroll 1
  for (int s = 10; s >= 0; --s) {
    uint32_t acc[23];
#pragma unroll
    for (int r = 0; r < 23; ++r) acc[r] = 0;
    const int ilo = s > 5 ? s - 5 : 0;
    const int iend = (s < 5 ? s : 5) + 1;
    Oct r0 = lds8(arow + 16 * ilo), r1;
    Hex c0 = lds16(b + 16 * (s - ilo)), c1;
    int I = ilo;
#pragma unroll 1
    for (; I + 1 < iend; I += 2) {  // operands one tile ahead, ping-pong
      r1 = lds8(arow + 16 * (I + 1));
      c1 = lds16(b + 16 * (s - I - 1));
      tile_mac(acc, r0, c0);
      if (I + 2 < iend) {
        r0 = lds8(arow + 16 * (I + 2));
        c0 = lds16(b + 16 * (s - I - 2));
      }
      tile_mac(acc, r1, c1);
    }
    if (I < iend) tile_mac(acc, r0, c0);

    // Lane g holds outputs 16s + 8g + r, r < 23.  Block s+1 (16s+16 ..
    // 16s+31): lane 0 takes 16..23 (its own 16..22 and lane 1's 16..23),
    // lane 1 takes 24..31 (its own only).  The low half of anti-diagonal s
    // stays pending for block s: lane 0 holds 0..7 (its own only), lane 1
    // 8..15 (its own and lane 0's).  So each lane sends its accumulators
    // 8..15 to the other.
    uint32_t out[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const uint32_t recv = __shfl_xor_sync(mask, acc[8 + k], kPairXor);
      out[k] = (k < 7 ? acc[16 + k] : 0u) + pend[k] + (g ? 0u : recv);
      pend[k] = acc[k] + (g ? recv : 0u);
    }
    const int B = s + 1;
    if (B >= 6) {
      // rank-1 part: c_k += a_96 b_{k-96} + b_96 a_{k-96}, k = 16B + 8g + j
      const int i0 = 16 * (B - 6) + 8 * static_cast<int>(g);
      const Oct x = lds8(a + i0);
      const Oct y = lds8(b + i0);
#pragma unroll
      for (int j = 0; j < 8; ++j) out[j] += a96 * y.v[j] + b96 * x.v[j];
      st4(R + i0, out[0], out[1], out[2], out[3]);
      st4(R + i0 + 4, out[4], out[5], out[6], out[7]);
      // coefficient 96: c_96 + h_65 - h_32 (h_j = c_{97+j} = R[j+1])
      if (B == 6 && g == 0) a[96] = out[0] + R[66] - R[33];
    } else {
      reduce_low_dispatch(B, a, R, g, out);
    }
    __syncwarp(mask);
  }
  reduce_low<0>(a, R, g, pend);
  __syncwarp(mask);
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

// kBits (<= 32) bits of E starting at bit p (p >= 0).
template <int kBits>
__device__ __forceinline__ uint32_t exp_bits(const uint32_t (&E)[kMaxExpWords], int p) {
  const int w = p >> 5, sh = p & 31;
  const uint32_t lo = exp_word(E, w);
  const uint32_t hi = (w + 1 < kMaxExpWords) ? exp_word(E, w + 1) : 0u;
  return __funnelshift_r(lo, hi, sh) & ((1u << kBits) - 1u);
}

// The leading (up to) kLeadBits bits v0 of an exponent whose bit length is
// at most L, and the bit below them (-1 when they are all of E): the
// square-and-multiply starts from t^v0 mod phi.
constexpr int kLeadBits = 10;
__device__ __forceinline__ uint32_t exp_lead(const uint32_t (&E)[kMaxExpWords], int L, int& p) {
  if (L <= kLeadBits) {
    p = -1;
    return E[0] & ((1u << kLeadBits) - 1u);
  }
  p = L - kLeadBits - 1;
  return exp_bits<kLeadBits>(E, L - kLeadBits);
}

// dst = src (1 - t^64) mod phi at n = first + kStep k < 97 (0 <= first <
// kStep; src and dst distinct, 97 words each).  t^64 src folds in closed
// form (t^97 = 1 - t^64): for n <= 63 its coefficient is src_{n+33} - [n <=
// 30] src_{n+66}, for n >= 64 it is src_{n-64} - src_{n-31} + [n <= 94]
// src_{n+2}.  With v0 = 97 q + r, t^v0 = t^r (t^97)^q = t^r (1 - t^64)^q mod
// phi.  Unrolled over k, so the loads are independent and every range test
// that holds for the whole of n's range kStep k .. kStep k + kStep - 1 folds
// at compile time.
template <int kStep>
__device__ __forceinline__ void mul_one_minus_t64(const uint32_t* __restrict__ src,
                                                  uint32_t* __restrict__ dst, int first) {
#pragma unroll
  for (int k = 0; k < (kR + kStep - 1) / kStep; ++k) {
    const int lo = kStep * k, hi = kStep * k + kStep - 1;   // n's range
    const int n = first + lo;
    if (hi >= kR && n >= kR) continue;
    uint32_t v = src[n];
    if (hi <= 63 || (lo <= 63 && n <= 63)) {
      v -= src[n + 33];
      if (hi <= 30 || (lo <= 30 && n <= 30)) v += src[n + 66];
    } else {
      v -= src[n - 64];
      v += src[n - 31];
      if (hi <= 94 || (lo <= 94 && n <= 94)) v -= src[n + 2];
    }
    dst[n] = v;
  }
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

// dst = x P(A) with P = a (97 coefficients), and the c / pos jump by E.
// The extended window X is consumed through the 128-word region R used as a
// ring: X(0..96) is the base state, X(q) = X(q-97) - X(q-33) beyond.  Round m
// (m < 3) handles output blocks K = 2m + g (outputs 16K .. 16K+15), whose
// windows are X(16K .. 16K+111): six 16x16 tiles plus the rank-1 column of
// a_96 (X(96+16K .. 111+16K), the last window block).  Between rounds 32 new
// words replace the 32 oldest: every lane reads the words its new ones
// depend on before any lane writes.  Output 96 is a plain dot product of a
// with X(96..192).
__device__ __forceinline__ void apply_pair(const ranmar_state_t* __restrict__ base,
                                           const uint32_t (&E)[kMaxExpWords], bool active,
                                           ranmar_state_t* __restrict__ dst,
                                           const uint32_t* __restrict__ a,
                                           uint32_t* __restrict__ R, unsigned g) {
  constexpr int kRM = kRingWords - 1;
  uint32_t* ring = R;
  const uint32_t* bx = base->x;  // 16-byte aligned (checked on the host)
  for (int q = static_cast<int>(g); q < 24; q += 2)
    reinterpret_cast<uint4*>(ring)[q] = reinterpret_cast<const uint4*>(bx)[q];
  if (g == 0) ring[96] = bx[96];
  __syncwarp();
  for (int q = kR + static_cast<int>(g); q < kRingWords; q += 2) ring[q] = ring[q - kR] - ring[q - kS];
  __syncwarp();

  const uint32_t b96 = a[96];
  uint32_t* ox = dst->x;
#pragma unroll 1
  for (int m = 0; m < 3; ++m) {
    const int K = 2 * m + static_cast<int>(g);
    uint32_t acc[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) acc[r] = 0;
    // six tiles, fully unrolled so that the sliding window (blocks I+K and
    // I+K+1 of X) and the coefficient blocks are renamed, not moved
    Hex w0 = lds16(ring + ((16 * K) & kRM));
#pragma unroll
    for (int I = 0; I < 6; ++I) {
      const Hex bb = lds16(a + 16 * I);
      const Hex w1 = lds16(ring + ((16 * (I + 1 + K)) & kRM));
#pragma unroll
      for (int p2 = 0; p2 < 16; ++p2) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
          const int idx = p2 + r;
          acc[r] += bb.v[p2] * (idx < 16 ? w0.v[idx] : w1.v[idx - 16]);
        }
      }
      w0 = w1;
    }
#pragma unroll
    for (int r = 0; r < 16; ++r) acc[r] += b96 * w0.v[r];
    if (active) {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        st4(ox + 16 * K + 4 * q, acc[4 * q] & kMask24, acc[4 * q + 1] & kMask24,
            acc[4 * q + 2] & kMask24, acc[4 * q + 3] & kMask24);
    }
    __syncwarp();
    if (m < 2) {
      // X(q) for q = 32m + 128 + 16g + j, j < 16, into the slots of X(q - 128)
      uint32_t nx[16];
      const int q0 = 32 * m + kRingWords + 16 * static_cast<int>(g);
#pragma unroll
      for (int j = 0; j < 16; ++j)
        nx[j] = ring[(q0 + j - kR) & kRM] - ring[(q0 + j - kS) & kRM];
      __syncwarp();
#pragma unroll
      for (int q = 0; q < 4; ++q)
        st4(ring + ((q0 + 4 * q) & kRM), nx[4 * q], nx[4 * q + 1], nx[4 * q + 2], nx[4 * q + 3]);
      __syncwarp();
    }
  }
  // output 96 = sum_i a_i X(96 + i); the ring holds X(64..191), and
  // X(192) = X(95) - X(159).  Lane 0 takes blocks 0..2 and a_96, lane 1
  // blocks 3..5.
  uint32_t part = 0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int I = 3 * static_cast<int>(g) + i;
    const Hex bb = lds16(a + 16 * I);
    const Hex xx = lds16(ring + ((96 + 16 * I) & kRM));
#pragma unroll
    for (int p2 = 0; p2 < 16; ++p2) part += bb.v[p2] * xx.v[p2];
  }
  if (g == 0) part += b96 * (ring[95] - ring[159 & kRM]);
  part += __shfl_xor_sync(kFull, part, kPairXor);

  if (active && g == 0) {
    ox[96] = part & kMask24;
    const uint32_t e = exp_mod_m(E);
    // (c - e d) mod m = (c + (m - e) d) mod m, non-negative residue.
    const uint64_t cn =
        (static_cast<uint64_t>(base->c) + static_cast<uint64_t>(kModM - e) * kD) % kModM;
    dst->c = static_cast<uint32_t>(cn);
    dst->pos = base->pos + (static_cast<uint64_t>(E[1]) << 32 | E[0]);
  }
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

}  // namespace ranmar
