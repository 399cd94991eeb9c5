// jump.cuh -- batched jump-ahead (Sec. 3.1, Sec. 3.2).
//
// For each stream: P_E(t) = t^E mod phi(t), phi = t^97 + t^64 - 1 over
// Z/2^24, by left-to-right square-and-multiply (a 1 bit multiplies by t, a
// shift plus one fix-up); then the new state word k = sum_i b_i x_{i+k+1}
// (x extended by 96 steps of the recurrence), which equals the Horner form
// u P_E(A) of Sec. 3.1; then c_E = (c - E d) mod m (Sec. 3.2).
//
// Mapping: one stream per LANE, 32 streams per warp.  Every lane runs the
// same instruction stream on its own polynomial (no divergence), so the
// 97x97 products are register-blocked 8x8 tiles of 32-bit multiply-adds
// (mul.lo wraps mod 2^32, which is exact mod 2^24; masks only at the end).
// Each lane owns a private slice of shared memory: the polynomial a (104
// words, zero padded to 13 blocks of 8) and the 208-word product buffer,
// which is reused for the extended state window during the application.
// The slice stride is 324 words (= 4 mod 32) so that 16-byte loads of the
// 32 lanes fall in distinct bank groups.
#pragma once

#include "ranmar_device.cuh"

namespace ranmar {

constexpr int kPolyWords = 104;   // 13 blocks of 8 >= 97
constexpr int kProdWords = 208;   // 193 product words + tile overhang
constexpr int kLaneWords = 324;   // per-lane slice stride (4 mod 32)
constexpr int kJumpWarpsPerBlock = 1;
constexpr size_t kJumpSmemBytes =
    sizeof(uint32_t) * kLaneWords * 32 * kJumpWarpsPerBlock;
static_assert(kPolyWords + kProdWords <= kLaneWords, "slice");
static_assert(kLaneWords % 32 == 4, "bank spread");

struct ExpParams {
  uint32_t J[kMaxExpWords];  // partition mode: E = (k0 + i) * J
  uint32_t J_words;
  uint64_t k0;
};

__device__ __forceinline__ void load8(const uint32_t* p, uint32_t (&v)[8]) {
  const uint4 lo = *reinterpret_cast<const uint4*>(p);
  const uint4 hi = *reinterpret_cast<const uint4*>(p + 4);
  v[0] = lo.x; v[1] = lo.y; v[2] = lo.z; v[3] = lo.w;
  v[4] = hi.x; v[5] = hi.y; v[6] = hi.z; v[7] = hi.w;
}

__device__ __forceinline__ void store8(uint32_t* p, const uint32_t (&v)[8]) {
  *reinterpret_cast<uint4*>(p) = make_uint4(v[0], v[1], v[2], v[3]);
  *reinterpret_cast<uint4*>(p + 4) = make_uint4(v[4], v[5], v[6], v[7]);
}

// c[0..192] = a(t)^2, with the symmetric products of tiles (I, J), I <= J,
// summed along the anti-diagonal s = I + J (outputs 8s .. 8s+14) in
// registers; the upper 7 outputs carry into the next anti-diagonal.
__device__ __forceinline__ void poly_square(const uint32_t* __restrict__ a,
                                            uint32_t* __restrict__ c) {
  uint32_t carry[7];
#pragma unroll
  for (int r = 0; r < 7; ++r) carry[r] = 0;
#pragma unroll 1
  for (int s = 0; s <= 24; ++s) {
    uint32_t acc[15];
#pragma unroll
    for (int r = 0; r < 15; ++r) acc[r] = 0;
    const int ilo = s > 12 ? s - 12 : 0;
    const int ihi = s >> 1;
#pragma unroll 1
    for (int I = ilo; I <= ihi; ++I) {
      const int J = s - I;
      uint32_t ai[8], aj[8];
      load8(a + 8 * I, ai);
      if (I == J) {
#pragma unroll
        for (int p = 0; p < 8; ++p) {
          acc[2 * p] += ai[p] * ai[p];
          const uint32_t a2 = ai[p] << 1;
#pragma unroll
          for (int q = p + 1; q < 8; ++q) acc[p + q] += a2 * ai[q];
        }
      } else {
        load8(a + 8 * J, aj);
#pragma unroll
        for (int p = 0; p < 8; ++p) {
          const uint32_t a2 = ai[p] << 1;
#pragma unroll
          for (int q = 0; q < 8; ++q) acc[p + q] += a2 * aj[q];
        }
      }
    }
    uint32_t lo[8];
#pragma unroll
    for (int r = 0; r < 7; ++r) lo[r] = acc[r] + carry[r];
    lo[7] = acc[7];
    store8(c + 8 * s, lo);
#pragma unroll
    for (int r = 0; r < 7; ++r) carry[r] = acc[8 + r];
  }
}

// a = (c mod phi) * t^shift, shift in {0, 1}; c holds 193 words on entry.
// t^k = t^(k-97) - t^(k-33) for k >= 97, applied from the top.
__device__ __forceinline__ void poly_reduce_into(uint32_t* __restrict__ c,
                                                 uint32_t* __restrict__ a, uint32_t shift) {
#pragma unroll 4
  for (int k = 2 * kR - 2; k >= kR; --k) {
    const uint32_t h = c[k];
    c[k - kR] += h;
    c[k - kS] -= h;
  }
  // Multiplying by t moves word n to n+1; word 97 then folds back as
  // t^97 = 1 - t^64.
#pragma unroll 4
  for (int n = 0; n < kR; ++n) a[n + shift] = c[n];
  if (shift) {
    const uint32_t top = a[kR];
    a[0] = top;
    a[64] -= top;
    a[kR] = 0;
  }
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
__device__ __forceinline__ void exp_mul_add(uint32_t (&E)[kMaxExpWords],
                                            const uint32_t* J, uint32_t m, int shift) {
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

// state_out = f^E(base) for one lane's stream; all lanes of the warp call
// it together (the bit loop is warp-uniform).
__device__ __forceinline__ void jump_one(const ranmar_state_t* __restrict__ base,
                                         const uint32_t (&E)[kMaxExpWords], bool active,
                                         ranmar_state_t* __restrict__ dst,
                                         uint32_t* __restrict__ a, uint32_t* __restrict__ c) {
  const int nb = active ? exp_bitlen(E) : 0;
  const int L = __reduce_max_sync(kFull, static_cast<unsigned>(nb));

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
#pragma unroll 4
  for (int n = 0; n < kPolyWords; ++n) a[n] = 0;
  a[v0] = 1;

#pragma unroll 1
  for (; p >= 0; --p) {
    const uint32_t bit = active ? exp_bit(E, p) : 0u;
    poly_square(a, c);
    poly_reduce_into(c, a, bit);
  }

  // Application: X(0..96) = base x, X(97..192) by the recurrence, zero pad.
  uint32_t* X = c;
  const uint32_t* bx = base->x;
#pragma unroll 4
  for (int q = 0; q < kR; ++q) X[q] = bx[q];
#pragma unroll 4
  for (int q = kR; q < 2 * kR - 1; ++q) X[q] = X[q - kR] - X[q - kS];
#pragma unroll
  for (int q = 2 * kR - 1; q < kProdWords; ++q) X[q] = 0;

  uint32_t* ox = dst->x;
#pragma unroll 1
  for (int K = 0; K < 13; ++K) {
    uint32_t acc[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) acc[r] = 0;
#pragma unroll 1
    for (int I = 0; I < 13; ++I) {
      uint32_t b[8], w0[8], w1[8];
      load8(a + 8 * I, b);
      load8(X + 8 * (I + K), w0);
      load8(X + 8 * (I + K) + 8, w1);
#pragma unroll
      for (int p2 = 0; p2 < 8; ++p2) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const int idx = p2 + r;
          const uint32_t xv = idx < 8 ? w0[idx & 7] : w1[idx & 7];
          acc[r] += b[p2] * xv;
        }
      }
    }
    if (active) {
#pragma unroll
      for (int r = 0; r < 8; ++r)
        if (8 * K + r < kR) ox[8 * K + r] = acc[r] & kMask24;
    }
  }

  if (active) {
    const uint32_t e = exp_mod_m(E);
    // (c - e d) mod m = (c + (m - e) d) mod m, non-negative residue.
    const uint64_t cn =
        (static_cast<uint64_t>(base->c) + static_cast<uint64_t>(kModM - e) * kD) % kModM;
    dst->c = static_cast<uint32_t>(cn);
    dst->pos = base->pos + (static_cast<uint64_t>(E[1]) << 32 | E[0]);
  }
}

// mode 0: E_i from d_exp (exp_words per stream), base d_base[base_idx[i]].
// mode 1: E_i = (k0 + i) * J, base d_base[0].
__global__ void __launch_bounds__(32 * kJumpWarpsPerBlock) jump_kernel(
    const ranmar_state_t* __restrict__ d_base, uint64_t n_base,
    const uint32_t* __restrict__ d_base_idx, const uint32_t* __restrict__ d_exp,
    uint32_t exp_words, ExpParams part, int mode, ranmar_state_t* __restrict__ d_out,
    uint64_t n, uint32_t* status) {
  extern __shared__ __align__(16) uint32_t smem[];
  const unsigned lane = threadIdx.x & 31;
  const uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  uint32_t* slice = smem + threadIdx.x * kLaneWords;
  uint32_t* a = slice;
  uint32_t* c = slice + kPolyWords;
  (void)lane;

  bool active = i < n;
  uint32_t E[kMaxExpWords];
#pragma unroll
  for (int w = 0; w < kMaxExpWords; ++w) E[w] = 0;
  const ranmar_state_t* base = d_base;
  if (active) {
    if (mode == 0) {
      const uint32_t* ew = d_exp + i * exp_words;
#pragma unroll
      for (int w = 0; w < kMaxExpWords; ++w)
        if (w < static_cast<int>(exp_words)) E[w] = ew[w];
      const uint32_t bi = d_base_idx ? d_base_idx[i] : 0u;
      if (bi >= n_base) {
        flag_status(status, RANMAR_ST_BAD_INDEX);
        active = false;
      } else {
        base = d_base + bi;
      }
    } else {
      const uint64_t k = part.k0 + i;
      exp_mul_add(E, part.J, static_cast<uint32_t>(k), 0);
      exp_mul_add(E, part.J, static_cast<uint32_t>(k >> 32), 1);
    }
  }
  jump_one(base, E, active, d_out + (active ? i : 0), a, c);
}

}  // namespace ranmar
