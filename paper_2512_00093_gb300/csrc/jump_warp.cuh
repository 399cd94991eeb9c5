// jump_warp.cuh -- table jump with a whole warp per stream, for small batches.
//
// The pair kernels (jump_table_kernel, jump_jtable_kernel) give each stream
// two lanes, which is efficient when the batch fills the GPU but leaves a
// batch of a few hundred streams (the first streams of a partition plan, the
// segment jumps of a serving iteration) on a handful of SMs for ~20 us.
// Here a warp owns one stream, with the same arithmetic (Sec. 3.1: P_E = the
// product of the table rows of the nonzero digits, then the new state word
// k = sum_i p_i x_{i+k}; Sec. 3.2: the c jump):
//   * product c = a b (193 coefficients): lane l forms c_n for n = 6l ..
//     6l+5 as sum_{i<97} a_i b_{n-i} over a copy of b with 96 zeros on
//     either side (no bounds tests; twice the multiply-adds of the
//     triangle), its six b words in registers sliding by one word per step
//     (one shared-memory load per six multiply-adds, the a_i broadcast four
//     at a time), c_192 = a_96 b_96;
//   * reduction mod phi: t^k = t^{k-97} - t^{k-33} for k from 192 down to 97
//     in three blocks [160, 192], [127, 159], [97, 126]: the targets of a
//     block lie below it and are distinct, so each block is one parallel
//     step;
//   * application: the window X(0..192) (X(0..96) = the state, then the
//     recurrence in three parallel rounds of at most 33 words), lane l forms
//     outputs 3l .. 3l+2 with a sliding window of three X words (one load
//     per three multiply-adds), and output 96 is a lane-strided dot product
//     summed over the warp.
// Arithmetic is mod 2^32 (exact mod 2^24), masked when stored.
#pragma once

#include "jump_table.cuh"

namespace ranmar {

constexpr int kWarpJumpWarps = 4;  // warps (streams in flight) per CTA
// Per-warp slice (words): a = P (100) at 0; b with zero margins at 100
// (b_0 at 196, 288 words: indices n - i in [-96, 191]); the product c
// (193) or the window X (193) at 388.
constexpr int kWjA = 0, kWjBz = 100, kWjB0 = kWjBz + 96, kWjC = 388, kWjWords = 584;
constexpr size_t kWarpJumpSmemBytes = sizeof(uint32_t) * kWjWords * kWarpJumpWarps;
static_assert(kWjB0 + 192 <= kWjC && kWjC + 196 <= kWjWords, "slice");
static_assert(kWjWords % 4 == 0 && kWjB0 % 4 == 0 && kWjC % 4 == 0, "16-byte rows");

// a = a b mod phi; b sits at bz + 96 with zeros at bz[0..95] and
// bz[193..287] (a table row's words 97..99 are zero); c is scratch.
// Lane l forms c_n for n = 6l .. 6l+5 with a sliding window: at step i its
// six registers hold b_{6l+j-i}, and step i+1 shifts them by one and loads
// the single new word b_{6l-i-1} (rows of b 24 bytes apart per lane: at most
// two lanes per bank).
__device__ __forceinline__ void poly_mulmod_warp(uint32_t* __restrict__ a,
                                                 const uint32_t* __restrict__ bz,
                                                 uint32_t* __restrict__ c, unsigned lane) {
  const uint32_t* b0 = bz + 96;
  const int n0 = 6 * static_cast<int>(lane);
  uint32_t acc[6], w[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    acc[j] = 0;
    w[j] = b0[n0 + j];
  }
#pragma unroll
  for (int i4 = 0; i4 < kR; i4 += 4) {
    const uint4 a4 = *reinterpret_cast<const uint4*>(a + i4);  // a[96..99] for the last
    const uint32_t av[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int i = i4 + e;
      if (i < kR) {
#pragma unroll
        for (int j = 0; j < 6; ++j) acc[j] += av[e] * w[j];
        if (i + 1 < kR) {
#pragma unroll
          for (int j = 5; j >= 1; --j) w[j] = w[j - 1];
          w[0] = b0[n0 - i - 1];
        }
      }
    }
  }
  __syncwarp();
#pragma unroll
  for (int j = 0; j < 6; ++j) c[n0 + j] = acc[j];
  if (lane == 0) c[192] = a[96] * b0[96];
  __syncwarp();
  // fold the coefficients 192 .. 97, one block of distinct targets at a time
#pragma unroll
  for (int blk = 0; blk < 3; ++blk) {
    const int hi = blk == 0 ? 192 : (blk == 1 ? 159 : 126);
    const int lo = blk == 0 ? 160 : (blk == 1 ? 127 : 97);
    for (int k = hi - static_cast<int>(lane); k >= lo; k -= 32) {
      const uint32_t v = c[k];
      c[k - kR] += v;
      c[k - kS] -= v;
    }
    __syncwarp();
  }
  for (int n = static_cast<int>(lane); n < kR; n += 32) a[n] = c[n];
  __syncwarp();
}

// The first window at or after j whose base-256 digit of D is nonzero
// (nwin when there is none).
__device__ __forceinline__ int next_digit(const uint32_t (&D)[kMaxExpWords], int j, int nwin) {
  while (j < nwin && exp_digit(D, j) == 0) ++j;
  return j;
}

// This lane's 16-byte part of table row (j, d_j) (lanes 0..24 of a row of
// 100 words), held in registers until it is stored.
__device__ __forceinline__ uint4 row_part(const uint32_t* __restrict__ table,
                                          const uint32_t (&D)[kMaxExpWords], int j,
                                          unsigned lane) {
  const uint32_t* row =
      table + static_cast<size_t>(j * kTabDigits + exp_digit(D, j)) * kTabRowWords;
  return lane < kTabRowWords / 4 ? __ldg(reinterpret_cast<const uint4*>(row) + lane)
                                 : make_uint4(0u, 0u, 0u, 0u);
}

// a = prod over the nonzero base-256 digits d_j of D of table row (j, d_j)
// (the fixed-base table, or a table of the powers of t^J); a = 1 for D = 0.
// D is the same in every lane.  The row of the next product is loaded into
// registers before the current product starts, so that its latency is
// spent under the product's multiply-adds instead of before them.
__device__ __forceinline__ void table_poly_warp(const uint32_t* __restrict__ table,
                                                const uint32_t (&D)[kMaxExpWords],
                                                uint32_t* __restrict__ s, unsigned lane) {
  uint32_t* a = s + kWjA;
  const int nwin = (exp_bitlen(D) + kTabWindowBits - 1) / kTabWindowBits;
  int j = next_digit(D, 0, nwin);
  if (j >= nwin) {
    for (int q = static_cast<int>(lane); q < kR; q += 32) a[q] = q == 0 ? 1u : 0u;
    __syncwarp();
    return;
  }
  uint4 v = row_part(table, D, j, lane);
  if (lane < kTabRowWords / 4) reinterpret_cast<uint4*>(a)[lane] = v;
  j = next_digit(D, j + 1, nwin);
  if (j < nwin) v = row_part(table, D, j, lane);
  __syncwarp();
#pragma unroll 1
  while (j < nwin) {
    if (lane < kTabRowWords / 4) reinterpret_cast<uint4*>(s + kWjB0)[lane] = v;
    __syncwarp();
    const int jn = next_digit(D, j + 1, nwin);
    if (jn < nwin) v = row_part(table, D, jn, lane);   // in flight during the product
    poly_mulmod_warp(a, s + kWjBz, s + kWjC, lane);
    j = jn;
  }
}

// dst = x P(A) with P = s[kWjA..], and the c / pos jump by E.
__device__ __forceinline__ void apply_warp(const ranmar_state_t* __restrict__ base,
                                           const uint32_t (&E)[kMaxExpWords],
                                           ranmar_state_t* __restrict__ dst,
                                           uint32_t* __restrict__ s, unsigned lane) {
  const uint32_t* a = s + kWjA;
  uint32_t* X = s + kWjC;
  // X(0..99) from the state's 25 leading 16-byte words (words 97..99 are c
  // and pos; the recurrence overwrites them)
  if (lane < 25)
    reinterpret_cast<uint4*>(X)[lane] = reinterpret_cast<const uint4*>(base->x)[lane];
  __syncwarp();
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const int qend = kR + kS * (r + 1) < 2 * kR - 1 ? kR + kS * (r + 1) : 2 * kR - 1;
    for (int q = kR + kS * r + static_cast<int>(lane); q < qend; q += 32)
      X[q] = X[q - kR] - X[q - kS];
    __syncwarp();
  }
  // lane l: outputs 3l .. 3l+2, window registers X(3l + j + i) slid by one
  // word per step (3l mod 32 is distinct over the warp: no bank conflicts)
  const int k0 = 3 * static_cast<int>(lane);
  uint32_t acc[3], w[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    acc[j] = 0;
    w[j] = X[k0 + j];
  }
#pragma unroll
  for (int i4 = 0; i4 < kR; i4 += 4) {
    const uint4 a4 = *reinterpret_cast<const uint4*>(a + i4);
    const uint32_t av[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int i = i4 + e;
      if (i < kR) {
#pragma unroll
        for (int j = 0; j < 3; ++j) acc[j] += av[e] * w[j];
        if (i + 1 < kR) {
          w[0] = w[1];
          w[1] = w[2];
          w[2] = X[k0 + 3 + i];
        }
      }
    }
  }
  uint32_t p96 = 0;
  for (int i = static_cast<int>(lane); i < kR; i += 32) p96 += a[i] * X[96 + i];
  p96 = __reduce_add_sync(kFull, p96);
  uint32_t* ox = dst->x;
#pragma unroll
  for (int j = 0; j < 3; ++j) ox[k0 + j] = acc[j] & kMask24;
  if (lane == 0) {
    ox[96] = p96 & kMask24;
    const uint32_t e = exp_mod_m(E);
    // (c - e d) mod m = (c + (m - e) d) mod m, non-negative residue.
    const uint64_t cn =
        (static_cast<uint64_t>(base->c) + static_cast<uint64_t>(kModM - e) * kD) % kModM;
    dst->c = static_cast<uint32_t>(cn);
    dst->pos = base->pos + (static_cast<uint64_t>(E[1]) << 32 | E[0]);
  }
  __syncwarp();
}

// Zero margins of the b copy (set once per warp slice; rows and squared
// copies land only at b_0 .. b_99).
__device__ __forceinline__ void zero_margins_warp(uint32_t* __restrict__ s, unsigned lane) {
  for (int q = static_cast<int>(lane); q < 96; q += 32) s[kWjBz + q] = 0u;
  for (int q = kWjB0 + 97 + static_cast<int>(lane); q < kWjC; q += 32) s[q] = 0u;
  __syncwarp();
}

// Same contract as jump_table_kernel, one warp per stream.
__global__ void __launch_bounds__(32 * kWarpJumpWarps) jump_table_warp_kernel(
    const uint32_t* __restrict__ table, const ranmar_state_t* __restrict__ d_base,
    uint64_t n_base, const uint32_t* __restrict__ d_base_idx,
    const uint32_t* __restrict__ d_exp, uint32_t exp_words, ExpParams part, int mode,
    ranmar_state_t* __restrict__ d_out, uint64_t n, uint32_t* status,
    const uint32_t* __restrict__ d_dst_idx, uint64_t n_dst) {
  extern __shared__ __align__(16) uint32_t smem[];
  const unsigned lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t* s = smem + w * kWjWords;
  zero_margins_warp(s, lane);
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * kWarpJumpWarps;
#pragma unroll 1
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * kWarpJumpWarps + w; i < n; i += stride) {
    uint32_t E[kMaxExpWords];
    load_exponent(E, mode, d_exp, exp_words, part, i);
    const ranmar_state_t* base = d_base;
    if (mode == 0) {
      const uint32_t bi = d_base_idx ? d_base_idx[i] : 0u;
      if (bi >= n_base) {
        if (lane == 0) flag_status(status, RANMAR_ST_BAD_INDEX);
        continue;
      }
      base = d_base + bi;
    }
    uint64_t di = i;
    if (d_dst_idx) {
      di = d_dst_idx[i];
      if (di >= n_dst) {
        if (lane == 0) flag_status(status, RANMAR_ST_BAD_INDEX);
        continue;
      }
    }
    uint32_t Ep[kMaxExpWords];
#pragma unroll
    for (int q = 0; q < kMaxExpWords; ++q) Ep[q] = E[q];
    if (part.flags & RANMAR_JUMP_REDUCE_PERIOD) reduce_period(Ep);
    table_poly_warp(table, Ep, s, lane);
    apply_warp(base, E, d_out + di, s, lane);
  }
}

// Same contract as jump_jtable_kernel (stream i: k = k0 + i, P_{kJ} from the
// digits of k in a table of the powers of t^J), one warp per stream.
__global__ void __launch_bounds__(32 * kWarpJumpWarps) jump_jtable_warp_kernel(
    const uint32_t* __restrict__ jtable, const ranmar_state_t* __restrict__ d_base,
    ExpParams part, ranmar_state_t* __restrict__ d_out, uint64_t n) {
  extern __shared__ __align__(16) uint32_t smem[];
  const unsigned lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t* s = smem + w * kWjWords;
  zero_margins_warp(s, lane);
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * kWarpJumpWarps;
#pragma unroll 1
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * kWarpJumpWarps + w; i < n; i += stride) {
    uint32_t E[kMaxExpWords], K[kMaxExpWords];
    load_exponent(E, 1, nullptr, 0, part, i);
    const uint64_t k = part.k0 + i;
#pragma unroll
    for (int q = 0; q < kMaxExpWords; ++q) K[q] = 0;
    K[0] = static_cast<uint32_t>(k);
    K[1] = static_cast<uint32_t>(k >> 32);
    table_poly_warp(jtable, K, s, lane);
    apply_warp(d_base, E, d_out + i, s, lane);
  }
}

// ---------------------------------------------------------------------------
// Square-and-multiply with a warp per stream (Sec. 3.1, the paper's method):
// the same left-to-right exponentiation as poly_power_mirror, each squaring
// a warp product of a with a copy of itself (the symmetric half is not used:
// in lockstep the lanes would wait for the longest triangle anyway), a 1 bit
// a shift by t with the fold t^97 = 1 - t^64.  For small batches only: per
// stream it executes about three times the instructions of the pair kernel,
// but one squaring of one stream takes ~1.1 us instead of the pair kernel's
// ~2.2 us (one CTA alone on an SM).

// a = a^2 t^bit mod phi
__device__ __forceinline__ void square_times_warp(uint32_t* __restrict__ s, uint32_t bit,
                                                  unsigned lane) {
  uint32_t* a = s + kWjA;
  for (int q = static_cast<int>(lane); q < kR; q += 32) s[kWjB0 + q] = a[q];
  __syncwarp();
  poly_mulmod_warp(a, s + kWjBz, s + kWjC, lane);
  if (bit) {
    // t a: a_q <- a_{q-1}, a_0 <- a_96, a_64 <- a_63 - a_96
    const uint32_t top = a[kR - 1];
    uint32_t v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int q = static_cast<int>(lane) + 32 * k;
      v[k] = q < kR ? (q == 0 ? top : a[q - 1]) : 0u;
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int q = static_cast<int>(lane) + 32 * k;
      if (q < kR) a[q] = q == kR - kS ? v[k] - top : v[k];
    }
    __syncwarp();
  }
}

// a = t^E mod phi (a in s[kWjA..]); E is the same in every lane.
__device__ __forceinline__ void poly_power_warp(const uint32_t (&E)[kMaxExpWords],
                                                uint32_t* __restrict__ s, unsigned lane) {
  const int L = exp_bitlen(E);
  // leading (up to) ten bits v0 = 97 q + r: t^r (1 - t^64)^q, the factors
  // applied between a and the product scratch
  int pbit;
  const uint32_t v0 = exp_lead(E, L, pbit);
  const int q = static_cast<int>(v0 / kR), r = static_cast<int>(v0) - q * kR;
  uint32_t* a = s + kWjA;
  uint32_t* T = s + kWjC;
  for (int i = static_cast<int>(lane); i < kR; i += 32) a[i] = i == r ? 1u : 0u;
  __syncwarp();
#pragma unroll 1
  for (int st = 0; st < q; ++st) {
    mul_one_minus_t64<32>((st & 1) ? T : a, (st & 1) ? a : T, static_cast<int>(lane));
    __syncwarp();
  }
  if (q & 1) {
    for (int i = static_cast<int>(lane); i < kR; i += 32) a[i] = T[i];
    __syncwarp();
  }
#pragma unroll 1
  for (; pbit >= 0; --pbit) square_times_warp(s, exp_bit(E, pbit), lane);
}

// Same contract as poly_power_kernel, one warp per exponent.
__global__ void __launch_bounds__(32 * kWarpJumpWarps) poly_power_warp_kernel(
    const uint32_t* __restrict__ d_exp, uint32_t exp_words, uint32_t* __restrict__ d_poly,
    uint64_t n) {
  extern __shared__ __align__(16) uint32_t smem[];
  const unsigned lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t* s = smem + w * kWjWords;
  zero_margins_warp(s, lane);
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * kWarpJumpWarps;
  const ExpParams part{};
#pragma unroll 1
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * kWarpJumpWarps + w; i < n; i += stride) {
    uint32_t E[kMaxExpWords];
    load_exponent(E, 0, d_exp, exp_words, part, i);
    poly_power_warp(E, s, lane);
    uint32_t* dst = d_poly + i * kPolyWords;
    for (int q = static_cast<int>(lane); q < kPolyWords; q += 32)
      dst[q] = q < kR ? (s[kWjA + q] & kMask24) : 0u;
    __syncwarp();
  }
}

// Same contract as jump_kernel (modes 0 and 1, base and destination
// indices, the period reduction), one warp per stream.
__global__ void __launch_bounds__(32 * kWarpJumpWarps) jump_warp_kernel(
    const ranmar_state_t* __restrict__ d_base, uint64_t n_base,
    const uint32_t* __restrict__ d_base_idx, const uint32_t* __restrict__ d_exp,
    uint32_t exp_words, ExpParams part, int mode, ranmar_state_t* __restrict__ d_out,
    uint64_t n, uint32_t* status, const uint32_t* __restrict__ d_dst_idx, uint64_t n_dst) {
  extern __shared__ __align__(16) uint32_t smem[];
  const unsigned lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t* s = smem + w * kWjWords;
  zero_margins_warp(s, lane);
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * kWarpJumpWarps;
#pragma unroll 1
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * kWarpJumpWarps + w; i < n; i += stride) {
    uint32_t E[kMaxExpWords];
    load_exponent(E, mode, d_exp, exp_words, part, i);
    const ranmar_state_t* base = d_base;
    if (mode == 0) {
      const uint32_t bi = d_base_idx ? d_base_idx[i] : 0u;
      if (bi >= n_base) {
        if (lane == 0) flag_status(status, RANMAR_ST_BAD_INDEX);
        continue;
      }
      base = d_base + bi;
    }
    uint64_t di = i;
    if (d_dst_idx) {
      di = d_dst_idx[i];
      if (di >= n_dst) {
        if (lane == 0) flag_status(status, RANMAR_ST_BAD_INDEX);
        continue;
      }
    }
    uint32_t Ep[kMaxExpWords];
#pragma unroll
    for (int q = 0; q < kMaxExpWords; ++q) Ep[q] = E[q];
    if (part.flags & RANMAR_JUMP_REDUCE_PERIOD) reduce_period(Ep);
    poly_power_warp(Ep, s, lane);
    apply_warp(base, E, d_out + di, s, lane);
  }
}

}  // namespace ranmar
