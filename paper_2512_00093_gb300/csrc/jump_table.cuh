// jump_table.cuh -- jump-ahead with a fixed-base power table.
//
// The base of the exponentiation is always t, so every power t^{d 2^{8j}}
// mod phi can be computed once and shared by all streams (fixed-base
// windowed exponentiation).  With E = sum_j d_j 2^{8j} (base-256 digits,
// j < 20 for E < 2^160):
//     t^E mod phi = prod_{j : d_j != 0} T[j][d_j]   (mod phi),
// where T[j][d] = t^{d 2^{8j}} mod phi.  The table depends on nothing but
// phi (not on the seed, J or k); it has 20 x 256 rows of 100 words (97
// coefficients, 3 zeros), about 2 MB, which stays in L2.  A stream then needs
// (number of nonzero digits - 1) general products instead of bitlen(E)
// squarings: one product for E = k 2^40 with k < 2^16, at most 19 for any
// 160-bit E.  The result P_E is the same polynomial the left-to-right
// square-and-multiply gives (it is unique), so the jumped states are
// bit-identical.  The table rows themselves are built by that
// square-and-multiply (poly_power_mirror), with the exponent d 2^{8j}.
//
// For the streams of one partition (E = kJ) a second table, of the powers of
// t^J (rows t^{d 2^{8j} J}, built from the first), lets the product run over
// the digits of k instead of those of kJ (jtable_build_kernel,
// jump_jtable_kernel).
#pragma once

#include "square_mirror.cuh"

namespace ranmar {

constexpr int kTabWindowBits = 8;
constexpr int kTabWindows = 32 * kMaxExpWords / kTabWindowBits;  // 20
constexpr int kTabDigits = 1 << kTabWindowBits;                  // 256
constexpr int kTabRows = kTabWindows * kTabDigits;               // 5120
constexpr int kTabRowWords = 100;                                // 97 + 3 zeros
constexpr size_t kTabBytes = sizeof(uint32_t) * kTabRowWords * kTabRows;
// Per-stream slice of the table jump: a (100 words) at 0, R at 100, the table
// row b (100 words) at 200.  A product reads R only up to word 99 and writes
// it only up to word 96, so b may start at R + 100; the application's
// 128-word ring overlaps the start of b, which it no longer needs.  300
// words, stride 324 = 4 mod 32 (16-byte loads of a quarter warp: 8 distinct
// groups).
constexpr int kTabRowOffset = kPolyWords + 100;
constexpr int kTabStreamWords = 324;
constexpr size_t kTabSmemBytes = sizeof(uint32_t) * kTabStreamWords * kJumpStreamsPerWarp;
static_assert(kTabRowOffset + kTabRowWords <= kTabStreamWords, "slice");
static_assert(kPolyWords + kRingWords <= kTabStreamWords, "slice");
static_assert(kTabStreamWords % 32 == 4, "bank spread");

// Row (j * 256 + d) = t^{d 2^{8j}} mod phi, canonical 24-bit coefficients
// 0..96, then zeros.
__global__ void __launch_bounds__(kMirThreads) table_build_kernel(uint32_t* __restrict__ table) {
  extern __shared__ __align__(16) uint32_t smem[];
  const unsigned lane = threadIdx.x & 31;
  const unsigned g = lane >> 4, slot = lane & 15, w = threadIdx.x >> 5;
  const int row = blockIdx.x * kJumpStreamsPerWarp + static_cast<int>(slot);
  const bool active = row < kTabRows;
  uint32_t* slice = smem + slot * kMirStreamWords;
  uint32_t E[kMaxExpWords];
#pragma unroll
  for (int w = 0; w < kMaxExpWords; ++w) E[w] = 0;
  if (active) {
    const int j = row / kTabDigits, d = row % kTabDigits;
    const int bit = kTabWindowBits * j;  // d * 2^bit, d < 256, bit + 8 <= 160
    const uint64_t v = static_cast<uint64_t>(d) << (bit & 31);
    const int w0 = bit >> 5;
    E[w0] = static_cast<uint32_t>(v);
    if (w0 + 1 < kMaxExpWords) E[w0 + 1] = static_cast<uint32_t>(v >> 32);
  }
  poly_power_mirror(E, active, slice, g, w);
  if (active && w == 0) {
    uint32_t* dst = table + static_cast<size_t>(row) * kTabRowWords;
    const uint32_t* a = slice + kMirA;
    for (int q = static_cast<int>(g); q < kTabRowWords; q += 2) dst[q] = q < kR ? (a[q] & kMask24) : 0u;
  }
}

__device__ __forceinline__ uint32_t exp_digit(const uint32_t (&E)[kMaxExpWords], int j) {
  return (exp_word(E, j >> 2) >> (8 * (j & 3))) & 0xFFu;
}

// Copies one 100-word table row (25 x 16 bytes) into shared memory.
__device__ __forceinline__ void copy_row(uint32_t* __restrict__ dst,
                                         const uint32_t* __restrict__ src, unsigned g) {
  const uint4* s4 = reinterpret_cast<const uint4*>(src);
  uint4* d4 = reinterpret_cast<uint4*>(dst);
  for (int q = static_cast<int>(g); q < kTabRowWords / 4; q += 2) d4[q] = __ldg(s4 + q);
}

// a = prod over the nonzero base-256 digits d_j of D of table row (j, d_j):
// P_D for the fixed-base table (rows t^{d 2^{8j}}), P_{D J} for a table of
// the powers of t^J (rows t^{d 2^{8j} J}).  All 32 lanes call it; `active`
// false for lanes without a stream.  Slice: a at 0, R at kPolyWords, the
// row b at kTabRowOffset.
__device__ __forceinline__ void table_poly_pair(const uint32_t* __restrict__ table,
                                                const uint32_t (&D)[kMaxExpWords], bool active,
                                                uint32_t* __restrict__ a, unsigned g) {
  uint32_t* R = a + kPolyWords;
  uint32_t* b = a + kTabRowOffset;
  // a = 1 (t^0); b is always a whole copied row
  for (int q = static_cast<int>(g); q < kPolyWords / 4; q += 2)
    reinterpret_cast<uint4*>(a)[q] = make_uint4(q == 0 ? 1u : 0u, 0u, 0u, 0u);
  __syncwarp();
  // digit positions up to the highest nonzero digit of the warp's exponents
  const int nbits = active ? exp_bitlen(D) : 0;
  const int nwin = (static_cast<int>(__reduce_max_sync(kFull, static_cast<unsigned>(nbits))) +
                    kTabWindowBits - 1) / kTabWindowBits;
  bool have = false;
#pragma unroll 1
  for (int j = 0; j < nwin; ++j) {
    const uint32_t d = active ? exp_digit(D, j) : 0u;
    const bool first = d != 0 && !have;
    const bool mul = d != 0 && have;
    const uint32_t* row = table + static_cast<size_t>(j * kTabDigits + d) * kTabRowWords;
    if (first) copy_row(a, row, g);
    if (mul) copy_row(b, row, g);
    const unsigned mmask = __ballot_sync(kFull, mul);
    __syncwarp();
    if (mul) product_reduce_pair(a, b, R, g, mmask);
    __syncwarp();
    have = have || d != 0;
  }
}

// dst = f^E(base) for the stream of this lane pair, P_E from the fixed-base
// table (of E, or of E reduced by the period of t when flagged).
__device__ __forceinline__ void table_jump_pair(const uint32_t* __restrict__ table,
                                                const ranmar_state_t* __restrict__ base,
                                                const uint32_t (&E)[kMaxExpWords],
                                                uint32_t flags, bool active,
                                                ranmar_state_t* __restrict__ dst,
                                                uint32_t* __restrict__ a, unsigned g) {
  uint32_t Ep[kMaxExpWords];
#pragma unroll
  for (int w = 0; w < kMaxExpWords; ++w) Ep[w] = E[w];
  if (flags & RANMAR_JUMP_REDUCE_PERIOD) reduce_period(Ep);
  table_poly_pair(table, Ep, active, a, g);
  apply_pair(base, E, active, dst, a, a + kPolyWords, g);
  __syncwarp();
}

// A table of the powers of t^J for one J (Sec. 1: the partition's start
// states are f^{kJ}(base), so P_{kJ} = prod over the base-256 digits d_j of k
// of t^{d_j 2^{8j} J}): rows (j, d) = t^{d 2^{8j} J} mod phi for j < windows,
// built from the fixed-base table.  Stream k then costs (nonzero digits of
// k) - 1 products instead of (nonzero digits of kJ) - 1: none for k < 256,
// at most one for k < 2^16, whatever the size of J.
__global__ void __launch_bounds__(32) jtable_build_kernel(const uint32_t* __restrict__ table,
                                                          ExpParams part, int windows,
                                                          uint32_t* __restrict__ jtable) {
  extern __shared__ __align__(16) uint32_t smem[];
  const unsigned lane = threadIdx.x & 31;
  const unsigned g = lane >> 4, slot = lane & 15;
  const int row = blockIdx.x * kJumpStreamsPerWarp + static_cast<int>(slot);
  const bool active = row < windows * kTabDigits;
  uint32_t* a = smem + slot * kTabStreamWords;
  uint32_t E[kMaxExpWords];
#pragma unroll
  for (int w = 0; w < kMaxExpWords; ++w) E[w] = 0;
  if (active) {
    // E = d 2^{8j} J: d 2^{(8j) mod 32} < 2^32 at word (8j) / 32
    const int j = row / kTabDigits, d = row % kTabDigits;
    exp_mul_add(E, part.J, static_cast<uint32_t>(d) << ((8 * j) & 31), (8 * j) >> 5);
  }
  table_poly_pair(table, E, active, a, g);
  if (active) {
    uint32_t* dst = jtable + static_cast<size_t>(row) * kTabRowWords;
    for (int q = static_cast<int>(g); q < kTabRowWords; q += 2) dst[q] = q < kR ? (a[q] & kMask24) : 0u;
  }
}

// Partition by a table of the powers of t^J: stream i of the call is
// k = k0 + i, P_{kJ} from the digits of k, c and pos from E = kJ.
__global__ void __launch_bounds__(32) jump_jtable_kernel(
    const uint32_t* __restrict__ jtable, const ranmar_state_t* __restrict__ d_base,
    ExpParams part, ranmar_state_t* __restrict__ d_out, uint64_t n) {
  extern __shared__ __align__(16) uint32_t smem[];
  const unsigned lane = threadIdx.x & 31;
  const unsigned g = lane >> 4, slot = lane & 15;
  uint32_t* a = smem + slot * kTabStreamWords;
  const uint64_t groups = (n + kJumpStreamsPerWarp - 1) / kJumpStreamsPerWarp;
#pragma unroll 1
  for (uint64_t grp = blockIdx.x; grp < groups; grp += gridDim.x) {
    const uint64_t i = grp * kJumpStreamsPerWarp + slot;
    const bool active = i < n;
    uint32_t E[kMaxExpWords], K[kMaxExpWords];
    load_exponent(E, 1, nullptr, 0, part, active ? i : 0);
    const uint64_t k = part.k0 + (active ? i : 0);
#pragma unroll
    for (int w = 0; w < kMaxExpWords; ++w) K[w] = 0;
    K[0] = static_cast<uint32_t>(k);
    K[1] = static_cast<uint32_t>(k >> 32);
    table_poly_pair(jtable, K, active, a, g);
    apply_pair(d_base, E, active, d_out + (active ? i : 0), a, a + kPolyWords, g);
    __syncwarp();
  }
}

// Same contract as jump_kernel (modes 0 and 1, optional destination
// indices), with P_E from the table.
__global__ void __launch_bounds__(32) jump_table_kernel(
    const uint32_t* __restrict__ table, const ranmar_state_t* __restrict__ d_base,
    uint64_t n_base, const uint32_t* __restrict__ d_base_idx,
    const uint32_t* __restrict__ d_exp, uint32_t exp_words, ExpParams part, int mode,
    ranmar_state_t* __restrict__ d_out, uint64_t n, uint32_t* status,
    const uint32_t* __restrict__ d_dst_idx, uint64_t n_dst) {
  extern __shared__ __align__(16) uint32_t smem[];
  const unsigned lane = threadIdx.x & 31;
  const unsigned g = lane >> 4, slot = lane & 15;
  uint32_t* a = smem + slot * kTabStreamWords;
  const uint64_t groups = (n + kJumpStreamsPerWarp - 1) / kJumpStreamsPerWarp;
  // grid-stride over groups of 16 streams (the grid may be smaller than the
  // work, e.g. to leave SM resources to a concurrent generation kernel)
#pragma unroll 1
  for (uint64_t grp = blockIdx.x; grp < groups; grp += gridDim.x) {
  const uint64_t i = grp * kJumpStreamsPerWarp + slot;

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

  table_jump_pair(table, base, E, part.flags, active, d_out + (active ? di : 0), a, g);
  }
}

}  // namespace ranmar
