// square_mirror.cuh -- the squaring step of the paper's left-to-right
// square-and-multiply (Sec. 3.1, Sec. 4: t^E mod phi by binary
// exponentiation), a lane pair per stream, with the symmetric square's
// exact multiply-add count.
//
// For x of degree <= 96, c = x^2 has 193 coefficients and
//     c_n = 2 sum_{i<j, i+j=n} x_i x_j + [n even] x_{n/2}^2,
// 97 * 98 / 2 = 4,753 multiply-adds in all.  Lane 0 of the pair forms the
// low half c_0 .. c_95 from x; lane 1 runs the SAME instructions on the
// reversed polynomial xr_i = x_{96-i}, whose square is c reversed, so its
// c'_0 .. c'_95 are c_192 .. c_97.  Each lane's half is 2,352 multiply-adds
// (x_96 takes no part in c_0 .. c_95, nor xr_96 = x_0 in c'_0 .. c'_95), and
// c_96 (49) is split between the lanes.
//
// A lane forms its outputs block by block (16 coefficients, output block m
// = coefficients 16m .. 16m+15, m = 0..5), output-stationary.  The cross
// terms x_i x_{n-i} (i < n - i) of block m are taken in chunks of 8 values
// of i: the chunks i = 8c .. 8c+7 for c < m lie wholly below the diagonal
// (i < j for every output of the block), each an 8 x 16 parallelogram of
// 128 multiply-adds with the same code; the chunk at i = 8m holds the
// diagonal and keeps its terms with u < r/2.  Cross terms are summed once,
// doubled, then the squares x_{8m+r/2}^2 are added at the even outputs.  No
// partial sum crosses lanes.  Lane 0 stores its half to C[n] = c_n and lane
// 1 to Hr[k] = c_{192-k} (the same store pattern), so that h_j = c_{97+j} =
// Hr[95 - j].
//
// Reduction mod phi = t^97 + t^64 - 1 (t^k = t^{k-97} - t^{k-33}) in
// closed form: for n <= 95
//     a_n = c_n + h_n - h_{n+33}[n<=62] + h_{n+66}[n<=29]
//               - h_{n-64}[n>=64] + h_{n-31}[n>=64] - h_{n+2}[64<=n<=93],
//     a_96 = c_96 + h_65 - h_32,
// lane g taking n = 16 kB + 8 g + j (j < 8) of each block kB.  A 1 bit of
// the exponent multiplies by t: each lane's 8 results move up one position
// (the word below them comes from the partner lane by one shuffle), and the
// word pushed to t^97 (the old a_96) folds back as +a_96 at t^0 and -a_96
// at t^64.  The new polynomial is written forward to A and reversed to Bv.
//
// All arithmetic is 32-bit and wraps mod 2^32, which is exact mod 2^24;
// words are masked to 24 bits only when a result leaves the kernel.
//
// Shared memory per stream (words): A (100: x_0..x_96, pad), Bv (100: the
// reversed copy), C (96), Hr (96); stride 420 = 4 mod 32, so that the
// 16-byte accesses of a quarter warp (8 streams) fall in distinct bank
// groups.  The application that follows uses C/Hr as its 128-word ring.
#pragma once

#include "jump.cuh"

namespace ranmar {

constexpr int kMirA = 0;
constexpr int kMirB = 100;
constexpr int kMirC = 200;
constexpr int kMirH = 296;
constexpr int kMirStreamWords = 420;
constexpr size_t kMirSmemBytes = sizeof(uint32_t) * kMirStreamWords * kJumpStreamsPerWarp;
static_assert(kMirH + 96 <= kMirStreamWords, "slice");
static_assert(kMirC + kRingWords <= kMirStreamWords, "ring inside the slice");
static_assert(kMirStreamWords % 32 == 4, "bank spread");
static_assert(kMirB % 4 == 0 && kMirC % 4 == 0 && kMirH % 4 == 0, "16-byte alignment");

// acc[r] += sum_{p+q=r} x_p y_q: the low triangle of a 16 x 16 block product.
__device__ __forceinline__ void mir_tri_low(uint32_t (&acc)[16], const Hex& x, const Hex& y) {
#pragma unroll
  for (int p = 0; p < 16; ++p) {
#pragma unroll
    for (int q = 0; q < 16 - p; ++q) acc[p + q] += x.v[p] * y.v[q];
  }
}
// acc[r] += sum_{p+q=r+16} x_p y_q: the high triangle.
__device__ __forceinline__ void mir_tri_high(uint32_t (&acc)[16], const Hex& x, const Hex& y) {
#pragma unroll
  for (int p = 1; p < 16; ++p) {
#pragma unroll
    for (int q = 16 - p; q < 16; ++q) acc[p + q - 16] += x.v[p] * y.v[q];
  }
}
// Cross terms p < q of x^2 with p + q <= 15.
__device__ __forceinline__ void mir_sym_low(uint32_t (&acc)[16], const Hex& x) {
#pragma unroll
  for (int p = 0; p < 8; ++p) {
#pragma unroll
    for (int q = p + 1; q < 16 - p; ++q) acc[p + q] += x.v[p] * x.v[q];
  }
}
// Cross terms p < q of x^2 with p + q >= 16.
__device__ __forceinline__ void mir_sym_high(uint32_t (&acc)[16], const Hex& x) {
#pragma unroll
  for (int p = 1; p < 16; ++p) {
#pragma unroll
    for (int q = (p + 1 > 16 - p ? p + 1 : 16 - p); q < 16; ++q) acc[p + q - 16] += x.v[p] * x.v[q];
  }
}

// One full chunk of output block m: acc[r] += sum_{u<8} x_{8c+u} w[r-u+8]
// for r = 0..15, with w[k] = x_{16m-8c-8+k} (24 words); all its terms have
// i < j.  128 multiply-adds; each accumulator is updated every 16.
__device__ __forceinline__ void mir_para(uint32_t (&acc)[16], const Oct& x, const Hex& w0,
                                         const Oct& w1) {
#pragma unroll
  for (int u = 0; u < 8; ++u) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int k = r - u + 8;  // 1 .. 23
      acc[r] += x.v[u] * (k < 16 ? w0.v[k] : w1.v[k - 16]);
    }
  }
}

// The last chunk of output block m and the block's end: t = x_{8m} ..
// x_{8m+15}; the terms with i < j are t_u t_{r-u} for u < r/2.  Then the
// cross terms are doubled, the squares t_{r/2}^2 added at even r, the block
// stored to dst + 16m and acc cleared.
__device__ __forceinline__ void mir_tail(uint32_t (&acc)[16], const Hex& t,
                                         uint32_t* __restrict__ dst, int m) {
#pragma unroll
  for (int u = 0; u < 8; ++u) {
#pragma unroll
    for (int r = 2 * u + 1; r < 16; ++r) acc[r] += t.v[u] * t.v[r - u];
  }
#pragma unroll
  for (int r = 0; r < 16; ++r) acc[r] += acc[r];
#pragma unroll
  for (int u = 0; u < 8; ++u) acc[2 * u] += t.v[u] * t.v[u];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    st4(dst + 16 * m + 4 * q, acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
    acc[4 * q] = acc[4 * q + 1] = acc[4 * q + 2] = acc[4 * q + 3] = 0u;
  }
}

// v[j] += / -= h_{n+kOff} for the lane's n = 16 kB + 8 g + j, j < 8, with
// kLo <= n <= kHi; h_i = Hr[95 - i].  The 8 words are read as 16-byte loads
// of Hr at a rounded-down index and selected (in reverse) at compile time.
template <int kB, int kOff, int kLo, int kHi, bool kAdd>
__device__ __forceinline__ void mir_term(uint32_t (&v)[8], const uint32_t* __restrict__ Hg,
                                         unsigned g) {
  constexpr int n_first = 16 * kB, n_last = 16 * kB + 15;
  if constexpr (kHi >= n_first && kLo <= n_last) {
    // j -> Hr[95 - kOff - 16 kB - 8 g - j]; the lane's lowest index is
    // w - 8 g with w = 88 - kOff - 16 kB, for j = 7.
    constexpr int w = 88 - kOff - 16 * kB;
    constexpr int d = ((w % 4) + 4) % 4;
    static_assert(w - d - 8 >= -kMirH && w - d + 12 <= kMirStreamWords - kMirH, "Hr window");
    const uint32_t* p = Hg + (w - d);
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
      uint32_t x = t[d + 7 - j];
      if (ok0 != ok1) x = ((g != 0) ? ok1 : ok0) ? x : 0u;
      v[j] = kAdd ? v[j] + x : v[j] - x;
    }
  }
}

// Block kB of the reduced square at positions n = 16 kB + 8 g + j, moved up
// by `shift`, written to A (forward) and Bv (reversed).  prev7 carries lane
// 1's v[7] of the previous block (the word lane 0 needs below its first).
template <int kB>
__device__ __forceinline__ void mir_gather(uint32_t* __restrict__ A, uint32_t* __restrict__ Bv,
                                           const uint32_t* __restrict__ C,
                                           const uint32_t* __restrict__ Hr, unsigned g,
                                           uint32_t shift, uint32_t a96, uint32_t& prev7,
                                           uint32_t& last) {
  uint32_t v[8];
  const Oct cn = lds8(C + 16 * kB + 8 * g);
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = cn.v[j];
  const uint32_t* Hg = Hr - 8 * static_cast<int>(g);
  mir_term<kB, 0, 0, 95, true>(v, Hg, g);
  mir_term<kB, 33, 0, 62, false>(v, Hg, g);
  mir_term<kB, 66, 0, 29, true>(v, Hg, g);
  mir_term<kB, -64, 64, 96, false>(v, Hg, g);
  mir_term<kB, -31, 64, 96, true>(v, Hg, g);
  mir_term<kB, 2, 64, 93, false>(v, Hg, g);
  // the word below this lane's first position: lane 0 gets lane 1's v[7] of
  // the previous block (0 below block 0), lane 1 gets lane 0's current v[7]
  const uint32_t recv = __shfl_xor_sync(kFull, g ? prev7 : v[7], kPairXor);
  if (g) prev7 = v[7];
  last = v[7];
  uint32_t w[8];
  w[0] = shift ? recv : v[0];
#pragma unroll
  for (int j = 1; j < 8; ++j) w[j] = shift ? v[j - 1] : v[j];
  if constexpr (kB == 0) w[0] += (shift && g == 0) ? a96 : 0u;   // t^97 -> +t^0
  if constexpr (kB == 4) w[0] -= (shift && g == 0) ? a96 : 0u;   // t^97 -> -t^64
  const int pos = 16 * kB + 8 * static_cast<int>(g);
  st4(A + pos, w[0], w[1], w[2], w[3]);
  st4(A + pos + 4, w[4], w[5], w[6], w[7]);
  // Bv[96 - pos - j] = w[j]: one aligned quad (j = 4..1) and four words
  uint32_t* br = Bv + 96 - pos;
  st4(br - 4, w[4], w[3], w[2], w[1]);
  br[0] = w[0];
  br[-5] = w[5];
  br[-6] = w[6];
  br[-7] = w[7];
}

// x = x^2 t^shift mod phi in place (A forward, Bv reversed), lanes g = 0, 1
// of the pair cooperating; all 32 lanes of the warp call it together.
__device__ __forceinline__ void square_mirror_pair(uint32_t* __restrict__ slice, uint32_t shift,
                                                   unsigned g) {
  uint32_t* A = slice + kMirA;
  uint32_t* Bv = slice + kMirB;
  uint32_t* C = slice + kMirC;
  uint32_t* Hr = slice + kMirH;
  const uint32_t* X = g ? Bv : A;
  uint32_t* dst = g ? Hr : C;
  // c_96 = 2 sum_{i<48} x_i x_{96-i} + x_48^2: lane g takes i = 24g .. 24g+23
  // of its own copy (for lane 1, xr_i xr_{96-i} = x_{96-i} x_i).
  uint32_t part = 0;
  {
    const uint32_t* lo = X + 24 * g;        // x_{24g + i}
    const uint32_t* hi = X + 72 - 24 * g;   // hi[k] = x_{72 - 24g + k}; x_{96-24g-i} = hi[24 - i]
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      uint32_t l4[4], h4[4], h5[4];
      lds4_to(l4, lo + 4 * q);
      lds4_to(h4, hi + 20 - 4 * q);       // hi[20-4q .. 23-4q]
      lds4_to(h5, hi + 24 - 4 * q);       // hi[24-4q .. 27-4q]
      // i = 4q + u: x_{96-24g-i} = hi[24 - 4q - u]
      part += l4[0] * h5[0];
      part += l4[1] * h4[3];
      part += l4[2] * h4[2];
      part += l4[3] * h4[1];
    }
  }
  // This lane's half, output block by output block: block m = m full chunks
  // (c = 0 .. m-1) then the last chunk.  Two operand sets (P, Q) alternate so
  // that the next chunk's words load while the current one multiplies.
  uint32_t acc[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) acc[r] = 0;
#pragma unroll 1
  for (int m = 0; m < 6; ++m) {
    const uint32_t* wb = X + 16 * m - 8;   // window base of chunk c: wb - 8c
    int c = 0;
    if (m > 0) {
      Oct xp = lds8(X), wp1;
      Hex wp0 = lds16(wb);
      wp1 = lds8(wb + 16);
#pragma unroll 1
      for (; c + 1 < m; c += 2) {
        const Oct xq = lds8(X + 8 * (c + 1));
        const Hex wq0 = lds16(wb - 8 * (c + 1));
        const Oct wq1 = lds8(wb - 8 * (c + 1) + 16);
        mir_para(acc, xp, wp0, wp1);
        if (c + 2 < m) {
          xp = lds8(X + 8 * (c + 2));
          wp0 = lds16(wb - 8 * (c + 2));
          wp1 = lds8(wb - 8 * (c + 2) + 16);
        }
        mir_para(acc, xq, wq0, wq1);
      }
      if (c < m) mir_para(acc, xp, wp0, wp1);
    }
    mir_tail(acc, lds16(X + 8 * m), dst, m);
  }
  const uint32_t x48 = X[48];               // x_48 (the same word in both copies)
  const uint32_t c96 =
      2u * (part + __shfl_xor_sync(kFull, part, kPairXor)) + x48 * x48;
  __syncwarp();
  const uint32_t a96 = c96 + Hr[95 - 65] - Hr[95 - 32];
  uint32_t prev7 = 0, last = 0;
  mir_gather<0>(A, Bv, C, Hr, g, shift, a96, prev7, last);
  mir_gather<1>(A, Bv, C, Hr, g, shift, a96, prev7, last);
  mir_gather<2>(A, Bv, C, Hr, g, shift, a96, prev7, last);
  mir_gather<3>(A, Bv, C, Hr, g, shift, a96, prev7, last);
  mir_gather<4>(A, Bv, C, Hr, g, shift, a96, prev7, last);
  mir_gather<5>(A, Bv, C, Hr, g, shift, a96, prev7, last);
  if (g) {  // position 96: the old a_95 (lane 1's v[7] of block 5) or a_96
    const uint32_t w96 = shift ? last : a96;
    A[96] = w96;
    Bv[0] = w96;
  }
  __syncwarp();
}

// A = t^E mod phi (and Bv its reverse) for the stream of this lane pair by
// left-to-right square-and-multiply; all 32 lanes of the warp call it
// together (the bit loop runs over the longest exponent of the warp).
__device__ __forceinline__ void poly_power_mirror(const uint32_t (&E)[kMaxExpWords], bool active,
                                                  uint32_t* __restrict__ slice, unsigned g) {
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
  for (int q = static_cast<int>(g); q < (kMirB + 100) / 4; q += 2)
    reinterpret_cast<uint4*>(slice)[q] = make_uint4(0u, 0u, 0u, 0u);
  __syncwarp();
  if (g == 0) {
    slice[kMirA + v0] = 1u;
    slice[kMirB + 96 - v0] = 1u;
  }
  __syncwarp();
#pragma unroll 1
  for (; p >= 0; --p) {
    const uint32_t bit = active ? exp_bit(E, p) : 0u;
    square_mirror_pair(slice, bit, g);
  }
}

// Exponent of stream i: mode 0 reads it from d_exp, mode 1 forms (k0 + i) J
// (load_exponent in jump.cuh).  mode 0: base d_base[base_idx[i]]; mode 1:
// base d_base[0].  d_dst_idx (mode 0 only, may be null): stream i is written
// to d_out[d_dst_idx[i]] (index < n_dst) instead of d_out[i].
//
// dst = f^E(base) per stream: t^Ep mod phi by the square-and-multiply above
// (Ep = E, or E mod T for RANMAR_JUMP_REDUCE_PERIOD), the application x P(A)
// through the C/Hr region as its ring, and c / pos by the full E.
__global__ void __launch_bounds__(32, 8) jump_kernel(
    const ranmar_state_t* __restrict__ d_base, uint64_t n_base,
    const uint32_t* __restrict__ d_base_idx, const uint32_t* __restrict__ d_exp,
    uint32_t exp_words, ExpParams part, int mode, ranmar_state_t* __restrict__ d_out,
    uint64_t n, uint32_t* status, const uint32_t* __restrict__ d_dst_idx, uint64_t n_dst) {
  extern __shared__ __align__(16) uint32_t smem[];
  const unsigned lane = threadIdx.x & 31;
  const unsigned g = lane >> 4;
  const unsigned slot = lane & 15;
  const uint64_t i = static_cast<uint64_t>(blockIdx.x) * kJumpStreamsPerWarp + slot;
  uint32_t* slice = smem + slot * kMirStreamWords;

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
  poly_power_mirror(Ep, active, slice, g);
  apply_pair(base, E, active, d_out + (active ? di : 0), slice + kMirA, slice + kMirC, g);
}

// P_{E_i} = t^{E_i} mod phi alone (the polynomial part of a jump, Sec. 3.1),
// by the same square-and-multiply: d_poly[i] = coefficients 0..96 (24-bit),
// then three zero words.
__global__ void __launch_bounds__(32, 8) poly_power_kernel(const uint32_t* __restrict__ d_exp,
                                                           uint32_t exp_words,
                                                           uint32_t* __restrict__ d_poly,
                                                           uint64_t n) {
  extern __shared__ __align__(16) uint32_t smem[];
  const unsigned lane = threadIdx.x & 31;
  const unsigned g = lane >> 4;
  const unsigned slot = lane & 15;
  const uint64_t i = static_cast<uint64_t>(blockIdx.x) * kJumpStreamsPerWarp + slot;
  uint32_t* slice = smem + slot * kMirStreamWords;
  const bool active = i < n;
  uint32_t E[kMaxExpWords];
  const ExpParams part{};
  load_exponent(E, 0, d_exp, active ? exp_words : 0, part, active ? i : 0);
  poly_power_mirror(E, active, slice, g);
  if (active) {
    uint32_t* dst = d_poly + i * kPolyWords;
    const uint32_t* a = slice + kMirA;
    for (int q = static_cast<int>(g); q < kPolyWords; q += 2) dst[q] = q < kR ? (a[q] & kMask24) : 0u;
  }
}

}  // namespace ranmar
