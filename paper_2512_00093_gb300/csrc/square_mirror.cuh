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
// Mapping: a CTA of two warps takes 16 streams; in each warp lanes L and
// L + 16 are the pair of stream L.  The two warps share each stream's work
// (different output blocks, then different reduction blocks), so a batch
// of n streams runs on n/8 warps.
//
// All arithmetic is 32-bit and wraps mod 2^32, which is exact mod 2^24;
// words are masked to 24 bits only when a result leaves the kernel.
//
// Shared memory per stream (words): A (100: x_0..x_96, pad), Bv (100: the
// reversed copy), C (96), Hr (96), c_96 and the application's four partial
// sums; stride 420 = 4 mod 32, so that the 16-byte accesses of a quarter warp
// (8 streams) fall in distinct bank groups.  The application that follows
// (apply_mirror, all four threads of a stream) builds its window X(0..192)
// over C/Hr.
#pragma once

#include "jump.cuh"

namespace ranmar {

constexpr int kMirA = 0;
constexpr int kMirB = 100;
constexpr int kMirC = 200;
constexpr int kMirH = 296;
constexpr int kMirC96 = 392;          // c_96, handed from warp 0 to warp 1
constexpr int kMirP96 = 396;          // the application's four partial sums of output 96
constexpr int kMirStreamWords = 420;
constexpr int kMirWarps = 2;          // warps per CTA, sharing its 16 streams
constexpr int kMirThreads = 32 * kMirWarps;
constexpr size_t kMirSmemBytes = sizeof(uint32_t) * kMirStreamWords * kJumpStreamsPerWarp;
static_assert(kMirH + 96 <= kMirC96 && kMirC96 < kMirP96 && kMirP96 + 4 <= kMirStreamWords,
              "slice");
static_assert(kMirC + 193 <= kMirP96, "the application's window X(0..192) after C");
static_assert(kMirStreamWords % 32 == 4, "bank spread");
static_assert(kMirB % 4 == 0 && kMirC % 4 == 0 && kMirH % 4 == 0, "16-byte alignment");

// One full chunk of output block m: acc[r] += sum_{u<8} x_{8c+u} w[r-u+8]
// for r = 0..15, with w[k] = x_{16m-8c-8+k} (24 words as three octets:
// w[0..7] = lo, w[8..15] = mid, w[16..23] = hi); all its terms have i < j.
// 128 multiply-adds; each accumulator is updated every 16.
__device__ __forceinline__ void mir_para(uint32_t (&acc)[16], const Oct& x, const Oct& lo,
                                         const Oct& mid, const Oct& hi) {
#pragma unroll
  for (int u = 0; u < 8; ++u) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int k = r - u + 8;  // 1 .. 23
      const uint32_t w = k < 8 ? lo.v[k] : (k < 16 ? mid.v[k - 8] : hi.v[k - 16]);
      acc[r] += x.v[u] * w;
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

// acc[r] += sum over the chunks c = 0 .. nch-1 of sum_{u<8} x_{8c+u}
// y_{16m+r-8c-u} (part of output block m of x y).  The caller passes only
// chunks whose every term has i < j, 1 <= 16m+r-8c-u <= 95: for a square,
// the chunks below the diagonal (nch = m).  Chunk c's window is the octets O(2m-c-1), O(2m-c), O(2m-c+1) of y (O(k) =
// y_{8k} .. y_{8k+7}), so the next chunk needs one new octet: four octet
// registers rotate (period four, the loop unrolled by four) and each chunk
// loads the next chunk's new octet and x octet O(c+1) while it multiplies.
__device__ __forceinline__ void mir_chunks(uint32_t (&acc)[16], const uint32_t* __restrict__ X,
                                           const uint32_t* __restrict__ Y, int m, int nch) {
  if (nch <= 0) return;
  const uint32_t* ob = Y + 16 * m - 8;   // O_y(2m-1-c) = ob - 8c
  Oct w0 = lds8(ob), w1 = lds8(ob + 8), w2 = lds8(ob + 16), w3;
  Oct x0 = lds8(X), x1;
#pragma unroll 1
  for (int c = 0; c < nch; c += 4) {
    if (c + 1 < nch) {
      w3 = lds8(ob - 8 * (c + 1));
      x1 = lds8(X + 8 * (c + 1));
    }
    mir_para(acc, x0, w0, w1, w2);
    if (c + 1 >= nch) break;
    if (c + 2 < nch) {
      w2 = lds8(ob - 8 * (c + 2));
      x0 = lds8(X + 8 * (c + 2));
    }
    mir_para(acc, x1, w3, w0, w1);
    if (c + 2 >= nch) break;
    if (c + 3 < nch) {
      w1 = lds8(ob - 8 * (c + 3));
      x1 = lds8(X + 8 * (c + 3));
    }
    mir_para(acc, x0, w2, w3, w0);
    if (c + 3 >= nch) break;
    if (c + 4 < nch) {
      w0 = lds8(ob - 8 * (c + 4));
      x0 = lds8(X + 8 * (c + 4));
    }
    mir_para(acc, x1, w1, w2, w3);
  }
}

// a_47 of the reduced square (the word below block 3), for warp 1's lane 0
// at its first block: c_47 + h_47 - h_80 (the other terms of the gather do
// not reach n = 47).
__device__ __forceinline__ uint32_t mir_a47(const uint32_t* __restrict__ C,
                                            const uint32_t* __restrict__ Hr) {
  return C[47] + Hr[95 - 47] - Hr[95 - 80];
}

// a_63 of the reduced square (the word below block 4): c_63 + h_63 (63 is
// past the range of the h_{n+33} term and below that of the n >= 64 terms).
__device__ __forceinline__ uint32_t mir_a63(const uint32_t* __restrict__ C,
                                            const uint32_t* __restrict__ Hr) {
  return C[63] + Hr[95 - 63];
}

// a_31 (the word below block 2): c_31 + h_31 - h_64 (31 > 29: no h_{n+66}).
__device__ __forceinline__ uint32_t mir_a31(const uint32_t* __restrict__ C,
                                            const uint32_t* __restrict__ Hr) {
  return C[31] + Hr[95 - 31] - Hr[95 - 64];
}

// Warp 0 reduces blocks 0 .. kMirGatherSplit-1, warp 1 the rest (3 measured
// fastest; 2 and 4 took 1.5-2% longer at 16,384 large jumps).
constexpr int kMirGatherSplit = 3;

// After both warps have stored their blocks of c (C[n] = c_n, Hr[k] =
// c_{192-k}, *c96 = c_96): a CTA barrier, the closed-form reduction mod phi
// with the shift by t^shift (warp 0 blocks 0..kMirGatherSplit-1, warp 1 the
// rest and position 96), written forward to A and reversed to Bv, and a
// second barrier.
__device__ __forceinline__ void mir_reduce(uint32_t* __restrict__ A, uint32_t* __restrict__ Bv,
                                           const uint32_t* __restrict__ C,
                                           const uint32_t* __restrict__ Hr,
                                           const uint32_t* __restrict__ c96, uint32_t shift,
                                           unsigned g, unsigned w) {
  __syncthreads();
  const uint32_t a96 = *c96 + Hr[95 - 65] - Hr[95 - 32];
  uint32_t last = 0;
  constexpr int kSplit = kMirGatherSplit;
  static_assert(kSplit >= 2 && kSplit <= 4, "gather split");
  if (w == 0) {
    uint32_t prev7 = 0;                      // a_{-1} = 0 below block 0
    mir_gather<0>(A, Bv, C, Hr, g, shift, a96, prev7, last);
    mir_gather<1>(A, Bv, C, Hr, g, shift, a96, prev7, last);
    if constexpr (kSplit > 2) mir_gather<2>(A, Bv, C, Hr, g, shift, a96, prev7, last);
    if constexpr (kSplit > 3) mir_gather<3>(A, Bv, C, Hr, g, shift, a96, prev7, last);
  } else {
    // lane 1 hands lane 0 the word below warp 1's first block
    uint32_t prev7 = 0;
    if (g) prev7 = kSplit == 2 ? mir_a31(C, Hr) : kSplit == 3 ? mir_a47(C, Hr) : mir_a63(C, Hr);
    if constexpr (kSplit <= 2) mir_gather<2>(A, Bv, C, Hr, g, shift, a96, prev7, last);
    if constexpr (kSplit <= 3) mir_gather<3>(A, Bv, C, Hr, g, shift, a96, prev7, last);
    mir_gather<4>(A, Bv, C, Hr, g, shift, a96, prev7, last);
    mir_gather<5>(A, Bv, C, Hr, g, shift, a96, prev7, last);
    if (g) {  // position 96: the old a_95 (lane 1's v[7] of block 5) or a_96
      const uint32_t w96 = shift ? last : a96;
      A[96] = w96;
      Bv[0] = w96;
    }
  }
  __syncthreads();
}

// x = x^2 t^shift mod phi in place (A forward, Bv reversed).  Both warps of
// the CTA call it for the same 16 streams (lanes g = 0, 1 of each pair in
// each warp): warp 0 forms output blocks 5 and 3 of each lane's half and
// c_96, warp 1 blocks 4, 2, 1 and 0 (1,216 and 1,184 multiply-adds per
// lane); after a CTA barrier warp 0 reduces blocks 0..2 and warp 1 blocks
// 3..5 and position 96; a second barrier ends the squaring.
__device__ __forceinline__ void square_mirror_pair(uint32_t* __restrict__ slice, uint32_t shift,
                                                   unsigned g, unsigned w) {
  uint32_t* A = slice + kMirA;
  uint32_t* Bv = slice + kMirB;
  uint32_t* C = slice + kMirC;
  uint32_t* Hr = slice + kMirH;
  const uint32_t* X = g ? Bv : A;
  uint32_t* dst = g ? Hr : C;
  if (w == 0) {
    // c_96 = 2 sum_{i<48} x_i x_{96-i} + x_48^2: lane g takes i = 24g ..
    // 24g+23 of its own copy (for lane 1, xr_i xr_{96-i} = x_{96-i} x_i).
    uint32_t pq[4] = {0u, 0u, 0u, 0u};      // four independent chains
    const uint32_t* lo = X + 24 * g;        // x_{24g + i}
    const uint32_t* hi = X + 72 - 24 * g;   // hi[k] = x_{72 - 24g + k}; x_{96-24g-i} = hi[24 - i]
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      uint32_t l4[4], h4[4], h5[4];
      lds4_to(l4, lo + 4 * q);
      lds4_to(h4, hi + 20 - 4 * q);       // hi[20-4q .. 23-4q]
      lds4_to(h5, hi + 24 - 4 * q);       // hi[24-4q .. 27-4q]
      // i = 4q + u: x_{96-24g-i} = hi[24 - 4q - u]
      pq[0] += l4[0] * h5[0];
      pq[1] += l4[1] * h4[3];
      pq[2] += l4[2] * h4[2];
      pq[3] += l4[3] * h4[1];
    }
    const uint32_t part = (pq[0] + pq[1]) + (pq[2] + pq[3]);
    const uint32_t x48 = X[48];             // x_48 (the same word in both copies)
    const uint32_t c96 = 2u * (part + __shfl_xor_sync(kFull, part, kPairXor)) + x48 * x48;
    if (g == 0) slice[kMirC96] = c96;
  }
  // This warp's output blocks of the lane's half: block m = m full chunks
  // (c = 0 .. m-1, mir_chunks) then the last chunk (mir_tail).
  const uint32_t blocks = w ? 0x0124u : 0x35u;   // m, four bits each, first in the low bits
  const int nblocks = w ? 4 : 2;
  uint32_t acc[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) acc[r] = 0;
#pragma unroll 1
  for (int k = 0; k < nblocks; ++k) {
    const int m = static_cast<int>((blocks >> (4 * k)) & 15u);
    mir_chunks(acc, X, X, m, m);
    mir_tail(acc, lds16(X + 8 * m), dst, m);
  }
  mir_reduce(A, Bv, C, Hr, slice + kMirC96, shift, g, w);
}

// dst = x P(A) (Sec. 3.1: new state word k = sum_i p_i X(i + k), with
// X(0..96) the base state and X(q) = X(q - 97) - X(q - 33) beyond), c and pos
// by E (Sec. 3.2), shared by the four threads of the stream (t = 2w + g, both
// warps of the CTA call it: barriers inside).  The window X(0..192) is built
// once in W (193 words, the recurrence in three rounds whose inputs lie in
// the rounds before); worker t then forms the 8-output blocks B = t, t + 4,
// t + 8 (outputs 8B .. 8B+7: twelve chunks of 8 coefficients, each against
// two window octets, then the p_96 term) and a quarter of output 96, so the
// four workers each do 2,352 of the 9,409 multiply-adds.  P may hold
// unmasked words (arithmetic mod 2^32); outputs are masked to 24 bits.
__device__ __forceinline__ void apply_mirror(const ranmar_state_t* __restrict__ base,
                                             const uint32_t (&E)[kMaxExpWords], bool active,
                                             ranmar_state_t* __restrict__ dst,
                                             const uint32_t* __restrict__ P,
                                             uint32_t* __restrict__ W,
                                             uint32_t* __restrict__ part96, unsigned t) {
  const int ti = static_cast<int>(t);
  const uint4* bx = reinterpret_cast<const uint4*>(base->x);   // 16-byte aligned
  for (int q = ti; q < 24; q += 4) reinterpret_cast<uint4*>(W)[q] = bx[q];
  if (t == 0) W[96] = base->x[96];
  __syncthreads();
  for (int q = 97 + ti; q <= 129; q += 4) W[q] = W[q - kR] - W[q - kS];
  __syncthreads();
  for (int q = 130 + ti; q <= 162; q += 4) W[q] = W[q - kR] - W[q - kS];
  __syncthreads();
  for (int q = 163 + ti; q <= 192; q += 4) W[q] = W[q - kR] - W[q - kS];
  __syncthreads();
  // output 96 = sum_i p_i X(96 + i): worker t takes i = 24t .. 24t+23 (and 96)
  {
    uint32_t s96 = 0;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      uint32_t p4[4], x4[4];
      lds4_to(p4, P + 24 * ti + 4 * q);
      lds4_to(x4, W + 96 + 24 * ti + 4 * q);
#pragma unroll
      for (int u = 0; u < 4; ++u) s96 += p4[u] * x4[u];
    }
    if (t == 3) s96 += P[96] * W[192];
    part96[t] = s96;
  }
  const uint32_t p96 = P[96];
#pragma unroll 1
  for (int bi = 0; bi < 3; ++bi) {
    const int B = ti + 4 * bi;
    uint32_t acc[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) acc[r] = 0;
    Oct w0 = lds8(W + 8 * B);
#pragma unroll
    for (int c = 0; c < 12; ++c) {   // p_{8c+u} X(8B + 8c + u + r)
      const Oct w1 = lds8(W + 8 * (B + c + 1));
      const Oct pc = lds8(P + 8 * c);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
#pragma unroll
        for (int r = 0; r < 8; ++r) acc[r] += pc.v[u] * (r + u < 8 ? w0.v[r + u] : w1.v[r + u - 8]);
      }
      w0 = w1;
    }
    const Oct wl = lds8(W + 8 * B + 96);   // X(8B + 96 + r)
#pragma unroll
    for (int r = 0; r < 8; ++r) acc[r] += p96 * wl.v[r];
    if (active) {
      uint4* ox = reinterpret_cast<uint4*>(dst->x + 8 * B);
      ox[0] = make_uint4(acc[0] & kMask24, acc[1] & kMask24, acc[2] & kMask24, acc[3] & kMask24);
      ox[1] = make_uint4(acc[4] & kMask24, acc[5] & kMask24, acc[6] & kMask24, acc[7] & kMask24);
    }
  }
  __syncthreads();
  if (t == 0 && active) {
    dst->x[96] = (part96[0] + part96[1] + part96[2] + part96[3]) & kMask24;
    const uint32_t e = exp_mod_m(E);
    // (c - e d) mod m = (c + (m - e) d) mod m, non-negative residue.
    const uint64_t cn =
        (static_cast<uint64_t>(base->c) + static_cast<uint64_t>(kModM - e) * kD) % kModM;
    dst->c = static_cast<uint32_t>(cn);
    dst->pos = base->pos + (static_cast<uint64_t>(E[1]) << 32 | E[0]);
  }
}

// A = t^E mod phi (and Bv its reverse) for the stream of this lane pair by
// left-to-right square-and-multiply; both warps of the CTA call it together
// (the bit loop runs over the longest exponent of the CTA's 16 streams, the
// same for both warps).
__device__ __forceinline__ void poly_power_mirror(const uint32_t (&E)[kMaxExpWords], bool active,
                                                  uint32_t* __restrict__ slice, unsigned g,
                                                  unsigned w) {
  const int nb = active ? exp_bitlen(E) : 0;
  const int L = static_cast<int>(__reduce_max_sync(kFull, static_cast<unsigned>(nb)));
  // Leading (up to) ten bits v0 = 97 q + r: P = t^r (1 - t^64)^q, the q
  // factors applied by all four threads of the stream (T, in the C region,
  // and A take turns as source and destination: the result is in T for odd
  // q), then the forward and reversed copies.
  int p;
  uint32_t v0 = exp_lead(E, L, p);
  if (!active) v0 = 0;
  const uint32_t q = v0 / kR, r = v0 - q * kR;
  const int Q = static_cast<int>(__reduce_max_sync(kFull, q));   // the same in every warp
  for (int i = static_cast<int>(g + 2 * w); i < (kMirB + 100) / 4; i += 4)
    reinterpret_cast<uint4*>(slice)[i] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  if (g == 0 && w == 0) slice[kMirA + r] = 1u;
  __syncthreads();
  const int t = static_cast<int>(g + 2 * w);
  uint32_t* A = slice + kMirA;
  uint32_t* T = slice + kMirC;   // 97 words: C and the first word of Hr
#pragma unroll 1
  for (int s = 0; s < Q; ++s) {   // a stream whose q is reached sits out
    if (s < static_cast<int>(q)) mul_one_minus_t64<4>((s & 1) ? T : A, (s & 1) ? A : T, t);
    __syncthreads();
  }
  const uint32_t* res = (q & 1) ? T : A;
  for (int n = t; n < kR; n += 4) {
    const uint32_t v = res[n];
    A[n] = v;
    slice[kMirB + 96 - n] = v;
  }
  __syncthreads();
#pragma unroll 1
  for (; p >= 0; --p) {
    const uint32_t bit = active ? exp_bit(E, p) : 0u;
    square_mirror_pair(slice, bit, g, w);
  }
}

// Exponent of stream i: mode 0 reads it from d_exp, mode 1 forms (k0 + i) J
// (load_exponent in jump.cuh).  mode 0: base d_base[base_idx[i]]; mode 1:
// base d_base[0].  d_dst_idx (mode 0 only, may be null): stream i is written
// to d_out[d_dst_idx[i]] (index < n_dst) instead of d_out[i].
//
// dst = f^E(base) per stream: t^Ep mod phi by the square-and-multiply above
// (Ep = E, or E mod T for RANMAR_JUMP_REDUCE_PERIOD), the application x P(A)
// with its window in the C/Hr region, and c / pos by the full E.
__global__ void __launch_bounds__(kMirThreads, 7) jump_kernel(
    const ranmar_state_t* __restrict__ d_base, uint64_t n_base,
    const uint32_t* __restrict__ d_base_idx, const uint32_t* __restrict__ d_exp,
    uint32_t exp_words, ExpParams part, int mode, ranmar_state_t* __restrict__ d_out,
    uint64_t n, uint32_t* status, const uint32_t* __restrict__ d_dst_idx, uint64_t n_dst) {
  extern __shared__ __align__(16) uint32_t smem[];
  const unsigned lane = threadIdx.x & 31;
  const unsigned g = lane >> 4;
  const unsigned w = threadIdx.x >> 5;
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
  poly_power_mirror(Ep, active, slice, g, w);
  apply_mirror(base, E, active, d_out + (active ? di : 0), slice + kMirA, slice + kMirC,
               slice + kMirP96, 2 * w + g);
}

// P_{E_i} = t^{E_i} mod phi alone (the polynomial part of a jump, Sec. 3.1),
// by the same square-and-multiply: d_poly[i] = coefficients 0..96 (24-bit),
// then three zero words.
__global__ void __launch_bounds__(kMirThreads, 7) poly_power_kernel(const uint32_t* __restrict__ d_exp,
                                                           uint32_t exp_words,
                                                           uint32_t* __restrict__ d_poly,
                                                           uint64_t n) {
  extern __shared__ __align__(16) uint32_t smem[];
  const unsigned lane = threadIdx.x & 31;
  const unsigned g = lane >> 4;
  const unsigned w = threadIdx.x >> 5;
  const unsigned slot = lane & 15;
  const uint64_t i = static_cast<uint64_t>(blockIdx.x) * kJumpStreamsPerWarp + slot;
  uint32_t* slice = smem + slot * kMirStreamWords;
  const bool active = i < n;
  uint32_t E[kMaxExpWords];
  const ExpParams part{};
  load_exponent(E, 0, d_exp, active ? exp_words : 0, part, active ? i : 0);
  poly_power_mirror(E, active, slice, g, w);
  if (active && w == 0) {
    uint32_t* dst = d_poly + i * kPolyWords;
    const uint32_t* a = slice + kMirA;
    for (int q = static_cast<int>(g); q < kPolyWords; q += 2) dst[q] = q < kR ? (a[q] & kMask24) : 0u;
  }
}

}  // namespace ranmar
