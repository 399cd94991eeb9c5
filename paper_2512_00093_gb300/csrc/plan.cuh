// plan.cuh -- stream partitioning (Sec. 1) by levels of jump matrices: one
// dense contraction per level.
//
// The x part of a jump is linear over Z/2^24 (x' = x A^E, Sec. 3.1), so a
// jump by a fixed E of many states is one matrix product X' = X M_E, where
// row i of the 97x97 matrix M_E is the x part of the unit state e_i jumped
// by E (computed once, with the polynomial method).  For the streams
// k = k0 + i, i < n, of one base state: the first 256 are jumped directly
// (the fixed-base table), and a level with R streams known and radix rho
// (256 for the first level, 16 after) derives streams r R + i (r = 1 ..
// rho - 1, i < R) as
//     x_{k0 + rR + i} = x_{k0 + i} M_{rRJ},   c by the closed form (Sec. 3.2),
// so every stream costs one 97x97 vector-matrix product (9,409 multiply-
// adds) against a matrix shared by R streams: a blocked GEMM on the integer
// multiply-add pipe (32-bit mul.lo, exact mod 2^24).
//
// GEMM tile: a CTA of 256 threads takes 128 source rows and one r; thread
// (ty, tx) holds rows 8ty..8ty+7 x columns tx + 16j (j < 7) in 56
// accumulators.  Shared memory: the source rows transposed (k-major, stride
// 132 words so that a thread's 8 rows are one 32-byte aligned run) and the
// matrix (97 x 112, zero padded), 94,672 bytes: 2 CTAs per SM.
#pragma once

#include "ranmar_device.cuh"

namespace ranmar {

constexpr int kPlanBase = 256;      // streams jumped directly (the table jump)
constexpr int kPlanRadix0 = 256;    // first level: 256 -> 65,536 streams
constexpr int kPlanRadix = 16;      // later levels
constexpr int kPlanMaxLevels = 8;

// Radix of level t.
__host__ __device__ constexpr int plan_radix(int t) { return t == 0 ? kPlanRadix0 : kPlanRadix; }
constexpr int kPlanRows = 128;      // source rows per CTA
constexpr int kPlanCols = 112;      // 97 output words, zero padded (16 x 7)
constexpr int kPlanAStride = 132;   // words per k of the transposed source rows
constexpr int kPlanThreads = 256;
constexpr size_t kPlanSmemBytes = sizeof(uint32_t) * (kR * kPlanAStride + kR * kPlanCols);
static_assert(kPlanAStride % 4 == 0 && kPlanAStride >= kPlanRows, "A layout");
static_assert((kR * kPlanAStride) % 4 == 0, "B alignment");

// mats[q][w] = unit_jumped[q].x[w] for w < 97, 0 for 97 <= w < 112.
__global__ void plan_pack_kernel(const ranmar_state_t* __restrict__ unit_jumped,
                                 uint32_t* __restrict__ mats, uint64_t nrows) {
  for (uint64_t q = blockIdx.x; q < nrows; q += gridDim.x)
    for (int w = threadIdx.x; w < kPlanCols; w += blockDim.x)
      mats[q * kPlanCols + w] = w < kR ? unit_jumped[q].x[w] : 0u;
}

// One level: for r = blockIdx.y + 1 and source rows i = blockIdx.x * 128 +
// (0..127) < R, st[rR + i] = st[i] advanced by E_r = rRJ (rows >= n are
// skipped).  mats: the matrices of this level (97 x 112 each); cEd[r-1] =
// (E_r mod m) d mod m; posE[r-1] = E_r mod 2^64.
__global__ void __launch_bounds__(kPlanThreads, 2) plan_level_kernel(
    ranmar_state_t* __restrict__ st, uint64_t R, uint64_t n, const uint32_t* __restrict__ mats,
    const uint32_t* __restrict__ cEd, const uint64_t* __restrict__ posE) {
  extern __shared__ __align__(16) uint32_t sm[];
  uint32_t* At = sm;                        // At[k * kPlanAStride + row]
  uint32_t* Bs = sm + kR * kPlanAStride;    // Bs[k * kPlanCols + col]
  const uint64_t r = blockIdx.y + 1;
  const uint64_t i0 = static_cast<uint64_t>(blockIdx.x) * kPlanRows;
  if (i0 >= R || r * R + i0 >= n) return;  // uniform over the CTA
  const int tid = threadIdx.x;
  for (int q = tid; q < kPlanRows * kR; q += kPlanThreads) {
    const int row = q / kR, k = q - row * kR;
    const uint64_t gi = i0 + row;
    At[k * kPlanAStride + row] = gi < R ? st[gi].x[k] : 0u;
  }
  const uint4* B4 = reinterpret_cast<const uint4*>(mats + (r - 1) * kR * kPlanCols);
  for (int q = tid; q < kR * kPlanCols / 4; q += kPlanThreads)
    reinterpret_cast<uint4*>(Bs)[q] = B4[q];
  __syncthreads();

  const int tx = tid & 15, ty = tid >> 4;
  uint32_t acc[8][7];
#pragma unroll
  for (int p = 0; p < 8; ++p)
#pragma unroll
    for (int j = 0; j < 7; ++j) acc[p][j] = 0;
#pragma unroll 4
  for (int k = 0; k < kR; ++k) {
    const uint4 a0 = *reinterpret_cast<const uint4*>(At + k * kPlanAStride + 8 * ty);
    const uint4 a1 = *reinterpret_cast<const uint4*>(At + k * kPlanAStride + 8 * ty + 4);
    const uint32_t a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    uint32_t b[7];
#pragma unroll
    for (int j = 0; j < 7; ++j) b[j] = Bs[k * kPlanCols + tx + 16 * j];
#pragma unroll
    for (int p = 0; p < 8; ++p)
#pragma unroll
      for (int j = 0; j < 7; ++j) acc[p][j] += a[p] * b[j];
  }

  const uint32_t ced = cEd[r - 1];
  const uint64_t pe = posE[r - 1];
#pragma unroll
  for (int p = 0; p < 8; ++p) {
    const uint64_t i = i0 + 8 * ty + p;
    const uint64_t d = r * R + i;
    if (i >= R || d >= n) continue;
    ranmar_state_t* dst = st + d;
#pragma unroll
    for (int j = 0; j < 7; ++j) {
      const int col = tx + 16 * j;
      if (col < kR) dst->x[col] = acc[p][j] & kMask24;
    }
    if (tx == 0) {
      dst->c = sub_mod_m(st[i].c, ced);
      dst->pos = st[i].pos + pe;
    }
  }
}

}  // namespace ranmar
