// plan_mma.cuh -- a partition-plan level (X' = X M_E mod 2^24, see plan.cuh)
// on the 5th-generation tensor cores (tcgen05, accumulators in TMEM).
//
// Exact integer arithmetic on fp16 inputs: every 24-bit word v is split
// into three balanced 8-bit limbs, v = v0 + 2^8 v1 + 2^16 v2 (mod 2^24),
// v_i in [-128, 127] (exact in fp16).  Along K, A holds [A0 | A1 | A2] and
// B holds [B2 | B1 | B0], each limb block 104 wide (97 padded), then 8 zero
// columns (K = 320).  The product sums with equal K positions give the
// weight-2^16 terms A0 B2 + A1 B1 + A2 B0, split at K = 160 into D2a and
// D2b; A's K positions [0, 208) against B's [104, 312) give D1 = A0 B1 +
// A1 B0, and [0, 112) against [208, 320) give D0 = A0 B0 (the last 8 B
// columns are zero).  Every accumulator sums at most 194 products of
// magnitude <= 2^14, so it and its partial sums stay below 2^22: the fp32
// accumulation is exact, each value converts to an integer by one add of
// 1.5 * 2^23 (its bits are then 0x4B400000 + D), and
//     x'_w = (D0 + 2^8 D1 + 2^16 (D2a + D2b)) mod 2^24.
//
// Tile: 128 source rows (M, one TMEM lane each) x 112 output words (N) x
// 320 (K): 40 MMAs of 128x112x16 per (tile, r).  A CTA of 256 threads owns
// a balanced contiguous range of (tile, r) items.  Per tile, one bulk async
// copy (TMA) brings the 128 consecutive source states (51 KB) into a staging
// buffer, from which the warps build the limb image.  Per item, a bulk copy
// brings the B image (70 KB, precomputed at plan creation), one thread
// issues the MMAs, the eight warps read the accumulators back (warps w and
// w+4 share TMEM lanes 32(w%4).. and split the columns), recombine the limbs
// and assemble the 128 new states in the staging buffer, and one bulk async
// store writes them (they are consecutive rows of the output).  The next B
// copy and the previous store overlap the MMAs and the read-back.
//
// Shared-memory operand layout (no swizzle, K-major): 8x8 fp16 core matrices
// of 128 contiguous bytes; A at ((k/8) * 16 + m/8) * 128 + (m%8) * 16 +
// (k%8) * 2 (LBO = 2048 B between K-adjacent, SBO = 128 B between M-adjacent
// core matrices), B likewise with 14 N-groups (LBO = 1792 B).
//
// Every wait on an mbarrier is bounded; on a timeout the CTA flags
// RANMAR_ST_TIMEOUT, waits (bounded) for its own copy in flight, frees its
// TMEM and returns.
#pragma once

#include <cuda_fp16.h>

#include "ranmar_device.cuh"

namespace ranmar {

constexpr int kMmaM = 128;              // rows per tile = TMEM lanes
constexpr int kMmaN = 112;              // output words, 97 padded
constexpr int kLimbK = 104;             // K per limb block, 97 padded to 8
constexpr int kMmaK = 320;              // 3 limb blocks + 8 zero columns
constexpr int kMmaThreads = 256;
constexpr uint32_t kTmemCols = 512;     // D0 at 0, D1 at 128, D2a at 256, D2b at 384
constexpr uint32_t kMagicBits = 0x4B400000u;  // bits of 1.5 * 2^23
// kMagicBits (1 + 2^8 + 2 * 2^16): the bias of b0 + 2^8 b1 + 2^16 (b2a + b2b)
constexpr uint32_t kMagicMix = kMagicBits + (kMagicBits << 8) + (kMagicBits << 17);
constexpr uint32_t kAImgBytes = kMmaM * kMmaK * 2;   // 81,920
constexpr uint32_t kStageBytes = kMmaM * sizeof(ranmar_state_t);  // 51,200
constexpr uint32_t kBImgBytes = kMmaN * kMmaK * 2;   // 71,680
constexpr uint32_t kALbo = (kMmaM / 8) * 128;        // 2048
constexpr uint32_t kBLbo = (kMmaN / 8) * 128;        // 1792
constexpr uint32_t kCoreSbo = 128;
constexpr int kKGroups = kMmaK / 8;     // 40 core matrices along K
// Operand images, the staging buffer, then barriers and the TMEM address:
// 204,864 B, so that a 20,736 B CTA of the table jump fits beside it on an
// SM.  An MMA reads K groups g, g + 1 from its start; the starts below reach
// at most group 38 (A and B), i.e. inside the images.
constexpr size_t kMmaSmemBytes = kAImgBytes + kBImgBytes + kStageBytes + 64;
static_assert(kMmaSmemBytes <= 232448, "smem");
static_assert(kKGroups * kALbo == kAImgBytes && kKGroups * kBLbo == kBImgBytes, "images");
static_assert(kLimbK % 8 == 0 && 3 * kLimbK + 8 == kMmaK && kMmaK % 16 == 0, "K layout");
constexpr uint32_t kMbarSpinLimit = 1u << 22;
static_assert(kBImgBytes % 32 == 0, "two 16-byte aligned halves");

// Instruction descriptor of tcgen05.mma kind::f16: D fp32 (bits 4-5 = 1), A
// and B fp16 (bits 7-9, 10-12 = 0), both K-major (bits 15, 16 = 0), N >> 3 at
// bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t kMmaIdesc = (1u << 4) | (static_cast<uint32_t>(kMmaN >> 3) << 17) |
                               (static_cast<uint32_t>(kMmaM >> 4) << 24);

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: start address >> 4 (bits 0-13), LBO >> 4
// (16-29), SBO >> 4 (32-45), the fixed 0b001 at bits 46-48, no swizzle.
__device__ __forceinline__ uint64_t mma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return static_cast<uint64_t>((addr & 0x3FFFFu) >> 4) |
         (static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16) |
         (static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Non-blocking probe of the phase with the given parity.
__device__ __forceinline__ bool mbar_test_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// A test of the timeout path (set only by ranmar_debug_set_wait_limit):
// when n > 0, the first wait of every CTA is made on a barrier that nothing
// completes, probed without blocking at most n times.
__device__ uint32_t g_wait_limit = 0;

// Bounded wait for the phase with the given parity (blocking polls, or
// non-blocking probes when `probe`); false on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity,
                                          uint32_t limit = kMbarSpinLimit, bool probe = false) {
  for (uint32_t it = 0; it < limit; ++it)
    if (probe ? mbar_test_wait(bar, parity) : mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void bulk_s2g(void* dst, uint32_t src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(src),
               "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// The staging buffer may be rewritten once the stores have read it.
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// A hint that brings `bytes` (a multiple of 16, 16-byte aligned) into L2.
__device__ __forceinline__ void prefetch_l2(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

// D[tmem] (+)= A[smem] B[smem], one 128 x 112 x 16 step.
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(kMmaIdesc), "r"(accumulate)
      : "memory");
}

// D[tmem] (+)= A B with the descriptors advanced by the constants kAOff /
// kBOff (added inside the statement, so that the 42 descriptors of an item
// are not all held in registers).
template <uint32_t kAOff, uint32_t kBOff>
__device__ __forceinline__ void mma_f16_at(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                           uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n .reg .b64 da, db;\n setp.ne.b32 p, %4, 0;\n"
      " add.s64 da, %1, %5;\n add.s64 db, %2, %6;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], da, db, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(kMmaIdesc), "r"(accumulate), "n"(kAOff), "n"(kBOff)
      : "memory");
}

// kSteps MMAs (16 K each) from the K group (8 columns) kA of A and kB of B
// on, into the accumulator at d (the first one overwrites it when `first`).
// Step j starts 2 j groups further: a constant added to the descriptor's
// start-address field (shared-memory addresses stay below 2^18).
template <int kSteps, int kA, int kB, int kJ = 0>
__device__ __forceinline__ void mma_run(uint32_t d, uint64_t ad, uint64_t bd, bool first) {
  if constexpr (kJ < kSteps) {
    static_assert(kA + 2 * kJ + 1 < kKGroups && kB + 2 * kJ + 1 < kKGroups, "K reach");
    mma_f16_at<(((kA + 2u * kJ) * kALbo) >> 4), (((kB + 2u * kJ) * kBLbo) >> 4)>(
        d, ad, bd, (first && kJ == 0) ? 0u : 1u);
    mma_run<kSteps, kA, kB, kJ + 1>(d, ad, bd, first);
  }
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::
                   "r"(bar)
               : "memory");
}

// 16 consecutive fp32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld1(uint32_t taddr, uint32_t (&v)[1]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(v[0]) : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// The registers of a tcgen05.ld hold their values only after the wait; an
// empty statement that "rewrites" them, placed after tmem_ld_wait, keeps the
// compiler from reading them earlier.
__device__ __forceinline__ void tmem_regs_fence(uint32_t (&v)[16]) {
  asm volatile(""
               : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]),
                 "+r"(v[6]), "+r"(v[7]), "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]),
                 "+r"(v[12]), "+r"(v[13]), "+r"(v[14]), "+r"(v[15]));
}
__device__ __forceinline__ void tmem_regs_fence(uint32_t (&v)[1]) {
  asm volatile("" : "+r"(v[0]));
}

// Output word j of the four accumulators D0, D1, D2a, D2b (fp32 bits):
// |D| < 2^22, so D + 1.5 * 2^23 is exact and its bits are 0x4B400000 + D;
// x' = (D0 + 2^8 D1 + 2^16 (D2a + D2b)) mod 2^24.
template <int kW>
__device__ __forceinline__ uint32_t limb_sum(const uint32_t (&f)[4][kW], int j) {
  const uint32_t b0 = __float_as_uint(__uint_as_float(f[0][j]) + 12582912.0f);
  const uint32_t b1 = __float_as_uint(__uint_as_float(f[1][j]) + 12582912.0f);
  const uint32_t b2 = __float_as_uint(__uint_as_float(f[2][j]) + 12582912.0f) +
                      __float_as_uint(__uint_as_float(f[3][j]) + 12582912.0f);
  return (b0 + (b1 << 8) + (b2 << 16) - kMagicMix) & kMask24;
}

// Balanced 8-bit limbs of two 24-bit words as fp16 pairs: h[s] = (limb s of
// a, limb s of b), v = l0 + 2^8 l1 + 2^16 l2 (mod 2^24), l_s in [-128, 127].
// (v + 0x808080) mod 2^24 has the bytes l_s + 128 (the balanced digits are
// unique); a byte u placed under the high byte 0x64 is the fp16 1024 + u,
// and one packed subtraction of 1152 leaves l_s (every value is exact).
__device__ __forceinline__ void limb_pairs(uint32_t a, uint32_t b, uint32_t (&h)[3]) {
  const uint32_t wa = ((a + 0x808080u) & kMask24) | 0x64000000u;
  const uint32_t wb = ((b + 0x808080u) & kMask24) | 0x64000000u;
  const __half2 bias = __float2half2_rn(1152.0f);
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    // result bytes: byte s of wa, 0x64, byte s of wb, 0x64
    const uint32_t bits = __byte_perm(wa, wb, s | (3u << 4) | ((4u + s) << 8) | (7u << 12));
    const __half2 v = __hsub2(*reinterpret_cast<const __half2*>(&bits), bias);
    h[s] = *reinterpret_cast<const uint32_t*>(&v);
  }
}

// Byte offset of element (row, k) in an operand image with `groups` 8-row
// groups (K-major, no swizzle).
__host__ __device__ constexpr uint32_t img_off(uint32_t row, uint32_t k, uint32_t groups) {
  return ((k / 8) * groups + row / 8) * 128 + (row % 8) * 16 + (k % 8) * 2;
}

// B image of one matrix: element (n, k') = limb (2 - k'/104) of M[k'%104][n]
// for k' < 312 (0 beyond 97 in either index), 0 for k' >= 312, so that K
// holds [B2 | B1 | B0 | 0].  One thread per (matrix, n, k-pair).
__global__ void plan_bimg_kernel(const ranmar_state_t* __restrict__ unit_jumped,
                                 uint8_t* __restrict__ bimg, uint32_t nmat) {
  const uint64_t total = static_cast<uint64_t>(nmat) * kMmaN * (kLimbK / 2);
  for (uint64_t q = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; q < total;
       q += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    const uint32_t mat = static_cast<uint32_t>(q / (kMmaN * (kLimbK / 2)));
    const uint32_t rem = static_cast<uint32_t>(q % (kMmaN * (kLimbK / 2)));
    const uint32_t nn = rem / (kLimbK / 2), k = 2 * (rem % (kLimbK / 2));
    uint32_t va = 0, vb = 0;
    if (nn < static_cast<uint32_t>(kR)) {
      const ranmar_state_t* rows = unit_jumped + static_cast<size_t>(mat) * kR;
      if (k < static_cast<uint32_t>(kR)) va = rows[k].x[nn];
      if (k + 1 < static_cast<uint32_t>(kR)) vb = rows[k + 1].x[nn];
    }
    uint32_t h[3];
    limb_pairs(va, vb, h);
    uint8_t* img = bimg + static_cast<size_t>(mat) * kBImgBytes;
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      const uint32_t kk = s * kLimbK + k;
      *reinterpret_cast<uint32_t*>(img + img_off(nn, kk, kMmaN / 8)) = h[2 - s];
    }
    if (k == 0)  // the 8 zero columns after the limb blocks
      *reinterpret_cast<uint4*>(img + img_off(nn, 3 * kLimbK, kMmaN / 8)) = make_uint4(0, 0, 0, 0);
  }
}

// One level on the tensor cores: items q = tile * r_count + (r - 1), tile <
// ceil(R / 128), r = 1..r_count; st[rR + i] = st[i] advanced by E_r for
// source rows i < R of the tile with rR + i < n.  bimg: this level's B
// images (one per r); cEd / posE as in plan_level_kernel.
__global__ void __launch_bounds__(kMmaThreads, 1) plan_level_mma_kernel(
    ranmar_state_t* __restrict__ st, uint64_t R, uint64_t n, uint32_t r_count, uint32_t items,
    const uint8_t* __restrict__ bimg, const uint32_t* __restrict__ cEd,
    const uint64_t* __restrict__ posE, uint32_t* status) {
  extern __shared__ __align__(16) uint32_t smem[];
  uint8_t* A = reinterpret_cast<uint8_t*>(smem);
  uint8_t* B = A + kAImgBytes;
  uint8_t* stage = B + kBImgBytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(stage + kStageBytes);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 4);
  const uint32_t bar_x = smem_addr(&bars[3]);  // never completed (the timeout test)
  const uint32_t bar_b = smem_addr(&bars[0]), bar_m = smem_addr(&bars[1]),
                 bar_s = smem_addr(&bars[2]);
  const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t test_limit = g_wait_limit;

  const uint32_t q0 = static_cast<uint32_t>(static_cast<uint64_t>(blockIdx.x) * items / gridDim.x);
  const uint32_t q1 =
      static_cast<uint32_t>(static_cast<uint64_t>(blockIdx.x + 1) * items / gridDim.x);
  if (q0 >= q1) return;

  auto load_b = [&](uint32_t q) {
    const uint32_t r = q % r_count + 1;
    const uint8_t* src = bimg + static_cast<size_t>(r - 1) * kBImgBytes;
    mbar_expect_tx(bar_b, kBImgBytes);
    bulk_g2s(smem_addr(B), src, kBImgBytes / 2, bar_b);
    bulk_g2s(smem_addr(B) + kBImgBytes / 2, src + kBImgBytes / 2, kBImgBytes / 2, bar_b);
  };
  // source rows of a tile into the staging buffer
  auto load_src = [&](uint64_t tile) {
    const uint64_t i0 = tile * kMmaM;
    const uint32_t bytes = static_cast<uint32_t>(R - i0 < kMmaM ? R - i0 : kMmaM) *
                           static_cast<uint32_t>(sizeof(ranmar_state_t));
    mbar_expect_tx(bar_s, bytes);
    bulk_g2s(smem_addr(stage), st + i0, bytes, bar_s);
  };

  // Thread 0 starts the copies of the first tile and the first B image at
  // once (they run under the TMEM allocation) and asks L2 for the CTA's
  // other B images and, if its range reaches a second tile, those rows.
  if (tid == 0) {
    mbar_init(bar_b, 1);
    mbar_init(bar_m, 1);
    mbar_init(bar_s, 1);
    mbar_init(bar_x, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    load_src(q0 / r_count);
    load_b(q0);
    for (uint32_t q = q0 + 1; q < q1; ++q)
      prefetch_l2(bimg + static_cast<size_t>(q % r_count) * kBImgBytes, kBImgBytes);
    const uint64_t t_last = (q1 - 1) / r_count;
    if (t_last != q0 / r_count) {
      const uint64_t i0 = t_last * kMmaM;
      prefetch_l2(st + i0, static_cast<uint32_t>(R - i0 < kMmaM ? R - i0 : kMmaM) *
                               static_cast<uint32_t>(sizeof(ranmar_state_t)));
    }
  }
  if (warp == 0) tmem_alloc(smem_addr(tmem_slot), kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  uint32_t ph_b = 0, ph_m = 0, ph_s = 0;  // ph_b: thread 0 only
  bool ok = true;
  bool b_in_flight = true, mma_in_flight = false, s_in_flight = true;  // thread 0's view
  int64_t cur_tile = -1;
  uint32_t src_c = 0;  // warps 0-3: c and pos of this thread's source row
  uint64_t src_pos = 0;
  const uint32_t quarter = warp & 3;
  const uint32_t m = quarter * 32 + lane;  // tile row = TMEM lane of this thread
#pragma unroll 1
  for (uint32_t q = q0; q < q1 && ok; ++q) {
    const uint64_t tile = q / r_count;
    const uint32_t r = q % r_count + 1;
    const uint64_t i0 = tile * kMmaM;
    const uint32_t nsrc = static_cast<uint32_t>(R - i0 < kMmaM ? R - i0 : kMmaM);
    if (static_cast<int64_t>(tile) != cur_tile) {
      // the tile's source states into the staging buffer (the first tile's
      // copy is already in flight; a later one waits until the last store
      // has read the buffer)
      if (tid == 0 && cur_tile >= 0) {
        bulk_wait_read();
        load_src(tile);
        s_in_flight = true;
      }
      const bool s_ok = test_limit ? mbar_wait(bar_x, 0, test_limit, true)
                                   : mbar_wait(bar_s, ph_s);
      ok = __syncthreads_and(s_ok);
      if (!ok) break;
      ph_s ^= 1;
      if (tid == 0) s_in_flight = false;
      // A image: warp w converts core matrices (mg, kg) with mg = w, w+8;
      // lane l -> row mg*8 + (l & 7), k pair 2 (l >> 3); then the 8 zero
      // columns after the limb blocks.
      if (tid < kMmaM)
        *reinterpret_cast<uint4*>(A + img_off(tid, 3 * kLimbK, kMmaM / 8)) = make_uint4(0, 0, 0, 0);
#pragma unroll 1
      for (uint32_t mg = warp; mg < kMmaM / 8; mg += kMmaThreads / 32) {
        const uint32_t row = mg * 8 + (lane & 7);
        const uint32_t* x = reinterpret_cast<const uint32_t*>(stage) + row * (sizeof(ranmar_state_t) / 4);
        const uint32_t kp = 2 * (lane >> 3);
#pragma unroll
        for (int kg = 0; kg < kLimbK / 8; ++kg) {
          const uint32_t k = 8 * kg + kp;  // even; x[k], x[k+1] (x[97] is c: dropped)
          uint2 v = make_uint2(0u, 0u);
          if (row < nsrc && k < static_cast<uint32_t>(kR)) {
            v = *reinterpret_cast<const uint2*>(x + k);
            if (k + 1 >= static_cast<uint32_t>(kR)) v.y = 0u;
          }
          uint32_t h[3];
          limb_pairs(v.x, v.y, h);
#pragma unroll
          for (int s = 0; s < 3; ++s)
            *reinterpret_cast<uint32_t*>(A + img_off(row, s * kLimbK + k, kMmaM / 8)) = h[s];
        }
      }
      if (warp < 4 && m < nsrc) {
        const ranmar_state_t* srow = reinterpret_cast<const ranmar_state_t*>(stage) + m;
        src_c = srow->c;
        src_pos = srow->pos;
      }
      fence_proxy_async_smem();
      __syncthreads();
      cur_tile = static_cast<int64_t>(tile);
    }
    if (tid == 0) {
      ok = mbar_wait(bar_b, ph_b);
      if (ok) {
        b_in_flight = false;
        ph_b ^= 1;
        tc_fence_after();
        // K groups of 8 (limb blocks of 13 groups: A = [A0 | A1 | A2 | 0], B
        // = [B2 | B1 | B0 | 0]).  D2a (col 256) and D2b (col 384): equal K
        // positions, groups 0-19 and 20-39; D1 (col 128): A groups 0-25
        // against B groups 13-38; D0 (col 0): A 0-13 against B 26-39.
        const uint64_t ad = mma_desc(smem_addr(A), kALbo, kCoreSbo);
        const uint64_t bd = mma_desc(smem_addr(B), kBLbo, kCoreSbo);
        constexpr int G = kLimbK / 8;                    // 13
        mma_run<10, 0, 0>(tmem + 256, ad, bd, true);     // D2a
        mma_run<10, 20, 20>(tmem + 384, ad, bd, true);   // D2b
        mma_run<G, 0, G>(tmem + 128, ad, bd, true);      // D1 = A0 B1 + A1 B0
        mma_run<7, 0, 2 * G>(tmem, ad, bd, true);        // D0 = A0 B0
        mma_commit(bar_m);
        mma_in_flight = true;
      }
    }
    // every thread: the MMAs of this item are complete (or thread 0 timed out)
    ok = __syncthreads_and(ok);
    if (!ok) break;
    const bool mma_ok = mbar_wait(bar_m, ph_m);
    ok = __syncthreads_and(mma_ok);
    if (!ok) break;
    ph_m ^= 1;
    tc_fence_after();
    if (tid == 0) {
      mma_in_flight = false;
      if (q + 1 < q1) {  // B is free: the next copy runs under the read-back
        load_b(q + 1);
        b_in_flight = true;
      }
      bulk_wait_read();  // the previous item's store has read the staging buffer
    }
    __syncthreads();
    // read-back: warps w and w+4 read TMEM lanes 32(w%4).. (tile rows);
    // warp w < 4 takes the column chunks 0-2 and column 96, warp w + 4 the
    // chunks 3-5 (16 columns each).  All loads of a phase are issued before
    // the one wait.  The states go to staging row m; destination rows rR +
    // i0 + (0 .. ndst): a prefix of the tile (i < R and rR + i < n),
    // possibly empty.
    const uint64_t dst0 = static_cast<uint64_t>(r) * R + i0;
    const uint32_t ndst =
        dst0 >= n ? 0u
                  : static_cast<uint32_t>(min(static_cast<uint64_t>(nsrc), n - dst0));
    uint32_t* srow = reinterpret_cast<uint32_t*>(stage) + m * (sizeof(ranmar_state_t) / 4);
    const uint32_t lane_base = tmem + ((quarter * 32u) << 16);
    const int c0 = warp < 4 ? 0 : 3;
    {
      uint32_t f[2][4][16];
#pragma unroll
      for (int cc = 0; cc < 2; ++cc)
#pragma unroll
        for (int d = 0; d < 4; ++d) tmem_ld16(lane_base + 128 * d + 16 * (c0 + cc), f[cc][d]);
      tmem_ld_wait();
#pragma unroll
      for (int cc = 0; cc < 2; ++cc)
#pragma unroll
        for (int d = 0; d < 4; ++d) tmem_regs_fence(f[cc][d]);
#pragma unroll
      for (int cc = 0; cc < 2; ++cc) {
        uint4* o4 = reinterpret_cast<uint4*>(srow + 16 * (c0 + cc));
#pragma unroll
        for (int j = 0; j < 4; ++j)
          o4[j] = make_uint4(limb_sum(f[cc], 4 * j), limb_sum(f[cc], 4 * j + 1),
                             limb_sum(f[cc], 4 * j + 2), limb_sum(f[cc], 4 * j + 3));
      }
    }
    {
      uint32_t f[4][16], g[4][1];
#pragma unroll
      for (int d = 0; d < 4; ++d) tmem_ld16(lane_base + 128 * d + 16 * (c0 + 2), f[d]);
      if (warp < 4) {
#pragma unroll
        for (int d = 0; d < 4; ++d) tmem_ld1(lane_base + 128 * d + 96, g[d]);
      }
      tmem_ld_wait();
#pragma unroll
      for (int d = 0; d < 4; ++d) {
        tmem_regs_fence(f[d]);
        tmem_regs_fence(g[d]);
      }
      uint4* o4 = reinterpret_cast<uint4*>(srow + 16 * (c0 + 2));
#pragma unroll
      for (int j = 0; j < 4; ++j)
        o4[j] = make_uint4(limb_sum(f, 4 * j), limb_sum(f, 4 * j + 1), limb_sum(f, 4 * j + 2),
                           limb_sum(f, 4 * j + 3));
      if (warp < 4) srow[96] = limb_sum(g, 0);
    }
    if (warp < 4) {
      ranmar_state_t* so = reinterpret_cast<ranmar_state_t*>(srow);
      so->c = sub_mod_m(src_c, cEd[r - 1]);
      so->pos = src_pos + posE[r - 1];
    }
    tc_fence_before();
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0 && ndst > 0)
      bulk_s2g(st + dst0, smem_addr(stage), ndst * static_cast<uint32_t>(sizeof(ranmar_state_t)));
  }
  if (!ok && tid == 0) {
    flag_status(status, RANMAR_ST_TIMEOUT);
    // bounded waits for this CTA's own asynchronous work still in flight
    if (b_in_flight) mbar_wait(bar_b, ph_b);
    if (s_in_flight) mbar_wait(bar_s, ph_s);
    if (mma_in_flight) mbar_wait(bar_m, ph_m);
  }
  // the staging buffer must outlive the reads of the last store; its writes
  // complete with the grid
  if (tid == 0) bulk_wait_read();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

}  // namespace ranmar
