// plan_mma.cuh -- a partition-plan level (X' = X M_E mod 2^24, see plan.cuh)
// on the 5th-generation tensor cores (tcgen05, accumulators in TMEM).
//
// Exact integer arithmetic on fp16 inputs: every 24-bit word v is split
// into three balanced 8-bit limbs, v = v0 + 2^8 v1 + 2^16 v2 (mod 2^24),
// v_i in [-128, 127] (exact in fp16).  With K = 97 terms per dot product the
// four accumulators
//     D0 = A0 B0,  D1 = A0 B1 + A1 B0,  D2a = A0 B2 + A2 B0,  D2b = A1 B1
// (and every partial sum of them) stay below 2 * 97 * 2^14 < 2^22 in
// magnitude, so the fp32 accumulation is exact, each value converts to an
// integer by one add of 1.5 * 2^23 (its bits are then 0x4B400000 + D), and
//     x'_w = (D0 + 2^8 D1 + 2^16 (D2a + D2b)) mod 2^24.
// A holds [A0 | A1 | A2] along K (3 x 112, 97 padded), B holds [B2 | B1 |
// B0]: each accumulator is a sum of K ranges of the two images.
//
// Tile: 128 source rows (M, one TMEM lane each) x 112 output words (N) x
// 336 (K): 42 MMAs of 128x112x16 per (tile, r).  A CTA of 256 threads owns
// a balanced contiguous range of (tile, r) items.  Per tile, one bulk async
// copy (TMA) brings the 128 consecutive source states (51 KB) into a staging
// buffer, from which the warps build the limb image.  Per item, a bulk copy
// brings the B image (75 KB, precomputed at plan creation), one thread
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
constexpr int kLimbK = 112;             // K per limb, 97 padded
constexpr int kMmaK = 3 * kLimbK;       // 336
constexpr int kMmaThreads = 256;
constexpr uint32_t kTmemCols = 512;     // D0 at 0, D1 at 128, D2a at 256, D2b at 384
constexpr uint32_t kMagicBits = 0x4B400000u;  // bits of 1.5 * 2^23
// kMagicBits (1 + 2^8 + 2 * 2^16): the bias of b0 + 2^8 b1 + 2^16 (b2a + b2b)
constexpr uint32_t kMagicMix = kMagicBits + (kMagicBits << 8) + (kMagicBits << 17);
constexpr uint32_t kAImgBytes = kMmaM * kMmaK * 2;   // 86,016
constexpr uint32_t kStageBytes = kMmaM * sizeof(ranmar_state_t);  // 51,200
constexpr uint32_t kBImgBytes = kMmaN * kMmaK * 2;   // 75,264
constexpr uint32_t kALbo = (kMmaM / 8) * 128;        // 2048
constexpr uint32_t kBLbo = (kMmaN / 8) * 128;        // 1792
constexpr uint32_t kCoreSbo = 128;
// Operand images, the staging buffer, then barriers and the TMEM address.
// The descriptors only reach inside the images (A start at most 40 LBO plus
// one LBO and 15 SBO; B at most 40 LBO plus one LBO and 13 SBO).
constexpr size_t kMmaSmemBytes = kAImgBytes + kBImgBytes + kStageBytes + 64;
static_assert(kMmaSmemBytes <= 232448, "smem");
static_assert(41 * kALbo + 15 * kCoreSbo + 128 <= kAImgBytes &&
                  41 * kBLbo + 13 * kCoreSbo + 128 <= kBImgBytes,
              "descriptor reach");
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

// Bounded wait for the phase with the given parity; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (uint32_t it = 0; it < kMbarSpinLimit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
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
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
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
__device__ __forceinline__ void tmem_ld_wait() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Balanced 8-bit limbs of a 24-bit word: v = l0 + 2^8 l1 + 2^16 l2 (mod 2^24).
__device__ __forceinline__ void limbs3(uint32_t v, int (&l)[3]) {
  l[0] = static_cast<int>((v & 0xFFu) ^ 0x80u) - 0x80;
  const uint32_t v1 = (v - static_cast<uint32_t>(l[0])) >> 8;
  l[1] = static_cast<int>((v1 & 0xFFu) ^ 0x80u) - 0x80;
  const uint32_t v2 = (v1 - static_cast<uint32_t>(l[1])) >> 8;
  l[2] = static_cast<int>((v2 & 0xFFu) ^ 0x80u) - 0x80;
}

__device__ __forceinline__ uint32_t pack_half2(int a, int b) {
  const __half2 h = __halves2half2(__int2half_rn(a), __int2half_rn(b));
  return *reinterpret_cast<const uint32_t*>(&h);
}

// Byte offset of element (row, k) in an operand image with `groups` 8-row
// groups (K-major, no swizzle).
__host__ __device__ constexpr uint32_t img_off(uint32_t row, uint32_t k, uint32_t groups) {
  return ((k / 8) * groups + row / 8) * 128 + (row % 8) * 16 + (k % 8) * 2;
}

// B image of one matrix: element (n, k') = limb (2 - k'/112) of M[k'%112][n]
// (0 beyond 97 in either index), so that K holds [B2 | B1 | B0].  One thread
// per (matrix, n, k-pair).
__global__ void plan_bimg_kernel(const ranmar_state_t* __restrict__ unit_jumped,
                                 uint8_t* __restrict__ bimg, uint32_t nmat) {
  const uint64_t total = static_cast<uint64_t>(nmat) * kMmaN * (kLimbK / 2);
  for (uint64_t q = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; q < total;
       q += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    const uint32_t mat = static_cast<uint32_t>(q / (kMmaN * (kLimbK / 2)));
    const uint32_t rem = static_cast<uint32_t>(q % (kMmaN * (kLimbK / 2)));
    const uint32_t nn = rem / (kLimbK / 2), k = 2 * (rem % (kLimbK / 2));
    int la[3] = {0, 0, 0}, lb[3] = {0, 0, 0};
    if (nn < static_cast<uint32_t>(kR)) {
      const ranmar_state_t* rows = unit_jumped + static_cast<size_t>(mat) * kR;
      if (k < static_cast<uint32_t>(kR)) limbs3(rows[k].x[nn], la);
      if (k + 1 < static_cast<uint32_t>(kR)) limbs3(rows[k + 1].x[nn], lb);
    }
    uint8_t* img = bimg + static_cast<size_t>(mat) * kBImgBytes;
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      const uint32_t kk = s * kLimbK + k;
      *reinterpret_cast<uint32_t*>(img + img_off(nn, kk, kMmaN / 8)) =
          pack_half2(la[2 - s], lb[2 - s]);
    }
  }
}

// One level on the tensor cores: items q = tile * r_count + (r - 1), tile <
// ceil(R / 128), r = 1..r_count; st[rR + i] = st[i] advanced by E_r for
// source rows i < R of the tile with rR + i < n.  bimg: this level's 15 B
// images; cEd / posE as in plan_level_kernel.
__global__ void __launch_bounds__(kMmaThreads, 1) plan_level_mma_kernel(
    ranmar_state_t* __restrict__ st, uint64_t R, uint64_t n, uint32_t r_count, uint32_t items,
    const uint8_t* __restrict__ bimg, const uint32_t* __restrict__ cEd,
    const uint64_t* __restrict__ posE, uint32_t* status) {
  extern __shared__ __align__(16) uint32_t smem[];
  uint8_t* A = reinterpret_cast<uint8_t*>(smem);
  uint8_t* B = A + kAImgBytes;
  uint8_t* stage = B + kBImgBytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(stage + kStageBytes);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3);
  const uint32_t bar_b = smem_addr(&bars[0]), bar_m = smem_addr(&bars[1]),
                 bar_s = smem_addr(&bars[2]);
  const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  const uint32_t q0 = static_cast<uint32_t>(static_cast<uint64_t>(blockIdx.x) * items / gridDim.x);
  const uint32_t q1 =
      static_cast<uint32_t>(static_cast<uint64_t>(blockIdx.x + 1) * items / gridDim.x);
  if (q0 >= q1) return;

  if (tid == 0) {
    mbar_init(bar_b, 1);
    mbar_init(bar_m, 1);
    mbar_init(bar_s, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(smem_addr(tmem_slot), kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  auto load_b = [&](uint32_t q) {
    const uint32_t r = q % r_count + 1;
    const uint8_t* src = bimg + static_cast<size_t>(r - 1) * kBImgBytes;
    mbar_expect_tx(bar_b, kBImgBytes);
    bulk_g2s(smem_addr(B), src, kBImgBytes / 2, bar_b);
    bulk_g2s(smem_addr(B) + kBImgBytes / 2, src + kBImgBytes / 2, kBImgBytes / 2, bar_b);
  };

  if (tid == 0) load_b(q0);
  uint32_t ph_b = 0, ph_m = 0, ph_s = 0;  // ph_b: thread 0 only
  bool ok = true;
  bool b_in_flight = true, mma_in_flight = false, s_in_flight = false;  // thread 0's view
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
      // the tile's source states into the staging buffer (after the last
      // store has read it)
      if (tid == 0) {
        bulk_wait_read();
        mbar_expect_tx(bar_s, nsrc * static_cast<uint32_t>(sizeof(ranmar_state_t)));
        bulk_g2s(smem_addr(stage), st + i0, nsrc * static_cast<uint32_t>(sizeof(ranmar_state_t)),
                 bar_s);
        s_in_flight = true;
      }
      const bool s_ok = mbar_wait(bar_s, ph_s);
      ok = __syncthreads_and(s_ok);
      if (!ok) break;
      ph_s ^= 1;
      if (tid == 0) s_in_flight = false;
      // A image: warp w converts core matrices (mg, kg) with mg = w, w+8;
      // lane l -> row mg*8 + (l & 7), k pair 2 (l >> 3).
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
          int la[3], lb[3];
          limbs3(v.x, la);
          limbs3(v.y, lb);
#pragma unroll
          for (int s = 0; s < 3; ++s)
            *reinterpret_cast<uint32_t*>(A + img_off(row, s * kLimbK + k, kMmaM / 8)) =
                pack_half2(la[s], lb[s]);
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
        const uint32_t a0 = smem_addr(A), b0 = smem_addr(B);
        // K ranges (units of 16): limb images A = [A0 | A1 | A2], B = [B2 | B1
        // | B0], 7 steps per limb.  D2a (col 256) = A0 B2 + A2 B0, D2b (col
        // 384) = A1 B1, D1 (col 128) = A0 B1 + A1 B0, D0 (col 0) = A0 B0.
        constexpr uint32_t L = kLimbK / 16;
        auto run = [&](uint32_t dcol, uint32_t astep, uint32_t bstep, uint32_t nsteps,
                       bool first) {
#pragma unroll 1
          for (uint32_t s2 = 0; s2 < nsteps; ++s2)
            mma_f16(tmem + dcol, mma_desc(a0 + 2 * (astep + s2) * kALbo, kALbo, kCoreSbo),
                    mma_desc(b0 + 2 * (bstep + s2) * kBLbo, kBLbo, kCoreSbo),
                    (first && s2 == 0) ? 0u : 1u);
        };
        run(256, 0, 0, L, true);          // A0 B2
        run(256, 2 * L, 2 * L, L, false); // A2 B0
        run(384, L, L, L, true);          // A1 B1
        run(128, 0, L, 2 * L, true);      // A0 B1 + A1 B0
        run(0, 0, 2 * L, L, true);        // A0 B0
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
    // read-back: warps w and w+4 read TMEM lanes 32(w%4).. (tile rows) and
    // split the 7 column chunks (4 + 3); the states go to staging row m
    // destination rows rR + i0 + (0 .. ndst): a prefix of the tile (i < R and
    // rR + i < n), possibly empty
    const uint64_t dst0 = static_cast<uint64_t>(r) * R + i0;
    const uint32_t ndst =
        dst0 >= n ? 0u
                  : static_cast<uint32_t>(min(static_cast<uint64_t>(nsrc), n - dst0));
    uint32_t* srow = reinterpret_cast<uint32_t*>(stage) + m * (sizeof(ranmar_state_t) / 4);
    const uint32_t lane_base = tmem + ((quarter * 32u) << 16);
    const int c_lo = warp < 4 ? 0 : 4, c_hi = warp < 4 ? 4 : kMmaN / 16;
#pragma unroll 1
    for (int c = c_lo; c < c_hi; ++c) {
      uint32_t f0[16], f1[16], f2[16], f3[16];
      tmem_ld16(lane_base + 16 * c, f0);
      tmem_ld16(lane_base + 128 + 16 * c, f1);
      tmem_ld16(lane_base + 256 + 16 * c, f2);
      tmem_ld16(lane_base + 384 + 16 * c, f3);
      tmem_ld_wait();
      uint32_t w[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        // |D| < 2^22: D + 1.5 * 2^23 is exact and its bits are 0x4B400000 + D
        const uint32_t b0 = __float_as_uint(__uint_as_float(f0[j]) + 12582912.0f);
        const uint32_t b1 = __float_as_uint(__uint_as_float(f1[j]) + 12582912.0f);
        const uint32_t b2 = __float_as_uint(__uint_as_float(f2[j]) + 12582912.0f) +
                            __float_as_uint(__uint_as_float(f3[j]) + 12582912.0f);
        w[j] = (b0 + (b1 << 8) + (b2 << 16) - kMagicMix) & kMask24;
      }
      if (c < kMmaN / 16 - 1) {
        uint4* o4 = reinterpret_cast<uint4*>(srow + 16 * c);
#pragma unroll
        for (int j = 0; j < 4; ++j)
          o4[j] = make_uint4(w[4 * j], w[4 * j + 1], w[4 * j + 2], w[4 * j + 3]);
      } else {
        srow[96] = w[0];
      }
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
  if (tid == 0) bulk_wait_all();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

}  // namespace ranmar
