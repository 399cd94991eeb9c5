// plan_mma2.cuh -- a partition-plan level on the tensor cores with the A
// operand in tensor memory and the items of a CTA pipelined.
//
// Same arithmetic as plan_mma.cuh (balanced 8-bit limbs in fp16, K = 320 =
// three limb blocks of 104 and 8 zero columns), with three accumulators:
// D0 = A0 B0 and D1 = A0 B1 + A1 B0 as there, and the whole weight-2^16 sum
// D2 = A0 B2 + A1 B1 + A2 B0 in one accumulator.  D2 sums at most 291
// products of magnitude <= 2^14, below 2^23: its fp32 accumulation is still
// exact, and it converts to an integer with cvt.rni (D0 and D1, below 2^22,
// keep the one-add conversion).
//
// Tensor memory (512 columns): the A image of the tile at columns 0..159
// (lane m = source row m; column c holds the fp16 pair K = 2c, 2c + 1),
// D0 at 160, D1 at 272, D2 at 384 (112 columns each).  With A out of
// shared memory, two B images fit there beside the staging buffer
// (143,360 + 51,200 B), so the next item's B arrives while the current one
// is multiplied.
//
// Roles: warp 8 (one thread) issues the copies of the B images and the MMAs;
// warps 0-7 build A (once per tile), read the accumulators back, assemble
// the new states in the staging buffer and store them.  The MMAs of item
// t+1 into an accumulator start as soon as the read-back of item t has
// released it (D2 first, then D1, D0), so the tensor core works while the
// previous item is read back, converted and stored.
//
// mbarriers (all waits bounded; after a timeout the role flags
// RANMAR_ST_TIMEOUT and stops, the other role stops at its next wait, each
// drains its own copies and MMAs in flight, and the CTA frees its tensor
// memory):
//   bfull[s]  the B image in slot s has landed        (copy, tx count)
//   bempty[s] the MMAs reading slot s are complete    (tcgen05.commit)
//   dfull[x]  accumulator x of the item is complete   (tcgen05.commit)
//   dempty[x] the 8 reading warps have loaded x       (8 arrivals)
//   aready    the tile's A image is in tensor memory  (8 arrivals)
//   src       the tile's source rows have landed      (copy, tx count)
//   drain     every MMA of the CTA is complete        (tcgen05.commit)
//   x         never completed: with a wait limit set for the timeout test,
//             each role's first wait is a bounded probe of it
// The 256 reading threads also meet at named barrier 1 (bar.red.and, so
// that a timeout seen by any of them is seen by all of them).
#pragma once

#include "plan_mma.cuh"

namespace ranmar {

constexpr int kM2Workers = 256;
constexpr int kM2Threads = kM2Workers + 32;
constexpr uint32_t kM2D0 = 160, kM2D1 = 272, kM2D2 = 384;
constexpr int kM2ACols = kMmaK / 2;  // 160
static_assert(kM2D2 + kMmaN <= kTmemCols && kM2ACols <= static_cast<int>(kM2D0), "tmem");
constexpr size_t kM2SmemBytes = 2 * static_cast<size_t>(kBImgBytes) + kStageBytes + 128;
static_assert(kM2SmemBytes <= 232448, "smem");

// tcgen05.mma with A from tensor memory: D (+)= A[a_tmem + kACol] B, B's
// descriptor advanced by kBOff (both added inside the statement).
template <uint32_t kACol, uint32_t kBOff>
__device__ __forceinline__ void mma_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n .reg .b32 ta;\n .reg .b64 db;\n setp.ne.b32 p, %4, 0;\n"
      " add.u32 ta, %1, %5;\n add.s64 db, %2, %6;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], [ta], db, %3, p;\n}\n" ::"r"(d_tmem),
      "r"(a_tmem), "l"(bdesc), "r"(kMmaIdesc), "r"(accumulate), "n"(kACol), "n"(kBOff)
      : "memory");
}

// kSteps MMAs: step j takes A columns 8j .. 8j+7 (K 16j .. 16j+15) and B's
// K groups kB + 2j, kB + 2j + 1; the first overwrites the accumulator.
template <int kSteps, int kB, int kJ = 0>
__device__ __forceinline__ void mma_run_ta(uint32_t d, uint32_t a, uint64_t bd) {
  if constexpr (kJ < kSteps) {
    static_assert(8 * kJ + 8 <= kM2ACols && kB + 2 * kJ + 1 < kKGroups, "reach");
    mma_ta<8u * kJ, (((kB + 2u * kJ) * kBLbo) >> 4)>(d, a, bd, kJ == 0 ? 0u : 1u);
    mma_run_ta<kSteps, kB, kJ + 1>(d, a, bd);
  }
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
      "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]),
      "r"(v[15])
      : "memory");
}
__device__ __forceinline__ void tmem_st_wait() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// Named barrier 1 over the 256 reading threads; returns the AND of `p`.
__device__ __forceinline__ bool workers_sync_and(bool p) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred a, b;\n setp.ne.u32 a, %1, 0;\n bar.red.and.pred b, 1, %2, a;\n"
      " selp.u32 %0, 1, 0, b;\n}\n"
      : "=r"(r)
      : "r"(p ? 1u : 0u), "n"(kM2Workers)
      : "memory");
  return r != 0;
}

// Word j of this thread's read-back, from the three accumulators' fp32 bits.
__device__ __forceinline__ uint32_t d2_part(uint32_t f) {
  return static_cast<uint32_t>(__float2int_rn(__uint_as_float(f))) << 16;
}
__device__ __forceinline__ uint32_t small_part(uint32_t f) {  // |D| < 2^22
  return __float_as_uint(__uint_as_float(f) + 12582912.0f) - kMagicBits;
}

// One level, as plan_level_mma_kernel (same items, arguments and results).
__global__ void __launch_bounds__(kM2Threads, 1) plan_level_mma2_kernel(
    ranmar_state_t* __restrict__ st, uint64_t R, uint64_t n, uint32_t r_count, uint32_t items,
    const uint8_t* __restrict__ bimg, const uint32_t* __restrict__ cEd,
    const uint64_t* __restrict__ posE, uint32_t* status) {
  extern __shared__ __align__(16) uint32_t smem[];
  uint8_t* Bs = reinterpret_cast<uint8_t*>(smem);  // two B images
  uint8_t* stage = Bs + 2 * static_cast<size_t>(kBImgBytes);
  uint64_t* bars = reinterpret_cast<uint64_t*>(stage + kStageBytes);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 14);
  static_assert(14 * sizeof(uint64_t) + sizeof(uint32_t) <= 128, "barrier area");
  const uint32_t bfull0 = smem_addr(&bars[0]), bempty0 = smem_addr(&bars[2]);
  const uint32_t dfull0 = smem_addr(&bars[4]), dempty0 = smem_addr(&bars[7]);
  const uint32_t aready = smem_addr(&bars[10]), bar_src = smem_addr(&bars[11]);
  const uint32_t bar_drain = smem_addr(&bars[12]), bar_x = smem_addr(&bars[13]);
  const uint32_t test_limit = g_wait_limit;
  const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  const uint32_t q0 = static_cast<uint32_t>(static_cast<uint64_t>(blockIdx.x) * items / gridDim.x);
  const uint32_t q1 =
      static_cast<uint32_t>(static_cast<uint64_t>(blockIdx.x + 1) * items / gridDim.x);
  if (q0 >= q1) return;
  const uint32_t count = q1 - q0;

  auto b_addr = [&](uint32_t s) { return smem_addr(Bs) + s * kBImgBytes; };
  auto load_b = [&](uint32_t q, uint32_t s) {
    const uint8_t* src = bimg + static_cast<size_t>(q % r_count) * kBImgBytes;
    const uint32_t bar = bfull0 + 8 * s;
    mbar_expect_tx(bar, kBImgBytes);
    bulk_g2s(b_addr(s), src, kBImgBytes / 2, bar);
    bulk_g2s(b_addr(s) + kBImgBytes / 2, src + kBImgBytes / 2, kBImgBytes / 2, bar);
  };
  auto load_src = [&](uint64_t tile) {
    const uint64_t i0 = tile * kMmaM;
    const uint32_t bytes = static_cast<uint32_t>(R - i0 < kMmaM ? R - i0 : kMmaM) *
                           static_cast<uint32_t>(sizeof(ranmar_state_t));
    mbar_expect_tx(bar_src, bytes);
    bulk_g2s(smem_addr(stage), st + i0, bytes, bar_src);
  };

  if (tid == 0) {
    for (int b = 0; b < 7; ++b) mbar_init(smem_addr(&bars[b]), 1);             // bfull, bempty, dfull
    for (int b = 7; b < 11; ++b) mbar_init(smem_addr(&bars[b]), kM2Workers / 32);  // dempty, aready
    mbar_init(bar_src, 1);
    mbar_init(bar_drain, 1);
    mbar_init(bar_x, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    load_src(q0 / r_count);  // the first tile's rows, under the allocation
  }
  if (warp == 0) tmem_alloc(smem_addr(tmem_slot), kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  bool ok = true;

  if (warp == 8) {
    // ---------------- producer: B copies and MMAs (one thread) ----------------
    if (lane == 0) {
      uint32_t pend = 0;        // bit s: a copy into slot s not waited for yet
      uint32_t pend_par = 0;    // bit s: the parity that copy completes
      load_b(q0, 0);
      pend |= 1u;
      if (count > 1) {
        load_b(q0 + 1, 1);
        pend |= 2u;
      }
      // the CTA's later B images into L2 now, so that their copies into
      // shared memory, issued while the tensor core works, are short
      for (uint32_t qq = q0 + 2; qq < q1; ++qq)
        prefetch_l2(bimg + static_cast<size_t>(qq % r_count) * kBImgBytes, kBImgBytes);
      uint32_t tiles_seen = 0;
      int64_t cur_tile = -1;
      bool issued = false;
      if (test_limit) ok = mbar_wait(bar_x, 0, test_limit, true);
      for (uint32_t t = 0; t < count && ok; ++t) {
        const uint32_t q = q0 + t, s = t & 1u;
        const int64_t tile = static_cast<int64_t>(q / r_count);
        if (tile != cur_tile) {
          ok = mbar_wait(aready, tiles_seen & 1u);
          if (!ok) break;
          ++tiles_seen;
          cur_tile = tile;
        }
        ok = mbar_wait(bfull0 + 8 * s, (t >> 1) & 1u);
        if (!ok) break;
        pend &= ~(1u << s);
        tc_fence_after();
        const uint64_t bd = mma_desc(b_addr(s), kBLbo, kCoreSbo);
        // D2 (all K), D1 (A K [0,208) x B [104,312)), D0 (A [0,112) x B
        // [208,320)), each after the read-back of the previous item let it go
        if (t >= 1) {
          ok = mbar_wait(dempty0 + 8 * 2, (t - 1) & 1u);
          if (!ok) break;
          tc_fence_after();
        }
        mma_run_ta<20, 0>(tmem + kM2D2, tmem, bd);
        issued = true;
        mma_commit(dfull0 + 8 * 2);
        if (t >= 1 && t + 1 < count) {
          // item t+1 takes the slot of item t-1, free once its MMAs are done
          // (by now, behind this item's D2 group): its copy then lands while
          // the rest of this item is multiplied
          const uint32_t so = (t - 1) & 1u;
          ok = mbar_wait(bempty0 + 8 * so, ((t - 1) >> 1) & 1u);
          if (!ok) break;
          load_b(q + 1, so);
          pend |= 1u << so;
          pend_par = (pend_par & ~(1u << so)) | ((((t + 1) >> 1) & 1u) << so);
        }
        if (t >= 1) {
          ok = mbar_wait(dempty0 + 8 * 1, (t - 1) & 1u);
          if (!ok) break;
          tc_fence_after();
        }
        mma_run_ta<13, 13>(tmem + kM2D1, tmem, bd);
        mma_commit(dfull0 + 8 * 1);
        if (t >= 1) {
          ok = mbar_wait(dempty0 + 8 * 0, (t - 1) & 1u);
          if (!ok) break;
          tc_fence_after();
        }
        mma_run_ta<7, 26>(tmem + kM2D0, tmem, bd);
        mma_commit(dfull0 + 8 * 0);
        mma_commit(bempty0 + 8 * s);
      }
      if (!ok) flag_status(status, RANMAR_ST_TIMEOUT);
      // every MMA of the CTA done before the tensor memory is freed, every
      // copy into shared memory landed before the CTA exits (bounded)
      if (issued) {
        mma_commit(bar_drain);
        mbar_wait(bar_drain, 0);
      }
      for (uint32_t s = 0; s < 2; ++s)
        if (pend & (1u << s)) mbar_wait(bfull0 + 8 * s, (pend_par >> s) & 1u);
    }
  } else {
    // ---------------- readers: A build, read-back, stores ----------------
    const uint32_t quarter = warp & 3;
    const uint32_t m = quarter * 32 + lane;                 // tile row = TMEM lane
    const uint32_t lane_base = tmem + ((quarter * 32u) << 16);
    const bool lo_half = warp < 4;
    bool src_pending = (tid == 0);
    uint32_t changes = 0;
    int64_t cur_tile = -1;
    uint32_t src_c = 0;
    uint64_t src_pos = 0;
    for (uint32_t t = 0; t < count && ok; ++t) {
      const uint32_t q = q0 + t;
      const uint64_t tile = q / r_count;
      const uint32_t r = q % r_count + 1;
      const uint64_t i0 = tile * kMmaM;
      const uint32_t nsrc = static_cast<uint32_t>(R - i0 < kMmaM ? R - i0 : kMmaM);
      if (static_cast<int64_t>(tile) != cur_tile) {
        if (t > 0) {
          // the staging buffer holds the last store's rows until it has read them
          if (tid == 0) bulk_wait_read();
          ok = workers_sync_and(ok);
          if (!ok) break;
          if (tid == 0) {
            load_src(tile);
            src_pending = true;
          }
        }
        const bool s_ok = test_limit ? mbar_wait(bar_x, 0, test_limit, true)
                                     : mbar_wait(bar_src, changes & 1u);
        ok = workers_sync_and(s_ok);
        if (!ok) break;
        if (tid == 0) src_pending = false;
        // A image of row m: column c < 156 holds limb c / 52 of the words
        // (2(c % 52), 2(c % 52) + 1); columns 156..159 are zero.  Warp w < 4
        // writes columns 0..79 (limb 0, and limb 1 of the words 0..55),
        // warp w + 4 columns 80..159 (limb 1 of 56..103, limb 2, zeros).
        const uint32_t* x = reinterpret_cast<const uint32_t*>(stage) +
                            m * (sizeof(ranmar_state_t) / 4);
        uint32_t v[80];
#pragma unroll
        for (int pr = 0; pr < 52; ++pr) {
          const int k = 2 * pr;
          uint32_t a = 0, b = 0;
          if (m < nsrc) {
            if (k < kR) a = x[k];
            if (k + 1 < kR) b = x[k + 1];
          }
          uint32_t h[3];
          limb_pairs(a, b, h);
          if (lo_half) {
            v[pr] = h[0];                              // column pr
            if (pr < 28) v[52 + pr] = h[1];            // column 52 + pr
          } else {
            if (pr >= 28) v[pr - 28] = h[1];           // column 52 + pr (80 + pr - 28)
            v[24 + pr] = h[2];                         // column 104 + pr
          }
        }
        if (!lo_half) {
#pragma unroll
          for (int z = 76; z < 80; ++z) v[z] = 0u;     // columns 156..159
        }
        const uint32_t col0 = lo_half ? 0u : 80u;
#pragma unroll
        for (int c = 0; c < 5; ++c) tmem_st16(lane_base + col0 + 16 * c, v + 16 * c);
        tmem_st_wait();
        if (lo_half && m < nsrc) {
          const ranmar_state_t* srow = reinterpret_cast<const ranmar_state_t*>(stage) + m;
          src_c = srow->c;
          src_pos = srow->pos;
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(aready);
        ++changes;
        cur_tile = static_cast<int64_t>(tile);
      }

      // read-back: warp w < 4 takes the column chunks 0-2 and column 96,
      // warp w + 4 the chunks 3-5; D2, then D1, then D0, each released to the
      // next item's MMAs as soon as it is in registers
      const int c0 = lo_half ? 0 : 3;
      uint32_t p[49];
#pragma unroll
      for (int x = 2; x >= 0; --x) {
        const bool d_ok = mbar_wait(dfull0 + 8 * x, t & 1u);
        ok = workers_sync_and(d_ok);
        if (!ok) break;
        tc_fence_after();
        const uint32_t col = x == 2 ? kM2D2 : (x == 1 ? kM2D1 : kM2D0);
        uint32_t f[3][16], g[1] = {0u};
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) tmem_ld16(lane_base + col + 16 * (c0 + cc), f[cc]);
        if (lo_half) tmem_ld1(lane_base + col + 96, g);
        tmem_ld_wait();
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) tmem_regs_fence(f[cc]);
        tmem_regs_fence(g);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(dempty0 + 8 * x);
#pragma unroll
        for (int cc = 0; cc < 3; ++cc)
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const uint32_t fv = f[cc][j];
            if (x == 2) p[16 * cc + j] = d2_part(fv);
            else if (x == 1) p[16 * cc + j] += small_part(fv) << 8;
            else p[16 * cc + j] += small_part(fv);
          }
        if (x == 2) p[48] = d2_part(g[0]);
        else if (x == 1) p[48] += small_part(g[0]) << 8;
        else p[48] += small_part(g[0]);
      }
      if (!ok) break;

      // the new states into the staging buffer (after the last store read
      // it), then one bulk store of the tile's destination rows
      if (tid == 0) bulk_wait_read();
      ok = workers_sync_and(ok);
      if (!ok) break;
      const uint64_t dst0 = static_cast<uint64_t>(r) * R + i0;
      const uint32_t ndst =
          dst0 >= n ? 0u : static_cast<uint32_t>(min(static_cast<uint64_t>(nsrc), n - dst0));
      uint32_t* srow = reinterpret_cast<uint32_t*>(stage) + m * (sizeof(ranmar_state_t) / 4);
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) {
        uint4* o4 = reinterpret_cast<uint4*>(srow + 16 * (c0 + cc));
#pragma unroll
        for (int j = 0; j < 4; ++j)
          o4[j] = make_uint4(p[16 * cc + 4 * j] & kMask24, p[16 * cc + 4 * j + 1] & kMask24,
                             p[16 * cc + 4 * j + 2] & kMask24, p[16 * cc + 4 * j + 3] & kMask24);
      }
      if (lo_half) {
        srow[96] = p[48] & kMask24;
        ranmar_state_t* so = reinterpret_cast<ranmar_state_t*>(srow);
        so->c = sub_mod_m(src_c, cEd[r - 1]);
        so->pos = src_pos + posE[r - 1];
      }
      fence_proxy_async_smem();
      workers_sync_and(true);
      if (tid == 0 && ndst > 0)
        bulk_s2g(st + dst0, smem_addr(stage), ndst * static_cast<uint32_t>(sizeof(ranmar_state_t)));
    }
    if (!ok && tid == 0) flag_status(status, RANMAR_ST_TIMEOUT);
    if (tid == 0) {
      if (src_pending) mbar_wait(bar_src, changes & 1u);
      bulk_wait_read();
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

}  // namespace ranmar
