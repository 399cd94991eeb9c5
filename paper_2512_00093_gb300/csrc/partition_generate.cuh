// partition_generate.cuh -- stream partitioning (Sec. 1) fused with
// generation (Algorithm 2) in one kernel.
//
// Each CTA (one warp) takes a group of 16 consecutive streams k = k0 + i:
// the lane pairs jump them with the fixed-base table (P_E for E = k J, the
// application, c_E; integer multiply-add bound), then the whole warp
// generates the 16 streams, four at a time interleaved (HBM-store bound),
// and writes each advanced state back.  With several CTAs per SM at
// different points of this cycle, the jumps of some overlap the stores of
// others on the same SM, which two separate kernels on two streams do not
// achieve (each fills the SMs while it runs).
//
// The jumped state passes through d_states (400 bytes per stream, written
// by the pairs and read back by the whole warp after __syncwarp, which
// orders the warp's memory accesses); it stays in L2.
#pragma once

#include "generate.cuh"
#include "jump_table.cuh"

namespace ranmar {

// Stream i = grp * 16 + slot: E = (k0 + i) J; outputs out[i count .. (i+1)
// count); d_states[i] = f^{E + count}(base).
template <bool F32>
__global__ void __launch_bounds__(32) partition_generate_kernel(
    const uint32_t* __restrict__ table, const ranmar_state_t* __restrict__ d_base, ExpParams part,
    ranmar_state_t* __restrict__ d_states, uint64_t n, uint64_t count, void* out) {
  extern __shared__ __align__(16) uint32_t smem[];
  const unsigned lane = threadIdx.x & 31;
  const unsigned g = lane >> 4, slot = lane & 15;
  uint32_t* a = smem + slot * kTabStreamWords;
  const LaneConsts k = lane_consts<32>(lane);
  const uint64_t groups = (n + kJumpStreamsPerWarp - 1) / kJumpStreamsPerWarp;
#pragma unroll 1
  for (uint64_t grp = blockIdx.x; grp < groups; grp += gridDim.x) {
    const uint64_t i0 = grp * kJumpStreamsPerWarp;
    const uint64_t i = i0 + slot;
    const bool active = i < n;
    uint32_t E[kMaxExpWords];
    load_exponent(E, active ? 1 : 0, nullptr, 0, part, i);
    table_jump_pair(table, d_base, E, part.flags, active, d_states + (active ? i : 0), a, g);
    __syncwarp();
    constexpr int S = 4;
#pragma unroll 1
    for (int q = 0; q < kJumpStreamsPerWarp; q += S) {
      ranmar_state_t* st[S];
      uint64_t cnt[S], ob[S];
      bool wb[S], ok[S];
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const uint64_t is = i0 + q + s;
        ok[s] = is < n;
        st[s] = d_states + (ok[s] ? is : 0);
        cnt[s] = count;
        ob[s] = is * count;
        wb[s] = true;
      }
      generate_streams<32, F32, S>(st, cnt, out, ob, wb, ok, lane, kFull, k);
    }
    __syncwarp();
  }
}

}  // namespace ranmar
