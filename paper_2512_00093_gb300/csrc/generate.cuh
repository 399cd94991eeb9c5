// generate.cuh -- warp-step generation of RANMAR outputs (Algorithm 2).
//
// One warp owns one stream.  With the state as a sequence X(q), the new word
// X(q) = X(q-97) - X(q-33) only depends on words at least 33 positions back,
// so the 32 lanes compute 32 consecutive words per step.  Because 97 and 33
// are both 1 mod 32, the two inputs of lane L sit at lane L-1 of blocks b-3
// and b-1.  The window is therefore kept ROTATED by one lane: register
// R_b[L] = X(32b + L - 1), lane 0 taking the last word of the previous block
// from a carry.  A step is then
//     X(32b + L) = R_{b-3}[L] - R_{b-1}[L]          (no data movement)
//     R_b[L]     = shfl(X, L - 1), lane 0 <- carry  (one shuffle)
// and the 97 state words are exactly R_{b-3}, R_{b-2}, R_{b-1} and the carry.
// c_n of each lane comes in closed form (Sec. 3.2): lane L of step b uses
// c_{32b+L+1} = (c_{32b} - (L+1) d) mod m.  Output (X - c) mod 2^24 is stored
// coalesced (32 consecutive words per warp store, streaming hint).
#pragma once

#include "ranmar_device.cuh"

namespace ranmar {

template <bool F32>
__device__ __forceinline__ void store_output(void* out, uint64_t idx, uint32_t y) {
  if constexpr (F32) {
    // y < 2^24 converts exactly; the power-of-two scale is exact (Sec. 4).
    __stcs(static_cast<float*>(out) + idx, __uint2float_rn(y) * (1.0f / 16777216.0f));
  } else {
    __stcs(static_cast<uint32_t*>(out) + idx, y);
  }
}

struct LaneConsts {
  uint32_t delta_lane;  // (L + 1) d mod m
  uint32_t delta32;     // 32 d mod m
};

__device__ __forceinline__ LaneConsts lane_consts(unsigned lane) {
  return LaneConsts{mul_d_mod_m(lane + 1), mul_d_mod_m(32)};
}

// One 32-word step; `older` holds R_{b-3} on entry and R_b on exit,
// `newer` holds R_{b-1}.
template <bool F32>
__device__ __forceinline__ void warp_step(uint32_t& older, uint32_t newer, uint32_t& carry,
                                          uint32_t& cb, const LaneConsts& k, unsigned lane,
                                          void* out, uint64_t& o) {
  const uint32_t xv = older - newer;               // X(32b + L), kept mod 2^32
  const uint32_t cl = sub_mod_m(cb, k.delta_lane);  // c_{32b+L+1}
  store_output<F32>(out, o, (xv - cl) & kMask24);
  o += 32;
  cb = sub_mod_m(cb, k.delta32);
  const uint32_t t = __shfl_sync(kFull, xv, (lane + 31) & 31);
  older = (lane == 0) ? carry : t;
  carry = t;
}

// Generates `count` outputs of *st into out[out_base + n], n < count, and
// optionally writes the advanced state back.  Called by all 32 lanes.
template <bool F32>
__device__ void generate_stream(ranmar_state_t* st, uint64_t count, void* out, uint64_t out_base,
                                bool write_back, unsigned lane, const LaneConsts& k) {
  const uint32_t* xs = st->x;
  uint32_t s0 = xs[lane];       // R_{-3}[L] = X(-97 + L)
  uint32_t s1 = xs[32 + lane];  // R_{-2}[L]
  uint32_t s2 = xs[64 + lane];  // R_{-1}[L]
  uint32_t carry = xs[96];      // X(-1)
  uint32_t cb = st->c;          // c_0 of this call
  const uint64_t pos0 = st->pos;

  const uint64_t nblk = count >> 5;
  const unsigned rem = static_cast<unsigned>(count & 31);
  uint64_t o = out_base + lane;

  uint64_t b = 0;
#pragma unroll 1
  for (; b + 3 <= nblk; b += 3) {
    warp_step<F32>(s0, s2, carry, cb, k, lane, out, o);
    warp_step<F32>(s1, s0, carry, cb, k, lane, out, o);
    warp_step<F32>(s2, s1, carry, cb, k, lane, out, o);
  }
  const unsigned left = static_cast<unsigned>(nblk - b);
  if (left >= 1) warp_step<F32>(s0, s2, carry, cb, k, lane, out, o);
  if (left >= 2) warp_step<F32>(s1, s0, carry, cb, k, lane, out, o);

  // Canonical roles after B = nblk full blocks: R_{B-3}, R_{B-2}, R_{B-1}.
  uint32_t rm3, rm2, rm1;
  if (left == 0) {
    rm3 = s0; rm2 = s1; rm1 = s2;
  } else if (left == 1) {
    rm3 = s1; rm2 = s2; rm1 = s0;
  } else {
    rm3 = s2; rm2 = s0; rm1 = s1;
  }

  // Ragged tail: one more block with masked stores.
  uint32_t xb = 0;
  uint32_t c_end = cb;
  if (rem != 0) {
    xb = rm3 - rm1;  // X(32B + L)
    const uint32_t cl = sub_mod_m(cb, k.delta_lane);
    if (lane < rem) store_output<F32>(out, o, (xb - cl) & kMask24);
    c_end = __shfl_sync(kFull, cl, rem - 1);
  }

  if (!write_back) return;
  __syncwarp();
  // Positions relative to 32B: rm3 = X(L-97), rm2 = X(L-65), rm1 = X(L-33),
  // carry (lane 0) = X(-1), xb = X(L).  New state word q = X(rem - 97 + q).
  uint32_t* xw = st->x;
  if (lane >= rem) xw[lane - rem] = rm3 & kMask24;
  xw[lane + 32 - rem] = rm2 & kMask24;
  xw[lane + 64 - rem] = rm1 & kMask24;
  if (lane == 0) xw[96 - rem] = carry & kMask24;
  if (lane < rem) xw[lane + 97 - rem] = xb & kMask24;
  if (lane == 0) {
    st->c = c_end;
    st->pos = pos0 + count;
  }
}

// Batch of descriptors, one warp per descriptor (grid-stride over warps).
template <bool F32>
__global__ void __launch_bounds__(256) generate_desc_kernel(
    ranmar_state_t* __restrict__ states, uint64_t n_states,
    const ranmar_desc_t* __restrict__ desc, uint64_t n_desc, void* out, uint64_t out_len,
    uint32_t* status) {
  const unsigned lane = threadIdx.x & 31;
  const uint64_t warp = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
  const LaneConsts k = lane_consts(lane);
#pragma unroll 1
  for (uint64_t w = warp; w < n_desc; w += nwarps) {
    const ranmar_desc_t d = desc[w];
    if (d.state_idx >= n_states) {
      if (lane == 0) flag_status(status, RANMAR_ST_BAD_INDEX);
      continue;
    }
    if (d.count > out_len || d.out_offset > out_len - d.count) {
      if (lane == 0) flag_status(status, RANMAR_ST_OUT_RANGE);
      continue;
    }
    generate_stream<F32>(states + d.state_idx, d.count, out, d.out_offset,
                         (d.flags & RANMAR_DESC_WRITE_BACK) != 0, lane, k);
  }
}

// One stream per launch (the per-stream comparator path): one warp.
template <bool F32>
__global__ void __launch_bounds__(32) generate_plain_kernel(ranmar_state_t* st, uint64_t count,
                                                            void* out, int write_back) {
  const unsigned lane = threadIdx.x & 31;
  generate_stream<F32>(st, count, out, 0, write_back != 0, lane, lane_consts(lane));
}

}  // namespace ranmar
