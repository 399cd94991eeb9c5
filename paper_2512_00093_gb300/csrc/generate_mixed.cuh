// generate_mixed.cuh -- the persistent batch generation (Algorithm 2, the
// warp step of generate.cuh) for one descriptor list whose first n_u24
// descriptors produce 24-bit words and whose others produce float32 outputs
// (word * 2^-24), in ONE launch.  A serving iteration mixes both output
// types; two launches would each leave most of the GPU idle for the length
// of one segment.
#pragma once

#include "generate.cuh"

namespace ranmar {

// Checksums kept with the generation: item t (index0, result) applies to
// descriptor t's outputs, which the group reads back from memory after
// writing them (so the sum checks what was stored, as ranmar_checksum does).
struct MixedSums {
  const ranmar_sum_item_t* items;   // NULL: no checksums
  unsigned long long* results;
  uint64_t n_results;
};

// Descriptors [lo, hi) of one interleaved group (hi - lo <= S streams),
// all of one output type.
template <int W, int S, bool F32>
__device__ __forceinline__ void mixed_group(ranmar_state_t* __restrict__ states, uint64_t n_states,
                                            const ranmar_desc_t* __restrict__ desc, uint64_t lo,
                                            uint64_t hi, void* out, uint64_t out_len,
                                            uint32_t* status, unsigned gl, unsigned gmask,
                                            const LaneConsts& k, const MixedSums& sums) {
  ranmar_state_t* st[S];
  uint64_t cnt[S], ob[S];
  bool wb[S], ok[S];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const uint64_t t = lo + s;
    st[s] = states;
    cnt[s] = ob[s] = 0;
    wb[s] = ok[s] = false;
    if (t >= hi) continue;
    const ranmar_desc_t d = desc[t];
    if (!desc_ok(d, n_states, out_len, status, gl)) continue;
    st[s] = states + d.state_idx;
    cnt[s] = d.count;
    ob[s] = d.out_offset;
    wb[s] = (d.flags & RANMAR_DESC_WRITE_BACK) != 0;
    ok[s] = true;
  }
  generate_streams<W, F32, S, true>(st, cnt, out, ob, wb, ok, gl, gmask, k);
  if (sums.items == nullptr) return;
  __syncwarp(gmask);   // the group's stores are visible to the group
#pragma unroll
  for (int s = 0; s < S; ++s) {
    if (!ok[s]) continue;
    const ranmar_sum_item_t it = sums.items[lo + s];
    if (it.result >= sums.n_results) {
      if (gl == 0) flag_status(status, RANMAR_ST_OUT_RANGE);
      continue;
    }
    const uint32_t* p = static_cast<const uint32_t*>(out) + ob[s];
    const unsigned long long w0 = 2ull * it.index0 + 1ull;
    unsigned long long acc = 0;
#pragma unroll 4
    for (uint64_t i = gl; i < cnt[s]; i += W)
      acc += static_cast<unsigned long long>(p[i]) * (w0 + 2ull * i);
#pragma unroll
    for (int d = W / 2; d > 0; d >>= 1) acc += __shfl_xor_sync(gmask, acc, d, W);
    if (gl == 0) atomicAdd(&sums.results[it.result], acc);
  }
}

// Groups of W lanes pull `chunk` descriptors at a time from an atomic queue
// (*queue must be 0 at launch) in index order and generate them S at a time
// (interleaved; S = 1 when every descriptor can have a group of its own,
// which shortens the launch to the time of one stream); a group of streams
// that straddles n_u24 is generated as its u24 part, then its f32 part.
template <int W, int S>
__global__ void __launch_bounds__(256, 2) generate_persistent_mixed_kernel(ranmar_state_t* __restrict__ states,
                                                 uint64_t n_states,
                                                 const ranmar_desc_t* __restrict__ desc,
                                                 uint64_t n_desc, uint64_t n_u24, void* out,
                                                 uint64_t out_len, uint32_t* status,
                                                 unsigned long long* queue, uint32_t chunk,
                                                 MixedSums sums) {
  const unsigned lane = threadIdx.x & 31;
  const unsigned gl = lane % W;
  const unsigned gbase = lane - gl;
  const unsigned gmask = (W == 32) ? kFull : (((1u << W) - 1u) << gbase);
  const LaneConsts k = lane_consts<W>(gl);
#pragma unroll 1
  while (true) {
    unsigned long long base = 0;
    if (gl == 0) base = atomicAdd(queue, static_cast<unsigned long long>(chunk));
    base = __shfl_sync(gmask, base, gbase);
    if (base >= n_desc) break;
    const uint64_t end = min(static_cast<uint64_t>(base) + chunk, n_desc);
#pragma unroll 1
    for (uint64_t t0 = base; t0 < end; t0 += S) {
      const uint64_t hi = min(t0 + S, end);
      const uint64_t mid = min(max(t0, n_u24), hi);
      if (t0 < mid)
        mixed_group<W, S, false>(states, n_states, desc, t0, mid, out, out_len, status, gl, gmask,
                                 k, sums);
      if (mid < hi)
        mixed_group<W, S, true>(states, n_states, desc, mid, hi, out, out_len, status, gl, gmask,
                                k, sums);
    }
  }
}

}  // namespace ranmar
