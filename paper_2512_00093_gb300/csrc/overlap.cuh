// overlap.cuh -- the non-overlap condition of the partition (Sec. 1).
//
// Stream k of (base, J) owns the transitions [kJ, (k+1)J) of the base's
// sequence.  A generation of `count` outputs from a state at position pos
// (transitions since the base, kept mod 2^64 in the state) stays inside
// stream k iff off = pos - kJ satisfies off <= J and count <= J - off.  The
// check runs in 64-bit arithmetic: off = pos - k (J mod 2^64) mod 2^64,
// exact whenever the true offset is below 2^64; for J >= 2^64 only
// off + count > 2^64 can leave the stream.
#pragma once

#include "ranmar_device.cuh"

namespace ranmar {

// One thread per descriptor; flags RANMAR_ST_OVERLAP (or BAD_INDEX).
__global__ void __launch_bounds__(256) overlap_check_kernel(
    const ranmar_state_t* __restrict__ states, uint64_t n_states,
    const ranmar_desc_t* __restrict__ desc, uint64_t n_desc, const uint64_t* __restrict__ k,
    uint64_t J_lo, int J_big, uint32_t* status) {
  for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < n_desc;
       i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    const ranmar_desc_t d = desc[i];
    if (d.state_idx >= n_states) {
      flag_status(status, RANMAR_ST_BAD_INDEX);
      continue;
    }
    const uint64_t off = states[d.state_idx].pos - k[i] * J_lo;  // mod 2^64
    const bool leaves = J_big ? (off != 0 && d.count > 0ull - off)   // off + count > 2^64
                              : (off > J_lo || d.count > J_lo - off);
    if (leaves) flag_status(status, RANMAR_ST_OVERLAP);
  }
}

}  // namespace ranmar
