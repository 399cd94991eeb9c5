// ranmar_device.cuh -- constants and small device helpers shared by the
// libranmar kernels (RANMAR integer form, arXiv 2512.00093, Sec. 2-4).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "ranmar.h"

namespace ranmar {

// Parameters of Sec. 2 / Algorithm 3: lags (r, s) = (97, 33), M = 2^24,
// m = 2^24 - 3, d' = 7654321, c'_0 = 362436.
constexpr int kR = RANMAR_R;
constexpr int kS = RANMAR_S;
constexpr uint32_t kMask24 = 0x00FFFFFFu;
constexpr uint32_t kModM = 16777213u;
constexpr uint32_t kD = 7654321u;
constexpr uint32_t kC0 = 362436u;
constexpr int kMaxExpWords = RANMAR_MAX_EXP_WORDS;
constexpr unsigned kFull = 0xFFFFFFFFu;

static_assert(sizeof(ranmar_state_t) == 400, "state layout");
static_assert(sizeof(ranmar_desc_t) == 24, "descriptor layout");

// (a - b) mod m for a, b in [0, m).
__device__ __forceinline__ uint32_t sub_mod_m(uint32_t a, uint32_t b) {
  const uint32_t t = a - b;
  return (a < b) ? t + kModM : t;
}

// j * d mod m (one 64-bit product; used once per thread).
__device__ __forceinline__ uint32_t mul_d_mod_m(uint32_t j) {
  return static_cast<uint32_t>((static_cast<uint64_t>(j) * kD) % kModM);
}

__device__ __forceinline__ void flag_status(uint32_t* status, uint32_t bits) {
  if (status != nullptr) atomicOr(status, bits);
}

}  // namespace ranmar
