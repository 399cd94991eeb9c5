// ranmar.cu -- the C ABI of libranmar (declared in include/ranmar.h).
//
// Host side: argument checks, Algorithm 3 seeding, launch configuration and
// CUDA error mapping.  Device side: generate.cuh (Algorithm 2 warp step) and
// jump.cuh (Sec. 3.1 / 3.2 jump-ahead).
#include <cstdio>
#include <cstring>

#include "ranmar.h"
#include "ranmar_device.cuh"
#include "generate.cuh"
#include "jump.cuh"

namespace {

thread_local char g_cuda_err[256] = "";

int cuda_fail(cudaError_t e) {
  std::snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", cudaGetErrorName(e),
                cudaGetErrorString(e));
  return RANMAR_ECUDA;
}

int check_launch() {
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? RANMAR_OK : cuda_fail(e);
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return x < y + nb && y < x + na;
}

// The two sub-generators that Algorithm 3 (Appendix A) draws its bits from:
// a lag-3 multiplicative sequence mod 179 over (i, j, k) and the congruential
// sequence l -> 53 l + 1 mod 169; a bit is set when (l m mod 64) >= 32.
struct SeedBits {
  int32_t i, j, k, l;
  explicit SeedBits(int32_t seed) {
    const int32_t ij = (seed - 1) / 30082;
    const int32_t kl = (seed - 1) - 30082 * ij;
    i = (ij / 177) % 177 + 2;
    j = ij % 177 + 2;
    k = (kl / 169) % 178 + 1;
    l = kl % 169;
  }
  bool next() {
    const int32_t m = (((i * j) % 179) * k) % 179;
    i = j;
    j = k;
    k = m;
    l = (53 * l + 1) % 169;
    return (l * m) % 64 >= 32;
  }
};

int launch_generate(bool f32, ranmar_state_t* states, size_t n_states, const ranmar_desc_t* desc,
                    size_t n_desc, void* out, size_t out_len, uint32_t* status,
                    ranmar_stream_t stream) {
  if (n_desc == 0) return RANMAR_OK;
  if (!states || !desc || !out) return RANMAR_EINVAL;
  if (n_states == 0) return RANMAR_ERANGE;
  if (!aligned(states, 16) || !aligned(desc, 8) || !aligned(out, 4)) return RANMAR_EINVAL;
  const int threads = 256;
  const uint64_t warps_per_block = threads / 32;
  uint64_t blocks = (n_desc + warps_per_block - 1) / warps_per_block;
  if (blocks > (1u << 20)) blocks = 1u << 20;   // grid-stride beyond ~8.4M descriptors
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (f32)
    ranmar::generate_desc_kernel<true><<<static_cast<unsigned>(blocks), threads, 0, s>>>(
        states, n_states, desc, n_desc, out, out_len, status);
  else
    ranmar::generate_desc_kernel<false><<<static_cast<unsigned>(blocks), threads, 0, s>>>(
        states, n_states, desc, n_desc, out, out_len, status);
  return check_launch();
}

int launch_plain(bool f32, ranmar_state_t* st, uint64_t count, void* out, int write_back,
                 ranmar_stream_t stream) {
  if (!st) return RANMAR_EINVAL;
  if (count > 0 && !out) return RANMAR_EINVAL;
  if (!aligned(st, 16) || !aligned(out, 4)) return RANMAR_EINVAL;
  if (count == 0 && !write_back) return RANMAR_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (f32)
    ranmar::generate_plain_kernel<true><<<1, 32, 0, s>>>(st, count, out, write_back);
  else
    ranmar::generate_plain_kernel<false><<<1, 32, 0, s>>>(st, count, out, write_back);
  return check_launch();
}

int launch_jump(const ranmar_state_t* base, size_t n_base, const uint32_t* base_idx,
                const uint32_t* exp, uint32_t exp_words, const ranmar::ExpParams& part,
                int mode, ranmar_state_t* out, size_t n, uint32_t* status,
                ranmar_stream_t stream) {
  const uint64_t per_cta = ranmar::kJumpStreamsPerWarp;   // one warp per CTA
  const uint64_t blocks = (n + per_cta - 1) / per_cta;
  if (blocks > 0x7FFFFFFFull) return RANMAR_ERANGE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  ranmar::jump_kernel<<<static_cast<unsigned>(blocks), 32, ranmar::kJumpSmemBytes, s>>>(
      base, n_base, base_idx, exp, exp_words, part, mode, out, n, status);
  return check_launch();
}

}  // namespace

extern "C" {

int ranmar_abi_version(void) { return (1 << 16) | 0; }

const char* ranmar_strerror(int code) {
  switch (code) {
    case RANMAR_OK: return "RANMAR_OK";
    case RANMAR_EINVAL: return "RANMAR_EINVAL: invalid argument (null, misaligned, overlap or seed)";
    case RANMAR_ERANGE: return "RANMAR_ERANGE: size or exponent out of range";
    case RANMAR_ECUDA: return "RANMAR_ECUDA: CUDA error (see ranmar_last_cuda_error)";
    case RANMAR_ENOMEM: return "RANMAR_ENOMEM: allocation failed";
    case RANMAR_EDEVICE: return "RANMAR_EDEVICE: unsupported or unusable device";
    default: return "RANMAR: unknown status";
  }
}

const char* ranmar_last_cuda_error(void) { return g_cuda_err; }

int ranmar_seed(int32_t seed, ranmar_state_t* h_out) {
  if (!h_out || seed < 1 || seed > 900000000) return RANMAR_EINVAL;
  SeedBits src(seed);
  uint32_t u[ranmar::kR];
  for (int w = 0; w < ranmar::kR; ++w) {
    uint32_t v = 0;
    for (int b = 23; b >= 0; --b)   // first draw is the 2^-1 digit
      if (src.next()) v |= 1u << b;
    u[w] = v;
  }
  // LAMMPS starts with i = 97, j = 33: the oldest word is u_97.
  for (int q = 0; q < ranmar::kR; ++q) h_out->x[q] = u[ranmar::kR - 1 - q];
  h_out->c = ranmar::kC0;
  h_out->pos = 0;
  return RANMAR_OK;
}

int ranmar_jump(const ranmar_state_t* d_base, size_t n_base, const uint32_t* d_base_idx,
                const uint32_t* d_exp, uint32_t exp_words, ranmar_state_t* d_out, size_t n,
                uint32_t* d_status, ranmar_stream_t stream) {
  if (n == 0) return RANMAR_OK;
  if (!d_base || !d_exp || !d_out) return RANMAR_EINVAL;
  if (exp_words < 1 || exp_words > RANMAR_MAX_EXP_WORDS || n_base == 0) return RANMAR_ERANGE;
  if (!aligned(d_base, 16) || !aligned(d_out, 16) || !aligned(d_exp, 4)) return RANMAR_EINVAL;
  if (overlaps(d_base, n_base * sizeof(ranmar_state_t), d_out, n * sizeof(ranmar_state_t)))
    return RANMAR_EINVAL;
  ranmar::ExpParams part{};
  return launch_jump(d_base, n_base, d_base_idx, d_exp, exp_words, part, 0, d_out, n, d_status,
                     stream);
}

int ranmar_partition(const ranmar_state_t* d_base, const uint32_t* h_J, uint32_t J_words,
                     uint64_t k0, ranmar_state_t* d_out, size_t n, ranmar_stream_t stream) {
  if (n == 0) return RANMAR_OK;
  if (!d_base || !h_J || !d_out) return RANMAR_EINVAL;
  if (J_words < 1 || J_words > RANMAR_MAX_EXP_WORDS) return RANMAR_ERANGE;
  if (!aligned(d_base, 16) || !aligned(d_out, 16)) return RANMAR_EINVAL;
  if (overlaps(d_base, sizeof(ranmar_state_t), d_out, n * sizeof(ranmar_state_t)))
    return RANMAR_EINVAL;
  // k_max = k0 + n - 1 must not wrap, and k_max * J must fit in 160 bits.
  if (n - 1 > UINT64_MAX - k0) return RANMAR_ERANGE;
  const uint64_t kmax = k0 + (n - 1);
  int jbits = 0;
  for (int w = 0; w < static_cast<int>(J_words); ++w)
    if (h_J[w]) jbits = 32 * w + 32 - __builtin_clz(h_J[w]);
  const int kbits = kmax ? 64 - __builtin_clzll(kmax) : 0;
  if (jbits + kbits > 32 * RANMAR_MAX_EXP_WORDS) return RANMAR_ERANGE;
  ranmar::ExpParams part{};
  for (uint32_t w = 0; w < J_words; ++w) part.J[w] = h_J[w];
  part.J_words = J_words;
  part.k0 = k0;
  return launch_jump(d_base, 1, nullptr, nullptr, 0, part, 1, d_out, n, nullptr, stream);
}

int ranmar_generate_u24(ranmar_state_t* d_states, size_t n_states, const ranmar_desc_t* d_desc,
                        size_t n_desc, uint32_t* d_out, size_t out_len, uint32_t* d_status,
                        ranmar_stream_t stream) {
  return launch_generate(false, d_states, n_states, d_desc, n_desc, d_out, out_len, d_status,
                         stream);
}

int ranmar_generate_f32(ranmar_state_t* d_states, size_t n_states, const ranmar_desc_t* d_desc,
                        size_t n_desc, float* d_out, size_t out_len, uint32_t* d_status,
                        ranmar_stream_t stream) {
  return launch_generate(true, d_states, n_states, d_desc, n_desc, d_out, out_len, d_status,
                         stream);
}

int ranmar_generate_plain_u24(ranmar_state_t* d_state, uint64_t count, uint32_t* d_out,
                              int write_back, ranmar_stream_t stream) {
  return launch_plain(false, d_state, count, d_out, write_back, stream);
}

int ranmar_generate_plain_f32(ranmar_state_t* d_state, uint64_t count, float* d_out,
                              int write_back, ranmar_stream_t stream) {
  return launch_plain(true, d_state, count, d_out, write_back, stream);
}

}  // extern "C"
