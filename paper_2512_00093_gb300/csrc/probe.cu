// probe.cu -- roofline denominators measured on the running GPU (bench only).
//
// ranmar_probe_write: a store-only kernel over n 32-bit words (the HBM write
// ceiling for generation, which only stores), grid-stride;
// ranmar_probe_write_chunks: the same bytes written a chunk per warp (the
// store shape of generation; measured faster than the grid-stride order).  ranmar_probe_imad: independent
// chains of 32-bit multiply-add (the integer-pipe ceiling for the jump).
// Neither is part of the generator; both are timed by the caller with CUDA
// events on `stream`.  ranmar_probe_dadd: independent chains of
// double-precision adds (the FP64 rate that bounds Algorithm 1 in double).
#include <cstdint>
#include <cuda_runtime.h>

namespace {

__global__ void __launch_bounds__(256) probe_write_kernel(uint4* __restrict__ out, uint64_t n16,
                                                          uint32_t v) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n16;
       i += stride)
    __stcs(out + i, make_uint4(v, v + 1, v + 2, v + 3));
}

// Store-only, one warp per chunk of `chunk16` 16-byte words (the shape of
// generation, where a warp writes one stream's outputs): warp w writes
// chunk w with 512-byte warp stores, CTAs of 8 warps.
__global__ void __launch_bounds__(256) probe_write_chunks_kernel(uint4* __restrict__ out,
                                                                 uint32_t chunk16, uint32_t v) {
  const unsigned lane = threadIdx.x & 31;
  const uint64_t w = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  uint4* p = out + w * chunk16 + lane;
#pragma unroll 1
  for (uint32_t s = 0; s < chunk16; s += 32) __stcs(p + s, make_uint4(v, v + 1, v + 2, v + s));
}

// 16 independent multiply-add chains per thread, `iters` rounds each.
__global__ void __launch_bounds__(256) probe_imad_kernel(uint32_t* __restrict__ sink,
                                                         uint32_t iters, uint32_t seed) {
  uint32_t a[16];
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
  for (int k = 0; k < 16; ++k) a[k] = t * 2654435761u + seed + k;
  const uint32_t m = seed | 1u;
#pragma unroll 1
  for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 16; ++k) a[k] = a[k] * m + a[(k + 1) & 15];
  }
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < 16; ++k) s ^= a[k];
  if (s == 0x9E3779B9u) sink[t] = s;   // practically never; keeps the chains live
}

// 16 independent double-precision add chains per thread, `iters` rounds.
__global__ void __launch_bounds__(256) probe_dadd_kernel(double* __restrict__ sink,
                                                         uint32_t iters, double step) {
  double a[16];
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
  for (int k = 0; k < 16; ++k) a[k] = static_cast<double>(t + k) * 0.5;
#pragma unroll 1
  for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 16; ++k) a[k] = a[k] + step;
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 16; ++k) s += a[k];
  if (s == -1.0) sink[t] = s;   // never (all terms positive); keeps the chains live
}

}  // namespace

extern "C" {

int ranmar_probe_write(void* d_out, uint64_t n_words, uint32_t blocks, void* stream) {
  if (!d_out || (reinterpret_cast<uintptr_t>(d_out) & 15) || (n_words & 3)) return -1;
  probe_write_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      static_cast<uint4*>(d_out), n_words / 4, 0x1234u);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// n_words 32-bit words in chunks of chunk_words (a multiple of 128, dividing
// n_words into a multiple of 8 chunks), one warp per chunk.
int ranmar_probe_write_chunks(void* d_out, uint64_t n_words, uint32_t chunk_words, void* stream) {
  if (!d_out || (reinterpret_cast<uintptr_t>(d_out) & 15) || chunk_words == 0 ||
      (chunk_words % 128) || (n_words % (8ull * chunk_words)))
    return -1;
  const uint64_t blocks = n_words / chunk_words / 8;
  if (blocks > 0x7FFFFFFFull) return -2;
  probe_write_chunks_kernel<<<static_cast<unsigned>(blocks), 256, 0,
                              static_cast<cudaStream_t>(stream)>>>(static_cast<uint4*>(d_out),
                                                                   chunk_words / 4, 0x1234u);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// Multiply-adds issued: blocks * 256 * iters * 16.
int ranmar_probe_imad(uint32_t* d_sink, uint32_t blocks, uint32_t iters, void* stream) {
  if (!d_sink) return -1;
  probe_imad_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(d_sink, iters, 7u);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// Double-precision adds issued: blocks * 256 * iters * 16.
int ranmar_probe_dadd(double* d_sink, uint32_t blocks, uint32_t iters, void* stream) {
  if (!d_sink) return -1;
  probe_dadd_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(d_sink, iters,
                                                                          0.25);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // extern "C"
