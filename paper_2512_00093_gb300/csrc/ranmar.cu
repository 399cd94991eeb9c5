// ranmar.cu -- the C ABI of libranmar (declared in include/ranmar.h).
//
// Host side: argument checks, Algorithm 3 seeding, launch configuration and
// CUDA error mapping.  Device side: generate.cuh (Algorithm 2 warp step) and
// jump.cuh (Sec. 3.1 / 3.2 jump-ahead).
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>

#include <nvtx3/nvToolsExt.h>

#include "ranmar.h"
#include "ranmar_device.cuh"
#include "generate.cuh"
#include "jump.cuh"
#include "square_mirror.cuh"
#include "batch.cuh"
#include "jump_table.cuh"
#include "jump_warp.cuh"
#include "partition_generate.cuh"
#include "plan.cuh"
#include "plan_mma.cuh"
#include "plan_mma2.cuh"
#include "lfg.cuh"
#include "overlap.cuh"
#include "generate_mixed.cuh"

// Batch handle: the workspace of the persistent path on one device.
struct ranmar_batch {
  int device;
  int num_sms;
  size_t capacity;             // streams the workspace can pack
  unsigned char* ws;           // device workspace (one cudaMalloc)
  unsigned long long* queue;   // work-queue counter of the persistent kernel
  uint64_t* total;             // grand total of a pack
  uint32_t* hist;              // bucket histogram
  uint32_t* cursor;            // bucket cursors
  uint64_t* tile_sums;         // ceil(capacity / 1024) tile sums
  uint64_t* tile_extra;        // the same for the extra pieces of a split pack
  ranmar_batch_config_t cfg;
};

// Fixed-base power table on one device.
struct ranmar_table {
  int device;
  uint32_t* rows;     // kTabRows x kTabRowWords
  int num_sms;
  int ctas_per_sm;    // 0 = one CTA per group of 16 streams (full grid)
  int jump_map;       // RANMAR_JUMP_MAP_*: lanes per stream of the table jumps
};

struct ranmar_plan {
  int device;
  const ranmar_table_t* table;  // not owned
  uint32_t J[RANMAR_MAX_EXP_WORDS];
  uint32_t J_words;
  size_t max_n;
  int levels;          // level t: R_t known streams -> R_t * radix(t)
  int mat_off[ranmar::kPlanMaxLevels];  // first matrix of each level
  uint32_t* mats;      // per level radix - 1 matrices of 97 x 112: M_{r R_t J}
  uint8_t* bimg;       // fp16 limb images of the same matrices
  uint32_t* ced;       // per matrix: (E mod m) d mod m
  uint64_t* pose;      // per matrix: E mod 2^64
  uint32_t* status;    // device status word of the tensor-core levels
  int method;          // RANMAR_PLAN_TENSOR or RANMAR_PLAN_IMAD
  int num_sms;
  unsigned ctas;       // CTAs of a tensor-core level (0: one per SM)
  uint32_t* jtable;    // powers of t^J: rows (j, d) = t^{d 2^{8j} J}, j < jt_windows
  int jt_windows;      // base-256 digits of k it covers (0: none)
  int jump_map;        // RANMAR_JUMP_MAP_*: lanes per stream of its jumps
};

struct ranmar_graph {
  cudaGraph_t graph;
  cudaGraphExec_t exec;
};

// Scratch of ranmar_batch_pack_static, for callers that cannot allocate:
// [0] grand total, [256] bucket histogram, [768] bucket cursors, [1280] tile
// sums for up to RANMAR_PACK_STATIC_MAX streams.  9,472 bytes on every GPU
// that loads the library, kept until the process exits.
constexpr size_t kStaticTiles = RANMAR_PACK_STATIC_MAX / ranmar::kScanTile;
static_assert(RANMAR_PACK_STATIC_MAX % ranmar::kScanTile == 0, "whole tiles");
static __device__ __align__(256) unsigned char g_pack_static[1280 + kStaticTiles * 8];

namespace {

thread_local char g_cuda_err[256] = "";

int cuda_fail(cudaError_t e) {
  std::snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", cudaGetErrorName(e),
                cudaGetErrorString(e));
  return RANMAR_ECUDA;
}

}  // namespace

namespace ranmar {
namespace host {
// The library's CUDA error mapping, for its other translation units.
int cuda_fail(cudaError_t e) { return ::cuda_fail(e); }
}  // namespace host
}  // namespace ranmar

namespace {

// Host-side failure injection (ranmar_debug_fail_next): the next launch
// check returns this code once.
std::atomic<int> g_fail_next{0};

int check_launch() {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e);
  return g_fail_next.exchange(0);
}

// A named NVTX range over one entry point (host side: the enqueue), so that
// a timeline tool shows which call issued which kernels.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

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

// Algorithm 3 (Appendix A) on the device: one thread per seed, the same two
// sub-generators as the host SeedBits, 97 x 24 bit draws, then the LAMMPS
// ring order (x_1..x_97 = u_97, ..., u_1), c = 362436, pos = 0.
__global__ void __launch_bounds__(128) seed_kernel(const int32_t* __restrict__ seeds, uint64_t n,
                                                   ranmar_state_t* __restrict__ out,
                                                   uint32_t* status) {
  const uint64_t t = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int32_t seed = seeds[t];
  if (seed < 1 || seed > 900000000) {
    ranmar::flag_status(status, RANMAR_ST_BAD_SEED);
    return;
  }
  const int32_t ij = (seed - 1) / 30082;
  const int32_t kl = (seed - 1) - 30082 * ij;
  int32_t i = (ij / 177) % 177 + 2, j = ij % 177 + 2, k = (kl / 169) % 178 + 1, l = kl % 169;
  uint32_t* x = out[t].x;
#pragma unroll 1
  for (int w = 0; w < ranmar::kR; ++w) {
    uint32_t v = 0;
#pragma unroll 4
    for (int b = 23; b >= 0; --b) {
      const int32_t m = (((i * j) % 179) * k) % 179;
      i = j;
      j = k;
      k = m;
      l = (53 * l + 1) % 169;
      if ((l * m) % 64 >= 32) v |= 1u << b;
    }
    x[ranmar::kR - 1 - w] = v;  // u_{w+1} is x_{97-w}
  }
  out[t].c = ranmar::kC0;
  out[t].pos = 0;
}

// Weighted checksum of 32-bit words: result[item.result] +=
// sum_i word[offset + i] * (2 (index0 + i) + 1) mod 2^64, one CTA per item.
// Each thread issues its 16-byte loads of a pass before it uses any: the
// words are read once, so for items of a few thousand words the load
// latency, not the bandwidth, sets the time.  Four words x_0..x_3 of weights
// w, w + 2, w + 4, w + 6 add w (x_0 + x_1 + x_2 + x_3) + 2 x_1 + 4 x_2 + 6 x_3.
__global__ void __launch_bounds__(256) checksum_kernel(const uint32_t* __restrict__ data,
                                                      const ranmar_sum_item_t* __restrict__ items,
                                                      uint64_t n_items, uint64_t data_len,
                                                      unsigned long long* __restrict__ results,
                                                      uint64_t n_results, uint32_t* status) {
  constexpr int kPass = 4;    // 16-byte loads in flight per thread
  __shared__ unsigned long long part[32];
  const unsigned tid = threadIdx.x, nt = blockDim.x;
  for (uint64_t it = blockIdx.x; it < n_items; it += gridDim.x) {
    const ranmar_sum_item_t w = items[it];
    if (w.result >= n_results || w.count > data_len || w.offset > data_len - w.count) {
      if (tid == 0) ranmar::flag_status(status, RANMAR_ST_OUT_RANGE);
      continue;
    }
    const uint32_t* p = data + w.offset;
    const uint64_t mis = (reinterpret_cast<uintptr_t>(p) >> 2) & 3;   // words past a 16-byte line
    const uint64_t head = min(static_cast<uint64_t>((4 - mis) & 3), w.count);
    const uint64_t nvec = (w.count - head) >> 2;
    const uint64_t tail0 = head + 4 * nvec;
    const uint4* v = reinterpret_cast<const uint4*>(p + head);
    const unsigned long long w0 = 2ull * w.index0 + 1ull;
    unsigned long long acc = 0;
    if (tid < head) acc += static_cast<unsigned long long>(p[tid]) * (w0 + 2ull * tid);
    if (tid < w.count - tail0)
      acc += static_cast<unsigned long long>(p[tail0 + tid]) * (w0 + 2ull * (tail0 + tid));
    for (uint64_t b = tid; b < nvec; b += static_cast<uint64_t>(kPass) * nt) {
      uint4 x[kPass];
#pragma unroll
      for (int u = 0; u < kPass; ++u) {
        const uint64_t q = b + static_cast<uint64_t>(u) * nt;
        x[u] = q < nvec ? v[q] : make_uint4(0u, 0u, 0u, 0u);
      }
#pragma unroll
      for (int u = 0; u < kPass; ++u) {
        const uint64_t q = b + static_cast<uint64_t>(u) * nt;
        const unsigned long long wt = w0 + 2ull * (head + 4 * q);
        const unsigned long long sum = static_cast<unsigned long long>(x[u].x) + x[u].y +
                                       x[u].z + x[u].w;
        acc += wt * sum + 2ull * x[u].y + 4ull * x[u].z + 6ull * x[u].w;
      }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) acc += __shfl_xor_sync(ranmar::kFull, acc, d);
    if ((tid & 31) == 0) part[tid >> 5] = acc;
    __syncthreads();
    if (tid == 0) {
      unsigned long long tot = 0;
      for (unsigned q = 0; q < nt / 32; ++q) tot += part[q];
      atomicAdd(&results[w.result], tot);
    }
    __syncthreads();
  }
}

int launch_generate(bool f32, ranmar_state_t* states, size_t n_states, const ranmar_desc_t* desc,
                    size_t n_desc, void* out, size_t out_len, uint32_t* status,
                    ranmar_stream_t stream) {
  if (n_desc == 0) return RANMAR_OK;
  if (!states || !desc || !out) return RANMAR_EINVAL;
  if (n_states == 0) return RANMAR_ERANGE;
  if (!aligned(states, 16) || !aligned(desc, 8) || !aligned(out, 4)) return RANMAR_EINVAL;
  const int threads = 256;
  const uint64_t warps_per_block = threads / 32;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // Shared memory the kernel does not use, reserved only to cap residency at
  // four CTAs (32 warps, 32 streams being written) per SM: the HBM write
  // rate falls with the number of output regions written at once, and four
  // CTAs measured faster than the six that the registers allow (the 2^28-
  // output launch 0.170 against 0.173 ms).  Below the 48 KB that needs no
  // attribute.
  constexpr size_t kGenResidencyCapSmem = 46 * 1024;
  uint64_t blocks = (n_desc + warps_per_block - 1) / warps_per_block;
  if (blocks > (1u << 20)) blocks = 1u << 20;   // grid-stride beyond ~8.4M descriptors
  if (f32)
    ranmar::generate_desc_kernel<true><<<static_cast<unsigned>(blocks), threads,
                                         kGenResidencyCapSmem, s>>>(
        states, n_states, desc, n_desc, out, out_len, status);
  else
    ranmar::generate_desc_kernel<false><<<static_cast<unsigned>(blocks), threads,
                                          kGenResidencyCapSmem, s>>>(
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
                ranmar_stream_t stream, const uint32_t* dst_idx = nullptr, size_t n_dst = 0) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (n <= RANMAR_SQUARE_WARP_AUTO_MAX) {
    // a small batch: a warp per stream shortens each stream's chain of squarings
    const uint64_t wblocks = (n + ranmar::kWarpJumpWarps - 1) / ranmar::kWarpJumpWarps;
    ranmar::jump_warp_kernel<<<static_cast<unsigned>(wblocks), 32 * ranmar::kWarpJumpWarps,
                               ranmar::kWarpJumpSmemBytes, s>>>(
        base, n_base, base_idx, exp, exp_words, part, mode, out, n, status, dst_idx, n_dst);
    return check_launch();
  }
  const uint64_t per_cta = ranmar::kJumpStreamsPerWarp;   // 16 streams per CTA (two warps)
  const uint64_t blocks = (n + per_cta - 1) / per_cta;
  if (blocks > 0x7FFFFFFFull) return RANMAR_ERANGE;
  ranmar::jump_kernel<<<static_cast<unsigned>(blocks), ranmar::kMirThreads, ranmar::kMirSmemBytes,
                        s>>>(
      base, n_base, base_idx, exp, exp_words, part, mode, out, n, status, dst_idx, n_dst);
  return check_launch();
}

// Resident CTAs an SM of a kernel at `threads` threads a CTA on the current
// device, queried once per (kernel, device, threads) and kept: the query
// costs about a microsecond of host time, and the serving engine launches a
// persistent kernel every iteration.
constexpr int kOccDevices = 64;
using OccCache = std::atomic<int>[kOccDevices][33];

template <typename K>
int cached_occupancy(K kernel, OccCache& cache, int threads) {
  int dev = -1;
  const bool keep = cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < kOccDevices &&
                    threads >= 32 && threads <= 1024 && threads % 32 == 0;
  if (keep) {
    const int v = cache[dev][threads / 32].load(std::memory_order_relaxed);
    if (v > 0) return v;
  }
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, 0);
  if (keep && nb > 0) cache[dev][threads / 32].store(nb, std::memory_order_relaxed);
  return nb;
}

template <int W, bool F32>
int persistent_occupancy(int threads) {
  static OccCache cache;
  return cached_occupancy(ranmar::generate_persistent_kernel<W, F32>, cache, threads);
}

template <int W, bool F32>
void persistent_launch(unsigned grid, unsigned threads, cudaStream_t s, ranmar_state_t* states,
                       size_t n_states, const ranmar_desc_t* desc, size_t n_desc,
                       const uint32_t* order, void* out, size_t out_len, uint32_t* status,
                       unsigned long long* queue, uint32_t chunk, int allow_wb) {
  ranmar::generate_persistent_kernel<W, F32><<<grid, threads, 0, s>>>(
      states, n_states, desc, n_desc, order, out, out_len, status, queue, chunk, allow_wb);
}

bool config_ok(const ranmar_batch_config_t& c) {
  const int w = c.lanes_per_stream;
  return (w == 32 || w == 16 || w == 8 || w == 4) && c.threads_per_cta >= 32 &&
         c.threads_per_cta <= 1024 && c.threads_per_cta % 32 == 0 && c.ctas_per_sm >= 0 &&
         c.ctas_per_sm <= 64 && c.chunk >= 1;
}

bool on_device(const ranmar_batch* b) {
  int dev = -1;
  return b && cudaGetDevice(&dev) == cudaSuccess && dev == b->device;
}

// Enqueues queue reset + persistent kernel with config c.
int run_persistent(ranmar_batch* b, const ranmar_batch_config_t& c, bool f32,
                   ranmar_state_t* states, size_t n_states, const ranmar_desc_t* desc,
                   size_t n_desc, const uint32_t* order, void* out, size_t out_len,
                   uint32_t* status, cudaStream_t s, int allow_wb) {
  const int W = c.lanes_per_stream, T = c.threads_per_cta;
  int occ = 0;
#define RANMAR_OCC(WW) \
  occ = f32 ? persistent_occupancy<WW, true>(T) : persistent_occupancy<WW, false>(T)
  switch (W) {
    case 32: RANMAR_OCC(32); break;
    case 16: RANMAR_OCC(16); break;
    case 8: RANMAR_OCC(8); break;
    default: RANMAR_OCC(4); break;
  }
#undef RANMAR_OCC
  if (occ < 1) return cuda_fail(cudaErrorInvalidConfiguration);
  const int per_sm = c.ctas_per_sm > 0 ? (c.ctas_per_sm < occ ? c.ctas_per_sm : occ) : occ;
  // Enough CTAs for the work, at most one resident wave.
  const uint64_t groups_needed = (n_desc + c.chunk - 1) / c.chunk;
  const uint64_t groups_per_cta = static_cast<uint64_t>(T / W);
  uint64_t grid = static_cast<uint64_t>(per_sm) * b->num_sms;
  const uint64_t need = (groups_needed + groups_per_cta - 1) / groups_per_cta;
  if (need < grid) grid = need;
  if (grid < 1) grid = 1;
  cudaError_t e = cudaMemsetAsync(b->queue, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return cuda_fail(e);
#define RANMAR_LAUNCH(WW)                                                                      \
  do {                                                                                         \
    if (f32)                                                                                   \
      persistent_launch<WW, true>(static_cast<unsigned>(grid), T, s, states, n_states, desc,   \
                                  n_desc, order, out, out_len, status, b->queue, c.chunk,      \
                                  allow_wb);                                                   \
    else                                                                                       \
      persistent_launch<WW, false>(static_cast<unsigned>(grid), T, s, states, n_states, desc,  \
                                   n_desc, order, out, out_len, status, b->queue, c.chunk,     \
                                   allow_wb);                                                  \
  } while (0)
  switch (W) {
    case 32: RANMAR_LAUNCH(32); break;
    case 16: RANMAR_LAUNCH(16); break;
    case 8: RANMAR_LAUNCH(8); break;
    default: RANMAR_LAUNCH(4); break;
  }
#undef RANMAR_LAUNCH
  return check_launch();
}

template <int W, int S>
int mixed_occupancy(int threads) {
  static OccCache cache;
  return cached_occupancy(ranmar::generate_persistent_mixed_kernel<W, S>, cache, threads);
}

// Enqueues queue reset + the mixed-type persistent kernel with config c: a
// stream a group (S = 1) when every descriptor's group can be resident at
// once, else the interleaved width of the other persistent kernels.
template <int W>
int launch_mixed(ranmar_batch* b, const ranmar_batch_config_t& c, int T, ranmar_state_t* states,
                 size_t n_states, const ranmar_desc_t* desc, size_t n_desc, size_t n_u24,
                 uint32_t* out, size_t out_len, uint32_t* status, cudaStream_t s,
                 const ranmar::MixedSums& sums) {
  constexpr int kIlp = ranmar::persistent_ilp<W>();
  const int occ1 = mixed_occupancy<W, 1>(T);
  const int per_sm1 = c.ctas_per_sm > 0 && c.ctas_per_sm < occ1 ? c.ctas_per_sm : occ1;
  const uint64_t groups_per_cta = static_cast<uint64_t>(T / W);
  const uint64_t groups_needed = (n_desc + c.chunk - 1) / c.chunk;
  const bool one = kIlp == 1 || groups_needed <= static_cast<uint64_t>(per_sm1) *
                                                     b->num_sms * groups_per_cta;
  const int occ = one ? occ1 : mixed_occupancy<W, kIlp>(T);
  if (occ < 1) return cuda_fail(cudaErrorInvalidConfiguration);
  const int per_sm = c.ctas_per_sm > 0 ? (c.ctas_per_sm < occ ? c.ctas_per_sm : occ) : occ;
  uint64_t grid = static_cast<uint64_t>(per_sm) * b->num_sms;
  const uint64_t need = (groups_needed + groups_per_cta - 1) / groups_per_cta;
  if (need < grid) grid = need;
  if (grid < 1) grid = 1;
  cudaError_t e = cudaMemsetAsync(b->queue, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return cuda_fail(e);
  if (one)
    ranmar::generate_persistent_mixed_kernel<W, 1><<<static_cast<unsigned>(grid), T, 0, s>>>(
        states, n_states, desc, n_desc, n_u24, out, out_len, status, b->queue, c.chunk, sums);
  else
    ranmar::generate_persistent_mixed_kernel<W, kIlp><<<static_cast<unsigned>(grid), T, 0, s>>>(
        states, n_states, desc, n_desc, n_u24, out, out_len, status, b->queue, c.chunk, sums);
  return check_launch();
}

int run_persistent_mixed(ranmar_batch* b, const ranmar_batch_config_t& c, ranmar_state_t* states,
                         size_t n_states, const ranmar_desc_t* desc, size_t n_desc,
                         size_t n_u24, uint32_t* out, size_t out_len, uint32_t* status,
                         cudaStream_t s, const ranmar::MixedSums& sums) {
  // the kernel is compiled for at most 256 threads a CTA (two CTAs an SM)
  const int T = c.threads_per_cta < 256 ? c.threads_per_cta : 256;
  switch (c.lanes_per_stream) {
    case 32:
      return launch_mixed<32>(b, c, T, states, n_states, desc, n_desc, n_u24, out, out_len,
                              status, s, sums);
    case 16:
      return launch_mixed<16>(b, c, T, states, n_states, desc, n_desc, n_u24, out, out_len,
                              status, s, sums);
    case 8:
      return launch_mixed<8>(b, c, T, states, n_states, desc, n_desc, n_u24, out, out_len,
                             status, s, sums);
    default:
      return launch_mixed<4>(b, c, T, states, n_states, desc, n_desc, n_u24, out, out_len,
                             status, s, sums);
  }
}

int batch_generate(ranmar_batch* b, bool f32, ranmar_state_t* states, size_t n_states,
                   const ranmar_desc_t* desc, size_t n_desc, const uint32_t* order, void* out,
                   size_t out_len, uint32_t* status, ranmar_stream_t stream) {
  if (!on_device(b)) return RANMAR_EINVAL;
  if (n_desc == 0) return RANMAR_OK;
  if (!states || !desc || !out) return RANMAR_EINVAL;
  if (n_states == 0) return RANMAR_ERANGE;
  if (!aligned(states, 16) || !aligned(desc, 8) || !aligned(out, 4) || !aligned(order, 4))
    return RANMAR_EINVAL;
  return run_persistent(b, b->cfg, f32, states, n_states, desc, n_desc, order, out, out_len,
                        status, reinterpret_cast<cudaStream_t>(stream), 1);
}

// Device address of g_pack_static on the current device.  In host code the
// symbol is only a host-side stand-in, so the address is looked up once per
// device with cudaGetSymbolAddress (with that device current) and cached.
// The cache is not invalidated by cudaDeviceReset (which unloads the module),
// so a process that resets a device must not call the static pack on it
// afterwards.
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
unsigned char* g_static_addr[kMaxDevices] = {};

int static_scratch(unsigned char** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e);
  if (dev < 0 || dev >= kMaxDevices) return RANMAR_EDEVICE;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_pack_static);
    if (e != cudaSuccess) return cuda_fail(e);
    g_static_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_static_addr[dev];
  return RANMAR_OK;
}

template <typename F>
int launch_alg1(ranmar_state_t* states, size_t n_states, const ranmar_desc_t* desc,
                       size_t n_desc, F* out, size_t out_len, uint32_t* status,
                       ranmar_stream_t stream) {
  if (n_desc == 0) return RANMAR_OK;
  if (!states || !desc || !out) return RANMAR_EINVAL;
  if (n_states == 0) return RANMAR_ERANGE;
  if (!aligned(states, 16) || !aligned(desc, 8) || !aligned(out, sizeof(F))) return RANMAR_EINVAL;
  uint64_t blocks = (n_desc + 7) / 8;
  if (blocks > (1u << 20)) blocks = 1u << 20;
  ranmar::generate_alg1_kernel<F><<<static_cast<unsigned>(blocks), 256, 0,
                                    reinterpret_cast<cudaStream_t>(stream)>>>(
      states, n_states, desc, n_desc, out, out_len, status);
  return check_launch();
}

// Validates a partition request (E = (k0 + i) J for i < n must fit in
// RANMAR_MAX_EXP_WORDS words) and fills the kernel parameters.
int partition_params(const uint32_t* h_J, uint32_t J_words, uint64_t k0, size_t n,
                     uint32_t flags, ranmar::ExpParams& part) {
  if (flags & ~static_cast<uint32_t>(RANMAR_JUMP_REDUCE_PERIOD)) return RANMAR_EINVAL;
  if (J_words < 1 || J_words > RANMAR_MAX_EXP_WORDS) return RANMAR_ERANGE;
  if (n - 1 > UINT64_MAX - k0) return RANMAR_ERANGE;
  const uint64_t kmax = k0 + (n - 1);
  int jbits = 0;
  for (int w = 0; w < static_cast<int>(J_words); ++w)
    if (h_J[w]) jbits = 32 * w + 32 - __builtin_clz(h_J[w]);
  const int kbits = kmax ? 64 - __builtin_clzll(kmax) : 0;
  if (jbits + kbits > 32 * RANMAR_MAX_EXP_WORDS) return RANMAR_ERANGE;
  part = ranmar::ExpParams{};
  for (uint32_t w = 0; w < J_words; ++w) part.J[w] = h_J[w];
  part.J_words = J_words;
  part.k0 = k0;
  part.flags = flags;
  return RANMAR_OK;
}

template <bool F32>
int launch_partition_generate(const ranmar_table_t* t, const ranmar_state_t* d_base,
                              const uint32_t* h_J, uint32_t J_words, uint64_t k0, size_t n,
                              uint64_t count, uint32_t flags, ranmar_state_t* d_states,
                              void* d_out, ranmar_stream_t stream) {
  if (!t || (flags & ~static_cast<uint32_t>(RANMAR_JUMP_REDUCE_PERIOD))) return RANMAR_EINVAL;
  if (n == 0) return RANMAR_OK;
  if (!d_base || !h_J || !d_states || (count > 0 && !d_out)) return RANMAR_EINVAL;
  if (!aligned(d_base, 16) || !aligned(d_states, 16) || !aligned(d_out, 4)) return RANMAR_EINVAL;
  if (count > 0 && n > SIZE_MAX / 4 / count) return RANMAR_ERANGE;
  if (overlaps(d_base, sizeof(ranmar_state_t), d_states, n * sizeof(ranmar_state_t)))
    return RANMAR_EINVAL;
  if (count > 0 && (overlaps(d_base, sizeof(ranmar_state_t), d_out, n * count * 4) ||
                    overlaps(d_states, n * sizeof(ranmar_state_t), d_out, n * count * 4)))
    return RANMAR_EINVAL;
  ranmar::ExpParams part;
  const int rc = partition_params(h_J, J_words, k0, n, flags, part);
  if (rc != RANMAR_OK) return rc;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != t->device) return RANMAR_EINVAL;
  uint64_t blocks = (n + ranmar::kJumpStreamsPerWarp - 1) / ranmar::kJumpStreamsPerWarp;
  if (blocks > 0x7FFFFFFFull) blocks = 0x7FFFFFFFull;
  ranmar::partition_generate_kernel<F32>
      <<<static_cast<unsigned>(blocks), 32, ranmar::kTabSmemBytes,
         reinterpret_cast<cudaStream_t>(stream)>>>(t->rows, d_base, part, d_states, n, count,
                                                    d_out);
  return check_launch();
}

// Shape of a general-lag jump; false for arguments out of range.
constexpr size_t kLfgSmemMax = 200 * 1024;

bool lfg_shape(uint32_t r, uint32_t s, uint32_t e, int method, ranmar::LfgShape& sh) {
  if (r < 2 || r > static_cast<uint32_t>(ranmar::kLfgMaxR) || s < 1 || s >= r || e < 1 || e > 32)
    return false;
  // method: classical, Karatsuba with an automatic depth, or Karatsuba with
  // exactly L levels (RANMAR_LFG_KARATSUBA_LEVELS(L), L = 1..6)
  int want_L = -1;
  if (method == RANMAR_LFG_KARATSUBA) want_L = 0;
  else if (method >= RANMAR_LFG_KARATSUBA_LEVELS(1) && method <= RANMAR_LFG_KARATSUBA_LEVELS(6))
    want_L = method - RANMAR_LFG_KARATSUBA_LEVELS(0);
  else if (method != RANMAR_LFG_CLASSICAL) return false;
  sh = ranmar::LfgShape{};
  sh.r = static_cast<int>(r);
  sh.s = static_cast<int>(s);
  sh.mask = e == 32 ? 0xFFFFFFFFu : ((1u << e) - 1u);
  const int R = sh.r;
  const int xwin = ranmar::lfg_sk(2 * R + 3) + 1;   // the skewed extended window
  auto a4 = [](int w) { return (w + 3) & ~3; };
  if (want_L == 0) want_L = R >= 1024 ? 2 : (R >= 512 ? 1 : -1);  // measured on GB300
  if (want_L > 0) {
    for (int L = 6; L >= 1; --L) {
      if (L != want_L) continue;
      const int M = (R + (1 << L) - 1) >> L;
      if (M < 8) continue;
      int p3 = 1;
      for (int q = 0; q < L; ++q) p3 *= 3;
      const int opnd = ranmar::lfg_opnd_words(M);
      const int size_a = a4(std::max(p3 * 2 * M, xwin));
      const int size_b = a4((p3 / 3) * 4 * M);
      const int N = M << L;
      const int words = a4(N) + p3 * opnd + size_a + size_b;
      if (static_cast<size_t>(words) * 4 > kLfgSmemMax) continue;
      sh.L = L;
      sh.M = M;
      sh.N = N;
      sh.pow3L = p3;
      sh.opnd = opnd;
      sh.off_p = 0;
      sh.off_ops = a4(N);
      sh.off_a = sh.off_ops + p3 * opnd;
      sh.off_b = sh.off_a + size_a;
      sh.words = sh.off_b + size_b;
      return true;
    }
    return false;   // that depth does not fit
  }
  // the classical product (also Karatsuba's fallback when no level fits)
  sh.L = 0;
  sh.M = R;
  sh.N = R;
  sh.pow3L = 1;
  sh.opnd = ranmar::lfg_opnd_words(R);
  sh.off_p = 0;
  sh.off_ops = a4(R);
  sh.off_a = sh.off_ops + sh.opnd;
  sh.off_b = sh.off_a + a4(std::max(2 * R, xwin));
  sh.words = sh.off_b;
  return true;
}

}  // namespace

extern "C" {

int ranmar_abi_version(void) { return (1 << 16) | 1; }

const char* ranmar_strerror(int code) {
  switch (code) {
    case RANMAR_OK: return "RANMAR_OK";
    case RANMAR_EINVAL: return "RANMAR_EINVAL: invalid argument (null, misaligned, overlap or seed)";
    case RANMAR_ERANGE: return "RANMAR_ERANGE: size or exponent out of range";
    case RANMAR_ECUDA: return "RANMAR_ECUDA: CUDA error (see ranmar_last_cuda_error)";
    case RANMAR_ENOMEM: return "RANMAR_ENOMEM: allocation failed";
    case RANMAR_EDEVICE: return "RANMAR_EDEVICE: unsupported or unusable device";
    case RANMAR_ETIME: return "RANMAR_ETIME: the serving run passed its time limit";
    case RANMAR_ESTATUS: return "RANMAR_ESTATUS: a kernel set a RANMAR_ST_* status bit";
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
  NvtxRange nvtx_("ranmar_jump");
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

int ranmar_poly_power(const uint32_t* d_exp, uint32_t exp_words, size_t n, uint32_t* d_poly,
                      ranmar_stream_t stream) {
  NvtxRange nvtx_("ranmar_poly_power");
  if (n == 0) return RANMAR_OK;
  if (!d_exp || !d_poly) return RANMAR_EINVAL;
  if (exp_words < 1 || exp_words > RANMAR_MAX_EXP_WORDS) return RANMAR_ERANGE;
  if (!aligned(d_exp, 4) || !aligned(d_poly, 4)) return RANMAR_EINVAL;
  if (overlaps(d_exp, n * exp_words * sizeof(uint32_t), d_poly,
               n * ranmar::kPolyWords * sizeof(uint32_t)))
    return RANMAR_EINVAL;
  if (n <= RANMAR_SQUARE_WARP_AUTO_MAX) {
    const uint64_t wblocks = (n + ranmar::kWarpJumpWarps - 1) / ranmar::kWarpJumpWarps;
    ranmar::poly_power_warp_kernel<<<static_cast<unsigned>(wblocks), 32 * ranmar::kWarpJumpWarps,
                                     ranmar::kWarpJumpSmemBytes,
                                     reinterpret_cast<cudaStream_t>(stream)>>>(d_exp, exp_words,
                                                                               d_poly, n);
    return check_launch();
  }
  const uint64_t blocks = (n + ranmar::kJumpStreamsPerWarp - 1) / ranmar::kJumpStreamsPerWarp;
  if (blocks > 0x7FFFFFFFull) return RANMAR_ERANGE;
  ranmar::poly_power_kernel<<<static_cast<unsigned>(blocks), ranmar::kMirThreads,
                              ranmar::kMirSmemBytes,
                              reinterpret_cast<cudaStream_t>(stream)>>>(d_exp, exp_words, d_poly,
                                                                        n);
  return check_launch();
}

int ranmar_partition(const ranmar_state_t* d_base, const uint32_t* h_J, uint32_t J_words,
                     uint64_t k0, ranmar_state_t* d_out, size_t n, ranmar_stream_t stream) {
  NvtxRange nvtx_("ranmar_partition");
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
  NvtxRange nvtx_("ranmar_generate_u24");
  return launch_generate(false, d_states, n_states, d_desc, n_desc, d_out, out_len, d_status,
                         stream);
}

int ranmar_generate_f32(ranmar_state_t* d_states, size_t n_states, const ranmar_desc_t* d_desc,
                        size_t n_desc, float* d_out, size_t out_len, uint32_t* d_status,
                        ranmar_stream_t stream) {
  NvtxRange nvtx_("ranmar_generate_f32");
  return launch_generate(true, d_states, n_states, d_desc, n_desc, d_out, out_len, d_status,
                         stream);
}

int ranmar_check_overlap(const ranmar_state_t* d_states, size_t n_states,
                         const ranmar_desc_t* d_desc, size_t n_desc, const uint64_t* d_k,
                         const uint32_t* h_J, uint32_t J_words, uint32_t* d_status,
                         ranmar_stream_t stream) {
  NvtxRange nvtx_("ranmar_check_overlap");
  if (!h_J) return RANMAR_EINVAL;
  if (J_words < 1 || J_words > RANMAR_MAX_EXP_WORDS) return RANMAR_ERANGE;
  bool zero = true, big = false;
  for (uint32_t w = 0; w < J_words; ++w) {
    zero = zero && h_J[w] == 0;
    big = big || (w >= 2 && h_J[w] != 0);
  }
  if (zero) return RANMAR_ERANGE;
  if (n_desc == 0) return RANMAR_OK;
  if (!d_states || !d_desc || !d_k || !d_status) return RANMAR_EINVAL;
  if (n_states == 0) return RANMAR_ERANGE;
  if (!aligned(d_states, 16) || !aligned(d_desc, 8) || !aligned(d_k, 8)) return RANMAR_EINVAL;
  const uint64_t J_lo = static_cast<uint64_t>(h_J[0]) |
                        (J_words > 1 ? static_cast<uint64_t>(h_J[1]) << 32 : 0ull);
  uint64_t blocks = (n_desc + 255) / 256;
  if (blocks > (1u << 20)) blocks = 1u << 20;
  ranmar::overlap_check_kernel<<<static_cast<unsigned>(blocks), 256, 0,
                                 reinterpret_cast<cudaStream_t>(stream)>>>(
      d_states, n_states, d_desc, n_desc, d_k, J_lo, big ? 1 : 0, d_status);
  return check_launch();
}

int ranmar_generate_plain_u24(ranmar_state_t* d_state, uint64_t count, uint32_t* d_out,
                              int write_back, ranmar_stream_t stream) {
  return launch_plain(false, d_state, count, d_out, write_back, stream);
}

int ranmar_generate_plain_f32(ranmar_state_t* d_state, uint64_t count, float* d_out,
                              int write_back, ranmar_stream_t stream) {
  return launch_plain(true, d_state, count, d_out, write_back, stream);
}

int ranmar_batch_create(size_t capacity, ranmar_batch_t** out) {
  if (!out) return RANMAR_EINVAL;
  *out = nullptr;
  if (capacity == 0 || capacity >= (static_cast<size_t>(1) << 32)) return RANMAR_ERANGE;
  ranmar_batch* b = new (std::nothrow) ranmar_batch{};
  if (!b) return RANMAR_ENOMEM;
  cudaError_t e = cudaGetDevice(&b->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
  if (e != cudaSuccess) {
    delete b;
    return cuda_fail(e);
  }
  const size_t n_tiles = (capacity + ranmar::kScanTile - 1) / ranmar::kScanTile;
  // [0] queue, [8] total, [256] hist (65 words), [768] cursor (65 words),
  // [1280] tile sums, then the tile sums of the extra pieces (split packs).
  const size_t bytes = 1280 + 2 * n_tiles * sizeof(uint64_t);
  e = cudaMalloc(&b->ws, bytes);
  if (e != cudaSuccess) {
    delete b;
    if (e == cudaErrorMemoryAllocation) {
      cudaGetLastError();
      return RANMAR_ENOMEM;
    }
    return cuda_fail(e);
  }
  b->capacity = capacity;
  b->queue = reinterpret_cast<unsigned long long*>(b->ws);
  b->total = reinterpret_cast<uint64_t*>(b->ws + 8);
  b->hist = reinterpret_cast<uint32_t*>(b->ws + 256);
  b->cursor = reinterpret_cast<uint32_t*>(b->ws + 768);
  b->tile_sums = reinterpret_cast<uint64_t*>(b->ws + 1280);
  b->tile_extra = b->tile_sums + n_tiles;
  static_assert(ranmar::kBuckets * sizeof(uint32_t) <= 512, "workspace layout");
  b->cfg = ranmar_batch_config_t{32, 256, 0, 1};
  *out = b;
  return RANMAR_OK;
}

int ranmar_batch_destroy(ranmar_batch_t* b) {
  if (!b) return RANMAR_OK;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(b->device);
  cudaDeviceSynchronize();
  const cudaError_t e = cudaFree(b->ws);
  if (prev >= 0) cudaSetDevice(prev);
  delete b;
  return e == cudaSuccess ? RANMAR_OK : cuda_fail(e);
}

int ranmar_batch_set_config(ranmar_batch_t* b, const ranmar_batch_config_t* cfg) {
  if (!b || !cfg || !config_ok(*cfg)) return RANMAR_EINVAL;
  b->cfg = *cfg;
  return RANMAR_OK;
}

int ranmar_batch_get_config(const ranmar_batch_t* b, ranmar_batch_config_t* cfg) {
  if (!b || !cfg) return RANMAR_EINVAL;
  *cfg = b->cfg;
  return RANMAR_OK;
}

int ranmar_batch_pack(ranmar_batch_t* b, const uint64_t* d_counts, size_t n, uint32_t flags,
                      ranmar_desc_t* d_desc, uint32_t* d_order, uint64_t* d_total,
                      ranmar_stream_t stream) {
  NvtxRange nvtx_("ranmar_batch_pack");
  if (!on_device(b)) return RANMAR_EINVAL;
  if (n > b->capacity) return RANMAR_ERANGE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  uint64_t* total = d_total ? d_total : b->total;
  if (n == 0) {
    if (!d_total) return RANMAR_OK;
    const cudaError_t e = cudaMemsetAsync(d_total, 0, sizeof(uint64_t), s);
    return e == cudaSuccess ? RANMAR_OK : cuda_fail(e);
  }
  if (!d_counts || !d_desc) return RANMAR_EINVAL;
  if (!aligned(d_counts, 8) || !aligned(d_desc, 8) || !aligned(d_order, 4) ||
      !aligned(d_total, 8))
    return RANMAR_EINVAL;
  const unsigned tiles = static_cast<unsigned>((n + ranmar::kScanTile - 1) / ranmar::kScanTile);
  cudaError_t e = cudaMemsetAsync(b->hist, 0, 1024, s);   // hist + cursor
  if (e != cudaSuccess) return cuda_fail(e);
  ranmar::pack_tile_sums<<<tiles, ranmar::kScanThreads, 0, s>>>(d_counts, n, b->tile_sums,
                                                                  b->hist);
  ranmar::pack_scan_tiles<<<1, ranmar::kScanThreads, 0, s>>>(b->tile_sums, tiles, total,
                                                               b->hist, b->cursor);
  ranmar::pack_write<<<tiles, ranmar::kScanThreads, 0, s>>>(d_counts, n, b->tile_sums, flags,
                                                              d_desc, b->cursor, d_order);
  return check_launch();
}

int ranmar_batch_pack_split(ranmar_batch_t* b, const uint64_t* d_counts, size_t n, uint64_t seg,
                            size_t n_extra, uint32_t flags, ranmar_desc_t* d_desc,
                            uint32_t* d_src, uint32_t* d_exp, uint64_t* d_total,
                            uint32_t* d_status, ranmar_stream_t stream) {
  NvtxRange nvtx_("ranmar_batch_pack_split");
  if (!on_device(b)) return RANMAR_EINVAL;
  if (seg == 0) return RANMAR_EINVAL;
  if (n > b->capacity || n + n_extra >= (static_cast<uint64_t>(1) << 32)) return RANMAR_ERANGE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  uint64_t* total = d_total ? d_total : b->total;
  if (n == 0) {
    if (n_extra) return RANMAR_EINVAL;
    if (!d_total) return RANMAR_OK;
    const cudaError_t e = cudaMemsetAsync(d_total, 0, sizeof(uint64_t), s);
    return e == cudaSuccess ? RANMAR_OK : cuda_fail(e);
  }
  if (!d_counts || !d_desc || (n_extra && (!d_src || !d_exp))) return RANMAR_EINVAL;
  if (!aligned(d_counts, 8) || !aligned(d_desc, 8) || !aligned(d_src, 4) || !aligned(d_exp, 4) ||
      !aligned(d_total, 8) || !aligned(d_status, 4))
    return RANMAR_EINVAL;
  const unsigned tiles = static_cast<unsigned>((n + ranmar::kScanTile - 1) / ranmar::kScanTile);
  ranmar::split_tile_sums<<<tiles, ranmar::kScanThreads, 0, s>>>(d_counts, n, seg, b->tile_sums,
                                                                   b->tile_extra);
  ranmar::split_scan_tiles<<<1, ranmar::kScanThreads, 0, s>>>(
      b->tile_sums, b->tile_extra, tiles, n, n_extra, total, d_desc, d_src, d_exp, d_status);
  ranmar::split_write<<<tiles, ranmar::kScanThreads, 0, s>>>(
      d_counts, n, seg, n_extra, b->tile_sums, b->tile_extra, flags, d_desc, d_src, d_exp);
  return check_launch();
}

int ranmar_batch_split_finish(ranmar_state_t* d_states, size_t n, const uint32_t* d_src,
                              size_t n_extra, ranmar_stream_t stream) {
  NvtxRange nvtx_("ranmar_batch_split_finish");
  if (n_extra == 0) return RANMAR_OK;
  if (!d_states || !d_src) return RANMAR_EINVAL;
  if (!aligned(d_states, 16) || !aligned(d_src, 4)) return RANMAR_EINVAL;
  uint64_t blocks = (n_extra + ranmar::kScanThreads - 1) / ranmar::kScanThreads;
  if (blocks > 65536) blocks = 65536;
  ranmar::split_finish<<<static_cast<unsigned>(blocks), ranmar::kScanThreads, 0,
                         reinterpret_cast<cudaStream_t>(stream)>>>(d_states, n, d_src, n_extra);
  return check_launch();
}

int ranmar_batch_generate_u24(ranmar_batch_t* b, ranmar_state_t* d_states, size_t n_states,
                              const ranmar_desc_t* d_desc, size_t n_desc,
                              const uint32_t* d_order, uint32_t* d_out, size_t out_len,
                              uint32_t* d_status, ranmar_stream_t stream) {
  NvtxRange nvtx_("ranmar_batch_generate_u24");
  return batch_generate(b, false, d_states, n_states, d_desc, n_desc, d_order, d_out, out_len,
                        d_status, stream);
}

int ranmar_batch_generate_f32(ranmar_batch_t* b, ranmar_state_t* d_states, size_t n_states,
                              const ranmar_desc_t* d_desc, size_t n_desc,
                              const uint32_t* d_order, float* d_out, size_t out_len,
                              uint32_t* d_status, ranmar_stream_t stream) {
  NvtxRange nvtx_("ranmar_batch_generate_f32");
  return batch_generate(b, true, d_states, n_states, d_desc, n_desc, d_order, d_out, out_len,
                        d_status, stream);
}

int ranmar_batch_generate_mixed(ranmar_batch_t* b, ranmar_state_t* d_states, size_t n_states,
                                const ranmar_desc_t* d_desc, size_t n_desc, size_t n_u24,
                                uint32_t* d_out, size_t out_len,
                                const ranmar_sum_item_t* d_items, uint64_t* d_results,
                                size_t n_results, uint32_t* d_status, ranmar_stream_t stream) {
  NvtxRange nvtx_("ranmar_batch_generate_mixed");
  if (!on_device(b)) return RANMAR_EINVAL;
  if (n_u24 > n_desc) return RANMAR_ERANGE;
  if (n_desc == 0) return RANMAR_OK;
  if (!d_states || !d_desc || !d_out || (d_items && !d_results)) return RANMAR_EINVAL;
  if (n_states == 0) return RANMAR_ERANGE;
  if (!aligned(d_states, 16) || !aligned(d_desc, 8) || !aligned(d_out, 4) ||
      !aligned(d_items, 8) || !aligned(d_results, 8))
    return RANMAR_EINVAL;
  const ranmar::MixedSums sums{d_items, reinterpret_cast<unsigned long long*>(d_results),
                               d_items ? n_results : 0};
  return run_persistent_mixed(b, b->cfg, d_states, n_states, d_desc, n_desc, n_u24, d_out,
                              out_len, d_status, reinterpret_cast<cudaStream_t>(stream), sums);
}

int ranmar_batch_tune(ranmar_batch_t* b, int f32, ranmar_state_t* d_states, size_t n_states,
                      const ranmar_desc_t* d_desc, size_t n_desc, const uint32_t* d_order,
                      void* d_out, size_t out_len, ranmar_stream_t stream, float* best_ms) {
  NvtxRange nvtx_("ranmar_batch_tune");
  if (!on_device(b)) return RANMAR_EINVAL;
  if (n_desc == 0) return RANMAR_OK;
  if (!d_states || !d_desc || !d_out) return RANMAR_EINVAL;
  if (n_states == 0) return RANMAR_ERANGE;
  if (!aligned(d_states, 16) || !aligned(d_desc, 8) || !aligned(d_out, 4) ||
      !aligned(d_order, 4))
    return RANMAR_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return cuda_fail(cudaGetLastError());
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(cudaGetLastError());
  }
  const int widths[] = {32, 16, 8};
  const int threads[] = {128, 256, 512};
  const int chunks[] = {1, 8};
  float best = 0.0f;
  ranmar_batch_config_t best_cfg = b->cfg;
  int rc = RANMAR_OK;
  for (int w : widths) {
    for (int t : threads) {
      for (int ch : chunks) {
        const ranmar_batch_config_t c{w, t, 0, ch};
        float ms_min = -1.0f;
        for (int rep = 0; rep < 3 && rc == RANMAR_OK; ++rep) {
          cudaEventRecord(e0, s);
          rc = run_persistent(b, c, f32 != 0, d_states, n_states, d_desc, n_desc, d_order, d_out,
                              out_len, nullptr, s, 0);
          cudaEventRecord(e1, s);
          const cudaError_t es = cudaEventSynchronize(e1);
          if (rc == RANMAR_OK && es != cudaSuccess) rc = cuda_fail(es);
          float ms = 0.0f;
          cudaEventElapsedTime(&ms, e0, e1);
          if (rep > 0 && (ms_min < 0.0f || ms < ms_min)) ms_min = ms;  // rep 0 warms up
        }
        if (rc != RANMAR_OK) break;
        if (best == 0.0f || ms_min < best) {
          best = ms_min;
          best_cfg = c;
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != RANMAR_OK) return rc;
  b->cfg = best_cfg;
  if (best_ms) *best_ms = best;
  return RANMAR_OK;
}

int ranmar_graph_begin(ranmar_stream_t stream) {
  if (!stream) return RANMAR_EINVAL;
  const cudaError_t e = cudaStreamBeginCapture(reinterpret_cast<cudaStream_t>(stream),
                                               cudaStreamCaptureModeThreadLocal);
  return e == cudaSuccess ? RANMAR_OK : cuda_fail(e);
}

int ranmar_graph_end(ranmar_stream_t stream, ranmar_graph_t** out) {
  if (!stream || !out) return RANMAR_EINVAL;
  *out = nullptr;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(reinterpret_cast<cudaStream_t>(stream), &g);
  if (e != cudaSuccess) return cuda_fail(e);
  ranmar_graph* r = new (std::nothrow) ranmar_graph{g, nullptr};
  if (!r) {
    cudaGraphDestroy(g);
    return RANMAR_ENOMEM;
  }
  e = cudaGraphInstantiate(&r->exec, g, 0);
  // upload now, so that the first launch does not pay for it
  if (e == cudaSuccess) e = cudaGraphUpload(r->exec, reinterpret_cast<cudaStream_t>(stream));
  if (e == cudaSuccess) e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) {
    if (r->exec) cudaGraphExecDestroy(r->exec);
    cudaGraphDestroy(g);
    delete r;
    return cuda_fail(e);
  }
  *out = r;
  return RANMAR_OK;
}

int ranmar_graph_launch(const ranmar_graph_t* g, ranmar_stream_t stream) {
  if (!g) return RANMAR_EINVAL;
  const cudaError_t e = cudaGraphLaunch(g->exec, reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? RANMAR_OK : cuda_fail(e);
}

int ranmar_graph_destroy(ranmar_graph_t* g) {
  if (!g) return RANMAR_OK;
  cudaGraphExecDestroy(g->exec);
  cudaGraphDestroy(g->graph);
  delete g;
  return RANMAR_OK;
}

int ranmar_batch_pack_static(const uint64_t* d_counts, size_t n, uint32_t flags,
                             ranmar_desc_t* d_desc, uint32_t* d_order, uint64_t* d_total,
                             ranmar_stream_t stream) {
  NvtxRange nvtx_("ranmar_batch_pack_static");
  if (n > RANMAR_PACK_STATIC_MAX) return RANMAR_ERANGE;
  if (n > 0 && (!d_counts || !d_desc)) return RANMAR_EINVAL;
  if (!aligned(d_counts, 8) || !aligned(d_desc, 8) || !aligned(d_order, 4) ||
      !aligned(d_total, 8))
    return RANMAR_EINVAL;
  unsigned char* ws = nullptr;
  const int rc = static_scratch(&ws);
  if (rc != RANMAR_OK) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  uint64_t* total = d_total ? d_total : reinterpret_cast<uint64_t*>(ws);
  if (n == 0) {
    if (!d_total) return RANMAR_OK;
    const cudaError_t e = cudaMemsetAsync(d_total, 0, sizeof(uint64_t), s);
    return e == cudaSuccess ? RANMAR_OK : cuda_fail(e);
  }
  uint32_t* hist = reinterpret_cast<uint32_t*>(ws + 256);
  uint32_t* cursor = reinterpret_cast<uint32_t*>(ws + 768);
  uint64_t* tile_sums = reinterpret_cast<uint64_t*>(ws + 1280);
  // The array keeps the previous call's contents: clear histogram + cursors.
  cudaError_t e = cudaMemsetAsync(hist, 0, 1024, s);
  if (e != cudaSuccess) return cuda_fail(e);
  const unsigned tiles = static_cast<unsigned>((n + ranmar::kScanTile - 1) / ranmar::kScanTile);
  ranmar::pack_tile_sums<<<tiles, ranmar::kScanThreads, 0, s>>>(d_counts, n, tile_sums, hist);
  ranmar::pack_scan_tiles<<<1, ranmar::kScanThreads, 0, s>>>(tile_sums, tiles, total, hist,
                                                               cursor);
  ranmar::pack_write<<<tiles, ranmar::kScanThreads, 0, s>>>(d_counts, n, tile_sums, flags, d_desc,
                                                              cursor, d_order);
  return check_launch();
}

int ranmar_jump_scatter(const ranmar_state_t* d_base, size_t n_base, const uint32_t* d_base_idx,
                        const uint32_t* d_exp, uint32_t exp_words, ranmar_state_t* d_dst,
                        size_t n_dst, const uint32_t* d_dst_idx, size_t n, uint32_t* d_status,
                        ranmar_stream_t stream) {
  NvtxRange nvtx_("ranmar_jump_scatter");
  if (n == 0) return RANMAR_OK;
  if (!d_base || !d_exp || !d_dst || !d_dst_idx) return RANMAR_EINVAL;
  if (exp_words < 1 || exp_words > RANMAR_MAX_EXP_WORDS || n_base == 0 || n_dst == 0)
    return RANMAR_ERANGE;
  if (!aligned(d_base, 16) || !aligned(d_dst, 16) || !aligned(d_exp, 4) ||
      !aligned(d_dst_idx, 4) || !aligned(d_base_idx, 4))
    return RANMAR_EINVAL;
  ranmar::ExpParams part{};
  return launch_jump(d_base, n_base, d_base_idx, d_exp, exp_words, part, 0, d_dst, n, d_status,
                     stream, d_dst_idx, n_dst);
}

int ranmar_checksum(const uint32_t* d_data, size_t data_len, const ranmar_sum_item_t* d_items,
                    size_t n_items, uint64_t* d_results, size_t n_results, uint32_t* d_status,
                    ranmar_stream_t stream) {
  NvtxRange nvtx_("ranmar_checksum");
  if (n_items == 0) return RANMAR_OK;
  if (!d_data || !d_items || !d_results) return RANMAR_EINVAL;
  if (!aligned(d_data, 4) || !aligned(d_items, 8) || !aligned(d_results, 8)) return RANMAR_EINVAL;
  const uint64_t grid = n_items < (1u << 20) ? n_items : (1u << 20);
  checksum_kernel<<<static_cast<unsigned>(grid), 256, 0,
                    reinterpret_cast<cudaStream_t>(stream)>>>(
      d_data, d_items, n_items, data_len, reinterpret_cast<unsigned long long*>(d_results),
      n_results, d_status);
  return check_launch();
}

int ranmar_table_create(ranmar_table_t** out) {
  NvtxRange nvtx_("ranmar_table_create");
  if (!out) return RANMAR_EINVAL;
  *out = nullptr;
  ranmar_table* t = new (std::nothrow) ranmar_table{};
  if (!t) return RANMAR_ENOMEM;
  cudaError_t e = cudaGetDevice(&t->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&t->num_sms, cudaDevAttrMultiProcessorCount, t->device);
  if (e == cudaSuccess) e = cudaMalloc(&t->rows, ranmar::kTabBytes);
  if (e != cudaSuccess) {
    delete t;
    if (e == cudaErrorMemoryAllocation) {
      cudaGetLastError();
      return RANMAR_ENOMEM;
    }
    return cuda_fail(e);
  }
  cudaStream_t s = nullptr;
  e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) {
    const unsigned blocks = (ranmar::kTabRows + ranmar::kJumpStreamsPerWarp - 1) /
                            ranmar::kJumpStreamsPerWarp;
    ranmar::table_build_kernel<<<blocks, ranmar::kMirThreads, ranmar::kMirSmemBytes, s>>>(
        t->rows);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  if (e != cudaSuccess) {
    cudaFree(t->rows);
    delete t;
    return cuda_fail(e);
  }
  *out = t;
  return RANMAR_OK;
}

int ranmar_table_destroy(ranmar_table_t* t) {
  if (!t) return RANMAR_OK;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(t->device);
  cudaDeviceSynchronize();
  const cudaError_t e = cudaFree(t->rows);
  if (prev >= 0) cudaSetDevice(prev);
  delete t;
  return e == cudaSuccess ? RANMAR_OK : cuda_fail(e);
}

int ranmar_table_set_ctas_per_sm(ranmar_table_t* t, int ctas_per_sm) {
  if (!t || ctas_per_sm < 0 || ctas_per_sm > 64) return RANMAR_EINVAL;
  t->ctas_per_sm = ctas_per_sm;
  return RANMAR_OK;
}

int ranmar_table_set_jump_mapping(ranmar_table_t* t, int map) {
  if (!t || map < RANMAR_JUMP_MAP_AUTO || map > RANMAR_JUMP_MAP_WARP) return RANMAR_EINVAL;
  t->jump_map = map;
  return RANMAR_OK;
}

int ranmar_plan_set_jump_mapping(ranmar_plan_t* p, int map) {
  if (!p || map < RANMAR_JUMP_MAP_AUTO || map > RANMAR_JUMP_MAP_WARP) return RANMAR_EINVAL;
  p->jump_map = map;
  return RANMAR_OK;
}

int ranmar_table_rows(const ranmar_table_t* t, const uint32_t** d_rows) {
  if (!t || !d_rows) return RANMAR_EINVAL;
  *d_rows = t->rows;
  return RANMAR_OK;
}

// Two lanes per stream do less work per output and win once the batch is
// around ten thousand streams; below that a warp per stream finishes sooner.
static bool use_warp_jump(int map, size_t n) {
  if (map == RANMAR_JUMP_MAP_WARP) return true;
  if (map == RANMAR_JUMP_MAP_PAIR) return false;
  return n <= RANMAR_JUMP_WARP_AUTO_MAX;
}

static int launch_jump_table(const ranmar_table_t* t, const ranmar_state_t* base, size_t n_base,
                             const uint32_t* base_idx, const uint32_t* exp, uint32_t exp_words,
                             const ranmar::ExpParams& part, int mode, ranmar_state_t* out,
                             size_t n, uint32_t* status, ranmar_stream_t stream,
                             const uint32_t* dst_idx, size_t n_dst) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != t->device) return RANMAR_EINVAL;
  const bool warp = use_warp_jump(t->jump_map, n);
  const uint64_t per_cta = warp ? ranmar::kWarpJumpWarps : ranmar::kJumpStreamsPerWarp;
  uint64_t blocks = (n + per_cta - 1) / per_cta;
  if (t->ctas_per_sm > 0) {
    const uint64_t cap = static_cast<uint64_t>(t->ctas_per_sm) * t->num_sms;
    if (blocks > cap) blocks = cap;   // the kernel strides over the rest
  }
  if (blocks > 0x7FFFFFFFull) blocks = 0x7FFFFFFFull;
  if (warp) {
    ranmar::jump_table_warp_kernel<<<static_cast<unsigned>(blocks), 32 * ranmar::kWarpJumpWarps,
                                     ranmar::kWarpJumpSmemBytes,
                                     reinterpret_cast<cudaStream_t>(stream)>>>(
        t->rows, base, n_base, base_idx, exp, exp_words, part, mode, out, n, status, dst_idx,
        n_dst);
    return check_launch();
  }
  ranmar::jump_table_kernel<<<static_cast<unsigned>(blocks), 32, ranmar::kTabSmemBytes,
                              reinterpret_cast<cudaStream_t>(stream)>>>(
      t->rows, base, n_base, base_idx, exp, exp_words, part, mode, out, n, status, dst_idx,
      n_dst);
  return check_launch();
}

int ranmar_jump_tab(const ranmar_table_t* t, const ranmar_state_t* d_base, size_t n_base,
                    const uint32_t* d_base_idx, const uint32_t* d_exp, uint32_t exp_words,
                    ranmar_state_t* d_dst, size_t n_dst, const uint32_t* d_dst_idx, size_t n,
                    uint32_t* d_status, ranmar_stream_t stream) {
  NvtxRange nvtx_("ranmar_jump_tab");
  if (!t) return RANMAR_EINVAL;
  if (n == 0) return RANMAR_OK;
  if (!d_base || !d_exp || !d_dst) return RANMAR_EINVAL;
  if (exp_words < 1 || exp_words > RANMAR_MAX_EXP_WORDS || n_base == 0) return RANMAR_ERANGE;
  if (d_dst_idx ? n_dst == 0 : n_dst < n) return RANMAR_ERANGE;
  if (!aligned(d_base, 16) || !aligned(d_dst, 16) || !aligned(d_exp, 4) ||
      !aligned(d_base_idx, 4) || !aligned(d_dst_idx, 4))
    return RANMAR_EINVAL;
  if (!d_dst_idx &&
      overlaps(d_base, n_base * sizeof(ranmar_state_t), d_dst, n * sizeof(ranmar_state_t)))
    return RANMAR_EINVAL;
  ranmar::ExpParams part{};
  return launch_jump_table(t, d_base, n_base, d_base_idx, d_exp, exp_words, part, 0, d_dst, n,
                           d_status, stream, d_dst_idx, n_dst);
}

int ranmar_partition_tab(const ranmar_table_t* t, const ranmar_state_t* d_base,
                         const uint32_t* h_J, uint32_t J_words, uint64_t k0,
                         ranmar_state_t* d_out, size_t n, ranmar_stream_t stream) {
  NvtxRange nvtx_("ranmar_partition_tab");
  if (!t) return RANMAR_EINVAL;
  if (n == 0) return RANMAR_OK;
  if (!d_base || !h_J || !d_out) return RANMAR_EINVAL;
  if (J_words < 1 || J_words > RANMAR_MAX_EXP_WORDS) return RANMAR_ERANGE;
  if (!aligned(d_base, 16) || !aligned(d_out, 16)) return RANMAR_EINVAL;
  if (overlaps(d_base, sizeof(ranmar_state_t), d_out, n * sizeof(ranmar_state_t)))
    return RANMAR_EINVAL;
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
  return launch_jump_table(t, d_base, 1, nullptr, nullptr, 0, part, 1, d_out, n, nullptr, stream,
                           nullptr, n);
}


int ranmar_partition_generate_u24(const ranmar_table_t* t, const ranmar_state_t* d_base,
                                  const uint32_t* h_J, uint32_t J_words, uint64_t k0, size_t n,
                                  uint64_t count, uint32_t flags, ranmar_state_t* d_states,
                                  uint32_t* d_out, ranmar_stream_t stream) {
  NvtxRange nvtx_("ranmar_partition_generate_u24");
  return launch_partition_generate<false>(t, d_base, h_J, J_words, k0, n, count, flags, d_states,
                                          d_out, stream);
}

int ranmar_partition_generate_f32(const ranmar_table_t* t, const ranmar_state_t* d_base,
                                  const uint32_t* h_J, uint32_t J_words, uint64_t k0, size_t n,
                                  uint64_t count, uint32_t flags, ranmar_state_t* d_states,
                                  float* d_out, ranmar_stream_t stream) {
  NvtxRange nvtx_("ranmar_partition_generate_f32");
  return launch_partition_generate<true>(t, d_base, h_J, J_words, k0, n, count, flags, d_states,
                                         d_out, stream);
}

int ranmar_plan_create(const ranmar_table_t* t, const uint32_t* h_J, uint32_t J_words,
                       size_t max_n, ranmar_plan_t** out) {
  NvtxRange nvtx_("ranmar_plan_create");
  if (!out) return RANMAR_EINVAL;
  *out = nullptr;
  if (!t || !h_J) return RANMAR_EINVAL;
  if (J_words < 1 || J_words > RANMAR_MAX_EXP_WORDS || max_n == 0 || max_n > (1ull << 32))
    return RANMAR_ERANGE;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != t->device) return RANMAR_EINVAL;
  int levels = 0;
  {
    uint64_t known = ranmar::kPlanBase;
    for (; known < max_n; known *= ranmar::plan_radix(levels)) ++levels;
  }
  ranmar_plan* p = new (std::nothrow) ranmar_plan{};
  if (!p) return RANMAR_ENOMEM;
  p->device = dev;
  p->table = t;
  for (uint32_t w = 0; w < J_words; ++w) p->J[w] = h_J[w];
  p->J_words = J_words;
  p->max_n = max_n;
  p->levels = levels;
  p->method = RANMAR_PLAN_TENSOR_PIPELINED;
  {
    cudaError_t e0 = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e0 == cudaSuccess) e0 = cudaMalloc(&p->status, sizeof(uint32_t));
    if (e0 == cudaSuccess) e0 = cudaMemset(p->status, 0, sizeof(uint32_t));
    if (e0 != cudaSuccess) {
      cudaFree(p->status);
      delete p;
      if (e0 == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return RANMAR_ENOMEM;
      }
      return cuda_fail(e0);
    }
  }
  {
    // the table of the powers of t^J: windows j with 255 * 2^{8j} J < 2^160,
    // at most the 8 windows of a 64-bit k
    int jbits = 0;
    for (uint32_t w = 0; w < J_words; ++w)
      if (h_J[w]) jbits = 32 * static_cast<int>(w) + 32 - __builtin_clz(h_J[w]);
    const int W = std::min(8, (32 * RANMAR_MAX_EXP_WORDS - jbits) / 8);
    cudaError_t e0 = cudaSuccess;
    cudaStream_t s0 = nullptr;
    if (W > 0) {
      const int rows = W * ranmar::kTabDigits;
      e0 = cudaMalloc(&p->jtable, sizeof(uint32_t) * ranmar::kTabRowWords * rows);
      if (e0 == cudaSuccess) e0 = cudaStreamCreateWithFlags(&s0, cudaStreamNonBlocking);
      if (e0 == cudaSuccess) {
        ranmar::ExpParams jp{};
        for (uint32_t w = 0; w < J_words; ++w) jp.J[w] = h_J[w];
        jp.J_words = J_words;
        ranmar::jtable_build_kernel<<<(rows + ranmar::kJumpStreamsPerWarp - 1) /
                                          ranmar::kJumpStreamsPerWarp,
                                      32, ranmar::kTabSmemBytes, s0>>>(t->rows, jp, W,
                                                                       p->jtable);
        e0 = cudaGetLastError();
      }
      if (e0 == cudaSuccess) e0 = cudaStreamSynchronize(s0);
      if (s0) cudaStreamDestroy(s0);
    }
    if (e0 != cudaSuccess) {
      cudaFree(p->jtable);
      cudaFree(p->status);
      delete p;
      if (e0 == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return RANMAR_ENOMEM;
      }
      return cuda_fail(e0);
    }
    p->jt_windows = W;
  }
  if (levels == 0) {
    *out = p;
    return RANMAR_OK;
  }
  // Exponents E = r R_t J (r = 1 .. radix(t) - 1), one per matrix; each matrix
  // row i is the unit state e_i jumped by E.
  int nmat = 0;
  uint64_t level_known[ranmar::kPlanMaxLevels];
  {
    uint64_t known = ranmar::kPlanBase;
    for (int tl = 0; tl < levels; ++tl) {
      p->mat_off[tl] = nmat;
      level_known[tl] = known;
      nmat += ranmar::plan_radix(tl) - 1;
      known *= ranmar::plan_radix(tl);
    }
  }
  const size_t nrows = static_cast<size_t>(nmat) * RANMAR_R;
  uint32_t* hexp = new (std::nothrow) uint32_t[nrows * RANMAR_MAX_EXP_WORDS];
  uint32_t* hidx = new (std::nothrow) uint32_t[nrows];
  uint32_t* hced = new (std::nothrow) uint32_t[nmat];
  uint64_t* hpos = new (std::nothrow) uint64_t[nmat];
  ranmar_state_t* hunit = new (std::nothrow) ranmar_state_t[RANMAR_R];
  int rc = (hexp && hidx && hced && hpos && hunit) ? RANMAR_OK : RANMAR_ENOMEM;
  for (int m = 0; rc == RANMAR_OK && m < nmat; ++m) {
    int tl = 0;
    while (tl + 1 < levels && m >= p->mat_off[tl + 1]) ++tl;
    const int r = m - p->mat_off[tl] + 1;
    const uint64_t mult = static_cast<uint64_t>(r) * level_known[tl];  // < 2^40
    uint32_t E[RANMAR_MAX_EXP_WORDS] = {0, 0, 0, 0, 0};
    unsigned __int128 carry = 0;
    for (int w = 0; w < RANMAR_MAX_EXP_WORDS; ++w) {
      const unsigned __int128 v =
          static_cast<unsigned __int128>(w < static_cast<int>(J_words) ? h_J[w] : 0u) * mult + carry;
      E[w] = static_cast<uint32_t>(v);
      carry = v >> 32;
    }
    if (carry != 0) {
      rc = RANMAR_ERANGE;
      break;
    }
    uint64_t em = 0;  // E mod m by Horner over 32-bit words
    for (int w = RANMAR_MAX_EXP_WORDS - 1; w >= 0; --w) em = ((em << 32) | E[w]) % ranmar::kModM;
    hced[m] = static_cast<uint32_t>((em * ranmar::kD) % ranmar::kModM);
    hpos[m] = (static_cast<uint64_t>(E[1]) << 32) | E[0];
    for (int i = 0; i < RANMAR_R; ++i) {
      const size_t q = static_cast<size_t>(m) * RANMAR_R + i;
      hidx[q] = static_cast<uint32_t>(i);
      for (int w = 0; w < RANMAR_MAX_EXP_WORDS; ++w) hexp[q * RANMAR_MAX_EXP_WORDS + w] = E[w];
    }
  }
  if (rc == RANMAR_OK) {
    std::memset(hunit, 0, sizeof(ranmar_state_t) * RANMAR_R);
    for (int i = 0; i < RANMAR_R; ++i) hunit[i].x[i] = 1u;
  }
  ranmar_state_t *dunit = nullptr, *djumped = nullptr;
  uint32_t *dexp = nullptr, *didx = nullptr;
  cudaStream_t s = nullptr;
  cudaError_t e = cudaSuccess;
  if (rc == RANMAR_OK) {
    e = cudaMalloc(&p->mats, nrows * ranmar::kPlanCols * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&p->bimg, static_cast<size_t>(nmat) * ranmar::kBImgBytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(ranmar::plan_level_mma_kernel,
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               static_cast<int>(ranmar::kMmaSmemBytes));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(ranmar::plan_level_mma2_kernel,
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               static_cast<int>(ranmar::kM2SmemBytes));
    if (e == cudaSuccess) e = cudaMalloc(&p->ced, nmat * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&p->pose, nmat * sizeof(uint64_t));
    if (e == cudaSuccess) e = cudaMalloc(&dunit, RANMAR_R * sizeof(ranmar_state_t));
    if (e == cudaSuccess) e = cudaMalloc(&djumped, nrows * sizeof(ranmar_state_t));
    if (e == cudaSuccess) e = cudaMalloc(&dexp, nrows * RANMAR_MAX_EXP_WORDS * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&didx, nrows * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(p->ced, hced, nmat * sizeof(uint32_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(p->pose, hpos, nmat * sizeof(uint64_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dunit, hunit, RANMAR_R * sizeof(ranmar_state_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dexp, hexp, nrows * RANMAR_MAX_EXP_WORDS * sizeof(uint32_t),
                          cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(didx, hidx, nrows * sizeof(uint32_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(ranmar::plan_level_kernel,
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               static_cast<int>(ranmar::kPlanSmemBytes));
    if (e == cudaSuccess) {
      ranmar::ExpParams none{};
      const int jr = launch_jump_table(t, dunit, RANMAR_R, didx, dexp, RANMAR_MAX_EXP_WORDS, none,
                                       0, djumped, nrows, nullptr,
                                       reinterpret_cast<ranmar_stream_t>(s), nullptr, nrows);
      if (jr != RANMAR_OK) e = cudaErrorLaunchFailure;
    }
    if (e == cudaSuccess) {
      ranmar::plan_pack_kernel<<<1024, 128, 0, s>>>(djumped, p->mats, nrows);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      ranmar::plan_bimg_kernel<<<1024, 256, 0, s>>>(djumped, p->bimg,
                                                    static_cast<uint32_t>(nmat));
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (s) cudaStreamDestroy(s);
    if (e != cudaSuccess) rc = (e == cudaErrorMemoryAllocation) ? RANMAR_ENOMEM : cuda_fail(e);
  }
  cudaFree(dunit);
  cudaFree(djumped);
  cudaFree(dexp);
  cudaFree(didx);
  delete[] hexp;
  delete[] hidx;
  delete[] hced;
  delete[] hpos;
  delete[] hunit;
  if (rc != RANMAR_OK) {
    cudaFree(p->mats);
    cudaFree(p->bimg);
    cudaFree(p->ced);
    cudaFree(p->pose);
    cudaFree(p->status);
    cudaFree(p->jtable);
    delete p;
    if (rc == RANMAR_ENOMEM) cudaGetLastError();
    return rc;
  }
  *out = p;
  return RANMAR_OK;
}

int ranmar_plan_destroy(ranmar_plan_t* p) {
  if (!p) return RANMAR_OK;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(p->device);
  cudaFree(p->mats);
  cudaFree(p->bimg);
  cudaFree(p->ced);
  cudaFree(p->pose);
  cudaFree(p->status);
  cudaFree(p->jtable);
  if (prev >= 0) cudaSetDevice(prev);
  delete p;
  return RANMAR_OK;
}

int ranmar_plan_set_method(ranmar_plan_t* p, int method) {
  if (!p || (method != RANMAR_PLAN_TENSOR && method != RANMAR_PLAN_IMAD &&
             method != RANMAR_PLAN_TENSOR_PIPELINED))
    return RANMAR_EINVAL;
  p->method = method;
  return RANMAR_OK;
}

int ranmar_plan_set_ctas(ranmar_plan_t* p, unsigned ctas) {
  if (!p || ctas > 65535u) return RANMAR_EINVAL;
  p->ctas = ctas;
  return RANMAR_OK;
}

int ranmar_debug_fail_next(int code) {
  if (code > 0 || code < RANMAR_EDEVICE) return RANMAR_EINVAL;
  g_fail_next.store(code);
  return RANMAR_OK;
}

int ranmar_debug_set_wait_limit(uint32_t iterations) {
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(ranmar::g_wait_limit, &iterations, sizeof(iterations));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return e == cudaSuccess ? RANMAR_OK : cuda_fail(e);
}

int ranmar_plan_status(const ranmar_plan_t* p, uint32_t** d_status) {
  if (!p || !d_status) return RANMAR_EINVAL;
  *d_status = p->status;
  return RANMAR_OK;
}

int ranmar_plan_expand(const ranmar_plan_t* p, ranmar_state_t* d_states, size_t n,
                       ranmar_stream_t stream) {
  NvtxRange nvtx_("ranmar_plan_expand");
  if (!p) return RANMAR_EINVAL;
  if (n <= static_cast<size_t>(ranmar::kPlanBase)) return RANMAR_OK;
  if (!d_states) return RANMAR_EINVAL;
  if (n > p->max_n) return RANMAR_ERANGE;
  if (!aligned(d_states, 16)) return RANMAR_EINVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) return RANMAR_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  uint64_t R = ranmar::kPlanBase;
  for (int tl = 0; tl < p->levels && R < n; R *= ranmar::plan_radix(tl), ++tl) {
    const uint64_t rmax = static_cast<uint64_t>(ranmar::plan_radix(tl) - 1);
    const uint64_t rc = (n - 1) / R < rmax ? (n - 1) / R : rmax;  // r = 1..rc: rR < n
    const int mo = p->mat_off[tl];
    if (p->method == RANMAR_PLAN_TENSOR_PIPELINED) {
      const uint64_t tiles = (R + ranmar::kMmaM - 1) / ranmar::kMmaM;
      const uint64_t items = tiles * rc;
      const uint64_t want = p->ctas ? p->ctas : static_cast<uint64_t>(p->num_sms);
      const unsigned grid = static_cast<unsigned>(items < want ? items : want);
      ranmar::plan_level_mma2_kernel<<<grid, ranmar::kM2Threads, ranmar::kM2SmemBytes, s>>>(
          d_states, R, n, static_cast<uint32_t>(rc), static_cast<uint32_t>(items),
          p->bimg + static_cast<size_t>(mo) * ranmar::kBImgBytes, p->ced + mo, p->pose + mo,
          p->status);
    } else if (p->method == RANMAR_PLAN_TENSOR) {
      // items (tile, r): tiles of 128 source rows
      const uint64_t tiles = (R + ranmar::kMmaM - 1) / ranmar::kMmaM;
      const uint64_t items = tiles * rc;
      const uint64_t want = p->ctas ? p->ctas : static_cast<uint64_t>(p->num_sms);
      const unsigned grid = static_cast<unsigned>(items < want ? items : want);
      ranmar::plan_level_mma_kernel<<<grid, ranmar::kMmaThreads, ranmar::kMmaSmemBytes, s>>>(
          d_states, R, n, static_cast<uint32_t>(rc), static_cast<uint32_t>(items),
          p->bimg + static_cast<size_t>(mo) * ranmar::kBImgBytes, p->ced + mo, p->pose + mo,
          p->status);
    } else {
      const dim3 grid(static_cast<unsigned>((R + ranmar::kPlanRows - 1) / ranmar::kPlanRows),
                      static_cast<unsigned>(rc));
      ranmar::plan_level_kernel<<<grid, ranmar::kPlanThreads, ranmar::kPlanSmemBytes, s>>>(
          d_states, R, n, p->mats + static_cast<size_t>(mo) * RANMAR_R * ranmar::kPlanCols,
          p->ced + mo, p->pose + mo);
    }
    const int lr = check_launch();
    if (lr != RANMAR_OK) return lr;
  }
  return RANMAR_OK;
}

// Streams k0 .. k0+n-1 by the plan's table of the powers of t^J, when it
// covers k0 + n - 1 (else RANMAR_ERANGE, nothing launched).
static int launch_jtable_partition(const ranmar_plan_t* p, const ranmar_state_t* d_base,
                                   const ranmar::ExpParams& part, size_t n,
                                   ranmar_state_t* d_out, ranmar_stream_t stream) {
  const uint64_t kmax = part.k0 + (n - 1);
  const int kbits = kmax ? 64 - __builtin_clzll(kmax) : 0;
  if (!p->jtable || kbits > 8 * p->jt_windows) return RANMAR_ERANGE;
  const bool warp = use_warp_jump(p->jump_map, n);
  const uint64_t per_cta = warp ? ranmar::kWarpJumpWarps : ranmar::kJumpStreamsPerWarp;
  uint64_t blocks = (n + per_cta - 1) / per_cta;
  if (blocks > 0x7FFFFFFFull) blocks = 0x7FFFFFFFull;
  if (warp) {
    ranmar::jump_jtable_warp_kernel<<<static_cast<unsigned>(blocks), 32 * ranmar::kWarpJumpWarps,
                                      ranmar::kWarpJumpSmemBytes,
                                      reinterpret_cast<cudaStream_t>(stream)>>>(
        p->jtable, d_base, part, d_out, n);
    return check_launch();
  }
  ranmar::jump_jtable_kernel<<<static_cast<unsigned>(blocks), 32, ranmar::kTabSmemBytes,
                               reinterpret_cast<cudaStream_t>(stream)>>>(p->jtable, d_base,
                                                                         part, d_out, n);
  return check_launch();
}

int ranmar_plan_jump(const ranmar_plan_t* p, const ranmar_state_t* d_base, uint64_t k0,
                     size_t n, ranmar_state_t* d_out, ranmar_stream_t stream) {
  NvtxRange nvtx_("ranmar_plan_jump");
  if (!p) return RANMAR_EINVAL;
  if (n == 0) return RANMAR_OK;
  if (!d_base || !d_out) return RANMAR_EINVAL;
  if (!aligned(d_base, 16) || !aligned(d_out, 16)) return RANMAR_EINVAL;
  if (overlaps(d_base, sizeof(ranmar_state_t), d_out, n * sizeof(ranmar_state_t)))
    return RANMAR_EINVAL;
  ranmar::ExpParams part;
  const int rc = partition_params(p->J, p->J_words, k0, n, 0, part);
  if (rc != RANMAR_OK) return rc;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) return RANMAR_EINVAL;
  return launch_jtable_partition(p, d_base, part, n, d_out, stream);
}

int ranmar_partition_plan(const ranmar_plan_t* p, const ranmar_state_t* d_base, uint64_t k0,
                          size_t n, ranmar_state_t* d_out, ranmar_stream_t stream) {
  NvtxRange nvtx_("ranmar_partition_plan");
  if (!p) return RANMAR_EINVAL;
  if (n == 0) return RANMAR_OK;
  if (!d_base || !d_out) return RANMAR_EINVAL;
  if (n > p->max_n) return RANMAR_ERANGE;
  if (!aligned(d_base, 16) || !aligned(d_out, 16)) return RANMAR_EINVAL;
  if (overlaps(d_base, sizeof(ranmar_state_t), d_out, n * sizeof(ranmar_state_t)))
    return RANMAR_EINVAL;
  ranmar::ExpParams part;
  const int rc = partition_params(p->J, p->J_words, k0, n, 0, part);
  if (rc != RANMAR_OK) return rc;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) return RANMAR_EINVAL;
  const size_t n0 = n < static_cast<size_t>(ranmar::kPlanBase) ? n : ranmar::kPlanBase;
  // the first streams by the table of the powers of t^J where it covers
  // them, else by the fixed-base table
  int jr = launch_jtable_partition(p, d_base, part, n0, d_out, stream);
  if (jr == RANMAR_ERANGE)
    jr = launch_jump_table(p->table, d_base, 1, nullptr, nullptr, 0, part, 1, d_out, n0,
                           nullptr, stream, nullptr, n0);
  if (jr != RANMAR_OK) return jr;
  return ranmar_plan_expand(p, d_out, n, stream);
}

int ranmar_lfg_karatsuba_levels(uint32_t r, uint32_t s, uint32_t e, int method) {
  ranmar::LfgShape sh;
  if (!lfg_shape(r, s, e, method, sh)) return RANMAR_EINVAL;
  return sh.L;
}

// Threads of a jump CTA (one stream per CTA): enough for the widest
// CTA-parallel step (the 4-output blocks of the leaf squarings, of the
// application), in whole warps, at least 64 and at most kLfgThreads; a small
// r then leaves room for more streams per SM instead of idle warps.  Every
// thread holds at most ceil(r / threads) <= 8 words in the shift by t.
static int lfg_jump_threads(const ranmar::LfgShape& sh) {
  const int sq = sh.pow3L * ((2 * sh.M + 3) / 4);
  const int ap = (sh.r + 3) / 4;
  int t = std::max(sq, ap);
  t = (t + 31) / 32 * 32;
  t = std::min(ranmar::kLfgThreads, std::max(64, t));
  while (t < ranmar::kLfgThreads && (sh.r + t - 1) / t > 8) t += 32;
  return t;
}

int ranmar_lfg_jump(uint32_t r, uint32_t s, uint32_t e, int method, const uint32_t* d_x,
                    size_t n_base, const uint32_t* d_base_idx, const uint32_t* d_exp,
                    uint32_t exp_words, uint32_t* d_out, size_t n, uint32_t* d_status,
                    ranmar_stream_t stream) {
  NvtxRange nvtx_("ranmar_lfg_jump");
  ranmar::LfgShape sh;
  if (!lfg_shape(r, s, e, method, sh)) return RANMAR_EINVAL;
  if (n == 0) return RANMAR_OK;
  if (!d_x || !d_exp || !d_out) return RANMAR_EINVAL;
  if (exp_words < 1 || exp_words > RANMAR_MAX_EXP_WORDS || n_base == 0) return RANMAR_ERANGE;
  if (!aligned(d_x, 4) || !aligned(d_out, 4) || !aligned(d_exp, 4) || !aligned(d_base_idx, 4))
    return RANMAR_EINVAL;
  if (overlaps(d_x, n_base * r * sizeof(uint32_t), d_out, n * r * sizeof(uint32_t)))
    return RANMAR_EINVAL;
  if (sh.L == 0 && sh.r <= ranmar::kLfgWarpMaxR) {
    // a warp per stream (classical squaring)
    uint64_t blocks = (n + ranmar::kLfgWarpWarps - 1) / ranmar::kLfgWarpWarps;
    if (blocks > 0x7FFFFFFFull) blocks = 0x7FFFFFFFull;
    ranmar::lfg_jump_warp_kernel<<<static_cast<unsigned>(blocks), 32 * ranmar::kLfgWarpWarps,
                                   ranmar::kLfgWarpSmemBytes,
                                   reinterpret_cast<cudaStream_t>(stream)>>>(
        sh.r, sh.s, sh.mask, d_x, n_base, d_base_idx, d_exp, exp_words, d_out, n, d_status);
    return check_launch();
  }
  const size_t smem = static_cast<size_t>(sh.words) * sizeof(uint32_t);
  const int threads = lfg_jump_threads(sh);
  cudaError_t ce = cudaFuncSetAttribute(ranmar::lfg_jump_kernel,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        static_cast<int>(smem));
  if (ce != cudaSuccess) return cuda_fail(ce);
  int dev = -1, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, ranmar::lfg_jump_kernel, threads,
                                                    smem) != cudaSuccess)
    return cuda_fail(cudaGetLastError());
  if (per < 1) return RANMAR_ERANGE;
  uint64_t grid = static_cast<uint64_t>(sms) * per;
  if (grid > n) grid = n;
  ranmar::lfg_jump_kernel<<<static_cast<unsigned>(grid), threads, smem,
                            reinterpret_cast<cudaStream_t>(stream)>>>(
      sh, d_x, n_base, d_base_idx, d_exp, exp_words, d_out, n, d_status);
  return check_launch();
}

int ranmar_lfg_generate(uint32_t r, uint32_t s, uint32_t e, uint32_t* d_x, size_t n,
                        uint64_t count, uint32_t* d_out, ranmar_stream_t stream) {
  NvtxRange nvtx_("ranmar_lfg_generate");
  ranmar::LfgShape sh;
  if (!lfg_shape(r, s, e, RANMAR_LFG_CLASSICAL, sh)) return RANMAR_EINVAL;
  if (n == 0 || count == 0) return RANMAR_OK;
  if (!d_x || !d_out) return RANMAR_EINVAL;
  if (!aligned(d_x, 4) || !aligned(d_out, 4)) return RANMAR_EINVAL;
  if (count > SIZE_MAX / 4 / n) return RANMAR_ERANGE;
  if (overlaps(d_x, n * r * sizeof(uint32_t), d_out, n * count * sizeof(uint32_t)))
    return RANMAR_EINVAL;
  const size_t smem = static_cast<size_t>(ranmar::kLfgGenWarps) * r * sizeof(uint32_t);
  cudaError_t ce = cudaFuncSetAttribute(ranmar::lfg_generate_kernel,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        static_cast<int>(smem));
  if (ce != cudaSuccess) return cuda_fail(ce);
  uint64_t grid = (n + ranmar::kLfgGenWarps - 1) / ranmar::kLfgGenWarps;
  if (grid > (1u << 20)) grid = 1u << 20;
  ranmar::lfg_generate_kernel<<<static_cast<unsigned>(grid), 32 * ranmar::kLfgGenWarps, smem,
                                reinterpret_cast<cudaStream_t>(stream)>>>(
      static_cast<int>(r), static_cast<int>(s), sh.mask, d_x, n, count, d_out);
  return check_launch();
}

int ranmar_generate_alg1_f32(ranmar_state_t* d_states, size_t n_states,
                             const ranmar_desc_t* d_desc, size_t n_desc, float* d_out,
                             size_t out_len, uint32_t* d_status, ranmar_stream_t stream) {
  NvtxRange nvtx_("ranmar_generate_alg1_f32");
  return launch_alg1<float>(d_states, n_states, d_desc, n_desc, d_out, out_len, d_status, stream);
}

int ranmar_generate_alg1_f64(ranmar_state_t* d_states, size_t n_states,
                             const ranmar_desc_t* d_desc, size_t n_desc, double* d_out,
                             size_t out_len, uint32_t* d_status, ranmar_stream_t stream) {
  NvtxRange nvtx_("ranmar_generate_alg1_f64");
  return launch_alg1<double>(d_states, n_states, d_desc, n_desc, d_out, out_len, d_status,
                             stream);
}

int ranmar_partition_ex(const ranmar_table_t* t, const ranmar_state_t* d_base, const uint32_t* h_J,
                        uint32_t J_words, uint64_t k0, ranmar_state_t* d_out, size_t n,
                        uint32_t flags, ranmar_stream_t stream) {
  NvtxRange nvtx_("ranmar_partition_ex");
  if (flags & ~static_cast<uint32_t>(RANMAR_JUMP_REDUCE_PERIOD)) return RANMAR_EINVAL;
  if (n == 0) return RANMAR_OK;
  if (!d_base || !h_J || !d_out) return RANMAR_EINVAL;
  if (J_words < 1 || J_words > RANMAR_MAX_EXP_WORDS) return RANMAR_ERANGE;
  if (!aligned(d_base, 16) || !aligned(d_out, 16)) return RANMAR_EINVAL;
  if (overlaps(d_base, sizeof(ranmar_state_t), d_out, n * sizeof(ranmar_state_t)))
    return RANMAR_EINVAL;
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
  part.flags = flags;
  if (t)
    return launch_jump_table(t, d_base, 1, nullptr, nullptr, 0, part, 1, d_out, n, nullptr,
                             stream, nullptr, n);
  return launch_jump(d_base, 1, nullptr, nullptr, 0, part, 1, d_out, n, nullptr, stream);
}

int ranmar_seed_batch(const int32_t* d_seeds, size_t n, ranmar_state_t* d_out, uint32_t* d_status,
                      ranmar_stream_t stream) {
  NvtxRange nvtx_("ranmar_seed_batch");
  if (n == 0) return RANMAR_OK;
  if (!d_seeds || !d_out) return RANMAR_EINVAL;
  if (!aligned(d_seeds, 4) || !aligned(d_out, 16)) return RANMAR_EINVAL;
  const uint64_t blocks = (n + 127) / 128;
  if (blocks > 0x7FFFFFFFull) return RANMAR_ERANGE;
  seed_kernel<<<static_cast<unsigned>(blocks), 128, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      d_seeds, n, d_out, d_status);
  return check_launch();
}

int ranmar_host_device_pointer(void* h_ptr, void** d_ptr) {
  if (!h_ptr || !d_ptr) return RANMAR_EINVAL;
  *d_ptr = nullptr;
  int dev = -1, mapped = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&mapped, cudaDevAttrCanMapHostMemory, dev);
  if (e != cudaSuccess) return cuda_fail(e);
  if (!mapped) return RANMAR_EDEVICE;
  e = cudaHostGetDevicePointer(d_ptr, h_ptr, 0);
  if (e != cudaSuccess) {
    *d_ptr = nullptr;
    return cuda_fail(e);
  }
  return RANMAR_OK;
}

}  // extern "C"
