// batch.cuh -- packing a batch of uneven streams for the persistent kernel.
//
// From per-stream counts the device builds the descriptors (output offsets =
// exclusive prefix sum of the counts, so the outputs are packed back to
// back) and a longest-first visiting order (streams bucketed by
// floor(log2(count)), buckets in decreasing order), which keeps the
// persistent kernel's tail short.  The order within a bucket is whatever the
// atomics give; it does not affect any output, because every descriptor
// writes only its own slice.
//
// Prefix sum: three passes over tiles of kScanTile counts -- tile sums,
// one-CTA scan of the tile sums, then the tile-local scans -- with the tile
// sums in the batch workspace.
#pragma once

#include "ranmar_device.cuh"

namespace ranmar {

constexpr int kScanThreads = 256;
constexpr int kScanPerThread = 4;
constexpr int kScanTile = kScanThreads * kScanPerThread;  // 1024 counts per CTA
constexpr int kBuckets = 65;                               // 0, or floor(log2(count)) + 1

// Exclusive scan of one value per thread across the CTA; returns the
// exclusive prefix and writes the CTA total to *total.
__device__ __forceinline__ uint64_t cta_exclusive_scan(uint64_t v, uint64_t* total) {
  __shared__ uint64_t warp_sums[kScanThreads / 32];
  const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t inc = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint64_t t = __shfl_up_sync(kFull, inc, d);
    if (lane >= static_cast<unsigned>(d)) inc += t;
  }
  if (lane == 31) warp_sums[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    uint64_t w = lane < kScanThreads / 32 ? warp_sums[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint64_t t = __shfl_up_sync(kFull, w, d);
      if (lane >= static_cast<unsigned>(d)) w += t;
    }
    if (lane < kScanThreads / 32) warp_sums[lane] = w;  // inclusive warp prefix
  }
  __syncthreads();
  const uint64_t before = warp ? warp_sums[warp - 1] : 0;
  *total = warp_sums[kScanThreads / 32 - 1];
  __syncthreads();
  return before + inc - v;
}

__device__ __forceinline__ int count_bucket(uint64_t c) {
  return c ? 64 - __clzll(static_cast<long long>(c)) : 0;  // 0 for empty, else log2 + 1
}

// Pass 1: sum of each tile of counts; also the bucket histogram.
__global__ void __launch_bounds__(kScanThreads) pack_tile_sums(const uint64_t* __restrict__ counts,
                                                               uint64_t n,
                                                               uint64_t* __restrict__ tile_sums,
                                                               uint32_t* __restrict__ hist) {
  __shared__ uint32_t local[kBuckets];  // this tile's histogram (one global add per bucket)
  for (int b = threadIdx.x; b < kBuckets; b += kScanThreads) local[b] = 0;
  __syncthreads();
  const uint64_t base = static_cast<uint64_t>(blockIdx.x) * kScanTile;
  uint64_t s = 0;
#pragma unroll
  for (int j = 0; j < kScanPerThread; ++j) {
    const uint64_t i = base + static_cast<uint64_t>(j) * kScanThreads + threadIdx.x;
    if (i < n) {
      const uint64_t c = counts[i];
      s += c;
      atomicAdd(&local[count_bucket(c)], 1u);
    }
  }
  uint64_t total;
  (void)cta_exclusive_scan(s, &total);  // its barriers also complete the histogram
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
  for (int b = threadIdx.x; b < kBuckets; b += kScanThreads)
    if (local[b]) atomicAdd(&hist[b], local[b]);
}

// Pass 2 (one CTA): exclusive scan of the tile sums in place; *grand_total
// receives the sum of all counts.  Also turns the bucket histogram into
// start positions, largest bucket first (cursor[b] = first slot of bucket b).
__global__ void __launch_bounds__(kScanThreads) pack_scan_tiles(uint64_t* __restrict__ tile_sums,
                                                                uint64_t n_tiles,
                                                                uint64_t* __restrict__ grand_total,
                                                                const uint32_t* __restrict__ hist,
                                                                uint32_t* __restrict__ cursor) {
  uint64_t carry = 0;
#pragma unroll 1
  for (uint64_t b0 = 0; b0 < n_tiles; b0 += kScanThreads) {
    const uint64_t i = b0 + threadIdx.x;
    const uint64_t v = i < n_tiles ? tile_sums[i] : 0;
    uint64_t total;
    const uint64_t ex = cta_exclusive_scan(v, &total);
    if (i < n_tiles) tile_sums[i] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0) {
    *grand_total = carry;
    uint32_t pos = 0;
    for (int b = kBuckets - 1; b >= 0; --b) {
      cursor[b] = pos;
      pos += hist[b];
    }
  }
}

// Pass 3: descriptors with packed offsets, and the longest-first order.
__global__ void __launch_bounds__(kScanThreads) pack_write(const uint64_t* __restrict__ counts,
                                                           uint64_t n,
                                                           const uint64_t* __restrict__ tile_off,
                                                           uint32_t flags,
                                                           ranmar_desc_t* __restrict__ desc,
                                                           uint32_t* __restrict__ cursor,
                                                           uint32_t* __restrict__ order) {
  const uint64_t base = static_cast<uint64_t>(blockIdx.x) * kScanTile;
  // Thread t owns counts base + 4t .. 4t+3 so that its local scan is serial.
  uint64_t c[kScanPerThread];
  uint64_t s = 0;
#pragma unroll
  for (int j = 0; j < kScanPerThread; ++j) {
    const uint64_t i = base + static_cast<uint64_t>(threadIdx.x) * kScanPerThread + j;
    c[j] = i < n ? counts[i] : 0;
    s += c[j];
  }
  uint64_t total;
  uint64_t off = tile_off[blockIdx.x] + cta_exclusive_scan(s, &total);
#pragma unroll
  for (int j = 0; j < kScanPerThread; ++j) {
    const uint64_t i = base + static_cast<uint64_t>(threadIdx.x) * kScanPerThread + j;
    if (i < n) {
      ranmar_desc_t d;
      d.state_idx = static_cast<uint32_t>(i);
      d.flags = flags;
      d.out_offset = off;
      d.count = c[j];
      desc[i] = d;
    }
    off += c[j];
  }
  if (!order) return;  // uniform over the CTA
  // The order: the tile reserves one range per bucket with a single global
  // add (from its own histogram), then places its streams inside the range
  // with shared-memory counters.
  __shared__ uint32_t cnt[kBuckets], start[kBuckets];
  for (int b = threadIdx.x; b < kBuckets; b += kScanThreads) cnt[b] = 0;
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kScanPerThread; ++j) {
    const uint64_t i = base + static_cast<uint64_t>(threadIdx.x) * kScanPerThread + j;
    if (i < n) atomicAdd(&cnt[count_bucket(c[j])], 1u);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < kBuckets; b += kScanThreads) {
    start[b] = cnt[b] ? atomicAdd(&cursor[b], cnt[b]) : 0u;
    cnt[b] = 0;
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kScanPerThread; ++j) {
    const uint64_t i = base + static_cast<uint64_t>(threadIdx.x) * kScanPerThread + j;
    if (i < n) {
      const int b = count_bucket(c[j]);
      order[start[b] + atomicAdd(&cnt[b], 1u)] = static_cast<uint32_t>(i);
    }
  }
}

// ---- Splitting long streams into pieces started by extra jumps ----------
// A stream of count c > seg becomes ceil(c / seg) pieces of at most seg
// outputs: piece 0 runs from the stream's own state, piece q >= 1 from that
// state jumped by q seg (Sec. 3.1: a jump by any E), so the persistent kernel
// never has one warp on a long stream while the others idle.  Layout of the
// n + n_extra descriptors: piece 0 of stream i at i (state i), the extra
// pieces in stream order from n on (extra piece e uses state n + e, and
// src[e] = its stream, exp[e] = q seg as two words).  Only a stream's last
// piece keeps the write-back flag.

__device__ __forceinline__ uint64_t split_extra(uint64_t c, uint64_t seg) {
  return c > seg ? (c - 1) / seg : 0;   // ceil(c / seg) - 1
}

// Pass 1: per-tile sums of the counts and of the extra pieces.
__global__ void __launch_bounds__(kScanThreads) split_tile_sums(
    const uint64_t* __restrict__ counts, uint64_t n, uint64_t seg,
    uint64_t* __restrict__ tile_sums, uint64_t* __restrict__ tile_extra) {
  const uint64_t base = static_cast<uint64_t>(blockIdx.x) * kScanTile;
  uint64_t s = 0, x = 0;
#pragma unroll
  for (int j = 0; j < kScanPerThread; ++j) {
    const uint64_t i = base + static_cast<uint64_t>(j) * kScanThreads + threadIdx.x;
    if (i < n) {
      const uint64_t c = counts[i];
      s += c;
      x += split_extra(c, seg);
    }
  }
  uint64_t ts, tx;
  (void)cta_exclusive_scan(s, &ts);
  (void)cta_exclusive_scan(x, &tx);
  if (threadIdx.x == 0) {
    tile_sums[blockIdx.x] = ts;
    tile_extra[blockIdx.x] = tx;
  }
}

// Pass 2 (one CTA): exclusive scans of both tile arrays; *grand_total is the
// sum of the counts.  If the extra pieces do not number n_extra, the status
// gets RANMAR_ST_OUT_RANGE and the descriptors the caller sized for pieces
// that do not exist become empty ones (count 0, stream index UINT32_MAX).
__global__ void __launch_bounds__(kScanThreads) split_scan_tiles(
    uint64_t* __restrict__ tile_sums, uint64_t* __restrict__ tile_extra, uint64_t n_tiles,
    uint64_t n, uint64_t n_extra, uint64_t* __restrict__ grand_total,
    ranmar_desc_t* __restrict__ desc, uint32_t* __restrict__ src, uint32_t* __restrict__ exp,
    uint32_t* status) {
  uint64_t carry = 0, xcarry = 0;
#pragma unroll 1
  for (uint64_t b0 = 0; b0 < n_tiles; b0 += kScanThreads) {
    const uint64_t i = b0 + threadIdx.x;
    const uint64_t v = i < n_tiles ? tile_sums[i] : 0;
    const uint64_t w = i < n_tiles ? tile_extra[i] : 0;
    uint64_t total, xtotal;
    const uint64_t ex = cta_exclusive_scan(v, &total);
    const uint64_t xex = cta_exclusive_scan(w, &xtotal);
    if (i < n_tiles) {
      tile_sums[i] = carry + ex;
      tile_extra[i] = xcarry + xex;
    }
    carry += total;
    xcarry += xtotal;
  }
  if (threadIdx.x == 0) *grand_total = carry;
  if (xcarry != n_extra) {
    if (threadIdx.x == 0) flag_status(status, RANMAR_ST_OUT_RANGE);
    for (uint64_t e = xcarry + threadIdx.x; e < n_extra; e += kScanThreads) {
      ranmar_desc_t d;
      d.state_idx = static_cast<uint32_t>(n + e);
      d.flags = 0;
      d.out_offset = 0;
      d.count = 0;
      desc[n + e] = d;
      src[e] = 0xFFFFFFFFu;
      exp[2 * e] = 0u;
      exp[2 * e + 1] = 0u;
    }
  }
}

// Pass 3: the pieces' descriptors, and for the extra pieces their stream and
// jump exponent.
__global__ void __launch_bounds__(kScanThreads) split_write(
    const uint64_t* __restrict__ counts, uint64_t n, uint64_t seg, uint64_t n_extra,
    const uint64_t* __restrict__ tile_off, const uint64_t* __restrict__ tile_xoff, uint32_t flags,
    ranmar_desc_t* __restrict__ desc, uint32_t* __restrict__ src, uint32_t* __restrict__ exp) {
  const uint64_t base = static_cast<uint64_t>(blockIdx.x) * kScanTile;
  // Thread t owns counts base + 4t .. 4t+3 so that its local scans are serial.
  uint64_t c[kScanPerThread], x[kScanPerThread];
  uint64_t s = 0, xs = 0;
#pragma unroll
  for (int j = 0; j < kScanPerThread; ++j) {
    const uint64_t i = base + static_cast<uint64_t>(threadIdx.x) * kScanPerThread + j;
    c[j] = i < n ? counts[i] : 0;
    x[j] = split_extra(c[j], seg);
    s += c[j];
    xs += x[j];
  }
  uint64_t total;
  uint64_t off = tile_off[blockIdx.x] + cta_exclusive_scan(s, &total);
  uint64_t xo = tile_xoff[blockIdx.x] + cta_exclusive_scan(xs, &total);
  const uint32_t no_wb = flags & ~static_cast<uint32_t>(RANMAR_DESC_WRITE_BACK);
#pragma unroll
  for (int j = 0; j < kScanPerThread; ++j) {
    const uint64_t i = base + static_cast<uint64_t>(threadIdx.x) * kScanPerThread + j;
    if (i < n) {
      ranmar_desc_t d;
      d.state_idx = static_cast<uint32_t>(i);
      d.flags = x[j] ? no_wb : flags;
      d.out_offset = off;
      d.count = c[j] < seg ? c[j] : seg;
      desc[i] = d;
#pragma unroll 1
      for (uint64_t q = 1; q <= x[j]; ++q) {
        const uint64_t e = xo + q - 1;
        if (e >= n_extra) break;           // flagged by pass 2
        const uint64_t start = q * seg;
        const uint64_t left = c[j] - start;
        d.state_idx = static_cast<uint32_t>(n + e);
        d.flags = q == x[j] ? flags : no_wb;
        d.out_offset = off + start;
        d.count = left < seg ? left : seg;
        desc[n + e] = d;
        src[e] = static_cast<uint32_t>(i);
        exp[2 * e] = static_cast<uint32_t>(start);
        exp[2 * e + 1] = static_cast<uint32_t>(start >> 32);
      }
    }
    off += c[j];
    xo += x[j];
  }
}

// After the generation: the last piece of every split stream wrote its
// advanced state to its own slot n + e; copy it back to the stream's slot.
__global__ void __launch_bounds__(kScanThreads) split_finish(ranmar_state_t* __restrict__ states,
                                                             uint64_t n,
                                                             const uint32_t* __restrict__ src,
                                                             uint64_t n_extra) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t e = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < n_extra;
       e += stride) {
    const uint32_t i = src[e];
    if (i >= n) continue;
    if (e + 1 < n_extra && src[e + 1] == i) continue;   // not the stream's last piece
    const uint4* from = reinterpret_cast<const uint4*>(states + n + e);
    uint4* to = reinterpret_cast<uint4*>(states + i);
#pragma unroll 5
    for (int q = 0; q < static_cast<int>(sizeof(ranmar_state_t) / 16); ++q) to[q] = from[q];
  }
}

}  // namespace ranmar
