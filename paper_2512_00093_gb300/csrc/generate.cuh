// generate.cuh -- group-step generation of RANMAR outputs (Algorithm 2).
//
// A group of W lanes (W = 32, 16, 8 or 4) owns one stream.  With the state as
// a sequence X(q), the new word X(q) = X(q-97) - X(q-33) only depends on
// words at least 33 positions back, so the W lanes compute W consecutive
// words per step.  97 = (96/W) W + 1 and 33 = (32/W) W + 1, so the two
// inputs of lane L sit at lane L-1 of blocks b - 96/W and b - 32/W.  The
// window is therefore kept ROTATED by one lane: register R_b[L] =
// X(Wb + L - 1), lane 0 taking the last word of the previous block from a
// carry.  A step is then
//     X(Wb + L) = R_{b-96/W}[L] - R_{b-32/W}[L]     (no data movement)
//     R_b[L]    = shfl(X, L - 1), lane 0 <- carry   (one shuffle)
// and the 97 state words are exactly the 96/W ring registers of the group
// plus the carry.  c_n of each lane starts in closed form (Sec. 3.2): lane L
// begins at c_{L+1} = (c_0 - (L+1) d) mod m and every step moves it by W
// transitions, c <- (c - W d) mod m.  Output (X - c) mod 2^24 is stored
// coalesced (W consecutive words per step, streaming hint).
#pragma once

#include "ranmar_device.cuh"

namespace ranmar {

template <bool F32>
struct OutT {
  using type = uint32_t;
};
template <>
struct OutT<true> {
  using type = float;
};

template <bool F32>
__device__ __forceinline__ void store_output(typename OutT<F32>::type* p, uint32_t y) {
  if constexpr (F32) {
    // y < 2^24 converts exactly; the power-of-two scale is exact (Sec. 4).
    __stcs(p, __uint2float_rn(y) * (1.0f / 16777216.0f));
  } else {
    __stcs(p, y);
  }
}

// (c - delta) mod m for c, delta in [0, m): min(c - delta, c + (m - delta)) --
// exactly one of the two is below m (the other wrapped past 2^32 or is >= m).
__device__ __forceinline__ uint32_t step_c(uint32_t c, uint32_t delta, uint32_t m_minus_delta) {
  return min(c - delta, c + m_minus_delta);
}

struct LaneConsts {
  uint32_t delta_lane;  // (L + 1) d mod m
  uint32_t delta_w;     // W d mod m
};

template <int W>
__device__ __forceinline__ LaneConsts lane_consts(unsigned gl) {
  return LaneConsts{mul_d_mod_m(gl + 1), mul_d_mod_m(W)};
}

// Registers of one stream on its group of W lanes: the rotated ring, the
// carry (lane 0: the last word of the previous block), this lane's c and the
// output pointer.
//
// Store alignment: a step writes W consecutive outputs.  When the stream's
// output offset is not a multiple of W (a = out_base mod W, packed uneven
// batches), every such store would straddle two W-word windows.  The
// realigned mode rotates each step's outputs by a lanes (one more shuffle):
// lane L stores the output of lane (L - a) mod W, taken from the current
// step for L >= a and from the previous step (`up`) for L < a, so every
// store fills one aligned window; the first window (lanes below a skip it)
// and the last one or two are partial.
template <int W, bool F32>
struct GenCtx {
  static constexpr int NR = 96 / W;  // ring registers: blocks b-NR .. b-1
  static constexpr int Q = 32 / W;   // the newer input is block b-Q
  static_assert(NR * W == 96 && Q * W == 32, "group width");
  using T = typename OutT<F32>::type;
  uint32_t r[NR];
  uint32_t carry;
  uint32_t cl;     // c_{Wb+L+1} for the step b the lane is on
  T* p;            // out + (out_base - a) + L (a = 0 unless realigned)
  unsigned ssrc;   // the lane whose output this lane stores when realigned, (L - a) mod W
  bool lo;         // realigned: L < a (stores the previous step's output)
  uint32_t up;     // realigned: this lane's rotated output of the previous step
  uint32_t c0;     // kEarlyWb: the state's c and pos as loaded, for the
  uint64_t pos0;   // write-back (read with the window: the stream's end waits on no load)
};

// kRealign: prepare realigned stores (p at the aligned window, ssrc, lo);
// otherwise p = out + out_base + L and the stores are never realigned.
// kEarlyWb: also keep c and pos for the write-back (three registers), so
// that the end of the stream reads nothing; measured faster for the
// one-warp-per-stream kernels, where each warp's end is exposed.
template <int W, bool F32, bool kRealign, bool kEarlyWb = false>
__device__ __forceinline__ void gen_load(GenCtx<W, F32>& g, const ranmar_state_t* st, void* out,
                                         uint64_t out_base, unsigned gl, const LaneConsts& k) {
  const uint32_t* xs = st->x;
#pragma unroll
  for (int j = 0; j < GenCtx<W, F32>::NR; ++j) g.r[j] = xs[W * j + gl];  // R_{j-NR}[L] = X(W(j-NR) + L - 1)
  g.carry = xs[96];                                                       // X(-1)
  const uint32_t c = st->c;
  if constexpr (kEarlyWb) {
    g.c0 = c;
    g.pos0 = st->pos;
  }
  g.cl = sub_mod_m(c, k.delta_lane);                                      // c_{L+1}
  using T = typename GenCtx<W, F32>::T;
  g.up = 0;
  if constexpr (kRealign) {
    const unsigned a = static_cast<unsigned>(out_base % W);  // the same on the whole group
    g.ssrc = (gl + W - a) % W;
    g.lo = gl < a;
    g.p = static_cast<T*>(out) + (out_base - a) + gl;
  } else {
    g.ssrc = gl;
    g.lo = false;
    g.p = static_cast<T*>(out) + out_base + gl;
  }
}

// Step j of a ring turn: R_b into r[j] (= R_{b-NR} on entry), the outputs to
// window p[W j].  kRot: realigned stores; kFirst: the stream's first step
// (in the realigned mode the lanes below a have nothing to store yet).
template <int W, bool F32, bool kRot, bool kFirst>
__device__ __forceinline__ void gen_step(GenCtx<W, F32>& g, int j, unsigned gl, unsigned gmask,
                                         unsigned src, uint32_t dw, uint32_t mdw) {
  constexpr int NR = GenCtx<W, F32>::NR, Q = GenCtx<W, F32>::Q;
  const uint32_t xv = g.r[j] - g.r[(j + NR - Q) % NR];  // X(Wb + L), kept mod 2^32
  const uint32_t y = (xv - g.cl) & kMask24;
  if constexpr (kRot) {
    const uint32_t u = __shfl_sync(gmask, y, g.ssrc, W);
    const uint32_t v = g.lo ? g.up : u;
    g.up = u;
    if (!(kFirst && g.lo)) store_output<F32>(g.p + W * j, v);
  } else {
    store_output<F32>(g.p + W * j, y);
  }
  g.cl = step_c(g.cl, dw, mdw);
  const uint32_t t = __shfl_sync(gmask, xv, src, W);
  g.r[j] = (gl == 0) ? g.carry : t;
  g.carry = t;
}

// One ring turn of steps (the first step of the stream when kFirst).
template <int W, bool F32, bool kRot, bool kFirst>
__device__ __forceinline__ void gen_turn(GenCtx<W, F32>& g, unsigned gl, unsigned gmask,
                                         unsigned src, uint32_t dw, uint32_t mdw) {
  constexpr int NR = GenCtx<W, F32>::NR;
  gen_step<W, F32, kRot, kFirst>(g, 0, gl, gmask, src, dw, mdw);
#pragma unroll
  for (int j = 1; j < NR; ++j) gen_step<W, F32, kRot, false>(g, j, gl, gmask, src, dw, mdw);
  g.p += W * NR;
}

// Continues the stream from block b0 (a multiple of NR; the context holds
// R_{b0-NR} .. R_{b0-1}) to `count` outputs, then optionally writes the
// advanced state back.
template <int W, bool F32, bool kRot, bool kEarlyWb = false>
__device__ void gen_finish(GenCtx<W, F32>& g, ranmar_state_t* st, uint64_t count, uint64_t b0,
                           bool write_back, unsigned gl, unsigned gmask, const LaneConsts& k) {
  constexpr int NR = GenCtx<W, F32>::NR, Q = GenCtx<W, F32>::Q;
  const uint64_t nblk = count / W;
  const unsigned rem = static_cast<unsigned>(count % W);
  const unsigned src = (gl + W - 1) % W;
  const uint32_t dw = k.delta_w, mdw = kModM - k.delta_w;
  uint64_t b = b0;
  if (kRot && b == 0 && nblk >= NR) {
    gen_turn<W, F32, kRot, true>(g, gl, gmask, src, dw, mdw);
    b = NR;
  }
#pragma unroll 1
  for (; b + NR <= nblk; b += NR) gen_turn<W, F32, kRot, false>(g, gl, gmask, src, dw, mdw);
  // Remaining blocks: step, then shift the ring so that r[0] stays oldest.
#pragma unroll 1
  for (; b < nblk; ++b) {
    if (kRot && b == 0)
      gen_step<W, F32, kRot, true>(g, 0, gl, gmask, src, dw, mdw);
    else
      gen_step<W, F32, kRot, false>(g, 0, gl, gmask, src, dw, mdw);
    g.p += W;
    const uint32_t nw = g.r[0];
#pragma unroll
    for (int j = 0; j + 1 < NR; ++j) g.r[j] = g.r[j + 1];
    g.r[NR - 1] = nw;
  }

  // Ragged tail: one more block with masked stores.
  uint32_t xb = 0;
  if (rem != 0) xb = g.r[0] - g.r[NR - Q];  // X(WB + L)
  if constexpr (kRot) {
    // window nblk: lanes below a hold the last full step's outputs (position
    // W nblk - a + L), the others the tail's (W nblk + L - a); window nblk+1:
    // lanes below a, the tail's positions W (nblk + 1) + L - a
    const uint32_t ut = __shfl_sync(gmask, (xb - g.cl) & kMask24, g.ssrc, W);
    const int a = static_cast<int>((gl + W - g.ssrc) % W);
    const int64_t rel = static_cast<int64_t>(W * nblk) + static_cast<int>(gl) - a;
    if (rel >= 0 && rel < static_cast<int64_t>(count)) store_output<F32>(g.p, g.lo ? g.up : ut);
    if (g.lo && W + static_cast<int>(gl) - a < static_cast<int>(rem))
      store_output<F32>(g.p + W, ut);
  } else {
    if (gl < rem) store_output<F32>(g.p, (xb - g.cl) & kMask24);
  }

  if (!write_back) return;
  uint32_t c0;
  uint64_t pos0;
  if constexpr (kEarlyWb) {
    c0 = g.c0;
    pos0 = g.pos0;
  } else {
    c0 = st->c;
    pos0 = st->pos;
  }
  __syncwarp(gmask);
  // Positions relative to WB: r[j] = X(Wj + L - 97), carry (lane 0) = X(-1),
  // xb = X(L).  New state word q = X(rem - 97 + q).
  uint32_t* xw = st->x;
#pragma unroll
  for (int j = 0; j < NR; ++j) {
    const int q = W * j + static_cast<int>(gl) - static_cast<int>(rem);
    if (q >= 0) xw[q] = g.r[j] & kMask24;
  }
  if (gl == 0) xw[96 - rem] = g.carry & kMask24;
  if (gl < rem) xw[gl + 97 - rem] = xb & kMask24;
  __syncwarp(gmask);
  if (gl == 0) {
    // c after `count` transitions, in closed form (Sec. 3.2)
    const uint64_t e = count % kModM;
    st->c = static_cast<uint32_t>((static_cast<uint64_t>(c0) + (kModM - e) * kD) % kModM);
    st->pos = pos0 + count;
  }
}

// Generates `count` outputs of *st into out[out_base + n], n < count, and
// optionally writes the advanced state back.  Called by the W lanes of one
// group (gl = lane within the group, gmask = the group's lane mask).
// kRealign: realigned stores for offsets that are not multiples of W (the
// persistent batch kernel, whose packed outputs start anywhere); the
// one-warp-per-descriptor and fused kernels store unrealigned, which keeps
// their register count (and occupancy) of the aligned case.
template <int W, bool F32, bool kRealign = false>
__device__ void generate_stream(ranmar_state_t* st, uint64_t count, void* out, uint64_t out_base,
                                bool write_back, unsigned gl, unsigned gmask,
                                const LaneConsts& k) {
  GenCtx<W, F32> g;
  gen_load<W, F32, kRealign, true>(g, st, out, out_base, gl, k);
  if (kRealign && g.ssrc != gl)
    gen_finish<W, F32, kRealign, true>(g, st, count, 0, write_back, gl, gmask, k);
  else
    gen_finish<W, F32, false, true>(g, st, count, 0, write_back, gl, gmask, k);
}

// The interleaved part of generate_streams: `common` blocks (whole ring
// turns) of all S streams, their steps alternating.
template <int W, bool F32, int S, bool kRot>
__device__ __forceinline__ void gen_interleaved(GenCtx<W, F32> (&g)[S], uint64_t common,
                                                unsigned gl, unsigned gmask, unsigned src,
                                                uint32_t dw, uint32_t mdw) {
  constexpr int NR = GenCtx<W, F32>::NR;
  uint64_t b = 0;
  if (kRot && common > 0) {
#pragma unroll
    for (int s = 0; s < S; ++s) gen_step<W, F32, kRot, true>(g[s], 0, gl, gmask, src, dw, mdw);
#pragma unroll
    for (int j = 1; j < NR; ++j) {
#pragma unroll
      for (int s = 0; s < S; ++s) gen_step<W, F32, kRot, false>(g[s], j, gl, gmask, src, dw, mdw);
    }
#pragma unroll
    for (int s = 0; s < S; ++s) g[s].p += W * NR;
    b = NR;
  }
#pragma unroll 1
  for (; b < common; b += NR) {
#pragma unroll
    for (int j = 0; j < NR; ++j) {
#pragma unroll
      for (int s = 0; s < S; ++s) gen_step<W, F32, kRot, false>(g[s], j, gl, gmask, src, dw, mdw);
    }
#pragma unroll
    for (int s = 0; s < S; ++s) g[s].p += W * NR;
  }
}

// S streams on one group at once: their steps are independent dependency
// chains (shuffle -> subtract -> shuffle), so interleaving them hides the
// chain latency with S times fewer resident warps.  The blocks all S have
// (rounded down to whole ring turns) run interleaved (realigned for all S
// when any of them needs it: with a = 0 that mode stores the same words);
// each stream then finishes alone.  ok[s] = false skips stream s (and the
// interleaved part).
template <int W, bool F32, int S, bool kRealign = false>
__device__ void generate_streams(ranmar_state_t* const (&st)[S], const uint64_t (&count)[S],
                                 void* out, const uint64_t (&out_base)[S],
                                 const bool (&write_back)[S], const bool (&ok)[S], unsigned gl,
                                 unsigned gmask, const LaneConsts& k) {
  constexpr int NR = GenCtx<W, F32>::NR;
  GenCtx<W, F32> g[S];
  bool all = true, rot = false;
  uint64_t common = ~0ull;
#pragma unroll
  for (int s = 0; s < S; ++s) {
    all = all && ok[s];
    if (ok[s]) {
      gen_load<W, F32, kRealign>(g[s], st[s], out, out_base[s], gl, k);
      common = min(common, count[s] / W);
      rot = rot || g[s].ssrc != gl;
    }
  }
  if (!all) common = 0;
  common -= common % NR;
  const unsigned src = (gl + W - 1) % W;
  const uint32_t dw = k.delta_w, mdw = kModM - k.delta_w;
  if (kRealign && rot)
    gen_interleaved<W, F32, S, kRealign>(g, common, gl, gmask, src, dw, mdw);
  else
    gen_interleaved<W, F32, S, false>(g, common, gl, gmask, src, dw, mdw);
#pragma unroll
  for (int s = 0; s < S; ++s) {
    if (!ok[s]) continue;
    // a stream that ran realigned from block 0 continues realigned (its
    // last window is still pending in `up`); one with a = 0 has nothing
    // pending either way
    if (kRealign && g[s].ssrc != gl)
      gen_finish<W, F32, kRealign>(g[s], st[s], count[s], common, write_back[s], gl, gmask, k);
    else
      gen_finish<W, F32, false>(g[s], st[s], count[s], common, write_back[s], gl, gmask, k);
  }
}

// Algorithm 1 (Sec. 4, the LAMMPS floating-point form) with the same warp
// mapping (W = 32): the LFG words are reals in [0, 1) (x = u 2^-24),
//     y = x_{q-97} - x_{q-33}; if y < 0: y += 1
//     c = c - 32 cd; if c < 0: c += cm            (32 transitions per step)
//     out = y - c; if out < 0: out += 1
// in floating type F (float or double).  Every value is a multiple of 2^-24
// in [0, 1) (the per-lane offsets (L+1) cd mod cm and 32 cd mod cm are formed
// in integers, then scaled), so float and double are exact and both equal
// the integer form times 2^-24 (Sec. 3.1, the isomorphism sigma).  The state
// stays in its integer format at the boundary.
template <typename F>
__device__ void generate_stream_alg1(ranmar_state_t* st, uint64_t count, F* out, bool write_back,
                                     unsigned lane, const LaneConsts& k) {
  const F S = static_cast<F>(1.0 / 16777216.0);
  const uint32_t* xs = st->x;
  F r0 = static_cast<F>(xs[lane]) * S;   // R_{-3}
  F r1 = static_cast<F>(xs[32 + lane]) * S;
  F r2 = static_cast<F>(xs[64 + lane]) * S;
  F carry = static_cast<F>(xs[96]) * S;
  const uint32_t c0 = st->c;
  const uint64_t pos0 = st->pos;
  F cl = static_cast<F>(sub_mod_m(c0, k.delta_lane)) * S;  // c_{L+1}
  const F dw = static_cast<F>(k.delta_w) * S;
  const F cm = static_cast<F>(kModM) * S;
  const F one = static_cast<F>(1);
  const uint64_t nblk = count >> 5;
  const unsigned rem = static_cast<unsigned>(count & 31);
  F* p = out + lane;
  const unsigned src = (lane + 31) & 31;

  auto step = [&](F& older, F newer, int off) {
    F y = older - newer;
    if (y < 0) y += one;
    F o = y - cl;
    if (o < 0) o += one;
    __stcs(p + off, o);
    cl -= dw;
    if (cl < 0) cl += cm;
    const F t = __shfl_sync(kFull, y, src);
    older = (lane == 0) ? carry : t;
    carry = t;
  };

  uint64_t b = 0;
#pragma unroll 1
  for (; b + 3 <= nblk; b += 3) {
    step(r0, r2, 0);
    step(r1, r0, 32);
    step(r2, r1, 64);
    p += 96;
  }
  const unsigned left = static_cast<unsigned>(nblk - b);
  if (left >= 1) { step(r0, r2, 0); p += 32; }
  if (left >= 2) { step(r1, r0, 0); p += 32; }
  F rm3, rm2, rm1;
  if (left == 0) { rm3 = r0; rm2 = r1; rm1 = r2; }
  else if (left == 1) { rm3 = r1; rm2 = r2; rm1 = r0; }
  else { rm3 = r2; rm2 = r0; rm1 = r1; }
  F xb = 0;
  if (rem != 0) {
    xb = rm3 - rm1;
    if (xb < 0) xb += one;
    F o = xb - cl;
    if (o < 0) o += one;
    if (lane < rem) __stcs(p, o);
  }
  if (!write_back) return;
  __syncwarp();
  const F U = static_cast<F>(16777216.0);
  uint32_t* xw = st->x;
  if (lane >= rem) xw[lane - rem] = static_cast<uint32_t>(rm3 * U);
  xw[lane + 32 - rem] = static_cast<uint32_t>(rm2 * U);
  xw[lane + 64 - rem] = static_cast<uint32_t>(rm1 * U);
  if (lane == 0) xw[96 - rem] = static_cast<uint32_t>(carry * U);
  if (lane < rem) xw[lane + 97 - rem] = static_cast<uint32_t>(xb * U);
  if (lane == 0) {
    const uint64_t e = count % kModM;
    st->c = static_cast<uint32_t>((static_cast<uint64_t>(c0) + (kModM - e) * kD) % kModM);
    st->pos = pos0 + count;
  }
}

// Checks one descriptor on the device; returns false (and flags the status
// word from the group's first lane) when it must be skipped.
__device__ __forceinline__ bool desc_ok(const ranmar_desc_t& d, uint64_t n_states,
                                        uint64_t out_len, uint32_t* status, unsigned gl) {
  if (d.state_idx >= n_states) {
    if (gl == 0) flag_status(status, RANMAR_ST_BAD_INDEX);
    return false;
  }
  if (d.count > out_len || d.out_offset > out_len - d.count) {
    if (gl == 0) flag_status(status, RANMAR_ST_OUT_RANGE);
    return false;
  }
  return true;
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
  const LaneConsts k = lane_consts<32>(lane);
#pragma unroll 1
  for (uint64_t w = warp; w < n_desc; w += nwarps) {
    const ranmar_desc_t d = desc[w];
    if (!desc_ok(d, n_states, out_len, status, lane)) continue;
    generate_stream<32, F32>(states + d.state_idx, d.count, out, d.out_offset,
                             (d.flags & RANMAR_DESC_WRITE_BACK) != 0, lane, kFull, k);
  }
}

// Algorithm 1 over a batch of descriptors (one warp per descriptor).
template <typename F>
__global__ void __launch_bounds__(256) generate_alg1_kernel(
    ranmar_state_t* __restrict__ states, uint64_t n_states,
    const ranmar_desc_t* __restrict__ desc, uint64_t n_desc, F* out, uint64_t out_len,
    uint32_t* status) {
  const unsigned lane = threadIdx.x & 31;
  const uint64_t warp = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
  const LaneConsts k = lane_consts<32>(lane);
#pragma unroll 1
  for (uint64_t w = warp; w < n_desc; w += nwarps) {
    const ranmar_desc_t d = desc[w];
    if (!desc_ok(d, n_states, out_len, status, lane)) continue;
    generate_stream_alg1<F>(states + d.state_idx, d.count, out + d.out_offset,
                            (d.flags & RANMAR_DESC_WRITE_BACK) != 0, lane, k);
  }
}

// Streams a group interleaves in the persistent kernel: 4 for whole warps
// (3 ring registers each), 2 for half warps (6 each), 1 for narrower groups
// (whose rings are 12 or 24 registers).
template <int W>
__host__ __device__ constexpr int persistent_ilp() {
  return W == 32 ? 4 : (W == 16 ? 2 : 1);
}

// Persistent batch kernel: groups of W lanes pull `chunk` descriptors at a
// time from an atomic queue (*queue must be 0 at launch), in the order
// given by `order` (e.g. longest first) or in index order when it is null,
// and generate them persistent_ilp<W>() at a time (interleaved).
// `allow_write_back` = 0 ignores the write-back flags (used while tuning, so
// that timing runs leave the states untouched).
template <int W, bool F32>
__global__ void generate_persistent_kernel(ranmar_state_t* __restrict__ states,
                                           uint64_t n_states,
                                           const ranmar_desc_t* __restrict__ desc,
                                           uint64_t n_desc, const uint32_t* __restrict__ order,
                                           void* out, uint64_t out_len, uint32_t* status,
                                           unsigned long long* queue, uint32_t chunk,
                                           int allow_write_back) {
  constexpr int S = persistent_ilp<W>();
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
      ranmar_state_t* st[S];
      uint64_t cnt[S], ob[S];
      bool wb[S], ok[S];
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const uint64_t t = t0 + s;
        st[s] = states;
        cnt[s] = ob[s] = 0;
        wb[s] = ok[s] = false;
        if (t >= end) continue;
        const uint64_t di = order ? order[t] : t;
        if (di >= n_desc) {
          if (gl == 0) flag_status(status, RANMAR_ST_BAD_INDEX);
          continue;
        }
        const ranmar_desc_t d = desc[di];
        if (!desc_ok(d, n_states, out_len, status, gl)) continue;
        st[s] = states + d.state_idx;
        cnt[s] = d.count;
        ob[s] = d.out_offset;
        wb[s] = allow_write_back && (d.flags & RANMAR_DESC_WRITE_BACK) != 0;
        ok[s] = true;
      }
      generate_streams<W, F32, S, true>(st, cnt, out, ob, wb, ok, gl, gmask, k);
    }
  }
}

// One stream per launch (the per-stream comparator path): one warp.
template <bool F32>
__global__ void __launch_bounds__(32) generate_plain_kernel(ranmar_state_t* st, uint64_t count,
                                                            void* out, int write_back) {
  const unsigned lane = threadIdx.x & 31;
  generate_stream<32, F32>(st, count, out, 0, write_back != 0, lane, kFull, lane_consts<32>(lane));
}

}  // namespace ranmar
