// lfg.cuh -- jump-ahead and generation for lagged Fibonacci recurrences of
// general order (the concluding remarks of the paper):
//     x_n = x_{n-r} - x_{n-s} mod 2^e,   r > s >= 1, 1 <= e <= 32,
// whose transition has the characteristic polynomial phi(t) = t^r + t^{r-s} -
// 1 (Sec. 3.1 for r = 97, s = 33, e = 24).  The jump by E is x' = x P_E(A),
// P_E = t^E mod phi, by left-to-right binary exponentiation (a squaring per
// exponent bit, a shift by t on a 1 bit), then the dot-product application
// over the window extended by the recurrence.  The cost is the squarings:
// r^2 multiply-adds each with the classical product, about r^{log2 3} with
// Karatsuba's -- the trade-off the concluding remarks describe.
//
// One CTA jumps one stream (grid-stride over streams), with 64 to 256
// threads by the width of its widest step (the host's choice: a small r
// leaves room for more streams per SM); every step is CTA-parallel, in
// shared memory:
//   * classical squaring: the operand, skewed (word q at q + q/32, so that
//     the stride-4 sliding-window loads of 32 lanes hit distinct banks), and
//     blocks of 4 consecutive outputs per thread, Sum_i a_i a_{k-i} with the
//     window a_{k-i .. k-i+3} shifted through registers;
//   * Karatsuba squaring, breadth first: with N = M 2^L >= r, the operands
//     are split level by level (each node's lower half, upper half and their
//     sum), the 3^L leaves squared by the same batched classical kernel, and
//     the products recombined level by level, c = z0 + t^h (z1 - z0 - z2) +
//     t^{2h} z2, between two buffers (L chosen on the host or given);
//   * reduction of the 2r - 1 product coefficients mod phi from the top, in
//     blocks of s (t^k = t^{k-r} - t^{k-s}: a block only feeds coefficients
//     below it), then masking to e bits;
//   * the application: the window extended to 2r - 1 words in blocks of s,
//     then new word k = Sum_i p_i X_{i+k}, again 4 outputs per thread.
// 32-bit arithmetic wraps mod 2^32, which is exact mod 2^e; masks only after
// each reduction.
//
// Generation: one warp per stream over a ring of r words in shared memory;
// a step makes W = min(32, s) consecutive words (x_n depends on words at
// least s back), every lane reading both inputs before any lane writes (for
// r < 2s a lane's input slot can be another lane's output slot).
#pragma once

#include "ranmar_device.cuh"

namespace ranmar {

constexpr int kLfgThreads = 256;
constexpr int kLfgMaxR = 2048;
constexpr int kLfgPad = 4;                 // zero words before and after an operand
constexpr int kLfgGenWarps = 8;            // streams per generation CTA

// Skewed index: word q of an operand lives at q + q/32.
__host__ __device__ constexpr int lfg_sk(int q) { return q + (q >> 5); }
// Words of a skewed operand of len coefficients with kLfgPad zeros each side.
__host__ __device__ constexpr int lfg_opnd_words(int len) {
  return ((lfg_sk(len + 2 * kLfgPad) + 1) + 3) & ~3;
}

// Everything one (r, s, e, method) jump needs, computed on the host.
struct LfgShape {
  int r, s;
  uint32_t mask;
  int L;        // Karatsuba levels (0: classical product)
  int M;        // leaf length (classical: r)
  int N;        // M 2^L >= r
  int pow3L;    // 3^L
  int opnd;     // words per skewed leaf operand
  // shared-memory word offsets
  int off_p;    // p[N] (plain)
  int off_ops;  // 3^L skewed operands
  int off_a;    // leaf products [3^L][2M]; depth L-2, L-4, ...; the extended window
  int off_b;    // depth L-1, L-3, ...
  int words;    // total
};

// out[tau * ostr + k] = Sum_{i+j=k} a_tau[i] a_tau[j] for k < 2 len, tau <
// nprod, where a_tau[i] sits at opnd[tau * astr + lfg_sk(i + kLfgPad)] and is
// zero for i in [-kLfgPad, 0) and [len, len + kLfgPad).  (out[2 len - 1] = 0.)
__device__ __forceinline__ void lfg_batched_square(const uint32_t* __restrict__ opnd, int astr,
                                                   int len, int nprod,
                                                   uint32_t* __restrict__ out, int ostr) {
  const int nb = (2 * len + 3) / 4;
  const int items = nprod * nb;
  for (int q = threadIdx.x; q < items; q += blockDim.x) {
    const int tau = q / nb, kb = q - tau * nb;
    const int k0 = 4 * kb;
    const uint32_t* a = opnd + tau * astr;
    const int lo = max(0, k0 - (len - 1));
    const int hi = min(len - 1, k0 + 3);
    uint32_t acc0 = 0, acc1 = 0, acc2 = 0, acc3 = 0;
    if (lo <= hi) {
      // w_j = a[k0 + j - i] for the current i (indices >= -3 and <= len + 2)
      uint32_t w0 = a[lfg_sk(k0 - lo + kLfgPad)], w1 = a[lfg_sk(k0 - lo + 1 + kLfgPad)],
               w2 = a[lfg_sk(k0 - lo + 2 + kLfgPad)], w3 = a[lfg_sk(k0 - lo + 3 + kLfgPad)];
      for (int i = lo; i <= hi; ++i) {
        const uint32_t ai = a[lfg_sk(i + kLfgPad)];
        acc0 += ai * w0;
        acc1 += ai * w1;
        acc2 += ai * w2;
        acc3 += ai * w3;
        w3 = w2;
        w2 = w1;
        w1 = w0;
        w0 = a[lfg_sk(k0 - i - 1 + kLfgPad)];   // index >= -4
      }
    }
    uint32_t* o = out + tau * ostr + k0;
    o[0] = acc0;
    if (k0 + 1 < 2 * len) o[1] = acc1;
    if (k0 + 2 < 2 * len) o[2] = acc2;
    if (k0 + 3 < 2 * len) o[3] = acc3;
  }
}

// Writes a skewed operand: dst[lfg_sk(i + kLfgPad)] = src(i) for i < len,
// zeros in the pads; f(i) gives the value.
template <typename F>
__device__ __forceinline__ void lfg_put_operand(uint32_t* __restrict__ dst, int len, F f) {
  for (int i = static_cast<int>(threadIdx.x) - kLfgPad; i < len + kLfgPad; i += blockDim.x)
    dst[lfg_sk(i + kLfgPad)] = (i >= 0 && i < len) ? f(i) : 0u;
}

// prod[0 .. 2N) = p^2 (p[r..N) = 0).  Returns the buffer holding it.
__device__ uint32_t* lfg_square(const LfgShape& sh, uint32_t* smem) {
  uint32_t* p = smem + sh.off_p;
  uint32_t* ops = smem + sh.off_ops;
  uint32_t* A = smem + sh.off_a;
  uint32_t* B = smem + sh.off_b;
  if (sh.L == 0) {
    lfg_put_operand(ops, sh.r, [&](int i) { return p[i]; });
    __syncthreads();
    lfg_batched_square(ops, sh.opnd, sh.r, 1, A, 2 * sh.r);
    __syncthreads();
    return A;
  }
  // operands level by level: node nu of depth d (3^d nodes of N/2^d words)
  // has children 3nu (lower half), 3nu+1 (upper half), 3nu+2 (their sum);
  // depths 1 .. L-1 alternate between B and A (plain), the leaves (depth L,
  // M words) go skewed into `ops`
  const int M = sh.M, L = sh.L;
  const uint32_t* src = p;
  int len = sh.N;   // operand length at the current depth
  int nodes = 1;
  for (int d = 1; d <= L; ++d) {
    const int h = len / 2;
    const bool leaf = d == L;
    uint32_t* dst = (d & 1) ? B : A;
    const int w = leaf ? (M + 2 * kLfgPad) : h;   // written words per child
    for (int q = threadIdx.x; q < 3 * nodes * w; q += blockDim.x) {
      const int child = q / w;
      const int i = q - child * w - (leaf ? kLfgPad : 0);
      const int nu = child / 3, c = child - 3 * nu;
      uint32_t v = 0;
      if (i >= 0 && i < h) {
        const uint32_t* par = src + nu * len;
        v = c == 0 ? par[i] : (c == 1 ? par[h + i] : par[i] + par[h + i]);
      }
      if (leaf)
        ops[child * sh.opnd + lfg_sk(i + kLfgPad)] = v;
      else
        dst[child * h + i] = v;
    }
    __syncthreads();
    src = dst;
    len = h;
    nodes *= 3;
  }
  __syncthreads();
  lfg_batched_square(ops, sh.opnd, M, sh.pow3L, A, 2 * M);
  __syncthreads();
  // recombine: depth d from depth d + 1; node nu's children 3nu (lo), 3nu+1
  // (hi), 3nu+2 (lo+hi); child products of 2h words, parent of 4h
  uint32_t* psrc = A;
  uint32_t* pdst = B;
  nodes = sh.pow3L / 3;
  int h = M;
  for (int d = L - 1; d >= 0; --d) {
    const int n4 = 4 * h;
    for (int q = threadIdx.x; q < nodes * n4; q += blockDim.x) {
      const int nu = q / n4, k = q - nu * n4;
      const uint32_t* z0 = psrc + (3 * nu) * 2 * h;
      const uint32_t* z2 = z0 + 2 * h;
      const uint32_t* z1 = z2 + 2 * h;
      uint32_t v = 0;
      if (k < 2 * h) v += z0[k];
      if (k >= h && k < 3 * h) {
        const int u = k - h;
        v += z1[u] - z0[u] - z2[u];
      }
      if (k >= 2 * h) v += z2[k - 2 * h];
      pdst[nu * n4 + k] = v;
    }
    __syncthreads();
    uint32_t* tmp = psrc;
    psrc = pdst;
    pdst = tmp;
    nodes /= 3;
    h *= 2;
  }
  return psrc;   // depth 0: 2N words
}

// p = prod mod phi, masked (prod: 2r - 1 meaningful words, modified).
__device__ void lfg_reduce(const LfgShape& sh, uint32_t* __restrict__ prod, uint32_t* __restrict__ p) {
  const int r = sh.r, s = sh.s;
  // A block [bot, top] of width <= s only feeds coefficients below bot, and
  // each of its words is final (its contributions come from k + s, k + r >
  // top).  The two updates run as separate passes: for r < 2s a k - r of one
  // word can be the k' - s of another word of the same block.
  for (int top = 2 * r - 2; top >= r; top -= s) {
    const int bot = max(r, top - s + 1);
    for (int k = bot + static_cast<int>(threadIdx.x); k <= top; k += blockDim.x)
      prod[k - s] -= prod[k];
    __syncthreads();
    for (int k = bot + static_cast<int>(threadIdx.x); k <= top; k += blockDim.x)
      prod[k - r] += prod[k];
    __syncthreads();
  }
  for (int i = threadIdx.x; i < sh.N; i += blockDim.x) p[i] = i < r ? (prod[i] & sh.mask) : 0u;
  __syncthreads();
}

// p = p t mod phi: shift up by one, the word on t^r folds back as 1 - t^{r-s}.
__device__ void lfg_times_t(const LfgShape& sh, uint32_t* __restrict__ p) {
  const int r = sh.r;
  const uint32_t top = p[r - 1];
  uint32_t v[(kLfgMaxR + kLfgThreads - 1) / kLfgThreads];
  int c = 0;
  for (int i = threadIdx.x; i < r; i += blockDim.x) v[c++] = (i == 0) ? top : p[i - 1];
  __syncthreads();
  c = 0;
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    uint32_t w = v[c++];
    if (i == r - sh.s) w -= top;
    p[i] = w & sh.mask;
  }
  __syncthreads();
}

// out[k] = Sum_i p_i X_{i+k}, k < r, X the window x extended to 2r - 1 words.
__device__ void lfg_apply(const LfgShape& sh, uint32_t* smem, const uint32_t* __restrict__ x,
                          uint32_t* __restrict__ out) {
  const int r = sh.r, s = sh.s;
  const uint32_t* p = smem + sh.off_p;
  uint32_t* X = smem + sh.off_a;   // skewed: X_q at lfg_sk(q)
  for (int q = threadIdx.x; q < r; q += blockDim.x) X[lfg_sk(q)] = x[q];
  __syncthreads();
  for (int q0 = r; q0 < 2 * r - 1; q0 += s) {   // each block depends on words >= s back
    const int q1 = min(2 * r - 1, q0 + s);
    for (int q = q0 + static_cast<int>(threadIdx.x); q < q1; q += blockDim.x)
      X[lfg_sk(q)] = X[lfg_sk(q - r)] - X[lfg_sk(q - s)];
    __syncthreads();
  }
  for (int q = 2 * r - 1 + static_cast<int>(threadIdx.x); q < 2 * r + 3; q += blockDim.x)
    X[lfg_sk(q)] = 0u;   // read by the last window (multiplied by zero coefficients)
  __syncthreads();
  const int nb = (r + 3) / 4;
  for (int kb = threadIdx.x; kb < nb; kb += blockDim.x) {
    const int k0 = 4 * kb;
    uint32_t acc[4] = {0u, 0u, 0u, 0u};
    uint32_t w0 = X[lfg_sk(k0)], w1 = X[lfg_sk(k0 + 1)], w2 = X[lfg_sk(k0 + 2)];
    for (int i = 0; i < r; ++i) {
      const uint32_t w3 = X[lfg_sk(i + k0 + 3)];
      const uint32_t pi = p[i];
      acc[0] += pi * w0;
      acc[1] += pi * w1;
      acc[2] += pi * w2;
      acc[3] += pi * w3;
      w0 = w1;
      w1 = w2;
      w2 = w3;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (k0 + j < r) out[k0 + j] = acc[j] & sh.mask;
  }
  __syncthreads();
}

// d_out[i] = window d_x[base_idx[i] or 0] jumped by E_i (d_exp, exp_words per
// stream).  Windows are r words each, oldest first.
__global__ void __launch_bounds__(kLfgThreads) lfg_jump_kernel(
    LfgShape sh, const uint32_t* __restrict__ d_x, uint64_t n_base,
    const uint32_t* __restrict__ d_base_idx, const uint32_t* __restrict__ d_exp,
    uint32_t exp_words, uint32_t* __restrict__ d_out, uint64_t n, uint32_t* status) {
  extern __shared__ __align__(16) uint32_t smem[];
  uint32_t* p = smem + sh.off_p;
  for (uint64_t i = blockIdx.x; i < n; i += gridDim.x) {
    uint32_t E[kMaxExpWords];
#pragma unroll
    for (int w = 0; w < kMaxExpWords; ++w)
      E[w] = w < static_cast<int>(exp_words) ? d_exp[i * exp_words + w] : 0u;
    const uint32_t bi = d_base_idx ? d_base_idx[i] : 0u;
    if (bi >= n_base) {
      if (threadIdx.x == 0) flag_status(status, RANMAR_ST_BAD_INDEX);
      continue;
    }
    int nbits = 0;
#pragma unroll
    for (int w = 0; w < kMaxExpWords; ++w)
      if (E[w] != 0) nbits = 32 * w + 32 - __clz(E[w]);
    // leading bits while the value stays below r: P is the monomial t^v
    uint32_t v = 0;
    int pos = nbits - 1;
    while (pos >= 0) {
      const uint32_t bit = (E[pos >> 5] >> (pos & 31)) & 1u;
      if (2 * v + bit >= static_cast<uint32_t>(sh.r)) break;
      v = 2 * v + bit;
      --pos;
    }
    for (int q = threadIdx.x; q < sh.N; q += blockDim.x) p[q] = (q == static_cast<int>(v)) ? 1u : 0u;
    __syncthreads();
    for (; pos >= 0; --pos) {
      uint32_t* prod = lfg_square(sh, smem);
      lfg_reduce(sh, prod, p);
      if ((E[pos >> 5] >> (pos & 31)) & 1u) lfg_times_t(sh, p);
    }
    lfg_apply(sh, smem, d_x + static_cast<uint64_t>(bi) * sh.r, d_out + i * sh.r);
  }
}

// count words of each stream: out[i * count + j]; the window is advanced in
// place.  One warp per stream, kLfgGenWarps streams per CTA, rings of r words
// in shared memory.
__global__ void __launch_bounds__(32 * kLfgGenWarps) lfg_generate_kernel(
    int r, int s, uint32_t mask, uint32_t* __restrict__ d_x, uint64_t n, uint64_t count,
    uint32_t* __restrict__ d_out) {
  extern __shared__ __align__(16) uint32_t smem[];
  const unsigned lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  uint32_t* ring = smem + wi * r;
  const int W = s < 32 ? s : 32;
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * kLfgGenWarps + wi; i < n;
       i += static_cast<uint64_t>(gridDim.x) * kLfgGenWarps) {
    uint32_t* x = d_x + i * r;
    for (int q = lane; q < r; q += 32) ring[q] = x[q];
    __syncwarp();
    int h = 0;   // ring[h] = x_{t-r} for the next word x_t
    uint32_t* o = d_out + i * count;
    for (uint64_t t = 0; t < count; t += W) {
      const int L = static_cast<int>(lane);
      const bool on = L < W && t + L < count;
      uint32_t w = 0;
      int slot = h + L;
      if (slot >= r) slot -= r;
      if (on) {
        int sq = slot + (r - s);
        if (sq >= r) sq -= r;
        w = (ring[slot] - ring[sq]) & mask;
      }
      __syncwarp();
      if (on) {
        ring[slot] = w;
        o[t + L] = w;
      }
      __syncwarp();
      const int adv = static_cast<int>(count - t < static_cast<uint64_t>(W) ? count - t : W);
      h += adv;
      if (h >= r) h -= r;
    }
    for (int q = lane; q < r; q += 32) {
      int slot = h + q;
      if (slot >= r) slot -= r;
      x[q] = ring[slot];
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Jump with a warp per stream, classical squaring, r <= kLfgWarpMaxR.
//
// The same steps as lfg_jump_kernel (left-to-right binary exponentiation,
// reduction in blocks of s, the application over the extended window), with
// the CTA-wide steps replaced by warp-wide ones, so that small lags (r = 97:
// 49 four-output blocks per squaring) do not leave most of a CTA idle:
//   * squaring: lane l forms c_n for n = 8l .. 8l+7 as Sum_{i < R4} a_i
//     a_{n-i} (R4 = r rounded up to 4; a is zero outside [0, r), stored with
//     128 zero words below and up to 256 above, so there are no bounds
//     tests), its eight a words in registers sliding down by one per step:
//     one shared-memory load per eight multiply-adds; the operand is skewed
//     (word q at q + q/32) so that the stride-8 loads of a warp hit distinct
//     banks (lanes 0 and 31 can share one);
//   * application: lane l forms outputs 4l .. 4l+3 over the skewed window,
//     sliding up by one word per step.
constexpr int kLfgWarpMaxR = 128;
constexpr int kLfgWarpWarps = 4;                  // streams per CTA
// per-warp slice (words): the operand a (logical -128 .. 255, skewed), the
// product / the extended window
constexpr int kLfgWA = 0;
constexpr int kLfgWAWords = ((lfg_sk(384 - 1) + 1) + 3) & ~3;   // 396
constexpr int kLfgWC = kLfgWAWords;
constexpr int kLfgWCWords = ((lfg_sk(2 * kLfgWarpMaxR + 8) + 1) + 3) & ~3;
constexpr int kLfgWWords = kLfgWC + kLfgWCWords;
constexpr size_t kLfgWarpSmemBytes = sizeof(uint32_t) * kLfgWWords * kLfgWarpWarps;
static_assert(kLfgWAWords >= lfg_sk(383) + 1 && kLfgWCWords >= 256, "warp slice");

// a_m, m in [-128, 256): the skewed slot of logical index m
__device__ __forceinline__ int lfg_wa(int m) { return lfg_sk(m + 128); }

__global__ void __launch_bounds__(32 * kLfgWarpWarps) lfg_jump_warp_kernel(
    int r, int s, uint32_t mask, const uint32_t* __restrict__ d_x, uint64_t n_base,
    const uint32_t* __restrict__ d_base_idx, const uint32_t* __restrict__ d_exp,
    uint32_t exp_words, uint32_t* __restrict__ d_out, uint64_t n, uint32_t* status) {
  extern __shared__ __align__(16) uint32_t smem[];
  const int lane = static_cast<int>(threadIdx.x & 31), w = static_cast<int>(threadIdx.x >> 5);
  uint32_t* A = smem + w * kLfgWWords + kLfgWA;
  uint32_t* C = smem + w * kLfgWWords + kLfgWC;
  const int R4 = (r + 3) & ~3;
  for (int q = lane; q < kLfgWAWords; q += 32) A[q] = 0u;
  __syncwarp();
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * kLfgWarpWarps;
#pragma unroll 1
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * kLfgWarpWarps + w; i < n; i += stride) {
    uint32_t E[kMaxExpWords];
#pragma unroll
    for (int q = 0; q < kMaxExpWords; ++q)
      E[q] = q < static_cast<int>(exp_words) ? d_exp[i * exp_words + q] : 0u;
    const uint32_t bi = d_base_idx ? d_base_idx[i] : 0u;
    if (bi >= n_base) {
      if (lane == 0) flag_status(status, RANMAR_ST_BAD_INDEX);
      continue;
    }
    int nbits = 0;
#pragma unroll
    for (int q = 0; q < kMaxExpWords; ++q)
      if (E[q] != 0) nbits = 32 * q + 32 - __clz(E[q]);
    // leading bits while the value stays below r: P = t^v
    uint32_t v = 0;
    int pos = nbits - 1;
    while (pos >= 0) {
      const uint32_t bit = (E[pos >> 5] >> (pos & 31)) & 1u;
      if (2 * v + bit >= static_cast<uint32_t>(r)) break;
      v = 2 * v + bit;
      --pos;
    }
    for (int q = lane; q < r; q += 32) A[lfg_wa(q)] = q == static_cast<int>(v) ? 1u : 0u;
    __syncwarp();
#pragma unroll 1
    for (; pos >= 0; --pos) {
      // c = a^2 (c_n for n = 8 lane + j)
      const int n0 = 8 * lane;
      uint32_t acc[8], win[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        acc[j] = 0u;
        win[j] = A[lfg_wa(n0 + j)];
      }
#pragma unroll 1
      for (int i0 = 0; i0 < R4; i0 += 4) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int ii = i0 + e;
          const uint32_t ai = A[lfg_wa(ii)];
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[j] += ai * win[j];
#pragma unroll
          for (int j = 7; j >= 1; --j) win[j] = win[j - 1];
          win[0] = A[lfg_wa(n0 - ii - 1)];   // logical index >= -128
        }
      }
      __syncwarp();
#pragma unroll
      for (int j = 0; j < 8; ++j) C[n0 + j] = acc[j];
      __syncwarp();
      // mod phi from the top, blocks of s (t^k = t^{k-r} - t^{k-s})
      for (int top = 2 * r - 2; top >= r; top -= s) {
        const int bot = max(r, top - s + 1);
        for (int k = bot + lane; k <= top; k += 32) C[k - s] -= C[k];
        __syncwarp();
        for (int k = bot + lane; k <= top; k += 32) C[k - r] += C[k];
        __syncwarp();
      }
      // a = c mod phi, times t on a 1 bit (shift; the word on t^r folds back
      // as 1 - t^{r-s}), masked
      const bool bit = (E[pos >> 5] >> (pos & 31)) & 1u;
      const uint32_t topw = C[r - 1];
      for (int q = lane; q < r; q += 32) {
        uint32_t x = C[q];
        if (bit) {
          x = q == 0 ? topw : C[q - 1];
          if (q == r - s) x -= topw;
        }
        A[lfg_wa(q)] = x & mask;
      }
      __syncwarp();
    }
    // application: X_q = x_q (q < r), X_q = X_{q-r} - X_{q-s} up to 2r - 2,
    // zeros above (read only against zero coefficients); out_k = Sum_i p_i X_{i+k}
    const uint32_t* x = d_x + static_cast<uint64_t>(bi) * r;
    for (int q = lane; q < r; q += 32) C[lfg_sk(q)] = x[q];
    for (int q = 2 * r - 1 + lane; q < 2 * kLfgWarpMaxR + 8; q += 32) C[lfg_sk(q)] = 0u;
    __syncwarp();
    for (int q0 = r; q0 < 2 * r - 1; q0 += s) {
      const int q1 = min(2 * r - 1, q0 + s);
      for (int q = q0 + lane; q < q1; q += 32) C[lfg_sk(q)] = C[lfg_sk(q - r)] - C[lfg_sk(q - s)];
      __syncwarp();
    }
    const int k0 = 4 * lane;
    uint32_t acc[4], win[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      acc[j] = 0u;
      win[j] = C[lfg_sk(k0 + j)];
    }
#pragma unroll 1
    for (int i0 = 0; i0 < R4; i0 += 4) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int ii = i0 + e;
        const uint32_t pi = A[lfg_wa(ii)];
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[j] += pi * win[j];
#pragma unroll
        for (int j = 0; j < 3; ++j) win[j] = win[j + 1];
        win[3] = C[lfg_sk(k0 + ii + 4)];
      }
    }
    uint32_t* o = d_out + i * static_cast<uint64_t>(r);
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (k0 + j < r) o[k0 + j] = acc[j] & mask;
    __syncwarp();
  }
}

}  // namespace ranmar
