/*
 * ranmar.h -- C ABI of libranmar: bulk generation of non-overlapping RANMAR
 * streams on one GB300 GPU (sm_103a).
 *
 * Method: H. Haramoto and K. Suzuki, "Making the RANMAR pseudorandom number
 * generator in LAMMPS up to four times faster, with an implementation of
 * jump-ahead", arXiv 2512.00093.
 *
 * Notation (Sec. 2, Sec. 3, Algorithm 2):
 *   lagged Fibonacci word   x_n = (x_{n-97} - x_{n-33}) mod 2^24
 *   arithmetic sequence     c_n = (c_{n-1} - d) mod m,  d = 7654321,
 *                           m = 2^24 - 3, c_0 = 362436 after seeding
 *   output                  y_n = (x_{96+n} - c_n) mod 2^24   (1-based n,
 *                           x_1..x_97 the state), float y_n * 2^-24
 *   jump by E transitions   x P_E(A), P_E = t^E mod (t^97 + t^64 - 1) over
 *                           Z/2^24 (Sec. 3.1), c_E = (c_0 - E d) mod m
 *                           (Sec. 3.2).
 *
 * Conventions for every entry point:
 *   - Return 0 (RANMAR_OK) or a negative RANMAR_E* code; no exception ever
 *     crosses the ABI.  ranmar_strerror() names each code.
 *   - Pointers named d_* are device pointers on the current CUDA device;
 *     h_* are host pointers.  The caller owns every buffer; the library
 *     allocates nothing in these calls and keeps no pointer after return.
 *   - Device work is enqueued on `stream` (a cudaStream_t; NULL means the
 *     legacy default stream) and the call returns without waiting for it.
 *   - Arguments visible on the host are checked before anything is
 *     launched (RANMAR_EINVAL / RANMAR_ERANGE, nothing enqueued).  Values
 *     only the device sees (indices inside descriptor arrays) are checked by
 *     the kernel: a bad item is skipped and a RANMAR_ST_* bit is OR-ed into
 *     *d_status when d_status is not NULL.
 *   - RANMAR_ECUDA means a CUDA launch or query failed; the CUDA error
 *     string is available from ranmar_last_cuda_error().
 */
#ifndef RANMAR_H
#define RANMAR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RANMAR_R 97               /* lag r (Sec. 2) */
#define RANMAR_S 33               /* lag s (Sec. 2) */
#define RANMAR_MAX_EXP_WORDS 5    /* jump exponents up to 2^160 - 1 */

/* Return codes. */
#define RANMAR_OK 0
#define RANMAR_EINVAL (-1)        /* null pointer, misalignment, bad seed   */
#define RANMAR_ERANGE (-2)        /* size or exponent out of range          */
#define RANMAR_ECUDA (-3)         /* CUDA launch/runtime error              */
#define RANMAR_ENOMEM (-4)        /* workspace allocation failed            */
#define RANMAR_EDEVICE (-5)       /* device not sm_103a / not usable        */
#define RANMAR_ETIME (-6)         /* a serving run passed its time limit    */
#define RANMAR_ESTATUS (-7)       /* a kernel of a serving run set a        */
                                  /* RANMAR_ST_* bit (ranmar_serve_stats)    */

/* Bits OR-ed into *d_status by kernels. */
#define RANMAR_ST_BAD_INDEX 1u    /* state or base index out of range       */
#define RANMAR_ST_OUT_RANGE 2u    /* out_offset + count beyond out_len      */
#define RANMAR_ST_BAD_SEED 4u     /* seed outside 1..900000000              */
#define RANMAR_ST_TIMEOUT 8u      /* a bounded device wait ran out (the CTA  */
                                  /* left its work undone and returned)      */
#define RANMAR_ST_OVERLAP 16u     /* a generation would leave its stream     */
                                  /* (ranmar_check_overlap; not an error)    */

/* Descriptor flags. */
#define RANMAR_DESC_WRITE_BACK 1u /* store the advanced state after output  */

/*
 * Generator state S = (x_1, ..., x_97, c) of Sec. 2 in its integer form
 * (Sec. 3): x[q] = x_{q+1}, oldest word first, each in [0, 2^24); c is the
 * numerator c' in [0, m) after the last transition, so the next output uses
 * (c - d) mod m.  pos counts transitions applied since the caller's origin,
 * modulo 2^64 (informational: jumps add E mod 2^64, generation adds count).
 * 400 bytes; arrays of states must be 16-byte aligned.
 */
typedef struct ranmar_state {
    uint32_t x[RANMAR_R];
    uint32_t c;
    uint64_t pos;
} ranmar_state_t;

/*
 * One generation request: `count` consecutive outputs of the stream whose
 * state is states[state_idx], written to out[out_offset .. out_offset +
 * count).  With RANMAR_DESC_WRITE_BACK the state is advanced by `count`
 * transitions in place (resume).  Two descriptors of one call must not name
 * the same state with WRITE_BACK, nor overlapping output ranges.  24 bytes.
 */
typedef struct ranmar_desc {
    uint32_t state_idx;
    uint32_t flags;
    uint64_t out_offset;
    uint64_t count;
} ranmar_desc_t;

/* One checksum work item: words data[offset .. offset+count), whose first
 * word has index index0 within its request; added into results[result]. */
typedef struct ranmar_sum_item {
    uint64_t offset;
    uint64_t count;
    uint64_t index0;
    uint32_t result;
    uint32_t pad;
} ranmar_sum_item_t;   /* 32 bytes */

typedef struct CUstream_st *ranmar_stream_t;   /* == cudaStream_t */

/*
 * ranmar_seed -- Algorithm 3 (Appendix A): the LAMMPS RanMars seeding in
 * integer form.  Host only, no device work.  Writes the seeded state in
 * sequence order (x_1..x_97 = u_97, u_96, ..., u_1 with i = 97, j = 33),
 * c = 362436, pos = 0.
 * Errors: RANMAR_EINVAL if out is NULL or seed is outside 1..900000000 (the
 * seed bound of Sec. 1; seed 0 would make seed - 1 negative).
 */
int ranmar_seed(int32_t seed, ranmar_state_t *h_out);

/*
 * ranmar_seed_batch -- Algorithm 3 on the device for many seeds at once (one
 * thread per seed): d_out[i] = the seeded state of d_seeds[i], identical to
 * ranmar_seed.  Errors: RANMAR_EINVAL (NULL with n > 0, misaligned d_out).
 * Device: RANMAR_ST_BAD_SEED for a seed outside 1..900000000 (that d_out[i]
 * is left untouched).
 */
int ranmar_seed_batch(const int32_t *d_seeds, size_t n, ranmar_state_t *d_out,
                      uint32_t *d_status, ranmar_stream_t stream);

/*
 * ranmar_jump -- Sec. 3.1 and Sec. 3.2: d_out[i] = f^{E_i}(base), where base
 * is d_base[d_base_idx[i]] (or d_base[0] when d_base_idx is NULL) and E_i is
 * the little-endian integer d_exp[i*exp_words .. (i+1)*exp_words).  For each
 * i the kernel forms P = t^{E_i} mod (t^97 + t^64 - 1) over Z/2^24 by
 * left-to-right square-and-multiply, applies x P(A) as sum_j b_j x_{j+k},
 * and sets c = (c_base - E_i d) mod m, pos = pos_base + E_i mod 2^64.
 * A CTA of two warps serves 16 streams, two lanes per stream in each warp
 * (lane 0 forms the low half of each square, lane 1 the high half from the
 * reversed polynomial; the two warps share each square's output blocks and
 * the application's, four threads per stream); a
 * batch of at most RANMAR_SQUARE_WARP_AUTO_MAX streams instead gives each
 * stream a whole warp.  That cuts the LATENCY of one squaring about 5 times
 * (each stream's dependent chain is spread over 32 lanes instead of 4), not
 * the work: the warp mapping executes about three times the instructions
 * per stream, so larger batches keep the lane pairs.  Same results either
 * way.
 * d_out must not overlap d_base.  n = 0 is a no-op.
 * Errors: RANMAR_EINVAL (null pointer with n > 0, misaligned states,
 * overlapping in/out), RANMAR_ERANGE (exp_words not in 1..5, n_base = 0, or
 * n too large for one launch).  Device: RANMAR_ST_BAD_INDEX when
 * d_base_idx[i] >= n_base (that d_out[i] is left untouched).
 */
int ranmar_jump(const ranmar_state_t *d_base, size_t n_base,
                const uint32_t *d_base_idx,
                const uint32_t *d_exp, uint32_t exp_words,
                ranmar_state_t *d_out, size_t n,
                uint32_t *d_status, ranmar_stream_t stream);

/*
 * ranmar_poly_power -- Sec. 3.1, the polynomial part of a jump alone (what
 * the paper's Table 2 times): d_poly[i] = P_{E_i}(t) = t^{E_i} mod (t^97 +
 * t^64 - 1) over Z/2^24, by the same left-to-right square-and-multiply as
 * ranmar_jump, for E_i the little-endian integer d_exp[i*exp_words ..
 * (i+1)*exp_words) (device).  d_poly (device, n x 100 uint32, caller-owned):
 * coefficients 0..96 of P_{E_i} (24-bit canonical, coefficient j of t^j),
 * then three zero words.  Two lanes per exponent in each of two warps per
 * 16 exponents (a warp per exponent up to RANMAR_SQUARE_WARP_AUTO_MAX
 * exponents); asynchronous
 * on `stream`; n = 0 is a no-op.  Errors: RANMAR_EINVAL (NULL with n > 0,
 * misaligned or overlapping buffers), RANMAR_ERANGE (exp_words not in
 * 1..RANMAR_MAX_EXP_WORDS, or n too large for one launch).
 */
int ranmar_poly_power(const uint32_t *d_exp, uint32_t exp_words, size_t n, uint32_t *d_poly,
                      ranmar_stream_t stream);

/*
 * ranmar_jump_scatter -- ranmar_jump with per-stream destinations:
 * d_dst[d_dst_idx[i]] = f^{E_i}(d_base[d_base_idx[i]]) (d_base_idx NULL =
 * base 0).  For state pools that are read and written in place (a serving
 * engine's resident states): d_base and d_dst may be the same array, but in
 * one call no destination index may equal another destination or any base
 * index used by the call (those would race; not checked).
 * Errors: as ranmar_jump (RANMAR_ERANGE also for n_dst = 0).  Device:
 * RANMAR_ST_BAD_INDEX for d_base_idx[i] >= n_base or d_dst_idx[i] >= n_dst
 * (that stream is skipped).
 */
int ranmar_jump_scatter(const ranmar_state_t *d_base, size_t n_base,
                        const uint32_t *d_base_idx,
                        const uint32_t *d_exp, uint32_t exp_words,
                        ranmar_state_t *d_dst, size_t n_dst, const uint32_t *d_dst_idx,
                        size_t n, uint32_t *d_status, ranmar_stream_t stream);

/*
 * ranmar_partition -- stream partitioning of Sec. 1: d_out[i] is the start
 * of block k = k0 + i of length J of the sequence that starts at *d_base,
 * i.e. f^{kJ}(base), computed as in ranmar_jump with E = (k0 + i) J formed
 * on the device.  J is the little-endian host integer h_J[0..J_words).
 * Errors: RANMAR_EINVAL (null pointer, misalignment, overlap),
 * RANMAR_ERANGE (J_words not in 1..5, or (k0 + n - 1) J >= 2^160).
 */
int ranmar_partition(const ranmar_state_t *d_base, const uint32_t *h_J,
                     uint32_t J_words, uint64_t k0,
                     ranmar_state_t *d_out, size_t n, ranmar_stream_t stream);

/*
 * ranmar_generate_u24 / ranmar_generate_f32 -- Algorithm 2 over a batch of
 * descriptors: for each desc, `count` outputs y_n = (x_{96+n} - c_n) mod
 * 2^24 of its stream, as uint32 (u24) or as float y_n * 2^-24 (f32; exact,
 * in [0, 1), 0.0 possible).  One warp runs one stream, 32 consecutive
 * outputs per step (the lag 33 allows 32 in parallel), stores coalesced.
 * The launch reserves 46 KB of shared memory per 256-thread CTA that it
 * does not use, which holds it to four CTAs per SM (fewer output regions
 * written at once write HBM faster); kernels running beside it on other
 * streams share the rest.  A state written back must belong to one
 * descriptor of the batch only (descriptors run concurrently).
 * out_len is the element count of d_out.
 * Errors: RANMAR_EINVAL (null pointer with n_desc > 0, misaligned states or
 * output), RANMAR_ERANGE (n_states = 0 with n_desc > 0).  Device:
 * RANMAR_ST_BAD_INDEX (state_idx >= n_states), RANMAR_ST_OUT_RANGE
 * (out_offset + count > out_len); the bad descriptor is skipped.
 */
int ranmar_generate_u24(ranmar_state_t *d_states, size_t n_states,
                        const ranmar_desc_t *d_desc, size_t n_desc,
                        uint32_t *d_out, size_t out_len,
                        uint32_t *d_status, ranmar_stream_t stream);
int ranmar_generate_f32(ranmar_state_t *d_states, size_t n_states,
                        const ranmar_desc_t *d_desc, size_t n_desc,
                        float *d_out, size_t out_len,
                        uint32_t *d_status, ranmar_stream_t stream);

/*
 * ranmar_check_overlap -- the non-overlap condition of the partition
 * (Sec. 1): stream k of (base, J) owns the transitions [kJ, (k+1)J), so
 * `count` outputs from a state at position pos stay inside it iff off = pos
 * - kJ satisfies off <= J and count <= J - off.  For each descriptor i (its
 * state d_states[state_idx] as it is BEFORE the generation, d_k[i] the
 * stream index that state belongs to) a generation that would leave the
 * stream OR-s RANMAR_ST_OVERLAP into *d_status.  Nothing is refused or
 * changed: such outputs are still RANMAR outputs, only no longer disjoint
 * from stream k+1's.  off is computed mod 2^64 (the state keeps pos mod
 * 2^64), exact while the true offset is below 2^64; for J >= 2^64 only off
 * + count > 2^64 is flagged.  h_J: J as J_words little-endian 32-bit words.
 * Errors: RANMAR_EINVAL (a null pointer with n_desc > 0, d_status NULL,
 * misaligned states, descriptors or d_k), RANMAR_ERANGE (J_words not in
 * 1..5, J = 0, n_states = 0 with n_desc > 0).  Device: RANMAR_ST_BAD_INDEX
 * for state_idx >= n_states.
 */
int ranmar_check_overlap(const ranmar_state_t *d_states, size_t n_states,
                         const ranmar_desc_t *d_desc, size_t n_desc,
                         const uint64_t *d_k, const uint32_t *h_J, uint32_t J_words,
                         uint32_t *d_status, ranmar_stream_t stream);

/*
 * ranmar_generate_alg1_f32 / _f64 -- Algorithm 1 (Sec. 4, the floating-point
 * form LAMMPS uses) over the same descriptors: the lagged Fibonacci words,
 * the arithmetic sequence and the output are computed as reals in [0, 1)
 * with the "if negative, add 1 (or cm)" fix-ups, in float or double.  Every
 * value is a multiple of 2^-24, so both are exact and equal
 * ranmar_generate_f32's outputs (the integer form times 2^-24, Sec. 3.1);
 * they exist to compare the cost of the two forms on the GPU (Table 1).
 * The state format (and write-back) is the integer one.  Errors as
 * ranmar_generate_u24 (d_out aligned to its element size).
 */
int ranmar_generate_alg1_f32(ranmar_state_t *d_states, size_t n_states,
                             const ranmar_desc_t *d_desc, size_t n_desc,
                             float *d_out, size_t out_len,
                             uint32_t *d_status, ranmar_stream_t stream);
int ranmar_generate_alg1_f64(ranmar_state_t *d_states, size_t n_states,
                             const ranmar_desc_t *d_desc, size_t n_desc,
                             double *d_out, size_t out_len,
                             uint32_t *d_status, ranmar_stream_t stream);

/*
 * ranmar_generate_plain_u24 / _f32 -- Algorithm 2 for ONE stream in one
 * launch of one warp: `count` outputs of *d_state into d_out[0..count); if
 * write_back != 0 the state is advanced in place.  This is the
 * one-launch-per-stream path that the batched calls are measured against.
 * Errors: RANMAR_EINVAL (null pointer with count > 0, misalignment).
 */
int ranmar_generate_plain_u24(ranmar_state_t *d_state, uint64_t count,
                              uint32_t *d_out, int write_back,
                              ranmar_stream_t stream);
int ranmar_generate_plain_f32(ranmar_state_t *d_state, uint64_t count,
                              float *d_out, int write_back,
                              ranmar_stream_t stream);

/* ------------------------------------------------------------------------
 * Fixed-base table jump: the same states as ranmar_jump / ranmar_partition.
 * (Sec. 3.1: t^E mod phi, here as the product of precomputed powers.)
 * ------------------------------------------------------------------------ */

/* Opaque handle: T[j][d] = t^{d 2^{8j}} mod phi (j < 20, d < 256) on one
 * device, 5,120 rows of 100 words (2,048,000 bytes).  The table depends only
 * on phi = t^97 + t^64 - 1, not on seeds or jump sizes. */
typedef struct ranmar_table ranmar_table_t;

/* Allocates (cudaMalloc) and builds the table on the current device by
 * left-to-right square-and-multiply of each row's exponent; synchronous
 * (a few ms).  Errors: RANMAR_EINVAL, RANMAR_ENOMEM, RANMAR_ECUDA. */
int ranmar_table_create(ranmar_table_t **out);
/* Frees the table (synchronizes its device).  NULL is a no-op. */
int ranmar_table_destroy(ranmar_table_t *t);
/* Caps the table-jump launches at ctas_per_sm resident CTAs per SM (the
 * kernel then strides over the remaining streams), leaving SM resources to
 * work running concurrently on another stream (e.g. generation of the
 * previous batch).  0 (the default) launches one CTA per 16 streams.
 * Errors: RANMAR_EINVAL (NULL, or outside 0..64). */
int ranmar_table_set_ctas_per_sm(ranmar_table_t *t, int ctas_per_sm);
/* Lanes per stream of the table jumps (Sec. 3.1; same results either way):
 *   RANMAR_JUMP_MAP_AUTO (default): a warp per stream for batches of at most
 *     RANMAR_JUMP_WARP_AUTO_MAX streams, two lanes per stream above;
 *   RANMAR_JUMP_MAP_PAIR: two lanes per stream, 16 streams per warp (the
 *     97 x 97 products register-tiled in 16 x 16 blocks; the most work per
 *     SM, for batches that fill the GPU);
 *   RANMAR_JUMP_MAP_WARP: one warp per stream (each lane forms a few
 *     product coefficients and output words; the shortest time per stream,
 *     for small batches such as the first streams of a partition plan or
 *     the segment jumps of a serving iteration).
 * ranmar_table_set_jump_mapping sets it for the table's jumps and
 * partitions, ranmar_plan_set_jump_mapping for the plan's jumps by the
 * powers of t^J.  Errors: RANMAR_EINVAL (NULL, unknown mapping). */
#define RANMAR_JUMP_MAP_AUTO 0
#define RANMAR_JUMP_MAP_PAIR 1
#define RANMAR_JUMP_MAP_WARP 2
#define RANMAR_JUMP_WARP_AUTO_MAX 8192
/* The square-and-multiply jumps (ranmar_jump, ranmar_jump_scatter,
 * ranmar_partition, ranmar_partition_ex without a table) and
 * ranmar_poly_power take a warp per stream up to this many streams. */
#define RANMAR_SQUARE_WARP_AUTO_MAX 1536
int ranmar_table_set_jump_mapping(ranmar_table_t *t, int map);
/* Device address of the rows (row j*256 + d, 100 words each), for checks. */
int ranmar_table_rows(const ranmar_table_t *t, const uint32_t **d_rows);

/*
 * ranmar_jump_tab -- d_dst[d_dst_idx ? d_dst_idx[i] : i] = f^{E_i}(base_i)
 * exactly as ranmar_jump / ranmar_jump_scatter, with t^{E_i} mod phi formed
 * as the product of the table rows of E_i's nonzero base-256 digits (one
 * general polynomial product per digit after the first) instead of
 * bitlen(E_i) squarings.  Without d_dst_idx the destinations are d_dst[0..n)
 * (n_dst >= n, no overlap with d_base); with it the scatter rules of
 * ranmar_jump_scatter apply.  Errors: as ranmar_jump / ranmar_jump_scatter,
 * plus RANMAR_EINVAL for a NULL table or a table of another device.
 */
int ranmar_jump_tab(const ranmar_table_t *t, const ranmar_state_t *d_base, size_t n_base,
                    const uint32_t *d_base_idx, const uint32_t *d_exp, uint32_t exp_words,
                    ranmar_state_t *d_dst, size_t n_dst, const uint32_t *d_dst_idx,
                    size_t n, uint32_t *d_status, ranmar_stream_t stream);

/* ranmar_partition_tab -- ranmar_partition with the table jump. */
int ranmar_partition_tab(const ranmar_table_t *t, const ranmar_state_t *d_base,
                         const uint32_t *h_J, uint32_t J_words, uint64_t k0,
                         ranmar_state_t *d_out, size_t n, ranmar_stream_t stream);

/* Flag of ranmar_partition_ex: the polynomial part of each jump uses
 * E mod T, T = (2^97 - 1) 2^23 = 2^120 - 2^23, the multiplicative order of t
 * modulo phi over Z/2^24 (t^T = 1, so t^E = t^(E mod T)); c still uses
 * E mod m (Sec. 3.2).  The jumped states are identical; long exponents (the
 * paper's J ~ 2^120) get much shorter.  Not in the paper (which jumps with
 * the unreduced E); the period follows from its Sec. 2 (about 2^144 in all,
 * 2^120 of it from the lagged Fibonacci part). */
#define RANMAR_JUMP_REDUCE_PERIOD 1u

/*
 * ranmar_partition_ex -- ranmar_partition (t == NULL: square-and-multiply)
 * or ranmar_partition_tab (t != NULL) with flags (0 or
 * RANMAR_JUMP_REDUCE_PERIOD).  Errors: as those, plus RANMAR_EINVAL for an
 * unknown flag.
 */
int ranmar_partition_ex(const ranmar_table_t *t, const ranmar_state_t *d_base,
                        const uint32_t *h_J, uint32_t J_words, uint64_t k0,
                        ranmar_state_t *d_out, size_t n, uint32_t flags,
                        ranmar_stream_t stream);

/*
 * Partition plan: stream partitioning (Sec. 1) of one base state into
 * consecutive blocks k = k0 + i of length J, computed level by level with
 * jump matrices.  The x part of a jump is linear over Z/2^24 (x' = x A^E,
 * Sec. 3.1), so the jump of many states by one fixed E is one matrix
 * product; row i of the 97x97 matrix M_E is the x part of the unit state
 * e_i jumped by E (the polynomial method of Sec. 3.1, via the table).  The
 * first 256 streams are jumped directly; level 0 takes them to 65,536
 * (radix 256), each later level multiplies the count by 16.  A plan holds
 * M_E for E = r R_t J (R_t = streams known before level t, r = 1 .. radix-1)
 * for the levels max_n needs: 255 matrices (19 MB of device images) for
 * max_n <= 65,536, 15 more per further level.
 *
 * ranmar_plan_create: builds the matrices on the current device (which must
 * be the table's), and a table of the powers of t^J (rows t^{d 2^{8j} J}
 * for the base-256 digits d of k, j < W with W = min(8, (160 - bitlen J)/8)),
 * and returns when they are ready (synchronous).  The plan
 * keeps a pointer to *t, which must outlive it.  Errors: RANMAR_EINVAL
 * (null pointer, table of another device), RANMAR_ERANGE (J_words not in
 * 1..5, max_n not in 1..2^32, r R_t J >= 2^160 for a needed matrix),
 * RANMAR_ENOMEM, RANMAR_ECUDA.
 */
typedef struct ranmar_plan ranmar_plan_t;
int ranmar_plan_create(const ranmar_table_t *t, const uint32_t *h_J, uint32_t J_words,
                       size_t max_n, ranmar_plan_t **out);
int ranmar_plan_destroy(ranmar_plan_t *p);

/*
 * ranmar_partition_plan -- the same states as ranmar_partition with the
 * plan's J: d_out[i] = f^{(k0+i) J}(*d_base), i < n <= max_n.  The first
 * 256 streams are jumped directly: by the plan's table of the powers of t^J
 * when it covers k0 + 255 (P_{kJ} from the digits of k: no product for
 * k < 256, at most one for k < 2^16), else by the fixed-base table; then each level derives
 * streams r R + i from streams i < R by x <- x M_{rRJ} (one dense GEMM per
 * level, 9,409 multiply-adds per stream against a matrix shared by all R
 * streams), c by the closed form of Sec. 3.2.  Asynchronous on `stream`.
 * Errors: RANMAR_EINVAL (null pointer, misalignment, d_out overlapping
 * *d_base, plan of another device), RANMAR_ERANGE (n > max_n,
 * (k0 + n - 1) J >= 2^160).
 */
int ranmar_partition_plan(const ranmar_plan_t *p, const ranmar_state_t *d_base, uint64_t k0,
                          size_t n, ranmar_state_t *d_out, ranmar_stream_t stream);

/*
 * ranmar_plan_expand -- the levels of ranmar_partition_plan alone: given
 * d_states[i] = f^{(k0+i) J}(base) for i < 256 (any k0, e.g. from
 * ranmar_partition_tab on another stream), fills d_states[256 .. n).  A
 * no-op for n <= 256.  Errors: RANMAR_EINVAL (null pointer, misalignment,
 * plan of another device), RANMAR_ERANGE (n > max_n).
 */
int ranmar_plan_expand(const ranmar_plan_t *p, ranmar_state_t *d_states, size_t n,
                       ranmar_stream_t stream);

/*
 * ranmar_plan_jump -- every stream by the plan's table of the powers of t^J
 * (Sec. 1 start states, the polynomial method of Sec. 3.1 with the product
 * over the base-256 digits of k instead of those of kJ): d_out[i] =
 * f^{(k0+i) J}(*d_base), i < n (any n), (nonzero digits of k) - 1 products
 * and the application per stream.  The same states as ranmar_partition.
 * Asynchronous on `stream`.  Errors: RANMAR_EINVAL (null pointer,
 * misalignment, d_out overlapping *d_base, plan of another device),
 * RANMAR_ERANGE ((k0 + n - 1) J >= 2^160, or k0 + n - 1 >= 256^W, W the
 * table's windows).
 */
int ranmar_plan_jump(const ranmar_plan_t *p, const ranmar_state_t *d_base, uint64_t k0,
                     size_t n, ranmar_state_t *d_out, ranmar_stream_t stream);

/*
 * How the plan's levels multiply (same results either way):
 *   RANMAR_PLAN_TENSOR: tcgen05 MMAs on fp16 limbs -- every 24-bit
 *     word split into three balanced 8-bit limbs (exact in fp16), the limb
 *     products accumulated exactly in fp32 in tensor memory and recombined
 *     mod 2^24; operands staged in shared memory (the matrix by a bulk async
 *     copy);
 *   RANMAR_PLAN_IMAD: blocked 32-bit integer multiply-adds;
 *   RANMAR_PLAN_TENSOR_PIPELINED (default): tcgen05 MMAs on the same limbs,
 *     with the limb image of the source rows in tensor memory, the whole
 *     weight-2^16 sum in one accumulator, two B images in shared memory and
 *     the MMAs of the next (tile, matrix) item running while the current one
 *     is read back.
 * ranmar_plan_set_method: RANMAR_EINVAL for an unknown method.
 * ranmar_plan_set_ctas: the number of CTAs a tensor-core level launches (one
 *   CTA per SM at most, each taking a balanced range of (tile, matrix)
 *   items); 0 (the default) = one per SM.  Fewer CTAs leave the other SMs
 *   to work on another stream at the same time (e.g. the generation of the
 *   previous batch).  RANMAR_EINVAL above 65535.
 * ranmar_plan_status: device pointer to the plan's status word (bit
 * RANMAR_ST_TIMEOUT if a tensor-core level gave up on a bounded wait; then
 * the states it was to write are not valid).  Cleared at plan creation.
 */
#define RANMAR_PLAN_TENSOR 0
#define RANMAR_PLAN_IMAD 1
#define RANMAR_PLAN_TENSOR_PIPELINED 2
int ranmar_plan_set_method(ranmar_plan_t *p, int method);
int ranmar_plan_set_ctas(ranmar_plan_t *p, unsigned ctas);
int ranmar_plan_set_jump_mapping(ranmar_plan_t *p, int map);

/*
 * ranmar_debug_set_wait_limit -- a test hook for the timeout path of the
 * bounded device waits of the tensor-core plan levels: with iterations > 0
 * the first wait of every CTA is made on a barrier that nothing completes,
 * probed without blocking at most `iterations` times, so that it runs out
 * without faulting or hanging anything (0 restores normal operation).  A
 * CTA whose wait ran out flags RANMAR_ST_TIMEOUT in the plan's status word,
 * still waits (bounded) for its own copies and MMAs in flight, frees its
 * tensor memory and returns.  Synchronizes the
 * device before and after.  Errors: RANMAR_ECUDA.
 */
int ranmar_debug_set_wait_limit(uint32_t iterations);

/*
 * ranmar_debug_fail_next -- host-side failure injection for tests: the next
 * entry point that launches a kernel returns `code` (a RANMAR_E* value, or 0
 * to clear) once, as if its launch had failed; the kernel itself was still
 * enqueued and runs normally.  Errors: RANMAR_EINVAL for a code that is not
 * 0 or a RANMAR_E* value.
 */
int ranmar_debug_fail_next(int code);
int ranmar_plan_status(const ranmar_plan_t *p, uint32_t **d_status);

/* ------------------------------------------------------------------------
 * Lagged Fibonacci recurrences of general order (the concluding remarks):
 * x_n = x_{n-r} - x_{n-s} mod 2^e, 2 <= r <= 2048, 1 <= s < r, 1 <= e <= 32;
 * for r = 97, s = 33, e = 24 the lagged Fibonacci part of RANMAR.  A state is
 * the window x_{n-r} .. x_{n-1}, r uint32 words, oldest first.  The jump by E
 * is x' = x P_E(A), P_E = t^E mod (t^r + t^{r-s} - 1) by binary
 * exponentiation (Sec. 3.1 with general lags), each squaring by the
 * classical product (r^2 multiply-adds) or by Karatsuba's (3^L products of
 * r/2^L coefficients with L levels, about r^{log2 3} for deep splits).
 * ------------------------------------------------------------------------ */
#define RANMAR_LFG_CLASSICAL 0
#define RANMAR_LFG_KARATSUBA 1                 /* depth chosen by the library */
#define RANMAR_LFG_KARATSUBA_LEVELS(L) (16 + (L))  /* exactly L = 1..6 levels */

/*
 * ranmar_lfg_jump -- d_out[i] = the window d_x[d_base_idx[i]] (or d_x[0]
 * when d_base_idx is NULL) jumped by E_i = d_exp[i * exp_words ..]
 * (little-endian 32-bit words, exp_words in 1..5).  d_x holds n_base windows
 * of r words, d_out n windows (must not overlap d_x).  One CTA per stream.
 * Errors: RANMAR_EINVAL (r, s, e or method out of range, null pointer,
 * misalignment, overlap), RANMAR_ERANGE (exp_words, n_base = 0, the shape
 * does not fit on the device).  Device: RANMAR_ST_BAD_INDEX for
 * d_base_idx[i] >= n_base (that stream is skipped).
 */
int ranmar_lfg_jump(uint32_t r, uint32_t s, uint32_t e, int method, const uint32_t *d_x,
                    size_t n_base, const uint32_t *d_base_idx, const uint32_t *d_exp,
                    uint32_t exp_words, uint32_t *d_out, size_t n, uint32_t *d_status,
                    ranmar_stream_t stream);

/*
 * ranmar_lfg_generate -- for each of the n windows d_x[i] (r words), the
 * next `count` words of the recurrence to d_out[i * count ..] (masked to e
 * bits), and the window advanced in place.  One warp per stream, min(32, s)
 * words per step.  Errors: RANMAR_EINVAL (r, s, e out of range, null
 * pointer, misalignment, overlap), RANMAR_ERANGE (n * count overflows).
 */
int ranmar_lfg_generate(uint32_t r, uint32_t s, uint32_t e, uint32_t *d_x, size_t n,
                        uint64_t count, uint32_t *d_out, ranmar_stream_t stream);

/*
 * ranmar_lfg_karatsuba_levels -- the number of Karatsuba levels the jump
 * uses for (r, s, e, method): 0 for the classical product.
 * RANMAR_LFG_KARATSUBA takes 2 levels for r >= 1024, 1 for 512 <= r < 1024
 * and the classical product below (the fastest on GB300 in a sweep of r =
 * 97, 607, 1279, 2048 and depths 0..5: a deeper split saves multiply-adds
 * but needs more shared memory, so fewer CTAs share an SM).
 * RANMAR_EINVAL for arguments out of range or an explicit depth that does
 * not fit (leaves of at least 8 coefficients within 200 KB of shared
 * memory).
 */
int ranmar_lfg_karatsuba_levels(uint32_t r, uint32_t s, uint32_t e, int method);

/*
 * ranmar_partition_generate_u24 / ranmar_partition_generate_f32 -- stream
 * partitioning (Sec. 1) and generation (Algorithm 2) fused in one kernel.
 * Stream i (block k = k0 + i of length J of the sequence that starts at
 * *d_base) is jumped to f^{kJ}(base) with the table (as
 * ranmar_partition_tab), then its first `count` outputs go to
 * d_out[i count .. (i+1) count) (u24 in uint32, or u24 * 2^-24 as float,
 * exact), and d_states[i] receives f^{kJ + count}(base), the state after
 * those outputs (for resume).  flags: 0 or RANMAR_JUMP_REDUCE_PERIOD.
 * d_states holds n states (the caller's, 16-byte aligned, not overlapping
 * *d_base); d_out holds n * count elements (aligned to the element size).
 * Same results as ranmar_partition_tab followed by ranmar_generate_* with
 * WRITE_BACK descriptors (state i, offset i count); one launch instead of
 * two, so that jumps and stores overlap on each SM.
 * Errors: RANMAR_EINVAL (null pointer with n > 0, misalignment, overlap,
 * unknown flag, table of another device), RANMAR_ERANGE (J_words not in
 * 1..5, (k0 + n - 1) J >= 2^160, n * count overflowing size_t).
 */
int ranmar_partition_generate_u24(const ranmar_table_t *t, const ranmar_state_t *d_base,
                                  const uint32_t *h_J, uint32_t J_words, uint64_t k0,
                                  size_t n, uint64_t count, uint32_t flags,
                                  ranmar_state_t *d_states, uint32_t *d_out,
                                  ranmar_stream_t stream);
int ranmar_partition_generate_f32(const ranmar_table_t *t, const ranmar_state_t *d_base,
                                  const uint32_t *h_J, uint32_t J_words, uint64_t k0,
                                  size_t n, uint64_t count, uint32_t flags,
                                  ranmar_state_t *d_states, float *d_out,
                                  ranmar_stream_t stream);

/* ------------------------------------------------------------------------
 * Persistent batch path: many streams of uneven lengths in one launch.
 * (Sec. 1 partitioning applied to a batch; Algorithm 2 per stream.)
 * ------------------------------------------------------------------------ */

/* Opaque handle: owns a device workspace on the device that was current at
 * creation (queue counter and prefix-sum scratch).  Calls that use one
 * handle must be ordered on one stream; use one handle per concurrent
 * stream. */
typedef struct ranmar_batch ranmar_batch_t;

/* Launch configuration of the persistent kernel. */
typedef struct ranmar_batch_config {
    int32_t lanes_per_stream;   /* 32, 16, 8 or 4 = outputs per group step */
    int32_t threads_per_cta;    /* multiple of 32, 32..1024 */
    int32_t ctas_per_sm;        /* resident CTAs per SM; 0 = as many as fit */
    int32_t chunk;              /* descriptors taken per queue pull, >= 1 */
} ranmar_batch_config_t;

/* ranmar_batch_create -- allocates the workspace (cudaMalloc) for batches of
 * up to `capacity` streams on the current device.  The default config is
 * {32, 256, 0, 1}.  Errors: RANMAR_EINVAL (out NULL), RANMAR_ERANGE
 * (capacity 0 or >= 2^32), RANMAR_ENOMEM, RANMAR_ECUDA. */
int ranmar_batch_create(size_t capacity, ranmar_batch_t **out);

/* Frees the workspace (synchronizes the device first).  NULL is a no-op. */
int ranmar_batch_destroy(ranmar_batch_t *b);

/* Set / read the persistent-kernel config.  RANMAR_EINVAL for a config
 * outside the ranges above. */
int ranmar_batch_set_config(ranmar_batch_t *b, const ranmar_batch_config_t *cfg);
int ranmar_batch_get_config(const ranmar_batch_t *b, ranmar_batch_config_t *cfg);

/* ranmar_batch_pack -- from per-stream counts (d_counts[i], device) builds
 * d_desc[i] = {state_idx i, flags, out_offset = sum_{j<i} counts[j],
 * count = counts[i]} (outputs packed back to back by an exclusive prefix
 * sum on the device), optionally d_order (a permutation of 0..n-1 visiting
 * streams longest first, by floor(log2(count)) bucket; NULL to skip) and
 * optionally *d_total (device, sum of all counts; NULL to skip).
 * Errors: RANMAR_EINVAL (NULL b/d_counts/d_desc with n > 0, b on another
 * device), RANMAR_ERANGE (n > capacity). */
int ranmar_batch_pack(ranmar_batch_t *b, const uint64_t *d_counts, size_t n,
                      uint32_t flags, ranmar_desc_t *d_desc, uint32_t *d_order,
                      uint64_t *d_total, ranmar_stream_t stream);

/* ranmar_batch_generate_u24 / _f32 -- the same outputs as
 * ranmar_generate_u24/_f32 for the same descriptors, from one persistent
 * launch: groups of lanes_per_stream lanes pull `chunk` descriptors at a
 * time from a device queue, in d_order's order (NULL = index order).  The
 * queue counter is reset on `stream` before the launch (capturable in a
 * CUDA graph).  Errors as ranmar_generate_u24, plus RANMAR_EINVAL for a NULL
 * or foreign-device handle.  Device: RANMAR_ST_BAD_INDEX also for
 * d_order[t] >= n_desc. */
int ranmar_batch_generate_u24(ranmar_batch_t *b, ranmar_state_t *d_states, size_t n_states,
                              const ranmar_desc_t *d_desc, size_t n_desc,
                              const uint32_t *d_order, uint32_t *d_out, size_t out_len,
                              uint32_t *d_status, ranmar_stream_t stream);
int ranmar_batch_generate_f32(ranmar_batch_t *b, ranmar_state_t *d_states, size_t n_states,
                              const ranmar_desc_t *d_desc, size_t n_desc,
                              const uint32_t *d_order, float *d_out, size_t out_len,
                              uint32_t *d_status, ranmar_stream_t stream);

/* ranmar_batch_generate_mixed -- one persistent launch for a descriptor list
 * whose first n_u24 descriptors produce 24-bit words (as
 * ranmar_batch_generate_u24) and whose others, d_desc[n_u24 .. n_desc),
 * produce float32 outputs (as ranmar_batch_generate_f32, their bit patterns
 * in the same word array d_out), in index order.  The outputs and write-backs
 * equal those of the two separate calls.  With d_items (device, n_desc
 * items, or NULL for none) the launch also adds the ranmar_checksum of each
 * descriptor's outputs, read back from d_out after they are stored, into
 * d_results[d_items[t].result] (device, n_results words, zeroed by the
 * caller), with word i of descriptor t weighted by 2 (d_items[t].index0 + i)
 * + 1; the items' offset and count are not read (the descriptor's are
 * used).  The handle's config applies, with at most 256 threads a CTA
 * (d_order is not taken).  Errors as ranmar_batch_generate_u24, plus
 * RANMAR_ERANGE for n_u24 > n_desc and RANMAR_EINVAL for d_items without
 * d_results.  Device: RANMAR_ST_OUT_RANGE for an item's result >= n_results
 * (its sum is skipped). */
int ranmar_batch_generate_mixed(ranmar_batch_t *b, ranmar_state_t *d_states, size_t n_states,
                                const ranmar_desc_t *d_desc, size_t n_desc, size_t n_u24,
                                uint32_t *d_out, size_t out_len,
                                const ranmar_sum_item_t *d_items, uint64_t *d_results,
                                size_t n_results, uint32_t *d_status, ranmar_stream_t stream);

/* ranmar_batch_tune -- autotuner: times every candidate config (group
 * width 32/16/8, 128/256/512 threads, chunk 1/8, all resident CTAs) on this
 * batch (write-back disabled, so the states are not advanced; the outputs
 * are written, with their correct values), keeps the fastest in the handle
 * and returns its time in *best_ms (may be NULL).  Synchronizes `stream`.
 * f32 != 0 tunes the float kernel.  Errors as ranmar_batch_generate_u24. */
int ranmar_batch_tune(ranmar_batch_t *b, int f32, ranmar_state_t *d_states, size_t n_states,
                      const ranmar_desc_t *d_desc, size_t n_desc, const uint32_t *d_order,
                      void *d_out, size_t out_len, ranmar_stream_t stream, float *best_ms);

/*
 * ranmar_batch_pack_split -- like ranmar_batch_pack, with every stream
 * longer than `seg` outputs split into ceil(count / seg) pieces of at most
 * seg outputs; piece q >= 1 of a stream starts from the stream's state
 * jumped by q seg (Sec. 3.1: the jump by any E), so that the persistent
 * kernel's warps share a long stream instead of one warp running it alone.
 * The outputs of every stream stay where ranmar_batch_pack puts them
 * (offsets = exclusive prefix sum of the counts).
 * Inputs: d_counts (device, n uint64, n <= the batch's capacity); seg >= 1;
 * n_extra = sum over the streams of max(0, ceil(count / seg) - 1), computed
 * by the caller (which sizes the outputs by it).
 * Outputs (device, caller-owned):
 *   d_desc[0 .. n + n_extra): piece 0 of stream i at i (state_idx i), the
 *     extra pieces in stream order from n on (extra piece e: state_idx
 *     n + e); only a stream's last piece keeps RANMAR_DESC_WRITE_BACK from
 *     `flags`;
 *   d_src[e] = the stream of extra piece e; d_exp[2e], d_exp[2e+1] = the
 *     little-endian jump exponent q seg of extra piece e;
 *   *d_total = sum of the counts (may be NULL).
 * To run a split batch: states d_states[0 .. n + n_extra) with the streams'
 * states in [0, n); fill [n, n + n_extra) by ranmar_jump_tab(table,
 * d_states, n, d_src, d_exp, 2, d_states + n, n_extra, NULL, n_extra, ...);
 * ranmar_batch_generate_* over the n + n_extra descriptors (no order needed:
 * no piece is longer than seg); with write-back, ranmar_batch_split_finish.
 * Errors: RANMAR_EINVAL (NULL pointers, seg = 0, n = 0 with n_extra > 0,
 * misalignment, foreign-device handle), RANMAR_ERANGE (n above capacity,
 * n + n_extra >= 2^32).  Device: RANMAR_ST_OUT_RANGE in *d_status when the
 * pieces do not number n_extra (pieces beyond n_extra are not written;
 * descriptors for missing ones get count 0 and d_src UINT32_MAX).
 * Not in the paper: load balance for the batched path.
 */
int ranmar_batch_pack_split(ranmar_batch_t *b, const uint64_t *d_counts, size_t n, uint64_t seg,
                            size_t n_extra, uint32_t flags, ranmar_desc_t *d_desc,
                            uint32_t *d_src, uint32_t *d_exp, uint64_t *d_total,
                            uint32_t *d_status, ranmar_stream_t stream);

/*
 * ranmar_batch_split_finish -- after the generation of a split batch with
 * write-back: copies the advanced state of each split stream's last piece
 * (d_states[n + e]) back to the stream's own slot d_states[d_src[e]], so
 * that the states end as ranmar_batch_pack + generate would leave them.
 * Entries with d_src[e] >= n are skipped.  Asynchronous on `stream`.
 * Errors: RANMAR_EINVAL (NULL or misaligned with n_extra > 0).
 */
int ranmar_batch_split_finish(ranmar_state_t *d_states, size_t n, const uint32_t *d_src,
                              size_t n_extra, ranmar_stream_t stream);

/*
 * ranmar_batch_pack_static -- the same result as ranmar_batch_pack, for
 * callers that cannot allocate device memory.  Some host programs own the
 * whole GPU heap through their own allocator (a simulation package or a
 * caching allocator that reserves device memory up front), so a cudaMalloc
 * from a library would fail or fragment their pool, and some must not make
 * allocation calls at all inside their time step.  This variant needs no
 * ranmar_batch_t: its scratch (tile sums of the prefix sum, the bucket
 * histogram and cursors) lives in a fixed 9,472-byte array compiled into the
 * library, which every GPU that loads the library keeps until the process
 * exits.  The paper has no counterpart; it is an interface convenience.
 * Limits and behaviour:
 *   - n <= RANMAR_PACK_STATIC_MAX streams, else RANMAR_ERANGE (nothing is
 *     enqueued).
 *   - The first call on a device looks up the array's device address (once
 *     per device, with that device current); make that first call before
 *     any stream capture.  The address is cached for the life of the
 *     process and does not survive cudaDeviceReset: after resetting a
 *     device, do not call this function on it again.
 *   - d_order may be NULL (descriptors only, no visiting order); d_total
 *     may be NULL (the grand total then goes only to the internal array).
 *     n == 0 enqueues nothing except *d_total = 0 when d_total is given.
 *   - All calls share the one array and each call clears the parts that must
 *     start at zero; two calls whose work overlaps on the GPU (different
 *     streams, or different host threads) race and give wrong results.
 *   - The caller still owns d_counts, d_desc, d_order and d_total; nothing
 *     is allocated or freed.
 * Errors: RANMAR_EINVAL (NULL d_counts/d_desc with n > 0, misalignment),
 * RANMAR_ERANGE, RANMAR_ECUDA.
 */
#define RANMAR_PACK_STATIC_MAX 1048576
int ranmar_batch_pack_static(const uint64_t *d_counts, size_t n, uint32_t flags,
                             ranmar_desc_t *d_desc, uint32_t *d_order, uint64_t *d_total,
                             ranmar_stream_t stream);

/* ------------------------------------------------------------------------
 * CUDA graphs: capture a sequence of the calls above on one stream and
 * replay it with one launch (buffers and arguments are frozen at capture).
 * ------------------------------------------------------------------------ */
typedef struct ranmar_graph ranmar_graph_t;

/* Starts capturing `stream` (thread-local capture mode).  The legacy NULL
 * stream cannot be captured: RANMAR_EINVAL. */
int ranmar_graph_begin(ranmar_stream_t stream);
/* Ends the capture, instantiates it into *out and uploads it to the device
 * (synchronizes `stream`). */
int ranmar_graph_end(ranmar_stream_t stream, ranmar_graph_t **out);
/* Replays the captured work on `stream`. */
int ranmar_graph_launch(const ranmar_graph_t *g, ranmar_stream_t stream);
/* Frees the graph.  NULL is a no-op. */
int ranmar_graph_destroy(ranmar_graph_t *g);

/* ------------------------------------------------------------------------
 * Output checksums (serving: outputs are consumed on the device).
 * ------------------------------------------------------------------------ */

/* (ranmar_sum_item_t: see the descriptor types above.) */

/*
 * ranmar_checksum -- for each item: results[item.result] += sum_i
 * data[offset + i] * (2 (index0 + i) + 1) mod 2^64 (32-bit words: the u24
 * values or the float32 bit patterns).  Items of one request split at any
 * boundaries sum to the same total.  The caller zeroes d_results first.
 * Not part of the paper's method: it lets a server consume outputs on the
 * device and check them against a reference.
 * Errors: RANMAR_EINVAL (NULL pointer with n_items > 0, misalignment).
 * Device: RANMAR_ST_OUT_RANGE for an item outside data_len or n_results
 * (skipped).
 */
int ranmar_checksum(const uint32_t *d_data, size_t data_len,
                    const ranmar_sum_item_t *d_items, size_t n_items,
                    uint64_t *d_results, size_t n_results,
                    uint32_t *d_status, ranmar_stream_t stream);

/* ------------------------------------------------------------------------
 * Serving engine: a native continuous-batching scheduler over the calls
 * above.  A request asks for the next `count` outputs of stream k of
 * (seed, J) -- the block that starts k J transitions after the seeded state
 * of `seed` (Sec. 1) -- from output `offset` of that block on.  The engine
 * keeps stream states resident in a device state pool, so that a request
 * that starts where an earlier one of the same stream ended needs no jump.
 * Every scheduler iteration admits arrived requests in arrival order while
 * the output pool and the state pool allow, cuts each into segments of at
 * most `seg` outputs (one state each), and enqueues:
 *   - on a stream of the engine's own: ONE host-to-device copy of a packed
 *     staging buffer (which also holds the iteration's zeroed checksum
 *     slots), the seeding of new seeds, and the jumps of the segment start
 *     states (from the seeded state by k J + offset + j seg, or from the
 *     resident state by j seg; Sec. 3.1 / 3.2);
 *   - then on the caller's stream: one persistent generation of all
 *     segments (ranmar_batch_generate_mixed) with the checksum of every
 *     request's outputs (summed inside that launch from the stored words,
 *     or by ranmar_checksum after it for an iteration of more than 4,096
 *     segments; the outputs are consumed on the device and their region is
 *     then recycled), and the copy of the checksums back.
 * An iteration's jumps thus run while earlier iterations generate.  Up to
 * max_inflight iterations are on the device while the host builds the next.
 * Unlike the calls above, an engine owns device memory (budget_bytes + 400
 * max_seeds bytes and small buffers) and a stream, and synchronizes the
 * caller's stream.  An engine is used by one host thread at a time.
 * ------------------------------------------------------------------------ */
typedef struct ranmar_serve ranmar_serve_t;

#define RANMAR_SERVE_SQUARE 1u      /* jumps by square-and-multiply           */
                                    /* (ranmar_jump_scatter), not the table   */
#define RANMAR_SERVE_HOST_ONLY 2u   /* no device at all: the scheduler alone, */
                                    /* which records its plan (tests)         */

typedef struct ranmar_serve_config {
    uint64_t budget_bytes;   /* state pool (400 bytes an entry) + output pool */
    uint64_t seg;            /* outputs per segment, >= 1 */
    uint32_t state_entries;  /* states of the pool, >= 1 */
    uint32_t max_seeds;      /* rows of the seeded-state table, >= 1 */
    uint32_t max_segments;   /* segments one iteration takes (a larger request */
                             /* still runs, alone in its iteration) */
    uint32_t max_inflight;   /* iterations on the device at once, >= 1 */
    uint32_t flags;          /* RANMAR_SERVE_* */
    uint32_t reserved;       /* 0 */
} ranmar_serve_config_t;   /* 40 bytes */

/* ranmar_request_t.status */
#define RANMAR_REQ_PENDING (-1)   /* not served (the run ended before it)     */
#define RANMAR_REQ_DONE 0
#define RANMAR_REQ_TOO_LARGE 1    /* more outputs than the output pool, or    */
                                  /* more segments than the state pool holds  */
#define RANMAR_REQ_BAD 2          /* seed outside 1..900000000, or            */
                                  /* k J + offset + count > 2^160             */

typedef struct ranmar_request {
    double   t;          /* in: arrival, seconds after the start of the run;
                            non-decreasing along the array */
    int32_t  seed;       /* in */
    uint32_t f32;        /* in: 0 = 24-bit words, else float32 (word 2^-24) */
    uint64_t k;          /* in: stream index */
    uint64_t J[2];       /* in: stream length, little-endian 128-bit */
    uint64_t offset;     /* in: outputs of (seed, k, J) taken by earlier
                            requests (the request starts at k J + offset) */
    uint64_t count;      /* in: outputs asked for (0 is served, checksum 0) */
    double   done;       /* out: when the device finished its iteration,
                            seconds after the start (CUDA events) */
    double   host_done;  /* out: when the scheduler saw it (host clock) */
    uint64_t checksum;   /* out: ranmar_checksum of its outputs, its first
                            output having index 0 */
    int32_t  status;     /* out: RANMAR_REQ_* */
    uint32_t iteration;  /* out: the scheduler iteration that served it */
} ranmar_request_t;     /* 88 bytes */

typedef struct ranmar_serve_stats {   /* totals over the engine's runs */
    uint64_t iterations, segments, base_jumps, pool_jumps;
    uint64_t resumed;        /* requests that started from a resident state */
    uint64_t evicted;        /* resident states taken back for other work */
    uint64_t rejected;       /* requests with status TOO_LARGE or BAD */
    uint64_t outputs;        /* outputs served */
    uint64_t new_seeds;      /* seeds seeded during runs */
    uint64_t slow_loops;     /* scheduler loop turns longer than 10 ms */
    uint64_t max_loop_ns;    /* longest scheduler loop turn */
    uint64_t max_inflight;   /* most iterations on the device at once */
    uint64_t host_ns;        /* host time spent building + enqueueing */
    uint64_t max_admit_ns;   /* longest admission (incl. evictions) */
    uint64_t max_enqueue_ns; /* longest build + enqueue of an iteration */
    uint64_t max_retire_ns;  /* longest retirement (incl. waiting for it) */
    uint64_t resident;       /* resident streams now */
    uint32_t status;         /* RANMAR_ST_* bits the kernels set */
    uint32_t pad;
} ranmar_serve_stats_t;

/* Trace of a RANMAR_SERVE_HOST_ONLY engine: one record per segment. */
#define RANMAR_SEG_FROM_SEED 0    /* state = f^E(seeded state of the seed)   */
#define RANMAR_SEG_FROM_POOL 1    /* state = f^E(pool state src)             */
#define RANMAR_SEG_RESIDENT 2     /* pool state `entry` as it stands         */
typedef struct ranmar_serve_seg {
    uint32_t iteration;
    uint32_t request;     /* index into the run's request array */
    uint32_t kind;        /* RANMAR_SEG_* */
    uint32_t entry;       /* pool state jumped into and generated from */
    uint32_t src;         /* FROM_SEED: row of the seed table; FROM_POOL: entry */
    uint32_t flags;       /* RANMAR_DESC_WRITE_BACK on a request's last segment */
    uint32_t exp[RANMAR_MAX_EXP_WORDS];   /* E, little-endian (FROM_*) */
    uint32_t live_until;  /* iterations enqueued when its iteration retired */
    uint64_t out_offset;  /* first word in the output pool */
    uint64_t count;
    uint64_t index0;      /* index of its first output within the request */
} ranmar_serve_seg_t;   /* 72 bytes */

/*
 * ranmar_serve_create -- allocates an engine on the current device (with
 * RANMAR_SERVE_HOST_ONLY: host memory only, no CUDA call).  The output pool
 * is (budget_bytes - 400 state_entries) / 4 words.  Errors: RANMAR_EINVAL
 * (NULL, a zero size, unknown flags or reserved != 0), RANMAR_ERANGE (budget
 * below the state pool), RANMAR_ENOMEM, RANMAR_ECUDA.
 */
int ranmar_serve_create(const ranmar_serve_config_t *cfg, ranmar_serve_t **out);
/* Waits for the device and frees everything (NULL is a no-op).  Errors:
 * RANMAR_EINVAL when called with another device current. */
int ranmar_serve_destroy(ranmar_serve_t *e);

/*
 * ranmar_serve_preload -- gives the seeds h_seeds[0..n) rows of the seeded
 * state table and seeds them on `stream` (Algorithm 3), synchronously.
 * Errors: RANMAR_EINVAL (NULL, a seed outside 1..900000000), RANMAR_ERANGE
 * (more distinct seeds than max_seeds), RANMAR_ENOMEM, RANMAR_ECUDA.
 */
int ranmar_serve_preload(ranmar_serve_t *e, const int32_t *h_seeds, size_t n,
                         ranmar_stream_t stream);

/*
 * ranmar_serve_run -- serves h_reqs[0..n) (host, caller-owned, read and
 * written during the call) and returns when all are done, refused, or the
 * run fails.  realtime != 0 replays the arrival times against the host
 * clock (a request is seen at h_reqs[i].t); realtime == 0 makes every
 * request available at once.  Writes each request's out fields.  Results do
 * not depend on how requests are batched: request i's outputs are outputs
 * offset .. offset + count - 1 of its stream whatever else runs.
 * Errors: RANMAR_EINVAL (NULL with n > 0, arrival times not sorted, an
 * engine whose earlier run failed), RANMAR_ERANGE (more distinct seeds than
 * max_seeds), RANMAR_ETIME (the run took longer than max_wait_s),
 * RANMAR_ESTATUS (a kernel set a status bit), and the errors of the calls
 * it makes.  After an error the engine refuses further runs; destroy it.
 */
int ranmar_serve_run(ranmar_serve_t *e, ranmar_request_t *h_reqs, size_t n, int realtime,
                     double max_wait_s, ranmar_stream_t stream);

/*
 * ranmar_serve_run_plain -- the comparator: every request alone, in
 * arrival order, with one square-and-multiply jump launch and one plain
 * one-warp generation launch (no batching, no segments, no resident
 * states), checksummed as above.  Same arguments, results and errors as
 * ranmar_serve_run (not on a host-only engine: RANMAR_EINVAL).
 */
int ranmar_serve_run_plain(ranmar_serve_t *e, ranmar_request_t *h_reqs, size_t n,
                           int realtime, double max_wait_s, ranmar_stream_t stream);

/* Totals over the engine's runs.  Errors: RANMAR_EINVAL (NULL). */
int ranmar_serve_get_stats(const ranmar_serve_t *e, ranmar_serve_stats_t *out);

/*
 * ranmar_serve_trace -- the segments a host-only engine planned, in the
 * order it planned them: copies min(cap, total) records to h_out and sets
 * *n_out = total.  A host-only engine runs no device work: its iterations
 * complete only when the scheduler must wait for one (so that as many as
 * max_inflight are in flight), and its checksums are 0.
 * Errors: RANMAR_EINVAL (NULL, or an engine with a device).
 */
int ranmar_serve_trace(const ranmar_serve_t *e, ranmar_serve_seg_t *h_out, size_t cap,
                       size_t *n_out);

/*
 * ranmar_host_device_pointer -- the device address of pinned (page-locked)
 * host memory, for generating straight into host memory: the kernels then
 * store over the CPU-GPU link instead of a separate device-to-host copy.
 * The memory must stay pinned while kernels use it.  Errors: RANMAR_EINVAL
 * (NULL, or memory that is not pinned: RANMAR_ECUDA), RANMAR_EDEVICE (the
 * device cannot map host memory).
 */
int ranmar_host_device_pointer(void *h_ptr, void **d_ptr);

/* Name of a return code (static string, never NULL). */
const char *ranmar_strerror(int code);

/* The CUDA error string behind the last RANMAR_ECUDA on this thread. */
const char *ranmar_last_cuda_error(void);

/* ABI version of this header: (major << 16) | minor. */
int ranmar_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RANMAR_H */
