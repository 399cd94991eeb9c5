"""RANMAR on GB300: bulk generation of non-overlapping streams of the 24-bit
integer RANMAR generator with exact polynomial jump-ahead (arXiv 2512.00093).

The compute path is libranmar (CUDA, sm_103a), reached through the C ABI in
include/ranmar.h; this package is its thin binding plus the build step.
"""
from .binding import (  # noqa: F401
    DESC_WRITE_BACK, MAX_EXP_WORDS, R, ST_BAD_INDEX, ST_OUT_RANGE, STATE_WORDS, Batch,
    BatchConfig, Graph, RanmarError, abi_version, capture, check_overlap, checksum, checksum_np,
    debug_fail_next, debug_set_wait_limit,
    exps_tensor, ST_OVERLAP, ST_TIMEOUT,
    JUMP_REDUCE_PERIOD, JUMP_MAP_AUTO, JUMP_MAP_PAIR, JUMP_MAP_WARP, JUMP_WARP_AUTO_MAX, SQUARE_WARP_AUTO_MAX,
    generate_alg1_f32, generate_alg1_f64, generate_f32, jump_scatter,
    partition_ex,
    generate_plain_f32, generate_plain_u24, generate_u24, jump, lib_path, make_desc,
    partition, poly_power, seed, seed_batch, ST_BAD_SEED, shape_bucket, state_words_np, Table, Plan,
    LFG_CLASSICAL, LFG_KARATSUBA, LFG_KARATSUBA_LEVELS, lfg_jump, lfg_generate, lfg_karatsuba_levels, tune_cached, words,
)
