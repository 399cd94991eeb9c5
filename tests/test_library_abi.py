"""CPU-side checks of libranmar: it loads, exports every symbol the header
declares, and its host logic (seeding, argument checks) is right.  No
compute call reaches a GPU here."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ranmar.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2512_00093_gb300.build import build_library
    path = build_library()
    from paper_2512_00093_gb300 import binding
    return binding._lib(), path


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ranmar_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for need in ["ranmar_seed", "ranmar_jump", "ranmar_partition", "ranmar_generate_u24",
                 "ranmar_generate_f32", "ranmar_generate_plain_u24", "ranmar_strerror"]:
        assert need in names


def test_library_exports_every_declared_symbol(lib):
    L, path = lib
    for name in declared_functions():
        assert hasattr(L, name), f"{name} declared in ranmar.h but not exported by {path}"


def test_abi_version_and_strerror(lib):
    L, _ = lib
    assert L.ranmar_abi_version() >> 16 == 1
    for code in (0, -1, -2, -3, -4, -5, -99):
        assert L.ranmar_strerror(code)


def test_host_seed_matches_oracle(orc):
    import paper_2512_00093_gb300 as rm
    rng = np.random.default_rng(0)
    seeds = [1, 2, 12345, 54217138, 900000000] + rng.integers(1, 900000001, 40).tolist()
    for s in seeds:
        st = rm.seed(int(s)).numpy().view(np.uint32)
        x, c = orc.seeded_state(int(s))
        assert np.array_equal(st[:97], x), s
        assert st[97] == c and st[98] == 0 and st[99] == 0


def test_seed_rejects_out_of_domain():
    import paper_2512_00093_gb300 as rm
    for bad in (0, -1, 900000001):
        with pytest.raises(rm.RanmarError):
            rm.seed(bad)


def test_host_argument_checks(lib):
    """Calls rejected by host checks return before any CUDA call."""
    L, _ = lib
    vp = ctypes.c_void_p
    fake = vp(0x10000)          # never dereferenced: every call below fails a host check
    assert L.ranmar_jump(None, 1, None, fake, 1, fake, 4, None, None) == -1
    assert L.ranmar_jump(fake, 1, None, fake, 0, vp(0x20000), 4, None, None) == -2
    assert L.ranmar_jump(fake, 1, None, fake, 6, vp(0x20000), 4, None, None) == -2
    assert L.ranmar_jump(fake, 0, None, fake, 1, vp(0x20000), 4, None, None) == -2
    assert L.ranmar_jump(fake, 4, None, fake, 1, vp(0x10000 + 400), 4, None, None) == -1  # overlap
    assert L.ranmar_jump(vp(0x10008), 1, None, fake, 1, vp(0x20000), 4, None, None) == -1  # align
    assert L.ranmar_jump(None, 0, None, None, 0, None, 0, None, None) == 0                  # n = 0
    J = (ctypes.c_uint32 * 5)(0, 0, 0, 0, 1 << 31)                                          # 2^159
    assert L.ranmar_partition(fake, J, 5, 1, vp(0x20000), 2, None) == -2                    # 2*2^159
    assert L.ranmar_partition(fake, J, 6, 0, vp(0x20000), 1, None) == -2
    assert L.ranmar_generate_u24(None, 1, fake, 1, fake, 10, None, None) == -1
    assert L.ranmar_generate_u24(fake, 0, fake, 1, fake, 10, None, None) == -2
    assert L.ranmar_generate_u24(fake, 1, fake, 0, fake, 10, None, None) == 0
    assert L.ranmar_generate_f32(fake, 1, fake, 1, vp(0x20002), 10, None, None) == -1
    assert L.ranmar_generate_plain_u24(None, 10, fake, 1, None) == -1
    assert L.ranmar_generate_plain_u24(fake, 10, None, 1, None) == -1
    L.ranmar_plan_set_ctas.argtypes = [ctypes.c_void_p, ctypes.c_uint]
    L.ranmar_debug_fail_next.argtypes = [ctypes.c_int]
    assert L.ranmar_debug_fail_next(1) == -1 and L.ranmar_debug_fail_next(-6) == -1
    assert L.ranmar_debug_fail_next(0) == 0
    assert L.ranmar_plan_set_ctas(None, 4) == -1
    L.ranmar_poly_power.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_size_t,
                                    ctypes.c_void_p, ctypes.c_void_p]
    assert L.ranmar_poly_power(None, 1, 1, fake, None) == -1
    assert L.ranmar_poly_power(fake, 0, 1, vp(0x20000), None) == -2
    assert L.ranmar_poly_power(fake, 6, 1, vp(0x20000), None) == -2
    assert L.ranmar_poly_power(None, 1, 0, None, None) == 0                              # n = 0
    L.ranmar_table_set_jump_mapping.argtypes = [ctypes.c_void_p, ctypes.c_int]
    L.ranmar_plan_set_jump_mapping.argtypes = [ctypes.c_void_p, ctypes.c_int]
    assert L.ranmar_table_set_jump_mapping(None, 0) == -1
    assert L.ranmar_plan_set_jump_mapping(None, 2) == -1
    L.ranmar_check_overlap.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                       ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p]
    jw = np.array([1000], dtype=np.uint32)
    zero = np.array([0, 0], dtype=np.uint32)
    d = jw.ctypes.data
    assert L.ranmar_check_overlap(fake, 1, fake, 1, fake, None, 1, fake, None) == -1  # J null
    assert L.ranmar_check_overlap(fake, 1, fake, 1, fake, d, 0, fake, None) == -2     # words
    assert L.ranmar_check_overlap(fake, 1, fake, 1, fake, d, 6, fake, None) == -2
    assert L.ranmar_check_overlap(fake, 1, fake, 1, fake, zero.ctypes.data, 2, fake,
                                  None) == -2                                          # J = 0
    assert L.ranmar_check_overlap(None, 0, None, 0, None, d, 1, None, None) == 0     # n = 0
    assert L.ranmar_check_overlap(fake, 1, fake, 1, fake, d, 1, None, None) == -1    # status
    assert L.ranmar_check_overlap(fake, 0, fake, 1, fake, d, 1, fake, None) == -2    # n_states
    L.ranmar_batch_generate_mixed.argtypes = [vp, vp, ctypes.c_size_t, vp, ctypes.c_size_t,
                                              ctypes.c_size_t, vp, ctypes.c_size_t, vp, vp]
    assert L.ranmar_batch_generate_mixed(None, fake, 1, fake, 1, 0, fake, 10, None,
                                         None) == -1                                   # handle
    L.ranmar_serve_create.argtypes = [vp, vp]
    L.ranmar_serve_run.argtypes = [vp, vp, ctypes.c_size_t, ctypes.c_int, ctypes.c_double, vp]
    L.ranmar_serve_get_stats.argtypes = [vp, vp]
    L.ranmar_serve_trace.argtypes = [vp, vp, ctypes.c_size_t, vp]
    L.ranmar_serve_destroy.argtypes = [vp]
    assert L.ranmar_serve_create(None, None) == -1
    assert L.ranmar_serve_run(None, None, 0, 0, 1.0, None) == -1
    assert L.ranmar_serve_get_stats(None, fake) == -1
    assert L.ranmar_serve_trace(None, None, 0, fake) == -1
    assert L.ranmar_serve_destroy(None) == 0


def test_workload_recipes():
    from paper_2512_00093_gb300 import workloads as wl
    lens = wl.BatchedUneven().lengths(200000)
    assert lens.min() >= 64 and lens.max() <= 65536
    # log-uniform on [64, 65536]: mean 64 * 1023 / ln 1024 ~ 9446
    assert abs(lens.mean() / 9446.0 - 1.0) < 0.02
    rows = wl.Partitioned().verify_rows()
    assert len(set(rows.tolist())) == 256 and rows.max() < 65536


def test_split_extra_counts_pieces():
    """Batch.split_extra (host): sum of max(0, ceil(c / seg) - 1), by brute force."""
    from paper_2512_00093_gb300.binding import Batch
    rng = np.random.default_rng(3)
    for seg in (1, 7, 64, 4096):
        c = np.concatenate([[0, 1, seg - 1, seg, seg + 1, 3 * seg], rng.integers(0, 70000, 500)])
        c = c[c >= 0]
        want = 0
        for x in c.tolist():
            pieces = 0
            left = x
            while left > 0:
                pieces += 1
                left -= seg
            want += max(0, pieces - 1)
        assert Batch.split_extra(c, seg) == want
    assert Batch.split_extra([], 10) == 0


def test_split_entry_points_reject_bad_arguments(lib):
    """Host checks of the split pack and its finish (no device work)."""
    L, _ = lib
    L.ranmar_batch_pack_split.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                          ctypes.c_uint64, ctypes.c_size_t, ctypes.c_uint32,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.ranmar_batch_split_finish.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                            ctypes.c_size_t, ctypes.c_void_p]
    fake = ctypes.c_void_p(0x10000)
    # no batch handle
    assert L.ranmar_batch_pack_split(None, fake, 4, 16, 0, 0, fake, None, None, None, None,
                                     None) == -1
    # finish: nothing to do with n_extra = 0; NULL or misaligned otherwise
    assert L.ranmar_batch_split_finish(None, 4, None, 0, None) == 0
    assert L.ranmar_batch_split_finish(None, 4, fake, 3, None) == -1
    assert L.ranmar_batch_split_finish(ctypes.c_void_p(0x10004), 4, fake, 3, None) == -1
