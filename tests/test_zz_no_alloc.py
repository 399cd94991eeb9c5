"""ranmar_batch_pack_static: packing without any device allocation.

Some programs that call this library cannot let it allocate GPU memory: the
host program's own allocator may already hold the device heap (so a
cudaMalloc from the library would fail or fragment that pool), or the
program must not allocate inside its time step.  For them the library has
a packing entry point whose scratch is a fixed array compiled into the
library.  These tests call it through the C ABI and check it against the
handle-based ranmar_batch_pack: descriptors and totals must be identical,
and the visiting order must be a permutation with the same longest-first
bucket sequence (the order inside one bucket is not fixed).  Two calls in a
row with different inputs check that the shared array is cleared between
calls.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch


def _lib():
    from paper_2512_00093_gb300.build import build_library
    build_library()
    from paper_2512_00093_gb300 import binding
    L = binding._lib()
    L.ranmar_batch_pack_static.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint32,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p]
    L.ranmar_batch_pack_static.restype = ctypes.c_int
    return L


def test_static_pack_rejects_oversized_batches():
    """Beyond RANMAR_PACK_STATIC_MAX (2^20 streams) the call fails before any
    device work (host check only, so it runs without a GPU)."""
    L = _lib()
    fake = ctypes.c_void_p(0x10000)
    assert L.ranmar_batch_pack_static(fake, (1 << 20) + 1, 0, fake, None, None, None) == -2


@pytest.mark.gpu
def test_static_pack_matches_handle_pack_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_00093_gb300 as rm
    L = _lib()
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream().cuda_stream
    # a large batch, then a smaller one with other counts: the second call must
    # not see the first call's histogram or tile sums
    for seed, n in [(1, 1 << 20), (2, 5003)]:
        rng = np.random.default_rng(seed)
        c = np.floor(64 * 1024.0 ** rng.random(n)).astype(np.int64)
        c[:6] = [0, 1, 31, 32, 33, 97]
        counts = torch.as_tensor(c, device=dev)
        b = rm.Batch(n)
        ref_desc, ref_order, ref_total = b.pack(counts, flags=rm.DESC_WRITE_BACK)
        desc = torch.full((n, 3), -1, dtype=torch.int64, device=dev)
        order = torch.full((n,), -1, dtype=torch.int32, device=dev)
        total = torch.full((1,), -1, dtype=torch.int64, device=dev)
        rc = L.ranmar_batch_pack_static(counts.data_ptr(), n, rm.DESC_WRITE_BACK,
                                        desc.data_ptr(), order.data_ptr(), total.data_ptr(),
                                        stream)
        assert rc == 0
        torch.cuda.synchronize()
        assert torch.equal(desc, ref_desc)
        assert int(total.item()) == int(ref_total.item()) == int(c.sum())
        o = order.cpu().numpy().astype(np.int64)
        ro = ref_order.cpu().numpy().astype(np.int64)
        assert np.array_equal(np.sort(o), np.arange(n))
        bits = np.array([int(x).bit_length() for x in c])
        assert np.array_equal(bits[o], bits[ro])
        assert np.all(np.diff(bits[o]) <= 0)
        b.close()


@pytest.mark.gpu
def test_static_pack_without_order_or_total_and_empty():
    """d_order = NULL and d_total = NULL give the same descriptors (the total
    then stays inside the library's array); n = 0 writes *d_total = 0."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_00093_gb300 as rm
    L = _lib()
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream().cuda_stream
    n = 3000
    c = np.floor(64 * 1024.0 ** np.random.default_rng(3).random(n)).astype(np.int64)
    counts = torch.as_tensor(c, device=dev)
    b = rm.Batch(n)
    ref_desc, _, _ = b.pack(counts, order=False)
    desc = torch.full((n, 3), -1, dtype=torch.int64, device=dev)
    assert L.ranmar_batch_pack_static(counts.data_ptr(), n, 0, desc.data_ptr(), None, None,
                                      stream) == 0
    torch.cuda.synchronize()
    assert torch.equal(desc, ref_desc)
    total = torch.full((1,), -1, dtype=torch.int64, device=dev)
    assert L.ranmar_batch_pack_static(counts.data_ptr(), 0, 0, desc.data_ptr(), None,
                                      total.data_ptr(), stream) == 0
    torch.cuda.synchronize()
    assert int(total.item()) == 0
    b.close()
