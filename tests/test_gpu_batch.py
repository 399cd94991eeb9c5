"""GPU parity of the persistent batch path: packing (prefix-sum offsets and
longest-first order), the persistent kernel at every group width, the
autotuner, CUDA-graph capture/replay, and the full-size uneven workload.
Tolerance 0: outputs are exact integers (or those integers times 2^-24)."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

F = 1.0 / 16777216.0


@pytest.fixture(scope="module")
def rm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_00093_gb300 as rm
    return rm


@pytest.fixture(scope="module")
def dev(rm):
    return torch.device("cuda:0")


def counts_mix(n, seed):
    rng = np.random.default_rng(seed)
    c = np.floor(64 * 1024.0 ** rng.random(n)).astype(np.int64)
    edge = np.array([0, 1, 2, 3, 4, 7, 8, 15, 16, 31, 32, 33, 63, 64, 65, 95, 96, 97, 98, 1000])
    c[: min(n, len(edge))] = edge[: min(n, len(edge))]
    return c


@pytest.mark.parametrize("n", [1, 5, 1023, 1024, 1025, 4097, 100_003])
def test_pack_offsets_and_order(rm, dev, n):
    c = counts_mix(n, n)
    b = rm.Batch(max(n, 1))
    desc, order, total = b.pack(torch.as_tensor(c, device=dev), flags=rm.DESC_WRITE_BACK)
    torch.cuda.synchronize()
    d = desc.cpu().numpy().view(np.uint64)
    assert np.array_equal(d[:, 0] & 0xFFFFFFFF, np.arange(n, dtype=np.uint64))
    assert np.all((d[:, 0] >> np.uint64(32)) == rm.DESC_WRITE_BACK)
    assert np.array_equal(d[:, 1], np.concatenate([[0], np.cumsum(c)[:-1]]).astype(np.uint64))
    assert np.array_equal(d[:, 2], c.astype(np.uint64))
    assert int(total.item()) == int(c.sum())
    o = order.cpu().numpy().astype(np.int64)
    assert np.array_equal(np.sort(o), np.arange(n))
    buckets = np.array([int(x).bit_length() for x in c[o]])
    assert np.all(np.diff(buckets) <= 0), "order must be longest bucket first"
    b.close()


def _reference_batch(rm, dev, states0, desc, total, f32):
    """The same batch through the one-warp-per-descriptor path (itself checked
    against the oracle in test_gpu_parity.py)."""
    st = states0.clone()
    out = torch.full((total + 3,), -1, dtype=torch.float32 if f32 else torch.int32, device=dev)
    (rm.generate_f32 if f32 else rm.generate_u24)(st, desc, out)
    return st, out


@pytest.mark.parametrize("lanes", [32, 16, 8, 4])
@pytest.mark.parametrize("f32", [False, True])
def test_persistent_equals_reference(rm, dev, orc, lanes, f32):
    n = 700
    c = counts_mix(n, 11)
    J = (1 << 64) + 3
    base = rm.seed(12345).to(dev)
    states0 = rm.partition(base, J, 5, n)
    b = rm.Batch(n)
    b.config = (lanes, 256, 0, 3)
    desc, order, total = b.pack(torch.as_tensor(c, device=dev), flags=rm.DESC_WRITE_BACK)
    tot = int(total.item())
    st_ref, out_ref = _reference_batch(rm, dev, states0, desc, tot, f32)
    st = states0.clone()
    out = torch.full_like(out_ref, -1)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    (b.generate_f32 if f32 else b.generate_u24)(st, desc, out, order=order, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert torch.equal(out, out_ref)
    assert torch.equal(st, st_ref)
    # and a few streams straight against the oracle
    got = out.cpu().numpy()
    offs = np.concatenate([[0], np.cumsum(c)[:-1]])
    for i in [0, 5, 19, 250, n - 1]:
        ref = orc.stream(12345, (5 + i) * J, int(c[i]))
        g = got[offs[i]:offs[i] + c[i]]
        if f32:
            assert np.array_equal(g, (ref.astype(np.float64) * F).astype(np.float32)), i
        else:
            assert np.array_equal(g.view(np.uint32), ref), i
    b.close()


@pytest.mark.parametrize("lanes,threads,ctas,n", [
    (32, 256, 0, 701), (16, 256, 0, 701), (8, 128, 0, 701), (4, 256, 0, 701),
    (32, 512, 0, 701),                           # more than 256 threads: clamped
    (32, 256, 1, 2001), (16, 128, 1, 2001)])     # more groups than resident: interleaved
def test_mixed_launch_equals_separate_calls(rm, dev, orc, lanes, threads, ctas, n):
    """ranmar_batch_generate_mixed: descriptors [0, n_u24) as 24-bit words,
    the rest as float32, in one launch, equal the two separate calls (outputs
    and written-back states), for a boundary inside an interleaved group and
    at the ends, with a stream a group (every group resident) and with
    interleaved groups (more descriptors than resident groups)."""
    c = counts_mix(n, 23)
    J = (1 << 100) + 77
    base = rm.seed(4242).to(dev)
    states0 = rm.partition(base, J, 0, n)
    b = rm.Batch(n)
    b.config = (lanes, threads, ctas, 1)
    desc, _, total = b.pack(torch.as_tensor(c, device=dev), flags=rm.DESC_WRITE_BACK)
    tot = int(total.item())
    for n_u24 in (0, 1, 350, 351, n - 3, n):
        st_ref = states0.clone()
        out_ref = torch.full((tot + 3,), -1, dtype=torch.int32, device=dev)
        rm.generate_u24(st_ref, desc[:n_u24], out_ref)
        rm.generate_f32(st_ref, desc[n_u24:], out_ref.view(torch.float32))
        st = states0.clone()
        out = torch.full_like(out_ref, -1)
        status = torch.zeros(1, dtype=torch.int32, device=dev)
        b.generate_mixed(st, desc, n_u24, out, status=status)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert torch.equal(out, out_ref), n_u24
        assert torch.equal(st, st_ref), n_u24
    # with the checksums kept by the launch: each descriptor's words, read
    # back after they are stored, into its slot (three descriptors a slot)
    idx0 = (np.arange(n) * 7919) % 100_003
    items = torch.tensor(np.stack([np.zeros(n), c, idx0, np.arange(n) // 3], 1).astype(np.int64),
                         device=dev)
    sums = torch.zeros((n + 2) // 3, dtype=torch.int64, device=dev)
    st3 = states0.clone()
    out3 = torch.full_like(out_ref, -1)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    b.generate_mixed(st3, desc, 351, out3, items=items, results=sums, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    ref_out = torch.full_like(out_ref, -1)
    st_ref = states0.clone()
    rm.generate_u24(st_ref, desc[:351], ref_out)
    rm.generate_f32(st_ref, desc[351:], ref_out.view(torch.float32))
    assert torch.equal(out3, ref_out) and torch.equal(st3, st_ref)
    words = ref_out.cpu().numpy().view(np.uint32)
    offs = np.concatenate([[0], np.cumsum(c)[:-1]])
    want = [0] * sums.numel()
    for i in range(n):
        want[i // 3] = (want[i // 3] + rm.checksum_np(words[offs[i]:offs[i] + c[i]],
                                                      index0=int(idx0[i]))) % (1 << 64)
    assert [int(x) for x in sums.cpu().numpy().astype(np.uint64)] == want
    got = out.cpu().numpy()
    for i in [0, 349, 350, n - 1]:         # n_u24 = n: all u24
        ref = orc.stream(4242, i * J, int(c[i]))
        assert np.array_equal(got[offs[i]:offs[i] + c[i]].view(np.uint32), ref), i
    with pytest.raises(rm.RanmarError):
        b.generate_mixed(st, desc, n + 1, out)
    b.close()


def test_tune_keeps_states_and_outputs(rm, dev):
    n = 3000
    c = counts_mix(n, 5)
    base = rm.seed(777).to(dev)
    states0 = rm.partition(base, 1 << 64, 0, n)
    b = rm.Batch(n)
    desc, order, total = b.pack(torch.as_tensor(c, device=dev), flags=rm.DESC_WRITE_BACK)
    tot = int(total.item())
    st_ref, out_ref = _reference_batch(rm, dev, states0, desc, tot, True)
    st = states0.clone()
    out = torch.zeros_like(out_ref)
    cfg, ms = b.tune(st, desc, out, order)
    torch.cuda.synchronize()
    assert torch.equal(st, states0), "tuning must not advance the states"
    assert cfg[0] in (32, 16, 8) and cfg[1] in (128, 256, 512) and cfg[3] in (1, 8) and ms > 0
    out[:tot] = -1
    b.generate_f32(st, desc, out, order=order)
    torch.cuda.synchronize()
    assert torch.equal(out[:tot], out_ref[:tot]) and torch.equal(st, st_ref)
    b.close()


def test_graph_capture_replay(rm, dev):
    """partition + pack + persistent generate captured once, replayed twice."""
    n = 2048
    c = counts_mix(n, 3)
    J = 1 << 64
    base = rm.seed(4242).to(dev)
    counts = torch.as_tensor(c, device=dev)
    tot = int(c.sum())
    b = rm.Batch(n)
    states = torch.empty((n, rm.STATE_WORDS), dtype=torch.int32, device=dev)
    desc = torch.empty((n, 3), dtype=torch.int64, device=dev)
    order = torch.empty(n, dtype=torch.int32, device=dev)
    total = torch.empty(1, dtype=torch.int64, device=dev)
    out = torch.zeros(tot, dtype=torch.float32, device=dev)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    import paper_2512_00093_gb300.binding as bd
    with rm.capture(s) as cap:
        rm.partition(base, J, 0, n, out=states, stream=s)
        bd._check(bd._lib().ranmar_batch_pack(b._h, counts.data_ptr(), n, 0, desc.data_ptr(),
                                              order.data_ptr(), total.data_ptr(), s.cuda_stream),
                  "pack")
        b.generate_f32(states, desc, out, order=order, stream=s)
    ref_states = rm.partition(base, J, 0, n)
    ref_desc = rm.make_desc(np.arange(n), np.concatenate([[0], np.cumsum(c)[:-1]]), c, 0,
                            device=dev)
    ref_out = torch.full_like(out, -1)
    rm.generate_f32(ref_states, ref_desc, ref_out)
    torch.cuda.synchronize()
    for _ in range(2):
        out.zero_()
        torch.cuda.synchronize()
        cap.graph.launch(s)
        s.synchronize()
        assert torch.equal(out, ref_out)
        assert int(total.item()) == tot
    cap.graph.close()
    b.close()


def test_batched_uneven_full_size_sampled(rm, dev, orc):
    """10^6 streams at k*2^64, lengths log-uniform [64, 65536] from seed 7, f32
    packed by prefix sum, one persistent launch; 48 streams checked."""
    from paper_2512_00093_gb300.workloads import BatchedUneven
    w = BatchedUneven()
    lens = w.lengths()
    n = w.n_streams
    base = rm.seed(w.seed).to(dev)
    states = rm.partition(base, w.J, 0, n)
    b = rm.Batch(n)
    desc, order, total = b.pack(torch.as_tensor(lens, device=dev))
    tot = int(total.item())
    assert tot == int(lens.sum())
    out = torch.empty(tot, dtype=torch.float32, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    b.generate_f32(states, desc, out, order=order, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    offs = np.concatenate([[0], np.cumsum(lens)[:-1]])
    rng = np.random.default_rng(8)
    rows = np.concatenate([[0, n - 1, int(np.argmax(lens)), int(np.argmin(lens))],
                           rng.choice(n, 44, replace=False)])
    for i in rows:
        i = int(i)
        ref = orc.stream(w.seed, i * w.J, int(lens[i]))
        g = out[int(offs[i]):int(offs[i] + lens[i])].cpu().numpy()
        assert np.array_equal(g, (ref.astype(np.float64) * F).astype(np.float32)), i
    del out
    b.close()


@pytest.mark.parametrize("seg", [64, 1000, 4096])
def test_split_pack_equals_unsplit_batch(rm, dev, orc, seg):
    """Splitting long streams (ranmar_batch_pack_split, the extra pieces'
    start states by the table jump by q seg, ranmar_batch_split_finish) gives
    the same outputs and the same advanced states as the unsplit batch, and
    the oracle's stream on sampled long streams.  Tolerance 0."""
    n = 3000
    c = counts_mix(n, 7)
    c[20:26] = [seg - 1, seg, seg + 1, 2 * seg, 2 * seg + 1, 65536]
    J = 1 << 64
    table = rm.Table()
    base = rm.seed(12345).to(dev)
    st0 = table.partition(base, J, 0, n)
    counts = torch.as_tensor(c, device=dev)
    total = int(c.sum())
    b = rm.Batch(n)
    desc, order, _ = b.pack(counts, flags=rm.DESC_WRITE_BACK)
    st_u = st0.clone()
    out_u = torch.full((total,), -1.0, dtype=torch.float32, device=dev)
    b.generate_f32(st_u, desc, out_u, order=order)
    n_extra = rm.Batch.split_extra(c, seg)
    assert n_extra == sum(max(0, -(-int(x) // seg) - 1) for x in c)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    sdesc, src, exps, tot = b.pack_split(counts, seg, n_extra, flags=rm.DESC_WRITE_BACK,
                                         status=status)
    st_s = torch.empty((n + n_extra, rm.STATE_WORDS), dtype=torch.int32, device=dev)
    st_s[:n] = st0
    if n_extra:
        table.jump(st_s[:n], exps, base_idx=src, out=st_s[n:], status=status)
    out_s = torch.full((total,), -1.0, dtype=torch.float32, device=dev)
    b.generate_f32(st_s, sdesc, out_s, status=status)
    rm.Batch.split_finish(st_s, n, src)
    torch.cuda.synchronize()
    assert int(status.item()) == 0 and int(tot.item()) == total
    d = sdesc.cpu().numpy().view(np.uint64)
    assert int(d[:, 2].max()) <= seg and int(d[:, 2].sum()) == total
    assert torch.equal(out_s.view(torch.int32), out_u.view(torch.int32))
    assert torch.equal(st_s[:n], st_u)
    offs = np.concatenate([[0], np.cumsum(c)[:-1]])
    got = out_s.cpu().numpy()
    for i in (20, 21, 22, 23, 24, 25, int(np.argmax(c))):
        ref = orc.stream(12345, i * J, int(c[i]))
        want = (ref.astype(np.float64) * F).astype(np.float32)
        assert np.array_equal(got[offs[i]: offs[i] + c[i]], want), i
    b.close()
    table.close()


def test_split_pack_wrong_extra_count_is_flagged(rm, dev):
    """n_extra that does not match the pieces sets RANMAR_ST_OUT_RANGE; the
    descriptors sized for missing pieces are empty ones."""
    c = np.array([10, 300, 5000, 64], dtype=np.int64)
    seg = 100
    n_extra = rm.Batch.split_extra(c, seg)          # 2 + 49 = 51
    counts = torch.as_tensor(c, device=dev)
    b = rm.Batch(4)
    for ne in (n_extra - 1, n_extra + 2):
        status = torch.zeros(1, dtype=torch.int32, device=dev)
        desc, src, exps, _ = b.pack_split(counts, seg, ne, status=status)
        torch.cuda.synchronize()
        assert int(status.item()) & rm.ST_OUT_RANGE
        if ne > n_extra:
            d = desc.cpu().numpy().view(np.uint64)
            assert np.all(d[4 + n_extra:, 2] == 0)
            assert np.all(src.cpu().numpy()[n_extra:].view(np.uint32) == 0xFFFFFFFF)
    b.close()


def test_split_pack_edge_shapes(rm, dev, orc):
    """n_extra = 0 (no stream longer than seg), every stream exactly seg,
    one stream of 65,536 outputs in pieces of 97, and no write-back: the
    split path still equals the unsplit batch (outputs; states untouched
    without write-back)."""
    J = 1 << 40
    table = rm.Table()
    base = rm.seed(54217138).to(dev)
    for c, seg, wb in [(np.array([5, 0, 64, 100]), 128, True),
                       (np.full(37, 256), 256, True),
                       (np.array([65536, 3]), 97, True),
                       (np.array([1000, 2000, 3000]), 512, False)]:
        n = len(c)
        flags = rm.DESC_WRITE_BACK if wb else 0
        counts = torch.as_tensor(c.astype(np.int64), device=dev)
        total = int(c.sum())
        st0 = table.partition(base, J, 11, n)
        b = rm.Batch(n)
        desc, order, _ = b.pack(counts, flags=flags)
        st_u = st0.clone()
        out_u = torch.full((total,), -1, dtype=torch.int32, device=dev)
        b.generate_u24(st_u, desc, out_u, order=order)
        n_extra = rm.Batch.split_extra(c, seg)
        status = torch.zeros(1, dtype=torch.int32, device=dev)
        sdesc, src, exps, _ = b.pack_split(counts, seg, n_extra, flags=flags, status=status)
        st_s = torch.empty((n + n_extra, rm.STATE_WORDS), dtype=torch.int32, device=dev)
        st_s[:n] = st0
        if n_extra:
            table.jump(st_s[:n], exps, base_idx=src, out=st_s[n:], status=status)
        out_s = torch.full((total,), -1, dtype=torch.int32, device=dev)
        b.generate_u24(st_s, sdesc, out_s, status=status)
        if wb:
            rm.Batch.split_finish(st_s, n, src)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert torch.equal(out_s, out_u), (c.tolist(), seg)
        assert torch.equal(st_s[:n], st_u if wb else st0), (c.tolist(), seg)
        i = int(np.argmax(c))
        offs = np.concatenate([[0], np.cumsum(c)[:-1]])
        ref = orc.stream(54217138, (11 + i) * J, int(c[i]))
        assert np.array_equal(out_s.cpu().numpy().view(np.uint32)[offs[i]: offs[i] + c[i]], ref)
        b.close()
    table.close()
