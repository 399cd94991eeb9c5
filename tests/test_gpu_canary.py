"""Guard words around every output slice: streams of ragged lengths written
at unaligned offsets with gaps between them (the persistent kernel's
realigned stores, every group width and both interleaving modes, and the
one-warp-per-descriptor kernel), then every gap word must still hold its
sentinel and every slice must equal the oracle's stream."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

SENT = 0x5A5A5A5A
J = 10**6


@pytest.fixture(scope="module")
def rm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_00093_gb300 as rm
    return rm


@pytest.fixture(scope="module")
def layout():
    rng = np.random.default_rng(31)
    n = 300
    lens = rng.integers(0, 5000, n)
    lens[:12] = [0, 1, 31, 32, 33, 95, 96, 97, 127, 128, 129, 3 * 96 + 5]
    gaps = rng.integers(0, 41, n + 1)
    offs = np.zeros(n, np.int64)
    pos = int(gaps[0])
    for i in range(n):
        offs[i] = pos
        pos += int(lens[i]) + int(gaps[i + 1])
    return lens.astype(np.int64), offs, pos


@pytest.fixture(scope="module")
def reference(orc, layout):
    lens, _, _ = layout
    return [orc.stream(12345, i * J, int(c)) for i, c in enumerate(lens)]


def _check(out_words, lens, offs, total, ref, f32):
    mask = np.ones(total, bool)
    for i, (o, c) in enumerate(zip(offs, lens)):
        mask[o:o + c] = False
        got = out_words[o:o + c]
        want = ref[i]
        if f32:
            want = (want.astype(np.float64) / 16777216.0).astype(np.float32).view(np.uint32)
        assert np.array_equal(got, want), f"stream {i} (offset {o}, length {c})"
    gaps = out_words[mask]
    assert np.all(gaps == SENT), f"{int(np.sum(gaps != SENT))} guard words overwritten"


@pytest.mark.parametrize("f32", [False, True])
@pytest.mark.parametrize("cfg", [(32, 128, 0, 1), (32, 256, 0, 8), (16, 128, 0, 1),
                                 (16, 256, 0, 8), (8, 128, 0, 2), (4, 64, 0, 1), None])
def test_guard_words_and_slices(rm, layout, reference, cfg, f32):
    dev = torch.device("cuda:0")
    lens, offs, total = layout
    n = len(lens)
    states = rm.partition(rm.seed(12345).to(dev), J, 0, n)
    out = torch.full((total,), SENT, dtype=torch.int32, device=dev)
    desc = rm.make_desc(np.arange(n), offs, lens, 0, device=dev)
    outv = out.view(torch.float32) if f32 else out
    if cfg is None:
        (rm.generate_f32 if f32 else rm.generate_u24)(states, desc, outv)
    else:
        b = rm.Batch(n)
        b.config = cfg
        order = torch.as_tensor(np.argsort(-lens, kind="stable").astype(np.int32), device=dev)
        (b.generate_f32 if f32 else b.generate_u24)(states, desc, outv, order=order)
    torch.cuda.synchronize()
    _check(out.cpu().numpy().view(np.uint32), lens, offs, total, reference, f32)
