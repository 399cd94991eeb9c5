"""The binding refuses buffers shorter than a call needs, before any launch:
the C ABI receives only pointers and sizes it is told, so a short output or
index tensor passed through would be read or written past its end."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_00093_gb300 as rm
    return rm


def test_short_buffers_are_refused(rm):
    dev = torch.device("cuda:0")
    W = rm.STATE_WORDS
    base = rm.seed(12345).to(dev)
    i32 = lambda *shape: torch.zeros(shape, dtype=torch.int32, device=dev)   # noqa: E731
    exps = rm.exps_tensor([5, 6, 7, 8], 2, device=dev)
    table = rm.Table()
    cases = [
        lambda: rm.seed_batch(torch.tensor([1, 2, 3], dtype=torch.int32, device=dev), out=i32(2, W)),
        lambda: rm.jump(base, exps, out=i32(3, W)),
        lambda: rm.jump(base, exps, base_idx=i32(3), out=i32(4, W)),
        lambda: rm.jump(base, exps, out=i32(4, W), status=i32(0)),
        lambda: rm.jump_scatter(base, exps, i32(8, W), i32(3)),
        lambda: rm.jump_scatter(base, exps, i32(8, W), i32(8), n=5),
        lambda: rm.partition(base, 1 << 40, 0, 4, out=i32(3, W)),
        lambda: rm.partition_ex(base, 1 << 40, 0, 4, out=i32(3, W)),
        lambda: table.partition(base, 1 << 40, 0, 4, out=i32(3, W)),
        lambda: table.jump(base, exps, out=i32(3, W)),
        lambda: table.jump(base, exps, base_idx=i32(2), out=i32(4, W)),
        lambda: rm.poly_power(exps, out=i32(3, W)),
        lambda: rm.lfg_generate(97, 33, 24, i32(2, 97), 64, out=i32(2, 63)),
        lambda: rm.check_overlap(i32(4, W), rm.make_desc(np.arange(4), np.arange(4) * 8, 8,
                                                         device=dev),
                                 torch.zeros(3, dtype=torch.int64, device=dev), 1 << 40),
        lambda: rm.Batch.split_finish(i32(4, W), 3, i32(2)),
    ]
    for i, fn in enumerate(cases):
        with pytest.raises(ValueError):
            fn()
    torch.cuda.synchronize()
    # the same calls with buffers of the right size go through
    out = rm.jump(base, exps, out=i32(4, W))
    torch.cuda.synchronize()
    assert out.abs().sum().item() > 0
