"""Algorithm 1 (floating-point form) on the GPU: bit-exact against the
oracle's Algorithm 1 in double, and equal to the integer path's f32 outputs
(every value is a multiple of 2^-24).  Tolerance 0."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

RAGGED = [0, 1, 31, 32, 33, 95, 96, 97, 98, 1000, 1013, 4096, 5000]


@pytest.fixture(scope="module")
def rm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_00093_gb300 as rm
    return rm


@pytest.mark.parametrize("dt", ["f32", "f64"])
def test_alg1_matches_oracle_alg1(rm, orc, dt):
    dev = torch.device("cuda:0")
    n = len(RAGGED)
    exps = [(i * 104729) << 30 for i in range(n)]
    states = rm.jump(rm.seed(2718).to(dev), rm.exps_tensor(exps, 2, device=dev))
    ref_states = states.clone()
    offs = np.concatenate([[0], np.cumsum(RAGGED)[:-1]])
    total = int(sum(RAGGED))
    desc = rm.make_desc(np.arange(n), offs, RAGGED, rm.DESC_WRITE_BACK, device=dev)
    torch_dt = torch.float32 if dt == "f32" else torch.float64
    out = torch.full((total,), -1.0, dtype=torch_dt, device=dev)
    (rm.generate_alg1_f32 if dt == "f32" else rm.generate_alg1_f64)(states, desc, out)
    outi = torch.empty(total, dtype=torch.float32, device=dev)
    rm.generate_f32(ref_states, desc, outi)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert torch.equal(states, ref_states), "write-back must equal the integer path's"
    assert np.array_equal(got.astype(np.float32), outi.cpu().numpy())
    x0, c0 = orc.seeded_state(2718)
    for i, cnt in enumerate(RAGGED):
        xs, cs = orc.jump(x0, c0, exps[i])
        ref = orc.generate_alg1(xs, cs, cnt)                   # double, Algorithm 1
        g = got[offs[i]:offs[i] + cnt]
        if dt == "f64":
            assert np.array_equal(g, ref), cnt
        else:
            assert np.array_equal(g, ref.astype(np.float32)), cnt
