"""ranmar_check_overlap: the non-overlap condition of the partition (Sec. 1)
-- stream k owns the transitions [kJ, (k+1)J) -- flagged on the device for
descriptors whose generation would run past the end of their stream, and
compared with the same condition evaluated in exact Python integers."""
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


def _pos(rm, states):
    w = rm.state_words_np(states).astype(np.uint64)
    return [int(a) | (int(b) << 32) for a, b in zip(w[:, 98], w[:, 99])]


def _flag(rm, states, idx, counts, ks, J):
    dev = states.device
    desc = rm.make_desc(np.asarray(idx), np.zeros(len(idx), np.int64), np.asarray(counts), 0,
                        device=dev)
    k = torch.as_tensor(np.asarray(ks, dtype=np.int64), device=dev)
    st = rm.check_overlap(states, desc, k, J)
    torch.cuda.synchronize()
    return int(st.item())


@pytest.mark.parametrize("J", [10**6, 1 << 40, (1 << 64) + 5, (1 << 120) + 12345])
def test_overlap_flag_matches_exact_condition(rm, J):
    dev = torch.device("cuda:0")
    base = rm.seed(12345).to(dev)
    k0 = 3
    states = rm.partition(base, J, k0, 4)
    pos = _pos(rm, states)
    for i in range(4):
        assert pos[i] == ((k0 + i) * J) % (1 << 64)
    for i in range(4):
        k = k0 + i
        for count in [0, 1, 4096, min(J, 1 << 40)]:
            exact = (count > J)                      # from the stream start (off = 0)
            got = _flag(rm, states, [i], [count], [k], J)
            assert bool(got & rm.ST_OVERLAP) == exact, (J, i, count)
    if J < (1 << 64):
        assert _flag(rm, states, [0], [J + 1], [k0], J) == rm.ST_OVERLAP
        assert _flag(rm, states, [0], [J], [k0], J) == 0
        # the state belongs to stream k0, not k0 + 1: off wraps, flagged
        assert _flag(rm, states, [0], [1], [k0 + 1], J) == rm.ST_OVERLAP
    else:
        # offsets past 2^64 cannot be told apart from the state's pos mod 2^64:
        # only off + count > 2^64 is flagged
        assert _flag(rm, states, [0], [1 << 40], [k0], J) == 0


def test_overlap_after_resume(rm):
    """After generating J - 5 outputs of stream k with write-back, 5 more stay
    inside the stream and 6 do not."""
    dev = torch.device("cuda:0")
    J = 10**6
    base = rm.seed(77).to(dev)
    states = rm.partition(base, J, 9, 2)
    out = torch.empty(J, dtype=torch.int32, device=dev)
    desc = rm.make_desc(np.array([0]), np.array([0]), J - 5, rm.DESC_WRITE_BACK, device=dev)
    rm.generate_u24(states, desc, out)
    torch.cuda.synchronize()
    assert _pos(rm, states)[0] == 9 * J + J - 5
    assert _flag(rm, states, [0], [5], [9], J) == 0
    assert _flag(rm, states, [0], [6], [9], J) == rm.ST_OVERLAP
    # a batch: only the offending descriptor sets the bit, the call refuses nothing
    assert _flag(rm, states, [0, 1, 1], [5, J, 3], [9, 10, 10], J) == 0
    assert _flag(rm, states, [0, 1, 1], [5, J + 1, 3], [9, 10, 10], J) == rm.ST_OVERLAP


def test_overlap_host_and_device_checks(rm):
    dev = torch.device("cuda:0")
    states = rm.partition(rm.seed(5).to(dev), 1000, 0, 2)
    assert _flag(rm, states, [2], [1], [0], 1000) == rm.ST_BAD_INDEX
    desc = rm.make_desc(np.array([0]), np.array([0]), 1, 0, device=dev)
    k = torch.zeros(1, dtype=torch.int64, device=dev)
    with pytest.raises(rm.RanmarError):
        rm.check_overlap(states, desc, k, 0)          # J = 0
    with pytest.raises(rm.RanmarError):
        rm.check_overlap(states, desc, k, 1 << 170)   # more than 5 words
