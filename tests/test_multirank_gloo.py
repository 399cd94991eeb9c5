"""The N > 1 path on CPU: two gloo ranks shard the partitioned workload by
stream index (weak scaling, no data-path collective), reduce the step time
with max-over-ranks, and each rank's first stream is the global stream the
shard names (checked with the CPU oracle)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, n, out_dir):
    import torch
    import torch.distributed as dist
    from oracle import oracle
    from paper_2512_00093_gb300.shard import max_over_ranks, shard
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    k0, cnt = shard(rank, world, n)
    o = oracle()
    J, seed, m = 1 << 40, 12345, 16
    first = o.stream(seed, k0 * J, m)
    last = o.stream(seed, (k0 + cnt - 1) * J, m)
    slowest = max_over_ranks(1.0 + rank, dist)          # ranks report 1.0 and 2.0
    got = [None] * world
    dist.all_gather_object(got, (k0, cnt, first.tolist(), last.tolist(), slowest))
    if rank == 0:
        np.save(os.path.join(out_dir, "gathered.npy"), np.array(got, dtype=object),
                allow_pickle=True)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_by_stream_index(tmp_path, orc):
    world, n = 2, 37
    port = _free_port()
    mp.start_processes(_rank_main, args=(world, port, n, str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    got = np.load(tmp_path / "gathered.npy", allow_pickle=True)
    (k0a, na, fa, la, sa), (k0b, nb, fb, lb, sb) = got
    assert (k0a, na, k0b, nb) == (0, n, n, n)            # disjoint, contiguous
    assert sa == sb == 2.0                               # max over ranks
    J = 1 << 40
    # rank 1's first stream is global stream n; rank 0's last is n - 1
    assert fb == orc.stream(12345, n * J, 16).tolist()
    assert la == orc.stream(12345, (n - 1) * J, 16).tolist()
    assert fa == orc.stream(12345, 0, 16).tolist()


def test_shard_rejects_bad_rank():
    from paper_2512_00093_gb300.shard import shard
    with pytest.raises(ValueError):
        shard(2, 2, 10)
