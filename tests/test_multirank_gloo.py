"""The N > 1 path on CPU: gloo ranks shard the partitioned workload by stream
index (weak scaling, no data-path collective) with the same per-step k-ranges
the benchmark uses (`shard.step_k0`), reduce the step time with
max-over-ranks, and each rank's boundary streams are the global streams its
ranges name (checked with the CPU oracle)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

SEED, J, M = 12345, 1 << 40, 16


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, n, steps, out_dir):
    import torch.distributed as dist
    from oracle import oracle
    from paper_2512_00093_gb300.shard import max_over_ranks, shard, step_k0
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    o = oracle()
    k0, cnt = shard(rank, world, n)
    ranges = []
    for i in range(steps):
        kf = step_k0(i, rank, world, n)
        # the first and last stream of this rank's batch i, as the rank computes them
        ranges.append((i, kf, o.stream(SEED, kf * J, M).tolist(),
                       o.stream(SEED, (kf + n - 1) * J, M).tolist()))
    slowest = max_over_ranks(1.0 + rank, dist)          # ranks report 1.0 and 2.0
    got = [None] * world
    dist.all_gather_object(got, (rank, k0, cnt, ranges, slowest))
    if rank == 0:
        np.save(os.path.join(out_dir, "gathered.npy"), np.array(got, dtype=object),
                allow_pickle=True)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_three_steps_tile_the_stream_indices(tmp_path, orc):
    world, n, steps = 2, 37, 3
    port = _free_port()
    mp.start_processes(_rank_main, args=(world, port, n, steps, str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    got = np.load(tmp_path / "gathered.npy", allow_pickle=True)
    covered = []
    for rank, k0, cnt, ranges, slowest in got:
        assert slowest == 2.0                            # max over ranks
        assert cnt == n and k0 == rank * n               # step 0 is the shard's block
        assert len(ranges) == steps
        for i, kf, first, last in ranges:
            covered.extend(range(kf, kf + n))
            # the rank's boundary streams are the global streams kf and kf + n - 1
            assert first == orc.stream(SEED, kf * J, M).tolist()
            assert last == orc.stream(SEED, (kf + n - 1) * J, M).tolist()
    # the (rank, step) ranges are disjoint and cover 0 .. world*steps*n - 1
    assert sorted(covered) == list(range(world * steps * n))


def test_step_k0_matches_the_block_order():
    from paper_2512_00093_gb300.shard import shard, step_k0
    world, n = 4, 10
    seen = [step_k0(i, r, world, n) for i in range(5) for r in range(world)]
    assert seen == [b * n for b in range(5 * world)]
    assert shard(3, world, n) == (30, n)


def test_shard_rejects_bad_rank():
    from paper_2512_00093_gb300.shard import shard, step_k0
    with pytest.raises(ValueError):
        shard(2, 2, 10)
    with pytest.raises(ValueError):
        step_k0(-1, 0, 2, 10)
