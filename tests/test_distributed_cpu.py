"""The multi-rank path on the CPU: two gloo ranks each integrate their shard of
a noisy ensemble (with the FP64 oracle standing in for the device kernels, since
this machine has no GPU) and combine the moments with
paper_1204_4255_gb300.distributed; the result must equal one process
integrating every path, because the noise counters carry the global path
index (path_offset)."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_covers_every_path_once():
    from paper_1204_4255_gb300.distributed import shard
    for total in (0, 1, 5, 64, 67):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                off, cnt = shard(total, r, world)
                seen.extend(range(off, off + cnt))
            assert seen == list(range(total))
    with pytest.raises(ValueError):
        shard(4, 2, 2)


def _workload():
    import workloads as W
    return W.truncated_wigner(npaths=7, n=64, nsteps=10, sample_every=5)


def _rank_main(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    from oracle import oracle as O
    from paper_1204_4255_gb300.distributed import combine_per_point, gather_per_path, shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = _workload()
        off, cnt = shard(w.npaths, rank, world)
        psi, pp, pq = O.run_workload(w, npaths=cnt, path0=off, threads=1)
        pq_t = combine_per_point(torch.from_numpy(pq), cnt, w.npaths)
        counts = [shard(w.npaths, r, world)[1] for r in range(world)]
        pp_t = gather_per_path(torch.from_numpy(pp), counts)
        psis = [None] * world
        dist.all_gather_object(psis, (off, psi))
        if rank == 0:
            full = np.concatenate([p for _, p in sorted(psis, key=lambda x: x[0])])
            np.savez(os.path.join(out_dir, "ranks.npz"), psi=full, pp=pp_t.numpy(), pq=pq_t.numpy())
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_single_process_ensemble(tmp_path):
    import torch.multiprocessing as mp
    from oracle import oracle as O
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    got = np.load(tmp_path / "ranks.npz")
    w = _workload()
    psi, pp, pq = O.run_workload(w, threads=1)
    assert np.array_equal(got["psi"], psi)
    assert np.array_equal(got["pp"], pp)
    np.testing.assert_allclose(got["pq"], pq, rtol=1e-13, atol=0)
