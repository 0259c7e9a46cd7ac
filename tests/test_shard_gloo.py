"""Multi-rank host logic on CPU (gloo, world size 2): band shards cover the
batch exactly once, a sharded transform (here the oracle, standing in for
each rank's plan) equals the unsharded one, and the step time reduces to the
maximum over ranks."""
import os
import socket

import numpy as np
import pytest

from paper_2406_05577_gb300.shard import band_shard


def test_band_shard_covers_batch():
    for total in (0, 1, 7, 64, 535):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                s, c = band_shard(total, world, r)
                seen.extend(range(s, s + c))
            assert seen == list(range(total))
            sizes = [band_shard(total, world, r)[1] for r in range(world)]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        band_shard(4, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, result_path):
    import torch
    import torch.distributed as dist
    import fftb_inputs as fi
    import oracle
    from paper_2406_05577_gb300.shard import band_shard, max_over_ranks
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n, r, total = (12, 10, 9), 2.5, 7
    g = oracle.sphere_gvectors(n, r)
    c = fi.complex_gaussian((total, len(g)), 5)          # the global batch
    start, count = band_shard(total, world, rank)
    mine = oracle.g2r(g, c[start:start + count], n).reshape(count, -1)
    # gather the shards on rank 0 (test only: the transform path has no collective)
    sizes = [band_shard(total, world, q)[1] for q in range(world)]
    pad = np.zeros((max(sizes), mine.shape[1]), np.complex128)
    pad[:count] = mine
    t = torch.from_numpy(np.stack([pad.real, pad.imag]))
    gathered = [torch.zeros_like(t) for _ in range(world)] if rank == 0 else None
    dist.gather(t, gathered, dst=0)
    step_ms = 1.0 + rank  # each rank's "step time"
    mx = max_over_ranks(step_ms)
    if rank == 0:
        parts = [(gt[0] + 1j * gt[1]).numpy()[:sizes[q]] for q, gt in enumerate(gathered)]
        full = oracle.g2r(g, c, n).reshape(total, -1)
        err = np.abs(np.concatenate(parts) - full).max()
        with open(result_path, "w") as f:
            f.write(f"{err} {mx}\n")
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharded_transform(tmp_path):
    import torch.multiprocessing as mp
    out = tmp_path / "r.txt"
    mp.spawn(_rank_main, args=(2, _free_port(), str(out)), nprocs=2, join=True)
    err, mx = map(float, out.read_text().split())
    assert err < 1e-12
    assert mx == 2.0
