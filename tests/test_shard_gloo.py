"""Multi-rank host logic on CPU (gloo, world size 2): band shards cover the
batch exactly once; the bench's own split (Workload.coefficients with rank
and world, the call each torchrun rank makes) gives each rank a contiguous
slice of one global batch, bit for bit; a transform of each shard (here the
oracle: the library's kernels need a GPU) equals the same rows of the
transform of the global batch; and the step time reduces to the maximum over
ranks with the bench's max_over_ranks."""
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
    import bench
    import fftb_inputs as fi
    import oracle
    from paper_2406_05577_gb300.shard import band_shard, max_over_ranks
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = bench.Workload("sphere64_rt")  # 64 bands per rank, |G| <= 16 on 64^3
    g = oracle.sphere_gvectors(w.n, w.radius)
    mine = w.coefficients([g], rank, world)[0]                 # what this rank's bench transforms
    start, count = band_shard(world * w.bands[0], world, rank)
    assert count == w.bands[0]                                 # weak scaling: B bands per rank
    # the global batch, drawn here in one piece
    full = fi.complex_gaussian_bands(0, world * w.bands[0], len(g), w.seed) * \
        fi.gaussian_envelope(g, w.envelope)[None, :]
    same = bool(np.array_equal(mine, full[start:start + count]))
    # two bands of the shard through the transform, against the global batch's rows
    sel = [0, count - 1]
    got = oracle.g2r(g, mine[sel], w.n)
    want = oracle.g2r(g, full[[start + q for q in sel]], w.n)
    err = float(np.abs(got - want).max())
    step_ms = 1.0 + rank  # each rank's "step time"
    mx = max_over_ranks(step_ms)
    flags = torch.tensor([1.0 if same else 0.0, err])
    gathered = [torch.zeros_like(flags) for _ in range(world)] if rank == 0 else None
    dist.gather(flags, gathered, dst=0)  # test only: the bench's data path has no collective
    if rank == 0:
        ok = all(t[0].item() == 1.0 for t in gathered)
        worst = max(t[1].item() for t in gathered)
        with open(result_path, "w") as f:
            f.write(f"{int(ok)} {worst} {mx}\n")
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharded_transform(tmp_path):
    import torch.multiprocessing as mp
    out = tmp_path / "r.txt"
    mp.spawn(_rank_main, args=(2, _free_port(), str(out)), nprocs=2, join=True)
    ok, err, mx = map(float, out.read_text().split())
    assert ok == 1.0
    assert err == 0.0
    assert mx == 2.0
