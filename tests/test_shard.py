"""Multi-GPU partition and reduction, tested on CPU with two gloo ranks.

The ranks shoot their ray ranges with the FP64 oracle (no GPU here) and sum
the integer maps with torch.distributed; the result must equal the one-rank
map bit for bit.
"""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2308_14278_gb300 import inputs, shard


def test_ray_ranges_cover_and_align():
    for n3x, n3y, n1y, world in [(100, 1000, 120, 2), (100, 1000, 120, 3), (7, 44281, 400, 8),
                                 (50, 70, 400, 4), (3, 5, 2, 8)]:
        rr = shard.ray_ranges(n3x, n3y, n1y, world)
        assert len(rr) == world
        assert rr[0][0] == 0 and rr[-1][1] == n3x * n3y
        for (a, b), (c, d) in zip(rr[:-1], rr[1:]):
            assert b == c and a <= b
        unit = n1y if (n3y + n1y - 1) // n1y >= world else 32
        for a, b in rr:
            assert a % n3x == 0
            assert (a // n3x) % unit == 0 or a == n3x * n3y
        sizes = [b - a for a, b in rr]
        assert max(sizes) - min(sizes) <= unit * n3x


def test_maps_for_rank_partition():
    rays = [int(v) for v in np.random.default_rng(0).integers(10**9, 10**10, 80)]
    world = 4
    parts = [shard.maps_for_rank(rays, r, world) for r in range(world)]
    assert sorted(i for p in parts for i in p) == list(range(80))
    loads = [sum(rays[i] for i in p) for p in parts]
    assert max(loads) - min(loads) <= max(rays)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_path):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = inputs.small_map(0)
    g = oracle.geometry_of(w)
    a, b = shard.ray_ranges(g.n3x, g.n3y, g.n1y, world)[rank]
    counts, stats = oracle.shoot_direct(g, w.lenses.x, w.lenses.y, w.lenses.m, a, b, threads=2)
    t = torch.from_numpy(counts.astype(np.int64))
    shard.reduce_counts(t, dst=0)            # the summed map is needed on rank 0 only
    st = torch.tensor([int(v) for v in stats], dtype=torch.int64)
    dist.all_reduce(st)
    if rank == 0:
        np.save(out_path, np.concatenate([t.numpy().ravel(), st.numpy()]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_one_rank_map(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    w = inputs.small_map(0)
    g = oracle.geometry_of(w)
    ref, stats = oracle.shoot_direct(g, w.lenses.x, w.lenses.y, w.lenses.m, 0, g.n_rays, threads=2)
    out = str(tmp_path / "sum.npy")
    mp.spawn(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True)
    got = np.load(out)
    n = g.mnx * g.mny
    assert np.array_equal(got[:n].reshape(g.mny, g.mnx), ref.astype(np.int64))
    assert list(got[n:]) == [int(v) for v in stats]


def _wrap_main(rank, world, port, out_path):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # uint32 counts near 2^32 travel as their int32 bit patterns
    u = np.array([4294967000, 7, 2147483647, 2147483648], np.uint32) + np.uint32(rank)
    t = torch.from_numpy(u.view(np.int32).copy())
    shard.reduce_counts(t, dst=0)
    if rank == 0:
        np.save(out_path, t.numpy().view(np.uint32))
    dist.barrier()
    dist.destroy_process_group()


def test_int32_transport_of_uint32_counts_sums_modulo_2_32(tmp_path):
    """The counts' int32 bit patterns sum to the uint32 sum's bits, wrapped
    modulo 2^32 like the one-GPU map would be."""
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    out = str(tmp_path / "wrap.npy")
    mp.spawn(_wrap_main, args=(2, _free_port(), out), nprocs=2, join=True)
    got = np.load(out)
    a = np.array([4294967000, 7, 2147483647, 2147483648], np.uint64)
    want = ((a + a + 1) % (1 << 32)).astype(np.uint32)
    assert np.array_equal(got, want)


@pytest.mark.gpu
def test_sharded_map_equals_the_one_gpu_map(ml):
    """The sharded path on one GPU: two fields shoot the two ranks' ray
    ranges, their count maps are summed and set into a third field, whose
    counts, mu and light curves must equal the map shot whole, bit for bit."""
    import torch
    w = inputs.paper_map(0, n_rays=2e9, map_px=1024)
    whole = ml.Field(w, precision=ml.PREC_MIXED)
    whole.shoot()
    info = whole.info
    parts = []
    for a, b in shard.ray_ranges(info["n_rays_x"], info["n_rays_y"], info["n1y"], 2):
        f = ml.Field(w, precision=ml.PREC_MIXED)
        f.shoot(a, b)
        parts.append(f)
    total = parts[0].counts() + parts[1].counts()
    ml.ml_field_set_counts(parts[0].h, total)
    assert torch.equal(parts[0].counts(), whole.counts())
    assert torch.equal(parts[0].mu("f32"), whole.mu("f32"))
    tracks = inputs.tracks(4, 1024, 1024, 3.0, seed=1)
    assert torch.equal(parts[0].light_curves(tracks, 256, 0.5), whole.light_curves(tracks, 256, 0.5))
    for f in parts + [whole]:
        f.close()


def _batch_rank_main(rank, world, port, out_path):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws = inputs.batched_maps(n_maps=12, seed=0, map_px=64, ray_range=(1e5, 1e6), tracks_per_map=1)
    mine = shard.maps_for_rank([w.n_av * w.map_n[0] * w.map_n[1] for w in ws], rank, world)
    rays = sum(oracle.geometry_of(ws[i]).n_rays for i in mine)
    r = torch.tensor([rays], dtype=torch.int64)
    dist.all_reduce(r)
    owner = torch.zeros(len(ws), dtype=torch.int64)
    owner[mine] = 1
    dist.all_reduce(owner)
    if rank == 0:
        np.save(out_path, np.concatenate([r.numpy(), owner.numpy()]))
    dist.barrier()
    dist.destroy_process_group()


def test_three_gloo_ranks_split_a_batch_by_whole_maps(tmp_path):
    """The batched workload split over ranks as the bench's --shard does it:
    every map is shot by exactly one rank, and the ranks' summed ray counts are
    the whole batch's."""
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ws = inputs.batched_maps(n_maps=12, seed=0, map_px=64, ray_range=(1e5, 1e6), tracks_per_map=1)
    total = sum(oracle.geometry_of(w).n_rays for w in ws)
    out = str(tmp_path / "batch.npy")
    mp.spawn(_batch_rank_main, args=(3, _free_port(), out), nprocs=3, join=True)
    got = np.load(out)
    assert int(got[0]) == total
    assert list(got[1:]) == [1] * len(ws)
