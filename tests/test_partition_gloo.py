"""The x-slab sharding with halo exchange reproduces the whole-cube result.

Two gloo ranks on the CPU each take their slab, exchange x halos with
torch.distributed send/recv, filter their slab from the extended slab with the
FP64 oracle, form window statistics and thresholds on their own windows, and
OR the filters; the concatenated slab masks and statistics must equal the
oracle on the whole cube exactly.

The same two ranks, exchanging on the CPU, then run their extended slabs
through the library (sf_detect_slab) on one GPU: the concatenated slab masks
and window statistics must equal sf_detect on the whole cube bit for bit.
"""
import os

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

BANK = ((0.0, 2.0), (1.5, 2.0), (3.0, 4.0))
WINDOW = (16, 16, 32)
SHAPE = (70, 40, 64)


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    import oracle
    from paper_1507_04941_gb300 import partition, synth

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cube = synth.make_cube(SHAPE, seed=41, n_sources=10, peak=(1.0, 5.0))
        slabs = partition.plan_slabs(SHAPE[0], WINDOW[0], world)
        x0, x1 = slabs[rank]
        halo = partition.halo_width(BANK, 3.0)
        mine = cube[x0:x1].contiguous()
        left, right = partition.exchange_halo(mine, rank, world, halo)
        ext = partition.extended_slab(mine, left, right).numpy()
        n = x1 - x0
        fire = np.zeros((n,) + SHAPE[1:], dtype=bool)
        stats = []
        for sxy, sz in BANK:
            c = oracle.filter_box(ext, sxy, sz, 3.0, box=((halo, halo + n), (0, SHAPE[1]), (0, SHAPE[2])))
            mean, std = oracle.window_stats(c, WINDOW)
            m, _ = oracle.threshold(c, WINDOW, mean, std, 4.0)
            fire |= oracle.unpack_bits(m, SHAPE[2])
            stats.append(np.stack([mean, std]))
        np.save(os.path.join(out_dir, f"fire{rank}.npy"), fire)
        np.save(os.path.join(out_dir, f"stats{rank}.npy"), np.stack(stats))
    finally:
        dist.destroy_process_group()


def _rank_gpu(rank, world, port, out_dir, shape, bank, window):
    import torch
    import torch.distributed as dist

    from paper_1507_04941_gb300 import SourceFinder, partition, synth

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cube = synth.make_cube(shape, seed=43, n_sources=12, peak=(1.0, 5.0), beam_sigma=1.5)
        x0, x1 = partition.plan_slabs(shape[0], window[0], world)[rank]
        halo = partition.halo_width(bank, 3.0)
        mine = cube[x0:x1].contiguous()
        left, right = partition.exchange_halo(mine, rank, world, halo)
        ext = partition.extended_slab(mine, left, right)
        dev = torch.device("cuda", 0)
        with SourceFinder(tuple(ext.shape), bank, 3.0, window, 4.0, device=dev) as sf:
            mask, mean, std = sf.detect_slab(ext.to(dev), halo, stats=True)
            torch.cuda.synchronize(dev)
            np.save(os.path.join(out_dir, f"gmask{rank}.npy"), mask.cpu().numpy())
            np.save(os.path.join(out_dir, f"gmean{rank}.npy"), mean.cpu().numpy())
            np.save(os.path.join(out_dir, f"gstd{rank}.npy"), std.cpu().numpy())
    finally:
        dist.destroy_process_group()


@pytest.mark.gpu
@pytest.mark.parametrize("shape,window", [((200, 64, 256), (32, 32, 64)),    # slabs of 128 + 72
                                          ((70, 40, 100), (16, 16, 32)),     # ragged nz, tail window
                                          ((70, 40, 101), (16, 16, 32))])    # padded rows
def test_two_rank_slabs_through_the_library(tmp_path, shape, window):
    import socket

    import torch
    from paper_1507_04941_gb300 import SourceFinder, synth
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    bank = ((0.0, 2.0), (1.5, 2.0), (3.0, 6.0))
    world = 2
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_gpu, args=(r, world, port, str(tmp_path), shape, bank, window))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(600)
        assert p.exitcode == 0
    got = np.concatenate([np.load(tmp_path / f"gmask{r}.npy") for r in range(world)], axis=0)
    gmean = np.concatenate([np.load(tmp_path / f"gmean{r}.npy") for r in range(world)], axis=1)
    gstd = np.concatenate([np.load(tmp_path / f"gstd{r}.npy") for r in range(world)], axis=1)
    dev = torch.device("cuda", 0)
    cube = synth.make_cube(shape, seed=43, n_sources=12, peak=(1.0, 5.0), beam_sigma=1.5)
    with SourceFinder(shape, bank, 3.0, window, 4.0, device=dev) as sf:
        mask, mean, std = sf.detect(cube.to(dev), stats=True)
        torch.cuda.synchronize(dev)
        want = mask.cpu().numpy()
    assert want.any()
    np.testing.assert_array_equal(got, want)
    np.testing.assert_array_equal(gmean, mean.cpu().numpy())
    np.testing.assert_array_equal(gstd, std.cpu().numpy())


def test_plan_slabs_whole_windows():
    from paper_1507_04941_gb300 import partition
    s = partition.plan_slabs(70, 16, 2)
    assert s == [(0, 48), (48, 70)]
    assert partition.plan_slabs(512, 32, 4) == [(0, 128), (128, 256), (256, 384), (384, 512)]
    for x0, x1 in partition.plan_slabs(1000, 32, 3):
        assert x0 % 32 == 0
    assert partition.halo_width(BANK, 3.0) == 9


def test_two_rank_slabs_equal_whole_cube(tmp_path):
    import socket

    import oracle
    from paper_1507_04941_gb300 import synth
    world = 2
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    fire = np.concatenate([np.load(tmp_path / f"fire{r}.npy") for r in range(world)], axis=0)
    stats = np.concatenate([np.load(tmp_path / f"stats{r}.npy") for r in range(world)], axis=2)
    cube = synth.make_cube(SHAPE, seed=41, n_sources=10, peak=(1.0, 5.0)).numpy()
    ref = oracle.detect(cube, BANK, 3.0, WINDOW, 4.0)
    want = oracle.unpack_bits(ref["mask"], SHAPE[2])
    assert want.sum() > 0
    np.testing.assert_array_equal(fire, want)
    np.testing.assert_allclose(stats[:, 0], ref["mean"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(stats[:, 1], ref["std"], rtol=1e-12, atol=1e-14)


def _rank_inplace(rank, world, port, out_dir):
    import torch.distributed as dist

    from paper_1507_04941_gb300 import partition

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        halo, s = 3, 7
        ext = torch.zeros((s + 2 * halo, 4, 5))
        ext[halo:halo + s] = torch.arange(s, dtype=torch.float32)[:, None, None] + 100.0 * rank
        partition.exchange_halo_into(ext, halo, rank, world)
        np.save(os.path.join(out_dir, f"ext{rank}.npy"), ext.numpy())
    finally:
        dist.destroy_process_group()


def test_inplace_halo_exchange_three_ranks(tmp_path):
    """The bench's in-place exchange: each rank's halo planes are its
    neighbours' edge planes, zeros at the ends of the cube."""
    import socket
    world = 3
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_inplace, args=(r, world, port, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    halo, s = 3, 7
    ext = [np.load(tmp_path / f"ext{r}.npy") for r in range(world)]
    for r in range(world):
        own = ext[r][halo:halo + s, 0, 0]
        assert np.array_equal(own, np.arange(s) + 100.0 * r)
        left, right = ext[r][:halo, 0, 0], ext[r][halo + s:, 0, 0]
        want_l = np.arange(s - halo, s) + 100.0 * (r - 1) if r > 0 else np.zeros(halo)
        want_r = np.arange(halo) + 100.0 * (r + 1) if r < world - 1 else np.zeros(halo)
        assert np.array_equal(left, want_l), (r, left)
        assert np.array_equal(right, want_r), (r, right)
