"""A cube past 2^32 voxels: 1100 x 1000 x 4000 (4.4e9 voxels, 17.6 GB in FP32),
ragged along every axis for 32 x 32 x 64 windows, the six-filter bank.

Voxel offsets pass 2^31 from x = 537 and 2^32 from x = 1074, so the sampled
windows lean towards the far end of the cube.  The oracle cannot take the
whole cube; each sampled window is checked on a block copied off the device:
the window plus one window of margin on each side (clipped at the cube's
faces).  The margin is wider than every filter radius (9 in x and y, 18 in
z), so inside the window the block's zero padding changes nothing, and the
window sits at a multiple of the window size inside the block, so the
oracle's window grid on the block puts the same window there.

FP32 storage: the parity bounds (1e-5 of max(std, |mean|) for the
statistics; masks bit-exact outside the guard band |c - T| < 1e-4 std).
FP16 storage (the tensor-core window kernel): the precision form's bounds
against the oracle on the FP16-rounded block.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

BANK6 = ((0.0, 2.0), (0.0, 6.0), (1.5, 2.0), (1.5, 6.0), (3.0, 2.0), (3.0, 6.0))
SHAPE = (1100, 1000, 4000)
WINDOW = (32, 32, 64)
K = 4.0


@pytest.fixture(scope="module")
def dev():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1507_04941_gb300 import build
    build.build()
    return torch.device("cuda", 0)


@pytest.fixture(scope="module")
def big_cube(dev):
    import torch
    from paper_1507_04941_gb300 import synth
    cube = synth.make_cube(SHAPE, 4242, 1500, (0.3, 5.0), 1.5, device=dev)
    torch.cuda.empty_cache()
    return cube


def _windows(grid):
    """The eight corners of the window grid, then windows past 2^31 and
    2^32 voxels (seeded)."""
    rng = np.random.default_rng(77)
    out = [(a, b, e) for a in (0, grid[0] - 1) for b in (0, grid[1] - 1) for e in (0, grid[2] - 1)]
    while len(out) < 20:
        a = int(rng.integers(grid[0] - 3, grid[0])) if len(out) < 16 else int(rng.integers(17, grid[0]))
        w = (a, int(rng.integers(0, grid[1])), int(rng.integers(0, grid[2])))
        if w not in out:
            out.append(w)
    return out


def _block(cube_d, widx):
    """The window's block (one window of margin, clipped) as float64 on the
    host, and the window's index on the block's own window grid."""
    lo, hi, sub = [], [], []
    for ax in range(3):
        w, n = WINDOW[ax], SHAPE[ax]
        o = widx[ax] * w
        b0 = max(0, o - w)
        lo.append(b0)
        hi.append(min(n, o + 2 * w))
        sub.append((o - b0) // w)
    blk = cube_d[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]].float().cpu().numpy().astype(np.float64)
    return blk, tuple(sub), tuple(lo)


def _run(dev, cube, storage):
    import torch
    from paper_1507_04941_gb300 import SourceFinder
    with SourceFinder(SHAPE, BANK6, 3.0, WINDOW, K, storage=storage, device=dev) as sf:
        grid = sf.grid
        mask, mean, std = sf.detect(cube, stats=True)
        torch.cuda.synchronize(dev)
        return grid, mask, mean.cpu().numpy(), std.cpu().numpy()


def test_past_2_32_voxels_f32(dev, oracle, big_cube):
    import torch
    from paper_1507_04941_gb300 import words_to_bits
    grid, mask, gm, gs = _run(dev, big_cube, "f32")
    total = 0
    for widx in _windows(grid):
        blk, sub, _ = _block(big_cube, widx)
        r = oracle.detect_window(blk, BANK6, 3.0, WINDOW, K, sub)
        x0, y0, z0 = (widx[i] * WINDOW[i] for i in range(3))
        ex, ey, ez = r["fire"].shape
        words = mask[x0:x0 + ex, y0:y0 + ey].cpu().numpy()
        got = words_to_bits(words, SHAPE[2])[:, :, z0:z0 + ez]
        want, sure = r["fire"].astype(bool), r["sure"].astype(bool)
        assert not ((got != want) & sure).any(), f"window {widx}: certain mask bits differ"
        a, b, e = widx
        scale = np.maximum(r["std"], np.abs(r["mean"]))
        assert (np.abs(gm[:, a, b, e] - r["mean"]) <= 1e-5 * scale).all(), f"window {widx} mean"
        assert (np.abs(gs[:, a, b, e] - r["std"]) <= 1e-5 * scale).all(), f"window {widx} std"
        total += int(want.sum())
    del mask
    torch.cuda.empty_cache()
    assert total > 0


def test_past_2_32_voxels_f16(dev, oracle, big_cube):
    """The tensor-core window kernel on the same cube stored in FP16."""
    import torch
    from paper_1507_04941_gb300 import words_to_bits
    cq = big_cube.to(torch.float16)
    grid, mask, gm, gs = _run(dev, cq, "f16")
    eps, floor = 2.0 ** -11, 1e-3
    total = n_dis = 0
    for widx in _windows(grid):
        blk, sub, lo = _block(cq, widx)
        r = oracle.detect_window(blk, BANK6, 3.0, WINDOW, K, sub)
        bx0, by0, bz0 = r["origin"]
        ex, ey, ez = r["fire"].shape
        box = ((bx0, bx0 + ex), (by0, by0 + ey), (bz0, bz0 + ez))
        unsure = np.zeros(r["fire"].shape, dtype=bool)
        sure_fire = np.zeros(r["fire"].shape, dtype=bool)
        a, b, e = widx
        for f, (sxy, sz) in enumerate(BANK6):
            A = oracle.filter_box(blk, sxy, sz, 3.0, box=box, take_abs=True)
            band = floor + (eps + 1e-5) * A + 1e-4 * r["std"][f]
            dlt = r["c"][f] - r["thr"][f]
            unsure |= np.abs(dlt) < band
            sure_fire |= dlt >= band
            sbound = floor + (eps + 1e-5) * A.max()
            assert abs(gm[f, a, b, e] - r["mean"][f]) <= sbound, f"window {widx} f{f} mean"
            assert abs(gs[f, a, b, e] - r["std"][f]) <= sbound, f"window {widx} f{f} std"
        x0, y0, z0 = (lo[i] + r["origin"][i] for i in range(3))
        words = mask[x0:x0 + ex, y0:y0 + ey].cpu().numpy()
        got = words_to_bits(words, SHAPE[2])[:, :, z0:z0 + ez]
        want = r["fire"].astype(bool)
        certain = sure_fire | ~unsure
        assert not ((got != want) & certain).any(), f"window {widx}: certain mask bits differ"
        n_dis += int((got != want).sum())
        total += int(want.sum())
    print(f"\n[f16 {SHAPE}] {total} oracle detections in the sampled windows, {n_dis} "
          f"differing bits, all inside the precision band")
    del mask, cq
    torch.cuda.empty_cache()
    assert total > 0
