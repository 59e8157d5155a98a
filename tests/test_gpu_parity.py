"""GPU parity of every step of the hot path against the FP64 oracle.

Tolerances (floating point, FP32 storage):
  filtered values  |gpu - ref| <= 1e-5 * max(|ref|, A),  A = the filter applied
                   to |d| (the scale of the rounding error of a sum of
                   products with positive taps);
  window stats     |d mean| <= 1e-5 * max(std, |mean|),
                   |d std|  <= 1e-5 * max(std, |mean|);
  masks            bit-exact wherever the oracle's decision is certain, i.e.
                   outside the guard band |c_f - T_f| < 1e-4 * std_f.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

BANK6 = ((0.0, 2.0), (0.0, 6.0), (1.5, 2.0), (1.5, 6.0), (3.0, 2.0), (3.0, 6.0))


@pytest.fixture(scope="module")
def dev():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1507_04941_gb300 import build
    build.build()
    return torch.device("cuda", 0)


def _cube(shape, seed, n_sources=8, peak=(1.0, 5.0), beam=None, device="cpu"):
    from paper_1507_04941_gb300 import synth
    return synth.make_cube(shape, seed, n_sources, peak, beam, device=device)


def _assert_filtered(gpu, ref, A, rel=1e-5, what=""):
    bound = rel * np.maximum(np.abs(ref), A)
    err = np.abs(gpu.astype(np.float64) - ref)
    bad = err > bound
    assert not bad.any(), (f"{what}: {int(bad.sum())} values outside tolerance, worst "
                           f"{float((err / np.maximum(bound, 1e-300)).max()):.3g} x bound")


def _assert_stats(gm, gs, rm, rs, rel=1e-5, what=""):
    scale = np.maximum(rs, np.abs(rm))
    dm = np.abs(gm.astype(np.float64) - rm)
    ds = np.abs(gs.astype(np.float64) - rs)
    assert (dm <= rel * scale).all(), f"{what}: mean off by {float((dm / scale).max()):.3g} x scale"
    assert (ds <= rel * scale).all(), f"{what}: std off by {float((ds / scale).max()):.3g} x scale"


def _assert_mask(got_bits, want_bits, sure_bits, what=""):
    """Bit-exact where the oracle's decision is certain; the differing bits
    inside the guard band are counted, printed and returned."""
    diff = (got_bits != want_bits) & sure_bits
    assert not diff.any(), f"{what}: {int(diff.sum())} certain mask bits differ"
    band = int((~sure_bits).sum())
    inside = int(((got_bits != want_bits) & ~sure_bits).sum())
    print(f"\n[{what}] guard band: {band} voxels, {inside} differing bits inside it")
    return inside


# --------------------------------------------------------------- taps ------
def test_taps_are_the_float32_rounded_oracle_taps(dev, oracle):
    from paper_1507_04941_gb300 import SourceFinder
    with SourceFinder((8, 8, 32), BANK6, 3.0, (8, 8, 32), device=dev) as sf:
        for f, (sxy, sz) in enumerate(BANK6):
            np.testing.assert_array_equal(sf.taps(f, 0), oracle.taps(sxy, 3.0).astype(np.float32))
            np.testing.assert_array_equal(sf.taps(f, 2), oracle.taps(sz, 3.0).astype(np.float32))


# ------------------------------------------------------------- filter ------
@pytest.mark.parametrize("shape", [(70, 45, 150), (33, 64, 128), (9, 7, 5)])
def test_filter_parity_every_bank_filter(dev, oracle, shape):
    from paper_1507_04941_gb300 import SourceFinder
    cube = _cube(shape, seed=21)
    d = cube.numpy()
    bank = BANK6 + ((1.0, 2.0),)
    with SourceFinder(shape, bank, 3.0, (32, 32, 64), device=dev) as sf:
        dc = cube.to(dev)
        for f, (sxy, sz) in enumerate(bank):
            got = sf.filter(dc, f).cpu().numpy()
            ref = oracle.filter_box(d, sxy, sz, 3.0)
            A = oracle.filter_box(d, sxy, sz, 3.0, take_abs=True)
            _assert_filtered(got, ref, A, what=f"filter {f} {shape}")


# -------------------------------------------------------------- stats ------
@pytest.mark.parametrize("stats_fp64", [False, True])
@pytest.mark.parametrize("window", [(32, 32, 64), (16, 16, 32), (7, 5, 13)])
def test_stats_parity(dev, oracle, window, stats_fp64):
    import torch
    from paper_1507_04941_gb300 import SourceFinder
    shape = (70, 45, 150)
    cube = _cube(shape, seed=22)
    with SourceFinder(shape, ((1.5, 2.0),), 3.0, window, device=dev, stats_fp64=stats_fp64) as sf:
        c = sf.filter(cube.to(dev), 0)
        # an offset makes the variance cancellation visible
        c += 3.0
        mean, std = sf.stats(c)
        torch.cuda.synchronize(dev)
        rm, rs = oracle.window_stats(c.cpu().numpy().astype(np.float64), window)
        _assert_stats(mean.cpu().numpy(), std.cpu().numpy(), rm, rs, what=f"window {window}")


# ---------------------------------------------------------- threshold ------
def test_threshold_parity(dev, oracle):
    from paper_1507_04941_gb300 import SourceFinder, words_to_bits
    shape = (40, 36, 100)
    window = (16, 16, 32)
    cube = _cube(shape, seed=23, n_sources=10, peak=(2.0, 6.0))
    with SourceFinder(shape, ((1.0, 2.0),), 3.0, window, k=3.0, device=dev) as sf:
        c = sf.filter(cube.to(dev), 0)
        mean, std = sf.stats(c)
        m = sf.threshold(c, mean, std)
        cn = c.cpu().numpy().astype(np.float64)
        want, amb = oracle.threshold(cn, window, mean.cpu().numpy(), std.cpu().numpy(), 3.0)
        got = words_to_bits(m.cpu().numpy(), shape[2])
        wb = oracle.unpack_bits(want, shape[2])
        sure = ~oracle.unpack_bits(amb, shape[2])
        assert wb.sum() > 0
        _assert_mask(got, wb, sure, "threshold")
        # accumulate ORs into an existing mask
        m2 = sf.threshold(c, mean, std, mask=m.clone().fill_(1), accumulate=True)
        g2 = words_to_bits(m2.cpu().numpy(), shape[2])
        assert g2[:, :, 0].all()


# ------------------------------------------------------------- detect ------
def _detect_vs_oracle(dev, oracle, shape, bank, window, k=4.0, seed=30, storage="f32",
                      cube=None, beam=None, stats_fp64=False, std_ddof=0):
    import torch
    from paper_1507_04941_gb300 import SourceFinder, words_to_bits
    if cube is None:
        cube = _cube(shape, seed=seed, n_sources=12, peak=(0.5, 5.0), beam=beam)
    with SourceFinder(shape, bank, 3.0, window, k=k, storage=storage, device=dev,
                      stats_fp64=stats_fp64, std_ddof=std_ddof) as sf:
        mask, mean, std = sf.detect(cube.to(dev), stats=True)
        torch.cuda.synchronize(dev)
        got = words_to_bits(mask.cpu().numpy(), shape[2])
        gm, gs = mean.cpu().numpy(), std.cpu().numpy()
    ref = oracle.detect(cube.numpy(), bank, 3.0, window, k, ddof=std_ddof)
    want = oracle.unpack_bits(ref["mask"], shape[2])
    sure = oracle.unpack_bits(ref["sure"], shape[2])
    _assert_mask(got, want, sure, f"detect {shape} {window}")
    _assert_stats(gm, gs, ref["mean"], ref["std"], what=f"detect stats {shape} {window}")
    # tail bits of every row are zero
    nz = shape[2]
    if nz % 32:
        words = mask.cpu().numpy().view(np.uint32)
        assert not (words[:, :, -1] >> np.uint32(nz % 32)).any()
    return want, got


def test_detect_tiny_workload(dev, oracle):
    from paper_1507_04941_gb300 import synth
    w = synth.TINY
    cube = synth.make(w)
    want, got = _detect_vs_oracle(dev, oracle, w.shape, w.bank, w.window, w.k, cube=cube)
    assert want.sum() > 0


@pytest.mark.parametrize("shape", [(72, 50, 200), (96, 64, 128), (40, 33, 70)])
def test_detect_bank6_ragged(dev, oracle, shape):
    _detect_vs_oracle(dev, oracle, shape, BANK6, (32, 32, 64), beam=1.5)


@pytest.mark.parametrize("shape,window", [((72, 50, 200), (32, 32, 64)), ((40, 33, 70), (16, 24, 48))])
def test_detect_stats_fp64(dev, oracle, shape, window):
    """FP64 combine of the window moments (fused kernel, and the composed
    path for the 16x24x48 windows): the same masks and statistics bounds."""
    _detect_vs_oracle(dev, oracle, shape, BANK6, window, beam=1.5, stats_fp64=True)


@pytest.mark.parametrize("shape,window", [((72, 50, 200), (32, 32, 64)), ((40, 33, 70), (8, 8, 8))])
def test_detect_sample_std(dev, oracle, shape, window):
    """std_ddof = 1 (squared deviations over n - 1) in the fused kernel and in
    the composed path (8x8x8 windows), against the oracle with ddof = 1."""
    _detect_vs_oracle(dev, oracle, shape, BANK6, window, beam=1.5, std_ddof=1)


def test_stats_sample_std(dev, oracle):
    import torch
    from paper_1507_04941_gb300 import SourceFinder
    shape, window = (70, 45, 150), (16, 16, 32)
    cube = _cube(shape, seed=24)
    with SourceFinder(shape, ((1.5, 2.0),), 3.0, window, device=dev, std_ddof=1) as sf:
        c = sf.filter(cube.to(dev), 0)
        mean, std = sf.stats(c)
        torch.cuda.synchronize(dev)
        rm, rs = oracle.window_stats(c.cpu().numpy().astype(np.float64), window, ddof=1)
        _assert_stats(mean.cpu().numpy(), std.cpu().numpy(), rm, rs, what="sample std")


@pytest.mark.parametrize("window", [(16, 24, 48), (8, 8, 8), (5, 7, 33)])
def test_detect_composed_path(dev, oracle, window):
    _detect_vs_oracle(dev, oracle, (40, 36, 100), ((0.0, 2.0), (1.0, 3.0)), window)


@pytest.mark.parametrize("shape,window", [((1, 1, 1), (8, 8, 32)), ((3, 5, 7), (16, 16, 32)),
                                          ((17, 9, 33), (16, 8, 32)), ((2, 40, 300), (2, 16, 64))])
def test_detect_edge_shapes(dev, oracle, shape, window):
    _detect_vs_oracle(dev, oracle, shape, ((0.0, 1.0), (1.0, 2.0)), window)


def test_detect_identity_filter_and_negative_k(dev, oracle):
    _detect_vs_oracle(dev, oracle, (32, 32, 64), ((0.0, 0.0),), (16, 16, 32), k=-0.5)


def test_detect_constant_cube_fires_nothing(dev):
    import torch
    from paper_1507_04941_gb300 import SourceFinder
    shape = (32, 32, 64)
    cube = torch.full(shape, 2.5, device=dev)
    with SourceFinder(shape, ((0.0, 2.0),), 3.0, (32, 32, 64), device=dev) as sf:
        # interior windows are constant: std 0, nothing fires; the edge roll-off is below mean
        mask, mean, std = sf.detect(cube, stats=True)
        assert int(mask.count_nonzero()) == 0


@pytest.mark.parametrize("shape,window", [((100, 40, 96), (16, 16, 32)), ((37, 33, 70), (8, 8, 32))])
def test_detect_host_pipelined_chunks(dev, shape, window):
    """sf_detect_host copies and computes in x chunks with an x halo."""
    import torch
    from paper_1507_04941_gb300 import SourceFinder
    cube = _cube(shape, seed=33, n_sources=10, peak=(2.0, 5.0))
    with SourceFinder(shape, BANK6, 3.0, window, device=dev) as sf:
        m_dev = sf.detect(cube.to(dev)).cpu()
        for _ in range(2):
            assert torch.equal(sf.detect_host(cube.pin_memory()), m_dev)


def test_detect_host_equals_device(dev):
    import torch
    from paper_1507_04941_gb300 import SourceFinder
    shape = (64, 48, 128)
    cube = _cube(shape, seed=31, n_sources=10, peak=(2.0, 5.0))
    with SourceFinder(shape, BANK6, 3.0, (32, 16, 64), device=dev) as sf:
        m_dev = sf.detect(cube.to(dev)).cpu()
        m_host = sf.detect_host(cube.pin_memory())
        assert torch.equal(m_dev, m_host)
        m_host2 = sf.detect_host(cube.contiguous())
        assert torch.equal(m_dev, m_host2)


def test_detect_repeatable_and_stream_ordered(dev):
    import torch
    from paper_1507_04941_gb300 import SourceFinder
    shape = (64, 64, 128)
    cube = _cube(shape, seed=32).to(dev)
    s = torch.cuda.Stream(dev)
    with SourceFinder(shape, BANK6, 3.0, (32, 32, 64), device=dev) as sf:
        a = sf.detect(cube, stats=True)
        with torch.cuda.stream(s):
            b = sf.detect(cube, stats=True)
        s.synchronize()
        for x, y in zip(a, b):
            assert torch.equal(x, y)


def test_invalid_calls_raise(dev):
    import torch
    from paper_1507_04941_gb300 import SfError, SourceFinder, lib
    shape = (16, 16, 32)
    with SourceFinder(shape, ((1.0, 2.0),), 3.0, (16, 16, 32), device=dev) as sf:
        cube = torch.zeros(shape, device=dev)
        with pytest.raises(ValueError):
            sf.detect(cube.double())
        with pytest.raises(SfError):
            sf.filter(cube, 5)
        mask = torch.zeros(sf.mask_shape, dtype=torch.int32, device=dev)
        # misaligned device pointer is rejected by the library
        buf = torch.zeros(shape[0] * shape[1] * shape[2] + 1, device=dev)
        st = lib().sf_detect(sf.handle, buf.data_ptr() + 4, mask.data_ptr(), None, None, None)
        assert st == 1


# ------------------------------------------------- full-size, sampled ------
def test_detect_tile_workload_sampled_windows(dev, oracle):
    """The 512x512x1024 six-filter workload in the bench's launch shape; the
    oracle recomputes a seeded sample of windows (corners included)."""
    import torch
    from paper_1507_04941_gb300 import SourceFinder, synth, words_to_bits
    w = synth.TILE
    cube_d = synth.make(w, device=dev)
    cube = cube_d.cpu().numpy()
    with SourceFinder(w.shape, w.bank, w.truncation, w.window, w.k, device=dev) as sf:
        mask, mean, std = sf.detect(cube_d, stats=True)
        torch.cuda.synchronize(dev)
        words = mask.cpu().numpy()
        gm, gs = mean.cpu().numpy(), std.cpu().numpy()
        grid = sf.grid
    rng = np.random.Generator(np.random.PCG64(5))
    sample = {(0, 0, 0), (grid[0] - 1, grid[1] - 1, grid[2] - 1), (0, grid[1] - 1, 7)}
    while len(sample) < 24:
        sample.add(tuple(int(rng.integers(0, g)) for g in grid))
    total = 0
    for widx in sorted(sample):
        r = oracle.detect_window(cube, w.bank, w.truncation, w.window, w.k, widx)
        x0, y0, z0 = r["origin"]
        ex, ey, ez = r["fire"].shape
        got = words_to_bits(words[x0:x0 + ex, y0:y0 + ey], w.shape[2])[:, :, z0:z0 + ez]
        _assert_mask(got, r["fire"].astype(bool), r["sure"].astype(bool), f"window {widx}")
        _assert_stats(gm[:, widx[0], widx[1], widx[2]], gs[:, widx[0], widx[1], widx[2]],
                      r["mean"], r["std"], what=f"window {widx}")
        total += int(r["fire"].sum())
    assert total > 0
