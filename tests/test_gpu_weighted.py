"""GPU parity of the weighted convolution (Eq. 1) against the FP64 oracle,
for both readings of the denominator (sum f w, and sum w as printed).

Tolerances as for the unweighted path:
  filtered values  |gpu - ref| <= 1e-5 * max(|ref|, A),  A = Eq. 1 applied to
                   |d| (the scale of the rounding error of the numerator);
  window stats     |d mean|, |d std| <= 1e-5 * max(std, |mean|);
  masks            bit-exact outside the guard band |c_f - T_f| < 1e-4 * std_f.
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


def _inputs(shape, seed):
    from paper_1507_04941_gb300 import synth
    d = synth.make_cube(shape, seed, 10, (1.0, 6.0), None)
    w = synth.make_weights(shape, seed, n_flagged=2, flag_width=(3, 9))
    return d, w


def _assert_filtered(gpu, ref, A, rel=1e-5, what=""):
    bound = rel * np.maximum(np.abs(ref), A)
    err = np.abs(gpu.astype(np.float64) - ref)
    bad = err > bound
    assert not bad.any(), (f"{what}: {int(bad.sum())} values outside tolerance, worst "
                           f"{float((err / np.maximum(bound, 1e-300)).max()):.3g} x bound")


@pytest.mark.parametrize("den", ["fw", "w"])
@pytest.mark.parametrize("shape", [(40, 36, 100), (9, 7, 5)])
def test_weighted_filter_parity(dev, oracle, den, shape):
    from paper_1507_04941_gb300 import SourceFinder
    d, w = _inputs(shape, 51)
    dn, wn = d.numpy(), w.numpy()
    with SourceFinder(shape, BANK6, 3.0, (16, 16, 32), device=dev) as sf:
        dd, wd = d.to(dev), w.to(dev)
        for f, (sxy, sz) in enumerate(BANK6):
            got = sf.weighted_filter(dd, wd, f, den).cpu().numpy()
            ref = oracle.weighted_filter_box(dn, wn, sxy, sz, 3.0, den)
            A = oracle.weighted_filter_box(np.abs(dn), wn, sxy, sz, 3.0, den)
            _assert_filtered(got, ref, A, what=f"filter {f} den={den} {shape}")
            # no weight in the support: exactly 0
            assert np.all(got[ref == 0.0] == 0.0)


def test_unit_weights_reduce_to_eq2(dev):
    import torch
    from paper_1507_04941_gb300 import SourceFinder
    shape = (30, 28, 90)
    d, _ = _inputs(shape, 52)
    with SourceFinder(shape, BANK6, 3.0, (16, 16, 32), device=dev) as sf:
        dd = d.to(dev)
        ones = torch.ones_like(dd)
        for f, (sxy, sz) in enumerate(BANK6):
            a = sf.weighted_filter(dd, ones, f, "fw").cpu().numpy()
            b = sf.filter(dd, f).cpu().numpy()
            rx, rz = int(np.ceil(3 * sxy)), int(np.ceil(3 * sz))
            inner = (slice(rx, shape[0] - rx), slice(rx, shape[1] - rx), slice(rz, shape[2] - rz))
            np.testing.assert_allclose(a[inner], b[inner], rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("den", ["fw", "w"])
def test_weighted_detect_parity(dev, oracle, den):
    import torch
    from paper_1507_04941_gb300 import SourceFinder, words_to_bits
    shape, window, k = (40, 36, 100), (16, 16, 32), 3.0
    d, w = _inputs(shape, 53)
    with SourceFinder(shape, BANK6, 3.0, window, k=k, device=dev) as sf:
        mask, mean, std = sf.weighted_detect(d.to(dev), w.to(dev), den, stats=True)
        torch.cuda.synchronize(dev)
        got = words_to_bits(mask.cpu().numpy(), shape[2])
        gm, gs = mean.cpu().numpy(), std.cpu().numpy()
    ref = oracle.weighted_detect(d.numpy(), w.numpy(), BANK6, 3.0, window, k, den)
    want = oracle.unpack_bits(ref["mask"], shape[2])
    sure = oracle.unpack_bits(ref["sure"], shape[2])
    assert want.sum() > 0
    diff = (got != want) & sure
    assert not diff.any(), f"{int(diff.sum())} certain mask bits differ"
    scale = np.maximum(ref["std"], np.abs(ref["mean"]))
    assert (np.abs(gm - ref["mean"]) <= 1e-5 * scale).all()
    assert (np.abs(gs - ref["std"]) <= 1e-5 * scale).all()


@pytest.mark.parametrize("opts", [dict(std_ddof=1), dict(stats_fp64=True)])
def test_weighted_detect_statistics_options(dev, oracle, opts):
    """The statistics options in the fused pair kernel (sample std against the
    oracle with ddof = 1; the FP64 combine against the population oracle)."""
    import torch
    from paper_1507_04941_gb300 import SourceFinder, words_to_bits
    shape, window, k = (40, 36, 100), (16, 16, 32), 3.0
    d, w = _inputs(shape, 56)
    with SourceFinder(shape, BANK6, 3.0, window, k=k, device=dev, **opts) as sf:
        mask, mean, std = sf.weighted_detect(d.to(dev), w.to(dev), "fw", stats=True)
        torch.cuda.synchronize(dev)
        got = words_to_bits(mask.cpu().numpy(), shape[2])
        gm, gs = mean.cpu().numpy(), std.cpu().numpy()
    ref = oracle.weighted_detect(d.numpy(), w.numpy(), BANK6, 3.0, window, k, "fw",
                                 ddof=opts.get("std_ddof", 0))
    want = oracle.unpack_bits(ref["mask"], shape[2])
    sure = oracle.unpack_bits(ref["sure"], shape[2])
    diff = (got != want) & sure
    assert not diff.any(), f"{opts}: {int(diff.sum())} certain mask bits differ"
    scale = np.maximum(ref["std"], np.abs(ref["mean"]))
    assert (np.abs(gm - ref["mean"]) <= 1e-5 * scale).all()
    assert (np.abs(gs - ref["std"]) <= 1e-5 * scale).all()


def test_weighted_full_tile_sampled(dev, oracle):
    """The tile workload's cube with its weights at full size: Eq. 1 of two
    bank filters at sampled voxels (some in flagged channels) against the
    oracle evaluated on those voxels alone."""
    import torch
    from paper_1507_04941_gb300 import SourceFinder, synth
    wk = synth.TILE
    d = synth.make(wk, device=dev)
    w = synth.make_weights(wk.shape, wk.seed, device=dev)
    dn, wn = d.cpu().numpy(), w.cpu().numpy()
    rng = np.random.default_rng(54)
    vox = np.stack([rng.integers(0, n, size=40) for n in wk.shape], axis=1)
    flagged = np.where(wn[0, 0, :] == 0.0)[0]
    vox[:5, 2] = flagged[:5]
    with SourceFinder(wk.shape, wk.bank, wk.truncation, wk.window, wk.k, device=dev) as sf:
        for f in (1, 5):
            for den in ("fw", "w"):
                got = sf.weighted_filter(d, w, f, den)
                torch.cuda.synchronize(dev)
                g = got.cpu().numpy()
                sxy, sz = wk.bank[f]
                for x, y, z in vox:
                    box = ((x, x + 1), (y, y + 1), (z, z + 1))
                    ref = oracle.weighted_filter_box(dn, wn, sxy, sz, wk.truncation, den, box)[0, 0, 0]
                    A = oracle.weighted_filter_box(np.abs(dn), wn, sxy, sz, wk.truncation, den, box)[0, 0, 0]
                    assert abs(g[x, y, z] - ref) <= 1e-5 * max(abs(ref), A), (f, den, x, y, z)


@pytest.mark.parametrize("composed,shape", [(True, (40, 36, 100)), (False, (24, 32, 70))])
def test_weighted_detect_paths(dev, oracle, monkeypatch, composed, shape):
    """The composed path (forced) and the fused kernel's cp.async slabs
    (nz % 4 != 0) against the oracle."""
    import torch
    from paper_1507_04941_gb300 import SourceFinder, words_to_bits
    if composed:
        monkeypatch.setenv("SF_WCOMPOSED", "1")
    window, k = (16, 16, 32), 3.0
    d, w = _inputs(shape, 55)
    for den in ("fw", "w"):
        with SourceFinder(shape, BANK6, 3.0, window, k=k, device=dev) as sf:
            mask, mean, std = sf.weighted_detect(d.to(dev), w.to(dev), den, stats=True)
            torch.cuda.synchronize(dev)
            got = words_to_bits(mask.cpu().numpy(), shape[2])
            gm, gs = mean.cpu().numpy(), std.cpu().numpy()
        ref = oracle.weighted_detect(d.numpy(), w.numpy(), BANK6, 3.0, window, k, den)
        want = oracle.unpack_bits(ref["mask"], shape[2])
        sure = oracle.unpack_bits(ref["sure"], shape[2])
        diff = (got != want) & sure
        assert not diff.any(), f"den={den}: {int(diff.sum())} certain mask bits differ"
        scale = np.maximum(ref["std"], np.abs(ref["mean"]))
        assert (np.abs(gm - ref["mean"]) <= 1e-5 * scale).all(), den
        assert (np.abs(gs - ref["std"]) <= 1e-5 * scale).all(), den
