"""Pins of the oracle's per-voxel local statistics (Sec. 3.3 read as a box of
half-widths (sx, sy, sz) around each voxel, clipped to the cube) against
values fixed independently of it: numpy slices of the same box, closed forms
(constant fields, a box covering the whole cube, linear ramps, zero
half-widths, the clipped count at a corner), and the sampled path of
local_detect against its whole-cube path."""
import math

import numpy as np
import pytest
import scipy.ndimage as ndi


@pytest.fixture(scope="module")
def rng():
    return np.random.default_rng(20260)


@pytest.mark.parametrize("shape,half", [((6, 7, 9), (1, 2, 3)), ((5, 4, 11), (2, 0, 4)),
                                        ((3, 8, 5), (0, 3, 1))])
def test_brute_force_every_voxel(oracle, rng, shape, half):
    c = rng.normal(size=shape) * 3.0 + 1.5
    m, s = oracle.local_stats(c, half)
    sx, sy, sz = half
    nx, ny, nz = shape
    for x in range(nx):
        for y in range(ny):
            for z in range(nz):
                blk = c[max(0, x - sx):x + sx + 1, max(0, y - sy):y + sy + 1, max(0, z - sz):z + sz + 1]
                assert m[x, y, z] == pytest.approx(blk.mean(), rel=1e-12, abs=1e-12)
                assert s[x, y, z] == pytest.approx(blk.std(), rel=1e-12, abs=1e-12)


def test_constant_field(oracle):
    c = np.full((5, 6, 7), 2.25)
    m, s = oracle.local_stats(c, (2, 1, 3))
    assert np.all(m == 2.25)
    assert np.allclose(s, 0.0, atol=1e-15)


def test_box_covering_the_cube_gives_global_moments(oracle, rng):
    c = rng.normal(size=(4, 5, 6))
    m, s = oracle.local_stats(c, (4, 5, 6))
    assert np.allclose(m, c.mean(), rtol=0, atol=1e-13)
    assert np.allclose(s, c.std(), rtol=0, atol=1e-13)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_linear_ramp_interior(oracle, axis):
    shape = (9, 10, 11)
    half = [1, 2, 3]
    idx = np.indices(shape)[axis].astype(np.float64)
    c = 0.5 * idx - 1.0
    m, s = oracle.local_stats(c, half)
    h = half[axis]
    # interior along the ramp axis: the box is centred, so mean = value and
    # std = 0.5 * sqrt(h (h + 1) / 3) (uniform on 2h+1 equally spaced points)
    sl = [slice(None)] * 3
    sl[axis] = slice(h, shape[axis] - h)
    sl = tuple(sl)
    assert np.allclose(m[sl], c[sl], atol=1e-12)
    assert np.allclose(s[sl], 0.5 * math.sqrt(h * (h + 1) / 3.0), atol=1e-12)


def test_zero_half_width_is_the_voxel(oracle, rng):
    c = rng.normal(size=(3, 4, 5))
    m, s = oracle.local_stats(c, (0, 0, 0))
    assert np.array_equal(m, c)
    assert np.all(s == 0.0)


def test_clipped_count_at_the_corners(oracle):
    shape, half = (7, 8, 9), (2, 3, 1)
    for corner in [(0, 0, 0), (6, 7, 8), (0, 7, 0), (6, 0, 8)]:
        c = np.zeros(shape)
        c[corner] = 1.0
        m, _ = oracle.local_stats(c, half)
        n = (half[0] + 1) * (half[1] + 1) * (half[2] + 1)
        assert m[corner] == pytest.approx(1.0 / n, rel=1e-14)


def test_indexed_voxels_match_the_full_cube(oracle, rng):
    c = rng.normal(size=(6, 5, 8))
    m, s = oracle.local_stats(c, (1, 2, 2))
    flat = rng.choice(c.size, size=17, replace=False)
    mi, si = oracle.local_stats(c, (1, 2, 2), flat)
    assert np.array_equal(mi, m.ravel()[flat])
    assert np.array_equal(si, s.ravel()[flat])


def test_local_detect_sampled_path_matches_whole_cube(oracle, rng):
    d = rng.normal(size=(20, 18, 40)).astype(np.float32)
    d[8:12, 7:11, 15:25] += 4.0
    bank = ((1.0, 2.0), (0.0, 3.0))
    half = (3, 2, 6)
    fire, sure, cv, mv, sv = oracle.local_detect(d, bank, 3.0, half, 3.0)
    vox = np.stack([rng.integers(0, n, size=40) for n in d.shape], axis=1)
    f2, s2, c2, m2, v2 = oracle.local_detect(d, bank, 3.0, half, 3.0, voxels=vox)
    flat = (vox[:, 0] * d.shape[1] + vox[:, 1]) * d.shape[2] + vox[:, 2]
    assert np.allclose(c2, cv[:, flat], rtol=0, atol=1e-12)
    assert np.allclose(m2, mv[:, flat], rtol=0, atol=1e-12)
    assert np.allclose(v2, sv[:, flat], rtol=0, atol=1e-12)
    assert np.array_equal(f2, fire[flat])
    # the selection is the stated comparison
    thr = mv + 3.0 * sv
    assert np.array_equal(fire.astype(bool), (cv > thr).any(axis=0))
    assert fire.sum() > 0 and fire.sum() < fire.size


# ---- z-score (c - mean) / std over the same box ----

def test_zscore_of_a_spike_is_sqrt_n_minus_1(oracle):
    """One voxel of height h among zeros, box of n voxels around it: mean
    h/n, population variance h^2 (n - 1) / n^2, so z at the spike is
    (h - h/n) / (h sqrt(n - 1) / n) = sqrt(n - 1); its neighbours in the box
    sit at -1/sqrt(n - 1)."""
    c = np.zeros((9, 9, 13))
    c[4, 4, 6] = 7.5
    half = (1, 2, 3)
    n = 3 * 5 * 7
    z = oracle.local_zscore(c, half)
    assert z[4, 4, 6] == pytest.approx(math.sqrt(n - 1), rel=1e-12)
    # a neighbour whose own box is interior and holds the spike
    assert z[4, 4, 7] == pytest.approx(-1.0 / math.sqrt(n - 1), rel=1e-12)
    # far from the spike every box is constant 0: std 0 gives z 0
    assert z[0, 0, 0] == 0.0


def test_zscore_invariances(oracle, rng):
    """z is unchanged by c -> a c + b (a > 0) and flips sign under c -> -c."""
    c = rng.normal(size=(6, 7, 10))
    half = (1, 2, 2)
    z = oracle.local_zscore(c, half)
    assert np.allclose(oracle.local_zscore(3.5 * c - 2.0, half), z, rtol=1e-10, atol=1e-10)
    assert np.allclose(oracle.local_zscore(-c, half), -z, rtol=1e-10, atol=1e-10)


def test_zscore_brute_force_and_sampled(oracle, rng):
    c = rng.normal(size=(5, 6, 8)) + 4.0
    half = (1, 1, 2)
    z = oracle.local_zscore(c, half)
    nx, ny, nz = c.shape
    for x in range(nx):
        for y in range(ny):
            for q in range(nz):
                blk = c[max(0, x - 1):x + 2, max(0, y - 1):y + 2, max(0, q - 2):q + 3]
                assert z[x, y, q] == pytest.approx((c[x, y, q] - blk.mean()) / blk.std(), rel=1e-10)
    idx = np.array([0, 17, 101, c.size - 1])
    assert np.allclose(oracle.local_zscore(c, half, idx), z.ravel()[idx], rtol=1e-14, atol=0)


def test_local_sample_std_flag(oracle, rng):
    """ddof = 1 in the local statistics: numpy's std(ddof=1) of the clipped box."""
    c = rng.normal(size=(5, 6, 9)) + 2.0
    half = (1, 2, 3)
    m, s = oracle.local_stats(c, half, ddof=1)
    for x in range(5):
        for y in range(6):
            for z in range(9):
                blk = c[max(0, x - 1):x + 2, max(0, y - 2):y + 3, max(0, z - 3):z + 4]
                assert s[x, y, z] == pytest.approx(blk.std(ddof=1), rel=1e-12)
    _, s0 = oracle.local_stats(c, (0, 0, 0), ddof=1)
    assert (s0 == 0).all()


# ---- the sliding-statistics detect: selection and OR pinned from outside ----

def _box_sums(a, half):
    """Sums of a over the clipped box of half-widths `half` around every
    voxel, by cumulative sums along each axis (a summed-area table): no
    per-voxel loop, nothing shared with the oracle's two-pass box."""
    out = np.asarray(a, dtype=np.float64)
    for axis, h in enumerate(half):
        n = out.shape[axis]
        s = np.concatenate([np.zeros_like(np.take(out, [0], axis=axis)),
                            np.cumsum(out, axis=axis)], axis=axis)
        hi = np.minimum(np.arange(n) + h + 1, n)
        lo = np.maximum(np.arange(n) - h, 0)
        out = np.take(s, hi, axis=axis) - np.take(s, lo, axis=axis)
    return out


def _independent_local_detect(d, bank, trunc, half, k):
    """scipy Gaussian filter with zero padding, box moments from summed-area
    tables (mean = S1/n, var = S2/n - mean^2), c > mean + k std, OR."""
    fire = np.zeros(d.shape, dtype=bool)
    n = _box_sums(np.ones(d.shape), half)
    for sxy, sz in bank:
        rxy = math.ceil(trunc * sxy) if sxy > 0 else 0
        rz = math.ceil(trunc * sz) if sz > 0 else 0
        c = ndi.gaussian_filter(d.astype(np.float64), sigma=(sxy, sxy, sz), mode="constant",
                                cval=0.0, radius=(rxy, rxy, rz))
        mean = _box_sums(c, half) / n
        var = np.maximum(_box_sums(c * c, half) / n - mean * mean, 0.0)
        fire |= c > mean + k * np.sqrt(var)
    return fire


def test_local_detect_matches_independent_pipeline(oracle):
    """The whole sliding-statistics detect against scipy + summed-area tables
    on a cube with sources, a three-filter bank and an asymmetric box: masks
    equal wherever the oracle's decision is certain.  A flipped sign, a
    dropped filter in the OR or a box taken on the wrong axis each change
    many voxels."""
    k = 2.5
    from paper_1507_04941_gb300 import synth
    d = synth.make_cube((24, 20, 56), seed=31, n_sources=5, peak=(2.0, 4.0)).numpy()
    bank = ((0.0, 2.0), (1.5, 4.0), (1.0, 2.0))
    half = (4, 3, 7)
    fire, sure, cv, mv, sv = oracle.local_detect(d, bank, 3.0, half, k)
    ref = _independent_local_detect(d, bank, 3.0, half, k).ravel()
    sure = sure.astype(bool)
    got = fire.astype(bool)
    assert ref.sum() > 100
    assert np.array_equal(got[sure], ref[sure])
    assert (~sure).sum() <= 4
    # the first and the last filter each select voxels no other filter
    # selects, so an OR that drops either cannot pass
    per_f = cv > mv + k * sv
    for f in (0, len(bank) - 1):
        others = np.delete(per_f, f, axis=0).any(axis=0)
        assert (per_f[f] & ~others).any(), f


def test_local_detect_whole_cube_box_equals_window_detect(oracle):
    """A cube that is exactly one statistics window and a box covering the
    whole cube from every voxel: the local statistics are the window's, so
    the sliding-statistics detect is the window detect (Sec. 3.3 both ways)."""
    from paper_1507_04941_gb300 import synth
    d = synth.make_cube((16, 12, 40), seed=32, n_sources=3, peak=(2.0, 4.0)).numpy()
    bank = ((0.0, 2.0), (1.0, 3.0))
    k = 2.5
    fire, sure, cv, mv, sv = oracle.local_detect(d, bank, 3.0, (16, 12, 40), k)
    ref = oracle.detect(d, bank, 3.0, d.shape, k, nthreads=1)
    bits = oracle.unpack_bits(ref["mask"], d.shape[2]).ravel()
    rsure = oracle.unpack_bits(ref["sure"], d.shape[2]).ravel()
    both = rsure & sure.astype(bool)
    assert bits.sum() > 20
    assert np.array_equal(fire.astype(bool)[both], bits[both])
    for f in range(len(bank)):
        np.testing.assert_allclose(mv[f], ref["mean"][f].ravel()[0], rtol=0, atol=1e-12)
        np.testing.assert_allclose(sv[f], ref["std"][f].ravel()[0], rtol=1e-12)


def test_local_detect_tie_does_not_fire(oracle):
    """Values +1 and -1 in equal numbers, the identity filter and a box over
    the whole cube: mean 0 and std 1 exactly, so with k = 1 the threshold is
    exactly 1 and the strict comparison selects nothing, while c >= T would
    select half the cube."""
    d = np.ones((6, 4, 8), dtype=np.float32)
    d.reshape(-1)[::2] = -1.0
    fire, _, cv, mv, sv = oracle.local_detect(d, ((0.0, 0.0),), 3.0, (6, 4, 8), 1.0)
    assert np.all(mv == 0.0) and np.all(sv == 1.0)
    assert fire.sum() == 0


@pytest.mark.parametrize("k", [3.0, 4.0])
def test_local_detect_pure_noise_false_positive_rate(oracle, k):
    """iid N(0, 2^2) noise, the identity filter and a 9x9x17 box: each voxel
    is selected with probability close to 1 - Phi(k) (the box estimates
    move it by a few percent).  With sigma 2 a threshold on the variance
    (mean + k var) or a flipped sign misses by orders of magnitude."""
    shape = (64, 64, 128)
    d = (2.0 * np.random.default_rng(777).standard_normal(shape)).astype(np.float32)
    fire, _, _, _, _ = oracle.local_detect(d, ((0.0, 0.0),), 3.0, (4, 4, 8), k)
    fired = int(fire.sum())
    expect = d.size * 0.5 * math.erfc(k / math.sqrt(2.0))
    assert abs(fired - expect) < 0.3 * expect + 5 * math.sqrt(expect), (fired, expect)
