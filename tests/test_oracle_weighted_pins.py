"""Pins of the oracle's weighted convolution (Eq. 1) against facts fixed
independently of it: a numpy triple sum with its own taps, the unweighted
case through scipy (w = 1: Eq. 2 inside, the normalised filter at the edges),
scale invariance in w, constant data (the constant itself for the normalised
denominator, the closed form kappa / F for the printed one), and zero weight."""
import math

import numpy as np
import pytest
import scipy.ndimage as ndi


def _taps(sigma, trunc):
    r = int(math.ceil(trunc * sigma)) if sigma > 0 else 0
    if r == 0:
        return np.ones(1)
    o = np.arange(-r, r + 1)
    g = np.exp(-o * o / (2.0 * sigma * sigma))
    return g / g.sum()


def _numpy_eq1(d, w, sxy, sz, trunc, den):
    gx = _taps(sxy, trunc)
    gz = _taps(sz, trunc)
    rx, rz = len(gx) // 2, len(gz) // 2
    f = gx[:, None, None] * gx[None, :, None] * gz[None, None, :]
    dp = np.pad(d.astype(np.float64), ((rx, rx), (rx, rx), (rz, rz)))
    wp = np.pad(w.astype(np.float64), ((rx, rx), (rx, rx), (rz, rz)))
    out = np.zeros(d.shape)
    for x in range(d.shape[0]):
        for y in range(d.shape[1]):
            for z in range(d.shape[2]):
                db = dp[x:x + 2 * rx + 1, y:y + 2 * rx + 1, z:z + 2 * rz + 1]
                wb = wp[x:x + 2 * rx + 1, y:y + 2 * rx + 1, z:z + 2 * rz + 1]
                num = (db * f * wb).sum()
                dd = (f * wb).sum() if den == "fw" else wb.sum()
                out[x, y, z] = num / dd if dd != 0 else 0.0
    return out


@pytest.fixture(scope="module")
def rng():
    return np.random.default_rng(1507)


@pytest.mark.parametrize("den", ["fw", "w"])
@pytest.mark.parametrize("sxy,sz", [(1.0, 1.5), (0.0, 2.0), (0.7, 0.0)])
def test_brute_force_triple_sum(oracle, rng, den, sxy, sz):
    d = rng.normal(size=(6, 7, 11)).astype(np.float32)
    w = rng.uniform(0.1, 2.0, size=d.shape).astype(np.float32)
    w[1, 2, 3] = 0.0
    got = oracle.weighted_filter_box(d, w, sxy, sz, 2.0, den)
    want = _numpy_eq1(d, w, sxy, sz, 2.0, den)
    np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-13)
    # the literal form at a corner and at the centre
    for v in [(0, 0, 0), (3, 3, 5), (5, 6, 10)]:
        assert oracle.weighted_direct_voxel(d, w, sxy, sz, 2.0, *v, den=den) == pytest.approx(
            want[v], rel=1e-11, abs=1e-13)


def test_unit_weights_are_the_normalised_gaussian(oracle, rng):
    d = rng.normal(size=(16, 15, 30)).astype(np.float32)
    w = np.ones_like(d)
    sxy, sz, tr = 1.5, 2.0, 3.0
    got = oracle.weighted_filter_box(d, w, sxy, sz, tr, "fw")
    trunc_xy, trunc_z = math.ceil(tr * sxy) / sxy, math.ceil(tr * sz) / sz
    num = ndi.gaussian_filter(d.astype(np.float64), (sxy, sxy, 0), mode="constant", truncate=trunc_xy)
    num = ndi.gaussian_filter(num, (0, 0, sz), mode="constant", truncate=trunc_z)
    one = ndi.gaussian_filter(np.ones(d.shape), (sxy, sxy, 0), mode="constant", truncate=trunc_xy)
    one = ndi.gaussian_filter(one, (0, 0, sz), mode="constant", truncate=trunc_z)
    np.testing.assert_allclose(got, num / one, rtol=1e-10, atol=1e-12)
    # inside (support within the cube) the normalised form is Eq. 2 itself
    rx, rz = math.ceil(tr * sxy), math.ceil(tr * sz)
    inner = (slice(rx, -rx), slice(rx, -rx), slice(rz, -rz))
    np.testing.assert_allclose(got[inner], num[inner], rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("den", ["fw", "w"])
def test_scale_invariance_in_the_weights(oracle, rng, den):
    d = rng.normal(size=(8, 9, 14)).astype(np.float32)
    w = rng.uniform(0.5, 1.5, size=d.shape).astype(np.float32)
    a = oracle.weighted_filter_box(d, w, 1.0, 2.0, 2.5, den)
    b = oracle.weighted_filter_box(d, (4.0 * w).astype(np.float32), 1.0, 2.0, 2.5, den)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-14)


def test_constant_data(oracle, rng):
    kappa = 2.5
    d = np.full((9, 10, 13), kappa, dtype=np.float32)
    w = rng.uniform(0.2, 3.0, size=d.shape).astype(np.float32)
    got = oracle.weighted_filter_box(d, w, 1.2, 1.8, 2.0, "fw")
    np.testing.assert_allclose(got, kappa, rtol=1e-13)
    # printed denominator, unit weights, support inside: kappa * sum f / F
    ones = np.ones_like(d)
    got_w = oracle.weighted_filter_box(d, ones, 1.0, 1.0, 2.0, "w")
    F = 5 * 5 * 5
    np.testing.assert_allclose(got_w[2:-2, 2:-2, 2:-2], kappa / F, rtol=1e-13)


@pytest.mark.parametrize("den", ["fw", "w"])
def test_zero_weight_gives_zero(oracle, rng, den):
    d = rng.normal(size=(10, 10, 20)).astype(np.float32)
    w = np.zeros_like(d)
    w[:2] = 1.0   # weight only in the first two x-planes
    got = oracle.weighted_filter_box(d, w, 1.0, 1.0, 2.0, den)
    # planes x >= 4 have no weight within their x radius of 2
    assert np.all(got[4:] == 0.0)
    assert np.any(got[:2] != 0.0)


# ---- the weighted detect (Eq. 1 filtering + window statistics + threshold) ----

def test_weighted_detect_constant_data_is_constant(oracle):
    """Normalised convolution (den = sum f w) of a constant cube is that
    constant everywhere, edges included: every window has the mean C and a
    std at the rounding level (the threshold decisions are then rounding's,
    and are not asserted)."""
    rng = np.random.default_rng(5)
    shape = (12, 10, 40)
    d = np.full(shape, 2.5, dtype=np.float32)
    w = (0.5 + rng.random(shape)).astype(np.float32)
    ref = oracle.weighted_detect(d, w, ((1.0, 2.0), (0.0, 3.0)), 3.0, (4, 5, 16), 3.0, "fw")
    np.testing.assert_allclose(ref["mean"], 2.5, rtol=1e-12)
    assert np.all(ref["std"] < 1e-12)


def test_weighted_detect_invariances(oracle):
    """c_w is invariant under w -> a w (a > 0) and linear in d: the masks
    stay the same, the statistics follow d."""
    rng = np.random.default_rng(6)
    shape = (10, 12, 48)
    d = rng.normal(size=shape).astype(np.float32)
    w = (0.2 + rng.random(shape)).astype(np.float32)
    bank = ((1.0, 2.0),)
    for den in ("fw", "w"):
        r0 = oracle.weighted_detect(d, w, bank, 3.0, (5, 6, 16), 2.0, den)
        r1 = oracle.weighted_detect(d, (4.0 * w).astype(np.float32), bank, 3.0, (5, 6, 16), 2.0, den)
        r2 = oracle.weighted_detect((2.0 * d).astype(np.float32), w, bank, 3.0, (5, 6, 16), 2.0, den)
        np.testing.assert_allclose(r1["mean"], r0["mean"], rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(r1["std"], r0["std"], rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(r2["mean"], 2.0 * r0["mean"], rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(r2["std"], 2.0 * r0["std"], rtol=1e-10, atol=1e-12)
        sure = r0["sure"] & r1["sure"] & r2["sure"]
        assert not ((r0["mask"] ^ r1["mask"]) & sure).any()
        assert not ((r0["mask"] ^ r2["mask"]) & sure).any()
        assert r0["mask"].any()


# ---- the weighted detect: selection and OR pinned from outside ----

def _independent_weighted_detect(d, w, bank, trunc, window, k, den):
    """scipy filters of d*w and of w (zero padding; the unit-tap box sum for
    the printed denominator), their ratio (0 where the denominator is 0),
    numpy window statistics by explicit slices, c > mean + k std, OR."""
    nx, ny, nz = d.shape
    wx, wy, wz = window
    fire = np.zeros(d.shape, dtype=bool)
    per_f = []
    dw = d.astype(np.float64) * w.astype(np.float64)
    for sxy, sz in bank:
        rxy = math.ceil(trunc * sxy) if sxy > 0 else 0
        rz = math.ceil(trunc * sz) if sz > 0 else 0
        num = ndi.gaussian_filter(dw, sigma=(sxy, sxy, sz), mode="constant", cval=0.0,
                                  radius=(rxy, rxy, rz))
        if den == "fw":
            dd = ndi.gaussian_filter(w.astype(np.float64), sigma=(sxy, sxy, sz), mode="constant",
                                     cval=0.0, radius=(rxy, rxy, rz))
        else:
            size = (2 * rxy + 1, 2 * rxy + 1, 2 * rz + 1)
            dd = ndi.uniform_filter(w.astype(np.float64), size=size, mode="constant",
                                    cval=0.0) * float(np.prod(size))
        c = np.where(dd != 0, num / np.where(dd != 0, dd, 1.0), 0.0)
        T = np.empty_like(c)
        for x0 in range(0, nx, wx):
            for y0 in range(0, ny, wy):
                for z0 in range(0, nz, wz):
                    blk = c[x0:x0 + wx, y0:y0 + wy, z0:z0 + wz]
                    T[x0:x0 + wx, y0:y0 + wy, z0:z0 + wz] = blk.mean() + k * blk.std()
        per_f.append(c > T)
        fire |= per_f[-1]
    return fire, np.array(per_f)


@pytest.mark.parametrize("den", ["fw", "w"])
def test_weighted_detect_matches_independent_pipeline(oracle, den):
    """The whole weighted detect against scipy + numpy on a cube with
    sources, flagged (zero-weight) channels, tail windows on every axis and a
    three-filter bank: masks equal wherever the oracle's decision is certain.
    A flipped sign, a dropped filter in the OR or a wrong window index in the
    broadcast of the statistics each change many voxels."""
    from paper_1507_04941_gb300 import synth
    shape = (22, 18, 72)
    d = synth.make_cube(shape, seed=41, n_sources=5, peak=(2.0, 4.0)).numpy()
    w = synth.make_weights(shape, 41).numpy()
    bank = ((0.0, 2.0), (1.5, 4.0), (1.0, 2.0))
    window, k = (8, 8, 32), 2.5
    ref = oracle.weighted_detect(d, w, bank, 3.0, window, k, den)
    fire, per_f = _independent_weighted_detect(d, w, bank, 3.0, window, k, den)
    got = oracle.unpack_bits(ref["mask"], shape[2])
    sure = oracle.unpack_bits(ref["sure"], shape[2])
    assert fire.sum() > 50
    assert np.array_equal(got[sure], fire[sure])
    assert (~sure).sum() <= 4
    for f in (0, len(bank) - 1):
        others = np.delete(per_f, f, axis=0).any(axis=0)
        assert (per_f[f] & ~others & sure).any(), f


def test_weighted_detect_unit_weights_identity_filter_is_detect(oracle):
    """w = 1, the normalised denominator and the identity filter give c_w = d
    exactly (Eq. 1 with one tap), so the weighted detect is the plain
    detect of the identity filter: same masks, same window statistics."""
    from paper_1507_04941_gb300 import synth
    shape = (20, 24, 70)
    d = synth.make_cube(shape, seed=42, n_sources=4, peak=(2.0, 4.0)).numpy()
    w = np.ones(shape, dtype=np.float32)
    bank, window, k = ((0.0, 0.0),), (8, 8, 32), 2.5
    got = oracle.weighted_detect(d, w, bank, 3.0, window, k, "fw")
    ref = oracle.detect(d, bank, 3.0, window, k, nthreads=1)
    assert np.array_equal(got["mask"], ref["mask"])
    assert ref["mask"].any()
    np.testing.assert_array_equal(got["mean"], ref["mean"])
    np.testing.assert_array_equal(got["std"], ref["std"])


@pytest.mark.parametrize("den", ["fw", "w"])
def test_weighted_detect_tie_does_not_fire(oracle, den):
    """Values +1 and -1 in equal numbers, w = 1, the identity filter and one
    window over the cube: c_w = d, mean 0 and std 1 exactly, so with k = 1
    the threshold is exactly 1 and the strict comparison selects nothing."""
    d = np.ones((4, 6, 8), dtype=np.float32)
    d.reshape(-1)[::2] = -1.0
    w = np.ones_like(d)
    ref = oracle.weighted_detect(d, w, ((0.0, 0.0),), 3.0, (4, 6, 8), 1.0, den)
    assert ref["mean"].ravel()[0] == 0.0 and ref["std"].ravel()[0] == 1.0
    assert not ref["mask"].any()


@pytest.mark.parametrize("k", [3.0, 4.0])
def test_weighted_detect_pure_noise_false_positive_rate(oracle, k):
    """iid N(0, 2^2) noise, random positive weights and the identity filter:
    c_w = d w / w = d, so each voxel fires with probability 1 - Phi(k) (the
    window estimates over 65536 voxels move it by far less than the
    binomial spread).  A flipped sign or a threshold on the variance misses
    by orders of magnitude."""
    shape = (128, 128, 256)
    rng = np.random.default_rng(4545)
    d = (2.0 * rng.standard_normal(shape)).astype(np.float32)
    w = (0.25 + rng.random(shape)).astype(np.float32)
    ref = oracle.weighted_detect(d, w, ((0.0, 0.0),), 3.0, (32, 32, 64), k, "fw")
    fired = int(oracle.unpack_bits(ref["mask"], shape[2]).sum())
    p = 0.5 * math.erfc(k / math.sqrt(2.0))
    n = d.size
    expect, sd = n * p, math.sqrt(n * p * (1 - p))
    assert abs(fired - expect) < 5 * sd + 0.02 * expect, (fired, expect)
