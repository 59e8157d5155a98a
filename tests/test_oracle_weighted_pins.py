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
