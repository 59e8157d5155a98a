"""Pins of the FP64 oracle against facts fixed outside the oracle itself.

Each check is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign or index, a transposed axis, a missing normalisation, an off-by-one
window) fails at least one of them:

* library routines: scipy.ndimage.gaussian_filter with zero padding is the same
  sampled, truncated, normalised Gaussian (Eq. 2 with f a product of 1D
  Gaussians), numpy mean/std is the window statistic;
* closed forms: impulse response, constant cube with edges, linear ramp,
  second moment of the taps, the 0..n-1 sequence;
* brute force: Eq. 2 written as a numpy triple sum on tiny cubes;
* hand-worked fixtures under tests/golden/.
"""
import math
import os

import numpy as np
import pytest
import scipy.ndimage as ndi

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(t) for t in line.split()])
    return rows


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


# ------------------------------------------------------------------ taps ----
def test_radii_match_hand_worked_table(oracle):
    for sigma, trunc, r in _golden("radii.txt"):
        assert oracle.radius(sigma, trunc) == int(r)


@pytest.mark.parametrize("sigma", [0.4, 1.0, 1.5, 2.0, 3.0, 6.0])
def test_taps_equal_scipy_impulse_response(oracle, sigma):
    g = oracle.taps(sigma, 3.0)
    r = (len(g) - 1) // 2
    imp = np.zeros(2 * r + 1 + 2 * r)
    imp[2 * r] = 1.0
    ref = ndi.gaussian_filter1d(imp, sigma, mode="constant", cval=0.0, radius=r)
    np.testing.assert_allclose(g, ref[r:3 * r + 1], rtol=0, atol=1e-15)


@pytest.mark.parametrize("sigma", [1.0, 1.5, 3.0, 6.0])
def test_taps_normalised_symmetric_and_second_moment(oracle, sigma):
    g = oracle.taps(sigma, 10.0)
    r = (len(g) - 1) // 2
    o = np.arange(-r, r + 1)
    assert abs(g.sum() - 1.0) < 1e-15
    np.testing.assert_array_equal(g, g[::-1])
    # Poisson summation: the unit-sum sampled Gaussian has second moment
    # (s^2 + 2 (s^2 - 4 pi^2 s^4) q) / (1 + 2 q), q = exp(-2 pi^2 s^2), up to
    # terms in q^4 (truncation at 10 sigma is far below double precision).
    q = math.exp(-2 * math.pi ** 2 * sigma ** 2)
    s2 = sigma * sigma
    m2 = (s2 + 2 * (s2 - 4 * math.pi ** 2 * s2 * s2) * q) / (1 + 2 * q)
    assert abs((o * o * g).sum() - m2) < 1e-13 * s2


def test_zero_sigma_is_identity(oracle):
    np.testing.assert_array_equal(oracle.taps(0.0, 3.0), [1.0])
    d = _rng(1).standard_normal((5, 6, 7)).astype(np.float32)
    np.testing.assert_array_equal(oracle.filter_box(d, 0.0, 0.0, 3.0), d.astype(np.float64))


# ---------------------------------------------------------------- filter ----
@pytest.mark.parametrize("sxy,sz", [(0.0, 2.0), (1.0, 2.0), (1.5, 6.0), (3.0, 2.0)])
def test_filter_equals_scipy_gaussian_filter(oracle, sxy, sz):
    d = _rng(2).standard_normal((23, 19, 53)).astype(np.float32)
    rxy, rz = oracle.radius(sxy, 3.0), oracle.radius(sz, 3.0)
    ref = ndi.gaussian_filter(d.astype(np.float64), sigma=(sxy, sxy, sz), mode="constant",
                              cval=0.0, radius=(rxy, rxy, rz))
    got = oracle.filter_box(d, sxy, sz, 3.0)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)


def _eq2_numpy(d, gx, gy, gz):
    """Eq. 2 as a numpy triple sum over filter offsets, zero padding."""
    rx, ry, rz = (len(gx) - 1) // 2, (len(gy) - 1) // 2, (len(gz) - 1) // 2
    nx, ny, nz = d.shape
    p = np.zeros((nx + 2 * rx, ny + 2 * ry, nz + 2 * rz))
    p[rx:rx + nx, ry:ry + ny, rz:rz + nz] = d
    out = np.zeros(d.shape)
    for ox in range(-rx, rx + 1):
        for oy in range(-ry, ry + 1):
            for oz in range(-rz, rz + 1):
                f = gx[ox + rx] * gy[oy + ry] * gz[oz + rz]
                out += f * p[rx + ox:rx + ox + nx, ry + oy:ry + oy + ny, rz + oz:rz + oz + nz]
    return out


@pytest.mark.parametrize("sxy,sz", [(1.0, 2.0), (1.5, 1.0), (0.0, 3.0)])
def test_separable_filter_equals_brute_force_eq2(oracle, sxy, sz):
    d = _rng(3).standard_normal((7, 9, 23)).astype(np.float32)
    g = oracle.taps(sxy, 3.0)
    gz = oracle.taps(sz, 3.0)
    ref = _eq2_numpy(d.astype(np.float64), g, g, gz)
    np.testing.assert_allclose(oracle.filter_box(d, sxy, sz, 3.0), ref, rtol=0, atol=1e-12)
    # the oracle's own literal triple sum agrees at a few voxels, edges included
    for (x, y, z) in [(0, 0, 0), (3, 4, 11), (6, 8, 22), (2, 0, 17)]:
        assert abs(oracle.filter_direct_voxel(d, sxy, sz, 3.0, x, y, z) - ref[x, y, z]) < 1e-12


def test_filter_box_equals_whole_cube_slice(oracle):
    d = _rng(4).standard_normal((20, 22, 40)).astype(np.float32)
    full = oracle.filter_box(d, 1.5, 2.0, 3.0)
    box = ((3, 17), (0, 9), (30, 40))
    part = oracle.filter_box(d, 1.5, 2.0, 3.0, box=box)
    np.testing.assert_array_equal(part, full[3:17, 0:9, 30:40])


def test_impulse_returns_the_filter(oracle):
    d = np.zeros((21, 21, 41), dtype=np.float32)
    d[10, 10, 20] = 1.0
    g = oracle.taps(1.5, 3.0)
    gz = oracle.taps(2.0, 3.0)
    c = oracle.filter_box(d, 1.5, 2.0, 3.0)
    kernel = g[:, None, None] * g[None, :, None] * gz[None, None, :]
    np.testing.assert_allclose(c[5:16, 5:16, 14:27], kernel, rtol=0, atol=1e-17)
    assert abs(c.sum() - 1.0) < 1e-14
    assert np.count_nonzero(c) == kernel.size


def test_constant_cube_closed_form_with_edges(oracle):
    C = 2.5
    d = np.full((12, 15, 30), C, dtype=np.float32)
    c = oracle.filter_box(d, 1.5, 2.0, 3.0)

    def partial(g, n):
        r = (len(g) - 1) // 2
        return np.array([sum(g[o + r] for o in range(-r, r + 1) if 0 <= i + o < n)
                         for i in range(n)])

    g = oracle.taps(1.5, 3.0)
    gz = oracle.taps(2.0, 3.0)
    ref = C * partial(g, 12)[:, None, None] * partial(g, 15)[None, :, None] * \
        partial(gz, 30)[None, None, :]
    np.testing.assert_allclose(c, ref, rtol=1e-14, atol=0)
    np.testing.assert_allclose(c[5:7, 5:10, 6:24], C, rtol=1e-14)  # interior stays C


def test_linear_ramp_preserved_in_interior(oracle):
    nx, ny, nz = 24, 24, 60
    x, y, z = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    d = (0.5 + 0.25 * x - 0.125 * y + 0.0625 * z).astype(np.float32)
    c = oracle.filter_box(d, 1.5, 2.0, 3.0)
    np.testing.assert_allclose(c[5:-5, 5:-5, 6:-6], d[5:-5, 5:-5, 6:-6], rtol=1e-13, atol=1e-13)
    # a quadratic along z gains the taps' second moment
    q = (np.zeros((1, 1, nz)) + np.arange(nz) ** 2).astype(np.float32)
    cq = oracle.filter_box(q, 0.0, 2.0, 3.0)
    gz = oracle.taps(2.0, 3.0)
    m2 = float((np.arange(-6, 7) ** 2 * gz).sum())
    np.testing.assert_allclose(cq[0, 0, 6:-6], np.arange(6, nz - 6) ** 2 + m2, rtol=1e-13)


def test_axes_are_not_transposed(oracle):
    # an impulse filtered with sigma only along z must spread only along z
    d = np.zeros((9, 9, 9), dtype=np.float32)
    d[4, 4, 4] = 1.0
    c = oracle.filter_box(d, 0.0, 1.0, 3.0)
    assert np.count_nonzero(c[:, :, 4]) == 1 and np.count_nonzero(c[4, 4, :]) == 7
    c2 = oracle.filter_box(d, 1.0, 0.0, 3.0)
    assert np.count_nonzero(c2[4, 4, :]) == 1 and np.count_nonzero(c2[:, :, 4]) == 49


# ----------------------------------------------------------------- stats ----
def test_window_sequence_closed_form(oracle):
    for n, mean, var in _golden("window_sequence.txt"):
        m, s = oracle.moments(np.arange(int(n), dtype=np.float64))
        assert m == pytest.approx(mean, rel=0, abs=1e-12 * max(1.0, mean))
        assert s * s == pytest.approx(var, rel=1e-12, abs=1e-15)


def test_window_stats_equal_numpy_with_tail_windows(oracle):
    c = _rng(5).standard_normal((37, 21, 45)) * 3.0 + 1.0
    w = (16, 16, 32)
    mean, std = oracle.window_stats(c, w)
    assert mean.shape == (3, 2, 2)
    for a in range(3):
        for b in range(2):
            for e in range(2):
                blk = c[a * 16:(a + 1) * 16, b * 16:(b + 1) * 16, e * 32:(e + 1) * 32]
                assert mean[a, b, e] == pytest.approx(blk.mean(), rel=1e-13, abs=1e-14)
                assert std[a, b, e] == pytest.approx(blk.std(ddof=0), rel=1e-13)


def test_constant_window_has_zero_std_and_fires_nothing(oracle):
    c = np.full((16, 16, 32), 7.25)
    mean, std = oracle.window_stats(c, (16, 16, 32))
    assert mean[0, 0, 0] == 7.25 and std[0, 0, 0] == 0.0
    mask, amb = oracle.threshold(c, (16, 16, 32), mean, std, 4.0)
    assert not mask.any() and not amb.any()


# ------------------------------------------------------ threshold / mask ----
def test_mask_packing_hand_worked(oracle):
    for nx, ny, nz, x, y, z, word, bit in _golden("mask_packing.txt"):
        nx, ny, nz, x, y, z, word, bit = (int(v) for v in (nx, ny, nz, x, y, z, word, bit))
        bits = np.zeros((nx, ny, nz), dtype=bool)
        bits[x, y, z] = True
        w = oracle.pack_bits(bits).ravel()
        assert np.flatnonzero(w).tolist() == [word]
        assert int(w[word]) == 1 << bit
        np.testing.assert_array_equal(oracle.unpack_bits(w.reshape(nx, ny, -1), nz), bits)


def test_threshold_strict_and_per_window(oracle):
    w = (4, 4, 8)
    c = np.zeros((8, 4, 8))
    mean = np.array([[[1.0]], [[2.0]]])
    std = np.array([[[0.5]], [[1.0]]])
    T0, T1 = 1.0 + 4 * 0.5, 2.0 + 4 * 1.0
    c[0, 0, 0] = T0                        # equal: does not fire (strict)
    c[0, 0, 1] = T0 + 1e-9                 # above, but inside the guard band
    c[1, 2, 3] = T0 + 1.0                  # fires
    c[4, 0, 0] = T0 + 1.0                  # window 1: below T1, no fire
    c[5, 3, 7] = T1 + 0.5                  # window 1: fires
    mask, amb = oracle.threshold(c, w, mean, std, 4.0, band_rel=1e-4)
    bits = oracle.unpack_bits(mask, 8)
    assert sorted(map(tuple, np.argwhere(bits))) == [(0, 0, 1), (1, 2, 3), (5, 3, 7)]
    abits = oracle.unpack_bits(amb, 8)
    assert sorted(map(tuple, np.argwhere(abits))) == [(0, 0, 0), (0, 0, 1)]


def _independent_detect(d, bank, trunc, window, k):
    """scipy filter + numpy window stats + numpy threshold, OR over the bank."""
    nx, ny, nz = d.shape
    wx, wy, wz = window
    fire = np.zeros(d.shape, dtype=bool)
    stats = []
    for sxy, sz in bank:
        r = (math.ceil(trunc * sxy) if sxy > 0 else 0, math.ceil(trunc * sz) if sz > 0 else 0)
        c = ndi.gaussian_filter(d.astype(np.float64), sigma=(sxy, sxy, sz), mode="constant",
                                cval=0.0, radius=(r[0], r[0], r[1]))
        T = np.empty_like(c)
        ms = []
        for x0 in range(0, nx, wx):
            for y0 in range(0, ny, wy):
                for z0 in range(0, nz, wz):
                    blk = c[x0:x0 + wx, y0:y0 + wy, z0:z0 + wz]
                    T[x0:x0 + wx, y0:y0 + wy, z0:z0 + wz] = blk.mean() + k * blk.std()
                    ms.append((blk.mean(), blk.std()))
        stats.append(ms)
        fire |= c > T
    return fire, np.array(stats)


def test_detect_equals_independent_pipeline(oracle):
    from paper_1507_04941_gb300 import synth
    d = synth.make_cube((40, 36, 96), seed=11, n_sources=6, peak=(2.0, 4.0)).numpy()
    bank = ((0.0, 2.0), (1.0, 2.0), (1.5, 6.0))
    window = (16, 16, 32)
    res = oracle.detect(d, bank, 3.0, window, 4.0, nthreads=2)
    fire, stats = _independent_detect(d, bank, 3.0, window, 4.0)
    got = oracle.unpack_bits(res["mask"], d.shape[2])
    sure = oracle.unpack_bits(res["sure"], d.shape[2])
    assert fire.sum() > 0
    assert np.array_equal(got[sure], fire[sure])
    assert (~sure).sum() <= 2
    np.testing.assert_allclose(res["mean"].reshape(len(bank), -1), stats[:, :, 0], atol=1e-13)
    np.testing.assert_allclose(res["std"].reshape(len(bank), -1), stats[:, :, 1], rtol=1e-12)


def test_detect_window_agrees_with_detect(oracle):
    from paper_1507_04941_gb300 import synth
    d = synth.make_cube((32, 32, 70), seed=12, n_sources=4).numpy()
    bank = ((1.0, 2.0), (0.0, 3.0))
    window = (16, 16, 32)
    full = oracle.detect(d, bank, 3.0, window, 4.0, nthreads=1)
    bits = oracle.unpack_bits(full["mask"], 70)
    for widx in [(0, 0, 0), (1, 1, 2), (0, 1, 1)]:
        r = oracle.detect_window(d, bank, 3.0, window, 4.0, widx)
        x0, y0, z0 = r["origin"]
        ex, ey, ez = r["fire"].shape
        np.testing.assert_array_equal(r["fire"].astype(bool), bits[x0:x0 + ex, y0:y0 + ey,
                                                                   z0:z0 + ez])
        np.testing.assert_array_equal(r["mean"], full["mean"][:, widx[0], widx[1], widx[2]])


def test_injected_source_recovered_at_centre(oracle):
    d = _rng(6).standard_normal((48, 48, 96)).astype(np.float32)
    x, y, z = np.meshgrid(np.arange(48), np.arange(48), np.arange(96), indexing="ij")
    d += (3.0 * np.exp(-((x - 20) ** 2 + (y - 27) ** 2) / (2 * 2.0 ** 2)
                       - (z - 50) ** 2 / (2 * 6.0 ** 2))).astype(np.float32)
    res = oracle.detect(d, ((1.5, 2.0), (3.0, 6.0)), 3.0, (16, 16, 32), 4.0, nthreads=2)
    bits = oracle.unpack_bits(res["mask"], 96)
    assert bits[20, 27, 50]
    # pure noise elsewhere rarely fires: far below 1% of voxels
    assert bits.mean() < 0.01


# ------------------------------------------------- threshold statistics ----
@pytest.mark.parametrize("k", [3.0, 4.0])
def test_pure_noise_false_positive_rate(oracle, k):
    """On iid N(0,1) noise with the identity filter, c > mean + k std fires
    with probability 1 - Phi(k) per voxel (the window estimates of mean and
    std over 65536 voxels move that by well under the binomial spread).  A
    threshold on the variance, a flipped sign or a wrong window would miss
    this by orders of magnitude."""
    shape = (128, 128, 256)
    d = _rng(4242).standard_normal(shape).astype(np.float32)
    ref = oracle.detect(d, ((0.0, 0.0),), 3.0, (32, 32, 64), k)
    fired = int(oracle.unpack_bits(ref["mask"], shape[2]).sum())
    p = 0.5 * math.erfc(k / math.sqrt(2.0))
    n = d.size
    expect, sd = n * p, math.sqrt(n * p * (1 - p))
    assert abs(fired - expect) < 5 * sd + 0.02 * expect, (fired, expect)


def test_smoothed_noise_false_positive_rate(oracle):
    """The same on noise smoothed by the (1.5, 2) filter: the filtered values
    are Gaussian again and the window statistics follow them, so the rate is
    still 1 - Phi(k); neighbouring voxels fire together, so the bound is
    loose (a third of the expectation)."""
    shape = (96, 96, 256)
    d = _rng(4343).standard_normal(shape).astype(np.float32)
    k = 3.0
    ref = oracle.detect(d, ((1.5, 2.0),), 3.0, (32, 32, 64), k)
    fired = int(oracle.unpack_bits(ref["mask"], shape[2]).sum())
    expect = d.size * 0.5 * math.erfc(k / math.sqrt(2.0))
    assert abs(fired - expect) < expect / 3, (fired, expect)


# ------------------------------------------------- std normaliser (ddof) ----
def test_sample_std_flag_equals_numpy(oracle):
    """ddof = 1 divides the squared deviations by n - 1 (numpy's ddof): per
    window, tail windows included, and through the detect path's statistics;
    a window of one voxel has std 0."""
    c = _rng(77).normal(size=(7, 9, 20)) * 2.0 + 1.0
    window = (3, 4, 8)
    m1, s1 = oracle.window_stats(c, window, ddof=1)
    for a in range(m1.shape[0]):
        for b in range(m1.shape[1]):
            for e in range(m1.shape[2]):
                blk = c[3 * a:3 * a + 3, 4 * b:4 * b + 4, 8 * e:8 * e + 8]
                assert m1[a, b, e] == pytest.approx(blk.mean(), rel=1e-13)
                assert s1[a, b, e] == pytest.approx(blk.std(ddof=1), rel=1e-13)
    m, s = oracle.moments([3.5], ddof=1)
    assert (m, s) == (3.5, 0.0)
    d = c.astype(np.float32)
    r0 = oracle.detect(d, ((0.0, 0.0),), 3.0, window, 1.0)
    r1 = oracle.detect(d, ((0.0, 0.0),), 3.0, window, 1.0, ddof=1)
    m0, s0 = oracle.window_stats(d.astype(np.float64), window)
    np.testing.assert_allclose(r1["std"][0], s0 * np.sqrt(_counts(d.shape, window) / (_counts(d.shape, window) - 1)),
                               rtol=1e-12)
    assert oracle.unpack_bits(r1["mask"], 20).sum() < oracle.unpack_bits(r0["mask"], 20).sum()


def _counts(shape, window):
    n = np.ones(oracle_grid(shape, window))
    for ax, (N, w) in enumerate(zip(shape, window)):
        ext = np.array([min(w, N - i * w) for i in range(-(-N // w))], dtype=float)
        sh = [1, 1, 1]
        sh[ax] = -1
        n = n * ext.reshape(sh)
    return n


def oracle_grid(shape, window):
    return tuple(-(-N // w) for N, w in zip(shape, window))


def test_detect_windows_counts_match_detect(oracle):
    """The per-window fired counts of detect_windows (the CPU baseline's
    sampled path) equal the fired bits of the whole-cube detect in those
    windows."""
    rng = _rng(88)
    shape, window = (20, 18, 70), (8, 6, 32)
    d = rng.normal(size=shape).astype(np.float32)
    bank = ((1.0, 2.0), (0.0, 3.0))
    full = oracle.detect(d, bank, 3.0, window, 2.5)
    bits = oracle.unpack_bits(full["mask"], shape[2])
    idx = [(0, 0, 0), (2, 2, 2), (1, 2, 0), (2, 0, 1)]
    fired, _ = oracle.detect_windows(d, bank, 3.0, window, 2.5, idx)
    for (a, b, e), n in zip(idx, fired):
        blk = bits[a * 8:(a + 1) * 8, b * 6:(b + 1) * 6, e * 32:(e + 1) * 32]
        assert n == int(blk.sum())
    assert fired.sum() > 0
