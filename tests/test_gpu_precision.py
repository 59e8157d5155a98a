"""Precision form: cube and x-filtered intermediates stored in FP16 / BF16,
FP32 arithmetic.

Gate (against the FP64 oracle run on the storage-rounded cube d_q):
  filtered values  |gpu - ref_q| <= 1e-3 sigma_noise + 2^-(p+1) A_q + 1e-5 A_q,
                   with A_q the filter applied to |d_q| and p the storage
                   mantissa bits (10 for FP16, 7 for BF16): the x-filtered
                   scratch is rounded to the storage type once, and positive
                   taps summing to one carry at most half an ulp of it;
  statistics       the same bound with the window's largest A_q;
  masks            bit-exact where |c_ref - T_ref| exceeds the same bound plus
                   the 1e-4 std guard band; elsewhere disagreements are counted.
Reported (printed, not gated): the error against the oracle on the FP32 cube.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

BANK6 = ((0.0, 2.0), (0.0, 6.0), (1.5, 2.0), (1.5, 6.0), (3.0, 2.0), (3.0, 6.0))
MANT = {"f16": 10, "bf16": 7}


@pytest.fixture(scope="module")
def dev():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1507_04941_gb300 import build
    build.build()
    return torch.device("cuda", 0)


def _tdtype(storage):
    import torch
    return {"f16": torch.float16, "bf16": torch.bfloat16}[storage]


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_filter_precision(dev, oracle, storage):
    from paper_1507_04941_gb300 import SourceFinder, synth
    shape = (48, 40, 128)
    cube = synth.make_cube(shape, 51, 10, (0.3, 5.0), 1.5)
    dq = cube.to(_tdtype(storage))
    d_q = dq.float().numpy()
    d32 = cube.numpy()
    eps = 2.0 ** -(MANT[storage] + 1)
    worst_gate, worst_f32 = 0.0, 0.0
    with SourceFinder(shape, BANK6, 3.0, (16, 16, 32), storage=storage, device=dev) as sf:
        for f, (sxy, sz) in enumerate(BANK6):
            got = sf.filter(dq.to(dev), f).cpu().numpy().astype(np.float64)
            ref_q = oracle.filter_box(d_q, sxy, sz, 3.0)
            A = oracle.filter_box(d_q, sxy, sz, 3.0, take_abs=True)
            bound = 1e-3 + eps * A + 1e-5 * A
            err = np.abs(got - ref_q)
            assert (err <= bound).all(), f"{storage} filter {f}: {(err / bound).max():.3g} x bound"
            worst_gate = max(worst_gate, float((err / bound).max()))
            worst_f32 = max(worst_f32, float(np.abs(got - oracle.filter_box(d32, sxy, sz, 3.0)).max()))
    print(f"\n[{storage}] filtered: worst |err|/bound {worst_gate:.3f}; "
          f"max |err| vs FP64 oracle on the FP32 cube {worst_f32:.3e} (noise sigma 1)")


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_detect_precision(dev, oracle, storage):
    import torch
    from paper_1507_04941_gb300 import SourceFinder, synth, words_to_bits
    shape = (64, 64, 192)
    window = (32, 32, 64)
    cube = synth.make_cube(shape, 52, 16, (0.3, 5.0), 1.5)
    dq = cube.to(_tdtype(storage))
    d_q = dq.float().numpy()
    eps = 2.0 ** -(MANT[storage] + 1)
    with SourceFinder(shape, BANK6, 3.0, window, storage=storage, device=dev) as sf:
        mask, mean, std = sf.detect(dq.to(dev), stats=True)
        torch.cuda.synchronize(dev)
        got = words_to_bits(mask.cpu().numpy(), shape[2])
        gm, gs = mean.cpu().numpy(), std.cpu().numpy()
        grid = sf.grid
    # FP32-storage run on the same rounded cube: the precision form's own effect
    with SourceFinder(shape, BANK6, 3.0, window, device=dev) as sf32:
        m32 = words_to_bits(sf32.detect(dq.float().to(dev)).cpu().numpy(), shape[2])
    n_dis = n_unsure = n_fire = 0
    worst_stat = 0.0
    for a in range(grid[0]):
        for b in range(grid[1]):
            for e in range(grid[2]):
                r = oracle.detect_window(d_q, BANK6, 3.0, window, 4.0, (a, b, e))
                x0, y0, z0 = r["origin"]
                ex, ey, ez = r["fire"].shape
                box = ((x0, x0 + ex), (y0, y0 + ey), (z0, z0 + ez))
                unsure = np.zeros(r["fire"].shape, dtype=bool)
                sure_fire = np.zeros(r["fire"].shape, dtype=bool)
                for f, (sxy, sz) in enumerate(BANK6):
                    A = oracle.filter_box(d_q, sxy, sz, 3.0, box=box, take_abs=True)
                    band = 1e-3 + (eps + 1e-5) * A + 1e-4 * r["std"][f]
                    dlt = r["c"][f] - r["thr"][f]
                    unsure |= np.abs(dlt) < band
                    sure_fire |= dlt >= band
                    sbound = 1e-3 + (eps + 1e-5) * A.max()
                    dm = abs(gm[f, a, b, e] - r["mean"][f])
                    ds = abs(gs[f, a, b, e] - r["std"][f])
                    assert dm <= sbound and ds <= sbound, f"{storage} stats window {(a, b, e)} f{f}"
                    worst_stat = max(worst_stat, dm / sbound, ds / sbound)
                certain = sure_fire | ~unsure
                g = got[x0:x0 + ex, y0:y0 + ey, z0:z0 + ez]
                want = r["fire"].astype(bool)
                assert not ((g != want) & certain).any(), f"{storage} window {(a, b, e)}"
                n_dis += int((g != want).sum())
                n_unsure += int((~certain).sum())
                n_fire += int(want.sum())
    print(f"\n[{storage}] detect: {n_fire} oracle detections, {n_unsure} voxels inside the "
          f"precision band, {n_dis} disagreements; vs FP32 storage on the same cube: "
          f"{int((got != m32).sum())} differing bits; stats worst {worst_stat:.3f} x bound")
    assert n_fire > 0
