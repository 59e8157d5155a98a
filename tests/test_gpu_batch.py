"""Batched form: many uneven cubes in one persistent launch replayed from a
CUDA graph, and the autotuner.  The batched path runs the same arithmetic as
the per-cube path, so masks and statistics must be bit-identical to
sf_detect on each cube alone; the per-cube path is pinned to the oracle by
test_gpu_parity.py, and one batch member is compared with the oracle here."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

BANK6 = ((0.0, 2.0), (0.0, 6.0), (1.5, 2.0), (1.5, 6.0), (3.0, 2.0), (3.0, 6.0))
SHAPES = [(70, 70, 131), (64, 64, 256), (33, 33, 200), (96, 96, 129), (41, 41, 130), (128, 128, 64)]


@pytest.fixture(scope="module")
def dev():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1507_04941_gb300 import build
    build.build()
    return torch.device("cuda", 0)


def _cubes(dev):
    from paper_1507_04941_gb300 import synth
    return [synth.make_cube(sh, 700 + i, 6, (0.5, 5.0), 1.5, device=dev) for i, sh in enumerate(SHAPES)]


def _single(dev, cube, window=(32, 32, 64)):
    import torch
    from paper_1507_04941_gb300 import SourceFinder
    with SourceFinder(tuple(cube.shape), BANK6, 3.0, window, device=dev) as sf:
        out = sf.detect(cube, stats=True)
        torch.cuda.synchronize(dev)
        return [t.cpu() for t in out]


def test_batch_equals_per_cube(dev, oracle):
    import torch
    from paper_1507_04941_gb300 import BatchSourceFinder, words_to_bits
    cubes = _cubes(dev)
    with BatchSourceFinder(SHAPES, BANK6, 3.0, (32, 32, 64), device=dev) as bf:
        for rep in range(2):   # the second call replays the graph with fresh tables
            masks, means, stds = bf.detect(cubes, stats=True)
            bf.synchronize()
            for i, cube in enumerate(cubes):
                m1, me1, sd1 = _single(dev, cube)
                assert torch.equal(masks[i].cpu(), m1), f"cube {i} mask (call {rep})"
                assert torch.equal(means[i].cpu(), me1), f"cube {i} mean"
                assert torch.equal(stds[i].cpu(), sd1), f"cube {i} std"
    # one member against the oracle
    i = 0
    ref = oracle.detect(cubes[i].cpu().numpy(), BANK6, 3.0, (32, 32, 64), 4.0)
    got = words_to_bits(masks[i].cpu().numpy(), SHAPES[i][2])
    sure = oracle.unpack_bits(ref["sure"], SHAPES[i][2])
    want = oracle.unpack_bits(ref["mask"], SHAPES[i][2])
    assert not ((got != want) & sure).any()


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_batch_padded_rows_equal_per_cube(dev, storage, monkeypatch):
    """Cubes whose rows are not 16-byte multiples (nz 131, 129, 130 in FP32;
    also 200 in FP16) take padded scratch rows and a padded copy of the cube
    written by the batched x pass, read by TMA: bit-identical to the per-cube
    path, which reads them unpadded by cp.async (the CUDA-core window kernel
    for FP16, as in the batch)."""
    import torch
    from paper_1507_04941_gb300 import BatchSourceFinder, SourceFinder
    dt = {"f32": torch.float32, "f16": torch.float16}[storage]
    cubes = [c.to(dt).contiguous() for c in _cubes(dev)]
    with BatchSourceFinder(SHAPES, BANK6, 3.0, (32, 32, 64), storage=storage, device=dev) as bf:
        masks, means, stds = bf.detect(cubes, stats=True)
        bf.synchronize()
    monkeypatch.setenv("SF_NO_TC", "1")
    for i, cube in enumerate(cubes):
        with SourceFinder(SHAPES[i], BANK6, 3.0, (32, 32, 64), storage=storage, device=dev) as sf:
            m1, me1, sd1 = sf.detect(cube, stats=True)
            torch.cuda.synchronize(dev)
        assert m1.any() or not masks[i].any()
        assert torch.equal(masks[i], m1), f"{storage} cube {i} {SHAPES[i]} mask"
        assert torch.equal(means[i], me1), f"{storage} cube {i} mean"
        assert torch.equal(stds[i], sd1), f"{storage} cube {i} std"


@pytest.mark.parametrize("opts", [dict(stats_fp64=True), dict(std_ddof=1)])
def test_batch_statistics_options(dev, opts):
    """The statistics options reach the persistent kernel: bit-identical to
    the per-cube path with the same options."""
    import torch
    from paper_1507_04941_gb300 import BatchSourceFinder, SourceFinder
    cubes = _cubes(dev)[:3]
    with BatchSourceFinder(SHAPES[:3], BANK6, 3.0, (32, 32, 64), device=dev, **opts) as bf:
        masks, means, stds = bf.detect(cubes, stats=True)
        bf.synchronize()
        for i, cube in enumerate(cubes):
            with SourceFinder(SHAPES[i], BANK6, 3.0, (32, 32, 64), device=dev, **opts) as sf:
                m1, me1, sd1 = sf.detect(cube, stats=True)
                torch.cuda.synchronize(dev)
            assert torch.equal(masks[i], m1), f"cube {i} mask {opts}"
            assert torch.equal(means[i], me1), f"cube {i} mean {opts}"
            assert torch.equal(stds[i], sd1), f"cube {i} std {opts}"


def test_batch_single_cube_and_no_spatial_filter(dev):
    import torch
    from paper_1507_04941_gb300 import BatchSourceFinder, SourceFinder, synth
    bank = ((0.0, 2.0), (0.0, 5.0))          # no x pass at all
    shape = (40, 40, 100)
    cube = synth.make_cube(shape, 91, 5, (1.0, 5.0), device=dev)
    with BatchSourceFinder([shape], bank, 3.0, (16, 16, 32), device=dev) as bf, \
            SourceFinder(shape, bank, 3.0, (16, 16, 32), device=dev) as sf:
        m = bf.detect([cube])[0]
        torch.cuda.synchronize(dev)
        assert torch.equal(m, sf.detect(cube))


def test_tune_keeps_results(dev):
    import json

    import torch
    from paper_1507_04941_gb300 import BatchSourceFinder, SourceFinder, synth
    shape = (256, 96, 256)
    cube = synth.make_cube(shape, 92, 30, (0.5, 5.0), 1.5, device=dev)
    with SourceFinder(shape, BANK6, 3.0, (32, 32, 64), device=dev) as sf:
        before = sf.detect(cube, stats=True)
        rep = json.loads(sf.tune(cube))
        assert rep[0]["path"].startswith("x pass") and len(rep) >= 3
        after = sf.detect(cube, stats=True)
        torch.cuda.synchronize(dev)
        for x, y in zip(before, after):
            assert torch.equal(x, y)
    cubes = _cubes(dev)
    with BatchSourceFinder(SHAPES, BANK6, 3.0, (32, 32, 64), device=dev) as bf:
        before = bf.detect(cubes)
        rep = json.loads(bf.tune(cubes))
        assert {r["path"] for r in rep} == {"persistent", "batched x pass + persistent windows"}
        after = bf.detect(cubes)
        bf.synchronize()
        for x, y in zip(before, after):
            assert torch.equal(x, y)


def test_bounded_wait_expires_and_context_recovers(dev):
    """The watchdog path: with the test hook, every window item of the
    persistent kernel waits for one x item more than its cube has, so each
    wait runs into its limit (1 ms here) and the CTA leaves; sf_synchronize
    reports SF_ETIMEOUT once.  The same context, with the hook off, then
    gives masks bit-identical to the per-cube path, and a fresh context works.
    Nothing faults: the waits are bounded spins on a counter."""
    import time

    import torch
    from paper_1507_04941_gb300 import BatchSourceFinder, SfError
    from paper_1507_04941_gb300.sf import SF_ETIMEOUT
    shapes = SHAPES[:3]
    cubes = _cubes(dev)[:3]
    with BatchSourceFinder(shapes, BANK6, 3.0, (32, 32, 64), device=dev) as bf:
        bf.set_wait_limit(1_000_000)
        bf.test_stall(1)
        t0 = time.perf_counter()
        bf.detect(cubes)
        with pytest.raises(SfError) as exc:
            bf.synchronize()
        assert exc.value.status == SF_ETIMEOUT
        assert time.perf_counter() - t0 < 10.0
        bf.synchronize()   # the flag was cleared
        bf.test_stall(0)
        bf.set_wait_limit(2_000_000_000)
        masks = bf.detect(cubes)
        bf.synchronize()
        for i, cube in enumerate(cubes):
            assert torch.equal(masks[i].cpu(), _single(dev, cube)[0]), f"cube {i} after recovery"
    with BatchSourceFinder(shapes, BANK6, 3.0, (32, 32, 64), device=dev) as bf2:
        masks = bf2.detect(cubes)
        bf2.synchronize()
        assert torch.equal(masks[0].cpu(), _single(dev, cubes[0])[0])


def test_wait_limit_and_stall_hook_arguments(dev):
    from paper_1507_04941_gb300 import BatchSourceFinder, SfError, SourceFinder
    with SourceFinder((32, 32, 64), BANK6, 3.0, (32, 32, 64), device=dev) as sf:
        with pytest.raises(SfError):
            sf.set_wait_limit(10)
        sf.set_wait_limit(5_000_000)
    with BatchSourceFinder(SHAPES[:2], BANK6, 3.0, (32, 32, 64), device=dev) as bf:
        with pytest.raises(SfError):
            bf.test_stall(-1)
