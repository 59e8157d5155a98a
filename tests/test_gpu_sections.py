"""Sectioned detect (Sec. 3.1: a cube larger than device memory cut along x
into sections with a halo) against the whole-cube detect on the same cube:
the masks must agree bit for bit, since every section sees exactly the planes
the whole-cube x pass reads and every statistics window lies in one section."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

BANK = ((0.0, 2.0), (1.5, 3.0), (3.0, 1.0))   # x radii 0, 5, 9: halo 16 for wx = 16


@pytest.fixture(scope="module")
def dev():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1507_04941_gb300 import build
    build.build()
    return torch.device("cuda", 0)


@pytest.mark.parametrize("shape,section,bank", [
    ((200, 40, 96), 64, BANK),          # four sections, the last one short
    ((205, 40, 96), 48, BANK),          # nx not a multiple of wx: last-section context
    ((96, 24, 70), 32, ((0.0, 2.0),)),  # no x filter: no halo; nz ragged
    ((60, 32, 64), 64, BANK),           # one section holds the cube
    ((130, 36, 64), 16, BANK),          # halo wider than the section
    ((150, 40, 101), 64, BANK),         # rows not 16-byte multiples: the padded layout
])
def test_sections_match_whole_cube(dev, shape, section, bank):
    import torch
    from paper_1507_04941_gb300 import SectionedSourceFinder, SourceFinder, synth
    cube = synth.make_cube(shape, 51, 12, (1.0, 5.0), None)
    window = (16, 16, 32)
    with SourceFinder(shape, bank, 3.0, window, k=3.0, device=dev) as sf:
        want = sf.detect(cube.to(dev))
        torch.cuda.synchronize(dev)
        want = want.cpu().numpy()
    h_cube = cube.contiguous().pin_memory()
    with SectionedSourceFinder(shape, bank, 3.0, window, k=3.0, section=section, device=dev) as ss:
        got = ss.detect_host(h_cube).numpy()
        again = ss.detect_host(h_cube).numpy()
    assert want.any()
    np.testing.assert_array_equal(got, want)
    np.testing.assert_array_equal(again, want)


def test_sectioned_context_refuses_device_entry_points(dev):
    import ctypes
    from paper_1507_04941_gb300 import SectionedSourceFinder, sf
    with SectionedSourceFinder((64, 16, 32), ((1.0, 2.0),), 3.0, (16, 16, 32), section=32,
                               device=dev) as ss:
        assert sf.lib().sf_detect(ss._h, None, None, None, None, None) == sf.SF_EINVAL
        n = ctypes.c_int64()
        assert sf.lib().sf_mask_words(ss._h, ctypes.byref(n)) in (sf.SF_EINVAL, sf.SF_OK)


def test_sections_sample_std(dev):
    """std_ddof = 1 reaches the section contexts."""
    import torch
    from paper_1507_04941_gb300 import SectionedSourceFinder, SourceFinder, synth
    shape = (130, 40, 96)
    cube = synth.make_cube(shape, 53, 12, (1.0, 5.0), None)
    window = (16, 16, 32)
    with SourceFinder(shape, BANK, 3.0, window, k=3.0, device=dev, std_ddof=1) as sf:
        want = sf.detect(cube.to(dev))
        torch.cuda.synchronize(dev)
        want = want.cpu().numpy()
    with SectionedSourceFinder(shape, BANK, 3.0, window, k=3.0, section=32, device=dev,
                               std_ddof=1) as ss:
        got = ss.detect_host(cube.contiguous().pin_memory()).numpy()
    np.testing.assert_array_equal(got, want)


def test_sections_fp16_storage(dev):
    """16-bit storage: the sections hold the cube in FP16 like the context."""
    import torch
    from paper_1507_04941_gb300 import SectionedSourceFinder, SourceFinder, synth
    shape = (150, 40, 96)
    cube = synth.make_cube(shape, 52, 12, (1.0, 5.0), None).to(torch.float16)
    window = (16, 16, 32)
    with SourceFinder(shape, BANK, 3.0, window, k=3.0, storage="f16", device=dev) as sf:
        want = sf.detect(cube.to(dev))
        torch.cuda.synchronize(dev)
        want = want.cpu().numpy()
    with SectionedSourceFinder(shape, BANK, 3.0, window, k=3.0, section=48, storage="f16",
                               device=dev) as ss:
        got = ss.detect_host(cube.contiguous().pin_memory()).numpy()
    assert want.any()
    np.testing.assert_array_equal(got, want)


def test_sections_tile_workload(dev):
    """The bench's tile workload (512x512x1024, six filters, 32x32x64 windows)
    in 128-plane sections: bit-identical to the whole-cube detect."""
    import torch
    from paper_1507_04941_gb300 import SectionedSourceFinder, SourceFinder, synth
    w = synth.TILE
    cube = synth.make(w, device=dev)
    with SourceFinder(w.shape, w.bank, w.truncation, w.window, w.k, device=dev) as sf:
        want = sf.detect(cube)
        torch.cuda.synchronize(dev)
        want = want.cpu().numpy()
    h_cube = cube.cpu().pin_memory()
    del cube
    with SectionedSourceFinder(w.shape, w.bank, w.truncation, w.window, w.k, section=128,
                               device=dev) as ss:
        got = ss.detect_host(h_cube).numpy()
    assert want.any()
    np.testing.assert_array_equal(got, want)
