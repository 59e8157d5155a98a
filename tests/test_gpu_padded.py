"""The padded layout of the detect path (rows that are not 16-byte multiples).

When nz * element size is not a multiple of 16 bytes the window kernels cannot
read the cube and its x-filtered scratch cubes by TMA.  The detect path then
writes the scratch cubes with padded rows and a padded copy of the cube (an
identity output of the x pass) and reads all of them by TMA.  The arithmetic
is unchanged, so masks and window statistics must be bit-identical to the
element-wise copies of the unpadded layout (SF_NO_PAD=1), from device and from
host buffers.  The unpadded path is pinned to the FP64 oracle by the parity
tests; one case here is compared with the oracle directly as well.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

BANK6 = ((0.0, 2.0), (0.0, 6.0), (1.5, 2.0), (1.5, 6.0), (3.0, 2.0), (3.0, 6.0))
WINDOW = (32, 32, 64)


@pytest.fixture(scope="module")
def dev():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1507_04941_gb300 import build
    build.build()
    return torch.device("cuda", 0)


def _run(dev, cube, storage, host=False):
    import torch
    from paper_1507_04941_gb300 import SourceFinder
    with SourceFinder(tuple(cube.shape), BANK6, 3.0, WINDOW, storage=storage, device=dev) as sf:
        if host:
            h = cube.cpu().pin_memory()
            mask = torch.empty(sf.mask_shape, dtype=torch.int32).pin_memory()
            sf.detect_host(h, mask)
            return mask.clone(), None, None
        m, me, sd = sf.detect(cube.to(dev), stats=True)
        torch.cuda.synchronize(dev)
        return m.cpu(), me.cpu(), sd.cpu()


# nz 131 and 130 (odd and even rows) in FP32; 100 (not a multiple of 8) and
# 131 in FP16, on the CUDA-core window kernel in both layouts
@pytest.mark.parametrize("storage,shape", [("f32", (70, 45, 131)), ("f32", (40, 70, 130)),
                                           ("f16", (37, 33, 100)), ("f16", (50, 40, 131))])
def test_padded_equals_unpadded(dev, monkeypatch, storage, shape):
    import torch
    from paper_1507_04941_gb300 import synth
    dt = {"f32": torch.float32, "f16": torch.float16}[storage]
    cube = synth.make_cube(shape, 811, 12, (0.5, 5.0), 1.5).to(dt).contiguous()
    monkeypatch.setenv("SF_NO_TC", "1")
    got = _run(dev, cube, storage)
    got_h, _, _ = _run(dev, cube, storage, host=True)
    monkeypatch.setenv("SF_NO_PAD", "1")
    want = _run(dev, cube, storage)
    assert want[0].any()
    for g, w, name in zip(got, want, ("mask", "mean", "std")):
        assert torch.equal(g, w), f"{storage} {shape} {name}"
    assert torch.equal(got_h, want[0]), f"{storage} {shape} host mask"


def test_padded_matches_oracle(dev, oracle):
    """FP32, nz = 131: the padded path against the FP64 oracle (bit-exact
    wherever the oracle's decision is farther from the threshold than the
    FP32 guard band)."""
    from paper_1507_04941_gb300 import synth, words_to_bits
    shape = (40, 36, 131)
    cube = synth.make_cube(shape, 812, 10, (0.5, 5.0), 1.5)
    mask, mean, std = _run(dev, cube, "f32")
    ref = oracle.detect(cube.numpy(), BANK6, 3.0, WINDOW, 4.0)
    got = words_to_bits(mask.numpy(), shape[2])
    want = oracle.unpack_bits(ref["mask"], shape[2])
    sure = oracle.unpack_bits(ref["sure"], shape[2])
    assert want.any()
    assert not ((got != want) & sure).any()
    # the parity tests' statistics bound: 1e-5 of max(std, |mean|) per window
    scale = np.maximum(ref["std"], np.abs(ref["mean"]))
    assert (np.abs(mean.numpy() - ref["mean"]) <= 1e-5 * scale).all()
    assert (np.abs(std.numpy() - ref["std"]) <= 1e-5 * scale).all()
