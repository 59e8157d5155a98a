"""sf_filter_noalloc: the filter entry point for callers that cannot allocate.

Some callers cannot call cudaMalloc (an allocation-free loop, or a host that
owns every device allocation), so they cannot create a context.  This entry
point keeps its two intermediate cubes in a fixed scratch array inside the
library.  Its output must match the context-based sf_filter, within the
filtered-value tolerance the parity tests use, on two calls in a row (the
second call reuses the scratch the first one left behind).  The file is named
so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_filter_matches_sf_filter_twice():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1507_04941_gb300 import SourceFinder, build, lib, synth
    build.build()
    dev = torch.device("cuda", 0)
    bank = ((1.5, 6.0), (3.0, 2.0))
    shapes = [(64, 48, 160), (37, 29, 91)]
    L = lib()
    for shape in shapes:
        cube = synth.make_cube(shape, 61, 8, (1.0, 5.0)).to(dev)
        with SourceFinder(shape, bank, 3.0, (16, 16, 32), device=dev) as sf:
            for f, (sxy, sz) in enumerate(bank):
                want = sf.filter(cube, f).cpu().numpy().astype(np.float64)
                A = sf.filter(cube.abs().contiguous(), f).cpu().numpy().astype(np.float64)
                out = torch.empty(shape, dtype=torch.float32, device=dev)
                for _ in range(2):
                    out.fill_(float("nan"))
                    st = L.sf_filter_noalloc(ctypes.c_void_p(cube.data_ptr()), shape[0], shape[1],
                                             shape[2], sxy, sz, 3.0,
                                             ctypes.c_void_p(out.data_ptr()),
                                             ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream))
                    assert st == 0
                    torch.cuda.synchronize(dev)
                    got = out.cpu().numpy().astype(np.float64)
                    bound = 1e-5 * np.maximum(np.abs(want), A)
                    assert (np.abs(got - want) <= bound).all(), f"shape {shape} filter {f}"


def test_noalloc_rejects_cubes_beyond_the_scratch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1507_04941_gb300 import lib
    dev = torch.device("cuda", 0)
    buf = torch.zeros(16, device=dev)
    # 8,388,609 voxels: one more than the fixed scratch holds (two FP32 cubes in 64 MiB)
    st = lib().sf_filter_noalloc(ctypes.c_void_p(buf.data_ptr()), 8388609, 1, 1, 1.0, 1.0, 3.0,
                                 ctypes.c_void_p(buf.data_ptr()), None)
    assert st == 1
    assert "exceed the fixed scratch" in lib().sf_last_error(None).decode()
