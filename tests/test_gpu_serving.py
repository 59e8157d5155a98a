"""Serving form: continuous batching with HBM-budget admission.

Each request's mask must be the same whether it runs alone or in a mix of
concurrently admitted requests (fixed reduction order: bit-identical); the
admitted footprint never exceeds the budget; a request larger than the
budget is rejected with SF_EBUDGET; evicting idle contexts keeps results."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

BANK6 = ((0.0, 2.0), (0.0, 6.0), (1.5, 2.0), (1.5, 6.0), (3.0, 2.0), (3.0, 6.0))
SHAPES = [(64, 64, 130), (40, 40, 96), (96, 96, 257), (33, 33, 200), (64, 64, 130), (72, 72, 64),
          (40, 40, 96), (128, 128, 128)]


@pytest.fixture(scope="module")
def dev():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1507_04941_gb300 import build
    build.build()
    return torch.device("cuda", 0)


def _requests(storage):
    import torch

    from paper_1507_04941_gb300 import synth
    dt = {"f16": torch.float16, "f32": torch.float32}[storage]
    cubes = [synth.make_cube(sh, 300 + i, 6, (0.5, 5.0), 1.5).to(dt).contiguous().pin_memory()
             for i, sh in enumerate(SHAPES)]
    masks = [torch.zeros((sh[0], sh[1], -(-sh[2] // 32)), dtype=torch.int32).pin_memory()
             for sh in SHAPES]
    return cubes, masks


def _alone(dev, cube, storage):
    from paper_1507_04941_gb300 import SourceFinder
    with SourceFinder(tuple(cube.shape), BANK6, 3.0, (32, 32, 64), storage=storage, device=dev) as sf:
        return sf.detect_host(cube).clone()


def _drain(srv, n, timeout=120.0):
    got, t0 = [], time.time()
    while len(got) < n and time.time() - t0 < timeout:
        got += srv.poll(timeout_ms=200)
    return got


@pytest.mark.parametrize("storage", ["f16", "f32"])
def test_mix_equals_alone(dev, storage):
    import torch
    from paper_1507_04941_gb300 import Server
    cubes, masks = _requests(storage)
    with Server(BANK6, storage=storage, budget_bytes=8 * 10 ** 9, max_inflight=4, device=0) as srv:
        ids = [srv.submit(c, m) for c, m in zip(cubes, masks)]
        done = _drain(srv, len(ids))
        assert sorted(i for i, _, _ in done) == sorted(ids)
        assert all(st == 0 for _, st, _ in done)
        assert all(lat > 0 for _, _, lat in done)
        stats = srv.stats()
        assert stats["completed"] == len(ids) and stats["rejected"] == 0
        assert stats["peak_bytes"] <= stats["budget"]
    for c, m in zip(cubes, masks):
        assert torch.equal(m, _alone(dev, c, storage))


def test_budget_admission_rejection_and_eviction(dev):
    import torch
    from paper_1507_04941_gb300 import Server
    cubes, masks = _requests("f16")

    def footprint(sh):
        # the server's accounting: cube + two x-filtered scratch cubes + mask
        up = lambda v: (v + 255) // 256 * 256  # noqa: E731
        cube = up(sh[0] * sh[1] * sh[2] * 2)
        return 3 * cube + up(sh[0] * sh[1] * (-(-sh[2] // 32)) * 4) + 4096

    # room for the largest request and a little more: admissions wait and
    # idle contexts of other shapes are evicted
    budget = int(1.5 * max(footprint(sh) for sh in SHAPES))
    with Server(BANK6, storage="f16", budget_bytes=budget, max_inflight=4, device=0) as srv:
        ids = [srv.submit(c, m) for c, m in zip(cubes, masks)]
        big = torch.zeros((512, 512, 1024), dtype=torch.float16)
        big_mask = torch.zeros((512, 512, 32), dtype=torch.int32)
        big_id = srv.submit(big, big_mask)
        done = _drain(srv, len(ids) + 1)
        st = {i: s for i, s, _ in done}
        assert st[big_id] == 3                      # SF_EBUDGET
        assert all(st[i] == 0 for i in ids)
        stats = srv.stats()
        assert stats["peak_bytes"] <= budget
        assert stats["evictions"] > 0
        assert srv.poll(timeout_ms=50) == []        # nothing pending: returns, no hang
    for c, m in zip(cubes, masks):
        assert torch.equal(m, _alone(dev, c, "f16"))
