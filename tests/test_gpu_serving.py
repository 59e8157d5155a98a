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


def test_cancel_queued_requests(dev):
    """With one slot, later requests wait in the queue: cancelling them
    completes them at once with SF_ECANCELED and leaves their masks untouched;
    a request already admitted cannot be cancelled and runs to its end."""
    import torch
    from paper_1507_04941_gb300 import Server
    from paper_1507_04941_gb300.sf import SF_ECANCELED
    cubes, masks = _requests("f16")
    for m in masks:
        m.fill_(-1)
    with Server(BANK6, storage="f16", budget_bytes=8 * 10 ** 9, max_inflight=1, device=0) as srv:
        ids = [srv.submit(c, m) for c, m in zip(cubes, masks)]
        cancelled = {i for i in ids[4:] if srv.cancel(i)}
        assert cancelled, "queued requests behind one slot must be cancellable"
        assert not srv.cancel(ids[4]) or ids[4] not in cancelled   # not twice
        done = _drain(srv, len(ids))
        st = {i: s for i, s, _ in done}
        assert sorted(st) == sorted(ids)
        for i, c, m in zip(ids, cubes, masks):
            if i in cancelled:
                assert st[i] == SF_ECANCELED
                assert bool((m == -1).all()), "a cancelled request's mask must stay untouched"
            else:
                assert st[i] == 0
                assert torch.equal(m, _alone(dev, c, "f16"))
        assert srv.stats()["cancelled"] == len(cancelled)
        assert not srv.cancel(10 ** 9)                   # unknown id


def test_served_sample_matches_oracle(dev, oracle):
    """A seeded sample of requests served together, each mask against the
    FP64 oracle on its FP16-rounded cube: bit-exact wherever the oracle's
    decision is certain (|c - T| beyond 1e-3 sigma + (2^-11 + 1e-5) A plus
    the 1e-4 std guard band, A the filter of |d|); the disagreements inside
    that band are counted and printed."""
    import torch
    from paper_1507_04941_gb300 import Server, synth, words_to_bits
    rng = np.random.default_rng(99)
    shapes = [(int(s), int(s), int(L)) for s, L in zip(rng.integers(24, 72, 6), rng.integers(64, 260, 6))]
    cubes = [synth.make_cube(sh, 900 + i, 5, (0.5, 5.0), 1.5).to(torch.float16).contiguous().pin_memory()
             for i, sh in enumerate(shapes)]
    masks = [torch.zeros((sh[0], sh[1], -(-sh[2] // 32)), dtype=torch.int32).pin_memory() for sh in shapes]
    with Server(BANK6, storage="f16", budget_bytes=8 * 10 ** 9, max_inflight=4, device=0) as srv:
        ids = [srv.submit(c, m) for c, m in zip(cubes, masks)]
        done = _drain(srv, len(ids))
        assert all(s == 0 for _, s, _ in done)
    eps = 2.0 ** -11
    n_dis = n_unsure = n_fire = 0
    for sh, c, m in zip(shapes, cubes, masks):
        d_q = c.float().numpy()
        ref = oracle.detect(d_q, BANK6, 3.0, (32, 32, 64), 4.0)
        want = oracle.unpack_bits(ref["mask"], sh[2])
        got = words_to_bits(m.numpy(), sh[2])
        unsure = np.zeros(sh, dtype=bool)
        sure_fire = np.zeros(sh, dtype=bool)
        wi = [np.arange(n) // w for n, w in zip(sh, (32, 32, 64))]
        for f, (sxy, sz) in enumerate(BANK6):
            cf = oracle.filter_box(d_q, sxy, sz, 3.0)
            A = oracle.filter_box(d_q, sxy, sz, 3.0, take_abs=True)
            mb = ref["mean"][f][np.ix_(*wi)]
            sb = ref["std"][f][np.ix_(*wi)]
            dlt = cf - (mb + 4.0 * sb)
            band = 1e-3 + (eps + 1e-5) * A + 1e-4 * sb
            unsure |= np.abs(dlt) < band
            sure_fire |= dlt >= band
        certain = sure_fire | ~unsure
        assert not ((got != want) & certain).any(), f"request {sh}"
        n_dis += int((got != want).sum())
        n_unsure += int((~certain).sum())
        n_fire += int(want.sum())
    assert n_fire > 0
    print(f"\n[serving f16] {len(shapes)} requests: {n_fire} oracle detections, {n_unsure} voxels in "
          f"the precision band, {n_dis} disagreements")
