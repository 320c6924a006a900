"""si_generate_noalloc: the entry point for callers that must not allocate
device memory during a call (their device memory is fully reserved by
another allocator, or their loop runs with a fixed footprint).  It keeps its
scratch in a static device array instead of the stream-ordered pool, so its
images must equal those of si_generate, call after call.

This file is collected last on purpose, so that a run that stops at the first
failure has already run every other test.
"""
import numpy as np
import pytest

from paper_1811_00901_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_00901_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)


def test_no_alloc_matches_allocating_entry_point_twice():
    import torch

    import paper_1811_00901_gb300 as spin
    dev = torch.device("cuda:0")
    pts, nrm = wl.heightfield(20000, 606)
    W, B, c = 32, 0.01, float(wl.cos_deg(60.0))
    n = pts.shape[0]
    mesh = spin.si_mesh_create(torch.from_numpy(pts).to(dev), torch.from_numpy(nrm).to(dev))
    try:
        sched_a = spin.make_schedule("GSS")
        sched_b = spin.make_schedule("FAC", min_chunk=2, group=8)
        spin.si_mesh_prepare(mesh, W, B, sched_a)
        spin.si_mesh_prepare(mesh, W, B, sched_b)
        rng = np.random.default_rng(3)
        q = torch.from_numpy(rng.integers(0, n, 3001).astype(np.int32)).to(dev)

        # reference images from the allocating entry point
        ref_all = torch.empty((n, W, W), dtype=torch.int32, device=dev)
        spin.si_generate(mesh, None, n, W, B, c, sched_a, ref_all)
        ref_q = torch.empty((3001, W, W), dtype=torch.int32, device=dev)
        spin.si_generate(mesh, q, 3001, W, B, c, sched_b, ref_q)

        # two calls in a row through the allocation-free entry point; the
        # library's allocation count and the pool's bytes in use must not move
        out1 = torch.full((n, W, W), -3, dtype=torch.int32, device=dev)
        out2 = torch.full((3001, W, W), -3, dtype=torch.int32, device=dev)
        torch.cuda.synchronize()
        calls0, used0, _ = spin.si_alloc_stats()
        spin.si_generate_noalloc(mesh, None, n, W, B, c, sched_a, out1)
        spin.si_generate_noalloc(mesh, q, 3001, W, B, c, sched_b, out2)
        torch.cuda.synchronize()
        calls1, used1, _ = spin.si_alloc_stats()
        assert calls1 == calls0
        assert used1 == used0
        spin.si_get_stats(mesh)

        # GPU-against-GPU results are compared bit for bit (the tolerance every
        # schedule comparison in these tests uses)
        assert torch.equal(out1, ref_all)
        assert torch.equal(out2, ref_q)
        # and, as a plain numeric check, within the oracle tolerance of 1e-4 L1/total
        a = out2.double() / 65536.0
        r = ref_q.double() / 65536.0
        l1 = (a - r).abs().sum((1, 2))
        assert bool((l1 <= 1e-4 * r.sum((1, 2)).clamp(min=1.0)).all())
    finally:
        spin.si_mesh_destroy(mesh)


@pytest.mark.parametrize("kind,min_chunk", [("STATIC", 1), ("SS", 1), ("SS", 3)])
def test_no_alloc_static_and_ss_on_a_prefix(kind, min_chunk):
    """STATIC and SS build their chunk tables with all threads of the set-up
    kernel (GSS and FAC with one); both on a call for the first m < n points
    (no query list), bit for bit against si_generate, twice in a row, with no
    allocation."""
    import torch

    import paper_1811_00901_gb300 as spin
    dev = torch.device("cuda:0")
    pts, nrm = wl.heightfield(12000, 91)
    W, B, c = 32, 0.01, float(wl.cos_deg(60.0))
    m = 5003
    mesh = spin.si_mesh_create(torch.from_numpy(pts).to(dev), torch.from_numpy(nrm).to(dev))
    try:
        sched = spin.make_schedule(kind, min_chunk=min_chunk, group=8)
        spin.si_mesh_prepare(mesh, W, B, sched)
        ref = torch.empty((m, W, W), dtype=torch.int32, device=dev)
        spin.si_generate(mesh, None, m, W, B, c, sched, ref)
        outs = [torch.full((m, W, W), -5, dtype=torch.int32, device=dev) for _ in range(2)]
        torch.cuda.synchronize()
        calls0, used0, _ = spin.si_alloc_stats()
        for o in outs:
            spin.si_generate_noalloc(mesh, None, m, W, B, c, sched, o)
        torch.cuda.synchronize()
        calls1, used1, _ = spin.si_alloc_stats()
        assert (calls1, used1) == (calls0, used0)
        spin.si_get_stats(mesh)
        for o in outs:
            assert torch.equal(o, ref)
    finally:
        spin.si_mesh_destroy(mesh)


def test_no_alloc_rejects_what_it_cannot_do_without_allocating():
    import torch

    import paper_1811_00901_gb300 as spin
    dev = torch.device("cuda:0")
    pts, nrm = wl.sphere(3000, 17)
    mesh = spin.si_mesh_create(torch.from_numpy(pts).to(dev), torch.from_numpy(nrm).to(dev))
    try:
        out = torch.empty((3000, 16, 16), dtype=torch.int32, device=dev)
        # no grid prepared for this resolution: it would have to be allocated
        with pytest.raises(spin.SpinError) as e:
            spin.si_generate_noalloc(mesh, None, 3000, 16, 0.05, 0.5, spin.make_schedule("GSS", grid_div=7), out)
        assert e.value.status == spin.SI_ERR_INVALID
        # more scheduling steps than the static scratch holds
        spin.si_mesh_prepare(mesh, 16, 0.05)
        with pytest.raises(spin.SpinError) as e:
            spin.si_generate_noalloc(mesh, None, 3000, 16, 0.05, 0.5,
                                     spin.make_schedule("STATIC", num_workers=200000), out)
        assert e.value.status == spin.SI_ERR_INVALID
        assert "scratch" in spin.si_last_error()
        # SS with one image per group over a 150,000-entry query list: 150,000
        # steps, refused before any work (the output is full size all the same)
        q = torch.randint(0, 3000, (150000,), dtype=torch.int32, device=dev)
        big_out = torch.empty((150000, 16, 16), dtype=torch.int32, device=dev)
        with pytest.raises(spin.SpinError) as e:
            spin.si_generate_noalloc(mesh, q, 150000, 16, 0.05, 0.5, spin.make_schedule("SS", group=1), big_out)
        assert e.value.status == spin.SI_ERR_INVALID
        assert "scratch" in spin.si_last_error()
        # a group's candidate stream split over several blocks needs a zeroed
        # output and per-image counts: not offered here
        with pytest.raises(spin.SpinError) as e:
            spin.si_generate_noalloc(mesh, None, 3000, 16, 0.05, 0.5, spin.make_schedule("GSS", slices=2), out)
        assert e.value.status == spin.SI_ERR_INVALID
        assert "slice" in spin.si_last_error()
        # the cost order needs scratch for its estimate and its sort: refused
        with pytest.raises(spin.SpinError) as e:
            spin.si_generate_noalloc(mesh, None, 3000, 16, 0.05, 0.5, spin.make_schedule("FAC", order=1), out)
        assert e.value.status == spin.SI_ERR_INVALID
        assert "order" in spin.si_last_error()
    finally:
        spin.si_mesh_destroy(mesh)
