"""Failure handling without a GPU fault: device allocations are made to fail
on the host (si_debug_fail_allocs), one at a time at every allocation a call
makes, and each call must return SI_ERR_OOM, give back what it had taken (the
pool's bytes in use return to where they were) and leave the library usable."""
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


def _used(spin):
    import torch
    torch.cuda.synchronize()
    return spin.si_alloc_stats()[1]


def _sweep(spin, attempt, max_fail_at=64):
    """Runs attempt() with the k-th allocation failing, k = 0, 1, ..., until an
    attempt succeeds with the injection unused.  attempt() returns a cleanup
    callable (or None) and must leave the pool as it found it after cleanup.
    Returns the number of attempts that failed."""
    failed = 0
    for k in range(max_fail_at):
        base = _used(spin)
        calls0 = spin.si_alloc_stats()[0]
        spin.si_debug_fail_allocs(k, 1)
        ok, cleanup = True, None
        try:
            cleanup = attempt()
        except spin.SpinError as e:
            assert e.status == spin.SI_ERR_OOM, str(e)
            assert "injected" in spin.si_last_error()
            ok = False
        finally:
            spin.si_debug_fail_allocs(0, 0)
        made = spin.si_alloc_stats()[0] - calls0
        if cleanup is not None:
            cleanup()
        assert _used(spin) == base, "pool bytes in use changed after failing allocation %d" % k
        if ok:
            # the call made fewer than k + 1 allocations, so nothing failed
            assert made <= k
            return failed
        failed += 1
    raise AssertionError("calls kept failing")


def _mesh_inputs(torch, n=6000, seed=21):
    pts, nrm = wl.heightfield(n, seed)
    dev = torch.device("cuda:0")
    return pts, nrm, torch.from_numpy(pts).to(dev), torch.from_numpy(nrm).to(dev)


def test_mesh_create_fails_cleanly_at_every_allocation():
    import torch

    import paper_1811_00901_gb300 as spin
    _, _, tp, tn = _mesh_inputs(torch)

    def attempt():
        mesh = spin.si_mesh_create(tp, tn)
        return lambda: spin.si_mesh_destroy(mesh)

    assert _sweep(spin, attempt) >= 3


def test_generate_fails_cleanly_at_every_allocation_and_then_works():
    import torch

    import paper_1811_00901_gb300 as spin
    pts, nrm, tp, tn = _mesh_inputs(torch)
    n, W, B, c = pts.shape[0], 32, 0.01, float(wl.cos_deg(60.0))
    dev = torch.device("cuda:0")
    q = torch.from_numpy(np.arange(0, n, 3).astype(np.int32)).to(dev)
    ref = torch.empty((q.numel(), W, W), dtype=torch.int32, device=dev)
    mesh = spin.si_mesh_create(tp, tn)
    spin.si_generate(mesh, q, q.numel(), W, B, c, spin.make_schedule("FAC"), ref)
    torch.cuda.synchronize()
    spin.si_mesh_destroy(mesh)
    out = torch.empty_like(ref)

    def attempt():
        # a fresh mesh each time, so the grid build's allocations are in the call
        mesh = spin.si_mesh_create(tp, tn)
        try:
            out.fill_(-1)
            spin.si_generate(mesh, q, q.numel(), W, B, c, spin.make_schedule("FAC"), out)
            torch.cuda.synchronize()
            spin.si_get_stats(mesh)
        except Exception:
            spin.si_mesh_destroy(mesh)
            raise
        return lambda: spin.si_mesh_destroy(mesh)

    assert _sweep(spin, attempt) >= 2
    assert torch.equal(out, ref)


def test_batched_call_fails_cleanly_at_every_allocation():
    import torch

    import paper_1811_00901_gb300 as spin
    dev = torch.device("cuda:0")
    a = _mesh_inputs(torch, 3000, 5)
    b = _mesh_inputs(torch, 4000, 6)
    ma = spin.si_mesh_create(a[2], a[3])
    mb = spin.si_mesh_create(b[2], b[3])
    try:
        oa = torch.empty((3000, 16, 16), dtype=torch.int32, device=dev)
        ob = torch.empty((4000, 32, 32), dtype=torch.int32, device=dev)
        ra, rb = torch.empty_like(oa), torch.empty_like(ob)
        spin.si_generate(ma, None, 3000, 16, 0.02, 0.5, spin.make_schedule("GSS"), ra)
        spin.si_generate(mb, None, 4000, 32, 0.01, 0.5, spin.make_schedule("GSS"), rb)
        torch.cuda.synchronize()
        stream = torch.cuda.Stream(dev)
        items = [dict(mesh=ma, query_idx=None, m=3000, W=16, bin_size=0.02, cos_s=0.5, out=oa),
                 dict(mesh=mb, query_idx=None, m=4000, W=32, bin_size=0.01, cos_s=0.5, out=ob)]

        def attempt():
            oa.fill_(-1)
            ob.fill_(-1)
            # the default stream takes the direct path, a side stream the graph cache
            spin.si_generate_batched(items, spin.make_schedule("GSS"), stream=None)
            with torch.cuda.stream(stream):
                spin.si_generate_batched(items, spin.make_schedule("GSS"), stream=stream)
            torch.cuda.synchronize()
            return None

        # both meshes' grids exist (the reference calls built them), so the pool
        # returns to its level after each attempt except for a cached graph's
        # scratch, which lives until its meshes go
        base = _used(spin)
        failed = 0
        for k in range(64):
            spin.si_debug_fail_allocs(k, 1)
            ok = True
            try:
                attempt()
            except spin.SpinError as e:
                assert e.status == spin.SI_ERR_OOM
                ok = False
            finally:
                spin.si_debug_fail_allocs(0, 0)
            torch.cuda.synchronize()
            if ok:
                break
            assert _used(spin) == base
            failed += 1
        assert failed >= 1
        assert torch.equal(oa, ra) and torch.equal(ob, rb)
    finally:
        spin.si_mesh_destroy(ma)
        spin.si_mesh_destroy(mb)
    # destroying the meshes drops the cached graph and its scratch
    assert _used(spin) <= base


def test_host_buffer_path_fails_cleanly_at_every_allocation():
    import torch

    import paper_1811_00901_gb300 as spin
    pts, nrm = wl.sphere(2000, 4)
    hp, hn = torch.from_numpy(pts), torch.from_numpy(nrm)
    W = 16
    ref = torch.empty((2000, W, W), dtype=torch.int32)
    spin.si_generate_host(hp, hn, 2000, None, 2000, W, 0.05, 0.5, spin.make_schedule("SS"), ref)
    out = torch.empty_like(ref)

    def attempt():
        out.fill_(-1)
        spin.si_generate_host(hp, hn, 2000, None, 2000, W, 0.05, 0.5, spin.make_schedule("SS"), out)
        return None

    assert _sweep(spin, attempt) >= 3
    assert torch.equal(out, ref)


def test_match_fails_cleanly_at_every_allocation():
    import torch

    import paper_1811_00901_gb300 as spin
    dev = torch.device("cuda:0")
    pts, nrm = wl.heightfield(3000, 8)
    imgs = torch.empty((3000, 16, 16), dtype=torch.int32, device=dev)
    mesh = spin.si_mesh_create(torch.from_numpy(pts).to(dev), torch.from_numpy(nrm).to(dev))
    spin.si_generate(mesh, None, 3000, 16, 0.02, 0.5, spin.make_schedule("GSS"), imgs)
    torch.cuda.synchronize()
    spin.si_mesh_destroy(mesh)
    k = 3
    ri = torch.empty((500, k), dtype=torch.int32, device=dev)
    rc = torch.empty((500, k), dtype=torch.float32, device=dev)
    spin.si_match(imgs[:500], 500, imgs, 3000, 16, k, spin.SI_MATCH_FP32, ri, rc)
    bi, bc = torch.empty_like(ri), torch.empty_like(rc)

    def attempt():
        bi.fill_(-1)
        spin.si_match(imgs[:500], 500, imgs, 3000, 16, k, spin.SI_MATCH_FP32, bi, bc)
        torch.cuda.synchronize()
        return None

    assert _sweep(spin, attempt) >= 1
    assert torch.equal(bi, ri)


def test_injection_arguments():
    import paper_1811_00901_gb300 as spin
    with pytest.raises(spin.SpinError) as e:
        spin.si_debug_fail_allocs(-1, 1)
    assert e.value.status == spin.SI_ERR_INVALID
    spin.si_debug_fail_allocs(0, 0)
