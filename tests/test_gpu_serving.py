"""Serving (continuous batching) and the autotuner on the GPU, through the C ABI."""
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


def _read_device(ptr, m, W):
    """Copy a server-owned output (raw device pointer) into a fresh tensor."""
    import torch

    import paper_1811_00901_gb300 as spin
    view = torch.as_tensor(spin.device_view(ptr, (m, W, W)), device="cuda:0")
    return view.clone()


def _meshes(torch, spin, dev):
    out = []
    for pts, nrm in (wl.sphere(6000, 41), wl.object_scene(9000, 42, n_objects=10)):
        mesh = spin.si_mesh_create(torch.from_numpy(pts).to(dev), torch.from_numpy(nrm).to(dev))
        out.append((mesh, pts.shape[0]))
    return out


def test_served_results_equal_direct_calls_alone_and_in_the_mix():
    import torch

    import paper_1811_00901_gb300 as spin
    dev = torch.device("cuda:0")
    meshes = _meshes(torch, spin, dev)
    srv = spin.si_serve_create(4 << 30, 64)
    try:
        for mesh, _ in meshes:
            spin.si_serve_add_mesh(srv, mesh)
        rng = np.random.default_rng(7)
        reqs = []
        for k in range(200):
            mesh, n = meshes[k % 2]
            m = int(rng.integers(1, 2500))
            W = int(rng.choice([16, 32]))
            B = 0.8 / W
            c = float(rng.choice([0.0, 0.5, 0.7071]))
            q = torch.from_numpy(rng.integers(0, n, m).astype(np.int32)).to(dev)
            own = k % 3 == 0
            out = None if own else torch.full((m, W, W), -9, dtype=torch.int32, device=dev)
            t = spin.si_serve_submit(srv, dict(mesh=mesh, query_idx=q, m=m, W=W, bin_size=B, cos_s=c, out=out))
            assert t is not None
            reqs.append((t, mesh, q, m, W, B, c, out))
        lat = []
        for t, mesh, q, m, W, B, c, out in reqs:
            assert spin.si_serve_wait(srv, t, 60000)
            ptr, us = spin.si_serve_result(srv, t)
            lat.append(us)
            got = out if out is not None else _read_device(ptr, m, W)
            ref = torch.empty((m, W, W), dtype=torch.int32, device=dev)
            spin.si_generate(mesh, q, m, W, B, c, spin.make_schedule("STATIC"), ref)
            torch.cuda.synchronize()
            assert torch.equal(got, ref)
            spin.si_serve_release(srv, t)
        assert min(lat) > 0
    finally:
        spin.si_serve_destroy(srv)
        for mesh, _ in meshes:
            spin.si_mesh_destroy(mesh)


def test_admission_by_memory_and_wait_timeout():
    """A request that does not fit next to an unreleased result waits (and a
    bounded wait times out); releasing the result admits it."""
    import torch

    import paper_1811_00901_gb300 as spin
    dev = torch.device("cuda:0")
    pts, nrm = wl.sphere(4000, 3)
    mesh = spin.si_mesh_create(torch.from_numpy(pts).to(dev), torch.from_numpy(nrm).to(dev))
    budget = 24 << 20
    srv = spin.si_serve_create(budget, 8)
    try:
        spin.si_serve_add_mesh(srv, mesh)
        # ~16 MB of server-owned output: 4000 images of 32 x 32
        big = dict(mesh=mesh, query_idx=None, m=4000, W=32, bin_size=0.025, cos_s=0.5, out=None)
        t1 = spin.si_serve_submit(srv, big)
        assert spin.si_serve_wait(srv, t1, 60000)
        t2 = spin.si_serve_submit(srv, big)  # fits the budget alone, not next to t1's output
        assert spin.si_serve_wait(srv, t2, 50) is False
        assert spin.si_serve_poll(srv, t2) is False
        spin.si_serve_release(srv, t1)
        assert spin.si_serve_wait(srv, t2, 60000)
        spin.si_serve_release(srv, t2)
        # larger than the whole budget: refused at submit
        huge = dict(big, m=4000, W=64)
        assert spin.si_serve_submit(srv, huge) is None
        # a mesh the server does not know is an argument error
        other = spin.si_mesh_create(torch.from_numpy(pts).to(dev), torch.from_numpy(nrm).to(dev))
        try:
            with pytest.raises(spin.SpinError):
                spin.si_serve_submit(srv, dict(big, mesh=other))
        finally:
            spin.si_mesh_destroy(other)
    finally:
        spin.si_serve_destroy(srv)
        spin.si_mesh_destroy(mesh)


def test_in_flight_limit_of_one_still_serves_everything():
    import torch

    import paper_1811_00901_gb300 as spin
    dev = torch.device("cuda:0")
    pts, nrm = wl.heightfield(3000, 5)
    mesh = spin.si_mesh_create(torch.from_numpy(pts).to(dev), torch.from_numpy(nrm).to(dev))
    srv = spin.si_serve_create(1 << 30, 1)
    try:
        spin.si_serve_add_mesh(srv, mesh)
        outs, ts = [], []
        for k in range(12):
            q = torch.arange(k, 3000, 13, dtype=torch.int32, device=dev)
            o = torch.empty((q.numel(), 16, 16), dtype=torch.int32, device=dev)
            ts.append(spin.si_serve_submit(srv, dict(mesh=mesh, query_idx=q, m=q.numel(), W=16, bin_size=0.03,
                                                     cos_s=0.5, out=o)))
            outs.append((q, o))
        for t in ts:
            assert spin.si_serve_wait(srv, t, 60000)
        for (q, o), t in zip(outs, ts):
            ref = torch.empty_like(o)
            spin.si_generate(mesh, q, q.numel(), 16, 0.03, 0.5, spin.make_schedule("GSS"), ref)
            torch.cuda.synchronize()
            assert torch.equal(o, ref)
            spin.si_serve_release(srv, t)
    finally:
        spin.si_serve_destroy(srv)
        spin.si_mesh_destroy(mesh)


def test_tuner_records_and_batched_uses_the_table(tmp_path):
    import torch

    import paper_1811_00901_gb300 as spin
    dev = torch.device("cuda:0")
    pts, nrm = wl.heightfield(8000, 6)
    n = pts.shape[0]
    mesh = spin.si_mesh_create(torch.from_numpy(pts).to(dev), torch.from_numpy(nrm).to(dev))
    try:
        spin.si_tune_clear()
        out = torch.empty((n, 32, 32), dtype=torch.int32, device=dev)
        best, ms = spin.si_tune_mesh(mesh, None, n, 32, 0.01, 0.5, out, reps=1)
        assert ms > 0 and best.kind in (0, 1, 2, 3) and best.group in (1, 2, 4, 8, 16, 32)
        got = spin.si_tune_lookup(32, n, n)
        assert got is not None and (got.kind, got.group, got.grid_div) == (best.kind, best.group, best.grid_div)
        path = str(tmp_path / "tune.json")
        spin.si_tune_save(path)
        spin.si_tune_clear()
        assert spin.si_tune_lookup(32, n, n) is None
        spin.si_tune_load(path)
        got = spin.si_tune_lookup(32, n, n)
        assert (got.kind, got.min_chunk, got.group, got.grid_div) == (best.kind, best.min_chunk, best.group,
                                                                      best.grid_div)
        ref = torch.empty_like(out)
        spin.si_generate(mesh, None, n, 32, 0.01, 0.5, spin.make_schedule("STATIC"), ref)
        out.fill_(0)
        spin.si_generate_batched([dict(mesh=mesh, query_idx=None, m=n, W=32, bin_size=0.01, cos_s=0.5, out=out)])
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    finally:
        spin.si_tune_clear()
        spin.si_mesh_destroy(mesh)
