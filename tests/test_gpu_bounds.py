"""The bounds-checking build (libspin_gb300_bounds.so: the spin kernel compiled
with SI_DEBUG_BOUNDS, whose index checks of shared and global accesses flag
and skip a bad access instead of trapping) on small cases of every path: no
check may fire, and the images must equal the normal build's bit for bit.
This stands in for a memory checker, which this GPU pool does not offer."""
import os

import numpy as np
import pytest

from paper_1811_00901_gb300 import workloads as wl

from spin_testlib import gpu_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_00901_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)


def _with_bounds_lib(fn):
    """Runs fn with every binding call going to the bounds-checking library."""
    import paper_1811_00901_gb300._binding as b
    from paper_1811_00901_gb300 import _build
    assert os.path.exists(_build.LIB_BOUNDS)
    old = b.load()
    b._lib = b.load(_build.LIB_BOUNDS)
    try:
        return fn()
    finally:
        b._lib = old


def _both(fn):
    """fn() with the normal build and with the bounds-checking build."""
    ref = fn()
    chk = _with_bounds_lib(fn)
    return ref, chk


CASES = {
    # (points, normals) generator, W, B, cos S, query list or None, schedule kwargs
    "sphere-W16-groups-of-32": (lambda: wl.sphere(4096, 3), 16, 0.05, 0.5, None, dict(kind="SS")),
    "heightfield-W32-FAC": (lambda: wl.heightfield(6000, 77), 32, 0.01, 0.5, None, dict(kind="FAC")),
    "heightfield-W32-query-list": (lambda: wl.heightfield(6000, 78), 32, 0.01, 0.5,
                                   np.r_[np.arange(0, 6000, 7), [5, 5, 5999]].astype(np.int32), dict(kind="GSS")),
    "heightfield-W32-five-queries-sliced": (lambda: wl.heightfield(20000, 79), 32, 0.01, 0.5,
                                            np.array([3, 900, 17000, 17001, 42], np.int32), dict(kind="GSS")),
    "scene-W64-producer-ring": (lambda: wl.object_scene(20000, 31), 64, 0.005, 0.0,
                                np.arange(0, 20000, 29).astype(np.int32), dict(kind="FAC")),
    "W5-runtime-shape": (lambda: wl.object_scene(3000, 8, n_objects=6), 5, 0.1, -1.0, None, dict(kind="GSS")),
    "W127-runtime-shape": (lambda: wl.object_scene(3000, 8, n_objects=6), 127, 0.004, 0.5,
                           np.arange(0, 3000, 11).astype(np.int32), dict(kind="SS")),
    "nearest-bin-W32": (lambda: wl.heightfield(6000, 80), 32, 0.01, 0.5, None, dict(kind="FAC", binning="NEAREST")),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_bounds_build_matches_and_flags_nothing(name):
    import paper_1811_00901_gb300 as spin
    gen, W, B, c, q, sk = CASES[name]
    pts, nrm = gen()

    def run():
        imgs, pr = gpu_run(pts, nrm, W, B, c, query_idx=q, schedule=spin.make_schedule(**sk), probe=False)
        return imgs

    # gpu_run reads si_get_stats, which raises on any device flag (a failed
    # index check included), before it returns the images
    ref, chk = _both(run)
    np.testing.assert_array_equal(chk, ref)


def test_bounds_build_probe_batched_and_no_alloc():
    """Probes, a batched launch mixing both ring disciplines and the wide
    instance (W = 128), and the allocation-free entry point."""
    import torch

    import paper_1811_00901_gb300 as spin
    dev = torch.device("cuda:0")
    specs = [(wl.sphere(3000, 5), 16, 0.05, 0.5), (wl.heightfield(4000, 6), 32, 0.01, 0.5),
             (wl.object_scene(5000, 7, n_objects=8), 64, 0.005, 0.0), (wl.object_scene(2000, 9, n_objects=4), 128,
                                                                       0.004, 0.5)]

    def run():
        meshes, items, outs = [], [], []
        try:
            for (pts, nrm), W, B, c in specs:
                mesh = spin.si_mesh_create(torch.from_numpy(pts).to(dev), torch.from_numpy(nrm).to(dev))
                meshes.append(mesh)
                m = min(pts.shape[0], 700)
                o = torch.full((m, W, W), -1, dtype=torch.int32, device=dev)
                outs.append(o)
                items.append(dict(mesh=mesh, query_idx=None, m=m, W=W, bin_size=B, cos_s=c, out=o))
            spin.si_generate_batched(items, spin.make_schedule("GSS"))
            # probes on the first mesh
            m0 = items[0]["m"]
            po = torch.empty_like(outs[0])
            cnt = {k: torch.zeros(m0, dtype=torch.int64, device=dev) for k in ("culled", "support", "angle")}
            spin.si_generate_probe(meshes[0], None, m0, 16, 0.05, 0.5, spin.make_schedule("FAC"), po, **cnt)
            # the allocation-free entry point on the second mesh
            na = torch.empty_like(outs[1])
            spin.si_mesh_prepare(meshes[1], 32, 0.01)
            spin.si_generate_noalloc(meshes[1], None, items[1]["m"], 32, 0.01, 0.5, spin.make_schedule("SS"), na)
            torch.cuda.synchronize()
            for mesh in meshes:
                spin.si_get_stats(mesh)
            return [o.cpu().numpy() for o in outs] + [po.cpu().numpy(), na.cpu().numpy()] + \
                [v.cpu().numpy() for v in cnt.values()]
        finally:
            for mesh in meshes:
                spin.si_mesh_destroy(mesh)

    ref, chk = _both(run)
    for a, b in zip(ref, chk):
        np.testing.assert_array_equal(b, a)
