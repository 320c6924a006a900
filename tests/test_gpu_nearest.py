"""Parity of the paper-literal count (SI_BIN_NEAREST: pixel (ceil(u), ceil(v))
+= 1, Algorithm 1) with the oracle.  Both sides decide every pixel index in
IEEE FP32 with the same roundings, so the images must be equal bit for bit."""
import numpy as np
import pytest

import oracle
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


def _nearest(spin, kind="GSS", **kw):
    return spin.make_schedule(kind, binning="NEAREST", **kw)


def test_sphere_every_image_bit_exact():
    import paper_1811_00901_gb300 as spin
    c = wl.plain_sphere()
    pts, nrm = c["points"], c["normals"]
    got, pr = gpu_run(pts, nrm, 16, 0.05, 0.5, schedule=_nearest(spin), probe=True)
    ref, sup, _ = oracle.spin_images_nearest(pts, nrm, 16, 0.05, 0.5)
    np.testing.assert_array_equal(got, ref)
    np.testing.assert_array_equal(pr["support"], sup)


@pytest.mark.parametrize("W,B", [(32, 0.01), (5, 0.04), (7, 0.03), (2, 0.1), (127, 0.002), (128, 0.002)])
def test_heightfield_sampled_images_bit_exact(W, B):
    import paper_1811_00901_gb300 as spin
    pts, nrm = wl.heightfield(6000, 21)
    c = float(wl.cos_deg(60.0))
    got, _ = gpu_run(pts, nrm, W, B, c, schedule=_nearest(spin, "FAC"))
    sample = np.arange(0, 6000, 3 if W < 64 else 29).astype(np.int32)
    ref, _, _ = oracle.spin_images_nearest(pts, nrm, W, B, c, query_idx=sample)
    np.testing.assert_array_equal(got[sample], ref)


def test_query_list_with_duplicates_and_scene():
    import paper_1811_00901_gb300 as spin
    pts, nrm = wl.object_scene(20_000, 4)
    rng = np.random.default_rng(3)
    q = rng.integers(0, 20_000, 700).astype(np.int32)
    q[10:20] = q[0]
    got, _ = gpu_run(pts, nrm, 64, 0.005, 0.0, query_idx=q, schedule=_nearest(spin, "SS"))
    ref, _, _ = oracle.spin_images_nearest(pts, nrm, 64, 0.005, 0.0, query_idx=q)
    np.testing.assert_array_equal(got, ref)


def test_every_rule_shape_and_slicing_gives_the_same_counts():
    import paper_1811_00901_gb300 as spin
    pts, nrm = wl.heightfield(4000, 22)
    W, B, c = 16, 0.02, 0.5
    ref, _ = gpu_run(pts, nrm, W, B, c, schedule=_nearest(spin, "STATIC"))
    for kind in ("SS", "GSS", "FAC", "FAC_PROB"):
        for group, workers, slices in [(1, 0, 1), (4, 7, 0), (32, 300, 1), (8, 0, 5)]:
            got, _ = gpu_run(pts, nrm, W, B, c,
                             schedule=_nearest(spin, kind, group=group, num_workers=workers, slices=slices,
                                               fac_cov=1.0))
            assert np.array_equal(got, ref), (kind, group, workers, slices)


def test_small_and_empty_calls():
    import paper_1811_00901_gb300 as spin
    pts, nrm = wl.heightfield(3000, 23)
    got, _ = gpu_run(pts, nrm, 16, 0.02, 0.5, query_idx=np.array([5], np.int32), schedule=_nearest(spin))
    ref, _, _ = oracle.spin_images_nearest(pts, nrm, 16, 0.02, 0.5, query_idx=np.array([5], np.int32))
    np.testing.assert_array_equal(got, ref)
    got, _ = gpu_run(pts, nrm, 16, 0.02, 0.5, query_idx=np.zeros(0, np.int32), schedule=_nearest(spin))
    assert got.shape == (0, 16, 16)


def test_batched_nearest_equals_single_calls():
    import torch

    import paper_1811_00901_gb300 as spin
    dev = torch.device("cuda:0")
    meshes, items, refs = [], [], []
    try:
        for k, (n, W, B, cs) in enumerate([(3000, 16, 0.05, 0.5), (1500, 32, 0.025, 0.0), (800, 7, 0.1, -1.0)]):
            pts, nrm = wl.sphere(n, 40 + k)
            mh = spin.si_mesh_create(torch.from_numpy(pts).to(dev), torch.from_numpy(nrm).to(dev))
            meshes.append(mh)
            out = torch.empty((n, W, W), dtype=torch.int32, device=dev)
            items.append(dict(mesh=mh, query_idx=None, m=n, W=W, bin_size=B, cos_s=cs, out=out))
            refs.append(oracle.spin_images_nearest(pts, nrm, W, B, cs)[0])
        spin.si_generate_batched(items, _nearest(spin, "GSS"))
        torch.cuda.synchronize()
        for it, ref in zip(items, refs):
            np.testing.assert_array_equal(it["out"].cpu().numpy(), ref)
    finally:
        for mh in meshes:
            spin.si_mesh_destroy(mh)
