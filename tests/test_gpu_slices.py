"""Candidate slices: several blocks share one group's candidate stream and add
their partial images into the output with integer atomics.  Images must be
bit-identical to unsliced generation, and the exact overflow check must still
see the summed pixels."""
import numpy as np
import pytest

from paper_1811_00901_gb300 import workloads as wl

from spin_testlib import compare_with_oracle, gpu_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_00901_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)


def test_slices_are_bit_identical_to_whole_groups():
    import paper_1811_00901_gb300 as spin
    pts, nrm = wl.heightfield(5000, 19)
    W, B, c = 32, 0.01, float(wl.cos_deg(60.0))
    ref, _ = gpu_run(pts, nrm, W, B, c, schedule=spin.make_schedule("STATIC", slices=1))
    for kind in ("STATIC", "SS", "GSS", "FAC"):
        for slices in (2, 3, 7, 64, 0):
            got, _ = gpu_run(pts, nrm, W, B, c, schedule=spin.make_schedule(kind, slices=slices))
            assert np.array_equal(got, ref), (kind, slices)


def test_small_request_on_a_big_mesh_is_sliced_and_exact():
    """A few queries on a large mesh: the automatic rule slices every group."""
    import paper_1811_00901_gb300 as spin
    pts, nrm = wl.sphere(120_000, 23)
    q = np.array([5, 77, 1000, 99_999, 5], np.int32)
    W, B, c = 16, 0.05, 0.5
    auto, _ = gpu_run(pts, nrm, W, B, c, query_idx=q)
    whole, _ = gpu_run(pts, nrm, W, B, c, query_idx=q, schedule=spin.make_schedule("GSS", slices=1))
    np.testing.assert_array_equal(auto, whole)
    compare_with_oracle(auto, pts, nrm, W, B, c, q, np.arange(len(q)))


def test_overflow_is_detected_across_slices():
    """40,000 coincident points: each slice's partial pixel fits in int32, the
    sum does not; the check after the kernel must flag it.  30,000 must not."""
    import torch

    import paper_1811_00901_gb300 as spin
    dev = torch.device("cuda:0")
    for n, expect in ((40000, spin.SI_ERR_OVERFLOW), (30000, spin.SI_OK)):
        pts = np.zeros((n, 3), np.float32)
        nrm = np.tile(np.array([[0, 0, 1]], np.float32), (n, 1))
        mesh = spin.si_mesh_create(torch.from_numpy(pts).to(dev), torch.from_numpy(nrm).to(dev))
        try:
            out = torch.empty((1, 8, 8), dtype=torch.int32, device=dev)
            spin.si_generate(mesh, torch.tensor([3], dtype=torch.int32, device=dev), 1, 8, 0.1, 0.0,
                             spin.make_schedule("GSS", slices=9), out)
            torch.cuda.synchronize()
            _, status = spin.si_get_stats(mesh, raise_on_flags=False)
            assert status == expect, n
        finally:
            spin.si_mesh_destroy(mesh)


def test_probes_use_whole_groups():
    import paper_1811_00901_gb300 as spin
    pts, nrm = wl.sphere(3000, 29)
    q = np.arange(0, 3000, 300).astype(np.int32)
    a, pa = gpu_run(pts, nrm, 16, 0.05, 0.5, query_idx=q, probe=True, schedule=spin.make_schedule("SS", slices=8))
    b, pb = gpu_run(pts, nrm, 16, 0.05, 0.5, query_idx=q, probe=True, schedule=spin.make_schedule("SS", slices=1))
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(pa["support"], pb["support"])
    np.testing.assert_array_equal(pa["culled"], pb["culled"])
