"""The cost order of the groups (si_schedule.order = 1): the dynamic rules hand
out the groups in decreasing estimated cost (the candidates of each group's
stencil).  Only the order of the work changes: every image must equal the
grid-order images bit for bit, each image must come from exactly one claim, and
the claims must follow the estimated cost."""
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


@pytest.mark.parametrize("kind", ["SS", "GSS", "FAC", "FAC_PROB", "AWF", "AF"])
def test_cost_order_changes_no_image(kind):
    import paper_1811_00901_gb300 as spin
    pts, nrm = wl.heightfield(6000, 91)
    W, B, c = 32, 0.01, wl.cos_deg(60.0)
    ref, _ = gpu_run(pts, nrm, W, B, c, schedule=spin.make_schedule("STATIC"))
    img, _ = gpu_run(pts, nrm, W, B, c, schedule=spin.make_schedule(kind, order=1, fac_cov=0.5))
    np.testing.assert_array_equal(img, ref)


@pytest.mark.parametrize("group,slices", [(8, 1), (16, 3), (1, 0), (32, 1)])
def test_cost_order_query_lists_and_slices(group, slices):
    """A query list with duplicates (sorted by the query sort, then ordered by
    cost), candidate slices and every group size."""
    import paper_1811_00901_gb300 as spin
    pts, nrm = wl.object_scene(20_000, 44, n_objects=12)
    rng = np.random.default_rng(group)
    q = np.r_[rng.choice(20_000, 1500, replace=False), [7, 7, 19_999]].astype(np.int32)
    W, B, c = 16, 0.02, 0.5
    ref, _ = gpu_run(pts, nrm, W, B, c, query_idx=q, schedule=spin.make_schedule("STATIC", group=group))
    img, _ = gpu_run(pts, nrm, W, B, c, query_idx=q,
                     schedule=spin.make_schedule("FAC", group=group, slices=slices, order=1))
    np.testing.assert_array_equal(img, ref)


def test_claims_follow_the_estimated_cost():
    """SS with one group per claim: the probe's examined count of an image is
    its group's stencil length, the quantity the order is built from; along
    the claims it must not increase by more than the bucket width (2^(1/32),
    one bucket of rounding either way), and every image comes from one claim."""
    import paper_1811_00901_gb300 as spin
    pts, nrm = wl.heightfield(20_000, 92)
    W, B, c = 32, 0.01, wl.cos_deg(60.0)
    group = 8
    import torch
    dev = torch.device("cuda:0")
    mesh = spin.si_mesh_create(torch.from_numpy(pts).to(dev), torch.from_numpy(nrm).to(dev))
    try:
        m = 20_000
        out = torch.empty((m, W, W), dtype=torch.int32, device=dev)
        step = torch.full((m,), -1, dtype=torch.int32, device=dev)
        examined = torch.full((m,), -1, dtype=torch.int64, device=dev)
        spin.si_generate_probe(mesh, None, m, W, B, c, spin.make_schedule("SS", group=group, order=1), out,
                               step=step, examined=examined)
        torch.cuda.synchronize()
        spin.si_get_stats(mesh)
        step, examined = step.cpu().numpy(), examined.cpu().numpy()
    finally:
        spin.si_mesh_destroy(mesh)
    assert (step >= 0).all()
    groups = -(-m // group)
    assert step.max() == groups - 1
    per_step = np.bincount(step, minlength=groups)
    assert per_step.sum() == m and (per_step[:-1] > 0).all()
    cost = np.zeros(groups)
    for s in range(groups):
        e = np.unique(examined[step == s])
        assert len(e) == 1  # one group per claim: all its images stream the same candidates
        cost[s] = e[0]
    later_max = np.maximum.accumulate(cost[::-1])[::-1]  # the costliest group at or after each claim
    assert np.all(cost >= later_max * 2.0 ** (-2.0 / 32) - 1), np.argmin(cost - later_max)
    assert cost[0] > 2 * np.median(cost)  # the heightfield's density varies: the order is not flat


def test_batched_items_in_cost_order():
    """One launch over items of three widths (and an empty one), each item's
    groups in its own cost order."""
    import torch

    import paper_1811_00901_gb300 as spin
    dev = torch.device("cuda:0")
    meshes, items, refs = [], [], []
    try:
        for k, (n, W, B, cs) in enumerate([(3000, 16, 0.05, 0.5), (1500, 32, 0.025, 0.0), (0, 16, 0.05, 0.5),
                                           (2500, 64, 0.01, 0.0)]):
            pts, nrm = wl.sphere(max(n, 10), 70 + k)
            mh = spin.si_mesh_create(torch.from_numpy(pts).to(dev), torch.from_numpy(nrm).to(dev))
            meshes.append(mh)
            out = torch.empty((n, W, W), dtype=torch.int32, device=dev)
            items.append(dict(mesh=mh, query_idx=None, m=n, W=W, bin_size=B, cos_s=cs, out=out))
            refs.append(gpu_run(pts, nrm, W, B, cs, m=n, schedule=spin.make_schedule("STATIC"))[0])
        for kind in ("FAC", "AWF"):
            for it in items:
                it["out"].fill_(-1)
            spin.si_generate_batched(items, spin.make_schedule(kind, order=1))
            torch.cuda.synchronize()
            for it, ref in zip(items, refs):
                np.testing.assert_array_equal(it["out"].cpu().numpy(), ref)
    finally:
        for mh in meshes:
            spin.si_mesh_destroy(mh)


def test_fac_batches_deal_the_costliest_groups():
    """FAC in cost order: within each batch of equal chunks the cost-sorted
    groups are dealt round-robin, so the chunks of the first batch (the
    costliest groups) carry nearly equal work, and the batches' groups get
    cheaper along the loop.  Every image still comes from exactly one claim."""
    import torch

    import paper_1811_00901_gb300 as spin
    pts, nrm = wl.heightfield(20_000, 93)
    W, B, c = 32, 0.01, wl.cos_deg(60.0)
    group, P, m = 8, 64, 20_000
    dev = torch.device("cuda:0")
    mesh = spin.si_mesh_create(torch.from_numpy(pts).to(dev), torch.from_numpy(nrm).to(dev))
    try:
        out = torch.empty((m, W, W), dtype=torch.int32, device=dev)
        step = torch.full((m,), -1, dtype=torch.int32, device=dev)
        examined = torch.full((m,), -1, dtype=torch.int64, device=dev)
        sched = spin.make_schedule("FAC", group=group, num_workers=P, order=1)
        spin.si_generate_probe(mesh, None, m, W, B, c, sched, out, step=step, examined=examined)
        torch.cuda.synchronize()
        spin.si_get_stats(mesh)
        step, examined = step.cpu().numpy(), examined.cpu().numpy()
    finally:
        spin.si_mesh_destroy(mesh)
    from oracle import dls
    groups = -(-m // group)
    starts = dls.chunk_starts(dls.FAC, groups, P, 1)
    assert (step >= 0).all() and step.max() == len(starts) - 2
    per_step_images = np.bincount(step, minlength=len(starts) - 1)
    sizes = np.diff(starts)
    np.testing.assert_array_equal(per_step_images[:-1], sizes[:-1] * group)  # the table's chunks, whole groups
    work = np.bincount(step, weights=examined.astype(np.float64), minlength=len(starts) - 1)  # pairs per claim
    first = work[:P]
    assert sizes[0] >= 10 and (sizes[:P] == sizes[0]).all()
    assert first.max() <= 1.25 * first.min(), (first.min(), first.max())
    per_group = work / (sizes * group)
    last_batch = per_group[len(sizes) - P:]
    assert per_group[:P].mean() > 1.2 * last_batch.mean()


def test_cost_order_from_host_buffers():
    """si_generate_host (host points, normals and output; mesh and grid built
    inside the call) in cost order gives the device path's images."""
    import torch

    import paper_1811_00901_gb300 as spin
    pts, nrm = wl.heightfield(8000, 94)
    W, B, c = 32, 0.01, wl.cos_deg(60.0)
    ref, _ = gpu_run(pts, nrm, W, B, c, schedule=spin.make_schedule("STATIC"))
    out = torch.empty((8000, W, W), dtype=torch.int32).pin_memory()
    spin.si_generate_host(torch.from_numpy(pts), torch.from_numpy(nrm), 8000, None, 8000, W, B, c,
                          spin.make_schedule("FAC", order=1), out)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.numpy(), ref)


def test_tuner_rebuilds_grids_and_the_mesh_stays_usable():
    """si_tune_mesh rebuilds the mesh's grids between its timed repetitions
    (forgetting the batch graphs that held them); afterwards the mesh, a
    batched call captured before the tuning and the tuner's choice all give
    the grid-order STATIC images."""
    import torch

    import paper_1811_00901_gb300 as spin
    pts, nrm = wl.heightfield(6000, 95)
    W, B, c = 32, 0.01, wl.cos_deg(60.0)
    ref, _ = gpu_run(pts, nrm, W, B, c, schedule=spin.make_schedule("STATIC"))
    dev = torch.device("cuda:0")
    mesh = spin.si_mesh_create(torch.from_numpy(pts).to(dev), torch.from_numpy(nrm).to(dev))
    try:
        out = torch.empty((6000, W, W), dtype=torch.int32, device=dev)
        item = [dict(mesh=mesh, query_idx=None, m=6000, W=W, bin_size=B, cos_s=c, out=out)]
        spin.si_generate_batched(item, spin.make_schedule("FAC"))  # a cached graph holding the grid
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), ref)
        spin.si_tune_clear()
        best, ms = spin.si_tune_mesh(mesh, None, 6000, W, B, c, out, reps=2)
        assert ms > 0 and best.kind in (0, 1, 2, 3) and best.order in (0, 1)
        for sched in (best, spin.make_schedule("FAC", order=1)):
            out.fill_(-1)
            spin.si_generate(mesh, None, 6000, W, B, c, sched, out)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(out.cpu().numpy(), ref)
        out.fill_(-1)
        spin.si_generate_batched(item, spin.make_schedule("FAC"))
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), ref)
        spin.si_get_stats(mesh)
    finally:
        spin.si_tune_clear()
        spin.si_mesh_destroy(mesh)
