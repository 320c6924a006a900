"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Bar: per-image L1 error / total weight <= 1e-4; membership may differ only on
pairs the oracle flags as boundary pairs; integer results (candidate sets,
counts) bit-exact; images bit-identical across schedules.
"""
import json
import os

import numpy as np
import pytest

import oracle
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


def _golden(golden_dir, name):
    with open(os.path.join(golden_dir, name)) as f:
        g = json.load(f)
    return g, np.array(g["points"], np.float32), np.array(g["normals"], np.float32)


@pytest.mark.parametrize("name", ["five_point.json", "edges.json"])
def test_hand_computed_images_exact(golden_dir, name):
    """Dyadic hand cases: the fixed-point image is exactly 65536 x the hand image."""
    g, pts, nrm = _golden(golden_dir, name)
    imgs, pr = gpu_run(pts, nrm, g["W"], g["bin_size"], g["cos_s"], query_idx=[g["query"]], probe=True)
    expect = (np.array(g["expected"]) * 65536).astype(np.int64)
    np.testing.assert_array_equal(imgs[0].astype(np.int64), expect)
    assert pr["support"][0] == g["support"]


def test_sphere_4096_full(golden_dir):
    """4,096 points on the unit sphere, every image, W=16, B=0.05, 60 deg."""
    c = wl.plain_sphere()
    imgs, pr = gpu_run(c["points"], c["normals"], c["W"], c["bin_size"], c["cos_s"], probe=True)
    worst = compare_with_oracle(imgs, c["points"], c["normals"], c["W"], c["bin_size"], c["cos_s"], None,
                                np.arange(c["m"]), support=pr["support"])
    assert worst < 1e-4


def test_heightfield_small_all_images():
    """Clustered heightfield, 6,000 points, every image (spans many groups and a ragged tail)."""
    pts, nrm = wl.heightfield(6000, 77)
    W, B, c = 32, 0.01, wl.cos_deg(60.0)
    imgs, pr = gpu_run(pts, nrm, W, B, c, probe=True)
    sample = np.arange(0, 6000, 3)
    compare_with_oracle(imgs, pts, nrm, W, B, c, None, sample, support=pr["support"])


def test_object_scene_w64_query_list():
    """64 posed objects, W=64, explicit query list with duplicates and a ragged count."""
    pts, nrm = wl.object_scene(20000, 31)
    rng = np.random.default_rng(5)
    q = rng.integers(0, 20000, 777).astype(np.int32)
    q[10] = q[11]
    W, B, c = 64, 0.005, wl.cos_deg(90.0)
    imgs, pr = gpu_run(pts, nrm, W, B, c, query_idx=q, probe=True)
    compare_with_oracle(imgs, pts, nrm, W, B, c, q, np.arange(0, 777, 2), support=pr["support"])
    np.testing.assert_array_equal(imgs[10], imgs[11])


def test_angle_probe_counts_angle_passing_candidates():
    """The angle probe counts the candidate-set points that pass the support-
    angle test: support <= angle <= culled for every image, and the count
    equals an FP64 count (|X - P|^2 <= Rc2 and n . n_X >= cos S) up to the
    pairs within 1e-5 of either threshold."""
    import torch

    import paper_1811_00901_gb300 as spin
    pts, nrm = wl.heightfield(5000, 19)
    W, B, c = 32, 0.01, float(wl.cos_deg(60.0))
    dev = torch.device("cuda:0")
    mesh = spin.si_mesh_create(torch.from_numpy(pts).to(dev), torch.from_numpy(nrm).to(dev))
    try:
        m = pts.shape[0]
        out = torch.empty((m, W, W), dtype=torch.int32, device=dev)
        pr = {k: torch.full((m,), -1, dtype=torch.int64, device=dev) for k in ("culled", "support", "angle")}
        spin.si_generate_probe(mesh, None, m, W, B, c, spin.make_schedule("FAC"), out, **pr)
        torch.cuda.synchronize()
        spin.si_get_stats(mesh)
        pr = {k: v.cpu().numpy() for k, v in pr.items()}
    finally:
        spin.si_mesh_destroy(mesh)
    assert np.all(pr["support"] <= pr["angle"]) and np.all(pr["angle"] <= pr["culled"])
    assert pr["angle"].sum() > pr["support"].sum()
    rc2 = float(spin.si_candidate_rc2(W, B))
    P = pts.astype(np.float64)
    N = nrm.astype(np.float64) / np.linalg.norm(nrm.astype(np.float64), axis=1, keepdims=True)
    for q in range(0, m, 97):
        d2 = ((P - P[q]) ** 2).sum(1)
        dot = N @ N[q]
        near = (np.abs(d2 - rc2) <= 1e-5 * rc2) | (np.abs(dot - c) <= 1e-5)
        expect = int(((d2 <= rc2) & (dot >= c)).sum())
        assert abs(int(pr["angle"][q]) - expect) <= int(near.sum())


@pytest.mark.parametrize("W", [16, 32, 64])
def test_near_axis_needle_and_layers(W):
    """Points on and next to each query's normal axis at distances up to the
    image half-height (a needle plus parallel discs, all sharing the axis as
    normal, S = 180 deg), every image: alpha is small next to |X - P| there,
    where |d|^2 - beta^2 in FP32 would lose alpha to cancellation.  No pair is
    near a threshold, so the bound holds with no flagged allowance."""
    h = 0.16
    B = float(np.float32(2 * h / W))
    pts, nrm, _, _ = wl.needle_layers(h, 1)
    imgs, pr = gpu_run(pts, nrm, W, B, -1.0, probe=True, schedule=None)
    worst = compare_with_oracle(imgs, pts, nrm, W, B, -1.0, None, np.arange(pts.shape[0]), support=pr["support"],
                                require_unflagged=True)
    assert worst <= 1e-4


@pytest.mark.parametrize("W,B,deg", [(2, 0.1, 180.0), (5, 0.1, 180.0), (7, 0.07, 45.0), (127, 0.004, 60.0),
                                     (128, 0.004, 60.0)])
def test_odd_widths(W, B, deg):
    """The paper's own W = 5 (Sec. 4.1) and other widths, including the extremes
    (W = 128 is the largest the library takes)."""
    pts, nrm = wl.object_scene(3000, 8, n_objects=6)
    c = wl.cos_deg(deg)
    imgs, pr = gpu_run(pts, nrm, W, B, c, query_idx=np.arange(0, 3000, 7).astype(np.int32), probe=True)
    q = np.arange(0, 3000, 7).astype(np.int32)
    compare_with_oracle(imgs, pts, nrm, W, B, c, q, np.arange(len(q)), support=pr["support"])


def test_candidate_sets_bit_exact():
    """The grid's candidate set equals the FP32 brute-force set (count and fingerprint)."""
    for pts, W, B in [(wl.heightfield(8000, 3)[0], 32, 0.01), (wl.object_scene(8000, 4)[0], 64, 0.005),
                      (wl.sphere(3000, 6)[0], 16, 0.05)]:
        nrm = np.tile(np.array([[0, 0, 1]], np.float32), (pts.shape[0], 1))
        q = np.arange(0, pts.shape[0], 11).astype(np.int32)
        for div in (1, 4, 9):
            import paper_1811_00901_gb300 as spin
            _, pr = gpu_run(pts, nrm, W, B, -1.0, query_idx=q, probe=True,
                            schedule=spin.make_schedule("GSS", grid_div=div))
            cnt, hs = oracle.candidates_fp32(pts, W, B, query_idx=q)
            np.testing.assert_array_equal(pr["culled"], cnt)
            np.testing.assert_array_equal(pr["cand_hash"], hs)


def test_candidate_sets_degenerate_meshes():
    """Coincident points, collinear points, a single point, points on cell faces."""
    rng = np.random.default_rng(2)
    cases = []
    cases.append(np.zeros((50, 3), np.float32))                                      # one location
    t = np.linspace(-1, 1, 400, dtype=np.float32)
    cases.append(np.stack([t, 2 * t, -t], 1))                                       # a line
    cases.append(np.array([[0.25, -0.5, 3.0]], np.float32))                          # single point
    g = (rng.integers(-6, 7, (600, 3)) * 0.125).astype(np.float32)                   # lattice on faces
    cases.append(g)
    for pts in cases:
        nrm = np.tile(np.array([[0, 1, 0]], np.float32), (pts.shape[0], 1))
        q = np.arange(pts.shape[0]).astype(np.int32)
        for W, B in [(8, 0.125), (16, 0.05)]:
            _, pr = gpu_run(pts, nrm, W, B, -1.0, query_idx=q, probe=True)
            cnt, hs = oracle.candidates_fp32(pts, W, B, query_idx=q)
            np.testing.assert_array_equal(pr["culled"], cnt)
            np.testing.assert_array_equal(pr["cand_hash"], hs)


def test_schedules_bit_identical():
    """Every schedule, worker count, group size and grid resolution gives the same int32 images."""
    import paper_1811_00901_gb300 as spin
    pts, nrm = wl.heightfield(5000, 9)
    W, B, c = 32, 0.01, wl.cos_deg(60.0)
    ref, _ = gpu_run(pts, nrm, W, B, c, schedule=spin.make_schedule("STATIC"))
    for kind in ("STATIC", "SS", "GSS", "FAC"):
        for workers, group, div, mc in [(0, 0, 0, 1), (1, 0, 0, 1), (7, 4, 2, 3), (300, 32, 8, 1), (13, 1, 1, 2)]:
            got, _ = gpu_run(pts, nrm, W, B, c,
                             schedule=spin.make_schedule(kind, min_chunk=mc, num_workers=workers, group=group,
                                                         grid_div=div))
            assert np.array_equal(got, ref), (kind, workers, group, div, mc)


def test_every_image_claimed_once_with_table_steps():
    """Probe worker/step: each image is produced once, by the step the chunk
    table assigns to its group; STATIC runs step b on block b."""
    import paper_1811_00901_gb300 as spin
    pts, nrm = wl.heightfield(4000, 10)
    W, B, c = 16, 0.02, 0.5
    for kind in ("STATIC", "SS", "GSS", "FAC"):
        workers, group = 9, 8
        _, pr = gpu_run(pts, nrm, W, B, c, probe=True,
                        schedule=spin.make_schedule(kind, num_workers=workers, group=group))
        assert (pr["worker"] >= 0).all() and (pr["worker"] < workers).all()
        units = -(-4000 // group)
        starts = spin.si_chunk_table(kind, units, workers, 1)
        nsteps = len(starts) - 1
        assert (pr["step"] >= 0).all() and (pr["step"] < nsteps).all()
        # images per step = the step's groups x group size (last group ragged)
        per_step = np.bincount(pr["step"], minlength=nsteps)
        for s in range(nsteps):
            lo, hi = starts[s] * group, min(starts[s + 1] * group, 4000)
            assert per_step[s] == max(0, hi - lo), (kind, s)
        if kind == "STATIC":
            np.testing.assert_array_equal(pr["worker"], pr["step"])


def test_m_zero_and_one():
    import torch

    import paper_1811_00901_gb300 as spin
    pts, nrm = wl.sphere(300, 4)
    imgs, _ = gpu_run(pts, nrm, 16, 0.05, 0.5, query_idx=np.array([123], np.int32))
    compare_with_oracle(imgs, pts, nrm, 16, 0.05, 0.5, np.array([123]), [0])
    dev = torch.device("cuda:0")
    mesh = spin.si_mesh_create(torch.from_numpy(pts).to(dev), torch.from_numpy(nrm).to(dev))
    try:
        out = torch.empty((0, 16, 16), dtype=torch.int32, device=dev)
        spin.si_generate(mesh, None, 0, 16, 0.05, 0.5, spin.make_schedule("SS"), out)
        torch.cuda.synchronize()
    finally:
        spin.si_mesh_destroy(mesh)


def test_invalid_arguments_are_rejected():
    import torch

    import paper_1811_00901_gb300 as spin
    dev = torch.device("cuda:0")
    pts, nrm = wl.sphere(100, 4)
    mesh = spin.si_mesh_create(torch.from_numpy(pts).to(dev), torch.from_numpy(nrm).to(dev))
    out = torch.empty((100, 16, 16), dtype=torch.int32, device=dev)
    try:
        bad = [dict(W=1), dict(W=129), dict(B=0.0), dict(B=float("inf")), dict(c=1.5), dict(m=101),
               dict(m=-1), dict(sched=spin.make_schedule("GSS", group=3)),
               dict(sched=spin.make_schedule(7))]
        for b in bad:
            with pytest.raises(spin.SpinError) as e:
                spin.si_generate(mesh, None, b.get("m", 100), b.get("W", 16), b.get("B", 0.05), b.get("c", 0.5),
                                 b.get("sched", spin.make_schedule("GSS")), out)
            assert e.value.status == spin.SI_ERR_INVALID
    finally:
        spin.si_mesh_destroy(mesh)
    bad_n = nrm.copy()
    bad_n[5] = 0
    bad_p = pts.copy()
    bad_p[7, 1] = np.nan
    # host inputs: rejected by si_mesh_create itself
    for p_, n_ in ((pts, bad_n), (bad_p, nrm)):
        with pytest.raises(spin.SpinError) as e:
            spin.si_mesh_create(torch.from_numpy(p_), torch.from_numpy(n_))
        assert e.value.status == spin.SI_ERR_INVALID
    # device inputs: checked on the device without a round trip, reported by si_get_stats
    for p_, n_ in ((pts, bad_n), (bad_p, nrm)):
        mesh = spin.si_mesh_create(torch.from_numpy(p_).to(dev), torch.from_numpy(n_).to(dev))
        try:
            spin.si_generate(mesh, None, 100, 16, 0.05, 0.5, spin.make_schedule("GSS"), out)
            st, status = spin.si_get_stats(mesh, raise_on_flags=False)
            assert status == spin.SI_ERR_INVALID and st["bad_input"] == 1
        finally:
            spin.si_mesh_destroy(mesh)
    # the host-buffer entry point checks on the device and reports before it returns
    hout = torch.empty((100, 16, 16), dtype=torch.int32)
    with pytest.raises(spin.SpinError) as e:
        spin.si_generate_host(torch.from_numpy(pts), torch.from_numpy(bad_n), 100, None, 100, 16, 0.05, 0.5,
                              spin.make_schedule("GSS"), hout)
    assert e.value.status == spin.SI_ERR_INVALID
    # a clean mesh reports nothing
    mesh = spin.si_mesh_create(torch.from_numpy(pts).to(dev), torch.from_numpy(nrm).to(dev))
    st, status = spin.si_get_stats(mesh, raise_on_flags=False)
    assert status == spin.SI_OK and st["bad_input"] == 0
    spin.si_mesh_destroy(mesh)


def test_overflow_is_detected():
    """40,000 coincident points put 40,000 x 65536 > INT32_MAX into one pixel."""
    import torch

    import paper_1811_00901_gb300 as spin
    n = 40000
    pts = np.zeros((n, 3), np.float32)
    nrm = np.tile(np.array([[0, 0, 1]], np.float32), (n, 1))
    dev = torch.device("cuda:0")
    mesh = spin.si_mesh_create(torch.from_numpy(pts).to(dev), torch.from_numpy(nrm).to(dev))
    try:
        out = torch.empty((2, 8, 8), dtype=torch.int32, device=dev)
        spin.si_generate(mesh, torch.tensor([0, 1], dtype=torch.int32, device=dev), 2, 8, 0.1, 0.0,
                         spin.make_schedule("GSS"), out)
        torch.cuda.synchronize()
        stats, status = spin.si_get_stats(mesh, raise_on_flags=False)
        assert status == spin.SI_ERR_OVERFLOW and stats["overflow"] == 1
        spin.si_reset_stats(mesh)
        # the flag is sticky until reset, and the same pixel overflows again
        spin.si_generate(mesh, torch.tensor([0], dtype=torch.int32, device=dev), 1, 8, 0.1, 0.0,
                         spin.make_schedule("GSS"), out)
        torch.cuda.synchronize()
        stats, status = spin.si_get_stats(mesh, raise_on_flags=False)
        assert status == spin.SI_ERR_OVERFLOW  # still 40,000 points in the pixel
    finally:
        spin.si_mesh_destroy(mesh)
    n = 30000
    mesh = spin.si_mesh_create(torch.from_numpy(np.zeros((n, 3), np.float32)).to(dev),
                               torch.from_numpy(np.tile(np.array([[0, 0, 1]], np.float32), (n, 1))).to(dev))
    try:
        out = torch.empty((1, 8, 8), dtype=torch.int32, device=dev)
        spin.si_generate(mesh, torch.tensor([0], dtype=torch.int32, device=dev), 1, 8, 0.1, 0.0,
                         spin.make_schedule("GSS"), out)
        torch.cuda.synchronize()
        stats, status = spin.si_get_stats(mesh, raise_on_flags=False)
        assert status == spin.SI_OK
        assert int(out[0, 4, 0]) == 30000 * 65536
    finally:
        spin.si_mesh_destroy(mesh)


def test_host_buffer_path_equals_device_path():
    import torch

    import paper_1811_00901_gb300 as spin
    pts, nrm = wl.heightfield(3000, 13)
    W, B, c = 16, 0.02, 0.5
    q = np.arange(0, 3000, 5).astype(np.int32)
    ref, _ = gpu_run(pts, nrm, W, B, c, query_idx=q)
    out = torch.empty((len(q), W, W), dtype=torch.int32).pin_memory()
    tp = torch.from_numpy(pts)
    tn = torch.from_numpy(nrm)
    tq = torch.from_numpy(q)
    spin.si_generate_host(tp, tn, 3000, tq, len(q), W, B, c, spin.make_schedule("FAC"), out)
    np.testing.assert_array_equal(out.numpy(), ref)


@pytest.mark.parametrize("explicit,pinned", [(False, True), (True, True), (False, False), (True, False)])
def test_host_buffer_path_large_calls(explicit, pinned):
    """Calls of 32,768 images or more: into page-locked output the kernel
    writes directly; into pageable output the call generates in query ranges
    whose downloads overlap the next range's generation.  Images equal the
    device path's either way."""
    import torch

    import paper_1811_00901_gb300 as spin
    n = 40_000
    pts, nrm = wl.heightfield(n, 15)
    W, B, c = 16, 0.02, 0.5
    q = np.random.default_rng(1).permutation(n)[:36_001].astype(np.int32) if explicit else None
    m = n if q is None else len(q)
    ref, _ = gpu_run(pts, nrm, W, B, c, query_idx=q)
    out = torch.full((m, W, W), -3, dtype=torch.int32)
    if pinned:
        out = out.pin_memory()
    tq = None if q is None else torch.from_numpy(q)
    spin.si_generate_host(torch.from_numpy(pts), torch.from_numpy(nrm), n, tq, m, W, B, c,
                          spin.make_schedule("FAC"), out)
    np.testing.assert_array_equal(out.numpy(), ref)


def test_batched_equals_single_calls():
    import torch

    import paper_1811_00901_gb300 as spin
    dev = torch.device("cuda:0")
    specs = [(wl.sphere(2000, 1), 16, 0.05, 0.5, None),
             (wl.heightfield(3000, 2), 32, 0.01, 0.5, np.arange(0, 3000, 3).astype(np.int32)),
             (wl.object_scene(2500, 3, n_objects=5), 64, 0.006, 0.0, None),
             (wl.sphere(10, 4), 8, 0.3, -1.0, np.array([9, 0, 9], np.int32))]
    meshes, items, refs = [], [], []
    try:
        for (pts, nrm), W, B, c, q in specs:
            ref, _ = gpu_run(pts, nrm, W, B, c, query_idx=q)
            refs.append(ref)
            mesh = spin.si_mesh_create(torch.from_numpy(pts).to(dev), torch.from_numpy(nrm).to(dev))
            meshes.append(mesh)
            m = pts.shape[0] if q is None else len(q)
            out = torch.full((m, W, W), -1, dtype=torch.int32, device=dev)
            tq = None if q is None else torch.from_numpy(q).to(dev)
            items.append(dict(mesh=mesh, query_idx=tq, m=m, W=W, bin_size=B, cos_s=c, out=out))
        for sched in (None, spin.make_schedule("STATIC"), spin.make_schedule("SS", num_workers=17),
                      spin.make_schedule("FAC", group=2)):
            for it in items:
                it["out"].fill_(-1)
            spin.si_generate_batched(items, sched)
            torch.cuda.synchronize()
            for it, ref in zip(items, refs):
                np.testing.assert_array_equal(it["out"].cpu().numpy(), ref)
    finally:
        for mesh in meshes:
            spin.si_mesh_destroy(mesh)


def test_bad_query_index_is_reported_not_read():
    """An out-of-range query index is detected on the device and never read:
    its image is not computed, the others are correct, and si_get_stats
    reports it."""
    import torch

    import paper_1811_00901_gb300 as spin
    pts, nrm = wl.sphere(500, 6)
    dev = torch.device("cuda:0")
    q = np.array([3, 500, 7, -2, 11], np.int32)
    mesh = spin.si_mesh_create(torch.from_numpy(pts).to(dev), torch.from_numpy(nrm).to(dev))
    try:
        out = torch.full((5, 16, 16), -5, dtype=torch.int32, device=dev)
        spin.si_generate(mesh, torch.from_numpy(q).to(dev), 5, 16, 0.05, 0.5, spin.make_schedule("GSS"), out)
        torch.cuda.synchronize()
        stats, status = spin.si_get_stats(mesh, raise_on_flags=False)
        assert status == spin.SI_ERR_INVALID and stats["bad_query"] == 1
        o = out.cpu().numpy()
    finally:
        spin.si_mesh_destroy(mesh)
    good = np.array([3, 7, 11], np.int32)
    ref, _ = gpu_run(pts, nrm, 16, 0.05, 0.5, query_idx=good)
    np.testing.assert_array_equal(o[[0, 2, 4]], ref)


@pytest.mark.parametrize("W,B", [(32, 0.01), (128, 0.003), (16, 0.05)])
def test_column_edge_pairs_keep_their_whole_weight(W, B):
    """Pairs whose alpha lies within a few ulps of (W-1) B: the column test is
    alpha^2 < ((W-1)B)^2, while v comes from an approximate reciprocal square
    root, so v may land a hair above W-1.  Every contributing pair must still
    put its whole weight 65536 inside the W x W image (the exact overflow check
    would otherwise report a pixel overflow)."""
    import paper_1811_00901_gb300 as spin
    edge = np.float32((W - 1) * B)
    ds = [edge]
    for _ in range(300):
        ds.append(np.nextafter(ds[-1], np.float32(0)))
    up = edge
    for _ in range(40):
        up = np.nextafter(up, np.float32(1))
        ds.append(up)
    ds = np.array(ds, np.float32)
    ang = np.linspace(0, 2 * np.pi, len(ds), endpoint=False)
    pts = np.zeros((len(ds) + 1, 3), np.float32)
    pts[1:, 0] = (ds * np.cos(ang)).astype(np.float32)
    pts[1:, 1] = (ds * np.sin(ang)).astype(np.float32)
    nrm = np.tile(np.array([[0, 0, 1]], np.float32), (len(pts), 1))
    q = np.array([0], np.int32)
    got, pr = gpu_run(pts, nrm, W, B, 0.0, query_idx=q, probe=True, schedule=spin.make_schedule("SS"))
    assert got[0].astype(np.int64).sum() == 65536 * int(pr["support"][0])
    compare_with_oracle(got, pts, nrm, W, B, 0.0, q, np.array([0]))


def test_bounded_device_wait_gives_up_and_the_context_stays_usable():
    """The spin kernel's mbarrier waits are bounded: a wait on a barrier that
    nothing arrives at gives up after its limit and reports it; work launched
    afterwards runs normally."""
    import paper_1811_00901_gb300 as spin
    timed_out, waited = spin.si_check_bounded_wait(50)
    assert timed_out
    assert 45.0 <= waited < 5000.0, waited
    pts, nrm = wl.sphere(1500, 77)
    got, _ = gpu_run(pts, nrm, 16, 0.05, 0.5)
    compare_with_oracle(got, pts, nrm, 16, 0.05, 0.5, None, np.arange(0, 1500, 97))


@pytest.mark.parametrize("group", [0, 1, 2])
def test_widest_images_with_every_group_that_fits(group):
    """W = 128 (the maximum): a group of one image needs ~100 KB of shared memory,
    two need ~166 KB; both run, and agree with each other and the oracle."""
    import paper_1811_00901_gb300 as spin
    pts, nrm = wl.heightfield(4000, 33)
    W, B, c = 128, 0.002, 0.5
    q = np.arange(0, 4000, 37).astype(np.int32)
    imgs, pr = gpu_run(pts, nrm, W, B, c, query_idx=q, probe=True,
                       schedule=spin.make_schedule("SS", group=group))
    compare_with_oracle(imgs, pts, nrm, W, B, c, q, np.arange(len(q)), support=pr["support"])
