"""The scheduling extensions: probabilistic factoring (FAC_PROB), adaptive
weighted factoring and adaptive factoring (AWF, AF: chunk sizes decided on the
device) and the heterogeneity emulation of the paper's Type1 + Type2 runs
(Sec. 5.2).  None may change an image; FAC_PROB's steps follow its chunk
table; AWF and AF hand out every group exactly once; slow workers take the
first steps."""
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


def test_fac_prob_images_and_steps():
    """FAC_PROB: images equal STATIC's bit for bit; each image comes from the
    step its group has in the table that the oracle's rule gives."""
    import paper_1811_00901_gb300 as spin
    from oracle import dls
    pts, nrm = wl.heightfield(4000, 10)
    W, B, c = 16, 0.02, 0.5
    ref, _ = gpu_run(pts, nrm, W, B, c, schedule=spin.make_schedule("STATIC"))
    workers, group = 9, 8
    units = -(-4000 // group)
    for cov in (0.0, 0.5, 2.0):
        img, pr = gpu_run(pts, nrm, W, B, c, probe=True,
                          schedule=spin.make_schedule("FAC_PROB", num_workers=workers, group=group, fac_cov=cov))
        np.testing.assert_array_equal(img, ref)
        starts = dls.chunk_starts(dls.FAC_PROB, units, workers, 1, cov=float(np.float32(cov)))
        nsteps = len(starts) - 1
        per_step = np.bincount(pr["step"], minlength=nsteps)
        assert len(per_step) == nsteps
        for s in range(nsteps):
            lo, hi = starts[s] * group, min(starts[s + 1] * group, 4000)
            assert per_step[s] == max(0, hi - lo), (cov, s)


@pytest.mark.parametrize("kind", ["STATIC", "SS", "GSS", "FAC", "FAC_PROB", "AWF", "AF"])
def test_slow_workers_change_no_image_and_take_the_first_steps(kind):
    import paper_1811_00901_gb300 as spin
    pts, nrm = wl.heightfield(6000, 12)
    W, B, c = 32, 0.01, wl.cos_deg(60.0)
    ref, _ = gpu_run(pts, nrm, W, B, c, schedule=spin.make_schedule("STATIC"))
    workers, slow = 24, 10
    img, pr = gpu_run(pts, nrm, W, B, c, probe=True,
                      schedule=spin.make_schedule(kind, num_workers=workers, group=8, slow_workers=slow,
                                                  slowdown=3.0, fac_cov=1.0))
    np.testing.assert_array_equal(img, ref)
    assert (pr["worker"] >= 0).all() and (pr["worker"] < workers).all()
    # step k < slow is run by slow worker k (the slow workers request first)
    first = pr["step"] < slow
    np.testing.assert_array_equal(pr["worker"][first], pr["step"][first])


def test_default_workers_match_the_default_launch():
    """si_default_workers is SMs x resident blocks; STATIC with num_workers = 0
    runs one step per worker.  The nearest-bin count runs the kernel instance
    that probe launches run, so the probe's step count is that number."""
    import torch

    import paper_1811_00901_gb300 as spin
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for W in (8, 16, 32, 64, 128):
        P = spin.si_default_workers(W)
        assert P % sms == 0 and 1 <= P // sms <= 2048 // 32, (W, P)
    W = 16
    sched = spin.make_schedule("STATIC", binning="NEAREST")
    P = spin.si_default_workers(W, sched)
    pts, nrm = wl.heightfield(40_000, 5)
    _, pr = gpu_run(pts, nrm, W, 0.02, 0.5, probe=True, schedule=sched)
    assert int(pr["step"].max()) + 1 == P
    assert len(np.unique(pr["worker"])) == P


def test_slow_workers_slow_static_down_more_than_self_scheduling():
    """Half the workers 6x slower: STATIC (equal blocks) takes several times as
    long; SS moves the work to the fast workers."""
    import torch

    import paper_1811_00901_gb300 as spin
    pts, nrm = wl.heightfield(30_000, 14)
    W, B, c = 32, 0.01, wl.cos_deg(60.0)
    dev = torch.device("cuda:0")
    tp, tn = torch.from_numpy(pts).to(dev), torch.from_numpy(nrm).to(dev)
    mesh = spin.si_mesh_create(tp, tn)
    out = torch.empty((30_000, W, W), dtype=torch.int32, device=dev)

    def kernel_ms(sched):
        spin.si_generate(mesh, None, 30_000, W, B, c, sched, out)
        torch.cuda.synchronize()
        spin.si_reset_stats(mesh)
        spin.si_set_timing(True)
        for _ in range(3):
            spin.si_generate(mesh, None, 30_000, W, B, c, sched, out)
        torch.cuda.synchronize()
        st, _ = spin.si_get_stats(mesh)
        spin.si_set_timing(False)
        return st["kernel_ms"] / st["kernel_launches"]

    try:
        P = spin.si_default_workers(W)
        hom = kernel_ms(spin.make_schedule("STATIC", num_workers=P))
        het_static = kernel_ms(spin.make_schedule("STATIC", num_workers=P, slow_workers=P // 2, slowdown=6.0))
        het_ss = kernel_ms(spin.make_schedule("SS", num_workers=P, slow_workers=P // 2, slowdown=6.0))
        assert het_static > 3.0 * hom, (hom, het_static)
        assert het_ss < 0.6 * het_static, (het_ss, het_static)
    finally:
        spin.si_mesh_destroy(mesh)


@pytest.mark.parametrize("kind", ["AWF", "AF"])
@pytest.mark.parametrize("group,workers,slices,mc", [(8, 0, 1, 1), (1, 37, 0, 1), (32, 300, 1, 3), (4, 9, 4, 2)])
def test_adaptive_rules_generate_every_group_once(kind, group, workers, slices, mc):
    """AWF and AF: images equal STATIC's; each image comes from exactly one
    claim, and each claim is one worker's."""
    import paper_1811_00901_gb300 as spin
    pts, nrm = wl.heightfield(5000, 31)
    W, B, c = 16, 0.02, 0.5
    ref, _ = gpu_run(pts, nrm, W, B, c, schedule=spin.make_schedule("STATIC"))
    img, pr = gpu_run(pts, nrm, W, B, c, probe=True,
                      schedule=spin.make_schedule(kind, group=group, num_workers=workers, slices=slices,
                                                  min_chunk=mc))
    np.testing.assert_array_equal(img, ref)
    assert (pr["step"] >= 0).all() and (pr["worker"] >= 0).all()
    # a claim is one worker's
    for s in np.unique(pr["step"]):
        assert len(np.unique(pr["worker"][pr["step"] == s])) == 1


@pytest.mark.parametrize("kind", ["AWF", "AF"])
def test_adaptive_batched_items_share_one_loop(kind):
    import torch

    import paper_1811_00901_gb300 as spin
    dev = torch.device("cuda:0")
    meshes, items, refs = [], [], []
    try:
        for k, (n, W, B, cs) in enumerate([(3000, 16, 0.05, 0.5), (1500, 32, 0.025, 0.0), (0, 16, 0.05, 0.5),
                                           (900, 7, 0.1, -1.0)]):
            pts, nrm = wl.sphere(max(n, 10), 50 + k)
            mh = spin.si_mesh_create(torch.from_numpy(pts).to(dev), torch.from_numpy(nrm).to(dev))
            meshes.append(mh)
            out = torch.empty((n, W, W), dtype=torch.int32, device=dev)
            items.append(dict(mesh=mh, query_idx=None, m=n, W=W, bin_size=B, cos_s=cs, out=out))
            refs.append(gpu_run(pts, nrm, W, B, cs, m=n, schedule=spin.make_schedule("STATIC"))[0])
        spin.si_generate_batched(items, spin.make_schedule(kind))
        torch.cuda.synchronize()
        for it, ref in zip(items, refs):
            np.testing.assert_array_equal(it["out"].cpu().numpy(), ref)
    finally:
        for mh in meshes:
            spin.si_mesh_destroy(mh)


def test_awf_balances_slow_workers():
    """With half the workers 4x slower (and requesting first), AWF moves work
    to the fast workers: it finishes well before STATIC (which waits for the
    slow workers' equal blocks) and before FAC, whose first batch of FAC2
    chunks is what sets its makespan at this slowdown (AWF's first batch is
    half as large and its later chunks follow the measured rates).  About 25
    groups per worker."""
    import torch

    import paper_1811_00901_gb300 as spin
    pts, nrm = wl.heightfield(60_000, 14)
    W, B, c = 32, 0.01, wl.cos_deg(60.0)
    dev = torch.device("cuda:0")
    mesh = spin.si_mesh_create(torch.from_numpy(pts).to(dev), torch.from_numpy(nrm).to(dev))
    out = torch.empty((60_000, W, W), dtype=torch.int32, device=dev)

    def kernel_ms(sched):
        spin.si_generate(mesh, None, 60_000, W, B, c, sched, out)
        torch.cuda.synchronize()
        spin.si_reset_stats(mesh)
        spin.si_set_timing(True)
        for _ in range(3):
            spin.si_generate(mesh, None, 60_000, W, B, c, sched, out)
        torch.cuda.synchronize()
        st, _ = spin.si_get_stats(mesh)
        spin.si_set_timing(False)
        return st["kernel_ms"] / st["kernel_launches"]

    try:
        P = spin.si_default_workers(W, spin.make_schedule("FAC", group=8))
        static = kernel_ms(spin.make_schedule("STATIC", num_workers=P, group=8, slow_workers=P // 2, slowdown=4.0))
        fac = kernel_ms(spin.make_schedule("FAC", num_workers=P, group=8, slow_workers=P // 2, slowdown=4.0))
        awf = kernel_ms(spin.make_schedule("AWF", num_workers=P, group=8, slow_workers=P // 2, slowdown=4.0))
        af = kernel_ms(spin.make_schedule("AF", num_workers=P, group=8, slow_workers=P // 2, slowdown=4.0))
        print("slow-worker balance (ms): STATIC %.3f FAC %.3f AWF %.3f AF %.3f" % (static, fac, awf, af))
        assert awf <= 0.7 * static, (awf, static)
        assert awf < fac, (awf, fac)
        assert af <= 0.7 * static, (af, static)
    finally:
        spin.si_mesh_destroy(mesh)


@pytest.mark.parametrize("kind", ["STATIC", "SS", "GSS", "FAC"])
def test_claim_trace_covers_every_step_once(kind):
    """si_generate_traced records one entry per scheduling claim: each step of
    the rule's chunk table exactly once (STATIC: one per worker), start before
    end, and the images are those of si_generate."""
    import torch

    import paper_1811_00901_gb300 as spin
    dev = torch.device("cuda:0")
    pts, nrm = wl.heightfield(20000, 51)
    W, B, c = 32, 0.01, float(wl.cos_deg(60.0))
    m = pts.shape[0]
    sched = spin.make_schedule(kind, group=16, slices=1)
    P = spin.si_default_workers(W, sched)
    mesh = spin.si_mesh_create(torch.from_numpy(pts).to(dev), torch.from_numpy(nrm).to(dev))
    try:
        ref = torch.empty((m, W, W), dtype=torch.int32, device=dev)
        spin.si_generate(mesh, None, m, W, B, c, sched, ref)
        out = torch.empty_like(ref)
        claims = torch.full((4 * P + 4096, 4), -1, dtype=torch.int64, device=dev)
        count = torch.zeros(1, dtype=torch.int64, device=dev)
        spin.si_generate_traced(mesh, None, m, W, B, c, sched, out, claims, count)
        torch.cuda.synchronize()
        spin.si_get_stats(mesh)
    finally:
        spin.si_mesh_destroy(mesh)
    assert torch.equal(out, ref)
    n = int(count.item())
    tr = claims[:n].cpu().numpy()
    units = (m + 15) // 16
    steps = len(spin.si_chunk_table(kind, units, P, 1)) - 1
    assert n == steps
    assert sorted(tr[:, 1].tolist()) == list(range(steps))
    assert np.all(tr[:, 2] <= tr[:, 3]) and np.all(tr[:, 0] >= 0) and np.all(tr[:, 0] < P)
    if kind == "STATIC":
        np.testing.assert_array_equal(np.sort(tr[:, 0]), np.arange(P))
        np.testing.assert_array_equal(tr[:, 0], tr[:, 1])  # worker k runs block k
