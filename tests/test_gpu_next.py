"""The scheduling extensions: probabilistic factoring (FAC_PROB) and the
heterogeneity emulation of the paper's Type1 + Type2 runs (Sec. 5.2).
Neither may change an image; FAC_PROB's steps follow its chunk table; slow
workers take the first steps."""
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


@pytest.mark.parametrize("kind", ["STATIC", "SS", "GSS", "FAC", "FAC_PROB"])
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
        P = 152 * 3
        hom = kernel_ms(spin.make_schedule("STATIC", num_workers=P))
        het_static = kernel_ms(spin.make_schedule("STATIC", num_workers=P, slow_workers=P // 2, slowdown=6.0))
        het_ss = kernel_ms(spin.make_schedule("SS", num_workers=P, slow_workers=P // 2, slowdown=6.0))
        assert het_static > 3.0 * hom, (hom, het_static)
        assert het_ss < 0.6 * het_static, (het_ss, het_static)
    finally:
        spin.si_mesh_destroy(mesh)
