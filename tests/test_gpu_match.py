"""Spin-image matching against the oracle: correlations within the bound of
the arithmetic, and best-k lists that are valid, sorted and exact where the
correlations are clearly apart."""
import numpy as np
import pytest

from oracle import match
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


def _images():
    """Model: images of a heightfield; scene: images of the same surface seen
    from a rigidly moved copy with extra points, plus a constant image."""
    pts, nrm = wl.heightfield(3000, 61)
    W, B, c = 16, 0.02, 0.5
    model, _ = gpu_run(pts, nrm, W, B, c)
    rng = np.random.default_rng(2)
    rot = np.linalg.qr(rng.normal(size=(3, 3)))[0]
    extra_p, extra_n = wl.heightfield(600, 62)
    p2 = np.concatenate([pts, extra_p]) @ rot.T + np.array([0.3, -0.2, 0.1])
    n2 = np.concatenate([nrm, extra_n]) @ rot.T
    q = np.arange(0, 3000, 7).astype(np.int32)
    scene, _ = gpu_run(p2.astype(np.float32), n2.astype(np.float32), W, B, c, query_idx=q)
    scene = np.concatenate([scene, np.full((1, W, W), 65536 * 3, np.int32)])
    return scene, model, W


@pytest.mark.parametrize("precision,tol", [("FP32", 1e-4), ("BF16", 2.0 ** -8 + 1e-4)])
def test_best_matches_against_the_oracle(precision, tol):
    import torch

    import paper_1811_00901_gb300 as spin
    scene, model, W = _images()
    k = 5
    dev = torch.device("cuda:0")
    ts, tm = torch.from_numpy(scene).to(dev), torch.from_numpy(model).to(dev)
    idx = torch.full((len(scene), k), -2, dtype=torch.int32, device=dev)
    val = torch.zeros((len(scene), k), dtype=torch.float32, device=dev)
    spin.si_match(ts, len(scene), tm, len(model), W, k, precision, idx, val)
    torch.cuda.synchronize()
    idx, val = idx.cpu().numpy(), val.cpu().numpy()
    r = match.correlations(scene, model)
    ref_idx, ref_val = match.best_matches(scene, model, k)
    for i in range(len(scene)):
        assert len(set(idx[i])) == k and (idx[i] >= 0).all()
        assert np.all(np.diff(val[i]) <= 0)
        # the reported values are the pairs' correlations ...
        assert np.all(np.abs(val[i] - r[i, idx[i]]) <= tol), i
        # ... and no model image left out beats the k-th reported one by more than the bound
        out = np.ones(len(model), bool)
        out[idx[i]] = False
        assert r[i, out].max() <= r[i, idx[i, k - 1]] + 2 * tol, i
        assert ref_val[i, k - 1] <= val[i, k - 1] + 2 * tol
        # where the oracle's ranking is separated by more than the bound on both
        # sides of a place, the lists agree at that place
        sv = np.sort(r[i])[::-1]
        for t in range(k):
            if sv[t] - sv[t + 1] > 2 * tol and (t == 0 or sv[t - 1] - sv[t] > 2 * tol):
                assert idx[i, t] == ref_idx[i, t], (i, t)
    # the constant image correlates 0 with everything
    assert np.all(val[-1] == 0.0)


def test_invalid_arguments():
    import torch

    import paper_1811_00901_gb300 as spin
    dev = torch.device("cuda:0")
    a = torch.zeros((2, 8, 8), dtype=torch.int32, device=dev)
    i = torch.zeros((2, 4), dtype=torch.int32, device=dev)
    v = torch.zeros((2, 4), dtype=torch.float32, device=dev)
    for args in [(a, 2, a, 2, 8, 4, 0), (a, 2, a, 2, 8, 0, 0), (a, 2, a, 2, 8, 17, 0), (a, 2, a, 2, 8, 2, 5)]:
        with pytest.raises(spin.SpinError):
            spin.si_match(*args, i, v)
