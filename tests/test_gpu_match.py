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


def _balanced_images(rng, n, W):
    """Images with exactly half of their W^2 pixels at 0 and half at one
    positive amplitude (its own per image): centred and scaled to unit length
    every pixel is +-1/W, exact in BF16 for W a power of two, whatever the
    rounding of the centring arithmetic.  Every correlation is then a multiple
    of 2/W^2, exact in FP32 accumulation."""
    K = W * W
    imgs = np.zeros((n, K), np.int32)
    for r in range(n):
        imgs[r, rng.permutation(K)[: K // 2]] = int(rng.integers(1, 30000)) * 65536 // 7
    return imgs.reshape(n, W, W)


def _run_bf16(scene, model, W, k, precision="BF16"):
    import torch

    import paper_1811_00901_gb300 as spin
    dev = torch.device("cuda:0")
    n_scene, n_model = len(scene), len(model)
    idx = torch.full((n_scene, k), -3, dtype=torch.int32, device=dev)
    val = torch.zeros((n_scene, k), dtype=torch.float32, device=dev)
    spin.si_match(torch.from_numpy(scene).to(dev), n_scene, torch.from_numpy(model).to(dev), n_model, W, k, precision,
                  idx, val)
    torch.cuda.synchronize()
    return idx.cpu().numpy(), val.cpu().numpy()


@pytest.mark.parametrize("W,k,n_scene,n_model,precision", [(16, 16, 257, 1025, "BF16"), (32, 5, 200, 3000, "BF16"),
                                                           (64, 3, 129, 600, "BF16"), (32, 7, 1000, 20000, "BF16"),
                                                           (32, 5, 300, 2000, "FP32"), (16, 3, 130, 700, "FP32"),
                                                           # both list lengths of the kernel (8 and 16 slots) at their edge
                                                           (32, 8, 300, 5000, "BF16"), (16, 9, 257, 1500, "FP32")])
def test_tensor_core_exact_products_and_ties(W, k, n_scene, n_model, precision):
    """BF16 matching on the tensor cores with operands that BF16 holds exactly
    (balanced two-level images): every reported value equals the FP64
    correlation exactly, and each list is exactly the k best, equal values by
    smaller model index (the images repeat, so there are many exact ties).
    Scene and model counts are ragged against the 128 x 256 tile."""
    rng = np.random.default_rng(W * 1000 + k)
    base = _balanced_images(rng, max(8, n_model // 3), W)
    model = base[rng.integers(0, len(base), n_model)]           # many duplicates: exact ties
    scene = base[rng.integers(0, len(base), n_scene)].copy()
    K = W * W
    for r in range(n_scene):                                      # move a few pixel pairs: near matches
        flat = scene[r].reshape(-1)
        on, off = np.nonzero(flat)[0], np.nonzero(flat == 0)[0]
        for _ in range(int(rng.integers(0, 4))):
            a, b = rng.choice(on), rng.choice(off)
            flat[a], flat[b] = 0, flat[a] if flat[a] else flat[on[0]]
            on, off = np.nonzero(flat)[0], np.nonzero(flat == 0)[0]
    idx, val = _run_bf16(scene, model, W, k, precision)
    r = match.correlations(scene, model)
    # the exact correlations are multiples of 2/K; the FP64 ones carry ~1e-16
    # of rounding, which must neither show in the values nor break ties
    steps = np.round(r * K / 2)
    assert np.all(np.abs(r * K / 2 - steps) < 1e-9)
    exact = steps * (2.0 / K)
    ref_idx = np.lexsort((np.broadcast_to(np.arange(n_model), exact.shape), -exact), axis=1)[:, :k]
    ref_val = np.take_along_axis(exact, ref_idx, axis=1)
    assert np.any(ref_val[:, :-1] == ref_val[:, 1:])  # the lists do hold exact ties
    np.testing.assert_array_equal(val, ref_val.astype(np.float32))
    np.testing.assert_array_equal(idx, ref_idx)


def test_tensor_core_padded_width():
    """W = 5: W^2 = 25 pixels padded to one 64-element K slice with zeros; the
    reported values are within the BF16 bound of the FP64 correlations and
    the lists are valid and sorted."""
    rng = np.random.default_rng(5)
    W, k, n_scene, n_model = 5, 4, 130, 300
    model = ((rng.random((n_model, W, W)) < 0.5) * rng.integers(0, 40 * 65536, (n_model, W, W))).astype(np.int32)
    scene = model[rng.integers(0, n_model, n_scene)].copy()
    scene += ((rng.random(scene.shape) < 0.1) * rng.integers(0, 65536 * 8, scene.shape)).astype(np.int32)
    idx, val = _run_bf16(scene, model, W, k)
    r = match.correlations(scene, model)
    tol = 2.0 ** -8 + 1e-4
    for i in range(n_scene):
        assert len(set(idx[i])) == k and (idx[i] >= 0).all()
        assert np.all(np.diff(val[i]) <= 0)
        assert np.all(np.abs(val[i] - r[i, idx[i]]) <= tol)
        out = np.ones(n_model, bool)
        out[idx[i]] = False
        assert r[i, out].max() <= r[i, idx[i, k - 1]] + 2 * tol


@pytest.mark.parametrize("precision", ["BF16", "FP32"])
def test_misaligned_images_take_the_scalar_centring(precision):
    """Images whose rows are 16-byte aligned are centred four pixels per lane
    step; images at a 4-byte offset take the one-pixel path.  Both must give
    the same lists (they differ only in the order of the FP32 sum of squares
    of each image, a relative 1e-6 of its norm)."""
    import torch

    import paper_1811_00901_gb300 as spin
    rng = np.random.default_rng(77)
    W, k, n_scene, n_model = 32, 5, 300, 4000
    model = ((rng.random((n_model, W, W)) < 0.4) * rng.integers(0, 50 * 65536, (n_model, W, W))).astype(np.int32)
    scene = model[rng.integers(0, n_model, n_scene)].copy()
    scene += ((rng.random(scene.shape) < 0.05) * rng.integers(0, 65536 * 8, scene.shape)).astype(np.int32)
    dev = torch.device("cuda:0")
    out = {}
    for off in (0, 1):
        bs = torch.zeros(scene.size + off, dtype=torch.int32, device=dev)
        bm = torch.zeros(model.size + off, dtype=torch.int32, device=dev)
        ts, tm = bs[off:].view(n_scene, W, W), bm[off:].view(n_model, W, W)
        ts.copy_(torch.from_numpy(scene))
        tm.copy_(torch.from_numpy(model))
        assert (ts.data_ptr() % 16 == 0) == (off == 0)
        idx = torch.full((n_scene, k), -3, dtype=torch.int32, device=dev)
        val = torch.zeros((n_scene, k), dtype=torch.float32, device=dev)
        spin.si_match(ts, n_scene, tm, n_model, W, k, precision, idx, val)
        torch.cuda.synchronize()
        out[off] = (idx.cpu().numpy(), val.cpu().numpy())
    (i0, v0), (i1, v1) = out[0], out[1]
    # a last-bit change of an image's norm can move a BF16 operand by one unit
    # (about 1e-4 of a pixel of a unit image of 1,024): a few 1e-6 per list value
    assert np.all(np.abs(v0 - v1) <= (1e-4 if precision == "BF16" else 1e-5))
    r = match.correlations(scene, model)
    for q in range(n_scene):
        sv = np.sort(r[q])[::-1]
        for t in range(k):
            if sv[t] - sv[t + 1] > 1e-3 and (t == 0 or sv[t - 1] - sv[t] > 1e-3):
                assert i0[q, t] == i1[q, t], (q, t)
