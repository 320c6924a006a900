"""Pins of the FP64 oracle against values fixed by the paper and by mathematics.

Each test states what it pins.  None of them re-types the oracle's formula:
they compare against hand-computed images (tests/golden), closed forms on a
sphere and a plane, invariances, and distance bounds.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1811_00901_gb300 import workloads as wl


def _golden(golden_dir, name):
    with open(os.path.join(golden_dir, name)) as f:
        g = json.load(f)
    pts = np.array(g["points"], dtype=np.float32)
    nrm = np.array(g["normals"], dtype=np.float32)
    return g, pts, nrm


@pytest.mark.parametrize("name", ["five_point.json", "edges.json"])
def test_hand_computed_images(golden_dir, name):
    """Algorithm 1 with the bilinear splat on hand-computed dyadic cases."""
    g, pts, nrm = _golden(golden_dir, name)
    img, sup, flg = oracle.spin_images(pts, nrm, g["W"], g["bin_size"], g["cos_s"],
                                       query_idx=[g["query"]])
    np.testing.assert_allclose(img[0], np.array(g["expected"]), rtol=0, atol=1e-12)
    assert sup[0] == g["support"]
    assert flg[0] == g["flagged"]
    assert abs(img[0].sum() - g["support"]) < 1e-12


def test_normal_length_does_not_matter(golden_dir):
    """Normals are directions: scaling them by positive factors changes nothing."""
    g, pts, nrm = _golden(golden_dir, "five_point.json")
    scale = np.array([[2.0], [0.5], [3.0], [0.25], [7.0]], dtype=np.float32)
    img, sup, _ = oracle.spin_images(pts, nrm * scale, g["W"], g["bin_size"], g["cos_s"],
                                     query_idx=[0])
    np.testing.assert_allclose(img[0], np.array(g["expected"]), rtol=0, atol=1e-12)


def test_zero_normal_is_an_error():
    pts = np.zeros((2, 3), np.float32)
    nrm = np.array([[0, 0, 1], [0, 0, 0]], np.float32)
    with pytest.raises(ValueError):
        oracle.spin_images(pts, nrm, 4, 1.0, 0.0, query_idx=[0])


def test_sphere_closed_form():
    """On a sphere of radius r with outward normals, beta = -|d|^2 / (2r), so every
    pair lies on alpha^2 + (beta + r)^2 = r^2 (to FP64 rounding)."""
    r = 1.7
    pts, nrm = wl.sphere(512, 7, radius=r)
    # radial normals recomputed from the FP32 points so the closed form is exact
    nrm = (pts / np.linalg.norm(pts.astype(np.float64), axis=1, keepdims=True)).astype(np.float32)
    for q in (0, 17, 300):
        a, b, ok = oracle.pair_coords(pts, nrm, q)
        # the FP32 normal is a rounded direction; the identity holds to ~1e-7 r
        resid = np.abs(a * a + (b + r) ** 2 - r * r)
        assert resid.max() < 5e-6 * r * r
        d = pts.astype(np.float64) - pts[q].astype(np.float64)
        d2 = (d * d).sum(1)
        assert np.all(b <= 1e-6)  # the sphere lies behind every tangent plane
        np.testing.assert_allclose(b, -d2 / (2 * r), rtol=0, atol=5e-6 * r)
        assert ok.all()  # cos S = -1 passes every pair


def test_sphere_image_hugs_the_curve():
    """Every nonzero pixel of a sphere image is adjacent to the curve
    alpha^2 + (beta + r)^2 = r^2 mapped to pixel coordinates."""
    r, W, B = 1.0, 16, 0.05
    pts, nrm = wl.sphere(2048, 11, radius=r)
    img, sup, _ = oracle.spin_images(pts, nrm, W, B, -1.0, query_idx=[0, 5, 9])
    h = W * B / 2
    # sample the curve densely: beta in [-2r, 0], alpha = sqrt(r^2 - (beta + r)^2)
    beta = np.linspace(-2 * r, 0, 200001)
    alpha = np.sqrt(np.maximum(0, r * r - (beta + r) ** 2))
    u = (h - beta) / B
    v = alpha / B
    near = set()
    for uu, vv in zip(np.floor(u).astype(int), np.floor(v).astype(int)):
        for di in (0, 1):
            for dj in (0, 1):
                near.add((uu + di, vv + dj))
    for k in range(3):
        nz = np.argwhere(img[k] > 0)
        assert len(nz) > 0
        for i, j in nz:
            assert (i, j) in near, (k, i, j)
        assert abs(img[k].sum() - sup[k]) < 1e-9


def test_plane_mass_in_middle_row():
    """Points in the plane z = 0 with normal (0,0,1): beta = 0, u = W/2 exactly,
    so all mass sits in row W/2 and row W/2 + 1 gets exactly 0."""
    rng = np.random.default_rng(3)
    n, W, B = 400, 16, 0.05
    xy = rng.uniform(-0.5, 0.5, (n, 2))
    pts = np.concatenate([xy, np.zeros((n, 1))], 1).astype(np.float32)
    nrm = np.tile(np.array([[0, 0, 1]], np.float32), (n, 1))
    img, sup, _ = oracle.spin_images(pts, nrm, W, B, 0.5, query_idx=np.arange(0, n, 37))
    for k in range(img.shape[0]):
        rows = img[k].sum(1)
        assert rows[W // 2 + 1] == 0.0
        assert abs(rows[W // 2] - sup[k]) < 1e-9
        assert abs(rows.sum() - rows[W // 2]) < 1e-9
        # support in the plane: alpha < (W-1) B
        d = np.linalg.norm(pts.astype(np.float64) - pts[k * 37].astype(np.float64), axis=1)
        assert sup[k] == int((d < (W - 1) * B).sum())


def test_angle_test_counts():
    """With S = 0 (cos S = 1) only pairs with identical normal directions pass;
    with S = pi (cos S = -1) the angle never rejects."""
    pts, nrm = wl.sphere(300, 5)
    nrm_flat = np.tile(np.array([[0, 0, 1]], np.float32), (300, 1))
    _, sup_all, _ = oracle.spin_images(pts, nrm_flat, 8, 0.3, -1.0, query_idx=[0, 1, 2])
    _, sup_one, _ = oracle.spin_images(pts, nrm_flat, 8, 0.3, 1.0, query_idx=[0, 1, 2])
    np.testing.assert_array_equal(sup_all, sup_one)  # identical normals pass at S = 0
    _, sup_radial, _ = oracle.spin_images(pts, nrm, 8, 0.3, 1.0, query_idx=[0, 1, 2])
    assert np.all(sup_radial == 1)  # only the self pair shares the exact direction


def _signed_permutation(pts, nrm, perm, signs, shift):
    p = pts[:, perm] * signs + shift
    n = nrm[:, perm] * signs
    return p.astype(np.float32), n.astype(np.float32)


def test_rigid_motion_invariance_exact():
    """Images are invariant under rigid motions.  A signed axis permutation is a
    rotation that is exact in FP32, and a dyadic shift of dyadic coordinates is
    exact too, so the moved input is the same geometry with no rounding."""
    rng = np.random.default_rng(8)
    n, W, B = 600, 8, 0.125
    pts = (np.round(rng.uniform(-1, 1, (n, 3)) * 1024) / 1024).astype(np.float32)
    nrm = rng.standard_normal((n, 3)).astype(np.float32)
    q = np.arange(0, n, 23).astype(np.int32)
    img0, sup0, flg0 = oracle.spin_images(pts, nrm, W, B, 0.2, query_idx=q)
    perm, signs = [2, 0, 1], np.array([-1.0, 1.0, -1.0])  # det = +1
    shift = np.array([0.375, -1.25, 2.5])
    p1, n1 = _signed_permutation(pts, nrm, perm, signs, shift)
    img1, sup1, flg1 = oracle.spin_images(p1, n1, W, B, 0.2, query_idx=q)
    for k in range(len(q)):
        tot = max(1.0, img0[k].sum())
        allow = flg0[k] + flg1[k]
        assert np.abs(img1[k] - img0[k]).sum() <= 1e-9 * tot + allow
        assert abs(int(sup1[k]) - int(sup0[k])) <= allow


def test_rigid_motion_invariance_general():
    """A general rotation and translation, rounded to FP32: images agree up to
    the input rounding (relative 1e-5 plus boundary pairs)."""
    pts, nrm = wl.heightfield(3000, 21)
    rng = np.random.default_rng(4)
    qv = rng.standard_normal(4)
    qv /= np.linalg.norm(qv)
    w, x, y, z = qv
    R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                  [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                  [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
    t = np.array([0.3, -0.7, 1.1])
    p1 = (pts.astype(np.float64) @ R.T + t).astype(np.float32)
    n1 = (nrm.astype(np.float64) @ R.T).astype(np.float32)
    q = np.arange(0, 3000, 97).astype(np.int32)
    W, B, c = 16, 0.02, 0.5
    img0, sup0, _ = oracle.spin_images(pts, nrm, W, B, c, query_idx=q)
    img1, sup1, _ = oracle.spin_images(p1, n1, W, B, c, query_idx=q)
    for k in range(len(q)):
        tot = img0[k].sum()
        # a pair whose threshold quantity moves across the threshold under the
        # ~1e-7 input rounding can flip; those are few and weigh at most 1 each
        flips = abs(int(sup1[k]) - int(sup0[k]))
        assert flips <= max(2, 1e-3 * sup0[k])
        assert np.abs(img1[k] - img0[k]).sum() <= 1e-4 * tot + 2.0 * (flips + 2)


def test_total_weight_equals_support_count():
    """Each pair splats total weight 1: the image sum equals the in-support count."""
    pts, nrm = wl.object_scene(4000, 9, n_objects=8)
    q = np.arange(0, 4000, 131).astype(np.int32)
    img, sup, _ = oracle.spin_images(pts, nrm, 12, 0.03, 0.0, query_idx=q)
    np.testing.assert_allclose(img.sum((1, 2)), sup, rtol=1e-12, atol=1e-9)
    assert np.all(img >= 0)
    assert sup.sum() > 0


def test_support_radius_bound():
    """Every in-support pair has |X - P| < R = sqrt(h^2 + ((W-1)B)^2), since
    |beta| <= h and alpha < (W - 1) B; and the FP32 candidate set brackets the
    exact-distance set."""
    pts, nrm = wl.heightfield(2500, 12)
    W, B = 16, 0.02
    R2 = oracle.support_radius2(W, B)
    assert R2 == pytest.approx((W * B / 2) ** 2 + ((W - 1) * B) ** 2, rel=1e-7)
    rc2 = float(oracle.candidate_rc2(W, B))
    assert rc2 == pytest.approx(R2 * (1 + 1e-5), rel=1e-7)
    q = np.arange(0, 2500, 53).astype(np.int32)
    cnt, hs = oracle.candidates_fp32(pts, W, B, query_idx=q)
    P64 = pts.astype(np.float64)
    for k, qi in enumerate(q):
        d2 = ((P64 - P64[qi]) ** 2).sum(1)
        lo = int((d2 <= rc2 * (1 - 1e-6)).sum())
        hi = int((d2 <= rc2 * (1 + 1e-6)).sum())
        assert lo <= cnt[k] <= hi
        a, b, ok = oracle.pair_coords(pts, nrm, qi, -1.0)
        u = (W * B / 2 - b) / B
        v = a / B
        inside = (u >= 0) & (u < W - 1) & (v < W - 1)
        assert np.all(d2[inside] < R2)
        # every in-support pair is a candidate
        assert int(inside.sum()) <= cnt[k]
        # the fingerprint depends on the set, not on the order of points
        assert hs[k] != 0 or cnt[k] == 0


def test_candidate_hash_is_order_independent():
    pts, _ = wl.sphere(700, 2)
    perm = np.random.default_rng(1).permutation(700)
    W, B = 8, 0.1
    cnt0, h0 = oracle.candidates_fp32(pts, W, B, query_idx=[0, 1, 2])
    # move the three query points to the front so their indices stay 0, 1, 2
    rest = [p for p in perm if p > 2]
    order = np.array([0, 1, 2] + rest)
    cnt1, h1 = oracle.candidates_fp32(pts[order], W, B, query_idx=[0, 1, 2])
    np.testing.assert_array_equal(cnt0, cnt1)
    # indices changed, so fingerprints generally differ; counts must not
    assert h0.shape == h1.shape


def test_query_subset_matches_full():
    """query_idx selects images; images do not depend on which others are made."""
    pts, nrm = wl.sphere(400, 3)
    full, sup_f, _ = oracle.spin_images(pts, nrm, 8, 0.2, 0.5)
    sub, sup_s, _ = oracle.spin_images(pts, nrm, 8, 0.2, 0.5, query_idx=[399, 0, 7, 7])
    np.testing.assert_array_equal(sub[0], full[399])
    np.testing.assert_array_equal(sub[1], full[0])
    np.testing.assert_array_equal(sub[2], full[7])
    np.testing.assert_array_equal(sub[3], full[7])
    assert sup_s[3] == sup_f[7]


def test_invalid_arguments():
    pts, nrm = wl.sphere(10, 1)
    with pytest.raises(ValueError):
        oracle.spin_images(pts, nrm, 1, 0.1, 0.0)
    with pytest.raises(ValueError):
        oracle.spin_images(pts, nrm, 4, 0.0, 0.0)
    with pytest.raises(ValueError):
        oracle.spin_images(pts, nrm, 4, 0.1, 1.5)
    with pytest.raises(ValueError):
        oracle.spin_images(pts, nrm, 4, 0.1, 0.0, query_idx=[10])
    with pytest.raises(ValueError):
        oracle.spin_images(pts, nrm, 4, float("nan"), 0.0)
    assert math.isfinite(oracle.support_radius2(4, 0.1))


@pytest.mark.parametrize("rule", ["static", "dynamic", "guided"])
def test_openmp_image_loop_equals_the_serial_oracle(rule):
    """The CPU baseline's parallel image loop computes the same images."""
    if not oracle.omp_available():
        pytest.skip("no OpenMP in the host compiler")
    pts, nrm = wl.heightfield(1500, 5)
    q = np.arange(0, 1500, 11).astype(np.int32)
    ref, sup, _ = oracle.spin_images(pts, nrm, 16, 0.02, 0.5, query_idx=q)
    img, sup2 = oracle.spin_images_omp(pts, nrm, 16, 0.02, 0.5, query_idx=q, rule=rule, threads=4)
    np.testing.assert_array_equal(img, ref)
    np.testing.assert_array_equal(sup2, sup)
