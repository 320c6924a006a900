"""Pins of the oracle's paper-literal binning (Algorithm 1's own count,
pixel (ceil(u), ceil(v)) += 1), evaluated in IEEE FP32.  Each pin comes from
outside the oracle: a hand-evaluated image, the flat-patch case that reduces
to a radial distance histogram, the sphere's closed-form (alpha, beta) curve,
the FP64 pair coordinates, and the radius bound that a culling grid uses."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1811_00901_gb300 import workloads as wl


def test_hand_evaluated_image(golden_dir):
    with open(os.path.join(golden_dir, "nearest_hand.json")) as f:
        g = json.load(f)
    pts = np.array(g["points"], np.float32)
    nrm = np.array(g["normals"], np.float32)
    cnt, sup, _ = oracle.spin_images_nearest(pts, nrm, g["W"], g["B"], g["cos_s"],
                                             query_idx=np.array([g["query"]], np.int32))
    np.testing.assert_array_equal(cnt[0], np.array(g["counts"]))
    assert sup[0] == g["support"]


def test_unnormalised_normals_give_the_same_counts(golden_dir):
    with open(os.path.join(golden_dir, "nearest_hand.json")) as f:
        g = json.load(f)
    pts = np.array(g["points"], np.float32)
    nrm = np.array(g["normals"], np.float32) * np.float32(4.0)   # power-of-two lengths stay exact
    cnt, _, _ = oracle.spin_images_nearest(pts, nrm, g["W"], g["B"], g["cos_s"],
                                           query_idx=np.array([g["query"]], np.int32))
    np.testing.assert_array_equal(cnt[0], np.array(g["counts"]))


def test_normal_length_does_not_matter_on_a_sphere():
    """Scaling every normal by 4 or 1/2 (exact in FP32) leaves the unit normals,
    and so every count, unchanged."""
    c = wl.plain_sphere()
    pts, nrm = c["points"][:1500], c["normals"][:1500]
    q = np.array([0, 9, 1000], np.int32)
    ref, _, _ = oracle.spin_images_nearest(pts, nrm, 16, 0.05, 0.5, query_idx=q)
    scale = np.where(np.arange(1500) % 2 == 0, np.float32(4.0), np.float32(0.5)).astype(np.float32)[:, None]
    got, _, _ = oracle.spin_images_nearest(pts, nrm * scale, 16, 0.05, 0.5, query_idx=q)
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("W,B", [(8, 0.05), (16, 0.02), (5, 0.1)])
def test_flat_patch_is_a_radial_histogram(W, B):
    """Coplanar points with the plane's normal: beta = 0 for every pair, so all
    counts sit in row ceil(W/2) and column l counts the points at distance in
    ((l-1)B, lB] -- a histogram of FP64 distances, away from bin edges."""
    rng = np.random.default_rng(5)
    n = 3000
    pts = np.zeros((n, 3), np.float32)
    pts[:, :2] = rng.uniform(-0.5, 0.5, (n, 2)).astype(np.float32)
    nrm = np.tile(np.array([[0, 0, 1]], np.float32), (n, 1))
    q = np.array([0, 17, 999], np.int32)
    cnt, sup, _ = oracle.spin_images_nearest(pts, nrm, W, B, -1.0, query_idx=q)
    row = int(np.ceil(W / 2))
    for k, qi in enumerate(q):
        other = np.delete(np.arange(W), row)
        assert cnt[k][other].sum() == 0
        d = np.sqrt(((pts.astype(np.float64) - pts[qi].astype(np.float64)) ** 2).sum(1)) / B
        edge = np.abs(d - np.round(d)) < 1e-4
        lcol = np.ceil(d).astype(np.int64)
        inside = lcol <= W - 1
        hist = np.bincount(lcol[inside & ~edge], minlength=W)[:W]
        n_edge = int((edge & (d <= W - 1 + 1e-4)).sum())
        diff = np.abs(cnt[k][row].astype(np.int64) - hist)
        assert diff.sum() <= n_edge, (qi, diff, n_edge)
        assert abs(int(sup[k]) - int(inside[~edge].sum())) <= n_edge


def test_sphere_counts_lie_on_the_closed_form_curve():
    """Unit sphere, radial normals: (alpha, beta) of every pair lies on
    alpha^2 + (beta + 1)^2 = 1.  A pixel (k, l) covers u in (k-1, k],
    v in (l-1, l]; every non-empty pixel must meet the curve."""
    pts, nrm = wl.plain_sphere()["points"][:1500], wl.plain_sphere()["normals"][:1500]
    W, B = 16, 0.05
    q = np.array([0, 3, 700], np.int32)
    cnt, _, _ = oracle.spin_images_nearest(pts, nrm, W, B, 0.5, query_idx=q)
    v = np.linspace(0.0, 1.0, 20001)
    for k in range(len(q)):
        ks, ls = np.nonzero(cnt[k])
        assert len(ks) > 3
        for i, j in zip(ks, ls):
            # on the curve, beta = -1 + sqrt(1 - alpha^2) (the near branch, n.n_X >= 0.5)
            a = (j - 1 + v) * B
            ok = a <= 1.0
            beta = -1.0 + np.sqrt(1.0 - a[ok] ** 2)
            u = W / 2 - beta / B
            assert np.any((u > i - 1 - 1e-3) & (u <= i + 1e-3)), (k, i, j)


def test_total_count_matches_fp64_coordinates():
    """The count per image equals the number of pairs with cos test passed,
    -1 < u <= W-1 and v <= W-1 in FP64, up to pairs within 1e-5 of an edge."""
    c = wl.plain_sphere()
    pts, nrm = c["points"][:2000], c["normals"][:2000]
    W, B, cs = 16, 0.05, 0.5
    for qi in (1, 42, 1999):
        alpha, beta, ok = oracle.pair_coords(pts, nrm, qi, cs)
        u = W / 2 - beta / B
        v = alpha / B
        inside = ok & (u > -1) & (u <= W - 1) & (v <= W - 1)
        tol = 1e-5 * np.maximum(1.0, np.abs(u))
        edge = (np.abs(u + 1) < tol) | (np.abs(u - (W - 1)) < tol) | (np.abs(v - (W - 1)) < 1e-5 * max(1, W))
        _, sup, _ = oracle.spin_images_nearest(pts, nrm, W, B, cs, query_idx=np.array([qi], np.int32))
        assert abs(int(sup[0]) - int(inside.sum())) <= int(edge.sum())


@pytest.mark.parametrize("W,B", [(16, 0.05), (32, 0.01), (4, 1.0)])
def test_counted_pairs_lie_within_the_nearest_bin_radius(W, B):
    """A counted pair has |beta| < (W/2 + 1) B and alpha <= (W-1) B, so
    |d|^2 < ((W/2+1)B)^2 + ((W-1)B)^2; the FP32 |d|^2 of every counted pair
    stays below that radius inflated by 1e-5 (the grid's culling threshold)."""
    c = wl.heightfield(3000, 3)
    pts, nrm = c[0], c[1]
    _, _, dmax = oracle.spin_images_nearest(pts, nrm, W, B, -1.0, query_idx=np.arange(0, 3000, 7).astype(np.int32))
    r2 = ((W / 2 + 1) * B) ** 2 + ((W - 1) * B) ** 2
    assert float(dmax.max()) <= np.float32(r2 * (1 + 1e-5))
