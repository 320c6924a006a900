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


_FMIX_C1, _FMIX_C2 = 0x85EBCA6B, 0xC2B2AE35


def _fmix32_np(h):
    """MurmurHash3's 32-bit finaliser (Appleby), restated in NumPy from its
    published definition: xor-shift 16, multiply, xor-shift 13, multiply,
    xor-shift 16, all modulo 2^32."""
    h = np.asarray(h, dtype=np.uint64) & 0xFFFFFFFF
    h ^= h >> 16
    h = (h * _FMIX_C1) & 0xFFFFFFFF
    h ^= h >> 13
    h = (h * _FMIX_C2) & 0xFFFFFFFF
    h ^= h >> 16
    return h


def _unfmix32_np(h):
    """Inverse of the finaliser: undo each xor-shift by repeated shifting and
    each multiply by the modular inverse of its odd constant."""
    def unxorshift(x, k):
        y = x.copy()
        for _ in range(32 // k + 1):
            y = x ^ (y >> k)
        return y
    h = np.asarray(h, dtype=np.uint64) & 0xFFFFFFFF
    h = unxorshift(h, 16)
    h = (h * pow(_FMIX_C2, -1, 1 << 32)) & 0xFFFFFFFF
    h = unxorshift(h, 13)
    h = (h * pow(_FMIX_C1, -1, 1 << 32)) & 0xFFFFFFFF
    h = unxorshift(h, 16)
    return h


def test_fmix32_restatement_is_the_published_bijection():
    """The NumPy finaliser maps 0 to 0 and inverts exactly (every step of
    fmix32 is a bijection of 32-bit words), so the restatement used below has
    the published structure."""
    x = np.random.default_rng(9).integers(0, 1 << 32, 100000, dtype=np.uint64)
    assert int(_fmix32_np(0)) == 0
    np.testing.assert_array_equal(_unfmix32_np(_fmix32_np(x)), x)
    # the finaliser avalanches: one flipped input bit flips about half the output bits
    flips = np.unpackbits((_fmix32_np(x) ^ _fmix32_np(x ^ 1)).astype(">u4").view(np.uint8)).mean() * 32
    assert 14.0 < flips < 18.0


def test_candidate_fingerprint_against_fp64_set():
    """The candidate fingerprint is the sum, modulo 2^32, of fmix32 over the
    ORIGINAL indices of the candidate set.  Pinned against an independent
    computation: the FP64 distance set (on points whose FP64 distance is far
    from the threshold, where FP32 rounding cannot decide membership) hashed
    with the NumPy restatement.  A hash of another quantity (sorted position,
    a position shifted by one, the query's own index) fails here."""
    pts, _ = wl.sphere(1500, 12)
    W, B = 8, 0.1
    rc2 = float(oracle.candidate_rc2(W, B))
    P64 = pts.astype(np.float64)
    q = np.arange(0, 1500, 29).astype(np.int32)
    cnt, hs = oracle.candidates_fp32(pts, W, B, query_idx=q)
    checked = 0
    for k, qi in enumerate(q):
        d2 = ((P64 - P64[qi]) ** 2).sum(1)
        if np.any(np.abs(d2 - rc2) <= 1e-5 * rc2):
            continue  # a point near the threshold: FP32 decides it, not this pin
        members = np.nonzero(d2 <= rc2)[0]
        assert cnt[k] == members.size
        expect = int(_fmix32_np(members).sum() & 0xFFFFFFFF)
        assert int(hs[k]) == expect
        checked += 1
    assert checked >= 40
    # the same set under a permutation of the point order (indices follow the
    # points) gives the same fingerprint
    perm = np.random.default_rng(1).permutation(1500)
    inv = np.argsort(perm)
    cnt_p, hs_p = oracle.candidates_fp32(pts[perm], W, B, query_idx=inv[q].astype(np.int32))
    np.testing.assert_array_equal(cnt_p, cnt)
    relabel = [int(_fmix32_np(inv[np.nonzero(((P64 - P64[qi]) ** 2).sum(1) <= rc2)[0]]).sum() & 0xFFFFFFFF)
               for qi in q]
    far = [k for k, qi in enumerate(q) if not np.any(np.abs(((P64 - P64[qi]) ** 2).sum(1) - rc2) <= 1e-5 * rc2)]
    assert all(int(hs_p[k]) == relabel[k] for k in far)


@pytest.mark.parametrize("W", [16, 32, 64, 128])
def test_near_axis_closed_form(W):
    """Points on and next to the query's normal axis, where alpha is small
    next to |X - P| (a needle and parallel discs, all with the axis as normal,
    S = 180 deg).  By construction beta = t_X - t_P (heights along the axis)
    and alpha = |lateral_X - lateral_P| (in-plane offsets), so the image is the
    bilinear splat of those closed-form coordinates.  The oracle must match it
    up to the FP32 rounding of the input points (about 1e-5 of the total), with
    the support counts exact."""
    h = 0.16
    B = np.float32(2 * h / W)
    pts, nrm, t, lat = wl.needle_layers(h, 1)
    q = np.arange(0, pts.shape[0], 37).astype(np.int32)
    img, sup, flg = oracle.spin_images(pts, nrm, W, float(B), -1.0, query_idx=q)
    assert int(flg.sum()) == 0
    Bd = float(B)
    for k, qi in enumerate(q):
        u = W / 2 - (t - t[qi]) / Bd
        v = np.hypot(lat[:, 0] - lat[qi, 0], lat[:, 1] - lat[qi, 1]) / Bd
        i, j = np.floor(u), np.floor(v)
        ok = (i >= 0) & (i + 1 <= W - 1) & (j + 1 <= W - 1)
        a, b = (u - i)[ok], (v - j)[ok]
        ii, jj = i[ok].astype(int), j[ok].astype(int)
        e = np.zeros((W, W))
        np.add.at(e, (ii, jj), (1 - a) * (1 - b))
        np.add.at(e, (ii + 1, jj), a * (1 - b))
        np.add.at(e, (ii, jj + 1), (1 - a) * b)
        np.add.at(e, (ii + 1, jj + 1), a * b)
        assert int(ok.sum()) == int(sup[k])
        assert np.abs(e - img[k]).sum() <= 5e-5 * e.sum()


def _numpy_spin_images(pts, nrm, W, B, cos_s, q):
    """An independent NumPy restatement for small inputs: alpha as the length
    of n x d (equal to sqrt(|d|^2 - beta^2) for a unit n), the four corners
    accumulated with np.add.at over all pairs at once."""
    P = pts.astype(np.float64)
    N = nrm.astype(np.float64)
    N = N / np.linalg.norm(N, axis=1, keepdims=True)
    out = np.zeros((len(q), W, W))
    sup = np.zeros(len(q), np.int64)
    for k, qi in enumerate(q):
        d = P - P[qi]
        beta = d @ N[qi]
        alpha = np.linalg.norm(np.cross(N[qi], d), axis=1)
        u = W / 2 - beta / B
        v = alpha / B
        i, j = np.floor(u), np.floor(v)
        ok = (N @ N[qi] >= cos_s) & (i >= 0) & (i + 1 <= W - 1) & (j + 1 <= W - 1)
        a, b = (u - i)[ok], (v - j)[ok]
        ii, jj = i[ok].astype(int), j[ok].astype(int)
        np.add.at(out[k], (ii, jj), (1 - a) * (1 - b))
        np.add.at(out[k], (ii + 1, jj), a * (1 - b))
        np.add.at(out[k], (ii, jj + 1), (1 - a) * b)
        np.add.at(out[k], (ii + 1, jj + 1), a * b)
        sup[k] = ok.sum()
    return out, sup


@pytest.mark.parametrize("seed,n,W,B,deg", [(1, 64, 6, 0.2, 60.0), (2, 50, 9, 0.11, 45.0), (3, 64, 4, 0.4, 180.0),
                                            (4, 33, 16, 0.05, 90.0)])
def test_numpy_cross_check_small(seed, n, W, B, deg):
    """Brute force on tiny inputs: the oracle against an independent NumPy
    restatement (cross-product alpha, vectorised splat) on n <= 64 points,
    every image; pairs the oracle flags may differ by at most their weight."""
    pts, nrm = wl.object_scene(n, seed, n_objects=3)
    c = float(wl.cos_deg(deg))
    q = np.arange(n).astype(np.int32)
    img, sup, flg = oracle.spin_images(pts, nrm, W, np.float32(B), c, query_idx=q)
    ref, rsup = _numpy_spin_images(pts, nrm, W, float(np.float32(B)), c, q)
    assert sup.sum() > n  # the inputs exercise more than the self pairs
    for k in range(n):
        assert abs(int(sup[k]) - int(rsup[k])) <= flg[k]
        assert np.abs(img[k] - ref[k]).sum() <= 1e-9 * max(1.0, ref[k].sum()) + flg[k]


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
