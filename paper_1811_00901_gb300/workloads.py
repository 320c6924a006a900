"""Seeded synthetic oriented-point sets and request streams.

This module generates INPUTS only (points, normals, query lists, parameters,
arrival times).  It holds none of the spin-image arithmetic, so both the CUDA
library's tests and the FP64 oracle can take their inputs from it.

The paper measures on the 3D mesh-watermarking data set (Sec. 4.1, Table 2:
ten meshes of roughly 3K to 826K points, Ramesses being the largest), which is
not available here.  These generators stand in for it with the same size range
and with the nonuniform point density that causes the load imbalance the
paper studies (Sec. 2.1, Fig. 2):

  sphere(n)           points uniform on the unit sphere, radial normals
  heightfield(n)      z = sum of 32 Gaussian bumps over [0,1]^2, xy density
                      varying 20:1 through 6 Gaussian clusters, analytic normals
  object_scene(n)     64 randomly posed tori and ellipsoids in [-1,1]^3 with
                      per-object density log-uniform in [1, 50], analytic normals

All generators take an explicit seed and use numpy's PCG64; the same seed
gives the same FP32 arrays on every machine.  Workload k uses seed
1811009010 + k.
"""
import math

import numpy as np

SEED_BASE = 1811009010


def _rng(seed):
    return np.random.Generator(np.random.PCG64(int(seed)))


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


# --------------------------------------------------------------------------
# geometry
# --------------------------------------------------------------------------

def sphere(n, seed, radius=1.0):
    """n points uniform on a sphere (normalised Gaussian triples), radial normals."""
    rng = _rng(seed)
    g = rng.standard_normal((n, 3))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    return _f32(g * radius), _f32(g)


def _bumps(rng, nbumps=32):
    amp = rng.uniform(-0.08, 0.08, nbumps)
    sig = rng.uniform(0.03, 0.12, nbumps)
    ctr = rng.uniform(0.0, 1.0, (nbumps, 2))
    return amp, sig, ctr


def _height_and_grad(xy, amp, sig, ctr):
    z = np.zeros(xy.shape[0])
    zx = np.zeros(xy.shape[0])
    zy = np.zeros(xy.shape[0])
    for a, s, c in zip(amp, sig, ctr):
        dx = xy[:, 0] - c[0]
        dy = xy[:, 1] - c[1]
        e = a * np.exp(-(dx * dx + dy * dy) / (2.0 * s * s))
        z += e
        zx += e * (-dx / (s * s))
        zy += e * (-dy / (s * s))
    return z, zx, zy


def _cluster_density(xy, cctr, csig):
    g = np.zeros(xy.shape[0])
    for c, s in zip(cctr, csig):
        d2 = (xy[:, 0] - c[0]) ** 2 + (xy[:, 1] - c[1]) ** 2
        g += np.exp(-d2 / (2.0 * s * s))
    return g


def heightfield(n, seed, ratio=20.0, nbumps=32, nclusters=6):
    """n points on z = sum_k A_k exp(-|xy - c_k|^2 / (2 s_k^2)) over [0,1]^2.

    A_k ~ U(-0.08, 0.08), s_k ~ U(0.03, 0.12), c_k ~ U[0,1]^2.  The xy
    sampling density is 1 + (ratio - 1) g(xy) / max g, g a sum of
    ``nclusters`` Gaussian clusters (sigma ~ U(0.05, 0.1)), drawn by
    rejection, so dense and sparse regions differ by ``ratio``.  Normals are
    the analytic (-z_x, -z_y, 1) / |.|.
    """
    rng = _rng(seed)
    amp, sig, ctr = _bumps(rng, nbumps)
    cctr = rng.uniform(0.0, 1.0, (nclusters, 2))
    csig = rng.uniform(0.05, 0.1, nclusters)
    gs = np.linspace(0.0, 1.0, 257)
    gx, gy = np.meshgrid(gs, gs)
    gmax = _cluster_density(np.stack([gx.ravel(), gy.ravel()], 1), cctr, csig).max()
    out = []
    have = 0
    while have < n:
        cand = rng.uniform(0.0, 1.0, (max(4 * (n - have), 1024), 2))
        rho = 1.0 + (ratio - 1.0) * _cluster_density(cand, cctr, csig) / gmax
        keep = rng.uniform(0.0, ratio, cand.shape[0]) < rho
        out.append(cand[keep])
        have += int(keep.sum())
    xy = np.concatenate(out)[:n]
    z, zx, zy = _height_and_grad(xy, amp, sig, ctr)
    pts = np.stack([xy[:, 0], xy[:, 1], z], 1)
    nrm = np.stack([-zx, -zy, np.ones_like(z)], 1)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    return _f32(pts), _f32(nrm)


def _random_rotation(rng):
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])


def _torus_points(rng, k, R, r):
    """k area-uniform points on a torus (major R, minor r) and their normals."""
    th_all, ph_all = [], []
    have = 0
    while have < k:
        m = max(2 * (k - have), 64)
        th = rng.uniform(0.0, 2 * math.pi, m)
        ph = rng.uniform(0.0, 2 * math.pi, m)
        keep = rng.uniform(0.0, R + r, m) < (R + r * np.cos(ph))
        th_all.append(th[keep])
        ph_all.append(ph[keep])
        have += int(keep.sum())
    th = np.concatenate(th_all)[:k]
    ph = np.concatenate(ph_all)[:k]
    ring = R + r * np.cos(ph)
    p = np.stack([ring * np.cos(th), ring * np.sin(th), r * np.sin(ph)], 1)
    nn = np.stack([np.cos(ph) * np.cos(th), np.cos(ph) * np.sin(th), np.sin(ph)], 1)
    return p, nn


def _ellipsoid_points(rng, k, ax):
    """k area-uniform points on an ellipsoid with semi-axes ax and normals."""
    a, b, c = ax
    gmax = max(b * c, a * c, a * b)
    out = []
    have = 0
    while have < k:
        m = max(2 * (k - have), 64)
        u = rng.standard_normal((m, 3))
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        g = np.sqrt((b * c * u[:, 0]) ** 2 + (a * c * u[:, 1]) ** 2 + (a * b * u[:, 2]) ** 2)
        keep = rng.uniform(0.0, gmax, m) < g
        out.append(u[keep])
        have += int(keep.sum())
    u = np.concatenate(out)[:k]
    p = u * np.array([a, b, c])
    nn = p / np.array([a * a, b * b, c * c])
    nn /= np.linalg.norm(nn, axis=1, keepdims=True)
    return p, nn


def _ellipsoid_area(ax):
    # Knud Thomsen's approximation (relative error below 1.1%); only used to
    # share the point budget between objects.
    p = 1.6075
    a, b, c = (x ** p for x in ax)
    return 4 * math.pi * ((a * b + a * c + b * c) / 3.0) ** (1.0 / p)


def object_scene(n, seed, n_objects=64, density_range=(1.0, 50.0)):
    """n points on randomly posed tori (first half) and ellipsoids (second half).

    Tori: R ~ U(0.08, 0.25), r ~ U(0.02, 0.08); ellipsoids: semi-axes
    ~ U(0.05, 0.25); uniform random rotation, centres ~ U[-0.8, 0.8]^3;
    per-object density log-uniform in ``density_range``; points shared in
    proportion to area x density, sampled area-uniformly.
    """
    rng = _rng(seed)
    objs = []
    for o in range(n_objects):
        if o < n_objects // 2:
            R = rng.uniform(0.08, 0.25)
            r = rng.uniform(0.02, 0.08)
            objs.append(("torus", (R, r), 4 * math.pi * math.pi * R * r))
        else:
            ax = tuple(rng.uniform(0.05, 0.25, 3))
            objs.append(("ellipsoid", ax, _ellipsoid_area(ax)))
    lo, hi = density_range
    dens = np.exp(rng.uniform(math.log(lo), math.log(hi), n_objects))
    w = np.array([o[2] for o in objs]) * dens
    counts = np.floor(n * w / w.sum()).astype(np.int64)
    counts[np.argsort(-w)[: n - int(counts.sum())]] += 1
    pts, nrms = [], []
    for (kind, prm, _), k in zip(objs, counts):
        rot = _random_rotation(rng)
        ctr = rng.uniform(-0.8, 0.8, 3)
        if k == 0:
            continue
        if kind == "torus":
            p, nn = _torus_points(rng, int(k), *prm)
        else:
            p, nn = _ellipsoid_points(rng, int(k), prm)
        pts.append(p @ rot.T + ctr)
        nrms.append(nn @ rot.T)
    return _f32(np.concatenate(pts)), _f32(np.concatenate(nrms))


def needle_layers(half_height, seed, axis=(0.31, -0.22, 0.93), origin=(0.4, 0.55, 0.3)):
    """Points along and across one tilted axis, all with the axis as normal:
    a needle of points on the axis (half of them exactly on it, half within
    0.02 h of it) at heights t = h (-0.9 + 0.00231 k), and five parallel discs
    (radius 0.3 h) perpendicular to the axis at heights h x {-0.75, -0.34, 0,
    0.28, 0.625}.  Pairs between them lie close to each other's normal axis at
    distances up to ~2h, the case where alpha, the distance from the axis, is
    small next to |X - P|.  No height difference comes within 5e-4 bins of a
    row threshold (u = 0 or u = W - 1) of a W x W image with half-height h
    for W in {16, 32, 64, 128}, and every alpha stays far below the last
    column, so no pair is near a support threshold.

    Returns (points, normals, t, lateral): t[k] the height along the axis and
    lateral[k] the in-plane offset (2 components) of point k before rounding
    to FP32."""
    rng = _rng(seed)
    h = float(half_height)
    n = np.asarray(axis, np.float64)
    n /= np.linalg.norm(n)
    e1 = np.cross(n, [1.0, 0.0, 0.0])
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(n, e1)
    t_needle = h * (-0.9 + 0.00231 * np.arange(int(1.85 / 0.00231) + 1))
    k = t_needle.size
    lat_needle = np.zeros((k, 2))
    r = rng.uniform(0.0, 0.02 * h, k // 2)
    a = rng.uniform(0.0, 2.0 * math.pi, k // 2)
    lat_needle[1::2][: k // 2] = np.stack([r * np.cos(a), r * np.sin(a)], 1)[: lat_needle[1::2].shape[0]]
    ts, lats = [t_needle], [lat_needle]
    for f in (-0.75, -0.34, 0.0, 0.28, 0.625):
        m = 400
        rr = 0.3 * h * np.sqrt(rng.uniform(0.0, 1.0, m))
        aa = rng.uniform(0.0, 2.0 * math.pi, m)
        ts.append(np.full(m, f * h))
        lats.append(np.stack([rr * np.cos(aa), rr * np.sin(aa)], 1))
    t = np.concatenate(ts)
    lat = np.concatenate(lats)
    pts = np.asarray(origin, np.float64) + t[:, None] * n + lat[:, :1] * e1 + lat[:, 1:] * e2
    nrm = np.tile(n, (t.size, 1))
    return _f32(pts), _f32(nrm), t, lat


def cos_deg(deg):
    """cos of a support angle in degrees, as the FP32 value passed to the library."""
    if deg >= 180.0:
        return np.float32(-1.0)
    return np.float32(math.cos(math.radians(deg)))


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------

def plain_sphere(n=4096):
    """4,096 points on the unit sphere; images for all points, W=16, B=0.05, 60 deg."""
    pts, nrm = sphere(n, SEED_BASE + 1)
    return dict(name="sphere-4096-W16", points=pts, normals=nrm, query_idx=None, m=n,
                W=16, bin_size=np.float32(0.05), cos_s=cos_deg(60.0))


def nonuniform_heightfield(n=100_000):
    """100,000-point clustered heightfield; images for all points, W=32, B=0.01, 60 deg."""
    pts, nrm = heightfield(n, SEED_BASE + 2)
    return dict(name="heightfield-100k-W32", points=pts, normals=nrm, query_idx=None, m=n,
                W=32, bin_size=np.float32(0.01), cos_s=cos_deg(60.0))


def large_scene(n=1_000_000, m=262_144):
    """1M points on 64 objects; 262,144 random queries, W=64, B=0.005, 90 deg."""
    pts, nrm = object_scene(n, SEED_BASE + 3)
    rng = _rng(SEED_BASE + 103)
    q = np.sort(rng.choice(n, size=m, replace=False)).astype(np.int32)
    return dict(name="scene-1M-W64", points=pts, normals=nrm, query_idx=q, m=m,
                W=64, bin_size=np.float32(0.005), cos_s=cos_deg(90.0))


def batched_spheres(count=512, n_range=(1_000, 200_000), seed=SEED_BASE + 4):
    """``count`` unit-sphere meshes, n log-uniform; per mesh W in {16,32,64},
    B = 0.8 / W, angle in {45, 60, 90} deg; images for all points."""
    rng = _rng(seed)
    lo, hi = n_range
    ns = np.exp(rng.uniform(math.log(lo), math.log(hi), count)).astype(np.int64)
    Ws = rng.choice([16, 32, 64], size=count)
    angs = rng.choice([45.0, 60.0, 90.0], size=count)
    items = []
    for k in range(count):
        pts, nrm = sphere(int(ns[k]), seed * 1000 + k)
        W = int(Ws[k])
        items.append(dict(points=pts, normals=nrm, query_idx=None, m=int(ns[k]), W=W,
                          bin_size=np.float32(0.8 / W), cos_s=cos_deg(float(angs[k]))))
    return items


def serving_pool(count=64, n_range=(10_000, 500_000), seed=SEED_BASE + 5):
    """``count`` resident meshes, n log-uniform; even slots spheres, odd slots
    object scenes."""
    rng = _rng(seed)
    lo, hi = n_range
    ns = np.exp(rng.uniform(math.log(lo), math.log(hi), count)).astype(np.int64)
    meshes = []
    for k in range(count):
        if k % 2 == 0:
            pts, nrm = sphere(int(ns[k]), seed * 1000 + k)
        else:
            pts, nrm = object_scene(int(ns[k]), seed * 1000 + k)
        meshes.append(dict(points=pts, normals=nrm))
    return meshes


def request_stream(mesh_sizes, count=10_000, rate_per_s=1000.0, m_range=(1, 10_000),
                   seed=SEED_BASE + 55):
    """Poisson request stream over a mesh pool.

    Each request: a mesh chosen uniformly, m log-uniform in ``m_range``
    query indices drawn uniformly (with replacement), W in {16, 32},
    B = 0.8 / W, support angle in {45, 60, 90} deg.  Arrival times are
    cumulative exponential gaps at ``rate_per_s``.
    """
    rng = _rng(seed)
    lo, hi = m_range
    gaps = rng.exponential(1.0 / rate_per_s, count)
    t = np.cumsum(gaps)
    reqs = []
    for k in range(count):
        mesh = int(rng.integers(0, len(mesh_sizes)))
        m = int(np.exp(rng.uniform(math.log(lo), math.log(hi + 1))))
        m = max(lo, min(hi, m))
        q = rng.integers(0, int(mesh_sizes[mesh]), m).astype(np.int32)
        W = int(rng.choice([16, 32]))
        ang = float(rng.choice([45.0, 60.0, 90.0]))
        reqs.append(dict(t=float(t[k]), mesh=mesh, query_idx=q, m=m, W=W,
                         bin_size=np.float32(0.8 / W), cos_s=cos_deg(ang)))
    return reqs
