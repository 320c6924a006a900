/*
 * spin_oracle.c -- plain, slow, single-threaded FP64 oracle for spin-image
 * generation.  TEST INFRASTRUCTURE ONLY: the tests, __graft_entry__.smoke()
 * and the CPU-baseline / reference legs of bench.py may load it; the product
 * path never does.  It shares no code, header or constant generator with the
 * CUDA library.
 *
 * What it computes (paper Sec. 2.1, Algorithm 1; Algorithm 2 is the same body
 * over an image range):
 *
 *   For every query oriented point P with normal n (normalised here in FP64)
 *   and EVERY oriented point X of the set OP (X = P included: the inner loop of
 *   Algorithm 1 runs over all M points):
 *
 *     angle test        n . n_X >= cos S          (acos(n . n_X) <= S)
 *     beta  = n . (X - P)
 *     alpha = sqrt(|X - P|^2 - beta^2)            (Algorithm 1's literal form)
 *     u = (h - beta) / B,  h = W*B/2              (row coordinate, from the top)
 *     v = alpha / B                               (column coordinate)
 *     support test      0 <= floor(u),  floor(u) + 1 <= W - 1,
 *                       floor(v) + 1 <= W - 1     (all four bilinear corners
 *                                                  inside the W x W image)
 *     splat             weight (1-a)(1-b), a(1-b), (1-a)b, ab at pixels
 *                       (i,j), (i+1,j), (i,j+1), (i+1,j+1), i = floor(u),
 *                       j = floor(v), a = u - i, b = v - j.
 *
 * Readings of the paper used here (the paper's Algorithm 1 counts the pixel
 * ceil((W/2 - beta)/B), ceil(alpha/B) with ++; the bilinear splat and the
 * "all four corners in range" support test replace that count):
 *   - W/2 in Algorithm 1 is read as the image half-height h = W*B/2 in length
 *     units, so u = (h - beta)/B = W/2 - beta/B.
 *   - B is the bin size in length units.
 *   - the angle test keeps the inclusive <=; S >= pi is passed as cos S = -1.
 *
 * Boundary flags.  FP32 evaluation can flip a pair's membership only when one
 * of its threshold quantities lies very close to its threshold.  A pair is
 * FLAGGED when every test it fails is near-threshold and at least one test is
 * near-threshold (so its membership could go either way):
 *   angle  near: |n.n_X - cos S| <= 1e-6 * max(1, |cos S|)
 *   u, v   near: |u - 0|, |u - (W-1)|, |v - (W-1)|  <=  1e-6 * s,
 *          s = max(1, |u|, |v|, |X-P|/B, h/B)
 * The scale s covers the FP32 rounding of beta and alpha, which grows with
 * |X - P|/B and h/B, not only with |u|, |v|.
 *
 * Candidate set (not in the paper; the paper is brute force over all M).  The
 * support test implies |X-P|^2 < R^2 = h^2 + ((W-1)B)^2.  The candidate set
 * is DEFINED in FP32 as { X : fl32(|X - P|^2) <= Rc2 } with
 *   d = fl32(X - P) componentwise,
 *   fl32(|d|^2) = fmaf(dz, dz, fmaf(dy, dy, dx*dx)),
 *   Rc2 = (float)(R^2 * (1 + 1e-5))  (R^2 evaluated in double),
 * the 1e-5 inflation keeping FP32 rounding of |d|^2 from dropping an
 * in-support pair.  oracle_candidates_fp32 evaluates exactly that definition
 * for every pair (compile with -ffp-contract=off so the compiler fuses nothing
 * beyond the fmaf calls written out).
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL -1
#define OR_EZERONORMAL -2

static int check_common(const float *points, const float *normals, int64_t n,
                        int32_t W, float bin_size)
{
    if (!points || !normals || n <= 0) return OR_EINVAL;
    if (W < 2) return OR_EINVAL;
    if (!(bin_size > 0.0f) || !isfinite(bin_size)) return OR_EINVAL;
    return OR_OK;
}

/* FP64 unit normal of oriented point k; returns 0 for a zero normal. */
static int unit_normal(const float *normals, int64_t k, double nu[3])
{
    double x = normals[3 * k], y = normals[3 * k + 1], z = normals[3 * k + 2];
    double len = sqrt(x * x + y * y + z * z);
    if (!(len > 0.0)) return 0;
    nu[0] = x / len;
    nu[1] = y / len;
    nu[2] = z / len;
    return 1;
}

/* Squared support radius R^2 = h^2 + ((W-1) B)^2 in double, h = W B / 2. */
double oracle_support_radius2(int32_t W, float bin_size)
{
    double B = (double)bin_size;
    double h = (double)W * B / 2.0;
    double r = (double)(W - 1) * B;
    return h * h + r * r;
}

/* Candidate-set threshold Rc2 = fl32(R^2 (1 + 1e-5)). */
float oracle_candidate_rc2(int32_t W, float bin_size)
{
    return (float)(oracle_support_radius2(W, bin_size) * (1.0 + 1e-5));
}

/*
 * Spin images of m query points (Algorithm 1 / 2 body), all pairs, FP64.
 *   points, normals : float[n][3]
 *   query_idx       : int32[m] indices into the point set, or NULL for 0..m-1
 *   img             : double[m][W][W] output (row i = u bin, column j = v bin)
 *   support         : int64[m] output, in-support pair count per image
 *   flagged         : int64[m] output, boundary-flagged pairs per image
 *                     (may be NULL)
 * Returns 0, OR_EINVAL, or OR_EZERONORMAL (a normal of length 0).
 */
int oracle_spin_images(const float *points, const float *normals, int64_t n,
                       const int32_t *query_idx, int64_t m, int32_t W,
                       float bin_size, float cos_s, double *img,
                       int64_t *support, int64_t *flagged)
{
    int rc = check_common(points, normals, n, W, bin_size);
    if (rc) return rc;
    if (m < 0 || (m > 0 && (!img || !support))) return OR_EINVAL;
    if (!(cos_s >= -1.0f && cos_s <= 1.0f)) return OR_EINVAL;

    const double B = (double)bin_size;
    const double h = (double)W * B / 2.0;
    const double cs = (double)cos_s;
    const double top = (double)(W - 1);
    const double angle_tol = 1e-6 * fmax(1.0, fabs(cs));
    const size_t npix = (size_t)W * (size_t)W;

    for (int64_t q = 0; q < m; ++q) {
        int64_t pi = query_idx ? (int64_t)query_idx[q] : q;
        if (pi < 0 || pi >= n) return OR_EINVAL;
        double *I = img + (size_t)q * npix;
        memset(I, 0, npix * sizeof(double));
        int64_t cnt = 0, nflag = 0;

        double np[3];
        if (!unit_normal(normals, pi, np)) return OR_EZERONORMAL;
        const double P[3] = {points[3 * pi], points[3 * pi + 1], points[3 * pi + 2]};

        for (int64_t j = 0; j < n; ++j) {
            double nx[3];
            if (!unit_normal(normals, j, nx)) return OR_EZERONORMAL;
            const double d[3] = {(double)points[3 * j] - P[0],
                                 (double)points[3 * j + 1] - P[1],
                                 (double)points[3 * j + 2] - P[2]};

            /* angle test: acos(n . n_X) <= S  <=>  n . n_X >= cos S */
            double c = np[0] * nx[0] + np[1] * nx[1] + np[2] * nx[2];
            int pass_a = c >= cs;
            int near_a = fabs(c - cs) <= angle_tol;

            /* beta, alpha as in Algorithm 1 */
            double beta = np[0] * d[0] + np[1] * d[1] + np[2] * d[2];
            double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            double a2 = d2 - beta * beta;
            double alpha = sqrt(a2 > 0.0 ? a2 : 0.0);

            double u = (h - beta) / B;
            double v = alpha / B;

            double s = 1.0;
            s = fmax(s, fabs(u));
            s = fmax(s, fabs(v));
            s = fmax(s, sqrt(d2) / B);
            s = fmax(s, h / B);
            double tol = 1e-6 * s;

            int pass_lo = u >= 0.0, near_lo = fabs(u) <= tol;
            int pass_hi = u < top, near_hi = fabs(u - top) <= tol;
            int pass_v = v < top, near_v = fabs(v - top) <= tol;

            int inside = pass_a && pass_lo && pass_hi && pass_v;
            int could = (pass_a || near_a) && (pass_lo || near_lo) &&
                        (pass_hi || near_hi) && (pass_v || near_v);
            int near_any = near_a || near_lo || near_hi || near_v;
            if (could && near_any) ++nflag;
            if (!inside) continue;

            ++cnt;
            double fi = floor(u), fj = floor(v);
            double a = u - fi, b = v - fj;
            size_t i = (size_t)fi, jj = (size_t)fj;
            I[i * W + jj] += (1.0 - a) * (1.0 - b);
            I[(i + 1) * W + jj] += a * (1.0 - b);
            I[i * W + jj + 1] += (1.0 - a) * b;
            I[(i + 1) * W + jj + 1] += a * b;
        }
        support[q] = cnt;
        if (flagged) flagged[q] = nflag;
    }
    return OR_OK;
}

/*
 * Pre-binning coordinates of every pair of one query, FP64 (for closed-form
 * checks): alpha[j], beta[j] as in Algorithm 1 and angle_ok[j] = (n.n_X >= cos S).
 */
int oracle_pair_coords(const float *points, const float *normals, int64_t n,
                       int64_t query, float cos_s, double *alpha, double *beta,
                       int32_t *angle_ok)
{
    if (!points || !normals || n <= 0 || query < 0 || query >= n) return OR_EINVAL;
    if (!alpha || !beta || !angle_ok) return OR_EINVAL;
    double np[3];
    if (!unit_normal(normals, query, np)) return OR_EZERONORMAL;
    const double P[3] = {points[3 * query], points[3 * query + 1], points[3 * query + 2]};
    for (int64_t j = 0; j < n; ++j) {
        double nx[3];
        if (!unit_normal(normals, j, nx)) return OR_EZERONORMAL;
        const double d[3] = {(double)points[3 * j] - P[0],
                             (double)points[3 * j + 1] - P[1],
                             (double)points[3 * j + 2] - P[2]};
        double b = np[0] * d[0] + np[1] * d[1] + np[2] * d[2];
        double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        double a2 = d2 - b * b;
        beta[j] = b;
        alpha[j] = sqrt(a2 > 0.0 ? a2 : 0.0);
        angle_ok[j] = (np[0] * nx[0] + np[1] * nx[1] + np[2] * nx[2]) >= (double)cos_s;
    }
    return OR_OK;
}

/* MurmurHash3's 32-bit finaliser (fmix32), as published by Austin Appleby. */
static uint32_t fmix32(uint32_t h)
{
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

/*
 * The FP32 candidate set of each query (definition in the header comment):
 * count[q] = |{X}| and hash[q] = sum over X of fmix32(index of X) mod 2^32
 * (an order-independent fingerprint of the set).
 */
int oracle_candidates_fp32(const float *points, int64_t n,
                           const int32_t *query_idx, int64_t m, int32_t W,
                           float bin_size, int64_t *count, uint32_t *hash)
{
    if (!points || n <= 0 || m < 0 || W < 2) return OR_EINVAL;
    if (!(bin_size > 0.0f) || !isfinite(bin_size)) return OR_EINVAL;
    if (m > 0 && (!count || !hash)) return OR_EINVAL;
    const float rc2 = oracle_candidate_rc2(W, bin_size);
    for (int64_t q = 0; q < m; ++q) {
        int64_t pi = query_idx ? (int64_t)query_idx[q] : q;
        if (pi < 0 || pi >= n) return OR_EINVAL;
        const float px = points[3 * pi], py = points[3 * pi + 1], pz = points[3 * pi + 2];
        int64_t c = 0;
        uint32_t hs = 0;
        for (int64_t j = 0; j < n; ++j) {
            float dx = points[3 * j] - px;
            float dy = points[3 * j + 1] - py;
            float dz = points[3 * j + 2] - pz;
            float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            if (d2 <= rc2) {
                ++c;
                hs += fmix32((uint32_t)j);
            }
        }
        count[q] = c;
        hash[q] = hs;
    }
    return OR_OK;
}

/*
 * Algorithm 1's own count ("nearest-bin" binning, the paper-literal form):
 * pixel (k, l) = (ceil(u), ceil(v)) of every pair that passes the angle test
 * gets 1 when 0 <= k <= W-1 and 0 <= l <= W-1, with u = W/2 - beta/B (the
 * half-height reading of Algorithm 1's W/2) and v = alpha/B.
 *
 * Precision.  ceil() turns a rounded coordinate into a pixel index, so this
 * function and the GPU take that decision in the same precision: IEEE FP32
 * (round to nearest even), every operation in this order (compile with
 * -ffp-contract=off so that only the fmaf calls written here fuse):
 *   unit normal   l2 = fmaf(nz, nz, fmaf(ny, ny, nx*nx)); s = sqrtf(l2);
 *                 inv = 1/s; n = (nx*inv, ny*inv, nz*inv)
 *   d             = X - P componentwise; |d|^2 = fmaf(dz, dz, fmaf(dy, dy, dx*dx))
 *   angle         fmaf(n.z, nX.z, fmaf(n.y, nX.y, n.x*nX.x)) >= cos S
 *   beta          = fmaf(n.z, dz, fmaf(n.y, dy, n.x*dx))
 *   alpha         = sqrtf(max(fmaf(-beta, beta, |d|^2), 0))
 *   u             = W/2 - beta/B;  v = alpha/B  (correctly rounded division)
 *   k, l          = ceilf(u), ceilf(v)
 * X = P is included (u = W/2, v = 0: pixel (ceil(W/2), 0)).
 *
 *   counts  : int32[m][W][W] output (row k, column l)
 *   support : int64[m] output, pairs counted per image
 *   max_d2  : float[m] output (may be NULL): the largest fl32 |d|^2 of a
 *             counted pair, 0 when none (bounds the radius a culling grid needs)
 * Returns 0, OR_EINVAL, or OR_EZERONORMAL.
 */
static int unit_normal_fp32(const float *normals, int64_t k, float nu[3])
{
    float x = normals[3 * k], y = normals[3 * k + 1], z = normals[3 * k + 2];
    float l2 = fmaf(z, z, fmaf(y, y, x * x));
    if (!(l2 > 0.0f) || !isfinite(l2)) return 0;
    float inv = 1.0f / sqrtf(l2);
    nu[0] = x * inv;
    nu[1] = y * inv;
    nu[2] = z * inv;
    return 1;
}

int oracle_spin_images_nearest(const float *points, const float *normals, int64_t n,
                               const int32_t *query_idx, int64_t m, int32_t W,
                               float bin_size, float cos_s, int32_t *counts,
                               int64_t *support, float *max_d2)
{
    int rc = check_common(points, normals, n, W, bin_size);
    if (rc) return rc;
    if (m < 0 || (m > 0 && (!counts || !support))) return OR_EINVAL;
    if (!(cos_s >= -1.0f && cos_s <= 1.0f)) return OR_EINVAL;
    const float half_w = 0.5f * (float)W;
    const float top = (float)(W - 1);
    const size_t npix = (size_t)W * (size_t)W;

    for (int64_t q = 0; q < m; ++q) {
        int64_t pi = query_idx ? (int64_t)query_idx[q] : q;
        if (pi < 0 || pi >= n) return OR_EINVAL;
        int32_t *C = counts + (size_t)q * npix;
        memset(C, 0, npix * sizeof(int32_t));
        float np[3];
        if (!unit_normal_fp32(normals, pi, np)) return OR_EZERONORMAL;
        const float px = points[3 * pi], py = points[3 * pi + 1], pz = points[3 * pi + 2];
        int64_t cnt = 0;
        float dmax = 0.0f;
        for (int64_t j = 0; j < n; ++j) {
            float nx[3];
            if (!unit_normal_fp32(normals, j, nx)) return OR_EZERONORMAL;
            const float dx = points[3 * j] - px;
            const float dy = points[3 * j + 1] - py;
            const float dz = points[3 * j + 2] - pz;
            const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            const float ca = fmaf(np[2], nx[2], fmaf(np[1], nx[1], np[0] * nx[0]));
            if (!(ca >= cos_s)) continue;
            const float beta = fmaf(np[2], dz, fmaf(np[1], dy, np[0] * dx));
            const float a2 = fmaf(-beta, beta, d2);
            const float alpha = sqrtf(a2 > 0.0f ? a2 : 0.0f);
            const float u = half_w - beta / bin_size;
            const float v = alpha / bin_size;
            const float k = ceilf(u), l = ceilf(v);
            if (!(k >= 0.0f && k <= top && l >= 0.0f && l <= top)) continue;
            C[(size_t)k * W + (size_t)l] += 1;
            ++cnt;
            if (d2 > dmax) dmax = d2;
        }
        support[q] = cnt;
        if (max_d2) max_d2[q] = dmax;
    }
    return OR_OK;
}
