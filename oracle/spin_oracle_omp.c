/*
 * spin_oracle_omp.c -- the FP64 oracle's all-pairs spin images, the image
 * loop spread over the host's cores with OpenMP.  TEST AND CPU-REFERENCE
 * INFRASTRUCTURE ONLY (bench.py's CPU baseline): it is the shared-memory CPU
 * analogue of the paper's PSIA-STATIC / EPSIA-SS / EPSIA-GSS (Sec. 2.2, 3),
 * the image loop scheduled by OpenMP's schedule(static), schedule(dynamic, 1)
 * and schedule(guided).  Every image is computed by oracle_spin_images of
 * spin_oracle.c, one query at a time, so the results equal the serial
 * oracle's.
 */
#include <omp.h>
#include <stdint.h>
#include <stddef.h>

int oracle_spin_images(const float *points, const float *normals, int64_t n,
                       const int32_t *query_idx, int64_t m, int32_t W,
                       float bin_size, float cos_s, double *img,
                       int64_t *support, int64_t *flagged);

/* rule: 0 static, 1 dynamic with chunk 1, 2 guided.  threads <= 0: all.
 * Returns the first nonzero oracle code, else 0. */
int oracle_spin_images_omp(const float *points, const float *normals, int64_t n,
                           const int32_t *query_idx, int64_t m, int32_t W,
                           float bin_size, float cos_s, double *img,
                           int64_t *support, int32_t rule, int32_t threads)
{
    if (rule < 0 || rule > 2 || m < 0) return -1;
    if (threads > 0) omp_set_num_threads(threads);
    const size_t npix = (size_t)W * (size_t)W;
    int rc = 0;
    if (rule == 0) {
#pragma omp parallel for schedule(static) reduction(| : rc)
        for (int64_t q = 0; q < m; ++q) {
            int32_t idx = query_idx ? query_idx[q] : (int32_t)q;
            rc |= oracle_spin_images(points, normals, n, &idx, 1, W, bin_size, cos_s, img + (size_t)q * npix,
                                     support + q, NULL);
        }
    } else if (rule == 1) {
#pragma omp parallel for schedule(dynamic, 1) reduction(| : rc)
        for (int64_t q = 0; q < m; ++q) {
            int32_t idx = query_idx ? query_idx[q] : (int32_t)q;
            rc |= oracle_spin_images(points, normals, n, &idx, 1, W, bin_size, cos_s, img + (size_t)q * npix,
                                     support + q, NULL);
        }
    } else {
#pragma omp parallel for schedule(guided) reduction(| : rc)
        for (int64_t q = 0; q < m; ++q) {
            int32_t idx = query_idx ? query_idx[q] : (int32_t)q;
            rc |= oracle_spin_images(points, normals, n, &idx, 1, W, bin_size, cos_s, img + (size_t)q * npix,
                                     support + q, NULL);
        }
    }
    return rc;
}

int oracle_omp_max_threads(void) { return omp_get_max_threads(); }
