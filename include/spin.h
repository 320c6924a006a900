/*
 * spin.h -- C ABI of the GB300 spin-image library (libspin_gb300.so).
 *
 * Spin images (Sec. 2.1, Algorithm 1): for every query oriented point P with
 * unit normal n and every oriented point X of the set (X = P included),
 *   beta  = n . (X - P),   alpha = sqrt(|X-P|^2 - beta^2),
 *   u = W/2 - beta/B (row, from the top),  v = alpha/B (column),
 * X contributes when n . n_X >= cos S (the support-angle test of Algorithm 1)
 * and all four bilinear corners lie inside the W x W image:
 *   0 <= floor(u),  floor(u) + 1 <= W - 1,  floor(v) + 1 <= W - 1.
 * Each contributing X adds weight 1, split bilinearly over the four corners.
 *
 * Output format (every entry point): int32 out[m][W][W], row-major, row i =
 * u bin, column j = v bin, value = weight x 65536 (16 fractional bits; with
 * SI_BIN_NEAREST, Algorithm 1's own count, the value is the count).  The
 * coordinates are quantised as U = rn(u * 65536), V = rn(v * 65536) (round to
 * nearest even); with A = U mod 65536, Bq = V mod 65536, i = U >> 16,
 * j = V >> 16 the corner weights are
 *   w11 = (A * Bq + 32768) >> 16,  w10 = A - w11,  w01 = Bq - w11,
 *   w00 = 65536 - A - Bq + w11      (all >= 0, sum exactly 65536),
 * added at (i,j) w00, (i+1,j) w10, (i,j+1) w01, (i+1,j+1) w11.  Integer
 * accumulation makes every image independent of scheduling, worker count and
 * batch composition: results are bit-identical across all of them.
 *
 * Image loop scheduling (Sec. 2.2 and Algorithm 3): the loop over images is
 * run by persistent thread blocks ("workers") that take chunks of the loop
 * under STATIC, SS, GSS or FAC (and FAC_PROB, AWF, AF).  The scheduled iteration
 * is one image GROUP:
 * `group` consecutive images (in grid order) that a worker generates together
 * against one shared stream of candidate points.
 *
 * Conventions
 *  - Status codes only; nothing throws across this boundary.
 *  - Argument errors are reported synchronously; no work is enqueued then.
 *  - Work is stream-ordered and asynchronous: a call returns after enqueueing.
 *    The caller synchronises its stream before reading `out`.
 *  - Device-side conditions (int32 pixel overflow, a bounded wait that gave
 *    up) are recorded on the mesh and reported by si_get_stats.
 *  - Pointers named "device" must be CUDA device memory of the current
 *    device; "host or device" pointers may be either (the library inspects
 *    them).  The caller owns every buffer it passes; buffers used by an
 *    enqueued call must stay valid until the stream reaches that point.
 *  - A NULL stream is the legacy default stream.
 *  - Handles are not thread-safe, except a server (si_serve_*), whose calls
 *    may come from any thread.
 *  - si_last_error() returns a thread-local message about the last failure.
 */
#ifndef SPIN_GB300_H
#define SPIN_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *si_stream; /* the same type as cudaStream_t */
typedef struct si_mesh_s *si_mesh_t;
typedef struct si_server_s *si_server_t;

typedef enum si_status {
    SI_OK = 0,
    SI_ERR_INVALID = 1,  /* bad argument; nothing was enqueued */
    SI_ERR_CUDA = 2,     /* a CUDA runtime call failed */
    SI_ERR_OOM = 3,      /* device or pinned-host allocation failed */
    SI_ERR_OVERFLOW = 4, /* a pixel exceeded INT32_MAX (more than 32767 points in one pixel) */
    SI_ERR_TIMEOUT = 5,  /* a wait ran out of time */
    SI_ERR_BUSY = 6      /* a server refused a request (memory budget / in-flight limit) */
} si_status;

/* Loop-scheduling rules, Sec. 2.2 (SS, GSS, FAC) and PSIA's static split. */
typedef enum si_sched_kind {
    SI_SCHED_STATIC = 0, /* worker k takes groups [floor(kU/P), floor((k+1)U/P)), no atomics */
    SI_SCHED_SS = 1,     /* one group (min_chunk groups) per request */
    SI_SCHED_GSS = 2,    /* ceil(remaining / P) groups per request, >= min_chunk */
    SI_SCHED_FAC = 3,    /* batches of P equal chunks of ceil(remaining / (2P)), >= min_chunk */
    SI_SCHED_FAC_PROB = 4 /* factoring with the batch size of its original probabilistic rule
                             (Hummel, Schonberg and Flynn, 1992 -- the paper's reference for FAC):
                             batch j hands out P chunks of ceil(R_j / (x_j P)), R_j what remains,
                             b_j = P / (2 sqrt(R_j)) * cov, x_0 = 1 + b_0^2 + b_0 sqrt(b_0^2 + 2),
                             x_j = 2 + b_j^2 + b_j sqrt(b_j^2 + 4) (j >= 1), cov = sigma / mu of the
                             iteration time (si_schedule.fac_cov), evaluated in IEEE double;
                             >= min_chunk */,
    SI_SCHED_AWF = 5      /* adaptive weighted factoring: batches of P chunks as FAC, the batch
                             chunk being FAC2 on the groups that remain at the claim, ceil(R / (2P)),
                             and half that for the first batch (claims 0 .. P-1, made before any
                             rate exists); each chunk scaled by the requesting worker's weight
                             w = rate / (mean rate of the workers measured so far), rate = its groups
                             done / its time so far (measured on the device, updated after every
                             chunk; w = 1 before a worker's first chunk ends; w clamped to
                             [0.05, 20]); chunk = max(min_chunk, round(w x batch chunk)).  Chunk
                             sizes depend on measured times and are decided on the device; every
                             group is still generated exactly once.  In a batched call every item
                             must use it. */,
    SI_SCHED_AF = 6       /* adaptive factoring (Banicescu and Liu, 2000; an adaptive rule of the kind
                             Sec. 2.2 leaves to future work): each worker measures the mean mu_i and
                             variance sigma_i^2 of its time per group (on the device; a chunk's
                             wall time, claim and any emulated slowdown included, spread over its
                             groups) and, with R groups remaining, D = sum sigma_j^2 / mu_j and
                             E = 1 / sum 1 / mu_j over the workers measured so far (scaled to all
                             P), takes ceil((D + 2ER - sqrt(D^2 + 4DER)) / (2 mu_i)) groups; before
                             its first chunk ends, ceil(R / (4P)).  Chunks are >= min_chunk and
                             are decided on the device; every group is still generated exactly
                             once.  In a batched call every item must use it. */
} si_sched_kind;

/* How a contributing pair is counted into its image. */
typedef enum si_binning {
    SI_BIN_BILINEAR = 0, /* weight 1 split over the four pixels around (u, v), fixed point x 65536 */
    SI_BIN_NEAREST = 1   /* Algorithm 1's own count: pixel (ceil(u), ceil(v)) += 1 for
                            0 <= ceil(u), ceil(v) <= W - 1, evaluated in IEEE FP32 as specified
                            at si_generate */
} si_binning;

/* Scheduling and launch shape.  Zero fields mean "choose automatically". */
typedef struct si_schedule {
    int32_t kind;        /* si_sched_kind */
    int32_t min_chunk;   /* lower bound of a dynamic chunk, in groups (0 -> 1) */
    int32_t num_workers; /* persistent thread blocks P (0 -> all SMs x blocks per SM, the count
                            si_default_workers returns) */
    int32_t group;       /* images per group: 1, 2, 4, 8, 16 or 32 (0 -> by W) */
    int32_t grid_div;    /* grid cells per candidate radius, 1..16 (0 -> 8, or 6 for W >= 64) */
    int32_t slices;      /* blocks that share one group's candidate stream, 1..64; each adds
                            its partial images into `out` with integer atomics (results are
                            unchanged).  0 -> auto: 1 when the call has enough groups to fill
                            the GPU, more for calls with few groups (small requests). */
    int32_t binning;     /* si_binning (0 -> bilinear) */
    int32_t slow_workers;/* heterogeneity emulation (the paper's Type1 + Type2 runs, Sec. 5.2):
                            workers 0 .. slow_workers-1 are slow.  They request first -- worker
                            k < slow_workers takes scheduling step k -- and after each step a slow
                            worker idles (slowdown - 1) x the time the step took (at most 1 s).
                            Results are unchanged.  0 -> no emulation.  For batched calls the
                            emulation comes from the override (or the first item's rule). */
    float slowdown;      /* >= 1 (0 -> 1) */
    float fac_cov;       /* SI_SCHED_FAC_PROB: sigma / mu of an iteration's time, finite, >= 0 */
    int32_t order;       /* order in which the dynamic rules hand out the groups: 0 -> grid order
                            (the loop as written); 1 -> decreasing estimated cost (the number of
                            candidates in each group's grid stencil, bucketed by 2^(1/32)), so
                            the cheapest groups come last and the last chunks balance the
                            workers' finishing times.  Within a run of equal chunks of the
                            rule's table (a FAC batch) the sorted groups are dealt round-robin
                            over the chunks, so that no chunk bundles the costliest ones.  The
                            estimate costs three small kernels per call.  Results are unchanged.
                            STATIC always runs grid order. */
} si_schedule;

/* Optional per-image probes (device buffers of m entries, each may be NULL).
 * Probing slows the kernel down; it is meant for tests and tuning. */
typedef struct si_probe {
    int64_t *culled;     /* |{X : fl32(|X-P|^2) <= Rc2}| (candidate set, see si_candidate_rc2) */
    uint32_t *cand_hash; /* sum over that set of fmix32(index of X), mod 2^32 */
    int64_t *support;    /* number of contributing X */
    int32_t *worker;     /* thread block that generated the image */
    int32_t *step;       /* scheduling step whose chunk contained the image */
    int64_t *examined;   /* candidate points the kernel streamed for the image (the grid
                            stencil; examined / culled is the culling overhead) */
    int64_t *angle;      /* candidates (culled set) that pass the support-angle test
                            n . n_X >= cos S */
} si_probe;

typedef struct si_stats {
    int64_t calls;          /* generate calls that used this mesh */
    int64_t images;         /* images enqueued on this mesh */
    int32_t overflow;       /* 1 if some pixel of some image exceeded INT32_MAX */
    int32_t timeout;        /* 1 if a bounded device wait gave up (images incomplete) */
    int32_t bad_query;      /* 1 if a query index was outside [0, n) (that image is not computed) */
    int32_t bad_input;      /* 1 if a device input point of the mesh had a non-finite coordinate or a
                               zero normal (si_mesh_create checks host inputs itself) */
    int64_t grid_cells;     /* cells of the most recently built grid */
    int64_t kernel_launches;/* timed spin-kernel launches (see si_set_timing) */
    double kernel_ms;       /* their summed device time, CUDA events on the launch stream */
} si_stats;

/* One item of a batched call: one mesh, its own parameters and output. */
typedef struct si_batch_item {
    si_mesh_t mesh;
    const int32_t *query_idx; /* device [m], or NULL for points 0..m-1 */
    int64_t m;
    int32_t W;
    float bin_size;
    float cos_support_angle;
    int32_t *out;             /* device [m][W][W] */
} si_batch_item;

/* ---------------------------------------------------------------- meshes --
 * si_mesh_create -- copy an oriented-point set into the library (the input
 * replication of Sec. 3, "the input data is replicated").
 *   points, normals : host or device, float[n][3] (x, y, z), n >= 1.
 *   Normals are normalised in FP32.  A zero or non-finite normal or a
 *   non-finite coordinate is SI_ERR_INVALID: here, synchronously, for host
 *   inputs; for device inputs the check runs on the device and si_get_stats
 *   reports it (bad_input; the mesh's images are then unspecified).
 * Stream-ordered: nothing is read back, the call does not synchronise (the
 * bounding box and the grids derived from it stay on the device).  The mesh
 * is bound to the current device. */
si_status si_mesh_create(const float *points, const float *normals, int64_t n,
                         si_stream stream, si_mesh_t *out_mesh);

/* Waits for the mesh's pending work and frees it. */
si_status si_mesh_destroy(si_mesh_t mesh);

/* Builds (and caches) the uniform grid that si_generate would use for this
 * W, bin size and grid_div, so that a later call does no allocation (e.g.
 * before CUDA-graph capture).  `schedule` may be NULL. */
si_status si_mesh_prepare(si_mesh_t mesh, int32_t W, float bin_size,
                          const si_schedule *schedule, si_stream stream);

/* si_default_workers -- the worker count P that num_workers = 0 gives a
 * single-item call of width W with `schedule`'s group and binning on the
 * current device: SMs x spin-kernel blocks resident per SM.  All P workers
 * run at once; a larger num_workers launches blocks that start only when
 * others have finished (Sec. 4's P processing elements are the resident
 * ones).  `schedule` may be NULL (defaults).
 *   workers : host int32, written on SI_OK.
 * SI_ERR_INVALID for W outside [2, 128], a bad group, or a shape that needs
 * more shared memory than a block has; SI_ERR_CUDA if the device query fails. */
si_status si_default_workers(int32_t W, const si_schedule *schedule, int32_t *workers);

/* -------------------------------------------------------------- generate --
 * si_generate -- spin images of m query points (Algorithm 1; the image range
 * of Algorithm 2 is the chunk a worker receives).
 *   query_idx : device int32[m] indices into the mesh, or NULL for 0..m-1
 *               (the paper's "first N oriented points"); m >= 0.
 *   W         : image width, 2 <= W <= 128.
 *   bin_size  : B > 0, finite, in the units of the points.
 *   cos_support_angle : cos S in [-1, 1]; S >= pi is -1 (no angle test).
 *   out       : device int32[m][W][W].
 * A query index outside [0, n) is detected on the device: its image is not
 * computed (its contents are unspecified) and si_get_stats reports SI_ERR_INVALID (bad_query). */
si_status si_generate(si_mesh_t mesh, const int32_t *query_idx, int64_t m, int32_t W,
                      float bin_size, float cos_support_angle, si_schedule schedule,
                      int32_t *out, si_stream stream);

/* si_generate with per-image probes (see si_probe). */
si_status si_generate_probe(si_mesh_t mesh, const int32_t *query_idx, int64_t m, int32_t W,
                            float bin_size, float cos_support_angle, si_schedule schedule,
                            int32_t *out, const si_probe *probe, si_stream stream);

/* Per-claim trace of the image loop (the GPU analogue of the per-rank finishing
 * times of Sec. 2.1, Fig. 2): one entry per scheduling claim a worker made. */
typedef struct si_trace {
    int64_t *claims;            /* device [capacity][4]: worker (thread block), scheduling step,
                                   start and end of the claim's work (ns of the GPU's global
                                   timer, %globaltimer; a slow worker of the heterogeneity
                                   emulation includes its idle) */
    int64_t capacity;           /* entries `claims` holds */
    unsigned long long *count;  /* device, zeroed by the caller: claims made (entries past
                                   `capacity` are counted and dropped) */
} si_trace;

/* si_generate with the claim trace (see si_trace); images are unchanged.
 * SI_ERR_INVALID if trace is NULL or its buffers are missing. */
si_status si_generate_traced(si_mesh_t mesh, const int32_t *query_idx, int64_t m, int32_t W,
                             float bin_size, float cos_support_angle, si_schedule schedule,
                             int32_t *out, const si_trace *trace, si_stream stream);

/* si_generate_batched -- many meshes, each with its own W, B, cos S, queries
 * and output, in ONE persistent launch: the concatenation of every item's
 * chunk list is scheduled as one loop (chunks never straddle items).  With
 * override_or_null == NULL each item's rule comes from the tuning table
 * (si_tune_*), falling back to GSS.  items: host array of `count` entries. */
si_status si_generate_batched(const si_batch_item *items, int32_t count,
                              const si_schedule *override_or_null, si_stream stream);

/* si_generate_host -- the whole path from HOST buffers: copies points and
 * normals in, builds a temporary mesh, generates, delivers the images to
 * host memory and synchronises `stream` before returning.
 *   points, normals : host float[n][3];  query_idx : host int32[m] or NULL;
 *   out             : host int32[m][W][W].
 * Delivery, for m >= 32768: page-locked `out` (mapped into the device's
 * address space, as cudaHostAlloc memory is) is written by the kernel itself
 * while it runs; pageable `out` is filled by downloads of query ranges that
 * overlap the generation of the next range.  Smaller calls download once.
 * Images are the same in every case. */
si_status si_generate_host(const float *points, const float *normals, int64_t n,
                           const int32_t *query_idx, int64_t m, int32_t W, float bin_size,
                           float cos_support_angle, si_schedule schedule, int32_t *out,
                           si_stream stream);

/* si_generate_noalloc -- si_generate for callers that must not allocate
 * device memory during the call.  The paper has no counterpart: it exists for
 * callers whose device memory is fully reserved by another allocator, or
 * whose loop runs with a fixed memory footprint and may not enter an
 * allocator, which si_generate's per-call scratch (from the stream-ordered
 * pool) and its on-demand grid build would do.
 *   Arguments, output and results are those of si_generate (images bit-
 *   identical); explicit query lists are processed in the order given.
 *   Scratch: one static 2 MiB device array in the library (held by every GPU
 *   that loads it until exit), enough for 100,000 scheduling steps; a call
 *   needing more steps is SI_ERR_INVALID (raise min_chunk or group).
 *   The mesh's grid for this W, bin size and grid_div must exist already
 *   (si_mesh_prepare); otherwise SI_ERR_INVALID.
 *   Schedules: STATIC, SS, GSS or FAC with bilinear binning, no slow
 *   workers, one slice per group (slices 0 or 1) and grid order (order 0);
 *   anything else is SI_ERR_INVALID.
 *   The first call on a device (with it current) looks up the array's device
 *   address; make that first call before any stream capture.
 *   Calls share the array: two calls whose work overlaps on the GPU race. */
si_status si_generate_noalloc(si_mesh_t mesh, const int32_t *query_idx, int64_t m, int32_t W,
                              float bin_size, float cos_support_angle, si_schedule schedule,
                              int32_t *out, si_stream stream);

/* ------------------------------------------------------------ scheduling --
 * si_chunk_table -- the chunk boundaries a rule hands out for `units`
 * iterations and `workers` workers (Algorithm 3's getChunk run to the end):
 * starts[0] = 0 < starts[1] < ... < starts[nsteps] = units.  For STATIC,
 * nsteps = workers and empty blocks repeat their start.  `starts` is host
 * memory of `capacity` entries; if it is too small, *nsteps is still set and
 * SI_ERR_INVALID is returned. */
si_status si_chunk_table(int32_t kind, int64_t units, int32_t workers, int32_t min_chunk,
                         int64_t *starts, int64_t capacity, int64_t *nsteps);

/* si_chunk_table for a whole schedule (kind, min_chunk and, for
 * SI_SCHED_FAC_PROB, fac_cov); si_chunk_table(kind, ...) is this with
 * fac_cov = 0.  SI_SCHED_AWF and SI_SCHED_AF have no table (their chunks are
 * decided on the device): SI_ERR_INVALID. */
si_status si_schedule_chunks(const si_schedule *schedule, int64_t units, int32_t workers, int64_t *starts,
                             int64_t capacity, int64_t *nsteps);

/* The FP32 candidate threshold Rc2 = fl32(R^2 (1 + 1e-5)), R^2 = h^2 +
 * ((W-1)B)^2, h = W B / 2: every contributing X has |X-P|^2 < R^2, and the
 * grid examines exactly { X : fl32(|X-P|^2) <= Rc2 } after culling. */
float si_candidate_rc2(int32_t W, float bin_size);

/* si_candidate_rc2 of a binning: SI_BIN_BILINEAR as above; SI_BIN_NEAREST
 * with R^2 = ((W/2 + 1) B)^2 + ((W-1)B)^2 (a counted pair has -1 < u <= W-1,
 * i.e. |beta| < (W/2 + 1) B, and alpha <= (W-1) B). */
float si_candidate_rc2_binned(int32_t W, float bin_size, int32_t binning);

/* ----------------------------------------------------------------- stats -- */
/* Synchronises the device and reads the mesh's flags.  Returns
 * SI_ERR_OVERFLOW, SI_ERR_TIMEOUT or SI_ERR_INVALID (bad query index) when the
 * corresponding flag is set (the stats are still filled in). */
si_status si_get_stats(si_mesh_t mesh, si_stats *out);
/* Clears the mesh's overflow / timeout flags and timing counters. */
si_status si_reset_stats(si_mesh_t mesh);
/* When enabled, every spin-kernel launch is bracketed by CUDA events on its
 * stream and the device time is summed into si_stats of its mesh(es). */
void si_set_timing(int32_t enabled);

/* --------------------------------------------------------------- tuning --
 * The autotuner times candidate (rule, min_chunk, workers, group, grid_div,
 * order) settings on a mesh and records the fastest per size class (W, log2
 * of the point count, log2 of the image count).  si_generate_batched consults
 * it.  Each timed repetition runs on a freshly built grid: the tuner drops the
 * mesh's grids (after synchronizing the device) and builds them again, so the
 * mesh must not be in use on another stream or thread during the call. */
si_status si_tune_mesh(si_mesh_t mesh, const int32_t *query_idx, int64_t m, int32_t W,
                       float bin_size, float cos_support_angle, int32_t *scratch_out,
                       int32_t reps, si_schedule *best, double *best_ms, si_stream stream);
/* Look up the tuned schedule of a size class; SI_ERR_INVALID if none. */
si_status si_tune_lookup(int32_t W, int64_t n, int64_t m, si_schedule *out);
/* Save / load the tuning table as JSON text. */
si_status si_tune_save(const char *path);
si_status si_tune_load(const char *path);
si_status si_tune_clear(void);

/* --------------------------------------------------------------- serving --
 * A server keeps meshes resident and runs spin-image requests with
 * continuous batching: requests that arrive while others are on the GPU are
 * admitted as memory and in-flight slots free up, packed into the next
 * batched launch, and run on several streams so their work overlaps.
 *   mem_budget_bytes : device bytes the server may hold for admitted
 *                      requests (scratch + outputs it allocates)
 *   max_inflight     : admitted requests at most (>= 1)
 * si_serve_submit copies req (its device buffers must stay valid until the
 * request completes).  If req->out is NULL the server allocates the output
 * from its budget and si_serve_result hands it out.  A request larger than
 * the whole budget is SI_ERR_BUSY.  Submit never blocks on the GPU. */
si_status si_serve_create(size_t mem_budget_bytes, int32_t max_inflight, si_server_t *out);
si_status si_serve_add_mesh(si_server_t s, si_mesh_t mesh, int32_t *mesh_slot);
si_status si_serve_submit(si_server_t s, const si_batch_item *req, uint64_t *ticket);
si_status si_serve_poll(si_server_t s, uint64_t ticket, int32_t *done);
/* Waits for a ticket; SI_ERR_TIMEOUT after timeout_ms (< 0: forever). */
si_status si_serve_wait(si_server_t s, uint64_t ticket, int32_t timeout_ms);
/* Device output of a completed ticket (server-allocated when req->out was
 * NULL) and the submit-to-completion latency in microseconds. */
si_status si_serve_result(si_server_t s, uint64_t ticket, int32_t **out, double *latency_us);
/* Releases a completed ticket (and its server-allocated output). */
si_status si_serve_release(si_server_t s, uint64_t ticket);
si_status si_serve_destroy(si_server_t s);

/* ----------------------------------------------------------------- misc -- */
const char *si_last_error(void);
/* Library version string. */
const char *si_version(void);
/* Kernels this library has launched in this process (all devices). */
int64_t si_kernel_launches(void);
/* Measures the current device's throughput of shared-memory int32 atomic
 * adds (atomics per second, all SMs): mode 0 = every lane in its own bank
 * (the peak), mode 1 = addresses spread over small interleaved images like
 * the spin kernel's splats.  The roofline denominator of the splat step
 * (Algorithm 1's tempSpinImage[k, l]++), which no vendor figure covers.
 * Synchronises `stream`. */
si_status si_peak_smem_atomics(int32_t mode, double *atomics_per_s, si_stream stream);

/* si_alloc_stats -- the library's device-memory accounting (the paper has no
 * counterpart; it lets a caller, or a test, see whether a call allocated).
 *   calls         : device allocations the library has made in this process
 *                   (all devices); every one goes through the current
 *                   device's default memory pool (cudaMallocAsync).
 *   pool_used     : bytes of the current device's default pool in use now,
 *   pool_reserved : bytes that pool holds from the device now (both count
 *                   every user of the default pool, not only this library).
 * Each pointer may be NULL.  SI_ERR_CUDA if the pool cannot be queried. */
si_status si_alloc_stats(int64_t *calls, int64_t *pool_used, int64_t *pool_reserved);

/* si_debug_fail_allocs -- host-side failure injection (the paper has no
 * counterpart): after `skip` more device allocations succeed, the library's
 * next `count` device allocations fail as if the device were out of memory,
 * so the calls that make them return SI_ERR_OOM, free what they had taken and
 * enqueue nothing more.  count = 0 disarms it.  Process-wide (all threads and
 * devices); no GPU fault is involved.  SI_ERR_INVALID for negative values. */
si_status si_debug_fail_allocs(int64_t skip, int64_t count);

/* ------------------------------------------------------------- matching --
 * si_match -- spin-image matching: for each scene image its k best model
 * images by the linear correlation coefficient over all W x W bins
 *   R(p, q) = (N sum pq - sum p sum q) / sqrt((N sum p^2 - (sum p)^2)(N sum q^2 - (sum q)^2)),
 * N = W^2, the similarity measure of spin-image matching (Johnson and Hebert,
 * 1999, the recognition work the paper cites); an image without variance
 * correlates 0.  Over all bins R is the dot product of the centred, unit-length
 * images, so the all-pairs step is one dense contraction; it runs on the
 * tensor cores (this library's tcgen05 kernel, FP32 accumulation) with the
 * k-best selection in the kernel's epilogue, so the correlation matrix is
 * never stored:
 *   SI_MATCH_BF16 -- the centred images rounded to BF16: |R error| <= 2^-8
 *     from the operand rounding plus the accumulation error below;
 *   SI_MATCH_FP32 -- each centred value split into three BF16 terms (24
 *     significant bits) and the six products of FP32 accuracy summed in one
 *     GEMM over 6 W^2: |R error| within the accumulation error below.
 *   Accumulation: each 16-term step enters the FP32 accumulator with up to one
 *   unit in its last place, i.e. about (K / 16) 2^-23 for K = W^2 (BF16) or
 *   6 W^2 (FP32) terms at worst.
 *   scene : device int32[n_scene][W][W], model : device int32[n_model][W][W]
 *           (images as si_generate writes them);
 *   best_idx, best_corr : device [n_scene][k], highest R first, equal values
 *           by smaller model index; 1 <= k <= min(16, n_model).
 * Scratch comes from the stream-ordered pool (the centred images, 2 bytes per
 * value in BF16 and 12 in FP32 mode, plus the k-best lists of the model
 * ranges).  Stream-ordered; argument errors are synchronous.  A bounded wait
 * of the kernel that gives up (which a correct run never meets) makes every
 * best_idx of the call -2.  The paper has no counterpart (its subject is
 * generation). */
typedef enum si_match_precision { SI_MATCH_FP32 = 0, SI_MATCH_BF16 = 1 } si_match_precision;
si_status si_match(const int32_t *scene, int64_t n_scene, const int32_t *model, int64_t n_model, int32_t W,
                   int32_t k, int32_t precision, int32_t *best_idx, float *best_corr, si_stream stream);

/* Self-check of the bounded device waits (the paper has no counterpart).
 * Every mbarrier wait of the spin kernel gives up after a time limit, sets the
 * mesh's timeout flag and lets the kernel return, so that a stalled copy can
 * never hang the GPU.  This launches a tiny kernel whose blocks wait, with a
 * limit of limit_ms (1..1000), on an mbarrier that nothing arrives at; on
 * return *timed_out is 1 when the wait gave up as it must, *waited_ms (may be
 * NULL) the longest wait seen.  Synchronises `stream`; the context stays
 * usable. */
si_status si_check_bounded_wait(int32_t limit_ms, int32_t *timed_out, double *waited_ms, si_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* SPIN_GB300_H */
