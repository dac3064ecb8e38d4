/*
 * qh.h: C ABI of the GB300 segmented-Quickhull library (libqh.so).
 *
 * The library computes convex hulls of float32 point sets on one CUDA
 * device with the segmented Quickhull of Tzeng & Owens, "Finding Convex
 * Hulls Using Quickhull on the GPU": the recursion of Quickhull (Section
 * 3.2, Algorithm 1) is replaced by a permutation of one flat point array
 * into segments (Section 3.1), and each iteration of the hot loop
 * (Algorithm 4, "Recursive Step") computes every live point's distance to
 * its segment's edge, reduces each segment to its farthest point, discards
 * the points inside the triangle it forms and permutes the survivors into
 * child segments (flagPermute, Section 4.1, and compact, Section 4.2, fused
 * into one pass).
 *
 * Conventions shared by every call
 *  - Points are structure-of-arrays float32: coordinate c of point i is at
 *    d_c[i * stride].  stride = 1 for separate arrays, stride = 2 (or 3)
 *    for interleaved xy (xyz) with d_y = d_x + 1 (d_z = d_x + 2).
 *  - n is limited to 0 <= n <= QH_MAX_POINTS (int32 indices).
 *  - Device pointers are named d_*, host pointers h_*.  The caller owns
 *    every buffer, including the workspace d_ws of qh_workspace_bytes_*()
 *    bytes (device memory, 256-byte aligned).  The library allocates no
 *    device memory and keeps no state between calls except a per-device
 *    cache of the occupancy query.
 *  - Work is issued on `stream` (0 = legacy default stream).  The *_async
 *    calls do not synchronise; results land in d_result when the stream
 *    reaches that point.  The other calls synchronise the stream before
 *    returning.
 *  - Nothing throws across the ABI.  A non-QH_OK status leaves every output
 *    unspecified (no partial output is valid).
 *  - Predicates are exact: every orientation sign and every distance
 *    comparison that decides the result is exact for the float32 inputs
 *    read as real numbers (FP32 or FP64 filter with a forward error bound,
 *    exact expansion arithmetic when the filter cannot decide).
 *  - Calls that overlap on the same workspace race; distinct workspaces
 *    may run concurrently on different streams.
 */
#ifndef QH_H
#define QH_H

#include <stddef.h>
#include <stdint.h>

#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QH_MAX_POINTS ((int64_t)2147483000)

typedef enum qh_status {
    QH_OK = 0,
    QH_ERR_INVALID_ARG = 1,   /* null pointer, negative n, bad stride, n too large */
    QH_ERR_NONFINITE = 2,     /* an input coordinate is NaN or +-Inf */
    QH_ERR_DEGENERATE = 3,    /* 3D input that does not span 3D */
    QH_ERR_NOMEM = 4,         /* workspace smaller than qh_workspace_bytes_*() */
    QH_ERR_CAPACITY = 5,      /* a table overflowed: 3D facets beyond qh_opts.max_facets, or an
                                 internal bound (which should not happen) */
    QH_ERR_TIMEOUT = 6,       /* a bounded device wait gave up (grid barrier) */
    QH_ERR_NO_CONVERGENCE = 7,/* iteration cap reached */
    QH_ERR_CUDA = 8,          /* a CUDA runtime call failed */
    QH_ERR_NOT_SUPPORTED = 9  /* option combination not available */
} qh_status;

/* Predicate arithmetic of the fast filter stage. */
#define QH_PRED_F32 0 /* FP32 values, FP32 static error bound (default) */
#define QH_PRED_F64 1 /* FP64 values, FP64 error bound: the plain path */

/* How the iterations are driven. */
#define QH_LOOP_PERSISTENT 0 /* one cooperative persistent kernel, grid barriers (default) */
#define QH_LOOP_HOST 1       /* one launch per phase, live count read back each iteration */

typedef struct qh_opts {
    int32_t pred_mode;    /* QH_PRED_* */
    int32_t loop_mode;    /* QH_LOOP_* */
    int32_t blocks_per_sm;/* persistent grid: CTAs per SM (0 = as many as fit) */
    int32_t block;        /* 3D: threads per CTA, 128, 256 or 512 (0 = 256) */
    int64_t max_iters;    /* iteration cap (0 = n + 8 in 2D, 4n + 16 in 3D) */
    int64_t wait_ns;      /* bound of every grid-barrier wait (0 = 2 s); a CTA's wait for its
                             own bulk copies has a fixed 2 s bound */
    int32_t items;        /* 3D: points per thread of the assign pass, 2, 4 or 8 (0 = 4) */
    int32_t max_ctas;     /* 2D persistent grid: at most this many CTAs (0 = no cap); lets
                             several hulls share the GPU on different streams */
    int32_t test_hold;    /* tests of the bounded waits only (0 = off): 1 = CTA 0 of the
                             persistent kernel does not arrive at its first grid barrier, so
                             that round never completes, every CTA's wait runs out after
                             wait_ns and the call reports QH_ERR_TIMEOUT.  The kernel then
                             leaves without starting another phase; the workspace is
                             reusable for the next call. */
    int32_t small_cloud;  /* batched 3D: clouds of 4 to small_cloud points are hulled whole by
                             one warp each during the setup (the small-cloud route), the rest
                             by the segmented iterations; 0 = every cloud through the
                             iterations (default); at most QH_SMALL_CLOUD_MAX */
    int64_t max_facets;   /* 3D: facets the workspace holds, counting every facet created in
                             the run (deleted ones too); 0 = the worst-case bound
                             6 n + 4 ncloud + 64.  A smaller capacity shrinks the workspace
                             (about 350 B a facet, and for one cloud its segment entries,
                             about 430 B each, are capped by the facets as well); a run that
                             needs more facets stops with QH_ERR_CAPACITY and the workspace
                             stays reusable.  Values below 4 ncloud + 256 (the first
                             polytope, the clouds' tetrahedra) are raised to it, values
                             above the bound lowered to it.  qh_workspace_bytes_3d* and the
                             hull call must see the same value. */
} qh_opts;

#define QH_SMALL_CLOUD_MAX 4096

/* Result record written by the device (async calls) and copied back by the
 * synchronous calls.  All counts are totals over the call. */
typedef struct qh_result {
    int64_t count;            /* 2D: hull vertices written to d_out_idx */
    int32_t status;           /* qh_status */
    int32_t reserved0;
    int64_t iterations;       /* Quickhull iterations (passes after the first split) */
    int64_t live_total;       /* sum over passes of live points read (incl. first split) */
    int64_t survivor_total;   /* sum over passes of points written */
    int64_t segments_total;   /* sum over iterations of segments */
    int64_t filter_fallbacks; /* predicate evaluations the fast filter could not decide */
    int64_t exact_argmax;     /* segments whose farthest point needed exact resolution */
    int64_t extra[4];         /* 2D persistent loop: nanoseconds spent in the pass,
                                 update, exact-argmax and other phases (device
                                 clock between grid barriers); 3D: [0] vertices,
                                 [1] faces, [2] face index total */
} qh_result;

/* Human-readable name of a status code (static storage). */
const char *qh_status_str(qh_status s);

/* Library version string, e.g. "qh 0.1 sm_103a". */
const char *qh_version(void);

/* Default options (persistent loop, FP32 filter). */
void qh_default_opts(qh_opts *opts);

/* ---------------------------------------------------------------------- */
/* 2D                                                                      */
/* ---------------------------------------------------------------------- */

/* Bytes of device workspace qh_hull2d* needs for n points. */
size_t qh_workspace_bytes_2d(int64_t n, const qh_opts *opts);

/*
 * qh_hull2d_async: convex hull of n float32 points in the plane (Algorithm
 * 4, 2DCUDAQuickhull: first split by the extrema along x, then repeated
 * farthest-point / triangle-discard / flagPermute iterations until no
 * segment has points; Section 4.3 states the problem as p_in -> ch_out).
 *
 *  d_x, d_y   device, n points, coordinate i at d_x[i*stride] (read only)
 *  d_out_idx  device int32[max(n,1)]: hull vertex indices in counter-
 *             clockwise order starting at the lexicographically smallest
 *             (x, y) vertex; a location present several times is reported
 *             as its lowest index; vertices in the middle of a straight
 *             boundary run are not vertices.  n = 1 or all points equal ->
 *             one index; all points collinear -> the two extreme points.
 *  d_result   device qh_result (count, status, statistics)
 *  d_ws       device workspace of qh_workspace_bytes_2d(n, opts) bytes
 *  opts       may be NULL (defaults)
 * Host-side argument errors are returned directly; data-dependent errors
 * (QH_ERR_NONFINITE, QH_ERR_TIMEOUT, ...) appear in d_result->status.
 * QH_LOOP_PERSISTENT (the default) runs the persistent kernel of
 * qh_hull2d_multi_async with this one cloud (n <= QH_MAX_POINTS - 2);
 * QH_LOOP_HOST synchronises the stream once per iteration.
 */
qh_status qh_hull2d_async(const float *d_x, const float *d_y, int64_t n, int64_t stride,
                          int32_t *d_out_idx, qh_result *d_result, void *d_ws, size_t ws_bytes,
                          const qh_opts *opts, cudaStream_t stream);

/* Synchronous form of qh_hull2d_async: returns the device status, the hull
 * size in *h_count and, when h_result is not NULL, the full result record.
 * d_result is taken from the workspace.  With QH_LOOP_HOST, hulls with more
 * than 4096 hull slots (the apexes found over all iterations, including
 * points later found collinear) are finished here by a second, single-block
 * output step; qh_hull2d_async reports QH_ERR_CAPACITY for them there (the
 * persistent loop returns them directly). */
qh_status qh_hull2d(const float *d_x, const float *d_y, int64_t n, int64_t stride,
                    int32_t *d_out_idx, int64_t *h_count, qh_result *h_result, void *d_ws,
                    size_t ws_bytes, const qh_opts *opts, cudaStream_t stream);

/*
 * Several 2D clouds in one persistent launch (no paper counterpart: the
 * clouds' live points share the segment table, so every iteration's pass,
 * update and grid barriers serve all of them, and each pass's tiles spread
 * the clouds' work over the whole GPU).  Each cloud's hull is the one
 * qh_hull2d_async returns for it alone.
 *
 *  k                1 <= k <= QH_MAX_CLOUDS_2D clouds
 *  h_dx[c], h_dy[c] host arrays of device pointers: cloud c's coordinates,
 *                   point i at d_x[i*stride] (read only)
 *  h_n[c]           points of cloud c (>= 0); the total is at most
 *                   QH_MAX_POINTS - 2 * k
 *  h_stride[c]      >= 1 (NULL: all 1)
 *  h_dout[c]        host array of device pointers: int32[max(n_c, 1)] hull
 *                   indices of cloud c, counter-clockwise from its
 *                   lexicographically smallest vertex (cloud-local indices)
 *  d_results        device qh_result[k]: per cloud count and status
 *                   (QH_ERR_NONFINITE for a cloud with NaN/Inf; a failure of
 *                   the shared iterations is reported in every record)
 *  d_ws             device workspace of qh_workspace_bytes_2d_multi bytes,
 *                   256-byte aligned
 * Only QH_LOOP_PERSISTENT.  qh_hull2d_multi synchronises, fills h_counts[k]
 * and h_results[k] (either may be NULL) and returns the first non-OK status
 * of the clouds. */
#define QH_MAX_CLOUDS_2D 8
size_t qh_workspace_bytes_2d_multi(int32_t k, const int64_t *h_n, const qh_opts *opts);
qh_status qh_hull2d_multi_async(int32_t k, const float *const *h_dx, const float *const *h_dy,
                                const int64_t *h_n, const int64_t *h_stride,
                                int32_t *const *h_dout, qh_result *d_results, void *d_ws,
                                size_t ws_bytes, const qh_opts *opts, cudaStream_t stream);
qh_status qh_hull2d_multi(int32_t k, const float *const *h_dx, const float *const *h_dy,
                          const int64_t *h_n, const int64_t *h_stride, int32_t *const *h_dout,
                          int64_t *h_counts, qh_result *h_results, void *d_ws, size_t ws_bytes,
                          const qh_opts *opts, cudaStream_t stream);

/* ---------------------------------------------------------------------- */
/* 3D                                                                      */
/* ---------------------------------------------------------------------- */

/* Bytes of device workspace qh_hull3d needs for n points
 * (n <= QH_MAX_POINTS_3D) and opts->max_facets (null opts: the worst case). */
#define QH_MAX_POINTS_3D ((int64_t)44000000)
size_t qh_workspace_bytes_3d(int64_t n, const qh_opts *opts);

/*
 * qh_hull3d: convex hull of n float32 points in space (Section 4.3, "3D and
 * Higher Dimensions": first split by a plane through the extrema, then
 * farthest-point insertion; read as Barber et al.'s Quickhull with several
 * non-conflicting apexes inserted per iteration).
 *
 *  d_x, d_y, d_z  device, coordinate i at d_c[i*stride] (read only)
 *  d_verts        device int32[max(n,1)]: the hull vertices, increasing index
 *  h_nv           host: number of vertices
 *  d_face_off     device int32[2n+1]: CSR offsets of the faces
 *  d_face_idx     device int32[6n]: face vertex indices; each face is a
 *                 maximal coplanar polygon, counter-clockwise seen from
 *                 outside, starting at its smallest index; faces are sorted
 *                 lexicographically
 *  h_nf           host: number of faces
 *  h_result       optional host qh_result (extra[0..2] = vertices, faces,
 *                 face index total)
 * Points that do not span 3D (n < 4, collinear, coplanar) give
 * QH_ERR_DEGENERATE; n = 0 gives QH_OK with no faces.  Only the persistent
 * loop is available (QH_LOOP_HOST returns QH_ERR_NOT_SUPPORTED).
 * Synchronises `stream`.
 */
qh_status qh_hull3d(const float *d_x, const float *d_y, const float *d_z, int64_t n,
                    int64_t stride, int32_t *d_verts, int64_t *h_nv, int32_t *d_face_off,
                    int32_t *d_face_idx, int64_t *h_nf, qh_result *h_result, void *d_ws,
                    size_t ws_bytes, const qh_opts *opts, cudaStream_t stream);

/*
 * Batched 3D hulls (no counterpart in the paper, whose input is one point
 * set; its segments are what makes a batch cheap: every cloud's root
 * segment simply joins the segment table of one persistent launch).
 *
 * The clouds are CSR: cloud c holds points [cloud_off[c], cloud_off[c+1])
 * of the shared coordinate arrays, cloud_off[0] = 0, cloud_off[ncloud] = n,
 * non-decreasing (empty clouds allowed).  1 <= ncloud and
 * n + ncloud <= QH_MAX_POINTS_3D.
 */
size_t qh_workspace_bytes_3d_batched(int64_t n, int32_t ncloud, const qh_opts *opts);

/*
 * qh_hull3d_batched: the hull of every cloud, in one call that never
 * synchronises the stream and allocates nothing, so it can be captured in a
 * CUDA graph (run it once before the capture: the first call on a device
 * queries the kernel occupancy).
 *
 *  d_cloud_off       device int64[ncloud+1] (checked on the device: bad
 *                    offsets give QH_ERR_INVALID_ARG in d_result->status)
 *  d_verts           device int32[n]: the vertices of all clouds, as global
 *                    point indices in increasing order (so grouped by cloud)
 *  d_cloud_vert_off  device int32[ncloud+1]: cloud c's vertices are
 *                    d_verts[d_cloud_vert_off[c] .. d_cloud_vert_off[c+1])
 *  d_face_off        device int32[2n+1], d_face_idx device int32[6n]: the
 *                    faces of all clouds as in qh_hull3d (global indices,
 *                    sorted, hence grouped by cloud)
 *  d_cloud_face_off  device int32[ncloud+1]: cloud c's faces are faces
 *                    d_cloud_face_off[c] .. d_cloud_face_off[c+1]
 *  d_cloud_status    device int32[ncloud]: QH_OK, QH_ERR_DEGENERATE (fewer
 *                    than 4 points or not spanning 3D: no faces) or
 *                    QH_ERR_NONFINITE (no faces) per cloud; an empty cloud
 *                    is QH_OK with no faces
 *  d_result          device qh_result: status of the whole call, vertex and
 *                    face totals (extra[0..2]) and statistics
 * opts->block and opts->items choose the launch shape (see
 * qh_autotune_3d_batched).  Returns QH_OK once the work is enqueued;
 * argument errors are returned at once.
 */
qh_status qh_hull3d_batched(const float *d_x, const float *d_y, const float *d_z, int64_t stride,
                            const int64_t *d_cloud_off, int32_t ncloud, int64_t n,
                            int32_t *d_verts, int32_t *d_cloud_vert_off, int32_t *d_face_off,
                            int32_t *d_face_idx, int32_t *d_cloud_face_off,
                            int32_t *d_cloud_status, qh_result *d_result, void *d_ws,
                            size_t ws_bytes, const qh_opts *opts, cudaStream_t stream);

/*
 * qh_autotune_3d_batched: times qh_hull3d_batched on the caller's batch for
 * every launch shape (threads per CTA 128/256/512 x points per thread
 * 2/4/8 x CTAs per SM 1/2/4, capped by occupancy), then, at the fastest
 * shape, for the small-cloud thresholds 0, 64, 256, 1024 and 4096
 * (qh_opts.small_cloud: the switchover below which one warp hulls a cloud
 * whole; no counterpart in the paper, which leaves switchover points to
 * future work in Section 6): one untimed run, then `reps` (1..64) runs timed
 * with CUDA events on `stream`; the median decides.
 *  h_best    in: base options (predicate mode); out: the fastest candidate
 *  h_ms      host float[max_cand]: median ms of each candidate that ran
 *  h_shape   host int32[4*max_cand]: (block, items, CTAs per SM,
 *            small-cloud threshold) of each
 *  h_ncand   host: candidates reported
 * Synchronises the stream; the outputs hold the hulls of the last run.
 */
qh_status qh_autotune_3d_batched(const float *d_x, const float *d_y, const float *d_z,
                                 int64_t stride, const int64_t *d_cloud_off, int32_t ncloud,
                                 int64_t n, int32_t *d_verts, int32_t *d_cloud_vert_off,
                                 int32_t *d_face_off, int32_t *d_face_idx,
                                 int32_t *d_cloud_face_off, int32_t *d_cloud_status,
                                 qh_result *d_result, void *d_ws, size_t ws_bytes, int32_t reps,
                                 qh_opts *h_best, float *h_ms, int32_t *h_shape, int32_t max_cand,
                                 int32_t *h_ncand, cudaStream_t stream);

/*
 * Batched 2D hulls (no counterpart in the paper): one CTA runs the whole
 * segmented Quickhull of one cloud, clouds taken from a queue by a
 * persistent grid.  Meant for many small or medium clouds (up to about 10^5
 * points each); large single clouds belong to qh_hull2d.  Clouds are CSR as
 * in qh_hull3d_batched (1 <= ncloud, n >= 1).
 *
 *  d_out_idx       device int32[n]: the hull of cloud c (counter-clockwise
 *                  from its lexicographically smallest point, collinear
 *                  points dropped, global indices) at
 *                  d_out_idx[cloud_off[c] .. cloud_off[c] + d_cloud_count[c])
 *  d_cloud_count   device int32[ncloud]: hull size per cloud (0 when empty
 *                  or non-finite, 1 when all points coincide)
 *  d_cloud_status  device int32[ncloud]: QH_OK or QH_ERR_NONFINITE
 *  d_result        device qh_result: whole-call status (QH_ERR_INVALID_ARG
 *                  for bad offsets), count = total hull vertices, iterations
 *                  = the largest per-cloud iteration count
 * Never synchronises; allocates nothing (capturable in a CUDA graph after
 * one call on the device).
 */
size_t qh_workspace_bytes_2d_batched(int64_t n, int32_t ncloud, const qh_opts *opts);
qh_status qh_hull2d_batched(const float *d_x, const float *d_y, int64_t stride,
                            const int64_t *d_cloud_off, int32_t ncloud, int64_t n,
                            int32_t *d_out_idx, int32_t *d_cloud_count, int32_t *d_cloud_status,
                            qh_result *d_result, void *d_ws, size_t ws_bytes, const qh_opts *opts,
                            cudaStream_t stream);

/*
 * Differentiable measures (no counterpart in the paper, which computes the
 * hull only).  On general-position inputs the hull's vertex set and faces
 * are locally constant, so each measure is a smooth function of the hull
 * vertices and its gradient is zero on every other point.  Sums are FP64.
 *
 * qh_measures2d: d_meas[2c] = perimeter, d_meas[2c+1] = area of cloud c's
 *   hull as written by qh_hull2d_batched (d_hull, d_cloud_count; a single
 *   qh_hull2d result is one cloud with offsets {0, n}).
 * qh_hull2d_backward: with d_grad[2c], d_grad[2c+1] = dL/dperimeter and
 *   dL/darea of cloud c, writes dL/dx, dL/dy of every point (float32, zero
 *   off the hull) to d_gx[i*gstride], d_gy[i*gstride].
 * qh_measures3d: d_meas[2c] = surface area, d_meas[2c+1] = volume of cloud
 *   c's hull (faces d_cloud_face_off[c] .. d_cloud_face_off[c+1] of the CSR
 *   face list of qh_hull3d / qh_hull3d_batched; faces are triangulated as
 *   fans from their first vertex).
 * qh_hull3d_backward: same for dL/darea, dL/dvolume; d_scratch is device
 *   FP64 scratch of 3n values (the per-point sums before rounding).
 * All four are asynchronous on `stream`.
 */
qh_status qh_measures2d(const float *d_x, const float *d_y, int64_t stride,
                        const int64_t *d_cloud_off, int32_t ncloud, const int32_t *d_hull,
                        const int32_t *d_cloud_count, double *d_meas, cudaStream_t stream);
qh_status qh_hull2d_backward(const float *d_x, const float *d_y, int64_t stride,
                             const int64_t *d_cloud_off, int32_t ncloud, int64_t n,
                             const int32_t *d_hull, const int32_t *d_cloud_count,
                             const double *d_grad, float *d_gx, float *d_gy, int64_t gstride,
                             cudaStream_t stream);
qh_status qh_measures3d(const float *d_x, const float *d_y, const float *d_z, int64_t stride,
                        int32_t ncloud, const int32_t *d_face_off, const int32_t *d_face_idx,
                        const int32_t *d_cloud_face_off, double *d_meas, cudaStream_t stream);
qh_status qh_hull3d_backward(const float *d_x, const float *d_y, const float *d_z, int64_t stride,
                             int32_t ncloud, int64_t n, const int32_t *d_face_off,
                             const int32_t *d_face_idx, const int32_t *d_cloud_face_off,
                             const double *d_grad, float *d_gx, float *d_gy, float *d_gz,
                             int64_t gstride, double *d_scratch, cudaStream_t stream);

/* ---------------------------------------------------------------------- */
/* 4D                                                                      */
/* ---------------------------------------------------------------------- */

/* Bytes of device workspace qh_hull4d needs for n points (0 when n is out
 * of range: 0 <= n <= 8,000,000). */
size_t qh_workspace_bytes_4d(int64_t n, const qh_opts *opts);

/*
 * qh_hull4d: convex hull of n float32 points in R^4 (Section 4.3, "3D and
 * Higher Dimensions": the recursion with a k-state flagPermute in higher
 * dimensions; read as Barber et al.'s Quickhull in R^4, several
 * non-conflicting apexes inserted per iteration, horizon ridges are
 * triangles).  The iterations are driven from the host (one launch per
 * phase; the header is read back once per batch of up to 4 iterations).
 *
 *  d_x .. d_w     device, coordinate i at d_c[i*stride] (read only)
 *  d_verts        device int32[max(n,1)]: the extreme points, increasing index
 *                 (a location present several times: its lowest index)
 *  h_nv           host: number of vertices
 *  d_facet_off    device int32[max_facets + 1]: CSR offsets of the facets
 *  d_facet_idx    device int32[max_idx]: for every facet (a maximal set of
 *                 boundary points on one supporting hyperplane), the sorted
 *                 extreme points on it; facets in lexicographic order of
 *                 these lists (compared on their first eight entries; lists
 *                 equal there appear in an unspecified order)
 *  h_nf           host: number of facets (also set when the capacities are
 *                 too small: then QH_ERR_CAPACITY, *h_nf and h_result->extra[2]
 *                 give the sizes needed)
 *  h_result       optional host qh_result (extra[0..2] = vertices, facets,
 *                 facet index total)
 * Points that do not span R^4 (n < 5 included) give QH_ERR_DEGENERATE;
 * n = 0 gives QH_OK with no facets; a non-finite coordinate gives
 * QH_ERR_NONFINITE.  The workspace holds up to 32 n + 1024 facets created
 * over the run (QH_ERR_CAPACITY beyond; inputs whose hull grows faster than
 * that are not supported).  Synchronises `stream`.
 */
qh_status qh_hull4d(const float *d_x, const float *d_y, const float *d_z, const float *d_w,
                    int64_t n, int64_t stride, int32_t *d_verts, int64_t *h_nv,
                    int32_t *d_facet_off, int64_t max_facets, int32_t *d_facet_idx,
                    int64_t max_idx, int64_t *h_nf, qh_result *h_result, void *d_ws,
                    size_t ws_bytes, const qh_opts *opts, cudaStream_t stream);

/*
 * qh_hull2d_noalloc: qh_hull2d for callers that cannot allocate device
 * memory while they run: plugins whose host owns every device allocation,
 * real-time loops that allocate only at start-up, and code that may not let
 * cudaMalloc/cudaFree synchronise the device.  (The paper has no
 * counterpart; this is an interface convenience.)
 *
 * Same inputs, output and result order as qh_hull2d, but no workspace
 * argument: the scratch is one fixed array of 32 MiB in device memory that
 * every device holds once the library is loaded on it, until the process
 * exits.  n may not exceed QH_NOALLOC_MAX_POINTS; larger n returns
 * QH_ERR_INVALID_ARG without touching the device.  Set-up happens on the
 * first call made on a device, with that device current: it looks up the
 * array's device address (cudaGetSymbolAddress) and keeps it for the
 * device.  That lookup is also what loads the library's module on the
 * device (CUDA loads modules lazily) and so reserves the 32 MiB; a device
 * without room for it gives QH_ERR_NOMEM.  Make that first call at start-up
 * and before any stream capture.  The kept address belongs to the device's
 * current context: after cudaDeviceReset (or any teardown of the primary
 * context) this entry point may not be called again in the process.  Every
 * call on a device shares the array and finds it as the last call left it
 * (the hull clears what it needs): calls that overlap on the GPU (other
 * streams, other host threads) race and must be serialised by the caller.
 * Nothing here calls cudaMalloc, cudaFree or an allocating library routine.
 * Synchronises `stream`.
 */
#define QH_NOALLOC_MAX_POINTS ((int64_t)131072)
qh_status qh_hull2d_noalloc(const float *d_x, const float *d_y, int64_t n, int64_t stride,
                            int32_t *d_out_idx, int64_t *h_count, cudaStream_t stream);

/* ---------------------------------------------------------------------- */
/* Diagnostics                                                             */
/* ---------------------------------------------------------------------- */

/* Per-iteration record of the last persistent-loop 2D call made on d_ws
 * (which must be the workspace of a call with the same n, finished or not
 * yet started on `stream`; the call synchronises the stream).  Row r holds
 * {r, L_r, S_r, pass_ns, update_ns}: r = 0 is the first split, L_r the live
 * points the pass of iteration r read, S_r its segments, then the device
 * time of that pass and of the update that followed.  At most 64 rows and
 * max_rows rows are written (h_rows: host int64[5 * max_rows]); *h_nrows
 * receives the count.  Timing comes from %globaltimer between grid
 * barriers. */
qh_status qh_debug_timeline_2d(const void *d_ws, int64_t n, int64_t *h_rows, int32_t max_rows,
                               int32_t *h_nrows, cudaStream_t stream);

/* Per-iteration record of the last qh_hull3d call made on d_ws (same n; the
 * call synchronises the stream).  Row r (h_rows: int64[10 * max_rows]) holds
 * {iteration, live points, segments, apexes inserted, then the device time in
 * ns of: visible-set search, selection rounds and cones, point assignment,
 * segment table, scatter and certification, exact farthest points}.  At most
 * 64 rows. */
qh_status qh_debug_timeline_3d(const void *d_ws, int64_t n, int64_t *h_rows, int32_t max_rows,
                               int32_t *h_nrows, cudaStream_t stream);

/* Record of the last qh_hull4d call made by the calling host thread, one
 * row per read of its header (the host loop reads it once per batch of up
 * to 4 iterations): row r (h_rows: int64[9 * max_rows]) holds {iterations
 * enqueued so far, segments, live points, apexes inserted in the last
 * iteration, apexes that needed the exact farthest-point step, host ns
 * since the previous row, then the candidates that claimed in selection
 * rounds 0, 1 and 2 of the last iteration}; at most 4096 rows.
 * Diagnostics only. */
qh_status qh_debug_timeline_4d(int64_t *h_rows, int32_t max_rows, int32_t *h_nrows);

/*
 * The paper's segmented primitives and a second workload built on them.
 * Arrays are int32 on the device; a segmented array of n elements carries
 * head flags s[i] != 0 at the first element of every segment (element 0
 * always starts a segment).  d_ws: qh_segmented_workspace_bytes(n, nseg)
 * bytes (nseg only matters for qh_select).  All three calls synchronise.
 *
 * qh_flag_permute (Section 4.1, Algorithm 2): states d_f[i] in [0, k),
 *   1 <= k <= 7.  d_p[i] = destination of element i when every segment is
 *   regrouped by state (stably); d_s_new[0..n) = head flags of the result
 *   (old heads plus one at every non-empty state group).  States outside
 *   [0, k) give QH_ERR_INVALID_ARG.
 * qh_compact (Section 4.2, Algorithm 3): flags d_b[i] in {0, 1}.  d_p[i] =
 *   number of true flags before i (the destination of the kept elements);
 *   *h_n_new = kept elements; d_s_new[0..n_new) = head flags of the kept
 *   array (a segment with nothing kept disappears); d_s_new has n entries.
 * qh_select (Section 6, k-th element selection: a 3-state flagPermute
 *   around each segment's pivot, then a compact that keeps the part holding
 *   the wanted rank): segments are CSR (d_seg_off[nseg+1], int64, every
 *   segment non-empty), d_k[c] (int64) the wanted rank in segment c
 *   (0 <= k < length).  d_out_idx[c] = index of the element of rank d_k[c]
 *   in the order (value, index), values ordered by their bit patterns like
 *   numbers (-0 before +0; NaNs at the ends).  *h_iters = rounds used.
 *   One persistent cooperative launch runs every round: segments longer
 *   than 4096 elements go through grid-wide rounds (counts around each
 *   segment's middle pivot, decisions, ordered scatter of the kept parts,
 *   separated by bounded grid barriers); a segment of at most 4096 elements
 *   is finished by one CTA in shared memory with the same rounds.  Nothing is
 *   read back between rounds.  QH_ERR_TIMEOUT if a grid barrier wait gives
 *   up, QH_ERR_NO_CONVERGENCE past 4n + 16 global rounds.
 * qh_select_host_loop: the same selection with one host iteration per round
 *   (the primitives' kernels, then the kept count read back), the
 *   round-by-round form; same arguments, results and round counts.
 */
size_t qh_segmented_workspace_bytes(int64_t n, int32_t nseg);
qh_status qh_flag_permute(const int32_t *d_f, const int32_t *d_s, int64_t n, int32_t k,
                          int32_t *d_p, int32_t *d_s_new, void *d_ws, size_t ws_bytes,
                          cudaStream_t stream);
qh_status qh_compact(const int32_t *d_b, const int32_t *d_s, int64_t n, int32_t *d_p,
                     int32_t *d_s_new, int64_t *h_n_new, void *d_ws, size_t ws_bytes,
                     cudaStream_t stream);
qh_status qh_select(const float *d_v, const int64_t *d_seg_off, int32_t nseg, int64_t n,
                    const int64_t *d_k, int32_t *d_out_idx, int64_t *h_iters, void *d_ws,
                    size_t ws_bytes, cudaStream_t stream);
qh_status qh_select_host_loop(const float *d_v, const int64_t *d_seg_off, int32_t nseg,
                              int64_t n, const int64_t *d_k, int32_t *d_out_idx,
                              int64_t *h_iters, void *d_ws, size_t ws_bytes,
                              cudaStream_t stream);

/* Device time of the last 3D call made on d_ws (qh_hull3d or
 * qh_hull3d_batched): h_ns[0..3] = initial simplex, first assignment, its
 * table, its scatter + certification + exact apexes; h_ns[4] = the whole
 * persistent kernel (ns, device clock).  Synchronises `stream`.
 * Diagnostics only. */
qh_status qh_debug_phases_3d(const void *d_ws, int64_t *h_ns, cudaStream_t stream);

/* ------------------------------------------------------------------------
 * One hull over several ranks (no counterpart in the paper, which runs one
 * GPU): the hull of a union is the hull of the union of the parts' hulls, so
 * every rank hulls a contiguous shard of each cloud, the shard hulls are
 * all-gathered (by the caller, e.g. NCCL), and one final hull of the
 * gathered candidates gives the answer.  These three calls are the device
 * steps around the exchange; none synchronises.
 *
 * qh_shard_block_words(dim, cap): int32 words of one cloud's rank block:
 *   1 + (1 + dim) * cap (0 for bad arguments).
 * qh_shard_local: the rank block for the all-gather.  h_dout[c] (device
 *   int32) holds the shard hull of cloud c with shard-local indices, its
 *   count and status in d_results[c] (device qh_result[k], as
 *   qh_hull2d_multi_async writes them); h_lo[c] is the shard's first global
 *   index; h_dcoord[c * dim + d] (device) the shard's coordinate d, point i
 *   at [i * stride] (may be null for an empty shard; a shard with points
 *   and a null coordinate array is reported as QH_ERR_INVALID_ARG through
 *   its count word).  Cloud c's block at d_block + c * words: word 0 =
 *   count, words 1 + j = h_lo[c] + local index j, words 1 + (1 + d) * cap + j
 *   = coordinate d of that point (float bits), for j < min(count, cap); a
 *   failed shard's count word is minus its status.
 * qh_shard_pack: d_gathered = the world rank blocks in rank order
 *   ([world][k][words]).  For every cloud c, the candidate cloud of
 *   m = world * cap slots: slot r * cap + j = rank r's j-th candidate, or the
 *   cloud's first candidate where rank r has fewer (a repeated point).
 *   d_cidx[c * m + s] = global index of slot s (-1 if no rank has any),
 *   d_ccoord[(d * k + c) * m + s] = its coordinate d.  dim 2 or 3.
 *   d_bad[c] (device int32[k], cleared by the caller) receives the status of
 *   a rank whose shard of cloud c failed, or QH_ERR_CAPACITY if a rank's
 *   count exceeds cap.
 * qh_shard_remap: after the final hull of the candidate clouds, h_dout[c]
 *   (device int32, its count in d_results[c]) holds candidate-local indices;
 *   each becomes d_cidx[c * m + local], the global index.
 * Candidate order makes the result equal the one-rank hull: ranks in rank
 * order hold increasing global indices, each shard hull already keeps the
 * lowest index of coincident points, and the final hull keeps the lowest
 * candidate slot, so coincident points keep their lowest global index.
 * 1 <= k <= 64; QH_ERR_INVALID_ARG for null pointers or bad sizes. */
int64_t qh_shard_block_words(int32_t dim, int32_t cap);
qh_status qh_shard_local(int32_t k, int32_t dim, const int32_t *const *h_dout,
                         const void *d_results, const int64_t *h_lo,
                         const float *const *h_dcoord, int64_t stride, int32_t cap,
                         int32_t *d_block, cudaStream_t stream);
qh_status qh_shard_pack(int32_t k, int32_t dim, const int32_t *d_gathered, int32_t world,
                        int32_t cap, float *d_ccoord, int32_t *d_cidx, int32_t *d_bad,
                        cudaStream_t stream);
qh_status qh_shard_remap(int32_t k, int32_t *const *h_dout, const void *d_results,
                         const int32_t *d_cidx, int64_t m, cudaStream_t stream);

/* ------------------------------------------------------------------------
 * Device-side checks (no counterpart in the paper: a debugging aid).
 *
 * A library built with -DQH_DEBUG=1 checks, on the device and before the
 * access: every bulk copy (16-byte aligned source and destination, a size
 * that is a positive multiple of 16, QH_DBG_BULK_ALIGN), every mbarrier's
 * 8-byte alignment (QH_DBG_MBAR_ALIGN), the range of the 2D bulk copies'
 * sources (QH_DBG_BULK_RANGE), the destination of every 2D and 3D point
 * scatter (QH_DBG_POINT_DST), the 2D tile map's segment indices
 * (QH_DBG_SEG_INDEX), the 2D hull slots written by the updates
 * (QH_DBG_HULL_SLOT) and the alignment of the 2D extrema's vector loads
 * (QH_DBG_VEC_ALIGN).  A failed check skips the access (the call's result is
 * then unspecified, and a skipped bulk copy ends in the bounded copy wait's
 * QH_ERR_TIMEOUT) and is counted; nothing traps.  The default build compiles
 * the checks out.
 *
 * qh_debug_checks() copies the record (failed checks since the last reset,
 * summed over the library's translation units, and the site and two values
 * of the first failure found) to *h_out and, when reset != 0, clears it.  It
 * synchronises the device.  Returns QH_ERR_NOT_SUPPORTED (with
 * h_out->enabled = 0) in a default build, QH_ERR_INVALID_ARG for a null
 * h_out, QH_ERR_CUDA if a copy fails. */
#define QH_DBG_BULK_ALIGN 1
#define QH_DBG_MBAR_ALIGN 2
#define QH_DBG_BULK_RANGE 3
#define QH_DBG_POINT_DST 4
#define QH_DBG_SEG_INDEX 5
#define QH_DBG_HULL_SLOT 6
#define QH_DBG_VEC_ALIGN 7
typedef struct qh_debug_record {
    int64_t failures;  /* failed checks since the last reset */
    int32_t site;      /* QH_DBG_* of the first failure (0: none) */
    int32_t enabled;   /* 1 in a -DQH_DEBUG=1 build */
    uint64_t a, b;     /* the first failure's values: address or index, and bound or size */
} qh_debug_record;
qh_status qh_debug_checks(qh_debug_record *h_out, int32_t reset);

#ifdef __cplusplus
}
#endif

#endif /* QH_H */
