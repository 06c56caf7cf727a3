/*
 * sbr.h -- C ABI of the GB300 shooting-and-bouncing-ray (SBR) library.
 *
 * The library implements the hot path of Zhou et al., "An Improved Equiangular Division
 * Algorithm for SBR based Ray Tracing Channel Modeling" (arXiv 2208.10009):
 *   equiangular ray launching (§II.B, Eq. 1-2), tracing with specular reflection and the
 *   reception judgment (§III.A, Fig. 4, Eq. 3), double-count removal (§III.A), the
 *   iterative precise algorithm (§III.B, Fig. 5, Eq. 10), the validity test (§III.A) and
 *   the channel outputs delay / AOD / AOA / power (§IV), plus a batched persistent
 *   refinement and the adjoint of the fixed-face-sequence unfolding.
 *
 * Conventions (every entry point):
 *   - Returns sbr_status; SBR_OK == 0.  On error, sbr_last_error(ctx) holds a message.
 *     No C++ exception crosses this boundary.
 *   - All GPU work is enqueued on the context's stream (sbr_ctx_create /
 *     sbr_ctx_set_stream) and is asynchronous unless the entry point says it
 *     synchronises.
 *   - Host input arrays are copied before the call returns; the caller keeps ownership.
 *     Pointers documented "host or device" are classified with cudaPointerGetAttributes.
 *   - Device memory owned by handles is obtained through the context's allocator
 *     callbacks (or cudaMallocAsync when none are given) and released by the matching
 *     destroy call.
 *   - Coordinates are metres in a right-handed frame; angles are radians; azimuth =
 *     atan2(y, x) in (-pi, pi], elevation = atan2(z, hypot(x, y)).
 *   - A "face" is a planar polygon given as triangles sharing a face id; path face
 *     sequences name faces.  At most SBR_MAX_ORDER reflections per path.
 */
#ifndef SBR_H_
#define SBR_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SBR_ABI_VERSION 3
#define SBR_MAX_ORDER 8

typedef enum {
    SBR_OK = 0,
    SBR_EINVAL = 1,      /* bad argument (null handle, size out of range, unknown K...) */
    SBR_ENOMEM = 2,      /* device or host allocation failed */
    SBR_ECUDA = 3,       /* a CUDA runtime call failed (message has the CUDA error) */
    SBR_ETIMEOUT = 4,    /* a bounded device-side wait gave up (persistent queue) */
    SBR_EOVERFLOW = 5,   /* a record or path buffer was too small; counts say how large */
    SBR_EDEGENERATE = 6, /* scene has NaN/Inf vertices, zero-area triangles or bad ids */
    SBR_ECOLLISION = 7,  /* two different face sequences shared a 64-bit dedup hash */
    SBR_ECHECK = 8       /* SBR_CHECKED builds: a device bounds check failed (see check_flags) */
} sbr_status;

typedef struct sbr_ctx sbr_ctx;
typedef struct sbr_scene sbr_scene;
typedef struct sbr_rxset sbr_rxset;
typedef struct sbr_paths sbr_paths;

/* Allocator callbacks: return a device pointer of at least `bytes` bytes usable on
 * `stream` (NULL on failure); free releases it.  `user` is passed through. */
typedef void *(*sbr_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*sbr_free_fn)(void *ptr, size_t bytes, void *stream, void *user);

/* ---------------------------------------------------------------- context */
/* Create a context on CUDA device `device` that enqueues work on `stream` (a
 * cudaStream_t; NULL = the legacy default stream).  alloc/free may both be NULL
 * (cudaMallocAsync / cudaFreeAsync on the stream are used then). */
sbr_status sbr_ctx_create(int device, void *stream, sbr_alloc_fn alloc, sbr_free_fn free_fn, void *user,
                          sbr_ctx **out);
sbr_status sbr_ctx_destroy(sbr_ctx *ctx);
sbr_status sbr_ctx_set_stream(sbr_ctx *ctx, void *stream);
/* Message of the last failed call on this context ("" if none).  Valid until the next call. */
const char *sbr_last_error(const sbr_ctx *ctx);
const char *sbr_status_string(sbr_status s);
int32_t sbr_abi_version(void);
/* Number of SMs of the context's device (for grid sizing by callers). */
int32_t sbr_ctx_num_sms(const sbr_ctx *ctx);

/* ---------------------------------------------------------------- launch geometry */
/* §III.B: rays launched at division level n (edges of the icosahedron split into n
 * equal angles): N = 10 n^2 + 2.  Returns -1 for n < 1. */
int64_t sbr_num_rays(int32_t n_div);
/* Eq. 8: cone half-angle theta_launch = theta_0 / (sqrt(3) n), theta_0 = acos(1/sqrt(5)). */
double sbr_theta_launch(int32_t n_div);
/* Sub-ray pattern of the precise algorithm (§III.B, Fig. 5) for K in {6, 7, 9, 16}:
 * ring radius rho[k] and azimuth phi[k] of each sub-ray, as a fraction of the cone
 * half-angle and in radians, and the per-iteration shrink factor.  rho and phi must
 * hold K doubles (host).  K = 6 is the paper's pattern (shrink 1/sqrt(3)). */
sbr_status sbr_subray_pattern(int32_t K, double *rho, double *phi, double *shrink);

/* a1 -- §II.B, Eq. 1-2: equiangular division of the regular icosahedron.  Writes the
 * N = 10 n^2 + 2 unit launch directions as float4 (x, y, z, 0) to the DEVICE buffer
 * `dirs` (capacity cap_rays rows).  Order: 12 icosahedron vertices; 30 edges x (n-1)
 * equal-angle points (lower to higher vertex id); then per face its interior points by
 * layer a = 1, 2, ... (3(n - 3a) points each) and, when n = 0 mod 3, the face centre.
 * SBR_EINVAL if n < 1 or n > 20000; SBR_EOVERFLOW if cap_rays < N. */
sbr_status sbr_raygen(sbr_ctx *ctx, int32_t n_div, float *dirs, int64_t cap_rays);

/* §II.A (ref. 9): equidistant division, the launcher the paper compares against.  Ray
 * points at equal intervals on each flat face of a regular polyhedron, projected onto the
 * unit sphere: poly = 20 (the icosahedron of sbr_raygen, N = 10 n^2 + 2) or poly = 8 (the
 * octahedron with vertices +-x, +-y, +-z, N = 4 n^2 + 2).  Order: vertices; edges (lower to
 * higher vertex id) with points j = 1..n-1 at lo + (j/n)(hi - lo); per face (lowest vertex A
 * first, outward orientation A, B, C) the interior points A + (i/n)(B - A) + (j/n)(C - A),
 * i = 1..n-2, j = 1..n-1-i.  Writes float4 (x, y, z, 0) to the DEVICE buffer dirs.
 * SBR_EINVAL for n < 1, n > 14000 or another poly; SBR_EOVERFLOW if cap_rays < N. */
sbr_status sbr_raygen_equidistant(sbr_ctx *ctx, int32_t n_div, int32_t poly, float *dirs, int64_t cap_rays);
/* Rays launched by launcher (0 = equiangular icosahedron, 20 = equidistant icosahedron,
 * 8 = equidistant octahedron) at division level n; -1 if invalid. */
int64_t sbr_num_rays_launcher(int32_t n_div, int32_t launcher);

/* ---------------------------------------------------------------- scene */
typedef struct {
    int64_t num_triangles;
    int32_t num_faces;
    int32_t bvh_nodes;
    int32_t bvh_depth;
    int32_t max_leaf;
    int64_t device_bytes;
    float bbox_lo[3], bbox_hi[3];
    int32_t num_wedges;      /* wedges found for order-1 diffraction (sbr_scene_wedges) */
} sbr_scene_info;

/* Upload a triangle scene and build its SAH BVH on the host.  verts: nv x 3 floats;
 * tris: nt x 3 vertex ids; tri_face: nt face ids in [0, nf); face_eps: nf relative
 * permittivities (NULL or values <= 0: perfect reflector).  All host pointers.  A face's
 * plane is taken from its first triangle.  SBR_EDEGENERATE for NaN/Inf vertices, ids
 * out of range or zero-area triangles. */
sbr_status sbr_scene_upload(sbr_ctx *ctx, const float *verts, int64_t nv, const int32_t *tris,
                            const int32_t *tri_face, int64_t nt, const float *face_eps, int32_t nf,
                            sbr_scene **out);
sbr_status sbr_scene_destroy(sbr_ctx *ctx, sbr_scene *scene);
/* Host only (no device, no context): the convex outlines the validity test's point-in-face
 * query uses (§III.A: each refined bounce point must lie on its face).  corners (nf int32,
 * host) receives, per face, the corner count of the convex polygon its triangles tile
 * exactly (such a face is tested against that polygon's edges), or 0 when they do not
 * (the face is tested triangle by triangle through the BVH).  A face's plane comes from
 * its first triangle, as in sbr_scene_upload; the triangles tile the hull when, on that
 * plane, each turns like the normal, each edge occurs at most once per direction, and the
 * edges without a reverse twin and the triangles add up to the hull's perimeter and area
 * (relative 1e-9).  Same arrays as sbr_scene_upload; SBR_EINVAL for null or negative
 * sizes, SBR_EDEGENERATE for ids out of range or zero-area triangles. */
sbr_status sbr_face_outline_corners(const float *verts, int64_t nv, const int32_t *tris, const int32_t *tri_face,
                                    int64_t nt, int32_t nf, int32_t *corners);
sbr_status sbr_scene_get_info(const sbr_scene *scene, sbr_scene_info *out);
/* The scene's wedges, where rays diffract (§III.A, Fig. 4; the paper does not define a
 * wedge, this library's reading): a side shared by two faces -- the same segment, with
 * identical endpoint coordinates, on the boundary of both (a face's boundary triangle
 * edges with collinear neighbours joined) -- whose half-planes meet at an interior angle
 * between 1 and 170 degrees; the solid fills the smaller sector, rays diffract into the
 * larger one.  Wedge ids follow the order of the face pairs (f1 < f2).  Writes
 * min(cap, count) wedges to host arrays ab (cap x 6 floats: end a xyz, end b xyz) and
 * faces (cap x 2: f1, f2); *count = the number of wedges.  SBR_EINVAL for null
 * arguments or cap < 0. */
sbr_status sbr_scene_wedges(const sbr_scene *scene, float *ab, int32_t *faces, int64_t cap, int64_t *count);

/* ---------------------------------------------------------------- receivers */
/* Upload nrx receiver positions (host, nrx x 3 floats) and build their BVH (used by the
 * reception judgment to find candidate Rx near a ray segment). */
sbr_status sbr_rx_upload(sbr_ctx *ctx, const float *rx, int32_t nrx, sbr_rxset **out);
sbr_status sbr_rx_destroy(sbr_ctx *ctx, sbr_rxset *rx);

/* ---------------------------------------------------------------- paths */
/* Device container for reception records and paths.  record_cap bounds the records one
 * launch may emit (before double-count removal), path_cap the unique paths. */
sbr_status sbr_paths_create(sbr_ctx *ctx, int64_t record_cap, int64_t path_cap, sbr_paths **out);
sbr_status sbr_paths_destroy(sbr_ctx *ctx, sbr_paths *paths);

typedef struct {
    int32_t n_div;           /* division level n >= 1 */
    int32_t max_order;       /* maximum reflections, 0..SBR_MAX_ORDER */
    float rx_angle_scale;    /* alpha: reception cone = alpha * theta_launch (1 = paper) */
    int32_t flags;           /* SBR_LAUNCH_* */
    int32_t dump_stride;     /* > 0: record per-ray face sequences of ray ids % stride == 0 */
    int32_t *dump_faces;     /* device, [ntx][ceil(N/stride)][max_order+1] face per segment
                                (-1 miss, -2 not traced), or NULL */
    int64_t dump_cap;        /* int32 entries in dump_faces; SBR_EINVAL if too small */
    int32_t grid_blocks;     /* persistent trace grid (0 = one wave over all SMs) */
    int32_t block_threads;   /* multiple of 32, at most 128 (0 = 128) */
    int32_t refill_min;      /* a warp takes new rays once this many of its lanes are idle
                                (1..32; 0 = 24: keeps a warp's rays neighbours in the lattice) */
    int32_t launcher;        /* 0 = equiangular (§II.B), 20 / 8 = equidistant icosahedron /
                                octahedron (§II.A); ray ids follow that launcher's order */
    int64_t ray_begin;       /* with SBR_LAUNCH_RAY_RANGE: trace only ray ids [ray_begin, ray_end) */
    int64_t ray_end;         /* of every transmitter (0 <= ray_begin <= ray_end <= N; rays are
                                independent, §III.A, so disjoint ranges split one launch) */
} sbr_launch_params;

#define SBR_LAUNCH_SYNC 1    /* synchronise at the end and report overflow / collisions */
#define SBR_LAUNCH_TIMING 2  /* record CUDA events around each kernel (read by get_stats) */
#define SBR_LAUNCH_DIFFRACTION 4 /* also search order-1 diffraction paths (§III.A, Fig. 4; §IV,
                                    Figs. 7c-d): a ray's first segment that passes a wedge
                                    inside its cone diffracts on the Keller cone, and a
                                    receiver in the wedge's exterior whose Eq. 3 error angle
                                    in the wedge's unfolded space (Rx rotated about the edge
                                    into the half-plane opposite Tx) is within the cone and
                                    whose segment from the edge is unblocked gets a record;
                                    the path has order 1 and faces[0] = -1 - wedge id */
#define SBR_LAUNCH_RAY_RANGE 8  /* trace only ray_begin..ray_end of each transmitter; record ray
                                   ids stay the lattice's own (position-independent records) */
#define SBR_LAUNCH_RECORDS_ONLY 16 /* stop after the reception judgment: the container keeps the
                                      reception records (sbr_records_read) and no paths */
#define SBR_LAUNCH_ID_ORDER 32 /* trace the rays in lattice id order.  By default a launch of a
                                  whole equiangular lattice takes them in compact tiles of
                                  each face's triangular grid (neighbouring directions together
                                  in a warp); the results are the same either way (§III.A:
                                  rays are independent) */

typedef struct {
    int64_t rays;            /* rays traced (ntx * N) */
    int64_t segments;        /* closest-hit queries = ray-bounces */
    int64_t node_visits;     /* 4-wide BVH nodes visited by the trace (four box tests each) */
    int64_t tri_tests;       /* ray-triangle tests */
    int64_t rx_tests;        /* candidate Rx tested */
    int64_t records;         /* reception records emitted (may exceed record_cap) */
    int64_t paths;           /* unique paths after double-count removal (may exceed path_cap) */
    int64_t collisions;      /* dedup hash collisions detected (must be 0) */
    int32_t ntx, nrx, n_div, max_order;
    float ms_raygen, ms_trace, ms_dedup; /* device time of each kernel group (SBR_LAUNCH_TIMING), else 0 */
    int32_t trace_grid, trace_block;     /* launch shape of the trace kernel */
    float ms_diffract;                   /* device time of the diffraction search (SBR_LAUNCH_TIMING) */
    int64_t wedge_tests;                 /* wedges tested by the diffraction search */
    int64_t diffraction_records;         /* diffraction records emitted */
    int64_t diffraction_candidates;      /* (ray, wedge) candidates (may exceed candidate_cap) */
    int64_t candidate_cap;               /* candidates the container holds: 1.25 x record_cap or more */
    int64_t check_flags;                 /* SBR_CHECK_* bits of failed device bounds checks of the
                                            container's work since its last launch (SBR_CHECKED
                                            builds; always 0 otherwise) */
} sbr_launch_stats;

/* a1-a5 -- §III.A / Fig. 4: launch N rays from each of ntx transmitters (tx: ntx x 3
 * floats, host or device), trace up to max_order specular reflections through the
 * scene's BVH (closest hit, watertight triangle test), run the reception judgment
 * against every receiver on every segment (Rx inside the cone alpha * theta_launch,
 * error angle Eq. 3) and remove double counts (per (Tx, Rx, face sequence) keep the
 * smallest error angle, ties to the lowest ray id).  The paths replace the container's
 * previous contents.  Asynchronous unless SBR_LAUNCH_SYNC; overflow is reported by
 * sbr_launch_get_stats (and by the SYNC return code). */
sbr_status sbr_launch(sbr_ctx *ctx, const sbr_scene *scene, const float *tx, int32_t ntx,
                      const sbr_rxset *rx, const sbr_launch_params *params, sbr_paths *paths);
/* Bounds checks of SBR_CHECKED builds (the library compiled with -DSBR_CHECKED; the
 * environment variable SBR_CHECKED_STACK_LIMIT, read at scene upload, lowers the traversal
 * stack entries a walk may use, to exercise the checks).  A failed check sets its bit in the
 * container's status word and stops the query that failed (a miss, or an unoccluded
 * segment): no assert, no trap.  sbr_launch with SBR_LAUNCH_SYNC and sbr_query then return
 * SBR_ECHECK, naming the failed checks in sbr_last_error. */
#define SBR_CHECK_TRACE_STACK 1      /* closest-hit walk of the trace */
#define SBR_CHECK_OCCLUSION_STACK 2  /* any-hit walk of the validity test */
#define SBR_CHECK_RX_STACK 4         /* receiver walk of the reception judgment */
#define SBR_CHECK_FACE_ID 8          /* a face id outside [0, num_faces) met on the device */
#define SBR_CHECK_BVH2_STACK 16      /* binary-BVH walks (point in face, wedge search) */

/* Synchronises the stream and reads the counters of the container's last launch. */
sbr_status sbr_launch_get_stats(sbr_ctx *ctx, const sbr_paths *paths, sbr_launch_stats *out);

/* ---------------------------------------------------------------- reception records */
/* One reception record of §III.A (Fig. 4): ray `ray` of transmitter `tx`, on the segment
 * after `order` reflections on faces[0..order), received Rx `rx` inside its cone with the
 * error angle of Eq. 3 and propagation distance dray to the foot of Rx.  Order-1
 * diffraction records have faces[0] = -1 - wedge id.  Records name lattice ray ids and hold
 * no buffer positions, so records of disjoint ray ranges can be concatenated. */
typedef struct {
    int32_t tx, rx, ray, order;
    int32_t faces[SBR_MAX_ORDER]; /* -1 padded */
    float err;               /* Eq. 3 error angle (rad) */
    float dray;              /* distance along the ray to the foot of Rx (m) */
    int32_t slot;            /* library-internal (dedup table slot); ignored on input */
    int32_t pad;
} sbr_reception_record;      /* 64 bytes */

/* Copy up to cap of the reception records the container's last sbr_launch emitted (before
 * double-count removal; order unspecified) to `out` (host or device); *written = records
 * copied.  The launch's total is sbr_launch_stats.records (records beyond record_cap were
 * dropped and are not copied).  Synchronises. */
sbr_status sbr_records_read(sbr_ctx *ctx, const sbr_paths *paths, sbr_reception_record *out, int64_t cap,
                            int64_t *written);
/* a5 -- §III.A, first path test, on a given record set: replace the container's records
 * with `count` records from `in` (host or device, e.g. the concatenated records of launches
 * over disjoint ray ranges) and remove double counts exactly as sbr_launch does (per (Tx,
 * Rx, face sequence) the smallest error angle, ties to the lowest ray id).  The paths that
 * replace the container's are those whose pair is owned by shard `rank` of `world`:
 * (tx * nrx + rx) mod world == rank (world = 1: all).  The container must hold a launch of
 * the same transmitters, receivers and division level (its refinement context is kept).
 * SBR_EOVERFLOW if count > record_cap; SBR_EINVAL unless 0 <= rank < world.  Asynchronous. */
sbr_status sbr_records_dedup(sbr_ctx *ctx, sbr_paths *paths, const sbr_reception_record *in, int64_t count,
                             int32_t rank, int32_t world);

/* ---------------------------------------------------------------- refinement */
typedef struct {
    int32_t max_iters;       /* iteration cap (>= 0) */
    int32_t subrays;         /* K in {6, 7, 9, 16} */
    double target_err_rad;   /* stop once the AOD error (the error angle) and the AOA error
                                are both <= this (<= 0: never early) */
    double fp64_below_rad;   /* run an iteration in FP64 once the cone half-angle is below
                                this (default 1e-5 when 0) */
    double freq_hz;          /* carrier for the power term (0: 2.4e9) */
    double ptx_dbm;          /* transmit power */
    int8_t *choice_log;      /* device [path_cap][max_iters], or NULL: per iteration the argmin
                                sub-ray k (bits 0-3) and the sub-cone frame's reference axis
                                0/1/2 = x/y/z (bits 4-5: the world axis of smallest |c_i|) */
} sbr_refine_params;

/* a6-a8 -- §III.B, Fig. 5, Eq. 10 and §III.A: refine every path of the container.  The
 * initial cone is centred on the path's rough launch direction with half-angle
 * max(theta_launch, rough error angle); each iteration traces K sub-rays through the
 * path's fixed face planes, keeps the one with the smallest error angle (Eq. 3) and
 * shrinks the cone, until the iteration cap or, with a target, until the path's AOD and
 * AOA errors both meet it (§III.B: iterate until the error satisfies the requirement;
 * the AOA error is measured exactly in the unfolded space).  Then the validity test
 * (bounce points inside their faces, no segment occluded) and the outputs (delay, AOD,
 * AOA, power).  One thread per path, static schedule. */
sbr_status sbr_refine(sbr_ctx *ctx, const sbr_scene *scene, sbr_paths *paths, const sbr_refine_params *params);
/* Same as sbr_refine restricted to the paths of one (tx, rx) pair: the per-pair form.  The
 * first call after a launch groups the paths by pair and reads the groups' ranges back to
 * the host once (synchronises); later calls are asynchronous. */
sbr_status sbr_refine_pair(sbr_ctx *ctx, const sbr_scene *scene, sbr_paths *paths, int32_t tx, int32_t rx,
                           const sbr_refine_params *params);

typedef struct {
    int32_t block_threads;   /* threads per block (0 = 128) */
    int32_t blocks_per_sm;   /* resident blocks per SM for the persistent grid (0 = max) */
    int32_t lanes_per_path;  /* lanes cooperating on one path: 1, 8, 16 or 32 (0 = 16) */
} sbr_batch_config;

/* a9 -- batched form of a6-a8: one persistent launch refines all paths of all (Tx, Rx)
 * pairs.  A group of lanes_per_path lanes owns one path: its lanes evaluate the K
 * sub-rays of an iteration in parallel (one lane: all K in turn, the form for many
 * paths); a group that finishes a path (iteration cap, target reached, stalled) takes the
 * next one from a device work queue (atomic head), so uneven iteration counts do not idle
 * the GPU.  With many paths (and always with one lane per path) a launch before it unfolds
 * every path's planes one path per thread and a launch after it runs the FP64 iterations
 * one path per thread.  A last launch runs the validity test and outputs (one thread per
 * path when there are many, one warp per path when there are few).  Results equal
 * sbr_refine's.  Capturable in a CUDA graph (no host synchronisation, no allocation). */
sbr_status sbr_batch_refine(sbr_ctx *ctx, const sbr_scene *scene, sbr_paths *paths,
                            const sbr_refine_params *params, const sbr_batch_config *cfg);

/* ---------------------------------------------------------------- results */
typedef struct {
    int32_t tx, rx;          /* transmitter / receiver index */
    int32_t ray;             /* lattice ray id of the rough path */
    int32_t order;           /* reflections */
    int32_t faces[SBR_MAX_ORDER]; /* face sequence, -1 padded */
    float rough_err;         /* Eq. 3 error angle of the rough path (rad) */
    float rough_dray;        /* propagation distance to the foot of Rx (m) */
    int32_t iters;           /* refinement iterations done */
    int32_t valid;           /* 1 if the validity test passed (after refinement) */
    double dir[3];           /* launch direction (refined if iters > 0) */
    double err;              /* Eq. 3 error angle of dir (rad) */
    double delay;            /* s */
    float aod[2];            /* azimuth, elevation of departure */
    float aoa[2];            /* azimuth, elevation of p_k - Rx (Tx - Rx for LOS) */
    float power_dbm;
    int32_t flags;           /* SBR_PATH_* */
} sbr_path_record;           /* 128 bytes */

#define SBR_PATH_REFINED 1
#define SBR_PATH_FP64 2      /* at least one iteration ran in FP64 */
#define SBR_PATH_TRACE_FAIL 4 /* all sub-rays invalid at some iteration */
#define SBR_PATH_STALLED 16   /* the refinement stopped early because the error angle exceeded
                                 R (1 / (1 - s) + 2 s) + 1e-6: the path can no longer pass the
                                 convergence condition and is invalid */
#define SBR_PATH_DIFFRACTED 8 /* order-1 diffraction path: faces[0] = -1 - wedge id; the
                                 refinement runs in the wedge's unfolded space, the validity
                                 test asks the diffraction point to lie on the wedge, both
                                 ends in its exterior and both legs unblocked; power is free-
                                 space loss only (the paper gives no diffraction coefficient) */

/* Number of the container's valid paths with a non-finite output (direction, error angle,
 * delay, AOD, AOA or power): a device scan, 0 when the outputs are sound.  Synchronises. */
sbr_status sbr_paths_nonfinite(sbr_ctx *ctx, const sbr_paths *paths, int64_t *count);

/* Number of paths in the container (synchronises). */
sbr_status sbr_paths_count(sbr_ctx *ctx, const sbr_paths *paths, int64_t *out);
/* Copy up to cap path records to `out` (host or device); *written = records copied.
 * Synchronises.  Record order is unspecified (sort by tx, rx, order, faces). */
sbr_status sbr_query(sbr_ctx *ctx, const sbr_paths *paths, sbr_path_record *out, int64_t cap, int64_t *written);
/* Replace the container's paths with `count` records (host or device), e.g. to resume
 * refinement from exported rough paths.  tx/rx positions are taken from `tx` (ntx x 3,
 * host or device) and the receiver set. */
sbr_status sbr_paths_import(sbr_ctx *ctx, sbr_paths *paths, const sbr_path_record *in, int64_t count,
                            const float *tx, int32_t ntx, const sbr_rxset *rx, int32_t n_div);

/* ---------------------------------------------------------------- unfolding + adjoint */
/* a10 -- fixed-face-sequence unfolding (the exact per-sequence geometry that the precise
 * algorithm converges to).  For path p with faces[p*8 .. p*8+order[p]) and mirror maps
 * M_f(x) = x - 2 (n.x - h) n: Rx' = M_f1(...M_fk(Rx)), w = Rx' - Tx, d = launch direction
 * of (az, el).  Outputs per path (8 floats): miss[3] = real-space vector from the foot of
 * Rx on the last leg to Rx, delay = |w| / c0, AOD (az, el) of w, AOA (az, el) of the last
 * Tx image minus Rx.  All pointers DEVICE: tx, rx [P][3]; az_el [P][2]; faces [P][8];
 * order [P]; out [P][8]. */
sbr_status sbr_unfold_fwd(sbr_ctx *ctx, const sbr_scene *scene, int64_t npaths, const float *tx,
                          const float *rx, const float *az_el, const int32_t *faces, const int32_t *order,
                          float *out);
/* Vector-Jacobian product of sbr_unfold_fwd: given grad_out [P][8], writes grad_tx,
 * grad_rx [P][3] and grad_az_el [P][2] (DEVICE).  Bounce state is recomputed, not read
 * from the forward pass.  A path with a face id outside [0, nf) gets NaN gradients.  When
 * every input array is 16-byte aligned and there are at least two 256-path tiles per SM,
 * the kernel stages whole tiles of the inputs in shared memory with bulk copies (same
 * results, bit for bit, as the unstaged form); should a tile's copies not arrive within
 * one second, the paths that block had left get NaN gradients instead of a hang. */
sbr_status sbr_unfold_bwd(sbr_ctx *ctx, const sbr_scene *scene, int64_t npaths, const float *tx,
                          const float *rx, const float *az_el, const int32_t *faces, const int32_t *order,
                          const float *grad_out, float *grad_tx, float *grad_rx, float *grad_az_el);

/* ---------------------------------------------------------------- allocation-free dedup */
/* The paper has no counterpart of this entry point; it serves callers that cannot let the
 * library allocate device memory while they call it, e.g. processes whose device memory is
 * fully reserved by another framework's pool.
 *
 * sbr_dedup_noalloc repeats the double-count removal of sbr_launch on the reception
 * records that the last sbr_launch left in `src`, writing the unique paths to `out`
 * (DEVICE, room for `cap` records, filled in unspecified order like sbr_query's) and
 * counts[0] = number of unique paths (may exceed cap; only cap are written),
 * counts[1] = hash collisions detected (0 when correct) to `counts` (DEVICE, 2 int64).
 * It allocates and frees nothing: its hash table is a fixed array of about 5.5 MiB in
 * device global memory that every GPU loading the library keeps until the process exits.
 * Limits and rules:
 *   - SBR_EINVAL if src's record capacity exceeds SBR_NOALLOC_MAX_RECORDS, or if the
 *     context's ray directions no longer belong to src's launch (another division level
 *     was launched since);
 *   - all calls share the array; each call clears it first, and calls whose GPU work
 *     overlaps (e.g. on two streams) race and corrupt each other's output;
 *   - the first call on a device looks up the array's device address for that device,
 *     and every call made while the context's stream is not capturing looks it up again
 *     (a device reset moves the array); make the first call on a device, and the first
 *     after a device reset, before any stream capture;
 *   - SBR_EINVAL if src's records do not live on the context's device.
 * Asynchronous on the context's stream. */
#define SBR_NOALLOC_MAX_RECORDS 131072
sbr_status sbr_dedup_noalloc(sbr_ctx *ctx, const sbr_paths *src, sbr_path_record *out, int64_t cap,
                             int64_t *counts);

#ifdef __cplusplus
}
#endif
#endif /* SBR_H_ */
