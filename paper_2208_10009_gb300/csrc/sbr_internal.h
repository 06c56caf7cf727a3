// sbr_internal.h -- device layouts and launch wrappers shared by the library's
// translation units.  Not part of the public ABI (include/sbr.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/sbr.h"

#ifdef SBR_CHECKED
#define SBR_CHECKED_BUILD 1
#else
#define SBR_CHECKED_BUILD 0
#endif

namespace sbr {

constexpr int kMaxOrder = SBR_MAX_ORDER;
constexpr int kUnfStride = kMaxOrder + 2;   // float4 per path in the batched refinement's unf
constexpr double kC0 = 299792458.0;
constexpr int kLeafMax = 2;        // triangles per BVH leaf (target; 2 measured fastest: a
                                   // triangle test costs about half a 4-wide node visit)
constexpr int kStackDepth = 64;    // traversal stack entries (BVH depth is capped below this)
constexpr int kStack4 = 96;        // 4-wide traversal stack (the builder checks the bound)

// Device counters of one launch (int64 each).
enum Counter {
    kRays = 0, kSegments, kNodeVisits, kTriTests, kRxTests, kRecords, kPaths, kCollisions,
    kRayHead, kBatchHead, kBatchDone, kErrorFlags, kWedgeTests, kDiffRecords, kDiffCand, kNonFinite,
    kDiffPending,   // diffraction receptions parked at the top of the record array for diffract_occlusion
    kDiffBase,      // the record count before them (the trace's records)
    kNumCounters = 18
};

// BVH node: both children's boxes in one 64-byte node (4 x float4).
//   f[0] = (c0.lo.x, c0.lo.y, c0.lo.z, c0.hi.x)
//   f[1] = (c0.hi.y, c0.hi.z, c1.lo.x, c1.lo.y)
//   f[2] = (c1.lo.z, c1.hi.x, c1.hi.y, c1.hi.z)
//   f[3] = (child0 ref, child1 ref, -, -) as int bits
// A child ref >= 0 is an inner node index; a leaf ref has bit 31 set, 7 bits of
// primitive count (bits 24-30) and a 24-bit first-primitive index.
__host__ __device__ inline int leaf_ref(int first, int count) {
    return (int)(0x80000000u | ((unsigned)count << 24) | (unsigned)first);
}
__host__ __device__ inline bool is_leaf(int ref) { return ref < 0; }
__host__ __device__ inline int leaf_first(int ref) { return ref & 0xFFFFFF; }
__host__ __device__ inline int leaf_count(int ref) { return (ref >> 24) & 0x7F; }

// face plane in double: n.x = h
struct __align__(32) Plane64 {
    double x, y, z, w;
};

// BVH4 node (128 bytes = 8 x float4) used by the trace kernel: the four children's boxes
// in structure-of-arrays form, f[0] = lo.x of children 0..3, f[1] = hi.x, f[2] = lo.y,
// f[3] = hi.y, f[4] = lo.z, f[5] = hi.z; f[6] = the four child refs (same encoding as
// BVH2; an empty slot is a leaf with 0 primitives and a far-away point box); f[7] unused.

struct SceneDev {
    const float4 *nodes4;     // 8 per BVH4 node
    const float4 *nodes;      // 4 per node
    const float4 *tris;       // 3 per triangle: (v0, face id bits), (v1, 0), (v2, 0)
    const float4 *planes;     // per face: (n, h) with n.x = h on the plane
    const Plane64 *planes_d;  // same in double
    const float4 *planes_df;  // same as float pairs: 2 per face, (n, h) rounded and the residuals
    const float *face_eps;    // per face relative permittivity (<= 0: perfect reflector)
    const int *face_tri_off;  // CSR over faces -> triangle indices (BVH order)
    const int *face_tri_idx;
    const int2 *face_outline; // per face (first corner, count) of its convex outline, count 0:
                              // the face is tested triangle by triangle (build_face_outlines)
    const float4 *outline_v;  // outline corners, counter-clockwise about the face normal
    int nt, nf, nnodes;
    float tmin;               // hits need t > tmin (1e-7 x scene diagonal)
    // wedges (order-1 diffraction): per wedge 4 float4 in wedge-id order,
    // (a, f1 bits), (b, f2 bits), (w1, 0), (w2, 0); a BVH over them (same node layout as
    // the scene's) whose leaves index wedge_bvh_ids
    const float4 *wedges;
    const float4 *wnodes;
    const int *wedge_bvh_ids;
    int nw;
    // SBR_CHECKED builds: a failed bounds check ORs its SBR_CHECK_* bit into *status (the
    // running launch's counters[kErrorFlags]; null: not recorded) and the query that failed
    // stops; traversal walks push at most stack_limit entries (<= their array sizes)
    unsigned long long *status;
    int stack_limit;
};

struct RxDev {
    const float4 *nodes4;     // 4-wide BVH over receivers (same node layout as the scene's)
    const float4 *nodes;      // BVH over receivers (same node layout)
    const float4 *pts;        // BVH order: (x, y, z, original id bits)
    const float4 *by_id;      // original order: (x, y, z, 0)
    int nrx;
    float lo[3], hi[3];
};

// One reception record (64 bytes).
struct __align__(16) RecDev {
    int tx, rx, ray, order;
    int faces[kMaxOrder];
    float err, dray;
    int slot, pad;
};

// Lattice tables for ray generation at division level n.
struct LatticeDev {
    const float4 *ico;        // 12 vertices
    const int2 *edges;        // 30 edges (lo, hi)
    const float4 *centre;     // 20 face centre directions
    const float4 *layers;     // [20][nl][3]: (W_e.xyz, angle W_e -> W_{e+1})
    int n, nl;
    float edge_angle;         // theta_0
};

// Wedges of a triangle scene (host_wedges.cpp), ordered by face pair.
struct WedgeHost {
    float a[3], b[3];
    double w1[3], w2[3];
    int f1, f2;
};

// Flat-face tables for the equidistant launcher.
struct PolyDev {
    const float4 *v;          // vertices (unit)
    const int2 *edges;        // (lo, hi)
    const int4 *faces;        // (A, B, C, -) outward, lowest id first
    int nv, ne, nf, n;
};

}  // namespace sbr

// ---------------------------------------------------------------- host handle structs
struct sbr_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    sbr_alloc_fn alloc = nullptr;
    sbr_free_fn free_fn = nullptr;
    void *user = nullptr;
    std::string last_error;
    int num_sms = 0;
    int max_threads_per_sm = 0;
    // ray-generation workspace (directions for the last division level)
    void *dirs = nullptr;
    size_t dirs_bytes = 0;
    int dirs_n = 0;
    bool dirs_valid = false;
    // lattice tables
    void *lattice_mem = nullptr;
    size_t lattice_bytes = 0;
    int lattice_n = 0;
    sbr::LatticeDev lattice{};
    int dirs_launcher = 0;
    // equidistant launcher tables
    void *poly_mem = nullptr;
    size_t poly_bytes = 0;
    int poly_kind = 0;
    sbr::PolyDev poly{};
    // kernel timing events (SBR_LAUNCH_TIMING)
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
};

struct sbr_scene {
    void *mem = nullptr;
    size_t bytes = 0;
    sbr::SceneDev dev{};
    sbr_scene_info info{};
    std::vector<sbr::WedgeHost> wedges;   // host copy (sbr_scene_wedges)
};

struct sbr_rxset {
    void *mem = nullptr;
    size_t bytes = 0;
    sbr::RxDev dev{};
    std::vector<float> host;   // original order, 3 per receiver
};

struct sbr_paths {
    int64_t record_cap = 0, path_cap = 0;
    void *mem = nullptr;
    size_t bytes = 0;
    sbr::RecDev *recs = nullptr;
    sbr_path_record *paths = nullptr;
    float4 *unf = nullptr;                 // batched refinement: kUnfStride float4 per path
    int *order_idx = nullptr;              // batched refinement: path indices grouped by order
    unsigned long long *order_cnt = nullptr;   // [0, 10): paths per group; fill cursors: [16, 26) order_idx
                                               // from the front, [48, 58) from the back, [32, 42) fp64_idx
    int *fp64_idx = nullptr;               // batched refinement: paths handed to the FP64 tail
    unsigned long long *table = nullptr;   // dedup hash table: 2 x u64 per slot (key, value)
    int64_t table_slots = 0;
    long long *counters = nullptr;         // sbr::kNumCounters
    int *pair_off = nullptr;               // per-pair path ranges (sbr_refine_pair), lazily sized
    std::vector<int> pair_host;            // host copy of the per-pair offsets [npairs + 1]
    int64_t pair_cap = 0;
    void *pair_mem = nullptr;
    size_t pair_bytes = 0;
    // launch context kept for refinement
    float4 *tx = nullptr;                  // device, up to tx_cap transmitters
    int32_t tx_cap = 0;
    void *tx_mem = nullptr;
    size_t tx_bytes = 0;
    int32_t ntx = 0, nrx = 0, n_div = 0, max_order = 0, launcher = 0;
    const sbr_rxset *rx = nullptr;
    float alpha = 1.0f;
    int64_t ray_begin = 0, ray_count = 0;  // ray ids traced per transmitter by the last launch
    bool timed = false;                    // last launch recorded kernel events
    int trace_grid = 0, trace_block = 0;
};

// ---------------------------------------------------------------- internal helpers
namespace sbr {

// allocation through the context's callbacks (or cudaMallocAsync)
void *dev_alloc(sbr_ctx *ctx, size_t bytes);
void dev_free(sbr_ctx *ctx, void *p, size_t bytes);

// host geometry (host_geometry.cpp)
struct BvhOut {
    std::vector<float4> nodes;
    std::vector<float4> nodes4;    // the same tree collapsed to 4-wide nodes
    int max_stack4 = 0;            // worst-case 4-wide traversal stack use
    std::vector<int> prim_order;   // BVH leaf order -> original primitive index
    int depth = 0, max_leaf = 0;
};
// Build a binned-SAH BVH over boxes lo/hi (3 floats each) with centroids c.
bool build_bvh(const std::vector<float> &lo, const std::vector<float> &hi, int leaf_max, BvhOut &out,
               std::string &err);
// Lattice layer tables at division level n (host doubles -> float4 table).
void build_lattice_tables(int n, std::vector<float4> &ico, std::vector<int2> &edges, std::vector<float4> &centre,
                          std::vector<float4> &layers, int &nl);
// Sub-ray pattern constants.
int subray_pattern(int K, double *rho, double *phi, double *shrink);
bool build_wedges(const float *verts, int64_t nv, const int32_t *tris, const int32_t *tri_face, int64_t nt, int nf,
                  std::vector<WedgeHost> &out);
// Convex outlines of the faces whose triangles tile a convex polygon (host_faces.cpp).
constexpr int kMaxOutline = 32;
void build_face_outlines(const float *verts, const int32_t *tris, const int32_t *tri_face, int64_t nt, int nf,
                         const Plane64 *planes, std::vector<int2> &outline, std::vector<float4> &corners);
// Vertex / edge / face tables of the icosahedron (poly 20) or octahedron (poly 8).
bool build_polyhedron(int poly, std::vector<float4> &v, std::vector<int2> &e, std::vector<int4> &f);

// kernels (kernels_*.cu)
cudaError_t launch_raygen(const LatticeDev &lat, float4 *dirs, int64_t N, cudaStream_t s);
cudaError_t launch_raygen_equidistant(const PolyDev &p, float4 *dirs, int64_t N, cudaStream_t s);

struct TraceArgs {
    SceneDev scene;
    RxDev rx;
    const float4 *dirs;
    const float4 *tx;
    int ntx;
    int64_t nrays_per_tx;     // rays traced per transmitter: ids ray_begin .. ray_begin + nrays_per_tx
    int64_t ray_begin;
    int max_order;
    float cone;               // reception cone half-angle (rad)
    float tan_cone;
    float tan2_pre;           // tan^2(cone) (1 + 1e-4): conservative pre-test |q|^2 > tan2_pre d_ray^2
                              // rejects before the exact Eq. 3 test (INFINITY: no pre-test)
    RecDev *recs;
    int64_t rec_cap;
    long long *counters;
    int dump_stride;
    int *dump_faces;
    int64_t dump_per_tx;
    int refill_min;           // a warp takes new rays once at least this many lanes are idle
    int tiled_n;              // > 0: the launch traces the whole equiangular lattice of this
                              // division level, in the order of tiled_ray; 0: lattice id order
};
cudaError_t launch_trace(const TraceArgs &a, int grid, int block, cudaStream_t s);

struct DiffractArgs {
    SceneDev scene;
    RxDev rx;
    const float4 *dirs;
    const float4 *tx;
    int ntx;
    int64_t nrays_per_tx;     // rays searched per transmitter: ids ray_begin .. ray_begin + nrays_per_tx
    int64_t ray_begin;
    float cone, tan_cone;
    RecDev *recs;
    int64_t rec_cap;
    long long *counters;
    float4 *cand;             // candidate (ray, wedge) list, 2 float4 each (scratch)
    int64_t cand_cap;
    int tiled_n;              // as TraceArgs::tiled_n: the rays in the order of tiled_ray
};
cudaError_t launch_diffract(const DiffractArgs &a, int num_sms, cudaStream_t s);

struct DedupArgs {
    RecDev *recs;
    int64_t rec_cap;
    unsigned long long *table;
    int64_t slots;            // power of two
    sbr_path_record *paths;
    int64_t path_cap;
    const float4 *dirs;       // lattice directions (rough launch direction)
    long long *counters;
    int nrx;                  // paths of pair (tx, rx) are emitted iff (tx * nrx + rx) % shard_world
    int shard_rank, shard_world;   // == shard_rank
};
cudaError_t launch_dedup(const DedupArgs &a, int num_sms, cudaStream_t s);
// counters of a container whose records were replaced: kRecords = n, kPaths = kCollisions = 0
cudaError_t launch_records_reset(long long *counters, long long n, cudaStream_t s);
// counters[kNonFinite] = valid paths with a non-finite output
cudaError_t launch_nonfinite_scan(const sbr_path_record *paths, long long *counters, int64_t path_cap, int num_sms,
                                  cudaStream_t s);

struct RefineArgs {
    SceneDev scene;
    const float4 *tx;
    const float4 *rx;         // original order
    sbr_path_record *paths;
    long long *counters;      // kPaths holds the path count
    int64_t path_cap;
    const int *range;         // optional [begin, end) on device (per-pair form), or null
    const int *index;         // path indices addressed by range (per-pair form)
    int K;
    int max_iters;
    float theta_launch;
    double target;
    double tan2_target;       // tan^2(target) (early-stop test on |d x W|^2)
    float tan2_target_f;      // (float)tan2_target, for the FP32 phase
    int target_on;            // target > 0
    double fp64_below;
    float fp64_below_f;       // smallest float >= fp64_below: for a float x,
                              // x < fp64_below_f  <=>  x < fp64_below
    double freq;
    double ptx_dbm;
    int8_t *choice_log;
    float4 *unf;              // batched form, per path (kUnfStride float4): FP32 unfolded planes
                              // [0, kMaxOrder), W at kMaxOrder, rough direction at kMaxOrder + 1
    int *order_idx;           // batched form: path indices grouped by order (diffraction last)
    unsigned long long *order_cnt;   // batched form: group sizes [0, 10), fill cursors of order_idx
                                     // ([16, 26) from the front, [48, 58) from the back) and
                                     // [32, 42) of fp64_idx
    int *fp64_idx;            // batched form: paths whose FP64 iterations run in the tail kernel,
                              // grouped by order like order_idx
    int chunk;                // lanes per path in the batched kernel (8, 16, 32)
    long long split_min;      // batched form: from this many paths on, validity and outputs run
                              // one thread per path in a second kernel
    int ntx, nrx, nf, nw;     // bounds of the ids a path record may hold
};
cudaError_t launch_refine(const RefineArgs &a, int grid, int block, cudaStream_t s);
cudaError_t launch_batch_refine(const RefineArgs &a, int grid, int block, cudaStream_t s);
void refine_kernel_attrs(int *regs, int block, int *blocks_per_sm, bool batched, int lanes);
cudaError_t upload_subray_table(cudaStream_t s);

struct PairArgs {
    const sbr_path_record *paths;
    const long long *counters;
    int64_t path_cap;
    int nrx;
    int npairs;
    int *pair_count;          // [npairs + 1] scratch: counts then offsets
    int *pair_idx;            // [path_cap] path indices grouped by pair
};
cudaError_t launch_pair_bucket(const PairArgs &a, cudaStream_t s);

struct UnfoldArgs {
    SceneDev scene;
    int nf;
    int64_t n;
    const float *tx, *rx, *az_el;
    const int32_t *faces, *order;
    const float *grad_out;
    float *out, *grad_tx, *grad_rx, *grad_az_el;
};
cudaError_t launch_unfold_fwd(const UnfoldArgs &a, cudaStream_t s);
cudaError_t launch_unfold_bwd(const UnfoldArgs &a, cudaStream_t s);

int trace_blocks_per_sm(int block);

}  // namespace sbr
