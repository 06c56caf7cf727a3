// kernels_diffract.cu -- the rough search for order-1 diffraction paths (§III.A, Fig. 4:
// rays reflect on faces and diffract on wedges; §IV, Figs. 7c-d).
//
// Per (Tx, ray) (two passes, below).  A ray meets a wedge when the edge point X seen at the
// smallest angle to the ray lies inside the ray cone (angle <= cone) and ahead of Tx, Tx
// lies in the wedge's exterior, and X is visible from Tx (segment Tx -> X unblocked, the
// wedge's two faces excluded: a ray grazing one of them just before the edge still has
// the edge in its cone).  The diffracted rays leave X on its Keller cone; a receiver gets
// one when it lies in the exterior, its Eq. 3 error angle in the wedge's unfolded space --
// angle(d, Rx* - Tx), Rx* being Rx rotated about the edge line into the half-plane
// opposite Tx -- is within the cone, and the segment X -> Rx is unblocked (the wedge's two
// faces excluded).  Each such (ray, wedge, Rx) appends a record (order 1, faces[0] =
// -1 - wedge id) to the launch's record buffer, before double-count removal.
//
// Candidate wedges come from a BVH over the wedge segments, each node box grown by
// tan(cone) times the largest foot of its corners on the ray: every point of the box
// inside the ray cone then lies within that margin of the ray (see cone_box).
#include "lattice_order.cuh"
#include "sbr_device.cuh"

namespace sbr {

struct WedgeF {
    float3 a, b, w1, w2;
    int f1, f2;
};

__device__ __forceinline__ WedgeF load_wedge(const SceneDev &S, int id) {
    const float4 *p = S.wedges + 4 * (size_t)id;
    float4 A = __ldg(p), B = __ldg(p + 1), W1 = __ldg(p + 2), W2 = __ldg(p + 3);
    return {f3(A), f3(B), f3(W1), f3(W2), __float_as_int(A.w), __float_as_int(B.w)};
}

__device__ __forceinline__ float angle32(float3 d, float3 v) {
    float3 c = cross(d, v);
    return atan2f(sqrtf(dot(c, c)), dot(d, v));
}

// p lies outside the interior sector (the solid) between w1 and w2; e = edge direction
__device__ __forceinline__ bool exterior32(const WedgeF &w, float3 e, float3 p) {
    float3 q = p - w.a;
    q = q - e * dot(q, e);
    float3 n = cross(w.w1, w.w2);
    return !(dot(cross(w.w1, q), n) > 0.0f && dot(cross(q, w.w2), n) > 0.0f);
}

// the edge point seen from o at the smallest angle to d (segment end or the interior
// critical point of the angle along the edge line); returns that angle
__device__ __forceinline__ float nearest_seen(const WedgeF &w, float3 o, float3 d, float3 &X) {
    const float3 a0 = w.a - o, eb = w.b - w.a;
    const float al = dot(d, a0), be = dot(d, eb), c = dot(a0, a0), ep = dot(a0, eb), g = dot(eb, eb);
    float uc = -1.0f;
    const float den = be * ep - al * g;
    if (den != 0.0f) {
        float u = (al * ep - be * c) / den;
        if (u > 0.0f && u < 1.0f) uc = u;
    }
    float best = INFINITY;
    const float cand[3] = {0.0f, 1.0f, uc};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (cand[i] < 0.0f) continue;
        float3 v = a0 + eb * cand[i];
        float ang = angle32(d, v);
        if (ang < best) {
            best = ang;
            X = o + v;
        }
    }
    return best;
}

// Child box of a 2-wide node against the ray cone.  A box point X inside the cone has its
// foot s_X on the ray between 0 and s_max, the largest foot of any box corner, and lies
// within s_X tan(cone) <= s_max tan(cone) of the ray; so the box grown by that radius
// (plus a relative rounding margin) must meet the ray segment t in [0, s_max].  od = o . d.
__device__ __forceinline__ bool cone_box(float lx, float ly, float lz, float hx, float hy, float hz, const RayPre &r,
                                         float od, float tan_cone) {
    const float smax = (r.d.x > 0.0f ? hx : lx) * r.d.x + (r.d.y > 0.0f ? hy : ly) * r.d.y +
                       (r.d.z > 0.0f ? hz : lz) * r.d.z - od;
    if (!(smax > 0.0f)) return false;
    const float g = smax * (tan_cone * 1.001f + 1e-6f);
    const float t0x = (lx - g - r.o.x) * r.inv.x, t1x = (hx + g - r.o.x) * r.inv.x;
    const float t0y = (ly - g - r.o.y) * r.inv.y, t1y = (hy + g - r.o.y) * r.inv.y;
    const float t0z = (lz - g - r.o.z) * r.inv.z, t1z = (hz + g - r.o.z) * r.inv.z;
    const float tn = fmaxf(fmaxf(fminf(t0x, t1x), fminf(t0y, t1y)), fmaxf(fminf(t0z, t1z), 0.0f));
    const float tf = fminf(fminf(fmaxf(t0x, t1x), fmaxf(t0y, t1y)), fminf(fmaxf(t0z, t1z), smax * 1.000001f + g));
    return tn <= tf;
}

// Pass 1, one thread per (Tx, ray): candidate wedges of the ray (edge point X inside the
// cone, ahead of Tx, Tx in the exterior), appended to the candidate list as (X, ray) and
// (tx, wedge).  The walk advances one node or one wedge per loop turn, so the lanes of a
// warp append their candidates together (one atomic per turn).
__global__ void __launch_bounds__(128) diffract_candidates(DiffractArgs A) {
    const SceneDev &S = A.scene;
    const long long total = (long long)A.ntx * A.nrays_per_tx;
    const int lane = threadIdx.x & 31;
    unsigned tests = 0;
    // grid-stride in whole warps so that every lane reaches the warp-wide votes
    for (long long base = (blockIdx.x * (long long)blockDim.x + threadIdx.x) - lane; base < total;
         base += (long long)gridDim.x * blockDim.x) {
        const long long i = base + lane;
        bool done = i >= total, tail = false;
        const int txi = done ? 0 : (int)(i / A.nrays_per_tx);
        const int local = done ? 0 : (int)(i - (long long)txi * A.nrays_per_tx);
        const int ray = A.tiled_n > 0 ? tiled_ray(local, A.tiled_n) : (int)A.ray_begin + local;
        const float3 o = f3(__ldg(A.tx + txi));
        const float3 d = f3(__ldg(A.dirs + ray));
        const RayPre r = make_ray(o, d);
        const float od = dot(o, d);
        int stack[kStackDepth];
        int sp = 0, node = 0, li = 0, ln = 0;
        for (;;) {
            int cand = -1;
            float3 X = o;
            if (!done) {
                if (ln > 0) {
                    const int id = __ldg(S.wedge_bvh_ids + li);
                    const WedgeF w = load_wedge(S, id);
                    ++tests;
                    const float ang = nearest_seen(w, o, d, X);
                    if (ang <= A.cone && dot(X - o, d) > 0.0f) {
                        float3 eb = w.b - w.a;
                        if (exterior32(w, eb * (1.0f / sqrtf(dot(eb, eb))), o)) cand = id;
                    }
                    ++li;
                    --ln;
                    if (ln == 0 && tail) done = true;
                } else if (is_leaf(node)) {
                    li = leaf_first(node);
                    ln = leaf_count(node);
                    if (sp > 0) node = stack[--sp];
                    else tail = true;
                    if (ln == 0 && tail) done = true;
                } else {
                    const float4 *nd = S.wnodes + 4 * (size_t)node;
                    float4 p = __ldg(nd), q = __ldg(nd + 1), t = __ldg(nd + 2);
                    int4 refs = __ldg(reinterpret_cast<const int4 *>(nd + 3));
                    bool in0 = cone_box(p.x, p.y, p.z, p.w, q.x, q.y, r, od, A.tan_cone);
                    bool in1 = cone_box(q.z, q.w, t.x, t.y, t.z, t.w, r, od, A.tan_cone);
                    if (in0 && in1 && SBR_CHECKED_ON && sp >= min(S.stack_limit, kStackDepth)) {
                        check_fail(S, SBR_CHECK_BVH2_STACK);
                        done = true;
                    } else if (in0 && in1) {
                        stack[sp++] = refs.y;
                        node = refs.x;
                    } else if (in0) {
                        node = refs.x;
                    } else if (in1) {
                        node = refs.y;
                    } else if (sp > 0) {
                        node = stack[--sp];
                    } else {
                        done = true;
                    }
                }
            }
            const unsigned want = __ballot_sync(0xffffffffu, cand >= 0);
            if (want) {
                const int leader = __ffs(want) - 1;
                unsigned long long at = 0;
                if (lane == leader)
                    at = atomicAdd(reinterpret_cast<unsigned long long *>(A.counters + kDiffCand),
                                   (unsigned long long)__popc(want));
                at = __shfl_sync(0xffffffffu, at, leader);
                if (cand >= 0) {
                    const long long slot = (long long)at + __popc(want & ((1u << lane) - 1u));
                    if (slot < A.cand_cap) {
                        A.cand[2 * slot] = make_float4(X.x, X.y, X.z, __int_as_float(ray));
                        A.cand[2 * slot + 1] = make_float4(__int_as_float(txi), __int_as_float(cand), 0.0f, 0.0f);
                    }
                }
            }
            if (__all_sync(0xffffffffu, done)) break;
        }
    }
    tests = __reduce_add_sync(0xffffffffu, tests);
    if (lane == 0 && tests) atomicAdd(reinterpret_cast<unsigned long long *>(A.counters + kWedgeTests), tests);
}

// Pass 2, 32 candidates per warp: each lane checks that its candidate's edge point is
// visible from Tx; then for every visible candidate the whole warp tests the receivers
// (lane-strided): exterior, unfolded error angle within the cone, unblocked X -> Rx.
// Receptions waiting for their occlusion query (diffract_occlusion) are parked at the top of
// the record array, slot rec_cap - 1 - q for the q-th, while the final records grow from
// the trace's count n0 at the bottom; parking q < (rec_cap - n0) / 2 of them leaves room for
// all of them as final records, so the two ends never meet.  Past that bound the launch
// reports record overflow (the record count is raised above the capacity).
__device__ __forceinline__ long long park_limit(const DiffractArgs &A, long long n0) { return (A.rec_cap - n0) / 2; }

__global__ void __launch_bounds__(256) diffract_receive(DiffractArgs A) {
    const SceneDev &S = A.scene;
    long long ncand = A.counters[kDiffCand];
    if (ncand > A.cand_cap) ncand = A.cand_cap;
    const long long n0 = A.counters[kRecords];   // the trace's records; nothing appends here
    const long long limit = park_limit(A, n0);
    if (blockIdx.x == 0 && threadIdx.x == 0) A.counters[kDiffBase] = n0;
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long base = (long long)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < ncand;
         base += warps * 32) {
        const long long c = base + lane;
        bool vis = false;
        float4 c0 = make_float4(0, 0, 0, 0), c1 = make_float4(0, 0, 0, 0);
        if (c < ncand) {
            c0 = A.cand[2 * c];
            c1 = A.cand[2 * c + 1];
            const WedgeF w = load_wedge(S, __float_as_int(c1.y));
            const float3 o = f3(__ldg(A.tx + __float_as_int(c1.x)));
            vis = !any_hit4(S, make_ray(o, f3(c0) - o), 1e-6f, 1.0f - 1e-6f, w.f1, w.f2);
        }
        unsigned todo = __ballot_sync(0xffffffffu, vis);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const float4 x0 = make_float4(__shfl_sync(0xffffffffu, c0.x, src), __shfl_sync(0xffffffffu, c0.y, src),
                                          __shfl_sync(0xffffffffu, c0.z, src), __shfl_sync(0xffffffffu, c0.w, src));
            const int txi = __float_as_int(__shfl_sync(0xffffffffu, c1.x, src));
            const int id = __float_as_int(__shfl_sync(0xffffffffu, c1.y, src));
            const int ray = __float_as_int(x0.w);
            const WedgeF w = load_wedge(S, id);
            const float3 o = f3(__ldg(A.tx + txi));
            const float3 d = f3(__ldg(A.dirs + ray));
            const float3 X = f3(x0);
            const float3 eb = w.b - w.a;
            const float3 e = eb * (1.0f / sqrtf(dot(eb, eb)));
            // frame of the plane across the edge: b1 towards Tx, b2 = e x b1.  A point
            // q = p - a has coordinates (x, y, z) = (q.b1, q.b2, q.e); its image rotated
            // into the half-plane opposite Tx is a + z e - sqrt(x^2 + y^2) b1, and it lies in
            // the solid's sector iff it is strictly between w1 and w2 (2-D cross products)
            float3 pt = (o - w.a) - e * dot(o - w.a, e);
            const float rt = sqrtf(dot(pt, pt));
            if (!(rt > 0.0f)) continue;
            const float3 b1 = pt * (1.0f / rt), b2 = cross(e, b1);
            const float w1x = dot(w.w1, b1), w1y = dot(w.w1, b2), w2x = dot(w.w2, b1), w2y = dot(w.w2, b2);
            const float s12 = w1x * w2y - w1y * w2x;
            const float3 a0 = w.a - o;
            const float t2 = A.tan_cone * A.tan_cone * 1.0001f;   // pre-test, the exact test follows
            for (int rx = lane; rx < A.rx.nrx; rx += 32) {
                const float3 R = f3(__ldg(A.rx.by_id + rx));
                const float3 q = R - w.a;
                const float x = dot(q, b1), y = dot(q, b2), z = dot(q, e);
                const float c1 = w1x * y - w1y * x, c2 = x * w2y - y * w2x;
                if (c1 * s12 > 0.0f && c2 * s12 > 0.0f) continue;   // Rx inside the solid's sector
                const float3 W = a0 + e * z - b1 * sqrtf(x * x + y * y);
                const float3 cw = cross(d, W);
                const float dw = dot(d, W), cc = dot(cw, cw);
                if (!(dw > 0.0f) || cc > dw * dw * t2) continue;
                const float err = atan2f(sqrtf(cc), dw);
                if (!(err <= A.cone)) continue;
                // the segment X -> Rx is tested by diffract_occlusion, a query per thread in
                // full warps (here it would run in one lane while the warp waits); the
                // reception is parked with X in its unused face slots 1-3
                const long long pq = (long long)atomicAdd(reinterpret_cast<unsigned long long *>(A.counters + kDiffPending), 1ULL);
                if (pq >= limit) {
                    atomicMax(reinterpret_cast<unsigned long long *>(A.counters + kRecords),
                              (unsigned long long)A.rec_cap + 1ULL);
                    continue;
                }
                RecDev rec;
                rec.tx = txi;
                rec.rx = rx;
                rec.ray = ray;
                rec.order = 1;
                rec.faces[0] = -1 - id;
                rec.faces[1] = __float_as_int(X.x);
                rec.faces[2] = __float_as_int(X.y);
                rec.faces[3] = __float_as_int(X.z);
#pragma unroll
                for (int j = 4; j < kMaxOrder; ++j) rec.faces[j] = -1;
                rec.err = err;
                rec.dray = sqrtf(dot(W, W)) * cosf(err);
                rec.slot = -1;
                rec.pad = 0;
                A.recs[A.rec_cap - 1 - pq] = rec;
            }
        }
    }
}

// The occlusion queries of the parked diffraction receptions: a reception whose segment from
// the edge point X to Rx is unblocked (the wedge's two faces excluded) becomes a record,
// appended with one atomic per warp; blocked ones are dropped.
__global__ void __launch_bounds__(128) diffract_occlusion(DiffractArgs A) {
    const SceneDev &S = A.scene;
    long long P = A.counters[kDiffPending];
    const long long limit = park_limit(A, A.counters[kDiffBase]);
    if (P > limit) P = limit;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    unsigned emitted = 0;
    for (long long base = (long long)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < P;
         base += warps * 32) {
        const long long q = base + lane;
        RecDev rec;
        bool keep = false;
        if (q < P) {
            rec = A.recs[A.rec_cap - 1 - q];
            const float3 X = make_float3(__int_as_float(rec.faces[1]), __int_as_float(rec.faces[2]),
                                         __int_as_float(rec.faces[3]));
            const float3 R = f3(__ldg(A.rx.by_id + rec.rx));
            const WedgeF w = load_wedge(S, -1 - rec.faces[0]);
            keep = !any_hit4(S, make_ray(X, R - X), 1e-6f, 1.0f - 1e-6f, w.f1, w.f2);
        }
        const unsigned b = __ballot_sync(0xffffffffu, keep);
        if (!b) continue;
        unsigned long long at = 0;
        if (lane == 0) at = atomicAdd(reinterpret_cast<unsigned long long *>(A.counters + kRecords), (unsigned long long)__popc(b));
        at = __shfl_sync(0xffffffffu, at, 0) + __popc(b & lt);
        if (keep) {
            rec.faces[1] = rec.faces[2] = rec.faces[3] = -1;
            if ((long long)at < A.rec_cap) A.recs[at] = rec;
            ++emitted;
        }
    }
    emitted = __reduce_add_sync(0xffffffffu, emitted);
    if (lane == 0 && emitted) atomicAdd(reinterpret_cast<unsigned long long *>(A.counters + kDiffRecords), emitted);
}

cudaError_t launch_diffract(const DiffractArgs &a, int num_sms, cudaStream_t s) {
    if (a.scene.nw == 0 || a.rx.nrx == 0) return cudaSuccess;
    diffract_candidates<<<num_sms * 8, 128, 0, s>>>(a);
    diffract_receive<<<num_sms * 4, 256, 0, s>>>(a);
    diffract_occlusion<<<num_sms * 8, 128, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace sbr
