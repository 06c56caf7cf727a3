// sbr_device.cuh -- device-side geometry: vector helpers, ray/box slab test, watertight
// ray/triangle test, BVH closest-hit and any-hit traversal, receiver candidate query.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "sbr_internal.h"

namespace sbr {

__device__ __forceinline__ float3 f3(float4 v) { return make_float3(v.x, v.y, v.z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float3 a, float s) { return make_float3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float dot(float3 a, float3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ float3 cross(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float comp(float3 v, int i) { return i == 0 ? v.x : (i == 1 ? v.y : v.z); }

struct dvec3 {
    double x, y, z;
};
__device__ __forceinline__ dvec3 dv(double x, double y, double z) { return {x, y, z}; }
__device__ __forceinline__ dvec3 operator+(dvec3 a, dvec3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ dvec3 operator-(dvec3 a, dvec3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ dvec3 operator*(dvec3 a, double s) { return {a.x * s, a.y * s, a.z * s}; }
__device__ __forceinline__ double ddot(dvec3 a, dvec3 b) { return fma(a.x, b.x, fma(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ dvec3 dcross(dvec3 a, dvec3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ double dnorm(dvec3 a) { return sqrt(ddot(a, a)); }

// Per-ray precomputation for the slab test and the watertight triangle test.  The
// triangle test's axis permutation and shear are folded into three vectors, so that a
// vertex's sheared coordinates are plain dot products (FMA pipe, no per-component
// selects): with kz the dominant axis of d and (kx, ky) the other two in winding order,
// mx = e_kx - (d_kx / d_kz) e_kz, my = e_ky - (d_ky / d_kz) e_kz, mz = e_kz / d_kz.
struct RayPre {
    float3 o, d, inv;
    float3 mx, my, mz;
    int nx, ny, nz;   // 1 where 1/d < 0: the near slab plane is the box's hi side
};

__device__ __forceinline__ RayPre make_ray(float3 o, float3 d) {
    RayPre r;
    r.o = o;
    r.d = d;
    // A zero component is replaced by 1e-30 before inverting: the slab tests stay correct
    // for axis-parallel rays (huge but finite t), and box * inv - o * inv never forms
    // inf - inf.
    r.inv = make_float3(1.0f / (d.x != 0.0f ? d.x : 1e-30f), 1.0f / (d.y != 0.0f ? d.y : 1e-30f),
                        1.0f / (d.z != 0.0f ? d.z : 1e-30f));
    r.nx = r.inv.x < 0.0f;
    r.ny = r.inv.y < 0.0f;
    r.nz = r.inv.z < 0.0f;
    float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
    int kz = (ax > ay) ? (ax > az ? 0 : 2) : (ay > az ? 1 : 2);
    int kx = kz == 2 ? 0 : kz + 1;
    int ky = kx == 2 ? 0 : kx + 1;
    if (comp(d, kz) < 0.0f) {
        int t = kx;
        kx = ky;
        ky = t;
    }
    const float sz = 1.0f / comp(d, kz);
    const float sx = comp(d, kx) * sz, sy = comp(d, ky) * sz;
    r.mx = make_float3(kx == 0 ? 1.0f : (kz == 0 ? -sx : 0.0f), kx == 1 ? 1.0f : (kz == 1 ? -sx : 0.0f),
                       kx == 2 ? 1.0f : (kz == 2 ? -sx : 0.0f));
    r.my = make_float3(ky == 0 ? 1.0f : (kz == 0 ? -sy : 0.0f), ky == 1 ? 1.0f : (kz == 1 ? -sy : 0.0f),
                       ky == 2 ? 1.0f : (kz == 2 ? -sy : 0.0f));
    r.mz = make_float3(kz == 0 ? sz : 0.0f, kz == 1 ? sz : 0.0f, kz == 2 ? sz : 0.0f);
    return r;
}

// SBR_CHECKED builds: record a failed bounds check (bit = SBR_CHECK_*) in the launch's
// status word.  The caller then ends the query that failed; nothing traps.
__device__ __forceinline__ void check_fail(const SceneDev &S, unsigned bit) {
    if (S.status) atomicOr(S.status, (unsigned long long)bit);
}
#ifdef SBR_CHECKED
#define SBR_CHECKED_ON 1
#else
#define SBR_CHECKED_ON 0
#endif

// Three-input min / max (one instruction each on sm_100 and later).
__device__ __forceinline__ float max3f(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
__device__ __forceinline__ float min3f(float a, float b, float c) {
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
// Watertight ray/triangle intersection (Woop, Benthin, Wald, JCGT 2013): edge functions in a
// sheared, permuted frame; an exactly-zero edge function is re-evaluated in double so
// that rays through a shared edge or vertex hit at least one of the triangles.
// Returns t, or a negative value on a miss.
__device__ __forceinline__ float tri_watertight(const RayPre &r, float4 A4, float4 B4, float4 C4) {
    float3 A = f3(A4) - r.o, B = f3(B4) - r.o, C = f3(C4) - r.o;
    float Ax = dot(A, r.mx), Ay = dot(A, r.my), Az = dot(A, r.mz);
    float Bx = dot(B, r.mx), By = dot(B, r.my), Bz = dot(B, r.mz);
    float Cx = dot(C, r.mx), Cy = dot(C, r.my), Cz = dot(C, r.mz);
    float U = Cx * By - Cy * Bx;
    float V = Ax * Cy - Ay * Cx;
    float W = Bx * Ay - By * Ax;
    if (min3f(fabsf(U), fabsf(V), fabsf(W)) == 0.0f) {
        U = (float)((double)Cx * (double)By - (double)Cy * (double)Bx);
        V = (float)((double)Ax * (double)Cy - (double)Ay * (double)Cx);
        W = (float)((double)Bx * (double)Ay - (double)By * (double)Ax);
    }
    // outside if the edge functions have mixed signs
    if (min3f(U, V, W) < 0.0f && max3f(U, V, W) > 0.0f) return -1.0f;
    float det = U + V + W;
    if (det == 0.0f) return -1.0f;
    float T = U * Az + V * Bz + W * Cz;   // mz carries the 1 / d_kz scale
    return T / det;
}

// Two FMAs in one packed f32x2 instruction: (a.x * b + c, a.y * b + c).
__device__ __forceinline__ float2 fma2s(float ax, float ay, float b, float c) {
    float2 r;
    asm("{\n\t.reg .b64 pa, pb, pc, pd;\n\t"
        "mov.b64 pa, {%2, %3};\n\t"
        "mov.b64 pb, {%4, %4};\n\t"
        "mov.b64 pc, {%5, %5};\n\t"
        "fma.rn.f32x2 pd, pa, pb, pc;\n\t"
        "mov.b64 {%0, %1}, pd;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(ax), "f"(ay), "f"(b), "f"(c));
    return r;
}

// Pop the next stack entry whose entry distance (sdist, beside the refs in stack) is within
// tcull (the closest-hit range grown by the slab test's tolerance); false once the stack
// holds none.
__device__ __forceinline__ bool pop_near(const int *stack, const float *sdist, int &sp, float tcull, int &node) {
    while (sp > 0) {
        --sp;
        if (sdist[sp] <= tcull) {
            node = stack[sp];
            return true;
        }
    }
    return false;
}

// Closest hit through the 4-wide BVH.  The walk descends inner nodes in an inner loop and
// tests a leaf once it reaches one ("while-while"): a warp then runs the leaf branch only
// when its lanes stand at leaves, not on every step where one lane does.  Per node, slab
// tests of the four child boxes as
// t = plane * (1/d) - o * (1/d), the near / far planes picked by the ray's direction
// signs (so no per-axis min/max), two children per packed FMA and three-input min/max;
// the nearest hit child is visited next and the others are pushed with their entry
// distances; a popped entry whose entry distance already lies beyond the closest hit
// found since its push is dropped unvisited (the box test it would face against the
// shrunk range, so nothing it holds can win).  Closest hit along o + t d over t in (tmin, tmax],
// skipping triangles of face `skip`; ties in t go to the lower face id, then the lower
// triangle index.  Returns the triangle index (BVH order) or -1; t_out, face_out set on a
// hit.  nodes_visited counts 4-wide nodes (four box tests each).
__device__ __forceinline__ int closest_hit4(const SceneDev &S, const RayPre &r, float tmin, float tmax, int skip,
                                            float &t_out, int &face_out, unsigned &nodes_visited,
                                            unsigned &tris_tested) {
    int stack[kStack4];    // node or leaf refs
    float sdist[kStack4];  // their entry distances
    int sp = 0;
    int node = 0;
    float tbest = tmax;
    float tcull = tmax * 1.0000005f;   // entries entering beyond this are dropped at pop
    int best = -1, bface = 0x7fffffff;
    const float oix = r.o.x * r.inv.x, oiy = r.o.y * r.inv.y, oiz = r.o.z * r.inv.z;
    for (;;) {
        bool done = false;
        while (!is_leaf(node)) {
            ++nodes_visited;
            const float4 *nd = S.nodes4 + 8 * (size_t)node;
            float4 nxv = __ldg(nd + r.nx), fxv = __ldg(nd + 1 - r.nx);
            float4 nyv = __ldg(nd + 2 + r.ny), fyv = __ldg(nd + 3 - r.ny);
            float4 nzv = __ldg(nd + 4 + r.nz), fzv = __ldg(nd + 5 - r.nz);
            int4 refs = __ldg(reinterpret_cast<const int4 *>(nd + 6));
            const float2 nx01 = fma2s(nxv.x, nxv.y, r.inv.x, -oix), nx23 = fma2s(nxv.z, nxv.w, r.inv.x, -oix);
            const float2 fx01 = fma2s(fxv.x, fxv.y, r.inv.x, -oix), fx23 = fma2s(fxv.z, fxv.w, r.inv.x, -oix);
            const float2 ny01 = fma2s(nyv.x, nyv.y, r.inv.y, -oiy), ny23 = fma2s(nyv.z, nyv.w, r.inv.y, -oiy);
            const float2 fy01 = fma2s(fyv.x, fyv.y, r.inv.y, -oiy), fy23 = fma2s(fyv.z, fyv.w, r.inv.y, -oiy);
            const float2 nz01 = fma2s(nzv.x, nzv.y, r.inv.z, -oiz), nz23 = fma2s(nzv.z, nzv.w, r.inv.z, -oiz);
            const float2 fz01 = fma2s(fzv.x, fzv.y, r.inv.z, -oiz), fz23 = fma2s(fzv.z, fzv.w, r.inv.z, -oiz);
            const float tnx[4] = {nx01.x, nx01.y, nx23.x, nx23.y}, tfx[4] = {fx01.x, fx01.y, fx23.x, fx23.y};
            const float tny[4] = {ny01.x, ny01.y, ny23.x, ny23.y}, tfy[4] = {fy01.x, fy01.y, fy23.x, fy23.y};
            const float tnz[4] = {nz01.x, nz01.y, nz23.x, nz23.y}, tfz[4] = {fz01.x, fz01.y, fz23.x, fz23.y};
            float dist[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                // hit iff tn <= tf (1 + 5e-7): tn, or +inf on a miss, as an FMA, a product
                // with +inf (-inf or NaN on a hit) and a max, keeping the compare and select
                // off the busier ALU pipe
                float tn = max3f(tnx[c], tny[c], fmaxf(tnz[c], tmin));
                float tf = min3f(tfx[c], tfy[c], fminf(tfz[c], tbest));
                dist[c] = fmaxf(tn, fmaf(-tf, 1.0000005f, tn) * INFINITY);
            }
            float d0 = dist[0], d1 = dist[1], d2 = dist[2], d3 = dist[3];
            float dmin = fminf(min3f(d0, d1, d2), d3);
            if (dmin < INFINITY) {
                if (SBR_CHECKED_ON && sp + 3 > S.stack_limit) {   // up to three pushes follow
                    check_fail(S, SBR_CHECK_TRACE_STACK);
                    t_out = tbest;
                    face_out = bface;
                    return -1;
                }
                int pick = d0 == dmin ? 0 : (d1 == dmin ? 1 : (d2 == dmin ? 2 : 3));
                if (d3 < INFINITY && pick != 3) { stack[sp] = refs.w; sdist[sp++] = d3; }
                if (d2 < INFINITY && pick != 2) { stack[sp] = refs.z; sdist[sp++] = d2; }
                if (d1 < INFINITY && pick != 1) { stack[sp] = refs.y; sdist[sp++] = d1; }
                if (d0 < INFINITY && pick != 0) { stack[sp] = refs.x; sdist[sp++] = d0; }
                node = pick == 0 ? refs.x : (pick == 1 ? refs.y : (pick == 2 ? refs.z : refs.w));
                continue;
            }
            if (!pop_near(stack, sdist, sp, tcull, node)) {
                done = true;
                break;
            }
        }
        if (done) break;
        {
            int first = leaf_first(node), cnt = leaf_count(node);
            for (int i = first; i < first + cnt; ++i) {
                const float4 *t = S.tris + 3 * (size_t)i;
                float4 a = __ldg(t), b = __ldg(t + 1), c = __ldg(t + 2);
                int f = __float_as_int(a.w);
                if (f == skip) continue;
                ++tris_tested;
                float th = tri_watertight(r, a, b, c);
                if (!(th > tmin) || th > tbest) continue;
                if (th < tbest || f < bface || (f == bface && i < best)) {
                    tbest = th;
                    best = i;
                    bface = f;
                }
            }
            tcull = tbest * 1.0000005f;
        }
        if (!pop_near(stack, sdist, sp, tcull, node)) break;
    }
    t_out = tbest;
    face_out = bface;
    return best;
}

// Any hit of the segment o + t d, t in (tmin, tmax), ignoring faces fa and fb, over the
// 4-wide BVH; inner nodes and leaves in nested loops as in closest_hit4.
__device__ __forceinline__ bool any_hit4(const SceneDev &S, const RayPre &r, float tmin, float tmax, int fa, int fb) {
    int stack[kStack4];
    int sp = 0;
    int node = 0;
    const float oix = r.o.x * r.inv.x, oiy = r.o.y * r.inv.y, oiz = r.o.z * r.inv.z;
    for (;;) {
        bool done = false;
        while (!is_leaf(node)) {
            const float4 *nd = S.nodes4 + 8 * (size_t)node;
            float4 nxv = __ldg(nd + r.nx), fxv = __ldg(nd + 1 - r.nx);
            float4 nyv = __ldg(nd + 2 + r.ny), fyv = __ldg(nd + 3 - r.ny);
            float4 nzv = __ldg(nd + 4 + r.nz), fzv = __ldg(nd + 5 - r.nz);
            int4 refs = __ldg(reinterpret_cast<const int4 *>(nd + 6));
            const float2 nx01 = fma2s(nxv.x, nxv.y, r.inv.x, -oix), nx23 = fma2s(nxv.z, nxv.w, r.inv.x, -oix);
            const float2 fx01 = fma2s(fxv.x, fxv.y, r.inv.x, -oix), fx23 = fma2s(fxv.z, fxv.w, r.inv.x, -oix);
            const float2 ny01 = fma2s(nyv.x, nyv.y, r.inv.y, -oiy), ny23 = fma2s(nyv.z, nyv.w, r.inv.y, -oiy);
            const float2 fy01 = fma2s(fyv.x, fyv.y, r.inv.y, -oiy), fy23 = fma2s(fyv.z, fyv.w, r.inv.y, -oiy);
            const float2 nz01 = fma2s(nzv.x, nzv.y, r.inv.z, -oiz), nz23 = fma2s(nzv.z, nzv.w, r.inv.z, -oiz);
            const float2 fz01 = fma2s(fzv.x, fzv.y, r.inv.z, -oiz), fz23 = fma2s(fzv.z, fzv.w, r.inv.z, -oiz);
            const float tnx[4] = {nx01.x, nx01.y, nx23.x, nx23.y}, tfx[4] = {fx01.x, fx01.y, fx23.x, fx23.y};
            const float tny[4] = {ny01.x, ny01.y, ny23.x, ny23.y}, tfy[4] = {fy01.x, fy01.y, fy23.x, fy23.y};
            const float tnz[4] = {nz01.x, nz01.y, nz23.x, nz23.y}, tfz[4] = {fz01.x, fz01.y, fz23.x, fz23.y};
            const int rf[4] = {refs.x, refs.y, refs.z, refs.w};
            int next = 0x7fffffff;
            if (SBR_CHECKED_ON && sp + 3 > S.stack_limit) {   // up to three pushes follow
                check_fail(S, SBR_CHECK_OCCLUSION_STACK);
                return false;
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float tn = max3f(tnx[c], tny[c], fmaxf(tnz[c], tmin));
                float tf = min3f(tfx[c], tfy[c], fminf(tfz[c], tmax)) * 1.0000005f;
                if (tn <= tf) {
                    if (next == 0x7fffffff) next = rf[c];
                    else stack[sp++] = rf[c];
                }
            }
            if (next != 0x7fffffff) {
                node = next;
                continue;
            }
            if (sp == 0) {
                done = true;
                break;
            }
            node = stack[--sp];
        }
        if (done) break;
        {
            int first = leaf_first(node), cnt = leaf_count(node);
            for (int i = first; i < first + cnt; ++i) {
                const float4 *t = S.tris + 3 * (size_t)i;
                float4 a = __ldg(t), b = __ldg(t + 1), c = __ldg(t + 2);
                int f = __float_as_int(a.w);
                if (f == fa || f == fb) continue;
                float th = tri_watertight(r, a, b, c);
                if (th > tmin && th < tmax) return true;
            }
        }
        if (sp == 0) break;
        node = stack[--sp];
    }
    return false;
}

// Largest foot parameter s = (p - o).d of any point p of box [lo, hi].
__device__ __forceinline__ float max_foot(const RxDev &R, float3 o, float3 d) {
    float s = (d.x > 0 ? R.hi[0] : R.lo[0]) * d.x + (d.y > 0 ? R.hi[1] : R.lo[1]) * d.y +
              (d.z > 0 ? R.hi[2] : R.lo[2]) * d.z;
    return s - dot(o, d);
}

}  // namespace sbr
