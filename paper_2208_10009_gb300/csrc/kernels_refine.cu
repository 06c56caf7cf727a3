// kernels_refine.cu -- a6 the iterative precise algorithm (§III.B, Fig. 5, Eq. 10), a7 the
// validity test (§III.A, second path test), a8 the channel outputs (§IV), and a9 the
// batched persistent form that refines all (Tx, Rx) pairs' paths from one device work
// queue.
//
// Per path: the cone is centred on the rough launch direction c with half-angle
// R = max(theta_launch, rough error angle), which always contains the exact direction
// (the rough error angle IS the angle to it).  Each iteration sends K sub-rays through
// the sub-cone centres d_k = cos(rho_k R) c + sin(rho_k R)(cos phi_k u + sin phi_k v),
// traces each through the path's fixed face planes, evaluates Eq. 3 at Rx, keeps the
// smallest (lowest k on ties) and shrinks R by the pattern's factor.  Iterations run in
// FP32 while R >= fp64_below and in FP64 after that.
#include "sbr_device.cuh"

namespace sbr {

struct SubTab {
    int off[17];                 // first entry of pattern K (K = 6, 7, 9, 16)
    float rho[38], cphi[38], sphi[38];
    double rho_d[38], cphi_d[38], sphi_d[38];
    double shrink[17];
};
__constant__ SubTab c_sub;

cudaError_t upload_subray_table(cudaStream_t s) {
    SubTab t;
    memset(&t, 0, sizeof(t));
    int at = 0;
    const int Ks[4] = {6, 7, 9, 16};
    for (int q = 0; q < 4; ++q) {
        double rho[16], phi[16], sh;
        int K = subray_pattern(Ks[q], rho, phi, &sh);
        t.off[Ks[q]] = at;
        t.shrink[Ks[q]] = sh;
        for (int k = 0; k < K; ++k, ++at) {
            t.rho[at] = (float)rho[k];
            t.cphi[at] = (float)cos(phi[k]);
            t.sphi[at] = (float)sin(phi[k]);
            t.rho_d[at] = rho[k];
            t.cphi_d[at] = cos(phi[k]);
            t.sphi_d[at] = sin(phi[k]);
        }
    }
    return cudaMemcpyToSymbolAsync(c_sub, &t, sizeof(t), 0, cudaMemcpyHostToDevice, s);
}

struct PathGeo {
    float3 tx, rx;
    dvec3 txd, rxd;
    int k;
    int faces[kMaxOrder];
};

// Records can come from sbr_paths_import, so every id is checked before it is used.
__device__ __forceinline__ bool path_ids_ok(const RefineArgs &A, const sbr_path_record &p) {
    if (p.tx < 0 || p.tx >= A.ntx || p.rx < 0 || p.rx >= A.nrx || p.order < 0 || p.order > kMaxOrder) return false;
    for (int j = 0; j < p.order; ++j)
        if (p.faces[j] < 0 || p.faces[j] >= A.nf) return false;
    return true;
}

__device__ __forceinline__ void load_path(const RefineArgs &A, const sbr_path_record &p, PathGeo &g) {
    float4 t = __ldg(A.tx + p.tx), r = __ldg(A.rx + p.rx);
    g.tx = f3(t);
    g.rx = f3(r);
    g.txd = dv(t.x, t.y, t.z);
    g.rxd = dv(r.x, r.y, r.z);
    g.k = p.order;
#pragma unroll
    for (int j = 0; j < kMaxOrder; ++j) g.faces[j] = p.faces[j];
}

// Eq. 3 error angle at Rx of direction d traced from Tx through the fixed face planes;
// +inf if a segment length is not positive or the foot distance is not positive.
__device__ __forceinline__ float eval32(const SceneDev &S, const PathGeo &g, float3 d) {
    float3 o = g.tx;
    float L = 0.0f;
#pragma unroll
    for (int j = 0; j < kMaxOrder; ++j) {
        if (j >= g.k) break;
        float4 pl = __ldg(S.planes + g.faces[j]);
        float3 n = f3(pl);
        float den = dot(n, d);
        if (den == 0.0f) return INFINITY;
        float t = (pl.w - dot(n, o)) / den;
        if (!(t > 0.0f)) return INFINITY;
        o = o + d * t;
        L += t;
        d = d - n * (2.0f * dot(d, n));
    }
    float3 w = g.rx - o;
    float s = dot(w, d);
    float3 q = w - d * s;
    float dray = L + s;
    if (!(dray > 0.0f)) return INFINITY;
    return atan2f(sqrtf(dot(q, q)), dray);
}

__device__ __forceinline__ double eval64(const SceneDev &S, const PathGeo &g, dvec3 d) {
    dvec3 o = g.txd;
    double L = 0.0;
#pragma unroll
    for (int j = 0; j < kMaxOrder; ++j) {
        if (j >= g.k) break;
        Plane64 pl = S.planes_d[g.faces[j]];
        dvec3 n = dv(pl.x, pl.y, pl.z);
        double den = ddot(n, d);
        if (den == 0.0) return INFINITY;
        double t = (pl.w - ddot(n, o)) / den;
        if (!(t > 0.0)) return INFINITY;
        o = o + d * t;
        L += t;
        d = d - n * (2.0 * ddot(d, n));
    }
    dvec3 w = g.rxd - o;
    double s = ddot(w, d);
    dvec3 q = w - d * s;
    double dray = L + s;
    if (!(dray > 0.0)) return INFINITY;
    return atan2(dnorm(q), dray);
}

// sub-cone frame: u = normalize(c x e), e the world axis with the smallest |c_i| (lowest
// index on ties), v = c x u
__device__ __forceinline__ void frame32(float3 c, float3 &u, float3 &v) {
    float ax = fabsf(c.x), ay = fabsf(c.y), az = fabsf(c.z);
    float3 e = make_float3(1, 0, 0);
    if (ay < ax && ay <= az) e = make_float3(0, 1, 0);
    else if (az < ax && az < ay) e = make_float3(0, 0, 1);
    u = cross(c, e);
    u = u * (1.0f / sqrtf(dot(u, u)));
    v = cross(c, u);
}

__device__ __forceinline__ void frame64(dvec3 c, dvec3 &u, dvec3 &v) {
    double ax = fabs(c.x), ay = fabs(c.y), az = fabs(c.z);
    dvec3 e = dv(1, 0, 0);
    if (ay < ax && ay <= az) e = dv(0, 1, 0);
    else if (az < ax && az < ay) e = dv(0, 0, 1);
    u = dcross(c, e);
    u = u * (1.0 / dnorm(u));
    v = dcross(c, u);
}

// One iteration: returns the chosen sub-ray (or -1 if all are invalid); updates c, err.
__device__ __forceinline__ int iterate32(const SceneDev &S, const PathGeo &g, int K, int off, double R, dvec3 &c,
                                         double &err) {
    float3 cf = make_float3((float)c.x, (float)c.y, (float)c.z);
    float3 u, v;
    frame32(cf, u, v);
    float best = INFINITY;
    int bk = -1;
    float3 bd = cf;
    const float Rf = (float)R;
    for (int k = 0; k < K; ++k) {
        float sa, ca;
        sincosf(c_sub.rho[off + k] * Rf, &sa, &ca);
        float3 dk = cf * ca + (u * c_sub.cphi[off + k] + v * c_sub.sphi[off + k]) * sa;
        float e = eval32(S, g, dk);
        if (e < best) {
            best = e;
            bk = k;
            bd = dk;
        }
    }
    if (bk >= 0) {
        float inv = 1.0f / sqrtf(dot(bd, bd));
        c = dv(bd.x * inv, bd.y * inv, bd.z * inv);
        err = best;
    }
    return bk;
}

__device__ __forceinline__ int iterate64(const SceneDev &S, const PathGeo &g, int K, int off, double R, dvec3 &c,
                                         double &err) {
    dvec3 u, v;
    frame64(c, u, v);
    double best = INFINITY;
    int bk = -1;
    dvec3 bd = c;
    for (int k = 0; k < K; ++k) {
        double sa, ca;
        sincos(c_sub.rho_d[off + k] * R, &sa, &ca);
        dvec3 dk = c * ca + (u * c_sub.cphi_d[off + k] + v * c_sub.sphi_d[off + k]) * sa;
        double e = eval64(S, g, dk);
        if (e < best) {
            best = e;
            bk = k;
            bd = dk;
        }
    }
    if (bk >= 0) {
        c = bd * (1.0 / dnorm(bd));
        err = best;
    }
    return bk;
}

// ----------------------------------------------------------------------------- a7/a8
__device__ __forceinline__ bool point_in_face(const SceneDev &S, int f, dvec3 p) {
    Plane64 pl = S.planes_d[f];
    dvec3 n = dv(pl.x, pl.y, pl.z);
    const float px = (float)p.x, py = (float)p.y, pz = (float)p.z;
    const float tol = 1e-6f * (fabsf(px) + fabsf(py) + fabsf(pz)) + 1e-6f;
    int stack[kStackDepth];
    int sp = 0;
    int node = 0;
    for (;;) {
        if (!is_leaf(node)) {
            const float4 *nd = S.nodes + 4 * (size_t)node;
            float4 a = __ldg(nd), b = __ldg(nd + 1), c = __ldg(nd + 2);
            int4 refs = __ldg(reinterpret_cast<const int4 *>(nd + 3));
            bool in0 = px >= a.x - tol && py >= a.y - tol && pz >= a.z - tol && px <= a.w + tol && py <= b.x + tol &&
                       pz <= b.y + tol;
            bool in1 = px >= b.z - tol && py >= b.w - tol && pz >= c.x - tol && px <= c.y + tol && py <= c.z + tol &&
                       pz <= c.w + tol;
            if (in0 && in1) {
                stack[sp++] = refs.y;
                node = refs.x;
                continue;
            } else if (in0) {
                node = refs.x;
                continue;
            } else if (in1) {
                node = refs.y;
                continue;
            }
        } else {
            int first = leaf_first(node), cnt = leaf_count(node);
            for (int i = first; i < first + cnt; ++i) {
                const float4 *t = S.tris + 3 * (size_t)i;
                float4 A = __ldg(t), B = __ldg(t + 1), C = __ldg(t + 2);
                if (__float_as_int(A.w) != f) continue;
                dvec3 a = dv(A.x, A.y, A.z), b = dv(B.x, B.y, B.z), c = dv(C.x, C.y, C.z);
                double ea = ddot(dcross(b - a, p - a), n);
                double eb = ddot(dcross(c - b, p - b), n);
                double ec = ddot(dcross(a - c, p - c), n);
                if ((ea >= 0 && eb >= 0 && ec >= 0) || (ea <= 0 && eb <= 0 && ec <= 0)) return true;
            }
        }
        if (sp == 0) break;
        node = stack[--sp];
    }
    return false;
}

__device__ __forceinline__ double fresnel_perp_abs(double ci, double eps) {
    if (eps <= 0.0) return 1.0;
    double r = sqrt(eps - (1.0 - ci * ci));
    return fabs((ci - r) / (ci + r));
}

__device__ __forceinline__ void az_el(dvec3 v, float *out) {
    out[0] = (float)atan2(v.y, v.x);
    out[1] = (float)atan2(v.z, sqrt(v.x * v.x + v.y * v.y));
}

// Upper bound on the final error angle of a refined path whose exact direction lies in
// its cone: twice the Eq. 10 bound R0 * s^iters (R_final) plus the FP32 evaluation floor.
// A redundant path received through the cone's width for a face sequence without a
// specular solution stalls far above it and is rejected by the validity test.
__device__ __forceinline__ double converged_bound(int iters, double R_final) {
    return iters > 0 ? 2.0 * R_final + 1e-7 : INFINITY;
}

// Validity test and outputs for launch direction c; writes the result fields of p.
__device__ void finalize_path(const RefineArgs &A, const PathGeo &g, dvec3 c, sbr_path_record &p, double err_bound) {
    const SceneDev &S = A.scene;
    dvec3 pts[kMaxOrder];
    dvec3 o = g.txd, d = c;
    bool ok = true;
    double gain_db = 0.0;
#pragma unroll
    for (int j = 0; j < kMaxOrder; ++j) {
        if (j >= g.k) break;
        Plane64 pl = S.planes_d[g.faces[j]];
        dvec3 n = dv(pl.x, pl.y, pl.z);
        double den = ddot(n, d);
        double t = den != 0.0 ? (pl.w - ddot(n, o)) / den : -1.0;
        if (!(t > 0.0)) {
            ok = false;
            break;
        }
        o = o + d * t;
        pts[j] = o;
        gain_db += 20.0 * log10(fresnel_perp_abs(fabs(den), (double)__ldg(S.face_eps + g.faces[j])));
        d = d - n * (2.0 * den);
    }
    if (!ok) {
        p.valid = 0;
        p.flags |= SBR_PATH_TRACE_FAIL;
        p.delay = 0.0;
        return;
    }
    // Rx must be received on the last leg (its foot lies ahead of the last bounce point)
    // and the refinement must have converged
    bool valid = ddot(g.rxd - o, d) > 0.0 && p.err <= err_bound;
    for (int j = 0; j < g.k && valid; ++j) valid = point_in_face(S, g.faces[j], pts[j]);
    double len = 0.0;
    for (int j = 0; j <= g.k; ++j) {
        dvec3 from = j == 0 ? g.txd : pts[j - 1];
        dvec3 to = j == g.k ? g.rxd : pts[j];
        dvec3 seg = to - from;
        len += dnorm(seg);
        if (valid) {
            int fa = j == 0 ? -1 : g.faces[j - 1];
            int fb = j == g.k ? -1 : g.faces[j];
            RayPre r = make_ray(make_float3((float)from.x, (float)from.y, (float)from.z),
                                make_float3((float)seg.x, (float)seg.y, (float)seg.z));
            if (any_hit(S, r, 1e-6f, 1.0f - 1e-6f, fa, fb)) valid = false;
        }
    }
    p.valid = valid ? 1 : 0;
    p.delay = len / kC0;
    az_el(c, p.aod);
    az_el((g.k > 0 ? pts[g.k - 1] : g.txd) - g.rxd, p.aoa);
    double lam = kC0 / A.freq;
    p.power_dbm = (float)(A.ptx_dbm + 20.0 * log10(lam / (4.0 * 3.14159265358979323846 * len)) + gain_db);
}

__device__ __forceinline__ void store_result(sbr_path_record *dst, const sbr_path_record &p) {
    // result fields only (bytes 56..128)
    dst->iters = p.iters;
    dst->valid = p.valid;
    dst->dir[0] = p.dir[0];
    dst->dir[1] = p.dir[1];
    dst->dir[2] = p.dir[2];
    dst->err = p.err;
    dst->delay = p.delay;
    dst->aod[0] = p.aod[0];
    dst->aod[1] = p.aod[1];
    dst->aoa[0] = p.aoa[0];
    dst->aoa[1] = p.aoa[1];
    dst->power_dbm = p.power_dbm;
    dst->flags = p.flags;
}

__device__ __forceinline__ long long path_count(const RefineArgs &A) {
    long long n = A.counters[kPaths];
    return n < A.path_cap ? n : A.path_cap;
}

// a6-a8, one thread per path (static grid-stride schedule).
__global__ void __launch_bounds__(256) refine_kernel(RefineArgs A) {
    const long long total = A.range ? (long long)(A.range[1] - A.range[0]) : path_count(A);
    const int off = c_sub.off[A.K];
    const double shrink = c_sub.shrink[A.K];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        long long pi = A.range ? (long long)A.index[A.range[0] + i] : i;
        sbr_path_record p = A.paths[pi];
        if (!path_ids_ok(A, p)) {
            A.paths[pi].valid = 0;
            A.paths[pi].flags = SBR_PATH_TRACE_FAIL;
            continue;
        }
        PathGeo g;
        load_path(A, p, g);
        dvec3 c = dv(p.dir[0], p.dir[1], p.dir[2]);
        double R = fmax((double)A.theta_launch, (double)p.rough_err);
        double err = R < A.fp64_below ? eval64(A.scene, g, c)
                                      : (double)eval32(A.scene, g, make_float3((float)c.x, (float)c.y, (float)c.z));
        int it = 0, flags = 0;
        while (it < A.max_iters && !(A.target > 0.0 && err <= A.target)) {
            int bk;
            if (R < A.fp64_below) {
                bk = iterate64(A.scene, g, A.K, off, R, c, err);
                flags |= SBR_PATH_FP64;
            } else {
                bk = iterate32(A.scene, g, A.K, off, R, c, err);
            }
            if (bk < 0) {
                flags |= SBR_PATH_TRACE_FAIL;
                break;
            }
            if (A.choice_log) A.choice_log[pi * A.max_iters + it] = (int8_t)bk;
            R *= shrink;
            ++it;
        }
        p.iters = it;
        p.flags = flags | (it > 0 ? SBR_PATH_REFINED : 0);
        p.dir[0] = c.x;
        p.dir[1] = c.y;
        p.dir[2] = c.z;
        p.err = err;
        finalize_path(A, g, c, p, converged_bound(it, R));
        store_result(A.paths + pi, p);
    }
}

// a9: persistent work-queue form.  A group of G lanes (G = 8, 16 or 32) owns one path at a
// time: lane l evaluates the sub-rays k = l, l + G, ... of each iteration and the group
// takes the argmin with shuffles (lowest k on ties, as in the plain form); the validity
// queries of the path (one point-in-face per bounce, one occlusion test per segment) are
// spread over the lanes the same way.  When a path is finished (iteration cap, target
// reached, or all sub-rays invalid) the group takes the next path index from the device
// queue head with one atomic, so paths that stop early free their group at once.
template <int G>
__device__ __forceinline__ void group_argmin(float &e, int &k, unsigned gmask) {
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) {
        float e2 = __shfl_xor_sync(gmask, e, off, G);
        int k2 = __shfl_xor_sync(gmask, k, off, G);
        if (e2 < e || (e2 == e && k2 < k)) {
            e = e2;
            k = k2;
        }
    }
}

template <int G>
__device__ __forceinline__ void group_argmin64(double &e, int &k, unsigned gmask) {
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) {
        double e2 = __shfl_xor_sync(gmask, e, off, G);
        int k2 = __shfl_xor_sync(gmask, k, off, G);
        if (e2 < e || (e2 == e && k2 < k)) {
            e = e2;
            k = k2;
        }
    }
}

template <int G>
__device__ __forceinline__ int group_iterate32(const SceneDev &S, const PathGeo &g, int K, int off, double R,
                                               dvec3 &c, double &err, int gl, unsigned gmask) {
    float3 cf = make_float3((float)c.x, (float)c.y, (float)c.z);
    float3 u, v;
    frame32(cf, u, v);
    float best = INFINITY;
    int bk = 0x7fffffff;
    const float Rf = (float)R;
    for (int k = gl; k < K; k += G) {
        float sa, ca;
        sincosf(c_sub.rho[off + k] * Rf, &sa, &ca);
        float3 dk = cf * ca + (u * c_sub.cphi[off + k] + v * c_sub.sphi[off + k]) * sa;
        float e = eval32(S, g, dk);
        if (e < best) {
            best = e;
            bk = k;
        }
    }
    group_argmin<G>(best, bk, gmask);
    if (!(best < INFINITY)) return -1;
    // every lane rebuilds the winning direction (same arithmetic as the lane that found it)
    float sa, ca;
    sincosf(c_sub.rho[off + bk] * Rf, &sa, &ca);
    float3 bd = cf * ca + (u * c_sub.cphi[off + bk] + v * c_sub.sphi[off + bk]) * sa;
    float inv = 1.0f / sqrtf(dot(bd, bd));
    c = dv(bd.x * inv, bd.y * inv, bd.z * inv);
    err = best;
    return bk;
}

template <int G>
__device__ __forceinline__ int group_iterate64(const SceneDev &S, const PathGeo &g, int K, int off, double R,
                                               dvec3 &c, double &err, int gl, unsigned gmask) {
    dvec3 u, v;
    frame64(c, u, v);
    double best = INFINITY;
    int bk = 0x7fffffff;
    for (int k = gl; k < K; k += G) {
        double sa, ca;
        sincos(c_sub.rho_d[off + k] * R, &sa, &ca);
        dvec3 dk = c * ca + (u * c_sub.cphi_d[off + k] + v * c_sub.sphi_d[off + k]) * sa;
        double e = eval64(S, g, dk);
        if (e < best) {
            best = e;
            bk = k;
        }
    }
    group_argmin64<G>(best, bk, gmask);
    if (!(best < INFINITY)) return -1;
    double sa, ca;
    sincos(c_sub.rho_d[off + bk] * R, &sa, &ca);
    dvec3 bd = c * ca + (u * c_sub.cphi_d[off + bk] + v * c_sub.sphi_d[off + bk]) * sa;
    c = bd * (1.0 / dnorm(bd));
    err = best;
    return bk;
}

// Validity and outputs with the per-bounce / per-segment queries spread over the group.
template <int G>
__device__ void group_finalize(const RefineArgs &A, const PathGeo &g, dvec3 c, sbr_path_record &p, int gl,
                               unsigned gmask, double err_bound) {
    const SceneDev &S = A.scene;
    dvec3 pts[kMaxOrder];
    dvec3 o = g.txd, d = c;
    bool ok = true;
    double gain_db = 0.0;
#pragma unroll
    for (int j = 0; j < kMaxOrder; ++j) {
        if (j >= g.k) break;
        Plane64 pl = S.planes_d[g.faces[j]];
        dvec3 n = dv(pl.x, pl.y, pl.z);
        double den = ddot(n, d);
        double t = den != 0.0 ? (pl.w - ddot(n, o)) / den : -1.0;
        if (!(t > 0.0)) {
            ok = false;
            break;
        }
        o = o + d * t;
        pts[j] = o;
        gain_db += 20.0 * log10(fresnel_perp_abs(fabs(den), (double)__ldg(S.face_eps + g.faces[j])));
        d = d - n * (2.0 * den);
    }
    if (!ok) {
        p.valid = 0;
        p.flags |= SBR_PATH_TRACE_FAIL;
        p.delay = 0.0;
        return;
    }
    // Rx must be received on the last leg (its foot lies ahead of the last bounce point)
    // and the refinement must have converged
    bool mine_ok = ddot(g.rxd - o, d) > 0.0 && p.err <= err_bound;
    for (int j = gl; j < g.k && mine_ok; j += G) mine_ok = point_in_face(S, g.faces[j], pts[j]);
    bool valid = __all_sync(gmask, mine_ok);
    mine_ok = true;
    if (valid) {
        for (int j = gl; j <= g.k && mine_ok; j += G) {
            dvec3 from = j == 0 ? g.txd : pts[j - 1];
            dvec3 to = j == g.k ? g.rxd : pts[j];
            dvec3 seg = to - from;
            int fa = j == 0 ? -1 : g.faces[j - 1];
            int fb = j == g.k ? -1 : g.faces[j];
            RayPre r = make_ray(make_float3((float)from.x, (float)from.y, (float)from.z),
                                make_float3((float)seg.x, (float)seg.y, (float)seg.z));
            if (any_hit(S, r, 1e-6f, 1.0f - 1e-6f, fa, fb)) mine_ok = false;
        }
        valid = __all_sync(gmask, mine_ok);
    }
    double len = 0.0;
    for (int j = 0; j <= g.k; ++j) {
        dvec3 from = j == 0 ? g.txd : pts[j - 1];
        dvec3 to = j == g.k ? g.rxd : pts[j];
        len += dnorm(to - from);
    }
    p.valid = valid ? 1 : 0;
    p.delay = len / kC0;
    az_el(c, p.aod);
    az_el((g.k > 0 ? pts[g.k - 1] : g.txd) - g.rxd, p.aoa);
    double lam = kC0 / A.freq;
    p.power_dbm = (float)(A.ptx_dbm + 20.0 * log10(lam / (4.0 * 3.14159265358979323846 * len)) + gain_db);
}

template <int G>
__global__ void __launch_bounds__(256) batch_refine_kernel(RefineArgs A) {
    const long long total = path_count(A);
    const int off = c_sub.off[A.K];
    const double shrink = c_sub.shrink[A.K];
    const int lane = threadIdx.x & 31;
    const int gl = lane % G;
    const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane - gl));
    for (;;) {
        unsigned long long q = 0;
        if (gl == 0) q = atomicAdd(reinterpret_cast<unsigned long long *>(A.counters + kBatchHead), 1ULL);
        q = __shfl_sync(gmask, q, 0, G);
        if ((long long)q >= total) break;
        const long long pi = (long long)q;
        sbr_path_record p = A.paths[pi];
        if (!path_ids_ok(A, p)) {
            if (gl == 0) {
                A.paths[pi].valid = 0;
                A.paths[pi].flags = SBR_PATH_TRACE_FAIL;
            }
            continue;
        }
        PathGeo g;
        load_path(A, p, g);
        dvec3 c = dv(p.dir[0], p.dir[1], p.dir[2]);
        double R = fmax((double)A.theta_launch, (double)p.rough_err);
        double err = R < A.fp64_below ? eval64(A.scene, g, c)
                                      : (double)eval32(A.scene, g, make_float3((float)c.x, (float)c.y, (float)c.z));
        int it = 0, flags = 0;
        while (it < A.max_iters && !(A.target > 0.0 && err <= A.target)) {
            int bk;
            if (R < A.fp64_below) {
                bk = group_iterate64<G>(A.scene, g, A.K, off, R, c, err, gl, gmask);
                flags |= SBR_PATH_FP64;
            } else {
                bk = group_iterate32<G>(A.scene, g, A.K, off, R, c, err, gl, gmask);
            }
            if (bk < 0) {
                flags |= SBR_PATH_TRACE_FAIL;
                break;
            }
            if (A.choice_log && gl == 0) A.choice_log[pi * A.max_iters + it] = (int8_t)bk;
            R *= shrink;
            ++it;
        }
        p.iters = it;
        p.flags = flags | (it > 0 ? SBR_PATH_REFINED : 0);
        p.dir[0] = c.x;
        p.dir[1] = c.y;
        p.dir[2] = c.z;
        p.err = err;
        group_finalize<G>(A, g, c, p, gl, gmask, converged_bound(it, R));
        if (gl == 0) store_result(A.paths + pi, p);
    }
}

static const void *batch_fn(int lanes) {
    switch (lanes) {
        case 8: return (const void *)batch_refine_kernel<8>;
        case 32: return (const void *)batch_refine_kernel<32>;
        default: return (const void *)batch_refine_kernel<16>;
    }
}

void refine_kernel_attrs(int *regs, int block, int *blocks_per_sm, bool batched, int lanes) {
    const void *fn = batched ? batch_fn(lanes) : (const void *)refine_kernel;
    cudaFuncAttributes at;
    cudaFuncGetAttributes(&at, fn);
    if (regs) *regs = at.numRegs;
    if (blocks_per_sm) {
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, block, 0);
        *blocks_per_sm = nb > 0 ? nb : 1;
    }
}

cudaError_t launch_refine(const RefineArgs &a, int grid, int block, cudaStream_t s) {
    refine_kernel<<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_batch_refine(const RefineArgs &a, int grid, int block, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(a.counters + kBatchHead, 0, sizeof(long long), s);
    if (e != cudaSuccess) return e;
    switch (a.chunk) {
        case 8: batch_refine_kernel<8><<<grid, block, 0, s>>>(a); break;
        case 32: batch_refine_kernel<32><<<grid, block, 0, s>>>(a); break;
        default: batch_refine_kernel<16><<<grid, block, 0, s>>>(a); break;
    }
    return cudaGetLastError();
}

}  // namespace sbr
