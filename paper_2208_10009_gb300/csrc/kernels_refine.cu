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

// Validity test and outputs for launch direction c; writes the result fields of p.
__device__ void finalize_path(const RefineArgs &A, const PathGeo &g, dvec3 c, sbr_path_record &p) {
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
    bool valid = true;
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
__global__ void __launch_bounds__(128) refine_kernel(RefineArgs A) {
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
        finalize_path(A, g, c, p);
        store_result(A.paths + pi, p);
    }
}

// a9: persistent work-queue form.  Each lane owns one path at a time and advances it by
// up to `chunk` iterations per step; lanes whose path is finished run its validity test
// and outputs and take new path indices from the queue head (one atomic per warp via
// ballot/popc), so lanes freed by early-stopping paths are refilled at once.
__global__ void __launch_bounds__(128) batch_refine_kernel(RefineArgs A) {
    const long long total = path_count(A);
    const int off = c_sub.off[A.K];
    const double shrink = c_sub.shrink[A.K];
    const unsigned lane = threadIdx.x & 31, lt = (1u << lane) - 1u;
    long long pi = -1;
    bool empty = false;
    sbr_path_record p;
    PathGeo g;
    dvec3 c = dv(0, 0, 0);
    double R = 0, err = 0;
    int it = 0, flags = 0;
    bool done = false;
    for (;;) {
        unsigned need = __ballot_sync(0xffffffffu, pi < 0);
        if (need && !empty) {
            unsigned long long base = 0;
            if (lane == 0)
                base = atomicAdd(reinterpret_cast<unsigned long long *>(A.counters + kBatchHead),
                                 (unsigned long long)__popc(need));
            base = __shfl_sync(0xffffffffu, base, 0);
            if ((long long)base >= total) empty = true;
            if (pi < 0) {
                long long q = (long long)base + __popc(need & lt);
                if (q < total) {
                    pi = q;
                    p = A.paths[pi];
                    if (!path_ids_ok(A, p)) {
                        A.paths[pi].valid = 0;
                        A.paths[pi].flags = SBR_PATH_TRACE_FAIL;
                        pi = -1;
                    }
                }
                if (pi >= 0) {
                    load_path(A, p, g);
                    c = dv(p.dir[0], p.dir[1], p.dir[2]);
                    R = fmax((double)A.theta_launch, (double)p.rough_err);
                    err = R < A.fp64_below ? eval64(A.scene, g, c)
                                           : (double)eval32(A.scene, g, make_float3((float)c.x, (float)c.y, (float)c.z));
                    it = 0;
                    flags = 0;
                    done = false;
                }
            }
        }
        if (__ballot_sync(0xffffffffu, pi >= 0) == 0) break;
        if (pi < 0) continue;
        for (int step = 0; step < A.chunk && !done; ++step) {
            if (!(it < A.max_iters && !(A.target > 0.0 && err <= A.target))) {
                done = true;
                break;
            }
            int bk;
            if (R < A.fp64_below) {
                bk = iterate64(A.scene, g, A.K, off, R, c, err);
                flags |= SBR_PATH_FP64;
            } else {
                bk = iterate32(A.scene, g, A.K, off, R, c, err);
            }
            if (bk < 0) {
                flags |= SBR_PATH_TRACE_FAIL;
                done = true;
                break;
            }
            if (A.choice_log) A.choice_log[pi * A.max_iters + it] = (int8_t)bk;
            R *= shrink;
            ++it;
        }
        if (!done && !(it < A.max_iters && !(A.target > 0.0 && err <= A.target))) done = true;
        if (done) {
            p.iters = it;
            p.flags = flags | (it > 0 ? SBR_PATH_REFINED : 0);
            p.dir[0] = c.x;
            p.dir[1] = c.y;
            p.dir[2] = c.z;
            p.err = err;
            finalize_path(A, g, c, p);
            store_result(A.paths + pi, p);
            pi = -1;
        }
    }
}

void refine_kernel_attrs(int *regs, int block, int *blocks_per_sm, bool batched) {
    cudaFuncAttributes at;
    cudaFuncGetAttributes(&at, batched ? (const void *)batch_refine_kernel : (const void *)refine_kernel);
    if (regs) *regs = at.numRegs;
    if (blocks_per_sm) {
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &nb, batched ? (const void *)batch_refine_kernel : (const void *)refine_kernel, block, 0);
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
    batch_refine_kernel<<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace sbr
