// capi.cu -- the C ABI declared in include/sbr.h: handles, validation, memory, and the
// order in which the kernels of the SBR hot path are enqueued.
#include <algorithm>
#include <cstddef>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "nvtx_ranges.h"
#include "sbr_internal.h"

using namespace sbr;

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

sbr_status fail(sbr_ctx *ctx, sbr_status s, const std::string &msg) {
    if (ctx) ctx->last_error = msg;
    return s;
}

#define SBR_CUDA(call)                                                                                  \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess)                                                                          \
            return fail(ctx, SBR_ECUDA, std::string(#call) + " failed: " + cudaGetErrorString(e_));     \
    } while (0)

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Carves several arrays out of one allocation (256-byte aligned sub-blocks).
struct Carver {
    size_t total = 0;
    std::vector<std::pair<void **, size_t>> parts;
    template <class T>
    void add(T **p, size_t count) {
        parts.push_back({reinterpret_cast<void **>(p), count * sizeof(T)});
        total = align_up(total, 256) + count * sizeof(T);
    }
    void bind(void *base) {
        size_t off = 0;
        for (auto &pr : parts) {
            off = align_up(off, 256);
            *pr.first = static_cast<char *>(base) + off;
            off += pr.second;
        }
    }
};

int64_t rays_for(int n) { return 10LL * n * n + 2; }

int64_t rays_for_launcher(int n, int launcher) {
    if (n < 1) return -1;
    if (launcher == 0 || launcher == 20) return 10LL * n * n + 2;
    if (launcher == 8) return 4LL * n * n + 2;
    return -1;
}

float bits_as_float(int i) {
    float f;
    std::memcpy(&f, &i, sizeof(f));
    return f;
}

sbr_status ensure_lattice(sbr_ctx *ctx, int n) {
    if (ctx->lattice_n == n && ctx->lattice_mem) return SBR_OK;
    std::vector<float4> ico, centre, layers;
    std::vector<int2> edges;
    int nl = 0;
    build_lattice_tables(n, ico, edges, centre, layers, nl);
    float4 *d_ico = nullptr, *d_centre = nullptr, *d_layers = nullptr;
    int2 *d_edges = nullptr;
    Carver cv;
    cv.add(&d_ico, ico.size());
    cv.add(&d_edges, edges.size());
    cv.add(&d_centre, centre.size());
    cv.add(&d_layers, layers.size());
    if (ctx->lattice_bytes < cv.total) {
        dev_free(ctx, ctx->lattice_mem, ctx->lattice_bytes);
        ctx->lattice_mem = dev_alloc(ctx, cv.total);
        ctx->lattice_bytes = ctx->lattice_mem ? cv.total : 0;
        if (!ctx->lattice_mem) return fail(ctx, SBR_ENOMEM, "lattice tables: allocation failed");
    }
    cv.bind(ctx->lattice_mem);
    SBR_CUDA(cudaMemcpyAsync(d_ico, ico.data(), ico.size() * sizeof(float4), cudaMemcpyHostToDevice, ctx->stream));
    SBR_CUDA(cudaMemcpyAsync(d_edges, edges.data(), edges.size() * sizeof(int2), cudaMemcpyHostToDevice, ctx->stream));
    SBR_CUDA(cudaMemcpyAsync(d_centre, centre.data(), centre.size() * sizeof(float4), cudaMemcpyHostToDevice,
                             ctx->stream));
    SBR_CUDA(cudaMemcpyAsync(d_layers, layers.data(), layers.size() * sizeof(float4), cudaMemcpyHostToDevice,
                             ctx->stream));
    SBR_CUDA(cudaStreamSynchronize(ctx->stream));
    ctx->lattice.ico = d_ico;
    ctx->lattice.edges = d_edges;
    ctx->lattice.centre = d_centre;
    ctx->lattice.layers = d_layers;
    ctx->lattice.n = n;
    ctx->lattice.nl = nl;
    ctx->lattice.edge_angle = (float)std::acos(1.0 / std::sqrt(5.0));
    ctx->lattice_n = n;
    ctx->dirs_valid = false;
    return SBR_OK;
}

sbr_status ensure_poly(sbr_ctx *ctx, int poly, int n) {
    if (ctx->poly_kind != poly || !ctx->poly_mem) {
        std::vector<float4> v;
        std::vector<int2> e;
        std::vector<int4> f;
        if (!build_polyhedron(poly, v, e, f)) return fail(ctx, SBR_EINVAL, "equidistant: poly must be 20 or 8");
        float4 *dv;
        int2 *de;
        int4 *df;
        Carver cv;
        cv.add(&dv, v.size());
        cv.add(&de, e.size());
        cv.add(&df, f.size());
        if (ctx->poly_bytes < cv.total) {
            dev_free(ctx, ctx->poly_mem, ctx->poly_bytes);
            ctx->poly_mem = dev_alloc(ctx, cv.total);
            ctx->poly_bytes = ctx->poly_mem ? cv.total : 0;
            if (!ctx->poly_mem) return fail(ctx, SBR_ENOMEM, "equidistant tables: allocation failed");
        }
        cv.bind(ctx->poly_mem);
        SBR_CUDA(cudaMemcpyAsync(dv, v.data(), v.size() * sizeof(float4), cudaMemcpyHostToDevice, ctx->stream));
        SBR_CUDA(cudaMemcpyAsync(de, e.data(), e.size() * sizeof(int2), cudaMemcpyHostToDevice, ctx->stream));
        SBR_CUDA(cudaMemcpyAsync(df, f.data(), f.size() * sizeof(int4), cudaMemcpyHostToDevice, ctx->stream));
        SBR_CUDA(cudaStreamSynchronize(ctx->stream));
        ctx->poly.v = dv;
        ctx->poly.edges = de;
        ctx->poly.faces = df;
        ctx->poly.nv = (int)v.size();
        ctx->poly.ne = (int)e.size();
        ctx->poly.nf = (int)f.size();
        ctx->poly_kind = poly;
    }
    ctx->poly.n = n;
    return SBR_OK;
}

sbr_status ensure_dirs(sbr_ctx *ctx, int n, int launcher) {
    int64_t N = rays_for_launcher(n, launcher);
    if (N < 0) return fail(ctx, SBR_EINVAL, "launcher must be 0 (equiangular), 20 or 8 (equidistant)");
    size_t need = (size_t)N * sizeof(float4);
    if (ctx->dirs_bytes < need) {
        dev_free(ctx, ctx->dirs, ctx->dirs_bytes);
        ctx->dirs = dev_alloc(ctx, need);
        ctx->dirs_bytes = ctx->dirs ? need : 0;
        ctx->dirs_valid = false;
        if (!ctx->dirs) return fail(ctx, SBR_ENOMEM, "ray directions: allocation failed");
    }
    if (launcher == 0) {
        sbr_status st = ensure_lattice(ctx, n);
        if (st != SBR_OK) return st;
        SBR_CUDA(launch_raygen(ctx->lattice, static_cast<float4 *>(ctx->dirs), N, ctx->stream));
    } else {
        sbr_status st = ensure_poly(ctx, launcher, n);
        if (st != SBR_OK) return st;
        SBR_CUDA(launch_raygen_equidistant(ctx->poly, static_cast<float4 *>(ctx->dirs), N, ctx->stream));
    }
    ctx->dirs_n = n;
    ctx->dirs_launcher = launcher;
    ctx->dirs_valid = true;
    return SBR_OK;
}

// copy an n x 3 float array (host or device) into a float4 device array
sbr_status copy_points(sbr_ctx *ctx, float4 *dst, const float *src, int64_t n) {
    if (n == 0) return SBR_OK;
    if (is_device_ptr(src)) {
        SBR_CUDA(cudaMemcpy2DAsync(dst, sizeof(float4), src, 3 * sizeof(float), 3 * sizeof(float), (size_t)n,
                                   cudaMemcpyDeviceToDevice, ctx->stream));
    } else {
        std::vector<float4> tmp((size_t)n);
        for (int64_t i = 0; i < n; ++i) tmp[i] = make_float4(src[3 * i], src[3 * i + 1], src[3 * i + 2], 0.0f);
        SBR_CUDA(cudaMemcpyAsync(dst, tmp.data(), tmp.size() * sizeof(float4), cudaMemcpyHostToDevice, ctx->stream));
        SBR_CUDA(cudaStreamSynchronize(ctx->stream));
    }
    return SBR_OK;
}

}  // namespace

namespace sbr {
void *dev_alloc(sbr_ctx *ctx, size_t bytes) {
    if (bytes == 0) bytes = 256;
    if (ctx->alloc) return ctx->alloc(bytes, (void *)ctx->stream, ctx->user);
    void *p = nullptr;
    if (cudaMallocAsync(&p, bytes, ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}
void dev_free(sbr_ctx *ctx, void *p, size_t bytes) {
    if (!p) return;
    if (ctx->free_fn) ctx->free_fn(p, bytes, (void *)ctx->stream, ctx->user);
    else cudaFreeAsync(p, ctx->stream);
}
}  // namespace sbr

extern "C" {

int32_t sbr_abi_version(void) { return SBR_ABI_VERSION; }

const char *sbr_status_string(sbr_status s) {
    switch (s) {
        case SBR_OK: return "ok";
        case SBR_EINVAL: return "invalid argument";
        case SBR_ENOMEM: return "out of memory";
        case SBR_ECUDA: return "CUDA error";
        case SBR_ETIMEOUT: return "device wait timed out";
        case SBR_EOVERFLOW: return "buffer overflow";
        case SBR_EDEGENERATE: return "degenerate scene";
        case SBR_ECOLLISION: return "dedup hash collision";
    }
    return "unknown status";
}

const char *sbr_last_error(const sbr_ctx *ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

int64_t sbr_num_rays(int32_t n) { return n < 1 ? -1 : rays_for(n); }

int64_t sbr_num_rays_launcher(int32_t n, int32_t launcher) { return rays_for_launcher(n, launcher); }

sbr_status sbr_raygen_equidistant(sbr_ctx *ctx, int32_t n, int32_t poly, float *dirs, int64_t cap) {
    if (!ctx || !dirs) return fail(ctx, SBR_EINVAL, "sbr_raygen_equidistant: null argument");
    if (n < 1 || n > 14000) return fail(ctx, SBR_EINVAL, "sbr_raygen_equidistant: n_div out of range [1, 14000]");
    if (poly != 20 && poly != 8) return fail(ctx, SBR_EINVAL, "sbr_raygen_equidistant: poly must be 20 or 8");
    int64_t N = rays_for_launcher(n, poly);
    if (cap < N) return fail(ctx, SBR_EOVERFLOW, "sbr_raygen_equidistant: buffer smaller than the ray count");
    DeviceGuard g(ctx->device);
    sbr_status st = ensure_poly(ctx, poly, n);
    if (st != SBR_OK) return st;
    SBR_CUDA(launch_raygen_equidistant(ctx->poly, reinterpret_cast<float4 *>(dirs), N, ctx->stream));
    return SBR_OK;
}

double sbr_theta_launch(int32_t n) { return n < 1 ? -1.0 : std::acos(1.0 / std::sqrt(5.0)) / (std::sqrt(3.0) * n); }

sbr_status sbr_subray_pattern(int32_t K, double *rho, double *phi, double *shrink) {
    if (!rho || !phi || !shrink) return SBR_EINVAL;
    return subray_pattern(K, rho, phi, shrink) == K ? SBR_OK : SBR_EINVAL;
}

sbr_status sbr_ctx_create(int device, void *stream, sbr_alloc_fn alloc, sbr_free_fn free_fn, void *user,
                          sbr_ctx **out) {
    if (!out) return SBR_EINVAL;
    *out = nullptr;
    if ((alloc == nullptr) != (free_fn == nullptr)) return SBR_EINVAL;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
        cudaGetLastError();
        return SBR_EINVAL;
    }
    sbr_ctx *ctx = new (std::nothrow) sbr_ctx();
    if (!ctx) return SBR_ENOMEM;
    ctx->device = device;
    ctx->stream = static_cast<cudaStream_t>(stream);
    ctx->alloc = alloc;
    ctx->free_fn = free_fn;
    ctx->user = user;
    DeviceGuard g(device);
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    cudaDeviceGetAttribute(&ctx->max_threads_per_sm, cudaDevAttrMaxThreadsPerMultiProcessor, device);
    cudaError_t e = upload_subray_table(ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        delete ctx;
        return SBR_ECUDA;
    }
    *out = ctx;
    return SBR_OK;
}

sbr_status sbr_ctx_destroy(sbr_ctx *ctx) {
    if (!ctx) return SBR_EINVAL;
    DeviceGuard g(ctx->device);
    dev_free(ctx, ctx->dirs, ctx->dirs_bytes);
    dev_free(ctx, ctx->lattice_mem, ctx->lattice_bytes);
    dev_free(ctx, ctx->poly_mem, ctx->poly_bytes);
    cudaStreamSynchronize(ctx->stream);
    for (auto &e : ctx->ev)
        if (e) cudaEventDestroy(e);
    delete ctx;
    return SBR_OK;
}

sbr_status sbr_ctx_set_stream(sbr_ctx *ctx, void *stream) {
    if (!ctx) return SBR_EINVAL;
    ctx->stream = static_cast<cudaStream_t>(stream);
    return SBR_OK;
}

int32_t sbr_ctx_num_sms(const sbr_ctx *ctx) { return ctx ? ctx->num_sms : 0; }

sbr_status sbr_raygen(sbr_ctx *ctx, int32_t n, float *dirs, int64_t cap) {
    if (!ctx || !dirs) return fail(ctx, SBR_EINVAL, "sbr_raygen: null argument");
    if (n < 1 || n > 14000) return fail(ctx, SBR_EINVAL, "sbr_raygen: n_div out of range [1, 14000]");
    if (cap < rays_for(n)) return fail(ctx, SBR_EOVERFLOW, "sbr_raygen: buffer holds fewer than 10 n^2 + 2 rays");
    DeviceGuard g(ctx->device);
    sbr_status st = ensure_lattice(ctx, n);
    if (st != SBR_OK) return st;
    SBR_CUDA(launch_raygen(ctx->lattice, reinterpret_cast<float4 *>(dirs), rays_for(n), ctx->stream));
    return SBR_OK;
}

// ------------------------------------------------------------------------------ scene
sbr_status sbr_scene_upload(sbr_ctx *ctx, const float *verts, int64_t nv, const int32_t *tris,
                            const int32_t *tri_face, int64_t nt, const float *face_eps, int32_t nf,
                            sbr_scene **out) {
    if (!ctx || !out) return fail(ctx, SBR_EINVAL, "sbr_scene_upload: null argument");
    *out = nullptr;
    if (nv < 0 || nt < 0 || nf < 0 || (nt > 0 && (!verts || !tris || !tri_face)))
        return fail(ctx, SBR_EINVAL, "sbr_scene_upload: bad sizes or null arrays");
    if (nt >= (1LL << 24)) return fail(ctx, SBR_EINVAL, "sbr_scene_upload: more than 2^24 triangles");
    DeviceGuard g(ctx->device);
    // validation
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < 3 * nv; ++i)
        if (!std::isfinite(verts[i])) return fail(ctx, SBR_EDEGENERATE, "scene: non-finite vertex coordinate");
    for (int64_t i = 0; i < nv; ++i)
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::min(lo[a], (double)verts[3 * i + a]);
            hi[a] = std::max(hi[a], (double)verts[3 * i + a]);
        }
    std::vector<Plane64> planes((size_t)std::max(nf, 1), Plane64{0, 0, 0, 0});
    std::vector<char> seen((size_t)std::max(nf, 1), 0);
    std::vector<float> blo(3 * (size_t)nt), bhi(3 * (size_t)nt);
    double diag = nv > 0 ? std::sqrt((hi[0] - lo[0]) * (hi[0] - lo[0]) + (hi[1] - lo[1]) * (hi[1] - lo[1]) +
                                     (hi[2] - lo[2]) * (hi[2] - lo[2]))
                         : 1.0;
    if (!(diag > 0)) diag = 1.0;
    const float pad = (float)(1e-6 * diag);
    for (int64_t t = 0; t < nt; ++t) {
        int ia = tris[3 * t], ib = tris[3 * t + 1], ic = tris[3 * t + 2], f = tri_face[t];
        if (ia < 0 || ib < 0 || ic < 0 || ia >= nv || ib >= nv || ic >= nv)
            return fail(ctx, SBR_EDEGENERATE, "scene: vertex id out of range in triangle " + std::to_string(t));
        if (f < 0 || f >= nf) return fail(ctx, SBR_EDEGENERATE, "scene: face id out of range in triangle " + std::to_string(t));
        const float *A = verts + 3 * ia, *B = verts + 3 * ib, *C = verts + 3 * ic;
        double e1[3] = {(double)B[0] - A[0], (double)B[1] - A[1], (double)B[2] - A[2]};
        double e2[3] = {(double)C[0] - A[0], (double)C[1] - A[1], (double)C[2] - A[2]};
        double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        double len = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        if (!(len > 0.0)) return fail(ctx, SBR_EDEGENERATE, "scene: zero-area triangle " + std::to_string(t));
        if (!seen[f]) {
            seen[f] = 1;
            double u[3] = {n[0] / len, n[1] / len, n[2] / len};
            planes[f] = Plane64{u[0], u[1], u[2], u[0] * A[0] + u[1] * A[1] + u[2] * A[2]};
        }
        for (int a = 0; a < 3; ++a) {
            blo[3 * t + a] = std::min(A[a], std::min(B[a], C[a])) - pad;
            bhi[3 * t + a] = std::max(A[a], std::max(B[a], C[a])) + pad;
        }
    }
    BvhOut bvh;
    std::string err;
    if (!build_bvh(blo, bhi, kLeafMax, bvh, err)) return fail(ctx, SBR_EDEGENERATE, err);
    if (bvh.max_stack4 > kStack4)
        return fail(ctx, SBR_EDEGENERATE, "scene: BVH too deep for the traversal stack (" +
                                              std::to_string(bvh.max_stack4) + " entries)");
    // triangles in BVH order, face CSR
    std::vector<float4> tri4(3 * (size_t)nt);
    std::vector<int> off((size_t)nf + 1, 0), idx((size_t)nt);
    for (int64_t i = 0; i < nt; ++i) {
        int t = bvh.prim_order[i];
        int f = tri_face[t];
        for (int v = 0; v < 3; ++v) {
            const float *P = verts + 3 * tris[3 * t + v];
            tri4[3 * i + v] = make_float4(P[0], P[1], P[2], v == 0 ? bits_as_float(f) : 0.0f);
        }
        ++off[f + 1];
    }
    for (int f = 0; f < nf; ++f) off[f + 1] += off[f];
    {
        std::vector<int> cur(off.begin(), off.end() - 1);
        for (int64_t i = 0; i < nt; ++i) idx[cur[tri_face[bvh.prim_order[i]]]++] = (int)i;
    }
    // wedges (order-1 diffraction) in id order, and a BVH over their segments
    std::vector<WedgeHost> wl;
    build_wedges(verts, nv, tris, tri_face, nt, nf, wl);
    const int nw = (int)wl.size();
    std::vector<float4> w4(4 * (size_t)std::max(nw, 1), make_float4(0, 0, 0, 0));
    std::vector<float> wlo(3 * (size_t)nw), whi(3 * (size_t)nw);
    for (int i = 0; i < nw; ++i) {
        const WedgeHost &w = wl[i];
        w4[4 * i] = make_float4(w.a[0], w.a[1], w.a[2], bits_as_float(w.f1));
        w4[4 * i + 1] = make_float4(w.b[0], w.b[1], w.b[2], bits_as_float(w.f2));
        w4[4 * i + 2] = make_float4((float)w.w1[0], (float)w.w1[1], (float)w.w1[2], 0.0f);
        w4[4 * i + 3] = make_float4((float)w.w2[0], (float)w.w2[1], (float)w.w2[2], 0.0f);
        for (int a = 0; a < 3; ++a) {
            wlo[3 * i + a] = std::min(w.a[a], w.b[a]) - pad;
            whi[3 * i + a] = std::max(w.a[a], w.b[a]) + pad;
        }
    }
    BvhOut wbvh;
    if (nw > 0 && !build_bvh(wlo, whi, 2, wbvh, err)) return fail(ctx, SBR_EDEGENERATE, err);
    if (nw == 0) wbvh.nodes.assign(4, make_float4(0, 0, 0, 0));
    std::vector<int> wids(wbvh.prim_order.begin(), wbvh.prim_order.end());
    if (wids.empty()) wids.push_back(0);
    std::vector<float4> pl4((size_t)std::max(nf, 1));
    std::vector<float> eps((size_t)std::max(nf, 1), 0.0f);
    // the FP64 planes also as float pairs hi + lo (lo = the rounding residual), per face
    // (hi, lo): the compensated-FP32 unfolding of the refinement starts from them
    std::vector<float4> pldf(2 * pl4.size(), make_float4(0, 0, 0, 0));
    auto split = [](double x, float &hi, float &lo) {
        hi = (float)x;
        lo = (float)(x - (double)hi);
    };
    for (int f = 0; f < nf; ++f) {
        pl4[f] = make_float4((float)planes[f].x, (float)planes[f].y, (float)planes[f].z, (float)planes[f].w);
        split(planes[f].x, pldf[2 * f].x, pldf[2 * f + 1].x);
        split(planes[f].y, pldf[2 * f].y, pldf[2 * f + 1].y);
        split(planes[f].z, pldf[2 * f].z, pldf[2 * f + 1].z);
        split(planes[f].w, pldf[2 * f].w, pldf[2 * f + 1].w);
        if (face_eps) eps[f] = face_eps[f];
    }
    std::vector<int2> outline;
    std::vector<float4> corners;
    build_face_outlines(verts, tris, tri_face, nt, nf, planes.data(), outline, corners);
    sbr_scene *sc = new (std::nothrow) sbr_scene();
    if (!sc) return fail(ctx, SBR_ENOMEM, "scene: host allocation failed");
    int2 *d_ol;
    float4 *d_olv;
    float4 *d_nodes, *d_nodes4, *d_tris, *d_pl, *d_pldf;
    Plane64 *d_pld;
    float *d_eps;
    int *d_off, *d_idx, *d_wid;
    float4 *d_w, *d_wn;
    Carver cv;
    cv.add(&d_nodes, bvh.nodes.size());
    cv.add(&d_nodes4, bvh.nodes4.size());
    cv.add(&d_tris, tri4.size());
    cv.add(&d_pl, pl4.size());
    cv.add(&d_pld, planes.size());
    cv.add(&d_pldf, pldf.size());
    cv.add(&d_eps, eps.size());
    cv.add(&d_off, off.size());
    cv.add(&d_idx, std::max<size_t>(idx.size(), 1));
    cv.add(&d_w, w4.size());
    cv.add(&d_wn, wbvh.nodes.size());
    cv.add(&d_wid, wids.size());
    cv.add(&d_ol, outline.size());
    cv.add(&d_olv, corners.size());
    sc->mem = dev_alloc(ctx, cv.total);
    if (!sc->mem) {
        delete sc;
        return fail(ctx, SBR_ENOMEM, "scene: device allocation failed");
    }
    sc->bytes = cv.total;
    cv.bind(sc->mem);
    cudaStream_t s = ctx->stream;
    SBR_CUDA(cudaMemcpyAsync(d_nodes, bvh.nodes.data(), bvh.nodes.size() * sizeof(float4), cudaMemcpyHostToDevice, s));
    SBR_CUDA(cudaMemcpyAsync(d_nodes4, bvh.nodes4.data(), bvh.nodes4.size() * sizeof(float4), cudaMemcpyHostToDevice, s));
    if (nt) SBR_CUDA(cudaMemcpyAsync(d_tris, tri4.data(), tri4.size() * sizeof(float4), cudaMemcpyHostToDevice, s));
    SBR_CUDA(cudaMemcpyAsync(d_pl, pl4.data(), pl4.size() * sizeof(float4), cudaMemcpyHostToDevice, s));
    SBR_CUDA(cudaMemcpyAsync(d_pld, planes.data(), planes.size() * sizeof(Plane64), cudaMemcpyHostToDevice, s));
    SBR_CUDA(cudaMemcpyAsync(d_pldf, pldf.data(), pldf.size() * sizeof(float4), cudaMemcpyHostToDevice, s));
    SBR_CUDA(cudaMemcpyAsync(d_eps, eps.data(), eps.size() * sizeof(float), cudaMemcpyHostToDevice, s));
    SBR_CUDA(cudaMemcpyAsync(d_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    if (nt) SBR_CUDA(cudaMemcpyAsync(d_idx, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    SBR_CUDA(cudaMemcpyAsync(d_w, w4.data(), w4.size() * sizeof(float4), cudaMemcpyHostToDevice, s));
    SBR_CUDA(cudaMemcpyAsync(d_wn, wbvh.nodes.data(), wbvh.nodes.size() * sizeof(float4), cudaMemcpyHostToDevice, s));
    SBR_CUDA(cudaMemcpyAsync(d_wid, wids.data(), wids.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    SBR_CUDA(cudaMemcpyAsync(d_ol, outline.data(), outline.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
    SBR_CUDA(cudaMemcpyAsync(d_olv, corners.data(), corners.size() * sizeof(float4), cudaMemcpyHostToDevice, s));
    SBR_CUDA(cudaStreamSynchronize(s));
    sc->dev.nodes = d_nodes;
    sc->dev.nodes4 = d_nodes4;
    sc->dev.tris = d_tris;
    sc->dev.planes = d_pl;
    sc->dev.planes_d = d_pld;
    sc->dev.planes_df = d_pldf;
    sc->dev.face_eps = d_eps;
    sc->dev.face_tri_off = d_off;
    sc->dev.face_tri_idx = d_idx;
    sc->dev.face_outline = d_ol;
    sc->dev.outline_v = d_olv;
    sc->dev.nt = (int)nt;
    sc->dev.nf = nf;
    sc->dev.nnodes = (int)(bvh.nodes.size() / 4);
    sc->dev.tmin = (float)(1e-7 * diag);
    sc->dev.wedges = d_w;
    sc->dev.wnodes = d_wn;
    sc->dev.wedge_bvh_ids = d_wid;
    sc->dev.nw = nw;
    sc->dev.status = nullptr;
    sc->dev.stack_limit = kStack4;
#ifdef SBR_CHECKED
    if (const char *lim = std::getenv("SBR_CHECKED_STACK_LIMIT"))
        sc->dev.stack_limit = std::max(1, std::min(kStack4, std::atoi(lim)));
#endif
    sc->wedges = std::move(wl);
    sc->info.num_wedges = nw;
    sc->info.num_triangles = nt;
    sc->info.num_faces = nf;
    sc->info.bvh_nodes = sc->dev.nnodes;
    sc->info.bvh_depth = bvh.depth;
    sc->info.max_leaf = bvh.max_leaf;
    sc->info.device_bytes = (int64_t)cv.total;
    for (int a = 0; a < 3; ++a) {
        sc->info.bbox_lo[a] = (float)lo[a];
        sc->info.bbox_hi[a] = (float)hi[a];
    }
    *out = sc;
    return SBR_OK;
}

sbr_status sbr_face_outline_corners(const float *verts, int64_t nv, const int32_t *tris, const int32_t *tri_face,
                                    int64_t nt, int32_t nf, int32_t *corners) {
    if (nv < 0 || nt < 0 || nf < 0 || (nf > 0 && !corners) || (nt > 0 && (!verts || !tris || !tri_face)))
        return SBR_EINVAL;
    // face planes from each face's first triangle, as in sbr_scene_upload
    std::vector<Plane64> planes((size_t)std::max(nf, 1), Plane64{0, 0, 0, 0});
    std::vector<char> seen((size_t)std::max(nf, 1), 0);
    for (int64_t t = 0; t < nt; ++t) {
        int ia = tris[3 * t], ib = tris[3 * t + 1], ic = tris[3 * t + 2], f = tri_face[t];
        if (ia < 0 || ib < 0 || ic < 0 || ia >= nv || ib >= nv || ic >= nv || f < 0 || f >= nf)
            return SBR_EDEGENERATE;
        const float *A = verts + 3 * ia, *B = verts + 3 * ib, *C = verts + 3 * ic;
        double e1[3] = {(double)B[0] - A[0], (double)B[1] - A[1], (double)B[2] - A[2]};
        double e2[3] = {(double)C[0] - A[0], (double)C[1] - A[1], (double)C[2] - A[2]};
        double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        double len = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        if (!(len > 0.0)) return SBR_EDEGENERATE;
        if (!seen[f]) {
            seen[f] = 1;
            double u[3] = {n[0] / len, n[1] / len, n[2] / len};
            planes[f] = Plane64{u[0], u[1], u[2], u[0] * A[0] + u[1] * A[1] + u[2] * A[2]};
        }
    }
    std::vector<int2> outline;
    std::vector<float4> pts;
    build_face_outlines(verts, tris, tri_face, nt, nf, planes.data(), outline, pts);
    for (int f = 0; f < nf; ++f) corners[f] = outline[f].y;
    return SBR_OK;
}

sbr_status sbr_scene_wedges(const sbr_scene *scene, float *ab, int32_t *faces, int64_t cap, int64_t *count) {
    if (!scene || !count || cap < 0 || (cap > 0 && (!ab || !faces))) return SBR_EINVAL;
    *count = (int64_t)scene->wedges.size();
    for (int64_t i = 0; i < std::min<int64_t>(cap, *count); ++i) {
        const WedgeHost &w = scene->wedges[i];
        for (int a = 0; a < 3; ++a) {
            ab[6 * i + a] = w.a[a];
            ab[6 * i + 3 + a] = w.b[a];
        }
        faces[2 * i] = w.f1;
        faces[2 * i + 1] = w.f2;
    }
    return SBR_OK;
}

sbr_status sbr_scene_destroy(sbr_ctx *ctx, sbr_scene *sc) {
    if (!ctx || !sc) return SBR_EINVAL;
    DeviceGuard g(ctx->device);
    dev_free(ctx, sc->mem, sc->bytes);
    delete sc;
    return SBR_OK;
}

sbr_status sbr_scene_get_info(const sbr_scene *sc, sbr_scene_info *out) {
    if (!sc || !out) return SBR_EINVAL;
    *out = sc->info;
    return SBR_OK;
}

// ------------------------------------------------------------------------------ receivers
sbr_status sbr_rx_upload(sbr_ctx *ctx, const float *rx, int32_t nrx, sbr_rxset **out) {
    if (!ctx || !out) return fail(ctx, SBR_EINVAL, "sbr_rx_upload: null argument");
    *out = nullptr;
    if (nrx < 0 || (nrx > 0 && !rx)) return fail(ctx, SBR_EINVAL, "sbr_rx_upload: bad receiver array");
    DeviceGuard g(ctx->device);
    std::vector<float> host((size_t)3 * nrx);
    if (nrx) {
        if (is_device_ptr(rx)) {
            SBR_CUDA(cudaMemcpyAsync(host.data(), rx, host.size() * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
            SBR_CUDA(cudaStreamSynchronize(ctx->stream));
        } else {
            std::memcpy(host.data(), rx, host.size() * sizeof(float));
        }
    }
    for (float v : host)
        if (!std::isfinite(v)) return fail(ctx, SBR_EINVAL, "sbr_rx_upload: non-finite receiver coordinate");
    BvhOut bvh;
    std::string err;
    if (!build_bvh(host, host, 1, bvh, err)) return fail(ctx, SBR_EINVAL, err);
    if (bvh.max_stack4 > kStack4) return fail(ctx, SBR_EINVAL, "sbr_rx_upload: receiver BVH too deep");
    std::vector<float4> pts((size_t)std::max(nrx, 1)), by_id((size_t)std::max(nrx, 1));
    sbr_rxset *rs = new (std::nothrow) sbr_rxset();
    if (!rs) return fail(ctx, SBR_ENOMEM, "rx: host allocation failed");
    for (int a = 0; a < 3; ++a) {
        rs->dev.lo[a] = INFINITY;
        rs->dev.hi[a] = -INFINITY;
    }
    for (int i = 0; i < nrx; ++i) {
        int o = bvh.prim_order[i];
        pts[i] = make_float4(host[3 * o], host[3 * o + 1], host[3 * o + 2], bits_as_float(o));
        by_id[i] = make_float4(host[3 * i], host[3 * i + 1], host[3 * i + 2], 0.0f);
        for (int a = 0; a < 3; ++a) {
            rs->dev.lo[a] = std::min(rs->dev.lo[a], host[3 * i + a]);
            rs->dev.hi[a] = std::max(rs->dev.hi[a], host[3 * i + a]);
        }
    }
    float4 *d_nodes, *d_nodes4, *d_pts, *d_by;
    Carver cv;
    cv.add(&d_nodes, bvh.nodes.size());
    cv.add(&d_nodes4, bvh.nodes4.size());
    cv.add(&d_pts, pts.size());
    cv.add(&d_by, by_id.size());
    rs->mem = dev_alloc(ctx, cv.total);
    if (!rs->mem) {
        delete rs;
        return fail(ctx, SBR_ENOMEM, "rx: device allocation failed");
    }
    rs->bytes = cv.total;
    cv.bind(rs->mem);
    SBR_CUDA(cudaMemcpyAsync(d_nodes, bvh.nodes.data(), bvh.nodes.size() * sizeof(float4), cudaMemcpyHostToDevice,
                             ctx->stream));
    SBR_CUDA(cudaMemcpyAsync(d_nodes4, bvh.nodes4.data(), bvh.nodes4.size() * sizeof(float4), cudaMemcpyHostToDevice,
                             ctx->stream));
    SBR_CUDA(cudaMemcpyAsync(d_pts, pts.data(), pts.size() * sizeof(float4), cudaMemcpyHostToDevice, ctx->stream));
    SBR_CUDA(cudaMemcpyAsync(d_by, by_id.data(), by_id.size() * sizeof(float4), cudaMemcpyHostToDevice, ctx->stream));
    SBR_CUDA(cudaStreamSynchronize(ctx->stream));
    rs->dev.nodes = d_nodes;
    rs->dev.nodes4 = d_nodes4;
    rs->dev.pts = d_pts;
    rs->dev.by_id = d_by;
    rs->dev.nrx = nrx;
    rs->host = std::move(host);
    *out = rs;
    return SBR_OK;
}

sbr_status sbr_rx_destroy(sbr_ctx *ctx, sbr_rxset *rs) {
    if (!ctx || !rs) return SBR_EINVAL;
    DeviceGuard g(ctx->device);
    dev_free(ctx, rs->mem, rs->bytes);
    delete rs;
    return SBR_OK;
}

// ------------------------------------------------------------------------------ paths
sbr_status sbr_paths_create(sbr_ctx *ctx, int64_t record_cap, int64_t path_cap, sbr_paths **out) {
    if (!ctx || !out) return fail(ctx, SBR_EINVAL, "sbr_paths_create: null argument");
    *out = nullptr;
    if (record_cap < 1 || path_cap < 1 || record_cap > (1LL << 31) || path_cap > (1LL << 31))
        return fail(ctx, SBR_EINVAL, "sbr_paths_create: capacities must be in [1, 2^31]");
    DeviceGuard g(ctx->device);
    sbr_paths *p = new (std::nothrow) sbr_paths();
    if (!p) return fail(ctx, SBR_ENOMEM, "paths: host allocation failed");
    int64_t slots = 1024;
    while (slots < 2 * record_cap) slots <<= 1;
    unsigned long long *table;
    Carver cv;
    cv.add(&p->recs, (size_t)record_cap);
    cv.add(&p->paths, (size_t)path_cap);
    cv.add(&p->unf, (size_t)path_cap * kUnfStride);
    cv.add(&p->order_idx, (size_t)path_cap);
    cv.add(&p->order_cnt, (size_t)64);
    cv.add(&p->fp64_idx, (size_t)path_cap);
    cv.add(&table, (size_t)slots * 2 + (size_t)(slots + 1) / 2);   // (key, value) slots, winner ids
    cv.add(&p->counters, (size_t)kNumCounters);
    p->mem = dev_alloc(ctx, cv.total);
    if (!p->mem) {
        delete p;
        return fail(ctx, SBR_ENOMEM, "paths: device allocation failed");
    }
    p->bytes = cv.total;
    cv.bind(p->mem);
    p->table = table;
    p->table_slots = slots;
    p->record_cap = record_cap;
    p->path_cap = path_cap;
    SBR_CUDA(cudaMemsetAsync(p->counters, 0, kNumCounters * sizeof(long long), ctx->stream));
    *out = p;
    return SBR_OK;
}

sbr_status sbr_paths_destroy(sbr_ctx *ctx, sbr_paths *p) {
    if (!ctx || !p) return SBR_EINVAL;
    DeviceGuard g(ctx->device);
    dev_free(ctx, p->mem, p->bytes);
    dev_free(ctx, p->tx_mem, p->tx_bytes);
    dev_free(ctx, p->pair_mem, p->pair_bytes);
    delete p;
    return SBR_OK;
}

static sbr_status ensure_tx(sbr_ctx *ctx, sbr_paths *p, const float *tx, int32_t ntx) {
    if (ntx > p->tx_cap) {
        dev_free(ctx, p->tx_mem, p->tx_bytes);
        size_t b = (size_t)ntx * sizeof(float4);
        p->tx_mem = dev_alloc(ctx, b);
        p->tx_bytes = p->tx_mem ? b : 0;
        p->tx_cap = p->tx_mem ? ntx : 0;
        p->tx = static_cast<float4 *>(p->tx_mem);
        if (!p->tx_mem) return fail(ctx, SBR_ENOMEM, "paths: transmitter buffer allocation failed");
    }
    return copy_points(ctx, p->tx, tx, ntx);
}

static sbr_status report_checks(sbr_ctx *ctx, long long flags, const char *where);

static DedupArgs dedup_args(sbr_ctx *ctx, sbr_paths *paths, int nrx, int rank, int world) {
    DedupArgs d;
    d.recs = paths->recs;
    d.rec_cap = paths->record_cap;
    d.table = paths->table;
    d.slots = paths->table_slots;
    d.paths = paths->paths;
    d.path_cap = paths->path_cap;
    d.dirs = static_cast<const float4 *>(ctx->dirs);
    d.counters = paths->counters;
    d.nrx = nrx;
    d.shard_rank = rank;
    d.shard_world = world;
    return d;
}

sbr_status sbr_launch(sbr_ctx *ctx, const sbr_scene *scene, const float *tx, int32_t ntx, const sbr_rxset *rx,
                      const sbr_launch_params *prm, sbr_paths *paths) {
    if (!ctx || !scene || !tx || !rx || !prm || !paths) return fail(ctx, SBR_EINVAL, "sbr_launch: null argument");
    if (ntx < 1) return fail(ctx, SBR_EINVAL, "sbr_launch: ntx must be >= 1");
    if (prm->n_div < 1 || prm->n_div > 14000) return fail(ctx, SBR_EINVAL, "sbr_launch: n_div out of range [1, 14000]");
    if (prm->max_order < 0 || prm->max_order > SBR_MAX_ORDER)
        return fail(ctx, SBR_EINVAL, "sbr_launch: max_order out of range [0, 8]");
    if (!(prm->rx_angle_scale > 0.0f) || !std::isfinite(prm->rx_angle_scale))
        return fail(ctx, SBR_EINVAL, "sbr_launch: rx_angle_scale must be positive");
    if (rays_for_launcher(prm->n_div, prm->launcher) < 0)
        return fail(ctx, SBR_EINVAL, "sbr_launch: launcher must be 0 (equiangular), 20 or 8 (equidistant)");
    if (prm->dump_stride > 0) {
        if (!prm->dump_faces) return fail(ctx, SBR_EINVAL, "sbr_launch: dump_faces is null");
        int64_t per = (rays_for_launcher(prm->n_div, prm->launcher) + prm->dump_stride - 1) / prm->dump_stride;
        if (prm->dump_cap < (int64_t)ntx * per * (prm->max_order + 1))
            return fail(ctx, SBR_EINVAL, "sbr_launch: dump_cap smaller than ntx * ceil(N / stride) * (max_order + 1)");
    }
    const int64_t N = rays_for_launcher(prm->n_div, prm->launcher);
    int64_t ray_begin = 0, ray_count = N;
    if (prm->flags & SBR_LAUNCH_RAY_RANGE) {
        if (prm->ray_begin < 0 || prm->ray_end < prm->ray_begin || prm->ray_end > N)
            return fail(ctx, SBR_EINVAL, "sbr_launch: ray range must satisfy 0 <= ray_begin <= ray_end <= N");
        ray_begin = prm->ray_begin;
        ray_count = prm->ray_end - prm->ray_begin;
    }
    DeviceGuard g(ctx->device);
    sbr_status st = ensure_tx(ctx, paths, tx, ntx);
    if (st != SBR_OK) return st;
    const bool timing = (prm->flags & SBR_LAUNCH_TIMING) != 0;
    if (timing && !ctx->ev[0])
        for (auto &e : ctx->ev) SBR_CUDA(cudaEventCreate(&e));
    if (timing) SBR_CUDA(cudaEventRecord(ctx->ev[0], ctx->stream));
    {
        Range r("sbr_launch: raygen");
        st = ensure_dirs(ctx, prm->n_div, prm->launcher);
    }
    if (st != SBR_OK) return st;
    if (timing) SBR_CUDA(cudaEventRecord(ctx->ev[1], ctx->stream));
    SBR_CUDA(cudaMemsetAsync(paths->counters, 0, kNumCounters * sizeof(long long), ctx->stream));
    TraceArgs a;
    a.scene = scene->dev;
    a.scene.status = reinterpret_cast<unsigned long long *>(paths->counters + kErrorFlags);
    a.rx = rx->dev;
    a.dirs = static_cast<const float4 *>(ctx->dirs);
    a.tx = paths->tx;
    a.ntx = ntx;
    a.nrays_per_tx = ray_count;
    a.ray_begin = ray_begin;
    a.max_order = prm->max_order;
    double cone = prm->rx_angle_scale * sbr_theta_launch(prm->n_div);
    a.cone = (float)cone;
    a.tan_cone = (float)std::tan(cone);
    a.tan2_pre = cone < 1.5 ? (float)(std::tan(cone) * std::tan(cone) * (1.0 + 1e-4)) : INFINITY;
    a.recs = paths->recs;
    a.rec_cap = paths->record_cap;
    a.counters = paths->counters;
    a.dump_stride = prm->dump_stride;
    a.dump_faces = prm->dump_faces;
    a.dump_per_tx = prm->dump_stride > 0 ? (N + prm->dump_stride - 1) / prm->dump_stride : 0;
    a.refill_min = prm->refill_min > 0 ? std::min(prm->refill_min, 32) : 24;
    a.tiled_n = (prm->launcher == 0 && ray_begin == 0 && ray_count == N && !(prm->flags & SBR_LAUNCH_ID_ORDER))
                    ? prm->n_div : 0;
    int block = prm->block_threads > 0 ? prm->block_threads : 128;
    if (block % 32 != 0 || block > 128)
        return fail(ctx, SBR_EINVAL, "sbr_launch: block_threads must be a multiple of 32, at most 128");
    int grid = prm->grid_blocks > 0 ? prm->grid_blocks : ctx->num_sms * trace_blocks_per_sm(block);
    {
        Range r("sbr_launch: trace + reception");
        SBR_CUDA(launch_trace(a, grid, block, ctx->stream));
    }
    if (timing) SBR_CUDA(cudaEventRecord(ctx->ev[2], ctx->stream));
    if (prm->flags & SBR_LAUNCH_DIFFRACTION) {
        DiffractArgs df;
        df.scene = a.scene;
        df.rx = rx->dev;
        df.dirs = a.dirs;
        df.tx = paths->tx;
        df.ntx = ntx;
        df.nrays_per_tx = ray_count;
        df.ray_begin = ray_begin;
        df.cone = a.cone;
        df.tan_cone = a.tan_cone;
        df.recs = paths->recs;
        df.rec_cap = paths->record_cap;
        df.counters = paths->counters;
        // the candidate list borrows the dedup table, which is cleared after this step
        df.cand = reinterpret_cast<float4 *>(paths->table);
        df.cand_cap = paths->table_slots * 5 / 8;
        df.tiled_n = a.tiled_n;
        Range r("sbr_launch: diffraction");
        SBR_CUDA(launch_diffract(df, ctx->num_sms, ctx->stream));
    }
    if (timing) SBR_CUDA(cudaEventRecord(ctx->ev[4], ctx->stream));
    paths->trace_grid = grid;
    paths->trace_block = block;
    if (!(prm->flags & SBR_LAUNCH_RECORDS_ONLY)) {
        DedupArgs d = dedup_args(ctx, paths, rx->dev.nrx, 0, 1);
        Range r("sbr_launch: dedup");
        SBR_CUDA(launch_dedup(d, ctx->num_sms, ctx->stream));
    }
    if (timing) SBR_CUDA(cudaEventRecord(ctx->ev[3], ctx->stream));
    paths->timed = timing;
    paths->ntx = ntx;
    paths->nrx = rx->dev.nrx;
    paths->n_div = prm->n_div;
    paths->launcher = prm->launcher;
    paths->max_order = prm->max_order;
    paths->rx = rx;
    paths->alpha = prm->rx_angle_scale;
    paths->ray_begin = ray_begin;
    paths->ray_count = ray_count;
    paths->pair_cap = -1;   // per-pair buckets are stale
    if (prm->flags & SBR_LAUNCH_SYNC) {
        sbr_launch_stats s;
        st = sbr_launch_get_stats(ctx, paths, &s);
        if (st != SBR_OK) return st;
        if (s.records > paths->record_cap || s.paths > paths->path_cap || s.diffraction_candidates > s.candidate_cap)
            return fail(ctx, SBR_EOVERFLOW, "sbr_launch: " + std::to_string(s.records) + " records / " +
                                                std::to_string(s.paths) + " paths exceed the container");
        if (s.collisions) return fail(ctx, SBR_ECOLLISION, "sbr_launch: dedup hash collision");
        st = report_checks(ctx, s.check_flags, "sbr_launch");
        if (st != SBR_OK) return st;
    }
    return SBR_OK;
}

sbr_status sbr_launch_get_stats(sbr_ctx *ctx, const sbr_paths *paths, sbr_launch_stats *out) {
    if (!ctx || !paths || !out) return fail(ctx, SBR_EINVAL, "sbr_launch_get_stats: null argument");
    DeviceGuard g(ctx->device);
    long long c[kNumCounters];
    SBR_CUDA(cudaMemcpyAsync(c, paths->counters, sizeof(c), cudaMemcpyDeviceToHost, ctx->stream));
    SBR_CUDA(cudaStreamSynchronize(ctx->stream));
    out->rays = (int64_t)paths->ntx * paths->ray_count;
    out->segments = c[kSegments];
    out->node_visits = c[kNodeVisits];
    out->tri_tests = c[kTriTests];
    out->rx_tests = c[kRxTests];
    out->records = c[kRecords];
    out->paths = c[kPaths];
    out->collisions = c[kCollisions];
    out->ntx = paths->ntx;
    out->nrx = paths->nrx;
    out->n_div = paths->n_div;
    out->max_order = paths->max_order;
    out->ms_raygen = out->ms_trace = out->ms_dedup = out->ms_diffract = 0.0f;
    if (paths->timed && ctx->ev[0]) {
        SBR_CUDA(cudaEventElapsedTime(&out->ms_raygen, ctx->ev[0], ctx->ev[1]));
        SBR_CUDA(cudaEventElapsedTime(&out->ms_trace, ctx->ev[1], ctx->ev[2]));
        SBR_CUDA(cudaEventElapsedTime(&out->ms_diffract, ctx->ev[2], ctx->ev[4]));
        SBR_CUDA(cudaEventElapsedTime(&out->ms_dedup, ctx->ev[4], ctx->ev[3]));
    }
    out->wedge_tests = c[kWedgeTests];
    out->diffraction_records = c[kDiffRecords];
    out->diffraction_candidates = c[kDiffCand];
    out->candidate_cap = paths->table_slots * 5 / 8;
    out->trace_grid = paths->trace_grid;
    out->trace_block = paths->trace_block;
    out->check_flags = c[kErrorFlags];
    return SBR_OK;
}

// SBR_ECHECK with the failed checks named, when a container's status word has bits set
static sbr_status report_checks(sbr_ctx *ctx, long long flags, const char *where) {
    if (!flags) return SBR_OK;
    static const char *names[] = {"trace stack", "occlusion stack", "receiver stack", "face id", "binary-BVH stack"};
    std::string m = std::string(where) + ": device bounds checks failed:";
    for (int b = 0; b < 5; ++b)
        if (flags & (1LL << b)) m += std::string(" ") + names[b];
    return fail(ctx, SBR_ECHECK, m);
}

// ------------------------------------------------------------------------------ records
static_assert(sizeof(sbr_reception_record) == sizeof(RecDev), "reception record layout");
static_assert(offsetof(sbr_reception_record, err) == offsetof(RecDev, err), "reception record layout");
static_assert(offsetof(sbr_reception_record, slot) == offsetof(RecDev, slot), "reception record layout");

sbr_status sbr_records_read(sbr_ctx *ctx, const sbr_paths *paths, sbr_reception_record *out, int64_t cap,
                            int64_t *written) {
    if (!ctx || !paths || !written || cap < 0 || (cap > 0 && !out))
        return fail(ctx, SBR_EINVAL, "sbr_records_read: null argument or negative cap");
    DeviceGuard g(ctx->device);
    long long c = 0;
    SBR_CUDA(cudaMemcpyAsync(&c, paths->counters + kRecords, sizeof(c), cudaMemcpyDeviceToHost, ctx->stream));
    SBR_CUDA(cudaStreamSynchronize(ctx->stream));
    int64_t n = std::min<int64_t>(std::min<int64_t>(c, paths->record_cap), cap);
    if (n > 0) {
        cudaMemcpyKind kind = is_device_ptr(out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        SBR_CUDA(cudaMemcpyAsync(out, paths->recs, (size_t)n * sizeof(RecDev), kind, ctx->stream));
        SBR_CUDA(cudaStreamSynchronize(ctx->stream));
    }
    *written = n;
    return SBR_OK;
}

sbr_status sbr_records_dedup(sbr_ctx *ctx, sbr_paths *paths, const sbr_reception_record *in, int64_t count,
                             int32_t rank, int32_t world) {
    if (!ctx || !paths || count < 0 || (count > 0 && !in))
        return fail(ctx, SBR_EINVAL, "sbr_records_dedup: null argument or negative count");
    if (world < 1 || rank < 0 || rank >= world)
        return fail(ctx, SBR_EINVAL, "sbr_records_dedup: need 0 <= rank < world");
    if (!paths->rx || paths->ntx < 1 || paths->n_div < 1)
        return fail(ctx, SBR_EINVAL, "sbr_records_dedup: the container holds no launch");
    if (count > paths->record_cap)
        return fail(ctx, SBR_EOVERFLOW, "sbr_records_dedup: " + std::to_string(count) + " records exceed record_cap");
    DeviceGuard g(ctx->device);
    if (!(ctx->dirs_valid && ctx->dirs_n == paths->n_div && ctx->dirs_launcher == paths->launcher)) {
        sbr_status st = ensure_dirs(ctx, paths->n_div, paths->launcher);   // rough launch directions
        if (st != SBR_OK) return st;
    }
    if (count > 0) {
        cudaMemcpyKind kind = is_device_ptr(in) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        SBR_CUDA(cudaMemcpyAsync(paths->recs, in, (size_t)count * sizeof(RecDev), kind, ctx->stream));
    }
    SBR_CUDA(launch_records_reset(paths->counters, count, ctx->stream));
    DedupArgs d = dedup_args(ctx, paths, paths->nrx, rank, world);
    {
        Range r("sbr_records_dedup: dedup");
        SBR_CUDA(launch_dedup(d, ctx->num_sms, ctx->stream));
    }
    paths->pair_cap = -1;
    paths->timed = false;
    return SBR_OK;
}

// ------------------------------------------------------------------------------ refine
static sbr_status refine_args(sbr_ctx *ctx, const sbr_scene *scene, sbr_paths *paths, const sbr_refine_params *prm,
                              RefineArgs &A) {
    if (!ctx || !scene || !paths || !prm) return fail(ctx, SBR_EINVAL, "refine: null argument");
    double rho[16], phi[16], sh;
    if (subray_pattern(prm->subrays, rho, phi, &sh) != prm->subrays)
        return fail(ctx, SBR_EINVAL, "refine: subrays must be 6, 7, 9 or 16");
    if (prm->max_iters < 0 || prm->max_iters > 200) return fail(ctx, SBR_EINVAL, "refine: max_iters out of [0, 200]");
    if (!paths->rx || paths->ntx < 1) return fail(ctx, SBR_EINVAL, "refine: container holds no launch");
    A.scene = scene->dev;
    A.scene.status = reinterpret_cast<unsigned long long *>(paths->counters + kErrorFlags);
    A.tx = paths->tx;
    A.rx = paths->rx->dev.by_id;
    A.paths = paths->paths;
    A.unf = paths->unf;
    A.order_idx = paths->order_idx;
    A.order_cnt = paths->order_cnt;
    A.fp64_idx = paths->fp64_idx;
    A.counters = paths->counters;
    A.path_cap = paths->path_cap;
    A.range = nullptr;
    A.index = nullptr;
    A.K = prm->subrays;
    A.max_iters = prm->max_iters;
    A.theta_launch = (float)sbr_theta_launch(paths->n_div);
    A.target = prm->target_err_rad;
    A.tan2_target = prm->target_err_rad >= 1.5707963267948966 ? INFINITY
                                                               : std::pow(std::tan(prm->target_err_rad), 2.0);
    A.fp64_below = prm->fp64_below_rad > 0 ? prm->fp64_below_rad : 1e-5;
    A.tan2_target_f = (float)A.tan2_target;
    A.target_on = A.target > 0.0;
    A.fp64_below_f = (float)A.fp64_below;
    if ((double)A.fp64_below_f < A.fp64_below) A.fp64_below_f = std::nextafter(A.fp64_below_f, INFINITY);
    A.freq = prm->freq_hz > 0 ? prm->freq_hz : 2.4e9;
    A.ptx_dbm = prm->ptx_dbm;
    A.choice_log = prm->choice_log;
    A.chunk = 1;
    A.split_min = 16LL * 32 * std::max(ctx->num_sms, 1);   // 16 warps of paths per SM
    A.ntx = paths->ntx;
    A.nrx = paths->nrx;
    A.nf = scene->dev.nf;
    A.nw = scene->dev.nw;
    return SBR_OK;
}

sbr_status sbr_refine(sbr_ctx *ctx, const sbr_scene *scene, sbr_paths *paths, const sbr_refine_params *prm) {
    RefineArgs A;
    sbr_status st = refine_args(ctx, scene, paths, prm, A);
    if (st != SBR_OK) return st;
    DeviceGuard g(ctx->device);
    int nb = 1;
    refine_kernel_attrs(nullptr, 128, &nb, false, 0);
    {
        Range r("sbr_refine: iterations + validity + outputs");
        SBR_CUDA(launch_refine(A, ctx->num_sms * nb, 128, ctx->stream));
    }
    return SBR_OK;
}

sbr_status sbr_refine_pair(sbr_ctx *ctx, const sbr_scene *scene, sbr_paths *paths, int32_t tx, int32_t rx,
                           const sbr_refine_params *prm) {
    RefineArgs A;
    sbr_status st = refine_args(ctx, scene, paths, prm, A);
    if (st != SBR_OK) return st;
    if (tx < 0 || tx >= paths->ntx || rx < 0 || rx >= paths->nrx)
        return fail(ctx, SBR_EINVAL, "sbr_refine_pair: pair out of range");
    DeviceGuard g(ctx->device);
    const int npairs = paths->ntx * paths->nrx;
    if (paths->pair_cap != paths->path_cap) {
        size_t need = sizeof(int) * ((size_t)npairs + 1 + (size_t)paths->path_cap + (size_t)npairs);
        if (paths->pair_bytes < need) {
            dev_free(ctx, paths->pair_mem, paths->pair_bytes);
            paths->pair_mem = dev_alloc(ctx, need);
            paths->pair_bytes = paths->pair_mem ? need : 0;
            if (!paths->pair_mem) return fail(ctx, SBR_ENOMEM, "sbr_refine_pair: allocation failed");
        }
        paths->pair_off = static_cast<int *>(paths->pair_mem);
        PairArgs pa;
        pa.paths = paths->paths;
        pa.counters = paths->counters;
        pa.path_cap = paths->path_cap;
        pa.nrx = paths->nrx;
        pa.npairs = npairs;
        pa.pair_count = paths->pair_off;
        pa.pair_idx = paths->pair_off + npairs + 1;
        SBR_CUDA(launch_pair_bucket(pa, ctx->stream));
        // one host copy of every pair's range per launch, so that later calls size their
        // grid without a device round trip
        paths->pair_host.resize((size_t)npairs + 1);
        SBR_CUDA(cudaMemcpyAsync(paths->pair_host.data(), paths->pair_off, sizeof(int) * ((size_t)npairs + 1),
                                 cudaMemcpyDeviceToHost, ctx->stream));
        SBR_CUDA(cudaStreamSynchronize(ctx->stream));
        paths->pair_cap = paths->path_cap;
    }
    int p = tx * paths->nrx + rx;
    int count = paths->pair_host[p + 1] - paths->pair_host[p];
    if (count <= 0) return SBR_OK;
    A.range = paths->pair_off + p;
    A.index = paths->pair_off + npairs + 1;
    {
        Range r("sbr_refine_pair: iterations + validity + outputs");
        SBR_CUDA(launch_refine(A, (count + 127) / 128, 128, ctx->stream));
    }
    return SBR_OK;
}

sbr_status sbr_batch_refine(sbr_ctx *ctx, const sbr_scene *scene, sbr_paths *paths, const sbr_refine_params *prm,
                            const sbr_batch_config *cfg) {
    RefineArgs A;
    sbr_status st = refine_args(ctx, scene, paths, prm, A);
    if (st != SBR_OK) return st;
    DeviceGuard g(ctx->device);
    int block = cfg && cfg->block_threads > 0 ? cfg->block_threads : 128;
    if (block % 32 != 0 || block > 256)
        return fail(ctx, SBR_EINVAL, "sbr_batch_refine: block_threads must be a multiple of 32, at most 256");
    int lanes = cfg && cfg->lanes_per_path > 0 ? cfg->lanes_per_path : 16;
    if (lanes != 1 && lanes != 8 && lanes != 16 && lanes != 32)
        return fail(ctx, SBR_EINVAL, "sbr_batch_refine: lanes_per_path must be 1, 8, 16 or 32");
    int nb = 1;
    refine_kernel_attrs(nullptr, block, &nb, true, lanes);
    if (cfg && cfg->blocks_per_sm > 0) nb = std::min(nb, cfg->blocks_per_sm);
    A.chunk = lanes;
    if (lanes == 1) A.split_min = 0;   // the one-lane form runs with the unfold and FP64 tail kernels
    {
        Range r("sbr_batch_refine: unfold, iterations, FP64 tail, validity + outputs");
        SBR_CUDA(launch_batch_refine(A, ctx->num_sms * nb, block, ctx->stream));
    }
    return SBR_OK;
}

// ------------------------------------------------------------------------------ results
sbr_status sbr_paths_count(sbr_ctx *ctx, const sbr_paths *paths, int64_t *out) {
    if (!ctx || !paths || !out) return fail(ctx, SBR_EINVAL, "sbr_paths_count: null argument");
    DeviceGuard g(ctx->device);
    long long c = 0;
    SBR_CUDA(cudaMemcpyAsync(&c, paths->counters + kPaths, sizeof(c), cudaMemcpyDeviceToHost, ctx->stream));
    SBR_CUDA(cudaStreamSynchronize(ctx->stream));
    *out = std::min<int64_t>(c, paths->path_cap);
    return SBR_OK;
}

sbr_status sbr_query(sbr_ctx *ctx, const sbr_paths *paths, sbr_path_record *out, int64_t cap, int64_t *written) {
    if (!ctx || !paths || !written || (cap > 0 && !out)) return fail(ctx, SBR_EINVAL, "sbr_query: null argument");
    int64_t n = 0;
    sbr_status st = sbr_paths_count(ctx, paths, &n);
    if (st != SBR_OK) return st;
    if (SBR_CHECKED_BUILD) {
        long long flags = 0;
        DeviceGuard g0(ctx->device);
        SBR_CUDA(cudaMemcpyAsync(&flags, paths->counters + kErrorFlags, sizeof(flags), cudaMemcpyDeviceToHost,
                                 ctx->stream));
        SBR_CUDA(cudaStreamSynchronize(ctx->stream));
        st = report_checks(ctx, flags, "sbr_query");
        if (st != SBR_OK) return st;
    }
    n = std::min(n, cap);
    DeviceGuard g(ctx->device);
    if (n > 0) {
        cudaMemcpyKind kind = is_device_ptr(out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        SBR_CUDA(cudaMemcpyAsync(out, paths->paths, (size_t)n * sizeof(sbr_path_record), kind, ctx->stream));
        SBR_CUDA(cudaStreamSynchronize(ctx->stream));
    }
    *written = n;
    return SBR_OK;
}

sbr_status sbr_paths_nonfinite(sbr_ctx *ctx, const sbr_paths *paths, int64_t *count) {
    if (!ctx || !paths || !count) return fail(ctx, SBR_EINVAL, "sbr_paths_nonfinite: null argument");
    DeviceGuard g(ctx->device);
    SBR_CUDA(launch_nonfinite_scan(paths->paths, paths->counters, paths->path_cap, ctx->num_sms, ctx->stream));
    long long c = 0;
    SBR_CUDA(cudaMemcpyAsync(&c, paths->counters + kNonFinite, sizeof(c), cudaMemcpyDeviceToHost, ctx->stream));
    SBR_CUDA(cudaStreamSynchronize(ctx->stream));
    *count = c;
    return SBR_OK;
}

sbr_status sbr_paths_import(sbr_ctx *ctx, sbr_paths *paths, const sbr_path_record *in, int64_t count,
                            const float *tx, int32_t ntx, const sbr_rxset *rx, int32_t n_div) {
    if (!ctx || !paths || !tx || !rx || (count > 0 && !in)) return fail(ctx, SBR_EINVAL, "sbr_paths_import: null argument");
    if (count < 0 || count > paths->path_cap) return fail(ctx, SBR_EOVERFLOW, "sbr_paths_import: count exceeds path_cap");
    if (ntx < 1 || n_div < 1) return fail(ctx, SBR_EINVAL, "sbr_paths_import: ntx and n_div must be >= 1");
    DeviceGuard g(ctx->device);
    sbr_status st = ensure_tx(ctx, paths, tx, ntx);
    if (st != SBR_OK) return st;
    if (count > 0) {
        cudaMemcpyKind kind = is_device_ptr(in) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        SBR_CUDA(cudaMemcpyAsync(paths->paths, in, (size_t)count * sizeof(sbr_path_record), kind, ctx->stream));
    }
    long long c[kNumCounters] = {0};
    c[kPaths] = count;
    SBR_CUDA(cudaMemcpyAsync(paths->counters, c, sizeof(c), cudaMemcpyHostToDevice, ctx->stream));
    SBR_CUDA(cudaStreamSynchronize(ctx->stream));
    paths->ntx = ntx;
    paths->nrx = rx->dev.nrx;
    paths->n_div = n_div;
    paths->rx = rx;
    paths->pair_cap = -1;
    return SBR_OK;
}

// ------------------------------------------------------------------------------ unfold
static sbr_status unfold_common(sbr_ctx *ctx, const sbr_scene *scene, int64_t n, const float *tx, const float *rx,
                                const float *az_el, const int32_t *faces, const int32_t *order, UnfoldArgs &a) {
    if (!ctx || !scene || n < 0) return fail(ctx, SBR_EINVAL, "unfold: null argument");
    if (n > 0 && (!tx || !rx || !az_el || !faces || !order)) return fail(ctx, SBR_EINVAL, "unfold: null array");
    if ((reinterpret_cast<uintptr_t>(faces) & 15) != 0) return fail(ctx, SBR_EINVAL, "unfold: faces must be 16-byte aligned");
    a.scene = scene->dev;
    a.nf = scene->dev.nf;
    a.n = n;
    a.tx = tx;
    a.rx = rx;
    a.az_el = az_el;
    a.faces = faces;
    a.order = order;
    a.grad_out = nullptr;
    a.out = a.grad_tx = a.grad_rx = a.grad_az_el = nullptr;
    return SBR_OK;
}

sbr_status sbr_unfold_fwd(sbr_ctx *ctx, const sbr_scene *scene, int64_t n, const float *tx, const float *rx,
                          const float *az_el, const int32_t *faces, const int32_t *order, float *out) {
    UnfoldArgs a;
    sbr_status st = unfold_common(ctx, scene, n, tx, rx, az_el, faces, order, a);
    if (st != SBR_OK) return st;
    if (n > 0 && !out) return fail(ctx, SBR_EINVAL, "unfold: null output");
    if (n == 0) return SBR_OK;
    a.out = out;
    DeviceGuard g(ctx->device);
    SBR_CUDA(launch_unfold_fwd(a, ctx->stream));
    return SBR_OK;
}

sbr_status sbr_unfold_bwd(sbr_ctx *ctx, const sbr_scene *scene, int64_t n, const float *tx, const float *rx,
                          const float *az_el, const int32_t *faces, const int32_t *order, const float *grad_out,
                          float *grad_tx, float *grad_rx, float *grad_az_el) {
    UnfoldArgs a;
    sbr_status st = unfold_common(ctx, scene, n, tx, rx, az_el, faces, order, a);
    if (st != SBR_OK) return st;
    if (n > 0 && (!grad_out || !grad_tx || !grad_rx || !grad_az_el)) return fail(ctx, SBR_EINVAL, "unfold: null gradient array");
    if (n == 0) return SBR_OK;
    a.grad_out = grad_out;
    a.grad_tx = grad_tx;
    a.grad_rx = grad_rx;
    a.grad_az_el = grad_az_el;
    DeviceGuard g(ctx->device);
    SBR_CUDA(launch_unfold_bwd(a, ctx->stream));
    return SBR_OK;
}

}  // extern "C"
