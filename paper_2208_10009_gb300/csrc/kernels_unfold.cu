// kernels_unfold.cu -- a10 the fixed-face-sequence unfolding and its adjoint.
//
// Mirroring through face plane (n, h) is M(x) = H x + 2 h n with H = I - 2 n n^T.  For
// faces f_1..f_k: Rx' = M_1(...M_k(Rx)) = A Rx + a0 with A = H_1 ... H_k; the last Tx image
// Tx^(k) = M_k(...M_1(Tx)) = A^T Tx + b0.  With w = Rx' - Tx and d(az, el) the launch
// direction:
//   miss  = A^T (w - (w.d) d)     real-space vector from the foot of Rx on the last leg to Rx
//   delay = |w| / c0
//   AOD   = (atan2(w_y, w_x), atan2(w_z, hypot(w_x, w_y)))
//   AOA   = same angles of v = Tx^(k) - Rx
// Applying A to a vector is mirroring (linear part) through f_k first, then f_{k-1}, ..., f_1;
// A^T mirrors through f_1 first.  The adjoint recomputes w, v and d instead of storing them.
#include "sbr_device.cuh"

namespace sbr {

struct UnfoldPath {
    float3 tx, rx;
    float az, el;
    int k;
    int faces[kMaxOrder];
};

__device__ __forceinline__ void load_unfold(const UnfoldArgs &a, long long i, UnfoldPath &u) {
    u.tx = make_float3(a.tx[3 * i], a.tx[3 * i + 1], a.tx[3 * i + 2]);
    u.rx = make_float3(a.rx[3 * i], a.rx[3 * i + 1], a.rx[3 * i + 2]);
    u.az = a.az_el[2 * i];
    u.el = a.az_el[2 * i + 1];
    int k = a.order[i];
    u.k = k < 0 ? 0 : (k > kMaxOrder ? kMaxOrder : k);
    const int4 *f4 = reinterpret_cast<const int4 *>(a.faces + 8 * i);
    int4 lo = f4[0], hi = f4[1];
    u.faces[0] = lo.x; u.faces[1] = lo.y; u.faces[2] = lo.z; u.faces[3] = lo.w;
    u.faces[4] = hi.x; u.faces[5] = hi.y; u.faces[6] = hi.z; u.faces[7] = hi.w;
}

// face ids come from the caller: a path with an id outside [0, nf) yields NaN outputs
__device__ __forceinline__ bool unfold_ids_ok(const UnfoldArgs &a, const UnfoldPath &u) {
    for (int j = 0; j < u.k; ++j)
        if (u.faces[j] < 0 || u.faces[j] >= a.nf) return false;
    return true;
}

// x -> A x (reverse order), affine when `point`
__device__ __forceinline__ float3 apply_A(const SceneDev &S, const UnfoldPath &u, float3 x, bool point) {
#pragma unroll
    for (int j = kMaxOrder - 1; j >= 0; --j) {
        if (j >= u.k) continue;
        float4 pl = __ldg(S.planes + u.faces[j]);
        float3 n = f3(pl);
        float s = dot(n, x) - (point ? pl.w : 0.0f);
        x = x - n * (2.0f * s);
    }
    return x;
}

// x -> A^T x (forward order), affine when `point`
__device__ __forceinline__ float3 apply_AT(const SceneDev &S, const UnfoldPath &u, float3 x, bool point) {
#pragma unroll
    for (int j = 0; j < kMaxOrder; ++j) {
        if (j >= u.k) break;
        float4 pl = __ldg(S.planes + u.faces[j]);
        float3 n = f3(pl);
        float s = dot(n, x) - (point ? pl.w : 0.0f);
        x = x - n * (2.0f * s);
    }
    return x;
}

// The linear part of the unfolding as a matrix, A = H_1 ... H_k (row-major m[9]), built
// by right-multiplying the reflections H = I - 2 n n^T in path order: A H = A - 2 (A n) n^T.
// It runs beside the point chains, so the adjoint's linear pull-backs become 3 x 3
// products instead of further mirror chains after them.
__device__ __forceinline__ void build_A(const SceneDev &S, const UnfoldPath &u, float m[9]) {
    m[0] = 1.0f; m[1] = 0.0f; m[2] = 0.0f;
    m[3] = 0.0f; m[4] = 1.0f; m[5] = 0.0f;
    m[6] = 0.0f; m[7] = 0.0f; m[8] = 1.0f;
#pragma unroll
    for (int j = 0; j < kMaxOrder; ++j) {
        if (j >= u.k) break;
        const float3 n = f3(__ldg(S.planes + u.faces[j]));
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const float an = 2.0f * fmaf(m[3 * r], n.x, fmaf(m[3 * r + 1], n.y, m[3 * r + 2] * n.z));
            m[3 * r] = fmaf(-an, n.x, m[3 * r]);
            m[3 * r + 1] = fmaf(-an, n.y, m[3 * r + 1]);
            m[3 * r + 2] = fmaf(-an, n.z, m[3 * r + 2]);
        }
    }
}

__device__ __forceinline__ float3 mul_A(const float m[9], float3 x) {
    return make_float3(fmaf(m[0], x.x, fmaf(m[1], x.y, m[2] * x.z)), fmaf(m[3], x.x, fmaf(m[4], x.y, m[5] * x.z)),
                       fmaf(m[6], x.x, fmaf(m[7], x.y, m[8] * x.z)));
}

__device__ __forceinline__ float3 mul_AT(const float m[9], float3 x) {
    return make_float3(fmaf(m[0], x.x, fmaf(m[3], x.y, m[6] * x.z)), fmaf(m[1], x.x, fmaf(m[4], x.y, m[7] * x.z)),
                       fmaf(m[2], x.x, fmaf(m[5], x.y, m[8] * x.z)));
}

__device__ __forceinline__ void angles(float3 w, float &az, float &el) {
    az = atan2f(w.y, w.x);
    el = atan2f(w.z, sqrtf(w.x * w.x + w.y * w.y));
}

// gradient of (az, el) of w with respect to w
__device__ __forceinline__ void angles_grad(float3 w, float3 &gaz, float3 &gel) {
    float rho2 = w.x * w.x + w.y * w.y, rho = sqrtf(rho2), r2 = rho2 + w.z * w.z;
    gaz = make_float3(-w.y / rho2, w.x / rho2, 0.0f);
    float c = 1.0f / (r2 * rho);
    gel = make_float3(-w.x * w.z * c, -w.y * w.z * c, rho / r2);
}

__global__ void unfold_fwd_kernel(UnfoldArgs a) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < a.n; i += (long long)gridDim.x * blockDim.x) {
        UnfoldPath u;
        load_unfold(a, i, u);
        if (!unfold_ids_ok(a, u)) {
            for (int j = 0; j < 8; ++j) a.out[8 * i + j] = __int_as_float(0x7fc00000);
            continue;
        }
        float mA[9];
        build_A(a.scene, u, mA);
        float3 rxp = apply_A(a.scene, u, u.rx, true);
        float3 w = rxp - u.tx;
        float se, ce, sa, ca;
        sincosf(u.el, &se, &ce);
        sincosf(u.az, &sa, &ca);
        float3 d = make_float3(ce * ca, ce * sa, se);
        float3 m = w - d * dot(w, d);
        float3 miss = mul_AT(mA, m);
        float3 txk = apply_AT(a.scene, u, u.tx, true);
        float3 v = txk - u.rx;
        float *o = a.out + 8 * i;
        o[0] = miss.x;
        o[1] = miss.y;
        o[2] = miss.z;
        o[3] = sqrtf(dot(w, w)) * (float)(1.0 / kC0);
        angles(w, o[4], o[5]);
        angles(v, o[6], o[7]);
    }
}

// At most 64 registers a thread (four 256-thread blocks per SM): the kernel waits on its
// loads, and the extra resident warps keep more of them in flight (measured 15 % faster
// than 78 registers, three blocks).
__global__ void __launch_bounds__(256, 4) unfold_bwd_kernel(UnfoldArgs a) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < a.n; i += (long long)gridDim.x * blockDim.x) {
        UnfoldPath u;
        load_unfold(a, i, u);
        if (!unfold_ids_ok(a, u)) {
            const float nan = __int_as_float(0x7fc00000);
            for (int j = 0; j < 3; ++j) a.grad_tx[3 * i + j] = a.grad_rx[3 * i + j] = nan;
            a.grad_az_el[2 * i] = a.grad_az_el[2 * i + 1] = nan;
            continue;
        }
        // the row of 8 output gradients: two 16-byte loads when the array is 16-byte
        // aligned (every row then is), else eight 4-byte loads
        float g[8];
        if ((reinterpret_cast<uintptr_t>(a.grad_out) & 15) == 0) {
            const float4 g0 = __ldg(reinterpret_cast<const float4 *>(a.grad_out) + 2 * i);
            const float4 g1 = __ldg(reinterpret_cast<const float4 *>(a.grad_out) + 2 * i + 1);
            g[0] = g0.x; g[1] = g0.y; g[2] = g0.z; g[3] = g0.w;
            g[4] = g1.x; g[5] = g1.y; g[6] = g1.z; g[7] = g1.w;
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) g[j] = __ldg(a.grad_out + 8 * i + j);
        }
        // recompute the forward quantities
        float m[9];
        build_A(a.scene, u, m);
        float3 rxp = apply_A(a.scene, u, u.rx, true);
        float3 w = rxp - u.tx;
        float se, ce, sa, ca;
        sincosf(u.el, &se, &ce);
        sincosf(u.az, &sa, &ca);
        float3 d = make_float3(ce * ca, ce * sa, se);
        float3 d_az = make_float3(-ce * sa, ce * ca, 0.0f);
        float3 d_el = make_float3(-se * ca, -se * sa, ce);
        float3 txk = apply_AT(a.scene, u, u.tx, true);
        float3 v = txk - u.rx;
        float wd = dot(w, d);
        // miss = A^T (w - (w.d) d): pull g_miss back into unfolded space
        float3 gm = mul_A(m, make_float3(g[0], g[1], g[2]));
        float gmd = dot(gm, d);
        float3 gw = gm - d * gmd;
        float3 gd = (gm * wd + w * gmd) * -1.0f;
        // delay
        float wn = sqrtf(dot(w, w));
        gw = gw + w * (g[3] * (float)(1.0 / kC0) / wn);
        // AOD angles of w
        float3 gaz, gel;
        angles_grad(w, gaz, gel);
        gw = gw + gaz * g[4] + gel * g[5];
        // AOA angles of v = A^T Tx + b0 - Rx
        angles_grad(v, gaz, gel);
        float3 gv = gaz * g[6] + gel * g[7];
        float3 gtx = gw * -1.0f + mul_A(m, gv);
        float3 grx = mul_AT(m, gw) - gv;
        a.grad_tx[3 * i] = gtx.x;
        a.grad_tx[3 * i + 1] = gtx.y;
        a.grad_tx[3 * i + 2] = gtx.z;
        a.grad_rx[3 * i] = grx.x;
        a.grad_rx[3 * i + 1] = grx.y;
        a.grad_rx[3 * i + 2] = grx.z;
        a.grad_az_el[2 * i] = dot(gd, d_az);
        a.grad_az_el[2 * i + 1] = dot(gd, d_el);
    }
}

static int unfold_grid(long long n) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long want = (n + 255) / 256;
    long long cap = (long long)sms * 8;
    return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

cudaError_t launch_unfold_fwd(const UnfoldArgs &a, cudaStream_t s) {
    unfold_fwd_kernel<<<unfold_grid(a.n), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_unfold_bwd(const UnfoldArgs &a, cudaStream_t s) {
    unfold_bwd_kernel<<<unfold_grid(a.n), 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace sbr
