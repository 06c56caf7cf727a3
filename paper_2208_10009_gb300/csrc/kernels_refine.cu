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
#include "dfloat.cuh"
#include "nvtx_ranges.h"
#include "sbr_device.cuh"

namespace sbr {

struct SubTab {
    int off[17];                 // first entry of pattern K (K = 6, 7, 9, 16)
    float rho[38], cphi[38], sphi[38];
    double rho_d[38], cphi_d[38], sphi_d[38];
    double shrink[17];
    float shrink_f[17];          // the FP32 phase's factor: its cone radius is kept in FP32
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
        t.shrink_f[Ks[q]] = (float)sh;
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
    int k;        // planes to unfold (0 for a diffraction path)
    int wedge;    // wedge id of a diffraction path, else -1
    int faces[kMaxOrder];
};

// group of a path for the batched form's finalize lists: its order 0..8, diffraction 9
__device__ __forceinline__ int order_group(const PathGeo &g) { return g.wedge >= 0 ? 9 : g.k; }

// Records can come from sbr_paths_import, so every id is checked before it is used.
__device__ __forceinline__ bool path_ids_ok(const RefineArgs &A, const sbr_path_record &p) {
    if (p.tx < 0 || p.tx >= A.ntx || p.rx < 0 || p.rx >= A.nrx || p.order < 0 || p.order > kMaxOrder) return false;
    if (p.order == 1 && p.faces[0] < 0) return -1 - p.faces[0] < A.nw;
    for (int j = 0; j < p.order; ++j)
        if (p.faces[j] < 0 || p.faces[j] >= A.nf) return false;
    return true;
}

// ------------------------------------------------------------ order-1 diffraction (wedges)
struct WedgeD {
    dvec3 a, b, w1, w2;
    int f1, f2;
};

__device__ __forceinline__ WedgeD wedge64(const SceneDev &S, int id) {
    const float4 *p = S.wedges + 4 * (size_t)id;
    float4 A = __ldg(p), B = __ldg(p + 1), W1 = __ldg(p + 2), W2 = __ldg(p + 3);
    return {dv(A.x, A.y, A.z), dv(B.x, B.y, B.z), dv(W1.x, W1.y, W1.z), dv(W2.x, W2.y, W2.z), __float_as_int(A.w),
            __float_as_int(B.w)};
}

// p lies outside the interior sector (the solid) between w1 and w2; e = edge direction
__device__ __forceinline__ bool exterior64(const WedgeD &w, dvec3 e, dvec3 p) {
    dvec3 q = p - w.a;
    q = q - e * ddot(q, e);
    dvec3 n = dcross(w.w1, w.w2);
    return !(ddot(dcross(w.w1, q), n) > 0.0 && ddot(dcross(q, w.w2), n) > 0.0);
}

// W = Rx* - Tx with Rx* = Rx rotated about the edge line into the half-plane through the
// edge opposite Tx: the diffraction analogue of the mirror image, in whose space Eq. 3's
// error angle of a launch direction d is angle(d, W) (zero vector if Tx is on the line)
__device__ __forceinline__ dvec3 wedge_unfold(const SceneDev &S, int id, dvec3 tx, dvec3 rx) {
    WedgeD w = wedge64(S, id);
    dvec3 eb = w.b - w.a;
    dvec3 e = eb * (1.0 / dnorm(eb));
    dvec3 qt = tx - w.a, qr = rx - w.a;
    dvec3 pt = qt - e * ddot(qt, e);
    double zr = ddot(qr, e);
    dvec3 pr = qr - e * zr;
    double rt = dnorm(pt), rr = dnorm(pr);
    if (!(rt > 0.0)) return dv(0.0, 0.0, 0.0);
    return w.a + e * zr - pt * (rr / rt) - tx;
}

__device__ __forceinline__ void load_path(const RefineArgs &A, const sbr_path_record &p, PathGeo &g) {
    float4 t = __ldg(A.tx + p.tx), r = __ldg(A.rx + p.rx);
    g.tx = f3(t);
    g.rx = f3(r);
    g.txd = dv(t.x, t.y, t.z);
    g.rxd = dv(r.x, r.y, r.z);
    g.wedge = (p.order == 1 && p.faces[0] < 0) ? -1 - p.faces[0] : -1;
    g.k = g.wedge >= 0 ? 0 : p.order;
#pragma unroll
    for (int j = 0; j < kMaxOrder; ++j) g.faces[j] = p.faces[j];
}

// The sub-rays of a path are traced through its fixed face planes.  Mirroring is an
// isometry, so that trace is a straight line in the path's unfolded space: face j's plane
// seen through the mirrors of faces 1..j-1 is n'_j . x = h'_j, the sub-ray from Tx along d
// meets it at T_j = num_j / (n'_j . d) with num_j = h'_j - n'_j . Tx, and the real segment
// lengths are T_j - T_{j-1}.  The receiver's image Rx' (mirrored through faces k..1) makes
// Eq. 3 exact in the same space: with W = Rx' - Tx the foot distance d_ray is W . d and
// the distance of Rx from the ray d_Rx-ray is |d x W|, so the error angle is
// atan2(|d x W|, d . W).  A sub-ray costs one dot product per face and no division; the
// argmin compares |d x W|^2, which orders sub-rays like the angle (below pi/2; a sub-ray
// with d . W <= 0 or a non-positive segment is invalid, as in the real-space trace).
struct __align__(32) D4 {
    double x, y, z, w;
};
struct __align__(16) UnfF {
    float4 p[kMaxOrder];   // (n'_j, num_j)
    float4 w;              // (W, 0)
};
struct __align__(32) UnfD {
    D4 p[kMaxOrder];
    D4 w;
};

// plane of face j seen from Tx through the mirrors of faces j-1, ..., 0 (innermost first)
__device__ __forceinline__ D4 unfold_plane(const SceneDev &S, const PathGeo &g, int j) {
    Plane64 pl = S.planes_d[g.faces[j]];
    dvec3 n = dv(pl.x, pl.y, pl.z);
    double h = pl.w;
    for (int m = j - 1; m >= 0; --m) {
        Plane64 q = S.planes_d[g.faces[m]];
        dvec3 qn = dv(q.x, q.y, q.z);
        double nm = ddot(n, qn);
        n = n - qn * (2.0 * nm);
        h = fma(-2.0 * nm, q.w, h);
    }
    return {n.x, n.y, n.z, h - ddot(n, g.txd)};
}

// W = Rx' - Tx, Rx mirrored through faces k-1, ..., 0 (rotated about the edge line for a
// diffraction path)
__device__ __forceinline__ D4 unfold_rx(const SceneDev &S, const PathGeo &g) {
    if (g.wedge >= 0) {
        dvec3 W = wedge_unfold(S, g.wedge, g.txd, g.rxd);
        return {W.x, W.y, W.z, 0.0};
    }
    dvec3 x = g.rxd;
    for (int m = g.k - 1; m >= 0; --m) {
        Plane64 q = S.planes_d[g.faces[m]];
        dvec3 qn = dv(q.x, q.y, q.z);
        x = x - qn * (2.0 * (ddot(qn, x) - q.w));
    }
    x = x - g.txd;
    return {x.x, x.y, x.z, 0.0};
}

// The FP32 copies the FP32 iterations use: the same mirror chains in compensated FP32
// pairs (dfloat.cuh, about 44 bits) from the per-face pairs of the FP64 planes, rounded
// once to FP32 -- the value the FP64 chain rounds to, except within 2^-44 of a rounding
// boundary -- without GB300's 1/64-rate FP64 pipe.
__device__ __forceinline__ void plane_df(const SceneDev &S, int f, df3 &n, df &h) {
    const float4 a = __ldg(S.planes_df + 2 * f), b = __ldg(S.planes_df + 2 * f + 1);
    n = {{a.x, b.x}, {a.y, b.y}, {a.z, b.z}};
    h = {a.w, b.w};
}

__device__ __forceinline__ float df_round(df x) { return __fadd_rn(x.hi, x.lo); }
__device__ __forceinline__ float3 df3_round(const df3 &a) { return make_float3(df_round(a.x), df_round(a.y), df_round(a.z)); }
__device__ __forceinline__ dvec3 df3_double(const df3 &a) { return dv(df_to_double(a.x), df_to_double(a.y), df_to_double(a.z)); }

__device__ __noinline__ float4 unfold_plane32(const SceneDev &S, const PathGeo &g, int j) {
    df3 n;
    df h;
    plane_df(S, g.faces[j], n, h);
    for (int m = j - 1; m >= 0; --m) {
        df3 q;
        df qh;
        plane_df(S, g.faces[m], q, qh);
        const df nm2 = df_scale2(df_dot(n, q), 2.0f);
        n = df3_sub_scaled(n, nm2, q);
        h = df_sub(h, df_mul(nm2, qh));
    }
    const df3 t = {df_of(g.tx.x), df_of(g.tx.y), df_of(g.tx.z)};
    const df num = df_sub(h, df_dot(n, t));
    return make_float4(df_round(n.x), df_round(n.y), df_round(n.z), df_round(num));
}

__device__ __noinline__ float4 unfold_rx32(const SceneDev &S, const PathGeo &g) {
    if (g.wedge >= 0) {
        const dvec3 W = wedge_unfold(S, g.wedge, g.txd, g.rxd);
        return make_float4((float)W.x, (float)W.y, (float)W.z, 0.0f);
    }
    df3 x = {df_of(g.rx.x), df_of(g.rx.y), df_of(g.rx.z)};
    for (int m = g.k - 1; m >= 0; --m) {
        df3 q;
        df qh;
        plane_df(S, g.faces[m], q, qh);
        const df s2 = df_scale2(df_sub(df_dot(q, x), qh), 2.0f);
        x = df3_sub_scaled(x, s2, q);
    }
    return make_float4(df_round(df_sub(x.x, df_of(g.tx.x))), df_round(df_sub(x.y, df_of(g.tx.y))),
                       df_round(df_sub(x.z, df_of(g.tx.z))), 0.0f);
}

__device__ __forceinline__ void build_unf(const SceneDev &S, const PathGeo &g, UnfD &ud, UnfF &uf) {
    for (int j = 0; j < g.k; ++j) {
        ud.p[j] = unfold_plane(S, g, j);
        uf.p[j] = unfold_plane32(S, g, j);
    }
    ud.w = unfold_rx(S, g);
    uf.w = unfold_rx32(S, g);
}

// |d x W|^2 of sub-ray d (+inf if invalid); dw = d . W
__device__ __forceinline__ float key32(const UnfF &u, int k, float3 d, float &dw) {
    float pn = 0.0f, pd = 1.0f;   // T_{j-1} = pn / pd, T_0 = 0
#pragma unroll
    for (int j = 0; j < kMaxOrder; ++j) {
        if (j >= k) break;
        const float4 P = u.p[j];
        const float den = fmaf(P.x, d.x, fmaf(P.y, d.y, P.z * d.z));
        if (den == 0.0f) return INFINITY;
        // sign(T_j - T_{j-1}) = sign(x) * sign(den * pd)
        const float x = fmaf(P.w, pd, -pn * den);
        const bool same = (den > 0.0f) == (pd > 0.0f);
        if (!(same ? x > 0.0f : x < 0.0f)) return INFINITY;
        pn = P.w;
        pd = den;
    }
    const float3 W = make_float3(u.w.x, u.w.y, u.w.z);
    dw = dot(d, W);
    if (!(dw > 0.0f)) return INFINITY;
    const float3 c = cross(d, W);
    return dot(c, c);
}

// The FP64 form takes its sign tests on the doubles' bits with integer instructions: on
// GB300 a double compare occupies the 1/64-rate FP64 pipe like an FMA does.  den != 0 is
// (bits << 1) != 0, and T_j - T_{j-1} > 0 is x != 0 with the sign bits of x, den and
// T_{j-1}'s denominator XOR-ing to 0 (the same decisions as key32's compares).
__device__ __forceinline__ double key64(const UnfD &u, int k, dvec3 d, double &dw) {
    double pn = 0.0, pd = 1.0;
#pragma unroll
    for (int j = 0; j < kMaxOrder; ++j) {
        if (j >= k) break;
        const D4 P = u.p[j];
        const double den = fma(P.x, d.x, fma(P.y, d.y, P.z * d.z));
        const long long bd = __double_as_longlong(den);
        if ((bd << 1) == 0) return INFINITY;
        const double x = fma(P.w, pd, -pn * den);
        const long long bx = __double_as_longlong(x);
        if ((bx << 1) == 0 || (bx ^ bd ^ __double_as_longlong(pd)) < 0) return INFINITY;
        pn = P.w;
        pd = den;
    }
    const dvec3 W = dv(u.w.x, u.w.y, u.w.z);
    dw = ddot(d, W);
    if (__double_as_longlong(dw) <= 0) return INFINITY;   // dw > 0 (a positive double's bits are > 0)
    const dvec3 c = dcross(d, W);
    return ddot(c, c);
}

// The iteration stops early once the path meets the accuracy requirement (§III.B): its AOD
// error, which is Eq. 3's error angle, and its AOA error both <= target.  For an angle
// below pi/2, atan2(sqrt(key), dw) <= target  <=>  key <= dw^2 tan^2(target).
// The AOA is the direction from Rx to the path's last bounce point (a diffraction path's
// edge point Q).  Unfolding is an isometry, so the AOA error is the angle at Rx' between
// X - W and -W, with X the unfolded last point relative to Tx (T_k d for reflections, Q -
// Tx for diffraction: the rotation about the edge fixes Q): the exact last point lies on
// the segment Tx -> Rx'.  tan(AOA error) = |X x W| / (W . W - X . W).  LOS paths have no
// AOA error (their AOA points at Tx for every launch direction).  d is a unit vector.
// Operands by value: P = the unfolded last plane (n'_k, num_k) of a reflection path, W =
// Rx' - Tx, wp = the wedge record of a diffraction path (else null).
__device__ __forceinline__ bool aoa_within64(dvec3 d, D4 P, D4 Wv, const float4 *wp, dvec3 tx, double tan2) {
    dvec3 X;
    if (wp) {
        const float4 A0 = __ldg(wp), B0 = __ldg(wp + 1);
        const dvec3 a = dv(A0.x, A0.y, A0.z), eb = dv(B0.x, B0.y, B0.z) - a, w0 = tx - a;
        const double b = ddot(d, eb), den = ddot(eb, eb) - b * b;
        if (!(den > 0.0)) return false;
        X = eb * ((ddot(eb, w0) - b * ddot(d, w0)) / den) - w0;
    } else {
        X = d * (P.w / ddot(dv(P.x, P.y, P.z), d));
    }
    const dvec3 W = dv(Wv.x, Wv.y, Wv.z), c = dcross(X, W);
    const double h = ddot(W, W) - ddot(X, W);
    return h > 0.0 && ddot(c, c) <= h * h * tan2;
}

__device__ __forceinline__ bool aoa_within32(float3 d, float4 P, float4 Wv, const float4 *wp, float3 tx, float tan2) {
    float3 X;
    if (wp) {
        const float3 a = f3(__ldg(wp)), eb = f3(__ldg(wp + 1)) - a, w0 = tx - a;
        const float b = dot(d, eb), den = dot(eb, eb) - b * b;
        if (!(den > 0.0f)) return false;
        X = eb * ((dot(eb, w0) - b * dot(d, w0)) / den) - w0;
    } else {
        X = d * (P.w / dot(make_float3(P.x, P.y, P.z), d));
    }
    const float3 W = make_float3(Wv.x, Wv.y, Wv.z), c = cross(X, W);
    const float h = dot(W, W) - dot(X, W);
    return h > 0.0f && dot(c, c) <= h * h * tan2;
}

__device__ __forceinline__ bool reached(const RefineArgs &A, const PathGeo &g, const UnfD &ud, dvec3 c, double key,
                                        double dw) {
    if (!(A.target > 0.0 && key < INFINITY && key <= dw * dw * A.tan2_target)) return false;
    if (g.wedge < 0 && g.k == 0) return true;
    const float4 *wp = g.wedge >= 0 ? A.scene.wedges + 4 * (size_t)g.wedge : nullptr;
    return aoa_within64(c, wp ? ud.w : ud.p[g.k - 1], ud.w, wp, g.txd, A.tan2_target);
}

// A stalled path stops: once its error angle exceeds R (1 / (1 - s) + 2 s) + 1e-6 it can
// no longer meet the validity test's convergence condition (2 R_final + 1e-7), because
// later cone centres stay within R / (1 - s) of the current one and the error is the angle
// to the exact direction; valid paths never meet this.  (FP32 is ample against the 1e-6
// margin.)
__device__ __forceinline__ bool stalled(double key, double dw, double R, double stall) {
    if (!(key < INFINITY)) return true;
    return atan2f(sqrtf((float)key), (float)dw) > (float)(R * stall + 1e-6);
}

__device__ __forceinline__ bool reached32(const RefineArgs &A, const PathGeo &g, const UnfF &uf, float3 c, float key,
                                          float dw) {
    if (!(A.target_on && key < INFINITY && key <= dw * dw * A.tan2_target_f)) return false;
    if (g.wedge < 0 && g.k == 0) return true;
    const float4 *wp = g.wedge >= 0 ? A.scene.wedges + 4 * (size_t)g.wedge : nullptr;
    return aoa_within32(c, wp ? uf.w : uf.p[g.k - 1], uf.w, wp, g.tx, A.tan2_target_f);
}

__device__ __forceinline__ bool stalled32(float key, float dw, float Rf, float stall) {
    if (!(key < INFINITY)) return true;
    return atan2f(sqrtf(key), dw) > Rf * stall + 1e-6f;
}

// Why an iteration loop ended before its cap: the accuracy target met, or the error left
// the stall bound (a redundant path); recorded where the loop exits, so that the path's
// flags name the test that stopped it, in the precision it was taken in.
constexpr int kStopNone = 0, kStopReached = 1, kStopStalled = 2;

// Eq. 3 error angle from key and d . W, in the precision of the phase that produced them
__device__ __forceinline__ double error_angle(double key, double dw, float keyf, float dwf, bool fp64) {
    if (fp64) return key < INFINITY ? atan2(sqrt(key), dw) : INFINITY;
    return keyf < INFINITY ? (double)atan2f(sqrtf(keyf), dwf) : INFINITY;
}

// The cone radius R0 s^it of the FP64 phase: R0 = max(theta_launch, rough error), shrunk
// once per iteration in FP64.  (The FP32 phase keeps its own radius in FP32: on GB300
// every FP64 instruction, conversions and compares included, costs 64 times an FP32 one.)
__device__ __forceinline__ double cone_radius64(const RefineArgs &A, float rough_err, int it, double shrink) {
    double R = fmax((double)A.theta_launch, (double)rough_err);
    for (int i = 0; i < it; ++i) R *= shrink;
    return R;
}

// sin and cos of a small angle (|x| <= 1e-3) from their Taylor series; the first omitted
// terms are below 1e-27 of the result
__device__ __forceinline__ void sincos_small(double x, double &s, double &c) {
    const double x2 = x * x;
    s = x * (1.0 - x2 * (1.0 / 6.0) * (1.0 - x2 * (1.0 / 20.0) * (1.0 - x2 * (1.0 / 42.0))));
    c = 1.0 - x2 * 0.5 * (1.0 - x2 * (1.0 / 12.0) * (1.0 - x2 * (1.0 / 30.0)));
}

__device__ __forceinline__ void sincos_sub(double x, double &s, double &c) {
    if (fabs(x) <= 1e-3) sincos_small(x, s, c);
    else sincos(x, &s, &c);
}

// FP32 sine and cosine of a sub-ray's cone angle: for |x| <= 0.03 the Taylor polynomials
// x (1 - x^2/6 + x^4/120) and 1 - x^2/2 + x^4/24 (first omitted terms below 2e-13 of the
// result, far under FP32 rounding); wider cones use sincosf.
__device__ __forceinline__ void sincos_sub32(float x, float &s, float &c) {
    if (fabsf(x) <= 0.03f) {
        const float x2 = x * x;
        s = x * fmaf(x2, fmaf(x2, 1.0f / 120.0f, -1.0f / 6.0f), 1.0f);
        c = fmaf(x2, fmaf(x2, 1.0f / 24.0f, -0.5f), 1.0f);
    } else {
        sincosf(x, &s, &c);
    }
}

// sub-cone frame: u = normalize(c x e), e the world axis with the smallest |c_i| (lowest
// index on ties), v = c x u.  frame_axis* is that axis (0, 1, 2), also written to the
// choice log beside the argmin.
__device__ __forceinline__ int frame_axis32(float3 c) {
    float ax = fabsf(c.x), ay = fabsf(c.y), az = fabsf(c.z);
    return (ay < ax && ay <= az) ? 1 : ((az < ax && az < ay) ? 2 : 0);
}

__device__ __forceinline__ int frame_axis64(dvec3 c) {
    double ax = fabs(c.x), ay = fabs(c.y), az = fabs(c.z);
    return (ay < ax && ay <= az) ? 1 : ((az < ax && az < ay) ? 2 : 0);
}

__device__ __forceinline__ void frame32(float3 c, float3 &u, float3 &v) {
    const int a = frame_axis32(c);
    const float3 e = make_float3(a == 0, a == 1, a == 2);
    u = cross(c, e);
    u = u * (1.0f / sqrtf(dot(u, u)));
    v = cross(c, u);
}

__device__ __forceinline__ void frame64(dvec3 c, dvec3 &u, dvec3 &v) {
    const int a = frame_axis64(c);
    const dvec3 e = dv(a == 0, a == 1, a == 2);
    u = dcross(c, e);
    u = u * (1.0 / dnorm(u));
    v = dcross(c, u);
}

// choice-log entry of one iteration: the argmin sub-ray in bits 0-3, the frame axis in 4-5
__device__ __forceinline__ int8_t choice_entry(int bk, int axis) { return (int8_t)(bk | (axis << 4)); }

// One iteration: returns the chosen sub-ray (or -1 if all are invalid); updates the cone
// centre and its |d x W|^2 and d . W.  The FP32 phase keeps this state in FP32 registers
// (GB300's FP64 pipe runs at 1/64 of the FP32 rate, conversions included).
__device__ __forceinline__ int iterate32(const UnfF &uf, int nk, int K, int off, float Rf, float3 &cf, float &key_c,
                                         float &dw_c) {
    float3 u, v;
    frame32(cf, u, v);
    float best = INFINITY, bdw = 0.0f;
    int bk = -1;
    float3 bd = cf;
    // the patterns' sub-rays come ring by ring: one sine and cosine per ring radius
    float rho = -1.0f, sa = 0.0f, ca = 1.0f;
    for (int k = 0; k < K; ++k) {
        if (c_sub.rho[off + k] != rho) {
            rho = c_sub.rho[off + k];
            sincos_sub32(rho * Rf, sa, ca);
        }
        float3 dk = cf * ca + (u * c_sub.cphi[off + k] + v * c_sub.sphi[off + k]) * sa;
        float dw = 0.0f;
        float key = key32(uf, nk, dk, dw);
        if (key < best) {
            best = key;
            bdw = dw;
            bk = k;
            bd = dk;
        }
    }
    if (bk >= 0) {
        float inv = 1.0f / sqrtf(dot(bd, bd));
        cf = bd * inv;
        key_c = best;
        dw_c = bdw;
    }
    return bk;
}

__device__ __forceinline__ int iterate64(const UnfD &ud, int nk, int K, int off, double R, dvec3 &c, double &key_c,
                                         double &dw_c) {
    dvec3 u, v;
    frame64(c, u, v);
    double best = INFINITY, bdw = 0.0;
    int bk = -1;
    dvec3 bd = c;
    double rho = -1.0, sa = 0.0, ca = 1.0;
    for (int k = 0; k < K; ++k) {
        if (c_sub.rho_d[off + k] != rho) {
            rho = c_sub.rho_d[off + k];
            sincos_sub(rho * R, sa, ca);
        }
        dvec3 dk = c * ca + (u * c_sub.cphi_d[off + k] + v * c_sub.sphi_d[off + k]) * sa;
        double dw = 0.0;
        double key = key64(ud, nk, dk, dw);
        // key < best, both >= 0 (or +inf): their bits order like the values
        if (__double_as_longlong(key) < __double_as_longlong(best)) {
            best = key;
            bdw = dw;
            bk = k;
            bd = dk;
        }
    }
    if (bk >= 0) {
        c = bd * (1.0 / dnorm(bd));
        key_c = best;
        dw_c = bdw;
    }
    return bk;
}

// ----------------------------------------------------------------------------- a7/a8
// p lies in (or on the boundary of) face f's convex outline: every edge function
// cross(b - a, p - a) . n of the counter-clockwise corners is >= 0.  FP32 with the
// triangle test's rounding band below; a sign inside the band is decided in FP64.
__device__ __noinline__ bool point_in_outline(const SceneDev &S, int f, int2 ol, const df3 &pd) {
    const float3 nf = f3(__ldg(S.planes + f));
    const float3 P = df3_round(pd);
    const float pn = fabsf(P.x) + fabsf(P.y) + fabsf(P.z) + 1.0f;
    const float4 *cv = S.outline_v + ol.x;
    bool unsure = false;
    float3 a = f3(__ldg(cv + ol.y - 1));
    for (int i = 0; i < ol.y; ++i) {
        const float3 b = f3(__ldg(cv + i));
        const float3 e = b - a, q = P - a;
        const float s = dot(cross(e, q), nf);
        if (fabsf(s) > 1e-5f * sqrtf(dot(e, e)) * (pn + fabsf(q.x) + fabsf(q.y) + fabsf(q.z))) {
            if (s < 0.0f) return false;
        } else {
            unsure = true;
        }
        a = b;
    }
    if (!unsure) return true;
    const dvec3 p = df3_double(pd);
    const Plane64 pl = S.planes_d[f];
    const dvec3 n = dv(pl.x, pl.y, pl.z);
    float4 a4 = __ldg(cv + ol.y - 1);
    dvec3 ad = dv(a4.x, a4.y, a4.z);
    for (int i = 0; i < ol.y; ++i) {
        const float4 b4 = __ldg(cv + i);
        const dvec3 bd = dv(b4.x, b4.y, b4.z);
        if (ddot(dcross(bd - ad, p - ad), n) < 0.0) return false;
        ad = bd;
    }
    return true;
}

__device__ __forceinline__ bool point_in_face(const SceneDev &S, int f, const df3 &pd) {
    const int2 ol = __ldg(S.face_outline + f);
    if (ol.y > 0) return point_in_outline(S, f, ol, pd);
    const float3 nf = f3(__ldg(S.planes + f));   // the FP64 normal rounded to FP32
    const float3 Pf = df3_round(pd);
    const float px = Pf.x, py = Pf.y, pz = Pf.z;
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
                if (SBR_CHECKED_ON && sp >= min(S.stack_limit, kStackDepth)) {
                    check_fail(S, SBR_CHECK_BVH2_STACK);
                    return false;
                }
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
                // edge functions in FP32; a sign outside a generous rounding bound of zero
                // (1e-5 x |edge| x (|p| + |p - vertex| + 1), 1-norms) is the FP64 sign.  Two
                // such signs that differ put p outside; three that agree put it inside; any
                // other case is decided in FP64.
                const float3 P = make_float3(px, py, pz);
                const float3 ab = f3(B) - f3(A), bc = f3(C) - f3(B), ca = f3(A) - f3(C);
                const float3 pa = P - f3(A), pb = P - f3(B), pc = P - f3(C);
                const float ea = dot(cross(ab, pa), nf);
                const float eb = dot(cross(bc, pb), nf);
                const float ec = dot(cross(ca, pc), nf);
                const float pn = fabsf(px) + fabsf(py) + fabsf(pz) + 1.0f;
                auto bound = [&](float3 e, float3 q) {
                    return 1e-5f * sqrtf(dot(e, e)) * (pn + fabsf(q.x) + fabsf(q.y) + fabsf(q.z));
                };
                const bool sa = fabsf(ea) > bound(ab, pa), sb = fabsf(eb) > bound(bc, pb), sc = fabsf(ec) > bound(ca, pc);
                const bool pos = (sa && ea > 0.0f) || (sb && eb > 0.0f) || (sc && ec > 0.0f);
                const bool neg = (sa && ea < 0.0f) || (sb && eb < 0.0f) || (sc && ec < 0.0f);
                if (pos && neg) continue;
                if (sa && sb && sc) return true;
                const Plane64 pl = S.planes_d[f];
                const dvec3 n = dv(pl.x, pl.y, pl.z);
                const dvec3 p = df3_double(pd);
                dvec3 a = dv(A.x, A.y, A.z), b = dv(B.x, B.y, B.z), c = dv(C.x, C.y, C.z);
                double da = ddot(dcross(b - a, p - a), n);
                double db = ddot(dcross(c - b, p - b), n);
                double dc = ddot(dcross(a - c, p - c), n);
                if ((da >= 0 && db >= 0 && dc >= 0) || (da <= 0 && db <= 0 && dc <= 0)) return true;
            }
        }
        if (sp == 0) break;
        node = stack[--sp];
    }
    return false;
}

// |Gamma_perp| of a Fresnel reflection at incidence cosine ci on relative permittivity eps
__device__ __forceinline__ float fresnel_perp_abs(float ci, float eps) {
    float r = sqrtf(eps - (1.0f - ci * ci));
    return fabsf((ci - r) / (ci + r));
}

// (azimuth, elevation) of v; the record stores them in FP32
__device__ __forceinline__ void az_el(dvec3 v, float *out) {
    const float x = (float)v.x, y = (float)v.y, z = (float)v.z;
    out[0] = atan2f(y, x);
    out[1] = atan2f(z, sqrtf(x * x + y * y));
}

// The refined ray's walk through the path's fixed planes for the validity test and the
// outputs, in compensated FP32 pairs (dfloat.cuh, about 44 bits): bounce point o_j, den_j =
// n_j . d_j (the incidence cosine up to sign), leg direction d_j and the sum of the segment
// parameters t_j (each leg is t_j d_j with |d_j| = |c|: mirroring keeps the length).  The
// per-thread and group forms repeat the walk as they need its points (the arithmetic is
// deterministic, so every repetition gives the same points), which keeps the points out
// of local memory and the walk off GB300's 1/64-rate FP64 pipe.
struct BounceWalk {
    df3 o, d;
    df tsum;
    __device__ __forceinline__ void start(const PathGeo &g, dvec3 c) {
        o = df3_of(g.tx);
        d = {df_from_double(c.x), df_from_double(c.y), df_from_double(c.z)};
        tsum = df_of(0.0f);
    }
    // the bounce on face f; false if the segment length is not positive
    __device__ __forceinline__ bool step(const SceneDev &S, int f, df &den) {
        df3 n;
        df h;
        plane_df(S, f, n, h);
        den = df_dot(n, d);
        if (den.hi == 0.0f) return false;
        const df t = df_div(df_sub(h, df_dot(n, o)), den);
        if (!(t.hi > 0.0f)) return false;
        tsum = df_add(tsum, t);
        o = df3_add_scaled(o, t, d);
        d = df3_sub_scaled(d, df_scale2(den, 2.0f), n);
        return true;
    }
};

// First pass of the validity test and the outputs: the whole walk.  Returns false (trace
// failure) if a segment length is not positive; else the last bounce point (Tx for LOS),
// the last leg's direction, sum t_j and the Fresnel reflection loss (dB, FP32).
__device__ __forceinline__ bool walk_path(const RefineArgs &A, const PathGeo &g, dvec3 c, df3 &last, df3 &d_last,
                                          df &tsum, float &gain_db) {
    BounceWalk w;
    w.start(g, c);
    gain_db = 0.0f;
    for (int j = 0; j < g.k; ++j) {
        df den;
        if (!w.step(A.scene, g.faces[j], den)) return false;
        const float eps = __ldg(A.scene.face_eps + g.faces[j]);
        if (eps > 0.0f) gain_db += 20.0f * log10f(fresnel_perp_abs(fabsf(df_round(den)), eps));
    }
    last = w.o;
    d_last = w.d;
    tsum = w.tsum;
    return true;
}

// Rx is received on the last leg: its foot lies ahead of the last bounce point
__device__ __forceinline__ bool rx_ahead(const PathGeo &g, const df3 &last, const df3 &d_last) {
    return df_dot(df3_sub(df3_of(g.rx), last), d_last).hi > 0.0f;
}

// a8 outputs of a walked path: delay = polyline length / c0 with the legs up to the last
// bounce point as |c| sum t_j and the last one from its end points; AOD, AOA and power =
// ptx + free-space loss + Fresnel reflection losses in FP32, as the record stores them
__device__ __forceinline__ void path_outputs(const RefineArgs &A, const PathGeo &g, dvec3 c, const df3 &last,
                                             df tsum, float gain_db, sbr_path_record &p) {
    const df3 cd = {df_from_double(c.x), df_from_double(c.y), df_from_double(c.z)};
    const df3 v = df3_sub(last, df3_of(g.rx));
    df len = df_sqrt(df_dot(v, v));
    if (g.k > 0) len = df_add(len, df_mul(tsum, df_sqrt(df_dot(cd, cd))));
    const df c0 = {299792448.0f, 10.0f};   // 299792458 m/s as an exact pair
    p.delay = df_to_double(df_div(len, c0));
    az_el(c, p.aod);
    az_el(dv(df_round(v.x), df_round(v.y), df_round(v.z)), p.aoa);
    const float lam = (float)(kC0 / A.freq);
    p.power_dbm = (float)A.ptx_dbm + 20.0f * log10f(lam / (4.0f * 3.14159265f * df_round(len))) + gain_db;
}

// Upper bound on the final error angle of a refined path whose exact direction lies in
// its cone: twice the Eq. 10 bound R0 * s^iters (R_final) plus the FP32 evaluation floor.
// A redundant path received through the cone's width for a face sequence without a
// specular solution stalls far above it and is rejected by the validity test.
__device__ __forceinline__ double converged_bound(int iters, double R_final) {
    return iters > 0 ? 2.0 * R_final + 1e-7 : INFINITY;
}

// a7/a8 for a diffraction path: the diffraction point Q is the point of the edge line
// closest to the launched ray; valid iff Q lies on the edge segment and ahead of Tx, Tx and
// Rx lie in the wedge's exterior, the refinement converged, and Tx -> Q and Q -> Rx are
// unblocked (the wedge's faces excluded).  delay = (|Q - Tx| + |Rx - Q|) / c0, AOD = c,
// AOA = Q - Rx, power = ptx + free-space loss (no diffraction coefficient).
__device__ void wedge_finalize(const RefineArgs &A, const PathGeo &g, dvec3 c, sbr_path_record &p,
                               double err_bound) {
    const SceneDev &S = A.scene;
    const WedgeD w = wedge64(S, g.wedge);
    const dvec3 eb = w.b - w.a, w0 = g.txd - w.a;
    const double Ac = ddot(c, c), B = ddot(c, eb), C = ddot(eb, eb), D = ddot(c, w0), E = ddot(eb, w0);
    const double den = Ac * C - B * B;
    const double u = den != 0.0 ? (Ac * E - B * D) / den : -1.0;
    const double sq = den != 0.0 ? (B * E - C * D) / den : -1.0;
    const dvec3 Q = w.a + eb * u;
    const dvec3 e = eb * (1.0 / sqrt(C));
    bool valid = u >= 0.0 && u <= 1.0 && sq > 0.0 && exterior64(w, e, g.txd) && exterior64(w, e, g.rxd) &&
                 p.err <= err_bound;
    for (int j = 0; j < 2 && valid; ++j) {
        dvec3 from = j == 0 ? g.txd : Q, seg = (j == 0 ? Q : g.rxd) - from;
        RayPre r = make_ray(make_float3((float)from.x, (float)from.y, (float)from.z),
                            make_float3((float)seg.x, (float)seg.y, (float)seg.z));
        if (any_hit4(S, r, 1e-6f, 1.0f - 1e-6f, w.f1, w.f2)) valid = false;
    }
    const double len = dnorm(Q - g.txd) + dnorm(g.rxd - Q);
    p.valid = valid ? 1 : 0;
    p.delay = len / kC0;
    az_el(c, p.aod);
    az_el(Q - g.rxd, p.aoa);
    const float lam = (float)(kC0 / A.freq);
    p.power_dbm = (float)A.ptx_dbm + 20.0f * log10f(lam / (4.0f * 3.14159265f * (float)len));
    p.flags |= SBR_PATH_DIFFRACTED;
}

// Validity test and outputs for launch direction c; writes the result fields of p.
__device__ void finalize_path(const RefineArgs &A, const PathGeo &g, dvec3 c, sbr_path_record &p, double err_bound) {
    const SceneDev &S = A.scene;
    if (g.wedge >= 0) {
        wedge_finalize(A, g, c, p, err_bound);
        return;
    }
    df3 last, dl;
    df tsum;
    float gain_db;
    if (!walk_path(A, g, c, last, dl, tsum, gain_db)) {
        p.valid = 0;
        p.flags |= SBR_PATH_TRACE_FAIL;
        p.delay = 0.0;
        return;
    }
    // Rx must be received on the last leg and the refinement must have converged
    bool valid = rx_ahead(g, last, dl) && p.err <= err_bound;
    // the outputs need only the first pass: computed now, so that its results are not
    // held in registers through the occlusion queries
    path_outputs(A, g, c, last, tsum, gain_db, p);
    // Second pass: the walk again, each bounce point tested on its face and each leg for
    // occlusion as it is reached.  The lanes that arrive here together run the queries in
    // lockstep: loop bounds made uniform over them, a lane that has failed a test idles
    // through the rest, so that the lanes execute the same traversal code at the same time.
    const unsigned m = __activemask();
    const int kk = __reduce_max_sync(m, g.k);
    BounceWalk w;
    w.start(g, c);
    for (int j = 0; j <= kk; ++j) {
        if (!__any_sync(m, valid)) break;
        if (!valid || j > g.k) continue;
        const df3 from = w.o;
        df den;
        if (j < g.k) {
            w.step(S, g.faces[j], den);   // succeeded in the first pass
            if (!point_in_face(S, g.faces[j], w.o)) {
                valid = false;
                continue;
            }
        }
        const df3 to = j < g.k ? w.o : df3_of(g.rx);
        const int fa = j == 0 ? -1 : g.faces[j - 1];
        const int fb = j == g.k ? -1 : g.faces[j];
        const RayPre r = make_ray(df3_round(from), df3_round(df3_sub(to, from)));
        if (any_hit4(S, r, 1e-6f, 1.0f - 1e-6f, fa, fb)) valid = false;
    }
    p.valid = valid ? 1 : 0;
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
    const float shrinkf = c_sub.shrink_f[A.K];
    const double stall = 1.0 / (1.0 - shrink) + 2.0 * shrink;
    const float stallf = (float)stall;
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
        UnfD ud;
        UnfF uf;
        build_unf(A.scene, g, ud, uf);
        // FP32 phase while the cone radius is >= fp64_below (the radius R0 = max(theta_launch,
        // rough error) is a float, so the first test is exact)
        float Rf = fmaxf(A.theta_launch, p.rough_err);
        bool fp64 = Rf < A.fp64_below_f, fail = false;
        float3 cf = make_float3((float)p.dir[0], (float)p.dir[1], (float)p.dir[2]);
        float keyf = INFINITY, dwf = 0.0f;
        int it = 0, flags = 0, stop = kStopNone;
        if (!fp64) {
            keyf = key32(uf, g.k, cf, dwf);
            while (it < A.max_iters) {
                if (reached32(A, g, uf, cf, keyf, dwf)) {
                    stop = kStopReached;
                    break;
                }
                if (stalled32(keyf, dwf, Rf, stallf)) {
                    stop = kStopStalled;
                    break;
                }
                if (Rf < A.fp64_below_f) break;   // on to the FP64 iterations
                const int ax = A.choice_log ? frame_axis32(cf) : 0;
                const int bk = iterate32(uf, g.k, A.K, off, Rf, cf, keyf, dwf);
                if (bk < 0) {
                    fail = true;
                    break;
                }
                if (A.choice_log) A.choice_log[pi * A.max_iters + it] = choice_entry(bk, ax);
                Rf *= shrinkf;
                ++it;
            }
        }
        dvec3 c = dv(cf.x, cf.y, cf.z);
        double key = INFINITY, dw = 0.0;
        if (!fail && Rf < A.fp64_below_f) {
            double R = cone_radius64(A, p.rough_err, it, shrink);
            if (fp64) {
                c = dv(p.dir[0], p.dir[1], p.dir[2]);
                key = key64(ud, g.k, c, dw);
            } else {
                key = keyf;
                dw = dwf;
            }
            stop = kStopNone;   // the FP64 phase judges the state again
            while (it < A.max_iters) {
                if (reached(A, g, ud, c, key, dw)) {
                    stop = kStopReached;
                    break;
                }
                if (stalled(key, dw, R, stall)) {
                    stop = kStopStalled;
                    break;
                }
                const int ax = A.choice_log ? frame_axis64(c) : 0;
                const int bk = iterate64(ud, g.k, A.K, off, R, c, key, dw);
                if (bk < 0) {
                    fail = true;
                    break;
                }
                flags |= SBR_PATH_FP64;
                fp64 = true;
                if (A.choice_log) A.choice_log[pi * A.max_iters + it] = choice_entry(bk, ax);
                R *= shrink;
                ++it;
            }
        }
        if (fail) flags |= SBR_PATH_TRACE_FAIL;
        else if (stop == kStopStalled) flags |= SBR_PATH_STALLED;
        p.iters = it;
        p.flags = flags | (it > 0 ? SBR_PATH_REFINED : 0);
        p.dir[0] = c.x;
        p.dir[1] = c.y;
        p.dir[2] = c.z;
        p.err = error_angle(key, dw, keyf, dwf, fp64);
        finalize_path(A, g, c, p, converged_bound(it, cone_radius64(A, p.rough_err, it, shrink)));
        store_result(A.paths + pi, p);
    }
}

// Lists path pi in its order group for batch_finalize_kernel (group offsets from
// batch_unfold_kernel's counts), so that a warp there holds paths of one order.  Inside the
// group, paths whose error meets the convergence bound 2 R + 1e-7 (the validity test's
// condition; R is the cone radius after the iterations, here only an ordering hint) fill it
// from the front and the others, which the validity test rejects at once, from the back:
// a warp's lanes then run their BVH queries, or skip them, together.
__device__ __forceinline__ void list_for_finalize(const RefineArgs &A, const PathGeo &g, long long pi, double err,
                                                  double R) {
    const int grp = order_group(g);
    unsigned long long at = 0;
    for (int b = 0; b < grp; ++b) at += A.order_cnt[b];
    if (err <= 2.0 * R + 1e-7) at += atomicAdd(A.order_cnt + 16 + grp, 1ULL);
    else at += A.order_cnt[grp] - 1ULL - atomicAdd(A.order_cnt + 48 + grp, 1ULL);
    A.order_idx[at] = (int)pi;
}

// a9: persistent work-queue form.  A group of G lanes (G = 1, 8, 16 or 32) owns one path at
// a time: lane l evaluates the sub-rays k = l, l + G, ... of each iteration and the group
// takes the argmin with shuffles (lowest k on ties, as in the plain form; one lane runs
// the plain form's iterate32).  When a path is finished (iteration cap, target reached,
// stalled, or all sub-rays invalid) the group takes the next path index from the device
// queue head with one atomic, so paths that stop early free their group at once.  With
// many paths, a path whose cone falls below the FP64 threshold moves on to
// batch_refine64_kernel; the validity test and outputs follow in batch_finalize_kernel.
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
__device__ __forceinline__ int group_iterate32(const UnfF &uf, int nk, int K, int off, float Rf, float3 &cf,
                                               float &key_c, float &dw_c, int gl, unsigned gmask) {
    float3 u, v;
    frame32(cf, u, v);
    float best = INFINITY;
    int bk = 0x7fffffff;
    for (int k = gl; k < K; k += G) {
        float sa, ca;
        sincos_sub32(c_sub.rho[off + k] * Rf, sa, ca);
        float3 dk = cf * ca + (u * c_sub.cphi[off + k] + v * c_sub.sphi[off + k]) * sa;
        float dw;
        float key = key32(uf, nk, dk, dw);
        if (key < best) {
            best = key;
            bk = k;
        }
    }
    group_argmin<G>(best, bk, gmask);
    if (!(best < INFINITY)) return -1;
    // every lane rebuilds the winning direction (same arithmetic as the lane that found it)
    float sa, ca;
    sincos_sub32(c_sub.rho[off + bk] * Rf, sa, ca);
    float3 bd = cf * ca + (u * c_sub.cphi[off + bk] + v * c_sub.sphi[off + bk]) * sa;
    float dw = 0.0f;
    float key = key32(uf, nk, bd, dw);
    float inv = 1.0f / sqrtf(dot(bd, bd));
    cf = bd * inv;
    key_c = key;
    dw_c = dw;
    return bk;
}

template <int G>
__device__ __forceinline__ int group_iterate64(const UnfD &ud, int nk, int K, int off, double R, dvec3 &c,
                                               double &key_c, double &dw_c, int gl, unsigned gmask) {
    dvec3 u, v;
    frame64(c, u, v);
    double best = INFINITY;
    int bk = 0x7fffffff;
    for (int k = gl; k < K; k += G) {
        double sa, ca;
        sincos_sub(c_sub.rho_d[off + k] * R, sa, ca);
        dvec3 dk = c * ca + (u * c_sub.cphi_d[off + k] + v * c_sub.sphi_d[off + k]) * sa;
        double dw;
        double key = key64(ud, nk, dk, dw);
        if (key < best) {
            best = key;
            bk = k;
        }
    }
    group_argmin64<G>(best, bk, gmask);
    if (!(best < INFINITY)) return -1;
    double sa, ca;
    sincos_sub(c_sub.rho_d[off + bk] * R, sa, ca);
    dvec3 bd = c * ca + (u * c_sub.cphi_d[off + bk] + v * c_sub.sphi_d[off + bk]) * sa;
    double dw = 0.0;
    double key = key64(ud, nk, bd, dw);
    c = bd * (1.0 / dnorm(bd));
    key_c = key;
    dw_c = dw;
    return bk;
}

// Validity and outputs with the per-bounce / per-segment queries spread over the group.
// Lane 0 traces the bounce points once (FP64) and shares them through the group's slot
// of shared memory (sh.p[j] = (p_j, den_j), sh.w = (direction of the last leg, sum of
// the segment parameters, or -1 if the trace failed)).
template <int G>
__device__ void group_finalize(const RefineArgs &A, const PathGeo &g, dvec3 c, sbr_path_record &p, int gl,
                               unsigned gmask, double err_bound, UnfD &sh) {
    const SceneDev &S = A.scene;
    if (g.wedge >= 0) {   // group-uniform: one path per group
        if (gl == 0) wedge_finalize(A, g, c, p, err_bound);
        return;
    }
    // every lane walks the path (the same compensated-FP32 arithmetic as the per-thread
    // form, so the same points); then lane j tests bounce point j on its face and leg j for
    // occlusion, walking to it again
    df3 last, dl;
    df tsum;
    float gain_db;
    if (!walk_path(A, g, c, last, dl, tsum, gain_db)) {
        p.valid = 0;
        p.flags |= SBR_PATH_TRACE_FAIL;
        p.delay = 0.0;
        return;
    }
    // Rx must be received on the last leg and the refinement must have converged
    bool valid = rx_ahead(g, last, dl) && p.err <= err_bound;
    bool mine_ok = true;
    if (valid) {
        for (int j = gl; j <= g.k && mine_ok; j += G) {
            BounceWalk w;
            w.start(g, c);
            df den;
            for (int i = 0; i < j; ++i) w.step(S, g.faces[i], den);
            const df3 from = w.o;
            if (j < g.k) {
                w.step(S, g.faces[j], den);
                mine_ok = point_in_face(S, g.faces[j], w.o);
                if (!mine_ok) break;
            }
            const df3 to = j < g.k ? w.o : df3_of(g.rx);
            const int fa = j == 0 ? -1 : g.faces[j - 1];
            const int fb = j == g.k ? -1 : g.faces[j];
            const RayPre r = make_ray(df3_round(from), df3_round(df3_sub(to, from)));
            if (any_hit4(S, r, 1e-6f, 1.0f - 1e-6f, fa, fb)) mine_ok = false;
        }
        valid = __all_sync(gmask, mine_ok);
    }
    p.valid = valid ? 1 : 0;
    if (gl == 0) path_outputs(A, g, c, last, tsum, gain_db, p);
}

// At most 85 registers a thread, so that three 256-thread blocks fit on an SM (measured
// faster than the uncapped 124-128 registers of the 8- and 32-lane forms).
// G = 1 is the one-lane form: each thread evaluates all K sub-rays of its own path (no
// shuffles, no re-evaluation of the winner) and always runs with batch_unfold_kernel and
// the FP64 tail kernel (the host sets split_min = 0 for it).
template <int G>
__global__ void __launch_bounds__(256, 3) batch_refine_kernel(RefineArgs A) {
    // the unfolded planes of each group's current path (shared by its G lanes)
    __shared__ UnfD s_ud[G == 1 ? 1 : 256 / G];
    __shared__ UnfF s_uf[256 / G];
    UnfD &ud = s_ud[G == 1 ? 0 : threadIdx.x / G];   // unused by the one-lane form
    UnfF &uf = s_uf[threadIdx.x / G];
    const long long total = path_count(A);
    // batch_unfold_kernel ran (the one-lane form always runs with it: split_min = 0)
    const bool prebuilt = G == 1 || total >= A.split_min;
    const int off = c_sub.off[A.K];
    const double shrink = c_sub.shrink[A.K];
    const float shrinkf = c_sub.shrink_f[A.K];
    const double stall = 1.0 / (1.0 - shrink) + 2.0 * shrink;
    const float stallf = (float)stall;
    const int lane = threadIdx.x & 31;
    const int gl = lane % G;
    const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane - gl));
    for (;;) {
        unsigned long long q = 0;
        if (G == 1) {
            // the lanes that finished a path together take consecutive indices with one atomic
            const unsigned m = __activemask();
            const int leader = __ffs(m) - 1;
            if (lane == leader)
                q = atomicAdd(reinterpret_cast<unsigned long long *>(A.counters + kBatchHead),
                              (unsigned long long)__popc(m));
            q = __shfl_sync(m, q, leader) + __popc(m & ((1u << lane) - 1u));
        } else {
            if (gl == 0) q = atomicAdd(reinterpret_cast<unsigned long long *>(A.counters + kBatchHead), 1ULL);
            q = __shfl_sync(gmask, q, 0, G);
        }
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
        // the path's unfolded planes and W into the group's shared slot: with many paths
        // the FP32 copy computed by batch_unfold_kernel, with few computed here in FP64 by
        // lanes 0..k-1 (one plane each) and lane G-1 (the receiver; k <= 8 <= G).  The
        // previous path's data is no longer read once every lane has reached this point.
        __syncwarp(gmask);
        float3 cf;
        if (prebuilt) {
            for (int j = gl; j <= kMaxOrder; j += G)
                if (j < g.k || j == kMaxOrder) (j < kMaxOrder ? uf.p[j] : uf.w) = A.unf[kUnfStride * pi + j];
            cf = f3(A.unf[kUnfStride * pi + kMaxOrder + 1]);
        } else {
            for (int j = gl; j < g.k; j += G) {
                ud.p[j] = unfold_plane(A.scene, g, j);
                uf.p[j] = unfold_plane32(A.scene, g, j);
            }
            if (gl == G - 1) {
                ud.w = unfold_rx(A.scene, g);
                uf.w = unfold_rx32(A.scene, g);
            }
            cf = make_float3((float)p.dir[0], (float)p.dir[1], (float)p.dir[2]);
        }
        __syncwarp(gmask);
        // FP32 phase, every operand in FP32 (see cone_radius64); state identical in the G lanes
        float Rf = fmaxf(A.theta_launch, p.rough_err);
        bool fp64 = Rf < A.fp64_below_f, fail = false;
        float keyf = INFINITY, dwf = 0.0f;
        int it = 0, flags = 0, stop = kStopNone;
        if (!fp64) {
            keyf = key32(uf, g.k, cf, dwf);
            while (it < A.max_iters) {
                if (reached32(A, g, uf, cf, keyf, dwf)) {
                    stop = kStopReached;
                    break;
                }
                if (stalled32(keyf, dwf, Rf, stallf)) {
                    stop = kStopStalled;
                    break;
                }
                if (Rf < A.fp64_below_f) break;   // on to the FP64 iterations
                const int ax = A.choice_log ? frame_axis32(cf) : 0;
                const int bk = G == 1 ? iterate32(uf, g.k, A.K, off, Rf, cf, keyf, dwf)
                                      : group_iterate32<G>(uf, g.k, A.K, off, Rf, cf, keyf, dwf, gl, gmask);
                if (bk < 0) {
                    fail = true;
                    break;
                }
                if (A.choice_log && gl == 0) A.choice_log[pi * A.max_iters + it] = choice_entry(bk, ax);
                Rf *= shrinkf;
                ++it;
            }
        }
        dvec3 c;
        double key = INFINITY, dw = 0.0;
        if (!fail && Rf < A.fp64_below_f && prebuilt) {
            // many paths: the FP64 iterations run in batch_refine64_kernel, one thread per
            // path.  The record keeps the iterations done; the path's unf slot keeps the
            // cone centre and |d x W|^2 of the FP32 phase, the record's err field d . W.
            // Listed by order group (group offsets from batch_unfold_kernel's counts), so that
            // the tail kernel's warps run paths of one order.
            if (gl == 0) {
                sbr_path_record *dst = A.paths + pi;
                dst->iters = it;
                dst->err = dwf;
                A.unf[kUnfStride * pi + kMaxOrder + 1] = make_float4(cf.x, cf.y, cf.z, keyf);
                const int grp = order_group(g);
                unsigned long long at = 0;
                for (int b = 0; b < grp; ++b) at += A.order_cnt[b];
                at += atomicAdd(A.order_cnt + 32 + grp, 1ULL);
                A.fp64_idx[at] = (int)pi;
            }
            continue;
        }
        if (G != 1 && !fail && Rf < A.fp64_below_f) {
            double R = cone_radius64(A, p.rough_err, it, shrink);
            if (fp64) {
                c = dv(p.dir[0], p.dir[1], p.dir[2]);
                key = key64(ud, g.k, c, dw);
            } else {
                c = dv(cf.x, cf.y, cf.z);
                key = keyf;
                dw = dwf;
            }
            stop = kStopNone;   // the FP64 phase judges the state again
            while (it < A.max_iters) {
                if (reached(A, g, ud, c, key, dw)) {
                    stop = kStopReached;
                    break;
                }
                if (stalled(key, dw, R, stall)) {
                    stop = kStopStalled;
                    break;
                }
                const int ax = A.choice_log ? frame_axis64(c) : 0;
                const int bk = group_iterate64<G>(ud, g.k, A.K, off, R, c, key, dw, gl, gmask);
                if (bk < 0) {
                    fail = true;
                    break;
                }
                flags |= SBR_PATH_FP64;
                fp64 = true;
                if (A.choice_log && gl == 0) A.choice_log[pi * A.max_iters + it] = choice_entry(bk, ax);
                R *= shrink;
                ++it;
            }
        }
        if (fail) flags |= SBR_PATH_TRACE_FAIL;
        else if (stop == kStopStalled) flags |= SBR_PATH_STALLED;
        if (gl == 0) {
            if (!fp64) c = dv(cf.x, cf.y, cf.z);
            p.iters = it;
            p.flags = flags | (it > 0 ? SBR_PATH_REFINED : 0);
            p.dir[0] = c.x;
            p.dir[1] = c.y;
            p.dir[2] = c.z;
            p.err = error_angle(key, dw, keyf, dwf, fp64);
            if (prebuilt) list_for_finalize(A, g, pi, p.err, (double)Rf);
            // iteration results; the validity test and outputs follow in batch_finalize_kernel
            sbr_path_record *dst = A.paths + pi;
            dst->iters = p.iters;
            dst->dir[0] = p.dir[0];
            dst->dir[1] = p.dir[1];
            dst->dir[2] = p.dir[2];
            dst->err = p.err;
            dst->flags = p.flags;
        }
    }
}

// Batched form, FP64 tail (from split_min paths on), one thread per path: the paths whose
// cone fell below fp64_below in batch_refine_kernel continue here with the plain form's
// FP64 iterations (iterate64, all K sub-rays in one thread), so that each instruction of
// GB300's narrow FP64 pipe serves 32 paths, where a lane group serves one.  The state
// carried over, and the arithmetic, are those of the in-group FP64 phase: a path that
// started in FP64 (no iteration done) takes its FP64 rough direction; otherwise the FP32
// phase's centre with its |d x W|^2 and d . W.  The path is then listed in its order group
// for batch_finalize_kernel.
__global__ void __launch_bounds__(128) batch_refine64_kernel(RefineArgs A) {
    // the list holds group b's n_b paths from the group's offset (the sizes of groups < b)
    long long n = 0;
    for (int b = 0; b < 10; ++b) n += A.order_cnt[32 + b];
    const int off = c_sub.off[A.K];
    const double shrink = c_sub.shrink[A.K];
    const double stall = 1.0 / (1.0 - shrink) + 2.0 * shrink;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        long long slot = t, base = 0;
        for (int b = 0; b < 10; ++b) {
            const long long nb = (long long)A.order_cnt[32 + b];
            if (slot < nb) break;
            slot -= nb;
            base += (long long)A.order_cnt[b];
        }
        const long long pi = A.fp64_idx[base + slot];
        sbr_path_record p = A.paths[pi];
        PathGeo g;
        load_path(A, p, g);
        UnfD ud;
        const float4 *u = A.unf + kUnfStride * pi;
        for (int j = 0; j < g.k; ++j) ud.p[j] = unfold_plane(A.scene, g, j);
        ud.w = unfold_rx(A.scene, g);
        const float4 cu = u[kMaxOrder + 1];
        const float3 cf = f3(cu);
        const float keyf = cu.w, dwf = (float)p.err;
        int it = p.iters, flags = 0;
        bool fp64 = it == 0, fail = false;
        double R = cone_radius64(A, p.rough_err, it, shrink);
        dvec3 c;
        double key, dw = 0.0;
        if (fp64) {
            c = dv(p.dir[0], p.dir[1], p.dir[2]);
            key = key64(ud, g.k, c, dw);
        } else {
            c = dv(cf.x, cf.y, cf.z);
            key = keyf;
            dw = dwf;
        }
        int stop = kStopNone;
        while (it < A.max_iters) {
            if (reached(A, g, ud, c, key, dw)) {
                stop = kStopReached;
                break;
            }
            if (stalled(key, dw, R, stall)) {
                stop = kStopStalled;
                break;
            }
            const int ax = A.choice_log ? frame_axis64(c) : 0;
            const int bk = iterate64(ud, g.k, A.K, off, R, c, key, dw);
            if (bk < 0) {
                fail = true;
                break;
            }
            flags |= SBR_PATH_FP64;
            fp64 = true;
            if (A.choice_log) A.choice_log[pi * A.max_iters + it] = choice_entry(bk, ax);
            R *= shrink;
            ++it;
        }
        if (fail) flags |= SBR_PATH_TRACE_FAIL;
        else if (stop == kStopStalled) flags |= SBR_PATH_STALLED;
        if (!fp64) c = dv(cf.x, cf.y, cf.z);
        const double err = error_angle(key, dw, keyf, dwf, fp64);
        list_for_finalize(A, g, pi, err, R);
        sbr_path_record *dst = A.paths + pi;
        dst->iters = it;
        dst->dir[0] = c.x;
        dst->dir[1] = c.y;
        dst->dir[2] = c.z;
        dst->err = err;
        dst->flags = flags | (it > 0 ? SBR_PATH_REFINED : 0);
    }
}

// Batched form, first pass (from split_min paths on), one thread per path: the FP64
// unfolding of the path's face planes into Tx's space and of the receiver (the same
// arithmetic as the plain form's build_unf), stored rounded to FP32 for the iteration
// kernel, with the rough launch direction rounded to FP32.  GB300 runs FP64 at 1/64 of
// the FP32 rate; with one path per lane every FP64 instruction serves 32 paths, where the
// iteration kernel's lane groups would serve one.
// It also counts the paths of each order group so that the iteration kernel can list them
// group by group for the finalize kernel.
__global__ void __launch_bounds__(128) batch_unfold_kernel(RefineArgs A) {
    __shared__ unsigned hist[10];
    const long long total = path_count(A);
    if (total < A.split_min) return;   // few paths: the iteration kernel unfolds them itself
    if (threadIdx.x < 10) hist[threadIdx.x] = 0;
    __syncthreads();
    for (long long pi = blockIdx.x * (long long)blockDim.x + threadIdx.x; pi < total;
         pi += (long long)gridDim.x * blockDim.x) {
        const sbr_path_record p = A.paths[pi];
        if (!path_ids_ok(A, p)) continue;
        PathGeo g;
        load_path(A, p, g);
        atomicAdd(&hist[order_group(g)], 1u);
        float4 *u = A.unf + kUnfStride * pi;
        for (int j = 0; j < g.k; ++j) u[j] = unfold_plane32(A.scene, g, j);
        u[kMaxOrder] = unfold_rx32(A.scene, g);
        u[kMaxOrder + 1] = make_float4((float)p.dir[0], (float)p.dir[1], (float)p.dir[2], 0.0f);
    }
    __syncthreads();
    if (threadIdx.x < 10 && hist[threadIdx.x]) atomicAdd(A.order_cnt + threadIdx.x, (unsigned long long)hist[threadIdx.x]);
}

// a7/a8 of the batched form.  With many paths (>= split_min), one thread per path: every
// lane of a warp runs the same validity test and bounce-point walk on its own path, the
// paths taken in the lists the iteration kernels grouped by order.  With few paths, one
// warp per path with the point-in-face and occlusion queries spread over its lanes
// (latency).  The cone radius after `iters` iterations is recomputed with the same
// multiplications.  The queries are latency-bound: eight blocks per SM (64 registers,
// some spilled to L1) measured faster than four, five or six with fewer spills, and
// faster than the occlusion queries split into a kernel of their own with a thread per
// (path, leg) (which walks each path again for every leg).
__global__ void __launch_bounds__(128, 8) batch_finalize_kernel(RefineArgs A) {
    __shared__ UnfD s_sh[4];
    const long long total = path_count(A);
    const double shrink = c_sub.shrink[A.K];
    const bool per_thread = total >= A.split_min;
    const long long stride = per_thread ? (long long)gridDim.x * blockDim.x : (long long)gridDim.x * (blockDim.x >> 5);
    const long long first = per_thread ? blockIdx.x * (long long)blockDim.x + threadIdx.x
                                       : blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5);
    long long listed = total;
    if (per_thread) {   // paths with valid ids, listed by order group by the iteration kernel
        listed = 0;
        for (int b = 0; b < 10; ++b) listed += A.order_cnt[b];
    }
    for (long long t = first; t < listed; t += stride) {
        const long long pi = per_thread ? (long long)A.order_idx[t] : t;
        sbr_path_record p = A.paths[pi];
        if (!path_ids_ok(A, p)) continue;   // already flagged by the iteration kernel
        PathGeo g;
        load_path(A, p, g);
        const double R = cone_radius64(A, p.rough_err, p.iters, shrink);
        dvec3 c = dv(p.dir[0], p.dir[1], p.dir[2]);
        if (per_thread) {
            finalize_path(A, g, c, p, converged_bound(p.iters, R));
            store_result(A.paths + pi, p);
        } else {
            const int lane = threadIdx.x & 31;
            group_finalize<32>(A, g, c, p, lane, 0xffffffffu, converged_bound(p.iters, R), s_sh[threadIdx.x >> 5]);
            if (lane == 0) store_result(A.paths + pi, p);
        }
    }
}

static const void *batch_fn(int lanes) {
    switch (lanes) {
        case 1: return (const void *)batch_refine_kernel<1>;
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
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    static int unf_blocks = 0;
    if (!unf_blocks) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&unf_blocks, batch_unfold_kernel, 128, 0);
        if (unf_blocks < 1) unf_blocks = 1;
    }
    e = cudaMemsetAsync(a.order_cnt, 0, 64 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    {
        Range r("batch refine: plane unfolding");
        batch_unfold_kernel<<<sms * unf_blocks, 128, 0, s>>>(a);
    }
    {
        Range r("batch refine: iterations (work queue)");
        switch (a.chunk) {
            case 1: batch_refine_kernel<1><<<grid, block, 0, s>>>(a); break;
            case 8: batch_refine_kernel<8><<<grid, block, 0, s>>>(a); break;
            case 32: batch_refine_kernel<32><<<grid, block, 0, s>>>(a); break;
            default: batch_refine_kernel<16><<<grid, block, 0, s>>>(a); break;
        }
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    static int tail_blocks = 0;
    if (!tail_blocks) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&tail_blocks, batch_refine64_kernel, 128, 0);
        if (tail_blocks < 1) tail_blocks = 1;
    }
    {
        Range r("batch refine: FP64 tail");
        batch_refine64_kernel<<<sms * tail_blocks, 128, 0, s>>>(a);
    }
    static int fin_blocks = 0;
    if (!fin_blocks) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fin_blocks, batch_finalize_kernel, 128, 0);
        if (fin_blocks < 1) fin_blocks = 1;
    }
    {
        Range r("batch refine: validity + outputs");
        batch_finalize_kernel<<<sms * fin_blocks, 128, 0, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace sbr
