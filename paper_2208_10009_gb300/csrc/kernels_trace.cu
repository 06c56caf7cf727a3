// kernels_trace.cu -- a1 equiangular ray generation (§II.B, Eq. 1-2) and a2-a4 the
// persistent trace kernel: BVH closest hit with a watertight triangle test, specular
// reflection up to max_order (Fig. 4) and the reception judgment with the error angle
// of Eq. 3 on every segment.
#include "lattice_order.cuh"
#include "sbr_device.cuh"

namespace sbr {

// ----------------------------------------------------------------------------- a1
// Point j of m equal-angle steps along the great circle u -> v (angle om): Eq. 1 asks the
// points of a layer edge to subtend equal angles.  Normalised afterwards.
__device__ __forceinline__ float3 arc_point(float3 u, float3 v, float om, int j, int m) {
    float a = sinf(om * (float)(m - j) / (float)m);
    float b = sinf(om * (float)j / (float)m);
    float3 p = u * a + v * b;
    float inv = 1.0f / sqrtf(dot(p, p));
    return p * inv;
}


// One thread per ray; 32-bit index arithmetic (N < 2^31 for the supported n).
__global__ void raygen_kernel(LatticeDev L, float4 *__restrict__ dirs, int N) {
    const int n = L.n;
    const int n_edge = 30 * (n - 1);
    const int per_face = (n - 1) * (n - 2) / 2;
    const int layer_pts = layer_prefix(n, L.nl - 1);   // points on layers 1..nl-1
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < N; id += gridDim.x * blockDim.x) {
        float3 d;
        if (id < 12) {
            d = f3(__ldg(L.ico + id));
        } else if (id < 12 + n_edge) {
            int r = id - 12;
            int e = r / (n - 1), j = r - e * (n - 1) + 1;
            int2 ed = __ldg(L.edges + e);
            d = arc_point(f3(__ldg(L.ico + ed.x)), f3(__ldg(L.ico + ed.y)), L.edge_angle, j, n);
        } else {
            int r = id - 12 - n_edge;
            int f = r / per_face;
            int q = r - f * per_face;
            if (q >= layer_pts) {
                d = f3(__ldg(L.centre + f));   // n = 0 mod 3: the face centre ray
            } else {
                // layer a >= 1 with S(a-1) <= q < S(a): estimate from the quadratic, then fix
                float B = 3.0f * n - 4.5f;
                float disc = fmaxf(B * B - 18.0f * (float)q, 0.0f);
                int a = (int)((B - sqrtf(disc)) / 9.0f) + 1;
                if (a < 1) a = 1;
                if (a > L.nl - 1) a = L.nl - 1;
                while (a > 1 && layer_prefix(n, a - 1) > q) --a;
                while (layer_prefix(n, a) <= q) ++a;
                int b = q - layer_prefix(n, a - 1);
                int m = n - 3 * a;
                int e = b / m, j = b - e * m;
                const float4 *W = L.layers + ((size_t)f * L.nl + a) * 3;
                float4 w0 = __ldg(W + e), w1 = __ldg(W + (e == 2 ? 0 : e + 1));
                d = arc_point(f3(w0), f3(w1), w0.w, j, m);
            }
        }
        dirs[id] = make_float4(d.x, d.y, d.z, 0.0f);
    }
}

cudaError_t launch_raygen(const LatticeDev &lat, float4 *dirs, int64_t N, cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long want = (N + 255) / 256;
    int grid = (int)(want < (long long)sms * 16 ? want : (long long)sms * 16);
    if (grid < 1) grid = 1;
    raygen_kernel<<<grid, 256, 0, s>>>(lat, dirs, (int)N);
    return cudaGetLastError();
}

// §II.A equidistant division: flat-face points projected onto the sphere.
// interior rows before row i of a face: sum_{i'=1}^{i-1} (n - 1 - i')
__device__ __forceinline__ long long row_prefix(int n, long long i) { return (i - 1) * (n - 1) - (i - 1) * i / 2; }

__global__ void raygen_equidistant_kernel(PolyDev P, float4 *__restrict__ dirs, long long N) {
    const int n = P.n;
    const long long n_edge = (long long)P.ne * (n - 1);
    const long long per_face = (long long)(n - 1) * (n - 2) / 2;
    for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < N;
         id += (long long)gridDim.x * blockDim.x) {
        float3 p;
        if (id < P.nv) {
            p = f3(__ldg(P.v + id));
        } else if (id < P.nv + n_edge) {
            long long r = id - P.nv;
            int e = (int)(r / (n - 1)), j = (int)(r % (n - 1)) + 1;
            int2 ed = __ldg(P.edges + e);
            float3 lo = f3(__ldg(P.v + ed.x)), hi = f3(__ldg(P.v + ed.y));
            p = lo + (hi - lo) * ((float)j / (float)n);
        } else {
            long long r = id - P.nv - n_edge;
            int f = (int)(r / per_face);
            long long q = r % per_face;
            // row i >= 1 with row_prefix(i) <= q < row_prefix(i + 1): estimate, then fix
            float B = (float)n - 1.5f;
            float disc = fmaxf(B * B - 2.0f * (float)q, 0.0f);
            long long i = (long long)(B - sqrtf(disc)) + 1;
            if (i < 1) i = 1;
            if (i > n - 2) i = n - 2;
            while (i > 1 && row_prefix(n, i) > q) --i;
            while (i < n - 2 && row_prefix(n, i + 1) <= q) ++i;
            int j = (int)(q - row_prefix(n, i)) + 1;
            int4 fc = __ldg(P.faces + f);
            float3 A = f3(__ldg(P.v + fc.x)), Bv = f3(__ldg(P.v + fc.y)), C = f3(__ldg(P.v + fc.z));
            p = A + (Bv - A) * ((float)i / (float)n) + (C - A) * ((float)j / (float)n);
        }
        float inv = 1.0f / sqrtf(dot(p, p));
        dirs[id] = make_float4(p.x * inv, p.y * inv, p.z * inv, 0.0f);
    }
}

cudaError_t launch_raygen_equidistant(const PolyDev &P, float4 *dirs, int64_t N, cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long want = (N + 255) / 256;
    int grid = (int)(want < (long long)sms * 16 ? want : (long long)sms * 16);
    if (grid < 1) grid = 1;
    raygen_equidistant_kernel<<<grid, 256, 0, s>>>(P, dirs, (long long)N);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------- a2-a4
struct LaneRay {
    float3 o, d;
    float L;
    int k, prev, txi, ray;
};

// Receptions a lane buffers during one segment before its warp flushes them.  Emitting
// each record with its own atomic on the one record counter serialises the records at
// that counter's L2 slice (lanes are divergent inside the receiver leaves, so nothing
// aggregates them); the flush takes one atomic per warp step instead.  The buffer is a
// per-thread array in local memory (L1-cached); a segment can see many receivers when
// the cone has grown wide, so it holds kPend of them, and any further ones take their
// own slot at once.
constexpr int kPend = 16;

// Shared memory of a trace block: the faces of each thread's ray, [kMaxOrder][block].
size_t trace_smem(int block) { return (size_t)kMaxOrder * block * sizeof(int); }

// The lane's pending receptions: receiver id, error angle and ray length of each (arrays
// in the thread's local memory), their count and the order of their segment (registers).
struct Pending {
    int *rx;
    float *err, *dray;
    int n, k;
    __device__ __forceinline__ int &rx_at(int i) { return rx[i]; }
    __device__ __forceinline__ float &err_at(int i) { return err[i]; }
    __device__ __forceinline__ float &dray_at(int i) { return dray[i]; }
};

__device__ __forceinline__ void write_record(const TraceArgs &a, unsigned long long slot, const LaneRay &st, int k,
                                             int rx, float err, float dray, const int *faces_sh, int stride_sh) {
    if ((long long)slot >= a.rec_cap) return;
    RecDev rec;
    rec.tx = st.txi;
    rec.rx = rx;
    rec.ray = st.ray;
    rec.order = k;
#pragma unroll
    for (int j = 0; j < kMaxOrder; ++j) rec.faces[j] = j < k ? faces_sh[j * stride_sh] : -1;
    rec.err = err;
    rec.dray = dray;
    rec.slot = -1;
    rec.pad = 0;
    int4 *dst = reinterpret_cast<int4 *>(a.recs + slot);
    const int4 *src = reinterpret_cast<const int4 *>(&rec);
#pragma unroll
    for (int j = 0; j < 4; ++j) dst[j] = src[j];
}

// A reception past the lane's kPend pending ones (rare): its own slot, written at once.
__device__ __noinline__ void emit_direct(const TraceArgs &a, const LaneRay &st, int rx, float err, float dray,
                                         const int *faces_sh, int stride_sh) {
    const unsigned long long slot = atomicAdd(reinterpret_cast<unsigned long long *>(a.counters + kRecords), 1ULL);
    write_record(a, slot, st, st.k, rx, err, dray, faces_sh, stride_sh);
}

// Whole warp: every lane's pending receptions get consecutive slots from one atomic (lane
// order, then reception order) and are written out.
__device__ __forceinline__ void flush_records(const TraceArgs &a, const LaneRay &st, const int *faces_sh,
                                              int stride_sh, Pending &pd, unsigned lane) {
    if (__ballot_sync(0xffffffffu, pd.n > 0) == 0) return;
    int incl = pd.n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (unsigned)o) incl += t;
    }
    unsigned long long base = 0;
    if (lane == 31) base = atomicAdd(reinterpret_cast<unsigned long long *>(a.counters + kRecords), (unsigned long long)incl);
    base = __shfl_sync(0xffffffffu, base, 31) + (unsigned long long)(incl - pd.n);
    for (int i = 0; i < pd.n; ++i)
        write_record(a, base + i, st, pd.k, pd.rx_at(i), pd.err_at(i), pd.dray_at(i), faces_sh, stride_sh);
    pd.n = 0;
}

// Reception judgment on segment o + s d, s in [0, tseg], of a ray that has travelled L
// metres before it: every Rx whose foot lies on the segment and whose error angle
// (Eq. 3) is within the cone emits a record.  Candidates come from the receivers' 4-wide
// BVH, each box grown by the cone radius at the segment's far end; the growth is folded
// into the per-segment slab offsets (near: o/d + rad/|d|, far: o/d - rad/|d|), so a grown
// box costs what a plain one does.  Receptions go to the lane's pending buffer (past
// kPend in one segment, straight to the record array with their own atomic).
__device__ __forceinline__ void reception(const TraceArgs &a, const RayPre &r, const LaneRay &st, float tseg,
                                          const int *faces_sh, int stride_sh, Pending &pd, unsigned &rx_tests) {
    const RxDev &R = a.rx;
    if (R.nrx == 0) return;
    float tcap = fminf(tseg, max_foot(R, st.o, st.d));
    if (!(tcap >= 0.0f)) return;
    float rad = (st.L + tcap) * a.tan_cone * 1.001f + 1e-5f;
    const float oix = r.o.x * r.inv.x, oiy = r.o.y * r.inv.y, oiz = r.o.z * r.inv.z;
    const float gx = rad * fabsf(r.inv.x), gy = rad * fabsf(r.inv.y), gz = rad * fabsf(r.inv.z);
    const float cnx = oix + gx, cny = oiy + gy, cnz = oiz + gz;
    const float cfx = oix - gx, cfy = oiy - gy, cfz = oiz - gz;
    const float tfar = tcap * 1.0000005f + 1e-6f;
    {
        // the receivers' bounding box, grown like the node boxes: one slab test before the
        // walk (most segments, e.g. those rising above every receiver, end here; 2-3 %
        // of the trace measured on the canyon and the large city)
        const float nx = r.nx ? R.hi[0] : R.lo[0], fx = r.nx ? R.lo[0] : R.hi[0];
        const float ny = r.ny ? R.hi[1] : R.lo[1], fy = r.ny ? R.lo[1] : R.hi[1];
        const float nz = r.nz ? R.hi[2] : R.lo[2], fz = r.nz ? R.lo[2] : R.hi[2];
        const float tn = max3f(fmaf(nx, r.inv.x, -cnx), fmaf(ny, r.inv.y, -cny), fmaxf(fmaf(nz, r.inv.z, -cnz), 0.0f));
        const float tf = min3f(fmaf(fx, r.inv.x, -cfx), fmaf(fy, r.inv.y, -cfy), fminf(fmaf(fz, r.inv.z, -cfz), tfar));
        if (!(tn <= tf * 1.0000005f)) return;
    }
    int stack[kStack4];
    int sp = 0;
    int node = 0;
    for (;;) {
        if (!is_leaf(node)) {
            const float4 *nd = R.nodes4 + 8 * (size_t)node;
            float4 nxv = __ldg(nd + r.nx), fxv = __ldg(nd + 1 - r.nx);
            float4 nyv = __ldg(nd + 2 + r.ny), fyv = __ldg(nd + 3 - r.ny);
            float4 nzv = __ldg(nd + 4 + r.nz), fzv = __ldg(nd + 5 - r.nz);
            int4 refs = __ldg(reinterpret_cast<const int4 *>(nd + 6));
            const float2 nx01 = fma2s(nxv.x, nxv.y, r.inv.x, -cnx), nx23 = fma2s(nxv.z, nxv.w, r.inv.x, -cnx);
            const float2 fx01 = fma2s(fxv.x, fxv.y, r.inv.x, -cfx), fx23 = fma2s(fxv.z, fxv.w, r.inv.x, -cfx);
            const float2 ny01 = fma2s(nyv.x, nyv.y, r.inv.y, -cny), ny23 = fma2s(nyv.z, nyv.w, r.inv.y, -cny);
            const float2 fy01 = fma2s(fyv.x, fyv.y, r.inv.y, -cfy), fy23 = fma2s(fyv.z, fyv.w, r.inv.y, -cfy);
            const float2 nz01 = fma2s(nzv.x, nzv.y, r.inv.z, -cnz), nz23 = fma2s(nzv.z, nzv.w, r.inv.z, -cnz);
            const float2 fz01 = fma2s(fzv.x, fzv.y, r.inv.z, -cfz), fz23 = fma2s(fzv.z, fzv.w, r.inv.z, -cfz);
            const float tnx[4] = {nx01.x, nx01.y, nx23.x, nx23.y}, tfx[4] = {fx01.x, fx01.y, fx23.x, fx23.y};
            const float tny[4] = {ny01.x, ny01.y, ny23.x, ny23.y}, tfy[4] = {fy01.x, fy01.y, fy23.x, fy23.y};
            const float tnz[4] = {nz01.x, nz01.y, nz23.x, nz23.y}, tfz[4] = {fz01.x, fz01.y, fz23.x, fz23.y};
            const int rf[4] = {refs.x, refs.y, refs.z, refs.w};
            int next = 0x7fffffff;
            if (SBR_CHECKED_ON && sp + 3 > a.scene.stack_limit) {   // up to three pushes follow
                check_fail(a.scene, SBR_CHECK_RX_STACK);
                return;
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float tn = max3f(tnx[c], tny[c], fmaxf(tnz[c], 0.0f));
                float tf = min3f(tfx[c], tfy[c], fminf(tfz[c], tfar)) * 1.0000005f;
                if (tn <= tf) {
                    if (next == 0x7fffffff) next = rf[c];
                    else stack[sp++] = rf[c];
                }
            }
            if (next != 0x7fffffff) {
                node = next;
                continue;
            }
        } else {
            int first = leaf_first(node), cnt = leaf_count(node);
            for (int i = first; i < first + cnt; ++i) {
                float4 p = __ldg(R.pts + i);
                ++rx_tests;
                float3 w = f3(p) - st.o;
                float s = dot(w, st.d);
                if (s < 0.0f || s > tseg) continue;
                float3 q = w - st.d * s;
                const float q2 = dot(q, q), dray = st.L + s;
                // far outside the cone (a margin of 1e-4 on tan^2 dwarfs the FP32 rounding):
                // rejected without the square root and arc tangent of the exact test
                if (q2 > a.tan2_pre * dray * dray) continue;
                float err = atan2f(sqrtf(q2), dray);
                if (!(err <= a.cone)) continue;
                if (pd.n < kPend) {
                    pd.rx_at(pd.n) = __float_as_int(p.w);
                    pd.err_at(pd.n) = err;
                    pd.dray_at(pd.n) = dray;
                    ++pd.n;
                } else {
                    emit_direct(a, st, __float_as_int(p.w), err, dray, faces_sh, stride_sh);
                }
            }
        }
        if (sp == 0) break;
        node = stack[--sp];
    }
}

// Persistent trace kernel.  Each warp keeps 32 rays in registers; after a segment, once at
// least refill_min lanes hold a finished ray (miss or order cap), those lanes take fresh,
// consecutive places of the schedule (tiled_ray, or lattice ids) from a global counter with
// one warp-aggregated atomic (ballot + popc).  Waiting for several idle lanes keeps a warp's
// rays neighbours on the sphere (coherent traversal) while still keeping warps mostly full
// until the pool drains.  After
// every segment step the warp writes out its lanes' receptions together (flush_records).
// Seven 128-thread blocks per SM (72 registers, no spills) measured faster than eight (64
// registers, spilled).
__global__ void __launch_bounds__(128, 7) trace_kernel(TraceArgs a) {
    extern __shared__ int faces_sh_all[];   // trace_smem(blockDim.x) bytes
    int *faces_sh = faces_sh_all + threadIdx.x;
    const int stride_sh = blockDim.x;
    int pend_rx[kPend];
    float pend_err[kPend], pend_dray[kPend];
    Pending pd;
    pd.rx = pend_rx;
    pd.err = pend_err;
    pd.dray = pend_dray;
    pd.n = 0;
    const unsigned lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    const long long total = (long long)a.ntx * a.nrays_per_tx;
    unsigned seg = 0, nodes = 0, tris = 0, rxt = 0;
    bool alive = false, pool_empty = false;
    LaneRay st;
    st.o = st.d = make_float3(0, 0, 0);
    st.L = 0.0f;
    st.k = st.prev = st.txi = st.ray = 0;
    for (;;) {
        unsigned need = __ballot_sync(0xffffffffu, !alive);
        if (need && !pool_empty && (__popc(need) >= a.refill_min || need == 0xffffffffu)) {
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(reinterpret_cast<unsigned long long *>(a.counters + kRayHead),
                                            (unsigned long long)__popc(need));
            base = __shfl_sync(0xffffffffu, base, 0);
            if ((long long)base >= total) pool_empty = true;
            if (!alive) {
                long long gid = (long long)base + __popc(need & lt_mask);
                if (gid < total) {
                    st.txi = (int)(gid / a.nrays_per_tx);
                    const int local = (int)(gid - (long long)st.txi * a.nrays_per_tx);
                    st.ray = a.tiled_n > 0 ? tiled_ray(local, a.tiled_n) : (int)a.ray_begin + local;
                    st.o = f3(__ldg(a.tx + st.txi));
                    st.d = f3(__ldg(a.dirs + st.ray));
                    st.L = 0.0f;
                    st.k = 0;
                    st.prev = -1;
                    alive = true;
                    if (a.dump_stride > 0 && st.ray % a.dump_stride == 0) {
                        int *df = a.dump_faces + ((size_t)st.txi * a.dump_per_tx + st.ray / a.dump_stride) *
                                                     (a.max_order + 1);
                        for (int j = 0; j <= a.max_order; ++j) df[j] = -2;
                    }
                }
            }
        }
        if (__ballot_sync(0xffffffffu, alive) == 0) break;
        if (alive) {
            RayPre r = make_ray(st.o, st.d);
            float th;
            int face;
            const int hit = closest_hit4(a.scene, r, a.scene.tmin, INFINITY, st.prev, th, face, nodes, tris);
            ++seg;
            if (a.dump_stride > 0 && st.ray % a.dump_stride == 0)
                a.dump_faces[((size_t)st.txi * a.dump_per_tx + st.ray / a.dump_stride) * (a.max_order + 1) + st.k] =
                    hit >= 0 ? face : -1;
            float tseg = hit >= 0 ? th : INFINITY;
            pd.k = st.k;
            reception(a, r, st, tseg, faces_sh, stride_sh, pd, rxt);
            if (SBR_CHECKED_ON && hit >= 0 && (unsigned)face >= (unsigned)a.scene.nf) {
                check_fail(a.scene, SBR_CHECK_FACE_ID);
                alive = false;
            } else if (hit < 0 || st.k == a.max_order) {
                alive = false;
            } else {
                // specular reflection on the hit face's plane (faces_sh[j], j < pd.k, stay
                // as the pending receptions need them)
                float4 pl = __ldg(a.scene.planes + face);
                float3 nrm = f3(pl);
                st.o = st.o + st.d * th;
                st.d = st.d - nrm * (2.0f * dot(st.d, nrm));
                st.L += th;
                faces_sh[st.k * stride_sh] = face;
                st.prev = face;
                ++st.k;
            }
        }
        flush_records(a, st, faces_sh, stride_sh, pd, lane);
    }
    // one atomic per warp per counter
    unsigned s0 = __reduce_add_sync(0xffffffffu, seg), s1 = __reduce_add_sync(0xffffffffu, nodes);
    unsigned s2 = __reduce_add_sync(0xffffffffu, tris), s3 = __reduce_add_sync(0xffffffffu, rxt);
    if (lane == 0) {
        atomicAdd(reinterpret_cast<unsigned long long *>(a.counters + kSegments), (unsigned long long)s0);
        atomicAdd(reinterpret_cast<unsigned long long *>(a.counters + kNodeVisits), (unsigned long long)s1);
        atomicAdd(reinterpret_cast<unsigned long long *>(a.counters + kTriTests), (unsigned long long)s2);
        atomicAdd(reinterpret_cast<unsigned long long *>(a.counters + kRxTests), (unsigned long long)s3);
    }
}

int trace_blocks_per_sm(int block) {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, trace_kernel, block, trace_smem(block));
    return nb > 0 ? nb : 1;
}

cudaError_t launch_trace(const TraceArgs &a, int grid, int block, cudaStream_t s) {
    trace_kernel<<<grid, block, trace_smem(block), s>>>(a);
    return cudaGetLastError();
}

}  // namespace sbr
