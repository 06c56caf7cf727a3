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
// A, a0 and Tx^(k) come from one pass over the faces in path order (unfold_pass).  The
// adjoint recomputes w, v and d instead of storing them.
#include <algorithm>

#include "sbr_device.cuh"

namespace sbr {

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

// One pass over the path's faces in path order: the linear part A = H_1 ... H_k (row-major
// m), the offset a0 of the composed map Rx' = M_1(...M_k(Rx)) = A Rx + a0, and the last Tx
// image txk = M_k(...M_1(Tx)).  With C_j = M_1 o ... o M_j and M_j(x) = H_j x + 2 h_j n_j:
// C_j(x) = A_{j-1} H_j x + (a_{j-1} + 2 h_j A_{j-1} n_j), so each face costs one plane load
// and A n once.  The loop runs the path's own order (a warp: its longest path), not the
// maximum order.  face(j) gives face j's id; false if one lies outside [0, nf).
template <class FaceAt>
__device__ __forceinline__ bool unfold_pass(const SceneDev &S, int nf, int k, FaceAt face, float3 tx, float m[9],
                                            float3 &a0, float3 &txk) {
    m[0] = 1.0f; m[1] = 0.0f; m[2] = 0.0f;
    m[3] = 0.0f; m[4] = 1.0f; m[5] = 0.0f;
    m[6] = 0.0f; m[7] = 0.0f; m[8] = 1.0f;
    float o[3] = {0.0f, 0.0f, 0.0f};
    float3 x = tx;
    // the ids first (independent loads), so that the walk below can load each next plane
    // under the current face's arithmetic
#pragma unroll
    for (int j = 0; j < kMaxOrder; ++j) {
        if (j >= k) break;
        const int f = face(j);
        if (f < 0 || f >= nf) return false;
    }
    float4 pl = k > 0 ? __ldg(S.planes + face(0)) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll 1
    for (int j = 0; j < k; ++j) {
        const float4 pn = __ldg(S.planes + face(j + 1 < k ? j + 1 : j));
        const float3 n = f3(pl);
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const float an = 2.0f * fmaf(m[3 * r], n.x, fmaf(m[3 * r + 1], n.y, m[3 * r + 2] * n.z));
            o[r] = fmaf(an, pl.w, o[r]);
            m[3 * r] = fmaf(-an, n.x, m[3 * r]);
            m[3 * r + 1] = fmaf(-an, n.y, m[3 * r + 1]);
            m[3 * r + 2] = fmaf(-an, n.z, m[3 * r + 2]);
        }
        const float s = dot(n, x) - pl.w;
        x = x - n * (2.0f * s);
        pl = pn;
    }
    a0 = make_float3(o[0], o[1], o[2]);
    txk = x;
    return true;
}

// gradient of (az, el) of w with respect to w, with one reciprocal and one reciprocal
// square root: d az = (-w_y, w_x, 0) / rho^2, d el = (-w_x w_z, -w_y w_z, rho^2) / (r^2 rho)
__device__ __forceinline__ void angles_grad_fast(float3 w, float3 &gaz, float3 &gel) {
    const float rho2 = fmaf(w.x, w.x, w.y * w.y), r2 = fmaf(w.z, w.z, rho2);
    const float irho = rsqrtf(rho2), ir2 = 1.0f / r2;
    const float irho2 = irho * irho, c = ir2 * irho;
    gaz = make_float3(-w.y * irho2, w.x * irho2, 0.0f);
    gel = make_float3(-w.x * w.z * c, -w.y * w.z * c, rho2 * c);
}

__global__ void unfold_fwd_kernel(UnfoldArgs a) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < a.n; i += (long long)gridDim.x * blockDim.x) {
        const float3 tx = make_float3(a.tx[3 * i], a.tx[3 * i + 1], a.tx[3 * i + 2]);
        const float3 rx = make_float3(a.rx[3 * i], a.rx[3 * i + 1], a.rx[3 * i + 2]);
        const int ord = a.order[i];
        const int k = ord < 0 ? 0 : (ord > kMaxOrder ? kMaxOrder : ord);
        const int *fp = a.faces + 8 * i;
        float m[9];
        float3 a0, txk;
        float *o = a.out + 8 * i;
        if (!unfold_pass(a.scene, a.nf, k, [&](int j) { return __ldg(fp + j); }, tx, m, a0, txk)) {
            for (int j = 0; j < 8; ++j) o[j] = __int_as_float(0x7fc00000);
            continue;
        }
        const float3 w = mul_A(m, rx) + a0 - tx;
        float se, ce, sa, ca;
        sincosf(a.az_el[2 * i + 1], &se, &ce);
        sincosf(a.az_el[2 * i], &sa, &ca);
        const float3 d = make_float3(ce * ca, ce * sa, se);
        const float3 miss = mul_AT(m, w - d * dot(w, d));
        const float3 v = txk - rx;
        o[0] = miss.x;
        o[1] = miss.y;
        o[2] = miss.z;
        o[3] = sqrtf(dot(w, w)) * (float)(1.0 / kC0);
        angles(w, o[4], o[5]);
        angles(v, o[6], o[7]);
    }
}

__device__ __forceinline__ void load_grad_row(const UnfoldArgs &a, long long i, float g[8]) {
    // two 16-byte loads when the array is 16-byte aligned (every row then is), else eight
    // 4-byte loads
    if ((reinterpret_cast<uintptr_t>(a.grad_out) & 15) == 0) {
        const float4 g0 = __ldg(reinterpret_cast<const float4 *>(a.grad_out) + 2 * i);
        const float4 g1 = __ldg(reinterpret_cast<const float4 *>(a.grad_out) + 2 * i + 1);
        g[0] = g0.x; g[1] = g0.y; g[2] = g0.z; g[3] = g0.w;
        g[4] = g1.x; g[5] = g1.y; g[6] = g1.z; g[7] = g1.w;
    } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) g[j] = __ldg(a.grad_out + 8 * i + j);
    }
}

// The adjoint of one path from its loaded inputs (g: the row of 8 output gradients);
// face(j) gives its face ids.  A path with an id outside [0, nf) gets NaN gradients.
template <class FaceAt>
__device__ __forceinline__ void bwd_path(const UnfoldArgs &a, float3 tx, float3 rx, float az, float el, int k,
                                         FaceAt face, const float g[8], long long i) {
    float m[9];
    float3 a0, txk;
    if (!unfold_pass(a.scene, a.nf, k, face, tx, m, a0, txk)) {
        const float nan = __int_as_float(0x7fc00000);
        for (int j = 0; j < 3; ++j) a.grad_tx[3 * i + j] = a.grad_rx[3 * i + j] = nan;
        a.grad_az_el[2 * i] = a.grad_az_el[2 * i + 1] = nan;
        return;
    }
    const float3 w = mul_A(m, rx) + a0 - tx;
    float se, ce, sa, ca;
    __sincosf(el, &se, &ce);
    __sincosf(az, &sa, &ca);
    const float3 d = make_float3(ce * ca, ce * sa, se);
    const float3 d_az = make_float3(-ce * sa, ce * ca, 0.0f);
    const float3 d_el = make_float3(-se * ca, -se * sa, ce);
    const float3 v = txk - rx;
    const float wd = dot(w, d);
    // miss = A^T (w - (w.d) d): pull g_miss back into unfolded space
    const float3 gm = mul_A(m, make_float3(g[0], g[1], g[2]));
    const float gmd = dot(gm, d);
    float3 gw = gm - d * gmd;
    const float3 gd = (gm * wd + w * gmd) * -1.0f;
    // delay |w| / c0
    gw = gw + w * (g[3] * (float)(1.0 / kC0) * rsqrtf(dot(w, w)));
    // AOD angles of w
    float3 gaz, gel;
    angles_grad_fast(w, gaz, gel);
    gw = gw + gaz * g[4] + gel * g[5];
    // AOA angles of v = A^T Tx + b0 - Rx
    angles_grad_fast(v, gaz, gel);
    const float3 gv = gaz * g[6] + gel * g[7];
    const float3 gtx = gw * -1.0f + mul_A(m, gv);
    const float3 grx = mul_AT(m, gw) - gv;
    a.grad_tx[3 * i] = gtx.x;
    a.grad_tx[3 * i + 1] = gtx.y;
    a.grad_tx[3 * i + 2] = gtx.z;
    a.grad_rx[3 * i] = grx.x;
    a.grad_rx[3 * i + 1] = grx.y;
    a.grad_rx[3 * i + 2] = grx.z;
    a.grad_az_el[2 * i] = dot(gd, d_az);
    a.grad_az_el[2 * i + 1] = dot(gd, d_el);
}

// The inputs of path i other than its faces, straight from global memory.
__device__ __forceinline__ void bwd_direct_path(const UnfoldArgs &a, long long i) {
    const float3 tx = make_float3(a.tx[3 * i], a.tx[3 * i + 1], a.tx[3 * i + 2]);
    const float3 rx = make_float3(a.rx[3 * i], a.rx[3 * i + 1], a.rx[3 * i + 2]);
    const int ord = a.order[i];
    const int k = ord < 0 ? 0 : (ord > kMaxOrder ? kMaxOrder : ord);
    float g[8];
    load_grad_row(a, i, g);
    const int *fp = a.faces + 8 * i;
    bwd_path(a, tx, rx, a.az_el[2 * i], a.az_el[2 * i + 1], k, [&](int j) { return __ldg(fp + j); }, g, i);
}


// Grid-stride form, loads straight from global memory: used when an input array is not
// 16-byte aligned (the bulk copies of the staged form need that) or the batch is small.
// At most 64 registers a thread (four 256-thread blocks per SM).
__global__ void __launch_bounds__(256, 4) unfold_bwd_kernel(UnfoldArgs a) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < a.n; i += (long long)gridDim.x * blockDim.x)
        bwd_direct_path(a, i);
}

// ---------------------------------------------------------------- staged adjoint
// The adjoint reads 100 bytes per path (Tx, Rx, az/el, order, 8 face ids, 8 output
// gradients) and writes 32; per path it then walks the order's face planes (an L1-resident
// table) once.  Loading a path's inputs in the thread that computes it leaves the thread
// idle for a DRAM round trip per path.  Here each warp owns whole 32-path chunks
// (persistent, chunk += all warps): one lane issues six bulk copies (cp.async.bulk, one per
// input array: a chunk's part of every array is one contiguous, 16-byte aligned range) into
// the warp's shared-memory buffer, completing on that buffer's mbarrier, and the next
// chunk's copies are issued before the current chunk is computed (two buffers a warp), so
// the copies run under the arithmetic.  Warps never wait for one another.  The ragged last
// chunk is read from global memory.
constexpr int kChunk = 32;
constexpr int kStageWarps = 8;   // warps a block
constexpr unsigned kCTx = 12 * kChunk, kCAzEl = 8 * kChunk, kCOrder = 4 * kChunk, kCFaces = 32 * kChunk,
                   kCGrad = 32 * kChunk;
constexpr unsigned kOffTx = 0, kOffRx = kOffTx + kCTx, kOffAzEl = kOffRx + kCTx, kOffOrder = kOffAzEl + kCAzEl,
                   kOffFaces = kOffOrder + kCOrder, kOffGrad = kOffFaces + kCFaces,
                   kChunkBytes = kOffGrad + kCGrad;   // 3,200 bytes a chunk
constexpr unsigned kBarOff = kStageWarps * 2 * kChunkBytes;
constexpr unsigned kBwdSmem = kBarOff + kStageWarps * 16;   // two buffers + two mbarriers a warp
static_assert(kOffRx % 16 == 0 && kOffAzEl % 16 == 0 && kOffOrder % 16 == 0 && kOffFaces % 16 == 0 &&
              kOffGrad % 16 == 0 && kChunkBytes % 16 == 0, "bulk-copy alignment");
// an mbarrier wait that has not completed after this long gives up (nanoseconds)
constexpr unsigned long long kWaitLimitNs = 1000000000ull;

__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void bulk_g2s(unsigned dst, const void *src, unsigned bytes, unsigned mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(dst), "l"(src), "r"(bytes), "r"(mbar) : "memory");
}

// Issue the six copies of chunk c into the buffer at buf (one lane).
__device__ __forceinline__ void issue_chunk(const UnfoldArgs &a, long long c, unsigned buf, unsigned mbar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(mbar), "r"(kChunkBytes) : "memory");
    const long long p = c * kChunk;
    bulk_g2s(buf + kOffTx, a.tx + 3 * p, kCTx, mbar);
    bulk_g2s(buf + kOffRx, a.rx + 3 * p, kCTx, mbar);
    bulk_g2s(buf + kOffAzEl, a.az_el + 2 * p, kCAzEl, mbar);
    bulk_g2s(buf + kOffOrder, a.order + p, kCOrder, mbar);
    bulk_g2s(buf + kOffFaces, a.faces + 8 * p, kCFaces, mbar);
    bulk_g2s(buf + kOffGrad, a.grad_out + 8 * p, kCGrad, mbar);
}

// Wait for phase `parity` of the mbarrier, at most kWaitLimitNs; false on giving up.
__device__ __forceinline__ bool wait_parity(unsigned mbar, unsigned parity) {
    const unsigned long long t0 = global_ns();
    for (;;) {
        unsigned done;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
        if (done) return true;
        if (global_ns() - t0 > kWaitLimitNs) return false;
    }
}

#ifndef SBR_STAGE_BLOCKS
#define SBR_STAGE_BLOCKS 3
#endif
__global__ void __launch_bounds__(kStageWarps * 32, SBR_STAGE_BLOCKS) unfold_bwd_staged_kernel(UnfoldArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long full = a.n / kChunk;   // chunks read by bulk copies
    const long long chunks = (a.n + kChunk - 1) / kChunk;
    const long long nwarps = (long long)gridDim.x * kStageWarps;
    unsigned char *wbuf = smem + w * 2 * kChunkBytes;
    const unsigned base = smem_addr(wbuf);
    const unsigned mb0 = smem_addr(smem + kBarOff) + 16 * w, mb1 = mb0 + 8;
    if (lane == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mb0) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mb1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    long long c = (long long)blockIdx.x * kStageWarps + w;
    if (lane == 0 && c < full) issue_chunk(a, c, base, mb0);
    for (unsigned it = 0; c < chunks; ++it, c += nwarps) {
        if (c >= full) {   // the ragged last chunk
            const long long i = c * kChunk + lane;
            if (i < a.n) bwd_direct_path(a, i);
            continue;
        }
        const unsigned cur = it & 1, mbar = cur ? mb1 : mb0;
        const long long nxt = c + nwarps;
        // the other buffer was last read in the previous iteration, which ended with a
        // warp barrier: refill it with the next chunk before computing this one
        if (lane == 0 && nxt < full) issue_chunk(a, nxt, base + (cur ^ 1) * kChunkBytes, cur ? mb0 : mb1);
        const bool ok = wait_parity(mbar, (it >> 1) & 1);
        if (__any_sync(0xffffffffu, !ok)) {
            // the copies did not arrive in time: NaN gradients for this warp's remaining
            // paths, then wait (bounded) for the copies still in flight before leaving
            const float nan = __int_as_float(0x7fc00000);
            for (long long r = c; r < chunks; r += nwarps) {
                const long long i = r * kChunk + lane;
                if (i >= a.n) continue;
                for (int j = 0; j < 3; ++j) a.grad_tx[3 * i + j] = a.grad_rx[3 * i + j] = nan;
                a.grad_az_el[2 * i] = a.grad_az_el[2 * i + 1] = nan;
            }
            if (lane == 0) {
                wait_parity(mbar, (it >> 1) & 1);
                if (nxt < full) wait_parity(cur ? mb0 : mb1, ((it + 1) >> 1) & 1);
            }
            return;
        }
        const unsigned char *sb = wbuf + cur * kChunkBytes;
        const float *stx = reinterpret_cast<const float *>(sb + kOffTx) + 3 * lane;
        const float *srx = reinterpret_cast<const float *>(sb + kOffRx) + 3 * lane;
        const float2 ae = reinterpret_cast<const float2 *>(sb + kOffAzEl)[lane];
        const int *sf = reinterpret_cast<const int *>(sb + kOffFaces) + 8 * lane;
        const float4 *sg = reinterpret_cast<const float4 *>(sb + kOffGrad) + 2 * lane;
        const int ord = reinterpret_cast<const int *>(sb + kOffOrder)[lane];
        const int k = ord < 0 ? 0 : (ord > kMaxOrder ? kMaxOrder : ord);
        const float4 g0 = sg[0], g1 = sg[1];
        const float g[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
        bwd_path(a, make_float3(stx[0], stx[1], stx[2]), make_float3(srx[0], srx[1], srx[2]), ae.x, ae.y, k,
                 [&](int j) { return sf[j]; }, g, c * kChunk + lane);
        __syncwarp();   // this buffer is refilled in the next iteration
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

// The staged form needs every input array 16-byte aligned (each chunk's range then is) and
// pays off once there are a few chunks per warp; it runs persistent, four blocks per SM.
cudaError_t launch_unfold_bwd(const UnfoldArgs &a, cudaStream_t s) {
    auto al16 = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long chunks = (a.n + kChunk - 1) / kChunk;
    const bool staged = al16(a.tx) && al16(a.rx) && al16(a.az_el) && al16(a.order) && al16(a.faces) &&
                        al16(a.grad_out) && chunks >= 16LL * sms;
    if (!staged) {
        unfold_bwd_kernel<<<unfold_grid(a.n), 256, 0, s>>>(a);
        return cudaGetLastError();
    }
    static bool attr_set[64] = {};
    if (dev < 64 && !attr_set[dev]) {
        cudaError_t e = cudaFuncSetAttribute(unfold_bwd_staged_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kBwdSmem);
        if (e != cudaSuccess) return e;
        attr_set[dev] = true;
    }
    const long long grid = std::min<long long>((chunks + kStageWarps - 1) / kStageWarps, (long long)SBR_STAGE_BLOCKS * sms);
    unfold_bwd_staged_kernel<<<(int)grid, kStageWarps * 32, kBwdSmem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace sbr
