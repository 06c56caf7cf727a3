// probe_fp32.cu -- measurement utility (no counterpart in the paper): the FP32 FMA rate this
// GPU sustains, the denominator of the roofline of the ALU-bound kernels (trace, batched
// refinement).  Each thread runs eight independent FMA chains (enough independent work to
// hide the pipe latency) for `iters` steps, either as scalar fma.rn.f32 or as packed
// fma.rn.f32x2 (two FMAs per instruction), over a grid of blocks_per_sm x SMs.  Built as
// its own small library (libsbr_probe.so); the SBR library does not use it.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

__global__ void fma_scalar(float *out, int iters, float a, float b) {
    float x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = threadIdx.x * 1e-3f + j;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(x[j]) : "f"(a), "f"(b));
    }
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += x[j];
    if (s == 1234.5f) out[blockIdx.x] = s;   // keeps the chains live; never true for these inputs
}

__global__ void fma_packed(float *out, int iters, float a, float b) {
    unsigned long long x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        float lo = threadIdx.x * 1e-3f + j, hi = lo + 0.5f;
        asm("mov.b64 %0, {%1, %2};" : "=l"(x[j]) : "f"(lo), "f"(hi));
    }
    unsigned long long pa, pb;
    asm("mov.b64 %0, {%1, %1};" : "=l"(pa) : "f"(a));
    asm("mov.b64 %0, {%1, %1};" : "=l"(pb) : "f"(b));
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[j]) : "l"(pa), "l"(pb));
    }
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[j]));
        s += lo + hi;
    }
    if (s == 1234.5f) out[blockIdx.x] = s;
}

}  // namespace

extern "C" {

// FP32 FLOP/s of one timed launch (2 FLOP per FMA); returns 0 on success, the CUDA error
// code otherwise.  packed = 0: fma.rn.f32; 1: fma.rn.f32x2.  *ms = the launch's event time.
int sbr_probe_fp32(int device, int packed, int blocks_per_sm, int iters, double *flops_per_s, float *ms) {
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return (int)e;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int block = 256, grid = sms * blocks_per_sm;
    float *out = nullptr;
    if ((e = cudaMalloc(&out, sizeof(float) * grid)) != cudaSuccess) return (int)e;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    for (int rep = 0; rep < 2; ++rep) {   // the first launch warms up, the second is timed
        cudaEventRecord(a);
        if (packed) fma_packed<<<grid, block>>>(out, iters, 0.999f, 1e-3f);
        else fma_scalar<<<grid, block>>>(out, iters, 0.999f, 1e-3f);
        cudaEventRecord(b);
    }
    e = cudaEventSynchronize(b);
    float t = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(out);
    if (e != cudaSuccess) return (int)e;
    const double fmas = (double)grid * block * iters * 8.0 * (packed ? 2.0 : 1.0);
    *flops_per_s = 2.0 * fmas / (t * 1e-3);
    *ms = t;
    return 0;
}

}  // extern "C"
