// noalloc.cu -- sbr_dedup_noalloc: double-count removal that allocates nothing.
//
// Some callers cannot let a library allocate device memory while they call it, e.g.
// processes whose device memory is already fully reserved by another framework's pool,
// where an allocation would fail or fragment the pool.
// For them this entry point keeps its scratch -- the hash table that picks one path per
// (Tx, Rx, face sequence) -- in a fixed-size array in device global memory that is part
// of the library image.  The caller passes the input (a container filled by sbr_launch)
// and the output buffers; nothing is allocated or freed here.
//
// Costs and rules of the fixed array:
//   - every GPU that loads the library holds kScratchBytes (about 5.5 MiB) until exit;
//   - all calls share it and it keeps the last call's contents, so each call clears the
//     parts that must start empty, and calls whose GPU work overlaps (different streams
//     or devices' contexts racing on the same device) corrupt each other's results;
//   - the first call on a device looks the array's device address up for that device
//     (cudaGetSymbolAddress), and every call made while its stream is not capturing looks
//     it up again (so a call after a device reset sees the array's new address); make the
//     first call on a device, and the first after a device reset, before any stream capture.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>

#include "dedup_keys.cuh"

namespace {

constexpr int64_t kMaxRecords = SBR_NOALLOC_MAX_RECORDS;
constexpr int64_t kSlots = 2 * kMaxRecords;   // power of two
static_assert((kSlots & (kSlots - 1)) == 0, "slot count must be a power of two");

// layout of the scratch array
constexpr size_t kKeysOff = 0;
constexpr size_t kValsOff = kKeysOff + sizeof(unsigned long long) * kSlots;
constexpr size_t kWinOff = kValsOff + sizeof(unsigned long long) * kSlots;
constexpr size_t kSlotOff = kWinOff + sizeof(int) * kSlots;
constexpr size_t kCountOff = (kSlotOff + sizeof(int) * kMaxRecords + 255) / 256 * 256;
constexpr size_t kScratchBytes = kCountOff + 2 * sizeof(long long);

static __device__ __align__(256) unsigned char g_dedup_scratch[kScratchBytes];

struct NaArgs {
    unsigned char *scratch;          // device address of g_dedup_scratch
    const sbr::RecDev *recs;         // input records
    const long long *rec_count;      // device: records emitted by the launch
    int64_t rec_cap;
    const float4 *dirs;              // lattice directions of the launch
    sbr_path_record *out;            // output paths
    int64_t cap;
};

__device__ __forceinline__ long long na_count(const NaArgs &a) {
    long long n = *a.rec_count;
    return n < a.rec_cap ? n : a.rec_cap;
}

// the slots this call uses, from the record count on the device (as the launch's dedup)
__device__ __forceinline__ unsigned long long na_slots(const NaArgs &a) { return sbr::dedup_slots(na_count(a), kSlots); }

// empty keys, +inf values and no winners over the slots in use, zero counts: the array
// keeps the last call's contents
__global__ void na_clear(NaArgs a) {
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(a.scratch + kKeysOff);
    unsigned long long *vals = reinterpret_cast<unsigned long long *>(a.scratch + kValsOff);
    int *winner = reinterpret_cast<int *>(a.scratch + kWinOff);
    const unsigned long long m = na_slots(a);
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < m;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        keys[i] = ~0ULL;
        vals[i] = ~0ULL;
        winner[i] = -1;
    }
    if (blockIdx.x == 0 && threadIdx.x < 2) reinterpret_cast<long long *>(a.scratch + kCountOff)[threadIdx.x] = 0;
}

__global__ void na_insert(NaArgs a) {
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(a.scratch + kKeysOff);
    unsigned long long *vals = reinterpret_cast<unsigned long long *>(a.scratch + kValsOff);
    int *slot_of = reinterpret_cast<int *>(a.scratch + kSlotOff);
    const long long n = na_count(a);
    const unsigned long long used = na_slots(a), mask = used - 1;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        sbr::RecDev r = a.recs[i];
        unsigned long long h = sbr::rec_hash(r), s = h & mask;
        slot_of[i] = -1;
        for (unsigned long long probe = 0; probe < used; ++probe) {
            unsigned long long prev = atomicCAS(keys + s, ~0ULL, h);
            if (prev == ~0ULL || prev == h) {
                atomicMin(vals + s, sbr::rec_value(r));
                slot_of[i] = (int)s;
                break;
            }
            s = (s + 1) & mask;
        }
    }
}

__global__ void na_select(NaArgs a) {
    const unsigned long long *vals = reinterpret_cast<const unsigned long long *>(a.scratch + kValsOff);
    int *winner = reinterpret_cast<int *>(a.scratch + kWinOff);
    const int *slot_of = reinterpret_cast<const int *>(a.scratch + kSlotOff);
    long long *counts = reinterpret_cast<long long *>(a.scratch + kCountOff);
    const long long n = na_count(a);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int s = slot_of[i];
        if (s < 0) continue;
        sbr::RecDev r = a.recs[i];
        if (vals[s] != sbr::rec_value(r)) continue;
        winner[s] = (int)i;
        unsigned long long p = atomicAdd(reinterpret_cast<unsigned long long *>(counts), 1ULL);
        if ((long long)p >= a.cap) continue;
        sbr_path_record o;
        o.tx = r.tx;
        o.rx = r.rx;
        o.ray = r.ray;
        o.order = r.order;
        for (int j = 0; j < SBR_MAX_ORDER; ++j) o.faces[j] = r.faces[j];
        o.rough_err = r.err;
        o.rough_dray = r.dray;
        o.iters = 0;
        o.valid = 0;
        float4 d = a.dirs[r.ray];
        o.dir[0] = d.x;
        o.dir[1] = d.y;
        o.dir[2] = d.z;
        o.err = r.err;
        o.delay = 0.0;
        o.aod[0] = o.aod[1] = o.aoa[0] = o.aoa[1] = 0.0f;
        o.power_dbm = 0.0f;
        o.flags = 0;
        a.out[p] = o;
    }
}

__global__ void na_verify(NaArgs a) {
    const int *winner = reinterpret_cast<const int *>(a.scratch + kWinOff);
    const int *slot_of = reinterpret_cast<const int *>(a.scratch + kSlotOff);
    long long *counts = reinterpret_cast<long long *>(a.scratch + kCountOff);
    const long long n = na_count(a);
    unsigned bad = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int s = slot_of[i];
        int w = s < 0 ? -1 : winner[s];
        if (w < 0) {
            ++bad;
            continue;
        }
        if (!sbr::same_key(a.recs[i], a.recs[w])) ++bad;
    }
    if (bad) atomicAdd(reinterpret_cast<unsigned long long *>(counts + 1), (unsigned long long)bad);
}

// device address of the scratch array, looked up once per device
std::mutex g_mu;
void *g_addr[128] = {nullptr};

sbr_status na_fail(sbr_ctx *ctx, sbr_status s, const std::string &m) {
    ctx->last_error = m;
    return s;
}

}  // namespace

extern "C" sbr_status sbr_dedup_noalloc(sbr_ctx *ctx, const sbr_paths *src, sbr_path_record *out, int64_t cap,
                                        int64_t *counts) {
    if (!ctx) return SBR_EINVAL;
    if (!src || !counts || (cap > 0 && !out) || cap < 0)
        return na_fail(ctx, SBR_EINVAL, "sbr_dedup_noalloc: null argument or negative capacity");
    if (src->record_cap > kMaxRecords)
        return na_fail(ctx, SBR_EINVAL, "sbr_dedup_noalloc: the container's record capacity " +
                                            std::to_string(src->record_cap) + " exceeds the fixed maximum of " +
                                            std::to_string(kMaxRecords) + " records");
    if (src->n_div < 1 || !ctx->dirs || ctx->dirs_n != src->n_div || ctx->dirs_launcher != src->launcher)
        return na_fail(ctx, SBR_EINVAL, "sbr_dedup_noalloc: the container holds no launch whose ray directions "
                                        "are still current on this context");
    if (ctx->device < 0 || ctx->device >= 128) return na_fail(ctx, SBR_EINVAL, "sbr_dedup_noalloc: device id");
    {
        // the container's records must live on the context's device
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, src->recs) != cudaSuccess || at.type != cudaMemoryTypeDevice ||
            at.device != ctx->device) {
            cudaGetLastError();
            return na_fail(ctx, SBR_EINVAL, "sbr_dedup_noalloc: the container does not belong to the context's device");
        }
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != ctx->device) cudaSetDevice(ctx->device);
    void *base = nullptr;
    {
        // looked up again whenever the stream is not capturing: a device reset gives the
        // array a new address, and a lookup is not made during capture
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(ctx->stream, &cs) != cudaSuccess) {
            cudaGetLastError();
            cs = cudaStreamCaptureStatusNone;
        }
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[ctx->device] || cs == cudaStreamCaptureStatusNone) {
            cudaError_t e = cudaGetSymbolAddress(&g_addr[ctx->device], g_dedup_scratch);
            if (e != cudaSuccess) {
                g_addr[ctx->device] = nullptr;
                if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
                return na_fail(ctx, SBR_ECUDA, std::string("sbr_dedup_noalloc: cudaGetSymbolAddress failed: ") +
                                                   cudaGetErrorString(e));
            }
        }
        base = g_addr[ctx->device];
    }
    unsigned char *sc = static_cast<unsigned char *>(base);
    cudaStream_t s = ctx->stream;
    cudaError_t e = cudaSuccess;
    NaArgs a;
    a.scratch = sc;
    a.recs = src->recs;
    a.rec_count = src->counters + sbr::kRecords;
    a.rec_cap = src->record_cap;
    a.dirs = static_cast<const float4 *>(ctx->dirs);
    a.out = out;
    a.cap = cap;
    int grid = std::max(1, ctx->num_sms * 2);
    if (e == cudaSuccess) {
        na_clear<<<grid, 256, 0, s>>>(a);
        na_insert<<<grid, 256, 0, s>>>(a);
        na_select<<<grid, 256, 0, s>>>(a);
        na_verify<<<grid, 256, 0, s>>>(a);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(counts, sc + kCountOff, 2 * sizeof(long long), cudaMemcpyDeviceToDevice, s);
    if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
    if (e != cudaSuccess) return na_fail(ctx, SBR_ECUDA, std::string("sbr_dedup_noalloc: ") + cudaGetErrorString(e));
    return SBR_OK;
}
