// kernels_paths.cu -- a5 double-count removal (§III.A, first path test): among reception
// records with the same (Tx, Rx, face sequence) keep the one with the smallest error
// angle of Eq. 3, ties to the lowest ray id.  Implemented as an open-addressing hash table
// keyed by a 64-bit hash of the face sequence with a 64-bit atomicMin on
// (error-angle bits, ray id); a second pass checks every record against its slot's
// winner so that a hash collision is detected, never silently merged.
#include "dedup_keys.cuh"
#include "sbr_device.cuh"

namespace sbr {

__device__ __forceinline__ long long num_records(const DedupArgs &a) {
    long long n = a.counters[kRecords];
    return n < a.rec_cap ? n : a.rec_cap;
}

// slots in use for this launch (dedup_slots)
__device__ __forceinline__ unsigned long long used_slots(const DedupArgs &a) {
    return dedup_slots(num_records(a), a.slots);
}

// A slot is 16 bytes, its key then its value (one 32-byte sector holds two slots, so an
// insert's compare-and-swap and minimum touch one sector); the winners follow the slots.
// Keys and values to all-ones (empty / +inf), winners to -1, over the used slots.
__global__ void dedup_clear(DedupArgs a) {
    const unsigned long long m = used_slots(a);
    ulonglong2 *slot = reinterpret_cast<ulonglong2 *>(a.table);
    int *winner = reinterpret_cast<int *>(a.table + 2 * a.slots);
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < m;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        slot[i] = make_ulonglong2(~0ULL, ~0ULL);
        winner[i] = -1;
    }
}

__global__ void dedup_insert(DedupArgs a) {
    const long long n = num_records(a);
    unsigned long long *tab = a.table;   // key of slot s at 2 s, its value at 2 s + 1
    const unsigned long long used = used_slots(a), mask = used - 1;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        RecDev r = a.recs[i];
        unsigned long long h = rec_hash(r), v = rec_value(r);
        unsigned long long s = h & mask;
        for (unsigned long long probe = 0; probe < used; ++probe) {
            unsigned long long prev = atomicCAS(tab + 2 * s, ~0ULL, h);
            if (prev == ~0ULL || prev == h) {
                atomicMin(tab + 2 * s + 1, v);
                a.recs[i].slot = (int)s;
                break;
            }
            s = (s + 1) & mask;
        }
    }
}

__global__ void dedup_select(DedupArgs a) {
    const long long n = num_records(a);
    const unsigned long long *tab = a.table;
    int *winner = reinterpret_cast<int *>(a.table + 2 * a.slots);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        RecDev r = a.recs[i];
        if (r.slot < 0) continue;
        if (tab[2 * (long long)r.slot + 1] != rec_value(r)) continue;
        winner[r.slot] = (int)i;
        if (a.shard_world > 1 && (r.tx * a.nrx + r.rx) % a.shard_world != a.shard_rank) continue;
        unsigned long long p = atomicAdd(reinterpret_cast<unsigned long long *>(a.counters + kPaths), 1ULL);
        if ((long long)p >= a.path_cap) continue;
        sbr_path_record out;
        out.tx = r.tx;
        out.rx = r.rx;
        out.ray = r.ray;
        out.order = r.order;
        for (int j = 0; j < kMaxOrder; ++j) out.faces[j] = r.faces[j];
        out.rough_err = r.err;
        out.rough_dray = r.dray;
        out.iters = 0;
        out.valid = 0;
        float4 d = __ldg(a.dirs + r.ray);
        out.dir[0] = d.x;
        out.dir[1] = d.y;
        out.dir[2] = d.z;
        out.err = r.err;
        out.delay = 0.0;
        out.aod[0] = out.aod[1] = out.aoa[0] = out.aoa[1] = 0.0f;
        out.power_dbm = 0.0f;
        out.flags = 0;
        a.paths[p] = out;
    }
}

__global__ void dedup_verify(DedupArgs a) {
    const long long n = num_records(a);
    const int *winner = reinterpret_cast<const int *>(a.table + 2 * a.slots);
    unsigned bad = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const RecDev &r = a.recs[i];
        if (r.slot < 0) {
            ++bad;
            continue;
        }
        int w = winner[r.slot];
        if (w == (int)i) continue;   // the winner itself
        if (w < 0 || !same_key(r, a.recs[w])) ++bad;
    }
    if (bad) atomicAdd(reinterpret_cast<unsigned long long *>(a.counters + kCollisions), (unsigned long long)bad);
}

cudaError_t launch_dedup(const DedupArgs &a, int num_sms, cudaStream_t s) {
    int grid = num_sms * 4;
    dedup_clear<<<grid, 256, 0, s>>>(a);
    dedup_insert<<<grid, 256, 0, s>>>(a);
    dedup_select<<<grid, 256, 0, s>>>(a);
    dedup_verify<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

__global__ void records_reset(long long *counters, long long n) {
    counters[kRecords] = n;
    counters[kPaths] = 0;
    counters[kCollisions] = 0;
}

cudaError_t launch_records_reset(long long *counters, long long n, cudaStream_t s) {
    records_reset<<<1, 1, 0, s>>>(counters, n);
    return cudaGetLastError();
}

// Valid paths with a non-finite output: an output scan (NaN / Inf in a valid path's
// direction, error angle, delay, angles or power means a numerical fault).
__device__ __forceinline__ bool finite_path(const sbr_path_record &p) {
    bool ok = isfinite(p.dir[0]) && isfinite(p.dir[1]) && isfinite(p.dir[2]) && isfinite(p.err) && isfinite(p.delay);
    ok = ok && isfinite(p.aod[0]) && isfinite(p.aod[1]) && isfinite(p.aoa[0]) && isfinite(p.aoa[1]);
    return ok && isfinite(p.power_dbm);
}

__global__ void nonfinite_scan(const sbr_path_record *paths, long long *counters, long long cap) {
    long long n = counters[kPaths];
    if (n > cap) n = cap;
    unsigned bad = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const sbr_path_record &p = paths[i];
        if (p.valid && !finite_path(p)) ++bad;
    }
    bad = __reduce_add_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0 && bad)
        atomicAdd(reinterpret_cast<unsigned long long *>(counters + kNonFinite), (unsigned long long)bad);
}

cudaError_t launch_nonfinite_scan(const sbr_path_record *paths, long long *counters, int64_t path_cap, int num_sms,
                                  cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(counters + kNonFinite, 0, sizeof(long long), s);
    if (e != cudaSuccess) return e;
    nonfinite_scan<<<num_sms * 4, 256, 0, s>>>(paths, counters, path_cap);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------- pairs
// Group path indices by (tx, rx) pair: counts, exclusive scan (one block), scatter.
__global__ void pair_count(PairArgs a) {
    long long n = a.counters[kPaths];
    if (n > a.path_cap) n = a.path_cap;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int p = a.paths[i].tx * a.nrx + a.paths[i].rx;
        atomicAdd(a.pair_count + p, 1);
    }
}

__global__ void pair_scan(PairArgs a) {
    // single block: exclusive scan of pair_count[0..npairs) into pair_count, total at [npairs]
    __shared__ int carry;
    __shared__ int buf[1024];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < a.npairs; base += 1024) {
        int i = base + threadIdx.x;
        int v = i < a.npairs ? a.pair_count[i] : 0;
        buf[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {
            int t = threadIdx.x >= off ? buf[threadIdx.x - off] : 0;
            __syncthreads();
            buf[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < a.npairs) a.pair_count[i] = carry + buf[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += buf[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) a.pair_count[a.npairs] = carry;
}

__global__ void pair_scatter(PairArgs a, int *cursor) {
    long long n = a.counters[kPaths];
    if (n > a.path_cap) n = a.path_cap;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int p = a.paths[i].tx * a.nrx + a.paths[i].rx;
        int at = atomicAdd(cursor + p, 1);
        a.pair_idx[at] = (int)i;
    }
}

cudaError_t launch_pair_bucket(const PairArgs &a, cudaStream_t s) {
    // cursor lives after pair_idx: [npairs] ints (caller sized pair_idx + npairs)
    int *cursor = a.pair_idx + a.path_cap;
    cudaError_t e = cudaMemsetAsync(a.pair_count, 0, sizeof(int) * (size_t)(a.npairs + 1), s);
    if (e != cudaSuccess) return e;
    pair_count<<<256, 256, 0, s>>>(a);
    pair_scan<<<1, 1024, 0, s>>>(a);
    e = cudaMemcpyAsync(cursor, a.pair_count, sizeof(int) * (size_t)a.npairs, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    pair_scatter<<<256, 256, 0, s>>>(a, cursor);
    return cudaGetLastError();
}

}  // namespace sbr
