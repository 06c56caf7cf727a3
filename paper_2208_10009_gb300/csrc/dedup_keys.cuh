// dedup_keys.cuh -- the keys of double-count removal (§III.A, first path test), shared by
// sbr_launch's dedup kernels (kernels_paths.cu) and sbr_dedup_noalloc (noalloc.cu) so that
// both pick the same winner.
#pragma once

#include "sbr_internal.h"

namespace sbr {

// A 64-bit hash of (Tx, Rx, order,
// face sequence) (SplitMix64's finaliser as the mixing step), the value (error-angle bits,
// ray id) whose minimum wins (error angles are >= 0, so their IEEE bits order like the
// values; ties go to the lowest ray id), and the full key comparison that detects a hash
// collision.
__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
    x += 0x9E3779B97F4A7C15ULL;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
    return x ^ (x >> 31);
}

__device__ __forceinline__ unsigned long long rec_hash(const RecDev &r) {
    unsigned long long h = mix64(((unsigned long long)(unsigned)r.tx << 40) ^ ((unsigned long long)(unsigned)r.rx << 8) ^
                                 (unsigned long long)r.order);
    for (int j = 0; j < r.order; ++j) h = mix64(h ^ (unsigned long long)(unsigned)(r.faces[j] + 1));
    return h == ~0ULL ? 0x5bd1e995ULL : h;
}

__device__ __forceinline__ unsigned long long rec_value(const RecDev &r) {
    return ((unsigned long long)__float_as_uint(r.err) << 32) | (unsigned)r.ray;
}

__device__ __forceinline__ bool same_key(const RecDev &a, const RecDev &b) {
    if (a.tx != b.tx || a.rx != b.rx || a.order != b.order) return false;
    for (int j = 0; j < a.order; ++j)
        if (a.faces[j] != b.faces[j]) return false;
    return true;
}

// Hash-table slots a dedup pass over n records uses: the smallest power of two >= 2 n
// (at least 1024, at most `slots`), so that few records clear and probe a small table that
// stays in L2 (the distinct keys are at most n: load factor <= 1/2).
__device__ __forceinline__ unsigned long long dedup_slots(long long n, long long slots) {
    long long s = 1024;
    while (s < 2 * n && s < slots) s <<= 1;
    return (unsigned long long)(s < slots ? s : slots);
}

}  // namespace sbr
