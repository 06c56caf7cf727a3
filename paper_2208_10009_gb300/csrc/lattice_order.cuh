// lattice_order.cuh -- index arithmetic of the equiangular lattice (§II.B) shared by ray
// generation, the trace and the diffraction search: the layer prefix and the schedule in
// which a whole-lattice launch takes its rays.
#pragma once

#include <cuda_runtime.h>

namespace sbr {

// interior points of layers 1..a of a face: S(a) = sum_{a'=1..a} 3(n - 3a') (fits 32 bits
// for n <= 14000)
__device__ __forceinline__ int layer_prefix(int n, int a) { return (6 * n * a - 9 * a * a - 9 * a) / 2; }

// ------------------------------------------------------------------ trace schedule
// The order in which the trace and the diffraction search take the rays of a whole
// equiangular-lattice launch (rays are independent, §III.A, so no result depends on it).  Lattice id order runs along the rings
// of a face's layers (§II.B): the 24-32 consecutive ids of a warp's refill form a thin strip
// of directions.  The schedule maps work index w in [0, N) to a ray id so that they form a
// compact patch instead.  The vertex and edge rays keep their ids.  A face's interior points
// are the triangular grid p0 + p1 + p2 = n, every p_k >= 1: layer a is the ring min(p) = a,
// and its side e runs from the layer's vertex e (nearest the face's corner e) towards vertex
// e + 1, so the ring index of (p0, p1, p2) is e (n - 3a) + j with (e, j) = (0, p1 - a) where
// p2 = a < p0, (1, p2 - a) where p0 = a < p1, and (2, p0 - a) where p1 = a < p2.  The points
// are taken in tiles of kTileRows values of p0 by kTileCols of p1, a block of rows at a time:
// its full tiles, then the rest of its rows (the staircase under the grid's diagonal); every
// other block runs the other way, so consecutive tiles stay neighbours.
constexpr int kTileRows = 6, kTileCols = 4;

// interior points in rows p0 = 1..x of a face (row p0 holds n - 1 - p0 of them)
__device__ __forceinline__ int rows_before(int n, int x) { return x * (n - 1) - x * (x + 1) / 2; }

__device__ __forceinline__ int grid_ray(int n, int face_base, int p0, int p1) {
    const int p2 = n - p0 - p1;
    const int a = min(p0, min(p1, p2)), m = n - 3 * a;
    const int base = face_base + layer_prefix(n, a - 1);
    if (m == 0) return base;   // the face centre (n = 0 mod 3)
    if (p2 == a && p0 > a) return base + (p1 - a);
    if (p0 == a && p1 > a) return base + m + (p2 - a);
    return base + 2 * m + (p0 - a);
}

// point qs of the staircase of the block of rows s..e (full tiles cover columns 1..fw)
__device__ __forceinline__ int staircase_ray(int n, int face_base, int s, int e, int fw, int qs) {
    for (int p0 = s; p0 < e; ++p0) {
        const int len = n - 1 - p0 - fw;
        if (qs < len) return grid_ray(n, face_base, p0, fw + 1 + qs);
        qs -= len;
    }
    return grid_ray(n, face_base, e, fw + 1 + qs);
}

__device__ __forceinline__ int tiled_ray(int w, int n) {
    const int E = 12 + 30 * (n - 1);
    if (w < E) return w;
    const int per_face = (n - 1) * (n - 2) / 2;
    const int r = w - E, f = r / per_face, q = r - f * per_face;
    const int face_base = E + f * per_face;
    // q's row in plain row-major order: the largest x with rows_before(x) <= q, from the
    // quadratic, then fixed
    const float B = (float)(2 * n - 3);
    int x = (int)((B - sqrtf(fmaxf(B * B - 8.0f * (float)q, 0.0f))) * 0.5f);
    x = max(0, min(x, n - 3));
    while (x > 0 && rows_before(n, x) > q) --x;
    while (x < n - 3 && rows_before(n, x + 1) <= q) ++x;
    const int blk = x / kTileRows;
    const int s = blk * kTileRows + 1, e = min(s + kTileRows - 1, n - 2), h = e - s + 1;
    const int fw = (n - 1 - e) / kTileCols * kTileCols;   // columns of the full tiles
    const int full = fw * h;
    int qb = q - rows_before(n, s - 1);
    int t, rem;
    if (blk & 1) {
        const int stair = rows_before(n, e) - rows_before(n, s - 1) - full;
        if (qb < stair) return staircase_ray(n, face_base, s, e, fw, qb);
        qb -= stair;
        t = fw / kTileCols - 1 - qb / (kTileCols * h);
        rem = qb % (kTileCols * h);
    } else {
        if (qb >= full) return staircase_ray(n, face_base, s, e, fw, qb - full);
        t = qb / (kTileCols * h);
        rem = qb % (kTileCols * h);
    }
    return grid_ray(n, face_base, s + rem / kTileCols, 1 + t * kTileCols + rem % kTileCols);
}

}  // namespace sbr
