// host_faces.cpp -- convex outlines of planar faces, for the validity test's point-in-face
// query (§III.A: a refined path's bounce points must lie on their faces).
//
// A face is a set of triangles with one face id.  When those triangles tile a convex
// polygon exactly, "inside some triangle of the face" is "inside the polygon", and the
// device tests a bounce point against the polygon's few edges instead of walking the BVH
// down to the face's triangles (a tessellated wall has thousands).  Other faces keep the
// BVH query.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

#include "sbr_internal.h"

namespace sbr {

namespace {

struct P2 {
    double x, y;
    int src;   // index of the 3-D point it came from
};

double cross2(const P2 &o, const P2 &a, const P2 &b) { return (a.x - o.x) * (b.y - o.y) - (a.y - o.y) * (b.x - o.x); }

// Convex hull, counter-clockwise, collinear points dropped (Andrew's monotone chain).
std::vector<P2> hull2(std::vector<P2> p) {
    std::sort(p.begin(), p.end(), [](const P2 &a, const P2 &b) { return a.x < b.x || (a.x == b.x && a.y < b.y); });
    p.erase(std::unique(p.begin(), p.end(), [](const P2 &a, const P2 &b) { return a.x == b.x && a.y == b.y; }),
            p.end());
    if (p.size() < 3) return {};
    std::vector<P2> h(2 * p.size());
    size_t k = 0;
    for (size_t i = 0; i < p.size(); ++i) {
        while (k >= 2 && cross2(h[k - 2], h[k - 1], p[i]) <= 0.0) --k;
        h[k++] = p[i];
    }
    for (size_t i = p.size() - 1, t = k + 1; i-- > 0;) {
        while (k >= t && cross2(h[k - 2], h[k - 1], p[i]) <= 0.0) --k;
        h[k++] = p[i];
    }
    h.resize(k - 1);
    return h;
}

using Key = std::tuple<uint32_t, uint32_t, uint32_t>;

Key key_of(const float *v) {
    uint32_t b[3];
    std::memcpy(b, v, sizeof b);
    return Key{b[0], b[1], b[2]};
}

}  // namespace

// For every face whose triangles tile a convex polygon, the polygon's corners
// counter-clockwise about the face normal: outline[f] = (first corner, count) into
// corners, count 0 for a face left to the BVH query.  With the face's points projected on
// its plane, a face qualifies when its points lie on the plane (1e-6 of the face's size),
// every triangle turns like the normal, every directed edge (endpoints compared by their
// coordinates) occurs once at most, and the edges without a reverse twin (the boundary)
// add up to the convex hull's perimeter while the triangles add up to its area (both
// relative 1e-9).  Consistently oriented triangles that meet along twin edges, with a
// boundary as long as the hull's and the hull's area, cover the hull once: a point is in
// some triangle exactly when it is in the hull.
void build_face_outlines(const float *verts, const int32_t *tris, const int32_t *tri_face, int64_t nt, int nf,
                         const Plane64 *planes, std::vector<int2> &outline, std::vector<float4> &corners) {
    outline.assign((size_t)std::max(nf, 1), make_int2(0, 0));
    corners.clear();
    std::vector<int> off((size_t)nf + 1, 0), idx((size_t)nt);
    for (int64_t t = 0; t < nt; ++t) ++off[tri_face[t] + 1];
    for (int f = 0; f < nf; ++f) off[f + 1] += off[f];
    {
        std::vector<int> cur(off.begin(), off.end() - 1);
        for (int64_t t = 0; t < nt; ++t) idx[cur[tri_face[t]]++] = (int)t;
    }
    for (int f = 0; f < nf; ++f) {
        const int t0 = off[f], t1 = off[f + 1];
        if (t1 <= t0) continue;
        const Plane64 &pl = planes[f];
        const double n[3] = {pl.x, pl.y, pl.z};
        // in-plane basis u, v with u x v = n
        double e[3] = {0, 0, 0};
        e[std::fabs(n[0]) <= std::fabs(n[1]) && std::fabs(n[0]) <= std::fabs(n[2]) ? 0
          : (std::fabs(n[1]) <= std::fabs(n[2]) ? 1 : 2)] = 1.0;
        double u[3] = {e[1] * n[2] - e[2] * n[1], e[2] * n[0] - e[0] * n[2], e[0] * n[1] - e[1] * n[0]};
        const double ul = std::sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        for (double &c : u) c /= ul;
        const double v[3] = {n[1] * u[2] - n[2] * u[1], n[2] * u[0] - n[0] * u[2], n[0] * u[1] - n[1] * u[0]};
        auto proj = [&](const float *q, int src) {
            return P2{u[0] * q[0] + u[1] * q[1] + u[2] * q[2], v[0] * q[0] + v[1] * q[1] + v[2] * q[2], src};
        };
        std::vector<P2> pts;
        std::map<std::pair<Key, Key>, int> dir_edges;
        double area = 0.0, size = 0.0, max_off = 0.0;
        bool ok = true;
        for (int i = t0; i < t1 && ok; ++i) {
            const int t = idx[i];
            const float *q[3] = {verts + 3 * (size_t)tris[3 * t], verts + 3 * (size_t)tris[3 * t + 1],
                                 verts + 3 * (size_t)tris[3 * t + 2]};
            P2 a[3];
            for (int c = 0; c < 3; ++c) {
                a[c] = proj(q[c], tris[3 * t + c]);
                pts.push_back(a[c]);
                max_off = std::max(max_off, std::fabs(n[0] * q[c][0] + n[1] * q[c][1] + n[2] * q[c][2] - pl.w));
                size = std::max(size, std::fabs(a[c].x) + std::fabs(a[c].y));
            }
            const double s = cross2(a[0], a[1], a[2]);
            if (!(s > 0.0)) ok = false;
            area += 0.5 * s;
            for (int c = 0; c < 3; ++c) {
                auto k = std::make_pair(key_of(q[c]), key_of(q[(c + 1) % 3]));
                if (++dir_edges[k] > 1) ok = false;
            }
        }
        if (!ok || max_off > 1e-6 * (size + 1.0)) continue;
        double blen = 0.0;
        for (const auto &de : dir_edges) {
            if (dir_edges.count(std::make_pair(de.first.second, de.first.first))) continue;
            const Key &ka = de.first.first, &kb = de.first.second;
            float A[3], B[3];
            uint32_t ba[3] = {std::get<0>(ka), std::get<1>(ka), std::get<2>(ka)};
            uint32_t bb[3] = {std::get<0>(kb), std::get<1>(kb), std::get<2>(kb)};
            std::memcpy(A, ba, sizeof A);
            std::memcpy(B, bb, sizeof B);
            const P2 pa = proj(A, -1), pb = proj(B, -1);
            blen += std::hypot(pb.x - pa.x, pb.y - pa.y);
        }
        const std::vector<P2> h = hull2(pts);
        if (h.size() < 3 || h.size() > (size_t)kMaxOutline) continue;
        double harea = 0.0, hper = 0.0;
        for (size_t i = 0; i < h.size(); ++i) {
            const P2 &a = h[i], &b = h[(i + 1) % h.size()];
            harea += 0.5 * (a.x * b.y - a.y * b.x);
            hper += std::hypot(b.x - a.x, b.y - a.y);
        }
        if (!(std::fabs(area - harea) <= 1e-9 * harea) || !(std::fabs(blen - hper) <= 1e-9 * hper)) continue;
        outline[f] = make_int2((int)corners.size(), (int)h.size());
        for (const P2 &c : h) {
            const float *q = verts + 3 * (size_t)c.src;
            corners.push_back(make_float4(q[0], q[1], q[2], 0.0f));
        }
    }
    if (corners.empty()) corners.push_back(make_float4(0, 0, 0, 0));
}

}  // namespace sbr
