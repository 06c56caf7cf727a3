// host_wedges.cpp -- the scene's wedges for order-1 diffraction (§III.A: rays diffract on
// the scene's wedges; both path tests name faces and wedges).
//
// A wedge is a side shared by two faces -- the same segment, with identical endpoint
// coordinates, on the boundary of both -- whose half-planes meet at an interior angle
// between 1 and 170 degrees.  A face's sides are its boundary triangle edges (edges no
// other triangle of the same face uses, matched by vertex id) with collinear neighbours
// that share a vertex joined.  The solid fills the smaller sector between the two
// half-planes; w1, w2 are the unit vectors perpendicular to the edge pointing into face f1
// and f2 (towards the mean of each face's triangle vertices).  Wedges are numbered in
// the order of their face pairs (f1 < f2), the ids the path records carry.
#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <tuple>

#include "sbr_internal.h"

namespace sbr {

namespace {

struct V3 {
    double x, y, z;
};
V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
V3 operator*(V3 a, double s) { return {a.x * s, a.y * s, a.z * s}; }
double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
V3 cross(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
double len(V3 a) { return std::sqrt(dot(a, a)); }
V3 unit(V3 a) { return a * (1.0 / len(a)); }

struct Side {
    int ia, ib;   // vertex ids of the ends
};

}  // namespace

bool build_wedges(const float *verts, int64_t nv, const int32_t *tris, const int32_t *tri_face, int64_t nt, int nf,
                  std::vector<WedgeHost> &out) {
    out.clear();
    if (nt <= 0 || nf <= 0) return true;
    auto P = [&](int i) { return V3{verts[3 * i], verts[3 * i + 1], verts[3 * i + 2]}; };
    // triangle edges keyed by (face, lower vertex id, higher vertex id); boundary = used once
    std::vector<std::tuple<int, int, int, int, int>> edges;   // face, lo, hi, a, b (a -> b as in the triangle)
    edges.reserve(3 * (size_t)nt);
    std::vector<V3> centre((size_t)nf, V3{0, 0, 0});
    std::vector<double> count((size_t)nf, 0.0);
    for (int64_t t = 0; t < nt; ++t) {
        int f = tri_face[t];
        for (int k = 0; k < 3; ++k) {
            int a = tris[3 * t + k], b = tris[3 * t + (k + 1) % 3];
            edges.emplace_back(f, std::min(a, b), std::max(a, b), a, b);
            V3 p = P(a);
            centre[f] = {centre[f].x + p.x, centre[f].y + p.y, centre[f].z + p.z};
            count[f] += 1.0;
        }
    }
    for (int f = 0; f < nf; ++f)
        if (count[f] > 0) centre[f] = centre[f] * (1.0 / count[f]);
    std::sort(edges.begin(), edges.end());
    // boundary edges per face, then collinear neighbours joined
    std::vector<std::vector<Side>> sides((size_t)nf);
    for (size_t i = 0; i < edges.size();) {
        size_t j = i;
        while (j < edges.size() && std::get<0>(edges[j]) == std::get<0>(edges[i]) &&
               std::get<1>(edges[j]) == std::get<1>(edges[i]) && std::get<2>(edges[j]) == std::get<2>(edges[i]))
            ++j;
        if (j - i == 1) sides[std::get<0>(edges[i])].push_back({std::get<3>(edges[i]), std::get<4>(edges[i])});
        i = j;
    }
    std::vector<std::tuple<std::array<float, 6>, int>> keyed;   // (lo xyz, hi xyz), face
    for (int f = 0; f < nf; ++f) {
        std::vector<Side> &S = sides[f];
        std::vector<char> alive(S.size(), 1);
        bool merged = true;
        while (merged) {
            merged = false;
            for (size_t i = 0; i < S.size(); ++i) {
                if (!alive[i]) continue;
                for (size_t j = 0; j < S.size(); ++j) {
                    if (j == i || !alive[j]) continue;
                    int pf, qf;   // far ends of i and j when they share a vertex
                    if (S[i].ib == S[j].ia) { pf = S[i].ia; qf = S[j].ib; }
                    else if (S[i].ib == S[j].ib) { pf = S[i].ia; qf = S[j].ia; }
                    else if (S[i].ia == S[j].ia) { pf = S[i].ib; qf = S[j].ib; }
                    else if (S[i].ia == S[j].ib) { pf = S[i].ib; qf = S[j].ia; }
                    else continue;
                    V3 d1 = P(S[i].ib) - P(S[i].ia), d2 = P(S[j].ib) - P(S[j].ia);
                    if (len(cross(d1, d2)) > 1e-6 * len(d1) * len(d2)) continue;
                    S[i] = {pf, qf};
                    alive[j] = 0;
                    merged = true;
                }
            }
        }
        for (size_t i = 0; i < S.size(); ++i) {
            if (!alive[i]) continue;
            std::array<float, 3> a = {verts[3 * S[i].ia], verts[3 * S[i].ia + 1], verts[3 * S[i].ia + 2]};
            std::array<float, 3> b = {verts[3 * S[i].ib], verts[3 * S[i].ib + 1], verts[3 * S[i].ib + 2]};
            if (b < a) std::swap(a, b);
            keyed.emplace_back(std::array<float, 6>{a[0], a[1], a[2], b[0], b[1], b[2]}, f);
        }
    }
    std::sort(keyed.begin(), keyed.end());
    for (size_t i = 0; i < keyed.size();) {
        size_t j = i;
        while (j < keyed.size() && std::get<0>(keyed[j]) == std::get<0>(keyed[i])) ++j;
        if (j - i == 2 && std::get<1>(keyed[i]) != std::get<1>(keyed[i + 1])) {
            const std::array<float, 6> &k = std::get<0>(keyed[i]);
            WedgeHost w;
            V3 a{k[0], k[1], k[2]}, b{k[3], k[4], k[5]};
            V3 e = unit(b - a);
            w.f1 = std::get<1>(keyed[i]);
            w.f2 = std::get<1>(keyed[i + 1]);
            V3 c1 = centre[w.f1] - a, c2 = centre[w.f2] - a;
            V3 w1 = unit(c1 - e * dot(c1, e)), w2 = unit(c2 - e * dot(c2, e));
            double phi = std::atan2(len(cross(w1, w2)), dot(w1, w2)) * (180.0 / 3.14159265358979323846);
            if (phi >= 1.0 && phi <= 170.0) {
                for (int q = 0; q < 3; ++q) {
                    w.a[q] = k[q];
                    w.b[q] = k[3 + q];
                }
                w.w1[0] = w1.x; w.w1[1] = w1.y; w.w1[2] = w1.z;
                w.w2[0] = w2.x; w.w2[1] = w2.y; w.w2[2] = w2.z;
                out.push_back(w);
            }
        }
        i = j;
    }
    std::sort(out.begin(), out.end(),
              [](const WedgeHost &p, const WedgeHost &q) { return std::tie(p.f1, p.f2) < std::tie(q.f1, q.f2); });
    (void)nv;
    return true;
}

}  // namespace sbr
