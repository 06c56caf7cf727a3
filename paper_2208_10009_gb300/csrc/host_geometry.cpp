// host_geometry.cpp -- host-side construction for the CUDA path: binned-SAH BVH, the
// equiangular lattice's layer tables (§II.B, Eq. 1-2) and the precise algorithm's
// sub-ray patterns (§III.B, Fig. 5).
#include <unistd.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <functional>
#include <mutex>
#include <numeric>
#include <system_error>
#include <thread>

#include "sbr_internal.h"

namespace sbr {

// ============================================================================ BVH
namespace {

struct Box {
    float lo[3] = {INFINITY, INFINITY, INFINITY};
    float hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    void grow(const float *l, const float *h) {
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::min(lo[a], l[a]);
            hi[a] = std::max(hi[a], h[a]);
        }
    }
    void grow(const Box &b) { grow(b.lo, b.hi); }
    float area() const {
        if (!(hi[0] >= lo[0])) return 0.0f;
        float dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
        return 2.0f * (dx * dy + dy * dz + dz * dx);
    }
};

struct TmpNode {
    Box box;
    int left = -1, right = -1;   // children (TmpNode ids) or -1 for a leaf
    int first = 0, count = 0;
};

// Right subtrees of at least this many primitives, within this many levels of the root,
// are built by the subtree pool's threads.
constexpr int kParallelMin = 256, kParallelDepth = 7;

// Worker threads for the builder's subtrees, started on first use and kept for the process
// (a thread start costs tens of microseconds, a good part of a small tree such as the
// receivers').  A thread that waits for a subtree runs queued subtrees meanwhile, so waits
// nested inside subtrees always leave a runnable task to some thread, and a process forked
// after the pool started (its workers do not exist there) runs every subtree itself.
class SubtreePool {
public:
    static SubtreePool &get() {
        static SubtreePool pool;
        return pool;
    }
    void submit(std::function<void()> f) {
        {
            std::lock_guard<std::mutex> l(m_);
            q_.push_back(std::move(f));
        }
        cv_.notify_one();
    }
    // runs one queued subtree; false if none was queued
    bool run_one() {
        std::function<void()> f;
        {
            std::lock_guard<std::mutex> l(m_);
            if (q_.empty()) return false;
            f = std::move(q_.front());
            q_.pop_front();
        }
        f();
        return true;
    }
    ~SubtreePool() {
        {
            std::lock_guard<std::mutex> l(m_);
            stop_ = true;
        }
        cv_.notify_all();
        for (auto &t : workers_) {
            if (getpid() == owner_ && t.joinable()) t.join();
            else if (t.joinable()) t.detach();
        }
    }

private:
    SubtreePool() : owner_(getpid()) {
        const unsigned hw = std::thread::hardware_concurrency();
        const unsigned n = hw > 1 ? std::min(hw - 1, 31u) : 0u;
        try {
            for (unsigned i = 0; i < n; ++i) workers_.emplace_back([this] { loop(); });
        } catch (const std::system_error &) {
            // fewer workers: waiting threads run the subtrees themselves
        }
    }
    void loop() {
        for (;;) {
            std::function<void()> f;
            {
                std::unique_lock<std::mutex> l(m_);
                cv_.wait(l, [this] { return stop_ || !q_.empty(); });
                if (q_.empty()) return;   // stopping
                f = std::move(q_.front());
                q_.pop_front();
            }
            f();
        }
    }
    std::mutex m_;
    std::condition_variable cv_;
    std::deque<std::function<void()>> q_;
    std::vector<std::thread> workers_;
    bool stop_ = false;
    pid_t owner_;
};

struct Builder {
    const std::vector<float> &lo, &hi;
    const std::vector<float> &cen;   // box centres, shared by the builders of one tree
    std::vector<int> &idx;           // primitive order, each builder permuting its own range
    std::vector<TmpNode> nodes;
    int leaf_max;
    int depth = 0, max_leaf = 0;

    Builder(const std::vector<float> &l, const std::vector<float> &h, const std::vector<float> &c,
            std::vector<int> &ix, int lm)
        : lo(l), hi(h), cen(c), idx(ix), leaf_max(lm) {}

    // The right subtree [mid, first + count) built by the subtree pool while this thread
    // builds the left one: it partitions only its own range of idx, and its nodes are
    // appended after the left subtree's, in the order the serial recursion gives them, so
    // the tree and its numbering do not depend on the threads.  Returns the subtree's root.
    int make_split(int first, int count, int mid, int d, int &l) {
        Builder rb(lo, hi, cen, idx, leaf_max);
        std::atomic<bool> done{false};
        SubtreePool &pool = SubtreePool::get();
        pool.submit([&rb, &done, mid, first, count, d] {
            rb.make(mid, first + count - mid, d + 1);
            done.store(true, std::memory_order_release);
        });
        l = make(first, mid - first, d + 1);
        while (!done.load(std::memory_order_acquire))
            if (!pool.run_one()) std::this_thread::yield();
        const int off = (int)nodes.size();
        for (TmpNode t : rb.nodes) {
            if (t.left >= 0) {
                t.left += off;
                t.right += off;
            }
            nodes.push_back(t);
        }
        depth = std::max(depth, rb.depth);
        max_leaf = std::max(max_leaf, rb.max_leaf);
        return off;
    }

    int make(int first, int count, int d) {
        depth = std::max(depth, d);
        int id = (int)nodes.size();
        nodes.emplace_back();
        Box b, cb;
        for (int i = first; i < first + count; ++i) {
            int p = idx[i];
            b.grow(&lo[3 * p], &hi[3 * p]);
            cb.grow(&cen[3 * p], &cen[3 * p]);
        }
        nodes[id].box = b;
        nodes[id].first = first;
        nodes[id].count = count;
        if (count <= leaf_max || d >= kStackDepth - 8) {
            max_leaf = std::max(max_leaf, count);
            return id;
        }
        // binned SAH over the centroid bounds
        const int B = 32;
        float best_cost = INFINITY;
        int best_axis = -1, best_split = 0;
        for (int a = 0; a < 3; ++a) {
            float ext = cb.hi[a] - cb.lo[a];
            if (!(ext > 0.0f)) continue;
            // only the occupied bins are set up and swept: the split cost is the same for
            // every bin boundary between two occupied bins, and the first of them (just past
            // the lower occupied bin) is the one the strict comparison keeps, so the choice
            // equals a sweep over all B boundaries at a cost that follows the node's size
            struct BinBox {
                float lo[3], hi[3];
            } bins[B];   // set when a bin is first occupied
            int cnt[B];
            unsigned occ = 0;
            float scale = B / ext;
            for (int i = first; i < first + count; ++i) {
                int p = idx[i];
                int k = std::min(B - 1, (int)((cen[3 * p + a] - cb.lo[a]) * scale));
                BinBox &bb = bins[k];
                if (!(occ >> k & 1u)) {
                    occ |= 1u << k;
                    for (int e = 0; e < 3; ++e) {
                        bb.lo[e] = lo[3 * p + e];
                        bb.hi[e] = hi[3 * p + e];
                    }
                    cnt[k] = 1;
                    continue;
                }
                for (int e = 0; e < 3; ++e) {
                    bb.lo[e] = std::min(bb.lo[e], lo[3 * p + e]);
                    bb.hi[e] = std::max(bb.hi[e], hi[3 * p + e]);
                }
                ++cnt[k];
            }
            int ob[B], no = 0;
            for (unsigned m = occ; m; m &= m - 1) ob[no++] = __builtin_ctz(m);
            float right_area[B];
            int right_cnt[B];
            Box acc;
            int c = 0;
            for (int j = no - 1; j >= 1; --j) {   // right side of the boundary below ob[j]
                acc.grow(bins[ob[j]].lo, bins[ob[j]].hi);
                c += cnt[ob[j]];
                right_area[j] = acc.area();
                right_cnt[j] = c;
            }
            Box lacc;
            int lc = 0;
            for (int j = 1; j < no; ++j) {
                lacc.grow(bins[ob[j - 1]].lo, bins[ob[j - 1]].hi);
                lc += cnt[ob[j - 1]];
                float cost = lacc.area() * lc + right_area[j] * right_cnt[j];
                if (cost < best_cost) {
                    best_cost = cost;
                    best_axis = a;
                    best_split = ob[j - 1] + 1;
                }
            }
        }
        int mid;
        if (best_axis < 0) {
            // all centroids coincide: split the range in half
            mid = first + count / 2;
        } else {
            float leaf_cost = b.area() * count;
            float inner_cost = 0.125f * b.area() + best_cost;  // traversal cost ~ 1/8 triangle
            if (inner_cost >= leaf_cost && count <= 2 * leaf_max) {
                max_leaf = std::max(max_leaf, count);
                return id;
            }
            float ext = cb.hi[best_axis] - cb.lo[best_axis];
            float scale = B / ext;
            auto it = std::partition(idx.begin() + first, idx.begin() + first + count, [&](int p) {
                int k = std::min(B - 1, (int)((cen[3 * p + best_axis] - cb.lo[best_axis]) * scale));
                return k < best_split;
            });
            mid = (int)(it - idx.begin());
            if (mid == first || mid == first + count) mid = first + count / 2;
        }
        int l = -1, r = -1;
        if (count >= kParallelMin && d <= kParallelDepth) {
            r = make_split(first, count, mid, d, l);
        } else {
            l = make(first, mid - first, d + 1);
            r = make(mid, first + count - mid, d + 1);
        }
        nodes[id].left = l;
        nodes[id].right = r;
        return id;
    }
};

void put_child(float4 *n, int slot, const Box &b) {
    float *f = reinterpret_cast<float *>(n);
    int o = slot == 0 ? 0 : 6;
    if (!(b.hi[0] >= b.lo[0])) {
        // empty child: a point far outside any scene (its leaf has no primitives)
        for (int a = 0; a < 6; ++a) f[o + a] = 1e30f;
        return;
    }
    f[o + 0] = b.lo[0]; f[o + 1] = b.lo[1]; f[o + 2] = b.lo[2];
    f[o + 3] = b.hi[0]; f[o + 4] = b.hi[1]; f[o + 5] = b.hi[2];
}

}  // namespace

bool build_bvh(const std::vector<float> &lo, const std::vector<float> &hi, int leaf_max, BvhOut &out,
               std::string &err) {
    size_t n = lo.size() / 3;
    if (n >= (1u << 24)) {
        err = "BVH: more than 2^24 primitives";
        return false;
    }
    std::vector<float> cen(3 * n);
    for (size_t i = 0; i < 3 * n; ++i) cen[i] = 0.5f * (lo[i] + hi[i]);
    std::vector<int> prims(n);
    std::iota(prims.begin(), prims.end(), 0);
    Builder b(lo, hi, cen, prims, leaf_max);
    if (n > 0) b.make(0, (int)n, 1);
    // Flatten: every inner TmpNode becomes one 64-byte node holding its children.
    std::vector<int> flat_id(b.nodes.size(), -1);
    std::vector<int> order;   // TmpNode ids of inner nodes, preorder
    std::vector<int> stack;
    if (!b.nodes.empty() && b.nodes[0].left >= 0) stack.push_back(0);
    while (!stack.empty()) {
        int id = stack.back();
        stack.pop_back();
        flat_id[id] = (int)order.size();
        order.push_back(id);
        const TmpNode &t = b.nodes[id];
        if (b.nodes[t.right].left >= 0) stack.push_back(t.right);
        if (b.nodes[t.left].left >= 0) stack.push_back(t.left);
    }
    out.nodes.clear();
    auto ref_of = [&](int id) {
        const TmpNode &t = b.nodes[id];
        return t.left >= 0 ? flat_id[id] : leaf_ref(t.first, t.count);
    };
    if (order.empty()) {
        // root is a leaf (or the scene is empty): one node with the leaf and an empty child
        float4 nd[4];
        std::memset(nd, 0, sizeof(nd));
        Box empty;
        Box root = b.nodes.empty() ? empty : b.nodes[0].box;
        put_child(nd, 0, root);
        put_child(nd, 1, empty);
        int *ref = reinterpret_cast<int *>(&nd[3]);
        ref[0] = leaf_ref(0, (int)n);
        ref[1] = leaf_ref(0, 0);
        out.nodes.assign(nd, nd + 4);
    } else {
        out.nodes.resize(order.size() * 4);
        for (size_t i = 0; i < order.size(); ++i) {
            const TmpNode &t = b.nodes[order[i]];
            float4 *nd = &out.nodes[4 * i];
            std::memset(nd, 0, 4 * sizeof(float4));
            put_child(nd, 0, b.nodes[t.left].box);
            put_child(nd, 1, b.nodes[t.right].box);
            int *ref = reinterpret_cast<int *>(&nd[3]);
            ref[0] = ref_of(t.left);
            ref[1] = ref_of(t.right);
        }
    }
    if (b.max_leaf > 127) {
        err = "BVH: leaf larger than 127 primitives (degenerate input)";
        return false;
    }
    // 4-wide collapse: a node adopts the children of its largest inner children until it
    // has four (or none of its children is inner).
    {
        std::vector<std::array<int, 4>> kids;
        std::vector<int> nkids;
        std::vector<int> wide_of(b.nodes.size(), -1);
        auto collapse = [&](int id) {
            std::array<int, 4> c = {-1, -1, -1, -1};
            int n = 0;
            const TmpNode &t = b.nodes[id];
            if (t.left < 0) {
                c[n++] = id;   // a leaf root
            } else {
                c[n++] = t.left;
                c[n++] = t.right;
                while (n < 4) {
                    int best = -1;
                    float area = -1.0f;
                    for (int i = 0; i < n; ++i) {
                        const TmpNode &ch = b.nodes[c[i]];
                        if (ch.left >= 0 && ch.box.area() > area) {
                            area = ch.box.area();
                            best = i;
                        }
                    }
                    if (best < 0) break;
                    int inner = c[best];
                    c[best] = b.nodes[inner].left;
                    c[n++] = b.nodes[inner].right;
                }
            }
            return std::make_pair(c, n);
        };
        std::vector<int> order4, st4;
        if (!b.nodes.empty()) st4.push_back(0);
        while (!st4.empty()) {
            int id = st4.back();
            st4.pop_back();
            wide_of[id] = (int)order4.size();
            order4.push_back(id);
            auto cn = collapse(id);
            kids.push_back(cn.first);
            nkids.push_back(cn.second);
            for (int i = cn.second - 1; i >= 0; --i)
                if (b.nodes[cn.first[i]].left >= 0 && cn.first[i] != id) st4.push_back(cn.first[i]);
        }
        out.nodes4.assign(order4.size() > 0 ? order4.size() * 8 : 8, make_float4(0, 0, 0, 0));
        auto put4 = [&](float4 *nd, int slot, const Box &bx) {
            float *f = reinterpret_cast<float *>(nd);
            bool empty = !(bx.hi[0] >= bx.lo[0]);
            for (int a = 0; a < 3; ++a) {
                f[(2 * a) * 4 + slot] = empty ? 1e30f : bx.lo[a];
                f[(2 * a + 1) * 4 + slot] = empty ? 1e30f : bx.hi[a];
            }
        };
        if (order4.empty()) {
            Box empty;
            for (int i = 0; i < 4; ++i) put4(&out.nodes4[0], i, empty);
            int *ref = reinterpret_cast<int *>(&out.nodes4[6]);
            for (int i = 0; i < 4; ++i) ref[i] = leaf_ref(0, 0);
        }
        // worst-case stack: along a root-to-leaf path every node pushes up to nkids - 1
        // siblings that stay on the stack while its subtree is traversed
        {
            std::vector<int> need(order4.size(), 0);
            for (size_t w = order4.size(); w-- > 0;) {
                int deepest = 0;
                for (int i = 0; i < nkids[w]; ++i) {
                    int c = kids[w][i];
                    if (b.nodes[c].left >= 0 && c != order4[w]) deepest = std::max(deepest, need[wide_of[c]]);
                }
                need[w] = nkids[w] - 1 + deepest;
            }
            out.max_stack4 = need.empty() ? 0 : need[0];
        }
        for (size_t w = 0; w < order4.size(); ++w) {
            float4 *nd = &out.nodes4[8 * w];
            int *ref = reinterpret_cast<int *>(&nd[6]);
            Box empty;
            for (int i = 0; i < 4; ++i) {
                int c = i < nkids[w] ? kids[w][i] : -1;
                if (c < 0) {
                    put4(nd, i, empty);
                    ref[i] = leaf_ref(0, 0);
                    continue;
                }
                const TmpNode &t = b.nodes[c];
                put4(nd, i, t.box);
                ref[i] = (t.left >= 0 && c != order4[w]) ? wide_of[c] : leaf_ref(t.first, t.count);
            }
        }
    }
    out.prim_order = b.idx;
    out.depth = b.depth;
    out.max_leaf = b.max_leaf;
    return true;
}

// ============================================================================ lattice
namespace {

struct D3 {
    double x, y, z;
};
D3 d3(double x, double y, double z) { return {x, y, z}; }
D3 operator+(D3 a, D3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
D3 operator-(D3 a, D3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
D3 operator*(D3 a, double s) { return {a.x * s, a.y * s, a.z * s}; }
double dot3(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
D3 cross3(D3 a, D3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
D3 normed(D3 a) { return a * (1.0 / std::sqrt(dot3(a, a))); }
double arc(D3 a, D3 b) { return std::atan2(std::sqrt(dot3(cross3(a, b), cross3(a, b))), dot3(a, b)); }

// point at fraction f along the great circle a -> b
D3 arc_point(D3 a, D3 b, double f) {
    double w = arc(a, b);
    return normed(a * std::sin((1.0 - f) * w) + b * std::sin(f * w));
}

}  // namespace

void build_lattice_tables(int n, std::vector<float4> &ico, std::vector<int2> &edges, std::vector<float4> &centre,
                          std::vector<float4> &layers, int &nl) {
    // Regular icosahedron: cyclic permutations of (0, +-1, +-phi), in this fixed order.
    const double g = 0.5 * (1.0 + std::sqrt(5.0));
    const double raw[12][3] = {{0, 1, g},  {0, -1, g},  {0, 1, -g},  {0, -1, -g}, {1, g, 0},  {-1, g, 0},
                               {1, -g, 0}, {-1, -g, 0}, {g, 0, 1},  {-g, 0, 1},  {g, 0, -1}, {-g, 0, -1}};
    D3 V[12];
    for (int i = 0; i < 12; ++i) V[i] = normed(d3(raw[i][0], raw[i][1], raw[i][2]));
    // adjacency: unnormalised vertices at distance 2
    auto adj = [&](int i, int j) {
        D3 a = d3(raw[i][0], raw[i][1], raw[i][2]), b = d3(raw[j][0], raw[j][1], raw[j][2]);
        return std::fabs(dot3(a - b, a - b) - 4.0) < 1e-9;
    };
    ico.assign(12, make_float4(0, 0, 0, 0));
    for (int i = 0; i < 12; ++i) ico[i] = make_float4((float)V[i].x, (float)V[i].y, (float)V[i].z, 0.0f);
    edges.clear();
    std::vector<int> F;   // 20 oriented faces, lowest vertex first
    for (int i = 0; i < 12; ++i)
        for (int j = i + 1; j < 12; ++j) {
            if (!adj(i, j)) continue;
            edges.push_back(make_int2(i, j));
            for (int k = j + 1; k < 12; ++k) {
                if (!adj(i, k) || !adj(j, k)) continue;
                D3 c = V[i] + V[j] + V[k];
                bool ccw = dot3(cross3(V[j] - V[i], V[k] - V[i]), c) > 0.0;
                F.push_back(i);
                F.push_back(ccw ? j : k);
                F.push_back(ccw ? k : j);
            }
        }
    nl = (n + 2) / 3;  // layers a >= 0 with n - 3a >= 1
    centre.assign(20, make_float4(0, 0, 0, 0));
    layers.assign((size_t)20 * nl * 3, make_float4(0, 0, 0, 0));
    for (int f = 0; f < 20; ++f) {
        D3 W[3] = {V[F[3 * f]], V[F[3 * f + 1]], V[F[3 * f + 2]]};
        D3 c = normed(W[0] + W[1] + W[2]);
        centre[f] = make_float4((float)c.x, (float)c.y, (float)c.z, 0.0f);
        for (int a = 0; a < nl; ++a) {
            for (int e = 0; e < 3; ++e) {
                D3 p = W[e], q = W[(e + 1) % 3];
                layers[((size_t)f * nl + a) * 3 + e] =
                    make_float4((float)p.x, (float)p.y, (float)p.z, (float)arc(p, q));
            }
            if (a + 1 == nl) break;
            // Eq. 2 (parallelogram rule): the next layer's vertex near W_e is W_e moved by
            // the vectors to its two layer-a neighbours, projected back onto the sphere.
            int m = n - 3 * a;
            D3 nw[3];
            for (int e = 0; e < 3; ++e) {
                D3 fwd = arc_point(W[e], W[(e + 1) % 3], 1.0 / m);
                D3 bwd = arc_point(W[e], W[(e + 2) % 3], 1.0 / m);
                nw[e] = normed(fwd + bwd - W[e]);
            }
            for (int e = 0; e < 3; ++e) W[e] = nw[e];
        }
    }
}

// ============================================================================ equidistant
bool build_polyhedron(int poly, std::vector<float4> &v, std::vector<int2> &e, std::vector<int4> &f) {
    std::vector<D3> V;
    if (poly == 20) {
        const double g = 0.5 * (1.0 + std::sqrt(5.0));
        const double raw[12][3] = {{0, 1, g},  {0, -1, g},  {0, 1, -g},  {0, -1, -g}, {1, g, 0},  {-1, g, 0},
                                   {1, -g, 0}, {-1, -g, 0}, {g, 0, 1},  {-g, 0, 1},  {g, 0, -1}, {-g, 0, -1}};
        for (auto &r : raw) V.push_back(normed(d3(r[0], r[1], r[2])));
    } else if (poly == 8) {
        const double raw[6][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
        for (auto &r : raw) V.push_back(d3(r[0], r[1], r[2]));
    } else {
        return false;
    }
    // neighbours subtend the polyhedron's smallest vertex angle
    double amin = 10.0;
    for (size_t i = 0; i < V.size(); ++i)
        for (size_t j = i + 1; j < V.size(); ++j) amin = std::min(amin, arc(V[i], V[j]));
    auto adj = [&](int i, int j) { return std::fabs(arc(V[i], V[j]) - amin) < 1e-9; };
    v.clear();
    e.clear();
    f.clear();
    for (auto &p : V) v.push_back(make_float4((float)p.x, (float)p.y, (float)p.z, 0.0f));
    int n = (int)V.size();
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            if (!adj(i, j)) continue;
            e.push_back(make_int2(i, j));
            for (int k = j + 1; k < n; ++k) {
                if (!adj(i, k) || !adj(j, k)) continue;
                D3 c = V[i] + V[j] + V[k];
                bool ccw = dot3(cross3(V[j] - V[i], V[k] - V[i]), c) > 0.0;
                f.push_back(make_int4(i, ccw ? j : k, ccw ? k : j, 0));
            }
        }
    return true;
}

// ============================================================================ sub-rays
// Sub-cone centres covering a cone of half-angle 1 (fractions of R) and the shrink factor
// (sub-cone half-angle / R).  K = 6 is the paper's ring of six at R/sqrt(3) (Fig. 5,
// Eq. 10).  K = 7, 9, 16 add a centre sub-ray and one or two rings; their radii are the
// smallest that still cover the disc (ring 5 and ring 10 radii for K = 16 were found by a
// covering search and are checked by sampling in the tests).
int subray_pattern(int K, double *rho, double *phi, double *shrink) {
    const double pi = 3.14159265358979323846;
    int k = 0;
    switch (K) {
        case 6:
            for (int j = 0; j < 6; ++j, ++k) { rho[k] = 0.57735026918962576; phi[k] = j * pi / 3.0; }
            *shrink = 0.57735026918962576;
            return 6;
        case 7:
            rho[k] = 0.0; phi[k] = 0.0; ++k;
            for (int j = 0; j < 6; ++j, ++k) { rho[k] = 0.86602540378443865; phi[k] = j * pi / 3.0; }
            *shrink = 0.5;
            return 7;
        case 9:
            rho[k] = 0.0; phi[k] = 0.0; ++k;
            for (int j = 0; j < 8; ++j, ++k) { rho[k] = 0.76536686473017954; phi[k] = j * pi / 4.0; }
            *shrink = 0.41421356237309505;
            return 9;
        case 16:
            rho[k] = 0.0; phi[k] = 0.0; ++k;
            for (int j = 0; j < 5; ++j, ++k) { rho[k] = 0.45963989297888640; phi[k] = j * 2.0 * pi / 5.0; }
            for (int j = 0; j < 10; ++j, ++k) { rho[k] = 0.82442949532182900; phi[k] = j * pi / 5.0; }
            *shrink = 0.33395494494483097;
            return 16;
        default:
            return -1;
    }
}

}  // namespace sbr
