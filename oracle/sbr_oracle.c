/*
 * sbr_oracle.c -- plain, slow, FP64 reference implementation of the SBR hot path of
 * "An Improved Equiangular Division Algorithm for SBR based Ray Tracing Channel
 * Modeling" (Zhou et al., arXiv 2208.10009).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA library is checked
 * against.  Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load it.  It shares no source, header, table or constant generator with the CUDA
 * path, and the CUDA path never calls it.
 *
 * Everything is double precision and deliberately unoptimised: brute-force intersection
 * against every triangle, brute-force occlusion, no acceleration structure.  Each
 * function cites the passage of the paper it follows.  Where the paper is silent or
 * ambiguous the reading taken is stated at the function.
 *
 * Parity status per function:
 *   lattice, trace, reception, refinement, validity, delay/AOD/AOA, image method,
 *   unfolding gradients: pinned by tests (closed forms, brute force, invariants).
 *   ora_path_eval power term: parity unpinned beyond the single-plane closed form
 *   (the paper gives no power formula; the Fresnel/free-space reading is ours).
 *   Order-1 diffraction (wedges, rough search, refinement, validity, outputs, exact
 *   diffraction point): pinned by tests; its power term is free-space loss only (the paper
 *   gives no diffraction coefficient): parity unpinned.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_MAX_ORDER 8
#define ORA_C0 299792458.0

/* ------------------------------------------------------------------------- */
/* small vector algebra                                                      */
/* ------------------------------------------------------------------------- */
typedef struct { double x, y, z; } vec3;

static vec3 mk(double x, double y, double z) { vec3 r; r.x = x; r.y = y; r.z = z; return r; }
static vec3 ld(const double *p) { return mk(p[0], p[1], p[2]); }
static void st(double *p, vec3 a) { p[0] = a.x; p[1] = a.y; p[2] = a.z; }
static vec3 add(vec3 a, vec3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
static vec3 sub(vec3 a, vec3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static vec3 scl(vec3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
static double dot(vec3 a, vec3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static vec3 cross(vec3 a, vec3 b) {
    return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static double norm(vec3 a) { return sqrt(dot(a, a)); }
static vec3 unit(vec3 a) { return scl(a, 1.0 / norm(a)); }
/* angle between two vectors, robust for tiny angles */
static double angle_between(vec3 a, vec3 b) { return atan2(norm(cross(a, b)), dot(a, b)); }

/* ------------------------------------------------------------------------- */
/* §II.B: the regular icosahedron                                            */
/* ------------------------------------------------------------------------- */
/* theta_0 = angle AOE between adjacent icosahedron vertices (§III.B, below Eq. 8). */
double ora_theta0(void) { return acos(1.0 / sqrt(5.0)); }

/* Eq. 8: cone half-angle of one ray for division level n. */
double ora_theta_launch(int n) { return ora_theta0() / (sqrt(3.0) * n); }

/* §III.B: total number of launched rays, N = 10 n^2 + 2. */
int64_t ora_num_rays(int n) { return 10 * (int64_t)n * n + 2; }

/*
 * The paper does not fix an orientation.  Reading: the canonical icosahedron whose
 * 12 vertices are the cyclic permutations of (0, +-1, +-phi), normalised, listed in the
 * fixed order below.  Faces are the vertex triples at mutual distance 2 (before
 * normalisation), in lexicographic order of the sorted triple, each oriented
 * counter-clockwise seen from outside and starting at its lowest vertex id.  Edges are
 * the vertex pairs at distance 2, lexicographic.
 */
static void ico_raw(vec3 V[12]) {
    double p = 0.5 * (1.0 + sqrt(5.0));
    double t[12][3] = {{0, 1, p},  {0, -1, p},  {0, 1, -p},  {0, -1, -p},
                       {1, p, 0},  {-1, p, 0},  {1, -p, 0},  {-1, -p, 0},
                       {p, 0, 1},  {-p, 0, 1},  {p, 0, -1},  {-p, 0, -1}};
    for (int i = 0; i < 12; ++i) V[i] = mk(t[i][0], t[i][1], t[i][2]);
}

static int ico_adjacent(vec3 a, vec3 b) { vec3 d = sub(a, b); return fabs(dot(d, d) - 4.0) < 1e-9; }

void ora_icosahedron(double *verts, int *faces, int *edges) {
    vec3 V[12];
    ico_raw(V);
    for (int i = 0; i < 12; ++i) st(verts + 3 * i, unit(V[i]));
    int nf = 0, ne = 0;
    for (int i = 0; i < 12; ++i)
        for (int j = i + 1; j < 12; ++j) {
            if (!ico_adjacent(V[i], V[j])) continue;
            edges[2 * ne] = i; edges[2 * ne + 1] = j; ++ne;
            for (int k = j + 1; k < 12; ++k) {
                if (!ico_adjacent(V[i], V[k]) || !ico_adjacent(V[j], V[k])) continue;
                vec3 c = add(add(V[i], V[j]), V[k]);
                int b = j, e = k;
                if (dot(cross(sub(V[j], V[i]), sub(V[k], V[i])), c) < 0) { b = k; e = j; }
                faces[3 * nf] = i; faces[3 * nf + 1] = b; faces[3 * nf + 2] = e; ++nf;
            }
        }
}

/* spherical linear interpolation: the point at fraction f of the great-circle arc u->v.
 * Consecutive fractions j/m give equal angles between neighbours, which is what Eq. 1
 * asks of the points on a layer edge. */
static vec3 slerp(vec3 u, vec3 v, double f) {
    double om = angle_between(u, v);
    double s = sin(om);
    return add(scl(u, sin((1.0 - f) * om) / s), scl(v, sin(f * om) / s));
}

/*
 * §II.B, Eq. 2: the three vertices of layer a+1 from layer a.  Layer a has vertices
 * W0, W1, W2 and m segments per edge.  The new vertex next to W0 is W0 moved by the
 * sum of the vectors to its two neighbours on layer a (parallelogram rule), i.e.
 * P1 + Plast - W0.  Reading: the sum leaves the sphere, so it is projected back onto
 * the unit sphere before the next layer is slerped.
 */
static void next_layer(const vec3 W[3], int m, vec3 out[3]) {
    for (int e = 0; e < 3; ++e) {
        vec3 here = W[e], fwd = W[(e + 1) % 3], bwd = W[(e + 2) % 3];
        vec3 p_next = slerp(here, fwd, 1.0 / m);
        vec3 p_prev = slerp(here, bwd, 1.0 / m);
        out[e] = unit(sub(add(p_next, p_prev), here));
    }
}

/*
 * Layer vertices of every face for division level n: L[(f * nl + a) * 3 + e], a = 0 .. nl-1,
 * nl = number of layers with m = n - 3a >= 1.
 */
static int num_layers(int n) { return (n + 2) / 3; } /* count of a >= 0 with n - 3a >= 1 */

static vec3 *build_layers(int n, vec3 ico[12], int F[60], vec3 centre[20]) {
    int nl = num_layers(n);
    vec3 *L = (vec3 *)malloc(sizeof(vec3) * 20 * nl * 3);
    for (int f = 0; f < 20; ++f) {
        vec3 W[3] = {ico[F[3 * f]], ico[F[3 * f + 1]], ico[F[3 * f + 2]]};
        centre[f] = unit(add(add(W[0], W[1]), W[2]));
        for (int a = 0; a < nl; ++a) {
            for (int e = 0; e < 3; ++e) L[(f * nl + a) * 3 + e] = W[e];
            if (a + 1 < nl) {
                vec3 nw[3];
                next_layer(W, n - 3 * a, nw);
                for (int e = 0; e < 3; ++e) W[e] = nw[e];
            }
        }
    }
    return L;
}

/*
 * Direction of ray `id` for division level n.  Canonical order (our reading; the paper
 * fixes only the per-face layering):
 *   [0, 12)                      the icosahedron vertices,
 *   [12, 12 + 30(n-1))           edge e, point j = 1..n-1 slerped from the lower to the
 *                                higher vertex id (layer 0 of both adjacent faces),
 *   then 20 faces x (n-1)(n-2)/2 interior points: layers a = 1, 2, ... (m = n - 3a
 *   segments per edge, 3m points b = 0..3m-1 walking W0->W1->W2->W0), and when the
 *   last m reaches 0 the single face-centre ray (§II.B: "one ray at the center").
 */
typedef struct {
    int n, nl;
    vec3 ico[12];
    int F[60], E[60];
    vec3 centre[20];
    vec3 *L;
} lattice;

static void lattice_init(lattice *lt, int n) {
    double v[36];
    lt->n = n;
    lt->nl = num_layers(n);
    ora_icosahedron(v, lt->F, lt->E);
    for (int i = 0; i < 12; ++i) lt->ico[i] = ld(v + 3 * i);
    lt->L = build_layers(n, lt->ico, lt->F, lt->centre);
}

static vec3 layer_point(const lattice *lt, int f, int a, int b) {
    int m = lt->n - 3 * a;
    const vec3 *W = lt->L + (f * lt->nl + a) * 3;
    int e = b / m, j = b % m;
    return slerp(W[e], W[(e + 1) % 3], (double)j / m);
}

static vec3 lattice_dir(const lattice *lt, int64_t id) {
    int n = lt->n;
    if (id < 12) return lt->ico[id];
    id -= 12;
    if (id < 30 * (int64_t)(n - 1)) {
        int e = (int)(id / (n - 1)), j = (int)(id % (n - 1)) + 1;
        return slerp(lt->ico[lt->E[2 * e]], lt->ico[lt->E[2 * e + 1]], (double)j / n);
    }
    id -= 30 * (int64_t)(n - 1);
    int64_t per_face = (int64_t)(n - 1) * (n - 2) / 2;
    int f = (int)(id / per_face);
    int64_t r = id % per_face;
    for (int a = 1;; ++a) {
        int m = n - 3 * a;
        if (m <= 0) return lt->centre[f];
        if (r < 3 * m) return layer_point(lt, f, a, (int)r);
        r -= 3 * m;
    }
}

/* All N directions (rows of 3 doubles).  Returns N. */
int64_t ora_lattice(int n, double *dirs) {
    lattice lt;
    lattice_init(&lt, n);
    int64_t N = ora_num_rays(n);
    for (int64_t i = 0; i < N; ++i) st(dirs + 3 * i, lattice_dir(&lt, i));
    free(lt.L);
    return N;
}

/* Directions of selected ray ids. */
void ora_lattice_ids(int n, const int64_t *ids, int64_t count, double *dirs) {
    lattice lt;
    lattice_init(&lt, n);
    for (int64_t i = 0; i < count; ++i) st(dirs + 3 * i, lattice_dir(&lt, ids[i]));
    free(lt.L);
}

/*
 * Face-local view of the lattice for tests: all points of face f including its shared
 * layer-0 boundary, computed from the face's own layer-0 edges (not the global edge
 * table), with their layer a and index b.  Returns the count, (n+1)(n+2)/2.
 */
int64_t ora_face_points(int n, int f, double *pts, int *layer, int *index) {
    lattice lt;
    lattice_init(&lt, n);
    int64_t c = 0;
    for (int a = 0; a < lt.nl; ++a) {
        int m = n - 3 * a;
        for (int b = 0; b < 3 * m; ++b) {
            st(pts + 3 * c, layer_point(&lt, f, a, b));
            layer[c] = a; index[c] = b; ++c;
        }
    }
    if (n - 3 * lt.nl == 0) {
        st(pts + 3 * c, lt.centre[f]);
        layer[c] = lt.nl; index[c] = 0; ++c;
    }
    free(lt.L);
    return c;
}

/* ------------------------------------------------------------------------- */
/* §II.A: equidistant division (the prior-art launcher the paper compares with) */
/* ------------------------------------------------------------------------- */
/*
 * Ray points at equal intervals on each flat face of a regular polyhedron, projected
 * onto the unit sphere (§II.A, ref. 9).  poly = 20: the icosahedron of the equiangular
 * lattice (same vertex, edge and face tables), N = 10 n^2 + 2; poly = 8: the octahedron
 * with vertices +-x, +-y, +-z in that order, N = 4 n^2 + 2.  Order: vertices; edges
 * (lower -> higher vertex id), points j = 1..n-1 at lo + (j/n)(hi - lo); per face (oriented,
 * lowest vertex A first, then B, C) the interior points A + (i/n)(B - A) + (j/n)(C - A) for
 * i = 1..n-2, j = 1..n-1-i.  Returns N, or -1 for an unknown polyhedron.
 */
static int octahedron_tables(vec3 V[6], int F[24], int E[24]) {
    vec3 t[6] = {mk(1, 0, 0), mk(-1, 0, 0), mk(0, 1, 0), mk(0, -1, 0), mk(0, 0, 1), mk(0, 0, -1)};
    int nf = 0, ne = 0;
    for (int i = 0; i < 6; ++i) V[i] = t[i];
    for (int i = 0; i < 6; ++i)
        for (int j = i + 1; j < 6; ++j) {
            if (fabs(dot(V[i], V[j])) > 1e-12) continue; /* antipodal pair */
            E[2 * ne] = i; E[2 * ne + 1] = j; ++ne;
            for (int k = j + 1; k < 6; ++k) {
                if (fabs(dot(V[i], V[k])) > 1e-12 || fabs(dot(V[j], V[k])) > 1e-12) continue;
                vec3 c = add(add(V[i], V[j]), V[k]);
                int b = j, e = k;
                if (dot(cross(sub(V[j], V[i]), sub(V[k], V[i])), c) < 0) { b = k; e = j; }
                F[3 * nf] = i; F[3 * nf + 1] = b; F[3 * nf + 2] = e; ++nf;
            }
        }
    return nf;
}

int64_t ora_equidistant(int n, int poly, double *dirs) {
    vec3 V[12];
    int F[60], E[60], nv, ne, nf;
    if (poly == 20) {
        double v[36];
        ora_icosahedron(v, F, E);
        for (int i = 0; i < 12; ++i) V[i] = ld(v + 3 * i);
        nv = 12; ne = 30; nf = 20;
    } else if (poly == 8) {
        nf = octahedron_tables(V, F, E);
        nv = 6; ne = 12;
    } else {
        return -1;
    }
    int64_t c = 0;
    for (int i = 0; i < nv; ++i) st(dirs + 3 * c++, V[i]);
    for (int e = 0; e < ne; ++e)
        for (int j = 1; j < n; ++j) {
            vec3 lo = V[E[2 * e]], hi = V[E[2 * e + 1]];
            st(dirs + 3 * c++, unit(add(lo, scl(sub(hi, lo), (double)j / n))));
        }
    for (int f = 0; f < nf; ++f) {
        vec3 A = V[F[3 * f]], B = V[F[3 * f + 1]], C = V[F[3 * f + 2]];
        for (int i = 1; i <= n - 2; ++i)
            for (int j = 1; j <= n - 1 - i; ++j)
                st(dirs + 3 * c++, unit(add(A, add(scl(sub(B, A), (double)i / n), scl(sub(C, A), (double)j / n)))));
    }
    return c;
}

/* ------------------------------------------------------------------------- */
/* §III.B: sub-ray patterns of the precise algorithm                          */
/* ------------------------------------------------------------------------- */
/*
 * The paper covers the ray cone (disc of angular radius R) by 6 smaller cones and sends
 * one sub-ray through the centre of each; the cone shrinks by 1/sqrt(3) per iteration
 * (Eq. 10).  Reading for K = 6: centres on a ring at R/sqrt(3), azimuths 60 deg * k,
 * sub-cone radius R/sqrt(3): adjacent sub-discs then meet exactly on the outer circle and
 * at the centre, so the six cover the disc.  K = 7, 9 and 16 are the same construction
 * with a centre disc and one or two rings; ring radii make each ring's worst (mid-gap)
 * point reach the next ring or the rim.  Output: rho[k] (ring radius / R), phi[k]
 * (azimuth, rad) and the shrink factor (sub-cone radius / R).  Returns K or -1.
 */
static void ring_extent(int m, double rho, double r, double *inner, double *outer) {
    double s = sin(M_PI / m), c = cos(M_PI / m);
    double q2 = r * r - rho * rho * s * s;
    if (q2 < 0) { *inner = 1e300; *outer = -1e300; return; }
    *inner = rho * c - sqrt(q2);
    *outer = rho * c + sqrt(q2);
}

/* smallest ring radius rho (for m discs of radius r) whose covered annulus reaches `target` */
static double ring_rho_reaching(int m, double r, double target) {
    double rmax = r / sin(M_PI / m), lo = 0, hi = -1, in, out;
    for (int i = 0; i <= 20000; ++i) { /* coarse scan for the first rho that reaches */
        double x = rmax * i / 20000.0;
        ring_extent(m, x, r, &in, &out);
        if (out >= target) { hi = x; lo = x - rmax / 20000.0; if (lo < 0) lo = 0; break; }
    }
    if (hi < 0) return -1;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        ring_extent(m, mid, r, &in, &out);
        if (out >= target) hi = mid; else lo = mid;
    }
    return hi;
}

/* K = 16 (centre + 5 + 10): the smallest r for which the two rings chain to the rim */
static int k16_feasible(double r, double *rho5, double *rho10) {
    double in10, out10, in5, out5;
    double r10 = ring_rho_reaching(10, r, 1.0);
    if (r10 < 0) return 0;
    ring_extent(10, r10, r, &in10, &out10);
    double r5 = ring_rho_reaching(5, r, in10);
    if (r5 < 0) return 0;
    ring_extent(5, r5, r, &in5, &out5);
    if (in5 > r) return 0;
    *rho5 = r5; *rho10 = r10;
    return 1;
}

int ora_subray_pattern(int K, double *rho, double *phi, double *shrink) {
    int k = 0;
    if (K == 6) {
        for (int j = 0; j < 6; ++j) { rho[k] = 1.0 / sqrt(3.0); phi[k] = M_PI / 3.0 * j; ++k; }
        *shrink = 1.0 / sqrt(3.0);
    } else if (K == 7) {
        rho[k] = 0; phi[k] = 0; ++k;
        for (int j = 0; j < 6; ++j) { rho[k] = sqrt(3.0) / 2.0; phi[k] = M_PI / 3.0 * j; ++k; }
        *shrink = 0.5;
    } else if (K == 9) {
        double r = sqrt(2.0) - 1.0;
        rho[k] = 0; phi[k] = 0; ++k;
        for (int j = 0; j < 8; ++j) {
            rho[k] = (1.0 + r) / (2.0 * cos(M_PI / 8.0)); phi[k] = M_PI / 4.0 * j; ++k;
        }
        *shrink = r;
    } else if (K == 16) {
        /* the search is deterministic; computed once per process */
        static double c_hi = 0, c_r5 = 0, c_r10 = 0;
        static int done = 0;
#pragma omp critical(ora_k16)
        if (!done) {
            double lo = 0.30, h = 0.36, a, b;
            for (int it = 0; it < 60; ++it) {
                double mid = 0.5 * (lo + h);
                if (k16_feasible(mid, &a, &b)) h = mid; else lo = mid;
            }
            k16_feasible(h, &c_r5, &c_r10);
            c_hi = h;
            done = 1;
        }
        double hi = c_hi, r5 = c_r5, r10 = c_r10;
        rho[k] = 0; phi[k] = 0; ++k;
        for (int j = 0; j < 5; ++j) { rho[k] = r5; phi[k] = 2.0 * M_PI / 5.0 * j; ++k; }
        for (int j = 0; j < 10; ++j) { rho[k] = r10; phi[k] = 2.0 * M_PI / 10.0 * j; ++k; }
        *shrink = hi;
    } else {
        return -1;
    }
    return k;
}

/* ------------------------------------------------------------------------- */
/* scene                                                                      */
/* ------------------------------------------------------------------------- */
typedef struct {
    int64_t nv, nt;
    int nf;
    vec3 *V;          /* vertices */
    int *T;           /* 3 vertex ids per triangle */
    int *tf;          /* face id per triangle */
    vec3 *fn;         /* unit plane normal per face */
    double *fh;       /* plane offset: n . x = h */
    double *eps;      /* relative permittivity per face (<= 0: perfect reflector) */
    unsigned char *boundary; /* 3 flags per triangle: edge (v_i, v_i+1) bounds its face */
    double scale;     /* bounding-box diagonal */
    struct wedge_s *wd;      /* wedges (diffraction), built on first use */
    int nw, wedges_built;
} scene;

typedef struct { int a, b, face; int64_t tri; int slot; } edge_rec;

static int edge_cmp(const void *x, const void *y) {
    const edge_rec *p = (const edge_rec *)x, *q = (const edge_rec *)y;
    if (p->a != q->a) return p->a < q->a ? -1 : 1;
    if (p->b != q->b) return p->b < q->b ? -1 : 1;
    if (p->face != q->face) return p->face < q->face ? -1 : 1;
    return 0;
}

/*
 * Scene upload.  A "face" is a planar polygon given as triangles sharing a face id
 * (§IV: the scene is made of faces; the face sequence of a path names faces).  The
 * plane of a face is taken from its first triangle.
 */
void *ora_scene_new(const double *verts, int64_t nv, const int32_t *tris, const int32_t *tri_face,
                    int64_t nt, const double *face_eps, int32_t nf) {
    scene *s = (scene *)calloc(1, sizeof(scene));
    s->nv = nv; s->nt = nt; s->nf = nf;
    s->V = (vec3 *)malloc(sizeof(vec3) * (nv > 0 ? nv : 1));
    s->T = (int *)malloc(sizeof(int) * 3 * (nt > 0 ? nt : 1));
    s->tf = (int *)malloc(sizeof(int) * (nt > 0 ? nt : 1));
    s->fn = (vec3 *)calloc(nf > 0 ? nf : 1, sizeof(vec3));
    s->fh = (double *)calloc(nf > 0 ? nf : 1, sizeof(double));
    s->eps = (double *)calloc(nf > 0 ? nf : 1, sizeof(double));
    s->boundary = (unsigned char *)calloc(3 * (nt > 0 ? nt : 1), 1);
    vec3 lo = mk(1e300, 1e300, 1e300), hi = mk(-1e300, -1e300, -1e300);
    for (int64_t i = 0; i < nv; ++i) {
        s->V[i] = ld(verts + 3 * i);
        lo = mk(fmin(lo.x, s->V[i].x), fmin(lo.y, s->V[i].y), fmin(lo.z, s->V[i].z));
        hi = mk(fmax(hi.x, s->V[i].x), fmax(hi.y, s->V[i].y), fmax(hi.z, s->V[i].z));
    }
    s->scale = nv > 0 ? norm(sub(hi, lo)) : 1.0;
    int *seen = (int *)calloc(nf > 0 ? nf : 1, sizeof(int));
    for (int64_t t = 0; t < nt; ++t) {
        for (int k = 0; k < 3; ++k) s->T[3 * t + k] = tris[3 * t + k];
        s->tf[t] = tri_face[t];
        int f = tri_face[t];
        if (!seen[f]) {
            vec3 a = s->V[tris[3 * t]], b = s->V[tris[3 * t + 1]], c = s->V[tris[3 * t + 2]];
            s->fn[f] = unit(cross(sub(b, a), sub(c, a)));
            s->fh[f] = dot(s->fn[f], a);
            seen[f] = 1;
        }
    }
    free(seen);
    for (int f = 0; f < nf; ++f) s->eps[f] = face_eps ? face_eps[f] : 0.0;
    /* an edge bounds its face unless another triangle of the same face shares it */
    edge_rec *er = (edge_rec *)malloc(sizeof(edge_rec) * 3 * (nt > 0 ? nt : 1));
    for (int64_t t = 0; t < nt; ++t)
        for (int k = 0; k < 3; ++k) {
            int a = s->T[3 * t + k], b = s->T[3 * t + (k + 1) % 3];
            edge_rec e; e.a = a < b ? a : b; e.b = a < b ? b : a; e.face = s->tf[t]; e.tri = t; e.slot = k;
            er[3 * t + k] = e;
        }
    qsort(er, 3 * nt, sizeof(edge_rec), edge_cmp);
    for (int64_t i = 0; i < 3 * nt;) {
        int64_t j = i;
        while (j < 3 * nt && edge_cmp(&er[i], &er[j]) == 0) ++j;
        for (int64_t k = i; k < j; ++k) s->boundary[3 * er[k].tri + er[k].slot] = (j - i == 1);
        i = j;
    }
    free(er);
    return s;
}

void ora_scene_free(void *p) {
    scene *s = (scene *)p;
    if (!s) return;
    free(s->V); free(s->T); free(s->tf); free(s->fn); free(s->fh); free(s->eps); free(s->boundary);
    free(s->wd);
    free(s);
}

void ora_scene_face_plane(void *p, int f, double *out4) {
    scene *s = (scene *)p;
    st(out4, s->fn[f]);
    out4[3] = s->fh[f];
}

double ora_scene_scale(void *p) { return ((scene *)p)->scale; }

/* Moller-Trumbore ray/triangle test in FP64; inclusive of the triangle's edges. */
static int tri_hit(const scene *s, int64_t t, vec3 o, vec3 d, double *tout) {
    vec3 a = s->V[s->T[3 * t]], b = s->V[s->T[3 * t + 1]], c = s->V[s->T[3 * t + 2]];
    vec3 e1 = sub(b, a), e2 = sub(c, a);
    vec3 p = cross(d, e2);
    double det = dot(e1, p);
    if (det == 0.0) return 0;
    double inv = 1.0 / det;
    vec3 w = sub(o, a);
    double u = dot(w, p) * inv;
    if (u < 0.0 || u > 1.0) return 0;
    vec3 q = cross(w, e1);
    double v = dot(d, q) * inv;
    if (v < 0.0 || u + v > 1.0) return 0;
    *tout = dot(e2, q) * inv;
    return 1;
}

/* smallest distance between segments o + s d (s in [0, S]) and a + u (b - a) (u in [0, 1]);
 * also returns s at the closest point */
static double seg_seg_dist(vec3 o, vec3 d, double S, vec3 a, vec3 b, double *s_at) {
    vec3 e = sub(b, a), w = sub(o, a);
    double A = dot(d, d), B = dot(d, e), C = dot(e, e), D = dot(d, w), E = dot(e, w);
    double den = A * C - B * B, s, u;
    if (den > 1e-14 * A * C) {
        s = (B * E - C * D) / den;
        if (s < 0) s = 0;
        if (s > S) s = S;
    } else {
        s = 0;
    }
    u = (B * s + E) / C;
    if (u < 0) u = 0;
    if (u > 1) u = 1;
    /* re-project s for the clamped u */
    s = (B * u - D) / A;
    if (s < 0) s = 0;
    if (s > S) s = S;
    *s_at = s;
    return norm(sub(add(o, scl(d, s)), add(a, scl(e, u))));
}

/* ------------------------------------------------------------------------- */
/* §III.A: tracing rays (Fig. 4), reception judgment and Eq. 3               */
/* ------------------------------------------------------------------------- */
/*
 * Closest hit of the ray o + t d over every triangle, skipping triangles of face `skip`
 * (a ray leaving a planar face cannot hit it again at once).  Hits need t > tmin.  Ties:
 * smaller t, then lower face id, then lower triangle id.  Returns the triangle or -1.
 */
static int64_t closest_hit(const scene *s, vec3 o, vec3 d, int skip, double tmin, double *t_out) {
    int64_t best = -1;
    double bt = INFINITY;
    for (int64_t t = 0; t < s->nt; ++t) {
        if (s->tf[t] == skip) continue;
        double th;
        if (!tri_hit(s, t, o, d, &th) || !(th > tmin)) continue;
        if (th < bt || (th == bt && s->tf[t] < s->tf[best])) { bt = th; best = t; }
    }
    *t_out = bt;
    return best;
}

/*
 * Angular edge margin of a segment: the smallest (distance to a face-boundary edge) /
 * (propagation distance there) over all triangles, for segment o + s d, s in [0, S],
 * after L metres of earlier segments.  Rays whose margin falls below 1e-6 rad can flip
 * their face sequence under rounding and are excluded from GPU parity.
 */
static double edge_margin(const scene *s, vec3 o, vec3 d, double S, double L) {
    double m = INFINITY;
    if (S > 1e7) S = 1e7;
    for (int64_t t = 0; t < s->nt; ++t)
        for (int k = 0; k < 3; ++k) {
            if (!s->boundary[3 * t + k]) continue;
            vec3 a = s->V[s->T[3 * t + k]], b = s->V[s->T[3 * t + (k + 1) % 3]];
            double sa;
            double dist = seg_seg_dist(o, d, S, a, b, &sa);
            double ang = dist / (L + sa + 1e-300);
            if (ang < m) m = ang;
        }
    return m;
}

/*
 * Trace rays from one Tx (Fig. 4): every ray goes through up to max_order specular
 * reflections; segment k (k = 0..max_order) runs from the k-th bounce point to the next
 * hit (or to infinity on a miss).  On every segment, each Rx is tested (reception
 * judgment, §III.A/§III.B): the foot of the Rx on the segment must lie on it, s in
 * [0, t_hit], and the error angle of Eq. 3, theta = arctan(d_Rx-ray / d_ray) with
 * d_ray = propagation distance to the foot, must not exceed the cone half-angle
 * `cone` (Rx inside the ray cone).  Each accepted (ray, Rx, segment) emits a record
 * (rx, ray id, order k, faces hit before the segment, theta, d_ray).  Rx are
 * transparent: the ray continues.
 *
 * Per ray, ray_nseg[i] = segments traced and ray_faces[i*(max_order+1) + k] = face hit by
 * segment k (-1 on a miss); ray_margin[i] (if want_margin) = min over segments of the
 * grazing cosine |d.n| at each hit and the angular edge margin.
 * Returns the number of records (only the first `cap` are written).
 */
int64_t ora_trace(void *sp, const double *tx3, const double *dirs, const int64_t *ray_ids, int64_t nrays,
                  const double *rx, int32_t nrx, int32_t max_order, double cone, int32_t want_margin,
                  int32_t *ray_nseg, int32_t *ray_faces, double *ray_margin,
                  int64_t cap, int32_t *rec_rx, int64_t *rec_ray, int32_t *rec_order, int32_t *rec_faces,
                  double *rec_err, double *rec_dray, int64_t *nsegments) {
    const scene *s = (const scene *)sp;
    vec3 tx = ld(tx3);
    int64_t nrec = 0, nseg_total = 0;
    double tmin = 1e-7 * s->scale;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : nseg_total)
    for (int64_t i = 0; i < nrays; ++i) {
        vec3 o = tx, d = ld(dirs + 3 * i);
        double L = 0.0, margin = INFINITY;
        int faces[ORA_MAX_ORDER + 1];
        int prev = -1, nseg = 0;
        for (int k = 0; k <= max_order; ++k) {
            double th;
            int64_t hit = closest_hit(s, o, d, prev, tmin, &th);
            ++nseg;
            int hf = hit >= 0 ? s->tf[hit] : -1;
            if (ray_faces) ray_faces[i * (max_order + 1) + k] = hf;
            /* reception judgment on this segment */
            for (int r = 0; r < nrx; ++r) {
                vec3 w = sub(ld(rx + 3 * r), o);
                double sf = dot(w, d);
                if (sf < 0.0 || sf > th) continue;
                double dperp = norm(sub(w, scl(d, sf)));
                double dray = L + sf;
                double err = atan(dperp / dray); /* Eq. 3 */
                if (!(err <= cone)) continue;
                int64_t slot;
#pragma omp atomic capture
                slot = nrec++;
                if (slot < cap) {
                    rec_rx[slot] = r;
                    rec_ray[slot] = ray_ids ? ray_ids[i] : i;
                    rec_order[slot] = k;
                    for (int q = 0; q < ORA_MAX_ORDER; ++q) rec_faces[slot * ORA_MAX_ORDER + q] = q < k ? faces[q] : -1;
                    rec_err[slot] = err;
                    rec_dray[slot] = dray;
                }
            }
            if (want_margin) {
                double em = edge_margin(s, o, d, th, L);
                if (em < margin) margin = em;
                if (hit >= 0) {
                    double g = fabs(dot(d, s->fn[hf]));
                    if (g < margin) margin = g;
                }
            }
            if (hit < 0 || k == max_order) break;
            /* specular reflection at the hit point */
            vec3 nrm = s->fn[hf];
            o = add(o, scl(d, th));
            d = sub(d, scl(nrm, 2.0 * dot(d, nrm)));
            L += th;
            faces[k] = hf;
            prev = hf;
        }
        for (int k = nseg; k <= max_order && ray_faces; ++k) ray_faces[i * (max_order + 1) + k] = -2;
        if (ray_nseg) ray_nseg[i] = nseg;
        if (ray_margin) ray_margin[i] = margin;
        nseg_total += nseg;
    }
    if (nsegments) *nsegments = nseg_total;
    return nrec;
}

/* ------------------------------------------------------------------------- */
/* §III.B: fixed-face-sequence tracing used by the precise algorithm         */
/* ------------------------------------------------------------------------- */
/*
 * Trace direction d from Tx through the planes of `faces` in order (polygon bounds
 * ignored: whether the bounce points lie inside their faces is the separate validity
 * test after refinement, §III.A).  Writes the k bounce points.  Returns the error angle
 * of Eq. 3 at Rx on the last segment (foot s may fall on either side of the last bounce,
 * d_ray = L + s), or +inf if any segment length t <= 0 or d_ray <= 0.
 */
static double trace_planes(const scene *s, vec3 tx, vec3 rx, int order, const int32_t *faces, vec3 d,
                           vec3 *pts, double *len) {
    vec3 o = tx;
    double L = 0.0;
    for (int k = 0; k < order; ++k) {
        vec3 nrm = s->fn[faces[k]];
        double den = dot(nrm, d);
        if (den == 0.0) return INFINITY;
        double t = (s->fh[faces[k]] - dot(nrm, o)) / den;
        if (!(t > 0.0)) return INFINITY;
        o = add(o, scl(d, t));
        if (pts) pts[k] = o;
        L += t;
        d = sub(d, scl(nrm, 2.0 * dot(d, nrm)));
    }
    vec3 w = sub(rx, o);
    double sf = dot(w, d);
    double dperp = norm(sub(w, scl(d, sf)));
    double dray = L + sf;
    if (len) *len = L;
    if (!(dray > 0.0)) return INFINITY;
    return atan2(dperp, dray);
}

static vec3 mirror(const scene *s, int f, vec3 x);

/*
 * AOA error of the path launched along d (§IV: AOA is the direction from Rx to the last
 * bounce point p_k): the angle at Rx between p_k - Rx and the exact direction, which
 * points at txk, Tx imaged through the k faces in order (the image method's last image
 * lies on the straight line from Rx through the exact p_k).  Zero for LOS, whose AOA
 * points at Tx for every launch direction; +inf if the fixed-face trace fails.
 */
static double aoa_error(const scene *s, vec3 tx, vec3 rx, int order, const int32_t *faces, vec3 d, vec3 txk) {
    if (order == 0) return 0.0;
    vec3 pts[ORA_MAX_ORDER];
    if (!(trace_planes(s, tx, rx, order, faces, d, pts, NULL) < INFINITY)) return INFINITY;
    return angle_between(sub(pts[order - 1], rx), sub(txk, rx));
}

/*
 * Sub-cone frame for cone centre c: u = normalize(c x e), e the world axis with the
 * smallest |c . e_i| (lowest index on ties); v = c x u.
 */
static int frame_axis(vec3 c) {
    double ax = fabs(c.x), ay = fabs(c.y), az = fabs(c.z);
    if (ay < ax && ay <= az) return 1;
    if (az < ax && az < ay) return 2;
    return 0;
}

static void frame_on_axis(vec3 c, int a, vec3 *u, vec3 *v) {
    vec3 e = mk(a == 0, a == 1, a == 2);
    *u = unit(cross(c, e));
    *v = cross(c, *u);
}

static void cone_frame(vec3 c, vec3 *u, vec3 *v) { frame_on_axis(c, frame_axis(c), u, v); }

/*
 * The iterative precise algorithm (§III.B, Fig. 5, Eq. 10).  The path's initial cone
 * is centred on its rough launch direction c0 with half-angle R0.  Each iteration sends
 * K sub-rays through the sub-cone centres (pattern above), traces each through the
 * path's fixed faces, evaluates Eq. 3 for each, keeps the sub-ray with the smallest
 * error (lowest k on ties; the parent ray does not compete) as the new centre and
 * shrinks the cone by the pattern's factor.  It stops after `iters` iterations or as
 * soon as the path meets the accuracy requirement (target <= 0: never early): the error
 * angle, which is the AOD error, and the AOA error (aoa_error) both <= target.  If every
 * sub-ray is
 * invalid the iteration stops.  Returns iterations done; writes the final direction, its
 * error, and per-iteration choice (argmin k) and error history (err_hist[0] = error of
 * c0).
 *
 * It also stops once the path can no longer pass the validity test's convergence
 * condition (error <= 2 R_final + 1e-7, see ora_path_eval) -- a stalled path, whose exact
 * direction has left the cone.  The error is the angle to the exact direction (Eq. 3 in
 * unfolded space); every later centre lies within R (1 + s + s^2 + ...) = R / (1 - s) of
 * the current one (sub-ray offsets are at most the cone half-angle), so later errors
 * exceed err - R / (1 - s), while after at least one more iteration 2 R_final + 1e-7 <=
 * 2 R s + 1e-7.  Once err > R (1 / (1 - s) + 2 s) + 1e-6 the path is rejected whatever
 * follows, and since 1 / (1 - s) + 2 s >= 2 for every pattern it is rejected now as well.
 * Valid paths never meet this condition, so their results are unchanged.
 */
static int refine_core(void *sp, const double *tx3, const double *rx3, int order, const int32_t *faces,
                       const double *c0, double R0, int K, int iters, double target, const int32_t *forced,
                       int stall_on, double *out_dir, double *out_err, int32_t *choice, double *err_hist,
                       double *sub_err, int32_t *axis_log, double *centre_log) {
    const scene *s = (const scene *)sp;
    double rho[16], phi[16], shrink;
    if (ora_subray_pattern(K, rho, phi, &shrink) != K) return -1;
    vec3 tx = ld(tx3), rx = ld(rx3), c = unit(ld(c0));
    vec3 txk = tx;
    for (int j = 0; j < order; ++j) txk = mirror(s, faces[j], txk);
    double R = R0;
    double err = trace_planes(s, tx, rx, order, faces, c, NULL, NULL);
    double aoa = target > 0 ? aoa_error(s, tx, rx, order, faces, c, txk) : INFINITY;
    if (err_hist) err_hist[0] = err;
    int it = 0;
    const double stall = 1.0 / (1.0 - shrink) + 2.0 * shrink;
    while (it < iters && !(target > 0 && err <= target && aoa <= target) &&
           !(stall_on && err > R * stall + 1e-6)) {
        vec3 u, v, best_d = c;
        double best = INFINITY;
        int bk = -1;
        const int fz = forced ? forced[it] : -1;
        if (axis_log) axis_log[it] = frame_axis(c);
        if (centre_log) st(centre_log + 3 * (size_t)it, c);
        frame_on_axis(c, fz >= 0 ? (fz >> 4) & 3 : frame_axis(c), &u, &v);
        for (int k = 0; k < K; ++k) {
            double a = rho[k] * R;
            vec3 dk = add(scl(c, cos(a)), scl(add(scl(u, cos(phi[k])), scl(v, sin(phi[k]))), sin(a)));
            double e = trace_planes(s, tx, rx, order, faces, dk, NULL, NULL);
            if (sub_err) sub_err[(size_t)it * K + k] = e;
            if (fz >= 0) {
                if (k == (fz & 15)) { best = e; bk = k; best_d = dk; }
            } else if (e < best) {
                best = e; bk = k; best_d = dk;
            }
        }
        if (bk < 0 || !(best < INFINITY)) break;
        c = best_d;
        err = best;
        if (target > 0) aoa = aoa_error(s, tx, rx, order, faces, c, txk);
        R *= shrink;
        if (choice) choice[it] = bk;
        ++it;
        if (err_hist) err_hist[it] = err;
    }
    st(out_dir, c);
    *out_err = err;
    return it;
}

int ora_refine(void *sp, const double *tx3, const double *rx3, int order, const int32_t *faces,
               const double *c0, double R0, int K, int iters, double target,
               double *out_dir, double *out_err, int32_t *choice, double *err_hist) {
    return refine_core(sp, tx3, rx3, order, faces, c0, R0, K, iters, target, NULL, 1, out_dir, out_err, choice,
                       err_hist, NULL, NULL, NULL);
}

/*
 * The same iteration with test hooks that leave its arithmetic unchanged: sub_err (iters x
 * K, or NULL) receives every sub-ray's error angle per iteration; axis_log (iters, or
 * NULL) the frame axis this implementation's own rule picks at each centre; centre_log
 * (iters x 3, or NULL) each iteration's cone centre; and forced (or
 * NULL) names, per iteration, the sub-ray to keep instead of the argmin (bits 0-3) and the
 * frame axis to use instead of the rule's (bits 4-5) -- a negative entry keeps the argmin
 * and the rule.  Replaying another implementation's logged choices this way gives the
 * exact FP64 state that implementation approximates, so each of its choices can be
 * compared with the best sub-ray of the same cone.  stall_on = 0 disables the stalled-
 * path exit (everything else as ora_refine).
 */
int ora_refine_ex(void *sp, const double *tx3, const double *rx3, int order, const int32_t *faces,
                  const double *c0, double R0, int K, int iters, double target, const int32_t *forced,
                  int stall_on, double *out_dir, double *out_err, int32_t *choice, double *err_hist,
                  double *sub_err, int32_t *axis_log, double *centre_log) {
    return refine_core(sp, tx3, rx3, order, faces, c0, R0, K, iters, target, forced, stall_on, out_dir, out_err,
                       choice, err_hist, sub_err, axis_log, centre_log);
}

/*
 * The two errors the early stop of the precise algorithm compares with its target, for a
 * path launched along dir: out[0] = the Eq. 3 error angle (the AOD error) and out[1] = the
 * AOA error (aoa_error).  +inf where the fixed-face trace fails.
 */
void ora_path_errors(void *sp, const double *tx3, const double *rx3, int order, const int32_t *faces,
                     const double *dir, double *out) {
    const scene *s = (const scene *)sp;
    vec3 tx = ld(tx3), rx = ld(rx3), d = unit(ld(dir)), txk = tx;
    for (int j = 0; j < order; ++j) txk = mirror(s, faces[j], txk);
    out[0] = trace_planes(s, tx, rx, order, faces, d, NULL, NULL);
    out[1] = aoa_error(s, tx, rx, order, faces, d, txk);
}

/* point-in-face: p lies inside (or on the boundary of) some triangle of face f */
static int in_face(const scene *s, int f, vec3 p) {
    vec3 n = s->fn[f];
    for (int64_t t = 0; t < s->nt; ++t) {
        if (s->tf[t] != f) continue;
        vec3 a = s->V[s->T[3 * t]], b = s->V[s->T[3 * t + 1]], c = s->V[s->T[3 * t + 2]];
        double ea = dot(cross(sub(b, a), sub(p, a)), n);
        double eb = dot(cross(sub(c, b), sub(p, b)), n);
        double ec = dot(cross(sub(a, c), sub(p, c)), n);
        if ((ea >= 0 && eb >= 0 && ec >= 0) || (ea <= 0 && eb <= 0 && ec <= 0)) return 1;
    }
    return 0;
}

/* segment p -> q blocked by any triangle not of faces fa, fb, strictly inside (eps, 1-eps) */
static int occluded(const scene *s, vec3 p, vec3 q, int fa, int fb) {
    vec3 d = sub(q, p);
    for (int64_t t = 0; t < s->nt; ++t) {
        if (s->tf[t] == fa || s->tf[t] == fb) continue;
        double th;
        if (tri_hit(s, t, p, d, &th) && th > 1e-6 && th < 1.0 - 1e-6) return 1;
    }
    return 0;
}

static void az_el(vec3 v, double *out) {
    out[0] = atan2(v.y, v.x);
    out[1] = atan2(v.z, sqrt(v.x * v.x + v.y * v.y));
}

/* |Gamma_perp| of a Fresnel reflection at incidence cosine ci on relative permittivity eps */
static double fresnel_perp(double ci, double eps) {
    if (eps <= 0) return 1.0;
    double s2 = 1.0 - ci * ci;
    double r = sqrt(eps - s2);
    return fabs((ci - r) / (ci + r));
}

/*
 * Validity test and channel outputs of one path for launch direction `dir` (§III.A
 * second path test; §IV outputs).  The bounce points p_1..p_k are recomputed through the
 * fixed planes; the path is valid iff every p_i lies in its face, the foot of Rx on the
 * last leg lies ahead of the last bounce point (the reception judgment's condition that
 * Rx is received on that segment, §III.A/B), no segment Tx->p_1->...->p_k->Rx is
 * blocked (endpoint faces excluded), and -- when err_bound > 0 -- the error angle of dir is
 * at most err_bound.  The caller passes twice the Eq. 10 bound of the refinement that
 * produced dir (plus the FP32 evaluation floor): a path whose exact direction lies in its
 * cone always meets the bound, while a redundant path received through the cone's width
 * for a face sequence with no specular solution stalls far above it (§III.A: such paths
 * are removed after the precise algorithm).  Outputs: delay = polyline
 * length to the exact Rx / c0; AOD = (azimuth, elevation) of dir; AOA = (azimuth,
 * elevation) of p_k - Rx (Tx - Rx for LOS); power (dBm) = ptx + 20 log10(lambda / (4 pi
 * length)) + sum 20 log10 |Gamma_perp| (parity unpinned beyond one plane); err = Eq. 3
 * error angle of dir.  Returns 0, or -1 if the fixed-plane trace fails.
 */
int ora_path_eval(void *sp, const double *tx3, const double *rx3, int order, const int32_t *faces,
                  const double *dir, double freq, double ptx_dbm, double err_bound, double *pts_out,
                  int32_t *valid, double *delay, double *aod, double *aoa, double *power, double *err) {
    const scene *s = (const scene *)sp;
    vec3 tx = ld(tx3), rx = ld(rx3), d = unit(ld(dir));
    vec3 P[ORA_MAX_ORDER];
    double L;
    double e = trace_planes(s, tx, rx, order, faces, d, P, &L);
    *err = e;
    *valid = 0;
    if (!isfinite(e)) return -1;
    int ok = 1;
    for (int k = 0; k < order; ++k) {
        if (pts_out) st(pts_out + 3 * k, P[k]);
        if (!in_face(s, faces[k], P[k])) ok = 0;
    }
    vec3 prev = tx;
    int fprev = -1;
    double len = 0.0, gain_db = 0.0;
    vec3 dd = d;
    for (int k = 0; k <= order && ok; ++k) {
        vec3 nxt = k < order ? P[k] : rx;
        int fn = k < order ? faces[k] : -1;
        if (occluded(s, prev, nxt, fprev, fn)) ok = 0;
        prev = nxt;
        fprev = fn;
    }
    prev = tx;
    for (int k = 0; k <= order; ++k) {
        vec3 nxt = k < order ? P[k] : rx;
        len += norm(sub(nxt, prev));
        if (k < order) {
            vec3 nrm = s->fn[faces[k]];
            double ci = fabs(dot(dd, nrm));
            gain_db += 20.0 * log10(fresnel_perp(ci, s->eps[faces[k]]));
            dd = sub(dd, scl(nrm, 2.0 * dot(dd, nrm)));
        }
        prev = nxt;
    }
    /* dd is now the direction of the last leg */
    if (dot(sub(rx, order > 0 ? P[order - 1] : tx), dd) <= 0.0) ok = 0;
    if (err_bound > 0.0 && !(e <= err_bound)) ok = 0;
    *valid = ok;
    *delay = len / ORA_C0;
    az_el(d, aod);
    az_el(sub(order > 0 ? P[order - 1] : tx, rx), aoa);
    double lam = ORA_C0 / freq;
    *power = ptx_dbm + 20.0 * log10(lam / (4.0 * M_PI * len)) + gain_db;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* image method (exact backward tracing; the comparison method of §IV)       */
/* ------------------------------------------------------------------------- */
static vec3 mirror(const scene *s, int f, vec3 x) {
    return sub(x, scl(s->fn[f], 2.0 * (dot(s->fn[f], x) - s->fh[f])));
}

/*
 * Image-method path for one face sequence: image Tx through the planes in order, then
 * back-trace from Rx: p_k is where the line image_k -> Rx crosses plane f_k, p_{k-1} where
 * image_{k-1} -> p_k crosses f_{k-1}, and so on; every crossing parameter must lie in
 * (0, 1).  Valid iff every p_i is inside its face and no segment is blocked.  Writes the
 * exact AOD direction (unit), delay |Rx - image_k| / c0, AOD/AOA angles and power.
 * Returns 1 if valid, 0 if not (geometry or validity), outputs written either way when
 * the back-trace succeeds; -1 if the back-trace itself fails.
 */
int ora_image_path(void *sp, const double *tx3, const double *rx3, int order, const int32_t *faces,
                   double freq, double ptx_dbm, double *pts_out, double *aod_dir, double *delay,
                   double *aod, double *aoa, double *power) {
    const scene *s = (const scene *)sp;
    vec3 tx = ld(tx3), rx = ld(rx3);
    vec3 img[ORA_MAX_ORDER + 1], P[ORA_MAX_ORDER];
    img[0] = tx;
    for (int k = 0; k < order; ++k) {
        if (k > 0 && faces[k] == faces[k - 1]) return -1;
        img[k + 1] = mirror(s, faces[k], img[k]);
    }
    vec3 q = rx;
    for (int k = order - 1; k >= 0; --k) {
        vec3 a = img[k + 1], dq = sub(q, a);
        vec3 nrm = s->fn[faces[k]];
        double den = dot(nrm, dq);
        if (den == 0.0) return -1;
        double u = (s->fh[faces[k]] - dot(nrm, a)) / den;
        if (!(u > 0.0 && u < 1.0)) return -1;
        P[k] = add(a, scl(dq, u));
        q = P[k];
    }
    vec3 first = order > 0 ? P[0] : rx;
    vec3 dir = unit(sub(first, tx));
    st(aod_dir, dir);
    *delay = norm(sub(rx, img[order])) / ORA_C0;
    az_el(dir, aod);
    az_el(sub(order > 0 ? P[order - 1] : tx, rx), aoa);
    int ok = 1;
    for (int k = 0; k < order; ++k) {
        if (pts_out) st(pts_out + 3 * k, P[k]);
        if (!in_face(s, faces[k], P[k])) ok = 0;
    }
    vec3 prev = tx, dd = dir;
    int fprev = -1;
    double gain_db = 0.0;
    for (int k = 0; k <= order; ++k) {
        vec3 nxt = k < order ? P[k] : rx;
        int fn = k < order ? faces[k] : -1;
        if (ok && occluded(s, prev, nxt, fprev, fn)) ok = 0;
        if (k < order) {
            vec3 nrm = s->fn[faces[k]];
            gain_db += 20.0 * log10(fresnel_perp(fabs(dot(dd, nrm)), s->eps[faces[k]]));
            dd = sub(dd, scl(nrm, 2.0 * dot(dd, nrm)));
        }
        prev = nxt;
        fprev = fn;
    }
    double lam = ORA_C0 / freq;
    *power = ptx_dbm + 20.0 * log10(lam / (4.0 * M_PI * norm(sub(rx, img[order])))) + gain_db;
    return ok;
}

/*
 * Exhaustive image method for small scenes: every face sequence of length 0..max_order
 * with no face repeated twice in a row.  Writes the valid ones (order, faces[8], exact AOD
 * direction, delay).  Returns the number of valid paths (only `cap` written).
 */
int64_t ora_image_enumerate(void *sp, const double *tx3, const double *rx3, int max_order, int64_t cap,
                            int32_t *out_order, int32_t *out_faces, double *out_dir, double *out_delay) {
    const scene *s = (const scene *)sp;
    int64_t count = 0;
    int32_t seq[ORA_MAX_ORDER];
    for (int k = 0; k <= max_order; ++k) {
        /* odometer over sequences of length k */
        for (int q = 0; q < k; ++q) seq[q] = 0;
        for (;;) {
            int okseq = 1;
            for (int q = 1; q < k; ++q) if (seq[q] == seq[q - 1]) okseq = 0;
            if (okseq) {
                double pts[3 * ORA_MAX_ORDER], dir[3], delay, aod[2], aoa[2], pw;
                int r = ora_image_path(sp, tx3, rx3, k, seq, 2.4e9, 0.0, pts, dir, &delay, aod, aoa, &pw);
                if (r == 1) {
                    if (count < cap) {
                        out_order[count] = k;
                        for (int q = 0; q < ORA_MAX_ORDER; ++q) out_faces[count * ORA_MAX_ORDER + q] = q < k ? seq[q] : -1;
                        for (int q = 0; q < 3; ++q) out_dir[3 * count + q] = dir[q];
                        out_delay[count] = delay;
                    }
                    ++count;
                }
            }
            int q = k - 1;
            while (q >= 0 && ++seq[q] == s->nf) seq[q--] = 0;
            if (q < 0) break;
        }
    }
    return count;
}

/* ------------------------------------------------------------------------- */
/* fixed-face-sequence unfolding and its closed-form gradients               */
/* ------------------------------------------------------------------------- */
/*
 * For a path with faces f_1..f_k, mirroring through the planes is x -> H x + b with
 * H = I - 2 n n^T.  Rx' = M_1(M_2(...M_k(Rx))) is Rx unfolded into Tx's space
 * (Rx' = A Rx + a0, A = H_1 ... H_k) and Tx^(k) = M_k(...M_1(Tx)) is the last Tx image
 * (Tx^(k) = B Tx + b0, B = H_k ... H_1 = A^T).
 *
 * Values (8): miss[3] = real-space vector from the foot of Rx on the last segment of the
 * ray launched at (az, el) to Rx, = A^T (w - (w.d) d) with w = Rx' - Tx; delay =
 * |w| / c0; AOD = az/el of w; AOA = az/el of Tx^(k) - Rx.
 * Jacobian J[8][8], rows = those 8 outputs, columns = (az, el, Tx xyz, Rx xyz).
 */
static void mat_mirror_apply(const scene *s, int f, const double M[9], double out[9]) {
    /* out = H_f M */
    vec3 n = s->fn[f];
    double nn[3] = {n.x, n.y, n.z};
    for (int c = 0; c < 3; ++c) {
        double nd = nn[0] * M[c] + nn[1] * M[3 + c] + nn[2] * M[6 + c];
        for (int r = 0; r < 3; ++r) out[3 * r + c] = M[3 * r + c] - 2.0 * nn[r] * nd;
    }
}

static void az_el_grad(vec3 w, double gaz[3], double gel[3]) {
    double rho2 = w.x * w.x + w.y * w.y, rho = sqrt(rho2), r2 = rho2 + w.z * w.z;
    gaz[0] = -w.y / rho2; gaz[1] = w.x / rho2; gaz[2] = 0.0;
    gel[0] = -w.x * w.z / (r2 * rho); gel[1] = -w.y * w.z / (r2 * rho); gel[2] = rho / r2;
}

void ora_unfold(void *sp, int order, const int32_t *faces, const double *tx3, const double *rx3, double az,
                double el, double *val, double *J) {
    const scene *s = (const scene *)sp;
    vec3 tx = ld(tx3), rx = ld(rx3);
    /* Rx' by mirroring in reverse order; A = H_1 ... H_k built the same way */
    vec3 rxp = rx, txk = tx;
    double A[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, tmp[9];
    for (int k = order - 1; k >= 0; --k) {
        rxp = mirror(s, faces[k], rxp);
        mat_mirror_apply(s, faces[k], A, tmp);
        memcpy(A, tmp, sizeof(A));
    }
    for (int k = 0; k < order; ++k) txk = mirror(s, faces[k], txk);
    vec3 d = mk(cos(el) * cos(az), cos(el) * sin(az), sin(el));
    vec3 d_az = mk(-cos(el) * sin(az), cos(el) * cos(az), 0.0);
    vec3 d_el = mk(-sin(el) * cos(az), -sin(el) * sin(az), cos(el));
    vec3 w = sub(rxp, tx);
    double wd = dot(w, d);
    vec3 m_unf = sub(w, scl(d, wd));
    /* A^T v */
#define AT(v) mk(A[0] * (v).x + A[3] * (v).y + A[6] * (v).z, A[1] * (v).x + A[4] * (v).y + A[7] * (v).z, \
                 A[2] * (v).x + A[5] * (v).y + A[8] * (v).z)
    vec3 miss = AT(m_unf);
    double dist = norm(w);
    double aod[2], aoa[2];
    az_el(w, aod);
    vec3 va = sub(txk, rx);
    az_el(va, aoa);
    if (val) {
        val[0] = miss.x; val[1] = miss.y; val[2] = miss.z;
        val[3] = dist / ORA_C0;
        val[4] = aod[0]; val[5] = aod[1]; val[6] = aoa[0]; val[7] = aoa[1];
    }
    if (!J) return;
    memset(J, 0, sizeof(double) * 64);
    /* d miss / d az, d el */
    vec3 dm_az = AT(scl(add(scl(d, dot(w, d_az)), scl(d_az, wd)), -1.0));
    vec3 dm_el = AT(scl(add(scl(d, dot(w, d_el)), scl(d_el, wd)), -1.0));
    J[0 * 8 + 0] = dm_az.x; J[1 * 8 + 0] = dm_az.y; J[2 * 8 + 0] = dm_az.z;
    J[0 * 8 + 1] = dm_el.x; J[1 * 8 + 1] = dm_el.y; J[2 * 8 + 1] = dm_el.z;
    /* d miss / d w = A^T (I - d d^T); w = A Rx + a0 - Tx */
    double P[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double dr = r == 0 ? d.x : r == 1 ? d.y : d.z, dc = c == 0 ? d.x : c == 1 ? d.y : d.z;
            P[3 * r + c] = (r == c) - dr * dc;
        }
    double ATP[9], ATPA[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double acc = 0;
            for (int q = 0; q < 3; ++q) acc += A[3 * q + r] * P[3 * q + c];
            ATP[3 * r + c] = acc;
        }
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double acc = 0;
            for (int q = 0; q < 3; ++q) acc += ATP[3 * r + q] * A[3 * q + c];
            ATPA[3 * r + c] = acc;
        }
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            J[r * 8 + 2 + c] = -ATP[3 * r + c];
            J[r * 8 + 5 + c] = ATPA[3 * r + c];
        }
    /* delay: d|w|/dw = w/|w| */
    vec3 uw = scl(w, 1.0 / dist);
    vec3 uA = AT(uw);
    double g3t[3] = {-uw.x / ORA_C0, -uw.y / ORA_C0, -uw.z / ORA_C0};
    double g3r[3] = {uA.x / ORA_C0, uA.y / ORA_C0, uA.z / ORA_C0};
    for (int c = 0; c < 3; ++c) { J[3 * 8 + 2 + c] = g3t[c]; J[3 * 8 + 5 + c] = g3r[c]; }
    /* AOD angles of w */
    double gaz[3], gel[3];
    az_el_grad(w, gaz, gel);
    vec3 gazA = AT(mk(gaz[0], gaz[1], gaz[2])), gelA = AT(mk(gel[0], gel[1], gel[2]));
    double gazAr[3] = {gazA.x, gazA.y, gazA.z}, gelAr[3] = {gelA.x, gelA.y, gelA.z};
    for (int c = 0; c < 3; ++c) {
        J[4 * 8 + 2 + c] = -gaz[c]; J[4 * 8 + 5 + c] = gazAr[c];
        J[5 * 8 + 2 + c] = -gel[c]; J[5 * 8 + 5 + c] = gelAr[c];
    }
    /* AOA angles of v = Tx^(k) - Rx = B Tx + b0 - Rx, B = A^T, so dv/dTx = A^T -> grad_Tx = A g */
    az_el_grad(va, gaz, gel);
    for (int c = 0; c < 3; ++c) {
        double a_az = A[3 * c] * gaz[0] + A[3 * c + 1] * gaz[1] + A[3 * c + 2] * gaz[2];
        double a_el = A[3 * c] * gel[0] + A[3 * c + 1] * gel[1] + A[3 * c + 2] * gel[2];
        J[6 * 8 + 2 + c] = a_az; J[6 * 8 + 5 + c] = -gaz[c];
        J[7 * 8 + 2 + c] = a_el; J[7 * 8 + 5 + c] = -gel[c];
    }
#undef AT
}

/* ora_unfold's values (no Jacobian) for P paths at once: order[p], faces[8 p ..], tx/rx
 * [3 p ..] -> vals[8 p ..].  The exact image-method delay, AOD and AOA of each face
 * sequence (the miss terms use az = el = 0). */
void ora_unfold_many(void *sp, int64_t P, const int32_t *order, const int32_t *faces, const double *tx,
                     const double *rx, double *vals) {
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < P; ++p)
        ora_unfold(sp, order[p], faces + 8 * p, tx + 3 * p, rx + 3 * p, 0.0, 0.0, vals + 8 * p, NULL);
}

int ora_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* order-1 diffraction: §III.A (Fig. 4, both path tests name faces and       */
/* wedges), §III.B last paragraph, §IV (Figs. 7c-d and 8b)                   */
/* ------------------------------------------------------------------------- */
/*
 * Wedges.  The paper diffracts rays at the wedges of its scenes without defining one; the
 * reading taken here: a wedge is a side shared by two faces -- the same segment, with
 * identical endpoint coordinates, on the boundary of both -- whose half-planes meet at an
 * interior angle between 1 and 170 degrees.  A face's sides are its boundary triangle
 * edges with collinear neighbours (sharing a vertex) merged.  The solid fills the smaller
 * of the two sectors the half-planes bound; the larger one (> pi) is the exterior, where
 * both ends of a diffracted path must lie.  Wedge ids follow the order of the face pairs
 * (f1 < f2).  w1, w2 are the unit vectors perpendicular to the edge pointing into face f1
 * and f2 (towards the mean of the face's triangle vertices).
 */
typedef struct wedge_s {
    vec3 a, b, e, w1, w2;
    int f1, f2;
} wedge_t;

typedef struct { vec3 pa, pb; int ia, ib, face, alive; } side_t;
typedef struct { double k[6]; int face; vec3 a, b; } side_key;

static int side_key_cmp(const void *x, const void *y) {
    const side_key *p = (const side_key *)x, *q = (const side_key *)y;
    for (int i = 0; i < 6; ++i)
        if (p->k[i] != q->k[i]) return p->k[i] < q->k[i] ? -1 : 1;
    return p->face < q->face ? -1 : (p->face > q->face ? 1 : 0);
}

static int lex_less(vec3 a, vec3 b) {
    if (a.x != b.x) return a.x < b.x;
    if (a.y != b.y) return a.y < b.y;
    return a.z < b.z;
}

static int wedge_cmp(const void *x, const void *y) {
    const wedge_t *p = (const wedge_t *)x, *q = (const wedge_t *)y;
    if (p->f1 != q->f1) return p->f1 < q->f1 ? -1 : 1;
    return p->f2 < q->f2 ? -1 : (p->f2 > q->f2 ? 1 : 0);
}

static vec3 perp_to(vec3 v, vec3 e) { return sub(v, scl(e, dot(v, e))); }

static void wedges_build(scene *s) {
    if (s->wedges_built) return;
    s->wedges_built = 1;
    /* boundary edges grouped by face */
    int64_t nb = 0;
    for (int64_t t = 0; t < s->nt; ++t)
        for (int k = 0; k < 3; ++k) nb += s->boundary[3 * t + k];
    side_t *sd = (side_t *)malloc(sizeof(side_t) * (nb > 0 ? nb : 1));
    int64_t *start = (int64_t *)calloc((size_t)s->nf + 1, sizeof(int64_t));
    for (int64_t t = 0; t < s->nt; ++t)
        for (int k = 0; k < 3; ++k)
            if (s->boundary[3 * t + k]) ++start[s->tf[t] + 1];
    for (int f = 0; f < s->nf; ++f) start[f + 1] += start[f];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * ((size_t)s->nf + 1));
    memcpy(fill, start, sizeof(int64_t) * ((size_t)s->nf + 1));
    vec3 *cen = (vec3 *)calloc((size_t)s->nf + 1, sizeof(vec3));
    double *cnt = (double *)calloc((size_t)s->nf + 1, sizeof(double));
    for (int64_t t = 0; t < s->nt; ++t) {
        int f = s->tf[t];
        for (int k = 0; k < 3; ++k) {
            cen[f] = add(cen[f], s->V[s->T[3 * t + k]]);
            cnt[f] += 1.0;
            if (!s->boundary[3 * t + k]) continue;
            side_t e;
            e.ia = s->T[3 * t + k];
            e.ib = s->T[3 * t + (k + 1) % 3];
            e.pa = s->V[e.ia];
            e.pb = s->V[e.ib];
            e.face = f;
            e.alive = 1;
            sd[fill[f]++] = e;
        }
    }
    for (int f = 0; f < s->nf; ++f)
        if (cnt[f] > 0) cen[f] = scl(cen[f], 1.0 / cnt[f]);
    /* merge collinear boundary edges of each face that share a vertex */
    for (int f = 0; f < s->nf; ++f) {
        int merged = 1;
        while (merged) {
            merged = 0;
            for (int64_t i = start[f]; i < start[f + 1]; ++i) {
                if (!sd[i].alive) continue;
                for (int64_t j = start[f]; j < start[f + 1]; ++j) {
                    if (j == i || !sd[j].alive) continue;
                    side_t *p = &sd[i], *q = &sd[j];
                    int shared, pfar, qfar;
                    vec3 pf, qf;
                    if (p->ib == q->ia) { shared = 1; pf = p->pa; pfar = p->ia; qf = q->pb; qfar = q->ib; }
                    else if (p->ib == q->ib) { shared = 1; pf = p->pa; pfar = p->ia; qf = q->pa; qfar = q->ia; }
                    else if (p->ia == q->ia) { shared = 1; pf = p->pb; pfar = p->ib; qf = q->pb; qfar = q->ib; }
                    else if (p->ia == q->ib) { shared = 1; pf = p->pb; pfar = p->ib; qf = q->pa; qfar = q->ia; }
                    else shared = 0;
                    if (!shared) continue;
                    vec3 d1 = sub(p->pb, p->pa), d2 = sub(q->pb, q->pa);
                    if (norm(cross(d1, d2)) > 1e-6 * norm(d1) * norm(d2)) continue;
                    p->pa = pf; p->ia = pfar;
                    p->pb = qf; p->ib = qfar;
                    q->alive = 0;
                    merged = 1;
                }
            }
        }
    }
    /* sides shared by exactly two faces */
    side_key *keys = (side_key *)malloc(sizeof(side_key) * (nb > 0 ? nb : 1));
    int64_t nk = 0;
    for (int64_t i = 0; i < nb; ++i) {
        if (!sd[i].alive) continue;
        vec3 lo = sd[i].pa, hi = sd[i].pb;
        if (lex_less(hi, lo)) { vec3 tmp = lo; lo = hi; hi = tmp; }
        side_key k;
        k.k[0] = lo.x; k.k[1] = lo.y; k.k[2] = lo.z; k.k[3] = hi.x; k.k[4] = hi.y; k.k[5] = hi.z;
        k.face = sd[i].face;
        k.a = lo;
        k.b = hi;
        keys[nk++] = k;
    }
    qsort(keys, (size_t)nk, sizeof(side_key), side_key_cmp);
    wedge_t *W = (wedge_t *)malloc(sizeof(wedge_t) * (nk > 0 ? nk : 1));
    int nw = 0;
    for (int64_t i = 0; i < nk;) {
        int64_t j = i;
        while (j < nk && memcmp(keys[j].k, keys[i].k, sizeof(keys[i].k)) == 0) ++j;
        if (j - i == 2 && keys[i].face != keys[i + 1].face) {
            wedge_t w;
            w.a = keys[i].a;
            w.b = keys[i].b;
            w.e = unit(sub(w.b, w.a));
            w.f1 = keys[i].face;
            w.f2 = keys[i + 1].face;
            w.w1 = unit(perp_to(sub(cen[w.f1], w.a), w.e));
            w.w2 = unit(perp_to(sub(cen[w.f2], w.a), w.e));
            double phi = angle_between(w.w1, w.w2) * 180.0 / M_PI;
            if (phi >= 1.0 && phi <= 170.0) W[nw++] = w;
        }
        i = j;
    }
    qsort(W, (size_t)nw, sizeof(wedge_t), wedge_cmp);
    s->wd = W;
    s->nw = nw;
    free(keys); free(sd); free(start); free(fill); free(cen); free(cnt);
}

/* Number of wedges; writes (a, b) as 6 doubles and (f1, f2) per wedge when non-null. */
int32_t ora_wedges(void *sp, double *ab, int32_t *faces) {
    scene *s = (scene *)sp;
    wedges_build(s);
    for (int i = 0; i < s->nw; ++i) {
        if (ab) { st(ab + 6 * i, s->wd[i].a); st(ab + 6 * i + 3, s->wd[i].b); }
        if (faces) { faces[2 * i] = s->wd[i].f1; faces[2 * i + 1] = s->wd[i].f2; }
    }
    return s->nw;
}

/* p lies in the wedge's exterior: not strictly inside the interior sector of w1, w2 */
static int wedge_exterior(const wedge_t *w, vec3 p) {
    vec3 q = perp_to(sub(p, w->a), w->e);
    vec3 nrm = cross(w->w1, w->w2);
    int inside = dot(cross(w->w1, q), nrm) > 0.0 && dot(cross(q, w->w2), nrm) > 0.0;
    return !inside;
}

int32_t ora_wedge_exterior(void *sp, int32_t wi, const double *p3) {
    scene *s = (scene *)sp;
    wedges_build(s);
    return wedge_exterior(&s->wd[wi], ld(p3));
}

/*
 * Unfolding across the edge line (the diffraction analogue of mirroring through a face
 * plane): Rx rotated about the edge line into the half-plane through the edge that is
 * opposite Tx.  Rotation about the edge keeps the angle to the edge, so a ray from Tx
 * that crosses the edge line and continues straight towards the image Rx* is, once
 * folded back, a ray on the Keller cone of diffraction (§III.B: the sub-rays diffract
 * along the recorded direction; the azimuth around the cone that reaches the receiver
 * is the limit of the rays sent to both sides of it).  Eq. 3's error angle of a launch
 * direction d is then angle(d, Rx* - Tx), and the exact diffraction point is where the
 * segment Tx -> Rx* crosses the edge line.  Returns 0 if Tx lies on the edge line.
 */
static int wedge_unfold_rx(const wedge_t *w, vec3 tx, vec3 rx, vec3 *out) {
    vec3 qt = sub(tx, w->a), qr = sub(rx, w->a);
    vec3 pt = perp_to(qt, w->e), pr = perp_to(qr, w->e);
    double rt = norm(pt), rr = norm(pr);
    if (!(rt > 0.0)) return 0;
    *out = add(w->a, sub(scl(w->e, dot(qr, w->e)), scl(pt, rr / rt)));
    return 1;
}

/* point of the edge segment seen from o at the smallest angle to d; returns that angle */
static double wedge_nearest_seen(const wedge_t *w, vec3 o, vec3 d, vec3 *x_out) {
    vec3 a0 = sub(w->a, o), eb = sub(w->b, w->a);
    double al = dot(d, a0), be = dot(d, eb), c = dot(a0, a0), ep = dot(a0, eb), g = dot(eb, eb);
    double cand[3] = {0.0, 1.0, -1.0};
    double den = be * ep - al * g;
    if (den != 0.0) {
        double u = (al * ep - be * c) / den;
        if (u > 0.0 && u < 1.0) cand[2] = u;
    }
    double best = INFINITY;
    for (int i = 0; i < 3; ++i) {
        if (cand[i] < 0.0) continue;
        vec3 v = add(a0, scl(eb, cand[i]));
        double ang = angle_between(d, v);
        if (ang < best) { best = ang; *x_out = add(o, v); }
    }
    return best;
}

/*
 * Rough order-1 diffraction search (§III.A, Fig. 4) for the rays of one Tx.  A ray from
 * Tx meets wedge w when the edge point X seen at the smallest angle to the ray lies inside
 * the ray cone (angle <= cone) and ahead of Tx (foot s_X > 0), Tx lies in the wedge's
 * exterior, and X is visible from Tx (the segment Tx -> X is not blocked, the wedge's two
 * faces excluded: a ray grazing one of them just before the edge still has the edge in
 * its cone).  The diffracted rays leave X on its Keller cone; receiver r receives one when
 * it lies in the exterior, its error angle of Eq. 3 in the unfolded space,
 * angle(d, Rx* - Tx), is <= cone, and the segment X -> Rx is not blocked (the wedge's faces
 * excluded).  Each such (ray, wedge, rx) is a record: error angle and d_ray = |Rx* - Tx|
 * cos(error).  Returns the record count (first `cap` written).
 */
int64_t ora_diffract(void *sp, const double *tx3, const double *dirs, const int64_t *ray_ids, int64_t nrays,
                     const double *rx, int32_t nrx, double cone, int64_t cap, int32_t *rec_rx, int64_t *rec_ray,
                     int32_t *rec_wedge, double *rec_err, double *rec_dray) {
    scene *s = (scene *)sp;
    wedges_build(s);
    vec3 tx = ld(tx3);
    int64_t nrec = 0;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < nrays; ++i) {
        vec3 d = ld(dirs + 3 * i);
        for (int wi = 0; wi < s->nw; ++wi) {
            const wedge_t *w = &s->wd[wi];
            vec3 X;
            double ang = wedge_nearest_seen(w, tx, d, &X);
            if (!(ang <= cone)) continue;
            double sx = dot(sub(X, tx), d);
            if (!(sx > 0.0)) continue;
            if (!wedge_exterior(w, tx)) continue;
            if (occluded(s, tx, X, w->f1, w->f2)) continue;
            for (int r = 0; r < nrx; ++r) {
                vec3 R = ld(rx + 3 * r), Rs;
                if (!wedge_exterior(w, R) || !wedge_unfold_rx(w, tx, R, &Rs)) continue;
                vec3 W = sub(Rs, tx);
                double err = angle_between(d, W);
                if (!(err <= cone)) continue;
                if (occluded(s, X, R, w->f1, w->f2)) continue;
                int64_t slot;
#pragma omp atomic capture
                slot = nrec++;
                if (slot < cap) {
                    rec_rx[slot] = r;
                    rec_ray[slot] = ray_ids ? ray_ids[i] : i;
                    rec_wedge[slot] = wi;
                    rec_err[slot] = err;
                    rec_dray[slot] = norm(W) * cos(err);
                }
            }
        }
    }
    return nrec;
}

/*
 * Diffraction point of the ray tx + s d (d unit): the point Q = a + u (b - a) of the edge
 * line closest to the ray.  Writes u and the ray parameter s of the closest approach
 * (both -1 for a ray parallel to the edge).
 */
static vec3 wedge_ray_point(const wedge_t *w, vec3 tx, vec3 d, double *u_out, double *s_out) {
    /* closest points of the lines tx + s d and a + u (b - a) */
    vec3 eb = sub(w->b, w->a), w0 = sub(tx, w->a);
    double A = 1.0, B = dot(d, eb), C = dot(eb, eb), D = dot(d, w0), E = dot(eb, w0);
    double den = A * C - B * B;
    double u = den != 0.0 ? (A * E - B * D) / den : -1.0;
    *u_out = u;
    *s_out = den != 0.0 ? (B * E - C * D) / den : -1.0;
    return add(w->a, scl(eb, u));
}

/*
 * Exact diffraction point Q* of the pair (tx, rx) at wedge w: along the edge at z_T + (z_R
 * - z_T) r_T / (r_T + r_R) (z: position along the edge, r: distance from it), where the
 * segment Tx -> Rx* crosses the edge line.  Writes z; returns 0 if Tx lies on the line.
 */
static int wedge_exact_point(const wedge_t *w, vec3 tx, vec3 rx, vec3 *q_out, double *z_out) {
    vec3 qt = sub(tx, w->a), qr = sub(rx, w->a);
    double zt = dot(qt, w->e), zr = dot(qr, w->e);
    double rt = norm(perp_to(qt, w->e)), rr = norm(perp_to(qr, w->e));
    if (!(rt > 0.0)) return 0;
    double z = zt + (zr - zt) * rt / (rt + rr);
    *z_out = z;
    *q_out = add(w->a, scl(w->e, z));
    return 1;
}

/*
 * The precise algorithm (§III.B, Fig. 5, Eq. 10) for a diffraction path at wedge wi: the
 * same sub-ray pattern, argmin and shrink as ora_refine, with Eq. 3 evaluated in the
 * unfolded space of the wedge (see wedge_unfold_rx): error(d) = angle(d, Rx* - Tx) for
 * d . (Rx* - Tx) > 0, else +inf.  The early stop needs, as for reflections, both that
 * error (the AOD error) and the AOA error <= target: the angle at Rx between the
 * directions to the diffraction point of the current ray (wedge_ray_point) and to the
 * exact one (wedge_exact_point).  Returns iterations done (-1 for a bad K or Tx on the
 * edge line).
 */
int ora_refine_wedge(void *sp, const double *tx3, const double *rx3, int32_t wi, const double *c0, double R0,
                     int K, int iters, double target, double *out_dir, double *out_err, int32_t *choice,
                     double *err_hist) {
    scene *s = (scene *)sp;
    wedges_build(s);
    double rho[16], phi[16], shrink;
    if (ora_subray_pattern(K, rho, phi, &shrink) != K) return -1;
    vec3 tx = ld(tx3), rx = ld(rx3), c = unit(ld(c0)), Rs;
    if (!wedge_unfold_rx(&s->wd[wi], tx, rx, &Rs)) return -1;
    vec3 W = sub(Rs, tx), Qs;
    double zs, uq, sq;
    wedge_exact_point(&s->wd[wi], tx, rx, &Qs, &zs);
    double R = R0;
    double err = dot(c, W) > 0.0 ? angle_between(c, W) : INFINITY;
    double aoa = angle_between(sub(wedge_ray_point(&s->wd[wi], tx, unit(c), &uq, &sq), rx), sub(Qs, rx));
    if (err_hist) err_hist[0] = err;
    int it = 0;
    const double stall = 1.0 / (1.0 - shrink) + 2.0 * shrink;   /* stalled paths stop, see ora_refine */
    while (it < iters && !(target > 0 && err <= target && aoa <= target) && !(err > R * stall + 1e-6)) {
        vec3 u, v, best_d = c;
        double best = INFINITY;
        int bk = -1;
        cone_frame(c, &u, &v);
        for (int k = 0; k < K; ++k) {
            double a = rho[k] * R;
            vec3 dk = add(scl(c, cos(a)), scl(add(scl(u, cos(phi[k])), scl(v, sin(phi[k]))), sin(a)));
            double e = dot(dk, W) > 0.0 ? angle_between(dk, W) : INFINITY;
            if (e < best) { best = e; bk = k; best_d = dk; }
        }
        if (bk < 0) break;
        c = best_d;
        err = best;
        aoa = angle_between(sub(wedge_ray_point(&s->wd[wi], tx, unit(c), &uq, &sq), rx), sub(Qs, rx));
        R *= shrink;
        if (choice) choice[it] = bk;
        ++it;
        if (err_hist) err_hist[it] = err;
    }
    st(out_dir, c);
    *out_err = err;
    return it;
}

/*
 * Validity test and outputs of a diffraction path launched along `dir` (§III.A second
 * path test: the path must touch its wedge; §IV outputs).  The diffraction point Q is
 * the point of the edge line closest to the launched ray.  Valid iff Q lies on the edge
 * segment and ahead of Tx, Tx and Rx lie in the wedge's exterior, Tx -> Q and Q -> Rx are
 * not blocked (the wedge's faces excluded) and -- when err_bound > 0 -- the error angle
 * is at most err_bound.  Outputs: delay = (|Q - Tx| + |Rx - Q|) / c0; AOD = dir; AOA =
 * Q - Rx; power = ptx + free-space loss over the path length (the paper gives no
 * diffraction coefficient; parity unpinned).  Writes Q to q_out.  Returns 0, or -1 if
 * Tx lies on the edge line.
 */
int ora_wedge_eval(void *sp, const double *tx3, const double *rx3, int32_t wi, const double *dir, double freq,
                   double ptx_dbm, double err_bound, double *q_out, int32_t *valid, double *delay, double *aod,
                   double *aoa, double *power, double *err) {
    scene *s = (scene *)sp;
    wedges_build(s);
    const wedge_t *w = &s->wd[wi];
    vec3 tx = ld(tx3), rx = ld(rx3), d = unit(ld(dir)), Rs;
    *valid = 0;
    if (!wedge_unfold_rx(w, tx, rx, &Rs)) return -1;
    vec3 W = sub(Rs, tx);
    double e = dot(d, W) > 0.0 ? angle_between(d, W) : INFINITY;
    *err = e;
    double u, sq;
    vec3 Q = wedge_ray_point(w, tx, d, &u, &sq);
    if (q_out) st(q_out, Q);
    int ok = u >= 0.0 && u <= 1.0 && sq > 0.0 && wedge_exterior(w, tx) && wedge_exterior(w, rx);
    if (ok && (occluded(s, tx, Q, w->f1, w->f2) || occluded(s, Q, rx, w->f1, w->f2))) ok = 0;
    if (err_bound > 0.0 && !(e <= err_bound)) ok = 0;
    *valid = ok;
    double len = norm(sub(Q, tx)) + norm(sub(rx, Q));
    *delay = len / ORA_C0;
    az_el(d, aod);
    az_el(sub(Q, rx), aoa);
    *power = ptx_dbm + 20.0 * log10(ORA_C0 / freq / (4.0 * M_PI * len));
    return 0;
}

/*
 * Exact order-1 diffraction path at wedge wi (the image-method counterpart): the point Q*
 * where Tx -> Rx* crosses the edge line, i.e. along the edge at z_T + (z_R - z_T) r_T /
 * (r_T + r_R) (z: position along the edge, r: distance from it), the minimum of |Tx - Q| +
 * |Q - Rx| over the line (Fermat) where Keller's law holds.  Returns 1 if valid (Q* on the
 * segment, both ends exterior, unblocked), 0 if not, -1 if Tx lies on the edge line.
 */
int ora_wedge_image(void *sp, const double *tx3, const double *rx3, int32_t wi, double freq, double ptx_dbm,
                    double *q_out, double *aod_dir, double *delay, double *aod, double *aoa, double *power) {
    scene *s = (scene *)sp;
    wedges_build(s);
    const wedge_t *w = &s->wd[wi];
    vec3 tx = ld(tx3), rx = ld(rx3), Q;
    double z;
    if (!wedge_exact_point(w, tx, rx, &Q, &z)) return -1;
    st(q_out, Q);
    vec3 dir = unit(sub(Q, tx));
    st(aod_dir, dir);
    double len = norm(sub(Q, tx)) + norm(sub(rx, Q));
    *delay = len / ORA_C0;
    az_el(dir, aod);
    az_el(sub(Q, rx), aoa);
    *power = ptx_dbm + 20.0 * log10(ORA_C0 / freq / (4.0 * M_PI * len));
    double L = norm(sub(w->b, w->a));
    int ok = z >= 0.0 && z <= L && wedge_exterior(w, tx) && wedge_exterior(w, rx);
    if (ok && (occluded(s, tx, Q, w->f1, w->f2) || occluded(s, Q, rx, w->f1, w->f2))) ok = 0;
    return ok;
}
