/*
 * Plain FP64 CPU oracle of the parallel heat method for geodesic distance
 * (Tao, Zhang, Deng, Fang, Peng, He: "Parallel and Scalable Heat Methods for
 * Geodesic Distance Computation", arXiv 1812.06060).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package's smoke check and
 * the CPU-baseline leg of the benchmark may load this library.  It shares no
 * code, header, table or helper with the CUDA library it checks.
 *
 * Every function is a slow restatement of one step of the paper, in the
 * paper's order and notation, with no blocking or fusion.  Readings of
 * passages the paper leaves open are marked READING.
 *
 * The same source builds two libraries: the plain one (compiled without
 * OpenMP, where every `omp` pragma is ignored: single-threaded) and a
 * level-parallel one (-fopenmp) for the large cases.  A pragma sits only on
 * a loop whose iterations write disjoint locations and read nothing another
 * iteration of the same loop writes -- the vertices of one breadth-first set
 * in a Gauss-Seidel sweep (Jacobi within a set, eq. HeatDiffusionUpdate) or
 * in the integration, the faces or edges of one ADMM block update -- and
 * every sum whose value depends on its order stays a sequential loop, so the
 * two libraries give bit-identical results.
 *
 * Numerical reading shared by the diffusion stages (READING, Sec. 3.1): the
 * heat solution u decays by roughly e^-1 per edge length away from the
 * sources, so on large meshes it spans far more than the double exponent
 * range and plain arithmetic underflows to zero.  The paper is silent on
 * this.  Here each vertex value is carried as a mantissa m (0.5 <= |m| < 1,
 * or m = 0) and a separate int32 binary exponent e, u = m * 2^e.  Scaling by
 * a power of two is exact, so the iterates are the plain ones wherever plain
 * double arithmetic does not underflow (orc_gs_plain is the plain form).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)
#define ORC_ENONMANIFOLD (-3)

/* exponent of an exact zero: far below any real exponent, and far enough
 * above INT32_MIN that differences of two exponents do not overflow */
#define ORC_ZERO_EXP (-(1 << 28))

/* threads the parallel loops use (1 in the plain build) */
int orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Connectivity (Sec. 3 mesh (V, E, F); Sec. 4.1 orientation halfedges)      */
/* ------------------------------------------------------------------------ */

static int cmp_i64(const void *a, const void *b) {
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

/* Undirected edges of the mesh, sorted by (min, max); edge id = rank.
 * edges_out must hold 2 * 3 * nf int32.  Returns the edge count. */
int64_t orc_edges(int64_t nv, int64_t nf, const int32_t *F, int32_t *edges_out) {
    if (nv <= 0 || nf <= 0) return ORC_EINVAL;
    int64_t *key = (int64_t *)malloc(sizeof(int64_t) * 3 * nf);
    if (!key) return ORC_ENOMEM;
    int bad = 0;
#pragma omp parallel for reduction(| : bad)
    for (int64_t f = 0; f < nf; ++f) {
        for (int k = 0; k < 3; ++k) {
            int32_t a = F[3 * f + k], b = F[3 * f + (k + 1) % 3];
            if (a < 0 || a >= nv || b < 0 || b >= nv || a == b) { bad = 1; key[3 * f + k] = 0; continue; }
            int32_t lo = a < b ? a : b, hi = a < b ? b : a;
            key[3 * f + k] = (int64_t)lo * nv + hi;
        }
    }
    if (bad) { free(key); return ORC_EINVAL; }
    qsort(key, (size_t)(3 * nf), sizeof(int64_t), cmp_i64);
    int64_t ne = 0;
    for (int64_t i = 0; i < 3 * nf; ++i) {
        if (i > 0 && key[i] == key[i - 1]) continue;
        edges_out[2 * ne] = (int32_t)(key[i] / nv);
        edges_out[2 * ne + 1] = (int32_t)(key[i] % nv);
        ++ne;
    }
    free(key);
    return ne;
}

/* id of edge {a, b} by binary search in the sorted edge list, -1 if absent */
static int64_t find_edge(int64_t ne, const int32_t *edges, int32_t a, int32_t b) {
    int32_t lo = a < b ? a : b, hi = a < b ? b : a;
    int64_t l = 0, r = ne - 1;
    while (l <= r) {
        int64_t m = (l + r) / 2;
        int32_t x = edges[2 * m], y = edges[2 * m + 1];
        if (x == lo && y == hi) return m;
        if (x < lo || (x == lo && y < hi)) l = m + 1; else r = m - 1;
    }
    return -1;
}

/* Tail and head of the orientation halfedge eta_e (Sec. 4.1): min -> max
 * unless flip[e] is set (the paper lets either halfedge be chosen). */
static void eta(const int32_t *edges, const uint8_t *flip, int64_t e, int32_t *tail, int32_t *head) {
    int f = flip ? flip[e] : 0;
    *tail = f ? edges[2 * e + 1] : edges[2 * e];
    *head = f ? edges[2 * e] : edges[2 * e + 1];
}

/*
 * Per-face and per-edge incidence.  Local edge k of face (a, b, c) is the
 * edge opposite corner k; the face loop runs a->b->c->a, so local edge 0 is
 * b->c, 1 is c->a, 2 is a->b.
 *   face_edge[3f+k]  edge id of local edge k
 *   face_sign[3f+k]  s_k^f of eq. (Integrability): +1 if eta_e is the loop
 *                    halfedge of f, else -1 (Sec. 4.1)
 *   edge_face[2e+j], edge_slot[2e+j]  the 1 or 2 faces of e in ascending face
 *                    order and the local slot there; -1 when absent
 *   rowptr, col      one-ring of each vertex, neighbours ascending
 *   col_edge         edge id of each (row, col) entry
 * Errors: an edge in more than two faces, or two faces that traverse an edge
 * in the same direction (not an oriented 2-manifold), give ORC_ENONMANIFOLD.
 */
int orc_connectivity(int64_t nv, int64_t nf, const int32_t *F, int64_t ne, const int32_t *edges,
                     const uint8_t *flip, int32_t *face_edge, int8_t *face_sign, int32_t *edge_face,
                     int32_t *edge_slot, int32_t *rowptr, int32_t *col, int32_t *col_edge) {
    for (int64_t e = 0; e < 2 * ne; ++e) { edge_face[e] = -1; edge_slot[e] = -1; }
    int missing = 0;
#pragma omp parallel for reduction(| : missing)
    for (int64_t f = 0; f < nf; ++f) {
        for (int k = 0; k < 3; ++k) {
            int32_t a = F[3 * f + (k + 1) % 3], b = F[3 * f + (k + 2) % 3]; /* loop a->b */
            int64_t e = find_edge(ne, edges, a, b);
            if (e < 0) { missing = 1; face_edge[3 * f + k] = -1; continue; }
            face_edge[3 * f + k] = (int32_t)e;
            int32_t t, h;
            eta(edges, flip, e, &t, &h);
            face_sign[3 * f + k] = (t == a && h == b) ? 1 : -1;
        }
    }
    if (missing) return ORC_EINVAL;
    /* the faces of each edge in ascending face order */
    for (int64_t f = 0; f < nf; ++f) {
        for (int k = 0; k < 3; ++k) {
            int64_t e = face_edge[3 * f + k];
            if (edge_face[2 * e] < 0) { edge_face[2 * e] = (int32_t)f; edge_slot[2 * e] = k; }
            else if (edge_face[2 * e + 1] < 0) { edge_face[2 * e + 1] = (int32_t)f; edge_slot[2 * e + 1] = k; }
            else return ORC_ENONMANIFOLD;
        }
    }
    for (int64_t e = 0; e < ne; ++e) {
        if (edge_face[2 * e + 1] >= 0) {
            int32_t f0 = edge_face[2 * e], f1 = edge_face[2 * e + 1];
            if (face_sign[3 * f0 + edge_slot[2 * e]] == face_sign[3 * f1 + edge_slot[2 * e + 1]])
                return ORC_ENONMANIFOLD;
        }
    }
    /* CSR: each undirected edge (lo, hi) appears in row lo and row hi; the
     * edge list is sorted, so filling rows in edge order keeps every row
     * ascending only for the hi > row part; rows are sorted afterwards. */
    for (int64_t v = 0; v <= nv; ++v) rowptr[v] = 0;
    for (int64_t e = 0; e < ne; ++e) { rowptr[edges[2 * e] + 1]++; rowptr[edges[2 * e + 1] + 1]++; }
    for (int64_t v = 0; v < nv; ++v) rowptr[v + 1] += rowptr[v];
    int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * (size_t)nv);
    if (!fill) return ORC_ENOMEM;
    for (int64_t v = 0; v < nv; ++v) fill[v] = rowptr[v];
    for (int64_t e = 0; e < ne; ++e) {
        int32_t a = edges[2 * e], b = edges[2 * e + 1];
        col[fill[a]] = b; col_edge[fill[a]++] = (int32_t)e;
        col[fill[b]] = a; col_edge[fill[b]++] = (int32_t)e;
    }
    free(fill);
#pragma omp parallel for
    for (int64_t v = 0; v < nv; ++v) { /* insertion sort of each short row */
        for (int32_t i = rowptr[v] + 1; i < rowptr[v + 1]; ++i) {
            int32_t c = col[i], ce = col_edge[i], j = i - 1;
            while (j >= rowptr[v] && col[j] > c) { col[j + 1] = col[j]; col_edge[j + 1] = col_edge[j]; --j; }
            col[j + 1] = c; col_edge[j + 1] = ce;
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Geometry (Sec. 3.1: A_v, cotangent Laplacian; eq. DiffusionTime)          */
/* ------------------------------------------------------------------------ */

static void sub3(const double *a, const double *b, double *o) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double *a, const double *b, double *o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
static double norm3(const double *a) { return sqrt(dot3(a, a)); }

/*
 * A_f  face area, |(p_b - p_a) x (p_c - p_a)| / 2
 * A_v  one third of the total area of the faces incident with v (Sec. 3.1)
 * cot  cot of the interior angle at each corner, cot[3f+k]
 * theta  per edge: coefficient of the cotangent Laplacian,
 *        theta_e = 1/2 * sum over the faces of e of cot(angle opposite e).
 *        READING: Sec. 3.1 only names "the coefficient of v_k for the
 *        cotangent Laplacian"; the 1/2 is the usual convention of the heat
 *        method it builds on and fixes the meaning of t = m h^2.
 * hbar  mean edge length (eq. DiffusionTime)
 */
int orc_geometry(int64_t nv, const double *P, int64_t nf, const int32_t *F, int64_t ne, const int32_t *edges,
                 const int32_t *edge_face, const int32_t *edge_slot, double *Af, double *Av, double *cot,
                 double *theta, double *hbar) {
#pragma omp parallel for
    for (int64_t f = 0; f < nf; ++f) {
        const double *p[3] = {P + 3 * F[3 * f], P + 3 * F[3 * f + 1], P + 3 * F[3 * f + 2]};
        double u[3], w[3], n[3];
        sub3(p[1], p[0], u);
        sub3(p[2], p[0], w);
        cross3(u, w, n);
        Af[f] = 0.5 * norm3(n);
        for (int k = 0; k < 3; ++k) {
            double a[3], b[3], c[3];
            sub3(p[(k + 1) % 3], p[k], a);
            sub3(p[(k + 2) % 3], p[k], b);
            cross3(a, b, c);
            cot[3 * f + k] = dot3(a, b) / norm3(c);
        }
    }
    /* vertex areas: sums in face order */
    for (int64_t v = 0; v < nv; ++v) Av[v] = 0.0;
    for (int64_t f = 0; f < nf; ++f)
        for (int k = 0; k < 3; ++k) Av[F[3 * f + k]] += Af[f] / 3.0;
#pragma omp parallel for
    for (int64_t e = 0; e < ne; ++e) {
        double th = 0.0;
        for (int j = 0; j < 2; ++j)
            if (edge_face[2 * e + j] >= 0) th += 0.5 * cot[3 * edge_face[2 * e + j] + edge_slot[2 * e + j]];
        theta[e] = th;
    }
    /* mean edge length: the sum in edge order */
    double sum = 0.0;
    for (int64_t e = 0; e < ne; ++e) {
        double d[3];
        sub3(P + 3 * edges[2 * e], P + 3 * edges[2 * e + 1], d);
        sum += norm3(d);
    }
    *hbar = sum / (double)ne;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Breadth-first vertex sets (eq. VertexSets; Sec. 3.3; Sec. 5.2)            */
/* ------------------------------------------------------------------------ */

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/*
 * One breadth-first traversal from the source set (Sec. 3.3: computed once,
 * reused by diffusion and integration).  D_0 = the sorted, de-duplicated
 * sources (Sec. 5.2 puts all sources in D_0).  A FIFO queue pops vertices in
 * order and scans each one-ring in ascending neighbour order; an undiscovered
 * neighbour joins the next set with the popped vertex as its parent.
 * READING: the paper says the pairing v_j -> v_k comes from the traversal;
 * here the parent is the first discoverer.
 *   level[v]   i with v in D_i, or -1 if unreachable from every source
 *   parent[v]  the pairing vertex in D_{i-1}; -1 for sources and unreachable
 *   order      vertices in FIFO order; D_i = order[level_off[i] .. level_off[i+1])
 * Returns the number of sets L, or ORC_EINVAL (empty set, index out of range).
 */
int orc_bfs(int64_t nv, const int32_t *rowptr, const int32_t *col, int64_t nsrc, const int32_t *src,
            int32_t *level, int32_t *parent, int32_t *order, int32_t *level_off) {
    if (nsrc <= 0) return ORC_EINVAL;
    int32_t *s = (int32_t *)malloc(sizeof(int32_t) * (size_t)nsrc);
    if (!s) return ORC_ENOMEM;
    memcpy(s, src, sizeof(int32_t) * (size_t)nsrc);
    qsort(s, (size_t)nsrc, sizeof(int32_t), cmp_i32);
    for (int64_t v = 0; v < nv; ++v) { level[v] = -1; parent[v] = -1; }
    int64_t tail = 0;
    for (int64_t i = 0; i < nsrc; ++i) {
        if (s[i] < 0 || s[i] >= nv) { free(s); return ORC_EINVAL; }
        if (i > 0 && s[i] == s[i - 1]) continue;
        level[s[i]] = 0;
        order[tail++] = s[i];
    }
    free(s);
    int32_t nlev = 1;
    level_off[0] = 0;
    for (int64_t head = 0; head < tail; ++head) {
        int32_t v = order[head];
        for (int32_t j = rowptr[v]; j < rowptr[v + 1]; ++j) {
            int32_t w = col[j];
            if (level[w] >= 0) continue;
            level[w] = level[v] + 1;
            parent[w] = v;
            if (level[w] + 1 > nlev) { level_off[nlev] = (int32_t)tail; nlev = level[w] + 1; }
            order[tail++] = w;
        }
    }
    level_off[nlev] = (int32_t)tail;
    return nlev;
}

/* ------------------------------------------------------------------------ */
/* Gauss-Seidel heat diffusion in breadth-first order (eq. heat,             */
/* eq. HeatDiffusionUpdate)                                                  */
/* ------------------------------------------------------------------------ */

/*
 * Solves (A - t L_c) u = u_0 by `sweeps` outer iterations.  u_0 is 1 at every
 * source and 0 elsewhere (Sec. 3.1; Sec. 5.2 for a source set).  In each
 * outer iteration the sets D_0, D_1, ... are visited in order; the vertices
 * of one set are updated simultaneously (Jacobi within the set) from the
 * latest neighbour values: neighbours in D_{i-1} carry this iteration's new
 * value, neighbours in D_i and D_{i+1} the previous iteration's.
 *   u_j <- (u_0(j) + t sum_k theta_jk u_k) / (A_j + t sum_k theta_jk)
 * The sum runs over the one-ring in ascending neighbour order.
 * READING: the initial guess is not stated; the caller passes it (the
 * pipeline starts from u = 0).  Unreachable vertices are never updated.
 * State in/out: u_j = um[j] * 2^ue[j] (see the file header).
 */
int orc_gs(int64_t nv, const int32_t *rowptr, const int32_t *col, const int32_t *col_edge, const double *theta,
           const double *Av, double t, const int32_t *order, const int32_t *level_off, int32_t nlev,
           int32_t sweeps, double *um, int32_t *ue) {
    double *nm = (double *)malloc(sizeof(double) * (size_t)nv);
    int32_t *ne_ = (int32_t *)malloc(sizeof(int32_t) * (size_t)nv);
    if (!nm || !ne_) { free(nm); free(ne_); return ORC_ENOMEM; }
    for (int32_t k = 0; k < sweeps; ++k) {
        for (int32_t i = 0; i < nlev; ++i) {
            /* new values of D_i into (nm, ne_), all from the state before D_i */
#pragma omp parallel for if (level_off[i + 1] - level_off[i] > 256)
            for (int32_t q = level_off[i]; q < level_off[i + 1]; ++q) {
                int32_t j = order[q];
                double u0 = (i == 0) ? 1.0 : 0.0;
                int32_t eref = ORC_ZERO_EXP;
                if (u0 != 0.0) eref = 1; /* frexp(1) = 0.5 * 2^1 */
                for (int32_t a = rowptr[j]; a < rowptr[j + 1]; ++a) {
                    int32_t kk = col[a];
                    if (um[kk] != 0.0 && ue[kk] > eref) eref = ue[kk];
                }
                double s = 0.0, ts = 0.0;
                for (int32_t a = rowptr[j]; a < rowptr[j + 1]; ++a) {
                    int32_t kk = col[a];
                    double th = theta[col_edge[a]];
                    s += th * ldexp(um[kk], ue[kk] - eref);
                    ts += th;
                }
                double num = ldexp(u0, -eref) + t * s;
                double val = num / (Av[j] + t * ts);
                int ex = 0;
                double mm = frexp(val, &ex);
                nm[j] = mm;
                ne_[j] = (mm == 0.0) ? ORC_ZERO_EXP : ex + eref;
            }
#pragma omp parallel for if (level_off[i + 1] - level_off[i] > 256)
            for (int32_t q = level_off[i]; q < level_off[i + 1]; ++q) {
                int32_t j = order[q];
                um[j] = nm[j];
                ue[j] = ne_[j];
            }
        }
    }
    free(nm);
    free(ne_);
    return ORC_OK;
}

/* The same iteration in plain double arithmetic (no separate exponent); it
 * underflows on large meshes and exists to pin orc_gs on small ones. */
int orc_gs_plain(int64_t nv, const int32_t *rowptr, const int32_t *col, const int32_t *col_edge,
                 const double *theta, const double *Av, double t, const int32_t *order,
                 const int32_t *level_off, int32_t nlev, int32_t sweeps, double *u) {
    double *nu = (double *)malloc(sizeof(double) * (size_t)nv);
    if (!nu) return ORC_ENOMEM;
    for (int32_t k = 0; k < sweeps; ++k) {
        for (int32_t i = 0; i < nlev; ++i) {
            for (int32_t q = level_off[i]; q < level_off[i + 1]; ++q) {
                int32_t j = order[q];
                double u0 = (i == 0) ? 1.0 : 0.0;
                double s = 0.0, ts = 0.0;
                for (int32_t a = rowptr[j]; a < rowptr[j + 1]; ++a) {
                    double th = theta[col_edge[a]];
                    s += th * u[col[a]];
                    ts += th;
                }
                nu[j] = (u0 + t * s) / (Av[j] + t * ts);
            }
            for (int32_t q = level_off[i]; q < level_off[i + 1]; ++q) u[order[q]] = nu[order[q]];
        }
    }
    free(nu);
    return ORC_OK;
}

/* E1 of eq. HeatSolutionError, ||(A - t L_c) u - u_0||_2, in plain double
 * (far-field values that underflow contribute nothing measurable). */
double orc_heat_residual(int64_t nv, const int32_t *rowptr, const int32_t *col, const int32_t *col_edge,
                         const double *theta, const double *Av, double t, const int32_t *level,
                         const double *um, const int32_t *ue) {
    double acc = 0.0;
    for (int64_t j = 0; j < nv; ++j) {
        double uj = ldexp(um[j], ue[j]);
        double r = Av[j] * uj;
        for (int32_t a = rowptr[j]; a < rowptr[j + 1]; ++a) {
            double uk = ldexp(um[col[a]], ue[col[a]]);
            r -= t * theta[col_edge[a]] * (uk - uj);
        }
        r -= (level[j] == 0) ? 1.0 : 0.0;
        acc += r * r;
    }
    return sqrt(acc);
}

/* ------------------------------------------------------------------------ */
/* Face-wise gradient normalisation (Algorithm 1; eq.                        */
/* HeatDiffusionNormalization)                                               */
/* ------------------------------------------------------------------------ */

/*
 * grad u on face (a, b, c) = 1/(2 A_f) sum_i u_i (N x e_i), e_i the edge
 * opposite corner i taken counter-clockwise and N the unit normal;
 * h = -grad u / |grad u|.  The three values are first brought to their
 * common largest exponent (exact).  READING: a face with grad u = 0 (not
 * reached, or an exact symmetry) gets h = 0.
 */
int orc_normalize(int64_t nv, const double *P, int64_t nf, const int32_t *F, const double *um, const int32_t *ue,
                  double *h) {
    (void)nv;
#pragma omp parallel for
    for (int64_t f = 0; f < nf; ++f) {
        int32_t v[3] = {F[3 * f], F[3 * f + 1], F[3 * f + 2]};
        const double *p[3] = {P + 3 * v[0], P + 3 * v[1], P + 3 * v[2]};
        int32_t eref = ORC_ZERO_EXP;
        for (int i = 0; i < 3; ++i) if (um[v[i]] != 0.0 && ue[v[i]] > eref) eref = ue[v[i]];
        double u1[3], u2[3], n[3];
        sub3(p[1], p[0], u1);
        sub3(p[2], p[0], u2);
        cross3(u1, u2, n);
        double twoA = norm3(n);
        double N[3] = {n[0] / twoA, n[1] / twoA, n[2] / twoA};
        double g[3] = {0, 0, 0};
        for (int i = 0; i < 3; ++i) {
            double e[3], ne[3];
            sub3(p[(i + 2) % 3], p[(i + 1) % 3], e);
            cross3(N, e, ne);
            double ui = ldexp(um[v[i]], ue[v[i]] - eref);
            g[0] += ui * ne[0]; g[1] += ui * ne[1]; g[2] += ui * ne[2];
        }
        g[0] /= twoA; g[1] /= twoA; g[2] /= twoA;
        double len = norm3(g);
        for (int c = 0; c < 3; ++c) h[3 * f + c] = (len > 0.0) ? -g[c] / len : 0.0;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Multi-source path constraints (Sec. 5.2, eq. MultiSourceConstraint,       */
/* eq. MultiSourceConstraintEdgeBased)                                       */
/* ------------------------------------------------------------------------ */

/*
 * npc linear constraints sum_i c_i . v_{var_i} = 0 on the variables of one
 * ADMM block: the edge differences x (dim 1) or the face gradients g (dim 3).
 * The entries of constraint j are [off[j], off[j+1]): variable var[i],
 * coefficient coef[dim i .. dim i + dim).
 *
 * READING: Sec. 5.2 says only that the extended problem stays convex and is
 * solved by ADMM.  Here the constraints join the block they act on.  That
 * block's subproblem is a separable quadratic 1/2 sum_v D_v |v - vhat_v|^2
 * around its unconstrained update vhat (D_e = |H_e| (1 + mu) for x, from the
 * objective 1/2 sum (x - z)^2 and the penalty; D_f = A_f (2 + mu n_f) for g,
 * from A_f |g - h|^2 and the M-weighted penalty over the face's n_f interior
 * slots).  Its minimiser under C v = 0 solves the KKT system:
 *   v = vhat - D^-1 C^T nu,   (C D^-1 C^T) nu = C vhat.
 * The Gram matrix C D^-1 C^T is factored once (Cholesky); a constraint whose
 * pivot is at most 1e-12 of its diagonal entry depends on the earlier ones
 * (or is empty) and is dropped: nu_j = 0.
 */
typedef struct {
    int32_t npc, dim, nu;  /* constraints, values per variable, distinct variables */
    int32_t *uvar;         /* [nu] the variable of each distinct entry */
    double *ucoef;         /* [nu][npc][dim] coefficients summed per variable */
    double *dinv;          /* [nu] 1 / D_v */
    double *L;             /* [npc][npc] lower Cholesky factor of the Gram matrix */
    int32_t *drop;         /* [npc] */
} orc_pc;

static void pc_free(orc_pc *pc) {
    free(pc->uvar); free(pc->ucoef); free(pc->dinv); free(pc->L); free(pc->drop);
    memset(pc, 0, sizeof(*pc));
}

/* the distinct variables of the entries (in order of first appearance) and
 * their coefficient rows; nvar = the block's variable count */
static int pc_build(orc_pc *pc, int64_t nvar, int32_t npc, int32_t dim, const int32_t *off, const int32_t *var,
                    const double *coef) {
    memset(pc, 0, sizeof(*pc));
    pc->npc = npc;
    pc->dim = dim;
    if (npc <= 0) return ORC_OK;
    int32_t nent = off[npc];
    int32_t *slot = (int32_t *)malloc(sizeof(int32_t) * (size_t)nvar);
    pc->uvar = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nent > 0 ? nent : 1));
    pc->ucoef = (double *)calloc((size_t)(nent > 0 ? nent : 1) * npc * dim, sizeof(double));
    pc->dinv = (double *)malloc(sizeof(double) * (size_t)(nent > 0 ? nent : 1));
    pc->L = (double *)calloc((size_t)npc * npc, sizeof(double));
    pc->drop = (int32_t *)calloc((size_t)npc, sizeof(int32_t));
    if (!slot || !pc->uvar || !pc->ucoef || !pc->dinv || !pc->L || !pc->drop) {
        free(slot);
        pc_free(pc);
        return ORC_ENOMEM;
    }
    for (int64_t v = 0; v < nvar; ++v) slot[v] = -1;
    for (int32_t j = 0; j < npc; ++j) {
        for (int32_t i = off[j]; i < off[j + 1]; ++i) {
            int32_t v = var[i];
            if (v < 0 || v >= nvar) { free(slot); pc_free(pc); return ORC_EINVAL; }
            if (slot[v] < 0) { slot[v] = pc->nu; pc->uvar[pc->nu++] = v; }
            for (int c = 0; c < dim; ++c)
                pc->ucoef[((size_t)slot[v] * npc + j) * dim + c] += coef[(size_t)dim * i + c];
        }
    }
    free(slot);
    return ORC_OK;
}

/* Gram matrix G_jk = sum_v c_vj . c_vk / D_v and its Cholesky factor
 * (dinv must be filled) */
static void pc_factor(orc_pc *pc) {
    int32_t n = pc->npc, dim = pc->dim;
    double *G = (double *)calloc((size_t)n * n + 1, sizeof(double));
    for (int32_t u = 0; u < pc->nu; ++u)
        for (int32_t j = 0; j < n; ++j)
            for (int32_t k = 0; k < n; ++k) {
                double s = 0.0;
                for (int c = 0; c < dim; ++c)
                    s += pc->ucoef[((size_t)u * n + j) * dim + c] * pc->ucoef[((size_t)u * n + k) * dim + c];
                G[j * n + k] += s * pc->dinv[u];
            }
    for (int32_t j = 0; j < n; ++j) {
        double d = G[j * n + j];
        for (int32_t m = 0; m < j; ++m) d -= pc->L[j * n + m] * pc->L[j * n + m];
        if (!(d > 1e-12 * G[j * n + j])) { pc->drop[j] = 1; continue; }   /* row j of L stays 0 */
        double ljj = sqrt(d);
        pc->L[j * n + j] = ljj;
        for (int32_t k = j + 1; k < n; ++k) {
            double s = G[k * n + j];
            for (int32_t m = 0; m < j; ++m) s -= pc->L[k * n + m] * pc->L[j * n + m];
            pc->L[k * n + j] = s / ljj;
        }
    }
    free(G);
}

/* v <- vhat - D^-1 C^T nu with (C D^-1 C^T) nu = C vhat; vals holds vhat */
static void pc_project(const orc_pc *pc, double *vals) {
    int32_t n = pc->npc, dim = pc->dim;
    if (n <= 0) return;
    double r[64], nu[64];
    for (int32_t j = 0; j < n; ++j) {
        double s = 0.0;
        for (int32_t u = 0; u < pc->nu; ++u)
            for (int c = 0; c < dim; ++c)
                s += pc->ucoef[((size_t)u * n + j) * dim + c] * vals[(size_t)dim * pc->uvar[u] + c];
        r[j] = s;
    }
    /* L L^T nu = r, dropped constraints held at 0 */
    for (int32_t j = 0; j < n; ++j) {
        if (pc->drop[j]) { nu[j] = 0.0; continue; }
        double s = r[j];
        for (int32_t m = 0; m < j; ++m) s -= pc->L[j * n + m] * nu[m];
        nu[j] = s / pc->L[j * n + j];
    }
    for (int32_t j = n - 1; j >= 0; --j) {
        if (pc->drop[j]) { nu[j] = 0.0; continue; }
        double s = nu[j];
        for (int32_t m = j + 1; m < n; ++m) s -= pc->L[m * n + j] * nu[m];
        nu[j] = s / pc->L[j * n + j];
    }
    for (int32_t u = 0; u < pc->nu; ++u)
        for (int c = 0; c < dim; ++c) {
            double s = 0.0;
            for (int32_t j = 0; j < n; ++j) s += pc->ucoef[((size_t)u * n + j) * dim + c] * nu[j];
            vals[(size_t)dim * pc->uvar[u] + c] -= pc->dinv[u] * s;
        }
}

/* ------------------------------------------------------------------------ */
/* Face-based integrable gradient field by ADMM (Sec. 3.2)                   */
/* ------------------------------------------------------------------------ */

/*
 * Minimises sum_i A_i |g_i - h_i|^2 subject to ebar.(g_1^e - g_2^e) = 0 on
 * every interior edge (eq. Integrable, eq. GradCompatibility), in the split
 * form of eq. NewTarget / eq. ADMMMatrixFormConstraint with one auxiliary
 * vector y per (face, interior edge) slot and M = diag(sqrt(A)).
 * Initialisation: g = y = h, lambda = 0.  Each iteration, in the paper's
 * order:
 *   Y: per interior edge with faces 1, 2 and q_i = g_i - lambda_i/(mu alpha_i):
 *        y_1 = q_1 + A_2/(A_1+A_2) ebar (ebar.(q_2 - q_1))
 *        y_2 = q_2 - A_1/(A_1+A_2) ebar (ebar.(q_2 - q_1))
 *   G: g_i = (2 h_i + mu sum_k (y_k + lambda_k/(mu alpha_i))) / (2 + mu |Y(i)|)
 *      (g_i = h_i when the face has no interior edge)
 *   lambda: lambda_k += mu alpha_i (y_k - g_i)
 * Storage per slot [3f+k]: y and lambda (NaN on boundary slots).
 * res (nullable) receives per iteration |r_primal|_F, |r_dual|_F and |M|_F
 * With early_stop the iterations end once |r_primal| <= |M|_F eps1 and
 * |r_dual| <= |M|_F eps2 (Sec. 3.2); done (nullable) receives the
 * iterations run.
 * with r_primal = M (Y - S G) and r_dual = mu M S dG.  READING: the dual
 * residual is printed with a matrix A that is never defined; it is read as M.
 */
int orc_face_admm(int64_t nv, const double *P, int64_t nf, int64_t ne, const int32_t *edges,
                  const int32_t *face_edge, const int32_t *edge_face, const int32_t *edge_slot, const double *Af,
                  const double *h, int32_t iters, double mu, double eps1, double eps2, int32_t early_stop,
                  int32_t npc, const int32_t *pc_off, const int32_t *pc_var, const double *pc_coef,
                  const double *eslot, double *g, double *y, double *lam, double *res, int32_t *done) {
    (void)nv;
    if (npc < 0 || npc > 64) return ORC_EINVAL;
    orc_pc pc;
    int rc = pc_build(&pc, nf, npc, 3, pc_off, pc_var, pc_coef);
    if (rc != ORC_OK) return rc;
    for (int32_t u = 0; u < pc.nu; ++u) {   /* D_f = A_f (2 + mu n_f) */
        int64_t f = pc.uvar[u];
        int n = 0;
        for (int k = 0; k < 3; ++k) n += edge_face[2 * face_edge[3 * f + k] + 1] >= 0;
        pc.dinv[u] = 1.0 / (Af[f] * (2.0 + mu * n));
    }
    pc_factor(&pc);
    double *gold = (double *)malloc(sizeof(double) * 3 * (size_t)nf);
    if (!gold) { pc_free(&pc); return ORC_ENOMEM; }
    for (int64_t f = 0; f < nf; ++f)
        for (int k = 0; k < 3; ++k)
            for (int c = 0; c < 3; ++c) { y[9 * f + 3 * k + c] = NAN; lam[9 * f + 3 * k + c] = NAN; }
    for (int64_t e = 0; e < ne; ++e) {
        if (edge_face[2 * e + 1] < 0) continue;
        for (int j = 0; j < 2; ++j) {
            int64_t f = edge_face[2 * e + j];
            int k = edge_slot[2 * e + j];
            for (int c = 0; c < 3; ++c) { y[9 * f + 3 * k + c] = h[3 * f + c]; lam[9 * f + 3 * k + c] = 0.0; }
        }
    }
    for (int64_t i = 0; i < 3 * nf; ++i) g[i] = h[i];
    double mnorm2 = 0.0;
    for (int64_t e = 0; e < ne; ++e)
        if (edge_face[2 * e + 1] >= 0) mnorm2 += Af[edge_face[2 * e]] + Af[edge_face[2 * e + 1]];

    for (int32_t it = 0; it < iters; ++it) {
        /* Y-update, one interior edge at a time */
#pragma omp parallel for
        for (int64_t e = 0; e < ne; ++e) {
            if (edge_face[2 * e + 1] < 0) continue;
            int64_t f1 = edge_face[2 * e], f2 = edge_face[2 * e + 1];
            int k1 = edge_slot[2 * e], k2 = edge_slot[2 * e + 1];
            double A1 = Af[f1], A2 = Af[f2];
            double a1 = sqrt(A1), a2 = sqrt(A2);
            double q1[3], q2[3];
            for (int c = 0; c < 3; ++c) {
                q1[c] = g[3 * f1 + c] - lam[9 * f1 + 3 * k1 + c] / (mu * a1);
                q2[c] = g[3 * f2 + c] - lam[9 * f2 + 3 * k2 + c] / (mu * a2);
            }
            if (eslot) {
                /* an intrinsic triangulation (Sec. 5.3): each face has its own
                 * frame and its own unit vector e_i of the edge; the condition
                 * e_1 . y_1 = e_2 . y_2 gives y_1 = q_1 + A2/(A1+A2) e_1 p,
                 * y_2 = q_2 - A1/(A1+A2) e_2 p, p = e_2 . q_2 - e_1 . q_1 */
                const double *v1 = eslot + 9 * f1 + 3 * k1, *v2 = eslot + 9 * f2 + 3 * k2;
                double n1 = norm3(v1), n2 = norm3(v2);
                double e1[3] = {v1[0] / n1, v1[1] / n1, v1[2] / n1}, e2[3] = {v2[0] / n2, v2[1] / n2, v2[2] / n2};
                double proj = dot3(e2, q2) - dot3(e1, q1);
                for (int c = 0; c < 3; ++c) {
                    y[9 * f1 + 3 * k1 + c] = q1[c] + A2 / (A1 + A2) * e1[c] * proj;
                    y[9 * f2 + 3 * k2 + c] = q2[c] - A1 / (A1 + A2) * e2[c] * proj;
                }
                continue;
            }
            double ev[3];
            sub3(P + 3 * edges[2 * e + 1], P + 3 * edges[2 * e], ev);
            double el = norm3(ev);
            double eb[3] = {ev[0] / el, ev[1] / el, ev[2] / el};
            double dq[3] = {q2[0] - q1[0], q2[1] - q1[1], q2[2] - q1[2]};
            double proj = dot3(eb, dq);
            for (int c = 0; c < 3; ++c) {
                y[9 * f1 + 3 * k1 + c] = q1[c] + A2 / (A1 + A2) * eb[c] * proj;
                y[9 * f2 + 3 * k2 + c] = q2[c] - A1 / (A1 + A2) * eb[c] * proj;
            }
        }
        /* G-update, one face at a time */
        for (int64_t i = 0; i < 3 * nf; ++i) gold[i] = g[i];
#pragma omp parallel for
        for (int64_t f = 0; f < nf; ++f) {
            double alpha = sqrt(Af[f]);
            double acc[3] = {0, 0, 0};
            int n = 0;
            for (int k = 0; k < 3; ++k) {
                if (edge_face[2 * face_edge[3 * f + k] + 1] < 0) continue; /* boundary edge: no y */
                for (int c = 0; c < 3; ++c) acc[c] += y[9 * f + 3 * k + c] + lam[9 * f + 3 * k + c] / (mu * alpha);
                ++n;
            }
            for (int c = 0; c < 3; ++c) g[3 * f + c] = (2.0 * h[3 * f + c] + mu * acc[c]) / (2.0 + mu * n);
        }
        /* the multi-source path constraints, if any, as part of the G-update */
        pc_project(&pc, g);
        /* lambda-update */
#pragma omp parallel for
        for (int64_t f = 0; f < nf; ++f) {
            double alpha = sqrt(Af[f]);
            for (int k = 0; k < 3; ++k) {
                if (edge_face[2 * face_edge[3 * f + k] + 1] < 0) continue;
                for (int c = 0; c < 3; ++c) lam[9 * f + 3 * k + c] += mu * (alpha * (y[9 * f + 3 * k + c] - g[3 * f + c]));
            }
        }
        /* the residual norms, summed in slot order */
        double rp = 0.0, rd = 0.0;
        for (int64_t f = 0; f < nf; ++f) {
            double alpha = sqrt(Af[f]);
            for (int k = 0; k < 3; ++k) {
                if (edge_face[2 * face_edge[3 * f + k] + 1] < 0) continue;
                for (int c = 0; c < 3; ++c) {
                    double r = alpha * (y[9 * f + 3 * k + c] - g[3 * f + c]);
                    rp += r * r;
                    double dg = mu * alpha * (g[3 * f + c] - gold[3 * f + c]);
                    rd += dg * dg;
                }
            }
        }
        if (res) { res[3 * it] = sqrt(rp); res[3 * it + 1] = sqrt(rd); res[3 * it + 2] = sqrt(mnorm2); }
        if (done) *done = it + 1;
        /* Sec. 3.2: stop once |r_primal| <= |M|_F eps1 and |r_dual| <= |M|_F eps2 */
        if (early_stop && sqrt(rp) <= sqrt(mnorm2) * eps1 && sqrt(rd) <= sqrt(mnorm2) * eps2) break;
    }
    if (done && iters <= 0) *done = 0;
    free(gold);
    pc_free(&pc);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Edge-based optimisation by ADMM (Sec. 4.1)                                */
/* ------------------------------------------------------------------------ */

/*
 * Target differences z = Z[3f+k] = h_f . e, e the vector of the orientation
 * halfedge (head - tail) of local edge k (eq. TargetDifference); z_in
 * (nullable) gives them instead (an intrinsic triangulation, whose edge
 * vectors live in each face's own frame, Sec. 5.3).
 * Minimises 1/2 sum_e sum_{h in H_e} (x_e - h_e)^2 subject to
 * sum_k s_k^f x_{e_k^f} = 0 on every face (eq. Integrability), split as
 * W - R X = 0.  Initialisation: lambda = 0, x_e = mean of its targets,
 * w = z.  Each iteration, in the paper's order:
 *   W: w_f = (I - q q^T / 3)(x_f - lambda_f / mu), q = the face's signs
 *   X: x_e = sum_{slots of e} (z + lambda + mu w) / (|H_e| (1 + mu))  (eq. xeupdate)
 *   lambda: lambda += mu (W - R X)
 * res (nullable) receives per iteration |W - RX| and |mu R dX|.  With
 * early_stop the iteration ends once |W - RX| <= |Z|_F eps1 and
 * |mu R dX| <= |Z|_F eps2; done (nullable) receives the iterations run.
 */
int orc_edge_admm(int64_t nv, const double *P, int64_t nf, const int32_t *F, int64_t ne, const int32_t *edges,
                  const uint8_t *flip, const int32_t *face_edge, const int8_t *face_sign, const int32_t *edge_face,
                  const int32_t *edge_slot, const double *h, int32_t iters, double mu, double eps1, double eps2,
                  int32_t early_stop, int32_t npc, const int32_t *pc_off, const int32_t *pc_var,
                  const double *pc_coef, const double *z_in, double *x, double *w, double *lam, double *z,
                  double *res, int32_t *done) {
    (void)nv; (void)F;
    if (npc < 0 || npc > 64) return ORC_EINVAL;
    orc_pc pc;
    int rc = pc_build(&pc, ne, npc, 1, pc_off, pc_var, pc_coef);
    if (rc != ORC_OK) return rc;
    for (int32_t u = 0; u < pc.nu; ++u) {   /* D_e = |H_e| (1 + mu) */
        int64_t e = pc.uvar[u];
        int n = (edge_face[2 * e] >= 0) + (edge_face[2 * e + 1] >= 0);
        pc.dinv[u] = 1.0 / (n * (1.0 + mu));
    }
    pc_factor(&pc);
    double *xold = (double *)malloc(sizeof(double) * (size_t)ne);
    if (!xold) { pc_free(&pc); return ORC_ENOMEM; }
#pragma omp parallel for
    for (int64_t f = 0; f < nf; ++f) {
        for (int k = 0; k < 3; ++k) {
            if (z_in) {   /* targets given (an intrinsic triangulation's local frames) */
                z[3 * f + k] = z_in[3 * f + k];
                continue;
            }
            int64_t e = face_edge[3 * f + k];
            int32_t ta, hd;
            eta(edges, flip, e, &ta, &hd);
            double ev[3];
            sub3(P + 3 * hd, P + 3 * ta, ev);
            z[3 * f + k] = dot3(h + 3 * f, ev);
        }
    }
#pragma omp parallel for
    for (int64_t e = 0; e < ne; ++e) {
        double s = 0.0;
        int n = 0;
        for (int j = 0; j < 2; ++j)
            if (edge_face[2 * e + j] >= 0) { s += z[3 * edge_face[2 * e + j] + edge_slot[2 * e + j]]; ++n; }
        x[e] = s / n;
    }
    for (int64_t i = 0; i < 3 * nf; ++i) { w[i] = z[i]; lam[i] = 0.0; }
    /* the scale of the edge form's residuals: |Z|_F, the norm of the targets
       (the paper prints no thresholds for this form; read as in Sec. 3.2 with
       |Z|_F in the place of |M|_F) */
    double znorm2 = 0.0;
    for (int64_t i = 0; i < 3 * nf; ++i) znorm2 += z[i] * z[i];

    for (int32_t it = 0; it < iters; ++it) {
        /* W-update per face */
#pragma omp parallel for
        for (int64_t f = 0; f < nf; ++f) {
            double v[3], q[3];
            for (int k = 0; k < 3; ++k) {
                v[k] = x[face_edge[3 * f + k]] - lam[3 * f + k] / mu;
                q[k] = (double)face_sign[3 * f + k];
            }
            double qv = dot3(q, v);
            for (int k = 0; k < 3; ++k) w[3 * f + k] = v[k] - q[k] * qv / 3.0;
        }
        /* X-update per edge */
#pragma omp parallel for
        for (int64_t e = 0; e < ne; ++e) {
            xold[e] = x[e];
            double s = 0.0;
            int n = 0;
            for (int j = 0; j < 2; ++j) {
                if (edge_face[2 * e + j] < 0) continue;
                int64_t sl = 3 * (int64_t)edge_face[2 * e + j] + edge_slot[2 * e + j];
                s += z[sl] + lam[sl] + mu * w[sl];
                ++n;
            }
            x[e] = s / (n * (1.0 + mu));
        }
        /* the multi-source path constraints, if any, as part of the X-update */
        pc_project(&pc, x);
        /* lambda-update per face slot */
#pragma omp parallel for
        for (int64_t f = 0; f < nf; ++f)
            for (int k = 0; k < 3; ++k) lam[3 * f + k] += mu * (w[3 * f + k] - x[face_edge[3 * f + k]]);
        /* the residual norms, summed in slot order */
        double rp = 0.0, rd = 0.0;
        for (int64_t f = 0; f < nf; ++f) {
            for (int k = 0; k < 3; ++k) {
                int64_t e = face_edge[3 * f + k];
                double r = w[3 * f + k] - x[e];
                rp += r * r;
                double d = mu * (x[e] - xold[e]);
                rd += d * d;
            }
        }
        if (res) { res[2 * it] = sqrt(rp); res[2 * it + 1] = sqrt(rd); }
        if (done) *done = it + 1;
        if (early_stop && sqrt(rp) <= sqrt(znorm2) * eps1 && sqrt(rd) <= sqrt(znorm2) * eps2) break;
    }
    if (done && iters <= 0) *done = 0;
    free(xold);
    pc_free(&pc);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Integration in breadth-first order (Sec. 3.3 eq. IntegrationStep; Sec. 4) */
/* ------------------------------------------------------------------------ */

/* edge id of {a, b} from the CSR row of a, -1 if not adjacent */
static int32_t csr_edge(const int32_t *rowptr, const int32_t *col, const int32_t *col_edge, int32_t a, int32_t b) {
    for (int32_t j = rowptr[a]; j < rowptr[a + 1]; ++j)
        if (col[j] == b) return col_edge[j];
    return -1;
}

/*
 * Face form: d = 0 on D_0; for D_1, D_2, ... in order, each v_j with its
 * pairing vertex v_k = parent[j] in D_{i-1}:
 *   d(v_j) = d(v_k) + 1/|T_jk| sum_{f in T_jk} g_f . (p_j - p_k)
 * where T_jk are the faces that contain both vertices.  Sources keep d = 0
 * (Sec. 5.2); unreachable vertices get +infinity.  eslot (nullable): an
 * intrinsic triangulation's slot edge vectors in each face's own frame
 * (lower -> higher vertex), which give p_j - p_k there (Sec. 5.3).
 */
int orc_integrate_face(int64_t nv, const double *P, const int32_t *rowptr, const int32_t *col,
                       const int32_t *col_edge, const int32_t *edge_face, const int32_t *edge_slot,
                       const double *eslot, const int32_t *order, const int32_t *level_off, int32_t nlev,
                       const int32_t *parent, const double *g, double *d) {
    for (int64_t v = 0; v < nv; ++v) d[v] = INFINITY;
    for (int32_t q = level_off[0]; q < level_off[1]; ++q) d[order[q]] = 0.0;
    for (int32_t i = 1; i < nlev; ++i) {
        int missing = 0;
#pragma omp parallel for reduction(| : missing) if (level_off[i + 1] - level_off[i] > 256)
        for (int32_t q = level_off[i]; q < level_off[i + 1]; ++q) {
            int32_t j = order[q], k = parent[j];
            int32_t e = csr_edge(rowptr, col, col_edge, k, j);
            if (e < 0) { missing = 1; continue; }
            double dp[3];
            sub3(P + 3 * j, P + 3 * k, dp);
            double s = 0.0;
            int n = 0;
            for (int a = 0; a < 2; ++a) {
                int32_t f = edge_face[2 * e + a];
                if (f < 0) continue;
                if (eslot) {   /* p_j - p_k in face f's own frame: its slot vector, lower -> higher */
                    const double *v = eslot + 9 * f + 3 * edge_slot[2 * e + a];
                    const double sg = (j > k) ? 1.0 : -1.0;
                    dp[0] = sg * v[0]; dp[1] = sg * v[1]; dp[2] = sg * v[2];
                }
                s += dot3(g + 3 * f, dp);
                ++n;
            }
            d[j] = d[k] + s / n;
        }
        if (missing) return ORC_EINVAL;
    }
    return ORC_OK;
}

/*
 * Edge form: the edge variable is the change of d along the orientation
 * halfedge, x_e = d(head) - d(tail) (Sec. 4: g.e = d(v1) - d(v2)), so
 * d(v_j) = d(v_k) + x_e when v_j is the head of eta_e and d(v_k) - x_e
 * otherwise, in the same breadth-first order.
 */
int orc_integrate_edge(int64_t nv, const int32_t *edges, const uint8_t *flip, const int32_t *rowptr,
                       const int32_t *col, const int32_t *col_edge, const int32_t *order, const int32_t *level_off,
                       int32_t nlev, const int32_t *parent, const double *x, double *d) {
    for (int64_t v = 0; v < nv; ++v) d[v] = INFINITY;
    for (int32_t q = level_off[0]; q < level_off[1]; ++q) d[order[q]] = 0.0;
    for (int32_t i = 1; i < nlev; ++i) {
        int missing = 0;
#pragma omp parallel for reduction(| : missing) if (level_off[i + 1] - level_off[i] > 256)
        for (int32_t q = level_off[i]; q < level_off[i + 1]; ++q) {
            int32_t j = order[q], k = parent[j];
            int32_t e = csr_edge(rowptr, col, col_edge, k, j);
            if (e < 0) { missing = 1; continue; }
            int32_t ta, hd;
            eta(edges, flip, e, &ta, &hd);
            d[j] = (hd == j) ? d[k] + x[e] : d[k] - x[e];
        }
        if (missing) return ORC_EINVAL;
    }
    return ORC_OK;
}
