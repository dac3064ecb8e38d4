/*
 * Oracle for segmented Quickhull (Tzeng & Owens, "Finding Convex Hulls Using
 * Quickhull on the GPU").  TEST INFRASTRUCTURE ONLY: the test suite, the
 * smoke check and the benchmark's CPU-baseline leg may load this library;
 * the product path never does.  It shares no code with the CUDA path.
 *
 * What it computes is the plain definition of the result:
 *   2D: the extreme points of the float32 input, read exactly as reals, in
 *       counter-clockwise order starting at the lexicographically smallest
 *       (x, y) vertex; a location present several times is reported as its
 *       lowest input index.
 *   3D: the face lattice of the convex hull: maximal coplanar faces as
 *       polygons, counter-clockwise seen from outside, each rotated to start
 *       at its smallest index, faces sorted lexicographically.
 *
 * It gets there by a sequential Quickhull in the paper's order of steps
 * (Algorithm 4 for 2D; Algorithm 1 with Barber et al.'s visible-set/horizon
 * reading for 3D), single-threaded, FP64 arithmetic, and exact signs for
 * every predicate: an FP64 evaluation with a forward error bound, and when
 * that cannot decide, an exact sum of the predicate's monomials held as a
 * non-overlapping floating-point expansion (Shewchuk 1997, "Adaptive
 * Precision Floating-Point Arithmetic and Fast Robust Geometric Predicates":
 * two-sum, two-product, grow-expansion).  Inputs are float32, so every
 * product of two coordinates is exact in FP64 and every product of three
 * is exact as a two-term expansion.
 *
 * Build with -ffp-contract=off: the error bounds assume separately rounded
 * products and sums.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_INVALID 1
#define OR_ERR_NONFINITE 2
#define OR_ERR_DEGENERATE 3
#define OR_ERR_NOMEM 4

/* ------------------------------------------------------------------------ */
/* Exact arithmetic                                                          */
/* ------------------------------------------------------------------------ */

static void two_sum(double a, double b, double *s, double *e)
{
    double x = a + b;
    double bv = x - a;
    double av = x - bv;
    *s = x;
    *e = (a - av) + (b - bv);
}

static void two_prod(double a, double b, double *p, double *e)
{
    double x = a * b;
    *p = x;
    *e = fma(a, b, -x);
}

/* Add b to the non-overlapping expansion e (increasing magnitude, length
 * *len); zero components are dropped.  h may alias e. */
static void grow(double *e, int *len, double b)
{
    double q = b;
    int out = 0;
    for (int i = 0; i < *len; i++) {
        double s, err;
        two_sum(q, e[i], &s, &err);
        q = s;
        if (err != 0.0)
            e[out++] = err;
    }
    if (q != 0.0 || out == 0)
        e[out++] = q;
    *len = out;
}

/* Exact sign of the sum of m doubles. */
static int exact_sign_of_sum(const double *t, int m)
{
    double e[160];
    int len = 0;
    for (int i = 0; i < m; i++)
        grow(e, &len, t[i]);
    double top = e[len - 1];
    return (top > 0.0) - (top < 0.0);
}

/* ------------------------------------------------------------------------ */
/* 2D predicates                                                             */
/* ------------------------------------------------------------------------ */

static const double EPS = 1.1102230246251565e-16; /* 2^-53 */

/* Sign of (p1 - p2) x (p3 - p4) = (p1x-p2x)(p3y-p4y) - (p1y-p2y)(p3x-p4x).
 * orient2d(a, b, c) is cross_diff(a, c, b, c): positive when a, b, c turn
 * counter-clockwise. */
static int cross_diff2(const double *p1, const double *p2, const double *p3, const double *p4)
{
    double l = (p1[0] - p2[0]) * (p3[1] - p4[1]);
    double r = (p1[1] - p2[1]) * (p3[0] - p4[0]);
    double det = l - r;
    double bound = (3.0 + 16.0 * EPS) * EPS * (fabs(l) + fabs(r));
    if (det > bound)
        return 1;
    if (-det > bound)
        return -1;
    /* monomials of (p1x-p2x)(p3y-p4y) - (p1y-p2y)(p3x-p4x) */
    double t[8] = {
        p1[0] * p3[1], -p1[0] * p4[1], -p2[0] * p3[1], p2[0] * p4[1],
        -p1[1] * p3[0], p1[1] * p4[0], p2[1] * p3[0], -p2[1] * p4[0],
    };
    return exact_sign_of_sum(t, 8);
}

static int orient2d(const double *a, const double *b, const double *c)
{
    return cross_diff2(a, c, b, c);
}

/* Compare the distances of p1 and p2 beyond the directed line a->b:
 * sign(orient2d(a,b,p1) - orient2d(a,b,p2)) = sign((b - a) x (p1 - p2)). */
static int cmp_dist2(const double *a, const double *b, const double *p1, const double *p2)
{
    return cross_diff2(b, a, p1, p2);
}

/* ------------------------------------------------------------------------ */
/* 3D predicates                                                             */
/* ------------------------------------------------------------------------ */

/* Append the 12 doubles whose exact sum is s * det[x; y; z]. */
static int det3_terms(const double *x, const double *y, const double *z, double s, double *out)
{
    static const int P[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    static const double SG[6] = {1, -1, -1, 1, 1, -1};
    for (int k = 0; k < 6; k++) {
        double xy = x[P[k][0]] * y[P[k][1]]; /* exact: two 24-bit mantissas */
        double hi, lo;
        two_prod(xy, z[P[k][2]], &hi, &lo);
        out[2 * k] = s * SG[k] * hi;
        out[2 * k + 1] = s * SG[k] * lo;
    }
    return 12;
}

/* Sign of det[u; v; w] for rows computed in FP64, with the forward error
 * bound (7 + 56 eps) eps * permanent (each entry a rounded difference of
 * exact inputs). Returns 2 when the bound cannot decide. */
static int det3_filter(const double *u, const double *v, const double *w)
{
    double m0 = v[1] * w[2], m1 = v[2] * w[1];
    double m2 = v[2] * w[0], m3 = v[0] * w[2];
    double m4 = v[0] * w[1], m5 = v[1] * w[0];
    double det = u[0] * (m0 - m1) + u[1] * (m2 - m3) + u[2] * (m4 - m5);
    double perm = fabs(u[0]) * (fabs(m0) + fabs(m1)) + fabs(u[1]) * (fabs(m2) + fabs(m3)) +
                  fabs(u[2]) * (fabs(m4) + fabs(m5));
    double bound = (7.0 + 56.0 * EPS) * EPS * perm;
    if (det > bound)
        return 1;
    if (-det > bound)
        return -1;
    return 2;
}

/* vol(a,b,c,p) = det[b-a; c-a; p-a]: positive when p lies on the side of
 * the normal (b-a) x (c-a), i.e. the side from which a, b, c appear
 * counter-clockwise. */
static int orient3d(const double *a, const double *b, const double *c, const double *p)
{
    double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double v[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    double w[3] = {p[0] - a[0], p[1] - a[1], p[2] - a[2]};
    int s = det3_filter(u, v, w);
    if (s != 2)
        return s;
    /* det[b-a, c-a, p-a] = det[b,c,p] - det[a,c,p] - det[b,a,p] - det[b,c,a] */
    double t[48];
    int m = 0;
    m += det3_terms(b, c, p, 1.0, t + m);
    m += det3_terms(a, c, p, -1.0, t + m);
    m += det3_terms(b, a, p, -1.0, t + m);
    m += det3_terms(b, c, a, -1.0, t + m);
    return exact_sign_of_sum(t, m);
}

/* sign(vol(a,b,c,p1) - vol(a,b,c,p2)) = sign(det[b-a; c-a; p1-p2]). */
static int cmp_dist3(const double *a, const double *b, const double *c, const double *p1,
                     const double *p2)
{
    double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double v[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    double w[3] = {p1[0] - p2[0], p1[1] - p2[1], p1[2] - p2[2]};
    int s = det3_filter(u, v, w);
    if (s != 2)
        return s;
    /* det[b-a, c-a, x] = det[b,c,x] - det[a,c,x] - det[b,a,x], linear in x */
    double t[72];
    int m = 0;
    m += det3_terms(b, c, p1, 1.0, t + m);
    m += det3_terms(a, c, p1, -1.0, t + m);
    m += det3_terms(b, a, p1, -1.0, t + m);
    m += det3_terms(b, c, p2, -1.0, t + m);
    m += det3_terms(a, c, p2, 1.0, t + m);
    m += det3_terms(b, a, p2, 1.0, t + m);
    return exact_sign_of_sum(t, m);
}

/* Exactly collinear in 3D: every coordinate-plane projection is collinear. */
static int collinear3(const double *a, const double *b, const double *c)
{
    double pa[2], pb[2], pc[2];
    for (int k = 0; k < 3; k++) {
        int i = k, j = (k + 1) % 3;
        pa[0] = a[i]; pa[1] = a[j];
        pb[0] = b[i]; pb[1] = b[j];
        pc[0] = c[i]; pc[1] = c[j];
        if (orient2d(pa, pb, pc) != 0)
            return 0;
    }
    return 1;
}

/* Exported for the predicate pins. */
int oracle_orient2d(const double *a, const double *b, const double *c) { return orient2d(a, b, c); }
int oracle_cmp_dist2(const double *a, const double *b, const double *p1, const double *p2)
{
    return cmp_dist2(a, b, p1, p2);
}
int oracle_orient3d(const double *a, const double *b, const double *c, const double *p)
{
    return orient3d(a, b, c, p);
}
int oracle_cmp_dist3(const double *a, const double *b, const double *c, const double *p1,
                     const double *p2)
{
    return cmp_dist3(a, b, c, p1, p2);
}

/* ------------------------------------------------------------------------ */
/* 2D Quickhull (Algorithm 4)                                                */
/* ------------------------------------------------------------------------ */

#define P2(i) (pts + 2 * (int64_t)(i))

/* Lexicographic (x, y) comparison of two points, exact on float32 data;
 * -0.0 and +0.0 compare equal. */
static int lex_cmp(const double *p, const double *q, int d)
{
    for (int k = 0; k < d; k++) {
        if (p[k] < q[k])
            return -1;
        if (p[k] > q[k])
            return 1;
    }
    return 0;
}

typedef struct {
    int32_t e0, e1;  /* segment edge: outside points p have orient2d(e0, e1, p) > 0 */
    int64_t lo, hi;  /* range of the work index array holding the segment's points */
    int32_t emit;    /* >= 0: this frame only emits vertex `emit` */
} frame2;

int oracle_hull2d(const float *x, const float *y, int64_t n, int32_t *out, int64_t *h_out,
                  int64_t *iterations)
{
    *h_out = 0;
    if (iterations)
        *iterations = 0;
    if (n < 0)
        return OR_ERR_INVALID;
    if (n == 0)
        return OR_OK;
    for (int64_t i = 0; i < n; i++)
        if (!isfinite(x[i]) || !isfinite(y[i]))
            return OR_ERR_NONFINITE;

    double *pts = (double *)malloc(sizeof(double) * 2 * (size_t)n);
    int32_t *work = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *chain = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    frame2 *stack = (frame2 *)malloc(sizeof(frame2) * (size_t)(2 * n + 4));
    if (!pts || !work || !chain || !stack) {
        free(pts); free(work); free(chain); free(stack);
        return OR_ERR_NOMEM;
    }
    for (int64_t i = 0; i < n; i++) {
        pts[2 * i] = (double)x[i] + 0.0; /* + 0.0 maps -0.0 to +0.0 */
        pts[2 * i + 1] = (double)y[i] + 0.0;
    }

    /* First split, step 1: extrema along x (lexicographic, ties to the
     * lowest index). */
    int32_t a = 0, b = 0;
    for (int64_t i = 1; i < n; i++) {
        if (lex_cmp(P2(i), P2(a), 2) < 0)
            a = (int32_t)i;
        if (lex_cmp(P2(i), P2(b), 2) > 0)
            b = (int32_t)i;
    }
    if (lex_cmp(P2(a), P2(b), 2) == 0) {
        out[0] = a;
        *h_out = 1;
        free(pts); free(work); free(chain); free(stack);
        return OR_OK;
    }

    /* First split, step 2: points strictly above a->b form one segment,
     * points strictly below (above b->a) the other; the rest is discarded. */
    int64_t nu = 0, nl = 0;
    for (int64_t i = 0; i < n; i++)
        if (orient2d(P2(a), P2(b), P2(i)) > 0)
            work[nu++] = (int32_t)i;
    for (int64_t i = 0; i < n; i++)
        if (orient2d(P2(b), P2(a), P2(i)) > 0)
            work[nu + nl++] = (int32_t)i;

    /* Recursive step with an explicit stack; frames pop in traversal order
     * e0 -> (vertices) -> e1, so `chain` fills clockwise from a. */
    int64_t hc = 0, sp = 0, iters = 0;
    chain[hc++] = a;
    stack[sp++] = (frame2){b, a, nu, nu + nl, -1};
    stack[sp++] = (frame2){-1, -1, 0, 0, b};
    stack[sp++] = (frame2){a, b, 0, nu, -1};
    while (sp > 0) {
        frame2 f = stack[--sp];
        if (f.emit >= 0) {
            chain[hc++] = f.emit;
            continue;
        }
        if (f.hi <= f.lo)
            continue;
        iters++;
        /* farthest point from the segment's line, ties to the lowest index */
        int32_t q = work[f.lo];
        for (int64_t k = f.lo + 1; k < f.hi; k++) {
            int32_t p = work[k];
            int c = cmp_dist2(P2(f.e0), P2(f.e1), P2(p), P2(q));
            if (c > 0 || (c == 0 && p < q))
                q = p;
        }
        /* triangle (e0, q, e1): interior points are discarded; the rest go
         * to the edge they are strictly outside of */
        int64_t w0 = f.lo;
        for (int64_t k = f.lo; k < f.hi; k++) {
            int32_t p = work[k];
            if (p != q && orient2d(P2(f.e0), P2(q), P2(p)) > 0) {
                int32_t t = work[w0];
                work[w0++] = p;
                work[k] = t;
            }
        }
        int64_t w1 = w0;
        for (int64_t k = w0; k < f.hi; k++) {
            int32_t p = work[k];
            if (p != q && orient2d(P2(q), P2(f.e1), P2(p)) > 0) {
                int32_t t = work[w1];
                work[w1++] = p;
                work[k] = t;
            }
        }
        stack[sp++] = (frame2){q, f.e1, w0, w1, -1};
        stack[sp++] = (frame2){-1, -1, 0, 0, q};
        stack[sp++] = (frame2){f.e0, q, f.lo, w0, -1};
    }

    /* chain is clockwise from a; reverse it to counter-clockwise from a */
    int32_t *ccw = work; /* reuse */
    ccw[0] = chain[0];
    for (int64_t k = 1; k < hc; k++)
        ccw[k] = chain[hc - k];
    /* a tied apex may sit inside a collinear run: drop vertices collinear
     * with their neighbours */
    int64_t h = 0;
    if (hc <= 2) {
        for (int64_t k = 0; k < hc; k++)
            out[h++] = ccw[k];
    } else {
        for (int64_t k = 0; k < hc; k++) {
            int32_t pv = ccw[(k + hc - 1) % hc], v = ccw[k], nx = ccw[(k + 1) % hc];
            if (orient2d(P2(pv), P2(v), P2(nx)) != 0)
                out[h++] = v;
        }
    }
    *h_out = h;
    if (iterations)
        *iterations = iters;
    free(pts); free(work); free(chain); free(stack);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* 3D Quickhull (Algorithm 1, Barber et al. visible set / horizon / cone)    */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t v[3];   /* counter-clockwise seen from outside */
    int32_t nb[3];  /* nb[i]: facet across edge (v[i], v[i+1]) */
    int32_t head;   /* first point of the outside set, -1 if empty */
    int32_t count;
    int32_t alive;
    int32_t mark;
} facet3;

typedef struct {
    facet3 *f;
    int64_t nf, cap;
} facets3;

static int push_facet(facets3 *F, int32_t a, int32_t b, int32_t c)
{
    if (F->nf == F->cap) {
        int64_t cap = F->cap ? 2 * F->cap : 64;
        facet3 *nf = (facet3 *)realloc(F->f, sizeof(facet3) * (size_t)cap);
        if (!nf)
            return -1;
        F->f = nf;
        F->cap = cap;
    }
    facet3 *t = &F->f[F->nf];
    t->v[0] = a; t->v[1] = b; t->v[2] = c;
    t->nb[0] = t->nb[1] = t->nb[2] = -1;
    t->head = -1;
    t->count = 0;
    t->alive = 1;
    t->mark = 0;
    return (int)(F->nf++);
}

#define P3(i) (pts + 3 * (int64_t)(i))

static int facet_side(const double *pts, const facet3 *f, int32_t p)
{
    return orient3d(P3(f->v[0]), P3(f->v[1]), P3(f->v[2]), P3(p));
}

/* union-find for merging coplanar triangles */
static int32_t uf_find(int32_t *par, int32_t x)
{
    while (par[x] != x) {
        par[x] = par[par[x]];
        x = par[x];
    }
    return x;
}

static int cmp_face(const int32_t *A, int la, const int32_t *B, int lb)
{
    int m = la < lb ? la : lb;
    for (int i = 0; i < m; i++) {
        if (A[i] != B[i])
            return A[i] < B[i] ? -1 : 1;
    }
    return (la > lb) - (la < lb);
}

typedef struct {
    int32_t *idx;
    int32_t len;
} face_ref;

static int face_qsort_cmp(const void *pa, const void *pb)
{
    const face_ref *A = (const face_ref *)pa, *B = (const face_ref *)pb;
    return cmp_face(A->idx, A->len, B->idx, B->len);
}

static int int_cmp(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/*
 * Outputs: verts (sorted unique vertex indices, capacity n), face_off
 * (nf + 1 entries, capacity 2n), face_idx (capacity 6n).  Returns
 * OR_ERR_DEGENERATE when the points do not span 3D (n in 1..3 included).
 */
int oracle_hull3d(const float *x, const float *y, const float *z, int64_t n, int32_t *verts,
                  int64_t *nv_out, int32_t *face_off, int32_t *face_idx, int64_t *nf_out,
                  int64_t *iterations)
{
    *nv_out = 0;
    *nf_out = 0;
    if (iterations)
        *iterations = 0;
    if (n < 0)
        return OR_ERR_INVALID;
    if (n == 0) {
        face_off[0] = 0;
        return OR_OK;
    }
    for (int64_t i = 0; i < n; i++)
        if (!isfinite(x[i]) || !isfinite(y[i]) || !isfinite(z[i]))
            return OR_ERR_NONFINITE;
    if (n < 4)
        return OR_ERR_DEGENERATE;

    int rc = OR_OK;
    double *pts = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    int32_t *nextp = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *start_at = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *end_at = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    facets3 F = {0, 0, 0};
    int32_t *queue = NULL, *visible = NULL, *pending = NULL, *par = NULL;
    if (!pts || !nextp || !start_at || !end_at) {
        rc = OR_ERR_NOMEM;
        goto done;
    }
    for (int64_t i = 0; i < n; i++) {
        pts[3 * i] = (double)x[i] + 0.0;
        pts[3 * i + 1] = (double)y[i] + 0.0;
        pts[3 * i + 2] = (double)z[i] + 0.0;
    }

    /* First split: extrema a, b along x (lexicographic, lowest index on ties) */
    int32_t a = 0, b = 0;
    for (int64_t i = 1; i < n; i++) {
        if (lex_cmp(P3(i), P3(a), 3) < 0)
            a = (int32_t)i;
        if (lex_cmp(P3(i), P3(b), 3) > 0)
            b = (int32_t)i;
    }
    if (lex_cmp(P3(a), P3(b), 3) == 0) {
        rc = OR_ERR_DEGENERATE;
        goto done;
    }
    /* c: farthest from the line ab (FP64 squared distance; exactness is not
     * needed for the choice, only for the non-collinearity check below) */
    int32_t c = -1;
    {
        double best = -1.0;
        const double *A = P3(a), *B = P3(b);
        double d[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
        for (int64_t i = 0; i < n; i++) {
            const double *p = P3(i);
            double w[3] = {p[0] - A[0], p[1] - A[1], p[2] - A[2]};
            double cx = d[1] * w[2] - d[2] * w[1];
            double cy = d[2] * w[0] - d[0] * w[2];
            double cz = d[0] * w[1] - d[1] * w[0];
            double s = cx * cx + cy * cy + cz * cz;
            if (s > best) {
                best = s;
                c = (int32_t)i;
            }
        }
        if (collinear3(P3(a), P3(b), P3(c))) {
            c = -1;
            for (int64_t i = 0; i < n && c < 0; i++)
                if (!collinear3(P3(a), P3(b), P3(i)))
                    c = (int32_t)i;
        }
        if (c < 0) {
            rc = OR_ERR_DEGENERATE;
            goto done;
        }
    }
    /* d: farthest from the plane abc (FP64 |vol|; the choice need not be
     * exact, only the non-coplanarity check) */
    int32_t d = -1;
    {
        double best = -1.0;
        const double *A = P3(a), *B = P3(b), *C = P3(c);
        double u[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
        double v[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
        double nrm[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
        for (int64_t i = 0; i < n; i++) {
            const double *p = P3(i);
            double s = fabs(nrm[0] * (p[0] - A[0]) + nrm[1] * (p[1] - A[1]) + nrm[2] * (p[2] - A[2]));
            if (s > best) {
                best = s;
                d = (int32_t)i;
            }
        }
        if (orient3d(P3(a), P3(b), P3(c), P3(d)) == 0) {
            d = -1;
            for (int64_t i = 0; i < n && d < 0; i++)
                if (orient3d(P3(a), P3(b), P3(c), P3(i)) != 0)
                    d = (int32_t)i;
        }
        if (d < 0) {
            rc = OR_ERR_DEGENERATE;
            goto done;
        }
    }

    /* Initial tetrahedron, facets oriented with the opposite vertex inside. */
    {
        int32_t tv[4] = {a, b, c, d};
        for (int o = 0; o < 4; o++) {
            int32_t f3[3];
            int k = 0;
            for (int j = 0; j < 4; j++)
                if (j != o)
                    f3[k++] = tv[j];
            if (orient3d(P3(f3[0]), P3(f3[1]), P3(f3[2]), P3(tv[o])) > 0) {
                int32_t t = f3[1];
                f3[1] = f3[2];
                f3[2] = t;
            }
            if (push_facet(&F, f3[0], f3[1], f3[2]) < 0) {
                rc = OR_ERR_NOMEM;
                goto done;
            }
        }
        for (int i = 0; i < 4; i++)
            for (int e = 0; e < 3; e++) {
                int32_t u = F.f[i].v[e], v = F.f[i].v[(e + 1) % 3];
                for (int j = 0; j < 4; j++) {
                    if (j == i)
                        continue;
                    for (int g = 0; g < 3; g++)
                        if (F.f[j].v[g] == v && F.f[j].v[(g + 1) % 3] == u)
                            F.f[i].nb[e] = j;
                }
            }
    }
    /* outside sets: each point goes to the first facet it is strictly above */
    for (int64_t i = n - 1; i >= 0; i--) {
        for (int k = 0; k < 4; k++) {
            if (facet_side(pts, &F.f[k], (int32_t)i) > 0) {
                nextp[i] = F.f[k].head;
                F.f[k].head = (int32_t)i;
                F.f[k].count++;
                break;
            }
        }
    }

    for (int64_t i = 0; i < n; i++)
        start_at[i] = end_at[i] = -1;

    int64_t qcap = 1024, qh = 0, qt = 0;
    queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)qcap);
    int64_t vcap = 1024;
    visible = (int32_t *)malloc(sizeof(int32_t) * (size_t)vcap);
    int64_t pcap = 1024;
    pending = (int32_t *)malloc(sizeof(int32_t) * (size_t)pcap);
    if (!queue || !visible || !pending) {
        rc = OR_ERR_NOMEM;
        goto done;
    }
    for (int k = 0; k < 4; k++)
        queue[qt++] = k;

    int32_t stamp = 0;
    int64_t iters = 0;
    while (qh < qt) {
        int32_t fi = queue[qh++];
        if (qh > 4096 && qh * 2 > qt) { /* compact the queue */
            memmove(queue, queue + qh, sizeof(int32_t) * (size_t)(qt - qh));
            qt -= qh;
            qh = 0;
        }
        if (!F.f[fi].alive || F.f[fi].head < 0)
            continue;
        iters++;
        /* farthest point of the outside set from the facet's plane */
        facet3 *f0 = &F.f[fi];
        int32_t q = f0->head;
        for (int32_t p = nextp[q]; p >= 0; p = nextp[p]) {
            int cmpv = cmp_dist3(P3(f0->v[0]), P3(f0->v[1]), P3(f0->v[2]), P3(p), P3(q));
            if (cmpv > 0 || (cmpv == 0 && p < q))
                q = p;
        }
        /* visible set: facets q is strictly above, connected to fi */
        stamp++;
        int64_t nvis = 0;
        visible[nvis++] = fi;
        F.f[fi].mark = stamp;
        for (int64_t k = 0; k < nvis; k++) {
            facet3 *g = &F.f[visible[k]];
            for (int e = 0; e < 3; e++) {
                int32_t h = g->nb[e];
                if (F.f[h].mark == stamp || F.f[h].mark == -stamp)
                    continue;
                if (facet_side(pts, &F.f[h], q) > 0) {
                    F.f[h].mark = stamp;
                    if (nvis == vcap) {
                        vcap *= 2;
                        int32_t *nvb = (int32_t *)realloc(visible, sizeof(int32_t) * (size_t)vcap);
                        if (!nvb) {
                            rc = OR_ERR_NOMEM;
                            goto done;
                        }
                        visible = nvb;
                    }
                    visible[nvis++] = h;
                } else {
                    F.f[h].mark = -stamp;
                }
            }
        }
        /* horizon edges -> cone facets (u, v, q) */
        int64_t first_new = F.nf;
        for (int64_t k = 0; k < nvis; k++) {
            int32_t gi = visible[k];
            for (int e = 0; e < 3; e++) {
                int32_t h = F.f[gi].nb[e];
                if (F.f[h].mark == stamp)
                    continue;
                int32_t u = F.f[gi].v[e], v = F.f[gi].v[(e + 1) % 3];
                int nfi = push_facet(&F, u, v, q);
                if (nfi < 0) {
                    rc = OR_ERR_NOMEM;
                    goto done;
                }
                F.f[nfi].nb[0] = h;
                for (int g = 0; g < 3; g++)
                    if (F.f[h].nb[g] == gi)
                        F.f[h].nb[g] = nfi;
                start_at[u] = nfi;
                end_at[v] = nfi;
            }
        }
        for (int64_t k = first_new; k < F.nf; k++) {
            facet3 *t = &F.f[k];
            t->nb[1] = start_at[t->v[1]]; /* edge (v, q): next cone facet */
            t->nb[2] = end_at[t->v[0]];   /* edge (q, u): previous cone facet */
        }
        /* gather the outside points of the visible facets and reassign them
         * to the first cone facet they are strictly above */
        int64_t npend = 0;
        for (int64_t k = 0; k < nvis; k++) {
            facet3 *g = &F.f[visible[k]];
            for (int32_t p = g->head; p >= 0; p = nextp[p]) {
                if (p == q)
                    continue;
                if (npend == pcap) {
                    pcap *= 2;
                    int32_t *np2 = (int32_t *)realloc(pending, sizeof(int32_t) * (size_t)pcap);
                    if (!np2) {
                        rc = OR_ERR_NOMEM;
                        goto done;
                    }
                    pending = np2;
                }
                pending[npend++] = p;
            }
            g->alive = 0;
            g->head = -1;
            g->count = 0;
        }
        for (int64_t k = npend - 1; k >= 0; k--) {
            int32_t p = pending[k];
            for (int64_t j = first_new; j < F.nf; j++) {
                if (facet_side(pts, &F.f[j], p) > 0) {
                    nextp[p] = F.f[j].head;
                    F.f[j].head = p;
                    F.f[j].count++;
                    break;
                }
            }
        }
        for (int64_t j = first_new; j < F.nf; j++) {
            if (qt == qcap) {
                qcap *= 2;
                int32_t *nq = (int32_t *)realloc(queue, sizeof(int32_t) * (size_t)qcap);
                if (!nq) {
                    rc = OR_ERR_NOMEM;
                    goto done;
                }
                queue = nq;
            }
            queue[qt++] = (int32_t)j;
        }
    }

    /* Merge coplanar neighbouring triangles into maximal faces. */
    par = (int32_t *)malloc(sizeof(int32_t) * (size_t)F.nf);
    if (!par) {
        rc = OR_ERR_NOMEM;
        goto done;
    }
    for (int64_t k = 0; k < F.nf; k++)
        par[k] = (int32_t)k;
    for (int64_t k = 0; k < F.nf; k++) {
        if (!F.f[k].alive)
            continue;
        for (int e = 0; e < 3; e++) {
            int32_t h = F.f[k].nb[e];
            if (h < (int32_t)k)
                continue;
            /* vertex of h opposite the shared edge */
            int32_t opp = -1;
            for (int g = 0; g < 3; g++) {
                int32_t w = F.f[h].v[g];
                if (w != F.f[k].v[e] && w != F.f[k].v[(e + 1) % 3])
                    opp = w;
            }
            if (facet_side(pts, &F.f[k], opp) == 0) {
                int32_t r1 = uf_find(par, (int32_t)k), r2 = uf_find(par, h);
                if (r1 != r2)
                    par[r1 < r2 ? r2 : r1] = r1 < r2 ? r1 : r2;
            }
        }
    }
    {
        /* boundary edges of each group: edges whose neighbour is in another
         * group; chain them with a successor map keyed by start vertex */
        int32_t *succ = start_at; /* reuse: succ[u] = v for boundary edge (u,v) */
        int32_t *gstamp = end_at; /* reuse: group of the successor entry */
        for (int64_t i = 0; i < n; i++)
            gstamp[i] = -1;
        /* collect groups */
        int64_t nface = 0, nidx = 0;
        int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)F.nf);
        int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * n + 2));
        int32_t *fidx_tmp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(6 * n + 16));
        int32_t *foff_tmp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * n + 16));
        if (!order || !tmp || !fidx_tmp || !foff_tmp) {
            free(order); free(tmp); free(fidx_tmp); free(foff_tmp);
            rc = OR_ERR_NOMEM;
            goto done;
        }
        /* sort alive facets by group root (counting through a bucket list) */
        int32_t *bucket_head = (int32_t *)malloc(sizeof(int32_t) * (size_t)F.nf);
        int32_t *bucket_next = (int32_t *)malloc(sizeof(int32_t) * (size_t)F.nf);
        if (!bucket_head || !bucket_next) {
            free(order); free(tmp); free(fidx_tmp); free(foff_tmp);
            free(bucket_head); free(bucket_next);
            rc = OR_ERR_NOMEM;
            goto done;
        }
        for (int64_t k = 0; k < F.nf; k++)
            bucket_head[k] = -1;
        for (int64_t k = F.nf - 1; k >= 0; k--) {
            if (!F.f[k].alive)
                continue;
            int32_t r = uf_find(par, (int32_t)k);
            bucket_next[k] = bucket_head[r];
            bucket_head[r] = (int32_t)k;
        }
        foff_tmp[0] = 0;
        for (int64_t r = 0; r < F.nf; r++) {
            if (bucket_head[r] < 0)
                continue;
            int32_t start_v = -1;
            for (int32_t k = bucket_head[r]; k >= 0; k = bucket_next[k]) {
                for (int e = 0; e < 3; e++) {
                    int32_t h = F.f[k].nb[e];
                    if (uf_find(par, h) == r)
                        continue;
                    int32_t u = F.f[k].v[e], v = F.f[k].v[(e + 1) % 3];
                    succ[u] = v;
                    gstamp[u] = (int32_t)r;
                    if (start_v < 0 || u < start_v)
                        start_v = u;
                }
            }
            /* walk the boundary cycle */
            int64_t len = 0;
            int32_t u = start_v;
            do {
                tmp[len++] = u;
                if (gstamp[u] != (int32_t)r || len > n) {
                    rc = OR_ERR_INVALID; /* cannot happen with exact predicates */
                    break;
                }
                u = succ[u];
            } while (u != start_v);
            if (rc != OR_OK) {
                free(order); free(tmp); free(fidx_tmp); free(foff_tmp);
                free(bucket_head); free(bucket_next);
                goto done;
            }
            /* drop vertices collinear with their polygon neighbours */
            int64_t m = 0;
            int32_t *keep = tmp + n + 1;
            for (int64_t k = 0; k < len; k++) {
                int32_t pv = tmp[(k + len - 1) % len], v = tmp[k], nx = tmp[(k + 1) % len];
                if (!collinear3(P3(pv), P3(v), P3(nx)))
                    keep[m++] = v;
            }
            /* rotate to start at the smallest index */
            int64_t arg = 0;
            for (int64_t k = 1; k < m; k++)
                if (keep[k] < keep[arg])
                    arg = k;
            for (int64_t k = 0; k < m; k++)
                fidx_tmp[nidx + k] = keep[(arg + k) % m];
            nidx += m;
            foff_tmp[++nface] = (int32_t)nidx;
        }
        free(bucket_head);
        free(bucket_next);
        /* sort faces lexicographically */
        face_ref *refs = (face_ref *)malloc(sizeof(face_ref) * (size_t)(nface + 1));
        if (!refs) {
            free(order); free(tmp); free(fidx_tmp); free(foff_tmp);
            rc = OR_ERR_NOMEM;
            goto done;
        }
        for (int64_t k = 0; k < nface; k++) {
            refs[k].idx = fidx_tmp + foff_tmp[k];
            refs[k].len = foff_tmp[k + 1] - foff_tmp[k];
        }
        qsort(refs, (size_t)nface, sizeof(face_ref), face_qsort_cmp);
        int64_t w = 0;
        face_off[0] = 0;
        for (int64_t k = 0; k < nface; k++) {
            memcpy(face_idx + w, refs[k].idx, sizeof(int32_t) * (size_t)refs[k].len);
            w += refs[k].len;
            face_off[k + 1] = (int32_t)w;
        }
        /* vertex set */
        int32_t *vv = fidx_tmp; /* reuse as scratch after copy-out */
        memcpy(vv, face_idx, sizeof(int32_t) * (size_t)w);
        qsort(vv, (size_t)w, sizeof(int32_t), int_cmp);
        int64_t nvv = 0;
        for (int64_t k = 0; k < w; k++)
            if (nvv == 0 || vv[k] != verts[nvv - 1])
                verts[nvv++] = vv[k];
        *nv_out = nvv;
        *nf_out = nface;
        free(refs);
        free(order);
        free(tmp);
        free(fidx_tmp);
        free(foff_tmp);
    }
    if (iterations)
        *iterations = iters;

done:
    free(pts);
    free(nextp);
    free(start_at);
    free(end_at);
    free(F.f);
    free(queue);
    free(visible);
    free(pending);
    free(par);
    return rc;
}
