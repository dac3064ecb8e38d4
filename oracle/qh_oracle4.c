/*
 * Oracle for the 4D hull (the paper's extension of Quickhull to higher
 * dimensions, Section 4.3, "3D and Higher Dimensions").  TEST
 * INFRASTRUCTURE ONLY, like qh_oracle.c: the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it; the product path never does.  It
 * shares no code with the CUDA path (nor with qh_oracle.c: the few exact
 * arithmetic helpers are written out again here).
 *
 * What it computes is the plain definition of the result for float32 points
 * in R^4 read exactly as reals:
 *   vertices  the extreme points, as sorted input indices (a location
 *             present several times is reported as its lowest index);
 *   facets    every facet of the convex hull (a maximal set of boundary
 *             points on one supporting hyperplane) as the sorted list of the
 *             extreme points on it, the facets sorted lexicographically.
 * For points in general position every facet is a tetrahedron (4 vertices).
 *
 * It gets there by a sequential Quickhull in Barber et al.'s form (the one
 * the paper builds on): a first simplex from extreme points, then for each
 * facet with outside points its farthest point, the facets it sees
 * (breadth-first from that facet), the horizon ridges (triangles), one new
 * facet per horizon ridge through the apex, and the reassignment of the
 * visible facets' points to the first new facet they are strictly above.
 * The final simplicial complex is then reduced to the definition above:
 * neighbouring simplices on one hyperplane are merged (union-find), and a
 * vertex v of the complex is kept exactly when no other vertex of the
 * simplices around v lies on every hyperplane through v (such a w exists
 * exactly when those hyperplanes meet in a line or more through v, i.e.
 * when v lies inside an edge, a 2-face or a facet).
 *
 * Predicates are exact.  orient4(a, b, c, d, p) = det[b-a; c-a; d-a; p-a]
 * (positive: p on the outer side of the facet a, b, c, d) is evaluated in
 * FP64 through the 2x2 minors of its first two and last two rows, with a
 * forward error bound; when the bound cannot decide, the determinant is
 * expanded into products of four float32 coordinates, each exact as a
 * four-term expansion (two-product), and the sign of their exact sum is
 * read from a non-overlapping expansion (Shewchuk 1997).
 *
 * Build with -ffp-contract=off: the error bound assumes separately rounded
 * products and sums.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define O4_OK 0
#define O4_ERR_INVALID 1
#define O4_ERR_NONFINITE 2
#define O4_ERR_DEGENERATE 3
#define O4_ERR_NOMEM 4

static const double EPS4 = 1.1102230246251565e-16; /* 2^-53 */

/* ------------------------------------------------------------------------ */
/* Exact arithmetic (Shewchuk's two-sum, two-product, grow-expansion)         */
/* ------------------------------------------------------------------------ */

static void t_sum(double a, double b, double *s, double *e)
{
    double x = a + b;
    double bv = x - a;
    double av = x - bv;
    *s = x;
    *e = (a - av) + (b - bv);
}

static void t_prod(double a, double b, double *p, double *e)
{
    double x = a * b;
    *p = x;
    *e = fma(a, b, -x);
}

/* Exact sign of the sum of m doubles (expansion grown term by term; zero
 * components dropped, so its length never exceeds the terms added). */
static int sign_of_sum(const double *t, int m)
{
    double *e = (double *)malloc(sizeof(double) * (size_t)(m + 1));
    if (!e)
        abort();
    int len = 0;
    for (int i = 0; i < m; i++) {
        double q = t[i];
        int out = 0;
        for (int j = 0; j < len; j++) {
            double s, err;
            t_sum(q, e[j], &s, &err);
            q = s;
            if (err != 0.0)
                e[out++] = err;
        }
        if (q != 0.0 || out == 0)
            e[out++] = q;
        len = out;
    }
    double top = e[len - 1];
    free(e);
    return (top > 0.0) - (top < 0.0);
}

/* Append the 96 doubles whose exact sum is s * det[x; y; z; w] (rows of
 * float32 values held in doubles): 24 signed products, each x_i y_j (exact)
 * times z_k (two-product: exact as two doubles) times w_l (two more
 * two-products: four doubles). */
static int det4_terms(const double *x, const double *y, const double *z, const double *w, double s,
                      double *out)
{
    int m = 0;
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) {
            if (j == i)
                continue;
            for (int k = 0; k < 4; k++) {
                if (k == i || k == j)
                    continue;
                int l = 6 - i - j - k;
                /* sign of the permutation (i, j, k, l): count inversions */
                int inv = (i > j) + (i > k) + (i > l) + (j > k) + (j > l) + (k > l);
                double sg = (inv & 1) ? -s : s;
                double xy = x[i] * y[j];
                double h, lo;
                t_prod(xy, z[k], &h, &lo);
                double h1, l1, h2, l2;
                t_prod(h, w[l], &h1, &l1);
                t_prod(lo, w[l], &h2, &l2);
                out[m++] = sg * h1;
                out[m++] = sg * l1;
                out[m++] = sg * h2;
                out[m++] = sg * l2;
            }
        }
    return m;
}

/* Sign of det[r0; r1; r2; r3] for rows of rounded FP64 differences, by the
 * 2x2 minors of rows 0-1 and rows 2-3 (Laplace); every monomial passes
 * through at most 12 roundings (4 differences, 2 products and a difference
 * per minor, the product of the minors, 3 levels of sums), so |det - D| <=
 * (12 eps + O(eps^2)) * permanent.  Returns 2 when the bound cannot decide. */
static int det4_filter(const double *r0, const double *r1, const double *r2, const double *r3)
{
    static const int C[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
    /* complement of pair q is pair 5 - q; sign of the split (Laplace) */
    static const double SG[6] = {1, -1, 1, 1, -1, 1};
    double t[6], perm = 0.0;
    for (int q = 0; q < 6; q++) {
        int i = C[q][0], j = C[q][1];
        int k = C[5 - q][0], l = C[5 - q][1];
        double a1 = r0[i] * r1[j], a2 = r0[j] * r1[i];
        double b1 = r2[k] * r3[l], b2 = r2[l] * r3[k];
        t[q] = SG[q] * ((a1 - a2) * (b1 - b2));
        perm += (fabs(a1) + fabs(a2)) * (fabs(b1) + fabs(b2));
    }
    double det = ((t[0] + t[1]) + (t[2] + t[3])) + (t[4] + t[5]);
    double bound = (12.0 + 256.0 * EPS4) * EPS4 * perm;
    if (det > bound)
        return 1;
    if (-det > bound)
        return -1;
    return 2;
}

/* orient4(a, b, c, d, p) = sign det[b-a; c-a; d-a; p-a]. */
static int orient4(const double *a, const double *b, const double *c, const double *d,
                   const double *p)
{
    double r0[4], r1[4], r2[4], r3[4];
    for (int i = 0; i < 4; i++) {
        r0[i] = b[i] - a[i];
        r1[i] = c[i] - a[i];
        r2[i] = d[i] - a[i];
        r3[i] = p[i] - a[i];
    }
    int s = det4_filter(r0, r1, r2, r3);
    if (s != 2)
        return s;
    /* multilinear in the rows: the four a-rows expand into five determinants
     * of raw points (terms with a twice vanish) */
    double *t = (double *)malloc(sizeof(double) * 5 * 96);
    if (!t)
        abort();
    int m = 0;
    m += det4_terms(b, c, d, p, 1.0, t + m);
    m += det4_terms(a, c, d, p, -1.0, t + m);
    m += det4_terms(b, a, d, p, -1.0, t + m);
    m += det4_terms(b, c, a, p, -1.0, t + m);
    m += det4_terms(b, c, d, a, -1.0, t + m);
    s = sign_of_sum(t, m);
    free(t);
    return s;
}

/* sign(orient4 value at p1 - value at p2) = sign det[b-a; c-a; d-a; p1-p2]. */
static int cmp_dist4(const double *a, const double *b, const double *c, const double *d,
                     const double *p1, const double *p2)
{
    double r0[4], r1[4], r2[4], r3[4];
    for (int i = 0; i < 4; i++) {
        r0[i] = b[i] - a[i];
        r1[i] = c[i] - a[i];
        r2[i] = d[i] - a[i];
        r3[i] = p1[i] - p2[i];
    }
    int s = det4_filter(r0, r1, r2, r3);
    if (s != 2)
        return s;
    /* det[b-a; c-a; d-a; x] = det[b;c;d;x] - det[a;c;d;x] - det[b;a;d;x]
     * - det[b;c;a;x], linear in x */
    double *t = (double *)malloc(sizeof(double) * 8 * 96);
    if (!t)
        abort();
    int m = 0;
    m += det4_terms(b, c, d, p1, 1.0, t + m);
    m += det4_terms(a, c, d, p1, -1.0, t + m);
    m += det4_terms(b, a, d, p1, -1.0, t + m);
    m += det4_terms(b, c, a, p1, -1.0, t + m);
    m += det4_terms(b, c, d, p2, -1.0, t + m);
    m += det4_terms(a, c, d, p2, 1.0, t + m);
    m += det4_terms(b, a, d, p2, 1.0, t + m);
    m += det4_terms(b, c, a, p2, 1.0, t + m);
    s = sign_of_sum(t, m);
    free(t);
    return s;
}

/* Exact sign of det[b-a; c-a; p-a] restricted to coordinates (i, j, k):
 * the 3D orientation of the projections. */
static int orient3_proj(const double *a, const double *b, const double *c, const double *p, int i,
                        int j, int k)
{
    /* det of 3x3 rows of raw projected points via the same expansion idea:
     * det[b-a; c-a; p-a] = det[b;c;p] - det[a;c;p] - det[b;a;p] - det[b;c;a];
     * each 3x3 determinant's 6 products of three float32 values are exact as
     * two doubles */
    const double *R[4][3] = {{b, c, p}, {a, c, p}, {b, a, p}, {b, c, a}};
    const double S[4] = {1, -1, -1, -1};
    const int I[3] = {i, j, k};
    double t[48];
    int m = 0;
    for (int q = 0; q < 4; q++)
        for (int s0 = 0; s0 < 3; s0++)
            for (int s1 = 0; s1 < 3; s1++) {
                if (s1 == s0)
                    continue;
                int s2 = 3 - s0 - s1;
                int inv = (s0 > s1) + (s0 > s2) + (s1 > s2);
                double sg = (inv & 1) ? -S[q] : S[q];
                double xy = R[q][0][I[s0]] * R[q][1][I[s1]];
                double h, lo;
                t_prod(xy, R[q][2][I[s2]], &h, &lo);
                t[m++] = sg * h;
                t[m++] = sg * lo;
            }
    return sign_of_sum(t, m);
}

/* p on the line ab (exactly): every 2x2 minor of [b-a; p-a] vanishes. */
static int on_line4(const double *a, const double *b, const double *p)
{
    for (int i = 0; i < 4; i++)
        for (int j = i + 1; j < 4; j++) {
            /* (b_i - a_i)(p_j - a_j) - (b_j - a_j)(p_i - a_i): monomials */
            double t[8] = {b[i] * p[j], -b[i] * a[j], -a[i] * p[j], a[i] * a[j],
                           -b[j] * p[i], b[j] * a[i], a[j] * p[i], -a[j] * a[i]};
            if (sign_of_sum(t, 8) != 0)
                return 0;
        }
    return 1;
}

/* p in the plane abc (exactly): every 3x3 minor of [b-a; c-a; p-a] vanishes. */
static int on_plane4(const double *a, const double *b, const double *c, const double *p)
{
    static const int T[4][3] = {{0, 1, 2}, {0, 1, 3}, {0, 2, 3}, {1, 2, 3}};
    for (int q = 0; q < 4; q++)
        if (orient3_proj(a, b, c, p, T[q][0], T[q][1], T[q][2]) != 0)
            return 0;
    return 1;
}

/* Exported for the predicate pins (points as 4 doubles holding float32 values). */
int oracle_orient4(const double *a, const double *b, const double *c, const double *d,
                   const double *p)
{
    return orient4(a, b, c, d, p);
}
int oracle_cmp_dist4(const double *a, const double *b, const double *c, const double *d,
                     const double *p1, const double *p2)
{
    return cmp_dist4(a, b, c, d, p1, p2);
}

/* ------------------------------------------------------------------------ */
/* 4D Quickhull                                                              */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t v[4];  /* orient4(v0, v1, v2, v3, x) > 0: x strictly outside */
    int32_t nb[4]; /* nb[k]: facet across the ridge opposite v[k] */
    int32_t head;  /* first point of the outside set, -1 if empty */
    int32_t alive;
    int32_t mark;
} facet4;

typedef struct {
    facet4 *f;
    int64_t nf, cap;
} facets4;

static int64_t push4(facets4 *F, const int32_t *v)
{
    if (F->nf == F->cap) {
        int64_t cap = F->cap ? 2 * F->cap : 64;
        facet4 *nf = (facet4 *)realloc(F->f, sizeof(facet4) * (size_t)cap);
        if (!nf)
            return -1;
        F->f = nf;
        F->cap = cap;
    }
    facet4 *t = &F->f[F->nf];
    for (int i = 0; i < 4; i++) {
        t->v[i] = v[i];
        t->nb[i] = -1;
    }
    t->head = -1;
    t->alive = 1;
    t->mark = 0;
    return F->nf++;
}

#define P4(i) (pts + 4 * (int64_t)(i))

static int side4(const double *pts, const facet4 *f, int32_t p)
{
    return orient4(P4(f->v[0]), P4(f->v[1]), P4(f->v[2]), P4(f->v[3]), P4(p));
}

static int lex4(const double *p, const double *q)
{
    for (int i = 0; i < 4; i++) {
        if (p[i] < q[i])
            return -1;
        if (p[i] > q[i])
            return 1;
    }
    return 0;
}

static int32_t uf4(int32_t *par, int32_t x)
{
    while (par[x] != x) {
        par[x] = par[par[x]];
        x = par[x];
    }
    return x;
}

static int i32cmp(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

static int i64cmp(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

typedef struct {
    int32_t *idx;
    int32_t len;
} list4;

static int list_cmp(const void *pa, const void *pb)
{
    const list4 *A = (const list4 *)pa, *B = (const list4 *)pb;
    int m = A->len < B->len ? A->len : B->len;
    for (int i = 0; i < m; i++)
        if (A->idx[i] != B->idx[i])
            return A->idx[i] < B->idx[i] ? -1 : 1;
    return (A->len > B->len) - (A->len < B->len);
}

/* Link new facets lo..hi-1 (each = a horizon ridge plus the apex q) across
 * their ridges through q: the ridge of facet f opposite vertex v[j] (j not
 * the apex slot) holds q and two ridge vertices, shared with exactly one
 * other new facet. */
static void link_new(facets4 *F, int64_t lo, int64_t hi, int32_t q)
{
    for (int64_t f = lo; f < hi; f++) {
        for (int j = 0; j < 4; j++) {
            if (F->f[f].v[j] == q || F->f[f].nb[j] >= 0)
                continue;
            /* the two non-apex vertices of this ridge */
            int32_t e[2], m = 0;
            for (int i = 0; i < 4; i++)
                if (i != j && F->f[f].v[i] != q)
                    e[m++] = F->f[f].v[i];
            for (int64_t g = lo; g < hi && F->f[f].nb[j] < 0; g++) {
                if (g == f)
                    continue;
                int has0 = 0, has1 = 0, jj = -1;
                for (int i = 0; i < 4; i++) {
                    int32_t x = F->f[g].v[i];
                    if (x == e[0])
                        has0 = 1;
                    else if (x == e[1])
                        has1 = 1;
                    else if (x != q)
                        jj = i;
                }
                if (has0 && has1 && jj >= 0) {
                    F->f[f].nb[j] = (int32_t)g;
                    F->f[g].nb[jj] = (int32_t)f;
                }
            }
        }
    }
}

/*
 * Outputs: verts (sorted extreme point indices, capacity n), facet_off
 * (nfacets + 1 entries) and facet_idx (CSR lists, sorted lexicographically);
 * capacities: facet_off >= fcap + 1, facet_idx >= icap (O4_ERR_NOMEM when
 * they do not suffice).  Returns O4_ERR_DEGENERATE when the points do not
 * span R^4 (n in 1..4 included).
 */
int oracle_hull4d(const float *x, const float *y, const float *z, const float *w, int64_t n,
                  int32_t *verts, int64_t *nv_out, int32_t *facet_off, int64_t fcap,
                  int32_t *facet_idx, int64_t icap, int64_t *nf_out, int64_t *iterations)
{
    *nv_out = 0;
    *nf_out = 0;
    if (iterations)
        *iterations = 0;
    if (n < 0 || fcap < 0 || icap < 0)
        return O4_ERR_INVALID;
    if (n == 0) {
        if (fcap >= 0)
            facet_off[0] = 0;
        return O4_OK;
    }
    for (int64_t i = 0; i < n; i++)
        if (!isfinite(x[i]) || !isfinite(y[i]) || !isfinite(z[i]) || !isfinite(w[i]))
            return O4_ERR_NONFINITE;
    if (n < 5)
        return O4_ERR_DEGENERATE;

    int rc = O4_OK;
    double *pts = (double *)malloc(sizeof(double) * 4 * (size_t)n);
    int32_t *nextp = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    facets4 F = {0, 0, 0};
    int32_t *queue = NULL, *vis = NULL, *cand = NULL, *par = NULL;
    int32_t *star_off = NULL, *star = NULL, *ext = NULL, *glist = NULL;
    list4 *lists = NULL;
    int64_t qcap = 1024, qh = 0, qt = 0, vcap = 1024, ccap = 1024;
    if (!pts || !nextp) {
        rc = O4_ERR_NOMEM;
        goto done;
    }
    for (int64_t i = 0; i < n; i++) {
        /* + 0.0 maps -0.0 to +0.0 (the same location) */
        pts[4 * i] = (double)x[i] + 0.0;
        pts[4 * i + 1] = (double)y[i] + 0.0;
        pts[4 * i + 2] = (double)z[i] + 0.0;
        pts[4 * i + 3] = (double)w[i] + 0.0;
    }

    /* ---- first simplex: lexicographic extrema a, b; c farthest from the
     * line ab; d farthest from the plane abc; e farthest from the hyperplane
     * abcd (FP64 magnitudes choose, exact tests confirm; an exact search
     * replaces a choice that is degenerate) */
    int32_t s[5];
    s[0] = s[1] = 0;
    for (int64_t i = 1; i < n; i++) {
        if (lex4(P4(i), P4(s[0])) < 0)
            s[0] = (int32_t)i;
        if (lex4(P4(i), P4(s[1])) > 0)
            s[1] = (int32_t)i;
    }
    if (lex4(P4(s[0]), P4(s[1])) == 0) {
        rc = O4_ERR_DEGENERATE;
        goto done;
    }
    for (int step = 2; step <= 4; step++) {
        /* orthonormal basis of the current affine span (Gram-Schmidt) */
        double B[3][4];
        int nb = step - 1;
        for (int k = 0; k < nb; k++) {
            for (int i = 0; i < 4; i++)
                B[k][i] = P4(s[k + 1])[i] - P4(s[0])[i];
            for (int r = 0; r < k; r++) {
                double dp = 0;
                for (int i = 0; i < 4; i++)
                    dp += B[k][i] * B[r][i];
                for (int i = 0; i < 4; i++)
                    B[k][i] -= dp * B[r][i];
            }
            double nr = 0;
            for (int i = 0; i < 4; i++)
                nr += B[k][i] * B[k][i];
            nr = sqrt(nr);
            for (int i = 0; i < 4; i++)
                B[k][i] = nr > 0 ? B[k][i] / nr : 0.0;
        }
        int32_t best = -1;
        double bd = -1.0;
        for (int64_t i = 0; i < n; i++) {
            double r[4];
            for (int k = 0; k < 4; k++)
                r[k] = P4(i)[k] - P4(s[0])[k];
            for (int k = 0; k < nb; k++) {
                double dp = 0;
                for (int q = 0; q < 4; q++)
                    dp += r[q] * B[k][q];
                for (int q = 0; q < 4; q++)
                    r[q] -= dp * B[k][q];
            }
            double dd = r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + r[3] * r[3];
            if (dd > bd) {
                bd = dd;
                best = (int32_t)i;
            }
        }
        int ok = 0;
        for (int pass = 0; pass < 2 && !ok; pass++) {
            for (int64_t i = (pass == 0 ? best : 0); i < n; i++) {
                const double *p = P4(i);
                int off;
                if (step == 2)
                    off = !on_line4(P4(s[0]), P4(s[1]), p);
                else if (step == 3)
                    off = !on_plane4(P4(s[0]), P4(s[1]), P4(s[2]), p);
                else
                    off = orient4(P4(s[0]), P4(s[1]), P4(s[2]), P4(s[3]), p) != 0;
                if (off) {
                    s[step] = (int32_t)i;
                    ok = 1;
                    break;
                }
                if (pass == 0)
                    break;
            }
        }
        if (!ok) {
            rc = O4_ERR_DEGENERATE;
            goto done;
        }
    }
    /* five facets, each the simplex minus one point, the missing point inside */
    for (int o = 0; o < 5; o++) {
        int32_t v[4], k = 0;
        for (int j = 0; j < 5; j++)
            if (j != o)
                v[k++] = s[j];
        if (orient4(P4(v[0]), P4(v[1]), P4(v[2]), P4(v[3]), P4(s[o])) > 0) {
            int32_t t = v[0];
            v[0] = v[1];
            v[1] = t;
        }
        if (push4(&F, v) < 0) {
            rc = O4_ERR_NOMEM;
            goto done;
        }
    }
    /* neighbours: facet i's ridge opposite v[k] is shared with the other
     * facet holding those three points */
    for (int i = 0; i < 5; i++)
        for (int k = 0; k < 4; k++)
            for (int j = 0; j < 5; j++) {
                if (j == i)
                    continue;
                int shared = 0;
                for (int a = 0; a < 4; a++) {
                    if (a == k)
                        continue;
                    for (int b = 0; b < 4; b++)
                        shared += F.f[i].v[a] == F.f[j].v[b];
                }
                if (shared == 3)
                    F.f[i].nb[k] = j;
            }
    /* outside sets: each point to the first facet it is strictly above */
    for (int64_t i = n - 1; i >= 0; i--)
        for (int k = 0; k < 5; k++)
            if (side4(pts, &F.f[k], (int32_t)i) > 0) {
                nextp[i] = F.f[k].head;
                F.f[k].head = (int32_t)i;
                break;
            }

    queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)qcap);
    vis = (int32_t *)malloc(sizeof(int32_t) * (size_t)vcap);
    cand = (int32_t *)malloc(sizeof(int32_t) * (size_t)ccap);
    if (!queue || !vis || !cand) {
        rc = O4_ERR_NOMEM;
        goto done;
    }
    for (int k = 0; k < 5; k++)
        queue[qt++] = k;

    int32_t stamp = 0;
    int64_t iters = 0;
    while (qh < qt) {
        int32_t fi = queue[qh++];
        if (qh > 4096 && qh * 2 > qt) {
            memmove(queue, queue + qh, sizeof(int32_t) * (size_t)(qt - qh));
            qt -= qh;
            qh = 0;
        }
        if (!F.f[fi].alive || F.f[fi].head < 0)
            continue;
        iters++;
        /* the outside set's farthest point (lowest index on exact ties) */
        const facet4 *f0 = &F.f[fi];
        int32_t q = f0->head;
        for (int32_t p = nextp[q]; p >= 0; p = nextp[p]) {
            int c = cmp_dist4(P4(f0->v[0]), P4(f0->v[1]), P4(f0->v[2]), P4(f0->v[3]), P4(p), P4(q));
            if (c > 0 || (c == 0 && p < q))
                q = p;
        }
        /* visible set: the facets q is strictly above, connected to fi */
        stamp++;
        int64_t nvis = 0;
        vis[nvis++] = fi;
        F.f[fi].mark = stamp;
        for (int64_t k = 0; k < nvis; k++) {
            for (int e = 0; e < 4; e++) {
                int32_t h = F.f[vis[k]].nb[e];
                if (F.f[h].mark == stamp || F.f[h].mark == -stamp)
                    continue;
                if (side4(pts, &F.f[h], q) > 0) {
                    F.f[h].mark = stamp;
                    if (nvis == vcap) {
                        vcap *= 2;
                        int32_t *nv = (int32_t *)realloc(vis, sizeof(int32_t) * (size_t)vcap);
                        if (!nv) {
                            rc = O4_ERR_NOMEM;
                            goto done;
                        }
                        vis = nv;
                    }
                    vis[nvis++] = h;
                } else {
                    F.f[h].mark = -stamp;
                }
            }
        }
        /* horizon ridges -> new facets (the visible facet with the ridge's
         * opposite vertex replaced by q keeps the outward orientation) */
        int64_t first_new = F.nf;
        for (int64_t k = 0; k < nvis; k++) {
            int32_t gi = vis[k];
            for (int e = 0; e < 4; e++) {
                int32_t h = F.f[gi].nb[e];
                if (F.f[h].mark == stamp)
                    continue;
                int32_t v[4];
                memcpy(v, F.f[gi].v, sizeof(v));
                v[e] = q;
                int64_t nf = push4(&F, v);
                if (nf < 0) {
                    rc = O4_ERR_NOMEM;
                    goto done;
                }
                F.f[nf].nb[e] = h;
                for (int t = 0; t < 4; t++)
                    if (F.f[h].nb[t] == gi)
                        F.f[h].nb[t] = (int32_t)nf;
            }
        }
        link_new(&F, first_new, F.nf, q);
        /* the visible facets' points: to the first new facet strictly below
         * them, else inside */
        int64_t ncand = 0;
        for (int64_t k = 0; k < nvis; k++) {
            facet4 *g = &F.f[vis[k]];
            g->alive = 0;
            for (int32_t p = g->head; p >= 0; p = nextp[p]) {
                if (ncand == ccap) {
                    ccap *= 2;
                    int32_t *nc = (int32_t *)realloc(cand, sizeof(int32_t) * (size_t)ccap);
                    if (!nc) {
                        rc = O4_ERR_NOMEM;
                        goto done;
                    }
                    cand = nc;
                }
                cand[ncand++] = p;
            }
            g->head = -1;
        }
        /* keep input order inside each new outside set (descending pushes) */
        qsort(cand, (size_t)ncand, sizeof(int32_t), i32cmp);
        for (int64_t k = ncand - 1; k >= 0; k--) {
            int32_t p = cand[k];
            if (p == q)
                continue;
            for (int64_t nf = first_new; nf < F.nf; nf++)
                if (side4(pts, &F.f[nf], p) > 0) {
                    nextp[p] = F.f[nf].head;
                    F.f[nf].head = p;
                    break;
                }
        }
        for (int64_t nf = first_new; nf < F.nf; nf++) {
            if (F.f[nf].head < 0)
                continue;
            if (qt == qcap) {
                qcap *= 2;
                int32_t *nq = (int32_t *)realloc(queue, sizeof(int32_t) * (size_t)qcap);
                if (!nq) {
                    rc = O4_ERR_NOMEM;
                    goto done;
                }
                queue = nq;
            }
            queue[qt++] = (int32_t)nf;
        }
    }
    if (iterations)
        *iterations = iters;

    /* ---- canonical output.  Simplices on one hyperplane are merged: a
     * neighbour is on the facet's hyperplane when its vertex opposite the
     * shared ridge is. */
    par = (int32_t *)malloc(sizeof(int32_t) * (size_t)F.nf);
    if (!par) {
        rc = O4_ERR_NOMEM;
        goto done;
    }
    for (int64_t f = 0; f < F.nf; f++)
        par[f] = (int32_t)f;
    for (int64_t f = 0; f < F.nf; f++) {
        if (!F.f[f].alive)
            continue;
        for (int k = 0; k < 4; k++) {
            const facet4 *g = &F.f[F.f[f].nb[k]];
            int32_t opp = -1;
            for (int t = 0; t < 4; t++) {
                int in = 0;
                for (int u = 0; u < 4; u++)
                    in |= g->v[t] == F.f[f].v[u];
                if (!in)
                    opp = g->v[t];
            }
            if (opp >= 0 && side4(pts, &F.f[f], opp) == 0) {
                int32_t a = uf4(par, (int32_t)f), b = uf4(par, F.f[f].nb[k]);
                if (a != b)
                    par[a > b ? a : b] = a < b ? a : b;
            }
        }
    }
    /* the star of every vertex of the complex: the simplices holding it */
    star_off = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    if (!star_off) {
        rc = O4_ERR_NOMEM;
        goto done;
    }
    int64_t nalive = 0;
    for (int64_t f = 0; f < F.nf; f++)
        if (F.f[f].alive) {
            nalive++;
            for (int k = 0; k < 4; k++)
                star_off[F.f[f].v[k] + 1]++;
        }
    for (int64_t i = 0; i < n; i++)
        star_off[i + 1] += star_off[i];
    star = (int32_t *)malloc(sizeof(int32_t) * (size_t)(4 * nalive + 1));
    int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!star || !fill) {
        free(fill);
        rc = O4_ERR_NOMEM;
        goto done;
    }
    memcpy(fill, star_off, sizeof(int32_t) * (size_t)n);
    for (int64_t f = 0; f < F.nf; f++)
        if (F.f[f].alive)
            for (int k = 0; k < 4; k++)
                star[fill[F.f[f].v[k]]++] = (int32_t)f;
    free(fill);
    /* extreme: no other vertex of the star lies on every hyperplane of the star */
    ext = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    if (!ext) {
        rc = O4_ERR_NOMEM;
        goto done;
    }
    for (int64_t v = 0; v < n; v++) {
        int32_t s0 = star_off[v], s1 = star_off[v + 1];
        if (s0 == s1)
            continue;
        int extreme = 1;
        for (int32_t a = s0; a < s1 && extreme; a++)
            for (int k = 0; k < 4 && extreme; k++) {
                int32_t wv = F.f[star[a]].v[k];
                if (wv == v)
                    continue;
                int on_all = 1;
                for (int32_t b = s0; b < s1 && on_all; b++)
                    on_all = side4(pts, &F.f[star[b]], wv) == 0;
                if (on_all)
                    extreme = 0;
            }
        ext[v] = extreme;
    }
    int64_t nv = 0;
    for (int64_t v = 0; v < n; v++)
        if (ext[v])
            verts[nv++] = (int32_t)v;
    /* facets: per merged group, the sorted extreme vertices on it */
    int64_t ngroups = 0;
    for (int64_t f = 0; f < F.nf; f++)
        if (F.f[f].alive && uf4(par, (int32_t)f) == f)
            ngroups++;
    if (ngroups + 1 > fcap) {
        rc = O4_ERR_NOMEM;
        goto done;
    }
    /* group members: sort alive facets by root */
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nalive + 1));
    glist = (int32_t *)malloc(sizeof(int32_t) * (size_t)(4 * nalive + 1));
    lists = (list4 *)malloc(sizeof(list4) * (size_t)(ngroups + 1));
    if (!order || !glist || !lists) {
        free(order);
        rc = O4_ERR_NOMEM;
        goto done;
    }
    {
        int64_t m = 0;
        for (int64_t f = 0; f < F.nf; f++)
            if (F.f[f].alive)
                order[m++] = ((int64_t)uf4(par, (int32_t)f) << 32) | f;
        qsort(order, (size_t)m, sizeof(int64_t), i64cmp); /* by root, then facet */
        int64_t g = 0, pos = 0;
        for (int64_t i = 0; i < m;) {
            int64_t j = i;
            int32_t root = (int32_t)(order[i] >> 32);
            int32_t st = (int32_t)pos;
            while (j < m && (int32_t)(order[j] >> 32) == root) {
                int32_t f = (int32_t)(order[j] & 0xffffffff);
                for (int k = 0; k < 4; k++)
                    if (ext[F.f[f].v[k]])
                        glist[pos++] = F.f[f].v[k];
                j++;
            }
            qsort(glist + st, (size_t)(pos - st), sizeof(int32_t), i32cmp);
            int32_t u = st;
            for (int32_t t = st; t < pos; t++)
                if (t == st || glist[t] != glist[t - 1])
                    glist[u++] = glist[t];
            pos = u;
            lists[g].idx = glist + st;
            lists[g].len = (int32_t)(pos - st);
            g++;
            i = j;
        }
        qsort(lists, (size_t)g, sizeof(list4), list_cmp);
        int64_t tot = 0;
        for (int64_t i = 0; i < g; i++)
            tot += lists[i].len;
        if (tot > icap) {
            free(order);
            rc = O4_ERR_NOMEM;
            goto done;
        }
        /* copy out (lists point into glist; copy through a temporary) */
        int64_t o = 0;
        int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(tot + 1));
        if (!tmp) {
            free(order);
            rc = O4_ERR_NOMEM;
            goto done;
        }
        for (int64_t i = 0; i < g; i++) {
            facet_off[i] = (int32_t)o;
            memcpy(tmp + o, lists[i].idx, sizeof(int32_t) * (size_t)lists[i].len);
            o += lists[i].len;
        }
        facet_off[g] = (int32_t)o;
        memcpy(facet_idx, tmp, sizeof(int32_t) * (size_t)o);
        free(tmp);
        *nf_out = g;
    }
    free(order);
    *nv_out = nv;

done:
    free(pts);
    free(nextp);
    free(F.f);
    free(queue);
    free(vis);
    free(cand);
    free(par);
    free(star_off);
    free(star);
    free(ext);
    free(glist);
    free(lists);
    return rc;
}
