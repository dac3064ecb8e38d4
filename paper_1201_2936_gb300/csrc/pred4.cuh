// Exact 4D predicates for the device path.
//
// orient4(a, b, c, d, p) = det[b-a; c-a; d-a; p-a] is positive when p lies
// on the outer side of the facet (a, b, c, d).  Signs go through
//   1. FP32 from the facet's cofactors (computed once per facet) with a
//      forward error bound,
//   2. FP64 with its bound,
//   3. exact: the determinant is multilinear in its rows, so the a-terms
//      expand it into five determinants of raw float32 points, each a signed
//      sum of 24 products of four coordinates.  x*y is exact in FP64, times z
//      exact as two doubles (two-product), times w exact as four; the sign
//      of the exact sum is read from a non-overlapping expansion grown term
//      by term with zero elimination (Shewchuk 1997).  Components of such an
//      expansion occupy disjoint bit ranges of the FP64 exponent range, so
//      its length stays small (tens) however many terms are added.
//
// Bound of stages 1 and 2.  With u, v, w the rounded rows b-a, c-a, d-a and
// t = p - a, D = (t0 C0 + t1 C1) + (t2 C2 + t3 C3) where C_i is the signed
// 3x3 minor of (u, v, w) without column i, each evaluated like det3_f32.
// Every monomial u_j v_k w_l t_i passes through at most twelve roundings
// (four differences, the product and difference inside a 2x2 minor, the
// product with the first row and two sums inside the 3x3 minor, the product
// with t_i, two sums), so |det - D| <= (12 eps + O(eps^2)) perm with perm =
// sum_i |t_i| M_i, M_i the permanent of minor i.  The code uses
// 12 eps (1 + 2^-10) perm.  FP32 products of four factors may underflow: the
// FP32 stage only decides when every non-zero difference is at least 2^-30
// (products then stay above 2^-120, and the absolute error of an underflowed
// sum stays far below the bound); a non-finite value never decides.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "pred2.cuh"
#include "pred3.cuh"

namespace qh {

constexpr float kC32_4 = 0x1.808p-21f;  // 12 * 2^-24 * (1 + 2^-10), rounded up
constexpr double kC64_4 = 0x1.808p-50;  // 12 * 2^-53 * (1 + 2^-10), rounded up
constexpr float kTiny4 = 0x1p-30f;

// A facet's filter data: base point a, cofactors n_i (D = t . n) and minor
// permanents m_i; f.x = 1 marks a facet with a non-zero component of u, v or
// w below 2^-30 (the FP32 stage never decides for it).
struct Plane4 {
    float4 a, n, m, f;
};

// det of the 3x3 matrix [r0; r1; r2] (rows of 3) and its permanent, FP32.
__device__ __forceinline__ void det3p_f32(const float *r0, const float *r1, const float *r2,
                                          float &d, float &p)
{
    const float m0a = __fmul_rn(r1[1], r2[2]), m0b = __fmul_rn(r1[2], r2[1]);
    const float m1a = __fmul_rn(r1[2], r2[0]), m1b = __fmul_rn(r1[0], r2[2]);
    const float m2a = __fmul_rn(r1[0], r2[1]), m2b = __fmul_rn(r1[1], r2[0]);
    d = __fadd_rn(__fadd_rn(__fmul_rn(r0[0], __fsub_rn(m0a, m0b)),
                            __fmul_rn(r0[1], __fsub_rn(m1a, m1b))),
                  __fmul_rn(r0[2], __fsub_rn(m2a, m2b)));
    p = __fadd_rn(__fadd_rn(__fmul_rn(fabsf(r0[0]), __fadd_rn(fabsf(m0a), fabsf(m0b))),
                            __fmul_rn(fabsf(r0[1]), __fadd_rn(fabsf(m1a), fabsf(m1b)))),
                  __fmul_rn(fabsf(r0[2]), __fadd_rn(fabsf(m2a), fabsf(m2b))));
}

__device__ __forceinline__ Plane4 make_plane4(const float *a, const float *b, const float *c,
                                              const float *d)
{
    float u[4], v[4], w[4];
    bool never = false;
    for (int i = 0; i < 4; i++) {
        u[i] = __fsub_rn(b[i], a[i]);
        v[i] = __fsub_rn(c[i], a[i]);
        w[i] = __fsub_rn(d[i], a[i]);
        never |= (u[i] != 0.0f && fabsf(u[i]) < kTiny4) || (v[i] != 0.0f && fabsf(v[i]) < kTiny4) ||
                 (w[i] != 0.0f && fabsf(w[i]) < kTiny4);
    }
    float n[4], m[4];
    for (int i = 0; i < 4; i++) {
        float r0[3], r1[3], r2[3];
        int k = 0;
        for (int j = 0; j < 4; j++) {
            if (j == i) continue;
            r0[k] = u[j];
            r1[k] = v[j];
            r2[k] = w[j];
            k++;
        }
        float dd, pp;
        det3p_f32(r0, r1, r2, dd, pp);
        // cofactor of row 3 (t), column i: (-1)^(3 + i)
        n[i] = (i & 1) ? dd : -dd;
        m[i] = pp;
    }
    Plane4 P;
    P.a = make_float4(a[0], a[1], a[2], a[3]);
    P.n = make_float4(n[0], n[1], n[2], n[3]);
    P.m = make_float4(m[0], m[1], m[2], m[3]);
    P.f = make_float4(never ? 1.0f : 0.0f, 0.0f, 0.0f, 0.0f);
    return P;
}

// FP32 value of orient4 at p and its bound (e = +inf: cannot decide).
__device__ __forceinline__ void plane4_value(const Plane4 &P, float4 p, float &d, float &e)
{
    const float t0 = __fsub_rn(p.x, P.a.x), t1 = __fsub_rn(p.y, P.a.y);
    const float t2 = __fsub_rn(p.z, P.a.z), t3 = __fsub_rn(p.w, P.a.w);
    d = __fadd_rn(__fadd_rn(__fmul_rn(t0, P.n.x), __fmul_rn(t1, P.n.y)),
                  __fadd_rn(__fmul_rn(t2, P.n.z), __fmul_rn(t3, P.n.w)));
    const float perm = __fadd_rn(__fadd_rn(__fmul_rn(fabsf(t0), P.m.x), __fmul_rn(fabsf(t1), P.m.y)),
                                 __fadd_rn(__fmul_rn(fabsf(t2), P.m.z), __fmul_rn(fabsf(t3), P.m.w)));
    e = __fmul_rn(kC32_4, perm);
    auto small = [](float t) { return t != 0.0f && fabsf(t) < kTiny4; };
    if (P.f.x != 0.0f || small(t0) || small(t1) || small(t2) || small(t3) || !isfinite(e) ||
        !isfinite(d))
        e = INFINITY;
}

// det[r0; r1; r2; r3] in FP64 through the 2x2 minors of rows 0-1 and 2-3,
// with its bound.
__device__ __forceinline__ void det4_f64(const double *r0, const double *r1, const double *r2,
                                         const double *r3, double &d, double &e)
{
    const int C[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
    const double SG[6] = {1, -1, 1, 1, -1, 1};  // Laplace signs of the column pairs
    double t[6], perm = 0.0;
#pragma unroll
    for (int q = 0; q < 6; q++) {
        const int i = C[q][0], j = C[q][1], k = C[5 - q][0], l = C[5 - q][1];
        const double a1 = __dmul_rn(r0[i], r1[j]), a2 = __dmul_rn(r0[j], r1[i]);
        const double b1 = __dmul_rn(r2[k], r3[l]), b2 = __dmul_rn(r2[l], r3[k]);
        t[q] = SG[q] * __dmul_rn(__dsub_rn(a1, a2), __dsub_rn(b1, b2));
        perm += (fabs(a1) + fabs(a2)) * (fabs(b1) + fabs(b2));
    }
    d = __dadd_rn(__dadd_rn(__dadd_rn(t[0], t[1]), __dadd_rn(t[2], t[3])), __dadd_rn(t[4], t[5]));
    e = kC64_4 * perm * (1.0 + 0x1p-40);
}

// Expansion accumulator: the exact sum of the terms added so far, as a
// non-overlapping expansion in increasing magnitude.
constexpr int kExpan = 96;
struct Expan {
    double e[kExpan];
    int len;
};

__device__ __forceinline__ void fast_two_sum_d(double a, double b, double &s, double &err)
{
    s = __dadd_rn(a, b);  // |a| >= |b|
    err = __dsub_rn(b, __dsub_rn(s, a));
}

// Shewchuk's Compress: the same value as a strongly non-overlapping
// expansion, whose length is bounded by the exponent range in use (for
// products of four float32 values a few tens of components), so a full
// buffer always gets room back.
__device__ __noinline__ void expan_compress(Expan &x)
{
    double g[kExpan];
    int bottom = x.len - 1;
    double Q = x.e[x.len - 1];
    for (int i = x.len - 2; i >= 0; i--) {
        double s, q;
        fast_two_sum_d(Q, x.e[i], s, q);
        if (q != 0.0) {
            g[bottom--] = s;
            Q = q;
        } else {
            Q = s;
        }
    }
    g[bottom] = Q;
    int top = 0;
    for (int i = bottom + 1; i < x.len; i++) {
        double s, q;
        fast_two_sum_d(g[i], Q, s, q);
        Q = s;
        if (q != 0.0) x.e[top++] = q;
    }
    x.e[top++] = Q;
    x.len = top;
}

__device__ __forceinline__ void expan_add(Expan &x, double b)
{
    if (x.len == kExpan) expan_compress(x);
    double q = b;
    int out = 0;
    for (int j = 0; j < x.len; j++) {
        double s, err;
        two_sum_d(q, x.e[j], s, err);
        q = s;
        if (err != 0.0) x.e[out++] = err;
    }
    if (q != 0.0 || out == 0) x.e[out++] = q;
    x.len = out;
}
__device__ __forceinline__ int expan_sign(const Expan &x)
{
    const double t = x.e[x.len - 1];
    return (t > 0.0) - (t < 0.0);
}

// Adds s * det[x; y; z; w] (raw float32 rows) exactly.
__device__ __noinline__ void det4_add(Expan &E, const float *x, const float *y, const float *z,
                                      const float *w, double s)
{
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) {
            if (j == i) continue;
            for (int k = 0; k < 4; k++) {
                if (k == i || k == j) continue;
                const int l = 6 - i - j - k;
                const int inv = (i > j) + (i > k) + (i > l) + (j > k) + (j > l) + (k > l);
                const double sg = (inv & 1) ? -s : s;
                const double xy = (double)x[i] * (double)y[j];  // exact
                double h, lo, h1, l1, h2, l2;
                two_prod_d(xy, (double)z[k], h, lo);
                two_prod_d(h, (double)w[l], h1, l1);
                two_prod_d(lo, (double)w[l], h2, l2);
                expan_add(E, sg * h1);
                expan_add(E, sg * l1);
                expan_add(E, sg * h2);
                expan_add(E, sg * l2);
            }
        }
}

// Exact sign of orient4(a, b, c, d, p) behind the FP64 filter.
__device__ __noinline__ int orient4_slow(const float *a, const float *b, const float *c,
                                         const float *d, const float *p)
{
    double r0[4], r1[4], r2[4], r3[4];
    for (int i = 0; i < 4; i++) {
        r0[i] = (double)b[i] - (double)a[i];
        r1[i] = (double)c[i] - (double)a[i];
        r2[i] = (double)d[i] - (double)a[i];
        r3[i] = (double)p[i] - (double)a[i];
    }
    double v, e;
    det4_f64(r0, r1, r2, r3, v, e);
    if (v > e) return 1;
    if (-v > e) return -1;
    Expan E;
    E.len = 0;
    det4_add(E, b, c, d, p, 1.0);
    det4_add(E, a, c, d, p, -1.0);
    det4_add(E, b, a, d, p, -1.0);
    det4_add(E, b, c, a, p, -1.0);
    det4_add(E, b, c, d, a, -1.0);
    return expan_sign(E);
}

// Exact sign of orient4 at p1 minus orient4 at p2 = det[b-a; c-a; d-a; p1-p2].
__device__ __noinline__ int cmp_dist4_slow(const float *a, const float *b, const float *c,
                                           const float *d, const float *p1, const float *p2)
{
    double r0[4], r1[4], r2[4], r3[4];
    for (int i = 0; i < 4; i++) {
        r0[i] = (double)b[i] - (double)a[i];
        r1[i] = (double)c[i] - (double)a[i];
        r2[i] = (double)d[i] - (double)a[i];
        r3[i] = (double)p1[i] - (double)p2[i];
    }
    double v, e;
    det4_f64(r0, r1, r2, r3, v, e);
    if (v > e) return 1;
    if (-v > e) return -1;
    Expan E;
    E.len = 0;
    det4_add(E, b, c, d, p1, 1.0);
    det4_add(E, a, c, d, p1, -1.0);
    det4_add(E, b, a, d, p1, -1.0);
    det4_add(E, b, c, a, p1, -1.0);
    det4_add(E, b, c, d, p2, -1.0);
    det4_add(E, a, c, d, p2, 1.0);
    det4_add(E, b, a, d, p2, 1.0);
    det4_add(E, b, c, a, p2, 1.0);
    return expan_sign(E);
}

// p on the line ab, exactly: every 2x2 minor of [b-a; p-a] vanishes.
__device__ __noinline__ bool on_line4(const float *a, const float *b, const float *p)
{
    for (int i = 0; i < 4; i++)
        for (int j = i + 1; j < 4; j++)
            if (orient_exact_sign(a[i], a[j], b[i], b[j], p[i], p[j]) != 0) return false;
    return true;
}

// p in the plane abc, exactly: every 3x3 minor of [b-a; c-a; p-a] vanishes.
__device__ __noinline__ bool on_plane4(const float *a, const float *b, const float *c,
                                       const float *p)
{
    const int T[4][3] = {{0, 1, 2}, {0, 1, 3}, {0, 2, 3}, {1, 2, 3}};
    for (int q = 0; q < 4; q++) {
        const float pa[3] = {a[T[q][0]], a[T[q][1]], a[T[q][2]]};
        const float pb[3] = {b[T[q][0]], b[T[q][1]], b[T[q][2]]};
        const float pc[3] = {c[T[q][0]], c[T[q][1]], c[T[q][2]]};
        const float pp[3] = {p[T[q][0]], p[T[q][1]], p[T[q][2]]};
        if (orient3d_exact_sign(pa, pb, pc, pp) != 0) return false;
    }
    return true;
}

}  // namespace qh
