// Exact 3D predicates for the device path.
//
// vol(a, b, c, p) = det[b-a; c-a; p-a] is positive when p lies on the side of
// the normal (b-a) x (c-a), i.e. the side from which a, b, c appear
// counter-clockwise.  Every sign goes through
//   1. FP32 (fast filter) or FP64 (plain path) with a forward error bound,
//   2. FP64 with its bound (behind the FP32 filter),
//   3. exact: det[b-a, c-a, p-a] = det[b,c,p] - det[a,c,p] - det[b,a,p] -
//      det[b,c,a] expands into 24 signed products of three float32
//      coordinates; x*y is exact in FP64 (two 24-bit significands) and
//      (x*y)*z is exact as a two-term expansion (two-product via fma), so the
//      determinant is the exact sum of 48 doubles, whose sign is read from a
//      non-overlapping expansion grown term by term (Shewchuk 1997).
//
// Bound of stages 1/2 for det = u.(v x w) evaluated as
// u0 (v1 w2 - v2 w1) + u1 (v2 w0 - v0 w2) + u2 (v0 w1 - v1 w0) with rounded
// differences: every monomial picks up at most eight roundings (three
// differences, the product inside the minor, the minor's subtraction, the
// product with u, two additions), so |det - D| <= (8u + O(u^2)) * perm with
// perm = sum |u_i| (|v_j w_k| + |v_k w_j|).  The code uses 8u(1 + 2^-10) perm.
// FP32 products may underflow, and an underflowed minor multiplied by a
// large u_i breaks a relative bound; the FP32 stage therefore only decides
// when every non-zero difference is at least 2^-40 in magnitude (all products
// then stay normal).  FP64 products of float32-derived values never underflow.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "pred2.cuh"

namespace qh {

constexpr float kC32_3 = 0x1.004p-21f;  // 8 * 2^-24 * (1 + 2^-10)
constexpr double kC64_3 = 0x1.004p-50;  // 8 * 2^-53 * (1 + 2^-10)
constexpr float kTiny3 = 0x1p-40f;      // smallest non-zero difference the FP32 stage accepts

// det[u; v; w] in FP32 with its bound; e = +inf when the stage cannot decide.
__device__ __forceinline__ void det3_f32(float u0, float u1, float u2, float v0, float v1,
                                         float v2, float w0, float w1, float w2, float &d,
                                         float &e)
{
    float m0a = __fmul_rn(v1, w2), m0b = __fmul_rn(v2, w1);
    float m1a = __fmul_rn(v2, w0), m1b = __fmul_rn(v0, w2);
    float m2a = __fmul_rn(v0, w1), m2b = __fmul_rn(v1, w0);
    float t0 = __fmul_rn(u0, __fsub_rn(m0a, m0b));
    float t1 = __fmul_rn(u1, __fsub_rn(m1a, m1b));
    float t2 = __fmul_rn(u2, __fsub_rn(m2a, m2b));
    d = __fadd_rn(__fadd_rn(t0, t1), t2);
    float perm = __fadd_rn(
        __fadd_rn(__fmul_rn(fabsf(u0), __fadd_rn(fabsf(m0a), fabsf(m0b))),
                  __fmul_rn(fabsf(u1), __fadd_rn(fabsf(m1a), fabsf(m1b)))),
        __fmul_rn(fabsf(u2), __fadd_rn(fabsf(m2a), fabsf(m2b))));
    e = __fmul_rn(kC32_3, perm);
    auto small = [](float t) { return t != 0.0f && fabsf(t) < kTiny3; };
    if (small(u0) || small(u1) || small(u2) || small(v0) || small(v1) || small(v2) ||
        small(w0) || small(w1) || small(w2))
        e = INFINITY;
}

__device__ __forceinline__ void det3_f64(double u0, double u1, double u2, double v0, double v1,
                                         double v2, double w0, double w1, double w2, double &d,
                                         double &e)
{
    double m0a = __dmul_rn(v1, w2), m0b = __dmul_rn(v2, w1);
    double m1a = __dmul_rn(v2, w0), m1b = __dmul_rn(v0, w2);
    double m2a = __dmul_rn(v0, w1), m2b = __dmul_rn(v1, w0);
    double t0 = __dmul_rn(u0, __dsub_rn(m0a, m0b));
    double t1 = __dmul_rn(u1, __dsub_rn(m1a, m1b));
    double t2 = __dmul_rn(u2, __dsub_rn(m2a, m2b));
    d = __dadd_rn(__dadd_rn(t0, t1), t2);
    double perm = fabs(u0) * (fabs(m0a) + fabs(m0b)) + fabs(u1) * (fabs(m1a) + fabs(m1b)) +
                  fabs(u2) * (fabs(m2a) + fabs(m2b));
    e = __dmul_rn(kC64_3, perm * (1.0 + 0x1p-50));
}

// Exact sign of the sum of sgn * det[x; y; z] terms appended to t.
__device__ __forceinline__ void det3_monomials(const float *x, const float *y, const float *z,
                                               double sgn, double *t, int &k)
{
    // det[x; y; z] = sum over permutations (i, j, l) of sign * x_i y_j z_l
    const int P[6][3] = {{0, 1, 2}, {1, 2, 0}, {2, 0, 1}, {0, 2, 1}, {1, 0, 2}, {2, 1, 0}};
#pragma unroll
    for (int q = 0; q < 6; q++) {
        double xy = (double)x[P[q][0]] * (double)y[P[q][1]];  // exact
        double h, l;
        two_prod_d(xy, (double)z[P[q][2]], h, l);
        double s = q < 3 ? sgn : -sgn;
        t[k++] = s * h;
        t[k++] = s * l;
    }
}

template <int M>
__device__ __forceinline__ int exact_sum_sign_n(const double *t, int m)
{
    double e[M];
    int len = 0;
#pragma unroll 1
    for (int i = 0; i < m; i++) {
        double q = t[i];
        int out = 0;
#pragma unroll 1
        for (int j = 0; j < len; j++) {
            double s, err;
            two_sum_d(q, e[j], s, err);
            q = s;
            if (err != 0.0) e[out++] = err;
        }
        if (q != 0.0 || out == 0) e[out++] = q;
        len = out;
    }
    double top = e[len - 1];
    return (top > 0.0) - (top < 0.0);
}

// Exact sign of vol(a, b, c, p).
static __device__ __noinline__ int orient3d_exact(const float *a, const float *b, const float *c,
                                           const float *p)
{
    double t[48];
    int k = 0;
    det3_monomials(b, c, p, 1.0, t, k);
    det3_monomials(a, c, p, -1.0, t, k);
    det3_monomials(b, a, p, -1.0, t, k);
    det3_monomials(b, c, a, -1.0, t, k);
    return exact_sum_sign_n<48>(t, k);
}

// Exact sign of vol(a,b,c,p1) - vol(a,b,c,p2) = det[b-a; c-a; p1-p2].
static __device__ __noinline__ int cmp_dist3_exact(const float *a, const float *b, const float *c,
                                            const float *p1, const float *p2)
{
    double t[72];
    int k = 0;
    det3_monomials(b, c, p1, 1.0, t, k);
    det3_monomials(a, c, p1, -1.0, t, k);
    det3_monomials(b, a, p1, -1.0, t, k);
    det3_monomials(b, c, p2, -1.0, t, k);
    det3_monomials(a, c, p2, 1.0, t, k);
    det3_monomials(b, a, p2, 1.0, t, k);
    return exact_sum_sign_n<72>(t, k);
}

// FP64 filter then exact, for vol(a, b, c, p).
static __device__ __noinline__ int orient3d_slow(const float *a, const float *b, const float *c,
                                          const float *p)
{
    double d, e;
    det3_f64(__dsub_rn(b[0], a[0]), __dsub_rn(b[1], a[1]), __dsub_rn(b[2], a[2]),
             __dsub_rn(c[0], a[0]), __dsub_rn(c[1], a[1]), __dsub_rn(c[2], a[2]),
             __dsub_rn(p[0], a[0]), __dsub_rn(p[1], a[1]), __dsub_rn(p[2], a[2]), d, e);
    if (d > e) return 1;
    if (-d > e) return -1;
    return orient3d_exact(a, b, c, p);
}

static __device__ __noinline__ int cmp_dist3_slow(const float *a, const float *b, const float *c,
                                           const float *p1, const float *p2)
{
    double d, e;
    det3_f64(__dsub_rn(b[0], a[0]), __dsub_rn(b[1], a[1]), __dsub_rn(b[2], a[2]),
             __dsub_rn(c[0], a[0]), __dsub_rn(c[1], a[1]), __dsub_rn(c[2], a[2]),
             __dsub_rn(p1[0], p2[0]), __dsub_rn(p1[1], p2[1]), __dsub_rn(p1[2], p2[2]), d, e);
    if (d > e) return 1;
    if (-d > e) return -1;
    return cmp_dist3_exact(a, b, c, p1, p2);
}

// Filter value of vol(a, b, c, p) and its bound, as float (keys of the
// farthest-point reduction).  MODE: QH_PRED_F32 or QH_PRED_F64.
template <int MODE>
__device__ __forceinline__ void orient3d_value(const float *a, const float *b, const float *c,
                                               const float *p, float &d, float &e)
{
    if (MODE == QH_PRED_F32) {
        det3_f32(__fsub_rn(b[0], a[0]), __fsub_rn(b[1], a[1]), __fsub_rn(b[2], a[2]),
                 __fsub_rn(c[0], a[0]), __fsub_rn(c[1], a[1]), __fsub_rn(c[2], a[2]),
                 __fsub_rn(p[0], a[0]), __fsub_rn(p[1], a[1]), __fsub_rn(p[2], a[2]), d, e);
    } else {
        double dd, ee;
        det3_f64(__dsub_rn(b[0], a[0]), __dsub_rn(b[1], a[1]), __dsub_rn(b[2], a[2]),
                 __dsub_rn(c[0], a[0]), __dsub_rn(c[1], a[1]), __dsub_rn(c[2], a[2]),
                 __dsub_rn(p[0], a[0]), __dsub_rn(p[1], a[1]), __dsub_rn(p[2], a[2]), dd, ee);
        d = __double2float_rn(dd);
        e = __double2float_ru(__dadd_ru(__dadd_ru(ee, __dmul_ru(fabs(dd), 0x1p-23)), 0x1p-146));
    }
}

// A facet's plane for the FP32 filter of many points against one facet.
// The same determinant det[u; v; w] (u = b - a, v = c - a, w = p - a)
// expanded along w instead: D = (w0 n0 + w1 n1) + w2 n2 with the minors
// n_i = u_j v_k - u_k v_j (each product and the difference rounded) and
// m_i = |u_j v_k| + |u_k v_j|.  Every monomial u_j v_k w_i still passes
// through eight roundings (w_i, u_j, v_k, the product u_j v_k, the minor's
// difference, the product with w_i, two sums), so the bound of det3_f32
// holds with its roles permuted: |det - D| <= 8u(1 + 2^-10) perm, perm =
// sum_i |w_i| m_i.  The minors are computed once per facet; a point then
// costs three differences and two short dot products.  a.w = 1 marks a facet
// with a non-zero component of u or v below 2^-40 (the filter never decides
// then, as in det3_f32); the same test on w is made per point.
struct Plane3 {
    float4 a, n, m;
};

__device__ __forceinline__ Plane3 make_plane3(const float *a, const float *b, const float *c)
{
    const float u0 = __fsub_rn(b[0], a[0]), u1 = __fsub_rn(b[1], a[1]), u2 = __fsub_rn(b[2], a[2]);
    const float v0 = __fsub_rn(c[0], a[0]), v1 = __fsub_rn(c[1], a[1]), v2 = __fsub_rn(c[2], a[2]);
    const float p0a = __fmul_rn(u1, v2), p0b = __fmul_rn(u2, v1);
    const float p1a = __fmul_rn(u2, v0), p1b = __fmul_rn(u0, v2);
    const float p2a = __fmul_rn(u0, v1), p2b = __fmul_rn(u1, v0);
    auto small = [](float t) { return t != 0.0f && fabsf(t) < kTiny3; };
    const bool never = small(u0) || small(u1) || small(u2) || small(v0) || small(v1) || small(v2);
    Plane3 P;
    P.a = make_float4(a[0], a[1], a[2], never ? 1.0f : 0.0f);
    P.n = make_float4(__fsub_rn(p0a, p0b), __fsub_rn(p1a, p1b), __fsub_rn(p2a, p2b), 0.0f);
    P.m = make_float4(__fadd_rn(fabsf(p0a), fabsf(p0b)), __fadd_rn(fabsf(p1a), fabsf(p1b)),
                      __fadd_rn(fabsf(p2a), fabsf(p2b)), 0.0f);
    return P;
}

// FP32 value of vol(a, b, c, p) and its bound from the facet's plane
// (e = +inf when the filter cannot decide).
__device__ __forceinline__ void plane3_value(const Plane3 &P, float px, float py, float pz,
                                             float &d, float &e)
{
    const float w0 = __fsub_rn(px, P.a.x), w1 = __fsub_rn(py, P.a.y), w2 = __fsub_rn(pz, P.a.z);
    d = __fadd_rn(__fadd_rn(__fmul_rn(w0, P.n.x), __fmul_rn(w1, P.n.y)), __fmul_rn(w2, P.n.z));
    const float perm = __fadd_rn(__fadd_rn(__fmul_rn(fabsf(w0), P.m.x), __fmul_rn(fabsf(w1), P.m.y)),
                                 __fmul_rn(fabsf(w2), P.m.z));
    e = __fmul_rn(kC32_3, perm);
    auto small = [](float t) { return t != 0.0f && fabsf(t) < kTiny3; };
    if (P.a.w != 0.0f || small(w0) || small(w1) || small(w2)) e = INFINITY;
}

// Exact sign of vol(a, b, c, p) given its filter value.
template <int MODE>
__device__ __forceinline__ int orient3d_sign(float d, float e, const float *a, const float *b,
                                             const float *c, const float *p, unsigned &fallbacks)
{
    if (d > e) return 1;
    if (-d > e) return -1;
    ++fallbacks;
    if (MODE == QH_PRED_F32) return orient3d_slow(a, b, c, p);
    return orient3d_exact(a, b, c, p);
}

__device__ __forceinline__ int orient3d_exact_sign(const float *a, const float *b, const float *c,
                                                   const float *p)
{
    float d, e;
    orient3d_value<QH_PRED_F32>(a, b, c, p, d, e);
    if (d > e) return 1;
    if (-d > e) return -1;
    return orient3d_slow(a, b, c, p);
}

__device__ __forceinline__ int cmp_dist3_exact_sign(const float *a, const float *b, const float *c,
                                                    const float *p1, const float *p2)
{
    float d, e;
    det3_f32(__fsub_rn(b[0], a[0]), __fsub_rn(b[1], a[1]), __fsub_rn(b[2], a[2]),
             __fsub_rn(c[0], a[0]), __fsub_rn(c[1], a[1]), __fsub_rn(c[2], a[2]),
             __fsub_rn(p1[0], p2[0]), __fsub_rn(p1[1], p2[1]), __fsub_rn(p1[2], p2[2]), d, e);
    if (d > e) return 1;
    if (-d > e) return -1;
    return cmp_dist3_slow(a, b, c, p1, p2);
}

}  // namespace qh
