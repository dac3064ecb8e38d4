// Exact 2D predicates for the device path.
//
// Every sign that decides the hull goes through three stages:
//   1. the fast filter: the determinant in FP32 (or FP64 on the plain path)
//      with a forward error bound; the sign is certain when |det| > bound;
//   2. FP64 with its own bound (only behind the FP32 filter);
//   3. exact: each coordinate difference as a two-term FP64 expansion
//      (two-sum), each product of expansion terms split exactly (two-product
//      via fma), and the sign of the exact sum of the 16 resulting doubles
//      from a non-overlapping expansion built by repeated two-sum
//      (Shewchuk 1997, grow-expansion with zero elimination).
//
// Error bound of stage 1/2 for det = fl(fl(fl(x1-x2) fl(y3-y4)) - fl(fl(y1-y2) fl(x3-x4))):
// with unit roundoff u, each product carries (1+u)^3 and the subtraction
// (1+u), so |det - D| <= (u + g3/(1-g3)) (|l| + |r|), g3 = (1+u)^3 - 1, i.e.
// 4u + O(u^2).  The code uses 4u(1 + 2^-10) on the computed |l| + |r|, which
// also covers the rounding of the bound itself.  FP32 products can underflow
// (absolute error <= 2^-150 each, sums of float32 values are exact when
// subnormal), hence the absolute term 2^-146.  Overflow gives Inf/NaN, which
// fails the filter and falls through to the exact stage.  Products in FP64 of
// float32-derived values neither underflow nor overflow.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "qh.h"

namespace qh {

constexpr float kC32 = 0x1.004p-22f;   // 4 * 2^-24 * (1 + 2^-10)
constexpr float kU32 = 0x1p-146f;      // absolute term for FP32 underflow
constexpr double kC64 = 0x1.004p-51;   // 4 * 2^-53 * (1 + 2^-10)

// ---------------------------------------------------------------- exact stage
__device__ __forceinline__ void two_sum_d(double a, double b, double &s, double &e)
{
    s = __dadd_rn(a, b);
    double bv = __dsub_rn(s, a);
    double av = __dsub_rn(s, bv);
    e = __dadd_rn(__dsub_rn(a, av), __dsub_rn(b, bv));
}

__device__ __forceinline__ void two_prod_d(double a, double b, double &p, double &e)
{
    p = __dmul_rn(a, b);
    e = __fma_rn(a, b, -p);
}

// Sign of the exact sum of t[0..m).  The running expansion e[] is kept
// non-overlapping in increasing magnitude; its sign is the sign of its
// largest component.
template <int M>
__device__ __forceinline__ int exact_sum_sign(const double (&t)[M])
{
    double e[M];
    int len = 0;
#pragma unroll 1
    for (int i = 0; i < M; i++) {
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

// Exact sign of (p1 - p2) x (p3 - p4) for float coordinates.
static __device__ __noinline__ int cross_diff_exact(float p1x, float p1y, float p2x, float p2y,
                                             float p3x, float p3y, float p4x, float p4y)
{
    double u[2], v[2], w[2], z[2];
    two_sum_d((double)p1x, -(double)p2x, u[1], u[0]);
    two_sum_d((double)p3y, -(double)p4y, v[1], v[0]);
    two_sum_d((double)p1y, -(double)p2y, w[1], w[0]);
    two_sum_d((double)p3x, -(double)p4x, z[1], z[0]);
    double t[16];
    int k = 0;
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 2; j++) {
            double p, e;
            two_prod_d(u[i], v[j], p, e);
            t[k++] = p;
            t[k++] = e;
            two_prod_d(w[i], z[j], p, e);
            t[k++] = -p;
            t[k++] = -e;
        }
    return exact_sum_sign(t);
}

// ---------------------------------------------------------------- FP64 stage
__device__ __forceinline__ void cross_diff_f64(float p1x, float p1y, float p2x, float p2y,
                                               float p3x, float p3y, float p4x, float p4y,
                                               double &det, double &err)
{
    double l = __dmul_rn(__dsub_rn(p1x, p2x), __dsub_rn(p3y, p4y));
    double r = __dmul_rn(__dsub_rn(p1y, p2y), __dsub_rn(p3x, p4x));
    det = __dsub_rn(l, r);
    err = __dmul_rn(kC64, __dadd_rn(fabs(l), fabs(r)));
}

// FP64 filter, then exact.
static __device__ __noinline__ int cross_diff_sign_slow(float p1x, float p1y, float p2x, float p2y,
                                                 float p3x, float p3y, float p4x, float p4y)
{
    double det, err;
    cross_diff_f64(p1x, p1y, p2x, p2y, p3x, p3y, p4x, p4y, det, err);
    if (det > err) return 1;
    if (-det > err) return -1;
    return cross_diff_exact(p1x, p1y, p2x, p2y, p3x, p3y, p4x, p4y);
}

// ---------------------------------------------------------------- FP32 stage
__device__ __forceinline__ void cross_diff_f32(float p1x, float p1y, float p2x, float p2y,
                                               float p3x, float p3y, float p4x, float p4y,
                                               float &det, float &err)
{
    float l = __fmul_rn(__fsub_rn(p1x, p2x), __fsub_rn(p3y, p4y));
    float r = __fmul_rn(__fsub_rn(p1y, p2y), __fsub_rn(p3x, p4x));
    det = __fsub_rn(l, r);
    err = __fadd_rn(__fmul_rn(kC32, __fadd_rn(fabsf(l), fabsf(r))), kU32);
}

// Predicate policies.  value() returns the filter value and a bound as float
// (used for the farthest-point keys); sign() returns the exact sign, using
// the value when it is decisive and counting the fallbacks.
struct PredF32 {
    static constexpr int kMode = QH_PRED_F32;
    __device__ __forceinline__ static void value(float p1x, float p1y, float p2x, float p2y,
                                                 float p3x, float p3y, float p4x, float p4y,
                                                 float &d, float &e)
    {
        cross_diff_f32(p1x, p1y, p2x, p2y, p3x, p3y, p4x, p4y, d, e);
    }
};

struct PredF64 {
    static constexpr int kMode = QH_PRED_F64;
    __device__ __forceinline__ static void value(float p1x, float p1y, float p2x, float p2y,
                                                 float p3x, float p3y, float p4x, float p4y,
                                                 float &d, float &e)
    {
        double dd, ee;
        cross_diff_f64(p1x, p1y, p2x, p2y, p3x, p3y, p4x, p4y, dd, ee);
        // the value is reported rounded to FP32; the bound adds that rounding
        // (<= 2^-24 |d|, plus 2^-150 when the result is subnormal)
        d = __double2float_rn(dd);
        e = __double2float_ru(__dadd_ru(__dadd_ru(ee, __dmul_ru(fabs(dd), 0x1p-23)), 0x1p-146));
    }
};

// Exact sign of (p1-p2) x (p3-p4) given the filter value/bound already
// computed by P::value for the same operands.
template <class P>
__device__ __forceinline__ int sign_from(float d, float e, float p1x, float p1y, float p2x,
                                         float p2y, float p3x, float p3y, float p4x, float p4y,
                                         unsigned &fallbacks)
{
    if (d > e) return 1;
    if (-d > e) return -1;
    ++fallbacks;
    if (P::kMode == QH_PRED_F32)
        return cross_diff_sign_slow(p1x, p1y, p2x, p2y, p3x, p3y, p4x, p4y);
    return cross_diff_exact(p1x, p1y, p2x, p2y, p3x, p3y, p4x, p4y);
}

// orient2d(a, b, c) = (a - c) x (b - c): positive when a, b, c turn
// counter-clockwise.
template <class P>
__device__ __forceinline__ void orient_value(float ax, float ay, float bx, float by, float cx,
                                             float cy, float &d, float &e)
{
    P::value(ax, ay, cx, cy, bx, by, cx, cy, d, e);
}

template <class P>
__device__ __forceinline__ int orient_sign(float d, float e, float ax, float ay, float bx,
                                           float by, float cx, float cy, unsigned &fallbacks)
{
    return sign_from<P>(d, e, ax, ay, cx, cy, bx, by, cx, cy, fallbacks);
}

// Exact orientation sign from scratch (used off the hot path).
__device__ __forceinline__ int orient_exact_sign(float ax, float ay, float bx, float by, float cx,
                                                 float cy)
{
    float d, e;
    cross_diff_f32(ax, ay, cx, cy, bx, by, cx, cy, d, e);
    if (d > e) return 1;
    if (-d > e) return -1;
    return cross_diff_sign_slow(ax, ay, cx, cy, bx, by, cx, cy);
}

// Exact comparison of the distances of p1 and p2 beyond the directed line
// a->b: sign(orient(a,b,p1) - orient(a,b,p2)) = sign((b - a) x (p1 - p2)).
__device__ __forceinline__ int cmp_dist_exact(float ax, float ay, float bx, float by, float p1x,
                                              float p1y, float p2x, float p2y)
{
    float d, e;
    cross_diff_f32(bx, by, ax, ay, p1x, p1y, p2x, p2y, d, e);
    if (d > e) return 1;
    if (-d > e) return -1;
    return cross_diff_sign_slow(bx, by, ax, ay, p1x, p1y, p2x, p2y);
}

}  // namespace qh
