// Hull measures and their gradients with respect to the input points
// (the paper computes hulls only; these kernels make the hull a
// differentiable layer).  The hull's combinatorial structure is piecewise
// constant in the input, so on general-position inputs each measure is a
// smooth function of the hull vertices alone and its gradient is zero on
// every other point.
//
//  2D, hull p_0 .. p_{h-1} counter-clockwise (cyclic):
//    perimeter P = sum |p_{i+1} - p_i|,
//      dP/dp_i = u(p_{i-1} -> p_i) - u(p_i -> p_{i+1}), u = unit vector;
//    area A = 1/2 sum (p_i - o) x (p_{i+1} - o)   (any fixed o),
//      dA/dx_i = (y_{i+1} - y_{i-1}) / 2,  dA/dy_i = (x_{i-1} - x_{i+1}) / 2.
//  3D, faces counter-clockwise from outside, split into fans (a, b, c):
//    area S = sum |n| / 2 with n = (b - a) x (c - a), n^ = n / |n|:
//      dS/da = (b - c) x n^ / 2, dS/db = (c - a) x n^ / 2, dS/dc = (a - b) x n^ / 2;
//    volume V = sum (a - o) . ((b - o) x (c - o)) / 6 for a fixed o:
//      dV/da = (b - o) x (c - o) / 6 and cyclically.  The terms in o sum to
//      zero over a closed surface, so o may be any point held constant (the
//      cloud's first face vertex).
// All sums in FP64; gradients are accumulated in FP64 and rounded once.
#include <algorithm>

#include "qh.h"
#include "qh_internal.h"

namespace qh {
namespace diff {

constexpr int kBlock = 256;

struct D3 {
    double x, y, z;
};
__device__ __forceinline__ D3 sub(D3 a, D3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ D3 cross(D3 a, D3 b)
{
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ double dot(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ D3 scale(D3 a, double s) { return {a.x * s, a.y * s, a.z * s}; }

__device__ __forceinline__ double block_sum(double v, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < nw; i++) t += sh[i];
    return t;  // valid in thread 0
}

struct Pts {
    const float *x, *y, *z;
    long long stride;
    __device__ __forceinline__ D3 at(int i) const
    {
        const long long o = (long long)i * stride;
        return {(double)x[o], (double)y[o], z ? (double)z[o] : 0.0};
    }
};

// ---------------------------------------------------------------- 2D
__global__ void __launch_bounds__(kBlock) k_meas2d(Pts P, const long long *coff, int ncloud,
                                                    const int32_t *hull, const int32_t *cnt,
                                                    double *meas)
{
    __shared__ double sh[32];
    for (int c = blockIdx.x; c < ncloud; c += gridDim.x) {
        const int lo = (int)coff[c], h = cnt[c];
        const int32_t *H = hull + lo;
        double per = 0.0, area = 0.0;
        if (h > 0) {
            const D3 o = P.at(H[0]);
            for (int i = threadIdx.x; i < h; i += blockDim.x) {
                const D3 a = P.at(H[i]), b = P.at(H[(i + 1) % h]);
                const D3 d = sub(b, a);
                per += sqrt(d.x * d.x + d.y * d.y);
                area += 0.5 * ((a.x - o.x) * (b.y - o.y) - (b.x - o.x) * (a.y - o.y));
            }
        }
        per = block_sum(per, sh);
        area = block_sum(area, sh);
        if (threadIdx.x == 0) {
            meas[2 * c + 0] = per;
            meas[2 * c + 1] = area;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kBlock) k_zero_grad(float *gx, float *gy, float *gz,
                                                       long long gstride, long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        gx[i * gstride] = 0.0f;
        gy[i * gstride] = 0.0f;
        if (gz) gz[i * gstride] = 0.0f;
    }
}

__global__ void __launch_bounds__(kBlock) k_bwd2d(Pts P, const long long *coff, int ncloud,
                                                   const int32_t *hull, const int32_t *cnt,
                                                   const double *g, float *gx, float *gy,
                                                   long long gstride)
{
    for (int c = blockIdx.x; c < ncloud; c += gridDim.x) {
        const int lo = (int)coff[c], h = cnt[c];
        const int32_t *H = hull + lo;
        const double wp = g[2 * c + 0], wa = g[2 * c + 1];
        for (int i = threadIdx.x; i < h; i += blockDim.x) {
            const int vi = H[i];
            const D3 p = P.at(vi), pj = P.at(H[(i + h - 1) % h]), pk = P.at(H[(i + 1) % h]);
            double dx = 0.0, dy = 0.0;
            const D3 a = sub(p, pj), b = sub(p, pk);
            const double la = sqrt(a.x * a.x + a.y * a.y), lb = sqrt(b.x * b.x + b.y * b.y);
            if (la > 0.0) {
                dx += wp * a.x / la;
                dy += wp * a.y / la;
            }
            if (lb > 0.0) {
                dx += wp * b.x / lb;
                dy += wp * b.y / lb;
            }
            dx += wa * 0.5 * (pk.y - pj.y);
            dy += wa * 0.5 * (pj.x - pk.x);
            gx[(long long)vi * gstride] = (float)dx;
            gy[(long long)vi * gstride] = (float)dy;
        }
    }
}

// ---------------------------------------------------------------- 3D
__global__ void __launch_bounds__(kBlock) k_meas3d(Pts P, int ncloud, const int32_t *foff,
                                                    const int32_t *fidx, const int32_t *cfoff,
                                                    double *meas)
{
    __shared__ double sh[32];
    for (int c = blockIdx.x; c < ncloud; c += gridDim.x) {
        const int f0 = cfoff[c], f1 = cfoff[c + 1];
        double area = 0.0, vol = 0.0;
        if (f1 > f0) {
            const D3 o = P.at(fidx[foff[f0]]);
            for (int f = f0 + threadIdx.x; f < f1; f += blockDim.x) {
                const int s = foff[f], m = foff[f + 1] - s;
                const D3 a = P.at(fidx[s]);
                for (int k = 1; k + 1 < m; k++) {
                    const D3 b = P.at(fidx[s + k]), cc = P.at(fidx[s + k + 1]);
                    const D3 nrm = cross(sub(b, a), sub(cc, a));
                    area += 0.5 * sqrt(dot(nrm, nrm));
                    vol += dot(sub(a, o), cross(sub(b, o), sub(cc, o))) / 6.0;
                }
            }
        }
        area = block_sum(area, sh);
        vol = block_sum(vol, sh);
        if (threadIdx.x == 0) {
            meas[2 * c + 0] = area;
            meas[2 * c + 1] = vol;
        }
        __syncthreads();
    }
}

// One thread per face (all clouds): its fan's contributions, accumulated
// per vertex with FP64 atomics.
__global__ void __launch_bounds__(kBlock) k_bwd3d(Pts P, int ncloud, const int32_t *foff,
                                                   const int32_t *fidx, const int32_t *cfoff,
                                                   const double *g, double *acc)
{
    const int nf = cfoff[ncloud];
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += gridDim.x * blockDim.x) {
        int lo = 0, hi = ncloud - 1;  // cloud of face f: last c with cfoff[c] <= f
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (cfoff[mid] <= f) lo = mid;
            else hi = mid - 1;
        }
        const int c = lo;
        const double ws = g[2 * c + 0], wv = g[2 * c + 1];
        const D3 o = P.at(fidx[foff[cfoff[c]]]);
        const int s = foff[f], m = foff[f + 1] - s;
        const int ia = fidx[s];
        const D3 a = P.at(ia);
        for (int k = 1; k + 1 < m; k++) {
            const int ib = fidx[s + k], ic = fidx[s + k + 1];
            const D3 b = P.at(ib), cc = P.at(ic);
            const D3 nrm = cross(sub(b, a), sub(cc, a));
            const double len = sqrt(dot(nrm, nrm));
            D3 ga = {0, 0, 0}, gb = {0, 0, 0}, gc = {0, 0, 0};
            if (len > 0.0) {
                const D3 u = scale(nrm, 0.5 * ws / len);
                ga = cross(sub(b, cc), u);
                gb = cross(sub(cc, a), u);
                gc = cross(sub(a, b), u);
            }
            const D3 ao = sub(a, o), bo = sub(b, o), co = sub(cc, o);
            const double v6 = wv / 6.0;
            const D3 va = scale(cross(bo, co), v6), vb = scale(cross(co, ao), v6),
                     vc = scale(cross(ao, bo), v6);
            const int id[3] = {ia, ib, ic};
            const D3 gg[3] = {{ga.x + va.x, ga.y + va.y, ga.z + va.z},
                              {gb.x + vb.x, gb.y + vb.y, gb.z + vb.z},
                              {gc.x + vc.x, gc.y + vc.y, gc.z + vc.z}};
            for (int t = 0; t < 3; t++) {
                atomicAdd(&acc[3ll * id[t] + 0], gg[t].x);
                atomicAdd(&acc[3ll * id[t] + 1], gg[t].y);
                atomicAdd(&acc[3ll * id[t] + 2], gg[t].z);
            }
        }
    }
}

__global__ void __launch_bounds__(kBlock) k_round3d(const double *acc, long long n, float *gx,
                                                     float *gy, float *gz, long long gstride)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        gx[i * gstride] = (float)acc[3 * i + 0];
        gy[i * gstride] = (float)acc[3 * i + 1];
        gz[i * gstride] = (float)acc[3 * i + 2];
    }
}

// grid-stride kernels: at most eight CTAs per SM of the current device
static int cloud_grid(int ncloud) { return std::max(1, std::min(ncloud, 8 * sm_count())); }
static int pts_grid(long long n)
{
    return (int)std::max(1ll, std::min((n + 255) / 256, 8ll * sm_count()));
}

}  // namespace diff
}  // namespace qh

using namespace qh::diff;

extern "C" qh_status qh_measures2d(const float *d_x, const float *d_y, int64_t stride,
                                   const int64_t *d_cloud_off, int32_t ncloud,
                                   const int32_t *d_hull, const int32_t *d_cloud_count,
                                   double *d_meas, cudaStream_t st)
{
    if (!d_x || !d_y || stride < 1 || !d_cloud_off || ncloud < 1 || !d_hull || !d_cloud_count ||
        !d_meas)
        return QH_ERR_INVALID_ARG;
    Pts P{d_x, d_y, nullptr, stride};
    k_meas2d<<<cloud_grid(ncloud), kBlock, 0, st>>>(P, (const long long *)d_cloud_off, ncloud,
                                                    d_hull, d_cloud_count, d_meas);
    return cudaGetLastError() == cudaSuccess ? QH_OK : QH_ERR_CUDA;
}

extern "C" qh_status qh_hull2d_backward(const float *d_x, const float *d_y, int64_t stride,
                                        const int64_t *d_cloud_off, int32_t ncloud, int64_t n,
                                        const int32_t *d_hull, const int32_t *d_cloud_count,
                                        const double *d_grad, float *d_gx, float *d_gy,
                                        int64_t gstride, cudaStream_t st)
{
    if (!d_x || !d_y || stride < 1 || !d_cloud_off || ncloud < 1 || n < 0 || !d_hull ||
        !d_cloud_count || !d_grad || !d_gx || !d_gy || gstride < 1)
        return QH_ERR_INVALID_ARG;
    Pts P{d_x, d_y, nullptr, stride};
    if (n > 0) k_zero_grad<<<pts_grid(n), kBlock, 0, st>>>(d_gx, d_gy, nullptr, gstride, n);
    k_bwd2d<<<cloud_grid(ncloud), kBlock, 0, st>>>(P, (const long long *)d_cloud_off, ncloud,
                                                   d_hull, d_cloud_count, d_grad, d_gx, d_gy,
                                                   gstride);
    return cudaGetLastError() == cudaSuccess ? QH_OK : QH_ERR_CUDA;
}

extern "C" qh_status qh_measures3d(const float *d_x, const float *d_y, const float *d_z,
                                   int64_t stride, int32_t ncloud, const int32_t *d_face_off,
                                   const int32_t *d_face_idx, const int32_t *d_cloud_face_off,
                                   double *d_meas, cudaStream_t st)
{
    if (!d_x || !d_y || !d_z || stride < 1 || ncloud < 1 || !d_face_off || !d_face_idx ||
        !d_cloud_face_off || !d_meas)
        return QH_ERR_INVALID_ARG;
    Pts P{d_x, d_y, d_z, stride};
    k_meas3d<<<cloud_grid(ncloud), kBlock, 0, st>>>(P, ncloud, d_face_off, d_face_idx,
                                                    d_cloud_face_off, d_meas);
    return cudaGetLastError() == cudaSuccess ? QH_OK : QH_ERR_CUDA;
}

extern "C" qh_status qh_hull3d_backward(const float *d_x, const float *d_y, const float *d_z,
                                        int64_t stride, int32_t ncloud, int64_t n,
                                        const int32_t *d_face_off, const int32_t *d_face_idx,
                                        const int32_t *d_cloud_face_off, const double *d_grad,
                                        float *d_gx, float *d_gy, float *d_gz, int64_t gstride,
                                        double *d_scratch, cudaStream_t st)
{
    if (!d_x || !d_y || !d_z || stride < 1 || ncloud < 1 || n < 0 || !d_face_off ||
        !d_face_idx || !d_cloud_face_off || !d_grad || !d_gx || !d_gy || !d_gz || gstride < 1 ||
        !d_scratch)
        return QH_ERR_INVALID_ARG;
    Pts P{d_x, d_y, d_z, stride};
    if (n == 0) return QH_OK;
    if (cudaMemsetAsync(d_scratch, 0, (size_t)n * 3 * sizeof(double), st) != cudaSuccess)
        return QH_ERR_CUDA;
    k_bwd3d<<<pts_grid(2 * n), kBlock, 0, st>>>(P, ncloud, d_face_off, d_face_idx,
                                                d_cloud_face_off, d_grad, d_scratch);
    k_round3d<<<pts_grid(n), kBlock, 0, st>>>(d_scratch, n, d_gx, d_gy, d_gz, gstride);
    return cudaGetLastError() == cudaSuccess ? QH_OK : QH_ERR_CUDA;
}
