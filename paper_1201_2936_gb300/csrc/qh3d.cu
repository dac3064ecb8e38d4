// 3D segmented Quickhull on one GPU.
//
// The paper extends its 2D algorithm to 3D by a first split with a triangle
// plane and a 3-state flagPermute in the recursion (Section 4.3, "3D and
// Higher Dimensions", Algorithm 1).  Splitting each face's points among the
// three faces of a tetrahedron built on it does not keep the partial hull
// convex, so this implementation follows the Quickhull of Barber et al. that
// the paper builds on: the farthest point of a facet's outside set (its
// "segment") becomes an apex, the facets it sees strictly form its visible
// set, the horizon of that set is coned to the apex, and the points of the
// visible facets are reassigned to the first cone facet they are strictly
// above (else discarded as interior).  Several apexes are inserted per
// iteration: each candidate claims its visible facets with a priority; a
// candidate whose visible set is entirely its own and whose horizon
// neighbours carry no higher-priority claim is inserted.  Two insertions
// chosen this way touch disjoint, non-adjacent facet sets, so they commute.
//
// Per iteration (persistent kernel, grid barriers between phases):
//   S  (select)   one thread per segment: visible-set BFS from the facet with
//                 exact orientation tests, priority claims.
//   C  (cone)     winners build their cone facets and relink neighbours.
//   A  (assign)   every live point: kept (its facet survives) or tested
//                 against its winner's cone facets; warp-aggregated counts,
//                 ranks and farthest-point keys per target facet.
//   T  (table)    scan of the new segment sizes (kept segments in order,
//                 then the new cone facets).
//   B  (scatter)  points to their new positions; certification of each new
//                 facet's farthest point (FP32 top-2 gap against the error
//                 bound), tile -> segment map.
//   X  (exact)    exact farthest point of uncertified facets.
// The output (maximal coplanar faces, canonical order) is produced by the
// kernels in qh3d_out.cu.

#include <climits>
#include <cstdio>
#include <cstring>

#include "pred3.cuh"
#include "qh3d_internal.cuh"
#include "qh_common.cuh"
#include "qh_internal.h"

namespace qh {
namespace d3 {

// ---------------------------------------------------------------- small helpers
__device__ __forceinline__ void set_status(Hdr3 *H, int st) { atomicCAS(&H->status, 0, st); }

__device__ __forceinline__ float4 load_input(const Params3 &A, long long i)
{
    const long long o = i * A.stride;
    return make_float4(__ldg(A.x + o), __ldg(A.y + o), __ldg(A.z + o), __int_as_float((int)i));
}

__device__ __forceinline__ void fac_pts(const Fac3 &f, const float *&a, const float *&b,
                                        const float *&c)
{
    a = f.p;
    b = f.p + 3;
    c = f.p + 6;
}

// Lexicographic (x, y, z, index) comparison for extrema; -0.0 == +0.0.
__device__ __forceinline__ bool lex_less(float4 p, float4 q)
{
    if (p.x != q.x) return p.x < q.x;
    if (p.y != q.y) return p.y < q.y;
    if (p.z != q.z) return p.z < q.z;
    return __float_as_int(p.w) < __float_as_int(q.w);
}
__device__ __forceinline__ bool lex_greater_lowidx(float4 p, float4 q)
{
    if (p.x != q.x) return p.x > q.x;
    if (p.y != q.y) return p.y > q.y;
    if (p.z != q.z) return p.z > q.z;
    return __float_as_int(p.w) < __float_as_int(q.w);
}

// Filter value of vol(facet g, p): the facet's plane in FP32 mode, the
// vertices (FP64 filter) in the plain mode.
template <int MODE>
__device__ __forceinline__ void facet_value(const Params3 &A, int g, const float *p, float &d,
                                            float &e)
{
    if (MODE == QH_PRED_F32) {
        const Plane3 P = A.plane[g];
        plane3_value(P, p[0], p[1], p[2], d, e);
    } else {
        const Fac3 &G = A.fac[g];
        orient3d_value<MODE>(G.p, G.p + 3, G.p + 6, p, d, e);
    }
}

// ---------------------------------------------------------------- initial simplex
// Block-level reductions write one candidate per block; block 0 reduces them
// after a grid barrier.

__device__ void extrema3d(const Params3 &A, SmemAll3 &sm, int bid, int nb)
{
    float4 mn = make_float4(INFINITY, INFINITY, INFINITY, __int_as_float(INT_MAX));
    float4 mx = make_float4(-INFINITY, -INFINITY, -INFINITY, __int_as_float(INT_MAX));
    int bad = 0;
    constexpr int kU = 4;  // points per thread in flight
    const long long step = (long long)nb * blockDim.x * kU;
    for (long long i0 = (long long)bid * blockDim.x * kU + threadIdx.x; i0 < A.n; i0 += step) {
        float4 q[kU];
#pragma unroll
        for (int k = 0; k < kU; k++) {
            const long long i = i0 + (long long)k * blockDim.x;
            q[k] = i < A.n ? load_input(A, i) : make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
        }
#pragma unroll
        for (int k = 0; k < kU; k++) {
            if (__float_as_int(q[k].w) < 0) continue;
            float4 p = q[k];
            p.x = canon0(p.x);
            p.y = canon0(p.y);
            p.z = canon0(p.z);
            bad |= !(isfinite(p.x) && isfinite(p.y) && isfinite(p.z));
            if (lex_less(p, mn)) mn = p;
            if (lex_greater_lowidx(p, mx)) mx = p;
        }
    }
    bad = __syncthreads_or(bad);
    sm.red.a[threadIdx.x] = mn;
    sm.red.b[threadIdx.x] = mx;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            if (lex_less(sm.red.a[threadIdx.x + s], sm.red.a[threadIdx.x]))
                sm.red.a[threadIdx.x] = sm.red.a[threadIdx.x + s];
            if (lex_greater_lowidx(sm.red.b[threadIdx.x + s], sm.red.b[threadIdx.x]))
                sm.red.b[threadIdx.x] = sm.red.b[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        A.blk_a[bid] = sm.red.a[0];
        A.blk_b[bid] = sm.red.b[0];
        if (bad) atomicExch(&A.hdr->nonfinite, 1);
    }
    __syncthreads();
}

// Farthest point from the line ab (kind 0) or from the plane abc (kind 1),
// FP32 magnitude, lowest index on ties.
__device__ void farthest3d(const Params3 &A, SmemAll3 &sm, int bid, int nb, int kind)
{
    const Hdr3 *H = A.hdr;
    const float a[3] = {H->pa.x, H->pa.y, H->pa.z};
    const float b[3] = {H->pb.x, H->pb.y, H->pb.z};
    const float c[3] = {H->pc.x, H->pc.y, H->pc.z};
    float best = -1.0f;
    int bi = INT_MAX;
    constexpr int kU = 4;  // points per thread in flight
    const long long step = (long long)nb * blockDim.x * kU;
    for (long long i0 = (long long)bid * blockDim.x * kU + threadIdx.x; i0 < A.n; i0 += step) {
      float4 q[kU];
#pragma unroll
      for (int k = 0; k < kU; k++) {
          const long long i = i0 + (long long)k * blockDim.x;
          q[k] = i < A.n ? load_input(A, i) : make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
      }
#pragma unroll
      for (int k = 0; k < kU; k++) {
        const long long i = i0 + (long long)k * blockDim.x;
        if (i >= A.n) continue;
        const float4 p = q[k];
        float v;
        if (kind == 0) {
            float ux = b[0] - a[0], uy = b[1] - a[1], uz = b[2] - a[2];
            float wx = p.x - a[0], wy = p.y - a[1], wz = p.z - a[2];
            float cx = uy * wz - uz * wy, cy = uz * wx - ux * wz, cz = ux * wy - uy * wx;
            v = cx * cx + cy * cy + cz * cz;
        } else {
            float q[3] = {p.x, p.y, p.z};
            float d, e;
            orient3d_value<QH_PRED_F32>(a, b, c, q, d, e);
            v = fabsf(d);
        }
        if (!(v <= best)) {  // NaN-safe: NaN never wins
            if (v > best || (v == best && (int)i < bi)) {
                best = v;
                bi = (int)i;
            }
        }
      }
    }
    sm.red.v[threadIdx.x] = best;
    sm.red.i[threadIdx.x] = bi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            float ov = sm.red.v[threadIdx.x + s];
            int oi = sm.red.i[threadIdx.x + s];
            if (ov > sm.red.v[threadIdx.x] || (ov == sm.red.v[threadIdx.x] && oi < sm.red.i[threadIdx.x])) {
                sm.red.v[threadIdx.x] = ov;
                sm.red.i[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        A.blk_v[bid] = sm.red.v[0];
        A.blk_i[bid] = sm.red.i[0];
    }
    __syncthreads();
}

__device__ __forceinline__ bool collinear3_exact(const float *a, const float *b, const float *c)
{
    for (int k = 0; k < 3; k++) {
        int i = k, j = (k + 1) % 3;
        if (orient_exact_sign(a[i], a[j], b[i], b[j], c[i], c[j]) != 0) return false;
    }
    return true;
}

// Any point not collinear with ab (kind 0) / not coplanar with abc (kind 1),
// lowest index: exact fallback when the FP32 choice turned out degenerate.
__device__ void exact_search3d(const Params3 &A, int bid, int nb, int kind)
{
    Hdr3 *H = A.hdr;
    const float a[3] = {H->pa.x, H->pa.y, H->pa.z};
    const float b[3] = {H->pb.x, H->pb.y, H->pb.z};
    const float c[3] = {H->pc.x, H->pc.y, H->pc.z};
    for (long long i = (long long)bid * blockDim.x + threadIdx.x; i < A.n;
         i += (long long)nb * blockDim.x) {
        float4 p = load_input(A, i);
        float q[3] = {p.x, p.y, p.z};
        bool ok = kind == 0 ? !collinear3_exact(a, b, q) : orient3d_exact_sign(a, b, c, q) != 0;
        if (ok) atomicMin(&H->search_idx, (int)i);
    }
}

// Block 0: reduce the per-block candidates of the previous phase (every
// thread of the block takes a stride of them, then a tree in shared memory).
__device__ void simplex_step(const Params3 &A, SmemAll3 &sm, int step, int nblk)
{
    Hdr3 *H = A.hdr;
    const int t = threadIdx.x;
    if (step == 0) {
        float4 mn = make_float4(INFINITY, INFINITY, INFINITY, __int_as_float(INT_MAX));
        float4 mx = make_float4(-INFINITY, -INFINITY, -INFINITY, __int_as_float(INT_MAX));
        bool any = false;
        for (int b = t; b < nblk; b += blockDim.x) {
            const float4 a = A.blk_a[b], c = A.blk_b[b];
            if (!any || lex_less(a, mn)) mn = a;
            if (!any || lex_greater_lowidx(c, mx)) mx = c;
            any = true;
        }
        sm.red.a[t] = mn;
        sm.red.b[t] = mx;
        sm.red.i[t] = any;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (t < s && sm.red.i[t + s]) {
                const bool mine = sm.red.i[t] != 0;
                if (!mine || lex_less(sm.red.a[t + s], sm.red.a[t])) sm.red.a[t] = sm.red.a[t + s];
                if (!mine || lex_greater_lowidx(sm.red.b[t + s], sm.red.b[t]))
                    sm.red.b[t] = sm.red.b[t + s];
                sm.red.i[t] = 1;
            }
            __syncthreads();
        }
        if (t == 0) {
            mn = sm.red.a[0];
            mx = sm.red.b[0];
            H->pa = mn;
            H->pb = mx;
            if (mn.x == mx.x && mn.y == mx.y && mn.z == mx.z) set_status(H, QH_ERR_DEGENERATE);
        }
        __syncthreads();
    } else {
        float bv = -2.0f;
        int bi = INT_MAX;
        for (int b = t; b < nblk; b += blockDim.x) {
            const float v = A.blk_v[b];
            const int i = A.blk_i[b];
            if (v > bv || (v == bv && i < bi)) {
                bv = v;
                bi = i;
            }
        }
        sm.red.v[t] = bv;
        sm.red.i[t] = bi;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (t < s) {
                const float ov = sm.red.v[t + s];
                const int oi = sm.red.i[t + s];
                if (ov > sm.red.v[t] || (ov == sm.red.v[t] && oi < sm.red.i[t])) {
                    sm.red.v[t] = ov;
                    sm.red.i[t] = oi;
                }
            }
            __syncthreads();
        }
        if (t == 0) {
            bi = sm.red.i[0];
            H->search_idx = INT_MAX;
            H->cand_idx = bi;
            // exact check of the FP32 choice
            bool ok = false;
            if (bi >= 0 && bi < A.n) {
                float4 p = load_input(A, bi);
                const float a[3] = {H->pa.x, H->pa.y, H->pa.z};
                const float b[3] = {H->pb.x, H->pb.y, H->pb.z};
                const float c[3] = {H->pc.x, H->pc.y, H->pc.z};
                float q[3] = {p.x, p.y, p.z};
                ok = step == 1 ? !collinear3_exact(a, b, q) : orient3d_exact_sign(a, b, c, q) != 0;
            }
            H->cand_ok = ok;
        }
        __syncthreads();
    }
}

__device__ void simplex_take(const Params3 &A, int step)
{
    Hdr3 *H = A.hdr;
    if (threadIdx.x != 0) return;
    int i = H->cand_ok ? H->cand_idx : H->search_idx;
    if (i == INT_MAX || i < 0) {
        set_status(H, QH_ERR_DEGENERATE);
        return;
    }
    float4 p = load_input(A, i);
    if (step == 1) H->pc = p;
    else H->pd = p;
}

// One thread: the tetrahedron (a, b, c, d) as facets base..base+3, oriented
// with the opposite vertex strictly inside, their neighbours, and the cone
// record of the cloud's pseudo facet.
__device__ void build_tetra_at(const Params3 &A, int base, const float4 *t, int pseudo)
{
    for (int o = 0; o < 4; o++) {
        int k[3], m = 0;
        for (int j = 0; j < 4; j++)
            if (j != o) k[m++] = j;
        float pa[3] = {t[k[0]].x, t[k[0]].y, t[k[0]].z};
        float pb[3] = {t[k[1]].x, t[k[1]].y, t[k[1]].z};
        float pc[3] = {t[k[2]].x, t[k[2]].y, t[k[2]].z};
        float po[3] = {t[o].x, t[o].y, t[o].z};
        if (orient3d_exact_sign(pa, pb, pc, po) > 0) {
            int s = k[1];
            k[1] = k[2];
            k[2] = s;
        }
        Fac3 f;
        for (int j = 0; j < 3; j++) {
            f.p[3 * j + 0] = t[k[j]].x;
            f.p[3 * j + 1] = t[k[j]].y;
            f.p[3 * j + 2] = t[k[j]].z;
            f.v[j] = __float_as_int(t[k[j]].w);
        }
        f.nb[0] = f.nb[1] = f.nb[2] = -1;
        f.alive = 1;
        A.fac[base + o] = f;
        A.plane[base + o] = make_plane3(f.p, f.p + 3, f.p + 6);
        Acc3 z = {};
        A.acc[base + o] = z;
        A.claim[0][base + o] = 0ull;
        A.claim[1][base + o] = 0ull;
        A.taken[base + o] = 0;
        A.big_mark[base + o] = -1;
    }
    for (int i = 0; i < 4; i++)
        for (int e = 0; e < 3; e++) {
            int u = A.fac[base + i].v[e], v = A.fac[base + i].v[(e + 1) % 3];
            for (int j = 0; j < 4; j++) {
                if (j == i) continue;
                for (int g = 0; g < 3; g++)
                    if (A.fac[base + j].v[g] == v && A.fac[base + j].v[(g + 1) % 3] == u)
                        A.fac[base + i].nb[e] = base + j;
            }
        }
    A.cone[pseudo] = make_int4(base, 4, -1, 0);
}

// Four dead facets (a cloud without a tetrahedron) and an empty cone.
__device__ void dead_tetra_at(const Params3 &A, int base, int pseudo)
{
    for (int o = 0; o < 4; o++) {
        Fac3 f = {};
        f.nb[0] = f.nb[1] = f.nb[2] = base + o;
        A.fac[base + o] = f;
        A.plane[base + o] = make_plane3(f.p, f.p + 3, f.p + 6);
        Acc3 z = {};
        A.acc[base + o] = z;
        A.claim[0][base + o] = 0ull;
        A.claim[1][base + o] = 0ull;
        A.taken[base + o] = 0;
        A.big_mark[base + o] = -1;
    }
    A.cone[pseudo] = make_int4(0, 0, -1, 0);
}

// Block 0 thread 0, single cloud: facets 0..3.
__device__ void build_tetra(const Params3 &A)
{
    Hdr3 *H = A.hdr;
    if (threadIdx.x != 0) return;
    const float4 t[4] = {H->pa, H->pb, H->pc, H->pd};
    build_tetra_at(A, 0, t, A.fcap);
    H->fcount = 4;
    H->hull_vertices = 4;
}

// ---------------------------------------------------------------- first polytope
// Direction k (0 <= k < kDirs) of the first polytope: the k-th non-zero
// vector of {-1, 0, 1}^3.
__device__ __forceinline__ void dir_of(int k, int &dx, int &dy, int &dz)
{
    const int i = k < 13 ? k : k + 1;
    dx = i / 9 - 1;
    dy = (i / 3) % 3 - 1;
    dz = i % 3 - 1;
}

// All CTAs: the extreme point of every direction (largest FP32 dot product,
// lowest index on ties; -0 counted as +0 so that copies of one location
// tie), kept in H->dirkey by one atomic per CTA and direction.  Which point
// each direction finds only shapes the first polytope: every point of it is
// an input point, so the hull does not depend on it.
// The directions the first polytope uses: all 26 (option 1), the 6 axes and
// the 8 diagonals (option 2), or the 6 axes (option 3).
constexpr int kNumDirs = kInitDirs == 1 ? kDirs : (kInitDirs == 3 ? 6 : 14);
__device__ __forceinline__ void used_dir(int k, int &dx, int &dy, int &dz)
{
    if (kInitDirs == 1) {
        dir_of(k, dx, dy, dz);
        return;
    }
    if (k < 6) {  // the axes
        dx = k / 2 == 0 ? (k & 1 ? -1 : 1) : 0;
        dy = k / 2 == 1 ? (k & 1 ? -1 : 1) : 0;
        dz = k / 2 == 2 ? (k & 1 ? -1 : 1) : 0;
    } else {      // the diagonals
        const int b = k - 6;
        dx = b & 1 ? -1 : 1;
        dy = b & 2 ? -1 : 1;
        dz = b & 4 ? -1 : 1;
    }
}

__device__ void dir_extrema3d(const Params3 &A, SmemAll3 &sm, int bid, int nb)
{
    Hdr3 *H = A.hdr;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    constexpr int kG = (kNumDirs + kDirGroup - 1) / kDirGroup;  // keys per pass: kDirGroup
#pragma unroll
    for (int g = 0; g < kG; g++) {
        const int k0 = kDirGroup * g, nk = kNumDirs - k0 < kDirGroup ? kNumDirs - k0 : kDirGroup;
        unsigned long long best[kDirGroup];
#pragma unroll
        for (int k = 0; k < kDirGroup; k++) best[k] = 0ull;
        for (long long i = (long long)bid * blockDim.x + threadIdx.x; i < A.n;
             i += (long long)nb * blockDim.x) {
            const float4 p = load_input(A, i);
            const unsigned lo = 0xffffffffu - (unsigned)i;
#pragma unroll
            for (int k = 0; k < kDirGroup; k++) {
                if (k >= nk) break;
                int dx, dy, dz;
                used_dir(k0 + k, dx, dy, dz);
                float sdot = 0.0f;
                if (dx) sdot += dx > 0 ? p.x : -p.x;
                if (dy) sdot += dy > 0 ? p.y : -p.y;
                if (dz) sdot += dz > 0 ? p.z : -p.z;
                sdot += 0.0f;
                const unsigned long long key = ((unsigned long long)ord_f32(sdot) << 32) | lo;
                best[k] = key > best[k] ? key : best[k];
            }
        }
#pragma unroll
        for (int k = 0; k < kDirGroup; k++) {
            if (k >= nk) break;
            unsigned long long b = best[k];
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long t = __shfl_xor_sync(0xffffffffu, b, o);
                b = t > b ? t : b;
            }
            if (lane == 0) sm.init.key[warp][k] = b;
        }
        __syncthreads();
        if (threadIdx.x < nk) {
            unsigned long long b = 0ull;
            for (int w = 0; w < nwarp; w++) {
                const unsigned long long t = sm.init.key[w][threadIdx.x];
                b = t > b ? t : b;
            }
            if (b) atomicMax(&H->dirkey[k0 + threadIdx.x], b);
        }
        __syncthreads();
    }
}

// Warp 0 of CTA 0, after the tetrahedron: insert the directions' extreme
// points one at a time (Barber et al.'s step with exact signs: the facets
// the point is strictly above, their horizon edges, one new facet per edge
// through the point), then write the polytope's facets to slots 0 .. F-1
// with their neighbours, and give the cloud's pseudo facet the cone of all
// of them, so the first assignment sends every point to the first facet it
// is strictly above.  A point on or inside the current polytope is skipped.
__device__ void expand_initial(const Params3 &A, SmemAll3 &sm)
{
    Hdr3 *H = A.hdr;
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    const unsigned lt = (1u << lane) - 1u;
    SmemInit &S = sm.init;
    // vertices get slots 0 .. nv-1 (point index in S.vid); a directed edge
    // (slot a -> slot b) of a facet that stays is bit b of S.emask[a]
    if (lane < 4) {
        const Fac3 F = A.fac[lane];
        for (int j = 0; j < 9; j++) S.p[lane][j] = F.p[j];
        for (int j = 0; j < 3; j++) S.v[lane][j] = F.v[j];
        S.vid[lane] = F.v[0];
    }
    __syncwarp();
    if (lane == 0) {
        // the four vertices: facet 0's three and the one facet 1 adds
        S.vid[0] = S.v[0][0];
        S.vid[1] = S.v[0][1];
        S.vid[2] = S.v[0][2];
        int o = S.v[1][0];
        for (int t = 0; t < 3; t++) {
            const int c = S.v[1][t];
            if (c != S.vid[0] && c != S.vid[1] && c != S.vid[2]) o = c;
        }
        S.vid[3] = o;
        // from here on a facet's vertices are slots
        for (int j = 0; j < 4; j++)
            for (int e = 0; e < 3; e++) {
                int r = 0;
                for (int t = 0; t < 4; t++)
                    if (S.vid[t] == S.v[j][e]) r = t;
                S.v[j][e] = r;
            }
        S.nf = 4;
        S.nv = 4;
    }
    __syncwarp();
    for (int k = 0; k < kNumDirs; k++) {
        const unsigned long long key = *(volatile unsigned long long *)&H->dirkey[k];
        const int qi = (int)(0xffffffffu - (unsigned)(key & 0xffffffffull));
        if (key == 0ull || qi < 0 || qi >= A.n || S.nv >= 32) continue;
        const float4 q4 = load_input(A, qi);
        const float q[3] = {q4.x, q4.y, q4.z};
        const int nf = S.nf;
        int nvis = 0;
        if (lane < 32) S.emask[lane] = 0u;
        __syncwarp();
        for (int j = lane; j < nf; j += 32) {
            const int vis = orient3d_exact_sign(S.p[j], S.p[j] + 3, S.p[j] + 6, q) > 0;
            S.vis[j] = vis;
            nvis += vis;
        }
        nvis = __reduce_add_sync(0xffffffffu, nvis);
        if (nvis == 0) continue;
        // the directed edges of the facets that stay
        for (int j = lane; j < nf; j += 32)
            if (!S.vis[j])
                for (int e = 0; e < 3; e++)
                    atomicOr(&S.emask[S.v[j][e]], 1u << S.v[j][e == 2 ? 0 : e + 1]);
        __syncwarp();
        // horizon edges: an edge of a visible facet whose reverse edge stays
        if (lane == 0) S.ne = 0;
        __syncwarp();
        for (int j = lane; j < nf; j += 32) {
            if (!S.vis[j]) continue;
            for (int e = 0; e < 3; e++) {
                const int e1 = e == 2 ? 0 : e + 1;
                if (!((S.emask[S.v[j][e1]] >> S.v[j][e]) & 1u)) continue;
                const int at = atomicAdd(&S.ne, 1);
                if (at >= kInitF) continue;
                S.eu[at] = S.v[j][e];
                S.ev[at] = S.v[j][e1];
                for (int t = 0; t < 3; t++) {
                    S.ep[at][t] = S.p[j][3 * e + t];
                    S.ep[at][3 + t] = S.p[j][3 * e1 + t];
                }
            }
        }
        __syncwarp();
        const int ne = S.ne;
        if (ne > kInitF || nf - nvis + ne > kInitF) continue;  // cannot happen (V <= 32)
        // the facets that stay, compacted in order (a chunk is read before it
        // is written; destinations never pass their sources), then the cone
        int w = 0;
        for (int j0 = 0; j0 < nf; j0 += 32) {
            const int j = j0 + lane;
            const bool keep = j < nf && !S.vis[j];
            float pp[9];
            int vv[3];
            if (keep) {
                for (int t = 0; t < 9; t++) pp[t] = S.p[j][t];
                for (int t = 0; t < 3; t++) vv[t] = S.v[j][t];
            }
            const unsigned b = __ballot_sync(0xffffffffu, keep);
            __syncwarp();
            if (keep) {
                const int d = w + __popc(b & lt);
                for (int t = 0; t < 9; t++) S.p[d][t] = pp[t];
                for (int t = 0; t < 3; t++) S.v[d][t] = vv[t];
            }
            w += __popc(b);
            __syncwarp();
        }
        for (int e = lane; e < ne; e += 32) {
            const int d = w + e;
            for (int t = 0; t < 6; t++) S.p[d][t] = S.ep[e][t];
            S.p[d][6] = q[0];
            S.p[d][7] = q[1];
            S.p[d][8] = q[2];
            S.v[d][0] = S.eu[e];
            S.v[d][1] = S.ev[e];
            S.v[d][2] = S.nv;
        }
        __syncwarp();
        if (lane == 0) {
            S.nf = w + ne;
            S.vid[S.nv] = qi;
            S.nv = S.nv + 1;
        }
        __syncwarp();
    }
    // buried vertices keep their slots (no facet uses them); the neighbours
    // from the edge slots
    const int nf = S.nf;
    for (int j = lane; j < nf; j += 32)
        for (int e = 0; e < 3; e++) S.eid[S.v[j][e]][S.v[j][e == 2 ? 0 : e + 1]] = j;
    __syncwarp();
    for (int j = lane; j < nf; j += 32) {
        Fac3 f;
        for (int t = 0; t < 9; t++) f.p[t] = S.p[j][t];
        for (int e = 0; e < 3; e++) {
            f.v[e] = S.vid[S.v[j][e]];
            f.nb[e] = S.eid[S.v[j][e == 2 ? 0 : e + 1]][S.v[j][e]];  // the facet with the reverse edge
        }
        f.alive = 1;
        A.fac[j] = f;
        A.plane[j] = make_plane3(f.p, f.p + 3, f.p + 6);
        Acc3 z = {};
        A.acc[j] = z;
        A.claim[0][j] = 0ull;
        A.claim[1][j] = 0ull;
        A.taken[j] = 0;
        A.big_mark[j] = -1;
    }
    if (lane == 0) {
        A.cone[A.fcap] = make_int4(0, nf, -1, 0);
        H->fcount = nf;
        H->hull_vertices = S.nv;
    }
}

// ---------------------------------------------------------------- clouds
__device__ __forceinline__ int cloud_start(const Params3 &A, int c)
{
    return A.cloud_off ? (int)A.cloud_off[c] : (c == 0 ? 0 : A.n);
}

// Cloud of point v: the last cloud starting at or before v.
__device__ __forceinline__ int cloud_of(const Params3 &A, int v)
{
    if (!A.cloud_off) return 0;
    int lo = 0, hi = A.ncloud - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (A.cloud_off[mid] <= v) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Block-wide reductions over a cloud for its initial simplex.
__device__ void block_lex_extrema(const Params3 &A, SmemAll3 &sm, int lo, int hi, float4 &mn,
                                  float4 &mx, bool &bad)
{
    float4 a = make_float4(INFINITY, INFINITY, INFINITY, __int_as_float(INT_MAX));
    float4 b = make_float4(-INFINITY, -INFINITY, -INFINITY, __int_as_float(INT_MAX));
    int nf = 0;
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        float4 p = load_input(A, i);
        p.x = canon0(p.x);
        p.y = canon0(p.y);
        p.z = canon0(p.z);
        nf |= !(isfinite(p.x) && isfinite(p.y) && isfinite(p.z));
        if (lex_less(p, a)) a = p;
        if (lex_greater_lowidx(p, b)) b = p;
    }
    bad = __syncthreads_or(nf);
    sm.red.a[threadIdx.x] = a;
    sm.red.b[threadIdx.x] = b;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            if (lex_less(sm.red.a[threadIdx.x + s], sm.red.a[threadIdx.x]))
                sm.red.a[threadIdx.x] = sm.red.a[threadIdx.x + s];
            if (lex_greater_lowidx(sm.red.b[threadIdx.x + s], sm.red.b[threadIdx.x]))
                sm.red.b[threadIdx.x] = sm.red.b[threadIdx.x + s];
        }
        __syncthreads();
    }
    mn = sm.red.a[0];
    mx = sm.red.b[0];
    __syncthreads();
}

// Farthest point of [lo, hi) from the line ab (kind 0) or the plane abc
// (kind 1), FP32 magnitude, lowest index on ties; then the exact check that
// it is off the line / plane, and if not, the lowest-index point that is.
// Returns the point index or -1 (all points on the line / plane).
__device__ int block_next_vertex(const Params3 &A, SmemAll3 &sm, int lo, int hi, const float *a,
                                 const float *b, const float *c, int kind)
{
    float best = -1.0f;
    int bi = INT_MAX;
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const float4 p = load_input(A, i);
        float v;
        if (kind == 0) {
            const float ux = b[0] - a[0], uy = b[1] - a[1], uz = b[2] - a[2];
            const float wx = p.x - a[0], wy = p.y - a[1], wz = p.z - a[2];
            const float cx = uy * wz - uz * wy, cy = uz * wx - ux * wz, cz = ux * wy - uy * wx;
            v = cx * cx + cy * cy + cz * cz;
        } else {
            const float q[3] = {p.x, p.y, p.z};
            float d, e;
            orient3d_value<QH_PRED_F32>(a, b, c, q, d, e);
            v = fabsf(d);
        }
        if (v > best || (v == best && i < bi)) {
            best = v;
            bi = i;
        }
    }
    sm.red.v[threadIdx.x] = best;
    sm.red.i[threadIdx.x] = bi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const float ov = sm.red.v[threadIdx.x + s];
            const int oi = sm.red.i[threadIdx.x + s];
            if (ov > sm.red.v[threadIdx.x] ||
                (ov == sm.red.v[threadIdx.x] && oi < sm.red.i[threadIdx.x])) {
                sm.red.v[threadIdx.x] = ov;
                sm.red.i[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    const int cand = sm.red.i[0];
    __syncthreads();
    if (threadIdx.x == 0) {
        bool ok = false;
        if (cand >= lo && cand < hi) {
            const float4 p = load_input(A, cand);
            const float q[3] = {p.x, p.y, p.z};
            ok = kind == 0 ? !collinear3_exact(a, b, q) : orient3d_exact_sign(a, b, c, q) != 0;
        }
        sm.red.flag = ok ? cand : INT_MAX;
    }
    __syncthreads();
    int r = sm.red.flag;
    if (r == INT_MAX) {
        // exact search (rare: the FP32 choice was degenerate)
        for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            const float4 p = load_input(A, i);
            const float q[3] = {p.x, p.y, p.z};
            const bool ok =
                kind == 0 ? !collinear3_exact(a, b, q) : orient3d_exact_sign(a, b, c, q) != 0;
            if (ok) atomicMin(&sm.red.flag, i);
        }
        __syncthreads();
        r = sm.red.flag;
    }
    __syncthreads();
    return r == INT_MAX ? -1 : r;
}

// ---------------------------------------------------------------- small-cloud route
// Below a size chosen by the autotuner (qh_opts.small_cloud) a cloud is
// cheaper to hull whole with one warp than to run through the segmented
// iterations (the switchover point the paper leaves to future work, Section
// 6).  Clouds of 4..small_cloud points get that route during the setup.
__device__ __forceinline__ bool is_small_cloud(const Params3 &A, int c)
{
    const int nc = cloud_start(A, c + 1) - cloud_start(A, c);
    return A.small_cloud > 0 && nc >= 4 && nc <= A.small_cloud;
}

// Exact: p strictly above facet g.
__device__ __forceinline__ bool above3(const Params3 &A, int g, const float *p, unsigned &fb)
{
    float d, e;
    facet_value<QH_PRED_F32>(A, g, p, d, e);
    if (d > e) return true;
    if (-d > e) return false;
    const Fac3 &G = A.fac[g];
    return orient3d_sign<QH_PRED_F32>(d, e, G.p, G.p + 3, G.p + 6, p, fb) > 0;
}

// One warp, one cloud: Quickhull inserting one apex at a time (Barber et
// al.): a tetrahedron of the cloud's extreme points (slots 4c..4c+3, exact
// tests), every point to the first facet strictly below it, then until no
// point is outside: the lowest outside point's facet, its farthest point
// (exact comparisons, lowest index on ties), every alive facet of the cloud
// strictly below it (the visible region of a convex polytope is connected,
// so no search is needed), its horizon, the cone (one facet per horizon
// edge, linked around the apex), and the visible facets' points to the first
// cone facet strictly below them.  The facets land in the global table like
// every other cloud's; the cloud's pseudo facet gets an empty cone, so the
// segmented passes drop its points.  Scratch borrowed while the pools are
// idle: the cloud's facet list in its candidate-list slice (kVCap per
// point), horizon edges in its neighbour slice (kNCap per point), each
// point's facet in code[].x.
__device__ void small_hull_warp(const Params3 &A, int c, unsigned &fb)
{
    Hdr3 *H = A.hdr;
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    const int lo = cloud_start(A, c), hi = cloud_start(A, c + 1), nc = hi - lo;
    const int base4 = 4 * c, pseudo = A.fcap + c;
    int *fl = A.vpool + (size_t)lo * kVCap;
    int *hz = A.npool + (size_t)lo * kNCap;
    const long long fl_cap = (long long)kVCap * nc, hz_cap = (long long)kNCap * nc;
    auto fail = [&](int st) {
        if (lane == 0) {
            dead_tetra_at(A, base4, pseudo);
            A.cloud_status[c] = st;
        }
        __syncwarp();
    };
    // ---- extrema (lexicographic, lowest index) and finiteness
    float4 mn = make_float4(INFINITY, INFINITY, INFINITY, __int_as_float(INT_MAX));
    float4 mx = make_float4(-INFINITY, -INFINITY, -INFINITY, __int_as_float(INT_MAX));
    bool bad = false;
    for (int i = lo + lane; i < hi; i += 32) {
        float4 p = load_input(A, i);
        p.x = canon0(p.x);
        p.y = canon0(p.y);
        p.z = canon0(p.z);
        bad |= !(isfinite(p.x) && isfinite(p.y) && isfinite(p.z));
        if (lex_less(p, mn)) mn = p;
        if (lex_greater_lowidx(p, mx)) mx = p;
    }
    if (__any_sync(0xffffffffu, bad)) return fail(QH_ERR_NONFINITE);
    for (int o = 16; o > 0; o >>= 1) {
        float4 a, b;
        a.x = __shfl_xor_sync(0xffffffffu, mn.x, o);
        a.y = __shfl_xor_sync(0xffffffffu, mn.y, o);
        a.z = __shfl_xor_sync(0xffffffffu, mn.z, o);
        a.w = __shfl_xor_sync(0xffffffffu, mn.w, o);
        b.x = __shfl_xor_sync(0xffffffffu, mx.x, o);
        b.y = __shfl_xor_sync(0xffffffffu, mx.y, o);
        b.z = __shfl_xor_sync(0xffffffffu, mx.z, o);
        b.w = __shfl_xor_sync(0xffffffffu, mx.w, o);
        if (lex_less(a, mn)) mn = a;
        if (lex_greater_lowidx(b, mx)) mx = b;
    }
    if (mn.x == mx.x && mn.y == mx.y && mn.z == mx.z) return fail(QH_ERR_DEGENERATE);
    float4 t[4] = {mn, mx, mn, mn};
    // ---- c: lowest index off the line ab; d: lowest index off the plane abc
    for (int step = 0; step < 2; step++) {
        const float a[3] = {t[0].x, t[0].y, t[0].z}, b[3] = {t[1].x, t[1].y, t[1].z};
        const float cc[3] = {t[2].x, t[2].y, t[2].z};
        int first = INT_MAX;
        for (int i = lo + lane; i < hi && first == INT_MAX; i += 32) {
            const float4 p4 = load_input(A, i);
            const float q[3] = {p4.x, p4.y, p4.z};
            const bool off =
                step == 0 ? !collinear3_exact(a, b, q) : orient3d_exact_sign(a, b, cc, q) != 0;
            if (off) first = i;
        }
        first = (int)__reduce_min_sync(0xffffffffu, (unsigned)first);
        if (first == INT_MAX) return fail(QH_ERR_DEGENERATE);
        t[2 + step] = load_input(A, first);
    }
    if (lane == 0) {
        build_tetra_at(A, base4, t, pseudo);
        A.cone[pseudo] = make_int4(0, 0, -1, 0);  // the segmented passes drop its points
        atomicAdd(&H->hull_vertices, 4);
    }
    if (lane < 4) fl[lane] = base4 + lane;
    int nf = 4;
    __syncwarp();
    for (int i = lo + lane; i < hi; i += 32) {
        const float4 p4 = load_input(A, i);
        const int idx = __float_as_int(p4.w);
        int g = -1;
        bool vtx = false;
        for (int k = 0; k < 4; k++) vtx |= idx == __float_as_int(t[k].w);
        const float p[3] = {p4.x, p4.y, p4.z};
        for (int k = 0; k < 4 && g < 0 && !vtx; k++)
            if (above3(A, base4 + k, p, fb)) g = base4 + k;
        A.code[i].x = g;
    }
    __syncwarp();
    // ---- insertions (each consumes its apex: at most nc)
    for (int it = 1; it <= nc; it++) {
        int cand = INT_MAX;
        for (int i = lo + lane; i < hi; i += 32)
            if (A.code[i].x >= 0) {
                cand = i;
                break;
            }
        cand = (int)__reduce_min_sync(0xffffffffu, (unsigned)cand);
        if (cand == INT_MAX) break;
        const int f = A.code[cand].x;
        const Fac3 F = A.fac[f];
        // farthest point of f's outside set
        int best = -1;
        float bx = 0.f, by = 0.f, bz = 0.f;
        for (int i = lo + lane; i < hi; i += 32) {
            if (A.code[i].x != f) continue;
            const float4 p4 = load_input(A, i);
            if (best >= 0) {
                const float p[3] = {p4.x, p4.y, p4.z}, q[3] = {bx, by, bz};
                const int sgn = cmp_dist3_exact_sign(F.p, F.p + 3, F.p + 6, p, q);
                if (!(sgn > 0 || (sgn == 0 && i < best))) continue;
            }
            best = i;
            bx = p4.x;
            by = p4.y;
            bz = p4.z;
        }
        for (int o = 16; o > 0; o >>= 1) {
            const int ob = __shfl_xor_sync(0xffffffffu, best, o);
            const float ox = __shfl_xor_sync(0xffffffffu, bx, o);
            const float oy = __shfl_xor_sync(0xffffffffu, by, o);
            const float oz = __shfl_xor_sync(0xffffffffu, bz, o);
            if (ob < 0) continue;
            bool take = best < 0;
            if (!take) {
                const float p[3] = {ox, oy, oz}, q[3] = {bx, by, bz};
                const int sgn = cmp_dist3_exact_sign(F.p, F.p + 3, F.p + 6, p, q);
                take = sgn > 0 || (sgn == 0 && ob < best);
            }
            if (take) {
                best = ob;
                bx = ox;
                by = oy;
                bz = oz;
            }
        }
        const float4 q4 = load_input(A, best);
        const float q[3] = {q4.x, q4.y, q4.z};
        const int qi = best;
        const unsigned long long key = ((unsigned long long)(unsigned)(c + 1) << 32) | (unsigned)it;
        // visible: every alive facet of the cloud strictly below q
        for (int j = lane; j < nf; j += 32) {
            const int g = fl[j];
            if (A.fac[g].alive && above3(A, g, q, fb)) A.claim[1][g] = key;
        }
        __syncwarp();
        // horizon edges: edges of visible facets whose neighbour is not visible
        int nh = 0;
        for (int j0 = 0; j0 < nf; j0 += 32) {
            const int j = j0 + lane;
            unsigned hm = 0;
            int g = -1;
            if (j < nf) {
                g = fl[j];
                if (A.claim[1][g] == key)
                    for (int k = 0; k < 3; k++)
                        if (A.claim[1][A.fac[g].nb[k]] != key) hm |= 1u << k;
            }
            const int cnt = __popc(hm);
            int inc = cnt;
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += v;
            }
            const int pos = nh + inc - cnt;
            int w = 0;
            for (int k = 0; k < 3; k++)
                if (hm & (1u << k)) {
                    if (pos + w < hz_cap) hz[pos + w] = g * 3 + k;
                    w++;
                }
            nh += __shfl_sync(0xffffffffu, inc, 31);
        }
        int base = 0;
        if (lane == 0) base = atomicAdd(&H->fcount, nh);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (nh > hz_cap || base + nh > A.fcap || nf + nh > fl_cap) {
            if (lane == 0) set_status(H, QH_ERR_CAPACITY);
            return fail(QH_ERR_CAPACITY);
        }
        __syncwarp();
        // cone facets, one per horizon edge (u, v, q), the outside
        // neighbour relinked
        for (int j = lane; j < nh; j += 32) {
            const int hf = hz[j] / 3, k = hz[j] - 3 * (hz[j] / 3), k1 = (k + 1) % 3;
            const Fac3 &G0 = A.fac[hf];
            Fac3 C;
            C.p[0] = G0.p[3 * k + 0]; C.p[1] = G0.p[3 * k + 1]; C.p[2] = G0.p[3 * k + 2];
            C.p[3] = G0.p[3 * k1 + 0]; C.p[4] = G0.p[3 * k1 + 1]; C.p[5] = G0.p[3 * k1 + 2];
            C.p[6] = q4.x; C.p[7] = q4.y; C.p[8] = q4.z;
            C.v[0] = G0.v[k];
            C.v[1] = G0.v[k1];
            C.v[2] = qi;
            const int g = G0.nb[k];
            C.nb[0] = g;
            C.nb[1] = -1;
            C.nb[2] = -1;
            C.alive = 1;
            A.fac[base + j] = C;
            A.plane[base + j] = make_plane3(C.p, C.p + 3, C.p + 6);
            Acc3 z = {};
            A.acc[base + j] = z;
            A.claim[0][base + j] = 0ull;
            A.claim[1][base + j] = 0ull;
            A.taken[base + j] = 0;
            A.big_mark[base + j] = -1;
            Fac3 &G = A.fac[g];
            for (int tt = 0; tt < 3; tt++)
                if (G.nb[tt] == hf) G.nb[tt] = base + j;
        }
        __syncwarp();
        // around q: edge (v, q) meets the cone facet whose horizon edge
        // starts at v, edge (q, u) the one whose horizon edge ends at u
        for (int j = lane; j < nh; j += 32) {
            const int u = A.fac[base + j].v[0], v = A.fac[base + j].v[1];
            int n1 = -1, n2 = -1;
            for (int i = 0; i < nh; i++) {
                const int du = A.fac[base + i].v[0], dv = A.fac[base + i].v[1];
                if (du == v) n1 = base + i;
                if (dv == u) n2 = base + i;
            }
            A.fac[base + j].nb[1] = n1;
            A.fac[base + j].nb[2] = n2;
        }
        for (int j = lane; j < nf; j += 32) {
            const int g = fl[j];
            if (A.claim[1][g] == key) A.fac[g].alive = 0;
        }
        for (int j = lane; j < nh; j += 32) fl[nf + j] = base + j;
        nf += nh;
        if (lane == 0) atomicAdd(&H->hull_vertices, 1);
        __syncwarp();
        // the visible facets' points: to the first cone facet strictly below
        for (int i = lo + lane; i < hi; i += 32) {
            const int g = A.code[i].x;
            if (g < 0 || A.claim[1][g] != key) continue;
            int tg = -1;
            if (i != qi) {
                const float4 p4 = load_input(A, i);
                const float p[3] = {p4.x, p4.y, p4.z};
                for (int jj = 0; jj < nh && tg < 0; jj++)
                    if (above3(A, base + jj, p, fb)) tg = base + jj;
            }
            A.code[i].x = tg;
        }
        __syncwarp();
    }
    if (lane == 0) A.cloud_status[c] = QH_OK;
    __syncwarp();
}

// Every warp takes small clouds from a queue (the others are init_clouds').
__device__ void small_clouds(const Params3 &A)
{
    Hdr3 *H = A.hdr;
    const int lane = threadIdx.x & 31;
    unsigned fb = 0;
    for (;;) {
        int c = 0;
        if (lane == 0) c = atomicAdd(&H->next_small, 1);
        c = __shfl_sync(0xffffffffu, c, 0);
        if (c >= A.ncloud) break;
        if (is_small_cloud(A, c)) small_hull_warp(A, c, fb);
    }
    const unsigned f = __reduce_add_sync(0xffffffffu, fb);
    if (lane == 0 && f) atomicAdd(&H->fallbacks, (unsigned long long)f);
}

// One block per cloud: its initial simplex as facets 4c..4c+3 (dead facets
// and a per-cloud status when the cloud does not span 3D or holds a
// non-finite coordinate).
__device__ void init_clouds(const Params3 &A, SmemAll3 &sm, int bid, int nb)
{
    Hdr3 *H = A.hdr;
    (void)bid;
    (void)nb;
    for (;;) {
        // clouds from a queue: a block that drew a large cloud does not hold
        // back the small ones
        __syncthreads();
        if (threadIdx.x == 0) sm.red.flag = atomicAdd(&H->next_cloud, 1);
        __syncthreads();
        const int c = sm.red.flag;
        if (c >= A.ncloud) break;
        if (is_small_cloud(A, c)) continue;  // hulled whole by one warp (small_clouds)
        const int lo = cloud_start(A, c), hi = cloud_start(A, c + 1);
        const int base = 4 * c, pseudo = A.fcap + c;
        int st = QH_OK;
        float4 t[4];
        if (hi - lo == 0) {
            st = -1;  // empty cloud: no faces, status OK
        } else if (hi - lo < 4) {
            st = QH_ERR_DEGENERATE;
        } else {
            bool bad;
            block_lex_extrema(A, sm, lo, hi, t[0], t[1], bad);
            if (bad) st = QH_ERR_NONFINITE;
            else if (t[0].x == t[1].x && t[0].y == t[1].y && t[0].z == t[1].z)
                st = QH_ERR_DEGENERATE;
        }
        for (int step = 0; step < 2 && st == QH_OK; step++) {
            const float a[3] = {t[0].x, t[0].y, t[0].z};
            const float b[3] = {t[1].x, t[1].y, t[1].z};
            const float cc[3] = {t[2].x, t[2].y, t[2].z};
            const int i = block_next_vertex(A, sm, lo, hi, a, b, cc, step);
            if (i < 0) st = QH_ERR_DEGENERATE;
            else t[2 + step] = load_input(A, i);
        }
        if (threadIdx.x == 0) {
            if (st == QH_OK) {
                build_tetra_at(A, base, t, pseudo);
                atomicAdd(&H->hull_vertices, 4);
            } else {
                dead_tetra_at(A, base, pseudo);
            }
            A.cloud_status[c] = st < 0 ? QH_OK : st;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- S: select
// One thread per segment (candidate): visible-set BFS from its facet with
// exact tests.  V: visible facets, N: their non-visible neighbours.  A
// candidate whose lists fit claims its visible facets for round 0 at once.
template <int MODE>
__device__ void select3d(const Params3 &A, int par, int iter, int bid, int nb)
{
    Hdr3 *H = A.hdr;
    const int ne = (int)(*(volatile unsigned long long *)&H->tab[par] >> 32);
    const Ent3 *ent = A.ent[par];
    unsigned fallbacks = 0;
    int nact = 0;
    const int per = (ne + nb - 1) / nb;
    const int e_lo = min(ne, bid * per), e_hi = min(ne, e_lo + per);
    for (int e = e_lo + threadIdx.x; e < e_hi; e += blockDim.x) {
        const Ent3 en = ent[e];
        const int f0 = en.f;
        const float4 q4 = A.apex[f0];
        const float q[3] = {q4.x, q4.y, q4.z};
        // the lists live in thread-local memory during the search (the
        // membership scans stay in L1) and are stored once at the end
        int V[kVCap], N[kNCap];
        int nv = 1, nn = 0;
        bool over = false;
        V[0] = f0;
        for (int i = 0; i < nv && !over; i++) {
            const int3 nbr = make_int3(A.fac[V[i]].nb[0], A.fac[V[i]].nb[1], A.fac[V[i]].nb[2]);
            for (int k = 0; k < 3 && !over; k++) {
                const int g = k == 0 ? nbr.x : (k == 1 ? nbr.y : nbr.z);
                bool seen = false;
                for (int j = 0; j < nv && !seen; j++) seen = V[j] == g;
                for (int j = 0; j < nn && !seen; j++) seen = N[j] == g;
                if (seen) continue;
                float d, err;
                facet_value<MODE>(A, g, q, d, err);
                bool vis = d > err;
                if (!vis && !(-d > err)) {
                    const Fac3 &G = A.fac[g];
                    vis = orient3d_sign<MODE>(d, err, G.p, G.p + 3, G.p + 6, q, fallbacks) > 0;
                }
                if (vis) {
                    if (nv == kVCap) over = true;
                    else V[nv++] = g;
                } else {
                    if (nn == kNCap) over = true;
                    else N[nn++] = g;
                }
            }
        }
        if (!over) {
            int *Vg = A.vpool + (size_t)e * kVCap;
            int *Ng = A.npool + (size_t)e * kNCap;
            for (int j = 0; j < nv; j++) Vg[j] = V[j];
            for (int j = 0; j < nn; j++) Ng[j] = N[j];
            const unsigned long long mine = claim_key(iter, 0, f0, en.len);
            for (int j = 0; j < nv; j++) atomicMax(&A.claim[0][V[j]], mine);
            nact++;
        }
        A.vn[e] = over ? make_int2(-1, -1) : make_int2(nv, nn);
        A.cstate[e] = over ? 2 : 0;
    }
    // one atomic per CTA on each header count (many candidates: every warp
    // of the grid has some)
    __shared__ unsigned long long s_cnt[2];
    if (threadIdx.x == 0) s_cnt[0] = s_cnt[1] = 0ull;
    __syncthreads();
    unsigned f = __reduce_add_sync(0xffffffffu, fallbacks);
    const int na = __reduce_add_sync(0xffffffffu, nact);
    if ((threadIdx.x & 31) == 0) {
        if (f) atomicAdd(&s_cnt[0], (unsigned long long)f);
        if (na) atomicAdd(&s_cnt[1], (unsigned long long)na);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_cnt[0]) atomicAdd(&H->fallbacks, s_cnt[0]);
        if (s_cnt[1]) atomicAdd(&H->nact[0], (int)s_cnt[1]);
    }
}

// The same search with one warp per candidate, level by level: the lanes
// take the unexpanded visible facets' neighbour slots of a level at once;
// a neighbour met by several lanes is tested by the lowest, one already
// listed is skipped; visible ones join V (expanded at the next level), the
// others N.  The lists (sets) are those of select3d.  Used when there are
// no more candidates than warps in the grid.
template <int MODE>
__device__ void select3d_warp(const Params3 &A, int par, int iter, SmemAll3 &sm, int bid, int nb)
{
    Hdr3 *H = A.hdr;
    const int ne = (int)(*(volatile unsigned long long *)&H->tab[par] >> 32);
    const Ent3 *ent = A.ent[par];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const unsigned lt = lanemask_lt();
    int *V = sm.bfs.V[warp];
    int *N = sm.bfs.N[warp];
    unsigned fallbacks = 0;
    int nact = 0;
    for (int e = bid * nwarp + warp; e < ne; e += nb * nwarp) {
        const Ent3 en = ent[e];
        const int f0 = en.f;
        const float4 q4 = A.apex[f0];
        const float q[3] = {q4.x, q4.y, q4.z};
        if (lane == 0) V[0] = f0;
        int nv = 1, nn = 0, done = 0;
        bool over = false;
        __syncwarp();
        while (done < nv && !over) {
            const int lo = done, cnt = 3 * (nv - done);
            done = nv;
            for (int b0 = 0; b0 < cnt && !over; b0 += 32) {
                const int it = b0 + lane;
                int g = -1;
                if (it < cnt) g = A.fac[V[lo + it / 3]].nb[it - 3 * (it / 3)];
                const unsigned same = __match_any_sync(0xffffffffu, g);
                bool keep = g >= 0 && lane == __ffs(same) - 1;
                for (int j = 0; j < nv && keep; j++) keep = V[j] != g;
                for (int j = 0; j < nn && keep; j++) keep = N[j] != g;
                bool vis = false;
                if (keep) {
                    float d, err;
                    facet_value<MODE>(A, g, q, d, err);
                    vis = d > err;
                    if (!vis && !(-d > err)) {
                        const Fac3 &G = A.fac[g];
                        vis = orient3d_sign<MODE>(d, err, G.p, G.p + 3, G.p + 6, q, fallbacks) > 0;
                    }
                }
                const unsigned bv = __ballot_sync(0xffffffffu, keep && vis);
                const unsigned bn = __ballot_sync(0xffffffffu, keep && !vis);
                if (nv + __popc(bv) > kVCap || nn + __popc(bn) > kNCap) {
                    over = true;
                } else {
                    if (keep && vis) V[nv + __popc(bv & lt)] = g;
                    if (keep && !vis) N[nn + __popc(bn & lt)] = g;
                    nv += __popc(bv);
                    nn += __popc(bn);
                }
                __syncwarp();
            }
        }
        if (!over) {
            int *Vg = A.vpool + (size_t)e * kVCap;
            int *Ng = A.npool + (size_t)e * kNCap;
            const unsigned long long mine = claim_key(iter, 0, f0, en.len);
            for (int j = lane; j < nv; j += 32) {
                Vg[j] = V[j];
                atomicMax(&A.claim[0][V[j]], mine);
            }
            for (int j = lane; j < nn; j += 32) Ng[j] = N[j];
            nact += lane == 0;
        }
        if (lane == 0) {
            A.vn[e] = over ? make_int2(-1, -1) : make_int2(nv, nn);
            A.cstate[e] = over ? 2 : 0;
        }
        __syncwarp();
    }
    unsigned f = __reduce_add_sync(0xffffffffu, fallbacks);
    if (lane == 0 && f) atomicAdd(&H->fallbacks, (unsigned long long)f);
    const int na = __reduce_add_sync(0xffffffffu, nact);
    if (lane == 0 && na) atomicAdd(&H->nact[0], na);
}

// Cone of one winner: horizon edges of V (edges whose neighbour is not in V),
// one facet (u, v, q) per horizon edge, neighbours relinked.  V and N are the
// winner's visible facets and horizon neighbours; hz is scratch for the
// horizon (capacity >= |V| + 2); cl holds the claims of `round`.
__device__ bool build_cone(const Params3 &A, int f0, int len, const int *V, int nv, int *hz,
                           int hcap, int iter, int round, const unsigned long long *cl)
{
    Hdr3 *H = A.hdr;
    const unsigned long long mine = claim_key(iter, round, f0, len);
    const float4 q4 = A.apex[f0];
    const int qi = __float_as_int(q4.w);
    int nh = 0;
    for (int i = 0; i < nv; i++) {
        const Fac3 &F = A.fac[V[i]];
        for (int k = 0; k < 3; k++) {
            int g = F.nb[k];
            if (cl[g] == mine) continue;  // g is in V
            if (nh == hcap) {  // a visible region that is not a disk: cannot happen
                set_status(H, QH_ERR_CAPACITY);
                return false;
            }
            hz[nh++] = V[i] * 3 + k;
        }
    }
    const int base = atomicAdd(&H->fcount, nh);
    if (base + nh > A.fcap) {
        set_status(H, QH_ERR_CAPACITY);
        return false;
    }
    for (int j = 0; j < nh; j++) {
        const int hf = hz[j] / 3;
        const Fac3 &F = A.fac[hf];
        const int k = hz[j] - 3 * hf;
        const int k1 = (k + 1) % 3;
        Fac3 C;
        C.p[0] = F.p[3 * k + 0]; C.p[1] = F.p[3 * k + 1]; C.p[2] = F.p[3 * k + 2];
        C.p[3] = F.p[3 * k1 + 0]; C.p[4] = F.p[3 * k1 + 1]; C.p[5] = F.p[3 * k1 + 2];
        C.p[6] = q4.x; C.p[7] = q4.y; C.p[8] = q4.z;
        C.v[0] = F.v[k];
        C.v[1] = F.v[k1];
        C.v[2] = qi;
        C.nb[0] = F.nb[k];
        C.nb[1] = -1;
        C.nb[2] = -1;
        C.alive = 1;
        A.fac[base + j] = C;
        A.plane[base + j] = make_plane3(C.p, C.p + 3, C.p + 6);
        Acc3 z = {};
        A.acc[base + j] = z;
        A.claim[0][base + j] = 0ull;
        A.claim[1][base + j] = 0ull;
        A.taken[base + j] = 0;
        A.big_mark[base + j] = -1;
        // the horizon neighbour now points at the cone facet
        Fac3 &G = A.fac[F.nb[k]];
        for (int g = 0; g < 3; g++)
            if (G.nb[g] == hf) G.nb[g] = base + j;
    }
    // cone facets around q: edge (v, q) meets the facet whose horizon edge
    // starts at v, edge (q, u) the facet whose horizon edge ends at u
    for (int j = 0; j < nh; j++) {
        Fac3 &C = A.fac[base + j];
        for (int i = 0; i < nh; i++) {
            const Fac3 &D = A.fac[base + i];
            if (D.v[0] == C.v[1]) C.nb[1] = base + i;
            if (D.v[1] == C.v[0]) C.nb[2] = base + i;
        }
    }
    for (int i = 0; i < nv; i++) {
        A.fac[V[i]].alive = 0;
        A.taken[V[i]] = iter;
        A.cone[V[i]] = make_int4(base, nh, qi, iter);
    }
    atomicAdd(&H->hull_vertices, 1);
    atomicAdd(&H->nwin, 1);
    return true;
}

// The cone of winner e (its visible set V of nv facets, all claimed by it
// in this round in cl), in two steps.  cone_horizon: its horizon edges
// (edges of V whose neighbour is not V) into hz, returns their count (a
// visible region that is not a disk cannot happen: QH_ERR_CAPACITY).
// cone_build: with the facet slots base .. base + nh - 1 reserved, one cone
// facet per horizon edge, the horizon neighbours relinked, the cone facets
// linked around the apex by matching edge ends across lanes (shuffles),
// and V deleted.  cone_warp reserves its own slots; the rounds with many
// winners per CTA reserve all of a CTA's slots with one atomic.
__device__ int cone_horizon(const Params3 &A, int f0, int len, const int *V, int nv, int *hz,
                            int iter, int round, const unsigned long long *cl)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    const unsigned long long mine = claim_key(iter, round, f0, len);
    int nh = 0;
    for (int p0 = 0; p0 < 3 * nv; p0 += 32) {
        const int p = p0 + lane;
        bool is_h = false;
        if (p < 3 * nv) {
            const int i = p / 3, k = p - 3 * (p / 3);
            is_h = cl[A.fac[V[i]].nb[k]] != mine;
        }
        const unsigned b = __ballot_sync(0xffffffffu, is_h);
        if (is_h) {
            const int pos = nh + __popc(b & lt);
            if (pos < kNCap) hz[pos] = V[p / 3] * 3 + (p - 3 * (p / 3));
        }
        nh += __popc(b);
    }
    if (nh > kNCap && lane == 0) set_status(A.hdr, QH_ERR_CAPACITY);
    __syncwarp();
    return nh;
}

__device__ void cone_build(const Params3 &A, int e, int f0, const int *V, int nv, const int *hz,
                           int nh, int base, int iter)
{
    const int lane = threadIdx.x & 31;
    const float4 q4 = A.apex[f0];
    const int qi = __float_as_int(q4.w);
    int u[2] = {-1, -1}, w[2] = {-1, -1};
#pragma unroll
    for (int r = 0; r < 2; r++) {
        const int j = lane + 32 * r;
        if (j >= nh) continue;
        const int hf = hz[j] / 3, k = hz[j] - 3 * (hz[j] / 3), k1 = (k + 1) % 3;
        const Fac3 &F = A.fac[hf];
        Fac3 C;
        C.p[0] = F.p[3 * k + 0]; C.p[1] = F.p[3 * k + 1]; C.p[2] = F.p[3 * k + 2];
        C.p[3] = F.p[3 * k1 + 0]; C.p[4] = F.p[3 * k1 + 1]; C.p[5] = F.p[3 * k1 + 2];
        C.p[6] = q4.x; C.p[7] = q4.y; C.p[8] = q4.z;
        C.v[0] = F.v[k];
        C.v[1] = F.v[k1];
        C.v[2] = qi;
        const int g = F.nb[k];
        C.nb[0] = g;
        C.nb[1] = -1;
        C.nb[2] = -1;
        C.alive = 1;
        u[r] = C.v[0];
        w[r] = C.v[1];
        A.fac[base + j] = C;
        A.plane[base + j] = make_plane3(C.p, C.p + 3, C.p + 6);
        Acc3 z = {};
        A.acc[base + j] = z;
        A.claim[0][base + j] = 0ull;
        A.claim[1][base + j] = 0ull;
        A.taken[base + j] = 0;
        A.big_mark[base + j] = -1;
        Fac3 &G = A.fac[g];
        for (int t = 0; t < 3; t++)
            if (G.nb[t] == hf) G.nb[t] = base + j;
    }
    // edge (w, q) of a cone facet meets the cone facet whose horizon edge starts
    // at w; edge (q, u) meets the one whose horizon edge ends at u
    int n1[2] = {-1, -1}, n2[2] = {-1, -1};
    for (int src = 0; src < 32; src++) {
#pragma unroll
        for (int r = 0; r < 2; r++) {
            const int su = __shfl_sync(0xffffffffu, u[r], src);
            const int sw = __shfl_sync(0xffffffffu, w[r], src);
            const int sj = src + 32 * r;
            if (sj >= nh) continue;
#pragma unroll
            for (int mr = 0; mr < 2; mr++) {
                if (u[mr] < 0) continue;
                if (su == w[mr]) n1[mr] = base + sj;
                if (sw == u[mr]) n2[mr] = base + sj;
            }
        }
    }
#pragma unroll
    for (int r = 0; r < 2; r++) {
        const int j = lane + 32 * r;
        if (j >= nh) continue;
        A.fac[base + j].nb[1] = n1[r];
        A.fac[base + j].nb[2] = n2[r];
    }
    for (int i = lane; i < nv; i += 32) {
        A.fac[V[i]].alive = 0;
        A.taken[V[i]] = iter;
        A.cone[V[i]] = make_int4(base, nh, qi, iter);
    }
    if (lane == 0) A.cstate[e] = 1;
}

__device__ void cone_warp(const Params3 &A, int e, int f0, int len, const int *V, int nv,
                          int *hz, int iter, int round, const unsigned long long *cl)
{
    Hdr3 *H = A.hdr;
    const int lane = threadIdx.x & 31;
    const int nh = cone_horizon(A, f0, len, V, nv, hz, iter, round, cl);
    if (nh > kNCap) return;
    int base = 0;
    if (lane == 0) base = atomicAdd(&H->fcount, nh);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base + nh > A.fcap) {
        if (lane == 0) set_status(H, QH_ERR_CAPACITY);
        return;
    }
    cone_build(A, e, f0, V, nv, hz, nh, base, iter);
    if (lane == 0) {
        atomicAdd(&H->hull_vertices, 1);
        atomicAdd(&H->nwin, 1);
    }
}

// Round r of the selection, one phase: every still-active candidate drops out
// if a winner of an earlier round deleted a facet of V or N (their regions
// would touch); else it wins when it owns every facet of V in this round's
// claims (claim[r & 1]) and no facet of N carries a higher claim.  A
// candidate that lost claims its visible facets for round r + 1 in the
// other claim array, which this round's checks and cones never read.  One
// warp checks a candidate (its lanes read the lists and the claims side by
// side) and, when it wins, builds its cone.  Winners of one round touch
// disjoint, non-adjacent facet
// sets (a facet of V_u in N_w would carry u's claim above w's, and one of
// V_w in N_u w's above u's), so their cones commute; a later round's winner
// re-checks against every earlier round's deletions.
__device__ void round3d_warp(const Params3 &A, int par, int iter, int r, bool last, SmemAll3 &sm,
                        int bid, int nb)
{
    (void)sm;
    Hdr3 *H = A.hdr;
    const int ne = (int)(*(volatile unsigned long long *)&H->tab[par] >> 32);
    const Ent3 *ent = A.ent[par];
    const unsigned long long *cl = A.claim[r & 1];
    unsigned long long *cn = A.claim[(r + 1) & 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    int nact = 0;
    // a contiguous chunk of candidates per CTA, one warp per candidate: the
    // lanes read the candidate's lists and their claims side by side, and a
    // winner's warp builds its cone at once
    const int per = (ne + nb - 1) / nb;
    const int e_lo = min(ne, bid * per), e_hi = min(ne, e_lo + per);
    for (int e = e_lo + warp; e < e_hi; e += nwarp) {
        if (A.cstate[e] != 0) continue;
        const int2 c = A.vn[e];
        const int *V = A.vpool + (size_t)e * kVCap;
        int *N = A.npool + (size_t)e * kNCap;
        const Ent3 en = ent[e];
        const unsigned long long mine = claim_key(iter, r, en.f, en.len);
        bool touched = false, lose = false;
        for (int j = lane; j < c.x; j += 32) {
            const int v = V[j];
            touched |= r > 0 && A.taken[v] == iter;
            lose |= cl[v] != mine;
        }
        for (int j = lane; j < c.y; j += 32) {
            const int v = N[j];
            touched |= r > 0 && A.taken[v] == iter;
            lose |= cl[v] >= mine;
        }
        touched = __any_sync(0xffffffffu, touched);
        lose = __any_sync(0xffffffffu, lose);
        if (touched) {
            if (lane == 0) A.cstate[e] = 2;
        } else if (!lose) {
            // the horizon list reuses the candidate's neighbour slice (>= |V| + 2)
            cone_warp(A, e, en.f, en.len, V, c.x, N, iter, r, cl);
        } else if (!last) {
            const unsigned long long next = claim_key(iter, r + 1, en.f, en.len);
            for (int j = lane; j < c.x; j += 32) atomicMax(&cn[V[j]], next);
            nact++;
        }
    }
    if (!last && lane == 0 && nact) atomicAdd(&H->nact[r + 1], nact);
}

// Many candidates per warp of the grid: one thread per candidate (the
// CTA's winners collected in shared memory, their cones built one warp per
// winner); the same decisions as round3d_warp.
__device__ void round3d_thread(const Params3 &A, int par, int iter, int r, bool last, SmemAll3 &sm,
                        int bid, int nb)
{
    Hdr3 *H = A.hdr;
    const int ne = (int)(*(volatile unsigned long long *)&H->tab[par] >> 32);
    const Ent3 *ent = A.ent[par];
    const unsigned long long *cl = A.claim[r & 1];
    unsigned long long *cn = A.claim[(r + 1) & 1];
    const int warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    int nact = 0;
    // a contiguous chunk of candidates per CTA: few candidates spread over
    // every SM (their winners' cones are built by the CTA's warps)
    const int per = (ne + nb - 1) / nb;
    const int e_lo = min(ne, bid * per), e_hi = min(ne, e_lo + per);
    for (int base = e_lo; base < e_hi; base += blockDim.x) {
        if (threadIdx.x == 0) sm.w.n = 0;
        __syncthreads();
        const int e = base + threadIdx.x;
        if (e < e_hi && A.cstate[e] == 0) {
            const int2 c = A.vn[e];
            const int *V = A.vpool + (size_t)e * kVCap;
            const int *N = A.npool + (size_t)e * kNCap;
            const Ent3 en = ent[e];
            const unsigned long long mine = claim_key(iter, r, en.f, en.len);
            // the lists' entries in groups of eight, each group's loads in
            // flight together (after round 0 a touched region decides
            // before a lost claim, so the scan goes on past a loss)
            bool touched = false, win = true;
            for (int j0 = 0; j0 < c.x + c.y && !touched && (win || r > 0); j0 += 8) {
                int g[8];
#pragma unroll
                for (int k = 0; k < 8; k++) {
                    const int j = j0 + k;
                    g[k] = j < c.x ? V[j] : (j < c.x + c.y ? N[j - c.x] : -1);
                }
#pragma unroll
                for (int k = 0; k < 8; k++) {
                    if (g[k] < 0) continue;
                    touched |= r > 0 && A.taken[g[k]] == iter;
                    const unsigned long long ck = cl[g[k]];
                    win &= j0 + k < c.x ? ck == mine : ck < mine;
                }
            }
            if (touched) {
                A.cstate[e] = 2;
            } else {
                if (win) {
                    sm.w.list[atomicAdd(&sm.w.n, 1)] = e;
                } else if (!last) {
                    const unsigned long long next = claim_key(iter, r + 1, en.f, en.len);
                    for (int j = 0; j < c.x; j++) atomicMax(&cn[V[j]], next);
                    nact++;
                }
            }
        }
        __syncthreads();
        const int nw = sm.w.n;
        if (nw > 0) {
            // the winners' horizons (one warp per winner; the horizon list
            // reuses the candidate's neighbour slice, >= |V| + 2), then one
            // reservation of facet slots for all of them, then the cones
            const int lane = threadIdx.x & 31;
            for (int i = warp; i < nw; i += nwarp) {
                const int ew = sm.w.list[i];
                const int nh = cone_horizon(A, ent[ew].f, ent[ew].len, A.vpool + (size_t)ew * kVCap,
                                            A.vn[ew].x, A.npool + (size_t)ew * kNCap, iter, r, cl);
                if (lane == 0) sm.w.nh[i] = nh <= kNCap ? nh : -1;
            }
            __syncthreads();
            const int t = threadIdx.x;
            const int my = t < nw && sm.w.nh[t] > 0 ? sm.w.nh[t] : 0;
            long long tot;
            const long long ex = block_excl_scan64(my, sm.w.wsum, &tot);
            if (t < nw) sm.w.base[t] = (int)ex;
            if (t == 0) {
                const int b0 = atomicAdd(&H->fcount, (int)tot);
                if (b0 + tot > A.fcap) {
                    set_status(H, QH_ERR_CAPACITY);
                    sm.w.base0 = -1;
                } else {
                    sm.w.base0 = b0;
                    atomicAdd(&H->hull_vertices, nw);
                    atomicAdd(&H->nwin, nw);
                }
            }
            __syncthreads();
            const int b0 = sm.w.base0;
            for (int i = warp; i < nw && b0 >= 0; i += nwarp) {
                const int nh = sm.w.nh[i];
                if (nh < 0) continue;
                const int ew = sm.w.list[i];
                cone_build(A, ew, ent[ew].f, A.vpool + (size_t)ew * kVCap, A.vn[ew].x,
                           A.npool + (size_t)ew * kNCap, nh, b0 + sm.w.base[i], iter);
            }
        }
        __syncthreads();  // the list is reused by the next chunk
    }
    if (!last) {
        // one atomic per CTA
        const int na = __syncthreads_count(nact != 0) ? __reduce_add_sync(0xffffffffu, nact) : 0;
        if (threadIdx.x == 0) sm.w.n = 0;
        __syncthreads();
        if ((threadIdx.x & 31) == 0 && na) atomicAdd(&sm.w.n, na);
        __syncthreads();
        if (threadIdx.x == 0 && sm.w.n) atomicAdd(&H->nact[r + 1], sm.w.n);
    }
}

__device__ void round3d(const Params3 &A, int par, int iter, int r, bool last, SmemAll3 &sm,
                        int bid, int nb)
{
    const int ne = (int)(*(volatile unsigned long long *)&A.hdr->tab[par] >> 32);
    if (ne <= kSelWarpMul * nb * (int)(blockDim.x >> 5))
        round3d_warp(A, par, iter, r, last, sm, bid, nb);
    else
        round3d_thread(A, par, iter, r, last, sm, bid, nb);
}

// No winner at all means the highest-priority candidate overflowed its
// fixed-size lists: insert it alone with the large scratch (one thread).
template <int MODE>
__device__ void fallback3d(const Params3 &A, int par, int iter)
{
    Hdr3 *H = A.hdr;
    if (threadIdx.x != 0) return;
    const int ne = (int)(H->tab[par] >> 32);
    const Ent3 *ent = A.ent[par];
    int f0 = INT_MAX, len = 0;
    for (int e = 0; e < ne; e++)
        if (ent[e].len > len || (ent[e].len == len && ent[e].f < f0)) {
            f0 = ent[e].f;
            len = ent[e].len;
        }
    if (f0 == INT_MAX) return;
    const float4 q4 = A.apex[f0];
    const float q[3] = {q4.x, q4.y, q4.z};
    int *V = A.big_v;
    int nv = 1;
    V[0] = f0;
    const unsigned long long mine = claim_key(iter, kRounds, f0, len);
    unsigned long long *cl = A.claim[kRounds & 1];  // round kRounds: above every claim
    cl[f0] = mine;
    unsigned fb = 0;
    for (int i = 0; i < nv; i++) {
        const Fac3 &F = A.fac[V[i]];
        for (int k = 0; k < 3; k++) {
            const int g = F.nb[k];
            if (cl[g] == mine || A.big_mark[g] == iter) continue;
            const Fac3 &G = A.fac[g];
            const float *a, *b, *c;
            fac_pts(G, a, b, c);
            float d, err;
            orient3d_value<MODE>(a, b, c, q, d, err);
            if (orient3d_sign<MODE>(d, err, a, b, c, q, fb) > 0) {
                cl[g] = mine;
                V[nv++] = g;
            } else {
                A.big_mark[g] = iter;
            }
        }
    }
    build_cone(A, f0, len, V, nv, A.big_h, A.fcap, iter, kRounds, cl);
}

// ---------------------------------------------------------------- A: assign
// Target of every live point whose facet was deleted this iteration: the
// first cone facet of its winner that it is strictly above (warp-aggregated
// count, rank and farthest-point key), else discarded (-1); code[v] receives
// (target, rank).  Points of surviving facets are left alone (the scatter
// moves their segments whole), and a tile that meets no deleted facet is
// skipped.  FIRST: the input points against the tetrahedron.
template <int MODE, int ITEMS, bool FIRST>
__device__ void assign3d(const Params3 &A, int par, SmemAll3 &sm, SmemSlots &ss, int bid, int nb)
{
    Hdr3 *H = A.hdr;
    const int L = FIRST ? A.n : (int)(*(volatile unsigned long long *)&H->tab[par] & 0xffffffffull);
    const Ent3 *ent = A.ent[par];
    const float4 *P = A.pts[par];
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    unsigned fallbacks = 0;
    // points per tile: blockDim.x * ITEMS, or fewer for a small table (so
    // that its tiles spread over the SMs)
    const int T = FIRST ? A.tile : *(volatile int *)&H->tile_sz[par];
    const int ntiles = (L + T - 1) / T;
    // Aggregation scope.  Few targets in the phase (the first assignment of
    // one cloud, the early iterations): the CTA's table spans all of its
    // tiles, so the few hot accumulators see one reservation per CTA instead
    // of one per tile.  Many targets: a table per tile, reserved at the
    // tile's end (contention is low, and the table would not hold them).
    const int ntarget = FIRST ? (A.cloud_off ? 4 * A.ncloud : *(volatile int *)&H->fcount)
                              : *(volatile int *)&H->fcount - *(volatile int *)&H->fc_iter[par];
    const bool per_tile = ntarget > (3 * kSlots) / 4;
    auto reset_slots = [&]() {
        for (int i = threadIdx.x; i < kSlots; i += blockDim.x) {
            ss.skey[i] = -1;
            ss.scnt[i] = 0;
            ss.sk1[i] = 0ull;
            ss.so2[i] = 0u;
            ss.sem[i] = 0u;
        }
    };
    // one reservation and key merge per used slot
    auto reserve_slots = [&]() {
        for (int i = threadIdx.x; i < kSlots; i += blockDim.x) {
            const int t = ss.skey[i];
            if (t < 0) continue;
            if (ss.scnt[i] >= (1 << kLocalBits)) set_status(H, QH_ERR_CAPACITY);
            Acc3 &ac = A.acc[t];
            ss.sbase[i] = (int)atomicAdd(&ac.cnt, (unsigned)ss.scnt[i]);
            const unsigned long long k1 = ss.sk1[i];
            const unsigned long long old = atomicMax(&ac.key1, k1);
            const unsigned long long lo2 = old < k1 ? old : k1;
            const unsigned lo_o = (unsigned)(lo2 >> 32);
            const unsigned o2 = ss.so2[i];
            atomicMax(&ac.o2, lo_o > o2 ? lo_o : o2);
            atomicMax(&ac.emax, ss.sem[i]);
        }
    };
    reset_slots();
    for (int tile = bid; tile < ntiles; tile += nb) {
        const int v0 = tile * T, v1 = min(v0 + T, L);
        __syncthreads();
        if (per_tile) {
            reset_slots();
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            if (FIRST) {  // entries = the clouds the tile meets
                const int c0 = cloud_of(A, v0);
                sm.a.e0 = c0;
                sm.a.m = cloud_of(A, v1 - 1) - c0 + 1;
            } else {
                sm.a.e0 = A.tile_ent[par][tile];
                sm.a.m = A.tile_m[par][tile];
            }
        }
        __syncthreads();
        const int e0 = sm.a.e0, m = sm.a.m;
        // FIRST: a tile that meets more clouds than the stage holds (runs of
        // empty clouds) searches the cloud offsets in global memory instead
        // entries: start, and the facet (>= 0) when it was deleted, -1 - facet
        // when it survives
        const bool staged = m <= kMaxTile;
        int dead = FIRST ? 1 : 0;
        for (int i = threadIdx.x; i < m && i < kMaxTile; i += blockDim.x) {
            if (FIRST) {
                sm.a.start[i] = cloud_start(A, e0 + i);
                sm.a.f[i] = A.fcap + e0 + i;
            } else {
                const Ent3 en = ent[e0 + i];
                const bool alive = A.fac[en.f].alive != 0;
                sm.a.start[i] = en.start;
                sm.a.f[i] = alive ? -1 - en.f : en.f;
                dead |= !alive;
            }
        }
        if (!__syncthreads_or(dead)) continue;  // every facet of the tile survives
        // ---- each item's facet (>= 0: deleted, to classify) and point,
        // every load issued before the first classification
        int fit[ITEMS];
        float4 pit[ITEMS];
#pragma unroll
        for (int k = 0; k < ITEMS; k++) {
            const int v = v0 + k * blockDim.x + threadIdx.x;
            fit[k] = -1;
            if (v < v1) {
                int lo = 0, hi = m - 1;
                if (FIRST && !staged) {
                    fit[k] = A.fcap + cloud_of(A, v);
                } else {
                    while (lo < hi) {
                        int mid = (lo + hi + 1) >> 1;
                        if (sm.a.start[mid] <= v) lo = mid;
                        else hi = mid - 1;
                    }
                    fit[k] = sm.a.f[lo];
                }
            }
            if (fit[k] >= 0) pit[k] = FIRST ? load_input(A, v) : P[v];
        }
        // ---- classify; cone targets get a slot of the table (shared hash),
        // or go straight to the global accumulator when it is full
        int tgt[ITEMS], rk[ITEMS], slot[ITEMS];
#pragma unroll
        for (int k = 0; k < ITEMS; k++) {
            const int v = v0 + k * blockDim.x + threadIdx.x;
            const bool valid = v < v1;
            int target = -1, rank = 0, s = -1;
            float d = 0.0f, err = 0.0f;
            int idx = 0;
            bool cone_t = false, f_dead = false;
            if (valid) {
                const int f = fit[k];
                f_dead = f >= 0;
                if (f_dead) {
                    const float4 p4 = pit[k];
                    idx = __float_as_int(p4.w);
                    const float p[3] = {p4.x, p4.y, p4.z};
                    const int4 cn = A.cone[f];
                    bool skip = idx == cn.z;  // the apex itself
                    if (FIRST && cn.y == 4) {
                        // the simplex vertices: facets 0 and 1 of the
                        // tetrahedron hold all four (exact zero tests else)
                        const Fac3 &F0 = A.fac[cn.x], &F1 = A.fac[cn.x + 1];
                        skip = idx == F0.v[0] || idx == F0.v[1] || idx == F0.v[2] ||
                               idx == F1.v[0] || idx == F1.v[1] || idx == F1.v[2];
                    }
                    if (!skip) {
                        // the first cone facet strictly below p: filter values
                        // four facets at a time (independent chains), then in
                        // order, an undecided one settled exactly
                        for (int c0 = 0; c0 < cn.y && !cone_t; c0 += 4) {
                            float dd[4], ee[4];
#pragma unroll
                            for (int j = 0; j < 4; j++) {
                                dd[j] = 0.0f;
                                ee[j] = 0.0f;
                                if (c0 + j < cn.y) facet_value<MODE>(A, cn.x + c0 + j, p, dd[j], ee[j]);
                            }
#pragma unroll
                            for (int j = 0; j < 4; j++) {
                                if (cone_t || c0 + j >= cn.y || -dd[j] > ee[j]) continue;
                                bool pos = dd[j] > ee[j];
                                if (!pos) {
                                    const Fac3 &C = A.fac[cn.x + c0 + j];
                                    // FIRST: the first polytope's vertices are
                                    // input points, each on its facets' planes
                                    // (sign 0 with no exact expansion: its
                                    // FP64 stage has no error bound to pass)
                                    if (FIRST && (idx == C.v[0] || idx == C.v[1] || idx == C.v[2]))
                                        continue;
                                    pos = orient3d_sign<MODE>(dd[j], ee[j], C.p, C.p + 3, C.p + 6, p,
                                                              fallbacks) > 0;
                                }
                                if (pos) {
                                    target = cn.x + c0 + j;
                                    d = dd[j];
                                    err = ee[j];
                                    cone_t = true;
                                }
                            }
                        }
                    }
                }
            }
            const unsigned act = __ballot_sync(0xffffffffu, cone_t);
            if (cone_t) {
                const unsigned grp = __match_any_sync(act, target);
                const int leader = __ffs(grp) - 1;
                const unsigned o = ord_f32(d);
                const unsigned top_o = __reduce_max_sync(grp, o);
                const unsigned cand = (o == top_o) ? (unsigned)idx : 0xffffffffu;
                const unsigned top_i = __reduce_min_sync(grp, cand);
                const unsigned sec = (o == top_o && (unsigned)idx == top_i) ? 0u : o;
                const unsigned sec_o = __reduce_max_sync(grp, sec);
                const unsigned em = __reduce_max_sync(grp, __float_as_uint(err));
                int base = 0;
                if (lane == leader) {
                    // find or insert the target's slot (linear probing, a
                    // bounded number of probes)
                    int h = (int)(((unsigned)target * 0x9E3779B1u) >> (32 - kSlotBits));
                    for (int probe = 0; probe < 16; probe++) {
                        const int prev = atomicCAS(&ss.skey[h], -1, target);
                        if (prev == -1 || prev == target) {
                            s = h;
                            break;
                        }
                        h = (h + 1) & (kSlots - 1);
                    }
                    const unsigned long long k1 =
                        ((unsigned long long)top_o << 32) | (0xffffffffu - top_i);
                    if (s >= 0) {
                        base = atomicAdd(&ss.scnt[s], __popc(grp));
                        const unsigned long long old = atomicMax(&ss.sk1[s], k1);
                        const unsigned long long lo2 = old < k1 ? old : k1;
                        const unsigned lo_o = (unsigned)(lo2 >> 32);
                        atomicMax(&ss.so2[s], lo_o > sec_o ? lo_o : sec_o);
                        atomicMax(&ss.sem[s], em);
                    } else {
                        // table full: straight to the global accumulator
                        Acc3 &ac = A.acc[target];
                        base = (int)atomicAdd(&ac.cnt, (unsigned)__popc(grp));
                        const unsigned long long old = atomicMax(&ac.key1, k1);
                        const unsigned long long lo2 = old < k1 ? old : k1;
                        const unsigned lo_o = (unsigned)(lo2 >> 32);
                        atomicMax(&ac.o2, lo_o > sec_o ? lo_o : sec_o);
                        atomicMax(&ac.emax, em);
                    }
                }
                base = __shfl_sync(grp, base, leader);
                s = __shfl_sync(grp, s, leader);
                rank = base + __popc(grp & lt);
            }
            // code: (target, (slot << kLocalBits) | rank in the CTA's count),
            // (target, -1 - global rank) with a per-tile table or past a full
            // one, (-1, 0) discarded
            tgt[k] = (valid && f_dead) ? target : -2;
            rk[k] = rank;
            slot[k] = cone_t ? s : -1;
            if (!per_tile && valid && f_dead) {
                const int r = !cone_t ? 0 : (s >= 0 ? (s << kLocalBits) | rank : -1 - rank);
                A.code[v] = make_int2(target, r);
            }
        }
        if (per_tile) {
            __syncthreads();
            reserve_slots();
            __syncthreads();
#pragma unroll
            for (int k = 0; k < ITEMS; k++) {
                const int v = v0 + k * blockDim.x + threadIdx.x;
                if (tgt[k] == -2) continue;
                const int r = tgt[k] < 0 ? 0 : -1 - (slot[k] >= 0 ? ss.sbase[slot[k]] + rk[k] : rk[k]);
                A.code[v] = make_int2(tgt[k], r);
            }
        }
    }
    // ---- CTA-wide table: one reservation and key merge per (CTA, target)
    __syncthreads();
    if (!per_tile) reserve_slots();
    unsigned fsum = __reduce_add_sync(0xffffffffu, fallbacks);
    if (lane == 0 && fsum) atomicAdd(&H->fallbacks, (unsigned long long)fsum);
}

// Destination of a point classified into a cone facet (code from assign3d,
// slot bases of the CTA that classified it: the same CTA as the caller).
__device__ __forceinline__ int code_dst(const Params3 &A, const SmemSlots &ss, int2 cr)
{
    if (cr.x < 0) return -1;
    const int r = cr.y >= 0 ? ss.sbase[cr.y >> kLocalBits] + (cr.y & ((1 << kLocalBits) - 1))
                            : -1 - cr.y;
    return A.nstart[cr.x] + r;
}

// ---------------------------------------------------------------- T: table
// New segment table (the other parity): the old segments whose facet
// survives and the cone facets created this iteration that received points.
// Each CTA takes blocks of items, scans a block in shared memory and
// reserves its entries and points with one 64-bit atomic ((entries << 32) |
// points), so entries come out sorted by start (the order of the blocks is
// whatever the atomics give; no hull result depends on it).  A new facet's
// FP32 farthest point is certified here (top-2 gap against twice the largest
// error bound) or queued for the exact phase; its apex is recorded.
__device__ void certify_new(const Params3 &A, int f, int e)
{
    Hdr3 *H = A.hdr;
    const Acc3 a = A.acc[f];
    const int qi = key_idx(a.key1);
    A.apex[f] = load_input(A, qi);
    bool cert = true;
    const float em = __uint_as_float(a.emax);
    const float d1 = key_dist(a.key1);
    if (a.cnt > 1) {
        const float d2 = unord_f32(a.o2);
        const double gap = ((double)d1 - (double)d2) * (1.0 - 0x1p-50);
        cert = gap > 2.0 * (double)em;
    }
    if (!cert) {
        const double thr = (double)d1 - 3.0 * (double)em - fabs((double)d1) * 0x1p-20;
        A.thr[f] = isfinite(thr) ? __double2float_rd(thr) : -INFINITY;
        A.uncert[atomicAdd(&H->n_uncert, 1)] = e;
    }
}

__device__ void table3d(const Params3 &A, int par, bool first, SmemAll3 &sm, int bid, int nb)
{
    Hdr3 *H = A.hdr;
    const int ne = first ? 0 : (int)(*(volatile unsigned long long *)&H->tab[par] >> 32);
    const int fc0 = first ? 0 : *(volatile int *)&H->fc_iter[par];
    const int fc1 = *(volatile int *)&H->fcount;
    const int m = ne + (fc1 - fc0);
    const Ent3 *old = A.ent[par];
    Ent3 *out = A.ent[par ^ 1];
    for (int base = bid * blockDim.x; base < m; base += nb * blockDim.x) {
        const int j = base + threadIdx.x;
        int f = -1, len = 0;
        if (j < ne) {
            const Ent3 en = old[j];
            f = en.f;
            len = A.fac[f].alive ? en.len : 0;
        } else if (j < m) {
            f = fc0 + (j - ne);
            len = (int)A.acc[f].cnt;
        }
        const long long s = len > 0 ? ((1ll << 32) | (long long)len) : 0ll;
        long long tot;
        const long long ex = block_excl_scan64(s, sm.t.wsum, &tot);
        if (threadIdx.x == 0)
            sm.t.base = tot ? atomicAdd(&H->tab[par ^ 1], (unsigned long long)tot) : 0ull;
        __syncthreads();
        if (len > 0) {
            const unsigned long long b = sm.t.base + (unsigned long long)ex;
            const int k = (int)(b >> 32), st = (int)(b & 0xffffffffull);
            Ent3 en;
            en.f = f;
            en.start = st;
            en.len = len;
            en.pad = 0;
            out[k] = en;
            A.nstart[f] = st;
            if (j >= ne) certify_new(A, f, k);
        }
        __syncthreads();  // sm.t.base is rewritten by the next block
    }
    if (bid == 0 && threadIdx.x == 0) {
        H->fc_lo_last = fc0;
        H->fc_iter[par ^ 1] = fc1;  // read by the next table phase (other parity)
        // round counters of the next iteration (its select counts round 0)
        for (int r = 0; r < kRounds; r++) H->nact[r] = 0;
    }
}

// ---------------------------------------------------------------- B: scatter
// Every live point of table `par` to its place in the other buffer: a point
// of a surviving facet keeps its offset in its segment (the segment moves
// whole, nstart[f] - start), a point of a deleted facet goes where its code
// says (or nowhere).  Then the tile map of the new table, for the next
// assign and scatter.  FIRST: the input points and their codes.
template <bool FIRST>
__device__ void scatter3d(const Params3 &A, int par, SmemAll3 &sm, const SmemSlots &ss, int bid,
                          int nb)
{
    Hdr3 *H = A.hdr;
    const int L = FIRST ? A.n : (int)(*(volatile unsigned long long *)&H->tab[par] & 0xffffffffull);
    const Ent3 *ent = A.ent[par];
    const float4 *P = A.pts[par];
    float4 *Q = A.pts[par ^ 1];
    const int T = FIRST ? A.tile : *(volatile int *)&H->tile_sz[par];
    constexpr int kSc = 4;  // points per thread in flight
    // the tiles of the assign phase, each on the CTA that classified it (the
    // codes' ranks are relative to that CTA's slot bases)
    if (FIRST) {
        const int ntiles = (L + T - 1) / T;
        for (int tile = bid; tile < ntiles; tile += nb) {
            const int v0 = tile * T, v1 = min(v0 + T, L);
            for (int vb = v0 + threadIdx.x; vb < v1; vb += blockDim.x * kSc) {
                int dst[kSc];
                float4 p[kSc];
#pragma unroll
                for (int k = 0; k < kSc; k++) {
                    const int v = vb + k * blockDim.x;
                    dst[k] = v < v1 ? code_dst(A, ss, A.code[v]) : -1;
                }
#pragma unroll
                for (int k = 0; k < kSc; k++)
                    if (dst[k] >= 0) p[k] = load_input(A, vb + k * blockDim.x);
#pragma unroll
                for (int k = 0; k < kSc; k++)
                    if (dst[k] >= 0 && dbg_ok(dst[k] < A.n, kDbgPointDst, dst[k], A.n)) Q[dst[k]] = p[k];
            }
        }
    } else {
        const int ntiles = (L + T - 1) / T;
        for (int tile = bid; tile < ntiles; tile += nb) {
            const int v0 = tile * T, v1 = min(v0 + T, L);
            __syncthreads();
            const int e0 = A.tile_ent[par][tile], m = A.tile_m[par][tile];
            // per entry: start, and the shift of a surviving segment (INT_MIN:
            // the facet was deleted, its points follow their codes)
            for (int i = threadIdx.x; i < m; i += blockDim.x) {
                const Ent3 en = ent[e0 + i];
                sm.a.start[i] = en.start;
                sm.a.f[i] = A.fac[en.f].alive ? A.nstart[en.f] - en.start : INT_MIN;
            }
            __syncthreads();
            for (int vb = v0 + threadIdx.x; vb < v1; vb += blockDim.x * kSc) {
                int dst[kSc];
                float4 p[kSc];
#pragma unroll
                for (int k = 0; k < kSc; k++) {
                    const int v = vb + k * blockDim.x;
                    dst[k] = -1;
                    if (v >= v1) continue;
                    int lo = 0, hi = m - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (sm.a.start[mid] <= v) lo = mid;
                        else hi = mid - 1;
                    }
                    const int sh = sm.a.f[lo];
                    if (sh != INT_MIN) {
                        dst[k] = v + sh;
                    } else {
                        dst[k] = code_dst(A, ss, A.code[v]);
                    }
                }
#pragma unroll
                for (int k = 0; k < kSc; k++) {
                    const int v = vb + k * blockDim.x;
                    if (dst[k] >= 0) p[k] = P[v];
                }
#pragma unroll
                for (int k = 0; k < kSc; k++)
                    if (dst[k] >= 0 && dbg_ok(dst[k] < A.n, kDbgPointDst, dst[k], A.n)) Q[dst[k]] = p[k];
            }
        }
    }
    // tile size and tile -> entries map of the new table: the largest tile
    // (blockDim.x * ITEMS) halved, down to kMinTile, until every CTA gets one
    const unsigned long long tb = *(volatile unsigned long long *)&H->tab[par ^ 1];
    const int ne1 = (int)(tb >> 32), L1 = (int)(tb & 0xffffffffull);
    const Ent3 *ent1 = A.ent[par ^ 1];
    int T1 = A.tile;
    while (T1 > kMinTile && (L1 + T1 - 1) / T1 < nb) T1 >>= 1;
    if (bid == 0 && threadIdx.x == 0) H->tile_sz[par ^ 1] = T1;
    const int nt1 = (L1 + T1 - 1) / T1;
    for (int t = bid * blockDim.x + threadIdx.x; t < nt1; t += nb * blockDim.x) {
        const int v = t * T1, vl = min(v + T1, L1) - 1;
        auto ent_of = [&](int x) {
            int lo = 0, hi = ne1 - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (ent1[mid].start <= x) lo = mid;
                else hi = mid - 1;
            }
            return lo;
        };
        const int s0 = ent_of(v);
        A.tile_ent[par ^ 1][t] = s0;
        A.tile_m[par ^ 1][t] = ent_of(vl) - s0 + 1;
    }
}

// ---------------------------------------------------------------- X: exact apex
// Chunks per uncertified facet: with fewer such facets than CTAs, each
// facet's points are split over several CTAs, whose bests (float4 with the
// index bits in w, -1 when the chunk has no candidate) go to the per-point
// code buffer, free between the scatter and the next assignment.
__device__ __forceinline__ int exact_chunks(const Params3 &A, int nu, int nb)
{
    if (nu <= 0) return 1;
    const long long cap = (long long)A.n / 2;  // float4 slots in the code buffer
    long long per = nb / nu;
    if (per * nu > cap) per = cap / nu;
    return per > 1 ? (int)per : 1;
}

template <int MODE>
__device__ void exact3d(const Params3 &A, int par, SmemAll3 &sm, int bid, int nb, int per)
{
    Hdr3 *H = A.hdr;
    const int nu = *(volatile int *)&H->n_uncert;
    const Ent3 *ent = A.ent[par ^ 1];
    const float4 *Q = A.pts[par ^ 1];
    float4 *part = reinterpret_cast<float4 *>(A.code);
    for (int w = bid; w < nu * per; w += nb) {
        const int u = w / per, ch = w - u * per;
        const Ent3 en = ent[A.uncert[u]];
        const Fac3 F = A.fac[en.f];
        const float *a, *b, *c;
        fac_pts(F, a, b, c);
        const float thr = A.thr[en.f];
        const int lo = (int)((long long)en.len * ch / per);
        const int hi = (int)((long long)en.len * (ch + 1) / per);
        int best = -1;
        float4 bp = make_float4(0, 0, 0, 0);
        for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            const float4 p4 = Q[en.start + i];
            const float p[3] = {p4.x, p4.y, p4.z};
            float d, e;
            orient3d_value<MODE>(a, b, c, p, d, e);
            if ((double)d + (double)e < (double)thr) continue;
            const int idx = __float_as_int(p4.w);
            if (best >= 0) {
                const float q[3] = {bp.x, bp.y, bp.z};
                const int s = cmp_dist3_exact_sign(a, b, c, p, q);
                if (!(s > 0 || (s == 0 && idx < best))) continue;
            }
            best = idx;
            bp = p4;
        }
        sm.x.idx[threadIdx.x] = best;
        sm.x.p[threadIdx.x] = bp;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) {
                const int oi = sm.x.idx[threadIdx.x + s];
                const int mi = sm.x.idx[threadIdx.x];
                if (oi >= 0) {
                    bool take = mi < 0;
                    if (!take) {
                        const float4 o = sm.x.p[threadIdx.x + s], me = sm.x.p[threadIdx.x];
                        const float po[3] = {o.x, o.y, o.z}, pm[3] = {me.x, me.y, me.z};
                        const int c2 = cmp_dist3_exact_sign(a, b, c, po, pm);
                        take = c2 > 0 || (c2 == 0 && oi < mi);
                    }
                    if (take) {
                        sm.x.idx[threadIdx.x] = oi;
                        sm.x.p[threadIdx.x] = sm.x.p[threadIdx.x + s];
                    }
                }
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            if (per > 1) {
                float4 r = sm.x.p[0];
                if (sm.x.idx[0] < 0) r.w = __int_as_float(-1);
                part[w] = r;
            } else if (sm.x.idx[0] >= 0) {
                A.apex[en.f] = sm.x.p[0];
            }
        }
        __syncthreads();
    }
}

// Split exact phase, second step (after a grid barrier): one thread per
// uncertified facet merges its chunks' bests with exact comparisons.
template <int MODE>
__device__ void exact3d_merge(const Params3 &A, int par, int bid, int nb, int per)
{
    Hdr3 *H = A.hdr;
    const int nu = *(volatile int *)&H->n_uncert;
    const Ent3 *ent = A.ent[par ^ 1];
    const float4 *part = reinterpret_cast<const float4 *>(A.code);
    for (int u = bid * blockDim.x + threadIdx.x; u < nu; u += nb * blockDim.x) {
        const Ent3 en = ent[A.uncert[u]];
        const Fac3 F = A.fac[en.f];
        const float *a, *b, *c;
        fac_pts(F, a, b, c);
        int best = -1;
        float4 bp = make_float4(0, 0, 0, 0);
        for (int ch = 0; ch < per; ch++) {
            const float4 p4 = part[u * per + ch];
            const int idx = __float_as_int(p4.w);
            if (idx < 0) continue;
            if (best >= 0) {
                const float p[3] = {p4.x, p4.y, p4.z}, q[3] = {bp.x, bp.y, bp.z};
                const int s = cmp_dist3_exact_sign(a, b, c, p, q);
                if (!(s > 0 || (s == 0 && idx < best))) continue;
            }
            best = idx;
            bp = p4;
        }
        if (best >= 0) A.apex[en.f] = bp;
    }
}

// ---------------------------------------------------------------- persistent kernel
template <int MODE, int ITEMS>
__global__ void __launch_bounds__(kMaxBlock) qh3d_persistent(Params3 A)
{
    __shared__ SmemAll3 sm;
    __shared__ SmemSlots ss;  // an assign phase's targets, read by the following scatter
    Hdr3 *H = A.hdr;
    int *fail = &H->status;
    const int bid = blockIdx.x, nb = gridDim.x;
    // every grid barrier returns the status, the same value in the whole
    // CTA; a phase runs only while it is zero, so after a failure no CTA
    // reads results that another CTA has not finished writing
    bool hold = A.test_hold != 0 && bid == 0;
    auto sync = [&]() {
        const int st = grid_sync_count(&H->bar, fail, A.wait_ns, hold);
        hold = false;
        return st == 0;
    };
    // phase clock of block 0, thread 0 (per-iteration record)
    const bool clk = bid == 0 && threadIdx.x == 0;
    unsigned long long tprev = clk ? globaltimer_ns() : 0;
    auto mark = [&](int it, int col) {
        if (!clk) return;
        const unsigned long long t = globaltimer_ns();
        if (it > 0 && it <= kTimeline3) H->tl[it - 1][col] += (long long)(t - tprev);
        tprev = t;
    };

    const unsigned long long t_start = tprev;
    auto setup_mark = [&](int k) {
        if (!clk) return;
        const unsigned long long t = globaltimer_ns();
        H->setup_ns[k] = (long long)(t - tprev);
        tprev = t;
    };
    bool go = status_uniform(fail) == 0;
    // ---- initial simplex: grid-wide for one cloud, one block per cloud for
    // a batch
    if (A.cloud_off) {
        if (go) {
            if (A.small_cloud > 0) small_clouds(A);  // one warp per small cloud
            init_clouds(A, sm, bid, nb);               // offsets checked before the launch
        }
        go = sync() && go;
    } else {
        if (go) {
            extrema3d(A, sm, bid, nb);
            go = sync();
        }
        if (go) {
            if (bid == 0) simplex_step(A, sm, 0, nb);
            go = sync();
        }
        if (go && *(volatile int *)&H->nonfinite) {
            if (bid == 0 && threadIdx.x == 0) set_status(H, QH_ERR_NONFINITE);
            go = sync();
        }
        for (int step = 1; step <= 2 && go; step++) {
            farthest3d(A, sm, bid, nb, step - 1);
            if (!(go = sync())) break;
            if (bid == 0) simplex_step(A, sm, step, nb);
            if (!(go = sync())) break;
            if (!*(volatile int *)&H->cand_ok) {
                exact_search3d(A, bid, nb, step - 1);
                if (!(go = sync())) break;
            }
            if (bid == 0) simplex_take(A, step);
            go = sync();
        }
        if (go) {
            if (bid == 0) build_tetra(A);
            go = sync();
        }
        // the first polytope: the tetrahedron and the directions' extreme points
        if (go && A.init_dirs) {
            dir_extrema3d(A, sm, bid, nb);
            go = sync();
            if (go) {
                if (bid == 0) expand_initial(A, sm);
                go = sync();
            }
        }
    }
    setup_mark(0);
    auto tab_ne = [&](int p) { return (int)(*(volatile unsigned long long *)&H->tab[p] >> 32); };
    auto tab_L = [&](int p) {
        return (int)(*(volatile unsigned long long *)&H->tab[p] & 0xffffffffull);
    };
    // exact farthest points of the facets the table phase left uncertified
    // (their points must be in place: after a scatter and a barrier); p is
    // the parity of the table the phase read (the new one is p ^ 1)
    auto exact_phase = [&](int p) {
        const int nu = *(volatile int *)&H->n_uncert;
        if (nu <= 0) return true;
        const int per = exact_chunks(A, nu, nb);
        exact3d<MODE>(A, p, sm, bid, nb, per);
        if (!sync()) return false;
        if (per > 1) {
            exact3d_merge<MODE>(A, p, bid, nb, per);
            if (!sync()) return false;
        }
        if (bid == 0 && threadIdx.x == 0) H->exact_argmax += nu;
        return true;
    };
    if (go) {
        // ---- first assignment: every input point against the tetrahedron;
        // table 1 / buffer 1 receive the result
        assign3d<MODE, ITEMS, true>(A, 0, sm, ss, bid, nb);
        go = sync();
        setup_mark(1);
        if (go) {
            table3d(A, 0, true, sm, bid, nb);
            go = sync();
        }
        setup_mark(2);
        if (go) {
            scatter3d<true>(A, 0, sm, ss, bid, nb);
            go = sync();
        }
        if (go) go = exact_phase(0);
        setup_mark(3);
    }
    // ---- iterations: table `cur` describes the live points in buffer `cur`.
    // Phases: [scatter of the previous iteration +] select with the claims of
    // round 0 | rounds 0 .. kRounds-1 (winners' cones, next round's claims) |
    // [lone-apex fallback] | assign | table (+ certification) | [scatter |
    // exact, when some apex is uncertified].
    int cur = 1;
    int iter = 0;
    bool scatter_due = false;  // the points of table `cur` are still in buffer cur ^ 1
    while (go && tab_ne(cur) > 0) {
        iter++;
        if (iter > A.max_iters) {
            if (bid == 0 && threadIdx.x == 0) set_status(H, QH_ERR_NO_CONVERGENCE);
            break;
        }
        if (bid == 0 && threadIdx.x == 0) {
            H->iter = iter;
            H->nwin = 0;  // counted from the rounds on (after this phase's barrier)
            H->seg_total += tab_ne(cur);
            H->surv_total += tab_L(cur);
            if (iter <= kTimeline3) {
                H->tl[iter - 1][0] = tab_L(cur);
                H->tl[iter - 1][1] = tab_ne(cur);
            }
        }
        mark(0, 0);
        if (scatter_due) scatter3d<false>(A, cur ^ 1, sm, ss, bid, nb);
        if (tab_ne(cur) <= kSelWarpMul * nb * (int)(blockDim.x >> 5)) {
            __syncthreads();  // the scatter's staging and the warps' lists share memory
            select3d_warp<MODE>(A, cur, iter, sm, bid, nb);
        } else {
            select3d<MODE>(A, cur, iter, bid, nb);
        }
        if (!sync()) break;
        mark(iter, 3);
        for (int r = 0; r < kRounds && go; r++) {
            if (*(volatile int *)&H->nact[r] == 0) break;
            round3d(A, cur, iter, r, r == kRounds - 1, sm, bid, nb);
            go = sync();
        }
        if (!go) break;
        if (*(volatile int *)&H->nwin == 0) {
            if (bid == 0) fallback3d<MODE>(A, cur, iter);
            if (!sync()) break;
        }
        if (clk && iter <= kTimeline3) H->tl[iter - 1][2] = H->nwin;
        mark(iter, 4);
        assign3d<MODE, ITEMS, false>(A, cur, sm, ss, bid, nb);
        if (bid == 0 && threadIdx.x == 0) {
            H->tab[cur ^ 1] = 0ull;  // the table of two iterations ago
            H->n_uncert = 0;
        }
        if (!sync()) break;
        mark(iter, 5);
        table3d(A, cur, false, sm, bid, nb);
        if (!sync()) break;
        mark(iter, 6);
        if (tab_ne(cur ^ 1) == 0) break;  // no point left outside the hull
        if (*(volatile int *)&H->n_uncert > 0) {
            scatter3d<false>(A, cur, sm, ss, bid, nb);
            if (!sync()) break;
            mark(iter, 7);
            if (!(go = exact_phase(cur))) break;
            scatter_due = false;
        } else {
            scatter_due = true;
        }
        mark(iter, 8);
        cur ^= 1;
    }
    if (clk) H->kernel_ns = (long long)(globaltimer_ns() - t_start);
}

// Kernel entry of the persistent 3D loop for a predicate mode and points per
// thread of the assign pass (2, 4 or 8; the launch happens in qh3d_out.cu).
const void *persistent_kernel(int mode, int items)
{
    if (mode == QH_PRED_F32) {
        if (items == 2) return (const void *)qh3d_persistent<QH_PRED_F32, 2>;
        if (items == 8) return (const void *)qh3d_persistent<QH_PRED_F32, 8>;
        return (const void *)qh3d_persistent<QH_PRED_F32, 4>;
    }
    if (items == 2) return (const void *)qh3d_persistent<QH_PRED_F64, 2>;
    if (items == 8) return (const void *)qh3d_persistent<QH_PRED_F64, 8>;
    return (const void *)qh3d_persistent<QH_PRED_F64, 4>;
}

}  // namespace d3
}  // namespace qh
