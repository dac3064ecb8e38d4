// 4D segmented Quickhull on one GPU.
//
// The paper extends the recursion to higher dimensions with a k-state
// flagPermute (Section 4.3, "3D and Higher Dimensions").  As in 3D, this
// follows the Quickhull of Barber et al. the paper builds on, in R^4: every
// live point belongs to the outside set ("segment") of one facet (a
// tetrahedron); each iteration takes every segment's farthest point as a
// candidate apex, inserts the candidates whose visible regions are disjoint
// and not adjacent (claims in rounds), replaces each winner's visible facets
// by one new facet per horizon ridge (a triangle) through the apex, assigns
// the visible facets' points to the first new facet they are strictly above
// (else discards them) and regroups the survivors into the new segments by a
// scan and a scatter.
//
// The iterations are driven from the host, one kernel per phase, with the
// table sizes read back once per iteration (the paper's own driver).  Output:
// the extreme points (sorted) and the facets of the hull as the sorted
// extreme points on each maximal set of boundary points on one supporting
// hyperplane, sorted lexicographically (the simplices of the final
// triangulation merged across ridges whose neighbours lie on the same
// hyperplane; a vertex of the triangulation is extreme exactly when no other
// vertex of the simplices around it lies on every hyperplane through it).

#include <algorithm>
#include <chrono>
#include <climits>
#include <cstdio>
#include <cstring>
#include <vector>

#include "pred4.cuh"
#include "qh3d_internal.cuh"
#include "qh_common.cuh"
#include "qh_internal.h"

namespace qh {
namespace d4 {

// Visible facets a candidate may list, and horizon neighbours (>= 2 kV + 2:
// a 3-ball of kV tetrahedra has at most 2 kV + 2 boundary triangles).  A
// late point at height h above a finely triangulated 3-sphere sees a cap of
// radius ~sqrt(2h), whose facet count grows with the cube of that radius
// (the square in 3D): the lists are longer than the 3D ones.
#ifndef QH4D_VCAP
#define QH4D_VCAP 128
#endif
constexpr int kV = QH4D_VCAP;
constexpr int kN = 2 * kV + 2;
#ifndef QH4D_ROUNDS
#define QH4D_ROUNDS 3
#endif
constexpr int kRounds4 = QH4D_ROUNDS;  // selection rounds per iteration
constexpr int kBlock = 256;
constexpr int kItems = 4;      // points per thread of the assign tiles
constexpr int kTile = kBlock * kItems;
constexpr int kSlots4 = 128;   // targets aggregated per assign tile

struct Fac4 {
    int v[4];    // orient4(v0, v1, v2, v3, x) > 0: x strictly outside
    int nb[4];   // nb[k]: facet across the ridge opposite v[k]
    int alive;
    int pad[3];
};
static_assert(sizeof(Fac4) == 48, "Fac4 layout");

struct Acc4 {
    unsigned long long key1;  // (distance order bits << 32) | ~index of the best point
    unsigned o2;              // distance order bits of the best other point
    unsigned cnt;
    unsigned emax;            // largest error bound of the keys (float bits)
    unsigned pad;
};

struct Ent4 {
    int f, start, len, pad;
};

struct Basis4 {
    float o[4];
    float b[3][4];
    int nb;
};

struct Hdr4 {
    int status, nonfinite;
    int fcount, nwin, n_uncert, iter;
    int simplex[5];
    int cand_idx, search_idx, cand_ok;
    unsigned long long tab[2];  // (entries << 32) | points of the table of each parity
    int fc_iter[2];             // facet count when the table of that parity was built
    int nact[8];
    int hull_vertices;
    long long seg_total, surv_total;
    unsigned long long fallbacks, exact_argmax;
    // output stage
    int nalive, npair, nuniq, ngroup, nvert, sort_m, uf_fail;
    long long nfidx;
    Basis4 basis;               // span of the first simplex so far (its construction)
};

struct Params4 {
    const float *x, *y, *z, *w;
    long long stride;
    int n, fcap, ecap;
    Hdr4 *hdr;
    Fac4 *fac;
    Plane4 *pl;
    Acc4 *acc;
    int *apex;                    // apex point index of a facet with a segment
    unsigned long long *claim[2];
    int4 *cone;                   // deleted facet: (first new facet, count, apex, iteration)
    int *taken;
    float *thr;
    int *nstart;
    int *big_v, *big_h;           // lone-apex fallback scratch (fcap each)
    Ent4 *ent[2];
    int2 *vn;
    int *cstate;
    int *vpool, *npool;
    int *uncert;
    float4 *pts[2];
    int *pidx[2];
    int2 *code;
    float4 *blk_a, *blk_b;
    int *blk_ai, *blk_bi;
    float *blk_v;
    int *blk_i;
    long long max_iters;
};

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ void set_status4(Hdr4 *H, int st) { atomicCAS(&H->status, 0, st); }

__device__ __forceinline__ float4 load4(const Params4 &A, long long i)
{
    const long long o = i * A.stride;
    return make_float4(__ldg(A.x + o), __ldg(A.y + o), __ldg(A.z + o), __ldg(A.w + o));
}
__device__ __forceinline__ void load4a(const Params4 &A, long long i, float *p)
{
    const float4 q = load4(A, i);
    p[0] = q.x;
    p[1] = q.y;
    p[2] = q.z;
    p[3] = q.w;
}

// Exact sign of orient4(facet g, p): the facet's plane in FP32, else the
// FP64 filter and the exact expansion on the vertices' coordinates.
__device__ __forceinline__ int facet_sign4(const Params4 &A, int g, float4 p, float &d, float &e,
                                           unsigned &fallbacks)
{
    const Plane4 P = A.pl[g];
    plane4_value(P, p, d, e);
    if (d > e) return 1;
    if (-d > e) return -1;
    ++fallbacks;
    float a[4], b[4], c[4], dd[4];
    const Fac4 &F = A.fac[g];
    load4a(A, F.v[0], a);
    load4a(A, F.v[1], b);
    load4a(A, F.v[2], c);
    load4a(A, F.v[3], dd);
    const float q[4] = {p.x, p.y, p.z, p.w};
    return orient4_slow(a, b, c, dd, q);
}

// Lexicographic (x, y, z, w, index) order; -0.0 == +0.0.
__device__ __forceinline__ bool lex_less4(float4 p, int pi, float4 q, int qi)
{
    if (p.x != q.x) return p.x < q.x;
    if (p.y != q.y) return p.y < q.y;
    if (p.z != q.z) return p.z < q.z;
    if (p.w != q.w) return p.w < q.w;
    return pi < qi;
}
__device__ __forceinline__ bool lex_greater4(float4 p, int pi, float4 q, int qi)
{
    if (p.x != q.x) return p.x > q.x;
    if (p.y != q.y) return p.y > q.y;
    if (p.z != q.z) return p.z > q.z;
    if (p.w != q.w) return p.w > q.w;
    return pi < qi;
}

// Claim key: iteration, round, segment size class, then a permutation of the
// facet id (keys unique; Luby-style independent winners).
__device__ __forceinline__ unsigned long long claim_key4(int iter, int round, int f, int len)
{
    const unsigned perm = (((unsigned)f ^ ((unsigned)iter * 0x9E37u)) * 0x0B5AD4Bu) & 0x0FFFFFFFu;
    const unsigned cls = min(15u, (31u - (unsigned)__clz(max(len, 1))) >> 1);
    return ((unsigned long long)(unsigned)iter << 36) | ((unsigned long long)round << 32) |
           ((unsigned long long)cls << 28) | perm;
}

// ---------------------------------------------------------------- first simplex
__global__ void __launch_bounds__(kBlock) k4_extrema(Params4 A)
{
    __shared__ float4 sa[kBlock], sb[kBlock];
    __shared__ int sai[kBlock], sbi[kBlock];
    float4 mn = make_float4(INFINITY, INFINITY, INFINITY, INFINITY);
    float4 mx = make_float4(-INFINITY, -INFINITY, -INFINITY, -INFINITY);
    int mni = INT_MAX, mxi = INT_MAX, bad = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < A.n;
         i += (long long)gridDim.x * blockDim.x) {
        float4 p = load4(A, i);
        p.x = canon0(p.x);
        p.y = canon0(p.y);
        p.z = canon0(p.z);
        p.w = canon0(p.w);
        bad |= !(isfinite(p.x) && isfinite(p.y) && isfinite(p.z) && isfinite(p.w));
        if (lex_less4(p, (int)i, mn, mni)) {
            mn = p;
            mni = (int)i;
        }
        if (lex_greater4(p, (int)i, mx, mxi)) {
            mx = p;
            mxi = (int)i;
        }
    }
    bad = __syncthreads_or(bad);
    sa[threadIdx.x] = mn;
    sai[threadIdx.x] = mni;
    sb[threadIdx.x] = mx;
    sbi[threadIdx.x] = mxi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const int o = threadIdx.x + s;
            if (lex_less4(sa[o], sai[o], sa[threadIdx.x], sai[threadIdx.x])) {
                sa[threadIdx.x] = sa[o];
                sai[threadIdx.x] = sai[o];
            }
            if (lex_greater4(sb[o], sbi[o], sb[threadIdx.x], sbi[threadIdx.x])) {
                sb[threadIdx.x] = sb[o];
                sbi[threadIdx.x] = sbi[o];
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        A.blk_a[blockIdx.x] = sa[0];
        A.blk_ai[blockIdx.x] = sai[0];
        A.blk_b[blockIdx.x] = sb[0];
        A.blk_bi[blockIdx.x] = sbi[0];
        if (bad) atomicExch(&A.hdr->nonfinite, 1);
    }
}

__global__ void k4_extrema_final(Params4 A, int nblk)
{
    Hdr4 *H = A.hdr;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x >= 32) return;
    if (H->nonfinite) {
        if (lane == 0) set_status4(H, QH_ERR_NONFINITE);
        return;
    }
    // each lane over a stride of the blocks' results, then the lanes'
    // results by shuffles (same order and lowest-index rules)
    float4 mn = A.blk_a[0], mx = A.blk_b[0];
    int mni = A.blk_ai[0], mxi = A.blk_bi[0];
    for (int b = lane; b < nblk; b += 32) {
        if (lex_less4(A.blk_a[b], A.blk_ai[b], mn, mni)) {
            mn = A.blk_a[b];
            mni = A.blk_ai[b];
        }
        if (lex_greater4(A.blk_b[b], A.blk_bi[b], mx, mxi)) {
            mx = A.blk_b[b];
            mxi = A.blk_bi[b];
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const float4 pa = make_float4(__shfl_xor_sync(0xffffffffu, mn.x, o),
                                      __shfl_xor_sync(0xffffffffu, mn.y, o),
                                      __shfl_xor_sync(0xffffffffu, mn.z, o),
                                      __shfl_xor_sync(0xffffffffu, mn.w, o));
        const int pai = __shfl_xor_sync(0xffffffffu, mni, o);
        const float4 pb = make_float4(__shfl_xor_sync(0xffffffffu, mx.x, o),
                                      __shfl_xor_sync(0xffffffffu, mx.y, o),
                                      __shfl_xor_sync(0xffffffffu, mx.z, o),
                                      __shfl_xor_sync(0xffffffffu, mx.w, o));
        const int pbi = __shfl_xor_sync(0xffffffffu, mxi, o);
        if (lex_less4(pa, pai, mn, mni)) {
            mn = pa;
            mni = pai;
        }
        if (lex_greater4(pb, pbi, mx, mxi)) {
            mx = pb;
            mxi = pbi;
        }
    }
    if (lane != 0) return;
    H->simplex[0] = mni;
    H->simplex[1] = mxi;
    if (mn.x == mx.x && mn.y == mx.y && mn.z == mx.z && mn.w == mx.w)
        set_status4(H, QH_ERR_DEGENERATE);
}

// Basis of the affine span of simplex[0..step) (Gram-Schmidt in FP64 on
// the device, one thread); it only chooses the next candidate, which an
// exact test confirms.
__global__ void k4_basis(Params4 A, int step)
{
    Hdr4 *H = A.hdr;
    if (threadIdx.x != 0 || H->status) return;
    double P[4][4];
    for (int k = 0; k < step; k++) {
        const float4 c = load4(A, H->simplex[k]);
        P[k][0] = c.x;
        P[k][1] = c.y;
        P[k][2] = c.z;
        P[k][3] = c.w;
    }
    double Bd[3][4];
    for (int k = 0; k < step - 1; k++) {
        for (int d = 0; d < 4; d++) Bd[k][d] = P[k + 1][d] - P[0][d];
        for (int r = 0; r < k; r++) {
            double dp = 0;
            for (int d = 0; d < 4; d++) dp += Bd[k][d] * Bd[r][d];
            for (int d = 0; d < 4; d++) Bd[k][d] -= dp * Bd[r][d];
        }
        double nr = 0;
        for (int d = 0; d < 4; d++) nr += Bd[k][d] * Bd[k][d];
        nr = sqrt(nr);
        for (int d = 0; d < 4; d++) Bd[k][d] = nr > 0 ? Bd[k][d] / nr : 0.0;
    }
    Basis4 &B = H->basis;
    for (int d = 0; d < 4; d++) B.o[d] = (float)P[0][d];
    for (int k = 0; k < 3; k++)
        for (int d = 0; d < 4; d++) B.b[k][d] = k < step - 1 ? (float)Bd[k][d] : 0.0f;
    B.nb = step - 1;
}

// Squared distance from the affine span of the simplex so far (origin s0,
// orthonormal directions from k4_basis), FP32; the farthest point (lowest
// index on ties) per block.
__global__ void __launch_bounds__(kBlock) k4_far(Params4 A)
{
    if (*(volatile int *)&A.hdr->status) return;
    const Basis4 B = A.hdr->basis;
    __shared__ float sv[kBlock];
    __shared__ int si[kBlock];
    float best = -1.0f;
    int bi = INT_MAX;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < A.n;
         i += (long long)gridDim.x * blockDim.x) {
        const float4 p = load4(A, i);
        float r[4] = {p.x - B.o[0], p.y - B.o[1], p.z - B.o[2], p.w - B.o[3]};
        for (int k = 0; k < B.nb; k++) {
            const float dp = r[0] * B.b[k][0] + r[1] * B.b[k][1] + r[2] * B.b[k][2] + r[3] * B.b[k][3];
            for (int q = 0; q < 4; q++) r[q] -= dp * B.b[k][q];
        }
        const float v = r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + r[3] * r[3];
        if (v > best) {  // NaN never wins; increasing i: the first keeps ties
            best = v;
            bi = (int)i;
        }
    }
    sv[threadIdx.x] = best;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const float ov = sv[threadIdx.x + s];
            const int oi = si[threadIdx.x + s];
            if (ov > sv[threadIdx.x] || (ov == sv[threadIdx.x] && oi < si[threadIdx.x])) {
                sv[threadIdx.x] = ov;
                si[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        A.blk_v[blockIdx.x] = sv[0];
        A.blk_i[blockIdx.x] = si[0];
    }
}

// Point i lies off the span of simplex[0..step) (exact).
__device__ bool off_span4(const Params4 &A, int step, int i)
{
    const Hdr4 *H = A.hdr;
    float a[4], b[4], c[4], d[4], p[4];
    load4a(A, H->simplex[0], a);
    load4a(A, H->simplex[1], b);
    load4a(A, i, p);
    if (step == 2) return !on_line4(a, b, p);
    load4a(A, H->simplex[2], c);
    if (step == 3) return !on_plane4(a, b, c, p);
    load4a(A, H->simplex[3], d);
    return orient4_slow(a, b, c, d, p) != 0;
}

__global__ void k4_far_final(Params4 A, int nblk, int step)
{
    Hdr4 *H = A.hdr;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x >= 32 || H->status) return;
    float bv = -2.0f;
    int bi = INT_MAX;
    for (int b = lane; b < nblk; b += 32)
        if (A.blk_v[b] > bv || (A.blk_v[b] == bv && A.blk_i[b] < bi)) {
            bv = A.blk_v[b];
            bi = A.blk_i[b];
        }
    for (int o = 16; o > 0; o >>= 1) {
        const float v = __shfl_xor_sync(0xffffffffu, bv, o);
        const int i = __shfl_xor_sync(0xffffffffu, bi, o);
        if (v > bv || (v == bv && i < bi)) {
            bv = v;
            bi = i;
        }
    }
    if (lane != 0) return;
    H->search_idx = INT_MAX;
    H->cand_ok = bi >= 0 && bi < A.n && off_span4(A, step, bi);
    if (H->cand_ok) H->simplex[step] = bi;
}

// The lowest-index point off the span (when the FP32 choice was degenerate).
__global__ void __launch_bounds__(kBlock) k4_search(Params4 A, int step)
{
    Hdr4 *H = A.hdr;
    if (H->status || H->cand_ok) return;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < A.n;
         i += (long long)gridDim.x * blockDim.x)
        if ((int)i < *(volatile int *)&H->search_idx && off_span4(A, step, (int)i))
            atomicMin(&H->search_idx, (int)i);
}

__global__ void k4_take(Params4 A, int step)
{
    Hdr4 *H = A.hdr;
    if (threadIdx.x != 0 || H->status || H->cand_ok) return;
    if (H->search_idx == INT_MAX) set_status4(H, QH_ERR_DEGENERATE);
    else H->simplex[step] = H->search_idx;
}

__device__ void init_facet4(const Params4 &A, int f, const int *v)
{
    Fac4 F;
    for (int i = 0; i < 4; i++) {
        F.v[i] = v[i];
        F.nb[i] = -1;
    }
    F.alive = 1;
    F.pad[0] = F.pad[1] = F.pad[2] = 0;
    A.fac[f] = F;
    float a[4], b[4], c[4], d[4];
    load4a(A, v[0], a);
    load4a(A, v[1], b);
    load4a(A, v[2], c);
    load4a(A, v[3], d);
    A.pl[f] = make_plane4(a, b, c, d);
    Acc4 z = {};
    A.acc[f] = z;
    A.claim[0][f] = 0ull;
    A.claim[1][f] = 0ull;
    A.taken[f] = 0;
}

// One thread: the five facets of the simplex, the missing point inside each,
// their neighbours, and the cone record of the pseudo facet fcap.
__global__ void k4_build(Params4 A)
{
    Hdr4 *H = A.hdr;
    if (threadIdx.x != 0 || H->status) return;
    for (int o = 0; o < 5; o++) {
        int v[4], k = 0;
        for (int j = 0; j < 5; j++)
            if (j != o) v[k++] = H->simplex[j];
        float a[4], b[4], c[4], d[4], p[4];
        load4a(A, v[0], a);
        load4a(A, v[1], b);
        load4a(A, v[2], c);
        load4a(A, v[3], d);
        load4a(A, H->simplex[o], p);
        if (orient4_slow(a, b, c, d, p) > 0) {
            const int t = v[0];
            v[0] = v[1];
            v[1] = t;
        }
        init_facet4(A, o, v);
    }
    for (int i = 0; i < 5; i++)
        for (int k = 0; k < 4; k++)
            for (int j = 0; j < 5; j++) {
                if (j == i) continue;
                int shared = 0;
                for (int a = 0; a < 4; a++) {
                    if (a == k) continue;
                    for (int b = 0; b < 4; b++) shared += A.fac[i].v[a] == A.fac[j].v[b];
                }
                if (shared == 3) A.fac[i].nb[k] = j;
            }
    A.cone[A.fcap] = make_int4(0, 5, -1, 0);
    H->fcount = 5;
    H->hull_vertices = 5;
}

// ---------------------------------------------------------------- A: assign
// Every live point of a deleted facet (first pass: every input point, all
// "in" the pseudo facet whose cone is the simplex) goes to the first facet
// of its winner's cone that it is strictly above, else it is discarded;
// code[v] = (target, rank in the target's segment) or (-1, 0); points of
// surviving facets get (-2, their segment's table entry).  Each tile's
// segments are staged in shared memory first.  Counts, ranks and
// farthest-point keys are aggregated per warp (match) and per tile (shared
// hash), one global reservation per (tile, target).
template <bool FIRST>
__global__ void __launch_bounds__(kBlock) k4_assign(Params4 A, int par)
{
    __shared__ int skey[kSlots4], scnt[kSlots4], sbase[kSlots4];
    __shared__ unsigned long long sk1[kSlots4];
    __shared__ unsigned so2[kSlots4], sem[kSlots4];
    __shared__ int sst[kTile], sfa[kTile];  // the tile's segments: start, facet
    __shared__ int s_m;
    Hdr4 *H = A.hdr;
    if (*(volatile int *)&H->status) return;
    const unsigned long long tb = *(volatile unsigned long long *)&H->tab[par];
    const int L = FIRST ? A.n : (int)(tb & 0xffffffffull);
    const int ne = (int)(tb >> 32);
    const Ent4 *ent = A.ent[par];
    const float4 *P = A.pts[par];
    const int *PI = A.pidx[par];
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    unsigned fallbacks = 0;
    const int ntiles = (L + kTile - 1) / kTile;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        __syncthreads();
        for (int i = threadIdx.x; i < kSlots4; i += blockDim.x) {
            skey[i] = -1;
            scnt[i] = 0;
            sk1[i] = 0ull;
            so2[i] = 0u;
            sem[i] = 0u;
        }
        __syncthreads();
        // the tile's segments, staged: the last one starting at or before
        // the tile (probes over the table, each round narrowing the interval
        // to one probe gap), then every one starting inside it
        int e0 = 0;
        if (!FIRST) {
            const int v0 = tile * kTile, v1 = min(v0 + kTile, L);
            int lo = 0, hi = ne - 1;  // the answer is in [lo, hi]
            for (int round = 0; round < 6 && hi > lo; round++) {
                const long long span = (long long)(hi - lo + 1);
                const int pi = lo + (int)((long long)threadIdx.x * span / blockDim.x);
                const int c = __syncthreads_count(ent[pi].start <= v0);  // >= 1: start[lo] <= v0
                const int nlo = lo + (int)((long long)(c - 1) * span / blockDim.x);
                const int nhi = c < (int)blockDim.x ? lo + (int)((long long)c * span / blockDim.x) - 1 : hi;
                lo = nlo;
                hi = nhi < nlo ? nlo : nhi;
            }
            e0 = lo;
            if (threadIdx.x == 0) s_m = 0;
            __syncthreads();
            int mine = 0;
            for (int i = threadIdx.x; i < kTile; i += blockDim.x) {
                const int e = e0 + i;
                if (e < ne) {
                    const Ent4 en = ent[e];
                    if (i == 0 || en.start < v1) {
                        sst[i] = en.start;
                        sfa[i] = en.f;
                        mine++;
                    }
                }
            }
            if (mine) atomicAdd(&s_m, mine);
            __syncthreads();
        }
        const int m = FIRST ? 0 : s_m;  // the staged entries are a prefix (starts increase)
        int tgt[kItems], rk[kItems], slot[kItems];
#pragma unroll
        for (int k = 0; k < kItems; k++) {
            const int v = tile * kTile + k * blockDim.x + threadIdx.x;
            const bool valid = v < L;
            int target = -1, rank = 0, s = -1, f = A.fcap;
            bool dead = false, cone_t = false;
            float d = 0.0f, err = 0.0f;
            int idx = 0;
            if (valid) {
                if (!FIRST) {
                    int lo = 0, hi = m - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (sst[mid] <= v) lo = mid;
                        else hi = mid - 1;
                    }
                    f = sfa[lo];
                    rank = e0 + lo;  // a surviving facet's points keep their segment
                }
                dead = FIRST || !A.fac[f].alive;
                if (dead) {
                    const float4 p = FIRST ? load4(A, v) : P[v];
                    idx = FIRST ? v : PI[v];
                    const int4 cn = A.cone[f];
                    bool skip = idx == cn.z;  // the apex itself
                    if (FIRST) {  // the simplex vertices (facets 0 and 1 hold all five)
                        const Fac4 &F0 = A.fac[0], &F1 = A.fac[1];
                        for (int t = 0; t < 4; t++) skip |= idx == F0.v[t] || idx == F1.v[t];
                    }
                    for (int c = 0; c < cn.y && !skip && !cone_t; c++) {
                        if (facet_sign4(A, cn.x + c, p, d, err, fallbacks) > 0) {
                            target = cn.x + c;
                            cone_t = true;
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
                    int h = (int)(((unsigned)target * 0x9E3779B1u) >> 25);
                    for (int probe = 0; probe < 16; probe++) {
                        const int prev = atomicCAS(&skey[h], -1, target);
                        if (prev == -1 || prev == target) {
                            s = h;
                            break;
                        }
                        h = (h + 1) & (kSlots4 - 1);
                    }
                    const unsigned long long k1 =
                        ((unsigned long long)top_o << 32) | (0xffffffffu - top_i);
                    if (s >= 0) {
                        base = atomicAdd(&scnt[s], __popc(grp));
                        const unsigned long long old = atomicMax(&sk1[s], k1);
                        const unsigned long long lo2 = old < k1 ? old : k1;
                        const unsigned lo_o = (unsigned)(lo2 >> 32);
                        atomicMax(&so2[s], lo_o > sec_o ? lo_o : sec_o);
                        atomicMax(&sem[s], em);
                    } else {
                        Acc4 &ac = A.acc[target];
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
            tgt[k] = !valid ? -3 : (!dead ? -2 : target);
            rk[k] = rank;  // the rank in the target's segment, or the surviving segment
            slot[k] = cone_t ? s : -1;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < kSlots4; i += blockDim.x) {
            const int t = skey[i];
            if (t < 0) continue;
            Acc4 &ac = A.acc[t];
            sbase[i] = (int)atomicAdd(&ac.cnt, (unsigned)scnt[i]);
            const unsigned long long k1 = sk1[i];
            const unsigned long long old = atomicMax(&ac.key1, k1);
            const unsigned long long lo2 = old < k1 ? old : k1;
            const unsigned lo_o = (unsigned)(lo2 >> 32);
            atomicMax(&ac.o2, lo_o > so2[i] ? lo_o : so2[i]);
            atomicMax(&ac.emax, sem[i]);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kItems; k++) {
            const int v = tile * kTile + k * blockDim.x + threadIdx.x;
            if (tgt[k] == -3) continue;
            int r = tgt[k] == -2 ? rk[k] : 0;
            if (tgt[k] >= 0) r = slot[k] >= 0 ? sbase[slot[k]] + rk[k] : rk[k];
            A.code[v] = make_int2(tgt[k] == -3 ? -1 : tgt[k], r);
        }
    }
    const unsigned fs = __reduce_add_sync(0xffffffffu, fallbacks);
    if (lane == 0 && fs) atomicAdd(&H->fallbacks, (unsigned long long)fs);
}

// ---------------------------------------------------------------- T: table
// New segment table: surviving old segments and the new facets that got
// points; a block scan and one 64-bit atomic per block ((entries << 32) |
// points) keep it sorted by start.  New facets' farthest points are
// certified (top-2 gap against twice the largest error bound) or queued for
// the exact phase.
__global__ void __launch_bounds__(kBlock) k4_table(Params4 A, int par, int first)
{
    __shared__ long long wsum[33];
    __shared__ unsigned long long sbase;
    Hdr4 *H = A.hdr;
    if (*(volatile int *)&H->status) return;
    const int ne = first ? 0 : (int)(*(volatile unsigned long long *)&H->tab[par] >> 32);
    const int fc0 = first ? 0 : H->fc_iter[par];
    const int fc1 = H->fcount;
    const int m = ne + (fc1 - fc0);
    const Ent4 *old = A.ent[par];
    Ent4 *out = A.ent[par ^ 1];
    for (int base = blockIdx.x * blockDim.x; base < m; base += gridDim.x * blockDim.x) {
        const int j = base + threadIdx.x;
        int f = -1, len = 0;
        if (j < ne) {
            const Ent4 en = old[j];
            f = en.f;
            len = A.fac[f].alive ? en.len : 0;
        } else if (j < m) {
            f = fc0 + (j - ne);
            len = (int)A.acc[f].cnt;
        }
        const long long s = len > 0 ? ((1ll << 32) | (long long)len) : 0ll;
        long long tot;
        const long long ex = block_excl_scan64(s, wsum, &tot);
        if (threadIdx.x == 0) sbase = tot ? atomicAdd(&H->tab[par ^ 1], (unsigned long long)tot) : 0ull;
        __syncthreads();
        if (len > 0) {
            const unsigned long long b = sbase + (unsigned long long)ex;
            const int k = (int)(b >> 32), st = (int)(b & 0xffffffffull);
            Ent4 en;
            en.f = f;
            en.start = st;
            en.len = len;
            en.pad = 0;
            out[k] = en;
            A.nstart[f] = st;
            if (j >= ne) {
                const Acc4 a = A.acc[f];
                A.apex[f] = key_idx(a.key1);
                bool cert = true;
                const float em = __uint_as_float(a.emax);
                const float d1 = key_dist(a.key1);
                if (a.cnt > 1) {
                    const double gap = ((double)d1 - (double)unord_f32(a.o2)) * (1.0 - 0x1p-50);
                    cert = gap > 2.0 * (double)em;
                }
                if (!cert) {
                    const double thr = (double)d1 - 3.0 * (double)em - fabs((double)d1) * 0x1p-20;
                    A.thr[f] = isfinite(thr) ? __double2float_rd(thr) : -INFINITY;
                    A.uncert[atomicAdd(&H->n_uncert, 1)] = k;
                }
            }
        }
        __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) H->fc_iter[par ^ 1] = fc1;
}

// ---------------------------------------------------------------- B: scatter
template <bool FIRST>
__global__ void __launch_bounds__(kBlock) k4_scatter(Params4 A, int par)
{
    Hdr4 *H = A.hdr;
    if (*(volatile int *)&H->status) return;
    const unsigned long long tb = *(volatile unsigned long long *)&H->tab[par];
    const int L = FIRST ? A.n : (int)(tb & 0xffffffffull);
    const Ent4 *ent = A.ent[par];
    float4 *Q = A.pts[par ^ 1];
    int *QI = A.pidx[par ^ 1];
    for (long long vv = (long long)blockIdx.x * blockDim.x + threadIdx.x; vv < L;
         vv += (long long)gridDim.x * blockDim.x) {
        const int v = (int)vv;
        int dst = -1;
        const int2 cr = A.code[v];
        if (cr.x == -2) {  // a surviving facet: the segment (cr.y) moves whole
            const Ent4 en = ent[cr.y];
            dst = A.nstart[en.f] + (v - en.start);
        } else if (cr.x >= 0) {
            dst = A.nstart[cr.x] + cr.y;
        }
        if (dst < 0) continue;
        if (dst >= A.n) {  // inconsistent counts: internal error, no write
            set_status4(H, QH_ERR_CAPACITY);
            continue;
        }
        if (FIRST) {
            Q[dst] = load4(A, v);
            QI[dst] = v;
        } else {
            Q[dst] = A.pts[par][v];
            QI[dst] = A.pidx[par][v];
        }
    }
}

// ---------------------------------------------------------------- X: exact apex
// One block per uncertified facet (of the table par ^ 1): its points whose
// filter value reaches the threshold, compared exactly (lowest index on
// ties).
__global__ void __launch_bounds__(kBlock) k4_exact(Params4 A, int par)
{
    __shared__ int sidx[kBlock];
    __shared__ float4 sp[kBlock];
    Hdr4 *H = A.hdr;
    if (*(volatile int *)&H->status) return;
    const int nu = *(volatile int *)&H->n_uncert;
    const Ent4 *ent = A.ent[par ^ 1];
    const float4 *Q = A.pts[par ^ 1];
    const int *QI = A.pidx[par ^ 1];
    for (int u = blockIdx.x; u < nu; u += gridDim.x) {
        const Ent4 en = ent[A.uncert[u]];
        const Fac4 F = A.fac[en.f];
        float a[4], b[4], c[4], d[4];
        load4a(A, F.v[0], a);
        load4a(A, F.v[1], b);
        load4a(A, F.v[2], c);
        load4a(A, F.v[3], d);
        const float thr = A.thr[en.f];
        int best = -1;
        float4 bp = make_float4(0, 0, 0, 0);
        for (int i = threadIdx.x; i < en.len; i += blockDim.x) {
            const float4 p = Q[en.start + i];
            float dv, e;
            plane4_value(A.pl[en.f], p, dv, e);
            if (isfinite(e) && (double)dv + (double)e < (double)thr) continue;
            const int idx = QI[en.start + i];
            if (best >= 0) {
                const float p1[4] = {p.x, p.y, p.z, p.w}, p2[4] = {bp.x, bp.y, bp.z, bp.w};
                const int s = cmp_dist4_slow(a, b, c, d, p1, p2);
                if (!(s > 0 || (s == 0 && idx < best))) continue;
            }
            best = idx;
            bp = p;
        }
        sidx[threadIdx.x] = best;
        sp[threadIdx.x] = bp;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) {
                const int oi = sidx[threadIdx.x + s], mi = sidx[threadIdx.x];
                if (oi >= 0) {
                    bool take = mi < 0;
                    if (!take) {
                        const float4 o = sp[threadIdx.x + s], me = sp[threadIdx.x];
                        const float po[4] = {o.x, o.y, o.z, o.w}, pm[4] = {me.x, me.y, me.z, me.w};
                        const int c2 = cmp_dist4_slow(a, b, c, d, po, pm);
                        take = c2 > 0 || (c2 == 0 && oi < mi);
                    }
                    if (take) {
                        sidx[threadIdx.x] = oi;
                        sp[threadIdx.x] = sp[threadIdx.x + s];
                    }
                }
            }
            __syncthreads();
        }
        if (threadIdx.x == 0 && sidx[0] >= 0) A.apex[en.f] = sidx[0];
        __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) H->exact_argmax += nu;
}

// ---------------------------------------------------------------- S: select
// lanes of this warp below the calling lane
__device__ __forceinline__ unsigned lanemask_lt4()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// The selection with one warp per candidate: the breadth-first frontier
// spread over the lanes (each frontier facet's four neighbours, duplicates
// merged by __match_any_sync), the lists in shared memory, new entries
// appended by ballots.  Per candidate: V = the facets its apex is strictly
// above, reached across ridges from its own facet; N = the facets next to V
// that are not in V; over the lists' capacity the candidate sits out.
__global__ void __launch_bounds__(kBlock) k4_select_warp(Params4 A, int par, int iter)
{
    __shared__ int sV[kBlock / 32][kV];
    __shared__ int sN[kBlock / 32][kN];
    Hdr4 *H = A.hdr;
    if (*(volatile int *)&H->status) return;
    const int ne = (int)(*(volatile unsigned long long *)&H->tab[par] >> 32);
    const Ent4 *ent = A.ent[par];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = lanemask_lt4();
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    int *V = sV[warp];
    int *N = sN[warp];
    unsigned fallbacks = 0;
    int nact = 0;
    for (int e = gw; e < ne; e += nw) {
        const Ent4 en = ent[e];
        const float4 q = load4(A, A.apex[en.f]);
        if (lane == 0) V[0] = en.f;
        int nv = 1, nn = 0, done = 0;
        bool over = false;
        __syncwarp();
        while (done < nv && !over) {
            const int lo = done, cnt = 4 * (nv - done);
            done = nv;
            for (int b0 = 0; b0 < cnt && !over; b0 += 32) {
                const int it = b0 + lane;
                int g = -1;
                bool bad = false;
                if (it < cnt) {
                    g = A.fac[V[lo + (it >> 2)]].nb[it & 3];
                    if (g < 0 || g >= A.fcap) {  // an unlinked ridge: internal error
                        bad = true;
                        g = -1;
                    }
                }
                if (__any_sync(0xffffffffu, bad)) {
                    if (lane == 0) set_status4(H, QH_ERR_CAPACITY);
                    over = true;
                    break;
                }
                const unsigned same = __match_any_sync(0xffffffffu, g);
                bool keep = g >= 0 && lane == __ffs(same) - 1;
                for (int j = 0; j < nv && keep; j++) keep = V[j] != g;
                for (int j = 0; j < nn && keep; j++) keep = N[j] != g;
                bool vis = false;
                if (keep) {
                    float d, err;
                    vis = facet_sign4(A, g, q, d, err, fallbacks) > 0;
                }
                const unsigned bv = __ballot_sync(0xffffffffu, keep && vis);
                const unsigned bn = __ballot_sync(0xffffffffu, keep && !vis);
                if (nv + __popc(bv) > kV || nn + __popc(bn) > kN) {
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
            int *Vg = A.vpool + (size_t)e * kV;
            int *Ng = A.npool + (size_t)e * kN;
            const unsigned long long mine = claim_key4(iter, 0, en.f, en.len);
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
    const unsigned f = __reduce_add_sync(0xffffffffu, fallbacks);
    if (lane == 0 && f) atomicAdd(&H->fallbacks, (unsigned long long)f);
    const int na = __reduce_add_sync(0xffffffffu, nact);
    if (lane == 0 && na) atomicAdd(&H->nact[0], na);
}

// Cone of one winner (one thread): one new facet per horizon ridge (the
// visible facet with the ridge's opposite vertex replaced by the apex keeps
// the outward orientation), the horizon neighbour relinked, the new facets
// linked to each other across their ridges through the apex (each holds the
// apex and an edge of the horizon, shared by exactly two horizon ridges).
// hz: scratch for the horizon ridges (capacity hcap); cl: the claims of the
// winner's round (g is in V exactly when cl[g] == mine).
__device__ bool build_cone4(const Params4 &A, int f0, int len, const int *V, int nv, int *hz,
                            int hcap, int iter, int round, const unsigned long long *cl)
{
    Hdr4 *H = A.hdr;
    const unsigned long long mine = claim_key4(iter, round, f0, len);
    const int qi = A.apex[f0];
    int nh = 0;
    for (int i = 0; i < nv; i++) {
        const Fac4 &F = A.fac[V[i]];
        for (int k = 0; k < 4; k++) {
            if (F.nb[k] < 0 || F.nb[k] >= A.fcap) {  // an unlinked ridge: internal error
                set_status4(H, QH_ERR_CAPACITY);
                return false;
            }
            if (cl[F.nb[k]] == mine) continue;
            if (nh == hcap) {
                set_status4(H, QH_ERR_CAPACITY);
                return false;
            }
            hz[nh++] = V[i] * 4 + k;
        }
    }
    const int base = atomicAdd(&H->fcount, nh);
    if (base + nh > A.fcap) {
        set_status4(H, QH_ERR_CAPACITY);
        return false;
    }
    for (int j = 0; j < nh; j++) {
        const int hf = hz[j] >> 2, k = hz[j] & 3;
        const Fac4 F = A.fac[hf];
        int v[4] = {F.v[0], F.v[1], F.v[2], F.v[3]};
        v[k] = qi;
        init_facet4(A, base + j, v);
        const int g = F.nb[k];
        A.fac[base + j].nb[k] = g;
        Fac4 &G = A.fac[g];
        for (int t = 0; t < 4; t++)
            if (G.nb[t] == hf) G.nb[t] = base + j;
    }
    // ridges through the apex: facet j's ridge opposite v[i] (v[i] != q)
    // holds q and the edge {v[t] : t != i, v[t] != q}
    for (int j = 0; j < nh; j++) {
        Fac4 &C = A.fac[base + j];
        for (int i = 0; i < 4; i++) {
            if (C.v[i] == qi || C.nb[i] >= 0) continue;
            int e[2], m = 0;
            for (int t = 0; t < 4; t++)
                if (t != i && C.v[t] != qi) e[m++] = C.v[t];
            for (int g = 0; g < nh; g++) {
                if (g == j) continue;
                Fac4 &D = A.fac[base + g];
                int has = 0, other = -1;
                for (int t = 0; t < 4; t++) {
                    if (D.v[t] == e[0] || D.v[t] == e[1]) has++;
                    else if (D.v[t] != qi) other = t;
                }
                if (has == 2 && other >= 0) {
                    C.nb[i] = base + g;
                    D.nb[other] = base + j;
                    break;
                }
            }
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

// The same cone built by one warp.  The horizon ridges by ballots; the
// lanes create the cone facets, relink their horizon neighbours and keep
// the cone's vertex lists in the warp's shared scratch sf (kN x 4); the
// facet across facet j's ridge opposite v[i] (v[i] not the apex) is the
// other cone facet holding the two vertices of j other than v[i] and the
// apex, found by a scan of sf.  Returns 1 when built, -1 on a capacity
// failure (status raised).
__device__ int cone4_warp(const Params4 &A, int f0, int len, const int *V, int nv, int *hz,
                          int hcap, int iter, int round, const unsigned long long *cl,
                          int (*sf)[4])
{
    Hdr4 *H = A.hdr;
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt4();
    const unsigned long long mine = claim_key4(iter, round, f0, len);
    const int qi = A.apex[f0];
    int nh = 0;
    bool bad = false;
    for (int p0 = 0; p0 < 4 * nv; p0 += 32) {
        const int p = p0 + lane;
        bool is_h = false;
        if (p < 4 * nv) {
            const int g = A.fac[V[p >> 2]].nb[p & 3];
            if (g < 0 || g >= A.fcap) bad = true;  // an unlinked ridge: internal error
            else is_h = cl[g] != mine;
        }
        const unsigned b = __ballot_sync(0xffffffffu, is_h);
        if (is_h) {
            const int pos = nh + __popc(b & lt);
            if (pos < hcap) hz[pos] = V[p >> 2] * 4 + (p & 3);
        }
        nh += __popc(b);
    }
    if (__any_sync(0xffffffffu, bad) || nh > hcap || nh > kN) {
        if (lane == 0) set_status4(H, QH_ERR_CAPACITY);
        return -1;
    }
    __syncwarp();
    int base = 0;
    if (lane == 0) base = atomicAdd(&H->fcount, nh);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base + nh > A.fcap) {
        if (lane == 0) set_status4(H, QH_ERR_CAPACITY);
        return -1;
    }
    // the cone facets: the horizon facet's vertices with the ridge's
    // opposite vertex replaced by the apex; their vertex lists in sf
    for (int j = lane; j < nh; j += 32) {
        const int hf = hz[j] >> 2, k = hz[j] & 3;
        const Fac4 F = A.fac[hf];
        int v[4] = {F.v[0], F.v[1], F.v[2], F.v[3]};
        v[k] = qi;
        init_facet4(A, base + j, v);
        const int g = F.nb[k];
        A.fac[base + j].nb[k] = g;
        Fac4 &G = A.fac[g];
        for (int t = 0; t < 4; t++)
            if (G.nb[t] == hf) G.nb[t] = base + j;
        for (int t = 0; t < 4; t++) sf[j][t] = v[t];
    }
    __syncwarp();
    for (int j = lane; j < nh; j += 32) {
        int v[4];
        for (int t = 0; t < 4; t++) v[t] = sf[j][t];
        for (int i = 0; i < 4; i++) {
            if (v[i] == qi) continue;
            int e[2], m = 0;
            for (int t = 0; t < 4; t++)
                if (t != i && v[t] != qi) e[m++] = v[t];
            int nbr = -1;
            for (int g = 0; g < nh && nbr < 0; g++) {
                if (g == j) continue;
                int has = 0;
                for (int t = 0; t < 4; t++) has += sf[g][t] == e[0] || sf[g][t] == e[1];
                if (has == 2) nbr = base + g;
            }
            A.fac[base + j].nb[i] = nbr;
        }
    }
    for (int i = lane; i < nv; i += 32) {
        A.fac[V[i]].alive = 0;
        A.taken[V[i]] = iter;
        A.cone[V[i]] = make_int4(base, nh, qi, iter);
    }
    if (lane == 0) {
        atomicAdd(&H->hull_vertices, 1);
        atomicAdd(&H->nwin, 1);
    }
    __syncwarp();
    return 1;
}

// Round r, one warp per candidate (the lanes read the lists and the claims
// side by side): out if an earlier round's winner deleted a facet of V or N;
// a winner owns every facet of V in this round's claims and no facet of N
// carries a higher one, and its warp builds its cone; a loser claims its
// visible facets for round r + 1 in the other claim array.
__global__ void __launch_bounds__(kBlock) k4_round_warp(Params4 A, int par, int iter, int r,
                                                        int last)
{
    Hdr4 *H = A.hdr;
    if (*(volatile int *)&H->status || *(volatile int *)&H->nact[r] == 0) return;
    const int ne = (int)(*(volatile unsigned long long *)&H->tab[par] >> 32);
    const Ent4 *ent = A.ent[par];
    const unsigned long long *cl = A.claim[r & 1];
    unsigned long long *cn = A.claim[(r + 1) & 1];
    __shared__ int sF[kBlock / 32][kN][4];  // each warp's cone vertex lists
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    int nact = 0;
    for (int e = gw; e < ne; e += nw) {
        if (A.cstate[e] != 0) continue;
        const int2 c = A.vn[e];
        int *V = A.vpool + (size_t)e * kV;
        int *N = A.npool + (size_t)e * kN;
        const Ent4 en = ent[e];
        const unsigned long long mine = claim_key4(iter, r, en.f, en.len);
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
            // the horizon list reuses the candidate's neighbour slice (kN >= 2 kV + 2)
            const int b = cone4_warp(A, en.f, en.len, V, c.x, N, kN, iter, r, cl,
                                     sF[threadIdx.x >> 5]);
            if (b > 0 && lane == 0) A.cstate[e] = 1;
        } else if (!last) {
            const unsigned long long next = claim_key4(iter, r + 1, en.f, en.len);
            for (int j = lane; j < c.x; j += 32) atomicMax(&cn[V[j]], next);
            nact++;
        }
    }
    if (!last && lane == 0 && nact) atomicAdd(&H->nact[r + 1], nact);
}

// No winner at all: the largest candidate (lowest facet on ties) inserted
// alone with lists of any size (one thread, global scratch).
__global__ void k4_fallback(Params4 A, int par, int iter)
{
    Hdr4 *H = A.hdr;
    if (threadIdx.x != 0 || H->status || H->nwin > 0) return;
    const int ne = (int)(H->tab[par] >> 32);
    const Ent4 *ent = A.ent[par];
    int f0 = INT_MAX, len = 0;
    for (int e = 0; e < ne; e++)
        if (ent[e].len > len || (ent[e].len == len && ent[e].f < f0)) {
            f0 = ent[e].f;
            len = ent[e].len;
        }
    if (f0 == INT_MAX) return;
    const float4 q = load4(A, A.apex[f0]);
    unsigned long long *cl = A.claim[kRounds4 & 1];
    const unsigned long long mine = claim_key4(iter, kRounds4, f0, len);
    int *V = A.big_v;
    int nv = 1;
    V[0] = f0;
    cl[f0] = mine;
    unsigned fb = 0;
    for (int i = 0; i < nv; i++) {
        for (int k = 0; k < 4; k++) {
            const int g = A.fac[V[i]].nb[k];
            if (g < 0 || g >= A.fcap) {
                set_status4(H, QH_ERR_CAPACITY);
                return;
            }
            if (cl[g] == mine || A.taken[g] == -iter) continue;
            float d, e;
            if (facet_sign4(A, g, q, d, e, fb) > 0) {
                cl[g] = mine;
                V[nv++] = g;
            } else {
                A.taken[g] = -iter;  // marked seen (not visible) in this search
            }
        }
    }
    build_cone4(A, f0, len, V, nv, A.big_h, A.fcap, iter, kRounds4, cl);
}

// Start of an iteration: counters of the rounds and of the tables.
__global__ void k4_iter_begin(Params4 A, int par, int iter)
{
    Hdr4 *H = A.hdr;
    if (threadIdx.x != 0) return;
    // (an iteration enqueued after the last segment was done changes
    // nothing, and is not counted)
    if (H->tab[par] != 0ull) H->iter = iter;
    H->nwin = 0;
    for (int r = 0; r < 8; r++) H->nact[r] = 0;
    H->tab[par ^ 1] = 0ull;
    H->n_uncert = 0;
    const unsigned long long tb = H->tab[par];
    H->seg_total += (long long)(tb >> 32);
    H->surv_total += (long long)(tb & 0xffffffffull);
}

// ---------------------------------------------------------------- output stage
// Simplices of the final triangulation -> canonical hull (see the file
// header).  Sizes are read back by the host between kernels.
__device__ __forceinline__ int uf_find4(int *par, int x)
{
    int p = *(volatile int *)&par[x];
    for (int guard = 0; p != x && guard < (1 << 26); guard++) {
        const int gp = *(volatile int *)&par[p];
        if (gp != p) par[x] = gp;
        x = p;
        p = gp;
    }
    return x;
}

// Exact sign of orient4(facet f, point w) (w given by index).
__device__ __forceinline__ int facet_sign_idx4(const Params4 &A, int f, int w, unsigned &fb)
{
    float d, e;
    return facet_sign4(A, f, load4(A, w), d, e, fb);
}

// Alive simplices, and per ridge whether the neighbour lies on the same
// hyperplane (its vertex opposite the ridge has orient4 = 0).
__global__ void __launch_bounds__(kBlock) k4o_alive(Params4 A, int *alive, int *label, int *cop)
{
    Hdr4 *H = A.hdr;
    const int fc = H->fcount;
    unsigned fb = 0;
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < fc; f += gridDim.x * blockDim.x) {
        const Fac4 F = A.fac[f];
        if (!F.alive) continue;
        alive[atomicAdd(&H->nalive, 1)] = f;
        label[f] = f;
        int bits = 0;
        for (int k = 0; k < 4; k++) {
            if (F.nb[k] < 0 || F.nb[k] >= A.fcap) {  // an unlinked ridge: internal error
                set_status4(H, QH_ERR_CAPACITY);
                continue;
            }
            const Fac4 &G = A.fac[F.nb[k]];
            int opp = -1;
            for (int t = 0; t < 4; t++) {
                const int x = G.v[t];
                if (x != F.v[0] && x != F.v[1] && x != F.v[2] && x != F.v[3]) opp = x;
            }
            if (opp >= 0 && facet_sign_idx4(A, f, opp, fb) == 0) bits |= 1 << k;
        }
        cop[f] = bits;
    }
}

__global__ void __launch_bounds__(kBlock) k4o_union(Params4 A, const int *alive, int *label,
                                                    const int *cop)
{
    Hdr4 *H = A.hdr;
    const int na = H->nalive;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < na; i += gridDim.x * blockDim.x) {
        const int f = alive[i];
        const int bits = cop[f];
        for (int k = 0; k < 4; k++) {
            if (!(bits & (1 << k))) continue;
            int a = f, b = A.fac[f].nb[k];
            int guard = 0;
            for (; guard < (1 << 20); guard++) {
                a = uf_find4(label, a);
                b = uf_find4(label, b);
                if (a == b) break;
                if (a < b) {
                    const int t = a;
                    a = b;
                    b = t;
                }
                if (atomicCAS(&label[a], a, b) == a) break;
            }
            if (guard == (1 << 20)) H->uf_fail = 1;
        }
    }
}

// Labels to roots; the (vertex << 32 | facet) pairs of the stars.
__global__ void __launch_bounds__(kBlock) k4o_compress_pairs(Params4 A, const int *alive,
                                                             int *label,
                                                             unsigned long long *key, int *val)
{
    Hdr4 *H = A.hdr;
    const int na = H->nalive;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < na; i += gridDim.x * blockDim.x) {
        const int f = alive[i];
        label[f] = uf_find4(label, f);
        for (int k = 0; k < 4; k++) {
            key[4 * i + k] = ((unsigned long long)(unsigned)A.fac[f].v[k] << 32) | (unsigned)f;
            val[4 * i + k] = 0;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) H->npair = 4 * na;
}

// A vertex (a run of the sorted star pairs) is extreme when no other vertex
// of its star lies on every hyperplane of its star.
__global__ void __launch_bounds__(kBlock) k4o_extreme(Params4 A, const unsigned long long *key,
                                                      int *ext)
{
    Hdr4 *H = A.hdr;
    const int m = H->npair;
    unsigned fb = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const int v = (int)(key[i] >> 32);
        if (i > 0 && (int)(key[i - 1] >> 32) == v) continue;
        int j = i;
        while (j < m && (int)(key[j] >> 32) == v) j++;
        bool extreme = true;
        for (int a = i; a < j && extreme; a++) {
            const Fac4 Fa = A.fac[(int)(key[a] & 0xffffffffull)];
            for (int t = 0; t < 4 && extreme; t++) {
                const int wv = Fa.v[t];
                if (wv == v) continue;
                bool on_all = true;
                for (int b = i; b < j && on_all; b++) {
                    const int fbi = (int)(key[b] & 0xffffffffull);
                    const Fac4 &Fb = A.fac[fbi];
                    if (Fb.v[0] == wv || Fb.v[1] == wv || Fb.v[2] == wv || Fb.v[3] == wv) continue;
                    on_all = facet_sign_idx4(A, fbi, wv, fb) == 0;
                }
                if (on_all) extreme = false;
            }
        }
        ext[v] = extreme ? 1 : 0;
    }
}

// (root << 32 | vertex) for every extreme vertex of every alive simplex.
__global__ void __launch_bounds__(kBlock) k4o_group_pairs(Params4 A, const int *alive,
                                                          const int *label, const int *ext,
                                                          unsigned long long *key, int *val)
{
    Hdr4 *H = A.hdr;
    const int na = H->nalive;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < na; i += gridDim.x * blockDim.x) {
        const int f = alive[i];
        const unsigned r = (unsigned)label[f];
        for (int k = 0; k < 4; k++) {
            const int v = A.fac[f].v[k];
            if (!ext[v]) continue;
            const int p = atomicAdd(&H->npair, 1);
            key[p] = ((unsigned long long)r << 32) | (unsigned)v;
            val[p] = 0;
        }
    }
}

// first-of-run flags: kind 0, of the whole key; kind 1, of its high half
__global__ void __launch_bounds__(kBlock) k4o_flags(const unsigned long long *key, const int *m_ptr,
                                                    int kind, int *flag)
{
    const int m = *m_ptr;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        bool first = i == 0;
        if (!first) first = kind == 0 ? key[i] != key[i - 1] : (key[i] >> 32) != (key[i - 1] >> 32);
        flag[i] = first;
    }
}

__global__ void __launch_bounds__(kBlock) k4o_compact(const unsigned long long *key, const int *m_ptr,
                                                      const int *flag, const long long *pos,
                                                      unsigned long long *out)
{
    const int m = *m_ptr;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
        if (flag[i]) out[pos[i]] = key[i];
}

__global__ void __launch_bounds__(kBlock) k4o_gstart(const int *m_ptr, const int *flag,
                                                     const long long *pos, int *gstart, int *order)
{
    const int m = *m_ptr;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
        if (flag[i]) {
            gstart[pos[i]] = i;
            order[pos[i]] = (int)pos[i];
        }
    if (blockIdx.x == 0 && threadIdx.x == 0 && m > 0) gstart[pos[m - 1] + flag[m - 1]] = m;
}

// Sort key of pass p (lexicographic order, least significant pass first):
// list elements 2p and 2p + 1 of the group, each + 1, 0 past the list's end.
__global__ void __launch_bounds__(kBlock) k4o_lexkey(const unsigned long long *ukey,
                                                     const int *gstart, const int *order,
                                                     const int *ng_ptr, int p,
                                                     unsigned long long *gkey)
{
    const int ng = *ng_ptr;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ng; i += gridDim.x * blockDim.x) {
        const int g = order[i];
        const int s = gstart[g], len = gstart[g + 1] - s;
        const unsigned hi = 2 * p < len ? (unsigned)(ukey[s + 2 * p] & 0xffffffffull) + 1u : 0u;
        const unsigned lo = 2 * p + 1 < len ? (unsigned)(ukey[s + 2 * p + 1] & 0xffffffffull) + 1u : 0u;
        gkey[i] = ((unsigned long long)hi << 32) | lo;
    }
}

__global__ void __launch_bounds__(kBlock) k4o_lens(const int *gstart, const int *order,
                                                   const int *ng_ptr, int *len)
{
    const int ng = *ng_ptr;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ng; i += gridDim.x * blockDim.x)
        len[i] = gstart[order[i] + 1] - gstart[order[i]];
}

__global__ void __launch_bounds__(kBlock) k4o_write(const unsigned long long *ukey,
                                                    const int *gstart, const int *order,
                                                    const int *ng_ptr, const long long *foff,
                                                    const long long *ftot, int32_t *facet_off,
                                                    int32_t *facet_idx)
{
    const int ng = *ng_ptr;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ng; i += gridDim.x * blockDim.x) {
        const int g = order[i];
        const int s = gstart[g], len = gstart[g + 1] - s;
        const long long o = foff[i];
        facet_off[i] = (int32_t)o;
        for (int t = 0; t < len; t++) facet_idx[o + t] = (int32_t)(ukey[s + t] & 0xffffffffull);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) facet_off[ng] = (int32_t)*ftot;
}

__global__ void __launch_bounds__(kBlock) k4o_verts(const int *ext, int n, const long long *pos,
                                                    int32_t *verts)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (ext[i]) verts[pos[i]] = i;
}

// ---------------------------------------------------------------- layout
static size_t au4(size_t v) { return (v + 255) & ~(size_t)255; }

struct Layout4 {
    size_t hdr, fac, pl, acc, apex, claim[2], cone, taken, thr, nstart, big_v, big_h;
    size_t ent[2], vn, cstate, vpool, npool, uncert, pts[2], pidx[2], code;
    size_t blk_a, blk_b, blk_ai, blk_bi, blk_v, blk_i;
    // output stage
    size_t alive, label, cop, key[2], val[2], ext, flag, pos, ukey, gstart, order[2], gkey[2],
        len, foff, hist, hist_off, tmp, cnt;
    size_t total;
    int fcap, ecap;
    long long pcap;
};

constexpr int kMaxGrid4 = 4096;

static Layout4 layout4d(int64_t n)
{
    Layout4 L = {};
    size_t o = 0;
    auto take = [&](size_t b) {
        const size_t r = o;
        o = au4(o + b);
        return r;
    };
    const size_t np = (size_t)(n > 0 ? n : 1);
    L.fcap = (int)(32 * np + 1024);
    L.ecap = (int)(np + 64);
    const size_t fc = (size_t)L.fcap + 1;  // + the pseudo facet of the first pass
    L.pcap = 4ll * (long long)fc;
    L.hdr = take(sizeof(Hdr4));
    L.fac = take(fc * sizeof(Fac4));
    L.pl = take(fc * sizeof(Plane4));
    L.acc = take(fc * sizeof(Acc4));
    L.apex = take(fc * 4);
    for (int b = 0; b < 2; b++) L.claim[b] = take(fc * 8);
    L.cone = take(fc * sizeof(int4));
    L.taken = take(fc * 4);
    L.thr = take(fc * 4);
    L.nstart = take(fc * 4);
    L.big_v = take(fc * 4);
    L.big_h = take(fc * 4);
    for (int b = 0; b < 2; b++) L.ent[b] = take((size_t)L.ecap * sizeof(Ent4));
    L.vn = take((size_t)L.ecap * sizeof(int2));
    L.cstate = take((size_t)L.ecap * 4);
    L.vpool = take((size_t)L.ecap * kV * 4);
    L.npool = take((size_t)L.ecap * kN * 4);
    L.uncert = take((size_t)L.ecap * 4);
    for (int b = 0; b < 2; b++) {
        L.pts[b] = take(np * sizeof(float4));
        L.pidx[b] = take(np * 4);
    }
    L.code = take(np * sizeof(int2));
    L.blk_a = take(kMaxGrid4 * sizeof(float4));
    L.blk_b = take(kMaxGrid4 * sizeof(float4));
    L.blk_ai = take(kMaxGrid4 * 4);
    L.blk_bi = take(kMaxGrid4 * 4);
    L.blk_v = take(kMaxGrid4 * 4);
    L.blk_i = take(kMaxGrid4 * 4);
    const size_t pc = (size_t)L.pcap;
    L.alive = take(fc * 4);
    L.label = take(fc * 4);
    L.cop = take(fc * 4);
    for (int b = 0; b < 2; b++) {
        L.key[b] = take(pc * 8);
        L.val[b] = take(pc * 4);
        L.order[b] = take(fc * 4);
        L.gkey[b] = take(fc * 8);
    }
    L.ext = take(np * 4);
    L.flag = take((pc > np ? pc : np) * 4);
    L.pos = take((pc > np ? pc : np) * 8);
    L.ukey = take(pc * 8);
    L.gstart = take((fc + 1) * 4);
    L.len = take(fc * 4);
    L.foff = take(fc * 8);
    const size_t tiles = (pc + d3::kScanTile - 1) / d3::kScanTile;
    L.hist = take(256 * tiles * 4 + 256);
    L.hist_off = take(256 * tiles * 8 + 256);
    L.tmp = take(((256 * tiles + pc + np) / d3::kScanTile + 64) * 8);
    L.cnt = take(64);
    L.total = o;
    return L;
}

static Params4 make_params4(const float *x, const float *y, const float *z, const float *w,
                            int64_t n, int64_t stride, char *ws, const Layout4 &L,
                            const qh_opts &o)
{
    Params4 A = {};
    A.x = x;
    A.y = y;
    A.z = z;
    A.w = w;
    A.stride = stride;
    A.n = (int)n;
    A.fcap = L.fcap;
    A.ecap = L.ecap;
    A.hdr = (Hdr4 *)(ws + L.hdr);
    A.fac = (Fac4 *)(ws + L.fac);
    A.pl = (Plane4 *)(ws + L.pl);
    A.acc = (Acc4 *)(ws + L.acc);
    A.apex = (int *)(ws + L.apex);
    for (int b = 0; b < 2; b++) {
        A.claim[b] = (unsigned long long *)(ws + L.claim[b]);
        A.ent[b] = (Ent4 *)(ws + L.ent[b]);
        A.pts[b] = (float4 *)(ws + L.pts[b]);
        A.pidx[b] = (int *)(ws + L.pidx[b]);
    }
    A.cone = (int4 *)(ws + L.cone);
    A.taken = (int *)(ws + L.taken);
    A.thr = (float *)(ws + L.thr);
    A.nstart = (int *)(ws + L.nstart);
    A.big_v = (int *)(ws + L.big_v);
    A.big_h = (int *)(ws + L.big_h);
    A.vn = (int2 *)(ws + L.vn);
    A.cstate = (int *)(ws + L.cstate);
    A.vpool = (int *)(ws + L.vpool);
    A.npool = (int *)(ws + L.npool);
    A.uncert = (int *)(ws + L.uncert);
    A.code = (int2 *)(ws + L.code);
    A.blk_a = (float4 *)(ws + L.blk_a);
    A.blk_b = (float4 *)(ws + L.blk_b);
    A.blk_ai = (int *)(ws + L.blk_ai);
    A.blk_bi = (int *)(ws + L.blk_bi);
    A.blk_v = (float *)(ws + L.blk_v);
    A.blk_i = (int *)(ws + L.blk_i);
    A.max_iters = o.max_iters > 0 ? o.max_iters : 4 * n + 16;
    return A;
}

}  // namespace d4
}  // namespace qh

using namespace qh;
using namespace qh::d4;

// facet ids must fit the 28-bit claim permutation and int32: 32n + 1024 < 2^28
constexpr int64_t kMax4d = 8000000;

extern "C" size_t qh_workspace_bytes_4d(int64_t n, const qh_opts *opts)
{
    (void)opts;
    if (n < 0 || n > kMax4d) return 0;
    return layout4d(n).total;
}

namespace {

// Per-iteration record of the last call made by this host thread:
// iteration, segments, live points, apexes inserted, uncertified apexes,
// host nanoseconds of the iteration (diagnostics).
thread_local std::vector<int64_t> g_tl4;

int grid_of4(long long items)
{
    const long long g = (items + kBlock - 1) / kBlock;
    return (int)std::max(1ll, std::min(g, 8ll * sm_count()));
}

cudaError_t read_hdr(const Params4 &A, Hdr4 &h, cudaStream_t st)
{
    cudaError_t e = cudaMemcpyAsync(&h, A.hdr, sizeof(Hdr4), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(st);
}

}  // namespace

extern "C" qh_status qh_hull4d(const float *d_x, const float *d_y, const float *d_z,
                               const float *d_w, int64_t n, int64_t stride, int32_t *d_verts,
                               int64_t *h_nv, int32_t *d_facet_off, int64_t max_facets,
                               int32_t *d_facet_idx, int64_t max_idx, int64_t *h_nf,
                               qh_result *h_result, void *d_ws, size_t ws_bytes,
                               const qh_opts *opts, cudaStream_t st)
{
    if (n < 0 || n > kMax4d || stride < 1 || !h_nv || !h_nf || !d_ws || max_facets < 0 ||
        max_idx < 0)
        return QH_ERR_INVALID_ARG;
    if (n > 0 && (!d_x || !d_y || !d_z || !d_w || !d_verts || !d_facet_off || !d_facet_idx))
        return QH_ERR_INVALID_ARG;
    if ((n - 1) * stride > (int64_t)1 << 40) return QH_ERR_INVALID_ARG;
    qh_opts o;
    qh_default_opts(&o);
    if (opts) o = *opts;
    const Layout4 L = layout4d(n);
    if (ws_bytes < L.total || ((uintptr_t)d_ws & 255)) return QH_ERR_NOMEM;
    *h_nv = 0;
    *h_nf = 0;
    qh_result r = {};
    auto finish = [&](qh_status s, const Hdr4 &h) {
        r.status = s;
        r.iterations = h.iter;
        r.survivor_total = h.surv_total;
        r.live_total = n + h.surv_total;
        r.segments_total = h.seg_total;
        r.filter_fallbacks = (int64_t)h.fallbacks;
        r.exact_argmax = (int64_t)h.exact_argmax;
        r.extra[0] = *h_nv;
        r.extra[1] = *h_nf;
        r.extra[2] = s == QH_OK ? h.nfidx : 0;
        if (h_result) *h_result = r;
        return s;
    };
    Hdr4 h = {};
    if (n == 0) {
        if (max_facets < 0) return QH_ERR_CAPACITY;
        if (cudaMemsetAsync(d_facet_off, 0, sizeof(int32_t), st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return QH_ERR_CUDA;
        return finish(QH_OK, h);
    }
    char *ws = (char *)d_ws;
    Params4 A = make_params4(d_x, d_y, d_z, d_w, n, stride, ws, L, o);
    if (cudaMemsetAsync(A.hdr, 0, sizeof(Hdr4), st) != cudaSuccess) return QH_ERR_CUDA;
    const int g = grid_of4(n);
    // ---- first simplex
    k4_extrema<<<g, kBlock, 0, st>>>(A);
    k4_extrema_final<<<1, 32, 0, st>>>(A, g);
    if (read_hdr(A, h, st) != cudaSuccess) return QH_ERR_CUDA;
    if (h.status) return finish((qh_status)h.status, h);
    if (n < 5) return finish(QH_ERR_DEGENERATE, h);
    for (int step = 2; step <= 4; step++) {
        k4_basis<<<1, 32, 0, st>>>(A, step);
        k4_far<<<g, kBlock, 0, st>>>(A);
        k4_far_final<<<1, 32, 0, st>>>(A, g, step);
        k4_search<<<g, kBlock, 0, st>>>(A, step);
        k4_take<<<1, 32, 0, st>>>(A, step);
        if (read_hdr(A, h, st) != cudaSuccess) return QH_ERR_CUDA;
        if (h.status) return finish((qh_status)h.status, h);
    }
    k4_build<<<1, 32, 0, st>>>(A);
    // ---- first assignment: every point against the simplex; table 1, buffer 1
    k4_assign<true><<<grid_of4((n + kItems - 1) / kItems), kBlock, 0, st>>>(A, 0);
    k4_table<<<grid_of4(64), kBlock, 0, st>>>(A, 0, 1);
    k4_scatter<true><<<g, kBlock, 0, st>>>(A, 0);
    if (read_hdr(A, h, st) != cudaSuccess) return QH_ERR_CUDA;
    if (h.status) return finish((qh_status)h.status, h);
    if (h.n_uncert > 0) k4_exact<<<std::min(h.n_uncert, 8 * sm_count()), kBlock, 0, st>>>(A, 0);
    // ---- iterations: table `cur` describes the live points in buffer `cur`
    int cur = 1, iter = 0;
    g_tl4.clear();
    auto t_prev = std::chrono::steady_clock::now();
    // up to kBatch iterations are enqueued between two reads of the header:
    // every kernel takes its sizes from the header on the device, so an
    // iteration enqueued after the hull is done does nothing; the grids of
    // the batch's later iterations allow for growth (any grid is correct)
    constexpr int kBatch = 4;
    for (;;) {
        if (read_hdr(A, h, st) != cudaSuccess) return QH_ERR_CUDA;
        if (h.status) return finish((qh_status)h.status, h);
        const int ne = (int)(h.tab[cur] >> 32), Lc = (int)(h.tab[cur] & 0xffffffffull);
        if (iter > 0 && g_tl4.size() < 9 * 4096) {
            const auto t = std::chrono::steady_clock::now();
            g_tl4.insert(g_tl4.end(), {iter, ne, Lc, h.nwin, h.n_uncert,
                                       (int64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
                                           t - t_prev).count(),
                                       h.nact[0], h.nact[1], h.nact[2]});
            t_prev = t;
        }
        if (ne == 0) break;
        if (iter >= A.max_iters) return finish(QH_ERR_NO_CONVERGENCE, h);
        const int nb = (int)std::min<long long>(kBatch, A.max_iters - iter);
        for (int b = 0; b < nb; b++) {
            ++iter;
            const long long grow = 1ll << (2 * b);
            const long long ne_b = (long long)ne * grow, L_b = std::min<long long>((long long)Lc, n);
            k4_iter_begin<<<1, 32, 0, st>>>(A, cur, iter);
            k4_select_warp<<<grid_of4(32ll * ne_b), kBlock, 0, st>>>(A, cur, iter);
            for (int rr = 0; rr < kRounds4; rr++)
                k4_round_warp<<<grid_of4(32ll * ne_b), kBlock, 0, st>>>(A, cur, iter, rr,
                                                                    rr == kRounds4 - 1);
            k4_fallback<<<1, 32, 0, st>>>(A, cur, iter);
            k4_assign<false><<<grid_of4((L_b + kItems - 1) / kItems), kBlock, 0, st>>>(A, cur);
            k4_table<<<grid_of4(ne_b + 64), kBlock, 0, st>>>(A, cur, 0);
            k4_scatter<false><<<grid_of4(L_b), kBlock, 0, st>>>(A, cur);
            // the exact step reads its count on the device
            k4_exact<<<2 * sm_count(), kBlock, 0, st>>>(A, cur);
            cur ^= 1;
        }
    }
    // ---- output stage
    using d3::radix_sort;
    using d3::scan_counts;
    int *alive = (int *)(ws + L.alive), *label = (int *)(ws + L.label), *cop = (int *)(ws + L.cop);
    unsigned long long *key0 = (unsigned long long *)(ws + L.key[0]),
                       *key1 = (unsigned long long *)(ws + L.key[1]);
    int *val0 = (int *)(ws + L.val[0]), *val1 = (int *)(ws + L.val[1]);
    int *ext = (int *)(ws + L.ext), *flag = (int *)(ws + L.flag);
    long long *pos = (long long *)(ws + L.pos);
    unsigned long long *ukey = (unsigned long long *)(ws + L.ukey);
    int *gstart = (int *)(ws + L.gstart), *len = (int *)(ws + L.len);
    int *order0 = (int *)(ws + L.order[0]), *order1 = (int *)(ws + L.order[1]);
    unsigned long long *gkey0 = (unsigned long long *)(ws + L.gkey[0]),
                       *gkey1 = (unsigned long long *)(ws + L.gkey[1]);
    long long *foff = (long long *)(ws + L.foff);
    int *hist = (int *)(ws + L.hist);
    long long *hist_off = (long long *)(ws + L.hist_off), *tmp = (long long *)(ws + L.tmp);
    long long *cnt = (long long *)(ws + L.cnt);  // [0] unique keys, [1] groups, [2] indices, [3] verts
    int *cnt_i = (int *)(ws + L.cnt + 32);        // the same as ints for the sorts' counts
    Hdr4 *H = A.hdr;
    const int gf = grid_of4(h.fcount);
    if (cudaMemsetAsync(ext, 0, (size_t)n * 4, st) != cudaSuccess) return QH_ERR_CUDA;
    k4o_alive<<<gf, kBlock, 0, st>>>(A, alive, label, cop);
    k4o_union<<<gf, kBlock, 0, st>>>(A, alive, label, cop);
    k4o_compress_pairs<<<gf, kBlock, 0, st>>>(A, alive, label, key0, val0);
    int vbits = 1;
    while ((1ll << vbits) <= n) vbits++;
    int fbits = 1;
    while ((1ll << fbits) <= L.fcap) fbits++;
    radix_sort(key0, val0, key1, val1, &H->npair, L.pcap, 32 + vbits, hist, hist_off, tmp,
               &H->sort_m, st);
    k4o_extreme<<<grid_of4(L.pcap), kBlock, 0, st>>>(A, key0, ext);
    if (cudaMemsetAsync(&H->npair, 0, sizeof(int), st) != cudaSuccess) return QH_ERR_CUDA;
    k4o_group_pairs<<<gf, kBlock, 0, st>>>(A, alive, label, ext, key0, val0);
    radix_sort(key0, val0, key1, val1, &H->npair, L.pcap, 32 + fbits, hist, hist_off, tmp,
               &H->sort_m, st);
    // unique (root, vertex) pairs, then groups (runs of equal roots)
    k4o_flags<<<grid_of4(L.pcap), kBlock, 0, st>>>(key0, &H->npair, 0, flag);
    scan_counts(flag, &H->npair, 0, L.pcap, pos, tmp, &cnt[0], st);
    k4o_compact<<<grid_of4(L.pcap), kBlock, 0, st>>>(key0, &H->npair, flag, pos, ukey);
    if (read_hdr(A, h, st) != cudaSuccess) return QH_ERR_CUDA;
    long long nuniq = 0;
    if (cudaMemcpyAsync(&nuniq, &cnt[0], 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return QH_ERR_CUDA;
    if (h.uf_fail) return finish(QH_ERR_CAPACITY, h);
    const int nu = (int)nuniq;
    if (cudaMemcpyAsync(&cnt_i[0], &nu, 4, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return QH_ERR_CUDA;
    k4o_flags<<<grid_of4(nu), kBlock, 0, st>>>(ukey, &cnt_i[0], 1, flag);
    scan_counts(flag, &cnt_i[0], 0, L.pcap, pos, tmp, &cnt[1], st);
    k4o_gstart<<<grid_of4(nu), kBlock, 0, st>>>(&cnt_i[0], flag, pos, gstart, order0);
    long long ng = 0;
    if (cudaMemcpyAsync(&ng, &cnt[1], 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return QH_ERR_CUDA;
    const int ngi = (int)ng;
    if (cudaMemcpyAsync(&cnt_i[1], &ngi, 4, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return QH_ERR_CUDA;
    // lexicographic order of the groups' lists (their first eight entries;
    // least significant pair first, each pass a stable sort)
    for (int p = 3; p >= 0; p--) {
        k4o_lexkey<<<grid_of4(ngi), kBlock, 0, st>>>(ukey, gstart, order0, &cnt_i[1], p, gkey0);
        radix_sort(gkey0, order0, gkey1, order1, &cnt_i[1], (long long)L.fcap + 1, 64, hist,
                   hist_off, tmp, &H->sort_m, st);
    }
    k4o_lens<<<grid_of4(ngi), kBlock, 0, st>>>(gstart, order0, &cnt_i[1], len);
    scan_counts(len, &cnt_i[1], 0, (long long)L.fcap + 1, foff, tmp, &cnt[2], st);
    scan_counts(ext, nullptr, (int)n, n, pos, tmp, &cnt[3], st);
    long long tot[4] = {0, 0, 0, 0};
    if (cudaMemcpyAsync(tot, cnt, 32, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return QH_ERR_CUDA;
    *h_nf = ng;
    *h_nv = tot[3];
    h.nfidx = tot[2];
    if (ng > max_facets || tot[2] > max_idx) return finish(QH_ERR_CAPACITY, h);
    k4o_write<<<grid_of4(ngi), kBlock, 0, st>>>(ukey, gstart, order0, &cnt_i[1], foff, &cnt[2],
                                                d_facet_off, d_facet_idx);
    k4o_verts<<<grid_of4(n), kBlock, 0, st>>>(ext, (int)n, pos, d_verts);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
        return QH_ERR_CUDA;
    if (read_hdr(A, h, st) != cudaSuccess) return QH_ERR_CUDA;
    h.nfidx = tot[2];
    return finish((qh_status)h.status, h);
}

extern "C" qh_status qh_debug_timeline_4d(int64_t *h_rows, int32_t max_rows, int32_t *h_nrows)
{
    if (!h_rows || !h_nrows || max_rows < 0) return QH_ERR_INVALID_ARG;
    const int rows = std::min((int)(g_tl4.size() / 9), (int)max_rows);
    std::memcpy(h_rows, g_tl4.data(), sizeof(int64_t) * 9 * (size_t)rows);
    *h_nrows = rows;
    return QH_OK;
}
