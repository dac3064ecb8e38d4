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

// ---------------------------------------------------------------- initial simplex
// Block-level reductions write one candidate per block; block 0 reduces them
// after a grid barrier.

__device__ void extrema3d(const Params3 &A, SmemAll3 &sm, int bid, int nb)
{
    float4 mn = make_float4(INFINITY, INFINITY, INFINITY, __int_as_float(INT_MAX));
    float4 mx = make_float4(-INFINITY, -INFINITY, -INFINITY, __int_as_float(INT_MAX));
    int bad = 0;
    for (long long i = (long long)bid * blockDim.x + threadIdx.x; i < A.n;
         i += (long long)nb * blockDim.x) {
        float4 p = load_input(A, i);
        p.x = canon0(p.x);
        p.y = canon0(p.y);
        p.z = canon0(p.z);
        bad |= !(isfinite(p.x) && isfinite(p.y) && isfinite(p.z));
        if (lex_less(p, mn)) mn = p;
        if (lex_greater_lowidx(p, mx)) mx = p;
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
    for (long long i = (long long)bid * blockDim.x + threadIdx.x; i < A.n;
         i += (long long)nb * blockDim.x) {
        float4 p = load_input(A, i);
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

// Block 0: reduce the per-block candidates of the previous phase.
__device__ void simplex_step(const Params3 &A, SmemAll3 &sm, int step, int nblk)
{
    Hdr3 *H = A.hdr;
    if (threadIdx.x != 0) return;
    if (step == 0) {
        float4 mn = A.blk_a[0], mx = A.blk_b[0];
        for (int b = 1; b < nblk; b++) {
            if (lex_less(A.blk_a[b], mn)) mn = A.blk_a[b];
            if (lex_greater_lowidx(A.blk_b[b], mx)) mx = A.blk_b[b];
        }
        H->pa = mn;
        H->pb = mx;
        if (mn.x == mx.x && mn.y == mx.y && mn.z == mx.z) set_status(H, QH_ERR_DEGENERATE);
    } else {
        float bv = A.blk_v[0];
        int bi = A.blk_i[0];
        for (int b = 1; b < nblk; b++) {
            if (A.blk_v[b] > bv || (A.blk_v[b] == bv && A.blk_i[b] < bi)) {
                bv = A.blk_v[b];
                bi = A.blk_i[b];
            }
        }
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
        Acc3 z = {};
        A.acc[base + o] = z;
        A.claim[base + o] = 0ull;
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
        Acc3 z = {};
        A.acc[base + o] = z;
        A.claim[base + o] = 0ull;
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
    if (bid == 0 && threadIdx.x == 0) H->fcount = 4 * A.ncloud;
}

// ---------------------------------------------------------------- S: select
// One thread per segment (candidate): visible-set BFS from its facet with
// exact tests.  V: visible facets, N: their non-visible neighbours.
template <int MODE>
__device__ void select3d(const Params3 &A, int par, int bid, int nb)
{
    Hdr3 *H = A.hdr;
    const int ne = *(volatile int *)&H->nent[par];
    const Ent3 *ent = A.ent[par];
    unsigned fallbacks = 0;
    for (int e = bid * blockDim.x + threadIdx.x; e < ne; e += nb * blockDim.x) {
        const int f0 = ent[e].f;
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
                const Fac3 &G = A.fac[g];
                const float *a, *b, *c;
                fac_pts(G, a, b, c);
                float d, err;
                orient3d_value<MODE>(a, b, c, q, d, err);
                if (orient3d_sign<MODE>(d, err, a, b, c, q, fallbacks) > 0) {
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
        }
        A.vn[e] = over ? make_int2(-1, -1) : make_int2(nv, nn);
        A.cstate[e] = over ? 2 : 0;
    }
    unsigned f = __reduce_add_sync(0xffffffffu, fallbacks);
    if ((threadIdx.x & 31) == 0 && f) atomicAdd(&H->fallbacks, (unsigned long long)f);
}

// Round `round` of the selection: every still-active candidate drops out if
// a winner of an earlier round deleted a facet of V or N (their regions would
// touch), else claims its visible facets.
__device__ void claim3d(const Params3 &A, int par, int iter, int round, int bid, int nb)
{
    Hdr3 *H = A.hdr;
    if (bid == 0 && threadIdx.x == 0) H->nactive[(round + 1) & 1] = 0;  // next round's counter
    const int ne = *(volatile int *)&H->nent[par];
    const Ent3 *ent = A.ent[par];
    for (int e = bid * blockDim.x + threadIdx.x; e < ne; e += nb * blockDim.x) {
        if (A.cstate[e] != 0) continue;
        const int2 c = A.vn[e];
        const int *V = A.vpool + (size_t)e * kVCap;
        const int *N = A.npool + (size_t)e * kNCap;
        bool touched = false;
        if (round > 0) {
            for (int j = 0; j < c.x && !touched; j++) touched = A.taken[V[j]] == iter;
            for (int j = 0; j < c.y && !touched; j++) touched = A.taken[N[j]] == iter;
        }
        if (touched) {
            A.cstate[e] = 2;
            continue;
        }
        const unsigned long long mine = claim_key(iter, round, ent[e].f, ent[e].len);
        for (int j = 0; j < c.x; j++) atomicMax(&A.claim[V[j]], mine);
        atomicAdd(&H->nactive[round & 1], 1);
    }
}

// Cone of one winner: horizon edges of V (edges whose neighbour is not in V),
// one facet (u, v, q) per horizon edge, neighbours relinked.  V and N are the
// winner's visible facets and horizon neighbours; hz is scratch for the
// horizon (capacity >= |V| + 2).
__device__ bool build_cone(const Params3 &A, int f0, int len, const int *V, int nv, int *hz,
                           int hcap, int iter, int round)
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
            if (A.claim[g] == mine) continue;  // g is in V
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
        Acc3 z = {};
        A.acc[base + j] = z;
        A.claim[base + j] = 0ull;
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

// ---------------------------------------------------------------- C: winners
// One warp per candidate that claimed in this round.  A winner owns every
// facet of V and no facet of N carries a higher claim; it builds its cone at
// once: horizon edges found by the lanes (ballot-compacted), one cone facet
// per horizon edge, the horizon neighbours relinked, and the cone facets
// linked around the apex by matching edge ends across lanes (shuffles).
__device__ void cone_warp(const Params3 &A, int e, int f0, int len, const int *V, int nv,
                          int *hz, int iter, int round)
{
    Hdr3 *H = A.hdr;
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    const unsigned long long mine = claim_key(iter, round, f0, len);
    const float4 q4 = A.apex[f0];
    const int qi = __float_as_int(q4.w);
    int nh = 0;
    for (int p0 = 0; p0 < 3 * nv; p0 += 32) {
        const int p = p0 + lane;
        bool is_h = false;
        if (p < 3 * nv) {
            const int i = p / 3, k = p - 3 * (p / 3);
            is_h = A.claim[A.fac[V[i]].nb[k]] != mine;
        }
        const unsigned b = __ballot_sync(0xffffffffu, is_h);
        if (is_h) {
            const int pos = nh + __popc(b & lt);
            if (pos < kNCap) hz[pos] = V[p / 3] * 3 + (p - 3 * (p / 3));
        }
        nh += __popc(b);
    }
    if (nh > kNCap) {  // a visible region that is not a disk: cannot happen
        if (lane == 0) set_status(H, QH_ERR_CAPACITY);
        return;
    }
    __syncwarp();
    int base = 0;
    if (lane == 0) base = atomicAdd(&H->fcount, nh);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base + nh > A.fcap) {
        if (lane == 0) set_status(H, QH_ERR_CAPACITY);
        return;
    }
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
        Acc3 z = {};
        A.acc[base + j] = z;
        A.claim[base + j] = 0ull;
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
    if (lane == 0) {
        atomicAdd(&H->hull_vertices, 1);
        atomicAdd(&H->nwin, 1);
        A.cstate[e] = 1;
    }
}

__device__ void cone3d(const Params3 &A, int par, int iter, int round, int bid, int nb)
{
    Hdr3 *H = A.hdr;
    const int ne = *(volatile int *)&H->nent[par];
    const Ent3 *ent = A.ent[par];
    const int lane = threadIdx.x & 31;
    const int gw = (bid * blockDim.x + threadIdx.x) >> 5, nw = (nb * blockDim.x) >> 5;
    // Candidates in groups of G per warp, G ~ candidates / warps (1..32): with
    // few candidates every candidate gets a warp (its lists checked by all
    // lanes, its cone built at once); with many, each lane checks one
    // candidate and the warp then builds the cones of the group's winners.
    const int G = min(32, max(1, (ne + nw - 1) / nw));
    for (int base = gw * G; base < ne; base += nw * G) {
        unsigned wins;
        if (G == 1) {
            const int e = base;
            bool ok = A.cstate[e] == 0;
            if (ok) {
                const int2 c = A.vn[e];
                const unsigned long long mine = claim_key(iter, round, ent[e].f, ent[e].len);
                const int *V = A.vpool + (size_t)e * kVCap;
                const int *N = A.npool + (size_t)e * kNCap;
                for (int j = lane; j < c.x; j += 32) ok &= A.claim[V[j]] == mine;
                for (int j = lane; j < c.y; j += 32) ok &= A.claim[N[j]] < mine;
            }
            wins = __all_sync(0xffffffffu, ok) ? 1u : 0u;
        } else {
            const int e = base + lane;
            bool win = false;
            if (lane < G && e < ne && A.cstate[e] == 0) {
                const int2 c = A.vn[e];
                const unsigned long long mine = claim_key(iter, round, ent[e].f, ent[e].len);
                const int *V = A.vpool + (size_t)e * kVCap;
                const int *N = A.npool + (size_t)e * kNCap;
                win = true;
                for (int j = 0; j < c.x && win; j++) win = A.claim[V[j]] == mine;
                for (int j = 0; j < c.y && win; j++) win = A.claim[N[j]] < mine;
            }
            wins = __ballot_sync(0xffffffffu, win);
        }
        while (wins) {
            const int l = __ffs(wins) - 1;
            wins &= wins - 1;
            const int ew = base + l;
            // the horizon list reuses the candidate's neighbour slice (>= |V| + 2)
            cone_warp(A, ew, ent[ew].f, ent[ew].len, A.vpool + (size_t)ew * kVCap,
                      A.vn[ew].x, A.npool + (size_t)ew * kNCap, iter, round);
        }
    }
}

// No winner at all means the highest-priority candidate overflowed its
// fixed-size lists: insert it alone with the large scratch (one thread).
template <int MODE>
__device__ void fallback3d(const Params3 &A, int par, int iter)
{
    Hdr3 *H = A.hdr;
    if (threadIdx.x != 0) return;
    const int ne = H->nent[par];
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
    A.claim[f0] = mine;
    unsigned fb = 0;
    for (int i = 0; i < nv; i++) {
        const Fac3 &F = A.fac[V[i]];
        for (int k = 0; k < 3; k++) {
            const int g = F.nb[k];
            if (A.claim[g] == mine || A.big_mark[g] == iter) continue;
            const Fac3 &G = A.fac[g];
            const float *a, *b, *c;
            fac_pts(G, a, b, c);
            float d, err;
            orient3d_value<MODE>(a, b, c, q, d, err);
            if (orient3d_sign<MODE>(d, err, a, b, c, q, fb) > 0) {
                A.claim[g] = mine;
                V[nv++] = g;
            } else {
                A.big_mark[g] = iter;
            }
        }
    }
    build_cone(A, f0, len, V, nv, A.big_h, A.fcap, iter, kRounds);
}

// ---------------------------------------------------------------- A: assign
// Target of every live point: its own facet if that facet survives (rank =
// position in the segment), else the first cone facet of its winner that it
// is strictly above (warp-aggregated count, rank and farthest-point key), else
// discarded (-1).  FIRST: the input points against the tetrahedron.
template <int MODE, int ITEMS, bool FIRST>
__device__ void assign3d(const Params3 &A, int par, SmemAll3 &sm, int bid, int nb)
{
    Hdr3 *H = A.hdr;
    const int L = FIRST ? A.n : *(volatile int *)&H->L[par];
    const Ent3 *ent = A.ent[par];
    const float4 *P = A.pts[par];
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    unsigned fallbacks = 0;
    const int T = A.tile;  // blockDim.x * ITEMS
    const int ntiles = (L + T - 1) / T;
    for (int tile = bid; tile < ntiles; tile += nb) {
        const int v0 = tile * T, v1 = min(v0 + T, L);
        __syncthreads();
        if (threadIdx.x == 0) {
            if (FIRST) {  // entries = the clouds the tile meets
                const int c0 = cloud_of(A, v0);
                sm.a.e0 = c0;
                sm.a.m = cloud_of(A, v1 - 1) - c0 + 1;
            } else {
                sm.a.e0 = A.tile_ent[tile];
                sm.a.m = A.tile_m[tile];
            }
        }
        for (int i = threadIdx.x; i < kSlots; i += blockDim.x) {
            sm.a.skey[i] = -1;
            sm.a.scnt[i] = 0;
            sm.a.sk1[i] = 0ull;
            sm.a.so2[i] = 0u;
            sm.a.sem[i] = 0u;
        }
        __syncthreads();
        const int e0 = sm.a.e0, m = sm.a.m;
        // FIRST: a tile that meets more clouds than the stage holds (runs of
        // empty clouds) searches the cloud offsets in global memory instead
        const bool staged = m <= kMaxTile;
        for (int i = threadIdx.x; i < m && i < kMaxTile; i += blockDim.x) {
            if (FIRST) {
                sm.a.start[i] = cloud_start(A, e0 + i);
                sm.a.f[i] = A.fcap + e0 + i;
            } else {
                sm.a.start[i] = ent[e0 + i].start;
                sm.a.f[i] = ent[e0 + i].f;
            }
        }
        __syncthreads();
        // ---- classify; cone targets get a tile-local slot (shared hash table)
        int tgt[ITEMS], rk[ITEMS], slot[ITEMS];
#pragma unroll
        for (int k = 0; k < ITEMS; k++) {
            const int v = v0 + k * blockDim.x + threadIdx.x;
            const bool valid = v < v1;
            int target = -1, rank = 0, s = -1;
            float d = 0.0f, err = 0.0f;
            int idx = 0;
            bool cone_t = false;
            if (valid) {
                int lo = 0, hi = m - 1, f;
                if (FIRST && !staged) {
                    lo = cloud_of(A, v) - e0;
                    f = A.fcap + e0 + lo;
                } else {
                    while (lo < hi) {
                        int mid = (lo + hi + 1) >> 1;
                        if (sm.a.start[mid] <= v) lo = mid;
                        else hi = mid - 1;
                    }
                    f = sm.a.f[lo];
                }
                const float4 p4 = FIRST ? load_input(A, v) : P[v];
                idx = __float_as_int(p4.w);
                const float p[3] = {p4.x, p4.y, p4.z};
                if (!FIRST && A.fac[f].alive) {
                    target = f;
                    rank = v - sm.a.start[lo];
                } else {
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
                        for (int c = 0; c < cn.y; c++) {
                            const Fac3 &C = A.fac[cn.x + c];
                            const float *a, *b, *cc;
                            fac_pts(C, a, b, cc);
                            orient3d_value<MODE>(a, b, cc, p, d, err);
                            if (orient3d_sign<MODE>(d, err, a, b, cc, p, fallbacks) > 0) {
                                target = cn.x + c;
                                cone_t = true;
                                break;
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
                    // find or insert the target's slot (linear probing)
                    int h = (int)(((unsigned)target * 0x9E3779B1u) >> (32 - kSlotBits));
                    for (int probe = 0; probe < kSlots; probe++) {
                        const int prev = atomicCAS(&sm.a.skey[h], -1, target);
                        if (prev == -1 || prev == target) {
                            s = h;
                            break;
                        }
                        h = (h + 1) & (kSlots - 1);
                    }
                    const unsigned long long k1 =
                        ((unsigned long long)top_o << 32) | (0xffffffffu - top_i);
                    if (s >= 0) {
                        base = atomicAdd(&sm.a.scnt[s], __popc(grp));
                        const unsigned long long old = atomicMax(&sm.a.sk1[s], k1);
                        const unsigned long long lo2 = old < k1 ? old : k1;
                        const unsigned lo_o = (unsigned)(lo2 >> 32);
                        atomicMax(&sm.a.so2[s], lo_o > sec_o ? lo_o : sec_o);
                        atomicMax(&sm.a.sem[s], em);
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
            tgt[k] = valid ? target : -2;
            rk[k] = rank;
            slot[k] = s;
        }
        __syncthreads();
        // ---- one global reservation and key merge per (tile, target)
        for (int i = threadIdx.x; i < kSlots; i += blockDim.x) {
            const int t = sm.a.skey[i];
            if (t < 0) continue;
            Acc3 &ac = A.acc[t];
            sm.a.sbase[i] = (int)atomicAdd(&ac.cnt, (unsigned)sm.a.scnt[i]);
            const unsigned long long k1 = sm.a.sk1[i];
            const unsigned long long old = atomicMax(&ac.key1, k1);
            const unsigned long long lo2 = old < k1 ? old : k1;
            const unsigned lo_o = (unsigned)(lo2 >> 32);
            const unsigned o2 = sm.a.so2[i];
            atomicMax(&ac.o2, lo_o > o2 ? lo_o : o2);
            atomicMax(&ac.emax, sm.a.sem[i]);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < ITEMS; k++) {
            const int v = v0 + k * blockDim.x + threadIdx.x;
            if (tgt[k] == -2) continue;
            const int r = (slot[k] >= 0) ? sm.a.sbase[slot[k]] + rk[k] : rk[k];
            A.code[v] = make_int2(tgt[k], r);
        }
    }
    unsigned fsum = __reduce_add_sync(0xffffffffu, fallbacks);
    if (lane == 0 && fsum) atomicAdd(&H->fallbacks, (unsigned long long)fsum);
}

// ---------------------------------------------------------------- T: table
// New segment table: the old segments whose facet survives (in order), then
// the cone facets created this iteration that received points.  Grid-wide
// exclusive scan in two steps (block sums, then offsets).
__device__ __forceinline__ int table_item_len(const Params3 &A, int par, int ne, int fc0, int j,
                                              int &f)
{
    if (j < ne) {
        const Ent3 en = A.ent[par][j];
        f = en.f;
        return A.fac[en.f].alive ? en.len : 0;
    }
    f = fc0 + (j - ne);
    return (int)A.acc[f].cnt;
}

__device__ void table_sum(const Params3 &A, int par, bool first, SmemAll3 &sm, int bid, int nb)
{
    Hdr3 *H = A.hdr;
    const int ne = first ? 0 : *(volatile int *)&H->nent[par];
    const int fc0 = first ? 0 : *(volatile int *)&H->fc_iter[par];
    const int fc1 = *(volatile int *)&H->fcount;
    const int m = ne + (fc1 - fc0);
    const int chunk = (m + nb - 1) / nb;
    const int j0 = bid * chunk, j1 = min(j0 + chunk, m);
    long long s = 0;
    for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        int f;
        int len = table_item_len(A, par, ne, fc0, j, f);
        s += ((long long)(len > 0) << 32) | (long long)len;
    }
    long long tot;
    block_excl_scan64(s, sm.t.wsum, &tot);
    if (threadIdx.x == 0) A.part[bid] = tot;
}

__device__ void table_write(const Params3 &A, int par, bool first, SmemAll3 &sm, int bid, int nb)
{
    Hdr3 *H = A.hdr;
    const int ne = first ? 0 : *(volatile int *)&H->nent[par];
    const int fc0 = first ? 0 : *(volatile int *)&H->fc_iter[par];
    const int fc1 = *(volatile int *)&H->fcount;
    const int m = ne + (fc1 - fc0);
    const int chunk = (m + nb - 1) / nb;
    const int j0 = bid * chunk, j1 = min(j0 + chunk, m);
    // prefix of the earlier blocks
    long long pre = 0;
    for (int b = threadIdx.x; b < bid; b += blockDim.x) pre += A.part[b];
    long long pre_tot;
    block_excl_scan64(pre, sm.t.wsum, &pre_tot);
    long long carry = pre_tot;
    Ent3 *out = A.ent[par ^ 1];
    for (int base = j0; base < j1; base += blockDim.x) {
        const int j = base + threadIdx.x;
        int f = -1, len = 0;
        if (j < j1) len = table_item_len(A, par, ne, fc0, j, f);
        long long s = ((long long)(len > 0) << 32) | (long long)len;
        long long tot;
        long long ex = block_excl_scan64(s, sm.t.wsum, &tot) + carry;
        if (len > 0) {
            const int k = (int)(ex >> 32), st = (int)(ex & 0xffffffffll);
            Ent3 en;
            en.f = f;
            en.start = st;
            en.len = len;
            en.pad = 0;
            out[k] = en;
            A.nstart[f] = st;
        }
        carry += tot;
    }
    if (bid == nb - 1 && threadIdx.x == 0) {
        H->nent[par ^ 1] = (int)(carry >> 32);
        H->L[par ^ 1] = (int)(carry & 0xffffffffll);
        H->fc_lo_last = fc0;
        H->fc_iter[par ^ 1] = fc1;  // read by the next table phase (other parity)
    }
}

// ---------------------------------------------------------------- B: scatter
template <bool FIRST>
__device__ void scatter3d(const Params3 &A, int par, int bid, int nb)
{
    Hdr3 *H = A.hdr;
    const int L = FIRST ? A.n : *(volatile int *)&H->L[par];
    const float4 *P = A.pts[par];
    float4 *Q = A.pts[par ^ 1];
    for (long long v = (long long)bid * blockDim.x + threadIdx.x; v < L;
         v += (long long)nb * blockDim.x) {
        const int2 cr = A.code[v];
        if (cr.x < 0) continue;
        const float4 p = FIRST ? load_input(A, v) : P[v];
        Q[A.nstart[cr.x] + cr.y] = p;
    }
}

// New facets: certify the FP32 farthest point (top-2 gap against twice the
// largest error bound) or queue it for the exact phase; record the apex.
// Also the tile -> entry map of the next assign phase.
__device__ void certify3d(const Params3 &A, int par, int bid, int nb)
{
    Hdr3 *H = A.hdr;
    const int ne = *(volatile int *)&H->nent[par ^ 1];
    const int L = *(volatile int *)&H->L[par ^ 1];
    const Ent3 *ent = A.ent[par ^ 1];
    for (int e = bid * blockDim.x + threadIdx.x; e < ne; e += nb * blockDim.x) {
        const int f = ent[e].f;
        const Acc3 a = A.acc[f];
        if (f >= *(volatile int *)&H->fc_lo_last) {
            // a facet created this iteration: its apex is new
            const int qi = key_idx(a.key1);
            const float4 q = load_input(A, qi);
            A.apex[f] = q;
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
    }
    const int T = A.tile;
    const int ntiles = (L + T - 1) / T;
    for (int t = bid * blockDim.x + threadIdx.x; t < ntiles; t += nb * blockDim.x) {
        const int v = t * T, vl = min(v + T, L) - 1;
        auto ent_of = [&](int x) {
            int lo = 0, hi = ne - 1;
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (ent[mid].start <= x) lo = mid;
                else hi = mid - 1;
            }
            return lo;
        };
        const int s0 = ent_of(v);
        A.tile_ent[t] = s0;
        A.tile_m[t] = ent_of(vl) - s0 + 1;
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
        if (go) init_clouds(A, sm, bid, nb);  // offsets checked before the launch
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
    }
    setup_mark(0);
    if (go) {
        // ---- first assignment: every input point against the tetrahedron;
        // table 1 / buffer 1 receive the result
        assign3d<MODE, ITEMS, true>(A, 0, sm, bid, nb);
        go = sync();
        setup_mark(1);
        if (go) {
            table_sum(A, 0, true, sm, bid, nb);
            go = sync();
        }
        if (go) {
            table_write(A, 0, true, sm, bid, nb);
            if (bid == 0 && threadIdx.x == 0) H->n_uncert = 0;
            go = sync();
        }
        setup_mark(2);
        if (go) {
            scatter3d<true>(A, 0, bid, nb);
            go = sync();
        }
        if (go) {
            certify3d(A, 0, bid, nb);
            go = sync();
        }
        if (go && *(volatile int *)&H->n_uncert > 0) {
            const int per = exact_chunks(A, *(volatile int *)&H->n_uncert, nb);
            exact3d<MODE>(A, 0, sm, bid, nb, per);
            go = sync();
            if (go && per > 1) {
                exact3d_merge<MODE>(A, 0, bid, nb, per);
                go = sync();
            }
        }
        setup_mark(3);
    }
    // ---- iterations: table `cur` describes the live points in buffer `cur`
    int cur = 1;
    int iter = 0;
    while (go && *(volatile int *)&H->nent[cur] > 0) {
        iter++;
        if (iter > A.max_iters) {
            if (bid == 0 && threadIdx.x == 0) set_status(H, QH_ERR_NO_CONVERGENCE);
            break;
        }
        if (bid == 0 && threadIdx.x == 0) {
            H->iter = iter;
            H->nwin = 0;
            H->seg_total += H->nent[cur];
            if (iter <= kTimeline3) {
                H->tl[iter - 1][0] = H->L[cur];
                H->tl[iter - 1][1] = H->nent[cur];
            }
        }
        mark(0, 0);
        select3d<MODE>(A, cur, bid, nb);
        if (!sync()) break;
        mark(iter, 3);
        if (bid == 0 && threadIdx.x == 0) H->nactive[0] = 0;
        if (!sync()) break;
        for (int round = 0; round < kRounds && go; round++) {
            claim3d(A, cur, iter, round, bid, nb);
            if (!(go = sync())) break;
            if (*(volatile int *)&H->nactive[round & 1] == 0) break;
            cone3d(A, cur, iter, round, bid, nb);
            go = sync();
        }
        if (!go) break;
        if (*(volatile int *)&H->nwin == 0) {
            if (bid == 0) fallback3d<MODE>(A, cur, iter);
            if (!sync()) break;
        }
        if (clk && iter <= kTimeline3) H->tl[iter - 1][2] = H->nwin;
        mark(iter, 4);
        assign3d<MODE, ITEMS, false>(A, cur, sm, bid, nb);
        if (!sync()) break;
        mark(iter, 5);
        table_sum(A, cur, false, sm, bid, nb);
        if (!sync()) break;
        table_write(A, cur, false, sm, bid, nb);
        if (bid == 0 && threadIdx.x == 0) H->n_uncert = 0;
        if (!sync()) break;
        mark(iter, 6);
        scatter3d<false>(A, cur, bid, nb);
        certify3d(A, cur, bid, nb);  // reads the table and accumulators only
        if (bid == 0 && threadIdx.x == 0) H->surv_total += H->L[cur ^ 1];
        if (!sync()) break;
        mark(iter, 7);
        if (*(volatile int *)&H->n_uncert > 0) {
            const int per = exact_chunks(A, *(volatile int *)&H->n_uncert, nb);
            exact3d<MODE>(A, cur, sm, bid, nb, per);
            if (!sync()) break;
            if (per > 1) {
                exact3d_merge<MODE>(A, cur, bid, nb, per);
                if (!sync()) break;
            }
            if (bid == 0 && threadIdx.x == 0) H->exact_argmax += H->n_uncert;
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
