// 2D segmented Quickhull on one GPU (Tzeng & Owens, Algorithm 4).
//
// Layout in device memory (one workspace, see layout2d):
//   * two point buffers (SoA x, y, idx) used ping-pong.  A segment owns a
//     fixed physical range [pstart, pstart + len) of the buffers; its
//     children are written into the same range of the other buffer, child 0
//     growing from the left end and child 1 from the right end, so no global
//     compaction of the array is ever needed and discarded points simply
//     leave a hole.  The "virtual" order of live points (segment by segment,
//     vstart = exclusive scan of live lengths) is what the pass tiles over.
//   * two segment tables (Seg2) and two child accumulators (Acc2: count,
//     top-2 farthest-point keys, max key error) by iteration parity.
//   * the hull as slots (0 = lexicographic min a, 1 = lexicographic max b,
//     then one slot per apex) with a successor link per slot; the links
//     always form the current hull polygon, clockwise from a.
//
// One iteration (the hot loop of Algorithm 4):
//   P  (pass2d_stream) every live point: classify against its segment's apex
//                 (outside edge e0-q -> child 0, outside q-e1 -> child 1,
//                 else discarded: inside the triangle, Algorithm 4 step 12),
//                 place it in its child's range and add it to the child's
//                 farthest-point reduction (the distance to the child edge
//                 is the classification value).  This fuses compact
//                 (Algorithm 3) and the 2-state flagPermute (Algorithm 2)
//                 with the next iteration's distance + segmented argmax
//                 (Algorithm 4 steps 9-14).  Warp-specialised: a producer
//                 warp streams tiles through a TMA ring and reserves each
//                 tile's output range with one atomic per child; consumer
//                 warps classify tile j and scatter tile j-1 (mbarrier
//                 hand-offs, no block barrier inside the pass).
//   U  (update2d) new segment table from the non-empty children, apex of
//                 each (certified exact when the FP32 top-2 gap exceeds the
//                 error bound), hull slots and links.
//   X  (exact2d)  only for uncertified segments: exact farthest point.
// The persistent kernel (qh2d_multi) runs all iterations of up to
// QH_MAX_CLOUDS_2D clouds with grid barriers over a shared segment table (a
// single-cloud call is one cloud): the streaming pass (pass2d_stream), a
// warp-per-segment pass once the segments are short (pass2d_warpseg), the
// update, and the exact argmax split over CTAs (exact2d_split).  The
// host-loop variant launches each phase (the synchronous pass pass2d) and
// reads the live counts back every iteration, as the paper's implementation
// does (Section 5 cost analysis).

#include <climits>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "pred2.cuh"
#include "qh_common.cuh"
#include "qh_internal.h"

namespace qh {

#ifndef QH2D_BLOCK
#define QH2D_BLOCK 256
#endif
#ifndef QH2D_ITEMS
#define QH2D_ITEMS 8
#endif
#ifndef QH2D_MINBLOCKS
#define QH2D_MINBLOCKS 2
#endif
#ifndef QH2D_SITEMS
#define QH2D_SITEMS 8
#endif
constexpr int kBlock = QH2D_BLOCK;
constexpr int kItems = QH2D_ITEMS;
constexpr int kTile = kBlock * kItems;   // points per tile
constexpr int kKeySeg = 64;              // segments per tile with shared-memory key slots
constexpr int kGeoCache = 64;            // segments per tile with geometry in shared memory
constexpr int kOutCap = 4096;            // hull slots ranked in one block's shared memory
constexpr int kMaxGrid = 4096;
constexpr int kMinBlocks = QH2D_MINBLOCKS;  // resident CTAs per SM the register budget targets
constexpr int kTimeline = 64;            // iterations recorded by the diagnostic timeline
// a pass whose segments average at most kWarpSegAvg points, none longer than
// kWarpSegMax, gives each segment to one warp (pass2d_warpseg)
constexpr int kWarpSegAvg = 64;
constexpr int kWarpSegMax = 2048;

struct Seg2 {
    float e0x, e0y, qx, qy, e1x, e1y;
    int q_idx, e0_slot, q_slot, e1_slot;
    int pstart, len, vstart;
    float thr;          // exact-argmax candidate threshold (uncertified segments)
    int pad[2];
};
static_assert(sizeof(Seg2) == 64, "Seg2 layout");

struct Acc2 {
    unsigned long long key1;  // best key of the child (distance order bits, ~index)
    unsigned int o2;          // distance order bits of the best other point
    unsigned int cnt;         // points in the child
    unsigned int emax;        // largest error bound of the child's keys (float bits)
    unsigned int pad[3];
};
static_assert(sizeof(Acc2) == 32, "Acc2 layout");

struct Hdr2 {
    GridBarrier bar;
    int status;
    int nonfinite;
    unsigned long long lexmin, lexmax;
    int a_idx, b_idx;
    int S[2];
    int L[2];
    int hull_count;
    int n_uncert;
    int iter;
    int maxlen;         // longest segment of the next pass (several-cloud kernel)
    long long seg_total, surv_total;
    unsigned long long fallbacks, exact_argmax;
    unsigned long long phase_ns[4];  // pass, update, exact, other (persistent kernel)
    // per-iteration record of the persistent kernel (first kTimeline iterations):
    // live points L, segments S, pass and update nanoseconds
    long long tl[kTimeline][4];
};

struct Params2 {
    const float *x, *y;
    long long stride;
    int n;
    int *out_idx;
    qh_result *res;
    Hdr2 *hdr;
    float2 *bxy[2];
    int *bi[2];
    Seg2 *seg[2];
    Acc2 *acc[2];
    int *tile_seg;
    int *tile_m;
    int *uncert;
    int *hull_idx;
    float *hull_x, *hull_y;
    int *next;
    long long max_iters;
    long long wait_ns;
    int test_hold;  // CTA 0 skips its first grid-barrier arrival (tests of the bounded wait)
    int cap_seg;
    int first_tma;  // first pass bulk copies: 0 none, 1 separate x, y arrays, 2 interleaved xy
    int cap_pts;    // entries of each point buffer (bounds of the debug build's checks)
    int cap_hull;   // hull slots
};

// ---------------------------------------------------------------- smem
// Geometry of a segment as the pass needs it.
struct Geo2 {
    float e0x, e0y, qx, qy, e1x, e1y;
    int q_idx, pstart, len, vstart;
};

// Farthest-point accumulator of one child: best key (distance order bits,
// then lowest index), order bits of the best distance among the other
// points, and the largest error bound of any key.
struct Top2 {
    unsigned long long k1;
    unsigned o2, em;
};

struct SmemPass {
    int vstart_l[kTile];
    unsigned short sb0[kTile], sb1[kTile];
    int gb0[kTile], gb1[kTile];
    unsigned long long sk1[kKeySeg][2];
    unsigned int so2[kKeySeg][2], sem[kKeySeg][2];
    Top2 carry[2];
    int wt0[kBlock / 32], wt1[kBlock / 32];
    int sfirst, m, carry_seg, par;
    Geo2 geo[kGeoCache];
};
struct SmemU {
    long long wsum[33];
    int vs[kTile];
    int small;
};
struct SmemX {
    int bidx[kBlock];
    float bx[kBlock], by[kBlock];
};
struct SmemOut {
    int succ[kOutCap];
    int dist[kOutCap];
    long long wsum[33];
};
union SmemAll {
    SmemPass pass;
    SmemU u;
    SmemX x;
    SmemOut out;
};

__device__ __forceinline__ int vload_i(const volatile int *p) { return *p; }

__device__ __forceinline__ void set_status(Hdr2 *H, int st) { atomicCAS(&H->status, 0, st); }

// ---------------------------------------------------------------- phase 0
__device__ void init2d(const Params2 &A)
{
    if (blockIdx.x != 0) return;
    Hdr2 *H = A.hdr;
    if (threadIdx.x == 0) {
        H->lexmin = ~0ull;
        H->lexmax = 0ull;
        H->a_idx = INT_MAX;
        H->b_idx = INT_MAX;
        H->S[0] = 1;
        H->L[0] = A.n;
        H->hull_count = 2;
    }
    if (threadIdx.x < 2) {
        Acc2 z = {};
        A.acc[0][threadIdx.x] = z;
    }
}

// ---------------------------------------------------------------- extrema
// Lexicographic min and max of (x, y) over all points (Algorithm 4 step 3,
// "min and max ... along the x axis", ties broken by y), each with the lowest
// index at which it occurs (the block's best pair is returned to thread 0;
// the persistent kernel settles the index once the global extremes are
// known).  Also flags non-finite input.
struct Ext2 {
    unsigned long long mn, mx;
    int mni, mxi;
};

__device__ Ext2 extrema2d(const Params2 &A, SmemAll &sm)
{
    unsigned long long mn = ~0ull, mx = 0ull;
    int mni = INT_MAX, mxi = INT_MAX;
    int bad = 0;
    // each thread visits its points in increasing index order, so a strict
    // comparison keeps the lowest index of its extreme key
    auto visit = [&](float xf, float yf, int i) {
        const float x = canon0(xf), y = canon0(yf);
        bad |= !(isfinite(x) && isfinite(y));
        const unsigned long long k = ((unsigned long long)ord_f32(x) << 32) | ord_f32(y);
        if (k < mn) {
            mn = k;
            mni = i;
        }
        if (k > mx) {
            mx = k;
            mxi = i;
        }
    };
    const long long s = A.stride;
    const long long nthr = (long long)gridDim.x * blockDim.x;
    const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    constexpr int U = 4;  // vector loads in flight per array and thread
    if (A.first_tma == 1 &&
        dbg_ok((((uintptr_t)A.x | (uintptr_t)A.y) & 15u) == 0u, kDbgVecAlign,
               (unsigned long long)(uintptr_t)A.x, (unsigned long long)(uintptr_t)A.y)) {
        // separate 16-byte aligned x and y arrays: four points per load
        const float4 *x4 = reinterpret_cast<const float4 *>(A.x);
        const float4 *y4 = reinterpret_cast<const float4 *>(A.y);
        const long long n4 = A.n / 4;
        for (long long q0 = gtid; q0 < n4; q0 += U * nthr) {
            float4 xs[U], ys[U];
#pragma unroll
            for (int u = 0; u < U; u++) {
                const long long q = q0 + u * nthr;
                xs[u] = q < n4 ? __ldg(x4 + q) : make_float4(0.f, 0.f, 0.f, 0.f);
                ys[u] = q < n4 ? __ldg(y4 + q) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < U; u++) {
                const long long q = q0 + u * nthr;
                if (q >= n4) continue;
                const int i = (int)(4 * q);
                visit(xs[u].x, ys[u].x, i);
                visit(xs[u].y, ys[u].y, i + 1);
                visit(xs[u].z, ys[u].z, i + 2);
                visit(xs[u].w, ys[u].w, i + 3);
            }
        }
        for (long long i = 4 * n4 + gtid; i < A.n; i += nthr) visit(__ldg(A.x + i), __ldg(A.y + i), (int)i);
    } else {
        constexpr int V = 8;
        for (long long i0 = gtid; i0 < A.n; i0 += V * nthr) {
            float xs[V], ys[V];
#pragma unroll
            for (int u = 0; u < V; u++) {
                const long long i = i0 + u * nthr;
                xs[u] = i < A.n ? __ldg(A.x + i * s) : 0.0f;
                ys[u] = i < A.n ? __ldg(A.y + i * s) : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < V; u++)
                if (i0 + u * nthr < A.n) visit(xs[u], ys[u], (int)(i0 + u * nthr));
        }
    }
    // (key, index) pairs: smaller key, then smaller index (max: larger key)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long a = __shfl_xor_sync(0xffffffffu, mn, o);
        const unsigned long long b = __shfl_xor_sync(0xffffffffu, mx, o);
        const int ai = __shfl_xor_sync(0xffffffffu, mni, o);
        const int bi = __shfl_xor_sync(0xffffffffu, mxi, o);
        if (a < mn || (a == mn && ai < mni)) {
            mn = a;
            mni = ai;
        }
        if (b > mx || (b == mx && bi < mxi)) {
            mx = b;
            mxi = bi;
        }
    }
    bad = __syncthreads_or(bad);
    unsigned long long *red = (unsigned long long *)sm.u.wsum;
    int *redi = sm.u.vs;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        red[w] = mn;
        red[16 + w] = mx;
        redi[w] = mni;
        redi[16 + w] = mxi;
    }
    __syncthreads();
    Ext2 r = {mn, mx, mni, mxi};
    if (threadIdx.x == 0) {
        for (int i = 1; i < (int)(blockDim.x >> 5); i++) {
            if (red[i] < r.mn || (red[i] == r.mn && redi[i] < r.mni)) {
                r.mn = red[i];
                r.mni = redi[i];
            }
            if (red[16 + i] > r.mx || (red[16 + i] == r.mx && redi[16 + i] < r.mxi)) {
                r.mx = red[16 + i];
                r.mxi = redi[16 + i];
            }
        }
        if (A.n > 0) {
            atomicMin(&A.hdr->lexmin, r.mn);
            atomicMax(&A.hdr->lexmax, r.mx);
        }
        if (bad) atomicExch(&A.hdr->nonfinite, 1);
    }
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------- the pass
__device__ __forceinline__ Geo2 geo_of(const Seg2 &g)
{
    Geo2 r;
    r.e0x = g.e0x; r.e0y = g.e0y; r.qx = g.qx; r.qy = g.qy; r.e1x = g.e1x; r.e1y = g.e1y;
    r.q_idx = g.q_idx; r.pstart = g.pstart; r.len = g.len; r.vstart = g.vstart;
    return r;
}

__device__ __forceinline__ void top2_add(Top2 &t, unsigned long long k, unsigned em)
{
    unsigned long long lo = k < t.k1 ? k : t.k1;
    t.k1 = k > t.k1 ? k : t.k1;
    unsigned lo_o = (unsigned)(lo >> 32);
    t.o2 = lo_o > t.o2 ? lo_o : t.o2;
    t.em = em > t.em ? em : t.em;
}

__device__ __forceinline__ void top2_join(Top2 &t, const Top2 &u)
{
    top2_add(t, u.k1, u.em);
    t.o2 = u.o2 > t.o2 ? u.o2 : t.o2;
}

// Insert an accumulator into memory (shared or global) with atomics: the key
// displaced from, or refused by, k1 offers its distance to o2.
__device__ __forceinline__ void top2_store(unsigned long long *k1, unsigned *o2, unsigned *em,
                                           const Top2 &t)
{
    if (!t.k1) return;
    unsigned long long old = atomicMax(k1, t.k1);
    unsigned long long lo = old < t.k1 ? old : t.k1;
    unsigned o = (unsigned)(lo >> 32);
    atomicMax(o2, o > t.o2 ? o : t.o2);
    atomicMax(em, t.em);
}

__device__ __forceinline__ void top2_warp(Top2 &t)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        Top2 u;
        u.k1 = __shfl_xor_sync(0xffffffffu, t.k1, o);
        u.o2 = __shfl_xor_sync(0xffffffffu, t.o2, o);
        u.em = __shfl_xor_sync(0xffffffffu, t.em, o);
        top2_join(t, u);
    }
}

__device__ __forceinline__ void acc_merge(Acc2 &ac, const Top2 &t)
{
    top2_store(&ac.key1, &ac.o2, &ac.emax, t);
}

// One tile of the pass.  SINGLE: the tile lies inside one segment (geometry
// in registers, no per-item segment search).
template <class P, bool FIRST, bool SINGLE>
__device__ __forceinline__ void pass_tile(const Params2 &A, SmemPass &sm, const Seg2 *seg,
                                          Acc2 *acc, int sf, int m, int v0, int v1,
                                          unsigned &fallbacks)
{
    Hdr2 *H = A.hdr;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    const float2 *ixy = A.bxy[FIRST ? 0 : (sm.par ^ 1)];
    const int *ii = A.bi[FIRST ? 0 : (sm.par ^ 1)];
    float2 *oxy = A.bxy[sm.par];
    int *oi = A.bi[sm.par];
    Geo2 g0;
    if (SINGLE) g0 = sm.geo[0];
    auto geo = [&](int ls) -> Geo2 {
        if (SINGLE) return g0;
        if (ls < kGeoCache) return sm.geo[ls];
        return geo_of(seg[sf + ls]);
    };

    // ---- load, classify, accumulate farthest-point keys
    float2 pxy[kItems];
    int pidx[kItems], pk[kItems];
    const int wbase = v0 + warp * 32 * kItems;
#pragma unroll
    for (int k = 0; k < kItems; k++) {
        int v = wbase + k * 32 + lane;
        pk[k] = 3;
        if (v < v1) {
            int ls = 0;
            if (!SINGLE) {
                int lo = 0, hi = m - 1;
                while (lo < hi) {
                    int mid = (lo + hi + 1) >> 1;
                    if (sm.vstart_l[mid] <= v) lo = mid;
                    else hi = mid - 1;
                }
                ls = lo;
            }
            pk[k] = (ls << 2) | 2;
            if (FIRST) {
                if (A.stride == 1) {
                    pxy[k].x = __ldg(A.x + v);
                    pxy[k].y = __ldg(A.y + v);
                } else {
                    pxy[k].x = __ldg(A.x + (long long)v * A.stride);
                    pxy[k].y = __ldg(A.y + (long long)v * A.stride);
                }
                pidx[k] = v;
            } else {
                int ps, vs;
                if (SINGLE) {
                    ps = g0.pstart;
                    vs = g0.vstart;
                } else if (ls < kGeoCache) {
                    ps = sm.geo[ls].pstart;
                    vs = sm.geo[ls].vstart;
                } else {
                    ps = seg[sf + ls].pstart;
                    vs = seg[sf + ls].vstart;
                }
                int pos = ps + (v - vs);
                pxy[k] = ixy[pos];
                pidx[k] = ii[pos];
            }
        }
    }
    int cur = -1;
    Top2 ta = {0ull, 0u, 0u}, tb = {0ull, 0u, 0u};
    auto flush = [&](int ls) {
        if (ls < 0) return;
        if (ls < kKeySeg) {
            top2_store(&sm.sk1[ls][0], &sm.so2[ls][0], &sm.sem[ls][0], ta);
            top2_store(&sm.sk1[ls][1], &sm.so2[ls][1], &sm.sem[ls][1], tb);
        } else {
            acc_merge(acc[2 * (sf + ls)], ta);
            acc_merge(acc[2 * (sf + ls) + 1], tb);
        }
    };
    int w0 = 0, w1 = 0;
#pragma unroll
    for (int k = 0; k < kItems; k++) {
        int c = 3;
        if (pk[k] != 3) {
            int ls = pk[k] >> 2;
            const Geo2 g = geo(ls);
            float x = pxy[k].x, y = pxy[k].y;
            c = 2;
            if (FIRST) {
                if (x == g.e0x && y == g.e0y) atomicMin(&H->a_idx, pidx[k]);
                if (x == g.qx && y == g.qy) atomicMin(&H->b_idx, pidx[k]);
            }
            if (pidx[k] != g.q_idx) {  // the apex itself joins the hull
                float d, e;
                orient_value<P>(g.e0x, g.e0y, g.qx, g.qy, x, y, d, e);
                if (orient_sign<P>(d, e, g.e0x, g.e0y, g.qx, g.qy, x, y, fallbacks) > 0) {
                    c = 0;
                } else {
                    orient_value<P>(g.qx, g.qy, g.e1x, g.e1y, x, y, d, e);
                    if (orient_sign<P>(d, e, g.qx, g.qy, g.e1x, g.e1y, x, y, fallbacks) > 0) c = 1;
                }
                if (c < 2) {
                    if (!SINGLE && ls != cur) {
                        flush(cur);
                        ta = {0ull, 0u, 0u};
                        tb = {0ull, 0u, 0u};
                    }
                    cur = ls;
                    // the distance to the child edge is the classification value
                    unsigned long long key = dist_key(d, pidx[k]);
                    if (c == 0) top2_add(ta, key, __float_as_uint(e));
                    else top2_add(tb, key, __float_as_uint(e));
                }
            }
            pk[k] = (ls << 2) | c;
        }
        w0 += __popc(__ballot_sync(0xffffffffu, c == 0));
        w1 += __popc(__ballot_sync(0xffffffffu, c == 1));
    }
    if (lane == 0) {
        sm.wt0[warp] = w0;
        sm.wt1[warp] = w1;
    }
    // warp-aggregated key flush when the warp ends in one segment
    {
        int lmax = SINGLE ? 0 : (int)__reduce_max_sync(0xffffffffu, (unsigned)(cur + 1)) - 1;
        bool same = SINGLE || __all_sync(0xffffffffu, cur == lmax || cur == -1);
        if (same && lmax >= 0) {
            top2_warp(ta);
            top2_warp(tb);
            if (lane == 0) flush(lmax);
        } else {
            flush(cur);
        }
    }
    __syncthreads();
    int base0 = 0, base1 = 0, tot0 = 0, tot1 = 0;
#pragma unroll
    for (int w = 0; w < kBlock / 32; w++) {
        int a = sm.wt0[w], b = sm.wt1[w];
        base0 += (w < warp) ? a : 0;
        base1 += (w < warp) ? b : 0;
        tot0 += a;
        tot1 += b;
    }
    if (!SINGLE) {
        // tile-local prefix at each segment start
        int r0 = base0, r1 = base1;
#pragma unroll
        for (int k = 0; k < kItems; k++) {
            int c = pk[k] & 3;
            unsigned b0 = __ballot_sync(0xffffffffu, c == 0);
            unsigned b1 = __ballot_sync(0xffffffffu, c == 1);
            int ls = pk[k] >> 2;
            int v = wbase + k * 32 + lane;
            if (c != 3 && ls > 0 && sm.vstart_l[ls] == v) {
                sm.sb0[ls] = (unsigned short)(r0 + __popc(b0 & lt));
                sm.sb1[ls] = (unsigned short)(r1 + __popc(b1 & lt));
            }
            r0 += __popc(b0);
            r1 += __popc(b1);
        }
        if (threadIdx.x == 0) {
            sm.sb0[0] = 0;
            sm.sb1[0] = 0;
        }
        __syncthreads();
    }
    // ---- global bases: one atomic per (tile, segment, child)
    for (int i = threadIdx.x; i < 2 * m; i += blockDim.x) {
        int ls = i >> 1, c = i & 1;
        int cnt;
        if (SINGLE) cnt = c ? tot1 : tot0;
        else if (c == 0) cnt = ((ls + 1 < m) ? sm.sb0[ls + 1] : tot0) - sm.sb0[ls];
        else cnt = ((ls + 1 < m) ? sm.sb1[ls + 1] : tot1) - sm.sb1[ls];
        int g = cnt ? (int)atomicAdd(&acc[2 * (sf + ls) + c].cnt, (unsigned)cnt) : 0;
        if (c == 0) sm.gb0[ls] = g;
        else sm.gb1[ls] = g;
    }
    __syncthreads();
    // ---- scatter survivors
    {
        int r0 = base0, r1 = base1;
#pragma unroll
        for (int k = 0; k < kItems; k++) {
            int c = pk[k] & 3;
            unsigned b0 = __ballot_sync(0xffffffffu, c == 0);
            unsigned b1 = __ballot_sync(0xffffffffu, c == 1);
            int pre0 = r0 + __popc(b0 & lt), pre1 = r1 + __popc(b1 & lt);
            r0 += __popc(b0);
            r1 += __popc(b1);
            if (c > 1) continue;
            int ls = pk[k] >> 2;
            int dst;
            if (SINGLE) {
                if (c == 0) dst = g0.pstart + sm.gb0[0] + pre0;
                else dst = g0.pstart + g0.len - 1 - (sm.gb1[0] + pre1);
            } else {
                int ps, ln;
                if (ls < kGeoCache) {
                    ps = sm.geo[ls].pstart;
                    ln = sm.geo[ls].len;
                } else {
                    ps = seg[sf + ls].pstart;
                    ln = seg[sf + ls].len;
                }
                if (c == 0) dst = ps + sm.gb0[ls] + (pre0 - sm.sb0[ls]);
                else dst = ps + ln - 1 - (sm.gb1[ls] + (pre1 - sm.sb1[ls]));
            }
            if (dbg_ok(dst >= 0 && dst < A.cap_pts, kDbgPointDst, dst, A.cap_pts)) {
                oxy[dst] = pxy[k];
                oi[dst] = pidx[k];
            }
        }
    }
}

template <class P, bool FIRST>
__device__ void pass2d(const Params2 &A, int par, SmemPass &sm, int bid, int nb)
{
    Hdr2 *H = A.hdr;
    const int L = FIRST ? A.n : vload_i(&H->L[par]);
    const int S = FIRST ? 1 : vload_i(&H->S[par]);
    const Seg2 *seg = A.seg[par];
    Acc2 *acc = A.acc[par];
    unsigned fallbacks = 0;
    const int ntiles = (L + kTile - 1) / kTile;
    // a contiguous run of tiles per block keeps consecutive tiles in the same
    // segment, so farthest-point keys are carried across tiles in shared memory
    const int per = ntiles / nb, rem = ntiles % nb;
    const int t_begin = bid * per + min(bid, rem);
    const int t_end = t_begin + per + (bid < rem ? 1 : 0);
    if (threadIdx.x == 0) {
        sm.carry_seg = -1;
        sm.par = par;
    }
    for (int tile = t_begin; tile < t_end; tile++) {
        const int v0 = tile * kTile;
        const int v1 = min(v0 + kTile, L);
        __syncthreads();  // shared memory of the previous tile is free
        if (threadIdx.x == 0) {
            int sf = FIRST ? 0 : A.tile_seg[tile];
            int mm = FIRST ? 1 : A.tile_m[tile];
            int cs = sm.carry_seg;
            if (cs >= 0 && cs != sf) {
                // the carried segment ended in the previous tile
                acc_merge(acc[2 * cs], sm.carry[0]);
                acc_merge(acc[2 * cs + 1], sm.carry[1]);
                sm.carry_seg = -1;
            }
            sm.sfirst = sf;
            sm.m = mm;
        }
        __syncthreads();
        const int sf = sm.sfirst, m = sm.m;
        const bool carry = sm.carry_seg == sf;
        for (int i = threadIdx.x; i < 2 * min(m, kKeySeg); i += blockDim.x) {
            int ls = i >> 1, c = i & 1;
            bool cin = carry && ls == 0;
            sm.sk1[ls][c] = cin ? sm.carry[c].k1 : 0ull;
            sm.so2[ls][c] = cin ? sm.carry[c].o2 : 0u;
            sm.sem[ls][c] = cin ? sm.carry[c].em : 0u;
        }
        if (m > 1)
            for (int i = threadIdx.x; i < m; i += blockDim.x) sm.vstart_l[i] = seg[sf + i].vstart;
        if (threadIdx.x < min(m, kGeoCache)) {
            Geo2 g;
            if (FIRST) {
                unsigned long long kmn = *(volatile unsigned long long *)&H->lexmin;
                unsigned long long kmx = *(volatile unsigned long long *)&H->lexmax;
                g.e0x = g.e1x = unord_f32((uint32_t)(kmn >> 32));
                g.e0y = g.e1y = unord_f32((uint32_t)kmn);
                g.qx = unord_f32((uint32_t)(kmx >> 32));
                g.qy = unord_f32((uint32_t)kmx);
                g.q_idx = -1;
                g.pstart = 0;
                g.len = A.n;
                g.vstart = 0;
            } else {
                g = geo_of(seg[sf + threadIdx.x]);
            }
            sm.geo[threadIdx.x] = g;
        }
        __syncthreads();
        if (m == 1) pass_tile<P, FIRST, true>(A, sm, seg, acc, sf, m, v0, v1, fallbacks);
        else pass_tile<P, FIRST, false>(A, sm, seg, acc, sf, m, v0, v1, fallbacks);
        __syncthreads();
        // ---- merge the key slots of segments that end in this tile; the last
        // segment is carried to the next tile of this block
        const int mk = min(m, kKeySeg);
        for (int i = threadIdx.x; i < 2 * mk; i += blockDim.x) {
            int ls = i >> 1, c = i & 1;
            Top2 t = {sm.sk1[ls][c], sm.so2[ls][c], sm.sem[ls][c]};
            if (ls == m - 1) sm.carry[c] = t;
            else acc_merge(acc[2 * (sf + ls) + c], t);
        }
        if (threadIdx.x == 0) sm.carry_seg = (m - 1 < kKeySeg) ? sf + m - 1 : -1;
    }
    __syncthreads();
    if (threadIdx.x == 0 && sm.carry_seg >= 0) {
        int cs = sm.carry_seg;
        acc_merge(acc[2 * cs], sm.carry[0]);
        acc_merge(acc[2 * cs + 1], sm.carry[1]);
    }
    // predicate fallback statistics
    unsigned f = __reduce_add_sync(0xffffffffu, fallbacks);
    if ((threadIdx.x & 31) == 0 && f) atomicAdd(&H->fallbacks, (unsigned long long)f);
}

// ---------------------------------------------------------------- streaming pass
// The persistent kernel's passes run as a warp-specialised pipeline over each
// CTA's run of tiles.  The CTA's last warp produces: it fills a ring of
// kRing shared-memory stages with the bulk-copy engine (TMA, non-tensor
// form), reserves each tile's output range in the segment's children with
// one global atomic per child, and merges the farthest-point slots of tiles
// that straddle segments.  The other kCW warps consume: they classify tile j
// and then scatter tile j-1, whose reserved bases the producer has published
// meanwhile, so the atomic's round trip overlaps a tile of work.  Producer and
// consumers hand off through mbarriers only (per stage: full, empty; per tile
// parity: counted, bases); there is no block-wide barrier inside the pass.
//
// A consumer keeps the farthest-point accumulators of its current segment in
// registers for as long as its run stays in that segment.  A tile that
// straddles segments is finished inside its classification step, warp by
// warp: each row of 32 points groups its survivors by (segment, child) with a
// match and reserves each group's range with one atomic.
constexpr int kCW = kBlock / 32 - 1;        // consumer warps
constexpr int kSItems = QH2D_SITEMS;        // points per consumer thread and tile
constexpr int kSTile = kCW * 32 * kSItems;  // points per streaming tile
constexpr int kRing = 4;                    // stages
constexpr int kStage = kSTile + 8;          // points per stage (16-byte alignment slack)
constexpr int kRun = 256;                   // tile-map entries of a CTA's run in shared memory
constexpr int kMSlot = 32;                  // segments of a multi-segment tile with key slots
static_assert(kSTile % 4 == 0, "tile starts must allow 16-byte bulk copies");

struct SmemStream {
    float2 sxy[kRing][kStage];
    int sidx[kRing][kStage];
    Seg2 sseg[kRing];                      // segment record of a single-segment tile
    unsigned long long sk1[2][kMSlot][2];  // key slots of a multi-segment tile, by tile parity
    unsigned so2[2][kMSlot][2], sem[2][kMSlot][2];
    int run_sf[kRun], run_m[kRun], run_ps[kRun], run_vs[kRun];
    int tilecnt[2][2];                     // survivors per child of a tile (consumers add)
    int gb[2][2];                          // the tile's reserved global base per child
    int shift[kRing];
};
static_assert(offsetof(SmemStream, sidx) % 16 == 0 && offsetof(SmemStream, sseg) % 16 == 0 &&
                  (sizeof(float2) * kStage) % 16 == 0 && (sizeof(int) * kStage) % 16 == 0,
              "stages and segment records must be 16-byte aligned");
// the run map's segment starts are staged in the (then idle) stage ring
constexpr int kStageInts = (int)(sizeof(float2) * kRing * kStage / sizeof(int));

// The pipeline's mbarriers (static shared memory of the persistent kernel,
// initialised once per launch) and each thread's phase parities.
struct PipeBars {
    unsigned long long full[kRing];   // producer: expect_tx arrive (or plain arrive)
    unsigned long long empty[kRing];  // one arrive per consumer warp after its scatter
    unsigned long long counted[2];    // one arrive per consumer warp after classifying
    unsigned long long bases[2];      // producer: bases published
};
// parity bits of the next phase to wait for, per thread
constexpr int kPhFull = 0, kPhBases = 4, kPhCounted = 8, kPhEmpty = 12;

__device__ __forceinline__ void mbar_arrive(unsigned long long *bar)
{
    if (!mbar_aligned(bar)) return;
    asm volatile("mbarrier.arrive.shared.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void fence_proxy_async_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Classification of one point against a segment (edge e0 -> e1, apex q):
// 0 = strictly outside e0 -> q, 1 = strictly outside q -> e1, 2 = neither
// (inside or on the triangle, or the apex itself).  d and e are the filter
// value and bound of the deciding orientation (the distance key of the child).
template <class P>
__device__ __forceinline__ int classify2d(const Geo2 &g, float x, float y, int idx, float &d,
                                          float &e, unsigned &fallbacks)
{
    if (idx == g.q_idx) return 2;
    orient_value<P>(g.e0x, g.e0y, g.qx, g.qy, x, y, d, e);
    if (orient_sign<P>(d, e, g.e0x, g.e0y, g.qx, g.qy, x, y, fallbacks) > 0) return 0;
    orient_value<P>(g.qx, g.qy, g.e1x, g.e1y, x, y, d, e);
    if (orient_sign<P>(d, e, g.qx, g.qy, g.e1x, g.e1y, x, y, fallbacks) > 0) return 1;
    return 2;
}

// One multi-segment tile, by one consumer warp (later passes only): its
// kSItems rows, classified, reserved per (segment, child) group and
// scattered.  Keys of the tile's first kMSlot segments go to the slots of
// parity p (merged by the producer), the others to the accumulators.
// The virtual starts of the tile's m segments are in tvs (shared memory).
template <class P>
__device__ __forceinline__ void multi_tile(SmemStream &sm, const Seg2 *seg, Acc2 *acc, int sf,
                                           int m, int v0, int v1, int p, const float2 *ixy,
                                           const int *ii, float2 *oxy, int *oi,
                                           unsigned &fallbacks, const int *tvs, int cap_pts)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    int mcur = -1;
    Top2 ma = {0ull, 0u, 0u}, mb = {0ull, 0u, 0u};
    auto mflush = [&]() {
        if (mcur < 0) return;
        if (mcur < kMSlot) {
            top2_store(&sm.sk1[p][mcur][0], &sm.so2[p][mcur][0], &sm.sem[p][mcur][0], ma);
            top2_store(&sm.sk1[p][mcur][1], &sm.so2[p][mcur][1], &sm.sem[p][mcur][1], mb);
        } else {
            acc_merge(acc[2 * (sf + mcur)], ma);
            acc_merge(acc[2 * (sf + mcur) + 1], mb);
        }
    };
    // rows in batches of kMB: classify and reserve every row of the batch,
    // then scatter (the reservations' round trips overlap)
    constexpr int kMB = 4;
    static_assert(kSItems % kMB == 0, "row batches");
    const int wbase = v0 + warp * 32 * kSItems;
#pragma unroll 1
    for (int k0 = 0; k0 < kSItems; k0 += kMB) {
        float2 pxy[kMB];
        int pidx[kMB], pk[kMB], pbase[kMB];
        unsigned pgrp[kMB];
#pragma unroll
        for (int k = 0; k < kMB; k++) {
            const int v = wbase + (k0 + k) * 32 + lane;
            int c = 3, ls = 0;
            if (v < v1) {
                // (the segment table is written inside this launch: plain loads)
                int lo = 0, hi = m - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (tvs[mid] <= v) lo = mid;
                    else hi = mid - 1;
                }
                ls = lo;
                const Seg2 &G = seg[sf + ls];
                Geo2 g;
                g.e0x = G.e0x; g.e0y = G.e0y;
                g.qx = G.qx;   g.qy = G.qy;
                g.e1x = G.e1x; g.e1y = G.e1y;
                g.q_idx = G.q_idx;
                const int pos = G.pstart + (v - G.vstart);
                pxy[k] = ixy[pos];
                pidx[k] = ii[pos];
                float d = 0.f, e = 0.f;
                c = classify2d<P>(g, pxy[k].x, pxy[k].y, pidx[k], d, e, fallbacks);
                if (c < 2) {
                    if (ls != mcur) {
                        mflush();
                        mcur = ls;
                        ma = {0ull, 0u, 0u};
                        mb = {0ull, 0u, 0u};
                    }
                    const unsigned long long key = dist_key(d, pidx[k]);
                    if (c == 0) top2_add(ma, key, __float_as_uint(e));
                    else top2_add(mb, key, __float_as_uint(e));
                }
            }
            pk[k] = (ls << 2) | c;
            // survivors of this row grouped by (segment, child); one atomic per group
            const unsigned gkey = c < 2 ? (unsigned)(ls * 2 + c) : 0x80000000u + (unsigned)lane;
            const unsigned grp = __match_any_sync(0xffffffffu, gkey);
            pgrp[k] = grp;
            pbase[k] = 0;
            if (c < 2 && lane == __ffs(grp) - 1)
                pbase[k] = (int)atomicAdd(&acc[2 * (sf + ls) + c].cnt, (unsigned)__popc(grp));
        }
#pragma unroll
        for (int k = 0; k < kMB; k++) {
            const unsigned grp = pgrp[k];
            const int base = __shfl_sync(0xffffffffu, pbase[k], __ffs(grp) - 1);
            const int c = pk[k] & 3;
            if (c < 2) {
                const Seg2 &G = seg[sf + (pk[k] >> 2)];
                const int rank = base + __popc(grp & lt);
                const int dst = c == 0 ? G.pstart + rank : G.pstart + G.len - 1 - rank;
                if (dbg_ok(dst >= 0 && dst < cap_pts, kDbgPointDst, dst, cap_pts)) {
                    oxy[dst] = pxy[k];
                    oi[dst] = pidx[k];
                }
            }
        }
    }
    mflush();
}

// A thread's farthest-point record of one child in the streaming pass: the order
// bits (ord_f32) of its best and second-best distance (0 = none: no distance
// that arithmetic produces maps to 0), the best point's index (the first one
// met among equal distances; a tie leaves o2 == o1, so the segment is never
// certified and its apex is found by the exact argmax) and the largest error
// bound.  Unsigned min/max order NaN distances like the 64-bit keys do.
struct Far2 {
    unsigned o1, o2, em;
    int i1;
};
__device__ __forceinline__ void far2_add(Far2 &a, unsigned o, int idx, unsigned eb)
{
    const bool gt = o > a.o1;
    a.o2 = max(a.o2, min(a.o1, o));
    a.o1 = max(a.o1, o);
    a.i1 = gt ? idx : a.i1;
    a.em = max(a.em, eb);
}
__device__ __forceinline__ Top2 far2_top2(const Far2 &a)
{
    Top2 t;
    t.k1 = a.o1 ? (((unsigned long long)a.o1 << 32) | (unsigned long long)(0xffffffffu - (uint32_t)a.i1))
                : 0ull;
    t.o2 = a.o2;
    t.em = a.em;
    return t;
}

// WEIGHTED: the CTAs' runs split the pass by cost rather than by tiles, a
// segment start counting as two more tiles (a tile that straddles segments
// is finished warp by warp with a chain of global round trips), so that runs
// over many small segments do not fall on a few CTAs.
// Single-segment tiles keep per-thread Far2 records and counts, the scatter
// loads a warp's items before storing them, the producer publishes a tile's
// bases as soon as they are reserved and stages the segment starts of a tile
// that straddles segments, and the cost-weighted run ends are found by all
// threads at once.
template <class P, bool FIRST, bool WEIGHTED = false>
__device__ void pass2d_stream(const Params2 &A, int par, SmemStream &sm, PipeBars &bars,
                              unsigned &ph, int bid, int nb)
{
    Hdr2 *H = A.hdr;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    const int L = FIRST ? A.n : vload_i(&H->L[par]);
    const int S = FIRST ? 1 : vload_i(&H->S[par]);
    const Seg2 *seg = A.seg[par];
    Acc2 *acc = A.acc[par];
    const float2 *ixy = A.bxy[par ^ 1];
    const int *ii = A.bi[par ^ 1];
    float2 *oxy = A.bxy[par];
    int *oi = A.bi[par];
    unsigned fallbacks = 0;
    // a pass never starts after a failure: no copy is issued that nobody
    // waits for (the same decision in every thread of the CTA)
    if (status_uniform(&H->status) != 0) return;
    const int ntiles = (L + kSTile - 1) / kSTile;
    const int per = ntiles / nb, rem = ntiles % nb;
    int t_begin = bid * per + min(bid, rem);
    int nt = per + (bid < rem ? 1 : 0);

    // ---- run map: tile -> (first segment, number of segments, the first
    // segment's physical and virtual start), by binary search of the tile's
    // first and last virtual positions in the segment starts (staged in the
    // idle stage ring when they fit)
    int *svs = reinterpret_cast<int *>(&sm.sxy[0][0]);
    const bool vs_smem = S <= kStageInts;
    auto seg_of = [&](int v, bool staged) {
        int lo = 0, hi = S - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            const int vs = staged ? svs[mid] : seg[mid].vstart;
            if (vs <= v) lo = mid;
            else hi = mid - 1;
        }
        return lo;
    };
    auto tile_segs = [&](int j, int &sf, int &m, bool staged) {
        const int v = (t_begin + j) * kSTile, vl = min(v + kSTile, L) - 1;
        sf = seg_of(v, staged);
        m = seg_of(vl, staged) - sf + 1;
        if (!dbg_ok(sf >= 0 && m >= 1 && sf + m <= S, kDbgSegIndex, sf + m, S)) {
            sf = 0;
            m = 1;
        }
    };
    if (WEIGHTED && !FIRST && ntiles > 0) {
        if (vs_smem)
            for (int i = threadIdx.x; i < S; i += blockDim.x) svs[i] = seg[i].vstart;
        __syncthreads();
        // cost of tiles [0, t): t plus twice the segment starts before
        // tile t (strictly increasing in t); run b covers the tiles
        // whose cost prefix falls in [b W / nb, (b+1) W / nb)
        auto cost = [&](int t) -> long long {
            return t == 0 ? 0ll : (long long)t + 2ll * (seg_of(t * kSTile - 1, vs_smem) + 1);
        };
        const long long W = cost(ntiles);
        // the first tile with cost >= target, for the run's two ends at
        // once (threads 0-127: its start, 128-255: its end): each round
        // probes 128 evenly spaced tiles of the interval [lo, hi] that
        // holds the answer and keeps the gap between the last probe
        // below the target and the first one at or above it
        static_assert(kBlock == 256, "two halves of 128 probes");
        const int half = threadIdx.x >> 7, hl = threadIdx.x & 127;
        const long long target = W * (bid + half) / nb;
        int *nbelow = sm.run_sf;  // per-warp counts (the run map is built later)
        int lo = 0, hi = ntiles;
        auto probe = [&](int i) { return lo + (int)(((long long)(i + 1) * (hi - lo)) >> 7); };
        for (int span = ntiles; span > 0; span >>= 7) {
            const bool below = cost(probe(hl)) < target;
            const unsigned b = __ballot_sync(0xffffffffu, below);
            if (lane == 0) nbelow[warp] = __popc(b);
            __syncthreads();
            const int q = half * 4;
            const int nf = nbelow[q] + nbelow[q + 1] + nbelow[q + 2] + nbelow[q + 3];
            __syncthreads();
            // probes 0..nf-1 are below the target, probe nf (<= 127) is not
            const int nlo = nf == 0 ? lo : probe(nf - 1) + 1, nhi = probe(nf);
            lo = nlo;
            hi = nhi;
        }
        if (hl == 0) sm.shift[half] = lo;  // (the stage shifts are not in use yet)
        __syncthreads();
        t_begin = sm.shift[0];
        nt = sm.shift[1] - sm.shift[0];
    }
    if (!FIRST && nt > 0) {
        if (vs_smem && !WEIGHTED)
            for (int i = threadIdx.x; i < S; i += blockDim.x) svs[i] = seg[i].vstart;
        __syncthreads();
        for (int j = threadIdx.x; j < min(nt, kRun); j += blockDim.x) {
            int sf, m;
            tile_segs(j, sf, m, vs_smem);
            sm.run_sf[j] = sf;
            sm.run_m[j] = m;
            sm.run_ps[j] = seg[sf].pstart;
            sm.run_vs[j] = vs_smem ? svs[sf] : seg[sf].vstart;
        }
    }
    for (int i = threadIdx.x; i < 2 * 2 * kMSlot; i += blockDim.x) {
        const int q = i / (2 * kMSlot), s = (i >> 1) % kMSlot, c = i & 1;
        sm.sk1[q][s][c] = 0ull;
        sm.so2[q][s][c] = 0u;
        sm.sem[q][s][c] = 0u;
    }
    if (threadIdx.x < 4) sm.tilecnt[threadIdx.x >> 1][threadIdx.x & 1] = 0;
    __syncthreads();
    auto tmap = [&](int j, int &sf, int &m) {
        if (FIRST) {
            sf = 0;
            m = 1;
        } else if (j < kRun) {
            sf = sm.run_sf[j];
            m = sm.run_m[j];
        } else {
            tile_segs(j, sf, m, false);  // runs longer than kRun tiles: searched again
        }
    };
    // bounded waits: after one has expired the others return at once, the
    // warp reads no staged data and no scatter uses a base that may not have
    // been published; the barrier arrivals go on, so no warp waits on this one
    bool dead = false;
    auto wait = [&](unsigned long long *bar, int bit) {
        if (!dead && !mbar_wait(bar, (ph >> bit) & 1u, kCopyWaitNs)) {
            dead = true;
            set_status(H, kStTimeout);
        }
        ph ^= 1u << bit;
    };

    if (warp == kCW) {
        // ======== producer warp (warp-uniform control; lane 0 issues)
        // the stage of tile j: later passes, single-segment tile: its range of
        // the point buffers rounded out to 16-byte boundaries (inside the
        // buffers' slack) and the segment record; first pass: the 16-byte
        // multiples of the tile in the caller's x and y (or interleaved xy),
        // never past the caller's arrays.  Other tiles: a plain arrive.
        // (warp-collective: every lane calls it; lane 0 issues the copies)
        auto issue = [&](int j) {
            const int s = j % kRing;
            const int v0 = (t_begin + j) * kSTile, v1 = min(v0 + kSTile, L), cnt = v1 - v0;
            if (FIRST) {
                int c = 0;
                if (A.first_tma == 1) c = cnt & ~3;
                else if (A.first_tma == 2) c = cnt & ~1;
                // the rest of the tile (a ragged end, or all of it when the
                // caller's layout allows no bulk copies) by plain loads
                float *xs = reinterpret_cast<float *>(sm.sxy[s]);
                for (int r = c + lane; r < cnt; r += 32) {
                    const long long v = (long long)(v0 + r) * A.stride;
                    const float x = __ldg(A.x + v), y = __ldg(A.y + v);
                    if (A.first_tma == 2) {
                        sm.sxy[s][r] = make_float2(x, y);
                    } else {
                        xs[r] = x;
                        xs[kStage + r] = y;
                    }
                }
                __syncwarp();
                if (lane != 0) return;
                if (c == 0) {
                    mbar_arrive(&bars.full[s]);
                    return;
                }
                if (!dbg_ok(v0 >= 0 && v0 + c <= A.n, kDbgBulkRange, v0 + c, A.n)) {
                    mbar_arrive(&bars.full[s]);
                    return;
                }
                fence_proxy_async();
                mbar_expect_tx(&bars.full[s], (unsigned)c * 8u);
                if (A.first_tma == 1) {
                    bulk_g2s(xs, A.x + v0, (unsigned)c * 4u, &bars.full[s]);
                    bulk_g2s(xs + kStage, A.y + v0, (unsigned)c * 4u, &bars.full[s]);
                } else {
                    bulk_g2s(sm.sxy[s], A.x + 2ll * v0, (unsigned)c * 8u, &bars.full[s]);
                }
                return;
            }
            int sf, m;
            if (j < kRun) {
                sf = sm.run_sf[j];
                m = sm.run_m[j];
            } else {
                tile_segs(j, sf, m, false);
            }
            if (m != 1) {
                // a tile that straddles segments: its segments' virtual
                // starts go to the stage's index area
                for (int i = lane; i < m; i += 32) sm.sidx[s][i] = seg[sf + i].vstart;
                __syncwarp();
                if (lane == 0) mbar_arrive(&bars.full[s]);
                return;
            }
            if (lane != 0) return;
            const int ps = j < kRun ? sm.run_ps[j] : seg[sf].pstart;
            const int vs = j < kRun ? sm.run_vs[j] : seg[sf].vstart;
            const int pos0 = ps + (v0 - vs);
            const int a0 = pos0 & ~3, a1 = (pos0 + cnt + 3) & ~3, nel = a1 - a0;
            sm.shift[s] = pos0 - a0;
            // inside the buffers and their 64-byte slack; a valid segment
            if (!dbg_ok(a0 >= 0 && a1 <= A.cap_pts + 8, kDbgBulkRange, a1, A.cap_pts) ||
                !dbg_ok(sf >= 0 && sf < A.cap_seg, kDbgSegIndex, sf, A.cap_seg)) {
                mbar_arrive(&bars.full[s]);
                return;
            }
            fence_proxy_async();
            mbar_expect_tx(&bars.full[s], (unsigned)nel * 12u + (unsigned)sizeof(Seg2));
            bulk_g2s(sm.sxy[s], ixy + a0, (unsigned)nel * 8u, &bars.full[s]);
            bulk_g2s(sm.sidx[s], ii + a0, (unsigned)nel * 4u, &bars.full[s]);
            bulk_g2s(&sm.sseg[s], seg + sf, (unsigned)sizeof(Seg2), &bars.full[s]);
        };
        // the point buffers were written by other CTAs' generic stores
        // before the grid barrier; order them before the bulk copies
        if (lane == 0) fence_proxy_async_global();
        for (int j = 0; j < min(nt, kRing); j++) issue(j);
        __syncwarp();
        for (int j = 0; j < nt; j++) {
            const int p = j & 1;
            wait(&bars.counted[p], kPhCounted + p);
            int sf, m;
            tmap(j, sf, m);
            unsigned r0 = 0u, r1 = 0u;
            if (m == 1 && lane == 0) {
                const int t0 = sm.tilecnt[p][0], t1 = sm.tilecnt[p][1];
                sm.tilecnt[p][0] = 0;
                sm.tilecnt[p][1] = 0;
                r0 = t0 ? atomicAdd(&acc[2 * sf].cnt, (unsigned)t0) : 0u;
                r1 = t1 ? atomicAdd(&acc[2 * sf + 1].cnt, (unsigned)t1) : 0u;
            }
            if (m > 1) {
                for (int i = lane; i < 2 * min(m, kMSlot); i += 32) {
                    const int ls = i >> 1, c = i & 1;
                    const Top2 t = {sm.sk1[p][ls][c], sm.so2[p][ls][c], sm.sem[p][ls][c]};
                    if (t.k1) acc_merge(acc[2 * (sf + ls) + c], t);
                    sm.sk1[p][ls][c] = 0ull;
                    sm.so2[p][ls][c] = 0u;
                    sm.sem[p][ls][c] = 0u;
                }
            }
            // every consumer warp has scattered tile j-2 (it did so
            // before classifying tile j): the bases of parity p are free
            __syncwarp();
            if (lane == 0) {
                sm.gb[p][0] = (int)r0;
                sm.gb[p][1] = (int)r1;
                mbar_arrive(&bars.bases[p]);
            }
            __syncwarp();
            if (j >= 1) {
                wait(&bars.empty[(j - 1) % kRing], kPhEmpty + (j - 1) % kRing);
                if (j - 1 + kRing < nt) issue(j - 1 + kRing);
            }
            __syncwarp();
        }
        if (nt > 0) wait(&bars.empty[(nt - 1) % kRing], kPhEmpty + (nt - 1) % kRing);
    } else {
        // ======== consumer warps
        // the first split's pseudo segment (edge a -> a, apex b) covers the input
        Geo2 gfirst = {};
        if (FIRST) {
            const unsigned long long kmn = *(volatile unsigned long long *)&H->lexmin;
            const unsigned long long kmx = *(volatile unsigned long long *)&H->lexmax;
            gfirst.e0x = gfirst.e1x = unord_f32((uint32_t)(kmn >> 32));
            gfirst.e0y = gfirst.e1y = unord_f32((uint32_t)kmn);
            gfirst.qx = unord_f32((uint32_t)(kmx >> 32));
            gfirst.qy = unord_f32((uint32_t)kmx);
            gfirst.q_idx = -1;
        }
        // point r of stage s in the first pass: interleaved xy, or x and y
        // as two arrays (the producer fills the stage either way)
        auto first_point = [&](int s, int r) {
            if (A.first_tma == 2) return sm.sxy[s][r];
            const float *xs = reinterpret_cast<const float *>(sm.sxy[s]);
            return make_float2(xs[r], xs[kStage + r]);
        };
        // farthest-point accumulators of segment `cur` (single-segment tiles)
        int cur = FIRST ? 0 : -1;
        Top2 ta = {0ull, 0u, 0u}, tb = {0ull, 0u, 0u};
        Far2 fa = {0u, 0u, 0u, 0}, fb = {0u, 0u, 0u, 0};
        const int first_tma = A.first_tma;
        auto flush = [&]() {
            if (cur < 0) return;
            ta = far2_top2(fa);
            tb = far2_top2(fb);
            top2_warp(ta);
            top2_warp(tb);
            if (lane == 0) {
                acc_merge(acc[2 * cur], ta);
                acc_merge(acc[2 * cur + 1], tb);
            }
        };
        unsigned cls = 0, cls_prev = 0;  // 2-bit classes of this thread's items
        int off0 = 0, off1 = 0, off0_prev = 0, off1_prev = 0;  // warp's offset in the tile
        bool single = false, prev_single = false;
        for (int j = 0; j <= nt; j++) {
            if (j < nt) {
                const int s = j % kRing, p = j & 1;
                const int v0 = (t_begin + j) * kSTile, v1 = min(v0 + kSTile, L);
                int sf, m;
                tmap(j, sf, m);
                single = m == 1;
                wait(&bars.full[s], kPhFull + s);
                if (single) {
                    const Geo2 g = FIRST ? gfirst : geo_of(sm.sseg[s]);
                    const int shift = FIRST ? 0 : sm.shift[s];
                    if (!FIRST && sf != cur) {
                        flush();
                        cur = sf;
                        fa = {0u, 0u, 0u, 0};
                        fb = {0u, 0u, 0u, 0};
                    }
                    // phase 1, branch-free: filter values and classes of all
                    // items (independent chains the compiler interleaves)
                    const int wbase = v0 + warp * 32 * kSItems;
                    float dsel[kSItems], esel[kSItems];
                    int pidx[kSItems];
                    unsigned unc = 0;
                    cls = 0;
#pragma unroll
                    for (int k = 0; k < kSItems; k++) {
                        const int v = wbase + k * 32 + lane;
                        const bool ok = v < v1;
                        const int r = ok ? v - v0 + shift : 0;
                        float2 pt;
                        if (FIRST) {
                            pt = first_point(s, r);
                            pidx[k] = v;
                        } else {
                            pt = sm.sxy[s][r];
                            pidx[k] = sm.sidx[s][r];
                        }
                        float d0, e0, d1, e1;
                        orient_value<P>(g.e0x, g.e0y, g.qx, g.qy, pt.x, pt.y, d0, e0);
                        if (FIRST) {
                            d1 = -d0;
                            e1 = e0;
                        } else {
                            orient_value<P>(g.qx, g.qy, g.e1x, g.e1y, pt.x, pt.y, d1, e1);
                        }
                        const bool pos0 = d0 > e0, neg0 = -d0 > e0, pos1 = d1 > e1, neg1 = -d1 > e1;
                        const bool apex = !FIRST && pidx[k] == g.q_idx;
                        int c = pos0 ? 0 : (pos1 ? 1 : 2);
                        c = apex ? 2 : c;
                        c = ok ? c : 3;
                        const bool u = ok && !apex && !pos0 && !(neg0 && (pos1 || neg1));
                        unc |= (unsigned)u << k;
                        dsel[k] = c == 0 ? d0 : d1;
                        esel[k] = c == 0 ? e0 : e1;
                        cls |= (unsigned)c << (2 * k);
                    }
                    // phase 2, rare: a thread with an item the filter cannot
                    // decide classifies all its items with exact signs
                    if (unc) {
                        cls = 0;
#pragma unroll
                        for (int k = 0; k < kSItems; k++) {
                            const int v = wbase + k * 32 + lane;
                            int c = 3;
                            if (v < v1) {
                                const int r = v - v0 + shift;
                                const float2 pt = FIRST ? first_point(s, r) : sm.sxy[s][r];
                                float d = 0.f, e = 0.f;
                                c = classify2d<P>(g, pt.x, pt.y, FIRST ? -2 : pidx[k], d, e,
                                                  fallbacks);
                                dsel[k] = d;
                                esel[k] = e;
                            }
                            cls |= (unsigned)c << (2 * k);
                        }
                    }
                    // phase 3, branch-free: farthest-point keys and counts
                    int w0 = 0, w1 = 0;
                    int n0 = 0, n1 = 0;
#pragma unroll
                    for (int k = 0; k < kSItems; k++) {
                        const int c = (int)((cls >> (2 * k)) & 3u);
                        const unsigned o = ord_f32(dsel[k]);
                        const unsigned eb = __float_as_uint(esel[k]);
                        far2_add(fa, c == 0 ? o : 0u, pidx[k], c == 0 ? eb : 0u);
                        far2_add(fb, c == 1 ? o : 0u, pidx[k], c == 1 ? eb : 0u);
                        n0 += c == 0;
                        n1 += c == 1;
                    }
                    w0 = __reduce_add_sync(0xffffffffu, n0);
                    w1 = __reduce_add_sync(0xffffffffu, n1);
                    if (lane == 0) {
                        off0 = atomicAdd(&sm.tilecnt[p][0], w0);
                        off1 = atomicAdd(&sm.tilecnt[p][1], w1);
                    }
                    off0 = __shfl_sync(0xffffffffu, off0, 0);
                    off1 = __shfl_sync(0xffffffffu, off1, 0);
                } else if (!dead) {
                    multi_tile<P>(sm, seg, acc, sf, m, v0, v1, p, ixy, ii, oxy, oi, fallbacks,
                                  sm.sidx[s], A.cap_pts);
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&bars.counted[p]);
            }
            if (j >= 1) {
                // scatter tile j-1 with the bases the producer published
                const int jp = j - 1, sp = jp % kRing, pp = jp & 1;
                wait(&bars.bases[pp], kPhBases + pp);
                if (prev_single && !dead) {
                    const int pv0 = (t_begin + jp) * kSTile;
                    const int shift = FIRST ? 0 : sm.shift[sp];
                    const int ps = FIRST ? 0 : sm.sseg[sp].pstart;
                    const int ln = FIRST ? A.n : sm.sseg[sp].len;
                    int base0 = sm.gb[pp][0] + off0_prev, base1 = sm.gb[pp][1] + off1_prev;
                    const int wbase = pv0 + warp * 32 * kSItems;
                    // destinations and stage reads of all items, then the stores
                    int dst[kSItems];
                    float2 spt[kSItems];
                    int sidx[kSItems];
                    const int r0 = wbase - pv0 + shift + lane;
                    int lo = ps + base0, hi = ps + ln - 1 - base1;
#pragma unroll
                    for (int k = 0; k < kSItems; k++) {
                        const int c = (int)((cls_prev >> (2 * k)) & 3u);
                        const unsigned b0 = __ballot_sync(0xffffffffu, c == 0);
                        const unsigned b1 = __ballot_sync(0xffffffffu, c == 1);
                        dst[k] = c == 0 ? lo + __popc(b0 & lt)
                                        : (c == 1 ? hi - __popc(b1 & lt) : -1);
                        lo += __popc(b0);
                        hi -= __popc(b1);
                        const int r = r0 + k * 32;
                        if (FIRST) {
                            if (first_tma == 2) {
                                spt[k] = sm.sxy[sp][r];
                            } else {
                                const float *xs = reinterpret_cast<const float *>(sm.sxy[sp]);
                                spt[k] = make_float2(xs[r], xs[kStage + r]);
                            }
                            sidx[k] = wbase + k * 32 + lane;
                        } else {
                            spt[k] = sm.sxy[sp][r];
                            sidx[k] = sm.sidx[sp][r];
                        }
                    }
#pragma unroll
                    for (int k = 0; k < kSItems; k++) {
                        if (dst[k] >= 0 &&
                            dbg_ok(dst[k] < A.cap_pts, kDbgPointDst, dst[k], A.cap_pts)) {
                            oxy[dst[k]] = spt[k];
                            oi[dst[k]] = sidx[k];
                        }
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&bars.empty[sp]);
            }
            prev_single = single;
            cls_prev = cls;
            off0_prev = off0;
            off1_prev = off1;
        }
        flush();
    }
    // after an expired wait, copies into the stage ring may still be in
    // flight: the CTA stays until the last copy issued to every stage has
    // landed (warp 0 counted every tile's phase of the full barriers, waited
    // for or not), bounded again; past that bound the CTA leaves best-effort
    if (__syncthreads_or(dead) && threadIdx.x == 0) {
        for (int s = 0; s < kRing; s++)
            mbar_wait(&bars.full[s], ((ph >> (kPhFull + s)) & 1u) ^ 1u, kCopyWaitNs);
    }
    const unsigned f = __reduce_add_sync(0xffffffffu, fallbacks);
    if (lane == 0 && f) atomicAdd(&H->fallbacks, (unsigned long long)f);
}

// ---------------------------------------------------------------- update
// Build the next segment table from the non-empty children (block 0 only).
// The tile -> segment map for the next pass is written when that pass has
// fewer than map_below live points (the passes of the persistent kernel's
// grid phase find their tiles' segments themselves).
__device__ void update2d(const Params2 &A, int par, bool first, SmemU &sm,
                         int map_below = INT_MAX)
{
    Hdr2 *H = A.hdr;
    Seg2 *so = A.seg[par];
    Acc2 *ac = A.acc[par];
    Seg2 *sn = A.seg[par ^ 1];
    Acc2 *an = A.acc[par ^ 1];
    if (first) {
        // the first split's pseudo segment: edge a -> a with apex b
        if (threadIdx.x == 0) {
            unsigned long long kmn = *(volatile unsigned long long *)&H->lexmin;
            unsigned long long kmx = *(volatile unsigned long long *)&H->lexmax;
            Seg2 g = {};
            g.e0x = g.e1x = unord_f32((uint32_t)(kmn >> 32));
            g.e0y = g.e1y = unord_f32((uint32_t)kmn);
            g.qx = unord_f32((uint32_t)(kmx >> 32));
            g.qy = unord_f32((uint32_t)kmx);
            g.q_idx = -1;
            g.e0_slot = 0;
            g.q_slot = 1;
            g.e1_slot = 0;
            g.pstart = 0;
            g.len = A.n;
            so[0] = g;
            int ai = *(volatile int *)&H->a_idx, bi = *(volatile int *)&H->b_idx;
            A.hull_idx[0] = ai;
            A.hull_x[0] = g.e0x;
            A.hull_y[0] = g.e0y;
            A.hull_idx[1] = bi;
            A.hull_x[1] = g.qx;
            A.hull_y[1] = g.qy;
            A.next[0] = 1;
            A.next[1] = 0;
        }
        __syncthreads();
    }
    const int S_old = *(volatile int *)&H->S[par];
    const int hull_base = *(volatile int *)&H->hull_count;
    if (threadIdx.x == 0) H->n_uncert = 0;
    __syncthreads();
    const int nslots = 2 * S_old;
    long long carry_k = 0, carry_v = 0;
    for (int base = 0; base < nslots; base += blockDim.x) {
        int i = base + threadIdx.x;
        unsigned cnt = (i < nslots) ? ac[i].cnt : 0u;
        long long packed = ((long long)(cnt > 0) << 32) | (long long)cnt;
        long long tot;
        long long ex = block_excl_scan64(packed, sm.wsum, &tot);
        if (cnt > 0 && carry_k + (ex >> 32) >= A.cap_seg) {
            set_status(H, kStCapacity);
        } else if (cnt > 0) {
            int k = (int)(carry_k + (ex >> 32));
            int vs = (int)(carry_v + (ex & 0xffffffffll));
            int j = i >> 1, c = i & 1;
            Seg2 o = so[j];
            Acc2 a = ac[i];
            Seg2 g = {};
            if (c == 0) {
                g.e0x = o.e0x; g.e0y = o.e0y; g.e0_slot = o.e0_slot;
                g.e1x = o.qx;  g.e1y = o.qy;  g.e1_slot = o.q_slot;
                g.pstart = o.pstart;
            } else {
                g.e0x = o.qx;  g.e0y = o.qy;  g.e0_slot = o.q_slot;
                g.e1x = o.e1x; g.e1y = o.e1y; g.e1_slot = o.e1_slot;
                g.pstart = o.pstart + o.len - (int)cnt;
            }
            g.len = (int)cnt;
            g.vstart = vs;
            int qi = key_idx(a.key1);
            g.q_idx = qi;
            g.qx = __ldg(A.x + (long long)qi * A.stride);
            g.qy = __ldg(A.y + (long long)qi * A.stride);
            int slot = hull_base + k;
            g.q_slot = slot;
            // certified when the FP32 gap between the two best keys exceeds
            // twice the largest error bound of the segment's keys
            bool cert = true;
            float em = __uint_as_float(a.emax);
            float d1 = key_dist(a.key1);
            if (cnt > 1) {
                float d2 = unord_f32(a.o2);
                double gap = ((double)d1 - (double)d2) * (1.0 - 0x1p-50);
                cert = gap > 2.0 * (double)em;
            }
            if (!cert) {
                double thr = (double)d1 - (double)em - 2.0 * (double)em - fabs((double)d1) * 0x1p-20;
                g.thr = isfinite(thr) ? __double2float_rd(thr) : -INFINITY;
                int u = atomicAdd(&H->n_uncert, 1);
                A.uncert[u] = k;
            }
            if (dbg_ok(slot < A.cap_hull && g.e0_slot >= 0 && g.e0_slot < A.cap_hull,
                       kDbgHullSlot, slot, A.cap_hull)) {
                A.hull_idx[slot] = qi;
                A.hull_x[slot] = g.qx;
                A.hull_y[slot] = g.qy;
                A.next[g.e0_slot] = slot;
                A.next[slot] = g.e1_slot;
            }
            Acc2 z = {};
            an[2 * k] = z;
            an[2 * k + 1] = z;
            sn[k] = g;
            if (k < kTile) sm.vs[k] = vs;
        }
        carry_k += tot >> 32;
        carry_v += tot & 0xffffffffll;
    }
    const int S_new = (int)carry_k, L_new = (int)carry_v;
    __syncthreads();
    // tile -> (first segment, number of segments) map for the next pass
    const int ntiles = (L_new + kTile - 1) / kTile;
    auto seg_of = [&](int v) {
        int lo = 0, hi = S_new - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            int vs = (S_new <= kTile) ? sm.vs[mid] : sn[mid].vstart;
            if (vs <= v) lo = mid;
            else hi = mid - 1;
        }
        return lo;
    };
    // (the persistent kernel's passes find their own tiles' segments)
    for (int t = threadIdx.x; L_new < map_below && t < ntiles; t += blockDim.x) {
        int v = t * kTile;
        int vl = min(v + kTile, L_new) - 1;
        int s0 = seg_of(v);
        A.tile_seg[t] = s0;
        A.tile_m[t] = seg_of(vl) - s0 + 1;
    }
    if (threadIdx.x == 0) {
        H->S[par ^ 1] = S_new;
        H->L[par ^ 1] = L_new;
        H->hull_count = hull_base + S_new;
        H->seg_total += S_new;
        H->surv_total += L_new;
        H->exact_argmax += H->n_uncert;
    }
    __syncthreads();
}

// ---------------------------------------------------------------- exact argmax
// Farthest point of each uncertified segment with exact comparisons
// (largest distance, then lowest index), one block per segment.
template <class P>
__device__ void exact2d(const Params2 &A, int par, SmemX &sm, int bid, int nb)
{
    Hdr2 *H = A.hdr;
    const int nu = *(volatile int *)&H->n_uncert;
    Seg2 *sn = A.seg[par ^ 1];
    const float2 *bxy = A.bxy[par];
    const int *bi = A.bi[par];
    for (int u = bid; u < nu; u += nb) {
        const int k = A.uncert[u];
        const Seg2 g = sn[k];
        int best = -1;
        float bxv = 0.f, byv = 0.f;
        for (int i = threadIdx.x; i < g.len; i += blockDim.x) {
            int pos = g.pstart + i;
            float2 p = bxy[pos];
            float x = p.x, y = p.y;
            int idx = bi[pos];
            float d, e;
            orient_value<P>(g.e0x, g.e0y, g.e1x, g.e1y, x, y, d, e);
            if ((double)d + (double)e < (double)g.thr) continue;
            if (best < 0) {
                best = idx; bxv = x; byv = y;
                continue;
            }
            int c = cmp_dist_exact(g.e0x, g.e0y, g.e1x, g.e1y, x, y, bxv, byv);
            if (c > 0 || (c == 0 && idx < best)) {
                best = idx; bxv = x; byv = y;
            }
        }
        sm.bidx[threadIdx.x] = best;
        sm.bx[threadIdx.x] = bxv;
        sm.by[threadIdx.x] = byv;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) {
                int o = threadIdx.x + s;
                int oi = sm.bidx[o];
                if (oi >= 0) {
                    int mi = sm.bidx[threadIdx.x];
                    bool take = mi < 0;
                    if (!take) {
                        int c = cmp_dist_exact(g.e0x, g.e0y, g.e1x, g.e1y, sm.bx[o], sm.by[o],
                                               sm.bx[threadIdx.x], sm.by[threadIdx.x]);
                        take = c > 0 || (c == 0 && oi < mi);
                    }
                    if (take) {
                        sm.bidx[threadIdx.x] = oi;
                        sm.bx[threadIdx.x] = sm.bx[o];
                        sm.by[threadIdx.x] = sm.by[o];
                    }
                }
            }
            __syncthreads();
        }
        if (threadIdx.x == 0 && sm.bidx[0] >= 0) {
            sn[k].q_idx = sm.bidx[0];
            sn[k].qx = sm.bx[0];
            sn[k].qy = sm.by[0];
            A.hull_idx[g.q_slot] = sm.bidx[0];
            A.hull_x[g.q_slot] = sm.bx[0];
            A.hull_y[g.q_slot] = sm.by[0];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- output
// Rank the hull links (clockwise from slot 0 = a) by pointer jumping,
// reverse to counter-clockwise, drop vertices collinear with their
// neighbours, write the indices (block 0 only).
__device__ void output2d(const Params2 &A, SmemOut &sm)
{
    Hdr2 *H = A.hdr;
    qh_result *R = A.res;
    int st = *(volatile int *)&H->status;
    long long count = 0;
    if (st == 0) {
        unsigned long long kmn = *(volatile unsigned long long *)&H->lexmin;
        unsigned long long kmx = *(volatile unsigned long long *)&H->lexmax;
        const int h = *(volatile int *)&H->hull_count;
        if (A.n == 0) {
            count = 0;
        } else if (kmn == kmx) {
            if (threadIdx.x == 0) A.out_idx[0] = *(volatile int *)&H->a_idx;
            count = 1;
        } else if (h > kOutCap) {
            st = QH_ERR_CAPACITY;
        } else {
            for (int i = threadIdx.x; i < h; i += blockDim.x) {
                int s = A.next[i];
                sm.succ[i] = (s == 0) ? -1 : s;
                sm.dist[i] = (s == 0) ? 0 : 1;
            }
            __syncthreads();
            constexpr int kPer = kOutCap / kBlock;
            for (int span = 1; span < h; span <<= 1) {
                int ns[kPer], nd[kPer];
#pragma unroll
                for (int r = 0; r < kPer; r++) {
                    int i = threadIdx.x + r * kBlock;
                    ns[r] = -1;
                    nd[r] = 0;
                    if (i < h) {
                        int s = sm.succ[i];
                        nd[r] = sm.dist[i];
                        ns[r] = s;
                        if (s >= 0) {
                            nd[r] += sm.dist[s];
                            ns[r] = sm.succ[s];
                        }
                    }
                }
                __syncthreads();
#pragma unroll
                for (int r = 0; r < kPer; r++) {
                    int i = threadIdx.x + r * kBlock;
                    if (i < h) {
                        sm.succ[i] = ns[r];
                        sm.dist[i] = nd[r];
                    }
                }
                __syncthreads();
            }
            // position counter-clockwise from a: pos = (h - rank) mod h with
            // rank = h - 1 - dist (clockwise position)
            for (int i = threadIdx.x; i < h; i += blockDim.x) {
                int rank = h - 1 - sm.dist[i];
                int pos = (h - rank) % h;
                sm.succ[pos] = i;  // succ reused as order[]
            }
            __syncthreads();
            int keep[kPer];
            long long my = 0;
#pragma unroll
            for (int r = 0; r < kPer; r++) {
                int p = threadIdx.x * kPer + r;
                keep[r] = 0;
                if (p < h) {
                    if (h <= 2) {
                        keep[r] = 1;
                    } else {
                        int sp = sm.succ[(p + h - 1) % h], sv = sm.succ[p], sx = sm.succ[(p + 1) % h];
                        keep[r] = orient_exact_sign(A.hull_x[sp], A.hull_y[sp], A.hull_x[sv],
                                                    A.hull_y[sv], A.hull_x[sx], A.hull_y[sx]) != 0;
                    }
                    my += keep[r];
                }
            }
            long long tot;
            long long off = block_excl_scan64(my, sm.wsum, &tot);
#pragma unroll
            for (int r = 0; r < kPer; r++) {
                int p = threadIdx.x * kPer + r;
                if (p < h && keep[r]) A.out_idx[off++] = A.hull_idx[sm.succ[p]];
            }
            count = tot;
        }
    }
    if (threadIdx.x == 0) {
        R->count = (st == 0) ? count : 0;
        R->status = st;
        R->iterations = *(volatile int *)&H->iter;
        R->survivor_total = *(volatile long long *)&H->surv_total;
        R->live_total = (long long)A.n + R->survivor_total;
        R->segments_total = *(volatile long long *)&H->seg_total;
        R->filter_fallbacks = *(volatile unsigned long long *)&H->fallbacks;
        R->exact_argmax = *(volatile unsigned long long *)&H->exact_argmax;
        for (int i = 0; i < 4; i++) R->extra[i] = (long long)*(volatile unsigned long long *)&H->phase_ns[i];
    }
}

// ---------------------------------------------------------------- persistent kernel
// Shared memory of the persistent kernel (dynamic): the phases' union and the
// pipelined pass's buffers alias; the bulk-copy barriers stay apart.
extern __shared__ __align__(16) unsigned char qh2d_dsm[];
constexpr size_t kPersistSmem =
    sizeof(SmemAll) > sizeof(SmemStream) ? sizeof(SmemAll) : sizeof(SmemStream);

// ---------------------------------------------------------------- several clouds
// qh_hull2d_multi: K independent clouds in one persistent launch.  The
// clouds' live points share the segment table and the point buffers (cloud c
// owns the physical range [off_c, off_c + n_c)), so every pass, update and
// grid barrier serves all of them, and the tiles of every pass balance the
// clouds' work over the whole grid.  Point records carry cloud-local
// indices; a segment carries its cloud (Seg2.pad[0]) for its apex's
// coordinates, a hull slot its cloud for the output step.  Each cloud has a
// header of its own for the extrema and the first split (lexmin, lexmax,
// lowest indices, non-finite flag) and its own output and result record.
constexpr int kMaxClouds = QH_MAX_CLOUDS_2D;

struct Cloud2 {
    const float *x, *y;
    long long stride;
    int n, first_tma;
    int off;           // physical start of the cloud's points in the point buffers
    int *out_idx;
    qh_result *res;
    Hdr2 *hdr;         // extrema and first-split state of the cloud
};

struct Params2M {
    Params2 A;         // the shared state: all clouds' points (N = sum of n_c)
    int K;
    int *hull_cloud;   // cloud of every hull slot
    Cloud2 c[kMaxClouds];
};

// Single-cloud parameters of cloud c for its extrema and its first split: its
// input and header, its accumulator pair, its range of the first buffer.
__device__ __forceinline__ Params2 cloud_params(const Params2M &M, int c)
{
    Params2 a = M.A;
    const Cloud2 &C = M.c[c];
    a.x = C.x;
    a.y = C.y;
    a.stride = C.stride;
    a.n = C.n;
    a.first_tma = C.first_tma;
    a.hdr = C.hdr;
    a.acc[0] = M.A.acc[0] + 2 * c;
    a.bxy[0] = M.A.bxy[0] + C.off;
    a.bi[0] = M.A.bi[0] + C.off;
    a.cap_pts = M.A.cap_pts - C.off;
    return a;
}

__device__ __forceinline__ bool cloud_live(const Params2M &M, int c)
{
    return M.c[c].n > 0 && !*(volatile int *)&M.c[c].hdr->nonfinite;
}

// update2d for several clouds: the first update lays out every cloud's first
// split (pseudo segment a_c -> b_c -> a_c over its physical range, hull slots
// 2c and 2c+1); later ones as update2d, with the apex read from the
// segment's cloud and every new hull slot tagged with it.
__device__ void update2d_m(const Params2M &M, int par, bool first, SmemU &sm, int map_below)
{
    const Params2 &A = M.A;
    Hdr2 *H = A.hdr;
    Seg2 *so = A.seg[par];
    Acc2 *ac = A.acc[par];
    Seg2 *sn = A.seg[par ^ 1];
    Acc2 *an = A.acc[par ^ 1];
    if (first) {
        for (int c = threadIdx.x; c < M.K; c += blockDim.x) {
            const Cloud2 &C = M.c[c];
            Hdr2 *Hc = C.hdr;
            const unsigned long long kmn = *(volatile unsigned long long *)&Hc->lexmin;
            const unsigned long long kmx = *(volatile unsigned long long *)&Hc->lexmax;
            Seg2 g = {};
            g.e0x = g.e1x = unord_f32((uint32_t)(kmn >> 32));
            g.e0y = g.e1y = unord_f32((uint32_t)kmn);
            g.qx = unord_f32((uint32_t)(kmx >> 32));
            g.qy = unord_f32((uint32_t)kmx);
            g.q_idx = -1;
            g.e0_slot = 2 * c;
            g.q_slot = 2 * c + 1;
            g.e1_slot = 2 * c;
            g.pstart = C.off;
            g.len = C.n;
            g.pad[0] = c;
            so[c] = g;
            A.hull_idx[2 * c] = *(volatile int *)&Hc->a_idx;
            A.hull_x[2 * c] = g.e0x;
            A.hull_y[2 * c] = g.e0y;
            A.hull_idx[2 * c + 1] = *(volatile int *)&Hc->b_idx;
            A.hull_x[2 * c + 1] = g.qx;
            A.hull_y[2 * c + 1] = g.qy;
            A.next[2 * c] = 2 * c + 1;
            A.next[2 * c + 1] = 2 * c;
            M.hull_cloud[2 * c] = c;
            M.hull_cloud[2 * c + 1] = c;
        }
        __syncthreads();
    }
    const int S_old = *(volatile int *)&H->S[par];
    const int hull_base = *(volatile int *)&H->hull_count;
    if (threadIdx.x == 0) {
        H->n_uncert = 0;
        H->maxlen = 0;
    }
    __syncthreads();
    unsigned longest = 0;
    const int nslots = 2 * S_old;
    long long carry_k = 0, carry_v = 0;
    for (int base = 0; base < nslots; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const unsigned cnt = (i < nslots) ? ac[i].cnt : 0u;
        longest = max(longest, cnt);
        const long long packed = ((long long)(cnt > 0) << 32) | (long long)cnt;
        long long tot;
        const long long ex = block_excl_scan64(packed, sm.wsum, &tot);
        if (cnt > 0 && carry_k + (ex >> 32) >= A.cap_seg) {
            set_status(H, kStCapacity);
        } else if (cnt > 0) {
            const int k = (int)(carry_k + (ex >> 32));
            const int vs = (int)(carry_v + (ex & 0xffffffffll));
            const int j = i >> 1, c = i & 1;
            const Seg2 o = so[j];
            const Acc2 a = ac[i];
            const int cl = o.pad[0];
            const Cloud2 &C = M.c[cl];
            Seg2 g = {};
            if (c == 0) {
                g.e0x = o.e0x; g.e0y = o.e0y; g.e0_slot = o.e0_slot;
                g.e1x = o.qx;  g.e1y = o.qy;  g.e1_slot = o.q_slot;
                g.pstart = o.pstart;
            } else {
                g.e0x = o.qx;  g.e0y = o.qy;  g.e0_slot = o.q_slot;
                g.e1x = o.e1x; g.e1y = o.e1y; g.e1_slot = o.e1_slot;
                g.pstart = o.pstart + o.len - (int)cnt;
            }
            g.len = (int)cnt;
            g.vstart = vs;
            g.pad[0] = cl;
            const int qi = key_idx(a.key1);
            g.q_idx = qi;
            g.qx = __ldg(C.x + (long long)qi * C.stride);
            g.qy = __ldg(C.y + (long long)qi * C.stride);
            const int slot = hull_base + k;
            g.q_slot = slot;
            // certified when the FP32 gap between the two best keys exceeds
            // twice the largest error bound of the segment's keys
            bool cert = true;
            const float em = __uint_as_float(a.emax);
            const float d1 = key_dist(a.key1);
            if (cnt > 1) {
                const float d2 = unord_f32(a.o2);
                const double gap = ((double)d1 - (double)d2) * (1.0 - 0x1p-50);
                cert = gap > 2.0 * (double)em;
            }
            if (!cert) {
                const double thr =
                    (double)d1 - (double)em - 2.0 * (double)em - fabs((double)d1) * 0x1p-20;
                g.thr = isfinite(thr) ? __double2float_rd(thr) : -INFINITY;
                const int u = atomicAdd(&H->n_uncert, 1);
                A.uncert[u] = k;
            }
            if (dbg_ok(slot < A.cap_hull && g.e0_slot >= 0 && g.e0_slot < A.cap_hull,
                       kDbgHullSlot, slot, A.cap_hull)) {
                A.hull_idx[slot] = qi;
                A.hull_x[slot] = g.qx;
                A.hull_y[slot] = g.qy;
                M.hull_cloud[slot] = cl;
                A.next[g.e0_slot] = slot;
                A.next[slot] = g.e1_slot;
            }
            const Acc2 z = {};
            an[2 * k] = z;
            an[2 * k + 1] = z;
            sn[k] = g;
            if (k < kTile) sm.vs[k] = vs;
        }
        carry_k += tot >> 32;
        carry_v += tot & 0xffffffffll;
    }
    const int S_new = (int)carry_k, L_new = (int)carry_v;
    longest = __reduce_max_sync(0xffffffffu, longest);
    if ((threadIdx.x & 31) == 0 && longest) atomicMax(&H->maxlen, (int)longest);
    __syncthreads();
    const int ntiles = (L_new + kTile - 1) / kTile;
    auto seg_of = [&](int v) {
        int lo = 0, hi = S_new - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            const int vs = (S_new <= kTile) ? sm.vs[mid] : sn[mid].vstart;
            if (vs <= v) lo = mid;
            else hi = mid - 1;
        }
        return lo;
    };
    for (int t = threadIdx.x; L_new < map_below && t < ntiles; t += blockDim.x) {
        const int v = t * kTile;
        const int vl = min(v + kTile, L_new) - 1;
        const int s0 = seg_of(v);
        A.tile_seg[t] = s0;
        A.tile_m[t] = seg_of(vl) - s0 + 1;
    }
    if (threadIdx.x == 0) {
        H->S[par ^ 1] = S_new;
        H->L[par ^ 1] = L_new;
        H->hull_count = hull_base + S_new;
        H->seg_total += S_new;
        H->surv_total += L_new;
        H->exact_argmax += H->n_uncert;
    }
    __syncthreads();
}

// The exact argmax of the several-cloud kernel.  With fewer uncertified
// segments than CTAs each segment's points are split into `per` chunks, one
// CTA each (a tie at the top of a large segment, e.g. a duplicated extreme
// point, would otherwise leave millions of points to one CTA).  A chunk's
// best (exact comparison, then lowest index) goes to slot w of the point
// buffers of the other parity, free until the next pass writes them, and
// exact2d_merge reduces the chunks after a grid barrier.  per = 1 is exact2d.
// Chunks of at least kExactChunk points (of the longest such segment): a
// shorter segment costs a CTA less than the extra barrier and merge.  Every
// CTA reads the same lengths, so all agree on per.
constexpr int kExactChunk = 65536;
__device__ int exact_chunks2d(const Params2 &A, int par, SmemX &sm, int nu, int nb)
{
    if (nu <= 0) return 1;
    long long cap = nb / nu;
    if (cap * nu > (long long)A.n) cap = A.n / nu;
    if (cap <= 1) return 1;
    const Seg2 *sn = A.seg[par ^ 1];
    int mx = 0;
    for (int u = threadIdx.x; u < nu; u += blockDim.x) mx = max(mx, sn[A.uncert[u]].len);
    mx = (int)__reduce_max_sync(0xffffffffu, (unsigned)mx);
    if ((threadIdx.x & 31) == 0) sm.bidx[threadIdx.x >> 5] = mx;
    __syncthreads();
    int m = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) m = max(m, sm.bidx[w]);
    __syncthreads();
    const long long want = ((long long)m + kExactChunk - 1) / kExactChunk;
    return (int)max(1ll, min(cap, want));
}

template <class P>
__device__ void exact2d_split(const Params2 &A, int par, SmemX &sm, int bid, int nb, int per)
{
    Hdr2 *H = A.hdr;
    const int nu = *(volatile int *)&H->n_uncert;
    Seg2 *sn = A.seg[par ^ 1];
    const float2 *bxy = A.bxy[par];
    const int *bi = A.bi[par];
    float2 *cxy = A.bxy[par ^ 1];
    int *ci = A.bi[par ^ 1];
    for (int w = bid; w < nu * per; w += nb) {
        const int u = w / per, q = w - u * per;
        const int k = A.uncert[u];
        const Seg2 g = sn[k];
        const int i0 = (int)((long long)g.len * q / per), i1 = (int)((long long)g.len * (q + 1) / per);
        int best = -1;
        float bxv = 0.f, byv = 0.f;
        for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
            const int pos = g.pstart + i;
            const float2 p = bxy[pos];
            const int idx = bi[pos];
            float d, e;
            orient_value<P>(g.e0x, g.e0y, g.e1x, g.e1y, p.x, p.y, d, e);
            if ((double)d + (double)e < (double)g.thr) continue;
            if (best >= 0) {
                const int c = cmp_dist_exact(g.e0x, g.e0y, g.e1x, g.e1y, p.x, p.y, bxv, byv);
                if (!(c > 0 || (c == 0 && idx < best))) continue;
            }
            best = idx;
            bxv = p.x;
            byv = p.y;
        }
        sm.bidx[threadIdx.x] = best;
        sm.bx[threadIdx.x] = bxv;
        sm.by[threadIdx.x] = byv;
        __syncthreads();
        for (int st = blockDim.x / 2; st > 0; st >>= 1) {
            if (threadIdx.x < st) {
                const int o = threadIdx.x + st;
                const int oi = sm.bidx[o];
                if (oi >= 0) {
                    const int mi = sm.bidx[threadIdx.x];
                    bool take = mi < 0;
                    if (!take) {
                        const int c = cmp_dist_exact(g.e0x, g.e0y, g.e1x, g.e1y, sm.bx[o], sm.by[o],
                                                     sm.bx[threadIdx.x], sm.by[threadIdx.x]);
                        take = c > 0 || (c == 0 && oi < mi);
                    }
                    if (take) {
                        sm.bidx[threadIdx.x] = oi;
                        sm.bx[threadIdx.x] = sm.bx[o];
                        sm.by[threadIdx.x] = sm.by[o];
                    }
                }
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            if (per > 1) {
                ci[w] = sm.bidx[0];
                cxy[w] = make_float2(sm.bx[0], sm.by[0]);
            } else if (sm.bidx[0] >= 0) {
                sn[k].q_idx = sm.bidx[0];
                sn[k].qx = sm.bx[0];
                sn[k].qy = sm.by[0];
                A.hull_idx[g.q_slot] = sm.bidx[0];
                A.hull_x[g.q_slot] = sm.bx[0];
                A.hull_y[g.q_slot] = sm.by[0];
            }
        }
        __syncthreads();
    }
}

// The chunks' bests of each uncertified segment, one thread per segment.
__device__ void exact2d_merge(const Params2 &A, int par, int bid, int nb, int per)
{
    Hdr2 *H = A.hdr;
    const int nu = *(volatile int *)&H->n_uncert;
    Seg2 *sn = A.seg[par ^ 1];
    const float2 *cxy = A.bxy[par ^ 1];
    const int *ci = A.bi[par ^ 1];
    for (int u = bid * blockDim.x + threadIdx.x; u < nu; u += nb * blockDim.x) {
        const int k = A.uncert[u];
        const Seg2 g = sn[k];
        int best = -1;
        float bxv = 0.f, byv = 0.f;
        for (int q = 0; q < per; q++) {
            const int idx = ci[u * per + q];
            if (idx < 0) continue;
            const float2 p = cxy[u * per + q];
            if (best >= 0) {
                const int c = cmp_dist_exact(g.e0x, g.e0y, g.e1x, g.e1y, p.x, p.y, bxv, byv);
                if (!(c > 0 || (c == 0 && idx < best))) continue;
            }
            best = idx;
            bxv = p.x;
            byv = p.y;
        }
        if (best >= 0) {
            sn[k].q_idx = best;
            sn[k].qx = bxv;
            sn[k].qy = byv;
            A.hull_idx[g.q_slot] = best;
            A.hull_x[g.q_slot] = bxv;
            A.hull_y[g.q_slot] = byv;
        }
    }
}

// A pass over short segments (several-cloud kernel): one warp per segment
// classifies its points 32 at a time (the next 32 loaded before the current
// ones are stored), writes child 0 from the left end of the segment's range
// and child 1 from the right end with ballot ranks, and stores both
// children's accumulators itself: the warp owns the segment, so there are no
// reservation or key atomics.
template <class P>
__device__ void pass2d_warpseg(const Params2 &A, int par, int bid, int nb)
{
    Hdr2 *H = A.hdr;
    const int S = vload_i(&H->S[par]);
    const Seg2 *seg = A.seg[par];
    Acc2 *acc = A.acc[par];
    const float2 *ixy = A.bxy[par ^ 1];
    const int *ii = A.bi[par ^ 1];
    float2 *oxy = A.bxy[par];
    int *oi = A.bi[par];
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    const int wpb = blockDim.x >> 5;
    unsigned fallbacks = 0;
    for (int sg = bid * wpb + (threadIdx.x >> 5); sg < S; sg += nb * wpb) {
        const Geo2 g = geo_of(seg[sg]);
        const int ps = g.pstart, len = g.len;
        Far2 fa = {0u, 0u, 0u, 0}, fb = {0u, 0u, 0u, 0};
        int n0 = 0, n1 = 0;
        float2 cp = make_float2(0.f, 0.f);
        int ci = 0;
        if (lane < len) {
            cp = ixy[ps + lane];
            ci = ii[ps + lane];
        }
        for (int b = 0; b < len; b += 32) {
            const int i = b + lane;
            float2 np = make_float2(0.f, 0.f);
            int ni = 0;
            if (i + 32 < len) {
                np = ixy[ps + i + 32];
                ni = ii[ps + i + 32];
            }
            int c = 3;
            float d = 0.f, e = 0.f;
            if (i < len) c = classify2d<P>(g, cp.x, cp.y, ci, d, e, fallbacks);
            const unsigned b0 = __ballot_sync(0xffffffffu, c == 0);
            const unsigned b1 = __ballot_sync(0xffffffffu, c == 1);
            if (c == 0) {
                const int dst = ps + n0 + __popc(b0 & lt);
                if (dbg_ok(dst >= 0 && dst < A.cap_pts, kDbgPointDst, dst, A.cap_pts)) {
                    oxy[dst] = cp;
                    oi[dst] = ci;
                }
                far2_add(fa, ord_f32(d), ci, __float_as_uint(e));
            } else if (c == 1) {
                const int dst = ps + len - 1 - (n1 + __popc(b1 & lt));
                if (dbg_ok(dst >= 0 && dst < A.cap_pts, kDbgPointDst, dst, A.cap_pts)) {
                    oxy[dst] = cp;
                    oi[dst] = ci;
                }
                far2_add(fb, ord_f32(d), ci, __float_as_uint(e));
            }
            n0 += __popc(b0);
            n1 += __popc(b1);
            cp = np;
            ci = ni;
        }
        Top2 ta = far2_top2(fa), tb = far2_top2(fb);
        top2_warp(ta);
        top2_warp(tb);
        if (lane == 0) {
            Acc2 a0 = {}, a1 = {};
            a0.key1 = ta.k1;
            a0.o2 = ta.o2;
            a0.cnt = (unsigned)n0;
            a0.emax = ta.em;
            a1.key1 = tb.k1;
            a1.o2 = tb.o2;
            a1.cnt = (unsigned)n1;
            a1.emax = tb.em;
            acc[2 * sg] = a0;
            acc[2 * sg + 1] = a1;
        }
    }
    const unsigned f = __reduce_add_sync(0xffffffffu, fallbacks);
    if (lane == 0 && f) atomicAdd(&H->fallbacks, (unsigned long long)f);
}

// Output of every cloud (block 0): the hull links of all clouds ranked at
// once by pointer jumping in global memory (each cloud's cycle ends at the
// link back to its slot a_c = 2c), then per cloud the collinear filter and
// the counter-clockwise compaction from a_c into its output.
__device__ void output2d_m(const Params2M &M, SmemOut &sm)
{
    const Params2 &A = M.A;
    Hdr2 *H = A.hdr;
    const int st = *(volatile int *)&H->status;
    const int h = *(volatile int *)&H->hull_count;
    int *hc = sm.succ;         // per cloud: hull slots of its cycle
    int *hbase = sm.succ + kMaxClouds;  // per cloud: first position of its order
    if (st == 0) {
        int *sa = A.bi[0], *sb = A.bi[1];
        int *da = reinterpret_cast<int *>(A.bxy[0]), *db = reinterpret_cast<int *>(A.bxy[1]);
        for (int i = threadIdx.x; i < h; i += blockDim.x) {
            const int s = A.next[i];
            const bool end = s == 2 * M.hull_cloud[i];
            sa[i] = end ? -1 : s;
            da[i] = end ? 0 : 1;
        }
        __syncthreads();
        for (int span = 1; span < h; span <<= 1) {
            for (int i = threadIdx.x; i < h; i += blockDim.x) {
                int s = sa[i], d = da[i];
                if (s >= 0) {
                    d += da[s];
                    s = sa[s];
                }
                sb[i] = s;
                db[i] = d;
            }
            __syncthreads();
            int *t = sa;
            sa = sb;
            sb = t;
            t = da;
            da = db;
            db = t;
        }
        if (threadIdx.x == 0) {
            int b = 0;
            for (int c = 0; c < M.K; c++) {
                hc[c] = da[2 * c] + 1;  // a_c is the farthest from its cycle's end
                hbase[c] = b;
                b += hc[c];
            }
        }
        __syncthreads();
        int *order = sb;  // hbase[c] + position counter-clockwise from a_c -> slot
        for (int i = threadIdx.x; i < h; i += blockDim.x) {
            const int c = M.hull_cloud[i], hh = hc[c];
            const int rank = hh - 1 - da[i];
            order[hbase[c] + (hh - rank) % hh] = i;
        }
        __syncthreads();
        for (int c = 0; c < M.K; c++) {
            const Cloud2 &C = M.c[c];
            Hdr2 *Hc = C.hdr;
            const bool nonfinite = C.n > 0 && *(volatile int *)&Hc->nonfinite;
            long long count = 0;
            if (C.n > 0 && !nonfinite) {
                const unsigned long long kmn = *(volatile unsigned long long *)&Hc->lexmin;
                const unsigned long long kmx = *(volatile unsigned long long *)&Hc->lexmax;
                if (kmn == kmx) {
                    if (threadIdx.x == 0) C.out_idx[0] = *(volatile int *)&Hc->a_idx;
                    count = 1;
                } else {
                    const int hh = hc[c], b0 = hbase[c];
                    long long off = 0;
                    for (int q = 0; q < hh; q += blockDim.x) {
                        const int p = q + threadIdx.x;
                        long long k = 0;
                        if (p < hh) {
                            if (hh <= 2) {
                                k = 1;
                            } else {
                                const int sp = order[b0 + (p + hh - 1) % hh], sv = order[b0 + p],
                                          sx = order[b0 + (p + 1) % hh];
                                k = orient_exact_sign(A.hull_x[sp], A.hull_y[sp], A.hull_x[sv],
                                                      A.hull_y[sv], A.hull_x[sx],
                                                      A.hull_y[sx]) != 0;
                            }
                        }
                        long long cnt;
                        const long long ex = block_excl_scan64(k, sm.wsum, &cnt);
                        if (k) C.out_idx[off + ex] = A.hull_idx[order[b0 + p]];
                        off += cnt;
                    }
                    count = off;
                }
            }
            if (threadIdx.x == 0) {
                qh_result *R = C.res;
                const int cst = nonfinite ? (int)QH_ERR_NONFINITE : 0;
                R->count = cst == 0 ? count : 0;
                R->status = cst;
                R->iterations = *(volatile int *)&H->iter;
                R->survivor_total = *(volatile long long *)&H->surv_total;
                R->live_total = (long long)A.n + R->survivor_total;
                R->segments_total = *(volatile long long *)&H->seg_total;
                R->filter_fallbacks = (long long)(*(volatile unsigned long long *)&H->fallbacks +
                                                  *(volatile unsigned long long *)&Hc->fallbacks);
                R->exact_argmax = *(volatile unsigned long long *)&H->exact_argmax;
                for (int i = 0; i < 4; i++)
                    R->extra[i] = (long long)*(volatile unsigned long long *)&H->phase_ns[i];
            }
            __syncthreads();
        }
    } else if (threadIdx.x == 0) {
        for (int c = 0; c < M.K; c++) {
            qh_result *R = M.c[c].res;
            R->count = 0;
            R->status = st;
            R->iterations = *(volatile int *)&H->iter;
        }
    }
}

template <class P>
__global__ void __launch_bounds__(kBlock, kMinBlocks) qh2d_multi(Params2M M)
{
    const Params2 &A = M.A;
    SmemAll &sm = *reinterpret_cast<SmemAll *>(qh2d_dsm);
    SmemStream &sp = *reinterpret_cast<SmemStream *>(qh2d_dsm);
    __shared__ PipeBars bars;
    __shared__ Ext2 ext_m[kMaxClouds];
    unsigned ph = 0;
    if (threadIdx.x == 0) {
        for (int b = 0; b < kRing; b++) {
            mbar_init(&bars.full[b], 1);
            mbar_init(&bars.empty[b], kCW);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&bars.counted[b], kCW);
            mbar_init(&bars.bases[b], 1);
        }
        fence_mbar_init();
    }
    __syncthreads();
    Hdr2 *H = A.hdr;
    int *fail = &H->status;
    const bool clk = blockIdx.x == 0 && threadIdx.x == 0;
    unsigned long long tprev = clk ? globaltimer_ns() : 0;
    int it = 0;
    // every grid barrier returns the status as one value for the whole CTA:
    // a phase starts only when it is zero, so after a failure (an expired
    // wait, a non-finite input) no CTA reads results another CTA has not
    // finished writing
    bool hold = A.test_hold != 0 && blockIdx.x == 0;
    auto sync_as = [&](int cat) {
        const int st = grid_sync_count(&H->bar, fail, A.wait_ns, hold);
        hold = false;
        if (clk) {
            const unsigned long long t = globaltimer_ns();
            H->phase_ns[cat] += t - tprev;
            if (it < kTimeline && cat < 2) {
                H->tl[it][2 + cat] += (long long)(t - tprev);
                if (cat == 0) {
                    H->tl[it][0] = *(volatile int *)&H->L[it & 1];
                    H->tl[it][1] = *(volatile int *)&H->S[it & 1];
                }
            }
            tprev = t;
        }
        return st;
    };
    // headers: the shared one (K pseudo segments, N live points, 2K hull
    // slots) and each cloud's
    if (blockIdx.x == 0) {
        for (int c = 0; c < M.K; c++) init2d(cloud_params(M, c));
        if (threadIdx.x == 0) {
            H->S[0] = M.K;
            H->L[0] = A.n;
            H->hull_count = 2 * M.K;
        }
    }
    if (sync_as(3) == 0) {
        for (int c = 0; c < M.K; c++) {
            if (M.c[c].n == 0) continue;
            const Ext2 e = extrema2d(cloud_params(M, c), sm);
            if (threadIdx.x == 0) ext_m[c] = e;
        }
        if (sync_as(3) == 0) {
            if (threadIdx.x == 0) {
                for (int c = 0; c < M.K; c++) {
                    if (M.c[c].n == 0) continue;
                    Hdr2 *Hc = M.c[c].hdr;
                    if (ext_m[c].mn == *(volatile unsigned long long *)&Hc->lexmin)
                        atomicMin(&Hc->a_idx, ext_m[c].mni);
                    if (ext_m[c].mx == *(volatile unsigned long long *)&Hc->lexmax)
                        atomicMin(&Hc->b_idx, ext_m[c].mxi);
                }
            }
            // the first split of every finite cloud, one after the other
            // (each over the whole grid; no barrier between them)
            for (int c = 0; c < M.K; c++)
                if (cloud_live(M, c))
                    pass2d_stream<P, true>(cloud_params(M, c), 0, sp, bars, ph, blockIdx.x,
                                           gridDim.x);
            int st = sync_as(0);
            // a bounded wait that expired in a cloud's first split stops every cloud
            if (st == 0) {
                int cst = 0;
                if (threadIdx.x == 0)
                    for (int c = 0; c < M.K; c++) cst |= *(volatile int *)&M.c[c].hdr->status;
                if (__syncthreads_or(cst != 0)) {
                    if (blockIdx.x == 0 && threadIdx.x == 0) set_status(H, kStTimeout);
                    st = kStTimeout;
                }
            }
            int t = 0;
            while (st == 0) {
                if (blockIdx.x == 0) update2d_m(M, t & 1, t == 0, sm.u, 0);
                if (sync_as(1) != 0) break;
                const int nu = *(volatile int *)&H->n_uncert;
                if (nu > 0) {
                    const int per = exact_chunks2d(A, t & 1, sm.x, nu, gridDim.x);
                    exact2d_split<P>(A, t & 1, sm.x, blockIdx.x, gridDim.x, per);
                    if (sync_as(2) != 0) break;
                    if (per > 1) {
                        exact2d_merge(A, t & 1, blockIdx.x, gridDim.x, per);
                        if (sync_as(2) != 0) break;
                    }
                }
                if (*(volatile int *)&H->S[(t + 1) & 1] == 0) break;
                t++;
                if (t > A.max_iters) {
                    if (blockIdx.x == 0 && threadIdx.x == 0) set_status(H, kStNoConv);
                    break;
                }
                const int Lt = *(volatile int *)&H->L[t & 1], St = *(volatile int *)&H->S[t & 1];
                if (blockIdx.x == 0 && threadIdx.x == 0) H->iter = t;
                it = t;
                if ((long long)Lt <= (long long)kWarpSegAvg * St &&
                    *(volatile int *)&H->maxlen <= kWarpSegMax)
                    pass2d_warpseg<P>(A, t & 1, blockIdx.x, gridDim.x);
                else
                    pass2d_stream<P, false, true>(A, t & 1, sp, bars, ph, blockIdx.x, gridDim.x);
                st = sync_as(0);
            }
        }
    }
    // the output step reads the status itself and writes only the result
    // records when it is not zero
    sync_as(3);
    if (blockIdx.x == 0) output2d_m(M, sm.out);
}

// ---------------------------------------------------------------- host-loop kernels
__global__ void __launch_bounds__(kBlock) k_init2d(Params2 A) { init2d(A); }
__global__ void __launch_bounds__(kBlock) k_extrema2d(Params2 A)
{
    __shared__ SmemAll sm;
    extrema2d(A, sm);
}
template <class P, bool FIRST>
__global__ void __launch_bounds__(kBlock, kMinBlocks) k_pass2d(Params2 A, int par)
{
    __shared__ SmemAll sm;
    pass2d<P, FIRST>(A, par, sm.pass, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(kBlock) k_update2d(Params2 A, int par, int first, int iter)
{
    __shared__ SmemAll sm;
    if (threadIdx.x == 0) A.hdr->iter = iter;
    update2d(A, par, first != 0, sm.u);
}
template <class P>
__global__ void __launch_bounds__(kBlock) k_exact2d(Params2 A, int par)
{
    __shared__ SmemAll sm;
    exact2d<P>(A, par, sm.x, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(kBlock) k_output2d(Params2 A, int nonfinite_check)
{
    __shared__ SmemAll sm;
    if (nonfinite_check && A.hdr->nonfinite && threadIdx.x == 0) set_status(A.hdr, kStNonfinite);
    __syncthreads();
    output2d(A, sm.out);
}

// ---------------------------------------------------------------- large-hull output
// The output step for hulls with more than kOutCap slots (output2d reports
// QH_ERR_CAPACITY for them): the same ranking of the hull links by pointer
// jumping, with the arrays in global memory (the point buffers are free once
// the last pass is done), by one block; then the collinear filter and the
// counter-clockwise compaction from a.  A separate launch, made by the
// synchronous entry point when the first output step reported the capacity.
__global__ void __launch_bounds__(kBlock) k_output2d_big(Params2 A)
{
    __shared__ long long wsum[33];
    Hdr2 *H = A.hdr;
    qh_result *R = A.res;
    const int h = *(volatile int *)&H->hull_count;
    const unsigned long long kmn = *(volatile unsigned long long *)&H->lexmin;
    const unsigned long long kmx = *(volatile unsigned long long *)&H->lexmax;
    if (*(volatile int *)&H->status != 0 || A.n == 0 || kmn == kmx || h <= kOutCap) return;
    int *sa = A.bi[0], *sb = A.bi[1];
    int *da = reinterpret_cast<int *>(A.bxy[0]), *db = reinterpret_cast<int *>(A.bxy[1]);
    for (int i = threadIdx.x; i < h; i += blockDim.x) {
        const int s = A.next[i];
        sa[i] = (s == 0) ? -1 : s;
        da[i] = (s == 0) ? 0 : 1;
    }
    __syncthreads();
    for (int span = 1; span < h; span <<= 1) {
        for (int i = threadIdx.x; i < h; i += blockDim.x) {
            int s = sa[i], d = da[i];
            if (s >= 0) {
                d += da[s];
                s = sa[s];
            }
            sb[i] = s;
            db[i] = d;
        }
        __syncthreads();
        int *t = sa;
        sa = sb;
        sb = t;
        t = da;
        da = db;
        db = t;
    }
    int *order = sb;  // position counter-clockwise from a -> slot
    for (int i = threadIdx.x; i < h; i += blockDim.x) {
        const int rank = h - 1 - da[i];
        order[(h - rank) % h] = i;
    }
    __syncthreads();
    long long off = 0;
    for (int q = 0; q < h; q += blockDim.x) {
        const int p = q + threadIdx.x;
        long long k = 0;
        if (p < h) {
            const int sp = order[(p + h - 1) % h], sv = order[p], sx = order[(p + 1) % h];
            k = orient_exact_sign(A.hull_x[sp], A.hull_y[sp], A.hull_x[sv], A.hull_y[sv],
                                  A.hull_x[sx], A.hull_y[sx]) != 0;
        }
        long long cnt;
        const long long ex = block_excl_scan64(k, wsum, &cnt);
        if (k) A.out_idx[off + ex] = A.hull_idx[order[p]];
        off += cnt;
    }
    if (threadIdx.x == 0) {
        R->count = off;
        R->status = QH_OK;
    }
}

// ---------------------------------------------------------------- host side
struct Layout2 {
    size_t hdr, bxy[2], bi[2], seg[2], acc[2], tile_seg, tile_m, uncert, hull_idx, hull_x, hull_y,
        next, res, total;
    int cap_seg;
    int64_t np;  // entries of each point buffer
};

static size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

static Layout2 layout2d(int64_t n)
{
    Layout2 L = {};
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t r = o;
        o = align_up(o + bytes);
        return r;
    };
    size_t np = (size_t)(n > 0 ? n : 1);
    L.np = (int64_t)np;
    // live segments never exceed 2(n-2)/3: a new segment needs a live point,
    // live points and earlier apexes are disjoint, and each old segment has at
    // most two children (S_new <= min(n - 2 - A, 2A) for A earlier apexes)
    L.cap_seg = (int)(2 * np / 3 + 8);
    L.hdr = take(sizeof(Hdr2));
    L.res = take(sizeof(qh_result));
    // point buffers: 64 bytes of slack after each (the bulk copies of a tile
    // round their range out to 16-byte boundaries)
    for (int b = 0; b < 2; b++) {
        L.bxy[b] = take(np * 8 + 64);
        L.bi[b] = take(np * 4 + 64);
    }
    for (int b = 0; b < 2; b++) L.seg[b] = take((size_t)L.cap_seg * sizeof(Seg2));
    for (int b = 0; b < 2; b++) L.acc[b] = take((size_t)2 * L.cap_seg * sizeof(Acc2));
    L.tile_seg = take((np / kTile + 2) * 4);
    L.tile_m = take((np / kTile + 2) * 4);
    L.uncert = take((size_t)L.cap_seg * 4);
    L.hull_idx = take((np + 2) * 4);
    L.hull_x = take((np + 2) * 4);
    L.hull_y = take((np + 2) * 4);
    L.next = take((np + 2) * 4);
    L.total = o;
    return L;
}

static Params2 make_params(const float *x, const float *y, int64_t n, int64_t stride,
                           int32_t *out, qh_result *res, char *ws, const Layout2 &L,
                           const qh_opts &o)
{
    Params2 A = {};
    A.x = x;
    A.y = y;
    A.stride = stride;
    A.n = (int)n;
    A.out_idx = out;
    A.res = res;
    A.hdr = (Hdr2 *)(ws + L.hdr);
    for (int b = 0; b < 2; b++) {
        A.bxy[b] = (float2 *)(ws + L.bxy[b]);
        A.bi[b] = (int *)(ws + L.bi[b]);
        A.seg[b] = (Seg2 *)(ws + L.seg[b]);
        A.acc[b] = (Acc2 *)(ws + L.acc[b]);
    }
    A.tile_seg = (int *)(ws + L.tile_seg);
    A.tile_m = (int *)(ws + L.tile_m);
    A.uncert = (int *)(ws + L.uncert);
    A.hull_idx = (int *)(ws + L.hull_idx);
    A.hull_x = (float *)(ws + L.hull_x);
    A.hull_y = (float *)(ws + L.hull_y);
    A.next = (int *)(ws + L.next);
    A.max_iters = o.max_iters > 0 ? o.max_iters : n + 8;
    A.cap_seg = L.cap_seg;
    A.cap_pts = (int)L.np;
    A.cap_hull = (int)L.np + 2;
    // the first pass may bulk-copy the caller's points when they are 16-byte
    // aligned separate arrays or one interleaved xy array
    if (stride == 1 && ((uintptr_t)x & 15) == 0 && ((uintptr_t)y & 15) == 0) A.first_tma = 1;
    else if (stride == 2 && y == x + 1 && ((uintptr_t)x & 15) == 0) A.first_tma = 2;
    A.wait_ns = o.wait_ns > 0 ? o.wait_ns : 2000000000ll;
    A.test_hold = o.test_hold;
    return A;
}

template <class P>
static qh_status run2d(const Params2 &A, const qh_opts &o, cudaStream_t st)
{
    if (cudaMemsetAsync(A.hdr, 0, sizeof(Hdr2), st) != cudaSuccess) return QH_ERR_CUDA;
    int grid = 0;
    // host-driven loop: one launch per phase, live counts read back each iteration
    grid = persistent_grid((const void *)k_pass2d<P, false>, kBlock, o.blocks_per_sm);
    if (grid <= 0) return QH_ERR_CUDA;
    grid = grid > kMaxGrid ? kMaxGrid : grid;
    Hdr2 hh;
    k_init2d<<<1, kBlock, 0, st>>>(A);
    k_extrema2d<<<grid, kBlock, 0, st>>>(A);
    if (cudaMemcpyAsync(&hh, A.hdr, sizeof(Hdr2), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return QH_ERR_CUDA;
    if (hh.nonfinite) {
        k_output2d<<<1, kBlock, 0, st>>>(A, 1);
        return cudaGetLastError() == cudaSuccess ? QH_OK : QH_ERR_CUDA;
    }
    k_pass2d<P, true><<<grid, kBlock, 0, st>>>(A, 0);
    int t = 0;
    for (;;) {
        k_update2d<<<1, kBlock, 0, st>>>(A, t & 1, t == 0, t);
        if (cudaMemcpyAsync(&hh, A.hdr, sizeof(Hdr2), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return QH_ERR_CUDA;
        if (hh.status) break;
        if (hh.n_uncert > 0) k_exact2d<P><<<grid, kBlock, 0, st>>>(A, t & 1);
        if (hh.S[(t + 1) & 1] == 0) break;
        t++;
        if (t > A.max_iters) {
            int s = QH_ERR_NO_CONVERGENCE;
            cudaMemcpyAsync(&A.hdr->status, &s, sizeof(int), cudaMemcpyHostToDevice, st);
            cudaStreamSynchronize(st);
            break;
        }
        int ntiles = (hh.S[(t) & 1] > 0) ? (hh.L[t & 1] + kTile - 1) / kTile : 0;
        int g = ntiles < grid ? (ntiles > 0 ? ntiles : 1) : grid;
        k_pass2d<P, false><<<g, kBlock, 0, st>>>(A, t & 1);
    }
    k_output2d<<<1, kBlock, 0, st>>>(A, 0);
    return cudaGetLastError() == cudaSuccess ? QH_OK : QH_ERR_CUDA;
}


// ---------------------------------------------------------------- several clouds: host side
struct Layout2M {
    Layout2 L;        // shared state for N points (+ two hull slots per cloud)
    size_t chdr;      // K cloud headers
    size_t hull_cloud;
    size_t res;       // K result records (used by the synchronous entry point)
    size_t total;
};

static Layout2M layout2d_multi(int k, int64_t N)
{
    Layout2M M;
    M.L = layout2d(N + 2 * (int64_t)k);
    size_t o = M.L.total;
    M.chdr = o;
    o = align_up(o + (size_t)k * align_up(sizeof(Hdr2)));
    M.hull_cloud = o;
    o = align_up(o + (size_t)(N + 2 * (int64_t)k + 2) * 4);
    M.res = o;
    o = align_up(o + (size_t)k * sizeof(qh_result));
    M.total = o;
    return M;
}

template <class P>
static qh_status run2d_multi(const Params2M &M, const Layout2M &LM, char *ws, const qh_opts &o,
                             cudaStream_t st)
{
    if (cudaMemsetAsync(ws + LM.L.hdr, 0, sizeof(Hdr2), st) != cudaSuccess ||
        cudaMemsetAsync(ws + LM.chdr, 0, (size_t)M.K * align_up(sizeof(Hdr2)), st) != cudaSuccess)
        return QH_ERR_CUDA;
    const void *fn = (const void *)qh2d_multi<P>;
    // the attribute belongs to the current device's context: set it on every
    // call (cheap), so that a process that uses several devices gets it on each
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kPersistSmem) != cudaSuccess)
        return QH_ERR_CUDA;
    int grid = persistent_grid_smem(fn, kBlock, o.blocks_per_sm, kPersistSmem);
    if (grid <= 0) return QH_ERR_CUDA;
    grid = grid > kMaxGrid ? kMaxGrid : grid;
    if (o.max_ctas > 0 && grid > o.max_ctas) grid = o.max_ctas;
    const int first_tiles = (int)((M.A.n + kTile - 1) / kTile);
    if (grid > first_tiles) grid = first_tiles > 0 ? first_tiles : 1;
    Params2M m = M;
    void *args[] = {&m};
    const cudaError_t e =
        cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kBlock), args, kPersistSmem, st);
    return e == cudaSuccess ? QH_OK : QH_ERR_CUDA;
}

// Checks the clouds and fills the several-cloud parameters (NOMEM when the
// workspace is too small or misaligned).
static qh_status multi_params(int32_t k, const float *const *h_dx, const float *const *h_dy,
                              const int64_t *h_n, const int64_t *h_stride, int32_t *const *h_dout,
                              qh_result *d_results, void *d_ws, size_t ws_bytes,
                              const qh_opts &o, Params2M &M, Layout2M &LM, int64_t &N)
{
    if (k < 1 || k > kMaxClouds || !h_n || !d_results || !d_ws) return QH_ERR_INVALID_ARG;
    if (o.pred_mode != QH_PRED_F32 && o.pred_mode != QH_PRED_F64) return QH_ERR_INVALID_ARG;
    if (o.loop_mode != QH_LOOP_PERSISTENT) return QH_ERR_INVALID_ARG;
    N = 0;
    for (int c = 0; c < k; c++) {
        const int64_t n = h_n[c];
        const int64_t s = h_stride ? h_stride[c] : 1;
        if (n < 0 || n > QH_MAX_POINTS || s < 1) return QH_ERR_INVALID_ARG;
        if (n > 0 && (!h_dx || !h_dy || !h_dout || !h_dx[c] || !h_dy[c] || !h_dout[c]))
            return QH_ERR_INVALID_ARG;
        if ((n - 1) * s > (int64_t)1 << 40) return QH_ERR_INVALID_ARG;
        N += n;
    }
    if (N > QH_MAX_POINTS - 2 * (int64_t)k) return QH_ERR_INVALID_ARG;
    LM = layout2d_multi(k, N);
    if (ws_bytes < LM.total || ((uintptr_t)d_ws & 255)) return QH_ERR_NOMEM;
    char *ws = (char *)d_ws;
    M = Params2M{};
    M.A = make_params(nullptr, nullptr, N, 1, nullptr, nullptr, ws, LM.L, o);
    M.A.first_tma = 0;
    M.K = k;
    M.hull_cloud = (int *)(ws + LM.hull_cloud);
    int64_t off = 0;
    for (int c = 0; c < k; c++) {
        Cloud2 &C = M.c[c];
        const int64_t n = h_n[c];
        const int64_t s = h_stride ? h_stride[c] : 1;
        C.n = (int)n;
        C.stride = s;
        C.off = (int)off;
        C.x = n > 0 ? h_dx[c] : nullptr;
        C.y = n > 0 ? h_dy[c] : nullptr;
        C.out_idx = n > 0 ? h_dout[c] : nullptr;
        C.res = d_results + c;
        C.hdr = (Hdr2 *)(ws + LM.chdr + (size_t)c * align_up(sizeof(Hdr2)));
        C.first_tma = 0;
        if (n > 0) {
            if (s == 1 && ((uintptr_t)C.x & 15) == 0 && ((uintptr_t)C.y & 15) == 0)
                C.first_tma = 1;
            else if (s == 2 && C.y == C.x + 1 && ((uintptr_t)C.x & 15) == 0)
                C.first_tma = 2;
        }
        off += n;
    }
    return QH_OK;
}

}  // namespace qh

extern "C" size_t qh_workspace_bytes_2d_multi(int32_t k, const int64_t *h_n, const qh_opts *opts)
{
    (void)opts;
    if (k < 1 || k > qh::kMaxClouds || !h_n) return 0;
    int64_t N = 0;
    for (int c = 0; c < k; c++) {
        if (h_n[c] < 0 || h_n[c] > QH_MAX_POINTS) return 0;
        N += h_n[c];
    }
    if (N > QH_MAX_POINTS - 2 * qh::kMaxClouds) return 0;
    return qh::layout2d_multi(k, N).total;
}

extern "C" qh_status qh_hull2d_multi_async(int32_t k, const float *const *h_dx,
                                           const float *const *h_dy, const int64_t *h_n,
                                           const int64_t *h_stride, int32_t *const *h_dout,
                                           qh_result *d_results, void *d_ws, size_t ws_bytes,
                                           const qh_opts *opts, cudaStream_t stream)
{
    using namespace qh;
    qh_opts o;
    qh_default_opts(&o);
    if (opts) o = *opts;
    Params2M M;
    Layout2M LM;
    int64_t N = 0;
    const qh_status s = multi_params(k, h_dx, h_dy, h_n, h_stride, h_dout, d_results, d_ws,
                                     ws_bytes, o, M, LM, N);
    if (s != QH_OK) return s;
    if (N == 0)
        return cudaMemsetAsync(d_results, 0, (size_t)k * sizeof(qh_result), stream) == cudaSuccess
                   ? QH_OK
                   : QH_ERR_CUDA;
    if (o.pred_mode == QH_PRED_F32) return run2d_multi<PredF32>(M, LM, (char *)d_ws, o, stream);
    return run2d_multi<PredF64>(M, LM, (char *)d_ws, o, stream);
}

extern "C" qh_status qh_hull2d_multi(int32_t k, const float *const *h_dx, const float *const *h_dy,
                                     const int64_t *h_n, const int64_t *h_stride,
                                     int32_t *const *h_dout, int64_t *h_counts,
                                     qh_result *h_results, void *d_ws, size_t ws_bytes,
                                     const qh_opts *opts, cudaStream_t stream)
{
    using namespace qh;
    if (k < 1 || k > kMaxClouds || !h_n || !d_ws) return QH_ERR_INVALID_ARG;
    int64_t N = 0;
    for (int c = 0; c < k; c++) N += h_n[c] > 0 ? h_n[c] : 0;
    const Layout2M LM = layout2d_multi(k, N);
    if (ws_bytes < LM.total || ((uintptr_t)d_ws & 255)) return QH_ERR_NOMEM;
    qh_result *d_res = (qh_result *)((char *)d_ws + LM.res);
    qh_status s = qh_hull2d_multi_async(k, h_dx, h_dy, h_n, h_stride, h_dout, d_res, d_ws,
                                        ws_bytes, opts, stream);
    if (s != QH_OK) return s;
    qh_result r[kMaxClouds];
    if (cudaMemcpyAsync(r, d_res, (size_t)k * sizeof(qh_result), cudaMemcpyDeviceToHost, stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return QH_ERR_CUDA;
    qh_status worst = QH_OK;
    for (int c = 0; c < k; c++) {
        if (h_counts) h_counts[c] = r[c].count;
        if (h_results) h_results[c] = r[c];
        if (r[c].status != QH_OK && worst == QH_OK) worst = (qh_status)r[c].status;
    }
    return worst;
}

using namespace qh;

extern "C" size_t qh_workspace_bytes_2d(int64_t n, const qh_opts *opts)
{
    (void)opts;
    if (n < 0 || n > QH_MAX_POINTS) return 0;
    // the persistent loop runs the several-cloud kernel with one cloud
    const size_t a = layout2d(n).total, b = layout2d_multi(1, n).total;
    return a > b ? a : b;
}

extern "C" qh_status qh_hull2d_async(const float *d_x, const float *d_y, int64_t n, int64_t stride,
                                     int32_t *d_out_idx, qh_result *d_result, void *d_ws,
                                     size_t ws_bytes, const qh_opts *opts, cudaStream_t stream)
{
    qh_opts o;
    qh_default_opts(&o);
    if (opts) o = *opts;
    if (n < 0 || n > QH_MAX_POINTS || stride < 1 || !d_result || !d_ws) return QH_ERR_INVALID_ARG;
    if (n > 0 && (!d_x || !d_y || !d_out_idx)) return QH_ERR_INVALID_ARG;
    if (o.pred_mode != QH_PRED_F32 && o.pred_mode != QH_PRED_F64) return QH_ERR_INVALID_ARG;
    if (o.loop_mode != QH_LOOP_PERSISTENT && o.loop_mode != QH_LOOP_HOST) return QH_ERR_INVALID_ARG;
    if ((n - 1) * stride > (int64_t)1 << 40) return QH_ERR_INVALID_ARG;
    if (ws_bytes < qh_workspace_bytes_2d(n, &o) || ((uintptr_t)d_ws & 255)) return QH_ERR_NOMEM;
    if (n == 0)
        return cudaMemsetAsync(d_result, 0, sizeof(qh_result), stream) == cudaSuccess ? QH_OK
                                                                                     : QH_ERR_CUDA;
    if (o.loop_mode == QH_LOOP_PERSISTENT) {
        // the several-cloud persistent kernel with one cloud
        const float *xs[1] = {d_x}, *ys[1] = {d_y};
        const int64_t ns[1] = {n}, ss[1] = {stride};
        int32_t *os[1] = {d_out_idx};
        return qh_hull2d_multi_async(1, xs, ys, ns, ss, os, d_result, d_ws, ws_bytes, &o, stream);
    }
    Layout2 L = layout2d(n);
    Params2 A = make_params(d_x, d_y, n, stride, d_out_idx, d_result, (char *)d_ws, L, o);
    if (o.pred_mode == QH_PRED_F32) return run2d<PredF32>(A, o, stream);
    return run2d<PredF64>(A, o, stream);
}

// ---------------------------------------------------------------- no-alloc variant
// Scratch for qh_hull2d_noalloc: a fixed array in device memory, created when
// the module is loaded on a device and kept until the process exits.  In host
// code the array's name is a host-side stand-in, not a device address: the
// device address is looked up once per device, with that device current,
// with cudaGetSymbolAddress (set-up on the first call made on the device).
constexpr size_t kNoAllocBytes = (size_t)32 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[64];
}  // namespace

extern "C" qh_status qh_hull2d_noalloc(const float *d_x, const float *d_y, int64_t n, int64_t stride,
                                       int32_t *d_out_idx, int64_t *h_count, cudaStream_t stream)
{
    if (n < 0 || n > QH_NOALLOC_MAX_POINTS || stride < 1 || !h_count) return QH_ERR_INVALID_ARG;
    if (n > 0 && (!d_x || !d_y || !d_out_idx)) return QH_ERR_INVALID_ARG;
    if (qh_workspace_bytes_2d(n, nullptr) > kNoAllocBytes) return QH_ERR_CAPACITY;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return QH_ERR_CUDA;
    void *ws = nullptr;
    {
        std::lock_guard<std::mutex> g(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            // set-up, first call on this device: this lookup loads the
            // module there (CUDA loads modules lazily), which reserves the
            // array; a device without room for it gives NOMEM
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                (void)cudaGetLastError();
                return e == cudaErrorMemoryAllocation ? QH_ERR_NOMEM : QH_ERR_CUDA;
            }
            g_noalloc_ptr[dev] = p;
        }
        ws = g_noalloc_ptr[dev];
    }
    return qh_hull2d(d_x, d_y, n, stride, d_out_idx, h_count, nullptr, ws, kNoAllocBytes, nullptr,
                     stream);
}

extern "C" qh_status qh_debug_timeline_2d(const void *d_ws, int64_t n, int64_t *h_rows,
                                          int32_t max_rows, int32_t *h_nrows, cudaStream_t stream)
{
    if (!d_ws || !h_rows || !h_nrows || max_rows < 0 || n < 0 || n > QH_MAX_POINTS)
        return QH_ERR_INVALID_ARG;
    Layout2 L = layout2d(n);
    Hdr2 hh;
    if (cudaMemcpyAsync(&hh, (const char *)d_ws + L.hdr, sizeof(Hdr2), cudaMemcpyDeviceToHost,
                        stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return QH_ERR_CUDA;
    int rows = hh.iter + 1;
    if (rows > kTimeline) rows = kTimeline;
    if (rows > max_rows) rows = max_rows;
    for (int r = 0; r < rows; r++) {
        h_rows[5 * r + 0] = r;
        for (int c = 0; c < 4; c++) h_rows[5 * r + 1 + c] = hh.tl[r][c];
    }
    *h_nrows = rows;
    return QH_OK;
}

extern "C" qh_status qh_hull2d(const float *d_x, const float *d_y, int64_t n, int64_t stride,
                               int32_t *d_out_idx, int64_t *h_count, qh_result *h_result,
                               void *d_ws, size_t ws_bytes, const qh_opts *opts,
                               cudaStream_t stream)
{
    if (n < 0 || n > QH_MAX_POINTS || !d_ws) return QH_ERR_INVALID_ARG;
    qh_opts o;
    qh_default_opts(&o);
    if (opts) o = *opts;
    if (ws_bytes < qh_workspace_bytes_2d(n, &o) || ((uintptr_t)d_ws & 255)) return QH_ERR_NOMEM;
    const bool host_loop = o.loop_mode == QH_LOOP_HOST;
    Layout2 L = layout2d(n);
    // the result record: a slot of the workspace the chosen loop leaves free
    qh_result *d_res =
        (qh_result *)((char *)d_ws + (host_loop ? L.res : layout2d_multi(1, n).res));
    qh_status s = qh_hull2d_async(d_x, d_y, n, stride, d_out_idx, d_res, d_ws, ws_bytes, &o, stream);
    if (s != QH_OK) return s;
    qh_result r;
    if (cudaMemcpyAsync(&r, d_res, sizeof(r), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return QH_ERR_CUDA;
    if (host_loop && r.status == QH_ERR_CAPACITY && n > 0) {
        // a hull with more slots than the host loop's output step ranks: the
        // large-hull output step (it leaves other capacity errors as they are)
        const Params2 A = make_params(d_x, d_y, n, stride, d_out_idx, d_res, (char *)d_ws, L, o);
        k_output2d_big<<<1, kBlock, 0, stream>>>(A);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(&r, d_res, sizeof(r), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
            cudaStreamSynchronize(stream) != cudaSuccess)
            return QH_ERR_CUDA;
    }
    if (h_count) *h_count = r.count;
    if (h_result) *h_result = r;
    return (qh_status)r.status;
}
