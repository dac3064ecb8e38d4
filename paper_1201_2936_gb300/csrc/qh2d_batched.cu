// Batched 2D hulls: one CTA per cloud, the whole segmented Quickhull of the
// cloud inside the CTA (block barriers only), clouds taken from a queue by a
// persistent grid.  Built for batches of small and medium clouds (thousands
// of clouds of a few thousand points, whose working set stays in L2), where
// the grid-wide kernel would spend its time in grid barriers.
//
// Per cloud (Algorithm 4 of the paper, restated per CTA):
//   extrema a (lexicographic min) and b (max); the first split is the
//   generic step applied to a pseudo segment (s = e = a, apex q = b), whose
//   children are the lower edge a->b and the upper edge b->a;
//   then, while segments remain:
//     certify   each segment's farthest point from its FP32 top-2 keys, or
//               resolve it exactly (block-wide, exact comparisons);
//               link it into the hull list between the segment's ends;
//     scatter   every live point (read segment by segment from the live
//               ranges, never the holes): child 0 (s, q) if strictly outside
//               s->q, child 1 (q, e) if strictly outside q->e, else discarded
//               (flagPermute with k = 3 states, Section 4.1); child 0 fills
//               the parent's range from the left, child 1 from the right, so
//               no scan is needed to place them (compact, Section 4.2, is the
//               holes left in between); the farthest-point key of the child
//               is accumulated on the way (the distance pass of the next
//               iteration fused into this one);
//     compact   the child table (block scan over the non-empty children).
//   The hull list is walked from a, vertices collinear with their
//   neighbours dropped.
// A segment (s, e) holds the points strictly to the right of s->e
// (orient(s, e, p) < 0); their distance is orient(e, s, p) > 0.
#include <algorithm>
#include <climits>

#include "pred2.cuh"
#include "qh_common.cuh"
#include "qh_internal.h"

namespace qh {
namespace b2 {

constexpr int kBlock = 256;

struct Rec {  // a live point: coordinates, index, raw id of its segment
    float x, y;
    int idx, raw;
};

struct SegB {
    float sx, sy, qx, qy, ex, ey;
    int si, qi, ei;
    int start, len, vstart;  // physical range of its points; virtual start (live order)
    unsigned long long key1;
    unsigned o2, emax;
};
static_assert(sizeof(SegB) == 64, "SegB layout");

struct AccB {
    unsigned long long key1;
    unsigned o2, emax;
};

struct HdrB {
    int next_cloud;
    int max_iter;
    unsigned long long fallbacks, exact_argmax;
    long long live_total, surv_total, seg_total, hull_total;
};

struct ParamsB {
    const float *x, *y;
    long long stride;
    const long long *cloud_off;
    int ncloud, n;
    int32_t *out, *count, *status;
    qh_result *res;
    HdrB *hdr;
    Rec *rec[2];
    SegB *tab[2];
    AccB *acc[2];
    int *cur0, *cur1;  // child cursors per segment
    int *next, *order, *unc;
};

struct Smem {
    long long wsum[33];
    float4 pa[kBlock], pb[kBlock];
    int ia[kBlock];
    int flag, m, nunc, cloud;
    unsigned long long surv;
};

__device__ __forceinline__ float4 load_pt(const ParamsB &A, long long i)
{
    const long long o = i * A.stride;
    return make_float4(canon0(__ldg(A.x + o)), canon0(__ldg(A.y + o)), 0.0f,
                       __int_as_float((int)i));
}

__device__ __forceinline__ bool lex_less2(float4 p, float4 q)
{
    if (p.x != q.x) return p.x < q.x;
    if (p.y != q.y) return p.y < q.y;
    return __float_as_int(p.w) < __float_as_int(q.w);
}
__device__ __forceinline__ bool lex_greater2(float4 p, float4 q)
{
    if (p.x != q.x) return p.x > q.x;
    if (p.y != q.y) return p.y > q.y;
    return __float_as_int(p.w) < __float_as_int(q.w);
}

// Exact farthest point of segment S (points tab.start .. +len of buf):
// candidates whose filter value can reach the best key's lower bound, then
// exact comparisons, lowest index on ties.
template <class P>
__device__ void exact_argmax(const ParamsB &A, Smem &sm, SegB &T, const Rec *buf, int base)
{
    const float d1 = key_dist(T.key1);
    const float em = __uint_as_float(T.emax);
    const double thr = (double)d1 - 3.0 * (double)em - fabs((double)d1) * 0x1p-20;
    int best = -1;
    float bx = 0.0f, by = 0.0f;
    unsigned fb = 0;
    for (int i = threadIdx.x; i < T.len; i += blockDim.x) {
        const Rec r = buf[base + T.start + i];
        float d, e;
        orient_value<P>(T.ex, T.ey, T.sx, T.sy, r.x, r.y, d, e);
        if ((double)d + (double)e < thr) continue;
        if (best >= 0) {
            const int s = cmp_dist_exact(T.ex, T.ey, T.sx, T.sy, r.x, r.y, bx, by);
            if (!(s > 0 || (s == 0 && r.idx < best))) continue;
        }
        best = r.idx;
        bx = r.x;
        by = r.y;
    }
    (void)fb;
    sm.ia[threadIdx.x] = best;
    sm.pa[threadIdx.x] = make_float4(bx, by, 0.0f, 0.0f);
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const int oi = sm.ia[threadIdx.x + s], mi = sm.ia[threadIdx.x];
            if (oi >= 0) {
                bool take = mi < 0;
                if (!take) {
                    const float4 o = sm.pa[threadIdx.x + s], me = sm.pa[threadIdx.x];
                    const int c = cmp_dist_exact(T.ex, T.ey, T.sx, T.sy, o.x, o.y, me.x, me.y);
                    take = c > 0 || (c == 0 && oi < mi);
                }
                if (take) {
                    sm.ia[threadIdx.x] = oi;
                    sm.pa[threadIdx.x] = sm.pa[threadIdx.x + s];
                }
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        T.qi = sm.ia[0];
        T.qx = sm.pa[0].x;
        T.qy = sm.pa[0].y;
    }
    __syncthreads();
}

// One pass over the live points of the cloud: classify against their
// segment's apex, place in the child range, accumulate the child's
// farthest-point key.  FIRST: the nc input points against the pseudo
// segment; else the nc live points of the m segments of T, in their virtual
// order (segment S covers [T[S].vstart, + len), physically from T[S].start;
// the starts are staged in shared memory when they fit), so that the holes
// the discarded points left are never read.
template <class P, bool FIRST>
__device__ void scatter_pass(const ParamsB &A, Smem &sm, int lo, int nc, int m, int par,
                             const SegB *T, unsigned &fb)
{
    const Rec *src = A.rec[par];
    Rec *dst = A.rec[par ^ 1];
    AccB *acc = A.acc[par ^ 1];
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    int *vst = reinterpret_cast<int *>(sm.pa);
    constexpr int kVstCap = (int)(2 * sizeof(sm.pa) / sizeof(int));  // pa and pb
    const bool staged = m <= kVstCap;
    if (!FIRST) {
        if (staged)
            for (int i = threadIdx.x; i < m; i += blockDim.x) vst[i] = T[i].vstart;
        __syncthreads();
    }
    for (int v0 = 0; v0 < nc; v0 += blockDim.x) {
        const int v = v0 + threadIdx.x;
        int child = -1, S = 0;
        Rec r;
        float d = 0.0f, e = 0.0f;
        if (v < nc) {
            if (FIRST) {
                const float4 p = load_pt(A, lo + v);
                r.x = p.x;
                r.y = p.y;
                r.idx = lo + v;
                r.raw = 0;
            } else {
                int a = 0, b = m - 1;
                while (a < b) {
                    const int mid = (a + b + 1) >> 1;
                    if ((staged ? vst[mid] : T[mid].vstart) <= v) a = mid;
                    else b = mid - 1;
                }
                S = a;
                r = src[lo + T[S].start + (v - T[S].vstart)];
            }
            {
                const SegB &G = T[S];
                if (r.idx != G.qi) {
                    float d0, e0;
                    orient_value<P>(G.sx, G.sy, G.qx, G.qy, r.x, r.y, d0, e0);
                    if (orient_sign<P>(d0, e0, G.sx, G.sy, G.qx, G.qy, r.x, r.y, fb) < 0) {
                        child = 0;
                        d = -d0;
                        e = e0;
                    } else {
                        float d1, e1;
                        orient_value<P>(G.qx, G.qy, G.ex, G.ey, r.x, r.y, d1, e1);
                        if (orient_sign<P>(d1, e1, G.qx, G.qy, G.ex, G.ey, r.x, r.y, fb) < 0) {
                            child = 1;
                            d = -d1;
                            e = e1;
                        }
                    }
                }
            }
        }
        const int raw = child >= 0 ? 2 * S + child : -1;
        const unsigned act = __ballot_sync(0xffffffffu, child >= 0);
        if (child >= 0) {
            const unsigned grp = __match_any_sync(act, raw);
            const int leader = __ffs(grp) - 1;
            const unsigned o = ord_f32(d);
            const unsigned top_o = __reduce_max_sync(grp, o);
            const unsigned cand = (o == top_o) ? (unsigned)r.idx : 0xffffffffu;
            const unsigned top_i = __reduce_min_sync(grp, cand);
            const unsigned sec = (o == top_o && (unsigned)r.idx == top_i) ? 0u : o;
            const unsigned sec_o = __reduce_max_sync(grp, sec);
            const unsigned em = __reduce_max_sync(grp, __float_as_uint(e));
            int base = 0;
            if (lane == leader) {
                base = atomicAdd(child == 0 ? &A.cur0[S] : &A.cur1[S], __popc(grp));
                AccB &ac = acc[raw];
                const unsigned long long k1 =
                    ((unsigned long long)top_o << 32) | (0xffffffffu - top_i);
                const unsigned long long old = atomicMax(&ac.key1, k1);
                const unsigned long long lo2 = old < k1 ? old : k1;
                const unsigned lo_o = (unsigned)(lo2 >> 32);
                atomicMax(&ac.o2, lo_o > sec_o ? lo_o : sec_o);
                atomicMax(&ac.emax, em);
            }
            base = __shfl_sync(grp, base, leader) + __popc(grp & lt);
            const SegB &G = T[S];
            const int pos = child == 0 ? G.start + base : G.start + G.len - 1 - base;
            Rec w;
            w.x = r.x;
            w.y = r.y;
            w.idx = r.idx;
            w.raw = raw;
            dst[lo + pos] = w;
        }
    }
}

template <class P>
__global__ void __launch_bounds__(kBlock) qh2d_batched_kernel(ParamsB A)
{
    __shared__ Smem sm;
    HdrB *H = A.hdr;
    unsigned fb = 0;
    for (;;) {
        if (threadIdx.x == 0) sm.cloud = atomicAdd(&H->next_cloud, 1);
        __syncthreads();
        const int c = sm.cloud;
        __syncthreads();
        if (c >= A.ncloud) break;
        const int lo = (int)A.cloud_off[c], nc = (int)A.cloud_off[c + 1] - lo;
        const int tb = lo + 2 * c;   // segment tables of this cloud: nc + 2 entries
        const int rb = 2 * tb;       // raw-indexed arrays: 2 (nc + 2) entries
        SegB *tab[2] = {A.tab[0] + tb, A.tab[1] + tb};
        if (nc == 0) {
            if (threadIdx.x == 0) {
                A.count[c] = 0;
                A.status[c] = QH_OK;
            }
            continue;
        }
        // ---- extrema
        float4 mn = make_float4(INFINITY, INFINITY, 0.0f, __int_as_float(INT_MAX));
        float4 mx = make_float4(-INFINITY, -INFINITY, 0.0f, __int_as_float(INT_MAX));
        int bad = 0;
        for (int i = threadIdx.x; i < nc; i += blockDim.x) {
            const float4 p = load_pt(A, lo + i);
            bad |= !(isfinite(p.x) && isfinite(p.y));
            if (lex_less2(p, mn)) mn = p;
            if (lex_greater2(p, mx)) mx = p;
        }
        bad = __syncthreads_or(bad);
        sm.pa[threadIdx.x] = mn;
        sm.pb[threadIdx.x] = mx;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) {
                if (lex_less2(sm.pa[threadIdx.x + s], sm.pa[threadIdx.x]))
                    sm.pa[threadIdx.x] = sm.pa[threadIdx.x + s];
                if (lex_greater2(sm.pb[threadIdx.x + s], sm.pb[threadIdx.x]))
                    sm.pb[threadIdx.x] = sm.pb[threadIdx.x + s];
            }
            __syncthreads();
        }
        const float4 a = sm.pa[0], b = sm.pb[0];
        __syncthreads();
        const int ai = __float_as_int(a.w), bi = __float_as_int(b.w);
        if (bad || (a.x == b.x && a.y == b.y)) {
            if (threadIdx.x == 0) {
                A.status[c] = bad ? QH_ERR_NONFINITE : QH_OK;
                A.count[c] = bad ? 0 : 1;
                if (!bad) A.out[lo] = ai;
            }
            __syncthreads();
            continue;
        }
        // ---- the pseudo segment (s = e = a, q = b) and the first split
        if (threadIdx.x == 0) {
            sm.surv = 0;
            SegB T = {};
            T.sx = a.x;
            T.sy = a.y;
            T.ex = a.x;
            T.ey = a.y;
            T.si = T.ei = ai;
            T.qx = b.x;
            T.qy = b.y;
            T.qi = bi;
            T.start = 0;
            T.len = nc;
            tab[1][0] = T;
            A.next[ai] = bi;
            A.next[bi] = ai;
            A.cur0[tb] = 0;
            A.cur1[tb] = 0;
        }
        for (int i = threadIdx.x; i < 2; i += blockDim.x) A.acc[0][rb + i] = AccB{0ull, 0u, 0u};
        __syncthreads();
        // table parity: tab[p] holds the segments of the records in rec[p]
        // (the pseudo segment: parity 1, the input as source)
        ParamsB Ac = A;
        Ac.cur0 = A.cur0 + tb;
        Ac.cur1 = A.cur1 + tb;
        for (int q = 0; q < 2; q++) Ac.acc[q] = A.acc[q] + rb;
        scatter_pass<P, true>(Ac, sm, lo, nc, 1, 1, tab[1], fb);
        __syncthreads();
        int par = 0;  // records now in rec[0], by the segments of tab[par ^ 1]
        int m_par = 1;
        int iter = 0;
        long long segs = 0;
        for (;;) {
            // ---- compact the children of tab[par ^ 1] (m_par parents) into tab[par]
            const SegB *Tp = tab[par ^ 1];
            SegB *Tn = tab[par];
            // (segment index, virtual start) of every non-empty child: one
            // packed scan
            long long carry = 0;
            unsigned long long nsurv = 0;
            for (int base = 0; base < 2 * m_par; base += blockDim.x) {
                const int raw = base + threadIdx.x;
                int cnt = 0;
                if (raw < 2 * m_par) cnt = (raw & 1) ? Ac.cur1[raw >> 1] : Ac.cur0[raw >> 1];
                nsurv += (unsigned long long)cnt;
                long long tot;
                const long long packed = ((long long)(cnt > 0) << 32) | (long long)cnt;
                const long long exp = block_excl_scan64(packed, sm.wsum, &tot) + carry;
                const long long ex = exp >> 32;
                if (raw < 2 * m_par) {
                    if (cnt > 0) {
                        const SegB &G = Tp[raw >> 1];
                        SegB T = {};
                        if (raw & 1) {
                            T.sx = G.qx; T.sy = G.qy; T.si = G.qi;
                            T.ex = G.ex; T.ey = G.ey; T.ei = G.ei;
                            T.start = G.start + G.len - cnt;
                        } else {
                            T.sx = G.sx; T.sy = G.sy; T.si = G.si;
                            T.ex = G.qx; T.ey = G.qy; T.ei = G.qi;
                            T.start = G.start;
                        }
                        T.len = cnt;
                        T.vstart = (int)(exp & 0xffffffffll);
                        const AccB ac = Ac.acc[par][raw];
                        T.key1 = ac.key1;
                        T.o2 = ac.o2;
                        T.emax = ac.emax;
                        T.qi = -1;
                        Tn[ex] = T;
                    }
                }
                carry += tot;
            }
            const int m = (int)(carry >> 32), live = (int)(carry & 0xffffffffll);
            nsurv = __reduce_add_sync(0xffffffffu, (unsigned)nsurv);
            if ((threadIdx.x & 31) == 0 && nsurv) atomicAdd(&sm.surv, nsurv);
            __syncthreads();
            if (m == 0) break;
            iter++;
            segs += m;
            // ---- reset cursors and the other accumulator for this round's children
            for (int i = threadIdx.x; i < m; i += blockDim.x) {
                Ac.cur0[i] = 0;
                Ac.cur1[i] = 0;
            }
            for (int i = threadIdx.x; i < 2 * m; i += blockDim.x)
                Ac.acc[par ^ 1][i] = AccB{0ull, 0u, 0u};
            if (threadIdx.x == 0) sm.nunc = 0;
            __syncthreads();
            // ---- certify the farthest points
            for (int S = threadIdx.x; S < m; S += blockDim.x) {
                SegB &T = Tn[S];
                bool cert = true;
                if (T.len > 1) {
                    const double gap = ((double)key_dist(T.key1) - (double)unord_f32(T.o2)) *
                                       (1.0 - 0x1p-50);
                    cert = gap > 2.0 * (double)__uint_as_float(T.emax);
                }
                if (cert) {
                    const int qi = key_idx(T.key1);
                    const float4 q = load_pt(A, qi);
                    T.qi = qi;
                    T.qx = q.x;
                    T.qy = q.y;
                } else {
                    A.unc[tb + atomicAdd(&sm.nunc, 1)] = S;
                }
            }
            __syncthreads();
            const int nu = sm.nunc;
            for (int u = 0; u < nu; u++) exact_argmax<P>(A, sm, Tn[A.unc[tb + u]], A.rec[par], lo);
            if (threadIdx.x == 0 && nu) atomicAdd(&H->exact_argmax, (unsigned long long)nu);
            __syncthreads();
            // ---- link the apexes into the hull list
            for (int S = threadIdx.x; S < m; S += blockDim.x) {
                const SegB &T = Tn[S];
                A.next[T.si] = T.qi;
                A.next[T.qi] = T.ei;
            }
            // ---- scatter the live points into the other buffer
            __syncthreads();
            scatter_pass<P, false>(Ac, sm, lo, live, m, par, Tn, fb);
            __syncthreads();
            // children counts are in cur0/cur1 of Tn's segments; their keys in
            // acc[par ^ 1]; records in rec[par ^ 1] carry raw ids 2S + k
            par ^= 1;
            m_par = m;
            // the compaction step reads tab[par ^ 1] = Tn as parents
        }
        // ---- walk the hull list from a; drop vertices collinear with their neighbours
        int *ord = A.order + lo;
        if (threadIdx.x == 0) {
            int h = 0, v = ai;
            do {
                ord[h++] = v;
                v = A.next[v];
            } while (v != ai && h < nc);
            sm.m = (v == ai) ? h : -1;
        }
        __syncthreads();
        const int h = sm.m;
        if (h < 0) {  // a broken hull list: cannot happen
            if (threadIdx.x == 0) {
                A.status[c] = QH_ERR_CAPACITY;
                A.count[c] = 0;
            }
            __syncthreads();
            continue;
        }
        long long carry = 0;
        for (int base = 0; base < h; base += blockDim.x) {
            const int i = base + threadIdx.x;
            int keep = 0, v = 0;
            if (i < h) {
                v = ord[i];
                keep = 1;
                if (h > 2) {
                    const float4 p = load_pt(A, ord[(i + h - 1) % h]);
                    const float4 q = load_pt(A, v);
                    const float4 r = load_pt(A, ord[(i + 1) % h]);
                    keep = orient_exact_sign(p.x, p.y, q.x, q.y, r.x, r.y) != 0;
                }
            }
            long long tot;
            const long long ex = block_excl_scan64(keep, sm.wsum, &tot) + carry;
            __syncthreads();  // every thread has read ord[] of this chunk's neighbours
            if (keep) A.out[lo + ex] = v;
            carry += tot;
        }
        if (threadIdx.x == 0) {
            A.count[c] = (int)carry;
            A.status[c] = QH_OK;
            atomicMax(&H->max_iter, iter);
            atomicAdd((unsigned long long *)&H->seg_total, (unsigned long long)segs);
            atomicAdd((unsigned long long *)&H->hull_total, (unsigned long long)carry);
            atomicAdd((unsigned long long *)&H->surv_total, sm.surv);
            atomicAdd((unsigned long long *)&H->live_total, (unsigned long long)nc + sm.surv);
        }
        __syncthreads();
    }
    unsigned f = __reduce_add_sync(0xffffffffu, fb);
    if ((threadIdx.x & 31) == 0 && f) atomicAdd(&H->fallbacks, (unsigned long long)f);
}

__global__ void k_finish_b2(ParamsB A)
{
    HdrB *H = A.hdr;
    qh_result r = {};
    r.status = QH_OK;
    r.count = H->hull_total;
    r.live_total = H->live_total;
    r.survivor_total = H->surv_total;
    r.iterations = H->max_iter;
    r.segments_total = H->seg_total;
    r.filter_fallbacks = (int64_t)H->fallbacks;
    r.exact_argmax = (int64_t)H->exact_argmax;
    *A.res = r;
}

__global__ void k_check_b2(ParamsB A)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < A.ncloud; c += gridDim.x * blockDim.x) {
        const long long a = A.cloud_off[c], b = A.cloud_off[c + 1];
        if ((c == 0 && a != 0) || b < a || (c == A.ncloud - 1 && b != A.n)) A.hdr->next_cloud = INT_MAX / 2;
    }
}

__global__ void k_status_b2(ParamsB A)
{
    if (A.hdr->next_cloud >= INT_MAX / 2) {
        qh_result r = {};
        r.status = QH_ERR_INVALID_ARG;
        *A.res = r;
    }
}

static size_t au(size_t v) { return (v + 255) & ~(size_t)255; }

struct LayoutB {
    size_t hdr, rec[2], tab[2], acc[2], cur0, cur1, next, order, unc, total;
};

static LayoutB layout_b2(int64_t n, int ncloud)
{
    LayoutB L = {};
    size_t o = 0;
    auto take = [&](size_t b) {
        size_t r = o;
        o = au(o + b);
        return r;
    };
    const size_t np = (size_t)std::max<int64_t>(n, 1);
    const size_t ts = np + 2 * (size_t)ncloud;  // table entries over all clouds
    L.hdr = take(sizeof(HdrB));
    for (int p = 0; p < 2; p++) {
        L.rec[p] = take(np * sizeof(Rec));
        L.tab[p] = take(ts * sizeof(SegB));
        L.acc[p] = take(2 * ts * sizeof(AccB));
    }
    L.cur0 = take(ts * 4);
    L.cur1 = take(ts * 4);
    L.next = take(np * 4);
    L.order = take(np * 4);
    L.unc = take(ts * 4);
    L.total = o;
    return L;
}

}  // namespace b2
}  // namespace qh

using namespace qh;
using namespace qh::b2;

extern "C" size_t qh_workspace_bytes_2d_batched(int64_t n, int32_t ncloud, const qh_opts *opts)
{
    (void)opts;
    if (n < 0 || ncloud < 1 || n + 2 * (int64_t)ncloud > QH_MAX_POINTS / 2) return 0;
    return layout_b2(n, ncloud).total;
}

extern "C" qh_status qh_hull2d_batched(const float *d_x, const float *d_y, int64_t stride,
                                       const int64_t *d_cloud_off, int32_t ncloud, int64_t n,
                                       int32_t *d_out_idx, int32_t *d_cloud_count,
                                       int32_t *d_cloud_status, qh_result *d_result, void *d_ws,
                                       size_t ws_bytes, const qh_opts *opts, cudaStream_t st)
{
    qh_opts o;
    qh_default_opts(&o);
    if (opts) o = *opts;
    if (n < 1 || ncloud < 1 || n + 2 * (int64_t)ncloud > QH_MAX_POINTS / 2 || stride < 1 ||
        !d_ws || !d_cloud_off || !d_x || !d_y || !d_out_idx || !d_cloud_count ||
        !d_cloud_status || !d_result)
        return QH_ERR_INVALID_ARG;
    if (o.pred_mode != QH_PRED_F32 && o.pred_mode != QH_PRED_F64) return QH_ERR_INVALID_ARG;
    const LayoutB L = layout_b2(n, ncloud);
    if (ws_bytes < L.total || ((uintptr_t)d_ws & 255)) return QH_ERR_NOMEM;
    char *ws = (char *)d_ws;
    ParamsB A = {};
    A.x = d_x;
    A.y = d_y;
    A.stride = stride;
    A.cloud_off = (const long long *)d_cloud_off;
    A.ncloud = ncloud;
    A.n = (int)n;
    A.out = d_out_idx;
    A.count = d_cloud_count;
    A.status = d_cloud_status;
    A.res = d_result;
    A.hdr = (HdrB *)(ws + L.hdr);
    for (int p = 0; p < 2; p++) {
        A.rec[p] = (Rec *)(ws + L.rec[p]);
        A.tab[p] = (SegB *)(ws + L.tab[p]);
        A.acc[p] = (AccB *)(ws + L.acc[p]);
    }
    A.cur0 = (int *)(ws + L.cur0);
    A.cur1 = (int *)(ws + L.cur1);
    A.next = (int *)(ws + L.next);
    A.order = (int *)(ws + L.order);
    A.unc = (int *)(ws + L.unc);
    if (cudaMemsetAsync(A.hdr, 0, sizeof(HdrB), st) != cudaSuccess) return QH_ERR_CUDA;
    k_check_b2<<<std::max(1, std::min((ncloud + 255) / 256, 1024)), 256, 0, st>>>(A);
    const void *fn = o.pred_mode == QH_PRED_F32 ? (const void *)qh2d_batched_kernel<PredF32>
                                                : (const void *)qh2d_batched_kernel<PredF64>;
    int grid = persistent_grid(fn, kBlock, o.blocks_per_sm);
    if (grid <= 0) return QH_ERR_CUDA;
    grid = std::min(grid, ncloud);
    if (o.pred_mode == QH_PRED_F32)
        qh2d_batched_kernel<PredF32><<<grid, kBlock, 0, st>>>(A);
    else
        qh2d_batched_kernel<PredF64><<<grid, kBlock, 0, st>>>(A);
    k_finish_b2<<<1, 1, 0, st>>>(A);
    k_status_b2<<<1, 1, 0, st>>>(A);
    return cudaGetLastError() == cudaSuccess ? QH_OK : QH_ERR_CUDA;
}
