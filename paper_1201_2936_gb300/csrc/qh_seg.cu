// The paper's segmented primitives as standalone GPU operations, and a
// second divide-and-conquer workload built on them (Section 6: k-th element
// selection, where a flagPermute splits every segment around a pivot and a
// compact throws away the parts that cannot hold the wanted rank).
//
//   flagPermute (Section 4.1, Algorithm 2): every element of a segmented
//     array carries a state in [0, k); within each segment the elements are
//     regrouped by state, stably, and a head flag starts every non-empty
//     state group.
//   compact (Section 4.2, Algorithm 3): the elements with a true flag are
//     kept, in order; a segment with no kept element disappears.
//
// Both reduce to global (unsegmented) exclusive counts: with C_j(i) the
// number of elements of state j before i and h the head of i's segment, the
// destination of i is  h + sum_{j < f_i} (C_j(end) - C_j(h)) + C_{f_i}(i) - C_{f_i}(h),
// so one vector scan of the state masks (and of the head flags, which
// number the segments) replaces the per-state segmented scans of the
// listing.  Scans are reduce-then-scan over tiles (three launches).
#include <algorithm>
#include <climits>
#include <vector>

#include "qh.h"
#include "qh_internal.h"

namespace qh {
namespace seg {

constexpr int kBlock = 256;
constexpr int kTileE = 4096;        // elements per scan tile
constexpr int kMaxK = 7;            // states (the eighth counter numbers the segments)
// grid-stride kernels: four CTAs per SM of the current device
static long long seg_grid() { return 4ll * sm_count(); }

struct Cnt8 {
    int c[8];
};

__device__ __forceinline__ Cnt8 zero8()
{
    Cnt8 r;
#pragma unroll
    for (int j = 0; j < 8; j++) r.c[j] = 0;
    return r;
}

// counters of element i: c[f] = 1 (state), c[7] = head flag (element 0 is a head)
__device__ __forceinline__ Cnt8 elem8(const int32_t *f, const int32_t *s, long long i)
{
    Cnt8 r = zero8();
    int st = f ? f[i] : 0;
    st = (st < 0 || st >= kMaxK) ? 0 : st;
    r.c[st] = 1;
    r.c[7] = (i == 0 || s[i] != 0) ? 1 : 0;
    return r;
}

// block-wide exclusive scan of Cnt8 (one value per thread), total in *tot
__device__ Cnt8 block_scan8(Cnt8 v, Cnt8 *sh, Cnt8 *tot)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    Cnt8 inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const int t = __shfl_up_sync(0xffffffffu, inc.c[j], o);
            if (lane >= o) inc.c[j] += t;
        }
    }
    if (lane == 31) sh[w] = inc;
    __syncthreads();
    if (w == 0) {
        Cnt8 x = lane < nw ? sh[lane] : zero8();
        Cnt8 xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
            for (int j = 0; j < 8; j++) {
                const int t = __shfl_up_sync(0xffffffffu, xi.c[j], o);
                if (lane >= o) xi.c[j] += t;
            }
        }
        if (lane < nw) {
            Cnt8 ex;
#pragma unroll
            for (int j = 0; j < 8; j++) ex.c[j] = xi.c[j] - x.c[j];
            sh[lane] = ex;
        }
        if (lane == nw - 1) sh[32] = xi;
    }
    __syncthreads();
    Cnt8 r;
#pragma unroll
    for (int j = 0; j < 8; j++) r.c[j] = sh[w].c[j] + inc.c[j] - v.c[j];
    *tot = sh[32];
    __syncthreads();
    return r;
}

// Pass 1: per-tile totals.
__global__ void __launch_bounds__(kBlock) k_tile_tot(const int32_t *f, const int32_t *s,
                                                      long long n, Cnt8 *tt)
{
    __shared__ Cnt8 sh[33];
    const long long nt = (n + kTileE - 1) / kTileE;
    for (long long t = blockIdx.x; t < nt; t += gridDim.x) {
        Cnt8 a = zero8();
        const long long b0 = t * kTileE;
        for (int i = threadIdx.x; i < kTileE; i += blockDim.x)
            if (b0 + i < n) {
                const Cnt8 e = elem8(f, s, b0 + i);
#pragma unroll
                for (int j = 0; j < 8; j++) a.c[j] += e.c[j];
            }
        Cnt8 tot;
        block_scan8(a, sh, &tot);
        if (threadIdx.x == 0) tt[t] = tot;
    }
}

// Pass 2: exclusive scan of the tile totals (one block); tt[nt] = grand total.
__global__ void __launch_bounds__(kBlock) k_tile_scan(Cnt8 *tt, long long nt)
{
    __shared__ Cnt8 sh[33];
    Cnt8 carry = zero8();
    for (long long b = 0; b < nt; b += blockDim.x) {
        const long long i = b + threadIdx.x;
        Cnt8 v = i < nt ? tt[i] : zero8();
        Cnt8 tot;
        Cnt8 ex = block_scan8(v, sh, &tot);
        if (i < nt) {
            Cnt8 o;
#pragma unroll
            for (int j = 0; j < 8; j++) o.c[j] = carry.c[j] + ex.c[j];
            tt[i] = o;
        }
#pragma unroll
        for (int j = 0; j < 8; j++) carry.c[j] += tot.c[j];
    }
    if (threadIdx.x == 0) tt[nt] = carry;
}

// Pass 3: per element, its segment number (segid), the exclusive count of its
// own state (cown); per segment its head index and the state counts before it
// (segC[seg * 8 + j], j < 7, and segC[seg * 8 + 7] = head index).
__global__ void __launch_bounds__(kBlock) k_apply(const int32_t *f, const int32_t *s, long long n,
                                                   const Cnt8 *tt, int32_t *segid, int32_t *cown,
                                                   int32_t *segC)
{
    __shared__ Cnt8 sh[33];
    const long long nt = (n + kTileE - 1) / kTileE;
    constexpr int kPer = kTileE / kBlock;
    for (long long t = blockIdx.x; t < nt; t += gridDim.x) {
        const long long b0 = t * kTileE + (long long)threadIdx.x * kPer;
        Cnt8 e[kPer];
        Cnt8 a = zero8();
#pragma unroll
        for (int r = 0; r < kPer; r++) {
            e[r] = (b0 + r < n) ? elem8(f, s, b0 + r) : zero8();
#pragma unroll
            for (int j = 0; j < 8; j++) a.c[j] += e[r].c[j];
        }
        Cnt8 tot;
        Cnt8 ex = block_scan8(a, sh, &tot);
        Cnt8 run;
#pragma unroll
        for (int j = 0; j < 8; j++) run.c[j] = tt[t].c[j] + ex.c[j];
#pragma unroll
        for (int r = 0; r < kPer; r++) {
            const long long i = b0 + r;
            if (i < n) {
                int st = f ? f[i] : 0;
                st = (st < 0 || st >= kMaxK) ? 0 : st;
                const int sg = run.c[7] + e[r].c[7] - 1;  // segments started up to i, minus 1
                segid[i] = sg;
                cown[i] = run.c[st];
                if (e[r].c[7]) {
#pragma unroll
                    for (int j = 0; j < 7; j++) segC[(long long)sg * 8 + j] = run.c[j];
                    segC[(long long)sg * 8 + 7] = (int)i;
                }
            }
#pragma unroll
            for (int j = 0; j < 8; j++) run.c[j] += e[r].c[j];
        }
    }
}

// The segment after the last: counts at n and head index n.
__global__ void k_seg_end(const Cnt8 *tt, long long nt, long long n, int32_t *segC, int32_t *nseg)
{
    const Cnt8 T = tt[nt];
    const int ns = T.c[7];
    for (int j = 0; j < 7; j++) segC[(long long)ns * 8 + j] = T.c[j];
    segC[(long long)ns * 8 + 7] = (int)n;
    *nseg = ns;
}

// flagPermute: destinations and new head flags.
__global__ void __launch_bounds__(kBlock) k_permute(const int32_t *f, long long n, int k,
                                                     const int32_t *segid, const int32_t *cown,
                                                     const int32_t *segC, int32_t *p,
                                                     int32_t *s_new)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int sg = segid[i];
        const int st = (f[i] < 0 || f[i] >= k) ? 0 : f[i];
        const int32_t *c0 = segC + (long long)sg * 8, *c1 = segC + (long long)(sg + 1) * 8;
        const int h = c0[7], e = c1[7];
        int loc = h;
        for (int j = 0; j < st; j++) loc += c1[j] - c0[j];
        p[i] = loc + cown[i] - c0[st];
        if (i == h) {
            // old head, plus a head at every state boundary inside the segment
            s_new[h] = 1;
            int cum = 0;
            for (int j = 0; j < k - 1; j++) {
                cum += c1[j] - c0[j];
                if (h + cum < e) s_new[h + cum] = 1;
            }
        }
    }
}

// compact: destinations (exclusive count of true flags, Algorithm 3's p for
// every element) and the new heads: a segment with a kept element starts
// where its first kept element lands, which is the kept count before the
// segment.  The flags were scanned as states 0 / 1.
__global__ void __launch_bounds__(kBlock) k_compact(const int32_t *b, long long n,
                                                     const int32_t *segid, const int32_t *cown,
                                                     const int32_t *segC, int32_t *p,
                                                     int32_t *s_new)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int sg = segid[i];
        const int32_t *c0 = segC + (long long)sg * 8, *c1 = segC + (long long)(sg + 1) * 8;
        p[i] = b[i] ? cown[i] : (int)(i - cown[i]);
        if (i == c0[7] && c1[1] > c0[1]) s_new[c0[1]] = 1;
    }
}

// States must lie in [0, k): anything else is reported (and counted as 0).
__global__ void k_check_states(const int32_t *f, long long n, int k, int32_t *bad)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        if (f[i] < 0 || f[i] >= k) *bad = 1;
}

static size_t au(size_t v) { return (v + 255) & ~(size_t)255; }

struct LayoutS {
    size_t tt, segid, cown, segC, nseg, total;
};

static LayoutS layout_s(long long n)
{
    LayoutS L = {};
    size_t o = 0;
    auto take = [&](size_t b) {
        size_t r = o;
        o = au(o + b);
        return r;
    };
    const size_t np = (size_t)std::max(n, 1ll);
    const size_t nt = (np + kTileE - 1) / kTileE;
    L.tt = take((nt + 1) * sizeof(Cnt8));
    L.segid = take(np * 4);
    L.cown = take(np * 4);
    L.segC = take((np + 2) * 8 * 4);
    L.nseg = take(16);
    L.total = o;
    return L;
}

static int grid_of(long long items)
{
    return (int)std::max(1ll, std::min((items + kBlock - 1) / kBlock, seg_grid()));
}

// The scan behind both primitives: segment numbers and counts.
static void scan_states(const int32_t *f, const int32_t *s, long long n, char *ws,
                        const LayoutS &L, cudaStream_t st)
{
    const long long nt = (n + kTileE - 1) / kTileE;
    Cnt8 *tt = (Cnt8 *)(ws + L.tt);
    const int g = (int)std::max(1ll, std::min(nt, seg_grid()));
    k_tile_tot<<<g, kBlock, 0, st>>>(f, s, n, tt);
    k_tile_scan<<<1, kBlock, 0, st>>>(tt, nt);
    k_apply<<<g, kBlock, 0, st>>>(f, s, n, tt, (int32_t *)(ws + L.segid),
                                  (int32_t *)(ws + L.cown), (int32_t *)(ws + L.segC));
    k_seg_end<<<1, 1, 0, st>>>(tt, nt, n, (int32_t *)(ws + L.segC), (int32_t *)(ws + L.nseg));
}

}  // namespace seg
}  // namespace qh

// ---------------------------------------------------------------- selection
namespace qh {
namespace seg {

// Total order of the selection: the float's bit pattern ordered like the
// number (-0 before +0, NaNs at the ends), then the index.
__device__ __forceinline__ unsigned long long sel_key(float v, int idx)
{
    unsigned u = __float_as_uint(v);
    u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return ((unsigned long long)u << 32) | (unsigned)idx;
}

// states around each segment's pivot (the element in the middle of the segment):
// 0 below, 1 the pivot, 2 above
__global__ void __launch_bounds__(kBlock) k_classify(const float *v, const int32_t *idx,
                                                      long long n, const int32_t *segid,
                                                      const int32_t *segC, int32_t *f)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int sg = segid[i];
        const int h = segC[(long long)sg * 8 + 7], e = segC[(long long)(sg + 1) * 8 + 7];
        const int m = h + (e - h) / 2;
        const unsigned long long kp = sel_key(v[m], idx[m]), ki = sel_key(v[i], idx[i]);
        f[i] = ki < kp ? 0 : (ki == kp ? 1 : 2);
    }
}

// per segment: keep the part holding rank k (0 below, 2 above with k reduced)
// or finish (the pivot is the answer)
__global__ void k_decide(int nseg, const int32_t *segC, const float *v, const int32_t *idx,
                         int32_t *kseg, const int32_t *orig, int32_t *keep, int32_t *out)
{
    for (int sg = blockIdx.x * blockDim.x + threadIdx.x; sg < nseg;
         sg += gridDim.x * blockDim.x) {
        const int32_t *c0 = segC + (long long)sg * 8, *c1 = segC + (long long)(sg + 1) * 8;
        const int below = c1[0] - c0[0];
        const int kk = kseg[sg];
        if (kk < below) {
            keep[sg] = 0;
        } else if (kk == below) {
            const int h = c0[7], e = c1[7];
            out[orig[sg]] = idx[h + (e - h) / 2];
            keep[sg] = -1;
        } else {
            keep[sg] = 2;
            kseg[sg] = kk - below - 1;
        }
    }
}

// the permuted array and its compaction flags (old segment bounds stay)
__global__ void __launch_bounds__(kBlock) k_scatter_sel(const float *v, const int32_t *idx,
                                                         long long n, const int32_t *f,
                                                         const int32_t *p, const int32_t *segid,
                                                         const int32_t *keep, float *v2,
                                                         int32_t *idx2, int32_t *b2)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int d = p[i];
        v2[d] = v[i];
        idx2[d] = idx[i];
        b2[d] = f[i] == keep[segid[i]];
    }
}

__global__ void __launch_bounds__(kBlock) k_gather_sel(const float *v2, const int32_t *idx2,
                                                        long long n, const int32_t *b2,
                                                        const int32_t *pc, float *v3,
                                                        int32_t *idx3)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        if (b2[i]) {
            v3[pc[i]] = v2[i];
            idx3[pc[i]] = idx2[i];
        }
}

// surviving segments keep their order: new number = survivors before them
__global__ void k_seg_compact(int nseg, const int32_t *keep, const int32_t *kseg,
                              const int32_t *orig, int32_t *kseg2, int32_t *orig2, int32_t *ns2)
{
    // one block: ordered compaction of nseg small entries
    __shared__ int base;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    for (int b = 0; b < nseg; b += blockDim.x) {
        const int sg = b + threadIdx.x;
        const bool sv = sg < nseg && keep[sg] >= 0;
        const unsigned bal = __ballot_sync(0xffffffffu, sv);
        __shared__ int wcount[32];
        const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (lane == 0) wcount[w] = __popc(bal);
        __syncthreads();
        int pre = base;
        for (int j = 0; j < w; j++) pre += wcount[j];
        pre += __popc(bal & ((1u << lane) - 1u));
        if (sv) {
            kseg2[pre] = kseg[sg];
            orig2[pre] = orig[sg];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int t = 0;
            for (int j = 0; j < (int)(blockDim.x >> 5); j++) t += wcount[j];
            base += t;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *ns2 = base;
}

__global__ void k_sel_init(const float *vin, long long n, const long long *off, int nseg,
                           const long long *kin, float *v, int32_t *idx, int32_t *s,
                           int32_t *kseg, int32_t *orig, int32_t *out, int32_t *bad)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (long long i = t0; i < n; i += stride) {
        v[i] = vin[i];
        idx[i] = (int)i;
        s[i] = 0;
    }
    for (long long c = t0; c < nseg; c += stride) {
        const long long a = off[c], b = off[c + 1];
        if (b <= a || (c == 0 && a != 0) || (c == nseg - 1 && b != n) || kin[c] < 0 ||
            kin[c] >= b - a)
            *bad = 1;
        kseg[c] = (int)kin[c];
        orig[c] = (int)c;
        out[c] = -1;
    }
}

__global__ void k_sel_heads(const long long *off, int nseg, long long n, int32_t *s)
{
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < nseg;
         c += (long long)gridDim.x * blockDim.x)
        if (off[c] < n) s[off[c]] = 1;
}

struct LayoutSel {
    LayoutS sc;
    size_t v[2], idx[2], s[2], f, p, b2, pc, keep, kseg[2], orig[2], ns, bad, total;
};

static LayoutSel layout_sel(long long n, int nseg)
{
    LayoutSel L = {};
    L.sc = layout_s(n);
    size_t o = L.sc.total;
    auto take = [&](size_t b) {
        size_t r = o;
        o = au(o + b);
        return r;
    };
    const size_t np = (size_t)std::max(n, 1ll), ns = (size_t)std::max(nseg, 1);
    for (int q = 0; q < 2; q++) {
        L.v[q] = take(np * 4);
        L.idx[q] = take(np * 4);
        L.s[q] = take(np * 4);
        L.kseg[q] = take(ns * 4);
        L.orig[q] = take(ns * 4);
    }
    L.f = take(np * 4);
    L.p = take(np * 4);
    L.b2 = take(np * 4);
    L.pc = take(np * 4);
    L.keep = take(ns * 4);
    L.ns = take(16);
    L.bad = take(16);
    L.total = o;
    return L;
}

}  // namespace seg
}  // namespace qh

using namespace qh::seg;

extern "C" size_t qh_segmented_workspace_bytes(int64_t n, int32_t nseg)
{
    if (n < 0 || n > QH_MAX_POINTS / 2 || nseg < 0) return 0;
    return std::max(layout_sel(n, nseg).total, qh::select_workspace_bytes(n, nseg));
}

extern "C" qh_status qh_flag_permute(const int32_t *d_f, const int32_t *d_s, int64_t n, int32_t k,
                                     int32_t *d_p, int32_t *d_s_new, void *d_ws, size_t ws_bytes,
                                     cudaStream_t st)
{
    if (n < 0 || n > QH_MAX_POINTS / 2 || k < 1 || k > kMaxK || !d_ws) return QH_ERR_INVALID_ARG;
    if (n == 0) return QH_OK;
    if (!d_f || !d_s || !d_p || !d_s_new) return QH_ERR_INVALID_ARG;
    const LayoutS L = layout_s(n);
    if (ws_bytes < L.total || ((uintptr_t)d_ws & 255)) return QH_ERR_NOMEM;
    char *ws = (char *)d_ws;
    int32_t *bad = (int32_t *)(ws + L.nseg) + 1;
    if (cudaMemsetAsync(bad, 0, 4, st) != cudaSuccess ||
        cudaMemsetAsync(d_s_new, 0, (size_t)n * 4, st) != cudaSuccess)
        return QH_ERR_CUDA;
    k_check_states<<<grid_of(n), kBlock, 0, st>>>(d_f, n, k, bad);
    scan_states(d_f, d_s, n, ws, L, st);
    k_permute<<<grid_of(n), kBlock, 0, st>>>(d_f, n, k, (int32_t *)(ws + L.segid),
                                              (int32_t *)(ws + L.cown), (int32_t *)(ws + L.segC),
                                              d_p, d_s_new);
    int hbad = 0;
    if (cudaMemcpyAsync(&hbad, bad, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return QH_ERR_CUDA;
    return hbad ? QH_ERR_INVALID_ARG : QH_OK;
}

extern "C" qh_status qh_compact(const int32_t *d_b, const int32_t *d_s, int64_t n, int32_t *d_p,
                                int32_t *d_s_new, int64_t *h_n_new, void *d_ws, size_t ws_bytes,
                                cudaStream_t st)
{
    if (n < 0 || n > QH_MAX_POINTS / 2 || !d_ws || !h_n_new) return QH_ERR_INVALID_ARG;
    *h_n_new = 0;
    if (n == 0) return QH_OK;
    if (!d_b || !d_s || !d_p || !d_s_new) return QH_ERR_INVALID_ARG;
    const LayoutS L = layout_s(n);
    if (ws_bytes < L.total || ((uintptr_t)d_ws & 255)) return QH_ERR_NOMEM;
    char *ws = (char *)d_ws;
    int32_t *bad = (int32_t *)(ws + L.nseg) + 1;
    if (cudaMemsetAsync(bad, 0, 4, st) != cudaSuccess ||
        cudaMemsetAsync(d_s_new, 0, (size_t)n * 4, st) != cudaSuccess)
        return QH_ERR_CUDA;
    k_check_states<<<grid_of(n), kBlock, 0, st>>>(d_b, n, 2, bad);
    scan_states(d_b, d_s, n, ws, L, st);
    k_compact<<<grid_of(n), kBlock, 0, st>>>(d_b, n, (int32_t *)(ws + L.segid),
                                              (int32_t *)(ws + L.cown), (int32_t *)(ws + L.segC),
                                              d_p, d_s_new);
    const long long nt = (n + kTileE - 1) / kTileE;
    Cnt8 tot;
    int hbad = 0;
    if (cudaMemcpyAsync(&tot, (Cnt8 *)(ws + L.tt) + nt, sizeof(Cnt8), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(&hbad, bad, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return QH_ERR_CUDA;
    if (hbad) return QH_ERR_INVALID_ARG;
    *h_n_new = tot.c[1];
    return QH_OK;
}

// The round-by-round form: one host iteration per round, the kept count and
// segment count read back after each (Section 5's host-driven loop).
extern "C" qh_status qh_select_host_loop(const float *d_v, const int64_t *d_seg_off, int32_t nseg, int64_t n,
                               const int64_t *d_k, int32_t *d_out_idx, int64_t *h_iters,
                               void *d_ws, size_t ws_bytes, cudaStream_t st)
{
    if (n < 1 || n > QH_MAX_POINTS / 2 || nseg < 1 || nseg > n || !d_v || !d_seg_off || !d_k ||
        !d_out_idx || !d_ws)
        return QH_ERR_INVALID_ARG;
    const LayoutSel L = layout_sel(n, nseg);
    if (ws_bytes < L.total || ((uintptr_t)d_ws & 255)) return QH_ERR_NOMEM;
    char *ws = (char *)d_ws;
    auto I = [&](size_t o) { return (int32_t *)(ws + o); };
    auto F = [&](size_t o) { return (float *)(ws + o); };
    int32_t *bad = I(L.bad);
    if (cudaMemsetAsync(bad, 0, 4, st) != cudaSuccess) return QH_ERR_CUDA;
    k_sel_init<<<grid_of(n), kBlock, 0, st>>>(d_v, n, (const long long *)d_seg_off, nseg,
                                               (const long long *)d_k, F(L.v[0]), I(L.idx[0]),
                                               I(L.s[0]), I(L.kseg[0]), I(L.orig[0]), d_out_idx,
                                               bad);
    int hbad = 0;
    if (cudaMemcpyAsync(&hbad, bad, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return QH_ERR_CUDA;
    if (hbad) return QH_ERR_INVALID_ARG;
    k_sel_heads<<<grid_of(nseg), kBlock, 0, st>>>((const long long *)d_seg_off, nseg, n, I(L.s[0]));
    long long cn = n;
    int cs = nseg, q = 0;
    long long iters = 0;
    const LayoutS &S = L.sc;
    while (cn > 0 && cs > 0) {
        if (++iters > 4 * n + 16) return QH_ERR_NO_CONVERGENCE;
        // pivot states: needs the segment table of the current array
        scan_states(nullptr, I(L.s[q]), cn, ws, S, st);
        k_classify<<<grid_of(cn), kBlock, 0, st>>>(F(L.v[q]), I(L.idx[q]), cn, I(S.segid),
                                                    I(S.segC), I(L.f));
        // flagPermute (3 states) of every segment around its pivot
        scan_states(I(L.f), I(L.s[q]), cn, ws, S, st);
        if (cudaMemsetAsync(I(L.b2), 0, (size_t)cn * 4, st) != cudaSuccess) return QH_ERR_CUDA;
        k_permute<<<grid_of(cn), kBlock, 0, st>>>(I(L.f), cn, 3, I(S.segid), I(S.cown),
                                                   I(S.segC), I(L.p), I(L.pc));
        k_decide<<<grid_of(cs), kBlock, 0, st>>>(cs, I(S.segC), F(L.v[q]), I(L.idx[q]),
                                                  I(L.kseg[q]), I(L.orig[q]), I(L.keep),
                                                  d_out_idx);
        // the decision reads the pivot from the unpermuted array above; now
        // permute, flag the kept part and compact it (old segment bounds)
        k_scatter_sel<<<grid_of(cn), kBlock, 0, st>>>(F(L.v[q]), I(L.idx[q]), cn, I(L.f),
                                                       I(L.p), I(S.segid), I(L.keep),
                                                       F(L.v[q ^ 1]), I(L.idx[q ^ 1]), I(L.b2));
        if (cudaMemsetAsync(I(L.s[q ^ 1]), 0, (size_t)cn * 4, st) != cudaSuccess)
            return QH_ERR_CUDA;
        scan_states(I(L.b2), I(L.s[q]), cn, ws, S, st);
        k_compact<<<grid_of(cn), kBlock, 0, st>>>(I(L.b2), cn, I(S.segid), I(S.cown), I(S.segC),
                                                   I(L.pc), I(L.s[q ^ 1]));
        k_gather_sel<<<grid_of(cn), kBlock, 0, st>>>(F(L.v[q ^ 1]), I(L.idx[q ^ 1]), cn, I(L.b2),
                                                      I(L.pc), F(L.v[q]), I(L.idx[q]));
        k_seg_compact<<<1, 1024, 0, st>>>(cs, I(L.keep), I(L.kseg[q]), I(L.orig[q]),
                                          I(L.kseg[q ^ 1]), I(L.orig[q ^ 1]), I(L.ns));
        const long long nt = (cn + kTileE - 1) / kTileE;
        Cnt8 tot;
        int ns2 = 0;
        if (cudaMemcpyAsync(&tot, (Cnt8 *)(ws + S.tt) + nt, sizeof(Cnt8), cudaMemcpyDeviceToHost,
                            st) != cudaSuccess ||
            cudaMemcpyAsync(&ns2, I(L.ns), 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return QH_ERR_CUDA;
        // the compacted values went back to buffer q; heads to s[q ^ 1]; the
        // segment tables to kseg/orig[q ^ 1]
        cn = tot.c[1];
        cs = ns2;
        if (cudaMemcpyAsync(I(L.s[q]), I(L.s[q ^ 1]), (size_t)std::max(cn, 1ll) * 4,
                            cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(I(L.kseg[q]), I(L.kseg[q ^ 1]), (size_t)std::max(cs, 1) * 4,
                            cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(I(L.orig[q]), I(L.orig[q ^ 1]), (size_t)std::max(cs, 1) * 4,
                            cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return QH_ERR_CUDA;
    }
    if (h_iters) *h_iters = iters;
    return cudaStreamSynchronize(st) == cudaSuccess ? QH_OK : QH_ERR_CUDA;
}
