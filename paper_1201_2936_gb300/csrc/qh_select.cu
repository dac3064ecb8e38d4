// k-th element selection with the round loop on the device (Section 6: a
// second divide-and-conquer workload on the segmented primitives).
//
// Every round splits each live segment around its pivot (the element in the
// middle of the segment: 3 states, below / the pivot / above, as a
// flagPermute would group them) and keeps, compacted and in order, the part
// that holds the wanted rank (compact); a segment whose rank falls on the
// pivot is finished.  The order is (value bits ordered like numbers, index),
// so every rank names one element.
//
// One persistent cooperative launch runs all rounds:
//   * segments longer than kSmall live in a global array; a round is three
//     phases between grid barriers: per-tile counts around the pivots, the
//     decisions and the new layout (CTA 0: scans over segments and tiles),
//     and the stable scatter of the kept parts;
//   * a segment of at most kSmall elements (from the input, or when its kept
//     part shrinks to that size) becomes a task that one CTA finishes in
//     shared memory with the same rounds (same pivot rule, same stable
//     partition), so results and round counts equal a loop of global rounds.
// Nothing is read back between rounds; the host reads the status and the
// round count once.
#include <climits>
#include <cstdint>
#include <cstring>

#include "qh_common.cuh"
#include "qh_internal.h"

namespace qh {
namespace sel {

constexpr int kBlock = 256;
constexpr int kSmall = 4096;  // segments of at most this many elements finish in shared memory
constexpr int kT = 4096;      // elements per tile of a global round (<= kSmall + 1: a tile
                              // meets at most two segments of the global array)
constexpr int kPer = kT / kBlock;
static_assert(kT <= kSmall + 1, "a tile meets at most two global segments");
static_assert(kT % kBlock == 0, "tile rows");

struct Hdr {
    GridBarrier bar;
    int status;
    int cs[2];           // live segments of the global array, by parity
    int cn[2];           // elements of the global array, by parity
    int ntask;           // small-segment tasks queued
    int next_task;       // tasks taken
    int rounds;          // largest round count of any segment
    int pool;            // pool elements used by the tasks so far
};

// A segment finished in shared memory: its elements at src (kind 0: the
// caller's values, index = position; kind 1: the pool, explicit indices),
// the wanted rank, its number in the caller's table, rounds already made.
struct Task {
    int src, len, k, orig, kind, rounds;
};

struct Params {
    const float *vin;
    const long long *off, *kin;
    int nseg, n;
    int *out;
    Hdr *H;
    float *v[2];
    int *idx[2];
    float *pv;
    int *pidx;
    int *start[2], *kseg[2], *orig[2];
    int *below, *keep, *dbase, *dpool;
    int4 *tc;
    int *tseg;
    int2 *tbase;
    Task *task;
    long long wait_ns, max_iters;
};

__device__ __forceinline__ unsigned long long sel_key(float v, int idx)
{
    unsigned u = __float_as_uint(v);
    u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return ((unsigned long long)u << 32) | (unsigned)idx;
}

__device__ __forceinline__ void set_st(Hdr *H, int st) { atomicCAS(&H->status, 0, st); }

// last segment whose start is <= j (start[0..cs] ascending, start[0] = 0)
__device__ __forceinline__ int seg_of(const int *start, int cs, int j)
{
    int lo = 0, hi = cs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= j) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ long long block_sum64(long long v, long long *wsum)
{
    long long tot;
    block_excl_scan64(v, wsum, &tot);
    return tot;
}

struct Smem {
    long long wsum[33];
    int bc[4];
    unsigned long long buf[2][kSmall];  // small tasks: keys, ping-pong; global rounds: tile keys
};

// ---------------------------------------------------------------- set-up
// CTA 0: check the table, queue the short segments as tasks, lay out the
// long ones as the first global array (their ranks and caller numbers).
__device__ void init_table(const Params &P, Smem &sm)
{
    Hdr *H = P.H;
    long long c_small = 0, c_large = 0, c_elems = 0;
    for (int b0 = 0; b0 < P.nseg; b0 += kBlock) {
        const int c = b0 + threadIdx.x;
        long long len = 0, k = 0;
        bool ok = true;
        if (c < P.nseg) {
            const long long a = P.off[c], b = P.off[c + 1];
            len = b - a;
            k = P.kin[c];
            ok = len >= 1 && (c != 0 || a == 0) && (c != P.nseg - 1 || b == P.n) && k >= 0 &&
                 k < len && b <= P.n;
        }
        if (!ok) set_st(H, QH_ERR_INVALID_ARG);
        const bool live = c < P.nseg && ok;
        const bool small = live && len <= kSmall, large = live && !small;
        long long t1, t2, t3;
        const long long e1 = block_excl_scan64(small ? 1 : 0, sm.wsum, &t1);
        const long long e2 = block_excl_scan64(large ? 1 : 0, sm.wsum, &t2);
        const long long e3 = block_excl_scan64(large ? len : 0, sm.wsum, &t3);
        if (small) {
            Task t;
            t.src = (int)P.off[c];
            t.len = (int)len;
            t.k = (int)k;
            t.orig = c;
            t.kind = 0;
            t.rounds = 0;
            P.task[c_small + e1] = t;
        }
        if (large) {
            const int j = (int)(c_large + e2);
            P.start[0][j] = (int)(c_elems + e3);
            P.kseg[0][j] = (int)k;
            P.orig[0][j] = c;
        }
        if (c < P.nseg) P.out[c] = -1;
        c_small += t1;
        c_large += t2;
        c_elems += t3;
    }
    if (threadIdx.x == 0) {
        P.start[0][c_large] = (int)c_elems;
        H->cs[0] = (int)c_large;
        H->cn[0] = (int)c_elems;
        H->ntask = (int)c_small;
        H->next_task = 0;
        H->rounds = 0;
        H->pool = 0;
    }
}

// all CTAs: the long segments' elements into the first global array
__device__ void init_copy(const Params &P, int bid, int nb)
{
    const Hdr *H = P.H;
    const int cs = *(volatile const int *)&H->cs[0], cn = *(volatile const int *)&H->cn[0];
    for (int j = bid * kBlock + threadIdx.x; j < cn; j += nb * kBlock) {
        const int s = seg_of(P.start[0], cs, j);
        const int src = (int)P.off[P.orig[0][s]] + (j - P.start[0][s]);
        P.v[0][j] = P.vin[src];
        P.idx[0][j] = src;
    }
    for (int s = bid * kBlock + threadIdx.x; s < cs; s += nb * kBlock) P.below[s] = 0;
}

// ---------------------------------------------------------------- a global round
// The pivot key of segment s of the array of parity q.
__device__ __forceinline__ unsigned long long pivot_key(const Params &P, int q, int s)
{
    const int h = P.start[q][s], e = P.start[q][s + 1];
    const int m = h + (e - h) / 2;
    return sel_key(P.v[q][m], P.idx[q][m]);
}

// Phase A: per tile, the elements below and above the pivot of each of the
// (at most two) segments it meets; per segment the elements below it.
__device__ void round_count(const Params &P, int q, Smem &sm, int bid, int nb)
{
    const int cs = *(volatile const int *)&P.H->cs[q], cn = *(volatile const int *)&P.H->cn[q];
    const int ntiles = (cn + kT - 1) / kT;
    for (int t = bid; t < ntiles; t += nb) {
        const int a = t * kT, b = min(a + kT, cn);
        const int s0 = seg_of(P.start[q], cs, a);
        const int e0 = P.start[q][s0 + 1];
        const bool two = e0 < b;
        const unsigned long long p0 = pivot_key(P, q, s0);
        const unsigned long long p1 = two ? pivot_key(P, q, s0 + 1) : 0ull;
        int b0 = 0, a0 = 0, b1 = 0, a1 = 0;
#pragma unroll 4
        for (int r = 0; r < kPer; r++) {
            const int j = a + r * kBlock + threadIdx.x;
            if (j >= b) break;
            const unsigned long long key = sel_key(P.v[q][j], P.idx[q][j]);
            if (j < e0) {
                b0 += key < p0;
                a0 += key > p0;
            } else {
                b1 += key < p1;
                a1 += key > p1;
            }
        }
        // two packed sums: (below, above) of each segment
        const long long s_0 = block_sum64(((long long)a0 << 32) | b0, sm.wsum);
        const long long s_1 = block_sum64(((long long)a1 << 32) | b1, sm.wsum);
        if (threadIdx.x == 0) {
            const int4 r = make_int4((int)(s_0 & 0xffffffff), (int)(s_0 >> 32),
                                     (int)(s_1 & 0xffffffff), (int)(s_1 >> 32));
            P.tc[t] = r;
            P.tseg[t] = s0;
            atomicAdd(&P.below[s0], r.x);
            if (two) atomicAdd(&P.below[s0 + 1], r.z);
        }
    }
}

// Phase B (CTA 0): each segment's decision (keep the part below the pivot,
// the part above with the rank reduced, or finish on the pivot); kept parts
// longer than kSmall form the next global array, shorter ones go to the pool
// as tasks; then every tile's destination base for its (at most two) parts.
// dbase[s] = destination of the segment's kept part minus the kept elements
// of all segments before it, so that the exclusive count over tiles lands
// each tile's part at its place.
__device__ void round_decide(const Params &P, int q, int round, Smem &sm)
{
    Hdr *H = P.H;
    const int cs = *(volatile int *)&H->cs[q], cn = *(volatile int *)&H->cn[q];
    const int ntask0 = *(volatile int *)&H->ntask, pool0 = *(volatile int *)&H->pool;
    long long cG = 0, cL = 0, cLE = 0, cS = 0, cSE = 0;
    for (int b0 = 0; b0 < cs; b0 += kBlock) {
        const int s = b0 + threadIdx.x;
        int keep = -1, kept = 0, knew = 0;
        if (s < cs) {
            const int h = P.start[q][s], e = P.start[q][s + 1];
            const int bl = P.below[s], k = P.kseg[q][s];
            P.below[s] = 0;
            if (k < bl) {
                keep = 0;
                kept = bl;
                knew = k;
            } else if (k == bl) {
                P.out[P.orig[q][s]] = P.idx[q][h + (e - h) / 2];
                atomicMax(&H->rounds, round + 1);
            } else {
                keep = 2;
                kept = e - h - bl - 1;
                knew = k - bl - 1;
            }
        }
        const bool big = kept > kSmall, small = kept > 0 && !big;
        long long tG, tL, tLE, tS, tSE;
        const long long eG = block_excl_scan64(kept, sm.wsum, &tG);
        const long long eL = block_excl_scan64(big ? 1 : 0, sm.wsum, &tL);
        const long long eLE = block_excl_scan64(big ? kept : 0, sm.wsum, &tLE);
        const long long eS = block_excl_scan64(small ? 1 : 0, sm.wsum, &tS);
        const long long eSE = block_excl_scan64(small ? kept : 0, sm.wsum, &tSE);
        if (s < cs) {
            P.keep[s] = keep;
            const long long g = cG + eG;
            if (big) {
                const int j = (int)(cL + eL), st = (int)(cLE + eLE);
                P.start[q ^ 1][j] = st;
                P.kseg[q ^ 1][j] = knew;
                P.orig[q ^ 1][j] = P.orig[q][s];
                P.dbase[s] = (int)(st - g);
                P.dpool[s] = 0;
            } else if (small) {
                const int po = pool0 + (int)(cSE + eSE);
                Task t;
                t.src = po;
                t.len = kept;
                t.k = knew;
                t.orig = P.orig[q][s];
                t.kind = 1;
                t.rounds = round + 1;
                P.task[ntask0 + cS + eS] = t;
                P.dbase[s] = (int)(po - g);
                P.dpool[s] = 1;
            }
        }
        cG += tG;
        cL += tL;
        cLE += tLE;
        cS += tS;
        cSE += tSE;
    }
    __syncthreads();
    // tiles: kept elements of each part, exclusive over (tile, part)
    const int ntiles = (cn + kT - 1) / kT;
    long long cE = 0;
    for (int b0 = 0; b0 < ntiles; b0 += kBlock) {
        const int t = b0 + threadIdx.x;
        int c0 = 0, c1 = 0, s0 = 0;
        bool two = false;
        if (t < ntiles) {
            const int4 r = P.tc[t];
            s0 = P.tseg[t];
            const int k0 = P.keep[s0];
            c0 = k0 == 0 ? r.x : (k0 == 2 ? r.y : 0);
            two = s0 + 1 < cs && P.start[q][s0 + 1] < min((t + 1) * kT, cn);
            if (two) {
                const int k1 = P.keep[s0 + 1];
                c1 = k1 == 0 ? r.z : (k1 == 2 ? r.w : 0);
            }
        }
        long long tE;
        const long long eE = block_excl_scan64(c0 + c1, sm.wsum, &tE);
        if (t < ntiles) {
            const long long e = cE + eE;
            P.tbase[t] = make_int2((int)(P.dbase[s0] + e),
                                   two ? (int)(P.dbase[s0 + 1] + e + c0) : 0);
        }
        cE += tE;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        P.start[q ^ 1][cL] = (int)cLE;
        H->cs[q ^ 1] = (int)cL;
        H->cn[q ^ 1] = (int)cLE;
        H->ntask = ntask0 + (int)cS;
        H->pool = pool0 + (int)cSE;
    }
}

// Stable compaction of [0, len) into two parts by warp spans: warp w takes
// the w-th run of consecutive positions, counts its kept elements of each
// part by ballots, and after one exchange of the warps' counts writes them
// in order (emit(r, part, rank within the part)).  part(r): 0 dropped, 1 or 2.
// Returns the kept counts packed as (part 2 << 32) | part 1.
template <class Part, class Emit>
__device__ __forceinline__ long long span_compact(int len, Part part, Emit emit, long long *wsum)
{
    constexpr int nw = kBlock / 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int span = (len + nw - 1) / nw;
    const int w0 = min(warp * span, len), w1 = min(w0 + span, len);
    int n1 = 0, n2 = 0;
    for (int c = w0; c < w1; c += 32) {
        const int r = c + lane;
        const int pt = r < w1 ? part(r) : 0;
        n1 += __popc(__ballot_sync(0xffffffffu, pt == 1));
        n2 += __popc(__ballot_sync(0xffffffffu, pt == 2));
    }
    __syncthreads();
    if (lane == 0) wsum[warp] = ((long long)n2 << 32) | n1;
    __syncthreads();
    long long pre = 0, tot = 0;
#pragma unroll
    for (int i = 0; i < nw; i++) {
        const long long x = wsum[i];
        pre += i < warp ? x : 0;
        tot += x;
    }
    __syncthreads();
    int b1 = (int)(pre & 0xffffffff), b2 = (int)(pre >> 32);
    for (int c = w0; c < w1; c += 32) {
        const int r = c + lane;
        const int pt = r < w1 ? part(r) : 0;
        const unsigned m1 = __ballot_sync(0xffffffffu, pt == 1);
        const unsigned m2 = __ballot_sync(0xffffffffu, pt == 2);
        if (pt == 1) emit(r, 1, b1 + __popc(m1 & lt));
        else if (pt == 2) emit(r, 2, b2 + __popc(m2 & lt));
        b1 += __popc(m1);
        b2 += __popc(m2);
    }
    return tot;
}

// One round of a short segment by warp spans: count both parts (below and
// above the pivot) in one pass, exchange the warps' counts once, let
// decide(totals) pick the part to keep (0: none), then write that part in
// order.  Returns the totals packed as (above << 32) | below.
template <class Part, class Decide, class Emit>
__device__ __forceinline__ long long span_split(int len, Part part, Decide decide, Emit emit,
                                                long long *wsum)
{
    constexpr int nw = kBlock / 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int span = (len + nw - 1) / nw;
    const int w0 = min(warp * span, len), w1 = min(w0 + span, len);
    int n1 = 0, n2 = 0;
    for (int c = w0; c < w1; c += 32) {
        const int r = c + lane;
        const int pt = r < w1 ? part(r) : 0;
        n1 += __popc(__ballot_sync(0xffffffffu, pt == 1));
        n2 += __popc(__ballot_sync(0xffffffffu, pt == 2));
    }
    __syncthreads();
    if (lane == 0) wsum[warp] = ((long long)n2 << 32) | n1;
    __syncthreads();
    long long pre = 0, tot = 0;
#pragma unroll
    for (int i = 0; i < nw; i++) {
        const long long x = wsum[i];
        pre += i < warp ? x : 0;
        tot += x;
    }
    const int keep = decide(tot);
    if (keep == 0) return tot;
    int b = keep == 1 ? (int)(pre & 0xffffffff) : (int)(pre >> 32);
    for (int c = w0; c < w1; c += 32) {
        const int r = c + lane;
        const bool k = r < w1 && part(r) == keep;
        const unsigned m = __ballot_sync(0xffffffffu, k);
        if (k) emit(r, b + __popc(m & lt));
        b += __popc(m);
    }
    return tot;
}

// Phase C: every tile writes its kept elements, in order, to its parts'
// bases (the next global array or the pool).  The tile's keys are staged in
// shared memory and compacted by warp spans.
__device__ void round_scatter(const Params &P, int q, Smem &sm, int bid, int nb)
{
    const int cs = *(volatile const int *)&P.H->cs[q], cn = *(volatile const int *)&P.H->cn[q];
    const int ntiles = (cn + kT - 1) / kT;
    unsigned long long *keys = sm.buf[0];
    for (int t = bid; t < ntiles; t += nb) {
        const int a = t * kT, b = min(a + kT, cn), len = b - a;
        const int s0 = P.tseg[t];
        const int e0 = P.start[q][s0 + 1] - a;  // tile-relative end of the first part
        const bool two = s0 + 1 < cs && e0 < len;
        const int k0 = P.keep[s0], k1 = two ? P.keep[s0 + 1] : -1;
        const unsigned long long p0 = pivot_key(P, q, s0);
        const unsigned long long p1 = two ? pivot_key(P, q, s0 + 1) : 0ull;
        const int2 base = P.tbase[t];
        const bool pool0 = P.dpool[s0] != 0, pool1 = two && P.dpool[s0 + 1] != 0;
        __syncthreads();  // the previous tile's keys are consumed
        for (int r = threadIdx.x; r < len; r += kBlock)
            keys[r] = sel_key(P.v[q][a + r], P.idx[q][a + r]);
        __syncthreads();
        // 0: dropped, 1: kept in the first part, 2: kept in the second
        auto part = [&](int r) -> int {
            const unsigned long long key = keys[r];
            if (r < e0) return ((k0 == 0 && key < p0) || (k0 == 2 && key > p0)) ? 1 : 0;
            return ((k1 == 0 && key < p1) || (k1 == 2 && key > p1)) ? 2 : 0;
        };
        auto emit = [&](int r, int pt, int rank) {
            const unsigned long long key = keys[r];
            const float v = unord_f32((unsigned)(key >> 32));
            const int id = (int)(unsigned)key;
            const int d = (pt == 1 ? base.x : base.y) + rank;
            if (!dbg_ok(d >= 0 && d < P.n, kDbgPointDst, d, P.n)) return;
            if (pt == 1 ? pool0 : pool1) {
                P.pv[d] = v;
                P.pidx[d] = id;
            } else {
                P.v[q ^ 1][d] = v;
                P.idx[q ^ 1][d] = id;
            }
        };
        span_compact(len, part, emit, sm.wsum);
    }
}

// ---------------------------------------------------------------- short segments
// Each CTA takes tasks until none is left and finishes each in shared
// memory: keys in one buffer, the kept part compacted in order into the
// other, the same pivot rule and decision as a global round.  Bounded: every
// round drops at least the pivot.
__device__ void small_tasks(const Params &P, Smem &sm)
{
    Hdr *H = P.H;
    const int ntask = *(volatile int *)&H->ntask;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) sm.bc[0] = atomicAdd(&H->next_task, 1);
        __syncthreads();
        const int ti = sm.bc[0];
        if (ti >= ntask) break;
        const Task T = P.task[ti];
        unsigned long long *A = sm.buf[0], *B = sm.buf[1];
        int len = T.len, k = T.k, rounds = T.rounds;
        if (!dbg_ok(len >= 1 && len <= kSmall && T.src >= 0 && T.src + len <= P.n, kDbgSegIndex,
                    T.src, len))
            continue;
        if (T.kind == 0) {
            for (int r = threadIdx.x; r < len; r += kBlock)
                A[r] = sel_key(P.vin[T.src + r], T.src + r);
        } else {
            for (int r = threadIdx.x; r < len; r += kBlock)
                A[r] = sel_key(P.pv[T.src + r], P.pidx[T.src + r]);
        }
        __syncthreads();
        while (len > 0) {
            rounds++;
            const unsigned long long pk = A[len / 2];
            auto part = [&](int r) -> int { return A[r] < pk ? 1 : (A[r] > pk ? 2 : 0); };
            auto decide = [&](long long tot) -> int {
                const int below = (int)(tot & 0xffffffff);
                return k == below ? 0 : (k < below ? 1 : 2);
            };
            auto emit = [&](int r, int rank) { B[rank] = A[r]; };
            const long long tot = span_split(len, part, decide, emit, sm.wsum);
            const int below = (int)(tot & 0xffffffff), keep = decide(tot);
            if (keep == 0) {
                if (threadIdx.x == 0) {
                    P.out[T.orig] = (int)(unsigned)pk;
                    atomicMax(&H->rounds, rounds);
                }
                break;
            }
            __syncthreads();
            if (keep == 2) k -= below + 1;
            len = keep == 1 ? below : (int)(tot >> 32);
            unsigned long long *t = A;
            A = B;
            B = t;
        }
    }
}

// ---------------------------------------------------------------- the kernel
extern __shared__ __align__(16) unsigned char sel_dsm[];

__global__ void __launch_bounds__(kBlock) k_select(Params P)
{
    Smem &sm = *reinterpret_cast<Smem *>(sel_dsm);
    Hdr *H = P.H;
    const int bid = blockIdx.x, nb = gridDim.x;
    auto sync = [&]() { return grid_sync_count(&H->bar, &H->status, P.wait_ns); };
    if (bid == 0) init_table(P, sm);
    if (sync() != 0) return;
    init_copy(P, bid, nb);
    if (sync() != 0) return;
    int q = 0;
    for (long long round = 0;; round++) {
        if (*(volatile int *)&H->cs[q] == 0) break;
        if (round >= P.max_iters) {
            if (bid == 0 && threadIdx.x == 0) set_st(H, QH_ERR_NO_CONVERGENCE);
            return;
        }
        round_count(P, q, sm, bid, nb);
        if (sync() != 0) return;
        if (bid == 0) round_decide(P, q, (int)round, sm);
        if (sync() != 0) return;
        round_scatter(P, q, sm, bid, nb);
        if (sync() != 0) return;
        q ^= 1;
    }
    small_tasks(P, sm);
}

}  // namespace sel
}  // namespace qh

// ---------------------------------------------------------------- host
namespace qh {
namespace sel {

struct Layout {
    size_t hdr, v[2], idx[2], pv, pidx, start[2], kseg[2], orig[2], below, keep, dbase, dpool, tc,
        tseg, tbase, task, total;
};

static size_t au(size_t v) { return (v + 255) & ~(size_t)255; }

static Layout layout(long long n, int nseg)
{
    Layout L = {};
    size_t o = 0;
    auto take = [&](size_t b) {
        const size_t r = o;
        o = au(o + b);
        return r;
    };
    const size_t np = (size_t)(n > 0 ? n : 1), ns = (size_t)(nseg > 0 ? nseg : 1);
    const size_t nt = np / kT + 2;
    L.hdr = take(sizeof(Hdr));
    for (int b = 0; b < 2; b++) {
        L.v[b] = take(np * 4);
        L.idx[b] = take(np * 4);
    }
    L.pv = take(np * 4);
    L.pidx = take(np * 4);
    for (int b = 0; b < 2; b++) {
        L.start[b] = take((ns + 1) * 4);
        L.kseg[b] = take(ns * 4);
        L.orig[b] = take(ns * 4);
    }
    L.below = take(ns * 4);
    L.keep = take(ns * 4);
    L.dbase = take(ns * 4);
    L.dpool = take(ns * 4);
    L.tc = take(nt * sizeof(int4));
    L.tseg = take(nt * 4);
    L.tbase = take(nt * sizeof(int2));
    L.task = take(ns * sizeof(Task));
    L.total = o;
    return L;
}

}  // namespace sel

size_t select_workspace_bytes(long long n, int nseg) { return sel::layout(n, nseg).total; }

}  // namespace qh

// Persistent form (see the comment at the top of this file); the round-by-
// round host loop is qh_select_host_loop.
extern "C" qh_status qh_select(const float *d_v, const int64_t *d_seg_off, int32_t nseg, int64_t n,
                               const int64_t *d_k, int32_t *d_out_idx, int64_t *h_iters,
                               void *d_ws, size_t ws_bytes, cudaStream_t st)
{
    using namespace qh::sel;
    if (n < 1 || n > QH_MAX_POINTS / 2 || nseg < 1 || nseg > n || !d_v || !d_seg_off || !d_k ||
        !d_out_idx || !d_ws)
        return QH_ERR_INVALID_ARG;
    const Layout L = layout(n, nseg);
    if (ws_bytes < L.total || ((uintptr_t)d_ws & 255)) return QH_ERR_NOMEM;
    char *ws = (char *)d_ws;
    Params P = {};
    P.vin = d_v;
    P.off = (const long long *)d_seg_off;
    P.kin = (const long long *)d_k;
    P.nseg = nseg;
    P.n = (int)n;
    P.out = d_out_idx;
    P.H = (Hdr *)(ws + L.hdr);
    for (int b = 0; b < 2; b++) {
        P.v[b] = (float *)(ws + L.v[b]);
        P.idx[b] = (int *)(ws + L.idx[b]);
        P.start[b] = (int *)(ws + L.start[b]);
        P.kseg[b] = (int *)(ws + L.kseg[b]);
        P.orig[b] = (int *)(ws + L.orig[b]);
    }
    P.pv = (float *)(ws + L.pv);
    P.pidx = (int *)(ws + L.pidx);
    P.below = (int *)(ws + L.below);
    P.keep = (int *)(ws + L.keep);
    P.dbase = (int *)(ws + L.dbase);
    P.dpool = (int *)(ws + L.dpool);
    P.tc = (int4 *)(ws + L.tc);
    P.tseg = (int *)(ws + L.tseg);
    P.tbase = (int2 *)(ws + L.tbase);
    P.task = (Task *)(ws + L.task);
    P.wait_ns = 2000000000ll;
    P.max_iters = 4 * n + 16;
    const size_t dsm = sizeof(Smem);
    if (cudaFuncSetAttribute(k_select, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm) !=
        cudaSuccess)
        return QH_ERR_CUDA;
    const int grid = qh::persistent_grid_smem((const void *)k_select, kBlock, 0, dsm);
    if (grid <= 0) return QH_ERR_CUDA;
    if (cudaMemsetAsync(P.H, 0, sizeof(Hdr), st) != cudaSuccess) return QH_ERR_CUDA;
    void *args[] = {&P};
    if (cudaLaunchCooperativeKernel((const void *)k_select, dim3(grid), dim3(kBlock), args, dsm,
                                    st) != cudaSuccess)
        return QH_ERR_CUDA;
    Hdr h;
    if (cudaMemcpyAsync(&h, P.H, sizeof(Hdr), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return QH_ERR_CUDA;
    if (h.status != 0) return (qh_status)h.status;
    if (h_iters) *h_iters = h.rounds;
    return QH_OK;
}
