// 3D hull: workspace layout, device scan and radix sort, the output stage
// (canonical face lattice) and the C entry points.
//
// Output (reading of the paper's ch_out for 3D): the faces of the hull as
// maximal coplanar polygons, counter-clockwise seen from outside, each
// rotated to start at its smallest point index, sorted lexicographically;
// vertices that lie inside a face or on an edge are not vertices.  From the
// final triangulation:
//   1. alive facets, and for each edge whether the neighbour across it is
//      coplanar (exact orientation of the neighbour's opposite vertex);
//   2. coplanar groups by minimum-label propagation;
//   3. boundary edges of every group, sorted by (group, start vertex): each
//      group's boundary is one cycle, walked by one thread;
//   4. vertices collinear with their cycle neighbours dropped (exact), cycle
//      rotated to its smallest index;
//   5. faces sorted by (first, second) vertex — unique, since two faces that
//      start at the same vertex leave it along different edges;
//   6. vertex list = vertices of the faces, in index order.

#include <algorithm>
#include <climits>
#include <cstring>

#include "pred3.cuh"
#include "qh3d_internal.cuh"
#include "qh_internal.h"

namespace qh {
namespace d3 {

// ---------------------------------------------------------------- layout
static size_t au(size_t v) { return (v + 255) & ~(size_t)255; }

// CTAs of the grid-stride output kernels: four per SM of the current device
static long long out_grid() { return 4ll * sm_count(); }

// Facet capacity: the worst case 6 n + 4 ncloud + 64 (facets are never
// reused within a run), or the caller's max_facets clamped to
// [4 ncloud + 256, worst case].  Segment entries: one cloud needs at most
// one per facet that can hold points, plus the pseudo facet; several clouds
// keep one per point (the small-cloud route uses the visible and horizon
// pools as per-point scratch).
Layout3 layout3d(int64_t n, int ncloud, bool single, int64_t max_facets)
{
    Layout3 L = {};
    size_t o = 0;
    auto take = [&](size_t b) {
        size_t r = o;
        o = au(o + b);
        return r;
    };
    const size_t np = (size_t)(n > 0 ? n : 1);
    const size_t nc = (size_t)(ncloud > 0 ? ncloud : 1);
    L.ncloud = (int)nc;
    const size_t worst = 6 * np + 4 * nc + 64;
    size_t fcap = worst;
    if (max_facets > 0) fcap = std::min(worst, std::max((size_t)max_facets, 4 * nc + 256));
    L.fcap = (int)fcap;
    L.ecap = (int)((single ? std::min(np, fcap) : np) + nc + 64);
    const size_t fc = (size_t)L.fcap + 1;
    L.hdr = take(sizeof(Hdr3));
    L.res = take(sizeof(qh_result));
    L.fac = take(fc * sizeof(Fac3));
    L.plane = take(fc * sizeof(Plane3));
    L.acc = take(fc * sizeof(Acc3));
    L.apex = take(fc * sizeof(float4));
    for (int b = 0; b < 2; b++) L.claim[b] = take(fc * 8);
    L.cone = take((fc + nc) * sizeof(int4));  // + the clouds' pseudo facets
    L.thr = take(fc * 4);
    L.nstart = take(fc * 4);
    L.big_mark = take(fc * 4);
    L.big_v = take(fc * 4);
    L.big_h = take(fc * 4);
    for (int b = 0; b < 2; b++) L.ent[b] = take((size_t)L.ecap * sizeof(Ent3));
    for (int b = 0; b < 2; b++) {
        L.tile_ent[b] = take((np / kMinTile + 2) * 4);
        L.tile_m[b] = take((np / kMinTile + 2) * 4);
    }
    L.vn = take((size_t)L.ecap * sizeof(int2));
    L.cstate = take((size_t)L.ecap * 4);
    L.taken = take(fc * 4);
    L.vpool = take((size_t)L.ecap * kVCap * 4);
    L.npool = take((size_t)L.ecap * kNCap * 4);
    L.uncert = take((size_t)L.ecap * 4);
    for (int b = 0; b < 2; b++) L.pts[b] = take(np * sizeof(float4));
    L.code = take(np * sizeof(int2));
    L.part = take(kMaxGrid * 8);
    L.blk_a = take(kMaxGrid * sizeof(float4));
    L.blk_b = take(kMaxGrid * sizeof(float4));
    L.blk_v = take(kMaxGrid * 4);
    L.blk_i = take(kMaxGrid * 4);
    // output stage: boundary edges <= 3 per alive facet, groups <= alive facets
    const size_t ecount = 3 * fc;
    L.alive = take(fc * 4);
    L.label = take(fc * 4);
    L.cop = take(fc * 4);
    for (int b = 0; b < 2; b++) {
        L.ekey[b] = take(ecount * 8);
        L.eval[b] = take(ecount * 4);
        L.fkey[b] = take(fc * 8);
        L.fval[b] = take(fc * 4);
    }
    L.hist_blocks = (int)((ecount + kScanTile - 1) / kScanTile);
    L.hist = take((size_t)256 * L.hist_blocks * 4 + 256);
    L.hist_off = take((size_t)256 * L.hist_blocks * 8 + 256);
    L.gstart = take((fc + 1) * 8);
    L.poly = take(ecount * 4);
    L.glen = take(fc * 4);
    L.vflag = take((np + 1) * 8);
    L.scan_tmp = take(((256 * (size_t)L.hist_blocks + ecount + np) / kScanTile + 64) * 8);
    L.total = o;
    return L;
}

Params3 make_params3(const float *x, const float *y, const float *z, int64_t n, int64_t stride,
                     char *ws, const Layout3 &L, const qh_opts &o)
{
    Params3 A = {};
    A.x = x;
    A.y = y;
    A.z = z;
    A.stride = stride;
    A.n = (int)n;
    A.fcap = L.fcap;
    A.ecap = L.ecap;
    A.ncloud = 1;
    A.hdr = (Hdr3 *)(ws + L.hdr);
    A.res = (qh_result *)(ws + L.res);
    A.fac = (Fac3 *)(ws + L.fac);
    A.plane = (Plane3 *)(ws + L.plane);
    A.acc = (Acc3 *)(ws + L.acc);
    A.apex = (float4 *)(ws + L.apex);
    for (int b = 0; b < 2; b++) A.claim[b] = (unsigned long long *)(ws + L.claim[b]);
    A.cone = (int4 *)(ws + L.cone);
    A.thr = (float *)(ws + L.thr);
    A.nstart = (int *)(ws + L.nstart);
    A.big_mark = (int *)(ws + L.big_mark);
    A.big_v = (int *)(ws + L.big_v);
    A.big_h = (int *)(ws + L.big_h);
    for (int b = 0; b < 2; b++) {
        A.ent[b] = (Ent3 *)(ws + L.ent[b]);
        A.pts[b] = (float4 *)(ws + L.pts[b]);
    }
    for (int b = 0; b < 2; b++) {
        A.tile_ent[b] = (int *)(ws + L.tile_ent[b]);
        A.tile_m[b] = (int *)(ws + L.tile_m[b]);
    }
    A.vn = (int2 *)(ws + L.vn);
    A.cstate = (int *)(ws + L.cstate);
    A.taken = (int *)(ws + L.taken);
    A.vpool = (int *)(ws + L.vpool);
    A.npool = (int *)(ws + L.npool);
    A.uncert = (int *)(ws + L.uncert);
    A.code = (int2 *)(ws + L.code);
    A.part = (long long *)(ws + L.part);
    A.blk_a = (float4 *)(ws + L.blk_a);
    A.blk_b = (float4 *)(ws + L.blk_b);
    A.blk_v = (float *)(ws + L.blk_v);
    A.blk_i = (int *)(ws + L.blk_i);
    A.max_iters = o.max_iters > 0 ? o.max_iters : 4 * n + 16;
    A.wait_ns = o.wait_ns > 0 ? o.wait_ns : 2000000000ll;
    A.test_hold = o.test_hold;
    A.small_cloud = o.small_cloud;
    // the first polytope pays off with the FP32 filter; with FP64 plane
    // tests its larger first assignment costs more than the iterations save
    A.init_dirs = o.pred_mode == QH_PRED_F32 ? kInitDirs : 0;
    const int block = o.block > 0 ? o.block : (o.pred_mode == QH_PRED_F64 ? kDefBlockF64 : kDefBlockF32);
    const int items = o.items > 0 ? o.items : kDefItems;
    A.tile = block * items;
    return A;
}

// ---------------------------------------------------------------- device scan
// Every size below is read on the device (a pointer to an int count, or a
// fixed count when the pointer is null), so the output stage runs without
// host round trips and can be captured in a CUDA graph.  Kernels stride
// over tiles of kScanTile elements with a bounded grid.
__device__ __forceinline__ int dev_count(const int *m_ptr, int m_fix)
{
    return m_ptr ? *(volatile const int *)m_ptr : m_fix;
}

// Exclusive scan of m int counts into long long offsets (3 kernels).
__global__ void __launch_bounds__(256) k_scan_sums(const int *in, const int *m_ptr, int m_fix,
                                                    long long *bsum)
{
    __shared__ long long ws[33];
    const int m = dev_count(m_ptr, m_fix);
    const int nt = (m + kScanTile - 1) / kScanTile;
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        const int b0 = t * kScanTile;
        long long s = 0;
        for (int i = threadIdx.x; i < kScanTile; i += blockDim.x)
            if (b0 + i < m) s += in[b0 + i];
        long long tot;
        block_excl_scan64(s, ws, &tot);
        if (threadIdx.x == 0) bsum[t] = tot;
    }
}

__global__ void __launch_bounds__(256) k_scan_top(long long *bsum, const int *m_ptr, int m_fix,
                                                   long long *total)
{
    __shared__ long long ws[33];
    const int m = dev_count(m_ptr, m_fix);
    const int nb = (m + kScanTile - 1) / kScanTile;
    long long carry = 0;
    for (int base = 0; base < nb; base += blockDim.x) {
        const int i = base + threadIdx.x;
        long long v = i < nb ? bsum[i] : 0;
        long long tot;
        long long ex = block_excl_scan64(v, ws, &tot);
        if (i < nb) bsum[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void __launch_bounds__(256) k_scan_apply(const int *in, const int *m_ptr, int m_fix,
                                                     const long long *bsum, long long *out)
{
    __shared__ long long ws[33];
    const int m = dev_count(m_ptr, m_fix);
    const int nt = (m + kScanTile - 1) / kScanTile;
    constexpr int kPer = kScanTile / 256;
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        const int b0 = t * kScanTile;
        long long v[kPer];
        long long s = 0;
#pragma unroll
        for (int r = 0; r < kPer; r++) {
            const int i = b0 + threadIdx.x * kPer + r;
            v[r] = i < m ? in[i] : 0;
            s += v[r];
        }
        long long tot;
        long long ex = block_excl_scan64(s, ws, &tot) + bsum[t];
#pragma unroll
        for (int r = 0; r < kPer; r++) {
            const int i = b0 + threadIdx.x * kPer + r;
            if (i < m) out[i] = ex;
            ex += v[r];
        }
    }
}

static int grid_for(long long items, int block)
{
    const long long g = (items + block - 1) / block;
    return (int)std::max(1ll, std::min(g, out_grid()));
}

static int tiles_grid(long long cap)
{
    const long long t = (cap + kScanTile - 1) / kScanTile;
    return (int)std::max(1ll, std::min(t, out_grid()));
}

// m_cap: an upper bound of the count (sizes the grid).
void scan_counts(const int *in, const int *m_ptr, int m_fix, long long m_cap,
                        long long *out, long long *tmp, long long *d_total, cudaStream_t st)
{
    const int g = tiles_grid(m_cap);
    k_scan_sums<<<g, 256, 0, st>>>(in, m_ptr, m_fix, tmp);
    k_scan_top<<<1, 256, 0, st>>>(tmp, m_ptr, m_fix, d_total);
    k_scan_apply<<<g, 256, 0, st>>>(in, m_ptr, m_fix, tmp, out);
}

// ---------------------------------------------------------------- radix sort
// Stable LSD radix sort of (u64 key, int value) pairs, 8-bit digits; the
// histogram of tile t for digit d sits at d * ntiles + t.
__global__ void __launch_bounds__(256) k_rs_hist(const unsigned long long *key, const int *m_ptr,
                                                  int shift, int *hist, int *hist_m)
{
    __shared__ int h[256];
    const int m = *(volatile const int *)m_ptr;
    const int nt = (m + kScanTile - 1) / kScanTile;
    if (blockIdx.x == 0 && threadIdx.x == 0) *hist_m = 256 * nt;
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        h[threadIdx.x] = 0;
        __syncthreads();
        const int b0 = t * kScanTile;
        for (int i = threadIdx.x; i < kScanTile; i += blockDim.x)
            if (b0 + i < m) atomicAdd(&h[(key[b0 + i] >> shift) & 255], 1);
        __syncthreads();
        hist[threadIdx.x * nt + t] = h[threadIdx.x];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) k_rs_scatter(const unsigned long long *key, const int *val,
                                                     const int *m_ptr, int shift,
                                                     const long long *off,
                                                     unsigned long long *okey, int *oval)
{
    __shared__ long long run[256];
    __shared__ int cnt[8][256];
    const int m = *(volatile const int *)m_ptr;
    const int nt = (m + kScanTile - 1) / kScanTile;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        __syncthreads();
        run[threadIdx.x] = off[threadIdx.x * nt + t];
        const int b0 = t * kScanTile;
        for (int sub = 0; sub < kScanTile; sub += 256) {
            for (int w = 0; w < 8; w++) cnt[w][threadIdx.x] = 0;
            __syncthreads();
            const int i = b0 + sub + threadIdx.x;
            const bool valid = i < m;
            unsigned long long k = valid ? key[i] : 0ull;
            const int d = valid ? (int)((k >> shift) & 255) : 256;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            const int wrank = __popc(peers & ((1u << lane) - 1u));
            if (valid && wrank == 0) cnt[warp][d] = __popc(peers);
            __syncthreads();
            if (valid) {
                long long pre = 0;
                for (int w = 0; w < warp; w++) pre += cnt[w][d];
                const long long dst = run[d] + pre + wrank;
                okey[dst] = k;
                oval[dst] = val[i];
            }
            __syncthreads();
            long long add = 0;
            for (int w = 0; w < 8; w++) add += cnt[w][threadIdx.x];
            run[threadIdx.x] += add;
            __syncthreads();
        }
    }
}

// Sorts keys/vals in place (ping-pong through tkey/tval); bits: key bits to
// sort; the count is *m_ptr (at most m_cap).
void radix_sort(unsigned long long *key, int *val, unsigned long long *tkey, int *tval,
                       const int *m_ptr, long long m_cap, int bits, int *hist, long long *hist_off,
                       long long *tmp, int *hist_m, cudaStream_t st)
{
    const int g = tiles_grid(m_cap);
    const long long hcap = 256 * ((m_cap + kScanTile - 1) / kScanTile);
    int passes = (bits + 7) / 8;
    if (passes & 1) passes++;  // even: the result ends in key/val
    for (int p = 0; p < passes; p++) {
        const int shift = 8 * p;
        unsigned long long *ik = (p & 1) ? tkey : key, *ok = (p & 1) ? key : tkey;
        int *iv = (p & 1) ? tval : val, *ov = (p & 1) ? val : tval;
        k_rs_hist<<<g, 256, 0, st>>>(ik, m_ptr, shift, hist, hist_m);
        scan_counts(hist, hist_m, 0, hcap, hist_off, tmp, nullptr, st);
        k_rs_scatter<<<g, 256, 0, st>>>(ik, iv, m_ptr, shift, hist_off, ok, ov);
    }
}

// ---------------------------------------------------------------- output kernels
struct OutBufs {
    int *alive, *label, *cop, *eval[2], *fval[2], *glen, *poly, *hist, *vflag;
    unsigned long long *ekey[2], *fkey[2];
    long long *gstart, *scan_tmp, *hist_off;
};

__device__ __forceinline__ void point_xyz(const Params3 &A, int i, float *p)
{
    const long long o = (long long)i * A.stride;
    p[0] = __ldg(A.x + o);
    p[1] = __ldg(A.y + o);
    p[2] = __ldg(A.z + o);
}

__device__ __forceinline__ void out_fail(Hdr3 *H, int st) { atomicCAS(&H->status, 0, st); }

__global__ void __launch_bounds__(256) k_alive(Params3 A, OutBufs O)
{
    Hdr3 *H = A.hdr;
    if (*(volatile int *)&H->status) return;
    const int fc = H->fcount;
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < fc; f += gridDim.x * blockDim.x) {
        const Fac3 F = A.fac[f];
        if (!F.alive) continue;
        O.alive[atomicAdd(&H->nalive, 1)] = f;
        O.label[f] = f;
        int bits = 0;
        for (int k = 0; k < 3; k++) {
            const Fac3 &G = A.fac[F.nb[k]];
            int opp = 0;
            for (int g = 0; g < 3; g++)
                if (G.v[g] != F.v[k] && G.v[g] != F.v[(k + 1) % 3]) opp = g;
            const float *q = G.p + 3 * opp;
            if (orient3d_exact_sign(F.p, F.p + 3, F.p + 6, q) == 0) bits |= 1 << k;
        }
        O.cop[f] = bits;
        if (bits) atomicAdd(&H->ncop, 1);
    }
}

// Coplanar groups by a concurrent union-find over the alive facets: a root
// is hooked under the smaller root (compare-and-swap), so every group ends
// with its smallest facet id as root whatever the order of the unions.
// Parents only move to ancestors, so the lock-free finds stay valid.
__device__ __forceinline__ int uf_find(int *par, int x)
{
    int p = *(volatile int *)&par[x];
    for (int guard = 0; p != x && guard < (1 << 26); guard++) {
        const int gp = *(volatile int *)&par[p];
        if (gp != p) par[x] = gp;  // path halving
        x = p;
        p = gp;
    }
    return x;
}

__global__ void __launch_bounds__(256) k_uf_union(Params3 A, OutBufs O)
{
    Hdr3 *H = A.hdr;
    if (*(volatile int *)&H->status) return;
    const int na = H->nalive;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < na; i += gridDim.x * blockDim.x) {
        const int f = O.alive[i];
        const int bits = O.cop[f];
        for (int k = 0; k < 3; k++) {
            if (!(bits & (1 << k))) continue;
            int a = f, b = A.fac[f].nb[k];
            int guard = 0;
            for (; guard < (1 << 20); guard++) {
                a = uf_find(O.label, a);
                b = uf_find(O.label, b);
                if (a == b) break;
                if (a < b) {
                    const int t = a;
                    a = b;
                    b = t;
                }
                if (atomicCAS(&O.label[a], a, b) == a) break;
            }
            if (guard == (1 << 20)) H->uf_fail = 1;
        }
    }
}

__global__ void __launch_bounds__(256) k_uf_compress(Params3 A, OutBufs O)
{
    Hdr3 *H = A.hdr;
    if (*(volatile int *)&H->status) return;
    if (H->uf_fail) {
        if (blockIdx.x == 0 && threadIdx.x == 0) out_fail(H, QH_ERR_CAPACITY);
        return;
    }
    const int na = H->nalive;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < na; i += gridDim.x * blockDim.x) {
        const int f = O.alive[i];
        if (O.cop[f]) O.label[f] = uf_find(O.label, f);
    }
}

__global__ void __launch_bounds__(256) k_bedges(Params3 A, OutBufs O)
{
    Hdr3 *H = A.hdr;
    if (*(volatile int *)&H->status) return;
    const int na = H->nalive;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < na; i += gridDim.x * blockDim.x) {
        const int f = O.alive[i];
        const int bits = O.cop[f];
        const Fac3 &F = A.fac[f];
        const int lab = O.label[f];
        for (int k = 0; k < 3; k++) {
            if (bits & (1 << k)) continue;
            const int slot = atomicAdd(&H->nbedge, 1);
            O.ekey[0][slot] = ((unsigned long long)(unsigned)lab << 32) | (unsigned)F.v[k];
            O.eval[0][slot] = F.v[(k + 1) % 3];
        }
    }
}

__global__ void __launch_bounds__(256) k_gmark(Params3 A, OutBufs O)
{
    const int ne = A.hdr->nbedge;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ne; i += gridDim.x * blockDim.x) {
        const bool st = i == 0 || (O.ekey[0][i] >> 32) != (O.ekey[0][i - 1] >> 32);
        O.poly[i] = st ? 1 : 0;  // poly doubles as the start-flag array here
    }
}

__global__ void __launch_bounds__(256) k_gwrite(Params3 A, OutBufs O, const long long *gidx)
{
    Hdr3 *H = A.hdr;
    const int ne = H->nbedge;
    if (ne == 0 && blockIdx.x == 0 && threadIdx.x == 0) {
        H->ngroup = 0;
        O.gstart[0] = 0;
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ne; i += gridDim.x * blockDim.x) {
        if (O.poly[i]) O.gstart[gidx[i]] = i;
        if (i == ne - 1) {
            const int ng = (int)gidx[i] + O.poly[i];
            H->ngroup = ng;
            O.gstart[ng] = ne;
            // a polytope has at most 2n - 4 faces
            if ((long long)ng > 2ll * A.n) out_fail(H, QH_ERR_CAPACITY);
        }
    }
}

__device__ __forceinline__ bool collinear3(const float *a, const float *b, const float *c)
{
    for (int k = 0; k < 3; k++) {
        const int i = k, j = (k + 1) % 3;
        if (orient_exact_sign(a[i], a[j], b[i], b[j], c[i], c[j]) != 0) return false;
    }
    return true;
}

// One thread per group: walk its boundary cycle from the smallest start
// vertex, drop vertices collinear with their neighbours, rotate to the
// smallest index.  The polygon is written into poly[gstart .. gstart+len).
__global__ void __launch_bounds__(128) k_walk(Params3 A, OutBufs O)
{
    Hdr3 *H = A.hdr;
    if (*(volatile int *)&H->status) return;
    const int ng = H->ngroup;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x) {
        const int s = (int)O.gstart[g], e = (int)O.gstart[g + 1];
        const int len = e - s;
        int *cyc = O.poly + s;            // cycle, then the kept vertices
        int *tmp = O.eval[1] + s;         // scratch of the same size
        const unsigned long long *key = O.ekey[0] + s;
        const int *nxt = O.eval[0] + s;
        int cur = (int)(unsigned)(key[0] & 0xffffffffu);
        const int first = cur;
        int got = 0;
        for (int step = 0; step < len; step++) {
            tmp[step] = cur;
            got++;
            int lo = 0, hi = len - 1;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if ((int)(unsigned)(key[mid] & 0xffffffffu) < cur) lo = mid + 1;
                else hi = mid;
            }
            cur = nxt[lo];
            if (cur == first) break;
        }
        int m = 0;
        for (int j = 0; j < got; j++) {
            float pp[3], pv[3], pn[3];
            point_xyz(A, tmp[(j + got - 1) % got], pp);
            point_xyz(A, tmp[j], pv);
            point_xyz(A, tmp[(j + 1) % got], pn);
            if (got < 3 || !collinear3(pp, pv, pn)) cyc[m++] = tmp[j];
        }
        int arg = 0;
        for (int j = 1; j < m; j++)
            if (cyc[j] < cyc[arg]) arg = j;
        for (int j = 0; j < m; j++) tmp[j] = cyc[(arg + j) % m];
        for (int j = 0; j < m; j++) cyc[j] = tmp[j];
        O.glen[g] = m;
        O.fkey[0][g] = ((unsigned long long)(unsigned)cyc[0] << 32) | (unsigned)(m > 1 ? cyc[1] : 0);
        O.fval[0][g] = g;
    }
}

__global__ void __launch_bounds__(256) k_fsizes(Params3 A, OutBufs O)
{
    const int ng = A.hdr->ngroup;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ng; i += gridDim.x * blockDim.x)
        O.eval[1][i] = O.glen[O.fval[0][i]];  // sizes in sorted face order
}

__global__ void __launch_bounds__(256) k_vclear(Params3 A, OutBufs O)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < A.n; i += gridDim.x * blockDim.x)
        O.vflag[i] = 0;
}

__global__ void __launch_bounds__(256) k_fcopy(Params3 A, OutBufs O, const long long *foff,
                                               int32_t *face_off, int32_t *face_idx)
{
    Hdr3 *H = A.hdr;
    // face indices: 2E <= 6n
    if (H->nfidx > 6ll * A.n) {
        if (blockIdx.x == 0 && threadIdx.x == 0) out_fail(H, QH_ERR_CAPACITY);
        return;
    }
    if (*(volatile int *)&H->status) return;
    const int ng = H->ngroup;
    if (ng == 0 && blockIdx.x == 0 && threadIdx.x == 0) face_off[0] = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ng; i += gridDim.x * blockDim.x) {
        const int g = O.fval[0][i];
        const int s = (int)O.gstart[g], m = O.glen[g];
        const long long o = foff[i];
        face_off[i] = (int32_t)o;
        for (int j = 0; j < m; j++) {
            const int v = O.poly[s + j];
            face_idx[o + j] = v;
            O.vflag[v] = 1;
        }
        if (i == ng - 1) face_off[ng] = (int32_t)(o + m);
    }
}

__global__ void __launch_bounds__(256) k_vpack(Params3 A, OutBufs O, const long long *voff,
                                               int32_t *verts)
{
    if (*(volatile int *)&A.hdr->status) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < A.n; i += gridDim.x * blockDim.x)
        if (O.vflag[i]) verts[voff[i]] = i;
}

// Result record; for a batch also each cloud's range of the vertex list
// and of the face list (faces are sorted by their smallest vertex, and a
// cloud's points are one index range, so each cloud's faces are contiguous).
__global__ void __launch_bounds__(256) k_finish(Params3 A, const int32_t *verts,
                                                const int32_t *face_off, const int32_t *face_idx,
                                                int32_t *cloud_voff, int32_t *cloud_foff)
{
    Hdr3 *H = A.hdr;
    const int st = *(volatile int *)&H->status;
    const long long nv = st ? 0 : H->nv_out;
    const int nf = st ? 0 : H->ngroup;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        qh_result r = {};
        r.status = st;
        r.count = nv;
        r.iterations = H->iter;
        r.survivor_total = H->surv_total;
        r.live_total = A.n + H->surv_total;
        r.segments_total = H->seg_total;
        r.filter_fallbacks = (int64_t)H->fallbacks;
        r.exact_argmax = (int64_t)H->exact_argmax;
        r.extra[0] = nv;
        r.extra[1] = nf;
        r.extra[2] = st ? 0 : H->nfidx;
        *A.res = r;
    }
    if (!cloud_voff) return;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c <= A.ncloud;
         c += gridDim.x * blockDim.x) {
        if (c == A.ncloud || st) {
            cloud_voff[c] = c == A.ncloud ? (int32_t)nv : 0;
            cloud_foff[c] = c == A.ncloud ? nf : 0;
            continue;
        }
        const long long lo = A.cloud_off[c];
        int a = 0, b = (int)nv;
        while (a < b) {
            const int mid = (a + b) >> 1;
            if (verts[mid] < lo) a = mid + 1;
            else b = mid;
        }
        cloud_voff[c] = a;
        a = 0;
        b = nf;
        while (a < b) {
            const int mid = (a + b) >> 1;
            if (face_idx[face_off[mid]] < lo) a = mid + 1;
            else b = mid;
        }
        cloud_foff[c] = a;
    }
}

// Batched input check: offsets start at 0, never decrease, end at n.
__global__ void k_check_clouds(Params3 A)
{
    // facet ids 4c..4c+3 are the clouds' simplices; the small-cloud route
    // allocates from here on during the setup
    if (blockIdx.x == 0 && threadIdx.x == 0) A.hdr->fcount = 4 * A.ncloud;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < A.ncloud; c += gridDim.x * blockDim.x) {
        const long long a = A.cloud_off[c], b = A.cloud_off[c + 1];
        if ((c == 0 && a != 0) || b < a || (c == A.ncloud - 1 && b != A.n))
            atomicCAS(&A.hdr->status, 0, QH_ERR_INVALID_ARG);
    }
}

static OutBufs out_bufs(char *ws, const Layout3 &L)
{
    OutBufs O;
    O.alive = (int *)(ws + L.alive);
    O.label = (int *)(ws + L.label);
    O.cop = (int *)(ws + L.cop);
    for (int b = 0; b < 2; b++) {
        O.ekey[b] = (unsigned long long *)(ws + L.ekey[b]);
        O.eval[b] = (int *)(ws + L.eval[b]);
        O.fkey[b] = (unsigned long long *)(ws + L.fkey[b]);
        O.fval[b] = (int *)(ws + L.fval[b]);
    }
    O.hist = (int *)(ws + L.hist);
    O.hist_off = (long long *)(ws + L.hist_off);
    O.gstart = (long long *)(ws + L.gstart);
    O.poly = (int *)(ws + L.poly);
    O.glen = (int *)(ws + L.glen);
    O.vflag = (int *)(ws + L.vflag);
    O.scan_tmp = (long long *)(ws + L.scan_tmp);
    return O;
}

// The whole call on the stream, no host synchronisation: header reset, the
// persistent kernel, the output stage, the result record (and cloud ranges).
static qh_status enqueue3d(Params3 &A, const Layout3 &L, char *ws, const qh_opts &o,
                           int32_t *d_verts, int32_t *d_face_off, int32_t *d_face_idx,
                           int32_t *cloud_voff, int32_t *cloud_foff, cudaStream_t st)
{
    const int block = o.block > 0 ? o.block : (o.pred_mode == QH_PRED_F64 ? kDefBlockF64 : kDefBlockF32);
    const int items = o.items > 0 ? o.items : kDefItems;
    if ((block != 128 && block != 256 && block != 512) || (items != 2 && items != 4 && items != 8))
        return QH_ERR_INVALID_ARG;
    if (cudaMemsetAsync(A.hdr, 0, sizeof(Hdr3), st) != cudaSuccess) return QH_ERR_CUDA;
    if (A.cloud_off) k_check_clouds<<<grid_for(A.ncloud, 256), 256, 0, st>>>(A);
    const void *fn = persistent_kernel(o.pred_mode, items);
    int grid = persistent_grid(fn, block, o.blocks_per_sm);
    if (grid <= 0) return QH_ERR_CUDA;
    grid = std::min(grid, kMaxGrid);
    void *args[] = {&A};
    if (cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(block), args, 0, st) != cudaSuccess)
        return QH_ERR_CUDA;
    // ---- output stage (sizes from the header on the device)
    OutBufs O = out_bufs(ws, L);
    Hdr3 *H = A.hdr;
    const long long fcap = L.fcap, ecap = 3ll * (L.fcap + 1), n = A.n;
    const int gf = (int)std::min<long long>(out_grid(), (fcap + 255) / 256);
    k_alive<<<gf, 256, 0, st>>>(A, O);
    k_uf_union<<<gf, 256, 0, st>>>(A, O);
    k_uf_compress<<<gf, 256, 0, st>>>(A, O);
    k_bedges<<<gf, 256, 0, st>>>(A, O);
    int lbits = 1;
    while ((1ll << lbits) <= fcap) lbits++;
    radix_sort(O.ekey[0], O.eval[0], O.ekey[1], O.eval[1], &H->nbedge, ecap, 32 + lbits, O.hist,
               O.hist_off, O.scan_tmp, &H->sort_m, st);
    const int ge = (int)std::min<long long>(out_grid(), (ecap + 255) / 256);
    k_gmark<<<ge, 256, 0, st>>>(A, O);
    // start-flag scan -> group index (the edge-sort scratch keys are free now)
    long long *gscan = (long long *)O.ekey[1];
    scan_counts(O.poly, &H->nbedge, 0, ecap, gscan, O.scan_tmp, nullptr, st);
    k_gwrite<<<ge, 256, 0, st>>>(A, O, gscan);
    k_walk<<<(int)std::min<long long>(out_grid() * 2, (fcap + 127) / 128), 128, 0, st>>>(A, O);
    int vbits = 1;
    while ((1ll << vbits) <= n) vbits++;
    radix_sort(O.fkey[0], O.fval[0], O.fkey[1], O.fval[1], &H->ngroup, fcap + 1, 32 + vbits,
               O.hist, O.hist_off, O.scan_tmp, &H->sort_m, st);
    k_fsizes<<<gf, 256, 0, st>>>(A, O);
    long long *foff = (long long *)O.ekey[1];
    scan_counts(O.eval[1], &H->ngroup, 0, fcap + 1, foff, O.scan_tmp, &H->nfidx, st);
    const int gn = (int)std::min<long long>(out_grid(), (n + 255) / 256);
    k_vclear<<<gn, 256, 0, st>>>(A, O);
    k_fcopy<<<gf, 256, 0, st>>>(A, O, foff, d_face_off, d_face_idx);
    long long *voff = (long long *)O.eval[1];  // n long longs fit: eval[1] holds 3 * fcap ints
    scan_counts(O.vflag, nullptr, (int)n, n, voff, O.scan_tmp, &H->nv_out, st);
    k_vpack<<<gn, 256, 0, st>>>(A, O, voff, d_verts);
    k_finish<<<cloud_voff ? grid_for(A.ncloud + 1, 256) : 1, 256, 0, st>>>(
        A, d_verts, d_face_off, d_face_idx, cloud_voff, cloud_foff);
    return cudaGetLastError() == cudaSuccess ? QH_OK : QH_ERR_CUDA;
}

}  // namespace d3
}  // namespace qh

using namespace qh;
using namespace qh::d3;

// facet ids must fit the 28-bit claim permutation: 6n + 4 ncloud + 64 < 2^28
constexpr int64_t kMax3d = 44000000;

static int64_t facet_hint(const qh_opts *opts) { return opts ? opts->max_facets : 0; }

extern "C" size_t qh_workspace_bytes_3d(int64_t n, const qh_opts *opts)
{
    if (n < 0 || n > kMax3d || facet_hint(opts) < 0) return 0;
    return layout3d(n, 1, true, facet_hint(opts)).total;
}

extern "C" size_t qh_workspace_bytes_3d_batched(int64_t n, int32_t ncloud, const qh_opts *opts)
{
    if (n < 0 || ncloud < 1 || n + ncloud > kMax3d || facet_hint(opts) < 0) return 0;
    return layout3d(n, ncloud, false, facet_hint(opts)).total;
}

extern "C" qh_status qh_debug_timeline_3d(const void *d_ws, int64_t n, int64_t *h_rows,
                                          int32_t max_rows, int32_t *h_nrows, cudaStream_t st)
{
    if (!d_ws || !h_rows || !h_nrows || max_rows < 0 || n < 0 || n > kMax3d)
        return QH_ERR_INVALID_ARG;
    const Layout3 L = layout3d(n, 1, true, 0);  // the header's offset does not depend on it
    Hdr3 hh;
    if (cudaMemcpyAsync(&hh, (const char *)d_ws + L.hdr, sizeof(Hdr3), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return QH_ERR_CUDA;
    int rows = std::min(std::min(hh.iter, kTimeline3), (int)max_rows);
    for (int r = 0; r < rows; r++) {
        h_rows[10 * r] = r + 1;
        for (int c = 0; c < 9; c++) h_rows[10 * r + 1 + c] = hh.tl[r][c];
    }
    *h_nrows = rows;
    return QH_OK;
}

extern "C" qh_status qh_debug_phases_3d(const void *d_ws, int64_t *h_ns, cudaStream_t st)
{
    if (!d_ws || !h_ns) return QH_ERR_INVALID_ARG;
    Hdr3 hh;
    if (cudaMemcpyAsync(&hh, (const char *)d_ws, sizeof(Hdr3), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return QH_ERR_CUDA;
    for (int k = 0; k < 4; k++) h_ns[k] = hh.setup_ns[k];
    h_ns[4] = hh.kernel_ns;
    return QH_OK;
}

static bool opts_ok(const qh_opts &o)
{
    return (o.pred_mode == QH_PRED_F32 || o.pred_mode == QH_PRED_F64) && o.small_cloud >= 0 &&
           o.small_cloud <= QH_SMALL_CLOUD_MAX && o.max_facets >= 0;
}

extern "C" qh_status qh_hull3d(const float *d_x, const float *d_y, const float *d_z, int64_t n,
                               int64_t stride, int32_t *d_verts, int64_t *h_nv, int32_t *d_face_off,
                               int32_t *d_face_idx, int64_t *h_nf, qh_result *h_result, void *d_ws,
                               size_t ws_bytes, const qh_opts *opts, cudaStream_t st)
{
    qh_opts o;
    qh_default_opts(&o);
    if (opts) o = *opts;
    if (h_nv) *h_nv = 0;
    if (h_nf) *h_nf = 0;
    if (n < 0 || n > kMax3d || stride < 1 || !d_ws || !h_nv || !h_nf)
        return QH_ERR_INVALID_ARG;
    if (n > 0 && (!d_x || !d_y || !d_z || !d_verts || !d_face_off || !d_face_idx))
        return QH_ERR_INVALID_ARG;
    if (!opts_ok(o)) return QH_ERR_INVALID_ARG;
    if (o.loop_mode != QH_LOOP_PERSISTENT) return QH_ERR_NOT_SUPPORTED;
    const Layout3 L = layout3d(n, 1, true, o.max_facets);
    if (ws_bytes < L.total || ((uintptr_t)d_ws & 255)) return QH_ERR_NOMEM;
    qh_result r = {};
    if (n == 0) {
        if (cudaMemsetAsync(d_face_off, 0, 4, st) != cudaSuccess) return QH_ERR_CUDA;
        if (h_result) *h_result = r;
        return cudaStreamSynchronize(st) == cudaSuccess ? QH_OK : QH_ERR_CUDA;
    }
    char *ws = (char *)d_ws;
    Params3 A = make_params3(d_x, d_y, d_z, n, stride, ws, L, o);
    qh_status s = enqueue3d(A, L, ws, o, d_verts, d_face_off, d_face_idx, nullptr, nullptr, st);
    if (s != QH_OK) return s;
    if (cudaMemcpyAsync(&r, A.res, sizeof(r), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return QH_ERR_CUDA;
    if (h_result) *h_result = r;
    if (r.status != 0) return (qh_status)r.status;
    *h_nv = r.extra[0];
    *h_nf = r.extra[1];
    return QH_OK;
}

extern "C" qh_status qh_hull3d_batched(const float *d_x, const float *d_y, const float *d_z,
                                       int64_t stride, const int64_t *d_cloud_off, int32_t ncloud,
                                       int64_t n, int32_t *d_verts, int32_t *d_cloud_vert_off,
                                       int32_t *d_face_off, int32_t *d_face_idx,
                                       int32_t *d_cloud_face_off, int32_t *d_cloud_status,
                                       qh_result *d_result, void *d_ws, size_t ws_bytes,
                                       const qh_opts *opts, cudaStream_t st)
{
    qh_opts o;
    qh_default_opts(&o);
    if (opts) o = *opts;
    if (n < 1 || ncloud < 1 || n + ncloud > kMax3d || stride < 1 || !d_ws || !d_cloud_off)
        return QH_ERR_INVALID_ARG;
    if (!d_x || !d_y || !d_z || !d_verts || !d_cloud_vert_off || !d_face_off || !d_face_idx ||
        !d_cloud_face_off || !d_cloud_status || !d_result)
        return QH_ERR_INVALID_ARG;
    if (!opts_ok(o)) return QH_ERR_INVALID_ARG;
    if (o.loop_mode != QH_LOOP_PERSISTENT) return QH_ERR_NOT_SUPPORTED;
    const Layout3 L = layout3d(n, ncloud, false, o.max_facets);
    if (ws_bytes < L.total || ((uintptr_t)d_ws & 255)) return QH_ERR_NOMEM;
    char *ws = (char *)d_ws;
    Params3 A = make_params3(d_x, d_y, d_z, n, stride, ws, L, o);
    A.cloud_off = (const long long *)d_cloud_off;
    A.ncloud = ncloud;
    A.cloud_status = d_cloud_status;
    A.res = d_result;
    return enqueue3d(A, L, ws, o, d_verts, d_face_off, d_face_idx, d_cloud_vert_off,
                     d_cloud_face_off, st);
}
