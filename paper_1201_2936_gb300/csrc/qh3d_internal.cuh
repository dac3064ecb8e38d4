// Data structures shared by the 3D kernels (qh3d.cu) and the 3D output and
// host code (qh3d_out.cu).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "qh.h"
#include "pred3.cuh"
#include "qh_common.cuh"

namespace qh {
namespace d3 {

// Launch shape of the persistent kernel: threads per CTA (runtime, up to
// kMaxBlock) and points per thread of the assign pass (template: 2, 4, 8).
constexpr int kMaxBlock = 512;
// default threads per CTA by predicate mode: the fastest of 128/256/512 on
// the 8M ball and the 1M sphere (FP32 filter: 512, FP64: 256)
constexpr int kDefBlockF32 = 512;
constexpr int kDefBlockF64 = 256;
constexpr int kDefItems = 4;
constexpr int kMaxTile = 4096;           // points per assign tile (block x items), upper bound
constexpr int kMinTile = 256;            // lower bound (sizes the tile maps)
#ifndef QH3D_VCAP
#define QH3D_VCAP 32
#endif
constexpr int kVCap = QH3D_VCAP;         // visible facets a candidate may list
constexpr int kNCap = 2 * kVCap;         // horizon neighbours a candidate may list (>= kVCap + 2)
constexpr int kMaxGrid = 4096;
constexpr int kDirs = 26;  // directions of the first polytope: the non-zero vectors of {-1, 0, 1}^3
#ifndef QH3D_INITDIRS
#define QH3D_INITDIRS 2
#endif
// single cloud: start from that polytope (0: the tetrahedron; 1: all 26
// directions; 2: the 14 of the axes and the diagonals; 3: the 6 axes)
constexpr int kInitDirs = QH3D_INITDIRS;
// the selection and its claim rounds take one warp per candidate while
// there are at most this many candidates per warp of the grid, else one
// thread per candidate
#ifndef QH3D_SELW
#define QH3D_SELW 2
#endif
constexpr int kSelWarpMul = QH3D_SELW;

// A facet of the current triangulated hull.
struct Fac3 {
    float p[9];   // vertex coordinates a, b, c, counter-clockwise seen from outside
    int v[3];     // vertex point indices
    int nb[3];    // nb[i]: facet across edge (v[i], v[i+1])
    int alive;
};
static_assert(sizeof(Fac3) == 64, "Fac3 layout");

// Farthest-point accumulator of a facet's outside set (its segment).
struct Acc3 {
    unsigned long long key1;  // (distance order bits << 32) | ~index of the best point
    unsigned o2;              // distance order bits of the best other point
    unsigned cnt;             // points
    unsigned emax;            // largest error bound of the keys (float bits)
    unsigned pad[3];
};
static_assert(sizeof(Acc3) == 32, "Acc3 layout");

// Segment table entry: facet and the range of its outside set in a buffer.
struct Ent3 {
    int f, start, len, pad;
};

struct Hdr3 {
    GridBarrier bar;
    int status, nonfinite;
    float4 pa, pb, pc, pd;  // initial simplex (w: point index bits)
    int search_idx, cand_idx, cand_ok;
    int fcount;             // facets created so far
    int fc_iter[2];         // facet count when the table of that parity was built
    int fc_lo_last;         // first facet id created in the last iteration
    int hull_vertices;
    int nwin, iter;
    int nact[8];            // candidates that claimed in round r (r < kRounds)
    // segment table of each parity: (entries << 32) | points, counted by the
    // table phase with one atomic per 512 items
    unsigned long long tab[2];
    int tile_sz[2];         // points per assign / scatter tile of each table
    int n_uncert;
    int next_cloud;         // queue of the per-cloud setup
    int next_small;         // queue of the small-cloud route (one warp per cloud)
    long long seg_total, surv_total;
    unsigned long long fallbacks, exact_argmax;
    // output stage
    int nalive, ncop, nbedge, ngroup;
    int sort_m;             // entries of the radix-sort histogram being scanned
    int uf_fail, pad1, pad2;
    long long nfidx, nv_out;
    // per-iteration record (first kTimeline3 iterations): live points,
    // segments, winners, then device time of select, rounds, assign, table,
    // scatter + certify, exact (ns)
    long long tl[64][9];
    // device time of the setup (initial simplex, first assignment, its table,
    // its scatter + certify + exact) and of the whole persistent kernel (ns)
    long long setup_ns[4], kernel_ns;
    // extreme point of each direction of the first polytope (single cloud):
    // (ordered dot product << 32) | ~index, the largest kept
    unsigned long long dirkey[kDirs];
};
constexpr int kTimeline3 = 64;

struct Params3 {
    const float *x, *y, *z;
    long long stride;
    int n;
    int fcap, ecap;
    int tile;                     // points per assign tile (block x items)
    // clouds: cloud c holds points [cloud_off[c], cloud_off[c+1]); a single
    // cloud when cloud_off is null
    const long long *cloud_off;
    int ncloud;
    int *cloud_status;            // per-cloud qh_status (batched calls)
    Hdr3 *hdr;
    qh_result *res;
    // facets
    Fac3 *fac;
    Plane3 *plane;                // FP32 filter plane of each facet (written with the facet)
    Acc3 *acc;
    float4 *apex;                 // apex (farthest point) of each facet with a segment
    unsigned long long *claim[2]; // claims of the even / odd selection rounds (claim_key)
    int4 *cone;                   // deleted facet: (first cone facet, count, apex index, iteration)
    float *thr;                   // exact-apex candidate threshold
    int *nstart;                  // new segment start of a facet
    int *big_mark;
    int *big_v, *big_h;
    // segments
    Ent3 *ent[2];
    int *tile_ent[2], *tile_m[2];  // per table: tile -> first entry, entries the tile meets
    int2 *vn;                     // (|V|, |N|) of a candidate, (-1,-1) on overflow
    int *cstate;                  // candidate state in an iteration: 0 active, 1 won, 2 out
    int *taken;                   // iteration whose winner deleted the facet
    int *vpool, *npool;
    int *uncert;
    // points
    float4 *pts[2];
    int2 *code;                   // (target facet, rank) of each live point
    // reductions
    long long *part;
    float4 *blk_a, *blk_b;
    float *blk_v;
    int *blk_i;
    long long max_iters, wait_ns;
    int test_hold;                // CTA 0 skips its first grid-barrier arrival (tests)
    int small_cloud;              // batched: clouds of 4..small_cloud points, one warp each
    int init_dirs;                // single cloud: first polytope from the directions' extreme points
};

// The pseudo facet of cloud c in the first assignment (every point of the
// cloud coned to its tetrahedron) is fcap + c; its cone record lists the
// tetrahedron's facets.

// Claim of a candidate (the facet f whose segment of `len` points it heads)
// in a selection round.  Later iterations and rounds win over earlier ones;
// within a round larger segments go first (size class = log2(len) / 2, so a
// segment with millions of points is not starved by small neighbours), then
// a bijective pseudo-random permutation of the facet ids (28 bits), which
// keeps keys unique and makes each round's winners a Luby-style independent
// set.  Bits: iteration 28 | round 4 | size class 4 | permutation 28.
#ifndef QH3D_ROUNDS
#define QH3D_ROUNDS 3
#endif
constexpr int kRounds = QH3D_ROUNDS;
static_assert(kRounds >= 1 && kRounds <= 7, "round numbers fit the claim key and nact[]");
__device__ __forceinline__ unsigned long long claim_key(int iter, int round, int f, int len)
{
    const unsigned perm = (((unsigned)f ^ ((unsigned)iter * 0x9E37u)) * 0x0B5AD4Bu) & 0x0FFFFFFFu;
    const unsigned cls = min(15u, (31u - (unsigned)__clz(max(len, 1))) >> 1);
    return ((unsigned long long)(unsigned)iter << 36) | ((unsigned long long)round << 32) |
           ((unsigned long long)cls << 28) | perm;
}

struct SmemRed {
    float4 a[kMaxBlock], b[kMaxBlock];
    float v[kMaxBlock];
    int i[kMaxBlock];
    int flag;
};
constexpr int kSlotBits = 7;
constexpr int kSlots = 1 << kSlotBits;   // distinct cone targets aggregated per assign tile
struct SmemAssign {
    int e0, m;
    int start[kMaxTile];
    int f[kMaxTile];
};
// The cone targets a CTA met in one assign phase, over all of its tiles (it
// lives outside the union: the scatter after the table phase, which visits
// the same tiles on the same CTA, reads the bases): points counted and
// farthest-point keys merged in shared memory, one reservation and key merge
// per (CTA, target) at the end of the phase.  A point's code then carries
// its slot and rank within the CTA's count.
constexpr int kLocalBits = 24;           // rank within a CTA's count of one target
struct SmemSlots {
    int skey[kSlots], scnt[kSlots], sbase[kSlots];
    unsigned long long sk1[kSlots];
    unsigned so2[kSlots], sem[kSlots];
};
struct SmemTable {
    long long wsum[33];
    unsigned long long base;
};
struct SmemWin {
    int n, base0;
    int list[kMaxBlock];
    int nh[kMaxBlock];    // a winner's horizon edges (-1: too many)
    int base[kMaxBlock];  // its first facet slot, from base0
    long long wsum[33];
};
// Visible-set search with one warp per candidate: the warp's lists.
struct SmemBfs {
    int V[kMaxBlock / 32][kVCap];
    int N[kMaxBlock / 32][kNCap];
};
struct SmemX3 {
    int idx[kMaxBlock];
    float4 p[kMaxBlock];
};
// The first polytope of a single cloud (built by one warp of CTA 0): the
// tetrahedron with the extreme points of kDirs directions inserted.
constexpr int kInitF = 128;         // facets while it is built (2 V - 4 <= 56 at the end)
constexpr int kDirGroup = 14;       // directions reduced per pass over the points
struct SmemInit {
    float p[kInitF][9];             // the three vertices' coordinates
    int v[kInitF][3];               // their point indices (outward: counter-clockwise)
    int vis[kInitF];
    int eu[kInitF], ev[kInitF];     // horizon edges of the point being inserted
    float ep[kInitF][6];
    int nf, ne, nv;
    int vid[32];                    // point index of each vertex slot
    unsigned emask[32];             // directed edges of the facets that stay, by slot
    int eid[32][32];                // the facet of each directed edge (neighbours at the end)
    unsigned long long key[32][14]; // per warp: the best key of each direction of a group
};
union SmemAll3 {
    SmemInit init;
    SmemRed red;
    SmemAssign a;
    SmemTable t;
    SmemX3 x;
    SmemWin w;
    SmemBfs bfs;
};

struct Layout3 {
    size_t hdr, res, fac, plane, acc, apex, claim[2], cone, thr, nstart, big_mark, big_v, big_h;
    size_t ent[2], tile_ent[2], tile_m[2], vn, cstate, taken, vpool, npool, uncert, pts[2], code, part,
        blk_a, blk_b, blk_v, blk_i;
    // output stage
    size_t alive, label, cop, ekey[2], eval[2], hist, hist_off, gstart, poly, glen, fkey[2], fval[2],
        vflag, scan_tmp;
    size_t total;
    int fcap, ecap, hist_blocks, ncloud;
};

Layout3 layout3d(int64_t n, int ncloud, bool single, int64_t max_facets);

// Device-sized scan and radix sort (qh3d_out.cu), shared with the 4D output
// stage.  Counts are read on the device (*m_ptr, or m_fix when m_ptr is
// null); m_cap bounds them and sizes the grids.  Scratch: tmp holds
// (256 * tiles(m_cap) + m_cap) / kScanTile + 64 long longs, hist 256 *
// tiles(m_cap) ints and hist_off as many long longs, tiles(m) = ceil(m /
// kScanTile).
constexpr int kScanTile = 2048;
void scan_counts(const int *in, const int *m_ptr, int m_fix, long long m_cap, long long *out,
                 long long *tmp, long long *d_total, cudaStream_t st);
void radix_sort(unsigned long long *key, int *val, unsigned long long *tkey, int *tval,
                const int *m_ptr, long long m_cap, int bits, int *hist, long long *hist_off,
                long long *tmp, int *hist_m, cudaStream_t st);
const void *persistent_kernel(int mode, int items);
Params3 make_params3(const float *x, const float *y, const float *z, int64_t n, int64_t stride,
                     char *ws, const Layout3 &L, const qh_opts &o);

}  // namespace d3
}  // namespace qh
