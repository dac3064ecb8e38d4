// Device utilities shared by the hull kernels: status codes, orderable
// float keys, grid-wide barrier with a bounded wait, small warp helpers.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "qh.h"

namespace qh {

constexpr int kStOk = QH_OK;
constexpr int kStNonfinite = QH_ERR_NONFINITE;
constexpr int kStDegenerate = QH_ERR_DEGENERATE;
constexpr int kStCapacity = QH_ERR_CAPACITY;
constexpr int kStTimeout = QH_ERR_TIMEOUT;
constexpr int kStNoConv = QH_ERR_NO_CONVERGENCE;

// ---------------------------------------------------------------- checks
// Device-side checks of the debug build (-DQH_DEBUG=1): alignment of every
// bulk copy and mbarrier, bounds of scatter destinations, segment indices and
// hull slots.  A failed check skips the access and is recorded (count, first
// site, its two values) in a per-translation-unit record that
// qh_debug_checks() reads; nothing traps.  In the default build the checks
// compile to nothing.
#ifndef QH_DEBUG
#define QH_DEBUG 0
#endif

struct DbgDev {
    unsigned long long n;
    int site, pad;
    unsigned long long a, b;
};
// host side: each translation unit registers a reader of its record
typedef int (*DbgReader)(DbgDev *out, int reset);
void dbg_register(DbgReader r);

#if QH_DEBUG
static __device__ DbgDev g_qh_dbg;
static __device__ __noinline__ void dbg_fail(int site, unsigned long long a, unsigned long long b)
{
    if (atomicAdd(&g_qh_dbg.n, 1ull) == 0ull) {
        g_qh_dbg.site = site;
        g_qh_dbg.a = a;
        g_qh_dbg.b = b;
    }
}
namespace {
int dbg_read_tu(DbgDev *out, int reset)
{
    if (cudaMemcpyFromSymbol(out, g_qh_dbg, sizeof(DbgDev)) != cudaSuccess) return 1;
    if (reset) {
        DbgDev z = {};
        if (cudaMemcpyToSymbol(g_qh_dbg, &z, sizeof(DbgDev)) != cudaSuccess) return 1;
    }
    return 0;
}
struct DbgRegistrar {
    DbgRegistrar() { dbg_register(&dbg_read_tu); }
};
DbgRegistrar g_dbg_registrar;
}  // namespace
#endif

// true when the condition holds; in the debug build a failure is recorded
__device__ __forceinline__ bool dbg_ok(bool c, int site, unsigned long long a,
                                       unsigned long long b)
{
#if QH_DEBUG
    if (!c) dbg_fail(site, a, b);
    return c;
#else
    (void)site; (void)a; (void)b;
    (void)c;
    return true;
#endif
}
constexpr int kDbgBulkAlign = QH_DBG_BULK_ALIGN;
constexpr int kDbgMbarAlign = QH_DBG_MBAR_ALIGN;
constexpr int kDbgBulkRange = QH_DBG_BULK_RANGE;
constexpr int kDbgPointDst = QH_DBG_POINT_DST;
constexpr int kDbgSegIndex = QH_DBG_SEG_INDEX;
constexpr int kDbgHullSlot = QH_DBG_HULL_SLOT;
constexpr int kDbgVecAlign = QH_DBG_VEC_ALIGN;

// Total order on float bits that matches the numeric order (-0 < +0 apart).
__device__ __forceinline__ uint32_t ord_f32(float f)
{
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float unord_f32(uint32_t o)
{
    uint32_t u = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
    return __uint_as_float(u);
}
// Coordinates enter keys and comparisons with -0.0 mapped to +0.0 (same point).
__device__ __forceinline__ float canon0(float f) { return f == 0.0f ? 0.0f : f; }

// Argmax key of a point: larger distance first, then lower index.
__device__ __forceinline__ unsigned long long dist_key(float d, int idx)
{
    return ((unsigned long long)ord_f32(d) << 32) | (unsigned long long)(0xffffffffu - (uint32_t)idx);
}
__device__ __forceinline__ int key_idx(unsigned long long k) { return (int)(0xffffffffu - (uint32_t)(k & 0xffffffffu)); }
__device__ __forceinline__ float key_dist(unsigned long long k) { return unord_f32((uint32_t)(k >> 32)); }

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

struct GridBarrier {
    unsigned int count;  // arrivals since the launch
};

// Grid-wide barrier for a cooperative launch (all CTAs co-resident), one
// global atomic per CTA and round: count only grows (zero at launch), arrival
// k of the grid belongs to round k / gridDim.x, and round r is complete once
// count reaches (r + 1) * gridDim.x.  The arrival releases the CTA's writes
// (ordered before it by the block barrier) and the polling load acquires the
// other CTAs'.  The wait is bounded by wait_ns; on expiry the barrier raises
// *fail (status QH_ERR_TIMEOUT) and returns so that the kernel can leave
// cleanly.
//
// Returns *fail as read by thread 0 after the wait, the same value in every
// thread of the CTA: callers branch on it without splitting the CTA around
// later block barriers.  skip_arrive (tests of the bounded wait only): this
// CTA waits without arriving, so the round cannot complete and every CTA's
// wait runs out.
__device__ __forceinline__ int grid_sync_count(GridBarrier *b, int *fail, long long wait_ns,
                                               bool skip_arrive = false)
{
    __shared__ int st_bcast;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int old;
        if (skip_arrive) {
            asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(old) : "l"(&b->count) : "memory");
        } else {
            asm volatile("atom.add.release.gpu.u32 %0, [%1], 1;"
                         : "=r"(old)
                         : "l"(&b->count)
                         : "memory");
        }
        const unsigned int target = (old / gridDim.x + 1u) * gridDim.x;
        unsigned long long t0 = 0;
        for (unsigned int spins = 0;; spins++) {
            unsigned int cur;
            asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(cur) : "l"(&b->count) : "memory");
            if ((int)(cur - target) >= 0) break;
            if (spins == 0) {
                t0 = globaltimer_ns();
            } else if ((spins & 255u) == 0u && (long long)(globaltimer_ns() - t0) > wait_ns) {
                atomicCAS(fail, 0, kStTimeout);
                break;
            }
        }
        st_bcast = *(volatile int *)fail;
    }
    __syncthreads();
    return st_bcast;
}

// CTA-uniform read of a status word (thread 0 reads; block barriers on both
// sides).
__device__ __forceinline__ int status_uniform(const int *st)
{
    __shared__ int st_u;
    __syncthreads();
    if (threadIdx.x == 0) st_u = *(volatile const int *)st;
    __syncthreads();
    return st_u;
}

// Bound of a CTA's wait for its own bulk copies (a few KB from device
// memory: microseconds).  Fixed, not the caller's wait_ns: an expired wait
// means the copy engine failed, not that another CTA is slow.
constexpr long long kCopyWaitNs = 2000000000ll;

// ---------------------------------------------------------------- shared addresses
__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

// Bulk copy engine (TMA, non-tensor form): `bytes` (a multiple of 16) from a
// 16-byte aligned global address to a 16-byte aligned shared address,
// completion counted on an mbarrier.
__device__ __forceinline__ bool mbar_aligned(const unsigned long long *bar)
{
    return dbg_ok((smem_u32(bar) & 7u) == 0u, kDbgMbarAlign, smem_u32(bar), 8);
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    if (!mbar_aligned(bar)) return;
    asm volatile("mbarrier.init.shared.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes)
{
    if (!mbar_aligned(bar)) return;
    asm volatile("mbarrier.arrive.expect_tx.shared.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes,
                                         unsigned long long *bar)
{
    // 16-byte aligned source and destination, a size that is a positive
    // multiple of 16 (a skipped copy leaves its barrier short: the bounded
    // wait gives up)
    if (!dbg_ok(((smem_u32(dst) | (unsigned)(uintptr_t)src | bytes) & 15u) == 0u && bytes > 0u,
                kDbgBulkAlign, (unsigned long long)(uintptr_t)src,
                ((unsigned long long)smem_u32(dst) << 32) | bytes) ||
        !mbar_aligned(bar))
        return;
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
// Wait until the mbarrier's phase `parity` has completed; bounded: gives up
// after about `max_ns` (returns false) so that a lost copy cannot hang the CTA.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity,
                                          long long max_ns)
{
    if (!mbar_aligned(bar)) return false;
    const unsigned a = smem_u32(bar);
    unsigned done = 0;
    unsigned long long t0 = 0;
    for (unsigned spins = 0;; spins++) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (spins == 0) t0 = globaltimer_ns();
        else if ((spins & 63u) == 0u && (long long)(globaltimer_ns() - t0) > max_ns) return false;
    }
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ long long warp_incl_scan64(long long v)
{
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Block-wide exclusive scan of a 64-bit value (blockDim.x <= 1024).  wsum
// must hold 33 entries.  Returns the exclusive prefix; *total gets the sum.
__device__ __forceinline__ long long block_excl_scan64(long long v, long long *wsum, long long *total)
{
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    long long inc = warp_incl_scan64(v);
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        long long s = lane < nw ? wsum[lane] : 0;
        long long si = warp_incl_scan64(s);
        if (lane < nw) wsum[lane] = si - s;
        if (lane == nw - 1) wsum[32] = si;
    }
    __syncthreads();
    long long r = wsum[w] + inc - v;
    *total = wsum[32];
    __syncthreads();
    return r;
}

}  // namespace qh
