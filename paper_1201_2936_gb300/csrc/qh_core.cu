// Status strings, defaults and the occupancy cache of libqh.
#include <cstring>
#include <mutex>
#include <map>
#include <tuple>

#include <vector>

#include "qh_common.cuh"
#include "qh_internal.h"

namespace qh {

// readers of the translation units' device-check records (debug build)
static std::mutex &dbg_mu()
{
    static std::mutex mu;
    return mu;
}
static std::vector<DbgReader> &dbg_readers()
{
    static std::vector<DbgReader> v;
    return v;
}
void dbg_register(DbgReader r)
{
    std::lock_guard<std::mutex> g(dbg_mu());
    dbg_readers().push_back(r);
}

int persistent_grid(const void *func, int block, int blocks_per_sm)
{
    return persistent_grid_smem(func, block, blocks_per_sm, 0);
}

int persistent_grid_smem(const void *func, int block, int blocks_per_sm, size_t dsmem)
{
    static std::mutex mu;
    // (func, device, block, dynamic shared memory)
    static std::map<std::tuple<uintptr_t, int, int, size_t>, int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    const auto key = std::make_tuple((uintptr_t)func, dev, block, dsmem);
    int per_sm = 0, sms = 0;
    {
        std::lock_guard<std::mutex> g(mu);
        auto it = cache.find(key);
        if (it != cache.end()) {
            per_sm = it->second & 0xffff;
            sms = it->second >> 16;
        }
    }
    if (sms == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, func, block, dsmem) != cudaSuccess)
            return 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return 0;
        std::lock_guard<std::mutex> g(mu);
        cache[key] = (sms << 16) | per_sm;
    }
    if (per_sm <= 0) return 0;
    if (blocks_per_sm > 0 && blocks_per_sm < per_sm) per_sm = blocks_per_sm;
    return per_sm * sms;
}

int sm_count()
{
    static std::mutex mu;
    static std::map<int, int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    {
        std::lock_guard<std::mutex> g(mu);
        auto it = cache.find(dev);
        if (it != cache.end()) return it->second;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        return 1;
    std::lock_guard<std::mutex> g(mu);
    cache[dev] = sms;
    return sms;
}

}  // namespace qh

extern "C" const char *qh_status_str(qh_status s)
{
    switch (s) {
    case QH_OK: return "QH_OK";
    case QH_ERR_INVALID_ARG: return "QH_ERR_INVALID_ARG: invalid argument";
    case QH_ERR_NONFINITE: return "QH_ERR_NONFINITE: input contains NaN or Inf";
    case QH_ERR_DEGENERATE: return "QH_ERR_DEGENERATE: points do not span the space";
    case QH_ERR_NOMEM: return "QH_ERR_NOMEM: workspace too small or misaligned";
    case QH_ERR_CAPACITY: return "QH_ERR_CAPACITY: internal table overflow";
    case QH_ERR_TIMEOUT: return "QH_ERR_TIMEOUT: a bounded device wait expired";
    case QH_ERR_NO_CONVERGENCE: return "QH_ERR_NO_CONVERGENCE: iteration cap reached";
    case QH_ERR_CUDA: return "QH_ERR_CUDA: CUDA runtime error";
    case QH_ERR_NOT_SUPPORTED: return "QH_ERR_NOT_SUPPORTED: option combination not available";
    }
    return "unknown qh_status";
}

extern "C" qh_status qh_debug_checks(qh_debug_record *h_out, int32_t reset)
{
    if (!h_out) return QH_ERR_INVALID_ARG;
    std::memset(h_out, 0, sizeof(*h_out));
    if (!QH_DEBUG) return QH_ERR_NOT_SUPPORTED;
    h_out->enabled = 1;
    if (cudaDeviceSynchronize() != cudaSuccess) return QH_ERR_CUDA;
    std::lock_guard<std::mutex> g(qh::dbg_mu());
    for (qh::DbgReader r : qh::dbg_readers()) {
        qh::DbgDev d = {};
        if (r(&d, reset) != 0) return QH_ERR_CUDA;
        if (d.n > 0 && h_out->failures == 0) {
            h_out->site = d.site;
            h_out->a = d.a;
            h_out->b = d.b;
        }
        h_out->failures += (int64_t)d.n;
    }
    return QH_OK;
}

extern "C" const char *qh_version(void) { return "qh 0.1 sm_103a"; }

extern "C" void qh_default_opts(qh_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->pred_mode = QH_PRED_F32;
    o->loop_mode = QH_LOOP_PERSISTENT;
}
