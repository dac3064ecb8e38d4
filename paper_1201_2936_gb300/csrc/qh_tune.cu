// Autotuner of the batched 3D launch: threads per CTA, points per thread of
// the assign pass and CTAs per SM of the persistent grid, then, at the
// fastest shape, the small-cloud threshold (clouds of at most that many
// points hulled whole by one warp: the switchover point below which that
// beats the segmented iterations).  Each candidate runs the caller's batch
// on the caller's stream (one untimed run, then `reps` runs timed with CUDA
// events); the fastest candidate whose runs all end with QH_OK is returned.
// The hull does not depend on these choices (every decision is an exact
// predicate or an index tie-break), so the outputs of the last run are
// valid for any candidate.
#include <algorithm>
#include <vector>

#include "qh.h"
#include "qh_internal.h"

namespace {

struct Cand {
    int block, items, bps, small;
};

// Events are created once per call and destroyed on every exit path.
struct Events {
    std::vector<cudaEvent_t> ev;
    explicit Events(int n) : ev(n, nullptr)
    {
        for (auto &e : ev)
            if (cudaEventCreate(&e) != cudaSuccess) e = nullptr;
    }
    ~Events()
    {
        for (auto e : ev)
            if (e) cudaEventDestroy(e);
    }
    bool ok() const
    {
        for (auto e : ev)
            if (!e) return false;
        return true;
    }
};

}  // namespace

extern "C" qh_status qh_autotune_3d_batched(
    const float *d_x, const float *d_y, const float *d_z, int64_t stride,
    const int64_t *d_cloud_off, int32_t ncloud, int64_t n, int32_t *d_verts,
    int32_t *d_cloud_vert_off, int32_t *d_face_off, int32_t *d_face_idx,
    int32_t *d_cloud_face_off, int32_t *d_cloud_status, qh_result *d_result, void *d_ws,
    size_t ws_bytes, int32_t reps, qh_opts *h_best, float *h_ms, int32_t *h_shape,
    int32_t max_cand, int32_t *h_ncand, cudaStream_t st)
{
    if (!h_best || !h_ncand || reps < 1 || reps > 64 || max_cand < 0 || (max_cand > 0 && (!h_ms || !h_shape)))
        return QH_ERR_INVALID_ARG;
    *h_ncand = 0;
    const qh_opts base = *h_best;
    std::vector<Cand> cands;
    for (int block : {128, 256, 512})
        for (int items : {2, 4, 8})
            for (int bps : {1, 2, 4}) cands.push_back({block, items, bps, base.small_cloud});
    const size_t nshape = cands.size();
    Events E(reps + 1);
    if (!E.ok()) return QH_ERR_CUDA;
    float best_ms = -1.0f;
    qh_opts best = base;
    int nc = 0;
    for (size_t ci = 0;; ci++) {
        if (ci == nshape && best_ms >= 0.0f) {
            // second stage: the small-cloud threshold at the fastest shape
            for (int sc : {0, 64, 256, 1024, 4096})
                if (sc != best.small_cloud)
                    cands.push_back({best.block, best.items, best.blocks_per_sm, sc});
        }
        if (ci >= cands.size()) break;
        const Cand c = cands[ci];
        qh_opts o = base;
        o.block = c.block;
        o.items = c.items;
        o.blocks_per_sm = c.bps;
        o.small_cloud = c.small;
        bool good = true;
        std::vector<float> ms;
        for (int r = 0; r <= reps && good; r++) {
            if (r > 0 && cudaEventRecord(E.ev[r - 1], st) != cudaSuccess) return QH_ERR_CUDA;
            const qh_status s = qh_hull3d_batched(d_x, d_y, d_z, stride, d_cloud_off, ncloud, n,
                                                  d_verts, d_cloud_vert_off, d_face_off,
                                                  d_face_idx, d_cloud_face_off, d_cloud_status,
                                                  d_result, d_ws, ws_bytes, &o, st);
            if (s == QH_ERR_INVALID_ARG || s == QH_ERR_NOMEM) return s;
            if (s != QH_OK) {
                good = false;
                break;
            }
            if (r > 0) {
                if (cudaEventRecord(E.ev[r], st) != cudaSuccess) return QH_ERR_CUDA;
                if (cudaEventSynchronize(E.ev[r]) != cudaSuccess) return QH_ERR_CUDA;
                float t = 0.0f;
                if (cudaEventElapsedTime(&t, E.ev[r - 1], E.ev[r]) != cudaSuccess)
                    return QH_ERR_CUDA;
                ms.push_back(t);
            }
            qh_result res;
            if (cudaMemcpyAsync(&res, d_result, sizeof(res), cudaMemcpyDeviceToHost, st) !=
                    cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess)
                return QH_ERR_CUDA;
            if (res.status != QH_OK) good = false;
        }
        if (!good) continue;
        std::sort(ms.begin(), ms.end());
        const float med = ms[ms.size() / 2];
        if (nc < max_cand) {
            h_ms[nc] = med;
            h_shape[4 * nc + 0] = c.block;
            h_shape[4 * nc + 1] = c.items;
            h_shape[4 * nc + 2] = c.bps;
            h_shape[4 * nc + 3] = c.small;
        }
        nc++;
        if (best_ms < 0.0f || med < best_ms) {
            best_ms = med;
            best = o;
        }
    }
    *h_ncand = std::min(nc, max_cand);
    if (best_ms < 0.0f) return QH_ERR_CUDA;
    *h_best = best;
    return QH_OK;
}
