// The device steps of one hull over several ranks (conv(P) = conv of the
// union of the shards' hulls): each rank's shard-hull indices packed into a
// fixed-size block for the all-gather, the gathered candidates' coordinates
// collected into one candidate cloud per input cloud, and the final hull's
// candidate-local indices mapped back to global indices.
//
// Candidate order: rank blocks in rank order, each rank's candidates as its
// shard hull lists them.  Coincident points keep their lowest index: inside a
// shard the shard hull already keeps only the lowest, and across shards the
// earlier rank block holds the lower global index, so the final hull's
// lowest-local-index rule picks the lowest global index.  Unused slots of a
// block repeat the cloud's first candidate (same point, same global index).
#include <climits>
#include <cstdint>

#include "qh_internal.h"

namespace qh {
namespace shard {

constexpr int kMaxK = 64;
constexpr int kMaxDim = 3;
constexpr int kBlock = 256;

// A rank block of cloud c: words [0] count, [1, 1 + cap) global indices,
// then dim runs of cap coordinates (float bits): (1 + dim * ... ) words.
__host__ __device__ __forceinline__ long long block_words(int dim, int cap)
{
    return 1 + (long long)(1 + dim) * cap;
}

struct LocalArgs {
    int k, dim, cap;
    long long stride;
    const int32_t *out[kMaxK];
    long long lo[kMaxK];
    const float *coord[kMaxK][kMaxDim];  // the shard's coordinates (shard-local index)
};

// block[c]: count (the shard hull's size; minus the status for a failed
// shard), lo + local index j and the point's coordinates for
// j < min(count, cap).  A count above cap is kept as is: the pack reports it.
__global__ void k_local(LocalArgs A, const qh_result *res, int32_t *block)
{
    const int c = blockIdx.y;
    int st = res[c].status;
    // an empty shard may come without coordinates; a shard with points may not
    bool have = true;
    for (int d = 0; d < A.dim; d++) have = have && A.coord[c][d] != nullptr;
    if (st == 0 && res[c].count > 0 && !have) st = QH_ERR_INVALID_ARG;
    const long long cnt = st == 0 ? res[c].count : 0;
    int32_t *b = block + (long long)c * block_words(A.dim, A.cap);
    if (blockIdx.x == 0 && threadIdx.x == 0) b[0] = st == 0 ? (int32_t)cnt : -st;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < cnt && j < A.cap;
         j += (long long)gridDim.x * blockDim.x) {
        const int32_t l = A.out[c][j];
        b[1 + j] = (int32_t)(l + A.lo[c]);
        for (int d = 0; d < A.dim; d++)
            b[1 + (long long)(1 + d) * A.cap + j] =
                __float_as_int(A.coord[c][d][(long long)l * A.stride]);
    }
}

// gathered[r][c] (rank r's block of cloud c) -> candidate cloud c: slot
// r * cap + j holds rank r's j-th candidate, or the cloud's first candidate
// when j >= that rank's count.  ccoord[d][c][m], cidx[c][m] with
// m = world * cap.  bad[c]: the first failed rank's status, or
// QH_ERR_CAPACITY for a count above cap.
__global__ void k_pack(int k, int dim, int world, int cap, const int32_t *gathered,
                       float *ccoord, int32_t *cidx, int32_t *bad)
{
    const int c = blockIdx.y;
    const long long m = (long long)world * cap, bw = block_words(dim, cap), blk = k * bw;
    __shared__ int first_r, first_j;
    if (threadIdx.x == 0) {
        first_r = -1;
        first_j = 0;
        for (int r = 0; r < world; r++) {
            const int32_t cnt = gathered[r * blk + c * bw];
            if (cnt < 0) atomicCAS(&bad[c], 0, -cnt);
            if (cnt > cap) atomicCAS(&bad[c], 0, (int32_t)QH_ERR_CAPACITY);
            if (first_r < 0 && cnt > 0) first_r = r;
        }
    }
    __syncthreads();
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < m;
         s += (long long)gridDim.x * blockDim.x) {
        int r = (int)(s / cap), j = (int)(s - (long long)r * cap);
        const int cnt = min(max(gathered[r * blk + c * bw], 0), cap);
        if (j >= cnt) {
            r = first_r;
            j = first_j;
        }
        if (r < 0) {
            cidx[c * m + s] = -1;
            for (int d = 0; d < dim; d++) ccoord[((long long)d * k + c) * m + s] = 0.f;
            continue;
        }
        const int32_t *b = gathered + r * blk + c * bw;
        cidx[c * m + s] = b[1 + j];
        for (int d = 0; d < dim; d++)
            ccoord[((long long)d * k + c) * m + s] = __int_as_float(b[1 + (long long)(1 + d) * cap + j]);
    }
}

struct RemapArgs {
    int k;
    long long m;
    int32_t *out[kMaxK];
};

// out[c][i] = cidx[c][out[c][i]] for the final hull's count entries
__global__ void k_remap(RemapArgs A, const qh_result *res, const int32_t *cidx)
{
    const int c = blockIdx.y;
    const long long cnt = res[c].status == 0 ? res[c].count : 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (long long)gridDim.x * blockDim.x) {
        const int32_t l = A.out[c][i];
        A.out[c][i] = (l >= 0 && l < A.m) ? cidx[c * A.m + l] : -1;
    }
}

static int grid_x(long long items)
{
    const long long g = (items + kBlock - 1) / kBlock;
    return (int)(g < 1 ? 1 : (g > 1024 ? 1024 : g));
}

}  // namespace shard
}  // namespace qh

using namespace qh::shard;

extern "C" int64_t qh_shard_block_words(int32_t dim, int32_t cap)
{
    if (dim < 2 || dim > kMaxDim || cap < 1) return 0;
    return block_words(dim, cap);
}

extern "C" qh_status qh_shard_local(int32_t k, int32_t dim, const int32_t *const *h_dout,
                                    const void *d_results, const int64_t *h_lo,
                                    const float *const *h_dcoord, int64_t stride, int32_t cap,
                                    int32_t *d_block, cudaStream_t st)
{
    if (k < 1 || k > kMaxK || dim < 2 || dim > kMaxDim || cap < 1 || stride < 1 || !h_dout ||
        !d_results || !h_lo || !h_dcoord || !d_block)
        return QH_ERR_INVALID_ARG;
    LocalArgs A = {};
    A.k = k;
    A.dim = dim;
    A.cap = cap;
    A.stride = stride;
    for (int c = 0; c < k; c++) {
        if (!h_dout[c] || h_lo[c] < 0) return QH_ERR_INVALID_ARG;
        A.out[c] = h_dout[c];
        A.lo[c] = h_lo[c];
        for (int d = 0; d < dim; d++) A.coord[c][d] = h_dcoord[c * dim + d];  // null: empty shard
    }
    k_local<<<dim3(grid_x(cap), k), kBlock, 0, st>>>(A, (const qh_result *)d_results, d_block);
    return cudaGetLastError() == cudaSuccess ? QH_OK : QH_ERR_CUDA;
}

extern "C" qh_status qh_shard_pack(int32_t k, int32_t dim, const int32_t *d_gathered,
                                   int32_t world, int32_t cap, float *d_ccoord, int32_t *d_cidx,
                                   int32_t *d_bad, cudaStream_t st)
{
    if (k < 1 || k > kMaxK || dim < 2 || dim > kMaxDim || world < 1 || cap < 1 ||
        (long long)world * cap > INT_MAX || !d_gathered || !d_ccoord || !d_cidx || !d_bad)
        return QH_ERR_INVALID_ARG;
    k_pack<<<dim3(grid_x((long long)world * cap), k), kBlock, 0, st>>>(
        k, dim, world, cap, d_gathered, d_ccoord, d_cidx, d_bad);
    return cudaGetLastError() == cudaSuccess ? QH_OK : QH_ERR_CUDA;
}

extern "C" qh_status qh_shard_remap(int32_t k, int32_t *const *h_dout, const void *d_results,
                                    const int32_t *d_cidx, int64_t m, cudaStream_t st)
{
    if (k < 1 || k > kMaxK || m < 1 || !h_dout || !d_results || !d_cidx)
        return QH_ERR_INVALID_ARG;
    RemapArgs A = {};
    A.k = k;
    A.m = m;
    for (int c = 0; c < k; c++) {
        if (!h_dout[c]) return QH_ERR_INVALID_ARG;
        A.out[c] = h_dout[c];
    }
    k_remap<<<dim3(grid_x(m), k), kBlock, 0, st>>>(A, (const qh_result *)d_results, d_cidx);
    return cudaGetLastError() == cudaSuccess ? QH_OK : QH_ERR_CUDA;
}
