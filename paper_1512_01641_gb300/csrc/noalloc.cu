// Allocation-free alignment of one document pair.
//
// Some callers cannot allocate device memory at call time: code running
// between the steps of a serving loop with a fixed memory budget, libraries
// embedded in a host framework that owns every device allocation, or code
// that must not pay cudaMalloc's implicit device synchronisation.  For them,
// mine_align_pair_noalloc aligns one pair without a plan and without any
// allocation: its scratch (traceback codes, boundary row, path cells) lives
// in one file-scope device array of fixed size, which every GPU that loads
// the library keeps until the process exits.
//
// The kernel runs, in one warp, the same device code as the batched path: the
// strip sweep of the fill, the register-blocked walk, the similarity of the
// path's cells from the cached counts, the FP64 pair sum and the compaction
// of the kept links; its results are bit-identical to mine_align's.
#include <mutex>

#include "fill.cuh"
#include "kernels.h"
#include "miner.h"

namespace gbm {
namespace {

constexpr int kMaxSide = MINE_NOALLOC_MAX_SIDE;
constexpr int64_t kMaxStrips = (kMaxSide + 31) / 32;
constexpr int64_t kTbWords = kMaxStrips * kMaxStrips * 32;  // uint64 traceback words
constexpr int64_t kScratchBytes = kTbWords * 8 + (int64_t)kMaxSide * 4 + 3 * (int64_t)kMaxSide * 4;

// The shared scratch of every call (see the header: overlapping calls race).
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

__global__ void __launch_bounds__(32)
align_pair_static_kernel(const int64_t *__restrict__ ssent, const int64_t *__restrict__ tsent, int N, int M,
                         const uint8_t *__restrict__ counts, DevParams P, unsigned char *__restrict__ scratch,
                         int32_t *__restrict__ link_i, int32_t *__restrict__ link_j, float *__restrict__ link_s,
                         int32_t *__restrict__ n_links, float *__restrict__ pair_score) {
    __shared__ SimCol colv[32];
    __shared__ __align__(16) unsigned char stage[2][32][kStageBytes];
    __shared__ uint64_t stage_bar[2];
    __shared__ uint32_t status;  // timeout bit of the staging waits
    const int lane = threadIdx.x;
    if (lane == 0) status = 0u;
    __syncwarp();
    const int nstrips = (N + 31) >> 5, nblk = (M + 31) >> 5;
    const int cap = min(N, M);
    uint64_t *tb = reinterpret_cast<uint64_t *>(scratch);
    float *hrow = reinterpret_cast<float *>(tb + (int64_t)nstrips * nblk * 32);
    int32_t *diag_i = reinterpret_cast<int32_t *>(hrow + M);
    int32_t *diag_j = diag_i + cap;
    float *diag_s = reinterpret_cast<float *>(diag_j + cap);

    if (N > 0 && M > 0) {
        FillCtx C;
        C.lane = lane;
        C.P = P;
        C.two_p = __fadd_rn(P.gap, P.gap);
        C.k = sim_const(P);
        C.colv = colv;
        C.counts = counts;
        C.counts_bytes = 2 * (int64_t)N * M;
        C.stage = stage;
        C.stage_bar = stage_bar;
        C.status = &status;
        C.blocked = false;
        fill_stage_init(C);
        C.N = N;
        C.M = M;
        C.c0 = 0;
        C.c1 = M;
        C.tsent = tsent;
        for (int s = 0; s < nstrips; ++s) {
            (void)fill_strip(C, s, ssent, counts, 0, hrow, tb, nblk, -C.two_p);
            __syncwarp();
        }
    }
    __syncwarp();
    const int nd = walk_pair(tb, N, M, lane, diag_i + cap, diag_j + cap);
    __syncwarp();
    const SimConst K = sim_const(P);
    const int64_t base = cap - nd;
    for (int x = lane; x < nd; x += 32) {
        const int i = diag_i[base + x], j = diag_j[base + x];
        const uchar2 q = reinterpret_cast<const uchar2 *>(counts)[(int64_t)i * M + j];
        diag_s[base + x] = similarity(q.x, q.y, sim_row((int)(ssent[i + 1] - ssent[i]), P),
                                      sim_col((int)(tsent[j + 1] - tsent[j]), P), K);
    }
    __syncwarp();
    double sum;
    int kept;
    pair_sum_warp(diag_s + base, nd, P.thr, lane, sum, kept);
    copy_kept_warp(diag_i + base, diag_j + base, diag_s + base, nd, P.thr, lane, link_i, link_j, link_s);
    __syncwarp();
    if (lane == 0) {
        if (status != 0u) {  // a staging wait gave up: the results are invalid
            *n_links = -1;
            *pair_score = __int_as_float(0x7fc00000);
        } else {
            *n_links = kept;
            *pair_score = (float)(sum - (double)P.gap * (double)(N + M - 2 * nd));
        }
    }
}

// Device address of the scratch array, looked up once per device (with that
// device current) and cached.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};

cudaError_t scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace gbm

extern "C" int mine_align_pair_noalloc(const int64_t *src_sent_off, const int64_t *tgt_sent_off, int32_t n,
                                       int32_t m, const uint8_t *counts, const mine_params *params,
                                       int32_t *link_i, int32_t *link_j, float *link_s, int32_t *n_links,
                                       float *pair_score, miner_stream_t stream) {
    using namespace gbm;
    if (!params || !n_links || !pair_score || n < 0 || m < 0) return MINE_EINVAL;
    if (n > kMaxSide || m > kMaxSide) return MINE_EINVAL;
    if ((n > 0 && !src_sent_off) || (m > 0 && !tgt_sent_off)) return MINE_EINVAL;
    if ((int64_t)n * m > 0 && !counts) return MINE_EINVAL;
    if (n > 0 && m > 0 && (!link_i || !link_j || !link_s)) return MINE_EINVAL;
    void *scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) {
        record_cuda_error((int)e);
        return MINE_ECUDA;
    }
    align_pair_static_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(src_sent_off, tgt_sent_off, n, m, counts,
                                                                 to_dev(*params), (unsigned char *)scratch,
                                                                 link_i, link_j, link_s, n_links, pair_score);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        record_cuda_error((int)e);
        return MINE_ECUDA;
    }
    return MINE_OK;
}
