// Needleman-Wunsch alignment of sentence sequences (Section 5.1, Eq. 1),
// traceback with the acceptance threshold (Section 4 / 5.2), link compaction,
// and the unfused similarity path (Section 4).
//
// The fill works on differences instead of absolute H values.  With
//   a(i,j) = H(i-1,j) - H(i-1,j-1) - p   (UP candidate, relative)
//   b(i,j) = H(i,j-1) - H(i-1,j-1) - p   (LEFT candidate, relative)
//   d(i,j) = H(i,j)   - H(i-1,j-1)       = max(s_ij, a, b)
// the next candidates are b(i,j+1) = d - a - 2p and a(i+1,j) = d - b - 2p, and
// the borders H(i,0) = -i p, H(0,j) = -j p give a = b = -2p on row 1 and
// column 1.  Every value stays within a few units of zero, so FP32 keeps
// ~1e-7 absolute precision however large the matrix (an absolute H of 5000
// would only keep ~5e-4), and the comparisons that pick the path are made on
// exactly the quantities the definition compares, shifted by a common term.
// H(N,M) itself is the score of the chosen path, summed in FP64 during the
// traceback.
//
// One warp owns a pair and sweeps it in strips of 32 rows (lane = row),
// skewed by one column per lane so that lane i handles column t - i at step
// t (the anti-diagonal wavefront of Figure 2, 32 cells wide); a(i,j) comes
// from the lane above by a register shuffle, and the last lane's outputs
// seed the next strip through a per-pair boundary row.
#include "kernels.h"

namespace gbm {
namespace {

constexpr int kAlignWarps = 4;

__global__ void __launch_bounds__(32 * kAlignWarps)
nw_counts_kernel(DevCorpus src, DevCorpus tgt, const PairGeom *__restrict__ geom,
                 const int32_t *__restrict__ order, int64_t n_pairs, DevParams P,
                 const uint8_t *__restrict__ counts, uint64_t *__restrict__ tb,
                 float *__restrict__ hrow) {
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const float p = P.gap;
    const float two_p = __fadd_rn(p, p);
    for (int64_t it = warp0; it < n_pairs; it += nwarps) {
        const int32_t k = order[it];
        const PairGeom g = geom[k];
        const int N = g.n, M = g.m;
        if (N == 0 || M == 0) continue;
        const int nblk = (M + 31) >> 5;
        const int64_t sbase = src.doc[k], tbase = tgt.doc[k];
        float *hb = hrow + g.hrow_off;
        uint64_t *tbp = tb + g.tb_off;
        const int nstrips = (N + 31) >> 5;
        for (int s = 0; s < nstrips; ++s) {
            const int r = 32 * s + lane;
            const bool rv = r < N;
            const int ls = rv ? (int)(src.sent[sbase + r + 1] - src.sent[sbase + r]) : 1;
            const uchar2 *crow = reinterpret_cast<const uchar2 *>(counts) + g.cell_off + (int64_t)r * M;
            float b = -two_p, a_down = 0.0f;
            uint64_t acc = 0;
            for (int t = 0; t < M + 31; ++t) {
                float a_up = __shfl_up_sync(kFull, a_down, 1);
                const int j = t - lane;
                if (lane == 0) a_up = (s == 0) ? -two_p : (t < M ? hb[t] : 0.0f);
                if (rv && j >= 0 && j < M) {
                    const uchar2 c = crow[j];
                    const int lt = (int)(tgt.sent[tbase + j + 1] - tgt.sent[tbase + j]);
                    const float sv = similarity(c.x, c.y, ls, lt, P);
                    const float d = fmaxf(fmaxf(sv, a_up), b);
                    const uint32_t code = (d == a_up) ? kUp : ((d == b) ? kLeft : kDiag);
                    const float e = __fsub_rn(d, two_p);
                    const float nb = __fsub_rn(e, a_up);
                    a_down = __fsub_rn(e, b);
                    b = nb;
                    acc |= (uint64_t)code << (2 * (j & 31));
                    if ((j & 31) == 31 || j == M - 1) {
                        tbp[((int64_t)s * nblk + (j >> 5)) * 32 + lane] = acc;
                        acc = 0;
                    }
                    if (lane == 31) hb[j] = a_down;
                }
            }
            __syncwarp();
        }
    }
}

// (ms, mt) of one cell by warp vote: lanes hold target positions (in chunks
// of 32); every dictionary translation of every source position is compared
// with all of them in one ballot.
__device__ __forceinline__ void ballot_counts(const int32_t *__restrict__ stok, int ls,
                                              const int32_t *__restrict__ ttok, int lt,
                                              const DevDict &dict, int lane, int &ms, int &mt) {
    const int nch = (lt + 31) >> 5;
    int32_t tq[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) tq[c] = (c < nch && c * 32 + lane < lt) ? ttok[c * 32 + lane] : -1;
    uint32_t hitq = 0;
    int msc = 0;
    for (int p = 0; p < ls; ++p) {
        const int32_t v = stok[p];
        uint32_t any = 0;
        for (int32_t e = dict.off[v]; e < dict.off[v + 1]; ++e) {
            const int32_t t = dict.tgt[e];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                if (c < nch) {
                    const bool eq = tq[c] == t;
                    any |= __ballot_sync(kFull, eq);
                    hitq |= eq ? (1u << c) : 0u;
                }
            }
        }
        msc += any != 0u;
    }
    int mtc = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c)
        if (c < nch) mtc += __popc(__ballot_sync(kFull, (hitq >> c) & 1u));
    ms = msc;
    mt = mtc;
}

// Walk back from (N,M) to (0,0) (one warp per pair).  A DIAG step links the
// cell; its counts are recomputed by warp vote and its similarity by the same
// function the fill used, and the link is kept iff s >= thr.  The path score
// (= H(N,M)) is summed in FP64.  Kept links land at the END of the pair's
// capacity window, so that they read in ascending order.
__global__ void __launch_bounds__(32 * kAlignWarps)
traceback_kernel(DevCorpus src, DevCorpus tgt, DevDict dict, const PairGeom *__restrict__ geom,
                 int64_t n_pairs, DevParams P, const uint64_t *__restrict__ tb,
                 int32_t *__restrict__ scr_i, int32_t *__restrict__ scr_j, float *__restrict__ scr_s,
                 int32_t *__restrict__ n_links, float *__restrict__ pair_score) {
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t k = warp0; k < n_pairs; k += nwarps) {
        const PairGeom g = geom[k];
        const int N = g.n, M = g.m;
        const int nblk = (M + 31) >> 5;
        const int cap = min(N, M);
        const int64_t sbase = src.doc[k], tbase = tgt.doc[k];
        const uint64_t *tbp = tb + g.tb_off;
        int i = N, j = M, n = 0;
        double score = 0.0;
        int64_t cached = -1;
        uint64_t word = 0;
        while (i > 0 || j > 0) {
            uint32_t code;
            if (i == 0) {
                code = kLeft;
            } else if (j == 0) {
                code = kUp;
            } else {
                const int rr = i - 1, cc = j - 1;
                const int64_t widx = ((int64_t)(rr >> 5) * nblk + (cc >> 5)) * 32 + (rr & 31);
                if (widx != cached) {
                    word = tbp[widx];
                    cached = widx;
                }
                code = (uint32_t)(word >> (2 * (cc & 31))) & 3u;
            }
            if (code == kDiag) {
                const int rr = i - 1, cc = j - 1;
                const int64_t s0 = src.sent[sbase + rr], s1 = src.sent[sbase + rr + 1];
                const int64_t t0 = tgt.sent[tbase + cc], t1 = tgt.sent[tbase + cc + 1];
                int ms, mt;
                ballot_counts(src.tok + s0, (int)(s1 - s0), tgt.tok + t0, (int)(t1 - t0), dict, lane, ms, mt);
                const float sv = similarity(ms, mt, (int)(s1 - s0), (int)(t1 - t0), P);
                score += (double)sv;
                if (sv >= P.thr) {
                    if (lane == 0) {
                        const int64_t at = g.link_off + cap - 1 - n;
                        scr_i[at] = rr;
                        scr_j[at] = cc;
                        scr_s[at] = sv;
                    }
                    ++n;
                }
                --i;
                --j;
            } else {
                score -= (double)P.gap;
                if (code == kUp) --i; else --j;
            }
        }
        if (lane == 0) {
            n_links[k] = n;
            pair_score[k] = (float)score;
        }
    }
}

// Exclusive scan of the per-pair link counts (one block; the pair count is a
// few hundred thousand at most, so a strided serial pass per thread is enough).
__global__ void __launch_bounds__(1024)
scan_kernel(const int32_t *__restrict__ n_links, int64_t n_pairs, int64_t *__restrict__ link_off) {
    __shared__ int64_t part[1024];
    const int t = threadIdx.x;
    const int64_t chunk = (n_pairs + 1023) / 1024;
    const int64_t a = t * chunk, b = min(n_pairs, a + chunk);
    int64_t sum = 0;
    for (int64_t x = a; x < b; ++x) sum += n_links[x];
    part[t] = sum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        int64_t v = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int64_t run = part[t] - sum;
    for (int64_t x = a; x < b; ++x) {
        link_off[x] = run;
        run += n_links[x];
    }
    if (t == 1023) link_off[n_pairs] = part[1023];
}

__global__ void __launch_bounds__(32 * kAlignWarps)
copy_links_kernel(const PairGeom *__restrict__ geom, int64_t n_pairs, const int32_t *__restrict__ n_links,
                  const int32_t *__restrict__ scr_i, const int32_t *__restrict__ scr_j,
                  const float *__restrict__ scr_s, const int64_t *__restrict__ link_off,
                  int32_t *__restrict__ out_i, int32_t *__restrict__ out_j, float *__restrict__ out_s) {
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t k = warp0; k < n_pairs; k += nwarps) {
        const PairGeom g = geom[k];
        const int n = n_links[k];
        const int cap = min(g.n, g.m);
        const int64_t from = g.link_off + cap - n, to = link_off[k];
        for (int x = lane; x < n; x += 32) {
            out_i[to + x] = scr_i[from + x];
            out_j[to + x] = scr_j[from + x];
            out_s[to + x] = scr_s[from + x];
        }
    }
}

// Unfused similarity of every cell from counts (one block per pair).
__global__ void __launch_bounds__(256)
score_kernel(DevCorpus src, DevCorpus tgt, const PairGeom *__restrict__ geom, DevParams P,
             const uint8_t *__restrict__ counts, float *__restrict__ s, float *__restrict__ feat) {
    const int64_t k = blockIdx.x;
    const PairGeom g = geom[k];
    const int64_t sbase = src.doc[k], tbase = tgt.doc[k];
    const int64_t cells = (int64_t)g.n * g.m;
    for (int64_t c = threadIdx.x; c < cells; c += blockDim.x) {
        const int i = (int)(c / g.m), j = (int)(c % g.m);
        const int ls = (int)(src.sent[sbase + i + 1] - src.sent[sbase + i]);
        const int lt = (int)(tgt.sent[tbase + j + 1] - tgt.sent[tbase + j]);
        const int ms = counts[2 * (g.cell_off + c)], mt = counts[2 * (g.cell_off + c) + 1];
        s[g.cell_off + c] = similarity(ms, mt, ls, lt, P);
        if (feat) {
            float f[4];
            features(ms, mt, ls, lt, f);
#pragma unroll
            for (int q = 0; q < 4; ++q) feat[4 * (g.cell_off + c) + q] = f[q];
        }
    }
}

int grid_for(int64_t warps_wanted, int warps_per_block, int n_sms, int per_sm) {
    int64_t blocks = (warps_wanted + warps_per_block - 1) / warps_per_block;
    int64_t cap = (int64_t)n_sms * per_sm;
    if (blocks > cap) blocks = cap;
    return (int)(blocks < 1 ? 1 : blocks);
}

}  // namespace

cudaError_t launch_nw_counts(const DevCorpus &src, const DevCorpus &tgt, const PairGeom *geom,
                             const int32_t *order, int64_t n_pairs, const DevParams &P,
                             const uint8_t *counts, uint64_t *tb, float *hrow, int n_sms,
                             cudaStream_t st) {
    if (n_pairs == 0) return cudaSuccess;
    int grid = grid_for(n_pairs, kAlignWarps, n_sms, 16);
    nw_counts_kernel<<<grid, 32 * kAlignWarps, 0, st>>>(src, tgt, geom, order, n_pairs, P, counts, tb, hrow);
    return cudaGetLastError();
}

cudaError_t launch_traceback(const DevCorpus &src, const DevCorpus &tgt, const DevDict &dict,
                             const PairGeom *geom, int64_t n_pairs, const DevParams &P,
                             const uint64_t *tb, int32_t *scr_i, int32_t *scr_j, float *scr_s,
                             int32_t *n_links, float *pair_score, cudaStream_t st) {
    if (n_pairs == 0) return cudaSuccess;
    int dev = 0, n_sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sms, cudaDevAttrMultiProcessorCount, dev);
    int grid = grid_for(n_pairs, kAlignWarps, n_sms, 16);
    traceback_kernel<<<grid, 32 * kAlignWarps, 0, st>>>(src, tgt, dict, geom, n_pairs, P, tb, scr_i, scr_j,
                                                        scr_s, n_links, pair_score);
    return cudaGetLastError();
}

cudaError_t launch_scan(const int32_t *n_links, int64_t n_pairs, int64_t *link_off, cudaStream_t st) {
    scan_kernel<<<1, 1024, 0, st>>>(n_links, n_pairs, link_off);
    return cudaGetLastError();
}

cudaError_t launch_copy_links(const PairGeom *geom, int64_t n_pairs, const int32_t *n_links,
                              const int32_t *scr_i, const int32_t *scr_j, const float *scr_s,
                              const int64_t *link_off, int32_t *out_i, int32_t *out_j, float *out_s,
                              cudaStream_t st) {
    if (n_pairs == 0) return cudaSuccess;
    int dev = 0, n_sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sms, cudaDevAttrMultiProcessorCount, dev);
    int grid = grid_for(n_pairs, kAlignWarps, n_sms, 16);
    copy_links_kernel<<<grid, 32 * kAlignWarps, 0, st>>>(geom, n_pairs, n_links, scr_i, scr_j, scr_s, link_off,
                                                         out_i, out_j, out_s);
    return cudaGetLastError();
}

cudaError_t launch_score(const DevCorpus &src, const DevCorpus &tgt, const PairGeom *geom,
                         int64_t n_pairs, const DevParams &P, const uint8_t *counts, float *s,
                         float *feat, cudaStream_t st) {
    if (n_pairs == 0) return cudaSuccess;
    score_kernel<<<(unsigned)n_pairs, 256, 0, st>>>(src, tgt, geom, P, counts, s, feat);
    return cudaGetLastError();
}

}  // namespace gbm
