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
// H(N,M) itself is the score of the chosen path, summed in FP64 after the
// traceback.
//
// Fill: a warp owns 32 rows (lane = row) and sweeps columns with a skew of one
// column per lane, so lane i handles column t - i at step t -- the
// anti-diagonal wavefront of Figure 2, 32 cells wide.  a(i,j) comes from the
// lane above through a register shuffle; the last lane's outputs seed the next
// strip through a boundary row.  Similarities of a 32 x 32 block are computed
// before its 32 DP steps, into registers in a rotated order (value for column
// c of lane i sits at index (c + i) mod 32) so that step u reads register u
// in every lane; the DP chain then carries only max/compare/add per step.
// A small pair is one work item (all its strips, all columns).  A large pair
// is cut into 32-row x cw-column tiles, each its own work item; a tile waits
// (bounded) on the completion flags of the tile above and the tile to its
// left, whose boundary row/column it reads from global memory.  Work items are
// handed out by an atomic counter in the planner's order.
#include "fill.cuh"
#include "kernels.h"

namespace gbm {
namespace {

constexpr int kFillWarps = 4;
constexpr int kTailWarps = 4;

// Bounded wait for a nonzero tile flag.
__device__ bool wait_flag(const int32_t *f, int64_t limit) {
    for (int64_t it = 0; it < limit; ++it) {
        if (ld_relaxed(f) != 0) return true;  // the caller acquires
        __nanosleep(200);
    }
    return false;
}

__global__ void __launch_bounds__(32 * kFillWarps, 4)
fill_kernel(DevCorpus src, DevCorpus tgt, const PairGeom *__restrict__ geom,
            const FillItem *__restrict__ items, int64_t n_items, DevParams P,
            const uint8_t *__restrict__ counts, int64_t counts_bytes, bool blocked, AlignScratch S,
            int64_t wait_limit, int64_t skip_flag) {
    __shared__ SimCol colv_all[kFillWarps][32];
    __shared__ __align__(16) unsigned char stage_all[kFillWarps][2][32][kStageBytes];
    __shared__ uint64_t bar_all[kFillWarps][2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    FillCtx C;
    C.lane = lane;
    C.P = P;
    C.two_p = __fadd_rn(P.gap, P.gap);
    C.k = sim_const(P);
    C.colv = colv_all[warp];
    C.counts = counts;
    C.counts_bytes = counts_bytes;
    C.stage = stage_all[warp];
    C.stage_bar = bar_all[warp];
    C.status = S.status;
    C.blocked = blocked;
    fill_stage_init(C);
    for (;;) {
        int64_t it = 0;
        if (lane == 0) it = atomicAdd(S.queue, 1);
        it = __shfl_sync(kFull, it, 0);
        if (it >= n_items) break;
        const FillItem w = items[it];
        const PairGeom g = geom[w.pair];
        C.N = g.n;
        C.M = g.m;
        if (C.N == 0 || C.M == 0) continue;
        C.c0 = w.cj * g.cw;
        C.c1 = min(C.M, C.c0 + g.cw);
        const bool tiled = g.flag_off >= 0;
        const int nblk_pair = (C.M + 31) >> 5;
        const int64_t sbase = src.doc[w.pair];
        C.tsent = tgt.sent + tgt.doc[w.pair];
        float *hrow = S.hrow + g.hrow_off;
        for (int s = w.s0; s < w.s1; ++s) {
            // the loads that do not depend on the neighbouring tiles go out
            // before the wait for them
            FillAhead ah;
            int nb;
            fill_strip_prepare(C, s, src.sent + sbase, g.cell_off, ah, nb, g.tb_off);
            if (tiled) {
                if (lane == 0) {
                    bool ok = true;
                    if (s > 0) ok &= wait_flag(S.flags + g.flag_off + (int64_t)(s - 1) * g.nchunk + w.cj, wait_limit);
                    if (w.cj > 0) ok &= wait_flag(S.flags + g.flag_off + (int64_t)s * g.nchunk + w.cj - 1, wait_limit);
                    if (!ok) atomicOr(S.status, kStTimeout);
                }
                __syncwarp();
                if (s > 0) (void)ld_acquire(S.flags + g.flag_off + (int64_t)(s - 1) * g.nchunk + w.cj);
                if (w.cj > 0) (void)ld_acquire(S.flags + g.flag_off + (int64_t)s * g.nchunk + w.cj - 1);
            }
            float b = -C.two_p;
            if (C.c0 > 0 && 32 * s + lane < C.N) b = __ldcg(S.vcol + g.vcol_off + 32 * s + lane);
            b = fill_strip_run(C, s, hrow, S.tb + g.tb_off, nblk_pair, b, ah, nb);
            if (tiled) {
                if (C.c1 < C.M && C.rv) __stcg(S.vcol + g.vcol_off + C.r, b);
                __threadfence();
                __syncwarp();
                const int64_t fi = g.flag_off + (int64_t)s * g.nchunk + w.cj;
                if (lane == 0 && fi != skip_flag) st_release(S.flags + fi, 1);
            } else {
                __syncwarp();
            }
        }
    }
}

// Walk back from (N,M) to (0,0), one warp per pair.  The 32 x 32 block of
// traceback codes around the current cell sits in registers (lane l holds the
// word of row l of the block), so a step costs a shuffle; leaving the block
// loads the next one with one coalesced 256-byte read.  Diagonal cells are
// written to the END of the pair's link window in ascending order.
__global__ void __launch_bounds__(32 * kTailWarps)
walk_kernel(const PairGeom *__restrict__ geom, const int32_t *__restrict__ order, int64_t n_pairs, AlignScratch S) {
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // largest pairs first: their serial walks start at once and run beside
    // the many short ones instead of after them
    for (int64_t x = warp0; x < n_pairs; x += nwarps) {
        const int32_t k = order[x];
        const PairGeom g = geom[k];
        const int N = g.n, M = g.m;
        const int cap = min(N, M);
        const int n = walk_pair(S.tb + g.tb_off, N, M, lane, S.diag_i + g.link_off + cap,
                                S.diag_j + g.link_off + cap);
        if (lane == 0) S.n_diag[k] = n;
    }
}

// Exclusive scan of int32 counts into int64 offsets, out[n] = total (one
// block; n is at most a few hundred thousand).  Tiles of 1024 consecutive
// counts: coalesced loads, warp scans by shuffle, a scan of the 32 warp
// totals, and a running carry from tile to tile.
template <typename OutT>
__global__ void __launch_bounds__(1024)
scan_kernel(const int32_t *__restrict__ in, int64_t n, OutT *__restrict__ out) {
    __shared__ int64_t wsum[32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    int64_t carry = 0;
    for (int64_t base = 0; base < n; base += 1024) {
        const int64_t x = base + t;
        const int64_t v = x < n ? (int64_t)in[x] : 0;
        int64_t s = v;  // inclusive scan within the warp
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int64_t y = __shfl_up_sync(kFull, s, off);
            if (lane >= off) s += y;
        }
        if (lane == 31) wsum[w] = s;
        __syncthreads();
        if (w == 0) {
            int64_t ws = wsum[lane];
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int64_t y = __shfl_up_sync(kFull, ws, off);
                if (lane >= off) ws += y;
            }
            wsum[lane] = ws;  // inclusive over warps
        }
        __syncthreads();
        if (x < n) out[x] = (OutT)(carry + (w > 0 ? wsum[w - 1] : 0) + s - v);
        carry += wsum[31];
        __syncthreads();  // wsum is rewritten by the next tile
    }
    if (t == 0) out[n] = (OutT)carry;
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

// Similarity of every diagonal cell of every path, by the same helper the fill
// used.  From the cached per-cell counts one thread handles a cell; without
// them (link recount) one warp per cell recounts the overlaps by warp vote.
__device__ __forceinline__ int64_t owner_pair(const int64_t *__restrict__ diag_off, int64_t n_pairs, int64_t f) {
    int64_t lo = 0, hi = n_pairs - 1;  // last k with diag_off[k] <= f
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (diag_off[mid] <= f) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(32 * kTailWarps)
link_score_cached_kernel(DevCorpus src, DevCorpus tgt, const PairGeom *__restrict__ geom, int64_t n_pairs,
                         DevParams P, AlignScratch S, const uint8_t *__restrict__ counts, bool blocked) {
    const int64_t total = S.diag_off[n_pairs];
    const SimConst K = sim_const(P);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < total; f += stride) {
        const int64_t k = owner_pair(S.diag_off, n_pairs, f);
        const PairGeom g = geom[k];
        const int64_t at = g.link_off + min(g.n, g.m) - S.n_diag[k] + (f - S.diag_off[k]);
        const int rr = S.diag_i[at], cc = S.diag_j[at];
        const int64_t sb = src.doc[k] + rr, tbs = tgt.doc[k] + cc;
        const int ls = (int)(src.sent[sb + 1] - src.sent[sb]), lt = (int)(tgt.sent[tbs + 1] - tgt.sent[tbs]);
        const int64_t cell = blocked ? 32 * g.tb_off + 1024 * ((int64_t)(rr >> 5) * ((g.m + 31) >> 5) + (cc >> 5)) +
                                           32 * (rr & 31) + (cc & 31)
                                     : g.cell_off + (int64_t)rr * g.m + cc;
        const uchar2 q = reinterpret_cast<const uchar2 *>(counts)[cell];
        S.diag_s[at] = similarity(q.x, q.y, sim_row(ls, P), sim_col(lt, P), K);
    }
}

__global__ void __launch_bounds__(32 * kTailWarps)
link_score_kernel(DevCorpus src, DevCorpus tgt, DevDict dict, const PairGeom *__restrict__ geom,
                  int64_t n_pairs, DevParams P, AlignScratch S) {
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t total = S.diag_off[n_pairs];
    const SimConst K = sim_const(P);
    for (int64_t f = warp0; f < total; f += nwarps) {
        const int64_t k = owner_pair(S.diag_off, n_pairs, f);
        const PairGeom g = geom[k];
        const int nd = S.n_diag[k];
        const int64_t at = g.link_off + min(g.n, g.m) - nd + (f - S.diag_off[k]);
        const int rr = S.diag_i[at], cc = S.diag_j[at];
        const int64_t sb = src.doc[k] + rr, tbs = tgt.doc[k] + cc;
        const int64_t s0 = src.sent[sb], s1 = src.sent[sb + 1];
        const int64_t t0 = tgt.sent[tbs], t1 = tgt.sent[tbs + 1];
        int ms, mt;
        ballot_counts(src.tok + s0, (int)(s1 - s0), tgt.tok + t0, (int)(t1 - t0), dict, lane, ms, mt);
        if (lane == 0)
            S.diag_s[at] = similarity(ms, mt, sim_row((int)(s1 - s0), P), sim_col((int)(t1 - t0), P), K);
    }
}

// Per pair: H(N,M) = sum of the path's similarities (FP64, fixed order) minus
// p per gap step, and the number of kept links (s >= thr).
__global__ void __launch_bounds__(32 * kTailWarps)
pair_sum_kernel(const PairGeom *__restrict__ geom, int64_t n_pairs, DevParams P, AlignScratch S,
                float *__restrict__ pair_score) {
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t k = warp0; k < n_pairs; k += nwarps) {
        const PairGeom g = geom[k];
        const int nd = S.n_diag[k];
        const int64_t base = g.link_off + min(g.n, g.m) - nd;
        double sum;
        int kept;
        pair_sum_warp(S.diag_s + base, nd, P.thr, lane, sum, kept);
        if (lane == 0) {
            const int gaps = g.n + g.m - 2 * nd;
            pair_score[k] = (float)(sum - (double)P.gap * (double)gaps);
            S.n_links[k] = kept;
        }
    }
}

// Kept links of each pair, compacted in ascending order at link_off[k].
__global__ void __launch_bounds__(32 * kTailWarps)
copy_links_kernel(const PairGeom *__restrict__ geom, int64_t n_pairs, DevParams P, AlignScratch S,
                  const int64_t *__restrict__ link_off, int32_t *__restrict__ out_i,
                  int32_t *__restrict__ out_j, float *__restrict__ out_s) {
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t k = warp0; k < n_pairs; k += nwarps) {
        const PairGeom g = geom[k];
        const int nd = S.n_diag[k];
        const int64_t base = g.link_off + min(g.n, g.m) - nd;
        copy_kept_warp(S.diag_i + base, S.diag_j + base, S.diag_s + base, nd, P.thr, lane, out_i + link_off[k],
                       out_j + link_off[k], out_s + link_off[k]);
    }
}

// Link quality against gold links (one 0/1 byte per cell): per pair, the
// number of links that are gold; plus the number of links and of gold cells.
// One warp per pair, integer sums (exact).
__global__ void __launch_bounds__(32 * kTailWarps)
link_gold_kernel(const PairGeom *__restrict__ geom, int64_t n_pairs, const int64_t *__restrict__ link_off,
                 const int32_t *__restrict__ li, const int32_t *__restrict__ lj, const uint8_t *__restrict__ gold,
                 unsigned long long *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long tp = 0, ng = 0, nl = 0;
    for (int64_t k = warp0; k < n_pairs; k += nwarps) {
        const PairGeom g = geom[k];
        for (int64_t x = link_off[k] + lane; x < link_off[k + 1]; x += 32) {
            tp += gold[g.cell_off + (int64_t)li[x] * g.m + lj[x]];
            ++nl;
        }
        const int64_t cells = (int64_t)g.n * g.m;
        for (int64_t c = lane; c < cells; c += 32) ng += gold[g.cell_off + c];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        tp += __shfl_xor_sync(kFull, tp, off);
        ng += __shfl_xor_sync(kFull, ng, off);
        nl += __shfl_xor_sync(kFull, nl, off);
    }
    if (lane == 0) {
        atomicAdd(out + 0, tp);
        atomicAdd(out + 1, nl);
        atomicAdd(out + 2, ng);
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
    const SimConst K = sim_const(P);
    for (int64_t c = threadIdx.x; c < cells; c += blockDim.x) {
        const int i = (int)(c / g.m), j = (int)(c % g.m);
        const int ls = (int)(src.sent[sbase + i + 1] - src.sent[sbase + i]);
        const int lt = (int)(tgt.sent[tbase + j + 1] - tgt.sent[tbase + j]);
        const int ms = counts[2 * (g.cell_off + c)], mt = counts[2 * (g.cell_off + c) + 1];
        s[g.cell_off + c] = similarity(ms, mt, sim_row(ls, P), sim_col(lt, P), K);
        if (feat) {
            float f[4];
            features(ms, mt, ls, lt, f);
#pragma unroll
            for (int q = 0; q < 4; ++q) feat[4 * (g.cell_off + c) + q] = f[q];
        }
    }
}

int tail_grid(int64_t warps_wanted, int n_sms) {
    int64_t blocks = (warps_wanted + kTailWarps - 1) / kTailWarps;
    int64_t cap = (int64_t)n_sms * 16;
    if (blocks > cap) blocks = cap;
    return (int)(blocks < 1 ? 1 : blocks);
}

}  // namespace

cudaError_t launch_fill(const DevCorpus &src, const DevCorpus &tgt, const PairGeom *geom,
                        const FillItem *items, int64_t n_items, const DevParams &P,
                        const uint8_t *counts, int64_t counts_bytes, bool blocked, const AlignScratch &S,
                        int64_t wait_limit, int64_t skip_flag, int n_sms, cudaStream_t st) {
    if (n_items == 0) return cudaSuccess;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fill_kernel, 32 * kFillWarps, 0);
    if (e != cudaSuccess) return e;
    int64_t blocks = (int64_t)n_sms * (per_sm > 0 ? per_sm : 1);
    const int64_t want = (n_items + kFillWarps - 1) / kFillWarps;
    if (blocks > want) blocks = want;
    e = cudaMemsetAsync(S.queue, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    fill_kernel<<<(unsigned)blocks, 32 * kFillWarps, 0, st>>>(src, tgt, geom, items, n_items, P, counts,
                                                               counts_bytes, blocked, S, wait_limit, skip_flag);
    return cudaGetLastError();
}

cudaError_t launch_walk(const PairGeom *geom, const int32_t *order, int64_t n_pairs, const AlignScratch &S,
                        int n_sms, cudaStream_t st) {
    if (n_pairs == 0) return cudaSuccess;
    walk_kernel<<<tail_grid(n_pairs, n_sms), 32 * kTailWarps, 0, st>>>(geom, order, n_pairs, S);
    return cudaGetLastError();
}

cudaError_t launch_scan(const int32_t *in, int64_t n, int64_t *out, cudaStream_t st) {
    scan_kernel<int64_t><<<1, 1024, 0, st>>>(in, n, out);
    return cudaGetLastError();
}

cudaError_t launch_scan32(const int32_t *in, int64_t n, int32_t *out, cudaStream_t st) {
    scan_kernel<int32_t><<<1, 1024, 0, st>>>(in, n, out);
    return cudaGetLastError();
}

cudaError_t launch_link_score(const DevCorpus &src, const DevCorpus &tgt, const DevDict &dict,
                              const PairGeom *geom, int64_t n_pairs, const DevParams &P,
                              const AlignScratch &S, const uint8_t *counts, bool blocked, int n_sms,
                              cudaStream_t st) {
    if (n_pairs == 0) return cudaSuccess;
    if (counts)
        link_score_cached_kernel<<<n_sms * 8, 32 * kTailWarps, 0, st>>>(src, tgt, geom, n_pairs, P, S, counts,
                                                                         blocked);
    else
        link_score_kernel<<<n_sms * 16, 32 * kTailWarps, 0, st>>>(src, tgt, dict, geom, n_pairs, P, S);
    return cudaGetLastError();
}

cudaError_t launch_pair_sum(const PairGeom *geom, int64_t n_pairs, const DevParams &P,
                            const AlignScratch &S, float *pair_score, int n_sms, cudaStream_t st) {
    if (n_pairs == 0) return cudaSuccess;
    pair_sum_kernel<<<tail_grid(n_pairs, n_sms), 32 * kTailWarps, 0, st>>>(geom, n_pairs, P, S, pair_score);
    return cudaGetLastError();
}

cudaError_t launch_copy_links(const PairGeom *geom, int64_t n_pairs, const DevParams &P,
                              const AlignScratch &S, const int64_t *link_off, int32_t *out_i,
                              int32_t *out_j, float *out_s, int n_sms, cudaStream_t st) {
    if (n_pairs == 0) return cudaSuccess;
    copy_links_kernel<<<tail_grid(n_pairs, n_sms), 32 * kTailWarps, 0, st>>>(geom, n_pairs, P, S, link_off,
                                                                             out_i, out_j, out_s);
    return cudaGetLastError();
}

cudaError_t launch_link_gold(const PairGeom *geom, int64_t n_pairs, const int64_t *link_off, const int32_t *li,
                             const int32_t *lj, const uint8_t *gold, unsigned long long *out, int n_sms,
                             cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out, 0, 3 * sizeof(unsigned long long), st);
    if (e != cudaSuccess || n_pairs == 0) return e;
    link_gold_kernel<<<tail_grid(n_pairs, n_sms), 32 * kTailWarps, 0, st>>>(geom, n_pairs, link_off, li, lj, gold,
                                                                            out);
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
