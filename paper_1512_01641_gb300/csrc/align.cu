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
#include "kernels.h"

namespace gbm {
namespace {

constexpr int kFillWarps = 4;
constexpr int kTailWarps = 4;

// Bounded wait for a nonzero tile flag.
__device__ bool wait_flag(const int32_t *f, int64_t limit) {
    for (int64_t it = 0; it < limit; ++it) {
        if (ld_acquire(f) != 0) return true;
        __nanosleep(200);
    }
    return false;
}

struct FillCtx {
    int lane, N, M, c0, c1, r;
    bool rv;
    float two_p;
    SimRow row;
    SimConst k;
    const uchar2 *rowp;   // counts of row r
    const int64_t *tsent; // target sentence offsets of the pair
    SimCol *colv;         // shared: per-column similarity constants of the current block
    DevParams P;
};

// One 32-column block iteration of a strip sweep.  cur receives the
// similarities of block jb (rotated); prev holds block jb-1.  rc/rp are the
// 64-bit traceback registers of this and the previous iteration.
__device__ __forceinline__ void fill_block(const FillCtx &C, int jb, int nb, bool first_strip,
                                           const float *__restrict__ hrow, float *__restrict__ hrow_w,
                                           float (&cur)[32], const float (&prev)[32], uint64_t &rc,
                                           const uint64_t &rp, float &a_down, float &b,
                                           uint64_t *__restrict__ tb_strip) {
    const int lane = C.lane;
    const int col_base = C.c0 + 32 * jb;
    const bool lane_col = col_base + lane < C.c1;
    // UP candidates of the first row of the strip for the 32 columns of this block
    const float hv = first_strip ? -C.two_p : (lane_col ? __ldcg(hrow + col_base + lane) : 0.0f);
    if (jb < nb) {
        __syncwarp();
        C.colv[lane] = sim_col(lane_col ? (int)(C.tsent[col_base + lane + 1] - C.tsent[col_base + lane]) : 1, C.P);
        __syncwarp();
#pragma unroll
        for (int x = 0; x < 32; ++x) {
            const int c = (x - lane) & 31;
            const int col = col_base + c;
            float v = 0.0f;
            if (C.rv && col < C.c1) {
                const uchar2 q = C.rowp[col];
                v = similarity(q.x, q.y, C.row, C.colv[c], C.k);
            }
            cur[x] = v;
        }
    }
    rc = 0;
#pragma unroll
    for (int u = 0; u < 32; ++u) {
        float a_up = __shfl_up_sync(kFull, a_down, 1);
        const float h0 = __shfl_sync(kFull, hv, u);
        if (lane == 0) a_up = h0;
        const int j = col_base + u - lane;
        const float sv = (u >= lane) ? cur[u] : prev[u];
        if (C.rv && j >= C.c0 && j < C.c1) {
            const float d = fmaxf(fmaxf(sv, a_up), b);
            const uint64_t bits = (d == a_up) ? (uint64_t)kUp << (2 * u)
                                              : ((d == b) ? (uint64_t)kLeft << (2 * u) : 0ull);
            rc |= bits;
            const float e = __fsub_rn(d, C.two_p);
            const float nb2 = __fsub_rn(e, a_up);
            a_down = __fsub_rn(e, b);
            b = nb2;
            if (lane == 31) __stcg(hrow_w + j, a_down);
        }
    }
    // the word of block jb-1 is complete: its columns came at steps u >= lane
    // of iteration jb-1 and u < lane of iteration jb
    if (jb > 0) {
        const int sh = 2 * lane;
        const uint64_t w = (rp >> sh) | (sh ? (rc << (64 - sh)) : 0ull);
        tb_strip[(int64_t)((C.c0 >> 5) + jb - 1) * 32 + lane] = w;
    }
}

__global__ void __launch_bounds__(32 * kFillWarps)
fill_kernel(DevCorpus src, DevCorpus tgt, const PairGeom *__restrict__ geom,
            const FillItem *__restrict__ items, int64_t n_items, DevParams P,
            const uint8_t *__restrict__ counts, AlignScratch S, int64_t wait_limit) {
    __shared__ SimCol colv_all[kFillWarps][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    FillCtx C;
    C.lane = lane;
    C.P = P;
    C.two_p = __fadd_rn(P.gap, P.gap);
    C.k = sim_const(P);
    C.colv = colv_all[warp];
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
        const int nb = (C.c1 - C.c0 + 31) >> 5;
        const int64_t sbase = src.doc[w.pair];
        C.tsent = tgt.sent + tgt.doc[w.pair];
        float *hrow = S.hrow + g.hrow_off;
        for (int s = w.s0; s < w.s1; ++s) {
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
            C.r = 32 * s + lane;
            C.rv = C.r < C.N;
            const int ls = C.rv ? (int)(src.sent[sbase + C.r + 1] - src.sent[sbase + C.r]) : 1;
            C.row = sim_row(ls, P);
            C.rowp = reinterpret_cast<const uchar2 *>(counts) + g.cell_off + (int64_t)C.r * C.M;
            float b = -C.two_p;
            if (C.c0 > 0 && C.rv) b = __ldcg(S.vcol + g.vcol_off + C.r);
            float a_down = 0.0f;
            float A[32], B[32];
#pragma unroll
            for (int x = 0; x < 32; ++x) B[x] = 0.0f;
            uint64_t RA = 0, RB = 0;
            uint64_t *tb_strip = S.tb + g.tb_off + (int64_t)s * nblk_pair * 32;
            for (int jb = 0; jb <= nb; jb += 2) {
                fill_block(C, jb, nb, s == 0, hrow, hrow, A, B, RA, RB, a_down, b, tb_strip);
                if (jb + 1 > nb) break;
                fill_block(C, jb + 1, nb, s == 0, hrow, hrow, B, A, RB, RA, a_down, b, tb_strip);
            }
            if (tiled) {
                if (C.c1 < C.M && C.rv) __stcg(S.vcol + g.vcol_off + C.r, b);
                __threadfence();
                __syncwarp();
                if (lane == 0) st_release(S.flags + g.flag_off + (int64_t)s * g.nchunk + w.cj, 1);
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
walk_kernel(const PairGeom *__restrict__ geom, int64_t n_pairs, AlignScratch S) {
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t k = warp0; k < n_pairs; k += nwarps) {
        const PairGeom g = geom[k];
        const int N = g.n, M = g.m;
        const int nblk = (M + 31) >> 5;
        const int cap = min(N, M);
        const uint64_t *tbp = S.tb + g.tb_off;
        int i = N, j = M, n = 0;
        int bs = -1, bj = -1;  // strip and column block held in `word`
        uint64_t word = 0;
        while (i > 0 && j > 0) {
            const int rr = i - 1, cc = j - 1;
            if ((rr >> 5) != bs || (cc >> 5) != bj) {
                bs = rr >> 5;
                bj = cc >> 5;
                word = tbp[((int64_t)bs * nblk + bj) * 32 + lane];
            }
            const uint64_t wr = __shfl_sync(kFull, word, rr & 31);
            const uint32_t code = (uint32_t)(wr >> (2 * (cc & 31))) & 3u;
            if (code == kUp) {
                --i;
            } else if (code == kLeft) {
                --j;
            } else {
                if (lane == 0) {
                    const int64_t at = g.link_off + cap - 1 - n;
                    S.diag_i[at] = rr;
                    S.diag_j[at] = cc;
                }
                ++n;
                --i;
                --j;
            }
        }
        if (lane == 0) S.n_diag[k] = n;
    }
}

// Exclusive scan of int32 counts into int64 offsets (one block; n is at most a
// few hundred thousand, so a strided serial pass per thread is enough).
__global__ void __launch_bounds__(1024)
scan_kernel(const int32_t *__restrict__ in, int64_t n, int64_t *__restrict__ out) {
    __shared__ int64_t part[1024];
    const int t = threadIdx.x;
    const int64_t chunk = (n + 1023) / 1024;
    const int64_t a = t * chunk, b = min(n, a + chunk);
    int64_t sum = 0;
    for (int64_t x = a; x < b; ++x) sum += in[x];
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
        out[x] = run;
        run += in[x];
    }
    if (t == 1023) out[n] = part[1023];
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

// Similarity of every diagonal cell of every path, one warp per cell, by the
// same helper the fill used.  The counts come from the cached per-cell counts
// when given, else they are recounted by warp vote from the tokens.
__global__ void __launch_bounds__(32 * kTailWarps)
link_score_kernel(DevCorpus src, DevCorpus tgt, DevDict dict, const PairGeom *__restrict__ geom,
                  int64_t n_pairs, DevParams P, AlignScratch S, const uint8_t *__restrict__ counts) {
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t total = S.diag_off[n_pairs];
    const SimConst K = sim_const(P);
    for (int64_t f = warp0; f < total; f += nwarps) {
        // pair owning flat diagonal f: last k with diag_off[k] <= f
        int64_t lo = 0, hi = n_pairs - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (S.diag_off[mid] <= f) lo = mid; else hi = mid - 1;
        }
        const int64_t k = lo;
        const PairGeom g = geom[k];
        const int nd = S.n_diag[k];
        const int64_t at = g.link_off + min(g.n, g.m) - nd + (f - S.diag_off[k]);
        const int rr = S.diag_i[at], cc = S.diag_j[at];
        const int64_t sb = src.doc[k] + rr, tbs = tgt.doc[k] + cc;
        const int64_t s0 = src.sent[sb], s1 = src.sent[sb + 1];
        const int64_t t0 = tgt.sent[tbs], t1 = tgt.sent[tbs + 1];
        int ms, mt;
        if (counts) {
            const uchar2 q = reinterpret_cast<const uchar2 *>(counts)[g.cell_off + (int64_t)rr * g.m + cc];
            ms = q.x;
            mt = q.y;
        } else {
            ballot_counts(src.tok + s0, (int)(s1 - s0), tgt.tok + t0, (int)(t1 - t0), dict, lane, ms, mt);
        }
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
        double sum = 0.0;
        int kept = 0;
        for (int x = lane; x < nd; x += 32) {
            const float s = S.diag_s[base + x];
            sum += (double)s;
            kept += s >= P.thr;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            sum += __shfl_xor_sync(kFull, sum, off);
            kept += __shfl_xor_sync(kFull, kept, off);
        }
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
        int64_t to = link_off[k];
        for (int x0 = 0; x0 < nd; x0 += 32) {
            const int x = x0 + lane;
            const bool in = x < nd;
            const float s = in ? S.diag_s[base + x] : 0.0f;
            const bool keep = in && s >= P.thr;
            const uint32_t m = __ballot_sync(kFull, keep);
            if (keep) {
                const int64_t o = to + __popc(m & ((1u << lane) - 1u));
                out_i[o] = S.diag_i[base + x];
                out_j[o] = S.diag_j[base + x];
                out_s[o] = s;
            }
            to += __popc(m);
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
                        const uint8_t *counts, const AlignScratch &S, int64_t wait_limit,
                        int n_sms, cudaStream_t st) {
    if (n_items == 0) return cudaSuccess;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fill_kernel, 32 * kFillWarps, 0);
    if (e != cudaSuccess) return e;
    int64_t blocks = (int64_t)n_sms * (per_sm > 0 ? per_sm : 1);
    const int64_t want = (n_items + kFillWarps - 1) / kFillWarps;
    if (blocks > want) blocks = want;
    e = cudaMemsetAsync(S.queue, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    fill_kernel<<<(unsigned)blocks, 32 * kFillWarps, 0, st>>>(src, tgt, geom, items, n_items, P, counts, S,
                                                               wait_limit);
    return cudaGetLastError();
}

cudaError_t launch_walk(const PairGeom *geom, int64_t n_pairs, const AlignScratch &S, int n_sms,
                        cudaStream_t st) {
    if (n_pairs == 0) return cudaSuccess;
    walk_kernel<<<tail_grid(n_pairs, n_sms), 32 * kTailWarps, 0, st>>>(geom, n_pairs, S);
    return cudaGetLastError();
}

cudaError_t launch_scan(const int32_t *in, int64_t n, int64_t *out, cudaStream_t st) {
    scan_kernel<<<1, 1024, 0, st>>>(in, n, out);
    return cudaGetLastError();
}

cudaError_t launch_link_score(const DevCorpus &src, const DevCorpus &tgt, const DevDict &dict,
                              const PairGeom *geom, int64_t n_pairs, const DevParams &P,
                              const AlignScratch &S, const uint8_t *counts, int n_sms, cudaStream_t st) {
    if (n_pairs == 0) return cudaSuccess;
    link_score_kernel<<<n_sms * 16, 32 * kTailWarps, 0, st>>>(src, tgt, dict, geom, n_pairs, P, S, counts);
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

cudaError_t launch_score(const DevCorpus &src, const DevCorpus &tgt, const PairGeom *geom,
                         int64_t n_pairs, const DevParams &P, const uint8_t *counts, float *s,
                         float *feat, cudaStream_t st) {
    if (n_pairs == 0) return cudaSuccess;
    score_kernel<<<(unsigned)n_pairs, 256, 0, st>>>(src, tgt, geom, P, counts, s, feat);
    return cudaGetLastError();
}

}  // namespace gbm
