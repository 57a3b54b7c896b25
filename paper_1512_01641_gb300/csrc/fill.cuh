// Device building blocks of the Needleman-Wunsch fill and traceback, shared
// by the batched kernels (align.cu) and the allocation-free single-pair
// variant (noalloc.cu), so that both run the same arithmetic.
#pragma once

#include "common.cuh"

namespace gbm {

// Bytes of one lane's staged count segment: 32 cells (64 bytes) inside
// their 16-byte-aligned cover.
constexpr int kStageBytes = 80;
constexpr int64_t kStageWaitLimit = 1 << 22;

struct FillCtx {
    int lane, N, M, c0, c1, r;
    bool rv;
    float two_p;
    SimRow row;
    SimConst k;
    const int64_t *tsent; // target sentence offsets of the pair
    SimCol *colv;         // shared: per-column similarity constants of the current block
    DevParams P;
    // staging of the count bytes (per warp, double-buffered by block parity)
    const uint8_t *counts;      // the whole counts array ...
    int64_t counts_bytes;       // ... and its length (a cover never reads past it)
    int64_t row_byte;           // byte offset of row r's first cell in counts
    unsigned char (*stage)[32][kStageBytes];  // shared [2][lane][byte]
    uint64_t *stage_bar;        // shared [2] mbarriers, 32 arrivals each
    uint32_t stage_phase;       // bit b: parity of buffer b's next completion
    int stage_off0, stage_off1; // byte offset of the segment in the lane's staged row, per buffer
    uint32_t *status;           // timeout bit (may be null)
    bool blocked;               // counts in the blocked layout: row_byte is the strip's first tile,
                                // block b of the pair at row_byte + 2048 b, row r at byte 64 r
};

// Per-warp setup of the staging barriers (lane 0 initialises, all lanes
// wait at the __syncwarp that follows).
__device__ __forceinline__ void fill_stage_init(FillCtx &C) {
    if (C.lane == 0) {
        mbar_init(C.stage_bar, 32);
        mbar_init(C.stage_bar + 1, 32);
    }
    C.stage_phase = 0;
    C.stage_off0 = C.stage_off1 = 0;
    __syncwarp();
}

// Start staging block jb's count bytes into buffer jb & 1: every lane copies
// its own row's 64 bytes with one bulk async copy of their cover aligned to
// 16-byte ADDRESSES (the array itself may start anywhere), or with plain
// loads when that cover would reach outside the array; then it arrives on
// the buffer's barrier.
__device__ __forceinline__ void fill_stage(FillCtx &C, int jb, int nb) {
    if (jb >= nb) return;
    const int buf = jb & 1;
    const int col_base = C.c0 + 32 * jb;
    const int ncol = min(32, C.c1 - col_base);
    uint64_t *bar = C.stage_bar + buf;
    if (C.blocked) {
        // the block's 32 rows are one aligned 2 KB tile: one copy for the warp
        if (C.lane == 0)
            bulk_copy_g2s(C.stage[buf], C.counts + C.row_byte + 2048 * (int64_t)(col_base >> 5), 2048u, bar);
        else
            mbar_arrive(bar);
        return;
    }
    unsigned char *dst = C.stage[buf][C.lane];
    int off = 0;
    if (C.rv) {
        const uintptr_t base = reinterpret_cast<uintptr_t>(C.counts);
        const uintptr_t a = base + (uintptr_t)(C.row_byte + 2 * (int64_t)col_base);
        const uintptr_t a16 = a & ~(uintptr_t)15, e16 = (a + 2 * ncol + 15) & ~(uintptr_t)15;
        off = (int)(a - a16);
        if (a16 >= base && e16 <= base + (uintptr_t)C.counts_bytes) {
            bulk_copy_g2s(dst, reinterpret_cast<const void *>(a16), (uint32_t)(e16 - a16), bar);
        } else {
            const uint8_t *src = reinterpret_cast<const uint8_t *>(a);
            for (int t = 0; t < 2 * ncol; ++t) dst[off + t] = src[t];
            mbar_arrive(bar);
        }
    } else {
        mbar_arrive(bar);
    }
    if (buf) C.stage_off1 = off;
    else C.stage_off0 = off;
}

// Wait until block jb's staged bytes have landed; returns the lane's row.
__device__ __forceinline__ const unsigned char *fill_stage_wait(FillCtx &C, int jb) {
    const int buf = jb & 1;
    if (!mbar_wait(C.stage_bar + buf, (C.stage_phase >> buf) & 1u, kStageWaitLimit) && C.status)
        atomicOr(C.status, kStTimeout);
    C.stage_phase ^= 1u << buf;
    if (C.blocked) return &C.stage[buf][0][0] + 64 * C.lane;
    return C.stage[buf][C.lane] + (buf ? C.stage_off1 : C.stage_off0);
}

// Values of the next block, loaded one block ahead so that their global
// latency overlaps the current block's sweep.
struct FillAhead {
    float hv;  // UP candidate of the strip's first row at this lane's column
    int lt;    // length of this lane's target sentence
};

// Loads the look-ahead values of block jb.
__device__ __forceinline__ void fill_ahead_hv(const FillCtx &C, int jb, int nb, bool first_strip,
                                              const float *__restrict__ hrow, FillAhead &A) {
    const int col = C.c0 + 32 * jb + C.lane;
    const bool in = jb < nb && col < C.c1;
    A.hv = first_strip ? -C.two_p : (in ? __ldcg(hrow + col) : 0.0f);
}
__device__ __forceinline__ void fill_ahead_lt(const FillCtx &C, int jb, int nb, FillAhead &A) {
    const int col = C.c0 + 32 * jb + C.lane;
    const bool in = jb < nb && col < C.c1;
    A.lt = in ? (int)(C.tsent[col + 1] - C.tsent[col]) : 1;
}
__device__ __forceinline__ void fill_ahead(const FillCtx &C, int jb, int nb, bool first_strip,
                                           const float *__restrict__ hrow, FillAhead &A) {
    fill_ahead_hv(C, jb, nb, first_strip, hrow, A);
    fill_ahead_lt(C, jb, nb, A);
}

// One 32-column block iteration of a strip sweep.  cur receives the
// similarities of block jb (rotated); prev holds block jb-1.  rc/rp are the
// 64-bit traceback registers of this and the previous iteration.  A holds
// block jb's look-ahead values on entry and block jb+1's on return.
__device__ __forceinline__ void fill_block(FillCtx &C, int jb, int nb, bool first_strip,
                                           const float *__restrict__ hrow, float *__restrict__ hrow_w,
                                           float (&cur)[32], const float (&prev)[32], uint64_t &rc,
                                           const uint64_t &rp, float &a_down, float &b,
                                           uint64_t *__restrict__ tb_strip, FillAhead &A) {
    const int lane = C.lane;
    const int col_base = C.c0 + 32 * jb;
    // UP candidates of the first row of the strip for the 32 columns of this block
    const float hv = A.hv;
    if (jb < nb) {
        __syncwarp();
        C.colv[lane] = sim_col(A.lt, C.P);
        __syncwarp();
        fill_ahead(C, jb + 1, nb, first_strip, hrow, A);
        fill_stage(C, jb + 1, nb);
        const unsigned char *st = fill_stage_wait(C, jb);
        // branch-free, so that the 32 independent cells overlap: every cell
        // is computed from the staged row (in bounds for any c); a cell
        // outside the pair gets a finite value from stale bytes, which only
        // feeds steps whose results are discarded
#pragma unroll
        for (int x = 0; x < 32; ++x) {
            const int c = (x - lane) & 31;
            const uint32_t q16 = *reinterpret_cast<const uint16_t *>(st + 2 * c);
            cur[x] = similarity_q16(q16, C.row, C.colv[c], C.k);
        }
    }
    uint32_t rup = 0u, rleft = 0u;
    // the cell of step u is column j = jl + u + c0 of this lane's row; it
    // exists when 0 <= jl + u < width (width 0 for a row below the pair)
    const int jl = col_base - lane - C.c0;
    const uint32_t width = C.rv ? (uint32_t)(C.c1 - C.c0) : 0u;
    float *const hrow_at = hrow_w + C.c0 + jl;  // lane 31 stores column j at hrow_at[u]
#pragma unroll
    for (int u = 0; u < 32; ++u) {
        float a_up = __shfl_up_sync(kFull, a_down, 1);
        const float h0 = __shfl_sync(kFull, hv, u);
        if (lane == 0) a_up = h0;
        const float sv = (u >= lane) ? cur[u] : prev[u];
        // branch-free step: computed in every lane, committed where the cell
        // exists (the skew leaves lanes outside the pair at both ends).  Only
        // one max waits for the shuffled value.  a_down needs no commit: a
        // lane's output of an invalid step reaches the next lane only at a
        // step where that lane is invalid too (before its first column, after
        // its last, or below the last row).  Nor do the code bits: those of
        // an invalid cell land in a word that is never stored (before the
        // first block) or at a cell the walk never visits.
        const bool valid = (uint32_t)(jl + u) < width;
        const float d = fmaxf(fmaxf(sv, b), a_up);
        rup |= eq_mask(d, a_up) & (1u << u);
        rleft |= eq_mask(d, b) & (1u << u);
        const float e = __fsub_rn(d, C.two_p);
        const float nb2 = __fsub_rn(e, a_up);
        a_down = __fsub_rn(e, b);
        b = valid ? nb2 : b;
        if (valid && lane == 31) __stcg(hrow_at + u, a_down);
    }
    rc = ((uint64_t)rleft << 32) | rup;
    // the word of block jb-1 is complete: its columns came at steps u >= lane
    // of iteration jb-1 and u < lane of iteration jb
    if (jb > 0) {
        const uint32_t wu = __funnelshift_r((uint32_t)rp, rup, lane);
        const uint32_t wl = __funnelshift_r((uint32_t)(rp >> 32), rleft, lane);
        tb_strip[(int64_t)((C.c0 >> 5) + jb - 1) * 32 + lane] = ((uint64_t)wl << 32) | wu;
    }
}


// First part of the sweep of strip s over columns [C.c0, C.c1): everything
// that does not depend on the strip above or the tile to the left -- row
// constants, block 0's target sentence lengths and the staging of its count
// bytes -- so that a tile can start these loads before it waits for its
// neighbours.  nb receives the number of 32-column blocks.
__device__ __forceinline__ void fill_strip_prepare(FillCtx &C, int s, const int64_t *__restrict__ ssent,
                                                   int64_t cell_off, FillAhead &ah, int &nb, int64_t tb_off = 0) {
    const int lane = C.lane;
    C.r = 32 * s + lane;
    C.rv = C.r < C.N;
    const int ls = C.rv ? (int)(ssent[C.r + 1] - ssent[C.r]) : 1;
    C.row = sim_row(ls, C.P);
    C.row_byte = C.blocked ? 64 * tb_off + 2048 * (int64_t)s * ((C.M + 31) >> 5)
                           : 2 * (cell_off + (int64_t)C.r * C.M);
    nb = (C.c1 - C.c0 + 31) >> 5;
    fill_ahead_lt(C, 0, nb, ah);
    fill_stage(C, 0, nb);
}

// The sweep itself, once the strip's boundaries are complete.  b0 holds the
// LEFT candidates of column c0 (-2p at the left border); returns each lane's
// LEFT candidate after the last column.  hrow holds the UP candidates of the
// row above the strip and receives those of the strip's last row (lane 31
// writes column j at the step after every lane has read it: block jb reads
// columns 32 jb .. 32 jb + 31 one block ahead, and lane 31 reaches them only
// in blocks jb and jb + 1).
__device__ __forceinline__ float fill_strip_run(FillCtx &C, int s, float *__restrict__ hrow,
                                                uint64_t *__restrict__ tb_pair, int nblk_pair, float b0,
                                                FillAhead &ah, int nb) {
    float b = b0, a_down = 0.0f;
    float A[32], B[32];
#pragma unroll
    for (int x = 0; x < 32; ++x) B[x] = 0.0f;
    uint64_t RA = 0, RB = 0;
    uint64_t *tb_strip = tb_pair + (int64_t)s * nblk_pair * 32;
    fill_ahead_hv(C, 0, nb, s == 0, hrow, ah);
    // one instance of the (fully unrolled) block body: the current block's
    // similarities become the previous block's by a register copy, which
    // keeps the loop's code half the size of two alternating instances
#pragma unroll 1
    for (int jb = 0; jb <= nb; ++jb) {
        fill_block(C, jb, nb, s == 0, hrow, hrow, A, B, RA, RB, a_down, b, tb_strip, ah);
#pragma unroll
        for (int x = 0; x < 32; ++x) B[x] = A[x];
        RB = RA;
    }
    return b;
}

// Sweep strip s (rows 32s..32s+31) over columns [C.c0, C.c1) in one go.
__device__ __forceinline__ float fill_strip(FillCtx &C, int s, const int64_t *__restrict__ ssent,
                                            const uint8_t *__restrict__ counts, int64_t cell_off,
                                            float *__restrict__ hrow, uint64_t *__restrict__ tb_pair,
                                            int nblk_pair, float b0) {
    (void)counts;  // read through C.counts (staged)
    FillAhead ah;
    int nb;
    fill_strip_prepare(C, s, ssent, cell_off, ah, nb);
    return fill_strip_run(C, s, hrow, tb_pair, nblk_pair, b0, ah, nb);
}

// Walk back from (N, M) to the border along the traceback codes (UP before
// LEFT before DIAG, as the fill recorded them), one warp per pair, and write
// the diagonal cells to the END of the pair's link window in ascending order
// (diag_*_end[-1] is the last); returns their number.  The 32 x 32 block of
// codes around the current cell sits in registers (lane l holds the word of
// row l of the block); leaving the block loads the next one with one
// coalesced 256-byte read.  A gap step costs a shuffle; a run of diagonal
// steps is taken at once: every lane reads the code of its own row's cell on
// the current diagonal, and a ballot finds where the run meets a cell that is
// not DIAG or the block's edge -- the cells the one-step walk would visit, in
// the same order.
__device__ __forceinline__ int walk_pair(const uint64_t *__restrict__ tbp, int N, int M, int lane,
                                         int32_t *diag_i_end, int32_t *diag_j_end) {
    const int nblk = (M + 31) >> 5;
    int i = N, j = M, n = 0;
    int bs = -1, bj = -1;
    uint64_t word = 0;
    while (i > 0 && j > 0) {
        const int rr = i - 1, cc = j - 1;
        if ((rr >> 5) != bs || (cc >> 5) != bj) {
            bs = rr >> 5;
            bj = cc >> 5;
            word = tbp[((int64_t)bs * nblk + bj) * 32 + lane];
            // the walk leaves this block into the one above, to the left or
            // above-left: start bringing their two 128-byte lines into L1
            if (lane < 6) {
                const int c = lane >> 1;
                const int pbs = bs - (c != 1), pbj = bj - (c != 0);
                if (pbs >= 0 && pbj >= 0) prefetch_l1(tbp + ((int64_t)pbs * nblk + pbj) * 32 + 16 * (lane & 1));
            }
        }
        const uint64_t wr = __shfl_sync(kFull, word, rr & 31);
        if ((wr >> (cc & 31)) & 1u) {  // UP
            --i;
        } else if ((wr >> (32 + (cc & 31))) & 1u) {  // LEFT
            --j;
        } else {
            // diagonal run from (rr, cc) upwards: lane l's cell on it is
            // (32 bs + l, cc - t) with t = rr - (32 bs + l) steps from here
            const int top = rr & 31;
            const int t = top - lane;
            const int cl = cc - t;
            bool stop = true;  // the run cannot pass this lane's cell
            if (t >= 0 && cl >= 32 * bj) stop = (((word >> (cl & 31)) | (word >> (32 + (cl & 31)))) & 1u) != 0;
            const uint32_t below = __ballot_sync(kFull, stop) & (0xFFFFFFFFu >> (31 - top));
            const int h = below ? 31 - __clz(below) : -1;  // the lane where the run ends (lane top is DIAG)
            if (lane > h && lane <= top) {
                diag_i_end[-1 - (n + t)] = rr - t;
                diag_j_end[-1 - (n + t)] = cl;
            }
            const int len = top - h;
            n += len;
            i -= len;
            j -= len;
        }
    }
    return n;
}

// Sum (FP64, fixed order: lane-strided partial sums, then a butterfly) of nd
// similarities, and the number of them >= thr; every lane gets the totals.
__device__ __forceinline__ void pair_sum_warp(const float *__restrict__ s, int nd, float thr, int lane,
                                              double &sum, int &kept) {
    sum = 0.0;
    kept = 0;
    for (int x = lane; x < nd; x += 32) {
        const float v = s[x];
        sum += (double)v;
        kept += v >= thr;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        sum += __shfl_xor_sync(kFull, sum, off);
        kept += __shfl_xor_sync(kFull, kept, off);
    }
}

// Copy the cells with s >= thr, in order, to out_*[0..).
__device__ __forceinline__ void copy_kept_warp(const int32_t *__restrict__ di, const int32_t *__restrict__ dj,
                                               const float *__restrict__ ds, int nd, float thr, int lane,
                                               int32_t *__restrict__ out_i, int32_t *__restrict__ out_j,
                                               float *__restrict__ out_s) {
    int64_t to = 0;
    for (int x0 = 0; x0 < nd; x0 += 32) {
        const int x = x0 + lane;
        const bool in = x < nd;
        const float s = in ? ds[x] : 0.0f;
        const bool keep = in && s >= thr;
        const uint32_t m = __ballot_sync(kFull, keep);
        if (keep) {
            const int64_t o = to + __popc(m & ((1u << lane) - 1u));
            out_i[o] = di[x];
            out_j[o] = dj[x];
            out_s[o] = s;
        }
        to += __popc(m);
    }
}

}  // namespace gbm
