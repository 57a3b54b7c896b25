// Launch wrappers and device-side layouts shared between the kernel
// translation units and the plan.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace gbm {

struct DevCorpus {
    const int64_t *doc;   // n_docs+1
    const int64_t *sent;  // n_sents+1
    const int32_t *tok;
    int64_t n_tok;        // tokens in tok (bounds of the bulk copies)
};

struct DevDict {
    const int32_t *off;
    const int32_t *tgt;
};

// One count work item: a 32 x 32 cell block of one pair.
struct CountItem {
    int32_t pair;
    int32_t strip_block;  // (row strip << 16) | column block
};

// One count work item of the strip kernel: rows [r_lo, r_hi) of a 32-row
// strip of one pair, all column blocks.
struct CountStripItem {
    int32_t pair;
    int32_t strip;
    int32_t r_lo, r_hi;
};

// Per-pair geometry the plan precomputes (device copy).
struct PairGeom {
    int64_t cell_off;  // first cell of the pair in per-cell buffers
    int64_t tb_off;    // first uint64 traceback word of the pair
    int64_t link_off;  // first slot of the pair's window of min(N,M) link slots
    int64_t hrow_off;  // first float of the pair's boundary row (M floats)
    int64_t vcol_off;  // first float of the pair's boundary column (N floats)
    int64_t flag_off;  // first tile flag (nstrips * nchunk ints), -1 if one warp does the pair
    int32_t n, m;      // sentence counts
    int64_t soft_off;  // first float of the pair's soft-alignment checkpoint rows (nstrips * M)
    int64_t ckw_off;   // first float of the pair's soft window checkpoints (nstrips * soft_ckw_floats(M))
    int32_t cw;        // fill column chunk width (multiple of 32)
    int32_t nchunk;    // number of column chunks
};

// One fill work item: strips [s0, s1) of column chunk cj of a pair.
struct FillItem {
    int32_t pair;
    int32_t s0, s1;
    int32_t cj;
};

// Plan-owned scratch of the alignment kernels.
struct AlignScratch {
    uint64_t *tb;      // traceback words: [strip][column block][row in strip]: UP bits low, LEFT bits high
    float *hrow;       // boundary row per pair (UP candidates of the next strip)
    float *vcol;       // boundary column per pair (LEFT candidates of the next chunk)
    int32_t *flags;    // tile completion flags
    int32_t *queue;    // dynamic work counter of the fill
    uint32_t *status;  // error bits
    int32_t *diag_i, *diag_j;  // diagonal cells of each path, in the pair's link window
    float *diag_s;
    int32_t *n_diag;
    int64_t *diag_off;  // exclusive scan of n_diag (n_pairs+1)
    int32_t *n_links;
};

cudaError_t launch_validate_corpus(const DevCorpus &c, int64_t n_sents, int64_t n_tok, int32_t vocab,
                                   uint32_t *status, int32_t *max_len, cudaStream_t st);
cudaError_t launch_block_tokens(const DevCorpus &tgt, const PairGeom *geom, int64_t n_pairs,
                                int32_t *max_block_tokens, cudaStream_t st);

cudaError_t launch_count(const DevCorpus &src, const DevCorpus &tgt, const DevDict &dict,
                         const PairGeom *geom, const CountItem *items, int64_t n_items,
                         int log_slots, int planes, uint8_t *counts, uint32_t *status,
                         int n_sms, cudaStream_t st);

cudaError_t launch_count_strips(const DevCorpus &src, const DevCorpus &tgt, const DevDict &dict,
                                const PairGeom *geom, const CountStripItem *items, int64_t n_items,
                                int log_slots, int planes, bool bulk_ok, uint8_t *counts, uint32_t *status,
                                int n_sms, cudaStream_t st);

// Fixed-width copy of a dictionary whose lists hold at most four targets.
cudaError_t launch_dict4(const DevDict &dict, int32_t v_src, int4 *dict4, cudaStream_t st);
// Every 32-row strip of every pair with targets as a count item, pairs in the
// given order (cnt: n ints, off: n + 1 int64 of scratch).
cudaError_t launch_strip_items(const PairGeom *geom, const int32_t *order, int64_t n, int32_t *cnt, int64_t *off,
                               CountStripItem *items, cudaStream_t st);
// Tile count kernel (sentences of at most 31 tokens, dictionary fan-out at
// most 4): blocked = true writes the blocked layout (pair k's 32 x 32 block
// (s, b) is the 2048-byte tile at byte 64 * tb_off + 2048 * (s * nblk + b),
// row r at byte 64 r of it, (ms, mt) per cell), false the row-major layout.
// queue: one int32 of device scratch (reset by the launch).
cudaError_t launch_count_tiles(const DevCorpus &src, const DevCorpus &tgt, const int4 *dict4, const PairGeom *geom,
                               const CountStripItem *items, int64_t n_items, int32_t *queue, bool bulk_ok,
                               bool blocked, uint8_t *counts, uint32_t *status, int n_sms, cudaStream_t st);
constexpr int kTileMaxFanout = 4;

constexpr int kStripLogSlots = 11;  // row-table slots of the strip count kernel (2^11)
constexpr int kStripMaxFanout = 46; // dictionary fan-out up to which one row always fits the row table

cudaError_t launch_score(const DevCorpus &src, const DevCorpus &tgt, const PairGeom *geom,
                         int64_t n_pairs, const DevParams &P, const uint8_t *counts, float *s,
                         float *feat, cudaStream_t st);

cudaError_t launch_fill(const DevCorpus &src, const DevCorpus &tgt, const PairGeom *geom,
                        const FillItem *items, int64_t n_items, const DevParams &P,
                        const uint8_t *counts, int64_t counts_bytes, bool blocked, const AlignScratch &S,
                        int64_t wait_limit, int64_t skip_flag, int n_sms, cudaStream_t st);

// order: the pairs by decreasing size (a permutation of 0..n_pairs-1)
cudaError_t launch_walk(const PairGeom *geom, const int32_t *order, int64_t n_pairs, const AlignScratch &S,
                        int n_sms, cudaStream_t st);

cudaError_t launch_scan(const int32_t *in, int64_t n, int64_t *out, cudaStream_t st);
// As launch_scan with int32 offsets (the caller knows the total fits).
cudaError_t launch_scan32(const int32_t *in, int64_t n, int32_t *out, cudaStream_t st);

// Bi-directional mining (bi.cu).
// Dictionary transpose: status bit 0 set for a malformed dictionary (checked
// by launch_dict_check before any other step reads it).
cudaError_t launch_dict_check(const int32_t *off, int32_t v_src, int64_t n_entries, const int32_t *tgt,
                              int32_t v_tgt, uint32_t *status, cudaStream_t st);
cudaError_t launch_dict_count(const int32_t *tgt, int64_t n_entries, int32_t *cnt, cudaStream_t st);
cudaError_t launch_dict_scatter(const int32_t *off, int32_t v_src, const int32_t *tgt, int32_t *cursor,
                                int32_t *tgt_out, cudaStream_t st);
cudaError_t launch_dict_sort(const int32_t *off_out, int32_t v_tgt, int32_t *tgt_out, cudaStream_t st);
// Anchor tokens (anchors.cu): status bit 0 set for malformed word offsets or
// anchor lists.
cudaError_t launch_anchor_check(const int64_t *woff, int64_t n_tok, const int64_t *aoff, int64_t n_sents,
                                const int32_t *ids, int64_t n_anchor_tok, int32_t v_anchor, uint32_t *status,
                                cudaStream_t st);
cudaError_t launch_anchor_merge(const int64_t *woff, const int32_t *words, const int64_t *aoff, const int32_t *ids,
                                int64_t n_sents, int32_t v_words, int64_t *out_off, int32_t *out, cudaStream_t st);
cudaError_t launch_anchor_dict(const int32_t *off, const int32_t *tgt, int32_t v_src, int32_t v_tgt,
                               int64_t n_entries, int32_t v_anchor, int32_t *off_out, int32_t *tgt_out,
                               cudaStream_t st);
// Link lists of a plan output (offsets per pair, i, j, s).
struct LinkView {
    const int64_t *off;
    const int32_t *i, *j;
    const float *s;
    int64_t cap;  // entries of i, j, s
};
// Per pair: count (out_i == nullptr) or write the merged links of fwd and
// rev (rev's link (i', j') is (j', i')); mode 0 union, 1 intersection;
// out_cap: entries of the output arrays.
cudaError_t launch_links_combine(LinkView fwd, LinkView rev, int64_t n_pairs, int mode, int32_t *count,
                                 int64_t out_cap, const int64_t *out_off, int32_t *out_i, int32_t *out_j,
                                 float *out_sf, float *out_sr, cudaStream_t st);

cudaError_t launch_link_score(const DevCorpus &src, const DevCorpus &tgt, const DevDict &dict,
                              const PairGeom *geom, int64_t n_pairs, const DevParams &P,
                              const AlignScratch &S, const uint8_t *counts, bool blocked, int n_sms,
                              cudaStream_t st);

cudaError_t launch_pair_sum(const PairGeom *geom, int64_t n_pairs, const DevParams &P,
                            const AlignScratch &S, float *pair_score, int n_sms, cudaStream_t st);

cudaError_t launch_copy_links(const PairGeom *geom, int64_t n_pairs, const DevParams &P,
                              const AlignScratch &S, const int64_t *link_off, int32_t *out_i,
                              int32_t *out_j, float *out_s, int n_sms, cudaStream_t st);

cudaError_t launch_link_gold(const PairGeom *geom, int64_t n_pairs, const int64_t *link_off, const int32_t *li,
                             const int32_t *lj, const uint8_t *gold, unsigned long long *out, int n_sms,
                             cudaStream_t st);

// Soft alignment: scalar arguments and the caller's workspace, carved up.
struct SoftArgs {
    float gamma, tau, eps, inv_cells;
    int64_t wait_limit;  // bounded spins of a strip wait (split pairs)
    uint32_t *status;    // plan status word (timeout bit)
    int split;           // 0: one warp per pair, 1: split long pairs, 2: split every pair of >= 2 strips
    int split_q4;        // split = 1: a pair splits when its chain exceeds split_q4 / 4 of the mean per warp
    int order;           // work list: 0 per split pair (its value sweep, then its adjoint), whole pairs last;
                         // 1 every value sweep, the whole pairs, every adjoint; 2 value sweeps, adjoints, whole
    int64_t skip_ctr;    // fault injection: this forward progress counter is never published (-1: off)
    float *hvp;          // backward: per cell H u (null: not wanted)
};
constexpr int kSoftSlots = 16;  // per strip: loss sum, the gradient's H u parts, its gate parts
constexpr int kSoftRedBlocks = 64;  // first-level blocks of the partial sums' reduction
// Work item of the sweep kernels: a whole pair (kind 0), or one strip of a
// split pair in the forward wavefront (kind 1) or in the adjoint wavefront
// (kind 2); ctr = the pair's first progress counter, slot = the pair's first
// strip slot of the partial sums.
struct SoftItem {
    int32_t pos, strip, kind, ctr, slot;
};
struct SoftScratch {
    double *partial;      // per strip slot: kSoftSlots sums
    double *vpart;        // per listed pair: V(N,M)
    double *red;          // kSoftRedBlocks x 8: first-level sums of the partial sums
    int32_t *queue;       // [0] work counter, [1] items, [2] strip slots
    SoftItem *items;      // sweep work list
    int32_t *prog1;       // per strip of a split pair: forward columns published
    int32_t *prog2;       // per strip of a split pair: adjoint steps published
    float *E;             // expected alignment per cell, per strip step-major (soft_e_index)
    float *ckv, *ckt;     // checkpoint rows (value, tangent), nstrips * M per pair at soft_off
    float *qrow, *qtrow;  // adjoint boundary rows (value, tangent), at soft_off
    float *ckw;           // per strip: the sweep state at the start of every window
    int64_t items_cap, slots_cap, ctr_cap;
};

int64_t soft_warps(int n_sms);
// Floats of one strip's window checkpoints in a pair of M target sentences
// (the adjoint sweeps recompute 8-step windows from them).
__host__ __device__ inline int64_t soft_ckw_floats(int M) { return 128 * (32 * ((M + 31) / 32 + 1) / 8); }

cudaError_t launch_soft_export_e(const PairGeom *geom, int64_t n_pairs, const float *E, float *out, cudaStream_t st);
cudaError_t launch_soft_forward(const DevCorpus &src, const DevCorpus &tgt, const PairGeom *geom,
                                const int32_t *order, int64_t n_pairs, const DevParams &P, const SoftArgs &A,
                                const uint8_t *counts, const uint8_t *gold, const SoftScratch &W, float *loss,
                                float *value, int n_sms, cudaStream_t st);

cudaError_t launch_soft_backward(const DevCorpus &src, const DevCorpus &tgt, const PairGeom *geom,
                                 const int32_t *order, int64_t n_pairs, const DevParams &P, const SoftArgs &A,
                                 const uint8_t *counts, const uint8_t *gold, const SoftScratch &W, float dloss,
                                 float *grad, float *hvp, int n_sms, cudaStream_t st);

// Unconstrained (Yalign A*) alignment: the caller's workspace, carved up.
struct UcScratch {
    const int64_t *a_off;     // per pair: first double of its two DP rows (2 (M+1))
    const int64_t *prev_off;  // per pair: first int of its predecessor pointers (N (M+1))
    const int64_t *link_off;  // per pair: first slot of its window of N matched cells
    int64_t *A;               // two score rows per pair (fixed point, units of 2^-k)
    int32_t *prev;
    int32_t *li, *lj;
    float *ls;
    int32_t *n_match;         // per pair: matched cells (at the end of the window)
};
// Pairs whose target has fewer than kUcShortCols sentences run with small
// shared rows and many warps per SM; the others with rows sized by max_m.
constexpr int kUcShortCols = 256;
// Scores, matches and per-pair kept-link counts (kept), then the compaction
// of the kept links (s >= thr) at out_off.  order: the pairs with
// M + 1 <= kUcShortCols first (n_short of them), then the rest; max_m: the
// largest M of the pairs.
cudaError_t launch_unconstrained(const DevCorpus &src, const DevCorpus &tgt, const PairGeom *geom, const int32_t *order,
                                 int64_t n_short, int64_t n_pairs, const DevParams &P, const uint8_t *counts,
                                 const UcScratch &W, float *pair_score, int max_m, int32_t *kept, int n_sms,
                                 cudaStream_t st);
cudaError_t launch_unconstrained_copy(const PairGeom *geom, int64_t n_pairs, float thr, const UcScratch &W,
                                      const int64_t *out_off, int32_t *out_i, int32_t *out_j, float *out_s, int n_sms,
                                      cudaStream_t st);

// Records e as this thread's last CUDA error (what mine_last_cuda_error
// returns) for entry points outside the plan's translation unit.
void record_cuda_error(int e);

// Kernel kinds of the per-kernel timing hook (order of MINE_KERNEL_KINDS).
enum KernelKind { kKCount = 0, kKFill, kKWalk, kKLinks, kKScan, kKScore, kKSoftFwd, kKSoftBwd, kKinds };

}  // namespace gbm
