// Launch wrappers shared between the kernel translation units and the plan.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace gbm {

struct DevCorpus {
    const int64_t *doc;   // n_docs+1
    const int64_t *sent;  // n_sents+1
    const int32_t *tok;
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

// Per-pair geometry the plan precomputes (device copy).
struct PairGeom {
    int64_t cell_off;  // first cell of the pair in per-cell buffers
    int64_t tb_off;    // first uint64 traceback word of the pair
    int64_t link_off;  // first link slot (capacity min(N,M) per pair)
    int64_t hrow_off;  // first float of the pair's boundary row buffer (M floats)
    int32_t n, m;      // sentence counts
};

cudaError_t launch_validate_corpus(const DevCorpus &c, int64_t n_sents, int64_t n_tok, int32_t vocab,
                                   uint32_t *status, int32_t *max_len, cudaStream_t st);
cudaError_t launch_block_tokens(const DevCorpus &tgt, const PairGeom *geom, int64_t n_pairs,
                                int32_t *max_block_tokens, cudaStream_t st);

cudaError_t launch_count(const DevCorpus &src, const DevCorpus &tgt, const DevDict &dict,
                         const PairGeom *geom, const CountItem *items, int64_t n_items,
                         int log_slots, int planes, uint8_t *counts, uint32_t *status,
                         int n_sms, cudaStream_t st);

cudaError_t launch_score(const DevCorpus &src, const DevCorpus &tgt, const PairGeom *geom,
                         int64_t n_pairs, const DevParams &P, const uint8_t *counts, float *s,
                         float *feat, cudaStream_t st);

cudaError_t launch_nw_counts(const DevCorpus &src, const DevCorpus &tgt, const PairGeom *geom,
                             const int32_t *order, int64_t n_pairs, const DevParams &P,
                             const uint8_t *counts, uint64_t *tb, float *hrow, int n_sms,
                             cudaStream_t st);

cudaError_t launch_traceback(const DevCorpus &src, const DevCorpus &tgt, const DevDict &dict,
                             const PairGeom *geom, int64_t n_pairs, const DevParams &P,
                             const uint64_t *tb, int32_t *scr_i, int32_t *scr_j, float *scr_s,
                             int32_t *n_links, float *pair_score, cudaStream_t st);

cudaError_t launch_scan(const int32_t *n_links, int64_t n_pairs, int64_t *link_off, cudaStream_t st);

cudaError_t launch_copy_links(const PairGeom *geom, int64_t n_pairs, const int32_t *n_links,
                              const int32_t *scr_i, const int32_t *scr_j, const float *scr_s,
                              const int64_t *link_off, int32_t *out_i, int32_t *out_j, float *out_s,
                              cudaStream_t st);

// Kernel kinds of the per-kernel timing hook (order of MINE_KERNEL_KINDS).
enum KernelKind { kKCount = 0, kKFill, kKTraceback, kKScan, kKCopy, kKScore, kKinds };

}  // namespace gbm
