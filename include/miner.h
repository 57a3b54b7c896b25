/*
 * miner.h - C ABI of the GB300 comparable-corpus miner.
 *
 * The method (Wolk & Marasek, arXiv:1512.01641):
 *   - every source x target sentence pair of a topic-aligned document pair gets
 *     a similarity in [0,1]: a linear classifier's decision value over
 *     dictionary/length features squashed by a sigmoid (Section 4);
 *   - the two sentence sequences are globally aligned by Needleman-Wunsch
 *     under a gap penalty (Section 5.1, Figure 1, Eq. 1): S(0,0) = 0, border
 *     cells initialised with the penalty, every other cell the max of
 *     diagonal + similarity, up - penalty and left - penalty;
 *   - aligned pairs whose similarity is below the acceptance threshold are
 *     dropped (Section 4; the threshold of Section 5.2).
 *
 * Conventions for every entry point:
 *   - all array pointers are DEVICE pointers unless the name says host_;
 *     buffers are owned by the caller, except what a plan allocates itself;
 *   - calls taking a stream are asynchronous on it, unless stated otherwise;
 *   - a negative return value is an error code (mine_strerror); 0 is success;
 *   - document pair k is source document k with target document k.
 *
 * Input corpus layout (CSR): document d owns sentences
 * doc_sent_off[d] .. doc_sent_off[d+1]-1; sentence s owns tokens
 * tok[sent_tok_off[s] .. sent_tok_off[s+1]-1], sorted ascending, 1..255 of
 * them.  The dictionary maps source id v to the sorted, distinct target ids
 * tgt[off[v] .. off[v+1]-1].
 *
 * Cell (i, j) of pair k is (source sentence i, target sentence j), 0-based.
 * Per-cell buffers are row-major per pair, pair k starting at cell offset
 * sum_{k'<k} N_k' * M_k' (mine_plan_cell_offsets).
 */
#ifndef GB300_MINER_H
#define GB300_MINER_H

#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *miner_stream_t; /* same handle as cudaStream_t */

/* error codes */
#define MINE_OK 0
#define MINE_EINVAL (-1)   /* malformed input (offsets, ids, ordering, sizes) */
#define MINE_ENOMEM (-2)   /* device or host allocation failed */
#define MINE_ECUDA (-3)    /* a CUDA call failed (mine_last_cuda_error) */
#define MINE_ETIMEOUT (-4) /* a device-side bounded wait gave up */
#define MINE_ENOTSUP (-5)  /* request outside what this build supports */

typedef struct {
    int64_t n_docs;               /* number of documents */
    int64_t n_sents;              /* total sentences (= doc_sent_off[n_docs]) */
    int64_t n_tok;                /* total tokens (= sent_tok_off[n_sents]) */
    const int64_t *doc_sent_off;  /* n_docs+1, device */
    const int64_t *sent_tok_off;  /* n_sents+1, device */
    const int32_t *tok;           /* n_tok, device, sorted per sentence */
} mine_corpus;

typedef struct {
    int32_t v_src;                /* source vocabulary size */
    int32_t v_tgt;                /* target vocabulary size */
    int64_t n_entries;            /* = off[v_src] */
    const int32_t *off;           /* v_src+1, device */
    const int32_t *tgt;           /* n_entries, device, sorted distinct per id */
} mine_dict;

/* Classifier and alignment parameters (Section 4 / Section 5.2):
 * similarity s = 1 / (1 + exp(-(w . f + b))) with
 * f = [ms/ls, mt/lt, |ls-lt|/max(ls,lt), min(ls,lt)/max(ls,lt)],
 * gap = penalty p per unmatched sentence, thr = acceptance threshold. */
typedef struct {
    float w[4];
    float b;
    float gap;
    float thr;
} mine_params;

/* Output of mine_pairs / mine_align (all device, caller-allocated).
 * Links of pair k are entries link_off[k] .. link_off[k+1]-1 of link_i,
 * link_j, link_s, ascending in i and j.  link_capacity must be at least
 * mine_plan_link_capacity() (the sum over pairs of min(N_k, M_k)). */
typedef struct {
    int64_t *link_off;     /* n_docs+1, filled by the library */
    int32_t *link_i;       /* source sentence index within the document */
    int32_t *link_j;       /* target sentence index within the document */
    float *link_s;         /* similarity of the linked pair (>= thr) */
    float *pair_score;     /* n_docs: Needleman-Wunsch value H(N_k, M_k) */
    int64_t link_capacity; /* entries available in link_i/link_j/link_s */
} mine_out;

typedef struct mine_plan mine_plan;

/* Validate the inputs and build a plan for mining every document pair:
 * document sizes, work order, per-pair offsets and the plan-owned scratch
 * (traceback bits, cached counts, boundary rows).  The input buffers must
 * stay alive and unchanged while the plan is used.  SYNCHRONOUS on the stream
 * (it reads the document offsets back and waits for the validation kernel).
 * Returns MINE_EINVAL for: n_docs mismatch, offsets not starting at 0 or not
 * monotone, an empty sentence or one longer than 255 tokens, a token id
 * outside its vocabulary, tokens not sorted within a sentence, dictionary
 * lists unsorted or repeated or out of range. */
int mine_plan_create(const mine_corpus *src, const mine_corpus *tgt, const mine_dict *dict,
                     mine_plan **out, miner_stream_t stream);
/* As mine_plan_create, with plan options (MINE_OPT_*, see below) set before
 * the work lists are built: options[x] takes values[x], in order.  Setting the
 * tiling options this way costs nothing, where mine_plan_set_option on an
 * existing plan rebuilds its fill work lists.  options and values: host
 * arrays of n_options entries (both may be NULL when n_options is 0).
 * MINE_EINVAL, before any device work, for n_options < 0, an unknown or
 * read-only option, or a value mine_plan_set_option would reject. */
int mine_plan_create_with_options(const mine_corpus *src, const mine_corpus *tgt, const mine_dict *dict,
                                  const int32_t *options, const int64_t *values, int n_options,
                                  mine_plan **out, miner_stream_t stream);
/* Releases the plan without waiting: its device memory returns to the
 * library's pool (a stream-ordered pool per device that keeps up to 16 GiB
 * of freed memory for later plans) once the work enqueued by the last call
 * that used the plan has finished on that call's stream.  Inputs may be freed
 * once that work has finished. */
void mine_plan_destroy(mine_plan *plan);

int64_t mine_plan_n_pairs(const mine_plan *plan);
int64_t mine_plan_n_cells(const mine_plan *plan);       /* sum N_k * M_k */
int64_t mine_plan_link_capacity(const mine_plan *plan); /* sum min(N_k, M_k) */
/* host_out: n_pairs+1 entries (host memory), cell offsets of each pair. */
int mine_plan_cell_offsets(const mine_plan *plan, int64_t *host_out);

/* Overlap counts of every cell (Section 4 similarity inputs, feature reading
 * above): counts[2*c] = ms, counts[2*c+1] = mt for cell c, uint8 each, exact
 * integers.  ms = source positions with a translation present in the target
 * sentence; mt = target positions whose token translates some source token.
 * counts must hold 2 * mine_plan_n_cells() bytes. */
int mine_count(mine_plan *plan, uint8_t *counts, miner_stream_t stream);

/* Features and similarity of every cell from counts (the unfused debug path of
 * Section 4's classifier): s[c] (FP32) and, if feat is not NULL, feat[4*c+k]
 * the four features, each an IEEE-rounded FP32 quotient. */
int mine_score(mine_plan *plan, const mine_params *params, const uint8_t *counts,
               float *s, float *feat, miner_stream_t stream);

/* Needleman-Wunsch alignment + threshold filter (Section 5.1, Eq. 1; Section
 * 4 threshold) of every pair from precomputed counts.  Ties in the traceback
 * prefer UP (source sentence unmatched), then LEFT, then DIAG (Figure 4). */
int mine_align(mine_plan *plan, const mine_params *params, const uint8_t *counts,
               mine_out *out, miner_stream_t stream);

/* The whole hot path: overlap counts, similarity, alignment, threshold
 * filter, for every document pair of the plan, as one CUDA graph launch
 * (MINE_OPT_USE_GRAPH).  Uses plan-owned scratch; no allocation after plan
 * creation.  The first call, and any call whose output buffers or parameters
 * differ from the previous one, captures the graph (on a plan-owned stream)
 * before launching it on `stream`. */
int mine_pairs(mine_plan *plan, const mine_params *params, mine_out *out,
               miner_stream_t stream);

/* The whole hot path from HOST buffers, for callers that hold the corpora in
 * host memory and have no device buffers of their own: the corpus and
 * dictionary structs' arrays are HOST pointers (pinned memory copies at full
 * speed, pageable memory works); the library uploads them into memory from its
 * pool, plans (with the options, as mine_plan_create_with_options; the CUDA
 * graph is off unless an option turns it on), runs mine_pairs, and writes the
 * results to the host arrays: link_off (n_docs+1), the links (link_capacity
 * entries, at least the sum over pairs of min(N_k, M_k)) and pair_score
 * (n_docs).  The upload overlaps the planning (from the host document
 * offsets); with MINE_OPT_HOST_CHUNKS the batch is mined in chunks of pairs,
 * the upload and plan of the next chunk overlapping the mining of the current
 * one; the results do not depend on the chunking.
 * SYNCHRONOUS: returns when the results are in host memory and everything the
 * call allocated is back in the pool.  Error codes as mine_plan_create and
 * mine_pairs, MINE_ETIMEOUT as mine_plan_check. */
int mine_pairs_host(const mine_corpus *src, const mine_corpus *tgt, const mine_dict *dict, const mine_params *params,
                    const int32_t *options, const int64_t *values, int n_options, int64_t *link_off,
                    int32_t *link_i, int32_t *link_j, float *link_s, float *pair_score, int64_t link_capacity,
                    miner_stream_t stream);

/* Link quality against gold links (gold: one 0/1 byte per cell, per-cell
 * layout as the counts): counts3[0] = links that are gold, counts3[1] =
 * links, counts3[2] = gold cells (device, 3 x uint64).  Micro precision =
 * [0]/[1], recall = [0]/[2]; the tuning evaluation of Section 5.2's
 * threshold/penalty search uses them. */
int mine_link_gold_counts(mine_plan *plan, const mine_out *out, const uint8_t *gold, uint64_t *counts3,
                          miner_stream_t stream);

/* ---- Bi-directional mining (Section 5.4, "BI": a second classifier mines
 * the reverse direction and the bi-sentences of both are kept) ----
 * The reverse direction is a second plan whose source corpus is this one's
 * target corpus and vice versa, with a dictionary from target ids to source
 * ids (the caller's own, or mine_dict_transpose of the forward one) and its
 * own parameters; mine_links_combine merges the links of the two plans pair
 * by pair. */

/* Transpose of a dictionary: for every target id t, the ascending source ids
 * v with t among tgt[off[v] .. off[v+1]-1].  off_out: v_tgt+1 int32, tgt_out:
 * n_entries int32 (device, caller-allocated).  SYNCHRONOUS on the stream (it
 * checks the dictionary first).  MINE_EINVAL for a NULL argument, sizes out of
 * range, offsets that do not start at 0, decrease or do not end at
 * n_entries, or a target id outside [0, v_tgt); the outputs are then
 * unspecified. */
int mine_dict_transpose(const mine_dict *dict, int32_t *off_out, int32_t *tgt_out, miner_stream_t stream);

/* ---- Anchors (Section 5.3: names, dates, numbers and references that two
 * Wikipedia sentences share mark them as likely translations) ----
 * An anchor is an id of its own vocabulary [0, v_anchor), the same in both
 * languages.  Reading: it takes part in the overlap counts of Section 4 as a
 * word that translates to itself -- anchor a of a sentence becomes token
 * v_words + a of its corpus (v_words: that corpus's vocabulary size), and the
 * dictionary gains the entries v_src + a -> {v_tgt + a}.  The extended
 * corpora and dictionary are then mined like any others. */

/* The corpus with every sentence's anchors appended to its tokens (as
 * v_words + a; anchors sort after every word, so sorted anchors keep the
 * sentence sorted).  anchor_off: n_sents+1 int64, anchor_ids: n_anchor_tok
 * int32 (device; per sentence sorted and distinct -- mine_plan_create rejects
 * the extended corpus otherwise).  Outputs (device, caller-allocated):
 * sent_tok_off_out n_sents+1 int64, tok_out n_tok + n_anchor_tok int32; the
 * document offsets are unchanged.  SYNCHRONOUS on the stream (it checks the
 * offsets first).  MINE_EINVAL for a NULL argument, v_words + v_anchor beyond
 * int32, word or anchor offsets that do not start at 0, decrease or do not
 * end at n_tok / n_anchor_tok, or an anchor id outside [0, v_anchor). */
int mine_corpus_add_anchors(const mine_corpus *words, int32_t v_words, const int64_t *anchor_off,
                            const int32_t *anchor_ids, int64_t n_anchor_tok, int32_t v_anchor,
                            int64_t *sent_tok_off_out, int32_t *tok_out, miner_stream_t stream);

/* The dictionary with the identity entries of v_anchor anchors appended:
 * off_out v_src + v_anchor + 1 int32, tgt_out n_entries + v_anchor int32
 * (device, caller-allocated).  SYNCHRONOUS on the stream (it checks the
 * dictionary first, as mine_dict_transpose does).  MINE_EINVAL, with nothing
 * written, for a NULL argument, sizes beyond int32, or offsets that do not
 * start at 0, decrease or do not end at n_entries, or a target id outside
 * [0, v_tgt). */
int mine_dict_add_anchors(const mine_dict *dict, int32_t v_anchor, int32_t *off_out, int32_t *tgt_out,
                          miner_stream_t stream);

#define MINE_BI_UNION 0     /* links kept by either direction */
#define MINE_BI_INTERSECT 1 /* links kept by both directions */

/* Output of mine_links_combine (device, caller-allocated).  Links of pair k
 * are entries link_off[k] .. link_off[k+1]-1, in forward coordinates
 * (link_i: source sentence, link_j: target sentence), ascending in (i, j)
 * lexicographically (a union of two monotone link lists need not be
 * monotone).  s_fwd / s_rev: the link's similarity in each direction, NaN
 * where that direction did not keep the link.  link_capacity must be at
 * least mine_plan_link_capacity(fwd) + mine_plan_link_capacity(rev). */
typedef struct {
    int64_t *link_off; /* n_docs+1 */
    int32_t *link_i;
    int32_t *link_j;
    float *s_fwd;
    float *s_rev;
    int64_t link_capacity;
} mine_bi_out;

/* Merge, per pair, the links of a forward plan (out_fwd, as mine_pairs or
 * mine_align wrote it on fwd) with those of the reverse plan (out_rev on
 * rev; its link (i', j') is the forward link (j', i')): their union or their
 * intersection (mode, MINE_BI_*).  rev must hold the same pairs with the roles
 * swapped, N_k(rev) = M_k(fwd) and M_k(rev) = N_k(fwd) (checked on the host:
 * MINE_EINVAL).  Asynchronous on the stream, after both outputs are complete
 * on it; uses a temporary of n_docs int32 from the library's pool.  Every
 * access stays inside the buffers' declared capacities even for outputs that
 * did not come from mining these plans (the links are then unspecified). */
int mine_links_combine(mine_plan *fwd, const mine_out *out_fwd, mine_plan *rev, const mine_out *out_rev,
                       int mode, mine_bi_out *out, miner_stream_t stream);

/* Plan options: the tuning knobs of the planner (defaults in parentheses).
 * Setting a tiling option to a new value rebuilds the plan's work lists on
 * the host and replaces them on the device after the plan's last enqueued
 * work (synchronous: returns once they are in place); set tiling options at
 * creation (mine_plan_create_with_options) where they are known then. */
#define MINE_OPT_TILE_COLS 1      /* fill tile width in columns, multiple of 32 (64) */
#define MINE_OPT_TILE_MIN_CELLS 2 /* a pair with at least this many cells ... (65536) */
#define MINE_OPT_TILE_MIN_ROWS 3  /* ... and this many rows is filled as tiles (64) */
#define MINE_OPT_WAIT_LIMIT 4     /* spin iterations before a tile wait gives up (2^24) */
#define MINE_OPT_LINK_RECOUNT 5   /* 1: recount the overlaps of aligned pairs by warp
                                     vote instead of reading the cached counts (0) */
#define MINE_OPT_USE_GRAPH 6      /* 1: mine_pairs captures its launches once into a
                                     CUDA graph and replays it (1); the graph is
                                     re-captured when the output buffers or the
                                     parameters change, and bypassed while per-kernel
                                     timing is on */
#define MINE_OPT_GRAPH_CAPTURES 7 /* read-only: graph captures made so far */
#define MINE_OPT_FAULT_SKIP_FLAG 8 /* fault injection for tests: the completion flag with
                                      this index is never published, so the tiles that
                                      wait on it give up after MINE_OPT_WAIT_LIMIT spins
                                      and mine_plan_check reports MINE_ETIMEOUT (-1: off) */
#define MINE_OPT_N_TILE_FLAGS 9   /* read-only: tile flags of the plan (tiled pairs) */
#define MINE_OPT_SOFT_SPLIT 10    /* softnw sweeps: 0 one warp per pair; 1 a pair whose
                                     serial chain (strips x (M + 32) steps) is above the
                                     mean per warp is split over warps, one strip each,
                                     in a wavefront; 2 every pair of two or more strips is
                                     split; 3 (default) every pair of two or more strips is
                                     split when some pair's chain is above the mean per
                                     warp, else none.  Same results in every mode. */
#define MINE_OPT_FAULT_SKIP_SOFT 11 /* fault injection for tests: the forward progress counter
                                       with this index (strips of split pairs, in the soft work
                                       list's order) is never published, so the strips that wait
                                       on it give up after MINE_OPT_WAIT_LIMIT polls and
                                       mine_plan_check reports MINE_ETIMEOUT (-1: off) */
#define MINE_OPT_SOFT_SPLIT_Q4 13  /* soft split modes 1 and 3: the chain threshold (of the
                                      pair, mode 1; of the longest pair, mode 3) in quarters of
                                      the mean chain per warp (4: the mean); 1 .. 4096.  Same
                                      results at any value. */
#define MINE_OPT_SOFT_ORDER 14    /* soft work list with split pairs: 0 each split pair's
                                     value-sweep strips then its adjoint strips, whole pairs
                                     last; 1 (default) every value-sweep strip, the whole pairs,
                                     every adjoint strip (the adjoint strips then seldom wait
                                     for their value sweep); 2 value sweeps, adjoints, whole.
                                     Every wait is on an item listed earlier in all three; same
                                     results in every order. */
#define MINE_OPT_HOST_CHUNKS 12   /* mine_pairs_host only (not a plan option): the batch is
                                     mined as this many contiguous chunks of pairs of about
                                     equal cells, the upload and the plan of the next chunk
                                     overlapping the mining of the current one (0, the
                                     default: one chunk, whose upload overlaps its planning;
                                     on a batch whose longest pairs end up in one chunk, more
                                     chunks lose the overlap of long and short pairs) */
int mine_plan_set_option(mine_plan *plan, int option, int64_t value);
/* Current value of an option, or MINE_EINVAL for an unknown option. */
int64_t mine_plan_get_option(const mine_plan *plan, int option);

/* Synchronise the stream and report device-side errors raised since the last
 * check: MINE_ETIMEOUT if a bounded wait of the cooperative fill or of a
 * split soft sweep gave up (its results are then invalid), MINE_EINVAL if a
 * count table overflowed or a soft work list did not fit the workspace
 * (repeated entries in softnw_opts.pairs), else MINE_OK.  Clears the recorded
 * errors. */
int mine_plan_check(mine_plan *plan, miner_stream_t stream);

/* Per-kernel timing (profiling aid).  When enabled, every kernel launch of the
 * plan is bracketed by CUDA events on the launching stream and its duration is
 * accumulated per kernel kind.  mine_plan_kernel_times synchronises the last
 * stream used, then writes up to n totals (milliseconds) into host_ms and the
 * matching launch counts into host_launches (either may be NULL); it returns
 * the number of kernel kinds (MINE_KERNEL_KINDS).  Kinds, in order: count,
 * fill, walk (traceback), links (link scoring, pair sums, compaction), scan,
 * score, soft forward, soft backward. */
#define MINE_KERNEL_KINDS 8
int mine_plan_set_timing(mine_plan *plan, int enable);
int mine_plan_kernel_times(mine_plan *plan, float *host_ms, int64_t *host_launches, int n);

/* ---------------------------------------------------------------------------
 * Soft (differentiable) alignment for tuning w, b, gap and thr.
 *
 * The paper tunes the threshold and the gap penalty by random search against
 * human alignments (Section 5.2).  This library replaces the search by
 * gradients of a smoothed alignment: every max of the Needleman-Wunsch fill
 * (Section 5.1, Eq. 1) becomes gamma * log-sum-exp(. / gamma), giving the
 * soft value V and the expected alignment E = dV(N,M)/ds (the probability
 * that the alignment pairs source sentence i with target sentence j).  With
 * gold links g (0/1 per cell) the loss is
 *   P = clamp(E * sigmoid((s - thr) / tau), eps, 1 - eps)
 *   L = mean over all cells of all pairs of -(g log P + (1-g) log(1-P)).
 * ------------------------------------------------------------------------- */
typedef struct {
    float gamma;           /* smoothing temperature (> 0); -> hard NW as gamma -> 0 */
    float tau;             /* gate temperature of the acceptance threshold (> 0) */
    float eps;             /* clamp of P (0 < eps < 0.5) */
    const int32_t *pairs;  /* device: the pairs to include (a minibatch, distinct
                              pair indices), or NULL for all */
    int64_t n_pairs;       /* number of entries of pairs (ignored when pairs is NULL) */
    int64_t n_cells;       /* cells of the listed pairs: the loss is their mean
                              (ignored when pairs is NULL) */
} softnw_opts;

/* Bytes of the caller-provided workspace of softnw_fwd / softnw_bwd. */
int64_t softnw_workspace_size(const mine_plan *plan);

/* Loss L (one float at *loss, device) from cached counts (as mine_count) and
 * gold (one byte per cell, 0 or 1).  Optional outputs (NULL to skip): value
 * (n_pairs floats, soft V(N,M) per pair) and expected (n_cells floats, E).
 * Keeps E in the workspace for softnw_bwd.  With opts->pairs set, only the
 * listed pairs are swept (E and value of the others are left untouched). */
int softnw_fwd(mine_plan *plan, const mine_params *params, const softnw_opts *opts, const uint8_t *counts,
               const uint8_t *gold, void *ws, float *loss, float *value, float *expected,
               miner_stream_t stream);

/* dloss * dL/d(w0, w1, w2, w3, b, gap, thr) into grad (7 floats, device).
 * hvp (optional, n_cells floats): the Hessian-vector product H u of V with
 * u = dL/dE, i.e. the derivative of E along u (dL/ds through E).
 * Must follow softnw_fwd with the same plan, arguments and workspace. */
int softnw_bwd(mine_plan *plan, const mine_params *params, const softnw_opts *opts, const uint8_t *counts,
               const uint8_t *gold, void *ws, float dloss, float *grad, float *hvp, miner_stream_t stream);

/* ---- Unconstrained alignment: the A* aligner of Yalign, the baseline that
 * Section 5.1 contrasts with Needleman-Wunsch (Figures 3 and 5 against 4 and
 * 6): with NW's similarities and gap penalty A* finds NW's alignment only if
 * its path may not go back up or left in the S matrix, and Yalign's may, so
 * a sentence can be aligned twice.  The paper gives no cost model for the
 * move back; reading used: source sentences are taken in order, each is
 * unmatched (-gap), matched ahead of the target pointer (the NW diagonal,
 * -gap for every target sentence skipped), or matched at or behind it (a
 * move back into the target sequence, -gap); target sentences after the
 * final pointer cost gap each.  Without the move back this is exactly NW.
 * Ties prefer unmatched, then ahead, then back; the nearest predecessor.
 * Scores in FP64 on the GPU (a comparison baseline, not the mining path). */

/* Bytes of the caller-provided workspace of mine_align_unconstrained. */
int64_t mine_unconstrained_workspace_size(const mine_plan *plan);
/* Links the output must hold: the sum over pairs of N_k (one per source
 * sentence at most; target sentences may repeat). */
int64_t mine_unconstrained_link_capacity(const mine_plan *plan);
/* Unconstrained alignment of every pair from counts (as mine_count) and the
 * classifier of params: out receives per pair the matched cells with s >= thr
 * in source order (target indices need not increase) and the score in
 * pair_score.  ws: mine_unconstrained_workspace_size bytes of device memory.
 * Asynchronous.  MINE_EINVAL for a NULL argument or an output of less than
 * mine_unconstrained_link_capacity links. */
int mine_align_unconstrained(mine_plan *plan, const mine_params *params, const uint8_t *counts, void *ws,
                             mine_out *out, miner_stream_t stream);

/* Allocation-free alignment of ONE document pair (the paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * device memory when they call -- a serving loop with a fixed memory budget,
 * a library embedded in a host framework that owns every device allocation,
 * or code that cannot afford cudaMalloc's implicit synchronisation).
 *
 * Same result as mine_align on a plan holding just this pair (bit-identical
 * links and score), from the pair's precomputed counts; no plan, no
 * allocation: the scratch (traceback codes, one boundary row, the path
 * cells) is one fixed device array of about 1.1 MB inside the library, which
 * every GPU that loads the library holds until the process exits.
 *   src_sent_off: n+1 sentence token offsets of the source document (device;
 *                 only their differences, the sentence lengths, are used)
 *   tgt_sent_off: m+1 likewise for the target document
 *   counts:       n*m*2 bytes, (ms, mt) per cell, row-major (as mine_count)
 *   link_i/j/s:   capacity min(n, m); the kept links, ascending
 *   n_links, pair_score: one int32 / one float (device)
 * n and m may be 0; each must be at most MINE_NOALLOC_MAX_SIDE, otherwise the
 * call returns MINE_EINVAL without launching anything.  Asynchronous on the
 * stream.  The first call on a device looks up the scratch array's device
 * address (once per device, with that device current): make that first call
 * before any stream capture.  Every call uses the same array, so calls whose
 * kernels overlap on the GPU (other streams, other threads) race and corrupt
 * each other's results; serialise them.  Nothing needs to be zero beforehand:
 * each call overwrites every scratch word it reads.
 * A device-side failure has no plan to report it through: if a bounded wait
 * for the staged counts gives up, the kernel writes *n_links = -1 and
 * *pair_score = NaN, and the links are then invalid (the call itself has
 * already returned MINE_OK; read n_links before using the links). */
#define MINE_NOALLOC_MAX_SIDE 2048
int mine_align_pair_noalloc(const int64_t *src_sent_off, const int64_t *tgt_sent_off, int32_t n, int32_t m,
                            const uint8_t *counts, const mine_params *params, int32_t *link_i,
                            int32_t *link_j, float *link_s, int32_t *n_links, float *pair_score,
                            miner_stream_t stream);

const char *mine_strerror(int code);
/* The cudaError_t value behind the last MINE_ECUDA of this thread. */
int mine_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GB300_MINER_H */
