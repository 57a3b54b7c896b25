// Overlap counts (ms, mt) of every cell: the integer inputs of Section 4's
// sentence-similarity classifier.
//
// One warp owns a 32 x 32 cell block (32 source rows x 32 target columns):
//   1. column pass: lane j inserts the tokens of target sentence j into a
//      shared-memory hash table keyed by target id; each slot keeps a 32-bit
//      mask of the columns whose sentence contains that id;
//   2. row pass: lane i walks source sentence i; for each position it ORs the
//      column masks of the position's dictionary translations into h (bit j
//      set iff some translation occurs in target sentence j) and adds h into
//      bit-sliced counters -> ms for all 32 columns at once; every translation
//      that hits also ORs bit i into its slot's row mask;
//   3. mt pass: lane j walks target sentence j again and adds the row mask of
//      each of its tokens into bit-sliced counters -> mt for all 32 rows;
//   4. the counters are expanded to bytes, transposed through shared memory,
//      and written as (ms, mt) byte pairs, one coalesced row at a time.
// Positions are counted with multiplicity on both sides, exactly as the
// definitions read: a source position counts once however many of its
// translations hit; a target position counts once however many source tokens
// translate to it.
#include <algorithm>
#include <cstddef>

#include "kernels.h"

namespace gbm {
namespace {

constexpr int kCountWarps = 2;
constexpr int kPad = 36;  // bytes per row of the transpose tiles (bank spread)

template <int LOG_SLOTS>
struct CountSmem {
    static constexpr int S = 1 << LOG_SLOTS;
    int32_t key[S];
    uint32_t colmask[S];
    uint32_t rowmask[S];
    uint8_t ms_t[32][kPad];  // [row][col]
    uint8_t mt_t[32][kPad];  // [col][row]
};

template <int LOG_SLOTS>
__device__ __forceinline__ int table_insert(int32_t *key, int32_t t) {
    constexpr uint32_t S = 1u << LOG_SLOTS;
    uint32_t h = hash_slot(t, LOG_SLOTS);
    for (uint32_t n = 0; n < S; ++n) {
        int32_t old = atomicCAS(&key[h], kEmpty, t);
        if (old == kEmpty || old == t) return (int)h;
        h = (h + 1) & (S - 1);
    }
    return -1;
}

// Continues a lookup of t at slot h (after a first probe that found
// neither t nor an empty slot).
template <int LOG_SLOTS>
__device__ __forceinline__ int table_find_from(const int32_t *key, int32_t t, uint32_t h) {
    constexpr uint32_t S = 1u << LOG_SLOTS;
    for (uint32_t n = 1; n < S; ++n) {
        const int32_t k = key[h];
        if (k == t) return (int)h;
        if (k == kEmpty) return -1;
        h = (h + 1) & (S - 1);
    }
    return -1;
}

template <int LOG_SLOTS>
__device__ __forceinline__ int table_find(const int32_t *key, int32_t t) {
    constexpr uint32_t S = 1u << LOG_SLOTS;
    uint32_t h = hash_slot(t, LOG_SLOTS);
    for (uint32_t n = 0; n < S; ++n) {
        int32_t k = key[h];
        if (k == t) return (int)h;
        if (k == kEmpty) return -1;
        h = (h + 1) & (S - 1);
    }
    return -1;
}

template <int LOG_SLOTS, int K>
__global__ void __launch_bounds__(32 * kCountWarps)
count_kernel(DevCorpus src, DevCorpus tgt, DevDict dict, const PairGeom *__restrict__ geom,
             const CountItem *__restrict__ items, int64_t n_items, uint8_t *__restrict__ counts,
             uint32_t *status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using Smem = CountSmem<LOG_SLOTS>;
    constexpr int S = Smem::S;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Smem &sm = reinterpret_cast<Smem *>(smem_raw)[warp];

    for (int64_t it = (int64_t)blockIdx.x * kCountWarps + warp; it < n_items;
         it += (int64_t)gridDim.x * kCountWarps) {
        const CountItem item = items[it];
        const PairGeom g = geom[item.pair];
        const int r0 = (item.strip_block >> 16) * 32, c0 = (item.strip_block & 0xFFFF) * 32;
        const int nr = min(32, g.n - r0), nc = min(32, g.m - c0);
        const int64_t ssent = src.doc[item.pair] + r0 + lane;
        const int64_t tsent = tgt.doc[item.pair] + c0 + lane;

        for (int x = lane; x < S; x += 32) {
            sm.key[x] = kEmpty;
            sm.colmask[x] = 0u;
            sm.rowmask[x] = 0u;
        }
        __syncwarp();

        // 1. column pass
        int64_t tq0 = 0, tq1 = 0;
        if (lane < nc) {
            tq0 = tgt.sent[tsent];
            tq1 = tgt.sent[tsent + 1];
            for (int64_t q = tq0; q < tq1; ++q) {
                int h = table_insert<LOG_SLOTS>(sm.key, tgt.tok[q]);
                if (h < 0) { atomicOr(status, kStTableFull); break; }
                atomicOr(&sm.colmask[h], 1u << lane);
            }
        }
        __syncwarp();

        // 2. row pass: ms for 32 columns
        BitCounter<K> ms;
        ms.clear();
        if (lane < nr) {
            const int64_t p0 = src.sent[ssent], p1 = src.sent[ssent + 1];
            for (int64_t p = p0; p < p1; ++p) {
                const int32_t v = src.tok[p];
                uint32_t h = 0u;
                for (int32_t e = dict.off[v]; e < dict.off[v + 1]; ++e) {
                    int slot = table_find<LOG_SLOTS>(sm.key, dict.tgt[e]);
                    if (slot >= 0) {
                        h |= sm.colmask[slot];
                        atomicOr(&sm.rowmask[slot], 1u << lane);
                    }
                }
                ms.add(h);
            }
        }
        __syncwarp();

        // 3. mt pass: mt for 32 rows
        BitCounter<K> mt;
        mt.clear();
        if (lane < nc) {
            for (int64_t q = tq0; q < tq1; ++q) {
                int slot = table_find<LOG_SLOTS>(sm.key, tgt.tok[q]);
                mt.add(slot >= 0 ? sm.rowmask[slot] : 0u);
            }
        }

        // 4. expand, transpose, write
        uint32_t w[8];
        ms.to_bytes(w);
#pragma unroll
        for (int m = 0; m < 8; ++m) *reinterpret_cast<uint32_t *>(&sm.ms_t[lane][4 * m]) = w[m];
        mt.to_bytes(w);
#pragma unroll
        for (int m = 0; m < 8; ++m) *reinterpret_cast<uint32_t *>(&sm.mt_t[lane][4 * m]) = w[m];
        __syncwarp();
        uint8_t *out = counts + 2 * (g.cell_off + (int64_t)r0 * g.m + c0);
        for (int i = 0; i < nr; ++i) {
            if (lane < nc) {
                uchar2 v = make_uchar2(sm.ms_t[i][lane], sm.mt_t[lane][i]);
                reinterpret_cast<uchar2 *>(out + 2 * ((int64_t)i * g.m))[lane] = v;
            }
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Strip kernel: one CTA of four warps owns the rows of a 32-row strip (or a
// row group of it) and sweeps all 32-column blocks of the pair.  Once per
// strip a shared-memory hash table is built over the dictionary translations
// of the strip's source positions:  RT[t] = mask of the rows i with t in T_i;
// every translation entry is kept as (table slot, source position).  The
// four warps then work on one 32 x 32 block at a time:
//   column pass (all threads, token by token): every target token of the
//     block looks itself up in RT; a hit records RT[t] (which rows'
//     translation sets contain it) and sets the token's column bit in the
//     slot's column mask;
//   then, side by side: warp 0 adds column j's recorded row masks into
//     bit-sliced counters (mt of 32 rows at once, lane = column), while
//     warps 1-3 OR the column mask of every entry's slot into the entry's
//     position word (bit j: the position has a translation in sentence j;
//     most masks are 0, so few atomics);
//   then warp 1 adds row i's position words into bit-sliced counters (ms of
//     32 columns at once, lane = row), clears them and expands its counters
//     to bytes, warp 0 expands the mt counters, warp 2 clears the column
//     masks, and warp 3 stages the next block's target tokens (bulk async
//     copy) so that the copy overlaps the rest of this block;
//   finally all threads write the (ms, mt) bytes of the block, transposed
//     through shared memory, one coalesced row at a time.
// Counters are carry-save (four words per step), bytes are expanded by
// multiply-spread.  One table per CTA serves four warps, so an SM holds five
// CTAs (20 warps) where a table per warp allowed six warps.
constexpr int kStripWarps = 4;
constexpr int kStripThreads = 32 * kStripWarps;
constexpr int kEntCap = 1440;  // translation entries of one row group
constexpr int kPosCap = 992;   // source positions per strip item (32 rows x 31 tokens)
constexpr int kTokCap = 992;   // target tokens per column block (32 sentences x 31 tokens)
constexpr int kColRounds = (kTokCap + kStripThreads - 1) / kStripThreads;  // target tokens per thread

template <int LOG_SLOTS>
struct alignas(16) StripSmem {
    static constexpr int S = 1 << LOG_SLOTS;
    uint64_t bar;          // completion barrier of the bulk copies
    uint32_t pad[2];
    int32_t key[S];
    uint32_t rowmask[S];
    uint32_t colmask[S];
    uint32_t gh[kTokCap + 8];  // staged tokens: the strip's source tokens, then each block's target tokens
                               // (replaced in place by their row masks)
    uint32_t hpos[kPosCap];    // per source position: column mask of the current block
    uint32_t ent[kEntCap];     // per translation entry: table slot | position << 16
    uint8_t ms_t[32][kPad];    // [row][col]
    uint8_t mt_t[32][kPad];    // [col][row]
    uint8_t colid[kTokCap];
    uint8_t rowid[kPosCap];
    int32_t ctpre[33];         // per column of the staged block: first token index; [32] = token count
    int32_t n_ent;             // translation entries of the row table
    int32_t full;              // the row group does not fit
    int32_t tsh;               // index in gh of the staged block's first token
    int32_t pad2[3];
};
static_assert(kTokCap >= kPosCap, "shared buffer sizes");
static_assert(offsetof(StripSmem<11>, gh) % 16 == 0 && sizeof(StripSmem<11>) % 16 == 0, "bulk copy alignment");
static_assert(offsetof(StripSmem<11>, key) % 16 == 0 && offsetof(StripSmem<11>, rowmask) % 16 == 0 &&
                  offsetof(StripSmem<11>, colmask) % 16 == 0 && offsetof(StripSmem<11>, hpos) % 16 == 0 &&
                  kPosCap % 4 == 0,
              "16-byte clears");
constexpr int64_t kBulkWaitLimit = 1 << 22;

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Start staging tokens [a, a+n) of `tok` into buf (called by one warp):
// returns the index of token a in buf.  A bulk copy moves the 16-byte-aligned
// cover of the range when the array allows it (bulk = true, completes on
// bar); otherwise the warp copies with plain loads.
__device__ __forceinline__ int stage_issue(const int32_t *__restrict__ tok, int64_t n_total, int64_t a, int n,
                                           uint32_t *buf, uint64_t *bar, bool bulk_ok, int lane, bool &bulk) {
    const int64_t a16 = a & ~3LL, b16 = (a + n + 3) & ~3LL;
    const int shift = (int)(a - a16);
    bulk = bulk_ok && n > 0 && b16 <= n_total;
    if (bulk) {
        if (lane == 0) bulk_copy_g2s(buf, tok + a16, (uint32_t)((b16 - a16) * 4), bar);
    } else {
        for (int x = lane; x < n; x += 32) buf[shift + x] = (uint32_t)tok[a + x];
    }
    return shift;
}

// All threads: wait for the staged copy (if any), agreeing on the outcome.  On
// a copy that never completes the status is flagged and false is returned
// (after a second bounded wait that lets the copy in flight land).
__device__ __forceinline__ bool stage_wait(bool bulk, uint64_t *bar, uint32_t &phase, uint32_t *status) {
    bool ok = true;
    if (bulk) {
        ok = mbar_wait(bar, phase, kBulkWaitLimit);
        if (!ok) (void)mbar_wait(bar, phase, kBulkWaitLimit);
        phase ^= 1u;
    }
    ok = __syncthreads_and(ok) != 0;
    if (!ok && threadIdx.x == 0) atomicOr(status, kStTimeout);
    return ok;
}

// Each thread: wait for the staged copy (if any), with no CTA barrier.  On a
// copy that never completes the status is flagged (after a second bounded
// wait that lets the copy in flight land) and the thread carries on: every
// index the block derives from the staged words stays in bounds, and the host
// discards the results of a launch that flagged a timeout.
__device__ __forceinline__ void stage_wait_own(bool bulk, uint64_t *bar, uint32_t &phase, uint32_t *status) {
    if (!bulk) return;
    if (!mbar_wait(bar, phase, kBulkWaitLimit)) {
        (void)mbar_wait(bar, phase, kBulkWaitLimit);
        atomicOr(status, kStTimeout);
    }
    phase ^= 1u;
}

// Adds n 0/1 words from shared memory into the counters, four per step.
template <int K>
__device__ __forceinline__ void acc_words(BitCounter<K> &c, const uint32_t *w, int n) {
    int t = 0;
    for (; t + 4 <= n; t += 4) c.add4(w[t], w[t + 1], w[t + 2], w[t + 3]);
    if (t < n) c.add4(w[t], t + 1 < n ? w[t + 1] : 0u, t + 2 < n ? w[t + 2] : 0u, 0u);
}

// As acc_words, and clears the words.
template <int K>
__device__ __forceinline__ void acc_words_clear(BitCounter<K> &c, uint32_t *w, int n) {
    int t = 0;
    for (; t + 4 <= n; t += 4) {
        c.add4(w[t], w[t + 1], w[t + 2], w[t + 3]);
        w[t] = w[t + 1] = w[t + 2] = w[t + 3] = 0u;
    }
    for (; t < n; ++t) {
        c.add(w[t]);
        w[t] = 0u;
    }
}

__device__ __forceinline__ int warp_excl_scan(int v, int lane, int &total) {
    int x = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(kFull, x, off);
        if (lane >= off) x += y;
    }
    total = __shfl_sync(kFull, x, 31);
    return x - v;
}

// The row group of an item starts as the whole strip; when its translations
// would overfill the entry buffer (kEntCap entries, which also keeps the row
// table at most 71 % full: at most one key per entry), the group is halved and
// rebuilt -- rows are independent, so any grouping gives the same counts.
static_assert(kEntCap * 100 <= (1 << kStripLogSlots) * 71, "entry cap bounds the row table's load");

template <int LOG_SLOTS, int K>
__global__ void __launch_bounds__(kStripThreads, 5)
count_strip_kernel(DevCorpus src, DevCorpus tgt, DevDict dict, const PairGeom *__restrict__ geom,
                   const CountStripItem *__restrict__ items, int64_t n_items, bool bulk_ok,
                   uint8_t *__restrict__ counts, uint32_t *status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using Smem = StripSmem<LOG_SLOTS>;
    constexpr int S = Smem::S;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
    if (tid == 0) mbar_init(&sm.bar);
    // column masks and position words return to zero at the end of every
    // block (and stay zero when a row group is rebuilt): cleared once here
    for (int x = tid; x < S / 4; x += kStripThreads) reinterpret_cast<uint4 *>(sm.colmask)[x] = make_uint4(0, 0, 0, 0);
    for (int x = tid; x < kPosCap / 4; x += kStripThreads) reinterpret_cast<uint4 *>(sm.hpos)[x] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    uint32_t phase = 0;

    for (int64_t it = blockIdx.x; it < n_items; it += gridDim.x) {
        const CountStripItem item = items[it];
        const PairGeom g = geom[item.pair];
        const int r0 = item.strip * 32;
        const int rend = min(item.r_hi, g.n - r0);
        const int64_t ssent0 = src.doc[item.pair] + r0;
        const int64_t tdoc = tgt.doc[item.pair];
        const int nblk = (g.m + 31) >> 5;
        uint8_t *out_strip = counts + 2 * (g.cell_off + (int64_t)r0 * g.m);
        int group = 32;
        for (int g_lo = item.r_lo; g_lo < rend;) {
            const int g_hi = min(g_lo + group, rend);
            const bool rv = lane >= g_lo && lane < g_hi;
            // source positions of the group's rows, flattened (rows are
            // consecutive sentences, so their tokens are contiguous); every
            // warp scans the 32 row lengths for itself
            const int my_len = rv ? (int)(src.sent[ssent0 + lane + 1] - src.sent[ssent0 + lane]) : 0;
            int n_pos;
            const int prow = warp_excl_scan(my_len, lane, n_pos);
            const int64_t ptok0 = src.sent[ssent0 + g_lo];
            for (int x = tid; x < S / 4; x += kStripThreads) {
                reinterpret_cast<int4 *>(sm.key)[x] = make_int4(kEmpty, kEmpty, kEmpty, kEmpty);
                reinterpret_cast<uint4 *>(sm.rowmask)[x] = make_uint4(0, 0, 0, 0);
            }
            if (tid == 0) {
                sm.n_ent = 0;
                sm.full = 0;
            }
            if (warp == 0)
                for (int t = 0; t < my_len; ++t) sm.rowid[prow + t] = (uint8_t)lane;
            fence_proxy_async();
            __syncthreads();
            bool bulk = false;
            int ssh = 0;
            if (warp == 0) ssh = stage_issue(src.tok, src.n_tok, ptok0, n_pos, sm.gh, &sm.bar, bulk_ok, lane, bulk);
            if (tid == 0) sm.tsh = ssh | (bulk ? 1 << 30 : 0);  // for every warp
            __syncthreads();
            bulk = (sm.tsh >> 30) & 1;
            ssh = sm.tsh & ((1 << 30) - 1);
            if (!stage_wait(bulk, &sm.bar, phase, status)) return;
            const int32_t *stok = reinterpret_cast<const int32_t *>(sm.gh) + ssh;
            // row table: positions in rounds of 128; each warp takes its
            // round's entry offsets with one shared atomic
            for (int base = 0; base < n_pos; base += kStripThreads) {
                const int p = base + tid;
                int32_t e0 = 0, e1 = 0;
                if (p < n_pos) {
                    const int32_t v = stok[p];
                    e0 = dict.off[v];
                    e1 = dict.off[v + 1];
                }
                int tot;
                const int ex = warp_excl_scan(e1 - e0, lane, tot);
                int o = 0;
                if (lane == 0 && tot > 0) o = atomicAdd(&sm.n_ent, tot);
                o = __shfl_sync(kFull, o, 0) + ex;
                if (o + (e1 - e0) > kEntCap) {
                    sm.full = 1;
                    continue;
                }
                if (p < n_pos) {
                    const uint32_t rbit = 1u << sm.rowid[p];
                    // the position's translations, four loads at a time
                    for (int32_t e = e0; e < e1; e += 4) {
                        int32_t tt[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) tt[u] = e + u < e1 ? dict.tgt[e + u] : kEmpty;
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            if (e + u >= e1) break;
                            const int h = table_insert<LOG_SLOTS>(sm.key, tt[u]);
                            if (h < 0) {
                                sm.full = 1;
                                sm.ent[o + (e + u - e0)] = (uint32_t)p << 16;
                                continue;
                            }
                            atomicOr(&sm.rowmask[h], rbit);
                            sm.ent[o + (e + u - e0)] = (uint32_t)h | ((uint32_t)p << 16);
                        }
                    }
                }
            }
            fence_proxy_async();  // the source tokens are read before a copy replaces them
            __syncthreads();
            const bool full = sm.full != 0;
            const int n_ent = min(sm.n_ent, kEntCap);
            if (full) {
                __syncthreads();  // everyone has read the flags before the rebuild clears them
                if (group == 1) {  // one row alone does not fit: give up on this item
                    if (tid == 0) atomicOr(status, kStTableFull);
                    break;
                }
                group >>= 1;
                continue;
            }

            // stage block jb's target tokens (warp 3): column ids and token
            // offsets into shared memory, then the copy
            int64_t nx_lo = 0, nx_hi = 0;  // warp 3: sentence offsets of the next block to stage
            auto offsets = [&](int jb) {
                const int c = 32 * jb + lane;
                if (jb < nblk && c < g.m) {
                    nx_lo = tgt.sent[tdoc + c];
                    nx_hi = tgt.sent[tdoc + c + 1];
                } else {
                    nx_lo = nx_hi = 0;
                }
            };
            auto stage_block = [&](int jb, bool &bulk_b) {
                const int nc = min(32, g.m - 32 * jb);
                const int my_lt = lane < nc ? (int)(nx_hi - nx_lo) : 0;
                const int64_t ttok0 = __shfl_sync(kFull, nx_lo, 0);
                int n_tok;
                const int tpre = warp_excl_scan(my_lt, lane, n_tok);
                sm.ctpre[lane] = tpre;
                if (lane == 0) sm.ctpre[32] = n_tok;
                for (int t = 0; t < my_lt; ++t) sm.colid[tpre + t] = (uint8_t)lane;
                const int sh = stage_issue(tgt.tok, tgt.n_tok, ttok0, n_tok, sm.gh, &sm.bar, bulk_ok, lane, bulk_b);
                if (lane == 0) sm.tsh = sh | (bulk_b ? 1 << 30 : 0);
            };
            if (warp == 3) {
                bool b;
                offsets(0);
                stage_block(0, b);
                offsets(1);
            }
            __syncthreads();  // block 0's ctpre, colid, tsh; later blocks are staged before the
                              // barrier that ends the previous block's ms phase
            for (int jb = 0; jb < nblk; ++jb) {
                const int c0 = jb * 32;
                const int nc = min(32, g.m - c0);
                // no CTA barrier here: the previous block's output (tiles) and
                // this block's column pass (tokens, column masks) share no data,
                // so one warp's stores overlap another's lookups
                const int tshw = sm.tsh;
                stage_wait_own((tshw >> 30) & 1, &sm.bar, phase, status);
                const int n_tok = sm.ctpre[32];
                uint32_t *tg = sm.gh + (tshw & ((1 << 30) - 1));
                // column pass (each token's row mask replaces it in place): the
                // first probe of all of a thread's tokens goes out as one batch
                // of loads; the rare longer probe chains continue one by one
                {
                    int32_t tk[kColRounds];
                    uint32_t hs[kColRounds];
                    int32_t k0[kColRounds];
#pragma unroll
                    for (int k = 0; k < kColRounds; ++k) {
                        const int x = tid + kStripThreads * k;
                        tk[k] = x < n_tok ? (int32_t)tg[x] : kEmpty;
                        hs[k] = hash_slot(tk[k], LOG_SLOTS);
                        k0[k] = x < n_tok ? sm.key[hs[k]] : kEmpty;
                    }
#pragma unroll
                    for (int k = 0; k < kColRounds; ++k) {
                        if (kStripThreads * k >= n_tok) break;  // same in every thread
                        const int x = tid + kStripThreads * k;
                        if (x < n_tok) {
                            int slot = -1;
                            if (k0[k] == tk[k])
                                slot = (int)hs[k];
                            else if (k0[k] != kEmpty)
                                slot = table_find_from<LOG_SLOTS>(sm.key, tk[k], (hs[k] + 1) & (S - 1));
                            uint32_t rm = 0u;
                            if (slot >= 0) {
                                rm = sm.rowmask[slot];
                                atomicOr(&sm.colmask[slot], 1u << sm.colid[x]);
                            }
                            tg[x] = rm;
                        }
                    }
                }
                __syncthreads();
                BitCounter<K> mt;  // warp 0: mt of 32 rows for column `lane`
                if (warp == 0) {
                    mt.clear();
                    const int t0 = sm.ctpre[lane];
                    acc_words(mt, tg + t0, lane < nc ? (lane < 31 ? sm.ctpre[lane + 1] : n_tok) - t0 : 0);
                } else {
                    // row pass: entries' column masks into their positions' words
#pragma unroll 4
                    for (int e = tid - 32; e < n_ent; e += kStripThreads - 32) {
                        const uint32_t en = sm.ent[e];
                        const uint32_t cm = sm.colmask[en & 0xFFFFu];
                        if (cm) atomicOr(&sm.hpos[en >> 16], cm);
                    }
                }
                fence_proxy_async();
                __syncthreads();
                if (warp == 1) {
                    // ms of 32 columns for row `lane` (clears the position words)
                    BitCounter<K> ms;
                    ms.clear();
                    acc_words_clear(ms, sm.hpos + prow, my_len);
                    uint32_t w[8];
                    ms.to_bytes(w);
#pragma unroll
                    for (int m = 0; m < 8; ++m) *reinterpret_cast<uint32_t *>(&sm.ms_t[lane][4 * m]) = w[m];
                } else if (warp == 0) {
                    // mt bytes, beside the ms accumulation
                    uint32_t w[8];
                    mt.to_bytes(w);
#pragma unroll
                    for (int m = 0; m < 8; ++m) *reinterpret_cast<uint32_t *>(&sm.mt_t[lane][4 * m]) = w[m];
                } else if (warp == 3) {
                    if (jb + 1 < nblk) {
                        bool b;
                        stage_block(jb + 1, b);
                        offsets(jb + 2);
                    }
                } else {
                    for (int x = lane; x < S / 4; x += 32)
                        reinterpret_cast<uint4 *>(sm.colmask)[x] = make_uint4(0, 0, 0, 0);
                }
                __syncthreads();
                // write the block's rows of the group
                for (int x = tid; x < 32 * 32; x += kStripThreads) {
                    const int i = x >> 5, c = x & 31;
                    if (i >= g_lo && i < g_hi && c < nc) {
                        const uchar2 v = make_uchar2(sm.ms_t[i][c], sm.mt_t[c][i]);
                        reinterpret_cast<uchar2 *>(out_strip + 2 * ((int64_t)i * g.m + c0))[c] = v;
                    }
                }
            }
            __syncthreads();  // the last block's tiles and tokens are read before the next group or item
            g_lo = g_hi;
        }
    }
}

// ---------------------------------------------------------------------------
// Tile kernel: the same strip table, with the per-block work spread evenly
// over the CTA's four warps and no shared atomics outside the column pass.
//
// Once per strip (row group) the table of the strip's translations is built
// from a fixed-width copy of the dictionary (dict4: the 1..4 translations of
// a source id in one 16-byte load, -1 padded), every thread holding all of
// its positions' loads in flight at once.  Each source position keeps a
// record of its translations' table slots (four 16-bit slots, padding = a
// slot whose column mask is always 0).  Per 32 x 32 block:
//   column pass (all threads, token by token): each target token looks
//     itself up; a hit replaces the token by RT[t] (the rows whose
//     translation sets contain t) and sets the token's column bit in the
//     slot's column mask CM[slot] (the columns whose sentence contains t);
//   quarter passes: warp w takes the w-th quarter of every column's tokens
//     (lane = column: their row masks into bit-sliced counters, mt) and of
//     every row's positions (lane = row: h = OR of CM over the position's
//     slots, into bit-sliced counters, ms);
//   combine: every warp adds the four quarters (bit-sliced, 4 planes each)
//     and expands one quarter of the bytes: columns 8w..8w+7 of ms (lane =
//     row), rows 8w..8w+7 of mt (lane = column, through a transpose tile);
//   output: lane = row interleaves (ms, mt) pairs by byte permutes and
//     writes 16 bytes: straight into the blocked layout (one 2 KB tile per
//     32 x 32 block, row r at byte 64 r) or, row-major, through a tile.
// The counts are the same integers as the other count kernels compute.
constexpr int kTileWarps = 8;
constexpr int kTileThreads = 32 * kTileWarps;
constexpr int kTileSlots = 1 << kStripLogSlots;  // 2048
constexpr int kTileZero = kTileSlots;            // CM index that stays 0
constexpr int kTilePosRounds = (kPosCap + kTileThreads - 1) / kTileThreads;
constexpr int kTileTokRounds = (kTokCap + kTileThreads - 1) / kTileThreads;

struct alignas(16) TileSmem {
    uint64_t bar;                   // completion barrier of the staged target tokens
    int32_t n_ent;                  // translation entries of the row group
    int32_t tsh;                    // staged block: index in tg of its first token | bulk << 30
    int2 ent[kTileSlots];           // hash table: (target id, row mask of the rows translating to it)
    uint32_t cm[kTileSlots + 4];    // column masks of the current block; cm[kTileZero] stays 0
    uint2 prec[kPosCap];            // per source position: byte offsets into cm of its translations' slots
    uint32_t tg[kTokCap + 8];       // staged target tokens, replaced in place by their row masks
    uint32_t part[kTileWarps][4][32];  // per warp: 4 planes of its quarter counters; then the output tile
    uint8_t mt_t[32][36];           // mt bytes [column][row]
    uint8_t colid[kTokCap];
    uint8_t rowid[kPosCap];
    int32_t ctpre[33];              // per column of the staged block: first token index; [32] = total
};
static_assert(offsetof(TileSmem, tg) % 16 == 0 && offsetof(TileSmem, ent) % 16 == 0 &&
                  offsetof(TileSmem, cm) % 16 == 0 && 4 * (kTileSlots + 3) < 65536,
              "tile kernel shared layout");

// Insert t into the interleaved table (linear probing): its slot, or -1 if
// the table is full.
__device__ __forceinline__ int ent_insert(int2 *ent, int32_t t) {
    uint32_t h = hash_slot(t, kStripLogSlots);
    for (int n = 0; n < kTileSlots; ++n) {
        const int32_t old = atomicCAS(&ent[h].x, kEmpty, t);
        if (old == kEmpty || old == t) return (int)h;
        h = (h + 1) & (kTileSlots - 1);
    }
    return -1;
}

// Continue a lookup of t at slot h (after a first probe that found neither t
// nor an empty slot): the slot's entry, key kEmpty if t is absent.
__device__ __forceinline__ int ent_find_from(const int2 *ent, int32_t t, uint32_t h, uint32_t &rm) {
    for (int n = 1; n < kTileSlots; ++n) {
        const int2 e = ent[h];
        if (e.x == t) {
            rm = (uint32_t)e.y;
            return (int)h;
        }
        if (e.x == kEmpty) return -1;
        h = (h + 1) & (kTileSlots - 1);
    }
    return -1;
}
static_assert(kEntCap * 100 <= kTileSlots * 71, "entry cap bounds the tile table's load");

// Sum of four 4-plane bit-sliced counters (each lane: 32 counters of at most
// 8) into 5 planes: ripple adds with three-input XOR / majority.
__device__ __forceinline__ void add4x4(const uint32_t (&a)[4], const uint32_t (&b)[4], const uint32_t (&c)[4],
                                       const uint32_t (&d)[4], uint32_t (&r)[5]) {
    uint32_t x[5], y[5];
    uint32_t cx = 0u, cy = 0u;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        x[k] = a[k] ^ b[k] ^ cx;
        cx = (a[k] & b[k]) | (cx & (a[k] ^ b[k]));
        y[k] = c[k] ^ d[k] ^ cy;
        cy = (c[k] & d[k]) | (cy & (c[k] ^ d[k]));
    }
    x[4] = cx;
    y[4] = cy;
    uint32_t cz = 0u;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        r[k] = x[k] ^ y[k] ^ cz;
        cz = (x[k] & y[k]) | (cz & (x[k] ^ y[k]));
    }
}

// Bytes of the counters for bit positions 4m .. 4m+3 (byte r <- position 4m+r).
__device__ __forceinline__ uint32_t nibble_bytes(const uint32_t (&p)[5], int m) {
    uint32_t w = 0u;
#pragma unroll
    for (int k = 0; k < 5; ++k) w |= (((p[k] >> (4 * m)) & 0xFu) * (0x00204081u << k)) & (0x01010101u << k);
    return w;
}

// Fixed-width dictionary: entry v holds the translations of source id v, -1
// padded (every list has at most four entries).
__global__ void dict4_kernel(DevDict d, int32_t v_src, int4 *__restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < v_src; v += stride) {
        const int32_t e0 = d.off[v], n = d.off[v + 1] - e0;
        int4 q = make_int4(-1, -1, -1, -1);
        if (n > 0) q.x = d.tgt[e0];
        if (n > 1) q.y = d.tgt[e0 + 1];
        if (n > 2) q.z = d.tgt[e0 + 2];
        if (n > 3) q.w = d.tgt[e0 + 3];
        out[v] = q;
    }
}

template <bool BLOCKED>
__global__ void __launch_bounds__(kTileThreads, 5)
count_tile_kernel(DevCorpus src, DevCorpus tgt, const int4 *__restrict__ dict4, const PairGeom *__restrict__ geom,
                  const CountStripItem *__restrict__ items, int64_t n_items, int32_t *queue, bool bulk_ok,
                  uint8_t *__restrict__ counts, uint32_t *status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TileSmem &sm = *reinterpret_cast<TileSmem *>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) mbar_init(&sm.bar);
    for (int x = tid; x < (kTileSlots + 4) / 4; x += kTileThreads)
        reinterpret_cast<uint4 *>(sm.cm)[x] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    uint32_t phase = 0;
    __shared__ int32_t item_sh;

    for (;;) {
        __syncthreads();  // everyone has read the previous item's index
        if (tid == 0) item_sh = atomicAdd(queue, 1);
        __syncthreads();
        const int64_t it = item_sh;
        if (it >= n_items) break;
        const CountStripItem item = items[it];
        const PairGeom g = geom[item.pair];
        const int r0 = item.strip * 32;
        const int rend = min(item.r_hi, g.n - r0);
        const int64_t ssent0 = src.doc[item.pair] + r0;
        const int64_t tdoc = tgt.doc[item.pair];
        const int nblk = (g.m + 31) >> 5;
        int group = 32;
        for (int g_lo = item.r_lo; g_lo < rend;) {
            const int g_hi = min(g_lo + group, rend);
            const bool rv = lane >= g_lo && lane < g_hi;
            const int my_len = rv ? (int)(src.sent[ssent0 + lane + 1] - src.sent[ssent0 + lane]) : 0;
            int n_pos;
            const int prow = warp_excl_scan(my_len, lane, n_pos);
            const int64_t ptok0 = src.sent[ssent0 + g_lo];
            // the group's positions, all loads in flight at once
            const int prounds = (n_pos + kTileThreads - 1) / kTileThreads;  // the same in every thread
            int32_t v[kTilePosRounds];
#pragma unroll
            for (int k = 0; k < kTilePosRounds; ++k) {
                const int p = tid + kTileThreads * k;
                v[k] = p < n_pos ? src.tok[ptok0 + p] : -1;
            }
            int4 d4[kTilePosRounds];
            int cnt = 0;
#pragma unroll
            for (int k = 0; k < kTilePosRounds; ++k) {
                d4[k] = v[k] >= 0 ? __ldg(dict4 + v[k]) : make_int4(-1, -1, -1, -1);
            }
#pragma unroll
            for (int k = 0; k < kTilePosRounds; ++k) {
                cnt += (d4[k].x >= 0) + (d4[k].y >= 0) + (d4[k].z >= 0) + (d4[k].w >= 0);
            }
            for (int x = tid; x < kTileSlots / 2; x += kTileThreads)
                reinterpret_cast<int4 *>(sm.ent)[x] = make_int4(kEmpty, 0, kEmpty, 0);
            // row of every position: warp w writes positions 4w .. 4w+3 of each row
            for (int t = 4 * warp; t < min(4 * warp + 4, my_len); ++t) sm.rowid[prow + t] = (uint8_t)lane;
            if (tid == 0) sm.n_ent = 0;
            __syncthreads();
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) cnt += __shfl_xor_sync(kFull, cnt, off);
            if (lane == 0 && cnt) atomicAdd(&sm.n_ent, cnt);
            __syncthreads();
            if (sm.n_ent > kEntCap) {
                __syncthreads();  // everyone has read n_ent before the rebuild resets it
                if (group == 1) {
                    if (tid == 0) atomicOr(status, kStTableFull);
                    break;
                }
                group >>= 1;
                continue;
            }
            // inserts: row masks and the positions' slot records
#pragma unroll
            for (int k = 0; k < kTilePosRounds; ++k) {
                if (k >= prounds) break;
                const int p = tid + kTileThreads * k;
                if (p < n_pos) {
                    const uint32_t rbit = 1u << sm.rowid[p];
                    const int32_t tt[4] = {d4[k].x, d4[k].y, d4[k].z, d4[k].w};
                    uint32_t sl[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        sl[u] = 4u * kTileZero;
                        if (tt[u] >= 0) {
                            const int h = ent_insert(sm.ent, tt[u]);
                            if (h < 0) {
                                atomicOr(status, kStTableFull);
                            } else {
                                atomicOr(reinterpret_cast<uint32_t *>(&sm.ent[h].y), rbit);
                                sl[u] = 4u * (uint32_t)h;
                            }
                        }
                    }
                    sm.prec[p] = make_uint2(sl[0] | (sl[1] << 16), sl[2] | (sl[3] << 16));
                }
            }

            // stage block jb's target tokens (warp 3)
            int64_t nx_lo = 0, nx_hi = 0;
            auto offsets = [&](int jb) {
                const int c = 32 * jb + lane;
                if (jb < nblk && c < g.m) {
                    nx_lo = tgt.sent[tdoc + c];
                    nx_hi = tgt.sent[tdoc + c + 1];
                } else {
                    nx_lo = nx_hi = 0;
                }
            };
            auto stage_block = [&](int jb) {
                const int nc = min(32, g.m - 32 * jb);
                const int my_lt = lane < nc ? (int)(nx_hi - nx_lo) : 0;
                const int64_t ttok0 = __shfl_sync(kFull, nx_lo, 0);
                int n_tok;
                const int tpre = warp_excl_scan(my_lt, lane, n_tok);
                sm.ctpre[lane] = tpre;
                if (lane == 0) sm.ctpre[32] = n_tok;
                for (int t = 0; t < my_lt; ++t) sm.colid[tpre + t] = (uint8_t)lane;
                bool bulk_b;
                const int sh = stage_issue(tgt.tok, tgt.n_tok, ttok0, n_tok, sm.tg, &sm.bar, bulk_ok, lane, bulk_b);
                if (lane == 0) sm.tsh = sh | (bulk_b ? 1 << 30 : 0);
            };
            if (warp == kTileWarps - 1) {
                offsets(0);
                stage_block(0);
                offsets(1);
            }
            fence_proxy_async();
            __syncthreads();  // table, position records and block 0's staging complete

            // warps 0-3 count ms, warps 4-7 mt, each over a quarter of every row's
            // positions / every column's tokens
            const bool ms_warp = warp < 4;
            const int quarter = warp & 3;
            const int lq0 = (quarter * my_len) >> 2, lq1 = ((quarter + 1) * my_len) >> 2;
            for (int jb = 0; jb < nblk; ++jb) {
                const int c0 = jb * 32;
                const int nc = min(32, g.m - c0);
                const int tshw = sm.tsh;
                stage_wait_own((tshw >> 30) & 1, &sm.bar, phase, status);
                const int n_tok = sm.ctpre[32];
                uint32_t *tg = sm.tg + (tshw & ((1 << 30) - 1));
                // column pass
                const int trounds = (n_tok + kTileThreads - 1) / kTileThreads;  // the same in every thread
                uint32_t hit[kTileTokRounds];
                {
                    int32_t tk[kTileTokRounds];
                    uint32_t hs[kTileTokRounds];
                    int32_t k0[kTileTokRounds];
#pragma unroll
                    for (int k = 0; k < kTileTokRounds; ++k) {
                        if (k >= trounds) break;
                        const int x = tid + kTileThreads * k;
                        tk[k] = x < n_tok ? (int32_t)tg[x] : kEmpty;
                        hs[k] = hash_slot(tk[k], kStripLogSlots);
                        k0[k] = x < n_tok ? sm.ent[hs[k]].x : kEmpty;
                    }
#pragma unroll
                    for (int k = 0; k < kTileTokRounds; ++k) {
                        hit[k] = kTileZero;
                        if (k >= trounds) break;
                        const int x = tid + kTileThreads * k;
                        if (x < n_tok) {
                            int slot = -1;
                            uint32_t rm = 0u;
                            if (k0[k] == tk[k]) {
                                slot = (int)hs[k];
                                rm = (uint32_t)sm.ent[slot].y;
                            } else if (k0[k] != kEmpty) {
                                slot = ent_find_from(sm.ent, tk[k], (hs[k] + 1) & (kTileSlots - 1), rm);
                            }
                            if (slot >= 0) {
                                atomicOr(&sm.cm[slot], 1u << sm.colid[x]);
                                hit[k] = (uint32_t)slot;
                            }
                            tg[x] = rm;
                        }
                    }
                }
                __syncthreads();
                // quarter passes
                {
                    BitCounter<4> q4;
                    q4.clear();
                    if (!ms_warp && lane < nc) {
                        const int t0 = sm.ctpre[lane];
                        const int t1 = lane < 31 ? sm.ctpre[lane + 1] : n_tok;
                        const int L = t1 - t0;
                        acc_words(q4, tg + t0 + ((quarter * L) >> 2), (((quarter + 1) * L) >> 2) - ((quarter * L) >> 2));
                    }
                    int p = prow + lq0;
                    const int pe = ms_warp ? prow + lq1 : p;
                    const unsigned char *cmb = reinterpret_cast<const unsigned char *>(sm.cm);
                    auto cmw = [&](uint32_t off) { return *reinterpret_cast<const uint32_t *>(cmb + off); };
                    for (; p + 2 <= pe; p += 2) {
                        const uint2 a = sm.prec[p], b = sm.prec[p + 1];
                        const uint32_t ha = cmw(a.x & 0xFFFFu) | cmw(a.x >> 16) | cmw(a.y & 0xFFFFu) | cmw(a.y >> 16);
                        const uint32_t hb = cmw(b.x & 0xFFFFu) | cmw(b.x >> 16) | cmw(b.y & 0xFFFFu) | cmw(b.y >> 16);
                        q4.add(ha);
                        q4.add(hb);
                    }
                    if (p < pe) {
                        const uint2 a = sm.prec[p];
                        q4.add(cmw(a.x & 0xFFFFu) | cmw(a.x >> 16) | cmw(a.y & 0xFFFFu) | cmw(a.y >> 16));
                    }
#pragma unroll
                    for (int k = 0; k < 4; ++k) sm.part[warp][k][lane] = q4.p[k];
                }
                fence_proxy_async();  // this block's accesses to tg come before the next block's copy into it
                __syncthreads();
                // column masks back to zero (every hit slot; repeats are harmless)
#pragma unroll
                for (int k = 0; k < kTileTokRounds; ++k) {
                    if (k >= trounds) break;
                    if (tid + kTileThreads * k < n_tok) sm.cm[hit[k]] = 0u;
                }
                // the next block's tokens go out now (tg, ctpre, colid are free)
                if (warp == kTileWarps - 1 && jb + 1 < nblk) {
                    stage_block(jb + 1);
                    offsets(jb + 2);
                }
                // combine the quarters; expand a quarter of the bytes: ms warps
                // columns 8q .. 8q+7 of row `lane`, mt warps rows 8q .. 8q+7 of
                // column `lane` (into the transpose tile)
                uint32_t msw0 = 0u, msw1 = 0u;
                {
                    const int base = ms_warp ? 0 : 4;
                    uint32_t q[4][4];
#pragma unroll
                    for (int w = 0; w < 4; ++w)
#pragma unroll
                        for (int k = 0; k < 4; ++k) q[w][k] = sm.part[base + w][k][lane];
                    uint32_t c5[5];
                    add4x4(q[0], q[1], q[2], q[3], c5);
                    const uint32_t b0 = nibble_bytes(c5, 2 * quarter), b1 = nibble_bytes(c5, 2 * quarter + 1);
                    if (ms_warp) {
                        msw0 = b0;
                        msw1 = b1;
                    } else {
                        *reinterpret_cast<uint32_t *>(&sm.mt_t[lane][8 * quarter]) = b0;
                        *reinterpret_cast<uint32_t *>(&sm.mt_t[lane][8 * quarter + 4]) = b1;
                    }
                }
                __syncthreads();
                // interleave (ms, mt) for row `lane`, columns 8q .. 8q+7 (ms warps)
                if (ms_warp) {
                    const int c = 8 * quarter;
                    const uint32_t mA = (uint32_t)sm.mt_t[c][lane] | ((uint32_t)sm.mt_t[c + 1][lane] << 8) |
                                        ((uint32_t)sm.mt_t[c + 2][lane] << 16) | ((uint32_t)sm.mt_t[c + 3][lane] << 24);
                    const uint32_t mB = (uint32_t)sm.mt_t[c + 4][lane] | ((uint32_t)sm.mt_t[c + 5][lane] << 8) |
                                        ((uint32_t)sm.mt_t[c + 6][lane] << 16) | ((uint32_t)sm.mt_t[c + 7][lane] << 24);
                    const uint4 o = make_uint4(__byte_perm(msw0, mA, 0x5140), __byte_perm(msw0, mA, 0x7362),
                                               __byte_perm(msw1, mB, 0x5140), __byte_perm(msw1, mB, 0x7362));
                    if (BLOCKED) {
                        if (rv) {
                            uint8_t *tile = counts + g.tb_off * 64 + ((int64_t)item.strip * nblk + jb) * 2048;
                            *reinterpret_cast<uint4 *>(tile + 64 * lane + 16 * quarter) = o;
                        }
                    } else {
                        uint32_t *ot = &sm.part[0][0][0];  // [32][17] words: the block's rows, interleaved
                        ot[17 * lane + 4 * quarter] = o.x;
                        ot[17 * lane + 4 * quarter + 1] = o.y;
                        ot[17 * lane + 4 * quarter + 2] = o.z;
                        ot[17 * lane + 4 * quarter + 3] = o.w;
                    }
                }
                if (!BLOCKED) {
                    __syncthreads();
                    const uint32_t *ot = &sm.part[0][0][0];
                    uint8_t *out_strip = counts + 2 * (g.cell_off + (int64_t)r0 * g.m + c0);
#pragma unroll
                    for (int q = 0; q < 32 / kTileWarps; ++q) {
                        const int i = (32 / kTileWarps) * warp + q;
                        if (i >= g_lo && i < g_hi && lane < nc) {
                            const uint32_t wd = ot[17 * i + (lane >> 1)];
                            reinterpret_cast<uint16_t *>(out_strip + 2 * (int64_t)i * g.m)[lane] =
                                (uint16_t)(lane & 1 ? wd >> 16 : wd & 0xFFFFu);
                        }
                    }
                }
            }
            __syncthreads();  // the last block is done before the next group's build
            g_lo = g_hi;
        }
    }
}

template <int LOG_SLOTS, int K>
cudaError_t launch_strip_t(const DevCorpus &src, const DevCorpus &tgt, const DevDict &dict,
                           const PairGeom *geom, const CountStripItem *items, int64_t n_items, bool bulk_ok,
                           uint8_t *counts, uint32_t *status, int n_sms, cudaStream_t st) {
    const size_t smem = sizeof(StripSmem<LOG_SLOTS>);
    auto kern = count_strip_kernel<LOG_SLOTS, K>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kStripThreads, smem);
    if (e != cudaSuccess) return e;
    int64_t cap = (int64_t)n_sms * (per_sm > 0 ? per_sm : 1);
    int grid = (int)(n_items < cap ? n_items : cap);
    if (grid < 1) return cudaSuccess;
    kern<<<grid, kStripThreads, smem, st>>>(src, tgt, dict, geom, items, n_items, bulk_ok, counts, status);
    return cudaGetLastError();
}

template <int LOG_SLOTS, int K>
cudaError_t launch_count_t(const DevCorpus &src, const DevCorpus &tgt, const DevDict &dict,
                           const PairGeom *geom, const CountItem *items, int64_t n_items,
                           uint8_t *counts, uint32_t *status, int n_sms, cudaStream_t st) {
    const size_t smem = sizeof(CountSmem<LOG_SLOTS>) * kCountWarps;
    auto kern = count_kernel<LOG_SLOTS, K>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * kCountWarps, smem);
    if (e != cudaSuccess) return e;
    int64_t want = (n_items + kCountWarps - 1) / kCountWarps;
    int64_t cap = (int64_t)n_sms * (per_sm > 0 ? per_sm : 1);
    int grid = (int)(want < cap ? want : cap);
    if (grid < 1) return cudaSuccess;
    kern<<<grid, 32 * kCountWarps, smem, st>>>(src, tgt, dict, geom, items, n_items, counts, status);
    return cudaGetLastError();
}


}  // namespace

cudaError_t launch_count_strips(const DevCorpus &src, const DevCorpus &tgt, const DevDict &dict,
                                const PairGeom *geom, const CountStripItem *items, int64_t n_items,
                                int log_slots, int planes, bool bulk_ok, uint8_t *counts, uint32_t *status,
                                int n_sms, cudaStream_t st) {
    if (n_items == 0) return cudaSuccess;
    if (log_slots == 11)
        return planes <= 5
                   ? launch_strip_t<11, 5>(src, tgt, dict, geom, items, n_items, bulk_ok, counts, status, n_sms, st)
                   : launch_strip_t<11, 8>(src, tgt, dict, geom, items, n_items, bulk_ok, counts, status, n_sms, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_dict4(const DevDict &dict, int32_t v_src, int4 *dict4, cudaStream_t st) {
    const int64_t blocks = std::min<int64_t>((v_src + 255) / 256, 4096);
    dict4_kernel<<<(unsigned)(blocks > 0 ? blocks : 1), 256, 0, st>>>(dict, v_src, dict4);
    return cudaGetLastError();
}

cudaError_t launch_count_tiles(const DevCorpus &src, const DevCorpus &tgt, const int4 *dict4, const PairGeom *geom,
                               const CountStripItem *items, int64_t n_items, int32_t *queue, bool bulk_ok,
                               bool blocked, uint8_t *counts, uint32_t *status, int n_sms, cudaStream_t st) {
    if (n_items == 0) return cudaSuccess;
    const size_t smem = sizeof(TileSmem);
    auto kern = blocked ? count_tile_kernel<true> : count_tile_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTileThreads, smem);
    if (e != cudaSuccess) return e;
    const int64_t cap = (int64_t)n_sms * (per_sm > 0 ? per_sm : 1);
    const int grid = (int)(n_items < cap ? n_items : cap);
    e = cudaMemsetAsync(queue, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    kern<<<grid, kTileThreads, smem, st>>>(src, tgt, dict4, geom, items, n_items, queue, bulk_ok, counts, status);
    return cudaGetLastError();
}

cudaError_t launch_count(const DevCorpus &src, const DevCorpus &tgt, const DevDict &dict,
                         const PairGeom *geom, const CountItem *items, int64_t n_items,
                         int log_slots, int planes, uint8_t *counts, uint32_t *status,
                         int n_sms, cudaStream_t st) {
#define GBM_COUNT_CASE(L)                                                                      \
    case L:                                                                                    \
        return planes <= 5 ? launch_count_t<L, 5>(src, tgt, dict, geom, items, n_items, counts, \
                                                  status, n_sms, st)                           \
                           : launch_count_t<L, 8>(src, tgt, dict, geom, items, n_items, counts, \
                                                  status, n_sms, st);
    switch (log_slots) {
        GBM_COUNT_CASE(10)
        GBM_COUNT_CASE(11)
        GBM_COUNT_CASE(12)
        GBM_COUNT_CASE(13)
        default:
            return cudaErrorInvalidValue;
    }
#undef GBM_COUNT_CASE
}

}  // namespace gbm
