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

// As table_insert, and tells whether this call created the key.
template <int LOG_SLOTS>
__device__ __forceinline__ bool table_insert_new(int32_t *key, int32_t t, int &slot) {
    constexpr uint32_t S = 1u << LOG_SLOTS;
    uint32_t h = hash_slot(t, LOG_SLOTS);
    for (uint32_t n = 0; n < S; ++n) {
        const int32_t old = atomicCAS(&key[h], kEmpty, t);
        if (old == kEmpty || old == t) {
            slot = (int)h;
            return old == kEmpty;
        }
        h = (h + 1) & (S - 1);
    }
    slot = -1;
    return false;
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
// Strip kernel: one warp owns the rows of a 32-row strip (or a row group of
// it) and sweeps all 32-column blocks of the pair.  Once per strip a
// shared-memory hash table is built over the dictionary translations of the
// strip's source positions:  RT[t] = mask of the rows i with t in T_i.  Every
// source position keeps the table slots of its translations.  Per block:
//   column pass: every target token of the block looks itself up in RT; a hit
//     records RT[t] (which rows' translation sets contain it) and sets the
//     token's column bit in the slot's column mask;
//   mt: lane j adds the recorded row masks of column j's tokens into
//     bit-sliced counters (mt of 32 rows at once);
//   row pass: every source position ORs the column masks of its translations
//     (bit j: the position has a translation in target sentence j);
//   ms: lane i adds the masks of row i's positions into bit-sliced counters
//     (ms of 32 columns at once).
// The table build, the column pass and the row pass are spread over the 32
// lanes token by token (position by position), so no lane waits for the
// longest sentence; only the two accumulations run one row (column) per lane.
// Counters are carry-save (four words per step), bytes are expanded by
// multiply-spread and transposed through shared memory for coalesced writes.
constexpr int kEntCap = 1440;  // translation entries of one row group
constexpr int kPosCap = 992;   // source positions per strip item (32 rows x 31 tokens)
constexpr int kTokCap = 992;   // target tokens per column block (32 sentences x 31 tokens)

template <int LOG_SLOTS>
struct alignas(16) StripSmem {
    static constexpr int S = 1 << LOG_SLOTS;
    uint64_t bar;          // completion barrier of the bulk copies
    uint32_t pad[2];
    int32_t key[S];
    uint32_t rowmask[S];
    uint32_t colmask[S];
    // staged tokens (the strip's source tokens, then each block's target
    // tokens, replaced in place by their row masks), then the positions'
    // column masks, then the byte tiles
    uint32_t gh[kTokCap + 8];
    uint16_t ent[kEntCap];
    uint16_t pos_off[kPosCap + 2];
    uint8_t colid[kTokCap];
    uint8_t rowid[kPosCap];
    int32_t n_keys;  // distinct keys of the row table being built
    int32_t pad2[3];
};
static_assert(kTokCap >= kPosCap && kTokCap * 4 >= 2 * 32 * kPad, "shared buffer sizes");
static_assert(offsetof(StripSmem<11>, gh) % 16 == 0 && sizeof(StripSmem<11>) % 16 == 0, "bulk copy alignment");
constexpr int64_t kBulkWaitLimit = 1 << 22;

// Stage tokens [a, a+n) of `tok` into buf; returns the index of token a in
// buf.  A bulk copy moves the 16-byte-aligned cover of the range when the array
// allows it, plain loads otherwise.  On a copy that never completes the status
// is flagged and ok is cleared (the caller stops).
__device__ __forceinline__ int stage_tokens(const int32_t *__restrict__ tok, int64_t n_total, int64_t a, int n,
                                            uint32_t *buf, uint64_t *bar, uint32_t &phase, bool bulk_ok, int lane,
                                            uint32_t *status, bool &ok) {
    const int64_t a16 = a & ~3LL, b16 = (a + n + 3) & ~3LL;
    const int shift = (int)(a - a16);
    __syncwarp();
    if (bulk_ok && n > 0 && b16 <= n_total) {
        if (lane == 0) bulk_copy_g2s(buf, tok + a16, (uint32_t)((b16 - a16) * 4), bar);
        ok = mbar_wait(bar, phase, kBulkWaitLimit);
        phase ^= 1u;
        if (!ok) {
            if (lane == 0) atomicOr(status, kStTimeout);
            (void)mbar_wait(bar, phase ^ 1u, kBulkWaitLimit);  // let the copy in flight land
        }
    } else {
        for (int x = lane; x < n; x += 32) buf[shift + x] = (uint32_t)tok[a + x];
        ok = true;
    }
    __syncwarp();
    return shift;
}

// Carry-save accumulation of 0/1 words into bit-sliced counters, four at a time.
template <int K>
struct Acc4 {
    BitCounter<K> c;
    uint32_t b0 = 0, b1 = 0, b2 = 0;
    int n = 0;
    __device__ __forceinline__ void add(uint32_t x) {
        if (n == 3) {
            c.add4(b0, b1, b2, x);
            n = 0;
        } else {
            b2 = b1;
            b1 = b0;
            b0 = x;
            ++n;
        }
    }
    __device__ __forceinline__ void finish() {
        if (n > 0) c.add4(b0, n > 1 ? b1 : 0u, n > 2 ? b2 : 0u, 0u);
        n = 0;
    }
};

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
// would fill the row table beyond kMaxLoad (or the entry buffer), the group is
// halved and rebuilt -- rows are independent, so any grouping gives the same
// counts.
constexpr float kMaxLoad = 0.85f;

template <int LOG_SLOTS, int K>
__global__ void __launch_bounds__(32 * kCountWarps)
count_strip_kernel(DevCorpus src, DevCorpus tgt, DevDict dict, const PairGeom *__restrict__ geom,
                   const CountStripItem *__restrict__ items, int64_t n_items, bool bulk_ok,
                   uint8_t *__restrict__ counts, uint32_t *status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using Smem = StripSmem<LOG_SLOTS>;
    constexpr int S = Smem::S;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Smem &sm = reinterpret_cast<Smem *>(smem_raw)[warp];
    if (lane == 0) mbar_init(&sm.bar);
    __syncwarp();
    uint32_t phase = 0;
    uint8_t(*ms_t)[kPad] = reinterpret_cast<uint8_t(*)[kPad]>(sm.gh);
    uint8_t(*mt_t)[kPad] = reinterpret_cast<uint8_t(*)[kPad]>(reinterpret_cast<uint8_t *>(sm.gh) + 32 * kPad);

    for (int64_t it = (int64_t)blockIdx.x * kCountWarps + warp; it < n_items;
         it += (int64_t)gridDim.x * kCountWarps) {
        const CountStripItem item = items[it];
        const PairGeom g = geom[item.pair];
        const int r0 = item.strip * 32;
        const int rend = min(item.r_hi, g.n - r0);
        const int64_t ssent0 = src.doc[item.pair] + r0;
        int group = 32;
        for (int g_lo = item.r_lo; g_lo < rend;) {
            const int g_hi = min(g_lo + group, rend);
            const bool rv = lane >= g_lo && lane < g_hi;
            // source positions of the group's rows, flattened (rows are
            // consecutive sentences, so their tokens are contiguous)
            const int my_len = rv ? (int)(src.sent[ssent0 + lane + 1] - src.sent[ssent0 + lane]) : 0;
            int n_pos;
            const int prow = warp_excl_scan(my_len, lane, n_pos);
            const int64_t ptok0 = src.sent[ssent0 + g_lo];
            for (int x = lane; x < S; x += 32) {
                sm.key[x] = kEmpty;
                sm.rowmask[x] = 0u;
                sm.colmask[x] = 0u;
            }
            if (lane == 0) sm.n_keys = 0;
            for (int t = 0; t < my_len; ++t) sm.rowid[prow + t] = (uint8_t)lane;
            bool ok;
            const int32_t *stok = reinterpret_cast<const int32_t *>(sm.gh) +
                                  stage_tokens(src.tok, src.n_tok, ptok0, n_pos, sm.gh, &sm.bar, phase, bulk_ok, lane,
                                               status, ok);
            if (!ok) return;
            // translation entry offsets of the positions
            int carry = 0;
            for (int base = 0; base < n_pos; base += 32) {
                const int p = base + lane;
                int f = 0;
                if (p < n_pos) {
                    const int32_t v = stok[p];
                    f = dict.off[v + 1] - dict.off[v];
                }
                int tot;
                const int ex = warp_excl_scan(f, lane, tot);
                if (p < n_pos) sm.pos_off[p] = (uint16_t)min(carry + ex, 0xFFFF);
                carry += tot;
            }
            if (lane == 0) sm.pos_off[n_pos] = (uint16_t)min(carry, 0xFFFF);
            // row table
            bool full = carry > kEntCap;
            __syncwarp();
            if (!full) {
                for (int p = lane; p < n_pos; p += 32) {
                    const int32_t v = stok[p];
                    const int32_t e0 = dict.off[v], e1 = dict.off[v + 1];
                    const uint32_t rbit = 1u << sm.rowid[p];
                    const int o = sm.pos_off[p];
                    for (int32_t e = e0; e < e1; ++e) {
                        int h;
                        const bool fresh = table_insert_new<LOG_SLOTS>(sm.key, dict.tgt[e], h);
                        if (h < 0) {
                            sm.ent[o + (e - e0)] = 0;
                            continue;
                        }
                        if (fresh) atomicAdd(&sm.n_keys, 1);
                        atomicOr(&sm.rowmask[h], rbit);
                        sm.ent[o + (e - e0)] = (uint16_t)h;
                    }
                }
                __syncwarp();
                full = sm.n_keys > (int)(kMaxLoad * S);
            }
            if (full) {
                if (group == 1) {  // one row alone does not fit: give up on this item
                    if (lane == 0) atomicOr(status, kStTableFull);
                    break;
                }
                group >>= 1;
                continue;
            }

            const int nblk = (g.m + 31) >> 5;
            const int64_t tdoc = tgt.doc[item.pair];
            uint8_t *out_strip = counts + 2 * (g.cell_off + (int64_t)r0 * g.m);
            for (int jb = 0; jb < nblk; ++jb) {
                const int c0 = jb * 32;
                const int nc = min(32, g.m - c0);
                const int64_t ts = tdoc + c0;
                const int my_lt = lane < nc ? (int)(tgt.sent[ts + lane + 1] - tgt.sent[ts + lane]) : 0;
                int n_tok;
                const int tpre = warp_excl_scan(my_lt, lane, n_tok);
                const int64_t ttok0 = tgt.sent[ts];
                for (int t = 0; t < my_lt; ++t) sm.colid[tpre + t] = (uint8_t)lane;
                const int tsh = stage_tokens(tgt.tok, tgt.n_tok, ttok0, n_tok, sm.gh, &sm.bar, phase, bulk_ok, lane,
                                             status, ok);
                if (!ok) return;
                // column pass (each token's row mask replaces it in place)
                uint32_t *tg = sm.gh + tsh;
                for (int x = lane; x < n_tok; x += 32) {
                    const int slot = table_find<LOG_SLOTS>(sm.key, (int32_t)tg[x]);
                    uint32_t rm = 0u;
                    if (slot >= 0) {
                        rm = sm.rowmask[slot];
                        atomicOr(&sm.colmask[slot], 1u << sm.colid[x]);
                    }
                    tg[x] = rm;
                }
                __syncwarp();
                Acc4<K> mt;
                mt.c.clear();
                for (int t = 0; t < my_lt; ++t) mt.add(tg[tpre + t]);
                mt.finish();
                __syncwarp();
                // row pass
                for (int p = lane; p < n_pos; p += 32) {
                    uint32_t h = 0u;
                    const int e1 = sm.pos_off[p + 1];
                    for (int e = sm.pos_off[p]; e < e1; ++e) h |= sm.colmask[sm.ent[e]];
                    sm.gh[p] = h;
                }
                __syncwarp();
                Acc4<K> ms;
                ms.c.clear();
                for (int t = 0; t < my_len; ++t) ms.add(sm.gh[prow + t]);
                ms.finish();
                __syncwarp();
                for (int x = lane; x < S / 4; x += 32) reinterpret_cast<uint4 *>(sm.colmask)[x] = make_uint4(0, 0, 0, 0);
                // expand, transpose, write
                uint32_t w[8];
                ms.c.to_bytes(w);
#pragma unroll
                for (int m = 0; m < 8; ++m) *reinterpret_cast<uint32_t *>(&ms_t[lane][4 * m]) = w[m];
                mt.c.to_bytes(w);
#pragma unroll
                for (int m = 0; m < 8; ++m) *reinterpret_cast<uint32_t *>(&mt_t[lane][4 * m]) = w[m];
                __syncwarp();
                if (lane < nc) {
                    for (int i = g_lo; i < g_hi; ++i) {
                        const uchar2 v = make_uchar2(ms_t[i][lane], mt_t[lane][i]);
                        reinterpret_cast<uchar2 *>(out_strip + 2 * ((int64_t)i * g.m + c0))[lane] = v;
                    }
                }
                __syncwarp();
            }
            g_lo = g_hi;
        }
    }
}

template <int LOG_SLOTS, int K>
cudaError_t launch_strip_t(const DevCorpus &src, const DevCorpus &tgt, const DevDict &dict,
                           const PairGeom *geom, const CountStripItem *items, int64_t n_items, bool bulk_ok,
                           uint8_t *counts, uint32_t *status, int n_sms, cudaStream_t st) {
    const size_t smem = sizeof(StripSmem<LOG_SLOTS>) * kCountWarps;
    auto kern = count_strip_kernel<LOG_SLOTS, K>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * kCountWarps, smem);
    if (e != cudaSuccess) return e;
    int64_t want = (n_items + kCountWarps - 1) / kCountWarps;
    int64_t cap = (int64_t)n_sms * (per_sm > 0 ? per_sm : 1);
    int grid = (int)(want < cap ? want : cap);
    if (grid < 1) return cudaSuccess;
    kern<<<grid, 32 * kCountWarps, smem, st>>>(src, tgt, dict, geom, items, n_items, bulk_ok, counts, status);
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
