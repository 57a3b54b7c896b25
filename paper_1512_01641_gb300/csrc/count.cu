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
// Strip kernel: one warp owns 32 source rows (a strip) and sweeps all column
// blocks of the pair.  The row table is built once per strip:
//   RT[t] = 32-bit mask of the strip's rows i with t in T_i (T_i = dictionary
//           translations of source sentence i),
// and every row keeps, in shared memory, the list of RT slots of its
// translations in position order (last translation of a position flagged).
// Per 32-column block:
//   column pass: lane j looks up each token of target sentence j in RT; a hit
//     adds RT[t] into the mt counters (mt for 32 rows) and sets bit j of the
//     slot's column mask;
//   row pass: lane i walks its slot list; the column masks of a position's
//     translations OR into h (bit j: the position is matched in column j), and
//     h is added into the ms counters (ms for 32 columns).
// No dictionary or hash work is left in the row pass, and the table build is
// paid once per strip instead of once per block.
template <int LOG_SLOTS, int LCAP>
struct StripSmem {
    static constexpr int S = 1 << LOG_SLOTS;
    int32_t key[S];
    uint32_t rowmask[S];
    uint32_t colmask[S];  // also holds the two 32 x 36 byte transpose tiles after the row pass
    uint16_t list[32][LCAP];
};
static_assert(sizeof(uint32_t) * 1024 >= 2 * 32 * kPad, "transpose tiles alias the column masks");

constexpr uint16_t kEndPos = 0x8000u;
// Per-row slot-list capacity: an odd number of 32-bit words per row keeps the
// lanes' list reads on distinct banks.
static_assert((kStripListCap / 2) % 2 == 1, "row lists need an odd word stride");

template <int LOG_SLOTS, int K, int LCAP>
__global__ void __launch_bounds__(32 * kCountWarps)
count_strip_kernel(DevCorpus src, DevCorpus tgt, DevDict dict, const PairGeom *__restrict__ geom,
                   const CountStripItem *__restrict__ items, int64_t n_items, uint8_t *__restrict__ counts,
                   uint32_t *status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using Smem = StripSmem<LOG_SLOTS, LCAP>;
    constexpr int S = Smem::S;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Smem &sm = reinterpret_cast<Smem *>(smem_raw)[warp];
    uint8_t(*ms_t)[kPad] = reinterpret_cast<uint8_t(*)[kPad]>(sm.colmask);
    uint8_t(*mt_t)[kPad] = reinterpret_cast<uint8_t(*)[kPad]>(reinterpret_cast<uint8_t *>(sm.colmask) + 32 * kPad);

    for (int64_t it = (int64_t)blockIdx.x * kCountWarps + warp; it < n_items;
         it += (int64_t)gridDim.x * kCountWarps) {
        const CountStripItem item = items[it];
        const PairGeom g = geom[item.pair];
        const int r0 = item.strip * 32;
        const bool rv = lane >= item.r_lo && lane < item.r_hi && r0 + lane < g.n;
        const int nr = min(item.r_hi, g.n - r0);  // rows [r_lo, nr) of the strip are written
        for (int x = lane; x < S; x += 32) {
            sm.key[x] = kEmpty;
            sm.rowmask[x] = 0u;
        }
        __syncwarp();

        // row table + slot lists
        int n_list = 0;
        if (rv) {
            const int64_t ssent = src.doc[item.pair] + r0 + lane;
            const int64_t p0 = src.sent[ssent], p1 = src.sent[ssent + 1];
            for (int64_t p = p0; p < p1; ++p) {
                const int32_t v = src.tok[p];
                const int32_t e0 = dict.off[v], e1 = dict.off[v + 1];
                for (int32_t e = e0; e < e1; ++e) {
                    const int h = table_insert<LOG_SLOTS>(sm.key, dict.tgt[e]);
                    if (h < 0 || n_list >= LCAP) {
                        atomicOr(status, kStTableFull);
                        break;
                    }
                    atomicOr(&sm.rowmask[h], 1u << lane);
                    sm.list[lane][n_list++] = (uint16_t)h | (e + 1 == e1 ? kEndPos : 0u);
                }
            }
        }
        __syncwarp();

        const int nblk = (g.m + 31) >> 5;
        const int64_t tdoc = tgt.doc[item.pair];
        uint8_t *out_strip = counts + 2 * (g.cell_off + (int64_t)r0 * g.m);
        for (int jb = 0; jb < nblk; ++jb) {
            const int c0 = jb * 32;
            const int nc = min(32, g.m - c0);
            for (int x = lane; x < S; x += 32) sm.colmask[x] = 0u;
            __syncwarp();
            // column pass: mt for 32 rows of column c0 + lane
            BitCounter<K> mt;
            mt.clear();
            if (lane < nc) {
                const int64_t q0 = tgt.sent[tdoc + c0 + lane], q1 = tgt.sent[tdoc + c0 + lane + 1];
                uint32_t b0 = 0, b1 = 0, b2 = 0;
                int nbuf = 0;
                for (int64_t q = q0; q < q1; ++q) {
                    const int slot = table_find<LOG_SLOTS>(sm.key, tgt.tok[q]);
                    if (slot < 0) continue;
                    const uint32_t rm = sm.rowmask[slot];
                    atomicOr(&sm.colmask[slot], 1u << lane);
                    if (nbuf == 3) {
                        mt.add4(b0, b1, b2, rm);
                        nbuf = 0;
                    } else {
                        b2 = b1;
                        b1 = b0;
                        b0 = rm;
                        ++nbuf;
                    }
                }
                if (nbuf > 0) mt.add4(b0, nbuf > 1 ? b1 : 0u, nbuf > 2 ? b2 : 0u, 0u);
            }
            __syncwarp();
            // row pass: ms for 32 columns of row r0 + lane
            BitCounter<K> ms;
            ms.clear();
            if (rv) {
                uint32_t b0 = 0, b1 = 0, b2 = 0, h = 0;
                int nbuf = 0;
                for (int x = 0; x < n_list; ++x) {
                    const uint16_t ent = sm.list[lane][x];
                    h |= sm.colmask[ent & 0x7FFF];
                    if (ent & kEndPos) {
                        if (nbuf == 3) {
                            ms.add4(b0, b1, b2, h);
                            nbuf = 0;
                        } else {
                            b2 = b1;
                            b1 = b0;
                            b0 = h;
                            ++nbuf;
                        }
                        h = 0;
                    }
                }
                if (nbuf > 0) ms.add4(b0, nbuf > 1 ? b1 : 0u, nbuf > 2 ? b2 : 0u, 0u);
            }
            __syncwarp();
            // expand, transpose (tiles alias the column masks), write
            uint32_t w[8];
            ms.to_bytes(w);
#pragma unroll
            for (int m = 0; m < 8; ++m) *reinterpret_cast<uint32_t *>(&ms_t[lane][4 * m]) = w[m];
            mt.to_bytes(w);
#pragma unroll
            for (int m = 0; m < 8; ++m) *reinterpret_cast<uint32_t *>(&mt_t[lane][4 * m]) = w[m];
            __syncwarp();
            if (lane < nc) {
                for (int i = item.r_lo; i < nr; ++i) {
                    const uchar2 v = make_uchar2(ms_t[i][lane], mt_t[lane][i]);
                    reinterpret_cast<uchar2 *>(out_strip + 2 * ((int64_t)i * g.m + c0))[lane] = v;
                }
            }
            __syncwarp();
        }
    }
}

template <int LOG_SLOTS, int K>
cudaError_t launch_strip_t(const DevCorpus &src, const DevCorpus &tgt, const DevDict &dict,
                           const PairGeom *geom, const CountStripItem *items, int64_t n_items,
                           uint8_t *counts, uint32_t *status, int n_sms, cudaStream_t st) {
    constexpr int LCAP = kStripListCap;
    const size_t smem = sizeof(StripSmem<LOG_SLOTS, LCAP>) * kCountWarps;
    auto kern = count_strip_kernel<LOG_SLOTS, K, LCAP>;
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

// Translation totals of every 32-row strip (sizes the row tables) and the
// largest per-sentence total (sizes the slot lists).
__global__ void strip_translations_kernel(DevCorpus src, DevDict dict, const PairGeom *__restrict__ geom,
                                          const int64_t *__restrict__ strip_off, int64_t n_pairs,
                                          int32_t *__restrict__ strip_tr, int32_t *__restrict__ max_row) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_pairs; k += stride) {
        const int N = geom[k].n;
        const int64_t base = src.doc[k];
        int best = 0;
        for (int s = 0; s * 32 < N; ++s) {
            int64_t tot = 0;
            for (int r = s * 32; r < min(N, s * 32 + 32); ++r) {
                int row = 0;
                for (int64_t p = src.sent[base + r]; p < src.sent[base + r + 1]; ++p) {
                    const int32_t v = src.tok[p];
                    row += dict.off[v + 1] - dict.off[v];
                }
                best = max(best, row);
                tot += row;
            }
            strip_tr[strip_off[k] + s] = (int32_t)(tot < 0x7fffffffLL ? tot : 0x7fffffffLL);
        }
        atomicMax(max_row, best);
    }
}

}  // namespace

cudaError_t launch_strip_translations(const DevCorpus &src, const DevDict &dict, const PairGeom *geom,
                                      const int64_t *strip_off, int64_t n_pairs, int32_t *strip_tr,
                                      int32_t *max_row, cudaStream_t st) {
    if (n_pairs == 0) return cudaSuccess;
    const int64_t blocks = (n_pairs + 127) / 128;
    strip_translations_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 128, 0, st>>>(
        src, dict, geom, strip_off, n_pairs, strip_tr, max_row);
    return cudaGetLastError();
}

cudaError_t launch_count_strips(const DevCorpus &src, const DevCorpus &tgt, const DevDict &dict,
                                const PairGeom *geom, const CountStripItem *items, int64_t n_items,
                                int log_slots, int planes, uint8_t *counts, uint32_t *status, int n_sms,
                                cudaStream_t st) {
    if (n_items == 0) return cudaSuccess;
    if (log_slots == 11)
        return planes <= 5 ? launch_strip_t<11, 5>(src, tgt, dict, geom, items, n_items, counts, status, n_sms, st)
                           : launch_strip_t<11, 8>(src, tgt, dict, geom, items, n_items, counts, status, n_sms, st);
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
