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
