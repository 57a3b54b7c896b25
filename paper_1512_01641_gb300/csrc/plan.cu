// Plan creation, input validation and the C ABI entry points of miner.h.
#include <algorithm>
#include <mutex>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <numeric>
#include <vector>

#include "kernels.h"
#include "miner.h"

namespace gbm {
namespace {

thread_local int g_last_cuda = 0;

// ---------------------------------------------------------------- validation
__global__ void validate_corpus_kernel(DevCorpus c, int64_t n_sents, int64_t n_tok, int32_t vocab,
                                       uint32_t *status, int32_t *max_len) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n_sents; s += stride) {
        const int64_t a = c.sent[s], b = c.sent[s + 1];
        if (a < 0 || b > n_tok || b - a < 1 || b - a > 255) {
            atomicOr(status, kStBadSentOff);
            continue;
        }
        atomicMax(max_len, (int32_t)(b - a));
        int32_t prev = -1;
        for (int64_t x = a; x < b; ++x) {
            const int32_t t = c.tok[x];
            if (t < 0 || t >= vocab) atomicOr(status, kStBadToken);
            if (t < prev) atomicOr(status, kStUnsorted);
            prev = t;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (c.sent[0] != 0 || c.sent[n_sents] != n_tok) atomicOr(status, kStBadSentOff);
    }
}

__global__ void validate_dict_kernel(DevDict d, int32_t v_src, int32_t v_tgt, int64_t n_entries,
                                     uint32_t *status, int32_t *max_fanout) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < v_src; v += stride) {
        const int64_t a = d.off[v], b = d.off[v + 1];
        if (a < 0 || b > n_entries || b < a) {
            atomicOr(status, kStBadDict);
            continue;
        }
        atomicMax(max_fanout, (int32_t)(b - a < 0x7fffffffLL ? b - a : 0x7fffffffLL));
        int32_t prev = -1;
        for (int64_t e = a; e < b; ++e) {
            const int32_t t = d.tgt[e];
            if (t < 0 || t >= v_tgt || t <= prev) atomicOr(status, kStBadDict);
            prev = t;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (d.off[0] != 0 || d.off[v_src] != n_entries) atomicOr(status, kStBadDict);
    }
}

// Largest token total of any 32-sentence target block (sizes the count hash).
__global__ void block_tokens_kernel(DevCorpus tgt, const PairGeom *geom, int64_t n_pairs, int32_t *out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_pairs; k += stride) {
        const int M = geom[k].m;
        const int64_t base = tgt.doc[k];
        for (int c0 = 0; c0 < M; c0 += 32) {
            const int c1 = min(M, c0 + 32);
            const int64_t tot = tgt.sent[base + c1] - tgt.sent[base + c0];
            atomicMax(out, (int32_t)tot);
        }
    }
}

// Plan scratch comes from a library-owned stream-ordered memory pool per
// device that keeps up to kPoolKeep bytes of freed memory for reuse, so that
// creating and destroying plans batch after batch neither maps new memory nor
// synchronises the device (beyond kPoolKeep, freed memory goes back to the
// system at the next synchronisation).
constexpr int kMaxDevices = 64;
constexpr uint64_t kPoolKeep = 16ull << 30;
cudaError_t scratch_pool(int device, cudaMemPool_t *out) {
    static std::mutex mu;
    static cudaMemPool_t pools[kMaxDevices] = {};
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!pools[device]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        cudaError_t e = cudaMemPoolCreate(&pools[device], &props);
        if (e != cudaSuccess) return e;
        uint64_t keep = kPoolKeep;
        e = cudaMemPoolSetAttribute(pools[device], cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) return e;
    }
    *out = pools[device];
    return cudaSuccess;
}

template <class T>
cudaError_t dalloc(T **p, size_t n, int device, cudaStream_t st) {
    *p = nullptr;
    if (n == 0) n = 1;
    cudaMemPool_t pool;
    const cudaError_t e = scratch_pool(device, &pool);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync((void **)p, n * sizeof(T), pool, st);
}

// Pinned staging for the tables a plan builds on the host (geometry, pair
// order, work lists).  A copy from pageable memory goes through the driver's
// small staging buffers and returns only once the copy engine has taken it,
// so while a large input upload was in flight (mine_pairs_host) plan creation
// stalled at its first table copy until the inputs had landed, and its
// remaining host work ran after them.  From pinned memory the copies are
// queued and the host goes on.  One grow-only buffer per device, reused once
// the copies of its previous use have completed.
struct HostStage {
    std::mutex mu;
    char *buf = nullptr;
    size_t cap = 0;
    cudaEvent_t used = nullptr;
};
HostStage g_stage[kMaxDevices];

struct StagePiece {
    const void *h;
    void *d;
    size_t bytes;
};

// Copies every piece (host source, device destination, bytes) to the device
// on st through the device's staging buffer.
cudaError_t staged_upload(int device, const StagePiece *pcs, int n, cudaStream_t st) {
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    HostStage &S = g_stage[device];
    std::lock_guard<std::mutex> lock(S.mu);
    size_t total = 0;
    for (int i = 0; i < n; ++i) total += (pcs[i].bytes + 255) & ~(size_t)255;
    cudaError_t e = S.used ? cudaEventSynchronize(S.used) : cudaEventCreateWithFlags(&S.used, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    if (total > S.cap) {
        if (S.buf) {
            e = cudaFreeHost(S.buf);
            S.buf = nullptr;
            S.cap = 0;
            if (e != cudaSuccess) return e;
        }
        const size_t cap = std::max(total + total / 4, (size_t)1 << 20);
        e = cudaMallocHost((void **)&S.buf, cap);
        if (e != cudaSuccess) return e;
        S.cap = cap;
    }
    size_t off = 0;
    for (int i = 0; i < n; ++i) {
        if (pcs[i].bytes == 0) continue;
        std::memcpy(S.buf + off, pcs[i].h, pcs[i].bytes);
        e = cudaMemcpyAsync(pcs[i].d, S.buf + off, pcs[i].bytes, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return e;
        off += (pcs[i].bytes + 255) & ~(size_t)255;
    }
    return cudaEventRecord(S.used, st);
}

}  // namespace

void record_cuda_error(int e) { g_last_cuda = e; }

cudaError_t launch_validate_corpus(const DevCorpus &c, int64_t n_sents, int64_t n_tok, int32_t vocab,
                                   uint32_t *status, int32_t *max_len, cudaStream_t st) {
    int64_t blocks = std::min<int64_t>((n_sents + 255) / 256, 4096);
    validate_corpus_kernel<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, st>>>(c, n_sents, n_tok, vocab,
                                                                                   status, max_len);
    return cudaGetLastError();
}

cudaError_t launch_block_tokens(const DevCorpus &tgt, const PairGeom *geom, int64_t n_pairs,
                                int32_t *max_block_tokens, cudaStream_t st) {
    if (n_pairs == 0) return cudaSuccess;
    int64_t blocks = std::min<int64_t>((n_pairs + 255) / 256, 4096);
    block_tokens_kernel<<<(unsigned)blocks, 256, 0, st>>>(tgt, geom, n_pairs, max_block_tokens);
    return cudaGetLastError();
}

}  // namespace gbm

using namespace gbm;

// Planner knobs (defaults; the tuner may override them per plan).
struct PlanKnobs {
    int64_t tile_min_cells = 1 << 16;  // pairs with at least this many cells are tiled
    int tile_min_rows = 64;            // ... and at least this many rows
    int tile_cols = 64;                // column chunk width of a tile (multiple of 32)
    int64_t wait_limit = 1 << 24;      // bounded spin iterations of a tile wait (~200 ns each)
    int link_recount = 0;              // 1: recount link overlaps by warp vote
    int use_graph = 1;                 // 1: mine_pairs replays a captured CUDA graph
    int64_t skip_flag = -1;            // fault injection: tile flag never published (tests)
    int soft_split = 3;                // soft sweeps: 0 never / 1 long pairs / 2 all pairs / 3 all once one must
    int soft_split_q4 = 4;             // split = 1: above this many quarters of the mean chain per warp
    int soft_order = 1;                // soft work list: 0 per pair, 1 value sweeps/whole/adjoints, 2 value/adjoints/whole
    int64_t skip_soft = -1;            // fault injection: soft progress counter never published (tests)
};

struct mine_plan {
    DevCorpus src{}, tgt{};
    DevDict dict{};
    int64_t n_pairs = 0, n_cells = 0, link_cap = 0, n_count_items = 0, n_fill_items = 0, n_flags = 0;
    std::vector<int64_t> cell_off_h;
    std::vector<PairGeom> geom_h;
    std::vector<int32_t> pair_order_h;  // pairs by decreasing size
    int32_t *pair_order = nullptr;
    int64_t soft_rows = 0;              // sum over pairs of nstrips * M
    int64_t soft_strips = 0;            // sum over pairs of nstrips
    int64_t soft_ckw = 0;               // floats of the soft window checkpoints
    int32_t max_m = 0;
    PlanKnobs knobs;
    PairGeom *geom = nullptr;
    CountItem *count_items = nullptr;
    CountStripItem *strip_items = nullptr;
    int64_t n_strip_items = 0;
    bool use_strips = false;  // strip count kernel (else the per-block kernel)
    bool use_tiles = false;   // tile count kernel (sentences <= 31 tokens, fan-out <= 4); mine_pairs
                              // then keeps its counts in the blocked layout
    int4 *dict4 = nullptr;    // fixed-width dictionary of the tile kernel
    int32_t *count_queue = nullptr;
    int32_t v_src = 0;
    int64_t counts_bytes = 0;  // plan-owned count buffer (blocked layout when use_tiles)
    bool bulk_ok = false;     // token arrays 16-byte aligned: bulk-copy staging
    FillItem *fill_items = nullptr;
    uint8_t *counts = nullptr;
    AlignScratch S{};
    int32_t *stats = nullptr;  // [max src len, max tgt len, max block tokens, max dictionary fan-out]
    int log_slots = 11, planes = 5, n_sms = 1, device = 0;
    // per-kernel timing hook
    bool timing = false;
    struct Pending {
        int kind;
        cudaEvent_t a, b;
    };
    std::vector<Pending> pending;
    double total_ms[kKinds] = {};
    int64_t launches[kKinds] = {};
    // whole-batch CUDA graph of mine_pairs, keyed by the output buffers and
    // the parameters baked into its kernel arguments
    cudaStream_t cap_stream = nullptr;
    cudaStream_t own_stream = nullptr;  // plan-owned: releases the scratch, rebuilds work lists
    cudaEvent_t done = nullptr;         // recorded after the work of every call that used the plan
    cudaGraphExec_t graph = nullptr;
    mine_out graph_out{};
    mine_params graph_params{};
    int64_t graph_captures = 0;
    std::vector<int64_t> uc_off_h;  // per-pair workspace offsets of the unconstrained aligner
    std::vector<int32_t> uc_order_h;  // its pair order: short targets first (uc_n_short of them)
    int64_t uc_n_short = 0;
};

// Launch f() on stream st; with timing enabled, bracket it by two events.
template <class F>
static cudaError_t timed(mine_plan *p, int kind, cudaStream_t st, F &&f) {
    if (!p->timing) return f();
    mine_plan::Pending q{kind, nullptr, nullptr};
    cudaError_t e = cudaEventCreate(&q.a);
    if (e == cudaSuccess) e = cudaEventCreate(&q.b);
    if (e == cudaSuccess) e = cudaEventRecord(q.a, st);
    if (e == cudaSuccess) e = f();
    if (e == cudaSuccess) e = cudaEventRecord(q.b, st);
    if (e == cudaSuccess) {
        p->pending.push_back(q);
    } else {
        if (q.a) cudaEventDestroy(q.a);
        if (q.b) cudaEventDestroy(q.b);
    }
    return e;
}

// Records the plan's completion event on the caller's stream when a call
// that enqueued work returns (not while the plan captures its own graph).
struct DoneMark {
    mine_plan *p;
    cudaStream_t st;
    ~DoneMark() {
        if (p && p->done && st != p->cap_stream) cudaEventRecord(p->done, st);
    }
};

static void drain_pending(mine_plan *p) {
    for (auto &q : p->pending) {
        float ms = 0.0f;
        if (cudaEventSynchronize(q.b) == cudaSuccess && cudaEventElapsedTime(&ms, q.a, q.b) == cudaSuccess) {
            p->total_ms[q.kind] += ms;
            p->launches[q.kind] += 1;
        }
        cudaEventDestroy(q.a);
        cudaEventDestroy(q.b);
    }
    p->pending.clear();
}

#define MINE_CK(x)                   \
    do {                             \
        cudaError_t e_ = (x);        \
        if (e_ != cudaSuccess) {     \
            g_last_cuda = (int)e_;   \
            return MINE_ECUDA;       \
        }                            \
    } while (0)

static void drop_graph(mine_plan *p) {
    if (p->graph) cudaGraphExecDestroy(p->graph);
    p->graph = nullptr;
}

static void plan_free(mine_plan *p) {
    if (!p) return;
    drain_pending(p);
    drop_graph(p);
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    void *bufs[] = {p->geom, p->pair_order, p->count_items, p->strip_items, p->dict4, p->count_queue,
                    p->fill_items, p->counts, p->S.tb, p->S.hrow, p->S.vcol,
                    p->S.flags, p->S.queue, p->S.status, p->S.diag_i, p->S.diag_j, p->S.diag_s, p->S.n_diag,
                    p->S.diag_off, p->S.n_links, p->stats};
    // back to the pool after the work last enqueued on the plan (the
    // caller's streams may be gone by now: the plan waits on its own event)
    if (p->own_stream) {
        if (p->done) cudaStreamWaitEvent(p->own_stream, p->done, 0);
        for (void *b : bufs)
            if (b) cudaFreeAsync(b, p->own_stream);
        cudaStreamDestroy(p->own_stream);
    }
    if (p->done) cudaEventDestroy(p->done);
    delete p;
}

static int validate_dict(const mine_dict *d, uint32_t *status, int32_t *max_fanout, cudaStream_t st) {
    int64_t blocks = std::min<int64_t>((d->v_src + 255) / 256, 4096);
    gbm::validate_dict_kernel<<<(unsigned)blocks, 256, 0, st>>>(DevDict{d->off, d->tgt}, d->v_src, d->v_tgt,
                                                                d->n_entries, status, max_fanout);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        g_last_cuda = (int)e;
        return MINE_ECUDA;
    }
    return MINE_OK;
}

// Indices 0..n-1 ordered by key (ascending, ties by index): a stable LSD
// radix sort on 11-bit digits; a pass whose digit is the same for every key
// is skipped (sizes fit two or three digits).
static void radix_order(const std::vector<uint64_t> &key, std::vector<int32_t> &order) {
    constexpr int kBits = 11;
    constexpr uint64_t kMask = (1u << kBits) - 1;
    const size_t n = key.size();
    std::vector<int32_t> a(n), b(n);
    std::iota(a.begin(), a.end(), 0);
    std::vector<uint32_t> cnt(kMask + 2);
    for (int shift = 0; shift < 64 && n > 1; shift += kBits) {
        const uint64_t d0 = (key[0] >> shift) & kMask;
        bool same = true;
        for (size_t i = 1; i < n && same; ++i) same = ((key[i] >> shift) & kMask) == d0;
        if (same) continue;
        std::fill(cnt.begin(), cnt.end(), 0u);
        for (size_t i = 0; i < n; ++i) ++cnt[((key[i] >> shift) & kMask) + 1];
        for (size_t d = 1; d < cnt.size(); ++d) cnt[d] += cnt[d - 1];
        for (size_t i = 0; i < n; ++i) b[cnt[(key[a[i]] >> shift) & kMask]++] = a[i];
        a.swap(b);
    }
    order.swap(a);
}

// Geometry, tiling and work order.  Tiled pairs are cut into 32-row x
// tile_cols tiles listed in anti-diagonal order (every tile after the tile
// above it and the tile to its left); whole small pairs (largest first) are
// interleaved between the diagonals so that warps find ready work while the
// wavefronts of the large pairs advance.
static void build_geometry(mine_plan *p, const std::vector<int64_t> &sd, const std::vector<int64_t> &td,
                           std::vector<FillItem> &fitems, int64_t &tbw, int64_t &hrow, int64_t &vcol) {
    const int64_t n = p->n_pairs;
    const PlanKnobs &K = p->knobs;
    p->geom_h.assign(n, PairGeom{});
    p->cell_off_h.assign(n + 1, 0);
    p->soft_rows = 0;
    p->soft_strips = 0;
    p->soft_ckw = 0;
    p->max_m = 0;
    int64_t cell = 0, link = 0, flags = 0;
    tbw = hrow = vcol = 0;
    // every work order below comes from one order of the pairs by size
    std::vector<uint64_t> size_key((size_t)n);  // ascending key = descending cells
    for (int64_t k = 0; k < n; ++k) {
        PairGeom &g = p->geom_h[k];
        g.n = (int32_t)(sd[k + 1] - sd[k]);
        g.m = (int32_t)(td[k + 1] - td[k]);
        g.cell_off = cell;
        g.tb_off = tbw;
        g.link_off = link;
        g.hrow_off = hrow;
        g.vcol_off = vcol;
        g.soft_off = p->soft_rows;
        g.ckw_off = p->soft_ckw;
        p->soft_ckw += ((g.n + 31) / 32) * soft_ckw_floats(g.m);
        p->soft_rows += ((g.n + 31) / 32) * (int64_t)g.m;
        p->soft_strips += (g.n + 31) / 32;
        p->max_m = std::max(p->max_m, g.m);
        p->cell_off_h[k] = cell;
        const int64_t ns = (g.n + 31) / 32, nb = (g.m + 31) / 32;
        const int64_t cells = (int64_t)g.n * g.m;
        const bool tile = cells >= K.tile_min_cells && g.n >= K.tile_min_rows && g.m > K.tile_cols;
        if (tile) {
            g.cw = K.tile_cols;
            g.nchunk = (g.m + g.cw - 1) / g.cw;
            g.flag_off = flags;
            flags += ns * g.nchunk;
        } else {
            g.cw = (int32_t)std::max<int64_t>(32, nb * 32);
            g.nchunk = 1;
            g.flag_off = -1;
        }
        size_key[(size_t)k] = (uint64_t)((int64_t)1 << 62) - (uint64_t)cells;
        cell += cells;
        tbw += ns * nb * 32;
        link += std::min(g.n, g.m);
        hrow += g.m;
        vcol += g.n;
    }
    p->cell_off_h[n] = cell;
    p->n_cells = cell;
    p->link_cap = link;
    p->n_flags = flags;

    // pairs by decreasing size, ties by index
    radix_order(size_key, p->pair_order_h);
    std::vector<int32_t> small, tiled;
    for (int32_t k : p->pair_order_h) {
        if (p->geom_h[k].flag_off >= 0)
            tiled.push_back(k);
        else if ((int64_t)p->geom_h[k].n * p->geom_h[k].m > 0)
            small.push_back(k);
    }

    // fill items: anti-diagonal d of the tile wavefronts holds the tiles
    // (s, c) with s + c = d of every tiled pair (pairs in size order, strips
    // ascending), and after each diagonal's tiles come per_diag whole small
    // pairs.  The tiles are bucketed by diagonal in one pass (a counting
    // sort, stable in pair and strip order), not found by a scan of every
    // pair's strips for every diagonal.
    fitems.clear();
    int64_t max_diag = 0, n_tiles = 0;
    for (int32_t k : tiled) {
        const PairGeom &g = p->geom_h[k];
        max_diag = std::max<int64_t>(max_diag, (g.n + 31) / 32 + g.nchunk - 1);
        n_tiles += (int64_t)((g.n + 31) / 32) * g.nchunk;
    }
    std::vector<int64_t> dpos((size_t)max_diag + 1, 0);
    for (int32_t k : tiled) {
        const PairGeom &g = p->geom_h[k];
        for (int s = 0; s < (g.n + 31) / 32; ++s) {  // diagonals s .. s + nchunk - 1, one tile each
            ++dpos[(size_t)s];
            --dpos[(size_t)(s + g.nchunk)];
        }
    }
    for (int64_t d = 0, run = 0, at = 0; d <= max_diag; ++d) {  // tiles per diagonal -> first index
        run += dpos[(size_t)d];
        dpos[(size_t)d] = at;
        at += run;
    }
    std::vector<FillItem> tiles((size_t)n_tiles);
    {
        std::vector<int64_t> put(dpos.begin(), dpos.end());
        for (int32_t k : tiled) {
            const PairGeom &g = p->geom_h[k];
            for (int s = 0; s < (g.n + 31) / 32; ++s)
                for (int32_t cj = 0; cj < g.nchunk; ++cj) tiles[(size_t)put[(size_t)(s + cj)]++] = {k, s, s + 1, cj};
        }
    }
    fitems.reserve((size_t)n_tiles + small.size());
    const int64_t per_diag = max_diag > 0 ? ((int64_t)small.size() + max_diag - 1) / max_diag : 0;
    size_t next_small = 0;
    for (int64_t d = 0; d < max_diag; ++d) {
        fitems.insert(fitems.end(), tiles.begin() + dpos[(size_t)d], tiles.begin() + dpos[(size_t)d + 1]);
        for (int64_t q = 0; q < per_diag && next_small < small.size(); ++q, ++next_small) {
            const int32_t k = small[next_small];
            fitems.push_back({k, 0, (p->geom_h[k].n + 31) / 32, 0});
        }
    }
    for (; next_small < small.size(); ++next_small) {
        const int32_t k = small[next_small];
        fitems.push_back({k, 0, (p->geom_h[k].n + 31) / 32, 0});
    }
    p->n_fill_items = (int64_t)fitems.size();
}

// Items of the per-block count kernel (used when the strip kernel cannot
// be): 32 x 32 blocks, large pairs first.
static void build_count_items(const mine_plan *p, std::vector<CountItem> &citems) {
    citems.clear();
    for (int32_t k : p->pair_order_h) {
        const int ns = (p->geom_h[k].n + 31) / 32, nb = (p->geom_h[k].m + 31) / 32;
        if ((int64_t)ns * nb == 0) continue;
        for (int s = 0; s < ns; ++s)
            for (int b = 0; b < nb; ++b) citems.push_back({k, (s << 16) | b});
    }
}

// What a knob change requires of an existing plan.
constexpr int kKnobPlain = 0;   // nothing (read at the next call)
constexpr int kKnobGraph = 1;   // the captured graph holds the value: drop it
constexpr int kKnobTiling = 2;  // the fill work lists and tile flags depend on it: rebuild

// Applies one option to a knob set (MINE_EINVAL for an unknown or read-only
// option or a value out of range; the knobs are then unchanged).
static int knob_apply(PlanKnobs &k, int option, int64_t value, int *effect) {
    *effect = kKnobPlain;
    switch (option) {
        case MINE_OPT_TILE_COLS:
            if (value < 32 || value % 32 || value > (1 << 20)) return MINE_EINVAL;
            k.tile_cols = (int)value;
            *effect = kKnobTiling;
            return MINE_OK;
        case MINE_OPT_TILE_MIN_CELLS:
            if (value < 1) return MINE_EINVAL;
            k.tile_min_cells = value;
            *effect = kKnobTiling;
            return MINE_OK;
        case MINE_OPT_TILE_MIN_ROWS:
            if (value < 1) return MINE_EINVAL;
            k.tile_min_rows = (int)std::min<int64_t>(value, 1 << 30);
            *effect = kKnobTiling;
            return MINE_OK;
        case MINE_OPT_WAIT_LIMIT:
            if (value < 1) return MINE_EINVAL;
            k.wait_limit = value;
            *effect = kKnobGraph;
            return MINE_OK;
        case MINE_OPT_LINK_RECOUNT:
            k.link_recount = value != 0;
            *effect = kKnobGraph;
            return MINE_OK;
        case MINE_OPT_USE_GRAPH:
            k.use_graph = value != 0;
            return MINE_OK;
        case MINE_OPT_FAULT_SKIP_FLAG:
            k.skip_flag = value < 0 ? -1 : value;
            *effect = kKnobGraph;
            return MINE_OK;
        case MINE_OPT_SOFT_SPLIT:
            if (value < 0 || value > 3) return MINE_EINVAL;
            k.soft_split = (int)value;
            return MINE_OK;
        case MINE_OPT_FAULT_SKIP_SOFT:
            k.skip_soft = value < 0 ? -1 : value;
            return MINE_OK;
        case MINE_OPT_SOFT_SPLIT_Q4:
            if (value < 1 || value > 4096) return MINE_EINVAL;
            k.soft_split_q4 = (int)value;
            return MINE_OK;
        case MINE_OPT_SOFT_ORDER:
            if (value < 0 || value > 2) return MINE_EINVAL;
            k.soft_order = (int)value;
            return MINE_OK;
        default:
            return MINE_EINVAL;
    }
}

extern "C" {

int mine_plan_create(const mine_corpus *src, const mine_corpus *tgt, const mine_dict *dict,
                     mine_plan **out, miner_stream_t stream) {
    return mine_plan_create_with_options(src, tgt, dict, nullptr, nullptr, 0, out, stream);
}

}  // extern "C"

// Plan creation.  host_sd / host_td (may be null): host copies of the
// document offsets, which spare the read-back of the device ones (and its
// wait for everything queued before it on the stream); inputs_ready (may be
// null): an event after which the token and dictionary arrays are in place,
// waited for before the first kernel reads them.
static int plan_create(const mine_corpus *src, const mine_corpus *tgt, const mine_dict *dict, const int32_t *options,
                       const int64_t *values, int n_options, mine_plan **out, miner_stream_t stream,
                       const int64_t *host_sd, const int64_t *host_td, cudaEvent_t inputs_ready) {
    if (!src || !tgt || !dict || !out) return MINE_EINVAL;
    *out = nullptr;
    if (n_options < 0 || (n_options > 0 && (!options || !values))) return MINE_EINVAL;
    PlanKnobs knobs;
    for (int x = 0; x < n_options; ++x) {
        int effect;
        if (knob_apply(knobs, options[x], values[x], &effect) != MINE_OK) return MINE_EINVAL;
    }
    if (src->n_docs != tgt->n_docs || src->n_docs < 0 || src->n_sents < 0 || tgt->n_sents < 0 ||
        src->n_tok < 0 || tgt->n_tok < 0 || dict->v_src <= 0 || dict->v_tgt <= 0 || dict->n_entries < 0)
        return MINE_EINVAL;
    if (!src->doc_sent_off || !src->sent_tok_off || !tgt->doc_sent_off || !tgt->sent_tok_off || !dict->off ||
        (src->n_tok > 0 && !src->tok) || (tgt->n_tok > 0 && !tgt->tok) || (dict->n_entries > 0 && !dict->tgt))
        return MINE_EINVAL;
    if (src->n_docs > INT32_MAX) return MINE_ENOTSUP;
    cudaStream_t st = (cudaStream_t)stream;
    mine_plan *p = new (std::nothrow) mine_plan();
    if (!p) return MINE_ENOMEM;
    p->knobs = knobs;
    DoneMark mark{nullptr, st};  // armed once the plan exists
    auto fail = [&](int code) {
        mark.p = nullptr;
        plan_free(p);
        return code;
    };
    cudaError_t e;
#define PLAN_CK(x)                                                                  \
    do {                                                                            \
        e = (x);                                                                    \
        if (e != cudaSuccess) {                                                     \
            g_last_cuda = (int)e;                                                   \
            return fail(e == cudaErrorMemoryAllocation ? MINE_ENOMEM : MINE_ECUDA); \
        }                                                                           \
    } while (0)
    PLAN_CK(cudaGetDevice(&p->device));
    PLAN_CK(cudaStreamCreateWithFlags(&p->own_stream, cudaStreamNonBlocking));
    PLAN_CK(cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming));
    mark.p = p;
    PLAN_CK(cudaDeviceGetAttribute(&p->n_sms, cudaDevAttrMultiProcessorCount, p->device));
    p->src = {src->doc_sent_off, src->sent_tok_off, src->tok, src->n_tok};
    p->tgt = {tgt->doc_sent_off, tgt->sent_tok_off, tgt->tok, tgt->n_tok};
    // token arrays starting on a 16-byte boundary can be staged by bulk copies
    p->bulk_ok = ((uintptr_t)src->tok % 16 == 0) && ((uintptr_t)tgt->tok % 16 == 0);
    p->dict = {dict->off, dict->tgt};
    const int64_t n = src->n_docs;
    p->n_pairs = n;

    // document sizes (the caller's host copies, or a synchronous read-back)
    std::vector<int64_t> sd(n + 1), td(n + 1);
    if (host_sd && host_td) {
        std::copy(host_sd, host_sd + n + 1, sd.begin());
        std::copy(host_td, host_td + n + 1, td.begin());
    } else {
        PLAN_CK(cudaMemcpyAsync(sd.data(), src->doc_sent_off, (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        PLAN_CK(cudaMemcpyAsync(td.data(), tgt->doc_sent_off, (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        PLAN_CK(cudaStreamSynchronize(st));
    }
    if (sd[0] != 0 || td[0] != 0 || sd[n] != src->n_sents || td[n] != tgt->n_sents) return fail(MINE_EINVAL);
    for (int64_t k = 0; k < n; ++k)
        if (sd[k + 1] < sd[k] || td[k + 1] < td[k] || sd[k + 1] - sd[k] > (1 << 21) || td[k + 1] - td[k] > (1 << 21))
            return fail(MINE_EINVAL);

    // validation kernels
    if (inputs_ready) PLAN_CK(cudaStreamWaitEvent(st, inputs_ready, 0));
    PLAN_CK(dalloc(&p->S.status, 4, p->device, st));
    PLAN_CK(dalloc(&p->stats, 4, p->device, st));
    PLAN_CK(cudaMemsetAsync(p->S.status, 0, 4 * sizeof(uint32_t), st));
    PLAN_CK(cudaMemsetAsync(p->stats, 0, 4 * sizeof(int32_t), st));
    if (src->n_sents > 0)
        PLAN_CK(launch_validate_corpus(p->src, src->n_sents, src->n_tok, dict->v_src, p->S.status, p->stats + 0, st));
    if (tgt->n_sents > 0)
        PLAN_CK(launch_validate_corpus(p->tgt, tgt->n_sents, tgt->n_tok, dict->v_tgt, p->S.status, p->stats + 1, st));
    {
        int r = validate_dict(dict, p->S.status, p->stats + 3, st);
        if (r != MINE_OK) return fail(r);
    }

    std::vector<FillItem> fitems;
    int64_t tbw = 0, hrow = 0, vcol = 0;
    build_geometry(p, sd, td, fitems, tbw, hrow, vcol);
    PLAN_CK(dalloc(&p->geom, n, p->device, st));
    PLAN_CK(dalloc(&p->pair_order, n, p->device, st));
    PLAN_CK(dalloc(&p->fill_items, fitems.size(), p->device, st));
    {
        const StagePiece pcs[3] = {{p->geom_h.data(), p->geom, n * sizeof(PairGeom)},
                                   {p->pair_order_h.data(), p->pair_order, n * sizeof(int32_t)},
                                   {fitems.data(), p->fill_items, fitems.size() * sizeof(FillItem)}};
        PLAN_CK(staged_upload(p->device, pcs, 3, st));
    }

    // scratch
    p->v_src = dict->v_src;
    PLAN_CK(dalloc(&p->S.tb, tbw, p->device, st));
    PLAN_CK(dalloc(&p->S.hrow, hrow, p->device, st));
    PLAN_CK(dalloc(&p->S.vcol, vcol, p->device, st));
    PLAN_CK(dalloc(&p->S.flags, p->n_flags, p->device, st));
    PLAN_CK(dalloc(&p->S.queue, 1, p->device, st));
    PLAN_CK(dalloc(&p->S.diag_i, p->link_cap, p->device, st));
    PLAN_CK(dalloc(&p->S.diag_j, p->link_cap, p->device, st));
    PLAN_CK(dalloc(&p->S.diag_s, p->link_cap, p->device, st));
    PLAN_CK(dalloc(&p->S.n_diag, n, p->device, st));
    PLAN_CK(dalloc(&p->S.diag_off, n + 1, p->device, st));
    PLAN_CK(dalloc(&p->S.n_links, n, p->device, st));
    PLAN_CK(launch_block_tokens(p->tgt, p->geom, n, p->stats + 2, st));
    // the strip count kernels' items (used if the validation's statistics
    // allow it), built on the device while the validation kernels run, in
    // scratch the walk overwrites later
    int64_t n_strips = 0;
    for (int64_t k = 0; k < n; ++k)
        if (p->geom_h[k].m > 0) n_strips += (p->geom_h[k].n + 31) / 32;
    PLAN_CK(dalloc(&p->strip_items, n_strips, p->device, st));
    PLAN_CK(launch_strip_items(p->geom, p->pair_order, n, p->S.n_diag, p->S.diag_off, p->strip_items, st));

    uint32_t status[4];
    int32_t stats[4];
    PLAN_CK(cudaMemcpyAsync(status, p->S.status, sizeof status, cudaMemcpyDeviceToHost, st));
    PLAN_CK(cudaMemcpyAsync(stats, p->stats, sizeof stats, cudaMemcpyDeviceToHost, st));
    PLAN_CK(cudaStreamSynchronize(st));
    if (status[0] != 0) return fail(MINE_EINVAL);

    // strip count kernel: one item per 32-row strip, largest pairs first (the
    // kernel itself halves a strip's row group when its translations would
    // overfill the row table); it needs sentences of at most 31 tokens (5
    // counter planes) and a dictionary fan-out small enough for one row to fit
    p->use_strips = std::max(stats[0], stats[1]) <= 31 && stats[3] <= kStripMaxFanout;
    p->use_tiles = p->use_strips && stats[3] <= kTileMaxFanout;
    p->counts_bytes = p->use_tiles ? 64 * tbw : 2 * p->n_cells;
    PLAN_CK(dalloc(&p->counts, p->counts_bytes, p->device, st));
    if (p->use_tiles) {
        PLAN_CK(dalloc(&p->dict4, (size_t)p->v_src, p->device, st));
        PLAN_CK(dalloc(&p->count_queue, 1, p->device, st));
    }
    if (p->use_strips) {
        p->n_strip_items = n_strips;
    } else {
        std::vector<CountItem> citems;
        build_count_items(p, citems);
        p->n_count_items = (int64_t)citems.size();
        PLAN_CK(dalloc(&p->count_items, citems.size(), p->device, st));
        PLAN_CK(cudaMemcpyAsync(p->count_items, citems.data(), citems.size() * sizeof(CountItem),
                                cudaMemcpyHostToDevice, st));
        PLAN_CK(cudaStreamSynchronize(st));
    }
    const int maxlen = std::max(stats[0], stats[1]);
    p->planes = maxlen <= 31 ? 5 : 8;
    const int btok = std::max(stats[2], 1);
    int ls = 10;
    while ((1 << ls) < btok + btok / 2 && ls < 13) ++ls;
    p->log_slots = ls;
    *out = p;
#undef PLAN_CK
    return MINE_OK;
}

extern "C" {

int mine_plan_create_with_options(const mine_corpus *src, const mine_corpus *tgt, const mine_dict *dict,
                                  const int32_t *options, const int64_t *values, int n_options,
                                  mine_plan **out, miner_stream_t stream) {
    return plan_create(src, tgt, dict, options, values, n_options, out, stream, nullptr, nullptr, nullptr);
}

void mine_plan_destroy(mine_plan *plan) { plan_free(plan); }

int64_t mine_plan_n_pairs(const mine_plan *p) { return p ? p->n_pairs : 0; }
int64_t mine_plan_n_cells(const mine_plan *p) { return p ? p->n_cells : 0; }
int64_t mine_plan_link_capacity(const mine_plan *p) { return p ? p->link_cap : 0; }

int mine_plan_cell_offsets(const mine_plan *p, int64_t *host_out) {
    if (!p || !host_out) return MINE_EINVAL;
    std::memcpy(host_out, p->cell_off_h.data(), p->cell_off_h.size() * sizeof(int64_t));
    return MINE_OK;
}

}  // extern "C"

// Counts of every cell into `counts`: row-major (the layout of mine_count) or,
// with the tile kernel, blocked (mine_pairs' own buffer).
static int count_into(mine_plan *p, uint8_t *counts, bool blocked, cudaStream_t st) {
    if (p->n_cells == 0) return MINE_OK;
    if (p->use_tiles) {
        MINE_CK(timed(p, kKCount, st, [&] {
            cudaError_t e = launch_dict4(p->dict, p->v_src, p->dict4, st);
            if (e != cudaSuccess) return e;
            return launch_count_tiles(p->src, p->tgt, p->dict4, p->geom, p->strip_items, p->n_strip_items,
                                      p->count_queue, p->bulk_ok, blocked, counts, p->S.status, p->n_sms, st);
        }));
    } else if (p->use_strips) {
        MINE_CK(timed(p, kKCount, st, [&] {
            return launch_count_strips(p->src, p->tgt, p->dict, p->geom, p->strip_items, p->n_strip_items,
                                       kStripLogSlots, p->planes, p->bulk_ok, counts, p->S.status, p->n_sms, st);
        }));
    } else {
        MINE_CK(timed(p, kKCount, st, [&] {
            return launch_count(p->src, p->tgt, p->dict, p->geom, p->count_items, p->n_count_items, p->log_slots,
                                p->planes, counts, p->S.status, p->n_sms, st);
        }));
    }
    return MINE_OK;
}

extern "C" {

int mine_count(mine_plan *p, uint8_t *counts, miner_stream_t stream) {
    if (!p || (!counts && p->n_cells > 0)) return MINE_EINVAL;
    if (p->n_cells == 0) return MINE_OK;
    cudaStream_t st = (cudaStream_t)stream;
    DoneMark mark{p, st};
    return count_into(p, counts, false, st);
}

int mine_score(mine_plan *p, const mine_params *params, const uint8_t *counts, float *s, float *feat,
               miner_stream_t stream) {
    if (!p || !params || ((!counts || !s) && p->n_cells > 0)) return MINE_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    DoneMark mark{p, st};
    const DevParams P = to_dev(*params);
    MINE_CK(timed(p, kKScore, st,
                  [&] { return launch_score(p->src, p->tgt, p->geom, p->n_pairs, P, counts, s, feat, st); }));
    return MINE_OK;
}

}  // extern "C"

static int align_from(mine_plan *p, const mine_params *params, const uint8_t *counts, bool blocked, mine_out *out,
                      cudaStream_t st);

extern "C" int mine_align(mine_plan *p, const mine_params *params, const uint8_t *counts, mine_out *out,
                          miner_stream_t stream) {
    if (!p || !params || !out || !out->link_off || (!out->pair_score && p->n_pairs > 0)) return MINE_EINVAL;
    if (out->link_capacity < p->link_cap) return MINE_EINVAL;
    if (p->link_cap > 0 && (!out->link_i || !out->link_j || !out->link_s)) return MINE_EINVAL;
    if (p->n_cells > 0 && !counts) return MINE_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    DoneMark mark{p, st};
    return align_from(p, params, counts, false, out, st);
}

// Fill, walk, link scoring and compaction from counts in either layout.
static int align_from(mine_plan *p, const mine_params *params, const uint8_t *counts, bool blocked, mine_out *out,
                      cudaStream_t st) {
    const DevParams P = to_dev(*params);
    const AlignScratch &S = p->S;
    const int64_t n = p->n_pairs;
    if (p->n_flags > 0) MINE_CK(cudaMemsetAsync(S.flags, 0, p->n_flags * sizeof(int32_t), st));
    MINE_CK(timed(p, kKFill, st, [&] {
        return launch_fill(p->src, p->tgt, p->geom, p->fill_items, p->n_fill_items, P, counts,
                           blocked ? p->counts_bytes : 2 * p->n_cells, blocked, S, p->knobs.wait_limit,
                           p->knobs.skip_flag, p->n_sms, st);
    }));
    MINE_CK(timed(p, kKWalk, st, [&] { return launch_walk(p->geom, p->pair_order, n, S, p->n_sms, st); }));
    MINE_CK(timed(p, kKScan, st, [&] { return launch_scan(S.n_diag, n, S.diag_off, st); }));
    MINE_CK(timed(p, kKLinks, st, [&] {
        return launch_link_score(p->src, p->tgt, p->dict, p->geom, n, P, S, p->knobs.link_recount ? nullptr : counts,
                                 blocked, p->n_sms, st);
    }));
    MINE_CK(timed(p, kKLinks, st, [&] { return launch_pair_sum(p->geom, n, P, S, out->pair_score, p->n_sms, st); }));
    MINE_CK(timed(p, kKScan, st, [&] { return launch_scan(S.n_links, n, out->link_off, st); }));
    MINE_CK(timed(p, kKLinks, st, [&] {
        return launch_copy_links(p->geom, n, P, S, out->link_off, out->link_i, out->link_j, out->link_s, p->n_sms, st);
    }));
    return MINE_OK;
}

static int enqueue_pairs(mine_plan *p, const mine_params *params, mine_out *out, cudaStream_t st) {
    if (!out->link_off || (!out->pair_score && p->n_pairs > 0) || out->link_capacity < p->link_cap ||
        (p->link_cap > 0 && (!out->link_i || !out->link_j || !out->link_s)))
        return MINE_EINVAL;
    int r = count_into(p, p->counts, p->use_tiles, st);
    if (r != MINE_OK) return r;
    return align_from(p, params, p->counts, p->use_tiles, out, st);
}

extern "C" {

int mine_pairs(mine_plan *p, const mine_params *params, mine_out *out, miner_stream_t stream) {
    if (!p || !params || !out) return MINE_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    DoneMark mark{p, st};
    if (p->timing || !p->knobs.use_graph) return enqueue_pairs(p, params, out, st);
    // capture once on a plan-owned stream (the caller's stream may be the
    // legacy default stream, which cannot be captured), replay on the caller's
    const bool same = p->graph && std::memcmp(&p->graph_out, out, sizeof *out) == 0 &&
                      std::memcmp(&p->graph_params, params, sizeof *params) == 0;
    if (!same) {
        if (!p->cap_stream) MINE_CK(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
        MINE_CK(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
        const int r = enqueue_pairs(p, params, out, p->cap_stream);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(p->cap_stream, &g);
        if (r != MINE_OK || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            if (e != cudaSuccess) g_last_cuda = (int)e;
            return r != MINE_OK ? r : MINE_ECUDA;
        }
        if (p->graph) {
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(p->graph, g, &info) != cudaSuccess) {
                (void)cudaGetLastError();
                drop_graph(p);
            }
        }
        if (!p->graph) {
            const cudaError_t ei = cudaGraphInstantiate(&p->graph, g, 0);
            if (ei != cudaSuccess) {
                cudaGraphDestroy(g);
                p->graph = nullptr;
                g_last_cuda = (int)ei;
                return MINE_ECUDA;
            }
        }
        cudaGraphDestroy(g);
        p->graph_out = *out;
        p->graph_params = *params;
        ++p->graph_captures;
    }
    MINE_CK(cudaGraphLaunch(p->graph, st));
    return MINE_OK;
}

// ------------------------------------------------------------- soft alignment
static int64_t align_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

struct SoftLayout {
    int64_t partial, vpart, red, queue, items, prog1, prog2, E, ckv, ckt, qrow, qtrow, ckw, total;
    int64_t items_cap, slots_cap, ctr_cap;
};

static SoftLayout soft_layout(const mine_plan *p) {
    SoftLayout L;
    L.items_cap = p->n_pairs + 2 * p->soft_strips;
    L.slots_cap = p->soft_strips;
    L.ctr_cap = p->soft_strips;
    int64_t o = 0;
    L.partial = o;
    o = align_up(o + std::max<int64_t>(L.slots_cap, 1) * kSoftSlots * (int64_t)sizeof(double), 256);
    L.vpart = o;
    o = align_up(o + std::max<int64_t>(p->n_pairs, 1) * (int64_t)sizeof(double), 256);
    L.red = o;
    o = align_up(o + kSoftRedBlocks * 8 * (int64_t)sizeof(double), 256);
    L.queue = o;
    o = align_up(o + 16, 256);
    L.items = o;
    o = align_up(o + std::max<int64_t>(L.items_cap, 1) * (int64_t)sizeof(SoftItem), 256);
    L.prog1 = o;
    o = align_up(o + std::max<int64_t>(L.ctr_cap, 1) * 4, 256);
    L.prog2 = o;
    o = align_up(o + std::max<int64_t>(L.ctr_cap, 1) * 4, 256);
    L.E = o;  // per strip, step-major: twice the window checkpoints
    o = align_up(o + std::max<int64_t>(2 * p->soft_ckw, 1) * 4, 256);
    const int64_t rows = std::max<int64_t>(p->soft_rows, 1) * 4;
    L.ckv = o;
    o = align_up(o + rows, 256);
    L.ckt = o;
    o = align_up(o + rows, 256);
    L.qrow = o;
    o = align_up(o + rows, 256);
    L.qtrow = o;
    o = align_up(o + rows, 256);
    L.ckw = o;
    o = align_up(o + std::max<int64_t>(p->soft_ckw, 1) * 4, 256);
    L.total = o;
    return L;
}

static SoftScratch soft_scratch(const mine_plan *p, void *ws) {
    const SoftLayout L = soft_layout(p);
    char *b = static_cast<char *>(ws);
    SoftScratch W;
    W.partial = reinterpret_cast<double *>(b + L.partial);
    W.vpart = reinterpret_cast<double *>(b + L.vpart);
    W.red = reinterpret_cast<double *>(b + L.red);
    W.queue = reinterpret_cast<int32_t *>(b + L.queue);
    W.items = reinterpret_cast<SoftItem *>(b + L.items);
    W.prog1 = reinterpret_cast<int32_t *>(b + L.prog1);
    W.prog2 = reinterpret_cast<int32_t *>(b + L.prog2);
    W.E = reinterpret_cast<float *>(b + L.E);
    W.ckv = reinterpret_cast<float *>(b + L.ckv);
    W.ckt = reinterpret_cast<float *>(b + L.ckt);
    W.qrow = reinterpret_cast<float *>(b + L.qrow);
    W.qtrow = reinterpret_cast<float *>(b + L.qtrow);
    W.ckw = reinterpret_cast<float *>(b + L.ckw);
    W.items_cap = L.items_cap;
    W.slots_cap = L.slots_cap;
    W.ctr_cap = L.ctr_cap;
    return W;
}

static bool soft_args(const mine_plan *p, const softnw_opts *o, SoftArgs &A, const int32_t *&order, int64_t &n) {
    if (!o || !(o->gamma > 0.0f) || !(o->tau > 0.0f) || !(o->eps > 0.0f) || !(o->eps < 0.5f)) return false;
    A.gamma = o->gamma;
    A.tau = o->tau;
    A.eps = o->eps;
    A.wait_limit = p->knobs.wait_limit;
    A.status = p->S.status;
    A.split = p->knobs.soft_split;
    A.split_q4 = p->knobs.soft_split_q4;
    A.order = p->knobs.soft_order;
    A.skip_ctr = p->knobs.skip_soft;
    A.hvp = nullptr;
    int64_t cells = p->n_cells;
    order = p->pair_order;
    n = p->n_pairs;
    if (o->pairs) {
        if (o->n_pairs < 0 || o->n_pairs > p->n_pairs || o->n_cells < 0 || o->n_cells > p->n_cells) return false;
        order = o->pairs;
        n = o->n_pairs;
        cells = o->n_cells;
    }
    A.inv_cells = cells > 0 ? (float)(1.0 / (double)cells) : 0.0f;
    return true;
}

int64_t softnw_workspace_size(const mine_plan *p) { return p ? soft_layout(p).total : MINE_EINVAL; }

int softnw_fwd(mine_plan *p, const mine_params *params, const softnw_opts *opts, const uint8_t *counts,
               const uint8_t *gold, void *ws, float *loss, float *value, float *expected, miner_stream_t stream) {
    SoftArgs A;
    const int32_t *order = nullptr;
    int64_t n = 0;
    if (!p || !params || !ws || !loss || !soft_args(p, opts, A, order, n)) return MINE_EINVAL;
    if (p->n_cells > 0 && (!counts || !gold)) return MINE_EINVAL;
    if (p->max_m > (1 << 20)) return MINE_ENOTSUP;
    cudaStream_t st = (cudaStream_t)stream;
    DoneMark mark{p, st};
    const SoftScratch W = soft_scratch(p, ws);
    const DevParams P = to_dev(*params);
    MINE_CK(timed(p, kKSoftFwd, st, [&] {
        return launch_soft_forward(p->src, p->tgt, p->geom, order, n, P, A, counts, gold, W, loss, value, p->n_sms,
                                   st);
    }));
    if (expected && p->n_cells > 0) MINE_CK(launch_soft_export_e(p->geom, p->n_pairs, W.E, expected, st));
    return MINE_OK;
}

int softnw_bwd(mine_plan *p, const mine_params *params, const softnw_opts *opts, const uint8_t *counts,
               const uint8_t *gold, void *ws, float dloss, float *grad, float *hvp, miner_stream_t stream) {
    SoftArgs A;
    const int32_t *order = nullptr;
    int64_t n = 0;
    if (!p || !params || !ws || !grad || !soft_args(p, opts, A, order, n)) return MINE_EINVAL;
    if (p->n_cells > 0 && (!counts || !gold)) return MINE_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    DoneMark mark{p, st};
    const SoftScratch W = soft_scratch(p, ws);
    const DevParams P = to_dev(*params);
    MINE_CK(timed(p, kKSoftBwd, st, [&] {
        return launch_soft_backward(p->src, p->tgt, p->geom, order, n, P, A, counts, gold, W, dloss, grad, hvp,
                                    p->n_sms, st);
    }));
    return MINE_OK;
}

int mine_link_gold_counts(mine_plan *p, const mine_out *out, const uint8_t *gold, uint64_t *counts3,
                          miner_stream_t stream) {
    if (!p || !out || !out->link_off || !counts3 || (p->n_cells > 0 && !gold)) return MINE_EINVAL;
    DoneMark mark{p, (cudaStream_t)stream};
    MINE_CK(launch_link_gold(p->geom, p->n_pairs, out->link_off, out->link_i, out->link_j, gold,
                             reinterpret_cast<unsigned long long *>(counts3), p->n_sms, (cudaStream_t)stream));
    return MINE_OK;
}

int mine_plan_check(mine_plan *p, miner_stream_t stream) {
    if (!p) return MINE_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    DoneMark mark{p, st};
    uint32_t status = 0;
    MINE_CK(cudaMemcpyAsync(&status, p->S.status, sizeof status, cudaMemcpyDeviceToHost, st));
    MINE_CK(cudaStreamSynchronize(st));
    MINE_CK(cudaMemsetAsync(p->S.status, 0, sizeof status, st));
    if (status & kStTimeout) return MINE_ETIMEOUT;
    if (status) return MINE_EINVAL;
    return MINE_OK;
}

int mine_plan_set_option(mine_plan *p, int option, int64_t value) {
    if (!p) return MINE_EINVAL;
    PlanKnobs k = p->knobs;
    int effect = 0;
    const int rc = knob_apply(k, option, value, &effect);
    if (rc != MINE_OK) return rc;
    const bool same_tiling = k.tile_cols == p->knobs.tile_cols && k.tile_min_cells == p->knobs.tile_min_cells &&
                             k.tile_min_rows == p->knobs.tile_min_rows;
    if (effect == kKnobTiling && same_tiling) return MINE_OK;
    if (effect != kKnobTiling) {
        if (effect == kKnobGraph) drop_graph(p);
        p->knobs = k;
        return MINE_OK;
    }
    drop_graph(p);
    // tiling changed: rebuild the work lists and the tile flags (synchronous)
    std::vector<int64_t> sd(p->n_pairs + 1, 0), td(p->n_pairs + 1, 0);
    for (int64_t x = 0; x < p->n_pairs; ++x) {
        sd[x + 1] = sd[x] + p->geom_h[x].n;
        td[x + 1] = td[x] + p->geom_h[x].m;
    }
    p->knobs = k;
    std::vector<FillItem> fitems;
    int64_t tbw, hrow, vcol;
    build_geometry(p, sd, td, fitems, tbw, hrow, vcol);
    // the old work lists and flags are released, and the geometry rewritten,
    // after the plan's last enqueued work (its completion event), on the
    // plan-owned stream; other work on the device is not waited for
    cudaStream_t st = p->own_stream;
    MINE_CK(cudaStreamWaitEvent(st, p->done, 0));
    MINE_CK(cudaFreeAsync(p->fill_items, st));
    MINE_CK(cudaFreeAsync(p->S.flags, st));
    p->fill_items = nullptr;
    p->S.flags = nullptr;
    MINE_CK(dalloc(&p->fill_items, fitems.size(), p->device, st));
    MINE_CK(dalloc(&p->S.flags, p->n_flags, p->device, st));
    MINE_CK(cudaMemcpyAsync(p->fill_items, fitems.data(), fitems.size() * sizeof(FillItem), cudaMemcpyHostToDevice,
                            st));
    MINE_CK(cudaMemcpyAsync(p->geom, p->geom_h.data(), p->n_pairs * sizeof(PairGeom), cudaMemcpyHostToDevice, st));
    MINE_CK(cudaStreamSynchronize(st));
    return MINE_OK;
}

int64_t mine_plan_get_option(const mine_plan *p, int option) {
    if (!p) return MINE_EINVAL;
    switch (option) {
        case MINE_OPT_TILE_COLS: return p->knobs.tile_cols;
        case MINE_OPT_TILE_MIN_CELLS: return p->knobs.tile_min_cells;
        case MINE_OPT_TILE_MIN_ROWS: return p->knobs.tile_min_rows;
        case MINE_OPT_WAIT_LIMIT: return p->knobs.wait_limit;
        case MINE_OPT_LINK_RECOUNT: return p->knobs.link_recount;
        case MINE_OPT_USE_GRAPH: return p->knobs.use_graph;
        case MINE_OPT_GRAPH_CAPTURES: return p->graph_captures;
        case MINE_OPT_FAULT_SKIP_FLAG: return p->knobs.skip_flag;
        case MINE_OPT_N_TILE_FLAGS: return p->n_flags;
        case MINE_OPT_SOFT_SPLIT: return p->knobs.soft_split;
        case MINE_OPT_FAULT_SKIP_SOFT: return p->knobs.skip_soft;
        case MINE_OPT_SOFT_SPLIT_Q4: return p->knobs.soft_split_q4;
        case MINE_OPT_SOFT_ORDER: return p->knobs.soft_order;
        default: return MINE_EINVAL;
    }
}

int mine_plan_set_timing(mine_plan *p, int enable) {
    if (!p) return MINE_EINVAL;
    drain_pending(p);
    p->timing = enable != 0;
    for (int k = 0; k < kKinds; ++k) {
        p->total_ms[k] = 0.0;
        p->launches[k] = 0;
    }
    return MINE_OK;
}

int mine_plan_kernel_times(mine_plan *p, float *host_ms, int64_t *host_launches, int n) {
    if (!p) return MINE_EINVAL;
    drain_pending(p);
    for (int k = 0; k < kKinds && k < n; ++k) {
        if (host_ms) host_ms[k] = (float)p->total_ms[k];
        if (host_launches) host_launches[k] = p->launches[k];
    }
    return kKinds;
}

const char *mine_strerror(int code) {
    switch (code) {
        case MINE_OK: return "ok";
        case MINE_EINVAL: return "invalid argument or malformed input";
        case MINE_ENOMEM: return "out of memory";
        case MINE_ECUDA: return "CUDA error";
        case MINE_ETIMEOUT: return "device-side wait timed out";
        case MINE_ENOTSUP: return "not supported";
        default: return "unknown error";
    }
}

int mine_last_cuda_error(void) { return g_last_cuda; }

}  // extern "C"

// A temporary from the library's pool, returned to it (stream-ordered) when
// the scope ends, on every path out of an entry point.
template <typename T>
struct PoolTemp {
    T *p = nullptr;
    cudaStream_t st;
    explicit PoolTemp(cudaStream_t s) : st(s) {}
    ~PoolTemp() {
        if (p) cudaFreeAsync(p, st);
    }
};

extern "C" {

int mine_dict_transpose(const mine_dict *d, int32_t *off_out, int32_t *tgt_out, miner_stream_t stream) {
    if (!d || !off_out || !d->off || d->v_src <= 0 || d->v_tgt <= 0 || d->n_entries < 0 ||
        d->n_entries > INT32_MAX || (d->n_entries > 0 && (!d->tgt || !tgt_out)))
        return MINE_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int device;
    MINE_CK(cudaGetDevice(&device));
    PoolTemp<uint32_t> status(st);
    PoolTemp<int32_t> cursor(st);
    MINE_CK(dalloc(&status.p, 1, device, st));
    MINE_CK(dalloc(&cursor.p, (size_t)d->v_tgt, device, st));
    MINE_CK(cudaMemsetAsync(status.p, 0, sizeof(uint32_t), st));
    MINE_CK(launch_dict_check(d->off, d->v_src, d->n_entries, d->tgt, d->v_tgt, status.p, st));
    uint32_t bad = 0;
    MINE_CK(cudaMemcpyAsync(&bad, status.p, sizeof bad, cudaMemcpyDeviceToHost, st));
    MINE_CK(cudaStreamSynchronize(st));
    if (bad) return MINE_EINVAL;
    // counts into off_out[0 .. v_tgt), scanned in place into offsets
    MINE_CK(cudaMemsetAsync(off_out, 0, ((size_t)d->v_tgt + 1) * sizeof(int32_t), st));
    MINE_CK(launch_dict_count(d->tgt, d->n_entries, off_out, st));
    MINE_CK(launch_scan32(off_out, d->v_tgt, off_out, st));
    MINE_CK(cudaMemcpyAsync(cursor.p, off_out, (size_t)d->v_tgt * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    MINE_CK(launch_dict_scatter(d->off, d->v_src, d->tgt, cursor.p, tgt_out, st));
    MINE_CK(launch_dict_sort(off_out, d->v_tgt, tgt_out, st));
    MINE_CK(cudaStreamSynchronize(st));
    return MINE_OK;
}

int mine_corpus_add_anchors(const mine_corpus *w, int32_t v_words, const int64_t *anchor_off,
                            const int32_t *anchor_ids, int64_t n_anchor_tok, int32_t v_anchor,
                            int64_t *sent_tok_off_out, int32_t *tok_out, miner_stream_t stream) {
    if (!w || !anchor_off || !sent_tok_off_out || !w->sent_tok_off || w->n_sents < 0 || w->n_tok < 0 ||
        n_anchor_tok < 0 || v_words <= 0 || v_anchor <= 0 || (int64_t)v_words + v_anchor > INT32_MAX ||
        (n_anchor_tok > 0 && !anchor_ids) || (w->n_tok > 0 && !w->tok) || (w->n_tok + n_anchor_tok > 0 && !tok_out))
        return MINE_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int device;
    MINE_CK(cudaGetDevice(&device));
    PoolTemp<uint32_t> status(st);
    MINE_CK(dalloc(&status.p, 1, device, st));
    MINE_CK(cudaMemsetAsync(status.p, 0, sizeof(uint32_t), st));
    MINE_CK(launch_anchor_check(w->sent_tok_off, w->n_tok, anchor_off, w->n_sents, anchor_ids, n_anchor_tok, v_anchor,
                                status.p, st));
    uint32_t bad = 0;
    MINE_CK(cudaMemcpyAsync(&bad, status.p, sizeof bad, cudaMemcpyDeviceToHost, st));
    MINE_CK(cudaStreamSynchronize(st));
    if (bad) return MINE_EINVAL;
    MINE_CK(launch_anchor_merge(w->sent_tok_off, w->tok, anchor_off, anchor_ids, w->n_sents, v_words,
                                sent_tok_off_out, tok_out, st));
    MINE_CK(cudaStreamSynchronize(st));
    return MINE_OK;
}

int mine_dict_add_anchors(const mine_dict *d, int32_t v_anchor, int32_t *off_out, int32_t *tgt_out,
                          miner_stream_t stream) {
    if (!d || !off_out || !tgt_out || !d->off || d->v_src <= 0 || d->v_tgt <= 0 || d->n_entries < 0 ||
        v_anchor <= 0 || (d->n_entries > 0 && !d->tgt) || (int64_t)d->v_src + v_anchor > INT32_MAX ||
        (int64_t)d->v_tgt + v_anchor > INT32_MAX || d->n_entries + v_anchor > INT32_MAX)
        return MINE_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int device;
    MINE_CK(cudaGetDevice(&device));
    // the offsets are copied and shifted as they are: check the dictionary
    // before anything is written
    PoolTemp<uint32_t> status(st);
    MINE_CK(dalloc(&status.p, 1, device, st));
    MINE_CK(cudaMemsetAsync(status.p, 0, sizeof(uint32_t), st));
    MINE_CK(launch_dict_check(d->off, d->v_src, d->n_entries, d->tgt, d->v_tgt, status.p, st));
    uint32_t bad = 0;
    MINE_CK(cudaMemcpyAsync(&bad, status.p, sizeof bad, cudaMemcpyDeviceToHost, st));
    MINE_CK(cudaStreamSynchronize(st));
    if (bad) return MINE_EINVAL;
    MINE_CK(launch_anchor_dict(d->off, d->tgt, d->v_src, d->v_tgt, d->n_entries, v_anchor, off_out, tgt_out, st));
    return MINE_OK;
}

int mine_links_combine(mine_plan *f, const mine_out *of, mine_plan *r, const mine_out *orv, int mode,
                       mine_bi_out *o, miner_stream_t stream) {
    if (!f || !r || !of || !orv || !o || (mode != MINE_BI_UNION && mode != MINE_BI_INTERSECT)) return MINE_EINVAL;
    if (f->n_pairs != r->n_pairs || !of->link_off || !orv->link_off || !o->link_off) return MINE_EINVAL;
    if (of->link_capacity < 0 || orv->link_capacity < 0) return MINE_EINVAL;
    for (int64_t k = 0; k < f->n_pairs; ++k)
        if (f->geom_h[k].n != r->geom_h[k].m || f->geom_h[k].m != r->geom_h[k].n) return MINE_EINVAL;
    const int64_t need = f->link_cap + r->link_cap;
    if (o->link_capacity < need) return MINE_EINVAL;
    if (f->link_cap > 0 && (!of->link_i || !of->link_j || !of->link_s)) return MINE_EINVAL;
    if (r->link_cap > 0 && (!orv->link_i || !orv->link_j || !orv->link_s)) return MINE_EINVAL;
    if (need > 0 && (!o->link_i || !o->link_j || !o->s_fwd || !o->s_rev)) return MINE_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = f->n_pairs;
    PoolTemp<int32_t> cnt(st);
    MINE_CK(dalloc(&cnt.p, (size_t)n, f->device, st));
    const LinkView F{of->link_off, of->link_i, of->link_j, of->link_s, of->link_capacity};
    const LinkView R{orv->link_off, orv->link_i, orv->link_j, orv->link_s, orv->link_capacity};
    MINE_CK(launch_links_combine(F, R, n, mode, cnt.p, 0, nullptr, nullptr, nullptr, nullptr, nullptr, st));
    MINE_CK(launch_scan(cnt.p, n, o->link_off, st));
    MINE_CK(launch_links_combine(F, R, n, mode, cnt.p, o->link_capacity, o->link_off, o->link_i, o->link_j, o->s_fwd,
                                 o->s_rev, st));
    return MINE_OK;
}

}  // extern "C"

// ------------------------------------------------- unconstrained alignment
namespace {

struct UcLayout {
    int64_t offs, order, n_match, kept, A, prev, li, lj, ls, total;
    int64_t a_total, prev_total, link_total;
};

UcLayout uc_layout(const mine_plan *p) {
    UcLayout L{};
    const int64_t n = p->n_pairs;
    for (const PairGeom &g : p->geom_h) {
        L.a_total += 2 * ((int64_t)g.m + 1);
        L.prev_total += (int64_t)g.n * ((int64_t)g.m + 1);
        L.link_total += g.n;
    }
    auto up = [](int64_t x) { return (x + 255) / 256 * 256; };
    int64_t o = 0;
    L.offs = o;
    o = up(o + 3 * std::max<int64_t>(n, 1) * 8);
    L.order = o;
    o = up(o + std::max<int64_t>(n, 1) * 4);
    L.n_match = o;
    o = up(o + std::max<int64_t>(n, 1) * 4);
    L.kept = o;
    o = up(o + std::max<int64_t>(n, 1) * 4);
    L.A = o;
    o = up(o + std::max<int64_t>(L.a_total, 1) * 8);
    L.prev = o;
    o = up(o + std::max<int64_t>(L.prev_total, 1) * 4);
    L.li = o;
    o = up(o + std::max<int64_t>(L.link_total, 1) * 4);
    L.lj = o;
    o = up(o + std::max<int64_t>(L.link_total, 1) * 4);
    L.ls = o;
    o = up(o + std::max<int64_t>(L.link_total, 1) * 4);
    L.total = o;
    return L;
}

}  // namespace

extern "C" {

int64_t mine_unconstrained_workspace_size(const mine_plan *p) { return p ? uc_layout(p).total : 0; }

int64_t mine_unconstrained_link_capacity(const mine_plan *p) { return p ? uc_layout(p).link_total : 0; }

int mine_align_unconstrained(mine_plan *p, const mine_params *params, const uint8_t *counts, void *ws, mine_out *out,
                             miner_stream_t stream) {
    if (!p || !params || !out || !ws || !out->link_off || (!out->pair_score && p->n_pairs > 0)) return MINE_EINVAL;
    const UcLayout L = uc_layout(p);
    if (out->link_capacity < L.link_total) return MINE_EINVAL;
    if (L.link_total > 0 && (!out->link_i || !out->link_j || !out->link_s)) return MINE_EINVAL;
    if (p->n_cells > 0 && !counts) return MINE_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    DoneMark mark{p, st};
    const int64_t n = p->n_pairs;
    if (p->uc_off_h.empty() && n > 0) {
        p->uc_off_h.resize(3 * (size_t)n);
        int64_t a = 0, pv = 0, lk = 0;
        for (int64_t k = 0; k < n; ++k) {
            const PairGeom &g = p->geom_h[k];
            p->uc_off_h[k] = a;
            p->uc_off_h[n + k] = pv;
            p->uc_off_h[2 * n + k] = lk;
            a += 2 * ((int64_t)g.m + 1);
            pv += (int64_t)g.n * ((int64_t)g.m + 1);
            lk += g.n;
        }
        // largest pairs first within each class
        p->uc_order_h.clear();
        p->uc_order_h.reserve((size_t)n);
        for (int32_t k : p->pair_order_h)
            if (p->geom_h[k].m + 1 <= kUcShortCols) p->uc_order_h.push_back(k);
        p->uc_n_short = (int64_t)p->uc_order_h.size();
        for (int32_t k : p->pair_order_h)
            if (p->geom_h[k].m + 1 > kUcShortCols) p->uc_order_h.push_back(k);
    }
    char *b = static_cast<char *>(ws);
    if (n > 0) {
        MINE_CK(cudaMemcpyAsync(b + L.offs, p->uc_off_h.data(), 3 * n * sizeof(int64_t), cudaMemcpyHostToDevice, st));
        MINE_CK(cudaMemcpyAsync(b + L.order, p->uc_order_h.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    }
    UcScratch W;
    W.a_off = reinterpret_cast<const int64_t *>(b + L.offs);
    W.prev_off = W.a_off + n;
    W.link_off = W.a_off + 2 * n;
    W.n_match = reinterpret_cast<int32_t *>(b + L.n_match);
    W.A = reinterpret_cast<int64_t *>(b + L.A);
    W.prev = reinterpret_cast<int32_t *>(b + L.prev);
    W.li = reinterpret_cast<int32_t *>(b + L.li);
    W.lj = reinterpret_cast<int32_t *>(b + L.lj);
    W.ls = reinterpret_cast<float *>(b + L.ls);
    int32_t *kept = reinterpret_cast<int32_t *>(b + L.kept);
    const DevParams P = to_dev(*params);
    MINE_CK(launch_unconstrained(p->src, p->tgt, p->geom, reinterpret_cast<const int32_t *>(b + L.order), p->uc_n_short,
                                 n, P, counts, W, out->pair_score, p->max_m, kept, p->n_sms, st));
    MINE_CK(launch_scan(kept, n, out->link_off, st));
    MINE_CK(launch_unconstrained_copy(p->geom, n, P.thr, W, out->link_off, out->link_i, out->link_j, out->link_s,
                                      p->n_sms, st));
    return MINE_OK;
}

}  // extern "C"

// ------------------------------------------------------- host-buffer mining
namespace gbm {
// Strip items of the count kernels, built on the device from the plan's
// geometry and size order: the number of 32-row strips of the pair at each
// position of the order (0 for a pair without targets) ...
__global__ void strip_counts_kernel(const PairGeom *__restrict__ geom, const int32_t *__restrict__ order, int64_t n,
                                    int32_t *__restrict__ cnt) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; pos < n; pos += stride) {
        const PairGeom g = geom[order[pos]];
        cnt[pos] = g.m > 0 ? (g.n + 31) / 32 : 0;
    }
}
// ... and, from their exclusive scan, every strip's item at its place (pairs
// largest first, strips in order, the whole 32-row group).
__global__ void strip_items_kernel(const PairGeom *__restrict__ geom, const int32_t *__restrict__ order, int64_t n,
                                   const int64_t *__restrict__ off, CountStripItem *__restrict__ items) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; pos < n; pos += stride) {
        const int32_t k = order[pos];
        const PairGeom g = geom[k];
        const int ns = g.m > 0 ? (g.n + 31) / 32 : 0;
        for (int sidx = 0; sidx < ns; ++sidx) items[off[pos] + sidx] = CountStripItem{k, sidx, 0, 32};
    }
}

cudaError_t launch_strip_items(const PairGeom *geom, const int32_t *order, int64_t n, int32_t *cnt, int64_t *off,
                               CountStripItem *items, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 4096);
    strip_counts_kernel<<<grid, 256, 0, st>>>(geom, order, n, cnt);
    cudaError_t e = launch_scan(cnt, n, off, st);
    if (e != cudaSuccess) return e;
    strip_items_kernel<<<grid, 256, 0, st>>>(geom, order, n, off, items);
    return cudaGetLastError();
}

// In place: x[i] -= base (a chunk's sentence offsets, rebased to its first token).
__global__ void rebase_offsets_kernel(int64_t *x, int64_t count, int64_t base) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) x[i] -= base;
}
}  // namespace gbm

namespace {

// One chunk of pairs [k0, k1) of mine_pairs_host: its device inputs (sentence
// offsets rebased to the chunk's first token, tokens in buffers of their own,
// so that every token array starts 16-byte aligned), its plan and outputs.
struct HostChunk {
    int64_t k0 = 0, k1 = 0, s0 = 0, s1 = 0, u0 = 0, u1 = 0;  // pairs, source sentences, target sentences
    std::vector<int64_t> sdoc_h, tdoc_h;                       // rebased document offsets (host)
    PoolTemp<int64_t> sdoc, ssent, tdoc, tsent, o_off;
    PoolTemp<int32_t> stok, ttok, o_i, o_j;
    PoolTemp<float> o_s, o_score;
    mine_plan *plan = nullptr;
    explicit HostChunk(cudaStream_t st)
        : sdoc(st), ssent(st), tdoc(st), tsent(st), o_off(st), stok(st), ttok(st), o_i(st), o_j(st), o_s(st),
          o_score(st) {}
    ~HostChunk() { mine_plan_destroy(plan); }
};

}  // namespace

extern "C" int mine_pairs_host(const mine_corpus *src, const mine_corpus *tgt, const mine_dict *dict,
                               const mine_params *params, const int32_t *options, const int64_t *values,
                               int n_options, int64_t *link_off, int32_t *link_i, int32_t *link_j, float *link_s,
                               float *pair_score, int64_t link_capacity, miner_stream_t stream) {
    if (!src || !tgt || !dict || !params || !link_off || (src->n_docs > 0 && !pair_score)) return MINE_EINVAL;
    if (src->n_docs != tgt->n_docs || src->n_docs < 0 || src->n_sents < 0 || tgt->n_sents < 0 || src->n_tok < 0 ||
        tgt->n_tok < 0 || dict->v_src <= 0 || dict->n_entries < 0 || link_capacity < 0)
        return MINE_EINVAL;
    if (!src->doc_sent_off || !src->sent_tok_off || !tgt->doc_sent_off || !tgt->sent_tok_off || !dict->off ||
        (src->n_tok > 0 && !src->tok) || (tgt->n_tok > 0 && !tgt->tok) || (dict->n_entries > 0 && !dict->tgt))
        return MINE_EINVAL;
    if (n_options < 0 || (n_options > 0 && (!options || !values))) return MINE_EINVAL;
    // a plan used once: no graph capture unless the caller's options ask for
    // it; MINE_OPT_HOST_CHUNKS is this call's own
    std::vector<int32_t> opt(1, MINE_OPT_USE_GRAPH);
    std::vector<int64_t> val(1, 0);
    int64_t want_chunks = 0;
    for (int x = 0; x < n_options; ++x) {
        if (options[x] == MINE_OPT_HOST_CHUNKS) {
            if (values[x] < 0) return MINE_EINVAL;
            want_chunks = values[x];
        } else {
            opt.push_back(options[x]);
            val.push_back(values[x]);
        }
    }
    const int64_t n = src->n_docs;
    const int64_t *sd = src->doc_sent_off, *td = tgt->doc_sent_off;  // host
    const int64_t *ss = src->sent_tok_off, *ts = tgt->sent_tok_off;  // host
    // the offsets that delimit the chunks (the plans check the rest)
    if (sd[0] != 0 || td[0] != 0 || sd[n] != src->n_sents || td[n] != tgt->n_sents) return MINE_EINVAL;
    int64_t cells = 0, need = 0;  // cells, and link capacity: the sum over pairs of min(N, M)
    for (int64_t k = 0; k < n; ++k) {
        if (sd[k + 1] < sd[k] || td[k + 1] < td[k]) return MINE_EINVAL;
        cells += (sd[k + 1] - sd[k]) * (td[k + 1] - td[k]);
        need += std::min(sd[k + 1] - sd[k], td[k + 1] - td[k]);
    }
    if (link_capacity < need || (need > 0 && (!link_i || !link_j || !link_s))) return MINE_EINVAL;
    if (ss[0] != 0 || ts[0] != 0 || ss[src->n_sents] != src->n_tok || ts[tgt->n_sents] != tgt->n_tok)
        return MINE_EINVAL;
    int64_t K = want_chunks > 0 ? want_chunks : 1;
    K = std::max<int64_t>(1, std::min<int64_t>(K, std::max<int64_t>(n, 1)));
    cudaStream_t st = (cudaStream_t)stream;
    int device;
    MINE_CK(cudaGetDevice(&device));

    // streams: copies (cs), plan creation of the next chunk (ps), mining (st);
    // every exit orders st after the copies and the plan work (the chunks'
    // buffers are freed on st)
    struct Streams {
        cudaStream_t main, cs = nullptr, ps = nullptr;
        cudaEvent_t ordered = nullptr, done_cs = nullptr, done_ps = nullptr;
        ~Streams() {
            for (cudaStream_t q : {cs, ps}) {
                if (!q) continue;
                cudaEvent_t ev = q == cs ? done_cs : done_ps;
                if (ev && cudaEventRecord(ev, q) == cudaSuccess)
                    (void)cudaStreamWaitEvent(main, ev, 0);
                else
                    (void)cudaStreamSynchronize(q);
            }
            for (cudaEvent_t ev : {ordered, done_cs, done_ps})
                if (ev) cudaEventDestroy(ev);
            if (cs) cudaStreamDestroy(cs);
            if (ps) cudaStreamDestroy(ps);
        }
    };
    // chunk bounds: about equal cells
    std::vector<int64_t> bounds(1, 0);
    {
        int64_t acc = 0, next = 1;
        for (int64_t k = 0; k < n && next < K; ++k) {
            acc += (sd[k + 1] - sd[k]) * (td[k + 1] - td[k]);
            if (acc * K >= next * cells && k + 1 < n) {
                bounds.push_back(k + 1);
                while (next < K && acc * K >= next * cells) ++next;
            }
        }
        bounds.push_back(n);
    }
    const int nc = (int)bounds.size() - 1;
    PoolTemp<int32_t> doff(st), dtgt(st);
    std::vector<std::unique_ptr<HostChunk>> ch;
    for (int c = 0; c < nc; ++c) {
        ch.emplace_back(new HostChunk(st));
        HostChunk &H = *ch.back();
        H.k0 = bounds[c];
        H.k1 = bounds[c + 1];
        H.s0 = sd[H.k0];
        H.s1 = sd[H.k1];
        H.u0 = td[H.k0];
        H.u1 = td[H.k1];
        const int64_t nk = H.k1 - H.k0;
        H.sdoc_h.resize(nk + 1);
        H.tdoc_h.resize(nk + 1);
        for (int64_t x = 0; x <= nk; ++x) {
            H.sdoc_h[x] = sd[H.k0 + x] - H.s0;
            H.tdoc_h[x] = td[H.k0 + x] - H.u0;
        }
        MINE_CK(dalloc(&H.sdoc.p, (size_t)nk + 1, device, st));
        MINE_CK(dalloc(&H.tdoc.p, (size_t)nk + 1, device, st));
        MINE_CK(dalloc(&H.ssent.p, (size_t)(H.s1 - H.s0) + 1, device, st));
        MINE_CK(dalloc(&H.tsent.p, (size_t)(H.u1 - H.u0) + 1, device, st));
        MINE_CK(dalloc(&H.stok.p, (size_t)std::max<int64_t>(ss[H.s1] - ss[H.s0], 1), device, st));
        MINE_CK(dalloc(&H.ttok.p, (size_t)std::max<int64_t>(ts[H.u1] - ts[H.u0], 1), device, st));
    }
    MINE_CK(dalloc(&doff.p, (size_t)dict->v_src + 1, device, st));
    MINE_CK(dalloc(&dtgt.p, (size_t)std::max<int64_t>(dict->n_entries, 1), device, st));
    Streams S{st};
    MINE_CK(cudaStreamCreateWithFlags(&S.cs, cudaStreamNonBlocking));
    MINE_CK(cudaStreamCreateWithFlags(&S.ps, cudaStreamNonBlocking));
    for (cudaEvent_t *ev : {&S.ordered, &S.done_cs, &S.done_ps})
        MINE_CK(cudaEventCreateWithFlags(ev, cudaEventDisableTiming));
    MINE_CK(cudaEventRecord(S.ordered, st));  // the allocations above
    MINE_CK(cudaStreamWaitEvent(S.cs, S.ordered, 0));
    std::vector<cudaEvent_t> ready(nc, nullptr);
    struct Events {
        std::vector<cudaEvent_t> &v;
        ~Events() {
            for (cudaEvent_t e : v)
                if (e) cudaEventDestroy(e);
        }
    } ev_guard{ready};
    // every upload is enqueued at once, chunk by chunk (the dictionary first)
    auto up = [&](void *d, const void *h, size_t bytes) {
        return bytes ? cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, S.cs) : cudaSuccess;
    };
    MINE_CK(up(doff.p, dict->off, ((size_t)dict->v_src + 1) * 4));
    MINE_CK(up(dtgt.p, dict->tgt, dict->n_entries * 4));
    for (int c = 0; c < nc; ++c) {
        HostChunk &H = *ch[c];
        const int64_t nk = H.k1 - H.k0;
        MINE_CK(up(H.sdoc.p, H.sdoc_h.data(), (nk + 1) * 8));
        MINE_CK(up(H.tdoc.p, H.tdoc_h.data(), (nk + 1) * 8));
        MINE_CK(up(H.ssent.p, ss + H.s0, (H.s1 - H.s0 + 1) * 8));
        MINE_CK(up(H.tsent.p, ts + H.u0, (H.u1 - H.u0 + 1) * 8));
        MINE_CK(up(H.stok.p, src->tok + ss[H.s0], (ss[H.s1] - ss[H.s0]) * 4));
        MINE_CK(up(H.ttok.p, tgt->tok + ts[H.u0], (ts[H.u1] - ts[H.u0]) * 4));
        if (ss[H.s0] != 0)
            gbm::rebase_offsets_kernel<<<64, 256, 0, S.cs>>>(H.ssent.p, H.s1 - H.s0 + 1, ss[H.s0]);
        if (ts[H.u0] != 0)
            gbm::rebase_offsets_kernel<<<64, 256, 0, S.cs>>>(H.tsent.p, H.u1 - H.u0 + 1, ts[H.u0]);
        MINE_CK(cudaGetLastError());
        MINE_CK(cudaEventCreateWithFlags(&ready[c], cudaEventDisableTiming));
        MINE_CK(cudaEventRecord(ready[c], S.cs));
    }
    const mine_dict dd{dict->v_src, dict->v_tgt, dict->n_entries, doff.p, dtgt.p};
    auto make_plan = [&](int c) -> int {
        HostChunk &H = *ch[c];
        const int64_t nk = H.k1 - H.k0;
        const mine_corpus ds{nk, H.s1 - H.s0, ss[H.s1] - ss[H.s0], H.sdoc.p, H.ssent.p, H.stok.p};
        const mine_corpus dt{nk, H.u1 - H.u0, ts[H.u1] - ts[H.u0], H.tdoc.p, H.tsent.p, H.ttok.p};
        int r = plan_create(&ds, &dt, &dd, opt.data(), val.data(), (int)opt.size(), &H.plan, (miner_stream_t)S.ps,
                            H.sdoc_h.data(), H.tdoc_h.data(), ready[c]);
        if (r != MINE_OK) return r;
        const int64_t cap = std::max<int64_t>(H.plan->link_cap, 1);
        MINE_CK(dalloc(&H.o_off.p, (size_t)nk + 1, device, S.ps));
        MINE_CK(dalloc(&H.o_i.p, (size_t)cap, device, S.ps));
        MINE_CK(dalloc(&H.o_j.p, (size_t)cap, device, S.ps));
        MINE_CK(dalloc(&H.o_s.p, (size_t)cap, device, S.ps));
        MINE_CK(dalloc(&H.o_score.p, (size_t)std::max<int64_t>(nk, 1), device, S.ps));
        MINE_CK(cudaStreamSynchronize(S.ps));  // the plan and its outputs exist before st uses them
        return MINE_OK;
    };
    std::vector<cudaEvent_t> mined(nc, nullptr);
    Events mined_guard{mined};
    auto mine = [&](int c) -> int {
        HostChunk &H = *ch[c];
        mine_out out{H.o_off.p, H.o_i.p, H.o_j.p, H.o_s.p, H.o_score.p, std::max<int64_t>(H.plan->link_cap, 1)};
        int r = mine_pairs(H.plan, params, &out, stream);
        if (r != MINE_OK) return r;
        MINE_CK(cudaEventCreateWithFlags(&mined[c], cudaEventDisableTiming));
        MINE_CK(cudaEventRecord(mined[c], st));
        return MINE_OK;
    };
    int r = make_plan(0);
    if (r == MINE_OK) r = mine(0);
    if (r != MINE_OK) return r;
    int64_t base = 0;
    for (int c = 0; c < nc; ++c) {
        // the next chunk's plan is built (its validation waits for its upload)
        // and its mining queued behind this chunk's
        if (c + 1 < nc) {
            r = make_plan(c + 1);
            if (r == MINE_OK) r = mine(c + 1);
            if (r != MINE_OK) return r;
        }
        // this chunk's results, its links after those of the chunks before it
        HostChunk &H = *ch[c];
        const int64_t nk = H.k1 - H.k0;
        int64_t total = 0;
        MINE_CK(cudaStreamWaitEvent(S.ps, mined[c], 0));
        if (nk > 0) {
            MINE_CK(cudaMemcpyAsync(link_off + H.k0, H.o_off.p, nk * 8, cudaMemcpyDeviceToHost, S.ps));
            MINE_CK(cudaMemcpyAsync(pair_score + H.k0, H.o_score.p, nk * 4, cudaMemcpyDeviceToHost, S.ps));
        }
        MINE_CK(cudaMemcpyAsync(&total, H.o_off.p + nk, 8, cudaMemcpyDeviceToHost, S.ps));
        r = mine_plan_check(H.plan, (miner_stream_t)S.ps);  // synchronises ps
        if (r != MINE_OK) return r;
        if (total < 0 || total > link_capacity - base) return MINE_EINVAL;
        if (total > 0) {
            MINE_CK(cudaMemcpyAsync(link_i + base, H.o_i.p, total * 4, cudaMemcpyDeviceToHost, S.ps));
            MINE_CK(cudaMemcpyAsync(link_j + base, H.o_j.p, total * 4, cudaMemcpyDeviceToHost, S.ps));
            MINE_CK(cudaMemcpyAsync(link_s + base, H.o_s.p, total * 4, cudaMemcpyDeviceToHost, S.ps));
        }
        for (int64_t x = 0; x < nk; ++x) link_off[H.k0 + x] += base;
        base += total;
    }
    link_off[n] = base;
    MINE_CK(cudaStreamSynchronize(S.ps));
    return MINE_OK;
}
