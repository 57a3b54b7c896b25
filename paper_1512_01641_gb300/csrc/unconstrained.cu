// Unconstrained sentence alignment: the A* aligner Yalign used, which Section
// 5.1 contrasts with Needleman-Wunsch (Figures 3 and 5 against 4 and 6).
//
// Source sentences (rows) are taken in order.  After row i-1 the target
// pointer is c (the last matched target sentence, 1-based; 0 before any
// match).  Row i is
//   unmatched:                    A(i, c)  = A(i-1, c) - p
//   matched ahead (c' > c):       A(i, c') = A(i-1, c) + s(i, c') - p (c' - c - 1)
//   matched back (c' <= c):       A(i, c') = A(i-1, c) + s(i, c') - p
// and the target sentences after the final pointer cost p each.  Without
// the move back these are exactly the Needleman-Wunsch alignments; the move
// back is what lets a target sentence be used twice (the paper's
// repetitions).  Per row, the best forward predecessor of c' is a prefix
// maximum of A(i-1, c) + p c over c < c', the best move back a suffix maximum
// of A(i-1, c) over c >= c': one warp per pair sweeps each row twice with
// warp scans.  Exact ties prefer unmatched, then a forward match, then a move
// back; among predecessors the nearest pointer; at the end the smallest final
// pointer.  Scores are exact: 64-bit integers in units of 2^-k, with k chosen
// per pair so that no value of the pair can overflow (similarities and p are
// rounded to that grid once; every sum, difference and comparison after that
// is exact).
#include <algorithm>
#include <cmath>

#include "kernels.h"

namespace gbm {
namespace {

constexpr int kUcWarps = 4;
constexpr int kUcShortWarps = 8;

using Fx = int64_t;                      // a score in units of 2^-k
constexpr Fx kNegFx = -(int64_t(1) << 62);  // below every reachable score (those stay within 2^61)

struct MaxArg {
    Fx v;
    int a;
};

// The grid of one pair: every score and every candidate is bounded by
// (N + M + 2)(1 + |p|) in magnitude, so 2^k times that bound stays below
// 2^61 (and kNegFx minus it above -2^63); k is at most 40 (similarities at
// or above 2^-16 are then exact).
struct FxGrid {
    float up, down;  // 2^k, 2^-k
};
__device__ __forceinline__ FxGrid fx_grid(int N, int M, float gap) {
    const float bound = __fmul_rn((float)(N + M + 2), __fadd_rn(1.0f, fabsf(gap)));  // >= 2, finite
    const int e = (int)((__float_as_uint(bound) >> 23) & 0xFFu) - 126;               // bound < 2^e
    const int k = max(-60, min(40, 61 - e));
    return {__uint_as_float((uint32_t)(127 + k) << 23), __uint_as_float((uint32_t)(127 - k) << 23)};
}
__device__ __forceinline__ Fx to_fx(float x, const FxGrid &G) { return __float2ll_rn(__fmul_rn(x, G.up)); }
__device__ __forceinline__ float from_fx(Fx v, const FxGrid &G) { return __fmul_rn(__ll2float_rn(v), G.down); }

// Inclusive warp scan of (value, index) maxima in lane order: ties keep the
// larger index (PREFER_HIGH) or the smaller one.
template <bool UP, bool PREFER_HIGH>
__device__ __forceinline__ MaxArg warp_max_scan(MaxArg x, int lane) {
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const Fx v = UP ? __shfl_up_sync(kFull, x.v, off) : __shfl_down_sync(kFull, x.v, off);
        const int a = UP ? __shfl_up_sync(kFull, x.a, off) : __shfl_down_sync(kFull, x.a, off);
        const bool in = UP ? lane >= off : lane + off < 32;
        if (in) {
            const bool take = v > x.v || (v == x.v && (PREFER_HIGH ? a > x.a : a < x.a));
            if (take) x = {v, a};
        }
    }
    return x;
}

__device__ __forceinline__ bool better(Fx v, int a, const MaxArg &b, bool prefer_high) {
    return v > b.v || (v == b.v && (prefer_high ? a > b.a : a < b.a));
}

__global__ void __launch_bounds__(32 * kUcWarps, 4)
unconstrained_kernel(DevCorpus src, DevCorpus tgt, const PairGeom *__restrict__ geom, const int32_t *__restrict__ order,
                     int64_t n_pairs, DevParams P, const uint8_t *__restrict__ counts, UcScratch W, float *pair_score) {
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const Fx NEG = kNegFx;
    const SimConst K = sim_const(P);
    for (int64_t x = warp0; x < n_pairs; x += nwarps) {
        const int32_t k = order[x];
        const PairGeom g = geom[k];
        const int N = g.n, M = g.m;
        const FxGrid G = fx_grid(N, M, P.gap);
        const Fx p = to_fx(P.gap, G);
        Fx *Aa = W.A + W.a_off[k], *Ab = Aa + (M + 1);
        int32_t *prev = W.prev + W.prev_off[k];
        const int64_t sdoc = src.doc[k], tdoc = tgt.doc[k];
        for (int c = lane; c <= M; c += 32) Aa[c] = c == 0 ? 0 : NEG;
        __syncwarp();
        for (int i = 1; i <= N; ++i) {
            const SimRow row = sim_row((int)(src.sent[sdoc + i] - src.sent[sdoc + i - 1]), P);
            const uchar2 *crow = reinterpret_cast<const uchar2 *>(counts) + g.cell_off + (int64_t)(i - 1) * M;
            int32_t *prow = prev + (int64_t)(i - 1) * (M + 1);
            // suffix maxima Q(c') = max_{c >= c'} A(i-1, c) (nearest: smallest c),
            // right to left; lane handles c' = 32 q + lane + 1 and keeps its value
            const int nq = (M + 32) / 32;  // chunks covering c' = 1 .. M (+ padding)
            // forward prefix maxima first, stored per chunk in registers is not
            // possible for any M: the suffix pass writes Q into Ab (scratch)
            MaxArg carry{NEG, 0x7fffffff};
            for (int q = nq - 1; q >= 0; --q) {
                const int c = 32 * q + lane + 1;
                MaxArg v{c <= M ? Aa[c] : NEG, c <= M ? c : 0x7fffffff};
                v = warp_max_scan<false, false>(v, lane);
                if (better(carry.v, carry.a, v, false)) v = carry;
                if (c <= M) {
                    Ab[c] = v.v;
                    prow[c] = v.a;  // provisional: the back predecessor of c
                }
                const Fx cv = __shfl_sync(kFull, v.v, 0);
                const int ca = __shfl_sync(kFull, v.a, 0);
                carry = {cv, ca};
            }
            __syncwarp();
            // left to right: prefix maxima F(c') = max_{c < c'} A(i-1, c) + p c
            // (nearest: largest c), then the three candidates of every c'
            MaxArg pc{NEG, -1};
            const Fx a0 = Aa[0];
            for (int q = 0; q < nq; ++q) {
                const int c = 32 * q + lane;  // predecessor pointer of c' = c + 1
                MaxArg v{c <= M ? Aa[c] + p * (Fx)c : NEG, c};
                v = warp_max_scan<true, true>(v, lane);
                if (better(pc.v, pc.a, v, true)) v = pc;
                const int c2 = c + 1;
                Fx a_un = 0;
                if (c2 <= M) a_un = Aa[c2];
                __syncwarp();
                if (c2 <= M) {
                    const int lt = (int)(tgt.sent[tdoc + c2] - tgt.sent[tdoc + c2 - 1]);
                    const uchar2 cq = crow[c2 - 1];
                    const Fx sim = to_fx(similarity(cq.x, cq.y, row, sim_col(lt, P), K), G);
                    Fx best = a_un - p;
                    int arg = -1;
                    const Fx fw = sim + v.v - p * (Fx)(c2 - 1);
                    if (fw > best) {
                        best = fw;
                        arg = v.a;
                    }
                    const Fx bk = sim - p + Ab[c2];
                    if (bk > best) {
                        best = bk;
                        arg = prow[c2];
                    }
                    prow[c2] = arg;
                    Ab[c2] = best;
                }
                pc = {__shfl_sync(kFull, v.v, 31), __shfl_sync(kFull, v.a, 31)};
            }
            if (lane == 0) {
                Ab[0] = a0 - p;
                prow[0] = -1;
            }
            __syncwarp();
            Fx *t = Aa;
            Aa = Ab;
            Ab = t;
        }
        // final pointer: max of A(N, c) - p (M - c), smallest c at ties
        MaxArg best{NEG, 0x7fffffff};
        for (int c = lane; c <= M; c += 32) {
            const Fx v = Aa[c] - p * (Fx)(M - c);
            if (better(v, c, best, false)) best = {v, c};
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const Fx v = __shfl_xor_sync(kFull, best.v, off);
            const int a = __shfl_xor_sync(kFull, best.a, off);
            if (better(v, a, best, false)) best = {v, a};
        }
        // traceback (one lane): the matched cells, written from the end of the
        // pair's window of N slots, and their similarities
        if (lane == 0) {
            int c = best.a;
            int n = 0;
            int32_t *li = W.li + W.link_off[k], *lj = W.lj + W.link_off[k];
            float *ls = W.ls + W.link_off[k];
            for (int i = N; i >= 1; --i) {
                const int a = prev[(int64_t)(i - 1) * (M + 1) + c];
                if (a != -1) {
                    const int slot = N - 1 - n;
                    const int lt = (int)(tgt.sent[tdoc + c] - tgt.sent[tdoc + c - 1]);
                    const uchar2 cq = reinterpret_cast<const uchar2 *>(counts)[g.cell_off + (int64_t)(i - 1) * M + c - 1];
                    li[slot] = i - 1;
                    lj[slot] = c - 1;
                    ls[slot] = similarity(cq.x, cq.y, sim_row((int)(src.sent[sdoc + i] - src.sent[sdoc + i - 1]), P),
                                          sim_col(lt, P), K);
                    ++n;
                    c = a;
                }
            }
            W.n_match[k] = n;
            pair_score[k] = from_fx(best.v, G);
        }
        __syncwarp();
    }
}

// The same DP with the row in shared memory and each row scanned in 32
// contiguous segments, one per lane: a lane's serial pass over its segment,
// then one warp scan of the 32 segment maxima, instead of a warp scan per 32
// columns.  Same candidates, same arithmetic, same tie rules.
__device__ __forceinline__ MaxArg excl_scan_left(MaxArg x, int lane) {  // max over lanes < lane, larger index at ties
    MaxArg y = warp_max_scan<true, true>(x, lane);
    MaxArg e{__shfl_up_sync(kFull, y.v, 1), __shfl_up_sync(kFull, y.a, 1)};
    if (lane == 0) e = {kNegFx, -1};
    return e;
}
__device__ __forceinline__ MaxArg excl_scan_right(MaxArg x, int lane) {  // max over lanes > lane, smaller index at ties
    MaxArg y = warp_max_scan<false, false>(x, lane);
    MaxArg e{__shfl_down_sync(kFull, y.v, 1), __shfl_down_sync(kFull, y.a, 1)};
    if (lane == 31) e = {kNegFx, 0x7fffffff};
    return e;
}

// Per warp, mcap columns of each: the score row (updated in place: every
// read of the previous row precedes the writes), the suffix maxima and their
// arguments, the row's similarities and the pair's per-column constants
// (1 / lt, lt) -- 32 bytes a column.
__global__ void __launch_bounds__(32 * kUcShortWarps, 3)
unconstrained_smem_kernel(DevCorpus src, DevCorpus tgt, const PairGeom *__restrict__ geom,
                          const int32_t *__restrict__ order, int64_t n_pairs, DevParams P,
                          const uint8_t *__restrict__ counts, UcScratch W, float *pair_score, int mcap) {
    extern __shared__ __align__(16) unsigned char uc_smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    Fx *A = reinterpret_cast<Fx *>(uc_smem) + (int64_t)warp * 2 * mcap;
    Fx *Qv = A + mcap;
    float2 *colc = reinterpret_cast<float2 *>(reinterpret_cast<Fx *>(uc_smem) + (int64_t)nw * 2 * mcap) +
                   (int64_t)warp * mcap;
    int32_t *Qa = reinterpret_cast<int32_t *>(reinterpret_cast<float2 *>(reinterpret_cast<Fx *>(uc_smem) +
                                                                         (int64_t)nw * 2 * mcap) +
                                              (int64_t)nw * mcap) +
                  (int64_t)warp * mcap;
    float *Sm = reinterpret_cast<float *>(Qa - (int64_t)warp * mcap + (int64_t)nw * mcap) + (int64_t)warp * mcap;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const Fx NEG = kNegFx;
    const SimConst K = sim_const(P);
    const float kb = __fmul_rn(-kLog2e, P.w[1]);  // SimCol.b = kb / lt, as sim_col rounds it
    for (int64_t x = warp0; x < n_pairs; x += nwarps) {
        const int32_t k = order[x];
        const PairGeom g = geom[k];
        const int N = g.n, M = g.m;
        const FxGrid G = fx_grid(N, M, P.gap);
        const Fx p = to_fx(P.gap, G);
        int32_t *prev = W.prev + W.prev_off[k];
        const int64_t sdoc = src.doc[k], tdoc = tgt.doc[k];
        const int L = (M + 1 + 31) / 32;  // columns 0..M in 32 segments
        const int lo = lane * L, hi = min(lo + L, M + 1);
        for (int c = lane; c <= M; c += 32) {
            A[c] = c == 0 ? 0 : NEG;
            if (c >= 1) {
                const int lt = (int)(tgt.sent[tdoc + c] - tgt.sent[tdoc + c - 1]);
                colc[c] = make_float2(__frcp_rn((float)lt), (float)lt);
            }
        }
        __syncwarp();
        for (int i = 1; i <= N; ++i) {
            const SimRow row = sim_row((int)(src.sent[sdoc + i] - src.sent[sdoc + i - 1]), P);
            const uchar2 *crow = reinterpret_cast<const uchar2 *>(counts) + g.cell_off + (int64_t)(i - 1) * M;
            int32_t *prow = prev + (int64_t)(i - 1) * (M + 1);
            // the row's similarities, lane-strided, four count loads in flight
            for (int cb = 1 + lane; cb <= M; cb += 128) {
                uchar2 q[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) q[u] = cb + 32 * u <= M ? crow[cb + 32 * u - 1] : make_uchar2(0, 0);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int c2 = cb + 32 * u;
                    if (c2 <= M) {
                        const float2 cc = colc[c2];
                        const SimCol col{__fmul_rn(kb, cc.x), cc.y, cc.x, 0.0f};
                        Sm[c2] = similarity(q[u].x, q[u].y, row, col, K);
                    }
                }
            }
            // suffix maxima of A(i-1, .) inside the segment, right to left
            MaxArg run{NEG, 0x7fffffff};
#pragma unroll 4
            for (int c = hi - 1; c >= lo; --c) {
                const Fx v = A[c];
                if (v >= run.v) run = {v, c};
                Qv[c] = run.v;
                Qa[c] = run.a;
            }
            const MaxArg right = excl_scan_right(run, lane);
            // prefix maxima of A(i-1, c) + p c over the lower lanes' segments
            MaxArg agg{NEG, -1};
#pragma unroll 4
            for (int c = lo; c < hi; ++c) {
                const Fx v = A[c] + p * (Fx)c;
                if (v >= agg.v) agg = {v, c};
            }
            MaxArg pre = excl_scan_left(agg, lane);
            __syncwarp();
            // candidates of c' in the segment, left to right (pre: the best
            // forward predecessor c < c'); A(i, c') replaces A(i-1, c') once
            // read
            for (int c2 = lo; c2 < hi; ++c2) {
                const Fx a_here = A[c2];
                if (c2 >= 1) {
                    const Fx sim = to_fx(Sm[c2], G);
                    Fx best = a_here - p;
                    int arg = -1;
                    const Fx fw = sim + pre.v - p * (Fx)(c2 - 1);
                    if (fw > best) {
                        best = fw;
                        arg = pre.a;
                    }
                    const MaxArg q = right.v > Qv[c2] ? right : MaxArg{Qv[c2], Qa[c2]};
                    const Fx bk = sim - p + q.v;
                    if (bk > best) {
                        best = bk;
                        arg = q.a;
                    }
                    A[c2] = best;
                    prow[c2] = arg;
                } else {
                    A[0] = a_here - p;
                    prow[0] = -1;
                }
                const Fx v = a_here + p * (Fx)c2;
                if (v >= pre.v) pre = {v, c2};
            }
            __syncwarp();
        }
        MaxArg best{NEG, 0x7fffffff};
        for (int c = lane; c <= M; c += 32) {
            const Fx v = A[c] - p * (Fx)(M - c);
            if (better(v, c, best, false)) best = {v, c};
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const Fx v = __shfl_xor_sync(kFull, best.v, off);
            const int a = __shfl_xor_sync(kFull, best.a, off);
            if (better(v, a, best, false)) best = {v, a};
        }
        if (lane == 0) {
            int c = best.a;
            int n = 0;
            int32_t *li = W.li + W.link_off[k], *lj = W.lj + W.link_off[k];
            float *ls = W.ls + W.link_off[k];
            for (int i = N; i >= 1; --i) {
                const int a = prev[(int64_t)(i - 1) * (M + 1) + c];
                if (a != -1) {
                    const int slot = N - 1 - n;
                    const int lt = (int)(tgt.sent[tdoc + c] - tgt.sent[tdoc + c - 1]);
                    const uchar2 cq = reinterpret_cast<const uchar2 *>(counts)[g.cell_off + (int64_t)(i - 1) * M + c - 1];
                    li[slot] = i - 1;
                    lj[slot] = c - 1;
                    ls[slot] = similarity(cq.x, cq.y, sim_row((int)(src.sent[sdoc + i] - src.sent[sdoc + i - 1]), P),
                                          sim_col(lt, P), K);
                    ++n;
                    c = a;
                }
            }
            W.n_match[k] = n;
            pair_score[k] = from_fx(best.v, G);
        }
        __syncwarp();
    }
}

// The same DP for long targets with one block of kUcCtaThreads threads per
// pair: columns 0..M in one contiguous segment per thread, the segment
// aggregates combined by block scans (a warp scan, then the warps' totals in
// shared memory), two block barriers per row.  Same candidates, same
// arithmetic, same tie rules.  Shared memory: mcap columns of A, Q (int64),
// colc (float2), Qa (int32), Sm (float), then the scans' warp totals.
constexpr int kUcCtaThreads = 128;
constexpr int kUcCtaWarps = kUcCtaThreads / 32;

__global__ void __launch_bounds__(kUcCtaThreads, 4)
unconstrained_cta_kernel(DevCorpus src, DevCorpus tgt, const PairGeom *__restrict__ geom,
                         const int32_t *__restrict__ order, int64_t n_pairs, DevParams P,
                         const uint8_t *__restrict__ counts, UcScratch W, float *pair_score, int mcap) {
    extern __shared__ __align__(16) unsigned char uc_smem[];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    Fx *A = reinterpret_cast<Fx *>(uc_smem);
    Fx *Qv = A + mcap;
    float2 *colc = reinterpret_cast<float2 *>(Qv + mcap);
    int32_t *Qa = reinterpret_cast<int32_t *>(colc + mcap);
    float *Sm = reinterpret_cast<float *>(Qa + mcap);
    MaxArg *tot_r = reinterpret_cast<MaxArg *>(Sm + mcap);  // at 32 mcap bytes: 8-byte aligned
    MaxArg *tot_l = tot_r + kUcCtaWarps;
    const Fx NEG = kNegFx;
    const SimConst K = sim_const(P);
    const float kb = __fmul_rn(-kLog2e, P.w[1]);
    for (int64_t x = blockIdx.x; x < n_pairs; x += gridDim.x) {
        const int32_t k = order[x];
        const PairGeom g = geom[k];
        const int N = g.n, M = g.m;
        const FxGrid G = fx_grid(N, M, P.gap);
        const Fx p = to_fx(P.gap, G);
        int32_t *prev = W.prev + W.prev_off[k];
        const int64_t sdoc = src.doc[k], tdoc = tgt.doc[k];
        const int L = (M + 1 + kUcCtaThreads - 1) / kUcCtaThreads;
        const int lo = min(t * L, M + 1), hi = min(lo + L, M + 1);
        __syncthreads();  // the previous pair is done with the rows
        for (int c = t; c <= M; c += kUcCtaThreads) {
            A[c] = c == 0 ? 0 : NEG;
            if (c >= 1) {
                const int lt = (int)(tgt.sent[tdoc + c] - tgt.sent[tdoc + c - 1]);
                colc[c] = make_float2(__frcp_rn((float)lt), (float)lt);
            }
        }
        __syncthreads();
        for (int i = 1; i <= N; ++i) {
            const SimRow row = sim_row((int)(src.sent[sdoc + i] - src.sent[sdoc + i - 1]), P);
            const uchar2 *crow = reinterpret_cast<const uchar2 *>(counts) + g.cell_off + (int64_t)(i - 1) * M;
            int32_t *prow = prev + (int64_t)(i - 1) * (M + 1);
            for (int cb = 1 + t; cb <= M; cb += 4 * kUcCtaThreads) {
                uchar2 q[4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    q[u] = cb + kUcCtaThreads * u <= M ? crow[cb + kUcCtaThreads * u - 1] : make_uchar2(0, 0);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int c2 = cb + kUcCtaThreads * u;
                    if (c2 <= M) {
                        const float2 cc = colc[c2];
                        const SimCol col{__fmul_rn(kb, cc.x), cc.y, cc.x, 0.0f};
                        Sm[c2] = similarity(q[u].x, q[u].y, row, col, K);
                    }
                }
            }
            MaxArg run{NEG, 0x7fffffff};
            for (int c = hi - 1; c >= lo; --c) {
                const Fx v = A[c];
                if (v >= run.v) run = {v, c};
                Qv[c] = run.v;
                Qa[c] = run.a;
            }
            MaxArg agg{NEG, -1};
            for (int c = lo; c < hi; ++c) {
                const Fx v = A[c] + p * (Fx)c;
                if (v >= agg.v) agg = {v, c};
            }
            // block scans: over the threads after t (smaller index at ties)
            // and before t (larger index at ties)
            const MaxArg ir = warp_max_scan<false, false>(run, lane);
            const MaxArg il = warp_max_scan<true, true>(agg, lane);
            if (lane == 0) tot_r[warp] = ir;
            if (lane == 31) tot_l[warp] = il;
            MaxArg right{__shfl_down_sync(kFull, ir.v, 1), __shfl_down_sync(kFull, ir.a, 1)};
            if (lane == 31) right = {NEG, 0x7fffffff};
            MaxArg pre{__shfl_up_sync(kFull, il.v, 1), __shfl_up_sync(kFull, il.a, 1)};
            if (lane == 0) pre = {NEG, -1};
            __syncthreads();  // warp totals, and the row's similarities, are visible
            for (int w = warp + 1; w < kUcCtaWarps; ++w)
                if (better(tot_r[w].v, tot_r[w].a, right, false)) right = tot_r[w];
            for (int w = 0; w < warp; ++w)
                if (better(tot_l[w].v, tot_l[w].a, pre, true)) pre = tot_l[w];
            for (int c2 = lo; c2 < hi; ++c2) {
                const Fx a_here = A[c2];
                if (c2 >= 1) {
                    const Fx sim = to_fx(Sm[c2], G);
                    Fx best = a_here - p;
                    int arg = -1;
                    const Fx fw = sim + pre.v - p * (Fx)(c2 - 1);
                    if (fw > best) {
                        best = fw;
                        arg = pre.a;
                    }
                    const MaxArg q = right.v > Qv[c2] ? right : MaxArg{Qv[c2], Qa[c2]};
                    const Fx bk = sim - p + q.v;
                    if (bk > best) {
                        best = bk;
                        arg = q.a;
                    }
                    A[c2] = best;
                    prow[c2] = arg;
                } else {
                    A[0] = a_here - p;
                    prow[0] = -1;
                }
                const Fx v = a_here + p * (Fx)c2;
                if (v >= pre.v) pre = {v, c2};
            }
            __syncthreads();  // the row is complete before the next one reads it
        }
        // final pointer: max of A(N, c) - p (M - c), smallest c at ties
        MaxArg best{NEG, 0x7fffffff};
        for (int c = t; c <= M; c += kUcCtaThreads) {
            const Fx v = A[c] - p * (Fx)(M - c);
            if (better(v, c, best, false)) best = {v, c};
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const Fx v = __shfl_xor_sync(kFull, best.v, off);
            const int a = __shfl_xor_sync(kFull, best.a, off);
            if (better(v, a, best, false)) best = {v, a};
        }
        if (lane == 0) tot_r[warp] = best;
        __syncthreads();
        if (t == 0) {
            for (int w = 1; w < kUcCtaWarps; ++w)
                if (better(tot_r[w].v, tot_r[w].a, best, false)) best = tot_r[w];
            int c = best.a;
            int n = 0;
            int32_t *li = W.li + W.link_off[k], *lj = W.lj + W.link_off[k];
            float *ls = W.ls + W.link_off[k];
            for (int i = N; i >= 1; --i) {
                const int a = prev[(int64_t)(i - 1) * (M + 1) + c];
                if (a != -1) {
                    const int slot = N - 1 - n;
                    const int lt = (int)(tgt.sent[tdoc + c] - tgt.sent[tdoc + c - 1]);
                    const uchar2 cq = reinterpret_cast<const uchar2 *>(counts)[g.cell_off + (int64_t)(i - 1) * M + c - 1];
                    li[slot] = i - 1;
                    lj[slot] = c - 1;
                    ls[slot] = similarity(cq.x, cq.y, sim_row((int)(src.sent[sdoc + i] - src.sent[sdoc + i - 1]), P),
                                          sim_col(lt, P), K);
                    ++n;
                    c = a;
                }
            }
            W.n_match[k] = n;
            pair_score[k] = from_fx(best.v, G);
        }
    }
}

// Links of every pair with s >= thr, in row order, compacted at out_off.
__global__ void __launch_bounds__(32 * kUcWarps)
uc_count_kernel(const PairGeom *__restrict__ geom, int64_t n_pairs, float thr, UcScratch W, int32_t *kept) {
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t k = warp0; k < n_pairs; k += nwarps) {
        const int N = geom[k].n, n = W.n_match[k];
        const float *ls = W.ls + W.link_off[k] + N - n;
        int c = 0;
        for (int x = lane; x < n; x += 32) c += ls[x] >= thr;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(kFull, c, off);
        if (lane == 0) kept[k] = c;
    }
}

__global__ void __launch_bounds__(32 * kUcWarps)
uc_copy_kernel(const PairGeom *__restrict__ geom, int64_t n_pairs, float thr, UcScratch W, const int64_t *out_off,
               int32_t *out_i, int32_t *out_j, float *out_s) {
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t k = warp0; k < n_pairs; k += nwarps) {
        const int N = geom[k].n, n = W.n_match[k];
        const int64_t base = W.link_off[k] + N - n;
        int64_t to = out_off[k];
        for (int x0 = 0; x0 < n; x0 += 32) {
            const int x = x0 + lane;
            const float s = x < n ? W.ls[base + x] : 0.0f;
            const bool keep = x < n && s >= thr;
            const uint32_t m = __ballot_sync(kFull, keep);
            if (keep) {
                const int64_t o = to + __popc(m & ((1u << lane) - 1u));
                out_i[o] = W.li[base + x];
                out_j[o] = W.lj[base + x];
                out_s[o] = s;
            }
            to += __popc(m);
        }
    }
}

int uc_grid(int64_t n_pairs, int n_sms) {
    int64_t b = (n_pairs + kUcWarps - 1) / kUcWarps;
    const int64_t cap = (int64_t)n_sms * 16;
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

namespace {

// The pairs order[0, n) on the shared-row kernel with rows of mcap columns
// (up to max_warps warps per block, as many as fit in 200 KB), or on the
// global-row kernel when one warp's rows do not fit.
cudaError_t launch_uc_rows(const DevCorpus &src, const DevCorpus &tgt, const PairGeom *geom, const int32_t *order,
                           int64_t n, const DevParams &P, const uint8_t *counts, const UcScratch &W, float *pair_score,
                           int mcap, int max_warps, int n_sms, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const int64_t per_warp = 32 * (int64_t)mcap;  // bytes per column: two score rows and the maxima (int64), arguments (int32), similarities (FP32)
    const int warps = (int)std::min<int64_t>(max_warps, (200 << 10) / per_warp);
    if (warps < 1) {
        unconstrained_kernel<<<uc_grid(n, n_sms), 32 * kUcWarps, 0, st>>>(src, tgt, geom, order, n, P, counts, W,
                                                                         pair_score);
        return cudaGetLastError();
    }
    const size_t smem = (size_t)(per_warp * warps);
    cudaError_t e = cudaFuncSetAttribute(unconstrained_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, unconstrained_smem_kernel, 32 * warps, smem);
    if (e != cudaSuccess) return e;
    int64_t blocks = (n + warps - 1) / warps;
    const int64_t cap = (int64_t)n_sms * (per_sm > 0 ? per_sm : 1);
    if (blocks > cap) blocks = cap;
    unconstrained_smem_kernel<<<(unsigned)blocks, 32 * warps, smem, st>>>(src, tgt, geom, order, n, P, counts, W,
                                                                        pair_score, mcap);
    return cudaGetLastError();
}

}  // namespace

// The pairs order[0, n) with one block of kUcCtaThreads per pair, rows of
// mcap columns in shared memory, or on the global-row kernel when they do not
// fit.
static cudaError_t launch_uc_cta(const DevCorpus &src, const DevCorpus &tgt, const PairGeom *geom, const int32_t *order,
                          int64_t n, const DevParams &P, const uint8_t *counts, const UcScratch &W, float *pair_score,
                          int mcap, int n_sms, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const int64_t bytes = 32 * (int64_t)mcap + 2 * kUcCtaWarps * (int64_t)sizeof(MaxArg);
    if (bytes > (200 << 10))
        return launch_uc_rows(src, tgt, geom, order, n, P, counts, W, pair_score, mcap, kUcWarps, n_sms, st);
    cudaError_t e = cudaFuncSetAttribute(unconstrained_cta_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)bytes);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, unconstrained_cta_kernel, kUcCtaThreads, (size_t)bytes);
    if (e != cudaSuccess) return e;
    int64_t blocks = n;
    const int64_t cap = (int64_t)n_sms * (per_sm > 0 ? per_sm : 1);
    if (blocks > cap) blocks = cap;
    unconstrained_cta_kernel<<<(unsigned)blocks, kUcCtaThreads, (size_t)bytes, st>>>(src, tgt, geom, order, n, P,
                                                                                    counts, W, pair_score, mcap);
    return cudaGetLastError();
}

cudaError_t launch_unconstrained(const DevCorpus &src, const DevCorpus &tgt, const PairGeom *geom, const int32_t *order,
                                 int64_t n_short, int64_t n_pairs, const DevParams &P, const uint8_t *counts,
                                 const UcScratch &W, float *pair_score, int max_m, int32_t *kept, int n_sms,
                                 cudaStream_t st) {
    if (n_pairs == 0) return cudaSuccess;
    // long targets first (few pairs: a block of threads each, rows sized by
    // the longest), then the short ones, eight warps per block on 8 KB of
    // rows each
    cudaError_t e = launch_uc_cta(src, tgt, geom, order + n_short, n_pairs - n_short, P, counts, W, pair_score,
                                  max_m + 1, n_sms, st);
    if (e != cudaSuccess) return e;
    e = launch_uc_rows(src, tgt, geom, order, n_short, P, counts, W, pair_score, kUcShortCols, kUcShortWarps, n_sms, st);
    if (e != cudaSuccess) return e;
    uc_count_kernel<<<uc_grid(n_pairs, n_sms), 32 * kUcWarps, 0, st>>>(geom, n_pairs, P.thr, W, kept);
    return cudaGetLastError();
}

cudaError_t launch_unconstrained_copy(const PairGeom *geom, int64_t n_pairs, float thr, const UcScratch &W,
                                      const int64_t *out_off, int32_t *out_i, int32_t *out_j, float *out_s, int n_sms,
                                      cudaStream_t st) {
    if (n_pairs == 0) return cudaSuccess;
    uc_copy_kernel<<<uc_grid(n_pairs, n_sms), 32 * kUcWarps, 0, st>>>(geom, n_pairs, thr, W, out_off, out_i, out_j,
                                                                     out_s);
    return cudaGetLastError();
}

}  // namespace gbm
