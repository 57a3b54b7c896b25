// Differentiable (soft) Needleman-Wunsch for parameter tuning.
//
// The paper tunes the acceptance threshold and the gap penalty by random
// search against human alignments (Section 5.2).  Here the max of the fill
// (Section 5.1, Eq. 1) is smoothed into gamma * log-sum-exp, which makes the
// alignment differentiable:
//   V(i,j) = gamma * LSE((V(i-1,j-1) + s_ij)/gamma, (V(i-1,j) - p)/gamma, (V(i,j-1) - p)/gamma)
// with the hard borders V(i,0) = -i p, V(0,j) = -j p.  E = dV(N,M)/ds is the
// expected alignment (the probability that the path takes cell (i,j)
// diagonally under the Gibbs distribution over paths); the tuning loss is
//   P = clamp(E * sigmoid((s - thr)/tau), eps, 1-eps),  L = mean BCE(P, gold).
// dL/ds needs the derivative of E, i.e. a Hessian-vector product of V, which
// is obtained forward-over-reverse: a tangent sweep along u = dL/dE, then the
// tangent of the adjoint sweep.
//
// Every sweep works on differences, as the hard fill does: with
//   A = V(i-1,j) - V(i-1,j-1) - p, B = V(i,j-1) - V(i-1,j-1) - p,
//   D = V(i,j) - V(i-1,j-1) = gamma LSE(s, A, B)/gamma,
// the softmax weights are wd = e^{(s-D)/g}, wu = e^{(A-D)/g}, wl = e^{(B-D)/g};
// the next candidates are D - B - 2p (down) and D - A - 2p (right).  The
// tangent V' along u has the same shape: with A' = V'(i-1,j) - V'(i-1,j-1),
// B' = V'(i,j-1) - V'(i-1,j-1):  D' = wd u + wu A' + wl B', down D' - B',
// right D' - A'.  All quantities stay O(1), so FP32 keeps its precision; the
// tangent differences are formed from pairwise candidate differences (see
// soft_fwd_strip) so that saturated cells (one weight ~ 1) do not cancel.
//
// Adjoint: Q(N,M) = 1, and every node pushes Q * w_k to its predecessor k;
// E = Q wd.  Its tangent: Q' pushes Q' w_k + Q w_k', w_k' = w_k (c_k - D')/g
// with c_d = u, c_u = A', c_l = B'; E' = Q' wd + Q wd' = (H u).
// Because every path takes N + M - 2 #diag gap steps, V(s,p) = V0(s + 2p) -
// p (N + M), so dE/dp = 2 H 1 and dL/dp (through E) = 2 sum(H u).
//
// Memory: per cell only E and u are kept (u is computed at the start of the
// backward and replaced by H u in place).  The
// forward sweeps checkpoint the boundary row of every 32-row strip; a backward
// sweep recomputes the strip's forward from its checkpoint into a per-warp
// strip buffer (anti-diagonal major, so that both the skewed forward and the
// reverse-skewed backward move 128 contiguous bytes per step) and then runs
// the reverse sweep over it.  One warp owns a pair.
//
// The sweeps carry only the recurrences: the similarities (and u) of a
// 32 x 32 block are computed before its 32 steps into shared memory (rotated,
// so that writes and the skewed reads hit distinct banks), and the reverse
// sweeps fetch their per-cell weights eight steps ahead.  The loss, u and the
// chain rule to the seven parameters are per-cell work, done by separate
// fully parallel kernels.
#include "kernels.h"

namespace gbm {
namespace {

constexpr int kSoftWarps = 4;
constexpr float kLn2 = 0.6931471805599453f;

__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct SoftCtx {
    int lane, N, M, nstrips;
    float two_p, gamma, kexp, kln, thr, ktau, eps, inv_cells;
    SimConst K;
    DevParams P;
    SimRow row;            // constants of this lane's source sentence (current strip)
    const int64_t *ssent, *tsent;
    const uchar2 *cnt;     // pair's counts
    const uint8_t *gold;   // pair's gold links (0/1 per cell)
    float *E;              // pair's expected alignment
    float *U;              // pair's tangent direction u = dL/dE, then H u
    SimCol *colv;          // shared: column constants of the block being prepared
    float (*svb)[32][32];  // shared: similarities of the current and previous block [2][row][col]
    float (*ub)[32][32];   // shared: u of the current and previous block
};

// Soft max of three candidates relative to a common base: returns D and the
// three weights.
__device__ __forceinline__ float soft3(float s, float a, float b, const SoftCtx &C, float &wd, float &wu, float &wl) {
    const float m = fmaxf(fmaxf(s, a), b);
    const float ed = ex2_approx(__fmul_rn(__fsub_rn(s, m), C.kexp));
    const float eu = ex2_approx(__fmul_rn(__fsub_rn(a, m), C.kexp));
    const float el = ex2_approx(__fmul_rn(__fsub_rn(b, m), C.kexp));
    const float z = __fadd_rn(__fadd_rn(ed, eu), el);
    const float rz = rcp_approx(z);
    wd = __fmul_rn(ed, rz);
    wu = __fmul_rn(eu, rz);
    wl = __fmul_rn(el, rz);
    return __fmaf_rn(C.kln, lg2_approx(z), m);
}

__device__ __forceinline__ float cell_similarity(const SoftCtx &C, const SimRow &row, int r, int j) {
    const uchar2 q = C.cnt[(int64_t)r * C.M + j];
    return similarity(q.x, q.y, row, sim_col((int)(C.tsent[j + 1] - C.tsent[j]), C.P), C.K);
}

// Gate, clamped P and dBCE/dP of one cell (dBCE/dP is 0 where P was clamped);
// the loss term of the cell goes to *bce when asked.
__device__ __forceinline__ float cell_dldp(float E, float sv, int g, const SoftCtx &C, float &G, float *bce) {
    G = rcp_approx(__fadd_rn(1.0f, ex2_approx(__fmul_rn(__fsub_rn(C.thr, sv), C.ktau))));
    const float Pr = __fmul_rn(E, G);
    const bool lo = Pr < C.eps, hi = Pr > 1.0f - C.eps;
    const float Pc = lo ? C.eps : (hi ? 1.0f - C.eps : Pr);
    if (bce) *bce = g ? -__fmul_rn(kLn2, lg2_approx(Pc)) : -__fmul_rn(kLn2, lg2_approx(__fsub_rn(1.0f, Pc)));
    if (lo || hi) return 0.0f;
    return __fmul_rn(g ? -rcp_approx(Pr) : rcp_approx(__fsub_rn(1.0f, Pr)), C.inv_cells);
}

// Similarities (and u) of block jb of the current strip into shared buffer
// jb & 1; lane = row, columns written in rotated order.
template <bool TAN>
__device__ __forceinline__ void soft_prep_block(const SoftCtx &C, int r, bool rv, int jb) {
    const int lane = C.lane;
    const int col0 = 32 * jb;
    __syncwarp();
    C.colv[lane] = sim_col(col0 + lane < C.M ? (int)(C.tsent[col0 + lane + 1] - C.tsent[col0 + lane]) : 1, C.P);
    __syncwarp();
    float(*sv)[32] = C.svb[jb & 1];
    float(*ub)[32] = C.ub[jb & 1];
    const uchar2 *rowc = C.cnt + (int64_t)r * C.M;
#pragma unroll 8
    for (int x = 0; x < 32; ++x) {
        const int c = (x + lane) & 31;
        const int col = col0 + c;
        float v = 0.0f, u = 0.0f;
        if (rv && col < C.M) {
            const uchar2 q = rowc[col];
            v = similarity(q.x, q.y, C.row, C.colv[c], C.K);
            if (TAN) u = C.U[(int64_t)r * C.M + col];
        }
        sv[lane][c] = v;
        if (TAN) ub[lane][c] = u;
    }
    __syncwarp();
}

// Forward sweep of strip s (rows 32s..32s+31, lane = row, skewed by lane).
//   TAN:   also run the tangent along u (needs U of the pair)
//   STORE: write the per-cell quantities the reverse sweep needs into sbuf,
//          anti-diagonal major: sbuf[k][t][lane] for step t, component k
// ck*_top: the strip above's checkpoint row (UP candidates of row 32s-1);
// ck*_out: this strip's checkpoint row (written by the last lane), may be null.
// vlast (may be null): receives the DOWN outputs of row N-1, V(N,j) - V(N,j-1) - p,
// from which V(N,M) is summed in FP64 outside the sweep.
template <bool TAN, bool STORE>
__device__ __forceinline__ void soft_fwd_strip(SoftCtx &C, int s, const float *__restrict__ ckv_top,
                                               const float *__restrict__ ckt_top, float *__restrict__ ckv_out,
                                               float *__restrict__ ckt_out, float *__restrict__ sbuf,
                                               float *__restrict__ vlast) {
    const int lane = C.lane;
    const int r = 32 * s + lane;
    const bool rv = r < C.N;
    C.row = sim_row(rv ? (int)(C.ssent[r + 1] - C.ssent[r]) : 1, C.P);
    const int64_t plane = (int64_t)(C.M + 31) * 32;
    const int nb = (C.M + 31) >> 5;
    float b = -C.two_p, a_down = 0.0f;
    float bt = 0.0f, at_down = 0.0f;
    for (int jb = 0; jb <= nb; ++jb) {
        if (jb < nb) soft_prep_block<TAN>(C, r, rv, jb);
        const int colx = 32 * jb + lane;
        const bool top = s > 0 && colx < C.M;
        const float hv = top ? __ldcg(ckv_top + colx) : -C.two_p;
        const float htv = (TAN && top) ? __ldcg(ckt_top + colx) : 0.0f;
#pragma unroll 4
        for (int u = 0; u < 32; ++u) {
            const int t = 32 * jb + u;
            float a_up = __shfl_up_sync(kFull, a_down, 1);
            float at_up = TAN ? __shfl_up_sync(kFull, at_down, 1) : 0.0f;
            const float h0 = __shfl_sync(kFull, hv, u);
            const float ht0 = TAN ? __shfl_sync(kFull, htv, u) : 0.0f;
            if (lane == 0) {
                a_up = h0;
                if (TAN) at_up = ht0;
            }
            const int j = t - lane;
            if (rv && j >= 0 && j < C.M) {
                const int bb = (j >> 5) & 1, c = j & 31;
                const float sv = C.svb[bb][lane][c];
                float wd, wu, wl;
                const float D = soft3(sv, a_up, b, C, wd, wu, wl);
                const float e = __fsub_rn(D, C.two_p);
                const float nb2 = __fsub_rn(e, a_up);
                a_down = __fsub_rn(e, b);
                // tangent: with the weights summing to one, every difference the
                // sweeps need is a weighted sum of pairwise candidate differences,
                // so nothing cancels when one weight is close to 1 (a saturated
                // alignment); e.g. u - D' = wu (u - A') + wl (u - B').
                float cd = 0.0f, cu = 0.0f, cl = 0.0f;
                if (TAN) {
                    const float uu = C.ub[bb][lane][c];
                    const float dua = __fsub_rn(uu, at_up), dub = __fsub_rn(uu, bt), dab = __fsub_rn(at_up, bt);
                    cd = __fmaf_rn(wu, dua, __fmul_rn(wl, dub));
                    cu = __fmaf_rn(wl, dab, -__fmul_rn(wd, dua));
                    cl = -__fmaf_rn(wd, dub, __fmul_rn(wu, dab));
                    at_down = __fmaf_rn(wd, dub, __fmul_rn(wu, dab));  // D' - B'
                    bt = __fmaf_rn(wd, dua, -__fmul_rn(wl, dab));      // D' - A'
                }
                b = nb2;
                if (STORE) {
                    float *q = sbuf + (int64_t)t * 32 + lane;
                    q[0] = wd;
                    q[plane] = wu;
                    q[2 * plane] = wl;
                    if (TAN) {
                        q[3 * plane] = cd;
                        q[4 * plane] = cu;
                        q[5 * plane] = cl;
                    }
                }
                if (lane == 31 && ckv_out) {
                    __stcg(ckv_out + j, a_down);
                    if (TAN) __stcg(ckt_out + j, at_down);
                }
                if (vlast && r == C.N - 1) __stcg(vlast + j, a_down);
            }
        }
    }
    __syncwarp();
}

// Reverse sweep over strip s with the weights the STORE forward left in sbuf:
// the adjoint Q (E = Q wd) and, with TAN, its tangent Q' (H u = Q' wd + Q wd').
// Reverse skew: lane i handles column M-1-(t-(31-i)) at step t, so that the
// cell below (lane i+1) was done one step earlier; its outflows come up by a
// shuffle, the strip below's through qrow/qtrow.
template <bool TAN>
__device__ __forceinline__ void soft_rev_strip(SoftCtx &C, int s, const float *__restrict__ sbuf, float *qrow,
                                               float *qtrow, float rgamma) {
    const int lane = C.lane;
    const int r = 32 * s + lane;
    const bool rv = r < C.N;
    const bool last = s == C.nstrips - 1;
    const int64_t plane = (int64_t)(C.M + 31) * 32;
    const int T = C.M + 31;
    float q_send = 0.0f, dflow = 0.0f, qright = 0.0f;
    float qt_send = 0.0f, dtflow = 0.0f, qtright = 0.0f;
    constexpr int NC = TAN ? 6 : 3;
    constexpr int CH = 8;  // steps per prefetched chunk
    // chunk loader: the weights of steps t0..t0+7 (registers) and, in lanes
    // 0..7, the inflow from the strip below for the columns lane 31 meets then
    auto load = [&](int t0, float (&w)[CH][NC], float &qb, float &qtb) {
#pragma unroll
        for (int k = 0; k < CH; ++k) {
            const int t = t0 + k;
            const float *q = sbuf + (int64_t)(C.M + 30 - t) * 32 + lane;
#pragma unroll
            for (int cpt = 0; cpt < NC; ++cpt) w[k][cpt] = t < T ? __ldcg(q + cpt * plane) : 0.0f;
        }
        const int jl = C.M - 1 - (t0 + lane);  // lane 31's column at step t0 + lane
        const bool in = !last && lane < CH && jl >= 0 && jl < C.M;
        qb = in ? __ldcg(qrow + jl) : 0.0f;
        qtb = (TAN && in) ? __ldcg(qtrow + jl) : 0.0f;
    };
    float wa[CH][NC], wb[CH][NC];
    float qa = 0.0f, qta = 0.0f, qb = 0.0f, qtb = 0.0f;
    load(0, wa, qa, qta);
    auto run = [&](int t0, const float (&w)[CH][NC], float qbl, float qtbl) {
#pragma unroll
        for (int k = 0; k < CH; ++k) {
            const int t = t0 + k;
            if (t >= T) break;
            float from_below = __shfl_down_sync(kFull, q_send, 1);
            float from_below_t = TAN ? __shfl_down_sync(kFull, qt_send, 1) : 0.0f;
            const float fb = __shfl_sync(kFull, qbl, k);
            const float fbt = TAN ? __shfl_sync(kFull, qtbl, k) : 0.0f;
            const int j = C.M - 1 - (t - (31 - lane));
            if (lane == 31) {
                from_below = fb;
                if (TAN) from_below_t = fbt;
            }
            if (rv && j >= 0 && j < C.M) {
                const float wd = w[k][0], wu = w[k][1], wl = w[k][2];
                float Q = __fadd_rn(from_below, qright);
                float Qt = TAN ? __fadd_rn(from_below_t, qtright) : 0.0f;
                if (r == C.N - 1 && j == C.M - 1) {
                    Q = 1.0f;
                    Qt = 0.0f;
                }
                const float Ec = __fmul_rn(Q, wd);
                qright = __fmul_rn(Q, wl);
                q_send = __fadd_rn(__fmul_rn(Q, wu), dflow);
                dflow = Ec;
                const int64_t c = (int64_t)r * C.M + j;
                if (TAN) {
                    // weight tangents w_k' = w_k (c_k - D') / gamma
                    const float wdt = __fmul_rn(__fmul_rn(wd, w[k][3]), rgamma);
                    const float wut = __fmul_rn(__fmul_rn(wu, w[k][4]), rgamma);
                    const float wlt = __fmul_rn(__fmul_rn(wl, w[k][5]), rgamma);
                    const float Hu = __fmaf_rn(Q, wdt, __fmul_rn(Qt, wd));
                    qtright = __fmaf_rn(Q, wlt, __fmul_rn(Qt, wl));
                    qt_send = __fadd_rn(__fmaf_rn(Q, wut, __fmul_rn(Qt, wu)), dtflow);
                    dtflow = Hu;
                    C.U[c] = Hu;
                    if (lane == 0) __stcg(qtrow + j, qt_send);
                } else {
                    C.E[c] = Ec;
                }
                if (lane == 0) __stcg(qrow + j, q_send);
            } else {
                q_send = dflow = qright = 0.0f;
                qt_send = dtflow = qtright = 0.0f;
            }
        }
    };
    // two chunks in flight: load chunk c+1 while chunk c runs
    for (int t0 = 0; t0 < T; t0 += 2 * CH) {
        if (t0 + CH < T) load(t0 + CH, wb, qb, qtb);
        run(t0, wa, qa, qta);
        if (t0 + CH >= T) break;
        if (t0 + 2 * CH < T) load(t0 + 2 * CH, wa, qa, qta);
        run(t0 + CH, wb, qb, qtb);
    }
    __syncwarp();
}

// Per-pair partial results, at the pair's position in the work order:
// [loss sum, V, dL/dw0..w3, dL/db, dL/dgap, dL/dthr]
constexpr int kSoftSlots = 9;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
    return v;
}

__device__ __forceinline__ bool next_pair(int32_t *queue, int64_t n, int lane, int64_t &it) {
    int64_t x = 0;
    if (lane == 0) x = atomicAdd(queue, 1);
    it = __shfl_sync(kFull, x, 0);
    return it < n;
}

__device__ __forceinline__ void ctx_for_pair(SoftCtx &C, const PairGeom &g, int64_t k, const DevCorpus &src,
                                             const DevCorpus &tgt, const uint8_t *counts, const uint8_t *gold,
                                             const SoftScratch &W) {
    C.N = g.n;
    C.M = g.m;
    C.nstrips = (g.n + 31) >> 5;
    C.ssent = src.sent + src.doc[k];
    C.tsent = tgt.sent + tgt.doc[k];
    C.cnt = reinterpret_cast<const uchar2 *>(counts) + g.cell_off;
    C.gold = gold + g.cell_off;
    C.E = W.E + g.cell_off;
    C.U = W.U + g.cell_off;
}

__device__ __forceinline__ SoftCtx make_ctx(const DevParams &P, const SoftArgs &A) {
    SoftCtx C;
    C.lane = threadIdx.x & 31;
    C.P = P;
    C.K = sim_const(P);
    C.two_p = __fadd_rn(P.gap, P.gap);
    C.gamma = A.gamma;
    C.kexp = kLog2e / A.gamma;
    C.kln = A.gamma * kLn2;
    C.thr = P.thr;
    C.ktau = kLog2e / A.tau;
    C.eps = A.eps;
    C.inv_cells = A.inv_cells;
    return C;
}

struct SoftSmem {
    float sv[2][32][32];
    float ub[2][32][32];
    SimCol colv[32];
};

__device__ __forceinline__ void bind_smem(SoftCtx &C, unsigned char *raw) {
    SoftSmem &sm = reinterpret_cast<SoftSmem *>(raw)[threadIdx.x >> 5];
    C.svb = sm.sv;
    C.ub = sm.ub;
    C.colv = sm.colv;
}

// Sweep 1 (value) + sweep 2 (adjoint): V(N,M) and E for every cell.
__global__ void __launch_bounds__(32 * kSoftWarps)
soft_forward_kernel(DevCorpus src, DevCorpus tgt, const PairGeom *__restrict__ geom, const int32_t *__restrict__ order,
                    int64_t n_pairs, DevParams P, SoftArgs A, const uint8_t *__restrict__ counts,
                    const uint8_t *__restrict__ gold, SoftScratch W) {
    extern __shared__ __align__(16) unsigned char soft_smem[];
    SoftCtx C = make_ctx(P, A);
    bind_smem(C, soft_smem);
    const int lane = C.lane;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    float *sbuf = W.sbuf + gw * W.sbuf_stride;
    int64_t it;
    while (next_pair(W.queue, n_pairs, lane, it)) {
        const int32_t k = order[it];
        const PairGeom g = geom[k];
        ctx_for_pair(C, g, k, src, tgt, counts, gold, W);
        if (C.N > 0 && C.M > 0) {
            float *ckv = W.ckv + g.soft_off;
            float *vlast = ckv + (int64_t)(C.nstrips - 1) * C.M;  // the last strip writes no checkpoint
            for (int s = 0; s < C.nstrips; ++s)
                soft_fwd_strip<false, false>(C, s, s > 0 ? ckv + (int64_t)(s - 1) * C.M : nullptr, nullptr,
                                             s + 1 < C.nstrips ? ckv + (int64_t)s * C.M : nullptr, nullptr, sbuf,
                                             s + 1 == C.nstrips ? vlast : nullptr);
            float *qrow = W.qrow + g.soft_off;
            for (int s = C.nstrips - 1; s >= 0; --s) {
                soft_fwd_strip<false, true>(C, s, s > 0 ? ckv + (int64_t)(s - 1) * C.M : nullptr, nullptr, nullptr,
                                            nullptr, sbuf, nullptr);
                soft_rev_strip<false>(C, s, sbuf, qrow, nullptr, 0.0f);
            }
        }
    }
}

// Sweep 3 (value + tangent, checkpoints) + sweep 4 (adjoint and its tangent):
// H u for every cell, written over u.
__global__ void __launch_bounds__(32 * kSoftWarps)
soft_backward_kernel(DevCorpus src, DevCorpus tgt, const PairGeom *__restrict__ geom, const int32_t *__restrict__ order,
                     int64_t n_pairs, DevParams P, SoftArgs A, const uint8_t *__restrict__ counts,
                     const uint8_t *__restrict__ gold, SoftScratch W) {
    extern __shared__ __align__(16) unsigned char soft_smem[];
    SoftCtx C = make_ctx(P, A);
    bind_smem(C, soft_smem);
    const int lane = C.lane;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    float *sbuf = W.sbuf + gw * W.sbuf_stride;
    const float rgamma = 1.0f / A.gamma;
    int64_t it;
    while (next_pair(W.queue, n_pairs, lane, it)) {
        const int32_t k = order[it];
        const PairGeom g = geom[k];
        ctx_for_pair(C, g, k, src, tgt, counts, gold, W);
        if (C.N > 0 && C.M > 0) {
            float *ckv = W.ckv + g.soft_off;
            float *ckt = W.ckt + g.soft_off;
            float *qrow = W.qrow + g.soft_off;
            float *qtrow = W.qtrow + g.soft_off;
            for (int s = 0; s + 1 < C.nstrips; ++s)
                soft_fwd_strip<true, false>(C, s, s > 0 ? ckv + (int64_t)(s - 1) * C.M : nullptr,
                                            s > 0 ? ckt + (int64_t)(s - 1) * C.M : nullptr, ckv + (int64_t)s * C.M,
                                            ckt + (int64_t)s * C.M, sbuf, nullptr);
            for (int s = C.nstrips - 1; s >= 0; --s) {
                soft_fwd_strip<true, true>(C, s, s > 0 ? ckv + (int64_t)(s - 1) * C.M : nullptr,
                                           s > 0 ? ckt + (int64_t)(s - 1) * C.M : nullptr, nullptr, nullptr, sbuf,
                                           nullptr);
                soft_rev_strip<true>(C, s, sbuf, qrow, qtrow, rgamma);
            }
        }
    }
}

// Per-cell work of the loss: gate, clamped P and BCE (summed per pair), or
// (WANT_U) the tangent direction u = dL/dE of the backward.  One block per
// listed pair.
template <bool WANT_U>
__global__ void __launch_bounds__(256)
soft_loss_kernel(DevCorpus src, DevCorpus tgt, const PairGeom *__restrict__ geom, const int32_t *__restrict__ order,
                 int64_t n_pairs, DevParams P, SoftArgs A, const uint8_t *__restrict__ counts,
                 const uint8_t *__restrict__ gold, SoftScratch W) {
    __shared__ double red[256];
    __shared__ double vred[256];
    SoftCtx C = make_ctx(P, A);
    for (int64_t it = blockIdx.x; it < n_pairs; it += gridDim.x) {
        const int32_t k = order[it];
        const PairGeom g = geom[k];
        const int64_t sb = src.doc[k], tb = tgt.doc[k];
        const int64_t cells = (int64_t)g.n * g.m;
        double acc = 0.0;
        for (int64_t c = threadIdx.x; c < cells; c += blockDim.x) {
            const int i = (int)(c / g.m), j = (int)(c - (int64_t)i * g.m);
            const uchar2 q = reinterpret_cast<const uchar2 *>(counts)[g.cell_off + c];
            const float sv = similarity(q.x, q.y, sim_row((int)(src.sent[sb + i + 1] - src.sent[sb + i]), P),
                                        sim_col((int)(tgt.sent[tb + j + 1] - tgt.sent[tb + j]), P), C.K);
            float G, bce;
            const float lp = cell_dldp(W.E[g.cell_off + c], sv, gold[g.cell_off + c], C, G, WANT_U ? nullptr : &bce);
            if (WANT_U)
                W.U[g.cell_off + c] = __fmul_rn(lp, G);
            else
                acc += (double)bce;
        }
        if (WANT_U) continue;
        // V(N,M) = -N p + sum_j (DOWN output of row N-1 at column j + p)
        double vs = 0.0;
        if (g.n > 0 && g.m > 0) {
            const float *vlast = W.ckv + g.soft_off + (int64_t)((g.n + 31) / 32 - 1) * g.m;
            for (int j = threadIdx.x; j < g.m; j += blockDim.x) vs += (double)vlast[j] + (double)P.gap;
        }
        red[threadIdx.x] = acc;
        vred[threadIdx.x] = vs;
        __syncthreads();
        for (int off = 128; off > 0; off >>= 1) {
            if ((int)threadIdx.x < off) {
                red[threadIdx.x] += red[threadIdx.x + off];
                vred[threadIdx.x] += vred[threadIdx.x + off];
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            W.partial[it * kSoftSlots + 0] = red[0];
            W.partial[it * kSoftSlots + 1] = (g.n > 0 && g.m > 0) ? vred[0] - (double)P.gap * (double)g.n
                                                                  : -(double)P.gap * (double)(g.n + g.m);
        }
        __syncthreads();
    }
}

// Per-cell chain rule: dL/ds = H u + dL/dP E dG/ds, then to w, b (through
// s(1-s) f), gap (2 H u) and thr (-dL/dP E dG/ds).  One block per listed pair.
__global__ void __launch_bounds__(256)
soft_chain_kernel(DevCorpus src, DevCorpus tgt, const PairGeom *__restrict__ geom, const int32_t *__restrict__ order,
                  int64_t n_pairs, DevParams P, SoftArgs A, const uint8_t *__restrict__ counts,
                  const uint8_t *__restrict__ gold, SoftScratch W, float *__restrict__ hvp) {
    __shared__ double red[7][256];
    SoftCtx C = make_ctx(P, A);
    for (int64_t it = blockIdx.x; it < n_pairs; it += gridDim.x) {
        const int32_t k = order[it];
        const PairGeom g = geom[k];
        const int64_t sb = src.doc[k], tb = tgt.doc[k];
        const int64_t cells = (int64_t)g.n * g.m;
        double gr[7] = {0, 0, 0, 0, 0, 0, 0};
        for (int64_t c = threadIdx.x; c < cells; c += blockDim.x) {
            const int i = (int)(c / g.m), j = (int)(c - (int64_t)i * g.m);
            const int ls = (int)(src.sent[sb + i + 1] - src.sent[sb + i]);
            const int lt = (int)(tgt.sent[tb + j + 1] - tgt.sent[tb + j]);
            const uchar2 q = reinterpret_cast<const uchar2 *>(counts)[g.cell_off + c];
            const float sv = similarity(q.x, q.y, sim_row(ls, P), sim_col(lt, P), C.K);
            const float Es = W.E[g.cell_off + c];
            const float Hu = W.U[g.cell_off + c];
            if (hvp) hvp[g.cell_off + c] = Hu;
            float G;
            const float lp = cell_dldp(Es, sv, gold[g.cell_off + c], C, G, nullptr);
            const float gg = __fmul_rn(__fmul_rn(G, __fsub_rn(1.0f, G)), C.ktau * kLn2);
            const float direct = __fmul_rn(__fmul_rn(lp, Es), gg);  // dL/ds through the gate
            const float dlds = __fadd_rn(Hu, direct);
            const float dz = __fmul_rn(dlds, __fmul_rn(sv, __fsub_rn(1.0f, sv)));
            float f[4];
            features(q.x, q.y, ls, lt, f);
#pragma unroll
            for (int q4 = 0; q4 < 4; ++q4) gr[q4] += (double)dz * (double)f[q4];
            gr[4] += (double)dz;
            gr[5] += 2.0 * (double)Hu;
            gr[6] -= (double)direct;
        }
#pragma unroll
        for (int q7 = 0; q7 < 7; ++q7) red[q7][threadIdx.x] = gr[q7];
        __syncthreads();
        for (int off = 128; off > 0; off >>= 1) {
            if ((int)threadIdx.x < off)
#pragma unroll
                for (int q7 = 0; q7 < 7; ++q7) red[q7][threadIdx.x] += red[q7][threadIdx.x + off];
            __syncthreads();
        }
        if (threadIdx.x < 7) W.partial[it * kSoftSlots + 2 + threadIdx.x] = red[threadIdx.x][0];
        __syncthreads();
    }
}

// Fixed-order reduction of the per-pair partials (one block).
__global__ void __launch_bounds__(256)
soft_reduce_kernel(const double *__restrict__ partial, int64_t n_pairs, int first, int count, float scale,
                   float *__restrict__ out) {
    __shared__ double red[256];
    for (int q = 0; q < count; ++q) {
        double v = 0.0;
        for (int64_t k = threadIdx.x; k < n_pairs; k += 256) v += partial[k * kSoftSlots + first + q];
        red[threadIdx.x] = v;
        __syncthreads();
        for (int off = 128; off > 0; off >>= 1) {
            if ((int)threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[q] = (float)(red[0] * (double)scale);
        __syncthreads();
    }
}

__global__ void copy_values_kernel(const double *__restrict__ partial, const int32_t *__restrict__ order,
                                   int64_t n_pairs, float *__restrict__ value) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n_pairs; x += stride)
        value[order[x]] = (float)partial[x * kSoftSlots + 1];
}

int soft_grid(int n_sms) { return n_sms * 3; }

}  // namespace

int64_t soft_warps(int n_sms) { return (int64_t)soft_grid(n_sms) * kSoftWarps; }

static cudaError_t set_soft_smem(const void *kern) {
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(SoftSmem) * kSoftWarps));
}

cudaError_t launch_soft_forward(const DevCorpus &src, const DevCorpus &tgt, const PairGeom *geom,
                                const int32_t *order, int64_t n_pairs, const DevParams &P, const SoftArgs &A,
                                const uint8_t *counts, const uint8_t *gold, const SoftScratch &W, float *loss,
                                float *value, int n_sms, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(W.queue, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    if (n_pairs > 0) {
        e = set_soft_smem((const void *)soft_forward_kernel);
        if (e != cudaSuccess) return e;
        soft_forward_kernel<<<soft_grid(n_sms), 32 * kSoftWarps, sizeof(SoftSmem) * kSoftWarps, st>>>(
            src, tgt, geom, order, n_pairs, P, A, counts, gold, W);
        const int64_t nb = n_pairs < (int64_t)n_sms * 16 ? n_pairs : (int64_t)n_sms * 16;
        soft_loss_kernel<false><<<(unsigned)nb, 256, 0, st>>>(src, tgt, geom, order, n_pairs, P, A, counts, gold, W);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    soft_reduce_kernel<<<1, 256, 0, st>>>(W.partial, n_pairs, 0, 1, A.inv_cells, loss);
    if (value && n_pairs > 0)
        copy_values_kernel<<<(unsigned)((n_pairs + 255) / 256), 256, 0, st>>>(W.partial, order, n_pairs, value);
    return cudaGetLastError();
}

cudaError_t launch_soft_backward(const DevCorpus &src, const DevCorpus &tgt, const PairGeom *geom,
                                 const int32_t *order, int64_t n_pairs, const DevParams &P, const SoftArgs &A,
                                 const uint8_t *counts, const uint8_t *gold, const SoftScratch &W, float dloss,
                                 float *grad, float *hvp, int n_sms, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(W.queue, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    if (n_pairs > 0) {
        e = set_soft_smem((const void *)soft_backward_kernel);
        if (e != cudaSuccess) return e;
        const int64_t nbu = n_pairs < (int64_t)n_sms * 16 ? n_pairs : (int64_t)n_sms * 16;
        soft_loss_kernel<true><<<(unsigned)nbu, 256, 0, st>>>(src, tgt, geom, order, n_pairs, P, A, counts, gold, W);
        soft_backward_kernel<<<soft_grid(n_sms), 32 * kSoftWarps, sizeof(SoftSmem) * kSoftWarps, st>>>(
            src, tgt, geom, order, n_pairs, P, A, counts, gold, W);
        const int64_t nb = n_pairs < (int64_t)n_sms * 16 ? n_pairs : (int64_t)n_sms * 16;
        soft_chain_kernel<<<(unsigned)nb, 256, 0, st>>>(src, tgt, geom, order, n_pairs, P, A, counts, gold, W, hvp);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    soft_reduce_kernel<<<1, 256, 0, st>>>(W.partial, n_pairs, 2, 7, dloss, grad);
    return cudaGetLastError();
}

}  // namespace gbm
