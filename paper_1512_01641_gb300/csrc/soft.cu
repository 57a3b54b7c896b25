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
// Memory: nothing per cell is kept but E.  The forward sweeps checkpoint the
// boundary row of every 32-row strip; a backward sweep recomputes the strip's
// forward from its checkpoint into a per-warp strip buffer (anti-diagonal
// major, so that both the skewed forward and the reverse-skewed backward read
// and write 128 contiguous bytes per step) and then runs the reverse sweep
// over it.  One warp owns a pair.
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
    const int64_t *ssent, *tsent;
    const uchar2 *cnt;     // pair's counts
    const uint8_t *gold;   // pair's gold links (0/1 per cell)
    float *E;              // pair's expected alignment
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

// Forward sweep of strip s (rows 32s..32s+31, lane = row, skewed by lane).
//   TAN:   also run the tangent along u = dL/dE (needs E of the pair)
//   STORE: write the per-cell quantities the reverse sweep needs into sbuf,
//          anti-diagonal major: sbuf[k][t][lane] for step t, component k
// ck*_top: the strip above's checkpoint row (UP candidates of row 32s-1);
// ck*_out: this strip's checkpoint row (written by the last lane), may be null.
// vsum accumulates V(N,M) + N p in the lane holding row N-1 (FP64).
template <bool TAN, bool STORE>
__device__ __forceinline__ void soft_fwd_strip(const SoftCtx &C, int s, const float *__restrict__ ckv_top,
                                               const float *__restrict__ ckt_top, float *__restrict__ ckv_out,
                                               float *__restrict__ ckt_out, float *__restrict__ sbuf, double &vsum) {
    const int lane = C.lane;
    const int r = 32 * s + lane;
    const bool rv = r < C.N;
    const SimRow row = sim_row(rv ? (int)(C.ssent[r + 1] - C.ssent[r]) : 1, C.P);
    const int64_t plane = (int64_t)(C.M + 31) * 32;
    float b = -C.two_p, a_down = 0.0f;
    float bt = 0.0f, at_down = 0.0f;
    const float p = 0.5f * C.two_p;
    for (int t = 0; t < C.M + 31; ++t) {
        float a_up = __shfl_up_sync(kFull, a_down, 1);
        float at_up = TAN ? __shfl_up_sync(kFull, at_down, 1) : 0.0f;
        if (lane == 0) {
            a_up = (s == 0 || t >= C.M) ? -C.two_p : __ldcg(ckv_top + t);
            if (TAN) at_up = (s == 0 || t >= C.M) ? 0.0f : __ldcg(ckt_top + t);
        }
        const int j = t - lane;
        if (rv && j >= 0 && j < C.M) {
            const float sv = cell_similarity(C, row, r, j);
            float wd, wu, wl;
            const float D = soft3(sv, a_up, b, C, wd, wu, wl);
            const float e = __fsub_rn(D, C.two_p);
            const float nb = __fsub_rn(e, a_up);
            a_down = __fsub_rn(e, b);
            // tangent: with the weights summing to one, every difference the
            // sweeps need is a weighted sum of pairwise candidate differences,
            // so nothing cancels when one weight is close to 1 (a saturated
            // alignment); e.g. u - D' = wu (u - A') + wl (u - B').
            float cd = 0.0f, cu = 0.0f, cl = 0.0f;
            if (TAN) {
                const int64_t c = (int64_t)r * C.M + j;
                float G;
                const float u = __fmul_rn(cell_dldp(C.E[c], sv, C.gold[c], C, G, nullptr), G);
                const float dua = __fsub_rn(u, at_up), dub = __fsub_rn(u, bt), dab = __fsub_rn(at_up, bt);
                cd = __fmaf_rn(wu, dua, __fmul_rn(wl, dub));
                cu = __fmaf_rn(wl, dab, -__fmul_rn(wd, dua));
                cl = -__fmaf_rn(wd, dub, __fmul_rn(wu, dab));
                const float down = __fmaf_rn(wd, dub, __fmul_rn(wu, dab));  // D' - B'
                const float right = __fmaf_rn(wd, dua, -__fmul_rn(wl, dab)); // D' - A'
                at_down = down;
                bt = right;
            }
            b = nb;
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
            if (r == C.N - 1) vsum += (double)a_down + (double)p;
        }
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
                                             float *E) {
    C.N = g.n;
    C.M = g.m;
    C.nstrips = (g.n + 31) >> 5;
    C.ssent = src.sent + src.doc[k];
    C.tsent = tgt.sent + tgt.doc[k];
    C.cnt = reinterpret_cast<const uchar2 *>(counts) + g.cell_off;
    C.gold = gold + g.cell_off;
    C.E = E + g.cell_off;
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

// Sweep 1 (value) + sweep 2 (adjoint): V(N,M), E for every cell, loss sum.
__global__ void __launch_bounds__(32 * kSoftWarps)
soft_forward_kernel(DevCorpus src, DevCorpus tgt, const PairGeom *__restrict__ geom, const int32_t *__restrict__ order,
                    int64_t n_pairs, DevParams P, SoftArgs A, const uint8_t *__restrict__ counts,
                    const uint8_t *__restrict__ gold, SoftScratch W) {
    SoftCtx C = make_ctx(P, A);
    const int lane = C.lane;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    float *sbuf = W.sbuf + gw * W.sbuf_stride;
    int64_t it;
    while (next_pair(W.queue, n_pairs, lane, it)) {
        const int32_t k = order[it];
        const PairGeom g = geom[k];
        ctx_for_pair(C, g, k, src, tgt, counts, gold, W.E);
        double vsum = 0.0, loss = 0.0;
        float *ckv = W.ckv + g.soft_off;
        if (C.N > 0 && C.M > 0) {
            for (int s = 0; s < C.nstrips; ++s)
                soft_fwd_strip<false, false>(C, s, s > 0 ? ckv + (int64_t)(s - 1) * C.M : nullptr, nullptr,
                                             s + 1 < C.nstrips ? ckv + (int64_t)s * C.M : nullptr, nullptr, sbuf, vsum);
            // adjoint, strips bottom to top
            float *qrow = W.qrow + g.soft_off;
            const int64_t plane = (int64_t)(C.M + 31) * 32;
            for (int s = C.nstrips - 1; s >= 0; --s) {
                double dummy = 0.0;
                soft_fwd_strip<false, true>(C, s, s > 0 ? ckv + (int64_t)(s - 1) * C.M : nullptr, nullptr, nullptr,
                                            nullptr, sbuf, dummy);
                const int r = 32 * s + lane;
                const bool rv = r < C.N;
                float q_send = 0.0f, dflow = 0.0f, qright = 0.0f;
                for (int t = 0; t < C.M + 31; ++t) {
                    float from_below = __shfl_down_sync(kFull, q_send, 1);
                    const int j = C.M - 1 - (t - (31 - lane));
                    if (lane == 31) from_below = (s == C.nstrips - 1 || j < 0 || j >= C.M) ? 0.0f : __ldcg(qrow + j);
                    if (rv && j >= 0 && j < C.M) {
                        const float *q = sbuf + (int64_t)(C.M + 30 - t) * 32 + lane;
                        const float wd = q[0], wu = q[plane], wl = q[2 * plane];
                        float Q = __fadd_rn(from_below, qright);
                        if (r == C.N - 1 && j == C.M - 1) Q = 1.0f;
                        const float Ec = __fmul_rn(Q, wd);
                        const int64_t c = (int64_t)r * C.M + j;
                        C.E[c] = Ec;
                        float G, bce;
                        const float sv = cell_similarity(C, sim_row((int)(C.ssent[r + 1] - C.ssent[r]), P), r, j);
                        (void)cell_dldp(Ec, sv, C.gold[c], C, G, &bce);
                        loss += (double)bce;
                        qright = __fmul_rn(Q, wl);
                        q_send = __fadd_rn(__fmul_rn(Q, wu), dflow);
                        dflow = Ec;
                        if (lane == 0) __stcg(qrow + j, q_send);
                    } else {
                        q_send = 0.0f;
                        dflow = 0.0f;
                        qright = 0.0f;
                    }
                }
                __syncwarp();
            }
        }
        vsum = warp_sum(vsum);
        loss = warp_sum(loss);
        if (lane == 0) {
            double *o = W.partial + it * kSoftSlots;
            o[0] = loss;
            o[1] = (C.N > 0 && C.M > 0) ? vsum - (double)P.gap * (double)C.N : -(double)P.gap * (double)(C.N + C.M);
        }
    }
}

// Sweep 3 (value + tangent, checkpoints) + sweep 4 (adjoint + its tangent):
// H u per cell, chained into the seven parameter gradients.
__global__ void __launch_bounds__(32 * kSoftWarps)
soft_backward_kernel(DevCorpus src, DevCorpus tgt, const PairGeom *__restrict__ geom, const int32_t *__restrict__ order,
                     int64_t n_pairs, DevParams P, SoftArgs A, const uint8_t *__restrict__ counts,
                     const uint8_t *__restrict__ gold, SoftScratch W, float *__restrict__ hvp) {
    SoftCtx C = make_ctx(P, A);
    const int lane = C.lane;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    float *sbuf = W.sbuf + gw * W.sbuf_stride;
    const float rgamma = 1.0f / A.gamma;
    int64_t it;
    while (next_pair(W.queue, n_pairs, lane, it)) {
        const int32_t k = order[it];
        const PairGeom g = geom[k];
        ctx_for_pair(C, g, k, src, tgt, counts, gold, W.E);
        double gr[7] = {0, 0, 0, 0, 0, 0, 0};  // w0..w3, b, gap, thr
        if (C.N > 0 && C.M > 0) {
            float *ckv = W.ckv + g.soft_off;
            float *ckt = W.ckt + g.soft_off;
            float *qrow = W.qrow + g.soft_off;
            float *qtrow = W.qtrow + g.soft_off;
            double dummy = 0.0;
            for (int s = 0; s + 1 < C.nstrips; ++s)
                soft_fwd_strip<true, false>(C, s, s > 0 ? ckv + (int64_t)(s - 1) * C.M : nullptr,
                                            s > 0 ? ckt + (int64_t)(s - 1) * C.M : nullptr, ckv + (int64_t)s * C.M,
                                            ckt + (int64_t)s * C.M, sbuf, dummy);
            const int64_t plane = (int64_t)(C.M + 31) * 32;
            for (int s = C.nstrips - 1; s >= 0; --s) {
                soft_fwd_strip<true, true>(C, s, s > 0 ? ckv + (int64_t)(s - 1) * C.M : nullptr,
                                           s > 0 ? ckt + (int64_t)(s - 1) * C.M : nullptr, nullptr, nullptr, sbuf,
                                           dummy);
                const int r = 32 * s + lane;
                const bool rv = r < C.N;
                const SimRow row = sim_row(rv ? (int)(C.ssent[r + 1] - C.ssent[r]) : 1, P);
                const int ls = rv ? (int)(C.ssent[r + 1] - C.ssent[r]) : 1;
                float q_send = 0.0f, dflow = 0.0f, qright = 0.0f;
                float qt_send = 0.0f, dtflow = 0.0f, qtright = 0.0f;
                for (int t = 0; t < C.M + 31; ++t) {
                    float from_below = __shfl_down_sync(kFull, q_send, 1);
                    float from_below_t = __shfl_down_sync(kFull, qt_send, 1);
                    const int j = C.M - 1 - (t - (31 - lane));
                    if (lane == 31) {
                        const bool edge = s == C.nstrips - 1 || j < 0 || j >= C.M;
                        from_below = edge ? 0.0f : __ldcg(qrow + j);
                        from_below_t = edge ? 0.0f : __ldcg(qtrow + j);
                    }
                    if (rv && j >= 0 && j < C.M) {
                        const float *q = sbuf + (int64_t)(C.M + 30 - t) * 32 + lane;
                        const float wd = q[0], wu = q[plane], wl = q[2 * plane];
                        const float cd = q[3 * plane], cu = q[4 * plane], cl = q[5 * plane];
                        float Q = __fadd_rn(from_below, qright);
                        float Qt = __fadd_rn(from_below_t, qtright);
                        if (r == C.N - 1 && j == C.M - 1) {
                            Q = 1.0f;
                            Qt = 0.0f;
                        }
                        // weight tangents w_k' = w_k (c_k - D') / gamma
                        const float wdt = __fmul_rn(__fmul_rn(wd, cd), rgamma);
                        const float wut = __fmul_rn(__fmul_rn(wu, cu), rgamma);
                        const float wlt = __fmul_rn(__fmul_rn(wl, cl), rgamma);
                        const float Ec = __fmul_rn(Q, wd);
                        const float Hu = __fmaf_rn(Q, wdt, __fmul_rn(Qt, wd));
                        qright = __fmul_rn(Q, wl);
                        qtright = __fmaf_rn(Q, wlt, __fmul_rn(Qt, wl));
                        q_send = __fadd_rn(__fmul_rn(Q, wu), dflow);
                        qt_send = __fadd_rn(__fmaf_rn(Q, wut, __fmul_rn(Qt, wu)), dtflow);
                        dflow = Ec;
                        dtflow = Hu;
                        if (lane == 0) {
                            __stcg(qrow + j, q_send);
                            __stcg(qtrow + j, qt_send);
                        }
                        // chain rule to the parameters
                        const int64_t c = (int64_t)r * C.M + j;
                        if (hvp) hvp[g.cell_off + c] = Hu;
                        const uchar2 cn = C.cnt[c];
                        const int lt = (int)(C.tsent[j + 1] - C.tsent[j]);
                        const float sv = similarity(cn.x, cn.y, row, sim_col(lt, P), C.K);
                        const float Es = C.E[c];
                        float G;
                        const float lp = cell_dldp(Es, sv, C.gold[c], C, G, nullptr);
                        const float gg = __fmul_rn(__fmul_rn(G, __fsub_rn(1.0f, G)), C.ktau * kLn2);
                        const float direct = __fmul_rn(__fmul_rn(lp, Es), gg);  // dL/ds through the gate
                        const float dlds = __fadd_rn(Hu, direct);
                        const float dz = __fmul_rn(dlds, __fmul_rn(sv, __fsub_rn(1.0f, sv)));
                        float f[4];
                        features(cn.x, cn.y, ls, lt, f);
#pragma unroll
                        for (int q4 = 0; q4 < 4; ++q4) gr[q4] += (double)dz * (double)f[q4];
                        gr[4] += (double)dz;
                        gr[5] += 2.0 * (double)Hu;
                        gr[6] -= (double)direct;
                    } else {
                        q_send = qt_send = dflow = dtflow = qright = qtright = 0.0f;
                    }
                }
                __syncwarp();
            }
        }
#pragma unroll
        for (int q7 = 0; q7 < 7; ++q7) gr[q7] = warp_sum(gr[q7]);
        if (lane == 0) {
            double *o = W.partial + it * kSoftSlots;
#pragma unroll
            for (int q7 = 0; q7 < 7; ++q7) o[2 + q7] = gr[q7];
        }
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

int soft_grid(int n_sms) { return n_sms * 8; }

}  // namespace

int64_t soft_warps(int n_sms) { return (int64_t)soft_grid(n_sms) * kSoftWarps; }

cudaError_t launch_soft_forward(const DevCorpus &src, const DevCorpus &tgt, const PairGeom *geom,
                                const int32_t *order, int64_t n_pairs, const DevParams &P, const SoftArgs &A,
                                const uint8_t *counts, const uint8_t *gold, const SoftScratch &W, float *loss,
                                float *value, int n_sms, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(W.queue, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    if (n_pairs > 0)
        soft_forward_kernel<<<soft_grid(n_sms), 32 * kSoftWarps, 0, st>>>(src, tgt, geom, order, n_pairs, P, A, counts,
                                                                           gold, W);
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
    if (n_pairs > 0)
        soft_backward_kernel<<<soft_grid(n_sms), 32 * kSoftWarps, 0, st>>>(src, tgt, geom, order, n_pairs, P, A,
                                                                            counts, gold, W, hvp);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    soft_reduce_kernel<<<1, 256, 0, st>>>(W.partial, n_pairs, 2, 7, dloss, grad);
    return cudaGetLastError();
}

}  // namespace gbm
