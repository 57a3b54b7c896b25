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
// Memory: per cell only E is kept.  The value sweeps checkpoint the boundary
// row of every 32-row strip and the sweep state at the start of every
// 8-step window; an adjoint sweep recomputes a window's forward steps from
// that state into shared memory and then runs the reverse steps over them.
// One warp owns a pair, or one strip of a pair split over warps.
//
// The sweeps carry the recurrences and the per-cell work: the similarities
// (and, in the backward, u = dL/dE from E and the gold links) of a 32 x 32
// block are computed before its 32 steps into shared memory (rotated, so
// that writes and the skewed reads hit distinct banks); the forward's reverse
// steps add each cell's loss term where E is formed, the backward's reverse
// steps each cell's chain rule to the seven parameters where H u is formed.
// Per strip the sums go, in a fixed order, to the strip's slot of the
// partial sums, so that splitting a pair over warps changes no bit.
#include <algorithm>

#include "kernels.h"

namespace gbm {
namespace {

constexpr int kSoftWarps = 4;
constexpr int kSoftBwdWarps = 2;  // 15 KB of shared memory per warp: six 2-warp CTAs per SM
constexpr int kWin = 8;  // steps of a window of the adjoint sweep's recompute
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
    float *E;              // pair's expected alignment, step-major per strip (soft_e_index)
    float *hvp;            // pair's H u output (backward, may be null)
    SimCol (*colb)[32];    // shared: column constants of the current and previous block [2][col]
    SimRow *rowv;          // shared: constants of the current strip's 32 rows
    float (*svb)[32][32];  // shared: similarities of the current and previous block [2][row][col]
    float (*wb)[kWin][32]; // shared: the recomputed window's per-cell weights [component][step][lane]
    int64_t wait_limit;    // bounded spins of a strip wait
    uint32_t *status;      // timeout bit
    bool failed;           // a wait of the current item gave up
};

// Bounded wait until the progress counter *ctr reaches need.  Every lane
// polls with relaxed loads and, once the whole warp has seen enough,
// acquires, so that its own later loads see what the producer wrote before
// it published (the acquired value is at least the polled one).  After
// wait_limit polls the wait gives up, sets the timeout bit and stops waiting
// for the rest of the item (its results are then invalid, the status says so).
__device__ __forceinline__ void soft_wait(SoftCtx &C, const int32_t *ctr, int need, int &have) {
    if (C.failed || __all_sync(kFull, have >= need)) return;
    for (int64_t it = 0;; ++it) {
        have = ld_relaxed(ctr);
        if (__all_sync(kFull, have >= need)) {
            have = ld_acquire(ctr);  // orders this lane's later loads after the producer's writes
            return;
        }
        if (it >= C.wait_limit) {
            C.failed = true;
            if (C.lane == 0) atomicOr(C.status, kStTimeout);
            return;
        }
        __nanosleep(100);
    }
}

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

// Similarities of block jb of strip s into shared buffer jb & 1 with the
// block's column constants.  Lane = column here: row i of the block is one
// coalesced 64-byte load across the warp (a lane-per-row load would touch 32
// cache lines per instruction), all 32 rows in flight at once; the rows'
// constants come from the warp's shared copy (rowv), the column's from a
// register.  sv[i][lane] for fixed i hits 32 distinct banks.
template <bool TAN>
__device__ __forceinline__ void soft_prep_block(const SoftCtx &C, int s, int jb) {
    const int lane = C.lane;
    const int col = 32 * jb + lane;
    const bool cok = col < C.M;
    const int nr = min(32, C.N - 32 * s);
    const uint16_t *cp = reinterpret_cast<const uint16_t *>(C.cnt) + (int64_t)(32 * s) * C.M + col;
    const int lt = cok ? (int)(C.tsent[col + 1] - C.tsent[col]) : 1;
    uint32_t q[16];
    SimCol *cv = C.colb[jb & 1];
    float(*sv)[32] = C.svb[jb & 1];
#pragma unroll
    for (int i = 0; i < 16; ++i) q[i] = (cok && i < nr) ? (uint32_t)cp[(int64_t)i * C.M] : 0u;
    const SimCol sc = sim_col(lt, C.P);
    __syncwarp();  // the previous readers of buffer jb & 1 are done
    cv[lane] = sc;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint32_t qn[16];
        if (h == 0) {
#pragma unroll
            for (int i = 0; i < 16; ++i) qn[i] = (cok && 16 + i < nr) ? (uint32_t)cp[(int64_t)(16 + i) * C.M] : 0u;
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int row = 16 * h + i;
            sv[row][lane] = (cok && row < nr) ? similarity_q16(q[i], C.rowv[row], sc, C.K) : 0.0f;
        }
        if (h == 0) {
#pragma unroll
            for (int i = 0; i < 16; ++i) q[i] = qn[i];
        }
    }
    __syncwarp();
}

// The inputs of u = dL/dE for the lane's cells of the kWin forward steps
// from t0 (column t0 + k - lane at step t0 + k): E and the gold links,
// loaded a window ahead of their use so that their latency overlaps a
// window of steps.
// E's place in the sweeps' layout: per strip, forward step t = j + lane
// major and lane minor, so that the 32 cells of one step (an anti-diagonal)
// are one 128-byte line for the reverse steps that write them and the
// backward's steps that read them (row-major, each step's cells would lie in
// 32 different lines).  A strip holds 32 (nb + 1) steps, twice its window
// checkpoints.
__host__ __device__ __forceinline__ int64_t soft_e_index(int M, int s, int t, int lane) {
    return (int64_t)s * 2 * soft_ckw_floats(M) + (int64_t)t * 32 + lane;
}

struct UIn {
    float e[kWin];
    uint32_t g;  // bit k: gold link of step k's cell
};
__device__ __forceinline__ void soft_u_inputs(const SoftCtx &C, int s, int t0, UIn &X) {
    const int lane = C.lane;
    const int r = 32 * s + lane;
    const bool rv = r < C.N;
    X.g = 0u;
#pragma unroll
    for (int k = 0; k < kWin; ++k) {
        const int j = t0 + k - lane;
        X.e[k] = 0.0f;
        if (rv && j >= 0 && j < C.M) {
            const int64_t c = (int64_t)r * C.M + j;
            X.e[k] = C.E[soft_e_index(C.M, s, t0 + k, lane)];
            X.g |= (uint32_t)(C.gold[c] != 0) << k;
        }
    }
}

// One cell of the forward recurrence (lane's row, column j): the soft max
// of the three candidates, its weights and the next DOWN / RIGHT differences
// (and, TAN, the tangents along u).  Tangent: with the weights summing to
// one, every difference the sweeps need is a weighted sum of pairwise
// candidate differences, so nothing cancels when one weight is close to 1 (a
// saturated alignment); e.g. u - D' = wu (u - A') + wl (u - B').  cd, cu, cl:
// the coefficients c_k - D' of the weight tangents.
template <bool TAN>
__device__ __forceinline__ void soft_cell(const SoftCtx &C, int lane, int j, float a_up, float at_up, float &b,
                                          float &bt, float &a_down, float &at_down, float &wd, float &wu, float &wl,
                                          float &cd, float &cu, float &cl, float ue = 0.0f, int ug = 0) {
    const int bb = (j >> 5) & 1, c = j & 31;
    const float sv = C.svb[bb][lane][c];
    const float D = soft3(sv, a_up, b, C, wd, wu, wl);
    const float e = __fsub_rn(D, C.two_p);
    const float nb2 = __fsub_rn(e, a_up);
    a_down = __fsub_rn(e, b);
    cd = cu = cl = 0.0f;
    if (TAN) {
        float G;  // u = dL/dE of the cell, from its E, similarity and gold link
        const float uu = __fmul_rn(cell_dldp(ue, sv, ug, C, G, nullptr), G);
        const float dua = __fsub_rn(uu, at_up), dub = __fsub_rn(uu, bt), dab = __fsub_rn(at_up, bt);
        cd = __fmaf_rn(wu, dua, __fmul_rn(wl, dub));
        cu = __fmaf_rn(wl, dab, -__fmul_rn(wd, dua));
        cl = -__fmaf_rn(wd, dub, __fmul_rn(wu, dab));
        at_down = __fmaf_rn(wd, dub, __fmul_rn(wu, dab));  // D' - B'
        bt = __fmaf_rn(wd, dua, -__fmul_rn(wl, dab));      // D' - A'
    }
    b = nb2;
}

// Forward (value) sweep of strip s (rows 32s..32s+31, lane = row, skewed by
// lane).
//   TAN:   also run the tangent along u (needs U of the pair)
// ck*_top: the strip above's checkpoint row (UP candidates of row 32s-1);
// ck*_out: this strip's checkpoint row (written by the last lane), may be null.
// ckw_out: the state of every lane at the start of every kWin-step window
// (b, a_down and, TAN, bt, at_down; 128 floats per window), from which the
// adjoint sweep recomputes the strip a window at a time.
// vlast (may be null): receives the DOWN outputs of row N-1, V(N,j) - V(N,j-1) - p,
// from which V(N,M) is summed in FP64 outside the sweep.
// Split pairs (strips on different warps): wait_top (may be null) counts the
// checkpoint columns the strip above has published, pub (may be null)
// receives this strip's count (lane 31 writes column j at step j + 31, so
// after block jb columns 0..32 jb are out).
template <bool TAN>
__device__ __forceinline__ void soft_fwd_strip(SoftCtx &C, int s, const float *__restrict__ ckv_top,
                                               const float *__restrict__ ckt_top, float *__restrict__ ckv_out,
                                               float *__restrict__ ckt_out, float *__restrict__ ckw_out,
                                               float *__restrict__ vlast, const int32_t *wait_top = nullptr,
                                               int32_t *pub = nullptr) {
    const int lane = C.lane;
    const int r = 32 * s + lane;
    const bool rv = r < C.N;
    C.row = sim_row(rv ? (int)(C.ssent[r + 1] - C.ssent[r]) : 1, C.P);
    __syncwarp();  // the previous strip's last block is prepared
    C.rowv[lane] = C.row;
    const int nb = (C.M + 31) >> 5;
    float b = -C.two_p, a_down = 0.0f;
    float bt = 0.0f, at_down = 0.0f;
    int have = 0;
    UIn Ucur, Unext;  // TAN: inputs of u for the current and the next window
    if (TAN) soft_u_inputs(C, s, 0, Ucur);
    for (int jb = 0; jb <= nb; ++jb) {
        if (jb < nb) soft_prep_block<TAN>(C, s, jb);
        const int colx = 32 * jb + lane;
        const bool top = s > 0 && colx < C.M;
        if (wait_top && 32 * jb < C.M) soft_wait(C, wait_top, min(32 * jb + 32, C.M), have);
        const float hv = top ? __ldcg(ckv_top + colx) : -C.two_p;
        const float htv = (TAN && top) ? __ldcg(ckt_top + colx) : 0.0f;
        for (int wi = 0; wi < 32 / kWin; ++wi) {
        if (TAN) soft_u_inputs(C, s, 32 * jb + kWin * (wi + 1), Unext);
#pragma unroll
        for (int k = 0; k < kWin; ++k) {
            const int u = kWin * wi + k;
            const int t = 32 * jb + u;
            if (ckw_out && k == 0) {
                float *q = ckw_out + (int64_t)(t / kWin) * 128 + lane;
                q[0] = b;
                q[32] = a_down;
                if (TAN) {
                    q[64] = bt;
                    q[96] = at_down;
                }
            }
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
                float wd, wu, wl, cd, cu, cl;
                soft_cell<TAN>(C, lane, j, a_up, at_up, b, bt, a_down, at_down, wd, wu, wl, cd, cu, cl,
                               TAN ? Ucur.e[k] : 0.0f, TAN ? (int)((Ucur.g >> k) & 1u) : 0);
                if (lane == 31 && ckv_out) {
                    __stcg(ckv_out + j, a_down);
                    if (TAN) __stcg(ckt_out + j, at_down);
                }
                if (vlast && r == C.N - 1) __stcg(vlast + j, a_down);
            }
        }
        if (TAN) Ucur = Unext;
        }
        if (pub && lane == 31) st_release(pub, min(32 * jb + 1, C.M));
    }
    __syncwarp();
}

// The adjoint sweep of a strip, a window of kWin anti-diagonals at a time
// from the right end: the window's forward steps are recomputed from the
// state the value sweep saved at its start (same arithmetic, so the same
// weights) into the warp's shared window buffer, then the reverse steps run
// over them.  Reverse: the adjoint Q (E = Q wd) and, with TAN, its tangent Q'
// (H u = Q' wd + Q wd').  Reverse step tr handles the cells of forward step
// t = M + 30 - tr (lane i, column t - i), so that the cell below (lane i+1)
// was done one step earlier; its outflows come up by a shuffle, the strip
// below's through qrow/qtrow (lane 0 writes column j of qrow at step
// M + 30 - j).  Split pairs: wait_below (may be null) counts the reverse steps
// the strip below has published, pub (may be null) receives this strip's.
// Floats of one strip's window checkpoints: 128 per window, the value sweep
// runs 32 (nb + 1) steps.
__device__ __forceinline__ int64_t soft_ckw_strip(int M) {
    static_assert(kWin == 8, "soft_ckw_floats assumes 8-step windows");
    return soft_ckw_floats(M);
}

struct RevState {
    float q_send, dflow, qright, qt_send, dtflow, qtright;
};

// Per-lane sums of the per-cell terms of a strip: the loss (forward) or the
// seven gradient components (backward), in FP32 over one 32-column block,
// then folded into FP64.
struct SoftAcc {
    float f[7];
    double d[7];
    __device__ __forceinline__ void clear() {
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            f[q] = 0.0f;
            d[q] = 0.0;
        }
    }
    template <int NV>
    __device__ __forceinline__ void fold() {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            d[q] += (double)f[q];
            f[q] = 0.0f;
        }
    }
};

template <bool TAN>
__device__ __forceinline__ void soft_fwd_window(SoftCtx &C, int s, int t0, float hv, float htv,
                                                const float *__restrict__ ckw_w, const UIn &U) {
    const int lane = C.lane;
    const bool rv = 32 * s + lane < C.N;
    float b = ckw_w[lane], a_down = ckw_w[32 + lane];
    float bt = TAN ? ckw_w[64 + lane] : 0.0f, at_down = TAN ? ckw_w[96 + lane] : 0.0f;
    const int u0 = t0 & 31;
#pragma unroll
    for (int k = 0; k < kWin; ++k) {
        const int t = t0 + k;
        float a_up = __shfl_up_sync(kFull, a_down, 1);
        float at_up = TAN ? __shfl_up_sync(kFull, at_down, 1) : 0.0f;
        const float h0 = __shfl_sync(kFull, hv, u0 + k);
        const float ht0 = TAN ? __shfl_sync(kFull, htv, u0 + k) : 0.0f;
        if (lane == 0) {
            a_up = h0;
            if (TAN) at_up = ht0;
        }
        const int j = t - lane;
        if (rv && j >= 0 && j < C.M) {
            float wd, wu, wl, cd, cu, cl;
            soft_cell<TAN>(C, lane, j, a_up, at_up, b, bt, a_down, at_down, wd, wu, wl, cd, cu, cl,
                           TAN ? U.e[k] : 0.0f, TAN ? (int)((U.g >> k) & 1u) : 0);
            C.wb[0][k][lane] = wd;
            C.wb[1][k][lane] = wu;
            C.wb[2][k][lane] = wl;
            if (TAN) {
                C.wb[3][k][lane] = cd;
                C.wb[4][k][lane] = cu;
                C.wb[5][k][lane] = cl;
            }
        }
    }
}

// The similarity's features of a cell (count pair in the low bytes of qg):
// ms / ls, mt / lt, 1 - q, q with q = min(ls / lt, lt / ls), through the rows'
// and columns' reciprocals (a rounding more than the IEEE quotients: far
// below the gradient's tolerance).
__device__ __forceinline__ void cell_features(const SoftCtx &C, uint32_t qg, const SimCol &sc, float (&f)[4]) {
    f[0] = __fmul_rn(small_int_float((int)(qg & 0xFFu)), C.row.rlen);
    f[1] = __fmul_rn(small_int_float((int)((qg >> 8) & 0xFFu)), sc.rlen);
    f[3] = fminf(__fmul_rn(C.row.len, sc.rlen), __fmul_rn(sc.len, C.row.rlen));
    f[2] = __fsub_rn(1.0f, f[3]);
}

// The per-cell inputs of a window's cells (forward step t0 + kk, lane's
// column t0 + kk - lane): the count pair and, in the forward, the gold link,
// loaded before the window's forward recompute so that their latency
// overlaps it.
struct CellIn {
    uint32_t qg[kWin];  // count pair (bytes 0, 1) | gold (byte 2)
};
template <bool TAN>
__device__ __forceinline__ void soft_cell_inputs(const SoftCtx &C, int s, int t0, CellIn &X) {
    const int lane = C.lane;
    const int r = 32 * s + lane;
    const bool rv = r < C.N;
#pragma unroll
    for (int kk = 0; kk < kWin; ++kk) {
        const int j = t0 + kk - lane;
        X.qg[kk] = 0u;
        if (rv && j >= 0 && j < C.M) {
            const int64_t c = (int64_t)r * C.M + j;
            const uchar2 q = C.cnt[c];
            X.qg[kk] = (uint32_t)q.x | ((uint32_t)q.y << 8);
            if (!TAN) X.qg[kk] |= (uint32_t)C.gold[c] << 16;
        }
    }
}

template <bool TAN>
__device__ __forceinline__ void soft_rev_window(SoftCtx &C, int s, int t0, RevState &R, SoftAcc &Z, const CellIn &X,
                                                float *qrow, float *qtrow, float rgamma, const int32_t *wait_below,
                                                int32_t *pub, int &have) {
    const int lane = C.lane;
    const int r = 32 * s + lane;
    const bool rv = r < C.N;
    const bool last = s == C.nstrips - 1;
    const int T = C.M + 31;
    const int tr0 = C.M + 30 - (t0 + kWin - 1);  // reverse step of the window's last forward step
    // the inflow from the strip below for the columns lane 31 meets in this
    // window (lane k: reverse step tr0 + k), which the strip below writes at
    // its step tr0 + k + 31
    if (wait_below) soft_wait(C, wait_below, min(tr0 + kWin + 31, T), have);
    const int jl = C.M - 1 - (tr0 + lane);
    const bool in = !last && lane < kWin && jl >= 0 && jl < C.M;
    const float qb = in ? __ldcg(qrow + jl) : 0.0f;
    const float qtb = (TAN && in) ? __ldcg(qtrow + jl) : 0.0f;
#pragma unroll
    for (int k = 0; k < kWin; ++k) {
        const int tr = tr0 + k;
        if (tr < 0) continue;  // forward steps past the strip's last cell
        float from_below = __shfl_down_sync(kFull, R.q_send, 1);
        float from_below_t = TAN ? __shfl_down_sync(kFull, R.qt_send, 1) : 0.0f;
        const float fb = __shfl_sync(kFull, qb, k);
        const float fbt = TAN ? __shfl_sync(kFull, qtb, k) : 0.0f;
        const int j = C.M - 1 - (tr - (31 - lane));
        if (lane == 31) {
            from_below = fb;
            if (TAN) from_below_t = fbt;
        }
        if (rv && j >= 0 && j < C.M) {
            const int kk = kWin - 1 - k;  // the forward step's slot in the window
            const float wd = C.wb[0][kk][lane], wu = C.wb[1][kk][lane], wl = C.wb[2][kk][lane];
            float Q = __fadd_rn(from_below, R.qright);
            float Qt = TAN ? __fadd_rn(from_below_t, R.qtright) : 0.0f;
            if (r == C.N - 1 && j == C.M - 1) {
                Q = 1.0f;
                Qt = 0.0f;
            }
            const float Ec = __fmul_rn(Q, wd);
            R.qright = __fmul_rn(Q, wl);
            R.q_send = __fadd_rn(__fmul_rn(Q, wu), R.dflow);
            R.dflow = Ec;
            const int64_t c = (int64_t)r * C.M + j;
            const float sv = C.svb[(j >> 5) & 1][lane][j & 31];
            if (TAN) {
                // weight tangents w_k' = w_k (c_k - D') / gamma
                const float wdt = __fmul_rn(__fmul_rn(wd, C.wb[3][kk][lane]), rgamma);
                const float wut = __fmul_rn(__fmul_rn(wu, C.wb[4][kk][lane]), rgamma);
                const float wlt = __fmul_rn(__fmul_rn(wl, C.wb[5][kk][lane]), rgamma);
                const float Hu = __fmaf_rn(Q, wdt, __fmul_rn(Qt, wd));
                R.qtright = __fmaf_rn(Q, wlt, __fmul_rn(Qt, wl));
                R.qt_send = __fadd_rn(__fmaf_rn(Q, wut, __fmul_rn(Qt, wu)), R.dtflow);
                R.dtflow = Hu;
                if (C.hvp) C.hvp[c] = Hu;
                if (lane == 0) __stcg(qtrow + j, R.qt_send);
                // the cell's chain rule, H u part: dL/ds gets H u, then to w
                // (through s(1-s) and the features), b and gap (2 H u); the
                // part through the gate (dL/dP E dG/ds) is summed by the forward
                const float dz = __fmul_rn(Hu, __fmul_rn(sv, __fsub_rn(1.0f, sv)));
                float f[4];
                cell_features(C, X.qg[kk], C.colb[(j >> 5) & 1][j & 31], f);
#pragma unroll
                for (int q4 = 0; q4 < 4; ++q4) Z.f[q4] = __fmaf_rn(dz, f[q4], Z.f[q4]);
                Z.f[4] = __fadd_rn(Z.f[4], dz);
                Z.f[5] = __fmaf_rn(2.0f, Hu, Z.f[5]);
            } else {
                C.E[soft_e_index(C.M, s, t0 + kk, lane)] = Ec;
                // the cell's loss term and the part of dL/ds through the gate,
                // dL/dP E dG/ds, to w (through s(1-s) and the features), b
                // and thr
                float G, bce;
                const float lp = cell_dldp(Ec, sv, (int)(X.qg[kk] >> 16), C, G, &bce);
                Z.f[0] = __fadd_rn(Z.f[0], bce);
                const float gg = __fmul_rn(__fmul_rn(G, __fsub_rn(1.0f, G)), C.ktau * kLn2);
                const float direct = __fmul_rn(__fmul_rn(lp, Ec), gg);
                const float dz = __fmul_rn(direct, __fmul_rn(sv, __fsub_rn(1.0f, sv)));
                float f[4];
                cell_features(C, X.qg[kk], C.colb[(j >> 5) & 1][j & 31], f);
#pragma unroll
                for (int q4 = 0; q4 < 4; ++q4) Z.f[1 + q4] = __fmaf_rn(dz, f[q4], Z.f[1 + q4]);
                Z.f[5] = __fadd_rn(Z.f[5], dz);
                Z.f[6] = __fsub_rn(Z.f[6], direct);
            }
            if (lane == 0) __stcg(qrow + j, R.q_send);
        } else {
            R.q_send = R.dflow = R.qright = 0.0f;
            R.qt_send = R.dtflow = R.qtright = 0.0f;
        }
    }
    if (pub && lane == 0) st_release(pub, min(max(tr0 + kWin, 0), T));
}

// The whole adjoint sweep of strip s (after its value sweep saved ckw).
template <bool TAN>
__device__ __forceinline__ void soft_adjoint_strip(SoftCtx &C, int s, const float *__restrict__ ckv_top,
                                                   const float *__restrict__ ckt_top, const float *__restrict__ ckw,
                                                   SoftAcc &Z, float *qrow, float *qtrow, float rgamma,
                                                   const int32_t *wait_below = nullptr, int32_t *pub = nullptr) {
    constexpr int NV = TAN ? 6 : 7;
    const int lane = C.lane;
    const int r = 32 * s + lane;
    const bool rv = r < C.N;
    C.row = sim_row(rv ? (int)(C.ssent[r + 1] - C.ssent[r]) : 1, C.P);
    __syncwarp();  // the previous strip's last block is prepared
    C.rowv[lane] = C.row;
    const int nb = (C.M + 31) >> 5;
    RevState R{0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    int have = 0;
    int cur = -1;  // the block whose windows run (blocks cur and cur - 1 are prepared)
    float hv = 0.0f, htv = 0.0f;
    UIn Ucur, Unext;  // TAN: inputs of u for the current and the next (left) window
    if (TAN) soft_u_inputs(C, s, ((C.M + 30) / kWin) * kWin, Ucur);
    for (int w = (C.M + 30) / kWin; w >= 0; --w) {
        const int t0 = w * kWin, jb = t0 >> 5;
        if (jb != cur) {
            Z.fold<NV>();
            // windows of block jb read blocks jb and jb - 1; going left, block jb
            // is ready from block jb + 1's windows except at the start
            if (cur < 0 && jb < nb) soft_prep_block<TAN>(C, s, jb);
            if (jb >= 1) soft_prep_block<TAN>(C, s, jb - 1);
            cur = jb;
            const int colx = 32 * jb + lane;
            const bool top = s > 0 && colx < C.M;
            hv = top ? __ldcg(ckv_top + colx) : -C.two_p;
            htv = (TAN && top) ? __ldcg(ckt_top + colx) : 0.0f;
        }
        if (TAN && w > 0) soft_u_inputs(C, s, t0 - kWin, Unext);
        CellIn X;
        soft_cell_inputs<TAN>(C, s, t0, X);
        soft_fwd_window<TAN>(C, s, t0, hv, htv, ckw + (int64_t)w * 128, Ucur);
        __syncwarp();
        soft_rev_window<TAN>(C, s, t0, R, Z, X, qrow, qtrow, rgamma, wait_below, pub, have);
        __syncwarp();
        if (TAN) Ucur = Unext;
    }
    Z.fold<NV>();
}

// The strip's sums over the warp (FP64 butterflies, a fixed order) into its
// slot of the partial sums.  Forward: the loss at slot[0], the gate parts of
// the gradient (w0..w3, b, thr) at slot[8 + q]; backward: the H u parts
// (w0..w3, b, gap) at slot[1 + q].
template <bool TAN>
__device__ __forceinline__ void soft_store_strip(const SoftAcc &Z, double *slot, int lane) {
    constexpr int kSlot[2][7] = {{0, 8, 9, 10, 11, 12, 14}, {1, 2, 3, 4, 5, 6, 7}};
#pragma unroll
    for (int q = 0; q < (TAN ? 6 : 7); ++q) {
        double v = Z.d[q];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
        if (lane == 0) slot[kSlot[TAN][q]] = v;
    }
    if (lane == 0) slot[TAN ? 7 : 13] = 0.0;  // no H u part of thr, no gate part of gap
}

__device__ __forceinline__ bool next_item(int32_t *queue, int32_t n, int lane, int32_t &it) {
    int32_t x = 0;
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
    C.E = W.E + 2 * g.ckw_off;
    C.hvp = nullptr;
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
    C.wait_limit = A.wait_limit;
    C.status = A.status;
    C.failed = false;
    return C;
}

// Per-warp shared memory of the sweep kernels (the value sweep of the
// forward needs no u).
struct SoftSmemFwd {
    float sv[2][32][32];
    float wb[3][kWin][32];
    SimCol colv[2][32];
    SimRow rowv[32];
};
struct SoftSmemBwd {
    float sv[2][32][32];
    float wb[6][kWin][32];
    SimCol colv[2][32];
    SimRow rowv[32];
};

template <bool TAN>
__device__ __forceinline__ void bind_smem(SoftCtx &C, unsigned char *raw) {
    if (TAN) {
        SoftSmemBwd &sm = reinterpret_cast<SoftSmemBwd *>(raw)[threadIdx.x >> 5];
        C.svb = sm.sv;
        C.wb = sm.wb;
        C.colb = sm.colv;
        C.rowv = sm.rowv;
    } else {
        SoftSmemFwd &sm = reinterpret_cast<SoftSmemFwd *>(raw)[threadIdx.x >> 5];
        C.svb = sm.sv;
        C.wb = sm.wb;
        C.colb = sm.colv;
        C.rowv = sm.rowv;
    }
}

// Sweep 1 (value) + sweep 2 (adjoint): V(N,M) and E for every cell.  A
// whole pair runs both sweeps strip by strip on one warp; a split pair's
// strips run on different warps, the value sweep top-down (kind 1) and the
// recompute + adjoint sweep bottom-up (kind 2), each strip a little behind
// its neighbour.  Every wait is on an item listed (so dequeued) earlier.
__global__ void __launch_bounds__(32 * kSoftWarps, 4)
soft_forward_kernel(DevCorpus src, DevCorpus tgt, const PairGeom *__restrict__ geom, const int32_t *__restrict__ order,
                    DevParams P, SoftArgs A, const uint8_t *__restrict__ counts, const uint8_t *__restrict__ gold,
                    SoftScratch W) {
    extern __shared__ __align__(16) unsigned char soft_smem[];
    SoftCtx C = make_ctx(P, A);
    bind_smem<false>(C, soft_smem);
    const int lane = C.lane;
    const int32_t n_items = W.queue[1];
    int32_t it;
    while (next_item(W.queue, n_items, lane, it)) {
        const SoftItem I = W.items[it];
        const int32_t k = order[I.pos];
        const PairGeom g = geom[k];
        ctx_for_pair(C, g, k, src, tgt, counts, gold, W);
        C.failed = false;
        if (C.N <= 0 || C.M <= 0) continue;
        const int S = C.nstrips;
        float *ckv = W.ckv + g.soft_off;
        float *vlast = ckv + (int64_t)(S - 1) * C.M;  // the last strip writes no checkpoint
        float *qrow = W.qrow + g.soft_off;
        auto top = [&](int s) { return s > 0 ? ckv + (int64_t)(s - 1) * C.M : nullptr; };
        auto ckw = [&](int s) { return W.ckw + g.ckw_off + (int64_t)s * soft_ckw_strip(C.M); };
        if (I.kind == 0) {
            for (int s = 0; s < S; ++s)
                soft_fwd_strip<false>(C, s, top(s), nullptr, s + 1 < S ? ckv + (int64_t)s * C.M : nullptr, nullptr,
                                      ckw(s), s + 1 == S ? vlast : nullptr);
            for (int s = S - 1; s >= 0; --s) {
                SoftAcc Z;
                Z.clear();
                soft_adjoint_strip<false>(C, s, top(s), nullptr, ckw(s), Z, qrow, nullptr, 0.0f);
                soft_store_strip<false>(Z, W.partial + (int64_t)(I.slot + s) * kSoftSlots, lane);
            }
        } else {
            const int s = I.strip;
            int32_t *p1 = W.prog1 + I.ctr, *p2 = W.prog2 + I.ctr;
            if (I.kind == 1) {
                soft_fwd_strip<false>(C, s, top(s), nullptr, s + 1 < S ? ckv + (int64_t)s * C.M : nullptr, nullptr,
                                      ckw(s), s + 1 == S ? vlast : nullptr, s > 0 ? p1 + s - 1 : nullptr,
                                      (int64_t)I.ctr + s == A.skip_ctr ? nullptr : p1 + s);
            } else {
                int have = 0;  // this strip's value sweep (and so the one above) complete
                soft_wait(C, p1 + s, C.M, have);
                SoftAcc Z;
                Z.clear();
                soft_adjoint_strip<false>(C, s, top(s), nullptr, ckw(s), Z, qrow, nullptr, 0.0f,
                                          s + 1 < S ? p2 + s + 1 : nullptr, p2 + s);
                soft_store_strip<false>(Z, W.partial + (int64_t)(I.slot + s) * kSoftSlots, lane);
            }
        }
    }
}

// Sweep 3 (value + tangent, checkpoints) + sweep 4 (adjoint and its tangent):
// H u for every cell (to the optional output) and the H u part of the
// gradient.  Same work list as the forward.
__global__ void __launch_bounds__(32 * kSoftBwdWarps, 6)
soft_backward_kernel(DevCorpus src, DevCorpus tgt, const PairGeom *__restrict__ geom, const int32_t *__restrict__ order,
                     DevParams P, SoftArgs A, const uint8_t *__restrict__ counts, const uint8_t *__restrict__ gold,
                     SoftScratch W) {
    extern __shared__ __align__(16) unsigned char soft_smem[];
    SoftCtx C = make_ctx(P, A);
    bind_smem<true>(C, soft_smem);
    const int lane = C.lane;
    const float rgamma = 1.0f / A.gamma;
    const int32_t n_items = W.queue[1];
    int32_t it;
    while (next_item(W.queue, n_items, lane, it)) {
        const SoftItem I = W.items[it];
        const int32_t k = order[I.pos];
        const PairGeom g = geom[k];
        ctx_for_pair(C, g, k, src, tgt, counts, gold, W);
        C.hvp = A.hvp ? A.hvp + g.cell_off : nullptr;
        C.failed = false;
        if (C.N <= 0 || C.M <= 0) continue;
        const int S = C.nstrips;
        float *ckv = W.ckv + g.soft_off;
        float *ckt = W.ckt + g.soft_off;
        float *qrow = W.qrow + g.soft_off;
        float *qtrow = W.qtrow + g.soft_off;
        auto topv = [&](int s) { return s > 0 ? ckv + (int64_t)(s - 1) * C.M : nullptr; };
        auto topt = [&](int s) { return s > 0 ? ckt + (int64_t)(s - 1) * C.M : nullptr; };
        auto ckw = [&](int s) { return W.ckw + g.ckw_off + (int64_t)s * soft_ckw_strip(C.M); };
        if (I.kind == 0) {
            for (int s = 0; s < S; ++s)
                soft_fwd_strip<true>(C, s, topv(s), topt(s), s + 1 < S ? ckv + (int64_t)s * C.M : nullptr,
                                     s + 1 < S ? ckt + (int64_t)s * C.M : nullptr, ckw(s), nullptr);
            for (int s = S - 1; s >= 0; --s) {
                SoftAcc Z;
                Z.clear();
                soft_adjoint_strip<true>(C, s, topv(s), topt(s), ckw(s), Z, qrow, qtrow, rgamma);
                soft_store_strip<true>(Z, W.partial + (int64_t)(I.slot + s) * kSoftSlots, lane);
            }
        } else {
            const int s = I.strip;
            int32_t *p1 = W.prog1 + I.ctr, *p2 = W.prog2 + I.ctr;
            if (I.kind == 1) {
                soft_fwd_strip<true>(C, s, topv(s), topt(s), s + 1 < S ? ckv + (int64_t)s * C.M : nullptr,
                                     s + 1 < S ? ckt + (int64_t)s * C.M : nullptr, ckw(s), nullptr,
                                     s > 0 ? p1 + s - 1 : nullptr,
                                     (int64_t)I.ctr + s == A.skip_ctr ? nullptr : p1 + s);
            } else {
                int have = 0;  // this strip's value sweep (and so the one above) complete
                soft_wait(C, p1 + s, C.M, have);
                SoftAcc Z;
                Z.clear();
                soft_adjoint_strip<true>(C, s, topv(s), topt(s), ckw(s), Z, qrow, qtrow, rgamma,
                                         s + 1 < S ? p2 + s + 1 : nullptr, p2 + s);
                soft_store_strip<true>(Z, W.partial + (int64_t)(I.slot + s) * kSoftSlots, lane);
            }
        }
    }
}

// Exclusive prefix sum over the block (blockDim.x a multiple of 32, at most
// 1024); total receives the block's sum.
__device__ int64_t block_scan(int64_t v, int64_t &total) {
    __shared__ int64_t ws[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int64_t w = lane < nw ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(kFull, w, o);
            if (lane >= o) w += y;
        }
        ws[lane] = w;
    }
    __syncthreads();
    const int64_t base = wid > 0 ? ws[wid - 1] : 0;
    total = ws[nw - 1];
    __syncthreads();
    return base + x - v;
}

// Work lists of one sweep (one block).  A listed pair of S >= 2 strips is
// split when its serial chain S (M + 32) exceeds split_q4 / 4 of the mean
// chain per warp (split = 1; every such pair with split = 2, none with
// split = 0).  List order 1: the value-sweep items of every split pair
// (S per pair, top-down), the whole pairs, then the adjoint items of every
// split pair (S per pair, bottom-up), so that an adjoint strip seldom waits
// for its own value sweep; order 0: each split pair's value-sweep items then
// its adjoint items, the whole pairs last; order 2: value sweeps, adjoints,
// whole pairs.  Every wait is on an item listed earlier.  Every
// listed pair with cells gets S slots of per-strip partial sums, in list
// order.  Zeroes the progress counters and the work counter.
__global__ void __launch_bounds__(1024)
soft_items_kernel(const PairGeom *__restrict__ geom, const int32_t *__restrict__ order, int64_t n_pairs,
                  int64_t n_warps, int split, int split_q4, int list_order, uint32_t *status, SoftScratch W) {
    auto strips = [&](int64_t pos, int32_t &n, int32_t &m) {
        const PairGeom g = geom[order[pos]];
        n = g.n;
        m = g.m;
        return (int64_t)((g.n + 31) >> 5);
    };
    __shared__ unsigned long long longest;  // the longest serial chain of a pair
    if (threadIdx.x == 0) longest = 0ull;
    __syncthreads();
    int64_t tot = 0, chain = 0, mx = 0;
    for (int64_t pos = threadIdx.x; pos < n_pairs; pos += blockDim.x) {
        int32_t n, m;
        const int64_t S = strips(pos, n, m);
        chain += S * (m + 32);
        mx = max(mx, S * (m + 32));
    }
    atomicMax(&longest, (unsigned long long)mx);
    (void)block_scan(chain, tot);  // its barriers also order the atomicMax before the read
    // mode 1: the pairs whose chain passes q4/4 of the mean chain per warp;
    // mode 3: every pair of two or more strips, once one pair's chain passes
    // it (that pair's wavefront then sets the pace, and a whole pair sweeping
    // value and adjoint in series on one warp would trail it), else none
    const int64_t mean_q = tot * split_q4 / (4 * (n_warps > 0 ? n_warps : 1));
    const int64_t thr = split == 2   ? 0
                        : split == 1 ? mean_q
                        : split == 3 ? ((int64_t)longest > mean_q ? 0 : INT64_MAX)
                                     : INT64_MAX;
    auto counts = [&](int64_t pos, int64_t &si, int64_t &sc, int64_t &wi, int64_t &sl) {
        int32_t n, m;
        const int64_t S = strips(pos, n, m);
        const bool sp = S >= 2 && m > 0 && S * (m + 32) > thr;
        si = sp ? 2 * S : 0;
        sc = sp ? S : 0;
        wi = sp ? 0 : 1;
        sl = m > 0 ? S : 0;
    };
    // totals, checked against the workspace
    int64_t a[4] = {0, 0, 0, 0};
    for (int64_t pos = threadIdx.x; pos < n_pairs; pos += blockDim.x) {
        int64_t si, sc, wi, sl;
        counts(pos, si, sc, wi, sl);
        a[0] += si;
        a[1] += sc;
        a[2] += wi;
        a[3] += sl;
    }
    int64_t T[4];
    for (int q = 0; q < 4; ++q) (void)block_scan(a[q], T[q]);
    const bool fits = T[0] + T[2] <= W.items_cap && T[1] <= W.ctr_cap && T[3] <= W.slots_cap;
    if (!fits) {
        if (threadIdx.x == 0) {
            atomicOr(status, kStBadList);
            W.queue[0] = 0;
            W.queue[1] = 0;
            W.queue[2] = 0;
        }
        return;
    }
    int64_t c_si = 0, c_sc = 0, c_wi = 0, c_sl = 0;
    for (int64_t base = 0; base < n_pairs; base += blockDim.x) {
        const int64_t pos = base + threadIdx.x;
        int64_t si = 0, sc = 0, wi = 0, sl = 0;
        if (pos < n_pairs) counts(pos, si, sc, wi, sl);
        int64_t t0, t1, t2, t3;
        const int64_t o_si = c_si + block_scan(si, t0);
        const int64_t o_sc = c_sc + block_scan(sc, t1);
        const int64_t o_wi = c_wi + block_scan(wi, t2);
        const int64_t o_sl = c_sl + block_scan(sl, t3);
        c_si += t0;
        c_sc += t1;
        c_wi += t2;
        c_sl += t3;
        if (pos >= n_pairs) continue;
        // item positions of the list order (T[1] value-sweep items, as many
        // adjoint items, T[2] whole pairs)
        const int64_t b1 = list_order == 0 ? o_si : o_sc;  // first value-sweep item of the pair
        const int64_t b2 = list_order == 0 ? o_si + sc : (list_order == 1 ? T[1] + T[2] + o_sc : T[1] + o_sc);
        const int64_t b0 = list_order == 2 ? 2 * T[1] : T[1];  // first whole pair (T[0] = 2 T[1])
        if (si) {
            const int32_t S = (int32_t)sc;
            for (int32_t s = 0; s < S; ++s) {
                W.items[b1 + s] = SoftItem{(int32_t)pos, s, 1, (int32_t)o_sc, (int32_t)o_sl};
                W.items[b2 + S - 1 - s] = SoftItem{(int32_t)pos, s, 2, (int32_t)o_sc, (int32_t)o_sl};
                W.prog1[o_sc + s] = 0;
                W.prog2[o_sc + s] = 0;
            }
        } else {
            W.items[(list_order == 0 ? T[0] : b0) + o_wi] = SoftItem{(int32_t)pos, 0, 0, 0, (int32_t)o_sl};
        }
    }
    if (threadIdx.x == 0) {
        W.queue[0] = 0;
        W.queue[1] = (int32_t)(T[0] + T[2]);
        W.queue[2] = (int32_t)T[3];
    }
}

// V(N,M) of every listed pair (one warp per pair) from the DOWN outputs of
// its last row, V(N,j) - V(N,j-1) - p (written by the value sweep):
// V(N,M) = -N p + sum_j (output_j + p), lane-strided FP32 partial sums and
// an FP64 butterfly in a fixed order.
__global__ void __launch_bounds__(256)
soft_value_kernel(const PairGeom *__restrict__ geom, const int32_t *__restrict__ order, int64_t n_pairs, DevParams P,
                  SoftScratch W) {
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t x = warp0; x < n_pairs; x += nwarps) {
        const PairGeom g = geom[order[x]];
        if (g.n <= 0 || g.m <= 0) {
            if (lane == 0) W.vpart[x] = -(double)P.gap * (double)(g.n + g.m);
            continue;
        }
        const float *vlast = W.ckv + g.soft_off + (int64_t)((g.n + 31) / 32 - 1) * g.m;
        float acc = 0.0f;
        for (int j = lane; j < g.m; j += 32) acc = __fadd_rn(acc, __fadd_rn(vlast[j], P.gap));
        double v = (double)acc;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
        if (lane == 0) W.vpart[x] = v - (double)P.gap * (double)g.n;
    }
}

// Fixed-order reduction of the per-strip partial sums in two launches:
// block b of kSoftRedBlocks sums the slots [b per, (b + 1) per) (thread t
// the slots t, t + 256, ... of that range, then a tree over the block) into
// red[b]; one block then sums red[0..] in order.  out[q] = scale * the sum of
// partial[first + q] (+ partial[first2 + q] when TWO), q < COUNT.
template <int COUNT, bool TWO>
__global__ void __launch_bounds__(256)
soft_reduce_kernel(const double *__restrict__ partial, const int32_t *__restrict__ queue, int first, int first2,
                   double *__restrict__ red) {
    __shared__ double sh[COUNT][256];
    const int64_t n = queue[2];
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t k0 = (int64_t)blockIdx.x * per, k1 = k0 + per < n ? k0 + per : n;
    double v[COUNT];
#pragma unroll
    for (int q = 0; q < COUNT; ++q) v[q] = 0.0;
    for (int64_t k = k0 + threadIdx.x; k < k1; k += 256) {
        const double *sl = partial + k * kSoftSlots;
#pragma unroll
        for (int q = 0; q < COUNT; ++q) v[q] += TWO ? sl[first + q] + sl[first2 + q] : sl[first + q];
    }
#pragma unroll
    for (int q = 0; q < COUNT; ++q) sh[q][threadIdx.x] = v[q];
    __syncthreads();
    for (int off = 128; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off)
#pragma unroll
            for (int q = 0; q < COUNT; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + off];
        __syncthreads();
    }
    if ((int)threadIdx.x < COUNT) red[(int64_t)blockIdx.x * 8 + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void soft_reduce_final_kernel(const double *__restrict__ red, int count, float scale, float *__restrict__ out) {
    if ((int)threadIdx.x < count) {
        double t = 0.0;
        for (int b = 0; b < kSoftRedBlocks; ++b) t += red[b * 8 + threadIdx.x];
        out[threadIdx.x] = (float)(t * (double)scale);
    }
}

__global__ void copy_values_kernel(const double *__restrict__ vpart, const int32_t *__restrict__ order,
                                   int64_t n_pairs, float *__restrict__ value) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n_pairs; x += stride)
        value[order[x]] = (float)vpart[x];
}

int soft_grid(int n_sms) { return n_sms * 3; }

}  // namespace

int64_t soft_warps(int n_sms) { return (int64_t)soft_grid(n_sms) * kSoftWarps; }

static cudaError_t set_soft_smem(const void *kern, size_t bytes) {
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

static void launch_soft_items(const PairGeom *geom, const int32_t *order, int64_t n_pairs, const SoftArgs &A,
                              const SoftScratch &W, int n_sms, cudaStream_t st) {
    soft_items_kernel<<<1, 1024, 0, st>>>(geom, order, n_pairs, soft_warps(n_sms), A.split, A.split_q4, A.order,
                                          A.status, W);
}

// E of every cell of the plan from the sweeps' layout into the caller's
// row-major cells (one block per pair).
__global__ void __launch_bounds__(256) soft_export_e_kernel(const PairGeom *__restrict__ geom,
                                                            const float *__restrict__ E, float *__restrict__ out) {
    const PairGeom g = geom[blockIdx.x];
    if (g.n <= 0 || g.m <= 0) return;
    const float *Ep = E + 2 * g.ckw_off;
    const int64_t cells = (int64_t)g.n * g.m;
    for (int64_t c = threadIdx.x; c < cells; c += blockDim.x) {
        const int i = (int)(c / g.m), j = (int)(c - (int64_t)i * g.m);
        out[g.cell_off + c] = Ep[soft_e_index(g.m, i >> 5, j + (i & 31), i & 31)];
    }
}

cudaError_t launch_soft_export_e(const PairGeom *geom, int64_t n_pairs, const float *E, float *out, cudaStream_t st) {
    if (n_pairs <= 0) return cudaSuccess;
    soft_export_e_kernel<<<(unsigned)n_pairs, 256, 0, st>>>(geom, E, out);
    return cudaGetLastError();
}

cudaError_t launch_soft_forward(const DevCorpus &src, const DevCorpus &tgt, const PairGeom *geom,
                                const int32_t *order, int64_t n_pairs, const DevParams &P, const SoftArgs &A,
                                const uint8_t *counts, const uint8_t *gold, const SoftScratch &W, float *loss,
                                float *value, int n_sms, cudaStream_t st) {
    launch_soft_items(geom, order, n_pairs, A, W, n_sms, st);
    if (n_pairs > 0) {
        cudaError_t e = set_soft_smem((const void *)soft_forward_kernel, sizeof(SoftSmemFwd) * kSoftWarps);
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, soft_forward_kernel, 32 * kSoftWarps,
                                                          sizeof(SoftSmemFwd) * kSoftWarps);
        if (e != cudaSuccess) return e;
        soft_forward_kernel<<<n_sms * (per_sm > 0 ? per_sm : 1), 32 * kSoftWarps, sizeof(SoftSmemFwd) * kSoftWarps, st>>>(
            src, tgt, geom, order, P, A, counts, gold, W);
        soft_value_kernel<<<(unsigned)std::min<int64_t>((n_pairs + 7) / 8, (int64_t)n_sms * 8), 256, 0, st>>>(
            geom, order, n_pairs, P, W);
    }
    soft_reduce_kernel<1, false><<<kSoftRedBlocks, 256, 0, st>>>(W.partial, W.queue, 0, 0, W.red);
    soft_reduce_final_kernel<<<1, 32, 0, st>>>(W.red, 1, A.inv_cells, loss);
    if (value && n_pairs > 0)
        copy_values_kernel<<<(unsigned)((n_pairs + 255) / 256), 256, 0, st>>>(W.vpart, order, n_pairs, value);
    return cudaGetLastError();
}

cudaError_t launch_soft_backward(const DevCorpus &src, const DevCorpus &tgt, const PairGeom *geom,
                                 const int32_t *order, int64_t n_pairs, const DevParams &P, const SoftArgs &A,
                                 const uint8_t *counts, const uint8_t *gold, const SoftScratch &W, float dloss,
                                 float *grad, float *hvp, int n_sms, cudaStream_t st) {
    launch_soft_items(geom, order, n_pairs, A, W, n_sms, st);
    if (n_pairs > 0) {
        cudaError_t e = set_soft_smem((const void *)soft_backward_kernel, sizeof(SoftSmemBwd) * kSoftBwdWarps);
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, soft_backward_kernel, 32 * kSoftBwdWarps,
                                                          sizeof(SoftSmemBwd) * kSoftBwdWarps);
        if (e != cudaSuccess) return e;
        SoftArgs Ah = A;
        Ah.hvp = hvp;
        soft_backward_kernel<<<n_sms * (per_sm > 0 ? per_sm : 1), 32 * kSoftBwdWarps, sizeof(SoftSmemBwd) * kSoftBwdWarps,
                               st>>>(src, tgt, geom, order, P, Ah, counts, gold, W);
    }
    soft_reduce_kernel<7, true><<<kSoftRedBlocks, 256, 0, st>>>(W.partial, W.queue, 1, 8, W.red);
    soft_reduce_final_kernel<<<1, 32, 0, st>>>(W.red, 7, dloss, grad);
    return cudaGetLastError();
}

}  // namespace gbm
