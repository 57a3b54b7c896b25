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
constexpr int kSoftBwdWarps = 2;  // the backward's 22.5 KB of shared memory per warp: five 2-warp CTAs per SM
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
    float *E;              // pair's expected alignment
    float *U;              // pair's tangent direction u = dL/dE, then H u
    SimCol *colv;          // shared: column constants of the block being prepared
    float (*svb)[32][32];  // shared: similarities of the current and previous block [2][row][col]
    float (*ub)[32][32];   // shared: u of the current and previous block (TAN)
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
                                          float &cd, float &cu, float &cl) {
    const int bb = (j >> 5) & 1, c = j & 31;
    const float sv = C.svb[bb][lane][c];
    const float D = soft3(sv, a_up, b, C, wd, wu, wl);
    const float e = __fsub_rn(D, C.two_p);
    const float nb2 = __fsub_rn(e, a_up);
    a_down = __fsub_rn(e, b);
    cd = cu = cl = 0.0f;
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
    const int nb = (C.M + 31) >> 5;
    float b = -C.two_p, a_down = 0.0f;
    float bt = 0.0f, at_down = 0.0f;
    int have = 0;
    for (int jb = 0; jb <= nb; ++jb) {
        if (jb < nb) soft_prep_block<TAN>(C, r, rv, jb);
        const int colx = 32 * jb + lane;
        const bool top = s > 0 && colx < C.M;
        if (wait_top && 32 * jb < C.M) soft_wait(C, wait_top, min(32 * jb + 32, C.M), have);
        const float hv = top ? __ldcg(ckv_top + colx) : -C.two_p;
        const float htv = (TAN && top) ? __ldcg(ckt_top + colx) : 0.0f;
#pragma unroll 4
        for (int u = 0; u < 32; ++u) {
            const int t = 32 * jb + u;
            if (ckw_out && (u % kWin) == 0) {
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
                soft_cell<TAN>(C, lane, j, a_up, at_up, b, bt, a_down, at_down, wd, wu, wl, cd, cu, cl);
                if (lane == 31 && ckv_out) {
                    __stcg(ckv_out + j, a_down);
                    if (TAN) __stcg(ckt_out + j, at_down);
                }
                if (vlast && r == C.N - 1) __stcg(vlast + j, a_down);
            }
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

template <bool TAN>
__device__ __forceinline__ void soft_fwd_window(SoftCtx &C, int s, int t0, float hv, float htv,
                                                const float *__restrict__ ckw_w) {
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
            soft_cell<TAN>(C, lane, j, a_up, at_up, b, bt, a_down, at_down, wd, wu, wl, cd, cu, cl);
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

template <bool TAN>
__device__ __forceinline__ void soft_rev_window(SoftCtx &C, int s, int t0, RevState &R, float *qrow, float *qtrow,
                                                float rgamma, const int32_t *wait_below, int32_t *pub, int &have) {
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
            if (TAN) {
                // weight tangents w_k' = w_k (c_k - D') / gamma
                const float wdt = __fmul_rn(__fmul_rn(wd, C.wb[3][kk][lane]), rgamma);
                const float wut = __fmul_rn(__fmul_rn(wu, C.wb[4][kk][lane]), rgamma);
                const float wlt = __fmul_rn(__fmul_rn(wl, C.wb[5][kk][lane]), rgamma);
                const float Hu = __fmaf_rn(Q, wdt, __fmul_rn(Qt, wd));
                R.qtright = __fmaf_rn(Q, wlt, __fmul_rn(Qt, wl));
                R.qt_send = __fadd_rn(__fmaf_rn(Q, wut, __fmul_rn(Qt, wu)), R.dtflow);
                R.dtflow = Hu;
                C.U[c] = Hu;
                if (lane == 0) __stcg(qtrow + j, R.qt_send);
            } else {
                C.E[c] = Ec;
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
                                                   float *qrow, float *qtrow, float rgamma,
                                                   const int32_t *wait_below = nullptr, int32_t *pub = nullptr) {
    const int lane = C.lane;
    const int r = 32 * s + lane;
    const bool rv = r < C.N;
    C.row = sim_row(rv ? (int)(C.ssent[r + 1] - C.ssent[r]) : 1, C.P);
    const int nb = (C.M + 31) >> 5;
    RevState R{0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    int have = 0;
    int cur = -1;  // the block whose windows run (blocks cur and cur - 1 are prepared)
    float hv = 0.0f, htv = 0.0f;
    for (int w = (C.M + 30) / kWin; w >= 0; --w) {
        const int t0 = w * kWin, jb = t0 >> 5;
        if (jb != cur) {
            // windows of block jb read blocks jb and jb - 1; going left, block jb
            // is ready from block jb + 1's windows except at the start
            if (cur < 0 && jb < nb) soft_prep_block<TAN>(C, r, rv, jb);
            if (jb >= 1) soft_prep_block<TAN>(C, r, rv, jb - 1);
            cur = jb;
            const int colx = 32 * jb + lane;
            const bool top = s > 0 && colx < C.M;
            hv = top ? __ldcg(ckv_top + colx) : -C.two_p;
            htv = (TAN && top) ? __ldcg(ckt_top + colx) : 0.0f;
        }
        soft_fwd_window<TAN>(C, s, t0, hv, htv, ckw + (int64_t)w * 128);
        __syncwarp();
        soft_rev_window<TAN>(C, s, t0, R, qrow, qtrow, rgamma, wait_below, pub, have);
        __syncwarp();
    }
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
    SimCol colv[32];
};
struct SoftSmemBwd {
    float sv[2][32][32];
    float ub[2][32][32];
    float wb[6][kWin][32];
    SimCol colv[32];
};

template <bool TAN>
__device__ __forceinline__ void bind_smem(SoftCtx &C, unsigned char *raw) {
    if (TAN) {
        SoftSmemBwd &sm = reinterpret_cast<SoftSmemBwd *>(raw)[threadIdx.x >> 5];
        C.svb = sm.sv;
        C.ub = sm.ub;
        C.wb = sm.wb;
        C.colv = sm.colv;
    } else {
        SoftSmemFwd &sm = reinterpret_cast<SoftSmemFwd *>(raw)[threadIdx.x >> 5];
        C.svb = sm.sv;
        C.ub = nullptr;
        C.wb = sm.wb;
        C.colv = sm.colv;
    }
}

// Sweep 1 (value) + sweep 2 (adjoint): V(N,M) and E for every cell.  A
// whole pair runs both sweeps strip by strip on one warp; a split pair's
// strips run on different warps, the value sweep top-down (kind 1) and the
// recompute + adjoint sweep bottom-up (kind 2), each strip a little behind
// its neighbour.  Every wait is on an item listed (so dequeued) earlier.
__global__ void __launch_bounds__(32 * kSoftWarps)
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
            for (int s = S - 1; s >= 0; --s) soft_adjoint_strip<false>(C, s, top(s), nullptr, ckw(s), qrow, nullptr, 0.0f);
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
                soft_adjoint_strip<false>(C, s, top(s), nullptr, ckw(s), qrow, nullptr, 0.0f,
                                          s + 1 < S ? p2 + s + 1 : nullptr, p2 + s);
            }
        }
    }
}

// Sweep 3 (value + tangent, checkpoints) + sweep 4 (adjoint and its tangent):
// H u for every cell, written over u.  Same work list as the forward.
__global__ void __launch_bounds__(32 * kSoftBwdWarps)
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
            for (int s = S - 1; s >= 0; --s)
                soft_adjoint_strip<true>(C, s, topv(s), topt(s), ckw(s), qrow, qtrow, rgamma);
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
                soft_adjoint_strip<true>(C, s, topv(s), topt(s), ckw(s), qrow, qtrow, rgamma,
                                         s + 1 < S ? p2 + s + 1 : nullptr, p2 + s);
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
// split when its serial chain S (M + 32) exceeds the mean chain per warp
// (split = 1; every such pair with split = 2, none with split = 0).  Split
// pairs come first, each as S value-sweep items (top-down) followed by S
// adjoint items (bottom-up), then the whole pairs in list order.  Every
// listed pair also gets ceil(cells / kSoftChunk) (at least one) chunks of
// per-cell work.  Zeroes the progress counters and the work counter.
__global__ void __launch_bounds__(1024)
soft_items_kernel(const PairGeom *__restrict__ geom, const int32_t *__restrict__ order, int64_t n_pairs,
                  int64_t n_warps, int split, uint32_t *status, SoftScratch W) {
    auto strips = [&](int64_t pos, int32_t &n, int32_t &m) {
        const PairGeom g = geom[order[pos]];
        n = g.n;
        m = g.m;
        return (int64_t)((g.n + 31) >> 5);
    };
    int64_t tot = 0, chain = 0;
    for (int64_t pos = threadIdx.x; pos < n_pairs; pos += blockDim.x) {
        int32_t n, m;
        const int64_t S = strips(pos, n, m);
        chain += S * (m + 32);
    }
    (void)block_scan(chain, tot);
    const int64_t thr = split == 2 ? 0 : (split == 1 ? tot / (n_warps > 0 ? n_warps : 1) : INT64_MAX);
    auto counts = [&](int64_t pos, int64_t &si, int64_t &sc, int64_t &wi, int64_t &ch) {
        int32_t n, m;
        const int64_t S = strips(pos, n, m);
        const bool sp = S >= 2 && m > 0 && S * (m + 32) > thr;
        si = sp ? 2 * S : 0;
        sc = sp ? S : 0;
        wi = sp ? 0 : 1;
        const int64_t cells = (int64_t)n * m;
        ch = cells > 0 ? (cells + kSoftChunk - 1) / kSoftChunk : 1;
    };
    // totals, checked against the workspace
    int64_t a[4] = {0, 0, 0, 0};
    for (int64_t pos = threadIdx.x; pos < n_pairs; pos += blockDim.x) {
        int64_t si, sc, wi, ch;
        counts(pos, si, sc, wi, ch);
        a[0] += si;
        a[1] += sc;
        a[2] += wi;
        a[3] += ch;
    }
    int64_t T[4];
    for (int q = 0; q < 4; ++q) (void)block_scan(a[q], T[q]);
    const bool fits = T[0] + T[2] <= W.items_cap && T[1] <= W.ctr_cap && T[3] <= W.chunks_cap;
    if (!fits) {
        if (threadIdx.x == 0) {
            atomicOr(status, kStBadList);
            W.queue[0] = 0;
            W.queue[1] = 0;
            W.queue[2] = 0;
        }
        return;
    }
    int64_t c_si = 0, c_sc = 0, c_wi = 0, c_ch = 0;
    for (int64_t base = 0; base < n_pairs; base += blockDim.x) {
        const int64_t pos = base + threadIdx.x;
        int64_t si = 0, sc = 0, wi = 0, ch = 0;
        if (pos < n_pairs) counts(pos, si, sc, wi, ch);
        int64_t t0, t1, t2, t3;
        const int64_t o_si = c_si + block_scan(si, t0);
        const int64_t o_sc = c_sc + block_scan(sc, t1);
        const int64_t o_wi = c_wi + block_scan(wi, t2);
        const int64_t o_ch = c_ch + block_scan(ch, t3);
        c_si += t0;
        c_sc += t1;
        c_wi += t2;
        c_ch += t3;
        if (pos >= n_pairs) continue;
        if (si) {
            const int32_t S = (int32_t)sc;
            for (int32_t s = 0; s < S; ++s) {
                W.items[o_si + s] = SoftItem{(int32_t)pos, s, 1, (int32_t)o_sc};
                W.items[o_si + 2 * S - 1 - s] = SoftItem{(int32_t)pos, s, 2, (int32_t)o_sc};
                W.prog1[o_sc + s] = 0;
                W.prog2[o_sc + s] = 0;
            }
        } else {
            W.items[T[0] + o_wi] = SoftItem{(int32_t)pos, 0, 0, 0};
        }
        for (int64_t c = 0; c < ch; ++c) W.chunks[o_ch + c] = SoftChunk{(int32_t)pos, 0, c * kSoftChunk};
    }
    if (threadIdx.x == 0) {
        W.queue[0] = 0;
        W.queue[1] = (int32_t)(T[0] + T[2]);
        W.queue[2] = (int32_t)T[3];
    }
}

// Sum over a block of 256 threads in a fixed order: FP32 butterflies within
// the warps (each thread's value is itself an FP32 sum of a few terms), then
// the eight warp sums in warp order in FP64; the total reaches thread 0.
__device__ __forceinline__ double block_sum256(float v, double *ws) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = __fadd_rn(v, __shfl_xor_sync(kFull, v, off));
    __syncthreads();  // the previous use of ws is complete
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = (double)v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < 8; ++w) t += ws[w];
    return t;
}

// NV sums over a block of 256 threads at once, in the same fixed order as
// block_sum256; thread q < NV receives sum q.
template <int NV>
__device__ __forceinline__ double block_sums256(const float (&v)[NV], double (*ws)[8]) {
    float x[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        x[q] = v[q];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) x[q] = __fadd_rn(x[q], __shfl_xor_sync(kFull, x[q], off));
    }
    __syncthreads();  // the previous use of ws is complete
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q) ws[q][threadIdx.x >> 5] = (double)x[q];
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < NV)
        for (int w = 0; w < 8; ++w) t += ws[threadIdx.x][w];
    return t;
}

// Row and column of the cells a thread visits in a chunk (cells c0 + t,
// c0 + t + 256, ... of a pair with M columns): one 32-bit division per thread
// and chunk, then constant steps; the sentence lengths of the current row and
// column are kept (the row changes rarely).
struct CellWalk {
    int i, j, si, sj;  // current cell, step per visit (256 = si M + sj)
    __device__ __forceinline__ CellWalk(int64_t c0, int t, int M) {
        const uint32_t i0 = (uint32_t)(c0 / M), j0 = (uint32_t)(c0 - (int64_t)i0 * M) + (uint32_t)t;
        i = (int)(i0 + j0 / (uint32_t)M);
        j = (int)(j0 % (uint32_t)M);
        si = 256 / M;
        sj = 256 % M;
    }
    __device__ __forceinline__ void next(int M) {
        i += si;
        j += sj;
        if (j >= M) {
            j -= M;
            ++i;
        }
    }
};

// Per-cell work of the loss: gate, clamped P and BCE (summed per chunk), or
// (WANT_U) the tangent direction u = dL/dE of the backward.  One block per
// chunk of kSoftChunk cells; the first chunk of a pair also sums V(N,M).
template <bool WANT_U>
__global__ void __launch_bounds__(256)
soft_loss_kernel(DevCorpus src, DevCorpus tgt, const PairGeom *__restrict__ geom, const int32_t *__restrict__ order,
                 DevParams P, SoftArgs A, const uint8_t *__restrict__ counts, const uint8_t *__restrict__ gold,
                 SoftScratch W) {
    __shared__ double ws[8];
    SoftCtx C = make_ctx(P, A);
    const int32_t n_chunks = W.queue[2];
    for (int32_t x = blockIdx.x; x < n_chunks; x += gridDim.x) {
        const SoftChunk ch = W.chunks[x];
        const int32_t k = order[ch.pos];
        const PairGeom g = geom[k];
        const int64_t sb = src.doc[k], tb = tgt.doc[k];
        const int64_t cells = (int64_t)g.n * g.m;
        const int64_t c1 = ch.c0 + kSoftChunk < cells ? ch.c0 + kSoftChunk : cells;
        float acc = 0.0f;  // at most kSoftChunk / 256 terms per thread
        CellWalk cw(ch.c0, threadIdx.x, g.m > 0 ? g.m : 1);
        int row_i = -1;
        SimRow srow{};
        for (int64_t c = ch.c0 + threadIdx.x; c < c1; c += blockDim.x, cw.next(g.m)) {
            if (cw.i != row_i) {
                row_i = cw.i;
                srow = sim_row((int)(src.sent[sb + row_i + 1] - src.sent[sb + row_i]), P);
            }
            const uchar2 q = __ldg(reinterpret_cast<const uchar2 *>(counts) + g.cell_off + c);
            const float sv = similarity(
                q.x, q.y, srow, sim_col((int)(__ldg(tgt.sent + tb + cw.j + 1) - __ldg(tgt.sent + tb + cw.j)), P), C.K);
            float G, bce;
            const float lp = cell_dldp(__ldg(W.E + g.cell_off + c), sv, __ldg(gold + g.cell_off + c), C, G,
                                       WANT_U ? nullptr : &bce);
            if (WANT_U)
                W.U[g.cell_off + c] = __fmul_rn(lp, G);
            else
                acc = __fadd_rn(acc, bce);
        }
        if (WANT_U) continue;
        // V(N,M) = -N p + sum_j (DOWN output of row N-1 at column j + p)
        float vs = 0.0f;  // at most M / 256 terms per thread
        if (ch.c0 == 0 && g.n > 0 && g.m > 0) {
            const float *vlast = W.ckv + g.soft_off + (int64_t)((g.n + 31) / 32 - 1) * g.m;
            for (int j = threadIdx.x; j < g.m; j += blockDim.x) vs = __fadd_rn(vs, __fadd_rn(vlast[j], P.gap));
        }
        const double lsum = block_sum256(acc, ws);
        const double vsum = ch.c0 == 0 ? block_sum256(vs, ws) : 0.0;
        if (threadIdx.x == 0) {
            W.partial[(int64_t)x * kSoftSlots] = lsum;
            if (ch.c0 == 0)
                W.vpart[ch.pos] = (g.n > 0 && g.m > 0) ? vsum - (double)P.gap * (double)g.n
                                                       : -(double)P.gap * (double)(g.n + g.m);
        }
    }
}

// Per-cell chain rule: dL/ds = H u + dL/dP E dG/ds, then to w, b (through
// s(1-s) f), gap (2 H u) and thr (-dL/dP E dG/ds).  One block per chunk.
__global__ void __launch_bounds__(256)
soft_chain_kernel(DevCorpus src, DevCorpus tgt, const PairGeom *__restrict__ geom, const int32_t *__restrict__ order,
                  DevParams P, SoftArgs A, const uint8_t *__restrict__ counts, const uint8_t *__restrict__ gold,
                  SoftScratch W, float *__restrict__ hvp) {
    __shared__ double ws[7][8];
    SoftCtx C = make_ctx(P, A);
    const int32_t n_chunks = W.queue[2];
    for (int32_t x = blockIdx.x; x < n_chunks; x += gridDim.x) {
        const SoftChunk ch = W.chunks[x];
        const int32_t k = order[ch.pos];
        const PairGeom g = geom[k];
        const int64_t sb = src.doc[k], tb = tgt.doc[k];
        const int64_t cells = (int64_t)g.n * g.m;
        const int64_t c1 = ch.c0 + kSoftChunk < cells ? ch.c0 + kSoftChunk : cells;
        float gr[7] = {0, 0, 0, 0, 0, 0, 0};  // at most kSoftChunk / 256 terms per thread
        CellWalk cw(ch.c0, threadIdx.x, g.m > 0 ? g.m : 1);
        int row_i = -1;
        SimRow srow{};
        for (int64_t c = ch.c0 + threadIdx.x; c < c1; c += blockDim.x, cw.next(g.m)) {
            if (cw.i != row_i) {
                row_i = cw.i;
                srow = sim_row((int)(src.sent[sb + row_i + 1] - src.sent[sb + row_i]), P);
            }
            const SimCol scol = sim_col((int)(__ldg(tgt.sent + tb + cw.j + 1) - __ldg(tgt.sent + tb + cw.j)), P);
            const uchar2 q = __ldg(reinterpret_cast<const uchar2 *>(counts) + g.cell_off + c);
            const float sv = similarity(q.x, q.y, srow, scol, C.K);
            const float Es = __ldg(W.E + g.cell_off + c);
            const float Hu = __ldg(W.U + g.cell_off + c);
            if (hvp) hvp[g.cell_off + c] = Hu;
            float G;
            const float lp = cell_dldp(Es, sv, __ldg(gold + g.cell_off + c), C, G, nullptr);
            const float gg = __fmul_rn(__fmul_rn(G, __fsub_rn(1.0f, G)), C.ktau * kLn2);
            const float direct = __fmul_rn(__fmul_rn(lp, Es), gg);  // dL/ds through the gate
            const float dlds = __fadd_rn(Hu, direct);
            const float dz = __fmul_rn(dlds, __fmul_rn(sv, __fsub_rn(1.0f, sv)));
            // the features through the rows' and columns' reciprocals (a rounding
            // more than the IEEE quotients: far below the gradient's tolerance)
            float f[4];
            f[0] = __fmul_rn(small_int_float(q.x), srow.rlen);
            f[1] = __fmul_rn(small_int_float(q.y), scol.rlen);
            f[3] = fminf(__fmul_rn(srow.len, scol.rlen), __fmul_rn(scol.len, srow.rlen));
            f[2] = __fsub_rn(1.0f, f[3]);
#pragma unroll
            for (int q4 = 0; q4 < 4; ++q4) gr[q4] = __fmaf_rn(dz, f[q4], gr[q4]);
            gr[4] = __fadd_rn(gr[4], dz);
            gr[5] = __fmaf_rn(2.0f, Hu, gr[5]);
            gr[6] = __fsub_rn(gr[6], direct);
        }
        const double t = block_sums256<7>(gr, ws);
        if (threadIdx.x < 7) W.partial[(int64_t)x * kSoftSlots + 1 + threadIdx.x] = t;
    }
}

// Fixed-order reduction of the per-chunk partials (one block).
__global__ void __launch_bounds__(256)
soft_reduce_kernel(const double *__restrict__ partial, const int32_t *__restrict__ queue, int first, int count,
                   float scale, float *__restrict__ out) {
    __shared__ double red[256];
    const int64_t n = queue[2];
    for (int q = 0; q < count; ++q) {
        double v = 0.0;
        for (int64_t k = threadIdx.x; k < n; k += 256) v += partial[k * kSoftSlots + first + q];
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
    soft_items_kernel<<<1, 1024, 0, st>>>(geom, order, n_pairs, soft_warps(n_sms), A.split, A.status, W);
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
        soft_loss_kernel<false><<<n_sms * 8, 256, 0, st>>>(src, tgt, geom, order, P, A, counts, gold, W);
    }
    soft_reduce_kernel<<<1, 256, 0, st>>>(W.partial, W.queue, 0, 1, A.inv_cells, loss);
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
        soft_loss_kernel<true><<<n_sms * 8, 256, 0, st>>>(src, tgt, geom, order, P, A, counts, gold, W);
        soft_backward_kernel<<<n_sms * (per_sm > 0 ? per_sm : 1), 32 * kSoftBwdWarps, sizeof(SoftSmemBwd) * kSoftBwdWarps,
                               st>>>(
            src, tgt, geom, order, P, A, counts, gold, W);
        soft_chain_kernel<<<n_sms * 8, 256, 0, st>>>(src, tgt, geom, order, P, A, counts, gold, W, hvp);
    }
    soft_reduce_kernel<<<1, 256, 0, st>>>(W.partial, W.queue, 1, 7, dloss, grad);
    return cudaGetLastError();
}

}  // namespace gbm
