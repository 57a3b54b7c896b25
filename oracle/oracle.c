/*
 * FP64 CPU oracle for the comparable-corpus miner (Wolk & Marasek,
 * arXiv:1512.01641).  TEST INFRASTRUCTURE ONLY: the product path never links,
 * loads or calls this file.  It is a plain, slow, obviously correct restatement
 * of the definitions, with no blocking, fusion or reordering.
 *
 *   Sentence similarity (Section 4): a classifier output squashed into [0,1]
 *     by a sigmoid of a linear decision value; here the decision value is
 *     w . f + b over four dictionary/length features of the sentence pair.
 *   Needleman-Wunsch alignment (Section 5.1, Figure 1, Eq. 1): S(0,0)=0, first
 *     row and column initialised by the gap penalty, every other cell is the
 *     max of diagonal + similarity, up - penalty, left - penalty, filled from
 *     the top-left to the bottom-right.
 *   Acceptance threshold (Section 4, Section 5.2): after alignment, a pair
 *     whose similarity is below the threshold is excluded.
 *   Tie rule (Figure 4): at an exact tie the traceback prefers UP (source
 *     sentence unmatched), then LEFT (target sentence unmatched), then DIAG.
 *
 * Readings of the paper used here (the paper is silent or garbled on them):
 *   features f = [ms/ls, mt/lt, |ls-lt|/max(ls,lt), min(ls,lt)/max(ls,lt)],
 *     ms = number of source positions with at least one translation present
 *     in the target sentence, mt = number of target positions whose token is a
 *     translation of some source token (positions counted with multiplicity);
 *   borders H(i,0) = -i p, H(0,j) = -j p (global alignment);
 *   the threshold is a post-filter on the optimal path (kept iff s >= thr).
 *
 * Soft alignment (smoothed max, gamma * log-sum-exp of the same three
 * candidates) is not in the paper; it is the differentiable relaxation used for
 * parameter tuning in place of the paper's random search (Section 5.2).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------------- */
/* Features of one sentence pair                                            */
/* ---------------------------------------------------------------------- */

/* Is token t one of tgt[0..lt)? (plain scan) */
static int contains(const int32_t *tgt, int64_t lt, int32_t t) {
    for (int64_t q = 0; q < lt; ++q)
        if (tgt[q] == t) return 1;
    return 0;
}

/* ms, mt for source sentence src[0..ls) and target sentence tgt[0..lt). */
void oracle_counts(const int32_t *src, int64_t ls, const int32_t *tgt, int64_t lt,
                   const int32_t *dict_off, const int32_t *dict_tgt,
                   int32_t *ms_out, int32_t *mt_out) {
    int32_t ms = 0, mt = 0;
    for (int64_t p = 0; p < ls; ++p) {
        int32_t v = src[p];
        int hit = 0;
        for (int32_t e = dict_off[v]; e < dict_off[v + 1]; ++e)
            if (contains(tgt, lt, dict_tgt[e])) hit = 1;
        ms += hit;
    }
    for (int64_t q = 0; q < lt; ++q) {
        int hit = 0;
        for (int64_t p = 0; p < ls; ++p) {
            int32_t v = src[p];
            for (int32_t e = dict_off[v]; e < dict_off[v + 1]; ++e)
                if (dict_tgt[e] == tgt[q]) hit = 1;
        }
        mt += hit;
    }
    *ms_out = ms;
    *mt_out = mt;
}

void oracle_features(int32_t ms, int32_t mt, int64_t ls, int64_t lt, double f[4]) {
    double a = (double)ls, b = (double)lt;
    double mx = a > b ? a : b, mn = a < b ? a : b;
    f[0] = (double)ms / a;
    f[1] = (double)mt / b;
    f[2] = fabs(a - b) / mx;
    f[3] = mn / mx;
}

double oracle_similarity(const double f[4], const double w[4], double bias) {
    double z = bias;
    for (int k = 0; k < 4; ++k) z += w[k] * f[k];
    return 1.0 / (1.0 + exp(-z));
}

/* ---------------------------------------------------------------------- */
/* Hard Needleman-Wunsch on an explicit similarity matrix                    */
/* ---------------------------------------------------------------------- */
enum { MOVE_DIAG = 0, MOVE_UP = 1, MOVE_LEFT = 2 };

/* H is (N+1) x (M+1), row-major; s is N x M row-major, s[(i-1)*M + (j-1)] is
 * the similarity of source sentence i and target sentence j (1-based cells). */
void oracle_nw_fill(int64_t N, int64_t M, const double *s, double p, double *H) {
    int64_t W = M + 1;
    H[0] = 0.0;
    for (int64_t i = 1; i <= N; ++i) H[i * W] = -(double)i * p;
    for (int64_t j = 1; j <= M; ++j) H[j] = -(double)j * p;
    for (int64_t i = 1; i <= N; ++i)
        for (int64_t j = 1; j <= M; ++j) {
            double diag = H[(i - 1) * W + (j - 1)] + s[(i - 1) * M + (j - 1)];
            double up = H[(i - 1) * W + j] - p;
            double left = H[i * W + (j - 1)] - p;
            double best = diag;
            if (up > best) best = up;
            if (left > best) best = left;
            H[i * W + j] = best;
        }
}

/* Walk back from (N,M) to (0,0).  moves[] receives the moves in walk order
 * (from the end); returns the number of moves.  Ties: UP, then LEFT, then DIAG. */
int64_t oracle_nw_traceback(int64_t N, int64_t M, double p, const double *H,
                            int8_t *moves) {
    int64_t W = M + 1, i = N, j = M, n = 0;
    while (i > 0 || j > 0) {
        int8_t mv;
        if (i == 0) mv = MOVE_LEFT;
        else if (j == 0) mv = MOVE_UP;
        else {
            double h = H[i * W + j];
            if (h == H[(i - 1) * W + j] - p) mv = MOVE_UP;
            else if (h == H[i * W + (j - 1)] - p) mv = MOVE_LEFT;
            else mv = MOVE_DIAG;
        }
        moves[n++] = mv;
        if (mv == MOVE_DIAG) { --i; --j; }
        else if (mv == MOVE_UP) --i;
        else --j;
    }
    return n;
}

/* ---------------------------------------------------------------------- */
/* Soft (log-sum-exp) Needleman-Wunsch on an explicit similarity matrix      */
/* ---------------------------------------------------------------------- */
static double lse3(double a, double b, double c, double g) {
    double m = a;
    if (b > m) m = b;
    if (c > m) m = c;
    return m + g * log(exp((a - m) / g) + exp((b - m) / g) + exp((c - m) / g));
}

/* V is (N+1) x (M+1); E is N x M with E = dV(N,M)/ds (the expected alignment);
 * *dVdp receives dV(N,M)/dp.  Q (adjoint of V) is (N+1) x (M+1) scratch. */
void oracle_soft_nw(int64_t N, int64_t M, const double *s, double p, double g,
                    double *V, double *E, double *Q, double *dVdp) {
    int64_t W = M + 1;
    V[0] = 0.0;
    for (int64_t i = 1; i <= N; ++i) V[i * W] = -(double)i * p;
    for (int64_t j = 1; j <= M; ++j) V[j] = -(double)j * p;
    for (int64_t i = 1; i <= N; ++i)
        for (int64_t j = 1; j <= M; ++j)
            V[i * W + j] = lse3(V[(i - 1) * W + (j - 1)] + s[(i - 1) * M + (j - 1)],
                                V[(i - 1) * W + j] - p, V[i * W + (j - 1)] - p, g);
    /* adjoint sweep: Q(i,j) = dV(N,M)/dV(i,j); every node passes its adjoint to
     * its predecessors in proportion to the softmax weight of each edge. */
    for (int64_t k = 0; k < (N + 1) * W; ++k) Q[k] = 0.0;
    Q[N * W + M] = 1.0;
    double dp = 0.0;
    for (int64_t i = N; i >= 0; --i)
        for (int64_t j = M; j >= 0; --j) {
            double q = Q[i * W + j];
            double v = V[i * W + j];
            if (i > 0 && j > 0) {
                double wd = exp((V[(i - 1) * W + (j - 1)] + s[(i - 1) * M + (j - 1)] - v) / g);
                double wu = exp((V[(i - 1) * W + j] - p - v) / g);
                double wl = exp((V[i * W + (j - 1)] - p - v) / g);
                E[(i - 1) * M + (j - 1)] = q * wd;
                Q[(i - 1) * W + (j - 1)] += q * wd;
                Q[(i - 1) * W + j] += q * wu;
                Q[i * W + (j - 1)] += q * wl;
                dp -= q * (wu + wl);
            } else if (i > 0) { /* j == 0: the border is one chain of UP moves */
                Q[(i - 1) * W] += q;
                dp -= q;
            } else if (j > 0) {
                Q[j - 1] += q;
                dp -= q;
            }
        }
    if (dVdp) *dVdp = dp;
}

/* ---------------------------------------------------------------------- */
/* Whole-batch mining, threaded over pairs                                  */
/* ---------------------------------------------------------------------- */
typedef struct {
    int64_t n_pairs;
    const int64_t *s_doc, *s_sent; const int32_t *s_tok;
    const int64_t *t_doc, *t_sent; const int32_t *t_tok;
    const int32_t *d_off, *d_tgt;
    double w[4], bias, gap;
    const int64_t *pairs;   /* which pairs to process (n_pairs of them) */
    const int64_t *out_off; /* per processed pair: offset into the diag arrays */
    double *pair_score;
    int64_t *n_diag;
    int32_t *diag_i, *diag_j;
    double *diag_s;
    int32_t *counts;        /* optional: 2 ints per cell, per processed pair at cell_off */
    double *sim;            /* optional: similarity per cell, per processed pair at cell_off */
    const int64_t *cell_off;
    int64_t next;           /* shared work counter */
    pthread_mutex_t lock;
} mine_job;

static void mine_one(mine_job *J, int64_t idx) {
    int64_t k = J->pairs[idx];
    int64_t sa = J->s_doc[k], N = J->s_doc[k + 1] - sa;
    int64_t ta = J->t_doc[k], M = J->t_doc[k + 1] - ta;
    double *S = (double *)malloc(sizeof(double) * (size_t)(N * M > 0 ? N * M : 1));
    double *H = (double *)malloc(sizeof(double) * (size_t)((N + 1) * (M + 1)));
    int8_t *mv = (int8_t *)malloc((size_t)(N + M + 1));
    for (int64_t i = 0; i < N; ++i) {
        const int32_t *src = J->s_tok + J->s_sent[sa + i];
        int64_t ls = J->s_sent[sa + i + 1] - J->s_sent[sa + i];
        for (int64_t j = 0; j < M; ++j) {
            const int32_t *tgt = J->t_tok + J->t_sent[ta + j];
            int64_t lt = J->t_sent[ta + j + 1] - J->t_sent[ta + j];
            int32_t ms, mt;
            double f[4];
            oracle_counts(src, ls, tgt, lt, J->d_off, J->d_tgt, &ms, &mt);
            if (J->counts) {
                int32_t *c = J->counts + 2 * (J->cell_off[idx] + i * M + j);
                c[0] = ms;
                c[1] = mt;
            }
            oracle_features(ms, mt, ls, lt, f);
            S[i * M + j] = oracle_similarity(f, J->w, J->bias);
            if (J->sim) J->sim[J->cell_off[idx] + i * M + j] = S[i * M + j];
        }
    }
    oracle_nw_fill(N, M, S, J->gap, H);
    int64_t n = oracle_nw_traceback(N, M, J->gap, H, mv);
    /* diag cells in ascending order: walk the moves backwards from (0,0) */
    int64_t i = 0, j = 0, nd = 0, base = J->out_off[idx];
    for (int64_t t = n - 1; t >= 0; --t) {
        if (mv[t] == MOVE_DIAG) {
            ++i; ++j;
            J->diag_i[base + nd] = (int32_t)(i - 1);
            J->diag_j[base + nd] = (int32_t)(j - 1);
            J->diag_s[base + nd] = S[(i - 1) * M + (j - 1)];
            ++nd;
        } else if (mv[t] == MOVE_UP) {
            ++i;
        } else {
            ++j;
        }
    }
    J->n_diag[idx] = nd;
    J->pair_score[idx] = H[N * (M + 1) + M];
    free(S); free(H); free(mv);
}

static void *mine_worker(void *arg) {
    mine_job *J = (mine_job *)arg;
    for (;;) {
        pthread_mutex_lock(&J->lock);
        int64_t idx = J->next++;
        pthread_mutex_unlock(&J->lock);
        if (idx >= J->n_pairs) break;
        mine_one(J, idx);
    }
    return NULL;
}

/* Mine the listed pairs.  For processed pair idx (0-based in pairs[]), the
 * diagonal cells of the chosen optimal path are written at out_off[idx] in
 * ascending order (capacity min(N,M)), with their similarity; pair_score[idx]
 * is H(N,M).  counts and sim (optional, NULL to skip) receive (ms, mt) and the
 * similarity per cell, row-major per pair at cell_off[idx].  Returns the number
 * of threads used. */
int oracle_mine(int64_t n_pairs, const int64_t *pairs,
                const int64_t *s_doc, const int64_t *s_sent, const int32_t *s_tok,
                const int64_t *t_doc, const int64_t *t_sent, const int32_t *t_tok,
                const int32_t *d_off, const int32_t *d_tgt,
                const double *w, double bias, double gap,
                const int64_t *out_off, double *pair_score, int64_t *n_diag,
                int32_t *diag_i, int32_t *diag_j, double *diag_s,
                int32_t *counts, double *sim, const int64_t *cell_off, int n_threads) {
    mine_job J;
    memset(&J, 0, sizeof J);
    J.n_pairs = n_pairs; J.pairs = pairs;
    J.s_doc = s_doc; J.s_sent = s_sent; J.s_tok = s_tok;
    J.t_doc = t_doc; J.t_sent = t_sent; J.t_tok = t_tok;
    J.d_off = d_off; J.d_tgt = d_tgt;
    for (int k = 0; k < 4; ++k) J.w[k] = w[k];
    J.bias = bias; J.gap = gap;
    J.out_off = out_off; J.pair_score = pair_score; J.n_diag = n_diag;
    J.diag_i = diag_i; J.diag_j = diag_j; J.diag_s = diag_s;
    J.counts = counts; J.sim = sim; J.cell_off = cell_off;
    pthread_mutex_init(&J.lock, NULL);
    if (n_threads < 1) n_threads = 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)n_threads);
    for (int t = 0; t < n_threads; ++t) pthread_create(&th[t], NULL, mine_worker, &J);
    for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
    free(th);
    pthread_mutex_destroy(&J.lock);
    return n_threads;
}
