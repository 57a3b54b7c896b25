// Anchor tokens (Section 5.3: shared names, dates, numbers and references
// mark parallel sentences): anchor a of a sentence becomes the token
// v_words + a of its corpus, and the dictionary gains the identity entries
// v_src + a -> {v_tgt + a}, so that the overlap counts of Section 4 count
// shared anchors like translated words.  Anchor ids are above every word id,
// so a sentence's tokens followed by its offset anchors stay sorted.
#include "kernels.h"

namespace gbm {
namespace {

// Word and anchor offsets start at 0, never decrease and end at n_tok and
// n_anchor_tok; anchor ids lie in [0, v_anchor).  Any violation sets status
// bit 0 (the merge indexes both token arrays through these offsets).
__global__ void anchor_check_kernel(const int64_t *__restrict__ woff, int64_t n_tok, const int64_t *__restrict__ aoff,
                                    int64_t n_sents, const int32_t *__restrict__ ids, int64_t n_anchor_tok,
                                    int32_t v_anchor, uint32_t *status) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t s = t0; s < n_sents; s += stride)
        if (aoff[s + 1] < aoff[s] || woff[s + 1] < woff[s]) atomicOr(status, 1u);
    if (t0 == 0 && (aoff[0] != 0 || aoff[n_sents] != n_anchor_tok || woff[0] != 0 || woff[n_sents] != n_tok))
        atomicOr(status, 1u);
    for (int64_t x = t0; x < n_anchor_tok; x += stride)
        if (ids[x] < 0 || ids[x] >= v_anchor) atomicOr(status, 1u);
}

// out_off[s] = word_off[s] + anchor_off[s]; then sentence s's words, then its
// anchors offset by v_words (one warp per sentence, lanes over tokens).
__global__ void anchor_merge_kernel(const int64_t *__restrict__ woff, const int32_t *__restrict__ words,
                                    const int64_t *__restrict__ aoff, const int32_t *__restrict__ ids, int64_t n_sents,
                                    int32_t v_words, int64_t *__restrict__ out_off, int32_t *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t s = warp0; s <= n_sents; s += nwarps) {
        const int64_t o = woff[s] + aoff[s];
        if (lane == 0) out_off[s] = o;
        if (s == n_sents) break;
        const int64_t w0 = woff[s], nw = woff[s + 1] - w0, a0 = aoff[s], na = aoff[s + 1] - a0;
        for (int64_t x = lane; x < nw; x += 32) out[o + x] = words[w0 + x];
        for (int64_t x = lane; x < na; x += 32) out[o + nw + x] = v_words + ids[a0 + x];
    }
}

// Dictionary copy plus one identity entry per anchor.
__global__ void anchor_dict_kernel(const int32_t *__restrict__ off, const int32_t *__restrict__ tgt, int32_t v_src,
                                   int32_t v_tgt, int64_t n_entries, int32_t v_anchor, int32_t *__restrict__ off_out,
                                   int32_t *__restrict__ tgt_out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t v = t0; v <= v_src; v += stride) off_out[v] = off[v];
    for (int64_t a = t0; a < v_anchor; a += stride) {
        off_out[v_src + 1 + a] = (int32_t)(n_entries + a + 1);
        tgt_out[n_entries + a] = v_tgt + (int32_t)a;
    }
    for (int64_t e = t0; e < n_entries; e += stride) tgt_out[e] = tgt[e];
}

int grid_of(int64_t n, int per_block) {
    int64_t g = (n + per_block - 1) / per_block;
    if (g > 65536) g = 65536;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t launch_anchor_check(const int64_t *woff, int64_t n_tok, const int64_t *aoff, int64_t n_sents,
                                const int32_t *ids, int64_t n_anchor_tok, int32_t v_anchor, uint32_t *status,
                                cudaStream_t st) {
    anchor_check_kernel<<<grid_of(n_sents > n_anchor_tok ? n_sents : n_anchor_tok, 256), 256, 0, st>>>(
        woff, n_tok, aoff, n_sents, ids, n_anchor_tok, v_anchor, status);
    return cudaGetLastError();
}

cudaError_t launch_anchor_merge(const int64_t *woff, const int32_t *words, const int64_t *aoff, const int32_t *ids,
                                int64_t n_sents, int32_t v_words, int64_t *out_off, int32_t *out, cudaStream_t st) {
    anchor_merge_kernel<<<grid_of((n_sents + 1) * 32, 256), 256, 0, st>>>(woff, words, aoff, ids, n_sents, v_words,
                                                                          out_off, out);
    return cudaGetLastError();
}

cudaError_t launch_anchor_dict(const int32_t *off, const int32_t *tgt, int32_t v_src, int32_t v_tgt,
                               int64_t n_entries, int32_t v_anchor, int32_t *off_out, int32_t *tgt_out,
                               cudaStream_t st) {
    const int64_t n = n_entries > (int64_t)v_src + 1 ? n_entries : (int64_t)v_src + 1;
    anchor_dict_kernel<<<grid_of(n > v_anchor ? n : v_anchor, 256), 256, 0, st>>>(off, tgt, v_src, v_tgt, n_entries,
                                                                                  v_anchor, off_out, tgt_out);
    return cudaGetLastError();
}

}  // namespace gbm
