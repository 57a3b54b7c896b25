// Bi-directional mining (Section 5.4, "BI"): the reverse direction is mined
// by a second plan with the corpora swapped and a dictionary from target ids
// to source ids; these kernels build that dictionary as the transpose of the
// forward one and merge the links of the two directions pair by pair.
#include <cmath>

#include "kernels.h"

namespace gbm {
namespace {

// Offsets start at 0, never decrease, end at n_entries; every target id is
// in [0, v_tgt).  Any violation sets status bit 0.
__global__ void dict_check_kernel(const int32_t *__restrict__ off, int32_t v_src, int64_t n_entries,
                                  const int32_t *__restrict__ tgt, int32_t v_tgt, uint32_t *status) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t v = t0; v < v_src; v += stride)
        if (off[v + 1] < off[v]) atomicOr(status, 1u);
    if (t0 == 0 && (off[0] != 0 || (int64_t)off[v_src] != n_entries)) atomicOr(status, 1u);
    for (int64_t e = t0; e < n_entries; e += stride) {
        const int32_t t = tgt[e];
        if (t < 0 || t >= v_tgt) atomicOr(status, 1u);
    }
}

// Entries per target id.
__global__ void dict_count_kernel(const int32_t *__restrict__ tgt, int64_t n_entries, int32_t *cnt) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_entries; e += stride)
        atomicAdd(&cnt[tgt[e]], 1);
}

// Source id v into the list of each of its targets (at a cursor that starts
// at the list's offset); the order within a list is fixed by dict_sort_kernel.
__global__ void dict_scatter_kernel(const int32_t *__restrict__ off, int32_t v_src, const int32_t *__restrict__ tgt,
                                    int32_t *cursor, int32_t *__restrict__ tgt_out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < v_src; v += stride)
        for (int32_t e = off[v]; e < off[v + 1]; ++e) tgt_out[atomicAdd(&cursor[tgt[e]], 1)] = (int32_t)v;
}

// Each reverse list ascending (insertion sort, one thread per list; the
// lists hold the few source ids that translate to one target id).
__global__ void dict_sort_kernel(const int32_t *__restrict__ off_out, int32_t v_tgt, int32_t *__restrict__ tgt_out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < v_tgt; t += stride) {
        const int32_t a = off_out[t], b = off_out[t + 1];
        for (int32_t x = a + 1; x < b; ++x) {
            const int32_t key = tgt_out[x];
            int32_t y = x - 1;
            while (y >= a && tgt_out[y] > key) {
                tgt_out[y + 1] = tgt_out[y];
                --y;
            }
            tgt_out[y + 1] = key;
        }
    }
}

// One thread per pair: merge the forward links (i, j) and the reverse links
// (i', j') -> (j', i'), both ascending in i and in j, into one list ascending
// in (i, j); a link in both lists appears once with both similarities.  Every
// range is clamped to its buffer's capacity and no write goes past the
// output's, so offsets that did not come from mining these plans cannot move
// an access out of bounds.
template <bool WRITE>
__global__ void links_combine_kernel(LinkView fwd, LinkView rev, int64_t n_pairs, int mode, int32_t *count,
                                     int64_t out_cap, const int64_t *__restrict__ out_off, int32_t *__restrict__ out_i,
                                     int32_t *__restrict__ out_j, float *__restrict__ out_sf,
                                     float *__restrict__ out_sr) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const float nan = __int_as_float(0x7fc00000);
    auto clamp = [](int64_t x, int64_t hi) { return x < 0 ? 0 : (x > hi ? hi : x); };
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_pairs; k += stride) {
        int64_t a = clamp(fwd.off[k], fwd.cap), c = clamp(rev.off[k], rev.cap);
        const int64_t ae = clamp(fwd.off[k + 1], fwd.cap), ce = clamp(rev.off[k + 1], rev.cap);
        int64_t o = WRITE ? out_off[k] : 0;
        int32_t n = 0;
        while (a < ae || c < ce) {
            const int64_t fk = a < ae ? ((int64_t)fwd.i[a] << 32) | (uint32_t)fwd.j[a] : INT64_MAX;
            const int64_t rk = c < ce ? ((int64_t)rev.j[c] << 32) | (uint32_t)rev.i[c] : INT64_MAX;
            const bool in_f = fk <= rk, in_r = rk <= fk;
            if (mode == 0 || (in_f && in_r)) {
                if (WRITE && o >= 0 && o < out_cap) {
                    const int64_t key = in_f ? fk : rk;
                    out_i[o] = (int32_t)(key >> 32);
                    out_j[o] = (int32_t)(key & 0xffffffff);
                    out_sf[o] = in_f ? fwd.s[a] : nan;
                    out_sr[o] = in_r ? rev.s[c] : nan;
                    ++o;
                } else if (!WRITE) {
                    ++n;
                }
            }
            a += in_f;
            c += in_r;
        }
        if (!WRITE) count[k] = n;
    }
}

int grid_for(int64_t n, int per_block) {
    int64_t g = (n + per_block - 1) / per_block;
    if (g > 65536) g = 65536;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t launch_dict_check(const int32_t *off, int32_t v_src, int64_t n_entries, const int32_t *tgt,
                              int32_t v_tgt, uint32_t *status, cudaStream_t st) {
    dict_check_kernel<<<grid_for(v_src > n_entries ? v_src : n_entries, 256), 256, 0, st>>>(off, v_src, n_entries, tgt,
                                                                                            v_tgt, status);
    return cudaGetLastError();
}

cudaError_t launch_dict_count(const int32_t *tgt, int64_t n_entries, int32_t *cnt, cudaStream_t st) {
    if (n_entries == 0) return cudaSuccess;
    dict_count_kernel<<<grid_for(n_entries, 256), 256, 0, st>>>(tgt, n_entries, cnt);
    return cudaGetLastError();
}

cudaError_t launch_dict_scatter(const int32_t *off, int32_t v_src, const int32_t *tgt, int32_t *cursor,
                                int32_t *tgt_out, cudaStream_t st) {
    dict_scatter_kernel<<<grid_for(v_src, 256), 256, 0, st>>>(off, v_src, tgt, cursor, tgt_out);
    return cudaGetLastError();
}

cudaError_t launch_dict_sort(const int32_t *off_out, int32_t v_tgt, int32_t *tgt_out, cudaStream_t st) {
    dict_sort_kernel<<<grid_for(v_tgt, 256), 256, 0, st>>>(off_out, v_tgt, tgt_out);
    return cudaGetLastError();
}

cudaError_t launch_links_combine(LinkView fwd, LinkView rev, int64_t n_pairs, int mode, int32_t *count,
                                 int64_t out_cap, const int64_t *out_off, int32_t *out_i, int32_t *out_j,
                                 float *out_sf, float *out_sr, cudaStream_t st) {
    if (n_pairs == 0) return cudaSuccess;
    if (out_i)
        links_combine_kernel<true><<<grid_for(n_pairs, 128), 128, 0, st>>>(fwd, rev, n_pairs, mode, count, out_cap,
                                                                          out_off, out_i, out_j, out_sf, out_sr);
    else
        links_combine_kernel<false><<<grid_for(n_pairs, 128), 128, 0, st>>>(fwd, rev, n_pairs, mode, count, out_cap,
                                                                           out_off, out_i, out_j, out_sf, out_sr);
    return cudaGetLastError();
}

}  // namespace gbm
