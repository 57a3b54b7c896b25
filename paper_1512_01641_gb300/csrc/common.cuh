// Device helpers shared by the mining kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "miner.h"

namespace gbm {

constexpr uint32_t kFull = 0xffffffffu;
constexpr int32_t kEmpty = -1;

// Traceback directions.  The fill stores, per cell, whether the UP and the
// LEFT candidate equal the cell's value (one bit each: per row and 32-column
// block a 64-bit word, UP bits low, LEFT bits high); the walk takes UP if
// set, else LEFT if set, else DIAG.
constexpr uint32_t kDiag = 0, kUp = 1, kLeft = 2;

struct DevParams {
    float w[4];
    float b;
    float gap;
    float thr;
};

inline DevParams to_dev(const mine_params &p) {
    DevParams d;
    for (int k = 0; k < 4; ++k) d.w[k] = p.w[k];
    d.b = p.b;
    d.gap = p.gap;
    d.thr = p.thr;
    return d;
}

// The four features of Section 4's classifier input, each an IEEE-rounded
// FP32 quotient of two small integers:
//   f0 = ms/ls, f1 = mt/lt, f2 = |ls-lt|/max(ls,lt), f3 = min(ls,lt)/max(ls,lt).
__device__ __forceinline__ void features(int ms, int mt, int ls, int lt, float f[4]) {
    int mx = max(ls, lt), mn = min(ls, lt);
    f[0] = __fdiv_rn((float)ms, (float)ls);
    f[1] = __fdiv_rn((float)mt, (float)lt);
    f[2] = __fdiv_rn((float)(mx - mn), (float)mx);
    f[3] = __fdiv_rn((float)mn, (float)mx);
}

// Similarity s = sigmoid(w . f + b) (Section 4: a linear decision value
// squashed into [0,1]), evaluated without divisions.  Since
// |ls-lt|/max + min/max = 1, the two length features fold into
//   w2 f2 + w3 f3 = w2 + (w3 - w2) * min(ls/lt, lt/ls),
// and with y = -log2(e) * (w . f + b) the similarity is 1 / (1 + 2^y):
//   y = A_i * ms + B_j * mt + C0 + C1 * min(ls / lt, lt / ls)
// where A_i = -log2(e) w0 / ls depends on the source sentence only, B_j on the
// target sentence only.  Every kernel that needs s goes through these
// helpers with explicitly rounded operations, so all of them produce the same
// float for the same cell.
constexpr float kLog2e = 1.4426950408889634f;

struct SimRow {  // per source sentence
    float a;     // -log2(e) w0 / ls
    float len;   // ls
    float rlen;  // 1 / ls
};
struct SimCol {  // per target sentence
    float b;     // -log2(e) w1 / lt
    float len;   // lt
    float rlen;  // 1 / lt
    float pad;
};
struct SimConst {
    float c0;  // -log2(e) (w2 + b)
    float c1;  // -log2(e) (w3 - w2)
};

__device__ __forceinline__ SimConst sim_const(const DevParams &P) {
    return {__fmul_rn(-kLog2e, __fadd_rn(P.w[2], P.b)), __fmul_rn(-kLog2e, __fsub_rn(P.w[3], P.w[2]))};
}
__device__ __forceinline__ SimRow sim_row(int ls, const DevParams &P) {
    const float r = __frcp_rn((float)ls);
    return {__fmul_rn(__fmul_rn(-kLog2e, P.w[0]), r), (float)ls, r};
}
__device__ __forceinline__ SimCol sim_col(int lt, const DevParams &P) {
    const float r = __frcp_rn((float)lt);
    return {__fmul_rn(__fmul_rn(-kLog2e, P.w[1]), r), (float)lt, r, 0.0f};
}
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// Exact float of a small non-negative integer (x < 2^23) with two full-rate
// operations: 2^23 + x has x in its low mantissa bits, so subtracting 2^23
// is exact.  Same value as (float)x, which is a quarter-rate conversion.
__device__ __forceinline__ float small_int_float(int x) {
    return __fsub_rn(__int_as_float(0x4B000000 | x), 8388608.0f);
}
// all-ones if a == b, else 0
__device__ __forceinline__ uint32_t eq_mask(float a, float b) {
    uint32_t m;
    asm("set.eq.u32.f32 %0, %1, %2;" : "=r"(m) : "f"(a), "f"(b));
    return m;
}
// Similarity of a cell from its two count bytes as one 16-bit word (ms in
// the low byte): each byte goes straight into the mantissa of 2^23 by a byte
// permute, the same floats small_int_float makes.
__device__ __forceinline__ float similarity_q16(uint32_t q16, const SimRow &r, const SimCol &c, const SimConst &k) {
    const float fs = __fsub_rn(__int_as_float(__byte_perm(q16, 0x4B000000u, 0x7540)), 8388608.0f);
    const float ft = __fsub_rn(__int_as_float(__byte_perm(q16, 0x4B000000u, 0x7541)), 8388608.0f);
    const float q = fminf(__fmul_rn(r.len, c.rlen), __fmul_rn(c.len, r.rlen));
    float y = __fmaf_rn(k.c1, q, k.c0);
    y = __fmaf_rn(c.b, ft, y);
    y = __fmaf_rn(r.a, fs, y);
    return rcp_approx(__fadd_rn(1.0f, ex2_approx(y)));
}
__device__ __forceinline__ float similarity(int ms, int mt, const SimRow &r, const SimCol &c, const SimConst &k) {
    const float q = fminf(__fmul_rn(r.len, c.rlen), __fmul_rn(c.len, r.rlen));
    float y = __fmaf_rn(k.c1, q, k.c0);
    y = __fmaf_rn(c.b, small_int_float(mt), y);
    y = __fmaf_rn(r.a, small_int_float(ms), y);
    return rcp_approx(__fadd_rn(1.0f, ex2_approx(y)));
}

// Hint: bring the cache line holding p into L1 (no effect on results).
__device__ __forceinline__ void prefetch_l1(const void *p) {
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// PTX acquire/release accesses for the tile flags of the cooperative fill.
// Waits poll with relaxed loads and acquire once the value is seen: an
// acquire at GPU scope must keep later loads off stale L1 lines, so polling
// with it would keep clearing the L1 that the SM's working warps rely on.
__device__ __forceinline__ int ld_relaxed(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(int *p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ---------------------------------------------------------------------------
// 1-D bulk async copy global -> shared (the copy engine behind TMA), with an
// mbarrier that counts the arriving bytes.  One elected lane issues; every
// lane waits with a bounded spin.
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t arrivals = 1) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(arrivals) : "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Plain arrival (no bytes expected) of this thread on bar.
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Order this thread's earlier shared-memory accesses before the async copy
// that will overwrite them, then start the copy of `bytes` (multiple of 16,
// both addresses 16-byte aligned) completing on `bar`.
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// Wait for the phase with the given parity to complete; false after `limit`
// polls (the caller reports a timeout and abandons the work item).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int64_t limit) {
    for (int64_t it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(smem_addr(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Multiplicative hash of a token id into a table of 2^log_slots slots.
__device__ __forceinline__ uint32_t hash_slot(int32_t t, int log_slots) {
    return ((uint32_t)t * 0x9E3779B1u) >> (32 - log_slots);
}

// Bit-sliced counters: plane k holds bit k of 32 independent counters (one
// per bit position).  add() adds a 0/1 word into all 32 counters at once.
template <int K>
struct BitCounter {
    uint32_t p[K];
    __device__ __forceinline__ void clear() {
#pragma unroll
        for (int k = 0; k < K; ++k) p[k] = 0u;
    }
    __device__ __forceinline__ void add(uint32_t x) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            uint32_t c = p[k] & x;
            p[k] ^= x;
            x = c;
        }
    }
    // Add four 0/1 words with a carry-save tree: two full adders into plane 0,
    // one into plane 1, then a ripple of the weight-4 carry (Harley-Seal).
    __device__ __forceinline__ void add4(uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
        const uint32_t s1 = p[0] ^ a ^ b;
        const uint32_t c1 = (p[0] & a) | (p[0] & b) | (a & b);
        const uint32_t s2 = s1 ^ c ^ d;
        const uint32_t c2 = (s1 & c) | (s1 & d) | (c & d);
        p[0] = s2;
        const uint32_t t = p[1] ^ c1 ^ c2;
        uint32_t x = (p[1] & c1) | (p[1] & c2) | (c1 & c2);
        p[1] = t;
#pragma unroll
        for (int k = 2; k < K; ++k) {
            const uint32_t y = p[k] & x;
            p[k] ^= x;
            x = y;
        }
    }
    // Counter for bit position 4m+r lands in byte r of out[m].
    __device__ __forceinline__ void to_bytes(uint32_t out[8]) const {
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            uint32_t w = 0;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                uint32_t nib = (p[k] >> (4 * m)) & 0xFu;
                w |= ((nib * 0x00204081u) & 0x01010101u) << k;
            }
            out[m] = w;
        }
    }
};

// Error bits of the device status word.
constexpr uint32_t kStBadDocOff = 1u << 0;
constexpr uint32_t kStBadSentOff = 1u << 1;
constexpr uint32_t kStBadToken = 1u << 2;
constexpr uint32_t kStUnsorted = 1u << 3;
constexpr uint32_t kStBadDict = 1u << 4;
constexpr uint32_t kStTableFull = 1u << 5;
constexpr uint32_t kStTimeout = 1u << 6;
constexpr uint32_t kStBadList = 1u << 7;  // soft work list over capacity (repeated pairs)

}  // namespace gbm
