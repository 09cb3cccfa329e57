// ffs_device.cuh -- device building blocks: Philox4x32-10, bounded bulk-copy staging of the
// instance tables into shared memory, and the warp-cooperative EDFFS decoder.
#pragma once
#include <stdint.h>
#include <climits>

#include "ffs_layout.h"

namespace edffs {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kOrderTopo = 0, kOrderStage = 1;
constexpr int kMachGene = 0, kMachEarliest = 1;

// ---------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror & Shaw, SC'11: ten rounds of the 4x32 Philox S-box with
// multipliers 0xD2511F53 / 0xCD9E8D57 and Weyl key increments 0x9E3779B9 / 0xBB67AE85.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

__device__ __forceinline__ uint32_t word_of(uint4 r, uint32_t w) {
    return w == 0 ? r.x : w == 1 ? r.y : w == 2 ? r.z : r.w;
}

// Block (d / 4) of the stream (purpose, instance, generation, slot) under key `seed`.
__device__ __forceinline__ uint4 stream_block(uint64_t seed, uint32_t purpose, uint32_t inst,
                                              uint32_t gen, uint32_t slot, uint32_t blk) {
    return philox4x32_10(make_uint4(blk, slot, gen, (purpose << 24) | (inst & 0xFFFFFFu)),
                         (uint32_t)seed, (uint32_t)(seed >> 32));
}

__device__ __forceinline__ uint32_t draw(uint64_t seed, uint32_t purpose, uint32_t inst,
                                         uint32_t gen, uint32_t slot, uint32_t d) {
    return word_of(stream_block(seed, purpose, inst, gen, slot, d >> 2), d & 3u);
}

// floor(u * n / 2^32): an integer in [0, n).
__device__ __forceinline__ uint32_t below(uint32_t u, uint32_t n) { return __umulhi(u, n); }

// ---------------------------------------------------------------- table staging
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Copies the instance blob (16-byte aligned, size a multiple of 16) into shared memory
// with cp.async.bulk completing on an mbarrier.  Every thread waits with an iteration
// limit; on timeout the error word gets kErrTimeout and false is returned.
__device__ __forceinline__ bool stage_tables(char *dst, const char *src, int bytes,
                                             uint64_t *mbar, int32_t *err) {
    const uint32_t bar = smem_u32(mbar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                     : "memory");
        constexpr int kChunk = 16384;
        for (int off = 0; off < bytes; off += kChunk) {
            const int n = bytes - off < kChunk ? bytes - off : kChunk;
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    smem_u32(dst + off)),
                "l"(src + off), "r"(n), "r"(bar)
                : "memory");
        }
    }
    bool done = false;
    for (int it = 0; it < (1 << 22) && !done; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar)
            : "memory");
        done = ok != 0;
    }
    if (!done) atomicOr(err, kErrTimeout);
    return __syncthreads_and(done) != 0;
}

// ---------------------------------------------------------------- decoder
struct DecodeOut {
    long long tard;  // sum_j T_j
    int cmax;        // C_max
    int status;      // 0 ok, 1 profile outgrew Hcap, 2 malformed chromosome
};

// Earliest start r >= t0 (slots past RS) such that headroom h[r .. r+p) >= q everywhere.
// Slots at or beyond the high-water mark hw were never touched and hold the full peak.
// Returns `limit` as soon as the answer cannot be below it.  One 32-slot window per step:
// a ballot finds the last violating slot and the candidate jumps past it.
__device__ __forceinline__ int earliest_start(const uint16_t *h, int hw, int t0, int p, unsigned q,
                                              int limit, int lane) {
    int run = t0, c = t0;
    for (;;) {
        if (run >= limit) return limit;
        const int end = run + p;
        if (c >= end || c >= hw) return run;
        const int pos = c + lane;
        const bool bad = pos < end && pos < hw && h[pos] < q;
        const unsigned bm = __ballot_sync(kFull, bad);
        if (bm == 0) {
            c += 32;
        } else {
            run = c + 32 - __clz(bm);  // one past the last violating slot
            c = run;
        }
    }
}

// Decodes one chromosome with the whole warp (Sec. 4.3, Alg. 1-2).  State lives in the
// caller's workspace: h [Hcap] headroom, C [N], mfree [M], inv [K+N], y [K], x [K].
// Schedule output (S_out/M_out, [N*g]) is written for free ops only when non-null.
template <int ORDER, int MACH>
__device__ DecodeOut decode_warp(const Tabs &T, uint16_t *h, int Hcap, int32_t *C, int32_t *mfree,
                                 int16_t *inv, const int16_t *y, const int8_t *x, int32_t *S_out,
                                 int32_t *M_out, int lane) {
    const int N = T.N, K = T.K, M = T.M, g = T.g, RS = T.RS;
    const unsigned Qmax = (unsigned)T.Qmax;

    if (T.E0 > Hcap) return {0, 0, 1};  // executing ops alone outgrow the profile slice
    for (int j = lane; j < N; j += 32) C[j] = T.C0[j];
    for (int m = lane; m < M; m += 32) mfree[m] = T.mfree0[m];
    for (int i = lane; i < T.E0; i += 32) h[i] = T.h0[i];
    int hw = T.E0;

    // Validate Y (a permutation of 1..K) and X, and build inv[K - y] = gene.
    for (int i = lane; i < K; i += 32) inv[i] = -1;
    __syncwarp();
    bool bad = false;
    for (int k = lane; k < K; k += 32) {
        const int v = y[k];
        if (v < 1 || v > K) bad = true;
        else inv[K - v] = (int16_t)k;
        if (MACH == kMachGene) {
            const int xm = x[k];
            if (xm < 0 || xm >= T.o[T.gstg[k]]) bad = true;
        }
    }
    __syncwarp();
    for (int i = lane; i < K; i += 32)
        if (inv[i] < 0) bad = true;
    if (__any_sync(kFull, bad)) return {0, 0, 2};

    int16_t *nxt = inv + K;  // Alg. 1 reading: next free gene of each job
    if (ORDER == kOrderTopo) {
        for (int j = lane; j < N; j += 32) nxt[j] = T.gfirst[j];
        __syncwarp();
    }

    // Assigns gene k (Alg. 2); returns false if the profile would outgrow Hcap.
    auto place = [&](int k) -> bool {
        const int j = T.gjob[k], s = T.gstg[k];
        const int p = T.p[j * g + s];
        const int est = max(RS, max(T.R[j], C[j])) - RS;
        const int mo = T.moff[s];
        int best_t = INT_MAX, best_m = 0;
        if (MACH == kMachGene) {
            best_m = x[k];
            best_t = earliest_start(h, hw, max(est, mfree[mo + best_m] - RS), p, (unsigned)T.q[mo + best_m],
                                    INT_MAX, lane);
        } else {
            const int os = T.o[s];
            for (int m = 0; m < os; ++m) {
                const int t0 = max(est, mfree[mo + m] - RS);
                if (t0 >= best_t) continue;  // cannot beat (or tie below) the best so far
                const int t = earliest_start(h, hw, t0, p, (unsigned)T.q[mo + m], best_t, lane);
                if (t < best_t) {
                    best_t = t;
                    best_m = m;
                }
            }
        }
        const int e = best_t + p;
        if (e > Hcap) return false;
        const unsigned qq = (unsigned)T.q[mo + best_m];
        const int lo = min(best_t, hw);
        for (int pos = lo + lane; pos < e; pos += 32) {
            unsigned v = pos < hw ? h[pos] : Qmax;
            if (pos >= best_t) v -= qq;
            h[pos] = (uint16_t)v;
        }
        hw = max(hw, e);
        __syncwarp();
        if (lane == 0) {
            mfree[mo + best_m] = e + RS;
            C[j] = e + RS;
            if (S_out) {
                S_out[j * g + s] = best_t + RS;
                M_out[j * g + s] = best_m;
            }
        }
        __syncwarp();
        return true;
    };

    if (ORDER == kOrderStage) {
        for (int s = 0; s < g; ++s) {
            for (int base = 0; base < K; base += 32) {
                const int i = base + lane;
                const int k = i < K ? inv[i] : -1;
                unsigned mask = __ballot_sync(kFull, k >= 0 && T.gstg[k] == s);
                while (mask) {
                    const int l = __ffs(mask) - 1;
                    mask &= mask - 1;
                    if (!place(__shfl_sync(kFull, k, l))) return {0, 0, 1};
                }
            }
        }
    } else {
        for (int n = 0; n < K; ++n) {
            int besty = 0, bestj = -1;
            for (int j = lane; j < N; j += 32) {
                const int k = nxt[j];
                if (k >= 0 && k < T.gfirst[j] + T.gcnt[j]) {
                    const int v = y[k];
                    if (v > besty) {
                        besty = v;
                        bestj = j;
                    }
                }
            }
#pragma unroll
            for (int off = 16; off; off >>= 1) {
                const int oy = __shfl_xor_sync(kFull, besty, off);
                const int oj = __shfl_xor_sync(kFull, bestj, off);
                if (oy > besty) {
                    besty = oy;
                    bestj = oj;
                }
            }
            const int k = nxt[bestj];
            __syncwarp();
            if (lane == 0) nxt[bestj] = (int16_t)(k + 1);
            __syncwarp();
            if (!place(k)) return {0, 0, 1};
        }
    }

    // Eq. (2)-(3) over every job, frozen ones included.
    long long tard = 0;
    int cmax = 0;
    for (int j = lane; j < N; j += 32) {
        const int cj = C[j];
        const long long d = (long long)cj - T.D[j];
        if (d > 0) tard += d;
        cmax = max(cmax, cj);
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        tard += __shfl_xor_sync(kFull, tard, off);
        cmax = max(cmax, __shfl_xor_sync(kFull, cmax, off));
    }
    return {tard, cmax, 0};
}

}  // namespace edffs
