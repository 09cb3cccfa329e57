// ffs_device.cuh -- device building blocks: Philox4x32-10, bounded bulk-copy staging of the
// instance tables into shared memory, and the warp-cooperative EDFFS decoder.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

#include <climits>

#include "ffs_layout.h"

namespace edffs {

constexpr unsigned kFull = 0xffffffffu;
// Ops placed per step of the stage-order loop on prefilled shared-memory profiles (2
// measured fastest on the dynamic job: 15.36 M decodes/s, against 14.17 M with 3 and
// 13.31 M with 4).
constexpr int kPlaceGroup = 2;
constexpr int kOrderTopo = 0, kOrderStage = 1;
constexpr int kMachGene = 0, kMachEarliest = 1;
// Kernel-side machine modes add the unrelated-machine variants (per-gene p and q per
// machine, the earliest completion instead of the earliest start).
constexpr int kMachGeneU = 2, kMachEarliestU = 3;
// Bit 2 (kPlaceInsert) selects idle-gap insertion placement.
constexpr int kPlaceInsert = 4;
__host__ __device__ constexpr bool mach_gene(int m) { return (m & 1) == 0; }
__host__ __device__ constexpr bool mach_unrel(int m) { return (m & 2) != 0; }
__host__ __device__ constexpr bool mach_insert(int m) { return (m & kPlaceInsert) != 0; }


// ---------------------------------------------------------------- bounds-checked builds
// With FFS_CHECKED, an index into a shared- or global-memory buffer that falls outside
// [0, n) is counted (per translation unit; bounds_faults_take reads and clears the count)
// and replaced by 0, so the access stays inside the buffer and control flow, which is
// warp-uniform, does not change.  Ordinary builds use the index as it is.
#ifdef FFS_CHECKED
static __device__ unsigned int g_bounds_faults;
__device__ __forceinline__ int checked_ix(int i, int n) {
    if ((unsigned)i >= (unsigned)n) {
        atomicAdd(&g_bounds_faults, 1u);
        return 0;
    }
    return i;
}
static inline unsigned int bounds_faults_take() {
    unsigned int v = 0, z = 0;
    if (cudaMemcpyFromSymbol(&v, g_bounds_faults, sizeof v) != cudaSuccess) return ~0u;
    if (cudaMemcpyToSymbol(g_bounds_faults, &z, sizeof z) != cudaSuccess) return ~0u;
    return v;
}
#define FFS_IX(i, n) ::edffs::checked_ix((i), (n))
#else
#define FFS_IX(i, n) (i)
#endif

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

// Iterations of the bounded wait for the instance tables.
constexpr int kStageWaitIters = 1 << 22;

// Copies the instance blob (16-byte aligned, size a multiple of 16) into shared memory
// with cp.async.bulk completing on an mbarrier.  Every thread waits with an iteration
// limit; on timeout the error word gets kErrTimeout and false is returned.  With `skip`
// (failure injection for tests) nothing is copied and nothing arrives, so the wait runs
// out with no copy in flight.
__device__ __forceinline__ bool stage_tables(char *dst, const char *src, int bytes,
                                             uint64_t *mbar, int32_t *err, bool skip = false,
                                             int iters = kStageWaitIters) {
    const uint32_t bar = smem_u32(mbar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0 && !skip) {
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
    for (int it = 0; it < iters && !done; ++it) {
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

// Expands bits 0/1 of m to the low/high halfword of a 32-bit word.
__device__ __forceinline__ uint32_t halves(unsigned m) {
    return (m & 1u) * 0xFFFFu + (m & 2u) * 0x7FFF8000u;
}

// Halfword masks of the slots [lo, hi) among b .. b+3 (x: slots b, b+1; y: b+2, b+3).
// PTX clamps a 64-bit shift amount at 64, so no range checks are needed.
__device__ __forceinline__ uint2 slot_mask(int b, int lo, int hi) {
    const uint32_t sl = (uint32_t)max(lo - b, 0) << 4, sh = (uint32_t)max(hi - b, 0) << 4;
    uint64_t a, c;
    asm("shl.b64 %0, %1, %2;" : "=l"(a) : "l"(~0ull), "r"(sl));
    asm("shl.b64 %0, %1, %2;" : "=l"(c) : "l"(~0ull), "r"(sh));
    const uint64_t m = a & ~c;
    return make_uint2((uint32_t)m, (uint32_t)(m >> 32));
}

// First slot >= t at which a machine is idle, from its occupancy bitmap (nw words): each
// step the warp looks at 32 words (1024 slots).  At least 32 nw if there is none below.
__device__ __forceinline__ int next_idle(const uint32_t *bm, int nw, int t, int lane) {
    for (int w0 = t >> 5; w0 < nw; w0 += 32) {
        const int w = w0 + lane;
        uint32_t fr = w < nw ? ~bm[w] : 0u;
        if (w == (t >> 5)) fr &= ~((1u << (t & 31)) - 1u);  // slots below t do not count
        const unsigned any = __ballot_sync(kFull, fr != 0u);
        if (any) {
            const int l = __ffs(any) - 1;
            return 32 * (w0 + l) + __ffs(__shfl_sync(kFull, fr, l)) - 1;
        }
    }
    return t > 32 * nw ? t : 32 * nw;
}

// Earliest start r >= t0 (slots past RS) such that headroom h[r .. r+p) >= q everywhere,
// slots at or beyond hw counting as full headroom (append placement, no occupancy).
// State: the candidate r, with [r, v) known to have headroom q.  Each step loads the 128
// slots from v & ~3 (4 per lane, below hw), marks the slots of [v, hw) lacking headroom,
// and then either confirms r (its clean run reaches p slots, or hw), or takes the first
// start right after a marked slot whose clean run reaches p.  Failing both, the start of
// the clean run that reaches the window's end becomes the candidate (v moves to that end),
// or the window's end itself when its last slot is marked.  Returns `limit` as soon as the
// answer cannot be below it.  Loads stay below hw <= Hcap (Hcap a multiple of 4).
__device__ __forceinline__ int earliest_start_win(const uint16_t *h, int hw, int t0, int p, uint32_t q2,
                                                  int limit, int lane) {
    int r = t0, v = t0;
    for (;;) {
        if (r >= limit) return limit;
        if (v >= hw || v - r >= p) return r;
        const int c = v & ~3, b = c + 4 * lane, wend = c + 128;
        const bool fin = wend >= hw;  // slots past the window are full headroom
        uint2 w = make_uint2(0u, 0u);
        if (b < hw) w = *reinterpret_cast<const uint2 *>(h + b);
        const uint32_t vx = ~((w.x | 0x80008000u) - q2), vy = ~((w.y | 0x80008000u) - q2);
        // bit k: slot b + k lacks headroom q; only slots of [v, hw) count
        unsigned nib = ((vx >> 15) & 1u) | ((vx >> 30) & 2u) | ((vy >> 13) & 4u) | ((vy >> 28) & 8u);
        nib &= (0xFu << min(max(v - b, 0), 4)) & ~(0xFu << min(max(hw - b, 0), 4));
        const unsigned anyv = __ballot_sync(kFull, nib != 0u);
        if (anyv == 0u) {  // r's run reaches the window's end
            if (fin) return r;
            v = wend;
            continue;
        }
        const unsigned b3 = __ballot_sync(kFull, (nib & 8u) != 0u);
        const int fvl = nib ? b + __ffs(nib) - 1 : INT_MAX;  // the lane's first marked slot
        const unsigned later = anyv & ~((2u << lane) - 1u);  // lanes above this one with one
        const int nfv = __shfl_sync(kFull, fvl, later ? __ffs(later) - 1 : 0);
        const int fv = __shfl_sync(kFull, fvl, __ffs(anyv) - 1);
        if (fv - r >= p) return r;
        // r fails: starts right after marked slots (a clean slot whose predecessor is marked)
        const int tail = fin ? INT_MAX : wend;  // where unknown slots begin
        const unsigned pv = (nib << 1) | (lane ? (b3 >> (lane - 1)) & 1u : 0u);
        const unsigned st = pv & ~nib & 0xFu;
        int best = INT_MAX, cont = INT_MAX;
        int nv = later ? nfv : tail;  // next marked slot above the one considered
#pragma unroll
        for (int k = 3; k >= 0; --k) {
            if ((nib >> k) & 1u) {
                nv = b + k;
            } else if ((st >> k) & 1u) {
                if (nv - (b + k) >= p) best = b + k;
                else if (nv == tail) cont = b + k;
            }
        }
        const unsigned fb = __ballot_sync(kFull, best != INT_MAX);
        if (fb) {
            const int rr = __shfl_sync(kFull, best, __ffs(fb) - 1);
            return rr < limit ? rr : limit;
        }
        const unsigned cb = __ballot_sync(kFull, cont != INT_MAX);
        r = cb ? __shfl_sync(kFull, cont, __ffs(cb) - 1) : wend;
        v = wend;
    }
}

// Earliest start r >= t0 (slots past RS) such that headroom h[r .. r+p) >= q everywhere.
// Append placement takes the window form above unless WIN is off.  Otherwise (the jump
// scan): slots at or beyond the high-water mark hw were never touched and hold the full
// peak, so only [r, min(r+p, hw)) needs checking.  Each lane reads 4 consecutive slots with one
// 64-bit load (128 slots per step) and compares both halfwords of a word at once: with
// headroom and q below 2^15, (h | 0x8000) - q keeps bit 15 set exactly when h >= q, and no
// borrow crosses into the next halfword.  A ballot finds the last violating slot and the
// candidate jumps past it.  Returns `limit` as soon as the answer cannot be below it.
// Loads stay below hw <= Hcap (Hcap a multiple of 4); lanes past the window load nothing.
// With INS, `bm` is the machine's occupancy bitmap (nw words; bit t: busy at slot t) and a
// slot also violates when the machine is busy there; a candidate start that falls in a
// busy stretch moves to the stretch's end directly.  Bits are only set below hw.
// Insertion placement: the earliest start r >= t0 at which the machine is idle (occupancy
// bitmap bm of nw words) and every slot of [r, r+p) has headroom q, slots at or beyond hw
// being idle with full headroom.  Each step looks at the 1024 slots of 32 whole bitmap
// words from the word that holds the candidate: lane l builds the violation bits of its
// word (busy, short of headroom, or before the candidate).  The first clean run of p slots
// is found from each word's clean slots at its start and end, the clean slots ending at
// the previous word's end (a ballot and two shuffles), and, for p <= 32, the runs inside
// one word; a clean run that reaches the step's end becomes the next step's candidate.
// For p <= 512 (each step then advances at least 512 slots).  Returns `limit` as soon as
// the answer cannot be below it.  Loads stay below hw <= Hcap (Hcap a multiple of 8).
__device__ __forceinline__ int earliest_start_ins(const uint16_t *h, int hw, int t0, int p, uint32_t q2, int limit,
                                                  int lane, const uint32_t *bm, int nw) {
    int cur = t0;
    for (;;) {
        if (cur >= limit) return limit;
        if (cur >= hw) return cur;  // idle with full headroom from there on
        const int base = cur & ~31, s0 = base + 32 * lane;
        uint32_t v = 0u;  // bit i: slot s0 + i violates
        if (s0 < hw) {
            uint32_t ok = 0u;  // bit i: slot s0 + i has headroom q (or lies at or past hw)
#pragma unroll
            for (int c = 0; c < 8; ++c) {  // four slots per load
                const int sc = s0 + 4 * c;
                uint32_t n = 0xFu;
                if (sc < hw) {
                    const uint2 w = *reinterpret_cast<const uint2 *>(h + sc);
                    // bit 15 of each halfword of (h | 0x8000) - q: the slot has headroom q.
                    // The bytes holding those bits, in slot order (bits 7, 15, 23, 31), then
                    // a multiply whose partial products never overlap moves them to bits 28..31.
                    const uint32_t t = __byte_perm((w.x | 0x80008000u) - q2, (w.y | 0x80008000u) - q2, 0x7531);
                    n = ((t & 0x80808080u) * 0x00204081u) >> 28;
                }
                ok |= n << (4 * c);
            }
            v = bm[FFS_IX(s0 >> 5, nw)] | ~ok;
            if (cur > s0) v |= cur - s0 >= 32 ? 0xFFFFFFFFu : ((1u << (cur - s0)) - 1u);
            if (hw - s0 < 32) v &= (1u << (hw - s0)) - 1u;
        }
        const int pre = v ? __ffs(v) - 1 : 32;  // clean slots at the word's start
        const int suf = __clz(v);               // clean slots at its end (32 if v == 0)
        // clean slots ending at this word's end: from the last word up to here with a violation
        const unsigned upto = __ballot_sync(kFull, v != 0u) & (0xFFFFFFFFu >> (31 - lane));
        const int j = upto ? 31 - __clz(upto) : 0;
        const int sufj = __shfl_sync(kFull, suf, j);
        const int E = upto ? sufj + 32 * (lane - j) : 32 * (lane + 1);
        int Eprev = __shfl_up_sync(kFull, E, 1);
        if (lane == 0) Eprev = 0;
        int cand = INT_MAX;  // the first clean run of p slots this lane sees, in step coordinates
        if (v != 0u) {
            if (Eprev + pre >= p) cand = 32 * lane - Eprev;  // the run across the word's start
            if (p <= 32) {                                  // runs inside the word
                uint32_t r = ~v;
                for (int have = 1; have < p;) {
                    const int sft = min(have, p - have);
                    r &= r >> sft;
                    have += sft;
                }
                if (r) cand = min(cand, 32 * lane + __ffs(r) - 1);
            }
        }
        if (lane == 31 && E >= p) cand = min(cand, 1024 - E);  // a run reaching the step's end
        const unsigned best = __reduce_min_sync(kFull, (unsigned)cand);
        if (best != (unsigned)INT_MAX) {
            const int r = base + (int)best;
            return r < limit ? r : limit;
        }
        cur = base + 1024 - __shfl_sync(kFull, E, 31);  // the clean run reaching the end, if any
    }
}

template <bool INS = false, bool WIN = true>
__device__ __forceinline__ int earliest_start(const uint16_t *h, int hw, int t0, int p, uint32_t q2,
                                              int limit, int lane, const uint32_t *bm = nullptr, int nw = 0) {
    if (!INS && WIN) return earliest_start_win(h, hw, t0, p, q2, limit, lane);
    if (INS && p <= 512) return earliest_start_ins(h, hw, t0, p, q2, limit, lane, bm, nw);
    int run = t0;
    if (INS && run < limit) run = next_idle(bm, nw, run, lane);
    if (run >= limit) return limit;
    int end = min(run + p, hw);
    int c = run & ~3;
    while (c < end) {
        const int b = c + 4 * lane;
        uint2 w = make_uint2(0u, 0u);
        if (b < end) w = *reinterpret_cast<const uint2 *>(h + b);
        const uint2 m = slot_mask(b, run, end);  // empty for lanes past the window
        // bit 15 of each halfword: the slot lacks headroom q (or, with INS, the machine is busy)
        uint32_t vx = ~((w.x | 0x80008000u) - q2), vy = ~((w.y | 0x80008000u) - q2);
        if (INS && b < end) {
            const unsigned busy = (bm[b >> 5] >> (b & 31)) & 0xFu;
            vx |= halves(busy);
            vy |= halves(busy >> 2);
        }
        vx &= m.x & 0x80008000u;
        vy &= m.y & 0x80008000u;
        // the lane's last violating slot among its four
        const int li = vy ? 2 + (int)(vy >> 31) : vx ? (int)(vx >> 31) : -1;
        const unsigned vm = __ballot_sync(kFull, li >= 0);
        if (vm == 0) {
            c += 128;
        } else {
            const int l = 31 - __clz(vm);
            run = c + 4 * l + __shfl_sync(kFull, li, l) + 1;  // one past the last violating slot
            if (INS && run < limit) run = next_idle(bm, nw, run, lane);
            if (run >= limit) return limit;
            end = min(run + p, hw);
            c = run & ~3;
        }
    }
    return run;
}

// Draws q on [t, e) of a profile initialised there.  Slots in [t, e) hold at least q, so
// the halfword subtraction never borrows.
__device__ __forceinline__ void commit_power_full(uint16_t *h, int t, int e, uint32_t q2, int lane) {
    for (int b = (t & ~3) + 4 * lane; b < e; b += 128) {
        const uint2 sub = slot_mask(b, t, e);
        uint2 w = *reinterpret_cast<const uint2 *>(h + b);
        w.x -= q2 & sub.x;
        w.y -= q2 & sub.y;
        *reinterpret_cast<uint2 *>(h + b) = w;
    }
}

// Profiles filled on demand: slots below the fill mark fl (a multiple of 4) are
// initialised, the rest not yet.  Advances fl past e in 256-slot steps, writing full
// headroom (each lane 2 x 4 slots a step, below Hcap).  Every lane then sees every slot
// below the new mark.
__device__ __forceinline__ void fill_to(uint16_t *h, int &fl, int e, int Hcap, uint32_t Q2, int lane) {
    if (fl >= e) return;
    do {
        const int b = fl + 4 * lane;
        if (b < Hcap) *reinterpret_cast<uint2 *>(h + b) = make_uint2(Q2, Q2);
        if (b + 128 < Hcap) *reinterpret_cast<uint2 *>(h + b + 128) = make_uint2(Q2, Q2);
        fl += 256;
    } while (fl < e);
    __syncwarp();
}

// The common case of one op on a profile initialised up to the op's end: when [t, t+p)
// lies within one 128-slot step from t & ~3 and every slot of it has headroom q, q is
// drawn there from the words the check loaded (no second read) and t is returned.  Otherwise nothing changes and the returned start is where the general scan
// may resume: one past the last slot lacking headroom (the jump its own first step would
// make), or t when the op spans more than one step.  Only lanes whose four slots start
// below t + p load and store.  The caller ensures t + p <= Hcap.
__device__ __forceinline__ int place_first(uint16_t *h, int t, int p, uint32_t q2, int lane, bool &placed,
                                           int Hcap) {
    placed = false;
    const int c = t & ~3, e = t + p;
    if (e - c > 128) return t;
    const int b = c + 4 * lane;
    const bool mine = b < e;
    uint2 w = make_uint2(0u, 0u);  // lanes past the window: no slot in it
    if (mine) w = *reinterpret_cast<const uint2 *>(h + FFS_IX(b, Hcap - 3));
    const uint2 m = slot_mask(b, t, e);
    // bit 15 of (h | 0x8000) - q is clear exactly where h < q (no borrow between halfwords)
    const uint32_t vx = ~((w.x | 0x80008000u) - q2) & m.x & 0x80008000u;
    const uint32_t vy = ~((w.y | 0x80008000u) - q2) & m.y & 0x80008000u;
    const unsigned vm = __ballot_sync(kFull, (vx | vy) != 0u);
    if (vm) {
        const int l = 31 - __clz(vm);
        const int li = vy ? 2 + (int)(vy >> 31) : (int)(vx >> 31);  // the lane's last violating slot
        return c + 4 * l + __shfl_sync(kFull, li, l) + 1;
    }
    if (mine) {
        w.x -= q2 & m.x;
        w.y -= q2 & m.y;
        *reinterpret_cast<uint2 *>(h + FFS_IX(b, Hcap - 3)) = w;
    }
    placed = true;
    return t;
}

// Insertion placement in one step, for identical machines and the earliest machine: the
// machines that become available first (lanes m with tl == t0) are checked at t0 together.
// Machine m fits if its occupancy bitmap is clear on [t0, t0+p) and every slot there has
// headroom for its power q_m (the window's least headroom, one reduction).  Since no
// machine can start before t0, the lowest machine that fits is the earliest-start choice;
// its power is drawn from the words already loaded.  Returns that machine, or -1 with
// nothing changed when none fits or the check does not fit one step (more than four
// machines, a window past one 128-slot step or past Hcap).  The profile must be initialised
// up to t0 + p.
__device__ __forceinline__ int place_first_ins(uint16_t *h, int Hcap, const uint32_t *busy, int words, int t0, int p,
                                               int tl, uint32_t q2, int os, int lane) {
    const int c = t0 & ~3, e = t0 + p;
    if (os > 4 || e > Hcap || e - c > 128) return -1;
    const int b = c + 4 * lane;
    const bool mine = b < e;
    uint2 w = make_uint2(0u, 0u);
    if (mine) w = *reinterpret_cast<const uint2 *>(h + FFS_IX(b, Hcap - 3));
    const uint2 m = slot_mask(b, t0, e);
    // least headroom over the window; slots outside it count as full
    const uint32_t mn = __vminu2(w.x | ~m.x, w.y | ~m.y);
    const unsigned least = __reduce_min_sync(kFull, min(mn & 0xFFFFu, mn >> 16));
    // occupancy: lane l reads word (t0 >> 5) + (l & 7) of machine l >> 3 (5 words cover 128 slots)
    const int bmach = lane >> 3, wd = (t0 >> 5) + (lane & 7);
    uint32_t bz = 0u;
    if (bmach < os && wd <= ((e - 1) >> 5)) {
        const int lo = max(t0 - 32 * wd, 0), hi = min(e - 32 * wd, 32);
        const uint32_t hm = hi >= 32 ? 0xFFFFFFFFu : ((1u << hi) - 1u);
        bz = busy[(size_t)bmach * words + FFS_IX(wd, words)] & hm & ~((1u << lo) - 1u);
    }
    const unsigned occ = __ballot_sync(kFull, bz != 0u);
    const bool fits = lane < os && tl == t0 && ((occ >> (8 * lane)) & 0xFFu) == 0u && (q2 & 0xFFFFu) <= least;
    const unsigned fm = __ballot_sync(kFull, fits);
    if (!fm) return -1;
    const int bm = __ffs(fm) - 1;
    const uint32_t bq2 = __shfl_sync(kFull, q2, bm);
    if (mine) {
        w.x -= bq2 & m.x;
        w.y -= bq2 & m.y;
        *reinterpret_cast<uint2 *>(h + FFS_IX(b, Hcap - 3)) = w;
    }
    return bm;
}

// Marks slots [t, e) busy in a machine's occupancy bitmap; lane l takes word (t >> 5) + l
// (+ 32 i), so no word has two writers.
__device__ __forceinline__ void commit_busy(uint32_t *bm, int t, int e, int lane) {
    for (int w = (t >> 5) + lane; w <= ((e - 1) >> 5); w += 32) {
        const int lo = max(t - 32 * w, 0), hi = min(e - 32 * w, 32);
        const uint32_t hm = hi >= 32 ? 0xFFFFFFFFu : ((1u << hi) - 1u);
        bm[w] |= hm & ~((1u << lo) - 1u);
    }
}

// Machine choice for one op among the lanes m < os of a stage, each holding its machine's
// availability t0 (slots past RS; INT_MAX elsewhere) and power q2.  Returns the
// lexicographic minimum of (earliest power-feasible start, machine): the machine that
// frees first is scanned first, another only if it could still start earlier.
// `from`: a start below which the first machine is already known to fail (its scan
// resumes there).
template <bool INS = false>
__device__ __forceinline__ void earliest_machine(const uint16_t *h, int hw, int t0, uint32_t q2, int os,
                                                 int p, int lane, int &best_t, int &best_m, uint32_t &best_q2,
                                                 const uint32_t *busy = nullptr, int words = 0, int from = 0) {
    const unsigned key = lane < os ? ((unsigned)t0 << 5) | (unsigned)lane : 0xFFFFFFFFu;
    const unsigned kmin = __reduce_min_sync(kFull, key);
    best_m = (int)(kmin & 31u);
    best_q2 = __shfl_sync(kFull, q2, best_m);
    best_t = earliest_start<INS>(h, hw, max((int)(kmin >> 5), from), p, best_q2, INT_MAX, lane,
                                 busy + (size_t)best_m * words, words);
    // if the first machine starts as soon as it frees, no machine can start earlier (every
    // other one frees no sooner, and equal times lose to its lower index)
    if (best_t == (int)(kmin >> 5)) return;
    unsigned cand = __ballot_sync(kFull, lane < os && lane != best_m && t0 < best_t + (lane < best_m));
    while (cand) {
        const int m = __ffs(cand) - 1;
        cand &= cand - 1;
        const int tm = __shfl_sync(kFull, t0, m);
        const int lim = best_t + (m < best_m ? 1 : 0);
        if (tm >= lim) continue;
        const uint32_t qm = __shfl_sync(kFull, q2, m);
        const int t = earliest_start<INS>(h, hw, tm, p, qm, lim, lane, busy + (size_t)m * words, words);
        if (t < lim) {
            best_t = t;
            best_m = m;
            best_q2 = qm;
        }
    }
}

// earliest_machine when the machine that frees first is already known (m0 with start t0m
// and power q0, the lexicographic minimum of (availability, machine)) and its scan may
// resume at `from`.
template <bool WIN = true>
__device__ __forceinline__ void earliest_machine_from(const uint16_t *h, int hw, int t0, uint32_t q2, int os, int p,
                                                      int lane, int m0, int t0m, uint32_t q0, int from, int &best_t,
                                                      int &best_m, uint32_t &best_q2) {
    best_m = m0;
    best_q2 = q0;
    best_t = earliest_start<false, WIN>(h, hw, max(t0m, from), p, q0, INT_MAX, lane);
    if (best_t == t0m) return;  // as in earliest_machine: nothing starts earlier
    unsigned cand = __ballot_sync(kFull, lane < os && lane != best_m && t0 < best_t + (lane < best_m));
    while (cand) {
        const int m = __ffs(cand) - 1;
        cand &= cand - 1;
        const int tm = __shfl_sync(kFull, t0, m);
        const int lim = best_t + (m < best_m ? 1 : 0);
        if (tm >= lim) continue;
        const uint32_t qm = __shfl_sync(kFull, q2, m);
        const int t = earliest_start<false, WIN>(h, hw, tm, p, qm, lim, lane);
        if (t < lim) {
            best_t = t;
            best_m = m;
            best_q2 = qm;
        }
    }
}

// One op of the stage-order loop on a profile initialised up to Hcap, after the one-step
// check of its first candidate failed: the general search from the machine that frees
// first (m0, starting at t0m with power q0), resuming at `from`, and the draw.  mf (the
// lane's machine availability) and hw follow.  Returns the op's end, or -1 when it would
// outgrow the slice.
__device__ __forceinline__ int place_general(uint16_t *h, int &hw, int Hcap, int est, int &mf, uint32_t q2, int os,
                                             int p, int lane, int m0, int t0m, uint32_t q0, int from, int &bt,
                                             int &bm) {
    uint32_t bq2;
    earliest_machine_from<false>(h, hw, lane < os ? max(est, mf) : INT_MAX, q2, os, p, lane, m0, t0m, q0, from, bt,
                                 bm, bq2);
    const int e = bt + p;
    if (e > Hcap) return -1;
    commit_power_full(h, bt, e, bq2, lane);
    if (lane == bm) mf = e;
    hw = max(hw, e);
    return e;
}

// One op from the true machine state: the machine that frees first (lowest index on
// ties), its one-step check and draw, else the general search.  As place_general.
__device__ __forceinline__ int place_single(uint16_t *h, int &hw, int Hcap, int est, int &mf, uint32_t q2, int os,
                                            int p, int lane, int &bt, int &bm) {
    const unsigned k = __reduce_min_sync(kFull, ((unsigned)max(est, mf) << 5) | (unsigned)lane);
    const int t0 = (int)(k >> 5), m0 = (int)(k & 31u);
    const uint32_t q0 = __shfl_sync(kFull, q2, m0);
    bool placed = false;
    int from = t0;
    if (t0 + p <= Hcap) from = place_first(h, t0, p, q0, lane, placed, Hcap);
    if (!placed) return place_general(h, hw, Hcap, est, mf, q2, os, p, lane, m0, t0, q0, from, bt, bm);
    bt = t0;
    bm = m0;
    if (lane == m0) mf = t0 + p;
    hw = max(hw, t0 + p);
    return t0 + p;
}

// Unrelated machines, after the one-step check failed: the general search over the stage's
// machines (lane m: availability mf, this op's time pl and power ql on machine m), and the
// draw.  Returns the op's end (-1 when it would outgrow the slice); bp: its time there.
template <bool INS = false>
__device__ __forceinline__ void earliest_machine_u(const uint16_t *h, int hw, int t0, uint32_t q2, int p, int os,
                                                   int lane, int &best_t, int &best_m, int &best_p,
                                                   const uint32_t *busy = nullptr, int words = 0);
__device__ __forceinline__ int place_general_u(uint16_t *h, int &hw, int Hcap, int est, int &mf, int pl,
                                               uint32_t ql, int os, int lane, int &bt, int &bm, int &bp) {
    earliest_machine_u<false>(h, hw, max(est, mf), ql, pl, os, lane, bt, bm, bp);
    const int e = bt + bp;
    if (e > Hcap) return -1;
    commit_power_full(h, bt, e, __shfl_sync(kFull, ql, bm), lane);
    if (lane == bm) mf = e;
    hw = max(hw, e);
    return e;
}

// Unrelated machines, from the true machine state: the machine whose completion bound is
// lowest (lowest index on ties), its one-step check and draw, else the general search.
__device__ __forceinline__ int place_single_u(uint16_t *h, int &hw, int Hcap, int est, int &mf, int pl, uint32_t ql,
                                              int os, int lane, int &bt, int &bm, int &bp) {
    const int tl = max(est, mf);
    const unsigned k = __reduce_min_sync(kFull, lane < os ? ((unsigned)(tl + pl) << 5) | (unsigned)lane : 0xFFFFFFFFu);
    const int m0 = (int)(k & 31u), p0 = __shfl_sync(kFull, pl, m0), t0 = (int)(k >> 5) - p0;
    const uint32_t q0 = __shfl_sync(kFull, ql, m0);
    bool placed = false;
    if (t0 + p0 <= Hcap) place_first(h, t0, p0, q0, lane, placed, Hcap);
    if (!placed) return place_general_u(h, hw, Hcap, est, mf, pl, ql, os, lane, bt, bm, bp);
    bt = t0;
    bm = m0;
    bp = p0;
    if (lane == m0) mf = t0 + p0;
    hw = max(hw, t0 + p0);
    return t0 + p0;
}

// Unrelated machines: lane m < os holds its machine's availability t0, power q2 and the
// op's processing time p on it.  Returns the lexicographic minimum of (earliest completion
// of a power-feasible start, machine) and that machine's p.  The machine whose completion
// bound t0 + p is lowest is scanned first; another only if its bound could still win.
template <bool INS>
__device__ __forceinline__ void earliest_machine_u(const uint16_t *h, int hw, int t0, uint32_t q2, int p, int os,
                                                   int lane, int &best_t, int &best_m, int &best_p,
                                                   const uint32_t *busy, int words) {
    const int c0 = lane < os ? t0 + p : INT_MAX;
    const unsigned key = lane < os ? ((unsigned)c0 << 5) | (unsigned)lane : 0xFFFFFFFFu;
    const unsigned kmin = __reduce_min_sync(kFull, key);
    best_m = (int)(kmin & 31u);
    best_p = __shfl_sync(kFull, p, best_m);
    best_t = earliest_start<INS>(h, hw, __shfl_sync(kFull, t0, best_m), best_p, __shfl_sync(kFull, q2, best_m),
                                 INT_MAX, lane, busy + (size_t)best_m * words, words);
    int best_c = best_t + best_p;
    if (best_c == (int)(kmin >> 5)) return;  // the completion bound itself: nothing beats it
    unsigned cand = __ballot_sync(kFull, lane < os && lane != best_m && c0 < best_c + (lane < best_m));
    while (cand) {
        const int m = __ffs(cand) - 1;
        cand &= cand - 1;
        const int tm = __shfl_sync(kFull, t0, m), pm = __shfl_sync(kFull, p, m);
        const int lim = best_c - pm + (m < best_m ? 1 : 0);  // starts below this complete earlier
        if (tm >= lim) continue;
        const int t = earliest_start<INS>(h, hw, tm, pm, __shfl_sync(kFull, q2, m), lim, lane,
                                          busy + (size_t)m * words, words);
        if (t < lim) {
            best_t = t;
            best_m = m;
            best_p = pm;
            best_c = t + pm;
        }
    }
}

// Decodes one chromosome with the whole warp (Sec. 4.3, Alg. 1-2).  State lives in the
// caller's workspace: h [Hcap] headroom, C [N], mfree [M], inv [K+N], y [K], x [K].  In
// stage order the priority list overwrites y once its inverse is built, so y must be a
// scratch copy.  Schedule output (S_out/M_out, [N*g]) is written for free ops only when
// non-null.
//
// C[j] (kept relative to RS) starts at the end of the job's frozen prefix, raised to R_j
// when the job still has free ops, so every op becomes available at RS + max(0, C[j]).
//
// FULL (shared-memory slices): the whole slice is filled first (the executing ops'
// profile, then Qmax).  Otherwise (global profiles of the full bound, too large to fill per
// decode) a fill mark runs ahead of every op's window and commit, so a decode initialises
// only the slots its schedule reaches.  Either way scans, the one-step check and commits
// read only initialised slots.
// PIPE selects the software-pipelined placement loop for identical machines (for kernels
// whose schedulers hold few warps, bound by each warp's dependency chain); without it the
// loop does less work per op (for kernels bound by issue slots).
template <int ORDER, int MACH, bool FULL = false, bool PIPE = true>
__device__ DecodeOut decode_warp(const Tabs &T, uint16_t *h, int Hcap, int32_t *C, int32_t *mfree,
                                 int16_t *inv, int16_t *y, const int8_t *x, int32_t *S_out,
                                 int32_t *M_out, int lane) {
    const int N = T.N, K = T.K, g = T.g, RS = T.RS;
    const uint32_t Q2 = (uint32_t)T.Qmax * 0x10001u;

    if (T.E0 > Hcap) return {0, 0, 1};  // executing ops alone outgrow the profile slice
    for (int j = lane; j < N; j += 32) C[j] = (T.gcnt[j] > 0 ? max(T.C0[j], T.R[j]) : T.C0[j]) - RS;
    for (int i = lane; i < T.E0; i += 32) h[i] = T.h0[i];
    int fl = Hcap;  // fill mark: slots below it are initialised
    {                // slots E0 .. Hcap (a multiple of 8) or up to the mark: full headroom
        const uint16_t Qm = (uint16_t)T.Qmax;
        for (int i = T.E0 + lane; i < min(Hcap, (T.E0 + 3) & ~3); i += 32) h[i] = Qm;
        __syncwarp();
        if (FULL) {
            for (int b = ((T.E0 + 3) & ~3) + 4 * lane; b < Hcap; b += 128)
                *reinterpret_cast<uint2 *>(h + b) = make_uint2(Q2, Q2);
            __syncwarp();
        } else {
            fl = min(Hcap, (T.E0 + 3) & ~3);
        }
    }
    // high-water mark: slots at or above it have never been drawn on (full headroom, and no
    // occupancy bits); scans stop there
    int hw = T.E0;
    // Insertion placement: occupancy bitmaps of the current stage's machines after the
    // profile slice (the caller sized it with profile_bytes(Hcap, maxo)).
    constexpr bool INS = mach_insert(MACH) && ORDER == kOrderStage;
    const int words = busy_words(Hcap);
    uint32_t *busy = reinterpret_cast<uint32_t *>(h + Hcap);
    if (INS)
        for (int i = lane; i < T.maxo * words; i += 32) busy[i] = 0u;

    // Validate Y (a permutation of 1..K) and X, and build inv[K - y] = gene.
    for (int i = lane; i < K; i += 32) inv[i] = -1;
    __syncwarp();
    bool bad = false;
    for (int k = lane; k < K; k += 32) {
        const int v = y[k];
        if (v < 1 || v > K) bad = true;
        else inv[FFS_IX(K - v, K)] = (int16_t)k;
        if (mach_gene(MACH)) {
            const int xm = x[k];
            if (xm < 0 || xm >= T.o[T.gstg[k]]) bad = true;
        }
    }
    __syncwarp();
    if (ORDER != kOrderStage) {
        for (int i = lane; i < K; i += 32)
            if (inv[i] < 0) bad = true;
        if (__any_sync(kFull, bad)) return {0, 0, 2};
    }

    if (ORDER == kOrderStage) {
        // Z: stage by stage, y descending.  One pass over inv in priority order sends each
        // gene to order[next[s]++] of its stage s: lanes of a chunk with the same stage
        // take consecutive places in lane order, and the group's last lane advances next[s]
        // (kept in the mfree scratch, which stage order does not use).  y is no longer
        // needed; a hole left in inv marks a chromosome that is no permutation.
        int16_t *order = y;
        int32_t *next = mfree;
        for (int s = lane; s < g; s += 32) next[s] = T.soff[s];
        __syncwarp();
        for (int base = 0; base < K; base += 32) {
            const int i = base + lane;
            const int k = i < K ? inv[i] : -1;
            if (i < K && k < 0) bad = true;
            const int s = k >= 0 ? (int)T.gstg[k] : -1;
            const unsigned grp = __match_any_sync(kFull, s);
            int at = 0;
            if (k >= 0) at = next[s] + __popc(grp & ((1u << lane) - 1u));
            __syncwarp();  // every lane has read next[s] before the group's last lane moves it
            if (k >= 0) {
                order[FFS_IX(at, K)] = (int16_t)k;
                if (lane == 31 - __clz(grp)) next[FFS_IX(s, g)] = at + 1;
            }
            __syncwarp();
        }
        if (__any_sync(kFull, bad)) return {0, 0, 2};
        // Identical machines, earliest start, prefilled shared-memory profile (the common
        // case): ops are placed G = kPlaceGroup at a time.  The group's first op's machine
        // and first candidate start are known on entry; each later op's are chosen (one
        // reduction) as if the ops before it in the group were placed at theirs, and the
        // next group's first op's as if all were.  Every window of the group is loaded
        // before any is drawn on, each with the earlier ops' draws subtracted where they
        // overlap, so the one-step checks and the reductions are in flight together.  When
        // every check passes the words are stored in order (a later op's words include the
        // earlier draws).  Otherwise the ops before the first failure are placed as checked,
        // the failing one takes the general search from its machine, past its last slot
        // short of headroom, and the rest are placed one at a time from the true machine
        // state; the next group's first machine is then chosen again.
        if (MACH == kMachEarliest && PIPE && FULL) {
            constexpr int G = kPlaceGroup;
            for (int s = 0; s < g; ++s) {
                const int lo = T.soff[s], hi = T.soff[s + 1];
                if (lo == hi) continue;
                const int mo = T.moff[s], os = T.o[s];
                constexpr int kNever = 0x07FFFFFF;  // lanes past the stage's machines never win
                int mf = kNever;
                uint32_t q2 = 0;
                if (lane < os) {
                    mf = T.mfree0[mo + lane] - RS;
                    q2 = (uint32_t)T.q[mo + lane] * 0x10001u;
                }
                // records of ops n .. n+G (this group and the next group's first op), and the
                // job completions before them
                uint2 gr[G + 1];
                int cj[G + 1];
#pragma unroll
                for (int u = 0; u <= G; ++u) {
                    gr[u] = T.grec[FFS_IX(order[FFS_IX(min(lo + u, hi - 1), K)], K)];
                    cj[u] = C[FFS_IX((int)(gr[u].x & 0xFFFFu), N)];
                }
                int est0 = max(cj[0], 0);
                const unsigned k0 = __reduce_min_sync(kFull, ((unsigned)max(est0, mf) << 5) | (unsigned)lane);
                int ct0 = (int)(k0 >> 5), cm0 = (int)(k0 & 31u);
                uint32_t cq0 = __shfl_sync(kFull, q2, cm0);
                int n = lo;
#pragma unroll 2
                for (; n + G - 1 < hi; n += G) {
                    int ct[G + 1], cm[G + 1], est[G + 1], e[G], cc[G], b[G], p[G], jj[G];
                    uint32_t cq[G + 1];
                    bool one[G], mine[G];
                    uint2 w[G], gn[G];
                    ct[0] = ct0;
                    cm[0] = cm0;
                    cq[0] = cq0;
                    est[0] = est0;
                    int mfc = mf;  // the machines as if ops 0 .. u of the group are placed
#pragma unroll
                    for (int u = 0; u < G; ++u) {
                        jj[u] = (int)(gr[u].x & 0xFFFFu);
                        p[u] = (int)(gr[u].y & 0xFFFFu);
                        e[u] = ct[u] + p[u];
                        cc[u] = ct[u] & ~3;
                        b[u] = cc[u] + 4 * lane;
                        one[u] = e[u] <= Hcap && e[u] - cc[u] <= 128;
                        mine[u] = one[u] && b[u] < e[u];
                        w[u] = make_uint2(0u, 0u);
                        if (mine[u]) w[u] = *reinterpret_cast<const uint2 *>(h + FFS_IX(b[u], Hcap - 3));
                        mfc = lane == cm[u] ? e[u] : mfc;
                        est[u + 1] = max(cj[u + 1], 0);
                        const unsigned k = __reduce_min_sync(kFull, ((unsigned)max(est[u + 1], mfc) << 5) | (unsigned)lane);
                        gn[u] = T.grec[FFS_IX(order[FFS_IX(min(n + G + 1 + u, hi - 1), K)], K)];
                        ct[u + 1] = (int)(k >> 5);
                        cm[u + 1] = (int)(k & 31u);
                        cq[u + 1] = __shfl_sync(kFull, q2, cm[u + 1]);
                    }
                    int cjn[G];
#pragma unroll
                    for (int u = 0; u < G; ++u) cjn[u] = C[FFS_IX((int)(gn[u].x & 0xFFFFu), N)];
                    uint2 m[G];
                    uint32_t vx[G], vy[G];
                    unsigned vm[G];
                    bool all = true;
#pragma unroll
                    for (int u = 0; u < G; ++u) {
#pragma unroll
                        for (int v = 0; v < u; ++v) {  // earlier ops' draws where they overlap
                            const uint2 o = slot_mask(b[u], ct[v], e[v]);
                            w[u].x -= cq[v] & o.x;
                            w[u].y -= cq[v] & o.y;
                        }
                        m[u] = slot_mask(b[u], ct[u], e[u]);
                        vx[u] = ~((w[u].x | 0x80008000u) - cq[u]) & m[u].x & 0x80008000u;
                        vy[u] = ~((w[u].y | 0x80008000u) - cq[u]) & m[u].y & 0x80008000u;
                        vm[u] = __ballot_sync(kFull, (vx[u] | vy[u]) != 0u);
                        all = all && one[u] && vm[u] == 0u;
                    }
                    int tt[G], mm[G], ee[G];
                    if (all) {  // every op placed: their words in order (later ones include earlier draws)
#pragma unroll
                        for (int u = 0; u < G; ++u) {
                            if (mine[u]) {
                                w[u].x -= cq[u] & m[u].x;
                                w[u].y -= cq[u] & m[u].y;
                                *reinterpret_cast<uint2 *>(h + FFS_IX(b[u], Hcap - 3)) = w[u];
                            }
                            tt[u] = ct[u];
                            mm[u] = cm[u];
                            ee[u] = e[u];
                            hw = max(hw, e[u]);
                        }
                        mf = mfc;
                    } else {
                        // ops before the first failure placed as checked; the first failure
                        // searched from its machine, past its last slot short of headroom;
                        // the rest one at a time from the true machine state
                        bool placed = true;
#pragma unroll
                        for (int u = 0; u < G; ++u) {
                            if (placed && one[u] && vm[u] == 0u) {
                                if (mine[u]) {
                                    w[u].x -= cq[u] & m[u].x;
                                    w[u].y -= cq[u] & m[u].y;
                                    *reinterpret_cast<uint2 *>(h + FFS_IX(b[u], Hcap - 3)) = w[u];
                                }
                                if (lane == cm[u]) mf = e[u];
                                hw = max(hw, e[u]);
                                tt[u] = ct[u];
                                mm[u] = cm[u];
                                ee[u] = e[u];
                            } else if (placed) {
                                int from = ct[u];
                                if (one[u]) {
                                    const int l = 31 - __clz(vm[u]);
                                    const int li = vy[u] ? 2 + (int)(vy[u] >> 31) : (int)(vx[u] >> 31);
                                    from = cc[u] + 4 * l + __shfl_sync(kFull, li, l) + 1;
                                }
                                ee[u] = place_general(h, hw, Hcap, est[u], mf, q2, os, p[u], lane, cm[u], ct[u], cq[u],
                                                      from, tt[u], mm[u]);
                                if (ee[u] < 0) return {0, 0, 1};
                                placed = false;
                            } else {
                                ee[u] = place_single(h, hw, Hcap, est[u], mf, q2, os, p[u], lane, tt[u], mm[u]);
                                if (ee[u] < 0) return {0, 0, 1};
                            }
                        }
                        const unsigned kr = __reduce_min_sync(kFull, ((unsigned)max(est[G], mf) << 5) | (unsigned)lane);
                        ct[G] = (int)(kr >> 5);
                        cm[G] = (int)(kr & 31u);
                        cq[G] = __shfl_sync(kFull, q2, cm[G]);
                    }
#pragma unroll
                    for (int u = 0; u < G; ++u) C[FFS_IX(jj[u], N)] = ee[u];  // every lane stores the same values
                    if (S_out && lane == 0) {
#pragma unroll
                        for (int u = 0; u < G; ++u) {
                            S_out[jj[u] * g + s] = tt[u] + RS;
                            M_out[jj[u] * g + s] = mm[u];
                        }
                    }
                    __syncwarp();
                    gr[0] = gr[G];
                    est0 = est[G];
                    ct0 = ct[G];
                    cm0 = cm[G];
                    cq0 = cq[G];
#pragma unroll
                    for (int u = 0; u < G; ++u) {
                        gr[u + 1] = gn[u];
                        cj[u + 1] = cjn[u];
                    }
                }
                // the stage's last ops when its count is not a multiple of G
#pragma unroll
                for (int u = 0; u + 1 < G; ++u) {
                    if (n + u < hi) {
                        const int ju = FFS_IX((int)(gr[u].x & 0xFFFFu), N);
                        int tu, mu;
                        const int e1 = place_single(h, hw, Hcap, u ? max(cj[u], 0) : est0, mf, q2, os,
                                                    (int)(gr[u].y & 0xFFFFu), lane, tu, mu);
                        if (e1 < 0) return {0, 0, 1};
                        C[ju] = e1;
                        if (S_out && lane == 0) {
                            S_out[ju * g + s] = tu + RS;
                            M_out[ju * g + s] = mu;
                        }
                        __syncwarp();
                    }
                }
            }
        } else
        // Unrelated machines, earliest completion, prefilled shared-memory profile: the same
        // grouped placement, where each op's time and power differ per machine (lane m
        // holds its machine's word p | q << 16 of the op) and the machine whose completion
        // bound is lowest is checked first.
        if (MACH == kMachEarliestU && PIPE && FULL) {
            constexpr int G = kPlaceGroup;
            for (int s = 0; s < g; ++s) {
                const int lo = T.soff[s], hi = T.soff[s + 1];
                if (lo == hi) continue;
                const int mo = T.moff[s], os = T.o[s];
                constexpr int kNever = 0x07FFFFFF;  // lanes past the stage's machines never win
                int mf = kNever;
                if (lane < os) mf = T.mfree0[mo + lane] - RS;
                // the machine an op would take next (the lowest completion bound, lowest index
                // on ties) given the machines' availability mv and the op's words pqv: its
                // start, machine, power and time there
                auto choose = [&](int est, int mv, uint32_t pqv, int &ct, int &cm, uint32_t &cq, int &pc) {
                    const int pl = (int)(pqv & 0xFFFFu);
                    const unsigned k = __reduce_min_sync(
                        kFull, lane < os ? ((unsigned)(max(est, mv) + pl) << 5) | (unsigned)lane : 0xFFFFFFFFu);
                    cm = (int)(k & 31u);
                    pc = __shfl_sync(kFull, pl, cm);
                    ct = (int)(k >> 5) - pc;
                    cq = __shfl_sync(kFull, (pqv >> 16) * 0x10001u, cm);
                };
                // this lane's machine word of gene k
                auto mword = [&](int k) -> uint32_t {
                    return lane < os ? T.gm[(size_t)FFS_IX(k, K) * T.maxo + lane] : 0u;
                };
                // records of ops n .. n+G (this group and the next group's first op), and the
                // job completions before them
                uint2 gr[G + 1];
                int cj[G + 1];
                uint32_t pq[G + 1];
#pragma unroll
                for (int u = 0; u <= G; ++u) {
                    const int ku = order[FFS_IX(min(lo + u, hi - 1), K)];
                    gr[u] = T.grec[FFS_IX(ku, K)];
                    pq[u] = mword(ku);
                    cj[u] = C[FFS_IX((int)(gr[u].x & 0xFFFFu), N)];
                }
                int est0 = max(cj[0], 0);
                int ct0, cm0, pc0 = 0;
                uint32_t cq0;
                choose(est0, mf, pq[0], ct0, cm0, cq0, pc0);
                int n = lo;
#pragma unroll 2
                for (; n + G - 1 < hi; n += G) {
                    int ct[G + 1], cm[G + 1], est[G + 1], pc[G + 1], e[G], cc[G], b[G], p[G], jj[G];
                    uint32_t cq[G + 1], pqn[G];
                    bool one[G], mine[G];
                    uint2 w[G], gn[G];
                    ct[0] = ct0;
                    cm[0] = cm0;
                    cq[0] = cq0;
                    pc[0] = pc0;
                    est[0] = est0;
                    int mfc = mf;  // the machines as if ops 0 .. u of the group are placed
#pragma unroll
                    for (int u = 0; u < G; ++u) {
                        jj[u] = (int)(gr[u].x & 0xFFFFu);
                        p[u] = pc[u];
                        e[u] = ct[u] + p[u];
                        cc[u] = ct[u] & ~3;
                        b[u] = cc[u] + 4 * lane;
                        one[u] = e[u] <= Hcap && e[u] - cc[u] <= 128;
                        mine[u] = one[u] && b[u] < e[u];
                        w[u] = make_uint2(0u, 0u);
                        if (mine[u]) w[u] = *reinterpret_cast<const uint2 *>(h + FFS_IX(b[u], Hcap - 3));
                        mfc = lane == cm[u] ? e[u] : mfc;
                        est[u + 1] = max(cj[u + 1], 0);
                        choose(est[u + 1], mfc, pq[u + 1], ct[u + 1], cm[u + 1], cq[u + 1], pc[u + 1]);
                        const int kn = order[FFS_IX(min(n + G + 1 + u, hi - 1), K)];
                        gn[u] = T.grec[FFS_IX(kn, K)];
                        pqn[u] = mword(kn);
                    }
                    int cjn[G];
#pragma unroll
                    for (int u = 0; u < G; ++u) cjn[u] = C[FFS_IX((int)(gn[u].x & 0xFFFFu), N)];
                    uint2 m[G];
                    uint32_t vx[G], vy[G];
                    unsigned vm[G];
                    bool all = true;
#pragma unroll
                    for (int u = 0; u < G; ++u) {
#pragma unroll
                        for (int v = 0; v < u; ++v) {  // earlier ops' draws where they overlap
                            const uint2 o = slot_mask(b[u], ct[v], e[v]);
                            w[u].x -= cq[v] & o.x;
                            w[u].y -= cq[v] & o.y;
                        }
                        m[u] = slot_mask(b[u], ct[u], e[u]);
                        vx[u] = ~((w[u].x | 0x80008000u) - cq[u]) & m[u].x & 0x80008000u;
                        vy[u] = ~((w[u].y | 0x80008000u) - cq[u]) & m[u].y & 0x80008000u;
                        vm[u] = __ballot_sync(kFull, (vx[u] | vy[u]) != 0u);
                        all = all && one[u] && vm[u] == 0u;
                    }
                    int tt[G], mm[G], ee[G];
                    if (all) {  // every op placed: their words in order (later ones include earlier draws)
#pragma unroll
                        for (int u = 0; u < G; ++u) {
                            if (mine[u]) {
                                w[u].x -= cq[u] & m[u].x;
                                w[u].y -= cq[u] & m[u].y;
                                *reinterpret_cast<uint2 *>(h + FFS_IX(b[u], Hcap - 3)) = w[u];
                            }
                            tt[u] = ct[u];
                            mm[u] = cm[u];
                            ee[u] = e[u];
                            hw = max(hw, e[u]);
                        }
                        mf = mfc;
                    } else {
                        // ops before the first failure placed as checked; the first failure
                        // searched from its machine, past its last slot short of headroom;
                        // the rest one at a time from the true machine state
                        bool placed = true;
#pragma unroll
                        for (int u = 0; u < G; ++u) {
                            if (placed && one[u] && vm[u] == 0u) {
                                if (mine[u]) {
                                    w[u].x -= cq[u] & m[u].x;
                                    w[u].y -= cq[u] & m[u].y;
                                    *reinterpret_cast<uint2 *>(h + FFS_IX(b[u], Hcap - 3)) = w[u];
                                }
                                if (lane == cm[u]) mf = e[u];
                                hw = max(hw, e[u]);
                                tt[u] = ct[u];
                                mm[u] = cm[u];
                                ee[u] = e[u];
                            } else if (placed) {
                                // (the search over every machine starts afresh)
                                int pu;
                                ee[u] = place_general_u(h, hw, Hcap, est[u], mf, (int)(pq[u] & 0xFFFFu),
                                                        (pq[u] >> 16) * 0x10001u, os, lane, tt[u], mm[u], pu);
                                if (ee[u] < 0) return {0, 0, 1};
                                placed = false;
                            } else {
                                int pu;
                                ee[u] = place_single_u(h, hw, Hcap, est[u], mf, (int)(pq[u] & 0xFFFFu),
                                                       (pq[u] >> 16) * 0x10001u, os, lane, tt[u], mm[u], pu);
                                if (ee[u] < 0) return {0, 0, 1};
                            }
                        }
                        choose(est[G], mf, pq[G], ct[G], cm[G], cq[G], pc[G]);
                    }
#pragma unroll
                    for (int u = 0; u < G; ++u) C[FFS_IX(jj[u], N)] = ee[u];  // every lane stores the same values
                    if (S_out && lane == 0) {
#pragma unroll
                        for (int u = 0; u < G; ++u) {
                            S_out[jj[u] * g + s] = tt[u] + RS;
                            M_out[jj[u] * g + s] = mm[u];
                        }
                    }
                    __syncwarp();
                    gr[0] = gr[G];
                    pq[0] = pq[G];
                    est0 = est[G];
                    ct0 = ct[G];
                    cm0 = cm[G];
                    cq0 = cq[G];
                    pc0 = pc[G];
#pragma unroll
                    for (int u = 0; u < G; ++u) {
                        gr[u + 1] = gn[u];
                        pq[u + 1] = pqn[u];
                        cj[u + 1] = cjn[u];
                    }
                }
                // the stage's last ops when its count is not a multiple of G
#pragma unroll
                for (int u = 0; u + 1 < G; ++u) {
                    if (n + u < hi) {
                        const int ju = FFS_IX((int)(gr[u].x & 0xFFFFu), N);
                        int tu, mu, pu;
                        const int eu = u ? max(cj[u], 0) : est0;
                        const int e1 = place_single_u(h, hw, Hcap, eu, mf, (int)(pq[u] & 0xFFFFu),
                                                      (pq[u] >> 16) * 0x10001u, os, lane, tu, mu, pu);
                        if (e1 < 0) return {0, 0, 1};
                        C[ju] = e1;
                        if (S_out && lane == 0) {
                            S_out[ju * g + s] = tu + RS;
                            M_out[ju * g + s] = mu;
                        }
                        __syncwarp();
                    }
                }
            }
        } else
        // Identical machines, earliest start, profile filled on demand: a software
        // pipeline.  While op n's window is loaded, checked and voted on, the
        // machine of op n+1 is chosen as if op n were placed at its first candidate start
        // (the one-step case, which most ops take); when op n needs the general search
        // instead, op n+1 is chosen again from the true machine state.  The statements
        // are ordered so that op n's load and op n+1's reduction are in flight together.
        if (MACH == kMachEarliest && PIPE) {
            for (int s = 0; s < g; ++s) {
                const int lo = T.soff[s], hi = T.soff[s + 1];
                if (lo == hi) continue;
                const int mo = T.moff[s], os = T.o[s];
                constexpr int kNever = 0x07FFFFFF;
                int mf = kNever;
                uint32_t q2 = 0;
                if (lane < os) {
                    mf = T.mfree0[mo + lane] - RS;
                    q2 = (uint32_t)T.q[mo + lane] * 0x10001u;
                }
                int k = order[lo];
                uint2 gr = T.grec[k];
                int est = max(C[gr.x & 0xFFFFu], 0);
                int kn = order[min(lo + 1, hi - 1)];
                uint2 grn = T.grec[kn];
                int cjn = C[grn.x & 0xFFFFu];
                // op n's machine (the one that frees first, lowest index on ties) and start
                unsigned kmin = __reduce_min_sync(kFull, ((unsigned)max(est, mf) << 5) | (unsigned)lane);
                int ct = (int)(kmin >> 5), cm = (int)(kmin & 31u);
                uint32_t cq = __shfl_sync(kFull, q2, cm);
#pragma unroll 4
                for (int n = lo; n < hi; ++n) {
                    const int j = (int)(gr.x & 0xFFFFu), p = (int)(gr.y & 0xFFFFu);
                    const int e = ct + p, c = ct & ~3, b = c + 4 * lane;
                    const bool one = e <= Hcap && e - c <= 128;  // one 128-slot step suffices
                    if (!FULL && one) fill_to(h, fl, e, Hcap, Q2, lane);
                    const bool mine = one && b < e;
                    uint2 w = make_uint2(0u, 0u);
                    if (mine) w = *reinterpret_cast<const uint2 *>(h + b);  // op n's window
                    // op n+1 as if op n is placed at ct on machine cm
                    const int estn = max(cjn, 0);
                    const int mfs = lane == cm ? e : mf;
                    const unsigned kminn = __reduce_min_sync(kFull, ((unsigned)max(estn, mfs) << 5) | (unsigned)lane);
                    const int kn2 = order[min(n + 2, hi - 1)];
                    const uint2 grn2 = T.grec[kn2];
                    const uint2 m = slot_mask(b, ct, e);
                    int nt = (int)(kminn >> 5), nm = (int)(kminn & 31u);
                    uint32_t nq = __shfl_sync(kFull, q2, nm);
                    const uint32_t vx = ~((w.x | 0x80008000u) - cq) & m.x & 0x80008000u;
                    const uint32_t vy = ~((w.y | 0x80008000u) - cq) & m.y & 0x80008000u;
                    const unsigned vm = __ballot_sync(kFull, (vx | vy) != 0u);
                    const int cjn2 = C[grn2.x & 0xFFFFu];
                    int best_t = ct, best_m = cm, ee = e;
                    if (one && vm == 0u) {  // placed at ct: draw q from the loaded words
                        if (mine) {
                            w.x -= cq & m.x;
                            w.y -= cq & m.y;
                            *reinterpret_cast<uint2 *>(h + b) = w;
                        }
                        mf = mfs;
                    } else {  // the general search, resuming past the last violating slot
                        int from = ct;
                        if (one) {
                            const int l = 31 - __clz(vm);
                            const int li = vy ? 2 + (int)(vy >> 31) : (int)(vx >> 31);
                            from = c + 4 * l + __shfl_sync(kFull, li, l) + 1;
                        }
                        uint32_t bq2;
                        // (few warps per scheduler: the jump scan, whose steps are shorter)
                        earliest_machine_from<false>(h, hw, lane < os ? max(est, mf) : INT_MAX, q2, os, p, lane, cm,
                                                     ct, cq, from, best_t, best_m, bq2);
                        ee = best_t + p;
                        if (ee > Hcap) return {0, 0, 1};
                        if (!FULL) fill_to(h, fl, ee, Hcap, Q2, lane);
                        commit_power_full(h, best_t, ee, bq2, lane);
                        if (lane == best_m) mf = ee;
                        // op n+1 from the true machine state
                        const unsigned kr = __reduce_min_sync(kFull, ((unsigned)max(estn, mf) << 5) | (unsigned)lane);
                        nt = (int)(kr >> 5);
                        nm = (int)(kr & 31u);
                        nq = __shfl_sync(kFull, q2, nm);
                    }
                    hw = max(hw, ee);
                    C[j] = ee;  // every lane stores the same value
                    if (S_out && lane == 0) {
                        S_out[j * g + s] = best_t + RS;
                        M_out[j * g + s] = best_m;
                    }
                    __syncwarp();
                    gr = grn;
                    est = estn;
                    ct = nt;
                    cm = nm;
                    cq = nq;
                    grn = grn2;
                    cjn = cjn2;
                }
            }
        } else
        // Place the ops; the stage's machines live in lanes (availability, power).
        for (int s = 0; s < g; ++s) {
            const int lo = T.soff[s], hi = T.soff[s + 1];
            if (lo == hi) continue;
            const int mo = T.moff[s], os = T.o[s];
            if (INS) {  // every bit set so far lies below hw
                __syncwarp();
                const int hwords = busy_words(hw);
                for (int i = lane; i < os * hwords; i += 32) busy[(i / hwords) * words + i % hwords] = 0u;
                __syncwarp();
            }
            // lane m < os: end of the last op on machine m past RS (with insertion: the end
            // of its frozen ops, before which it stays unavailable)
            // (lanes past the stage's machines hold an availability no machine reaches, so
            // their keys below lose without a lane test)
            constexpr int kNever = 0x07FFFFFF;
            int mf = kNever;
            uint32_t q2 = 0;
            if (lane < os) {
                mf = T.mfree0[mo + lane] - RS;
                q2 = (uint32_t)T.q[mo + lane] * 0x10001u;
            }
            // software pipeline: the next op's record and job completion are loaded early
            // (within a stage every job appears once, so C of the next job is final)
            int k = order[lo];
            uint2 gr = T.grec[k];
            int cj = C[gr.x & 0xFFFFu];
            for (int n = lo; n < hi; ++n) {
                const int kn = order[min(n + 1, hi - 1)];
                const uint2 grn = T.grec[kn];
                const int cjn = C[grn.x & 0xFFFFu];
                const int j = (int)(gr.x & 0xFFFFu);
                int p = (int)(gr.y & 0xFFFFu);
                uint32_t qo2 = q2;  // this op's power on the lane's machine
                if (mach_unrel(MACH)) {
                    const uint32_t pq = lane < os ? T.gm[(size_t)k * T.maxo + lane] : 0u;
                    p = (int)(pq & 0xFFFFu);
                    qo2 = (pq >> 16) * 0x10001u;
                }
                const int est = max(cj, 0);
                int best_t, best_m;
                uint32_t bq2;
                // fast path (append placement): the first candidate start is feasible and
                // the op is drawn in the same step
                constexpr bool kFast = !INS;
                bool placed = false;
                if (mach_gene(MACH)) {
                    best_m = x[k];
                    if (mach_unrel(MACH)) p = __shfl_sync(kFull, p, best_m);
                    bq2 = __shfl_sync(kFull, qo2, best_m);
                    const int t0 = max(est, __shfl_sync(kFull, mf, best_m));
                    int from = t0;
                    if (kFast && t0 + p <= Hcap) {
                        if (!FULL) fill_to(h, fl, t0 + p, Hcap, Q2, lane);
                        from = place_first(h, t0, p, bq2, lane, placed, Hcap);
                    }
                    if (placed)
                        best_t = t0;
                    else
                        best_t = earliest_start<INS>(h, hw, from, p, bq2, INT_MAX, lane, busy + (size_t)best_m * words,
                                                     words);
                } else if (mach_unrel(MACH)) {
                    if (kFast) {  // the machine whose completion bound is lowest (lowest index on ties):
                                  // starting as soon as it frees, nothing completes earlier
                        const int tl = max(est, mf);
                        const unsigned key =
                            lane < os ? ((unsigned)(tl + p) << 5) | (unsigned)lane : 0xFFFFFFFFu;
                        const unsigned kmin = __reduce_min_sync(kFull, key);
                        best_m = (int)(kmin & 31u);
                        const int t0 = __shfl_sync(kFull, tl, best_m), pb = __shfl_sync(kFull, p, best_m);
                        bq2 = __shfl_sync(kFull, qo2, best_m);
                        if (t0 + pb <= Hcap) {
                            if (!FULL) fill_to(h, fl, t0 + pb, Hcap, Q2, lane);
                            place_first(h, t0, pb, bq2, lane, placed, Hcap);
                        }
                        if (placed) {
                            best_t = t0;
                            p = pb;
                        }
                    }
                    if (!placed) {
                        earliest_machine_u<INS>(h, hw, max(est, mf), qo2, p, os, lane, best_t, best_m, p, busy, words);
                        bq2 = __shfl_sync(kFull, qo2, best_m);
                    }
                } else {
                    const int tl = lane < os ? max(est, mf) : INT_MAX;
                    int from = 0;
                    if (INS && !mach_unrel(MACH)) {  // every machine available first, checked at once
                        const unsigned kmin = __reduce_min_sync(kFull, ((unsigned)max(est, mf) << 5) | (unsigned)lane);
                        const int t0 = (int)(kmin >> 5);
                        if (t0 + p <= Hcap) {
                            if (!FULL) fill_to(h, fl, t0 + p, Hcap, Q2, lane);
                            const int bm = place_first_ins(h, Hcap, busy, words, t0, p, tl, q2, os, lane);
                            if (bm >= 0) {
                                placed = true;
                                best_t = t0;
                                best_m = bm;
                                bq2 = __shfl_sync(kFull, q2, bm);
                            }
                        }
                    }
                    if (kFast) {  // the machine that frees first (lowest index on ties)
                        const unsigned key = ((unsigned)max(est, mf) << 5) | (unsigned)lane;
                        const unsigned kmin = __reduce_min_sync(kFull, key);
                        const int t0 = (int)(kmin >> 5);
                        best_m = (int)(kmin & 31u);
                        bq2 = __shfl_sync(kFull, q2, best_m);
                        if (t0 + p <= Hcap) {
                            if (!FULL) fill_to(h, fl, t0 + p, Hcap, Q2, lane);
                            from = place_first(h, t0, p, bq2, lane, placed, Hcap);
                        }
                        if (placed) best_t = t0;
                    }
                    if (!placed)
                        earliest_machine<INS>(h, hw, tl, q2, os, p, lane, best_t, best_m, bq2, busy, words, from);
                }
                const int e = best_t + p;
                if (placed) {
                    hw = max(hw, e);
                } else if (e > Hcap) {
                    return {0, 0, 1};
                } else {
                    if (!FULL) fill_to(h, fl, e, Hcap, Q2, lane);
                    commit_power_full(h, best_t, e, bq2, lane);
                    hw = max(hw, e);
                }
                if (INS) commit_busy(busy + (size_t)best_m * words, best_t, e, lane);
                else if (lane == best_m) mf = e;
                if (lane == 0) {
                    C[j] = e;
                    if (S_out) {
                        S_out[j * g + s] = best_t + RS;
                        M_out[j * g + s] = best_m;
                    }
                }
                __syncwarp();
                k = kn;
                gr = grn;
                cj = cjn;
            }
        }
    } else {
        // Alg. 1 read as a topological order: the ready job head with the largest y.
        int16_t *nxt = inv + K;
        for (int j = lane; j < N; j += 32) nxt[j] = T.gfirst[j];
        for (int m = lane; m < T.M; m += 32) mfree[m] = T.mfree0[m];
        __syncwarp();
        for (int n = 0; n < K; ++n) {
            unsigned kmax = 0;  // (y << 15 | job) of the best ready job head
            for (int j = lane; j < N; j += 32) {
                const int k = nxt[j];
                if (k >= 0 && k < T.gfirst[j] + T.gcnt[j]) kmax = max(kmax, ((unsigned)y[k] << 15) | (unsigned)j);
            }
            const int bestj = (int)(__reduce_max_sync(kFull, kmax) & 0x7FFFu);
            const int k = nxt[bestj];
            const uint2 gr = T.grec[k];
            const int j = (int)(gr.x & 0xFFFFu), s = (int)((gr.x >> 16) & 0xFFu), os = (int)(gr.x >> 24);
            int p = (int)(gr.y & 0xFFFFu);
            const int mo = (int)(gr.y >> 16);
            int mf = INT_MAX;
            uint32_t q2 = 0;
            if (lane < os) {
                mf = mfree[mo + lane] - RS;
                q2 = (uint32_t)T.q[mo + lane] * 0x10001u;
            }
            if (mach_unrel(MACH)) {
                const uint32_t pq = lane < os ? T.gm[(size_t)k * T.maxo + lane] : 0u;
                p = (int)(pq & 0xFFFFu);
                q2 = (pq >> 16) * 0x10001u;
            }
            const int est = max(C[j], 0);
            int best_t, best_m;
            if (mach_gene(MACH)) {
                best_m = x[k];
                if (mach_unrel(MACH)) p = __shfl_sync(kFull, p, best_m);
                best_t = earliest_start(h, hw, max(est, __shfl_sync(kFull, mf, best_m)), p,
                                        __shfl_sync(kFull, q2, best_m), INT_MAX, lane);
            } else if (mach_unrel(MACH)) {
                earliest_machine_u(h, hw, max(est, mf), q2, p, os, lane, best_t, best_m, p);
            } else {
                uint32_t bq2_unused;
                earliest_machine(h, hw, lane < os ? max(est, mf) : INT_MAX, q2, os, p, lane, best_t, best_m,
                                 bq2_unused);
            }
            const int e = best_t + p;
            if (e > Hcap) return {0, 0, 1};
            const uint32_t bq2 = __shfl_sync(kFull, q2, best_m);
            if (!FULL) fill_to(h, fl, e, Hcap, Q2, lane);
            commit_power_full(h, best_t, e, bq2, lane);
            hw = max(hw, e);
            __syncwarp();
            if (lane == 0) {
                nxt[bestj] = (int16_t)(k + 1);
                mfree[mo + best_m] = e + RS;
                C[j] = e;
                if (S_out) {
                    S_out[j * g + s] = best_t + RS;
                    M_out[j * g + s] = best_m;
                }
            }
            __syncwarp();
        }
    }

    // Eq. (2)-(3) over every job, frozen ones included.
    long long tard = 0;
    int cmax = 0;
    for (int j = lane; j < N; j += 32) {
        const int cj = C[j] + RS;
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

// Surrogate input of one chromosome: f_k = 1 - r_k / n_s, where r_k is gene k's rank (0 =
// highest y) among the n_s genes of its stage.  BF16 bits go to row[0 .. Kpad), zero
// padded; `inv` is K entries of warp scratch.  Values of y outside 1..K are ignored (their
// genes keep 0), so a malformed row cannot index out of bounds.
__device__ __forceinline__ void stage_rank_row(const int16_t *y, int K, int Kpad, const int8_t *gstg,
                                               const int32_t *soff, int g, int16_t *inv, uint16_t *row, int lane) {
    for (int i = lane; i < K; i += 32) inv[i] = -1;
    for (int k = lane; k < Kpad; k += 32) row[k] = 0;
    __syncwarp();
    for (int k = lane; k < K; k += 32) {
        const int v = y[k];
        if (v >= 1 && v <= K) inv[K - v] = (int16_t)k;
    }
    __syncwarp();
    for (int s = 0; s < g; ++s) {
        const int n = soff[s + 1] - soff[s];
        if (n <= 0) continue;
        int pos = 0;
        for (int base = 0; base < K; base += 32) {
            const int i = base + lane;
            const int k = i < K ? inv[i] : -1;
            const bool sel = k >= 0 && gstg[k] == s;
            const unsigned mask = __ballot_sync(kFull, sel);
            if (sel) {
                const int r = pos + __popc(mask & ((1u << lane) - 1u));
                row[k] = __bfloat16_as_ushort(__float2bfloat16_rn(1.f - (float)r / (float)n));
            }
            pos += __popc(mask);
        }
    }
    __syncwarp();
}

}  // namespace edffs
