// ffs_kernels.cu -- EDFFS decode and GA kernels for sm_103a.
//
// Mapping: one warp per chromosome.  A CTA stages the instance tables (processing
// times, powers, releases, due dates, gene map, initial power profile) into shared memory
// with a single bulk copy; each warp then keeps its chromosome, per-job completion times,
// per-machine free times and the power headroom profile of its schedule in its own slice
// of shared memory.  The decoder's inner step scans 32 time slots per ballot.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <climits>
#include <map>
#include <mutex>

#include "ffs_device.cuh"
#include "ffs_ga.cuh"
#include "ffs_kernels.cuh"

namespace edffs {

namespace {

// Views of warp `warp`'s slice after the staged tables.
// With insertion placement the profile slice (shared, or global with gprof) is followed by
// the occupancy bitmaps of up to maxo machines.
__device__ __forceinline__ WarpPtrs warp_ptrs(char *tab, int blob_bytes, const Tabs &T, int Hcap,
                                              bool ga, bool gprof, uint16_t *gscratch, int warp, bool insert = false) {
    const WarpLayout L = warp_layout(T.N, T.M, T.K, gprof ? 0 : Hcap, ga, insert && !gprof ? T.maxo : 0);
    char *ws = tab + ((blob_bytes + 127) & ~127) + warp * L.bytes;
    return warp_view(ws, L, gprof ? gscratch + (size_t)(blockIdx.x * kWarpsPerBlock + warp) *
                                                   gwork_stride(Hcap, T.maxo, insert)
                                  : nullptr);
}

// ---------------------------------------------------------------- decode kernel
// At most 128 registers in this and the other per-warp kernels: no variant spills.
template <int ORDER, int MACH, bool GPROF>
__global__ void __maxnreg__(128) k_decode(DecodeArgs a) {
    extern __shared__ __align__(128) char smem[];
    char *tab = smem + 128;
    if (!stage_tables(tab, a.blob, a.blob_bytes, reinterpret_cast<uint64_t *>(smem), a.err, a.inject_skip != 0,
                      a.wait_iters > 0 ? a.wait_iters : kStageWaitIters))
        return;
    const Tabs T = tabs_view(tab);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const WarpPtrs w = warp_ptrs(tab, a.blob_bytes, T, a.Hcap, false, GPROF, a.gscratch, warp, mach_insert(MACH));
    const int buf = a.gdev ? ((a.gdev->gen + 1) & 1) : 0;
    const int n = a.list ? *a.list_count : a.count;
    const int K = T.K, NG = T.N * T.g;
    for (int c = blockIdx.x * kWarpsPerBlock + warp; c < n; c += gridDim.x * kWarpsPerBlock) {
        const int idx = a.list ? a.list[c] : c;
        const int16_t *yg = a.Y[buf] + (size_t)idx * K;
        for (int k = lane; k < K; k += 32) w.y[k] = yg[k];
        if (mach_gene(MACH)) {
            const int8_t *xg = a.X[buf] + (size_t)idx * K;
            for (int k = lane; k < K; k += 32) w.x[k] = xg[k];
        }
        int32_t *S = a.S ? a.S + (size_t)idx * NG : nullptr;
        int32_t *Mo = a.S ? a.Mo + (size_t)idx * NG : nullptr;
        if (S) {
            for (int i = lane; i < NG; i += 32)
                if (a.status[i] != kStFree) {
                    S[i] = a.S0[i];
                    Mo[i] = a.M0[i];
                }
        }
        __syncwarp();
        const DecodeOut r = decode_warp<ORDER, MACH, !GPROF>(T, w.h, a.Hcap, w.C, w.mfree, w.inv, w.y, w.x, S, Mo, lane);
        if (lane == 0) {
            if (r.status == 1) {
                if (GPROF) atomicOr(a.err, kErrOverflow);
                else a.over_list[atomicAdd(a.over_count, 1)] = idx;
            } else if (r.status == 2) {
                atomicOr(a.err, kErrBadChromosome);
                a.obj[buf][idx] = -1;
            } else {
                const long long o = (long long)T.WT * r.tard + r.cmax;
                a.obj[buf][idx] = o;
                if (a.tard) a.tard[idx] = r.tard;
                if (a.cmax) a.cmax[idx] = r.cmax;
                if (a.gdev) {
                    const long long f = a.gdev->emax - o;
                    a.fit[buf][idx] = f > 0 ? f : 0;
                }
            }
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------- GA: generation 0
template <int ORDER, int MACH>
__global__ void __maxnreg__(128) k_ga_init(GenArgs a) {
    extern __shared__ __align__(128) char smem[];
    char *tab = smem + 128;
    if (!stage_tables(tab, a.blob, a.blob_bytes, reinterpret_cast<uint64_t *>(smem), a.err)) return;
    const Tabs T = tabs_view(tab);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const WarpPtrs w = warp_ptrs(tab, a.blob_bytes, T, a.Hcap, true, false, nullptr, warp, mach_insert(MACH));
    const int K = T.K;
    for (int i = blockIdx.x * kWarpsPerBlock + warp; i < a.P; i += gridDim.x * kWarpsPerBlock) {
        int16_t *yo = a.Y[0] + (size_t)i * K;
        int8_t *xo = a.X[0] + (size_t)i * K;
        if (a.warm) {
            for (int k = lane; k < K; k += 32) w.y[k] = yo[k];
            if (mach_gene(MACH))
                for (int k = lane; k < K; k += 32) w.x[k] = xo[k];
            __syncwarp();
        } else {
            make_initial<MACH>(T, w, a.seed, a.instance_id, i, lane);
            for (int k = lane; k < K; k += 32) yo[k] = w.y[k];
            if (mach_gene(MACH))
                for (int k = lane; k < K; k += 32) xo[k] = w.x[k];
        }
        const DecodeOut r = decode_warp<ORDER, MACH, true>(T, w.h, a.Hcap, w.C, w.mfree, w.inv, w.y, w.x,
                                                     nullptr, nullptr, lane);
        if (lane == 0) {
            if (r.status == 1) a.over_list[atomicAdd(&a.dev->nover, 1)] = i;
            else if (r.status == 2) atomicOr(a.err, kErrBadChromosome);
            else a.obj[0][i] = (long long)T.WT * r.tard + r.cmax;
        }
        __syncwarp();
    }
}

// Called by every warp after writing its child.  The last warp to finish an island does
// the elitist replacement (Sec. 4.4: the island's best-ever individual overwrites its
// worst child) and, at migration generations, records the island's best and worst; the
// last island to finish performs the single-ring migration (island i's worst <- island
// i-1's best, from those records) and, at the last generation of a chain, advances the
// generation counter (islands count themselves only then or to migrate).  Completion is
// counted with atomics after a device-wide fence; nothing waits.
// Copies in this tail lie on the critical path of a generation (the last island's last
// warp runs them after every decode): 256 genes per chunk, one L2 round trip each.
constexpr int kTailU = 8;

template <typename Args>
__device__ void island_finish(const Args &a, int isl, int nx, int gen, int lane) {
    __threadfence();
    int ticket = 0;
    if (lane == 0) ticket = atomicAdd(a.isl_done + isl, 1);
    ticket = __shfl_sync(kFull, ticket, 0);
    if (ticket != a.I - 1) return;
    __threadfence();
    const int K = a.K;
    int16_t *Y = a.Y[nx];
    int8_t *X = a.X[nx];
    int64_t *obj = a.obj[nx], *fit = a.fit[nx];
    const bool migrate = a.migrate_every > 0 && gen % a.migrate_every == 0 && a.nisl > 1;
    island_replace<kTailU, true>(Y, X, obj, fit, a.bY, a.bX, a.bobj, a.bfit, isl, a.I, K, migrate, a.mY, a.mX, a.mobj,
                           a.mfit, a.mw, lane);
    if (lane == 0) a.isl_done[isl] = 0;
    // within a chain the counter is left as it was; islands meet only to migrate
    if (!a.publish && !migrate) return;
    __threadfence();
    if (lane == 0) ticket = atomicAdd(&a.dev->islands_done, 1);
    ticket = __shfl_sync(kFull, ticket, 0);
    if (ticket != a.nisl - 1) return;
    __threadfence();
    if (migrate) ring_migrate<kTailU>(Y, X, obj, fit, a.mY, a.mX, a.mobj, a.mfit, a.mw, a.nisl, K, lane);
    if (lane == 0) {
        a.dev->islands_done = 0;
        if (a.publish) {
            a.dev->nover = 0;
            __threadfence();
            a.dev->gen = gen;
        }
    }
}

// ---------------------------------------------------------------- GA: one generation
// Selection -> paired crossover + correction -> mutation -> decode, one child per warp.
// Each warp recomputes both parents of its pair from the counter-based stream, so the
// children of a pair are built independently by two warps.  An explicit cap of 168
// registers keeps every variant free of spills.  At that cap the register file holds 3
// CTAs of 128 threads per SM; profile slices of the usual size (112 KB of shared memory per
// CTA) allow 2 anyway.
template <int ORDER, int MACH>
__global__ void __maxnreg__(168) k_ga_generation(GenArgs a) {
    extern __shared__ __align__(128) char smem[];
    char *tab = smem + 128;
    if (!stage_tables(tab, a.blob, a.blob_bytes, reinterpret_cast<uint64_t *>(smem), a.err)) return;
    // Launched as a programmatic dependent, the kernel got here (tables staged, which no
    // generation changes) while the previous generation was draining: wait until it has
    // completed and its writes are visible, then let the next generation be scheduled.
    // Without such a launch both are no-ops.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const Tabs T = tabs_view(tab);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const WarpPtrs w = warp_ptrs(tab, a.blob_bytes, T, a.Hcap, true, false, nullptr, warp, mach_insert(MACH));
    const int K = T.K, I = a.I;
    const int g0 = a.dev->gen + a.gen_ofs;  // generations completed before this one
    const int cur = g0 & 1, nx = cur ^ 1;
    const uint32_t gen = (uint32_t)g0 + 1;
    const long long emax = a.dev->emax;
    const GASrc src{a.Y[cur], a.X[cur], a.fit[cur], a.P, a.I, K, a.tour_k, a.side, a.pc_thr, a.pm_thr, a.seed,
                    a.instance_id, 1};

    for (int i = blockIdx.x * kWarpsPerBlock + warp; i < a.P; i += gridDim.x * kWarpsPerBlock) {
        if (!a.cand_Y) {
            make_child<MACH>(T, w, src, i, gen, lane);
        } else if (a.cand_keep) {  // island top rule: the candidate chosen for this slot
            const size_t c = (size_t)__ldg(a.cand_keep + i);
            for (int k = lane; k < K; k += 32) w.y[k] = a.cand_Y[c * K + k];
            if (mach_gene(MACH))
                for (int k = lane; k < K; k += 32) w.x[k] = a.cand_X[c * K + k];
            for (int k = lane; k < a.Kpad; k += 32) a.kept_Yh[(size_t)i * a.Kpad + k] = a.cand_Yh[c * a.Kpad + k];
            __syncwarp();
        } else {
            // surrogate-assisted: the slot's first candidate decides, as a plain generation
            // would, between a parent's plain copy (kept as it is) and an offspring; a
            // screened offspring slot keeps the offspring with the lowest score among its
            // candidates (ties to the lower index; an undefined score counts as worst), an
            // unscreened one its first candidate
            const bool screen = a.cand_new[i] &&
                                (uint64_t)draw(a.seed, kPScreen, a.instance_id, gen, (uint32_t)i, 0) < a.screen_thr;
            float sc = INFINITY;
            int vi = screen ? INT_MAX : 0;
            // candidate f of slot i is row f P + i
            if (screen && lane < a.F && a.cand_new[(size_t)lane * a.P + i]) {
                sc = a.cand_out[(size_t)lane * a.P + i];
                if (isnan(sc)) sc = INFINITY;
                vi = lane;
            }
#pragma unroll
            for (int off = 16; off; off >>= 1) {
                const float os = __shfl_xor_sync(kFull, sc, off);
                const int ov = __shfl_xor_sync(kFull, vi, off);
                if (os < sc || (os == sc && ov < vi)) {
                    sc = os;
                    vi = ov;
                }
            }
            const size_t c = (size_t)vi * a.P + i;
            for (int k = lane; k < K; k += 32) w.y[k] = a.cand_Y[c * K + k];
            if (mach_gene(MACH))
                for (int k = lane; k < K; k += 32) w.x[k] = a.cand_X[c * K + k];
            for (int k = lane; k < a.Kpad; k += 32) a.kept_Yh[(size_t)i * a.Kpad + k] = a.cand_Yh[c * a.Kpad + k];
            __syncwarp();
        }
        int16_t *yo = a.Y[nx] + (size_t)i * K;
        for (int k = lane; k < K; k += 32) yo[k] = w.y[k];
        if (mach_gene(MACH)) {
            int8_t *xo = a.X[nx] + (size_t)i * K;
            for (int k = lane; k < K; k += 32) xo[k] = w.x[k];
        }
        DecodeOut r{0, 0, 1};
        if (a.Hcap > 0)
            r = decode_warp<ORDER, MACH, true>(T, w.h, a.Hcap, w.C, w.mfree, w.inv, w.y, w.x, nullptr, nullptr, lane);
        if (r.status == 1) {  // the schedule outgrew the shared slice: redo it in global memory
            for (int k = lane; k < K; k += 32) w.y[k] = yo[k];  // the decode reused w.y
            __syncwarp();
            uint16_t *hg = a.gscratch + (size_t)(blockIdx.x * kWarpsPerBlock + warp) *
                                            gwork_stride(a.H, T.maxo, mach_insert(MACH));
            r = decode_warp<ORDER, MACH>(T, hg, a.H, w.C, w.mfree, w.inv, w.y, w.x, nullptr, nullptr, lane);
        }
        if (lane == 0) {
            if (r.status != 0) {
                atomicOr(a.err, r.status == 2 ? kErrBadChromosome : kErrOverflow);
            } else {
                const long long o = (long long)T.WT * r.tard + r.cmax;
                a.obj[nx][i] = o;
                a.fit[nx][i] = emax - o > 0 ? emax - o : 0;
                if (a.kept_obj) a.kept_obj[i] = o;
            }
        }
        island_finish(a, i / I, nx, (int)gen, lane);
    }
}

// ---------------------------------------------------------------- warm start
// One CTA per new row.  Survivor priorities: a bit per old priority value marks the
// values held by genes that survive; the rank of value v among them is a popcount
// prefix, so survivors keep their relative order on top (n_new + rank) and the fresh
// genes take n_new .. 1 in index order.
constexpr int kRemapThreads = 256;
constexpr int kRemapWords = (kMaxK + 32) / 32;

__global__ void __launch_bounds__(kRemapThreads) k_warm_remap(WarmArgs a) {
    __shared__ uint32_t bits[kRemapWords];
    __shared__ int32_t pre[kRemapWords];
    const int nw = (a.Ko + 31) >> 5;
    const int ob = a.odev->gen & 1;
    for (int r = blockIdx.x; r < a.P; r += gridDim.x) {
        const int16_t *yo = a.Yo[ob] + (size_t)(r % a.Po) * a.Ko;
        const int8_t *xo = a.Xo[ob] + (size_t)(r % a.Po) * a.Ko;
        int16_t *y = a.Y + (size_t)r * a.K;
        int8_t *x = a.X + (size_t)r * a.K;
        for (int i = threadIdx.x; i < nw; i += blockDim.x) bits[i] = 0;
        __syncthreads();
        for (int k = threadIdx.x; k < a.Ko; k += blockDim.x) {
            if (a.map[k] < 0) continue;
            const int v = yo[k] - 1;
            if (v < 0 || v >= a.Ko) {
                atomicOr(a.err, kErrBadChromosome);
                continue;
            }
            atomicOr(&bits[v >> 5], 1u << (v & 31));
        }
        __syncthreads();
        if (threadIdx.x < 32) {  // exclusive prefix of the words' popcounts
            const int lane = threadIdx.x, per = (nw + 31) / 32;
            const int lo = min(nw, lane * per), hi = min(nw, lo + per);
            int s = 0;
            for (int i = lo; i < hi; ++i) s += __popc(bits[i]);
            int inc = s;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int t = __shfl_up_sync(kFull, inc, off);
                if (lane >= off) inc += t;
            }
            int run = inc - s;
            for (int i = lo; i < hi; ++i) {
                pre[i] = run;
                run += __popc(bits[i]);
            }
        }
        __syncthreads();
        for (int k = threadIdx.x; k < a.Ko; k += blockDim.x) {
            const int d = a.map[k];
            const int v = yo[k] - 1;
            if (d < 0 || v < 0 || v >= a.Ko) continue;
            const int rank = pre[v >> 5] + __popc(bits[v >> 5] & (0xFFFFFFFFu >> (31 - (v & 31))));
            y[d] = (int16_t)(a.n_new + rank);
            x[d] = xo[k];
        }
        for (int q = threadIdx.x; q < a.n_new; q += blockDim.x) {
            y[a.fresh[q]] = (int16_t)(a.n_new - q);
            x[a.fresh[q]] = 0;
        }
        __syncthreads();  // the next row reuses bits / pre
    }
}

// ---------------------------------------------------------------- surrogate candidates
// Over-generation for the surrogate: candidate c = f P + j is candidate f of population slot
// j, built with the usual operators from its own stream position (candidate 0 is the plain
// generation's child); its model input (the within-stage rank features, BF16, zero padded
// to Kpad) is written beside it.  Nothing is decoded here.
template <int MACH>
__global__ void __maxnreg__(128) k_candidates(GenArgs a) {
    extern __shared__ __align__(128) char smem[];
    char *tab = smem + 128;
    if (!stage_tables(tab, a.blob, a.blob_bytes, reinterpret_cast<uint64_t *>(smem), a.err)) return;
    const Tabs T = tabs_view(tab);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const WarpPtrs w = warp_ptrs(tab, a.blob_bytes, T, 0, true, false, nullptr, warp);
    const int K = T.K, cur = a.dev->gen & 1;
    const uint32_t gen = (uint32_t)a.dev->gen + 1;
    const GASrc src{a.Y[cur], a.X[cur], a.fit[cur], a.P, a.I, K, a.tour_k, a.side, a.pc_thr, a.pm_thr, a.seed,
                    a.instance_id, a.F};
    for (int c = blockIdx.x * kWarpsPerBlock + warp; c < a.P * a.F; c += gridDim.x * kWarpsPerBlock) {
        const bool fresh = make_child<MACH>(T, w, src, c, gen, lane);
        if (lane == 0) a.cand_new[c] = fresh ? 1 : 0;
        int16_t *yo = a.cand_Y + (size_t)c * K;
        for (int k = lane; k < K; k += 32) yo[k] = w.y[k];
        if (mach_gene(MACH)) {
            int8_t *xo = a.cand_X + (size_t)c * K;
            for (int k = lane; k < K; k += 32) xo[k] = w.x[k];
        }
        stage_rank_row(w.y, K, a.Kpad, T.gstg, T.soff, T.g, w.inv, a.cand_Yh + (size_t)c * a.Kpad, lane);
    }
}

// ---------------------------------------------------------------- surrogate: island top rule
// One CTA per island: its n = F I candidate rows get 64-bit keys (score made orderable as
// an unsigned integer, an undefined score ranking last | row), a bitonic sort in shared
// memory puts the I best first, and a block-wide prefix over the kept flags in row order
// gives each kept row its slot.  With is_new (offspring only), a slot whose first candidate
// is a parent's plain copy keeps that copy (the plain GA's copy rate), other copies rank
// last, and the offspring fill the remaining places by score.
constexpr int kTopThreads = 1024;

__device__ __forceinline__ uint32_t orderable(float f) {
    if (isnan(f)) return 0xFFFFFFFFu;
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__global__ void __launch_bounds__(kTopThreads) k_island_top(const float *__restrict__ score,
                                                             const uint8_t *__restrict__ is_new, int P, int F, int I,
                                                             int32_t *__restrict__ keep) {
    __shared__ unsigned long long key[kTopMax];
    __shared__ uint8_t kept[kTopMax];
    __shared__ int wsum[kTopThreads / 32];
    const int lo = blockIdx.x * I, n = F * I;
    int m = 1;
    while (m < n) m <<= 1;
    for (int l = threadIdx.x; l < m; l += blockDim.x) {  // local row l = f I + (j - lo)
        if (l < n) {
            const int f = l / I, j = lo + l % I;
            const size_t row = (size_t)f * P + j;
            unsigned hi = orderable(score[row]);
            if (is_new && !is_new[row]) hi = f == 0 ? 0u : 0xFFFFFFFFu;  // a copy slot keeps its copy; other copies last
            key[l] = ((unsigned long long)hi << 32) | (unsigned)l;
        } else {
            key[l] = ~0ull;  // padding sorts last
        }
        if (l < n) kept[l] = 0;
    }
    __syncthreads();
    for (int size = 2; size <= m; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < m / 2; t += blockDim.x) {
                const int a = 2 * t - (t & (stride - 1)), b = a + stride;
                const bool up = (a & size) == 0;
                const unsigned long long ka = key[a], kb = key[b];
                if ((ka > kb) == up) {
                    key[a] = kb;
                    key[b] = ka;
                }
            }
            __syncthreads();
        }
    for (int r = threadIdx.x; r < I; r += blockDim.x) kept[(int)(key[r] & 0xFFFFFFFFu)] = 1;
    __syncthreads();
    // slot of each kept row: the number of kept rows before it, in row order (chunks of
    // blockDim rows, a warp-shuffle scan within each warp, then across warps)
    int base = 0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c0 = 0; c0 < n; c0 += blockDim.x) {
        const int l = c0 + threadIdx.x;
        const int v = l < n ? kept[l] : 0;
        int inc = v;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int u = __shfl_up_sync(kFull, inc, off);
            if (lane >= off) inc += u;
        }
        if (lane == 31) wsum[wid] = inc;
        __syncthreads();
        int before = base;
        for (int q = 0; q < wid; ++q) before += wsum[q];
        if (v) {
            const int f = l / I, j = lo + l % I;
            keep[lo + before + inc - 1] = f * P + j;
        }
        int tot = 0;
        for (int q = 0; q < nw; ++q) tot += wsum[q];
        __syncthreads();
        base += tot;
    }
}

// ---------------------------------------------------------------- GA: generation 0 bookkeeping
constexpr int kReplThreads = 256;

// Block-wide best (largest fitness, lowest index) and worst (smallest fitness, lowest index).
__device__ void island_extremes(const int64_t *fit, int lo, int n, int &best, int &worst) {
    __shared__ long long sbf[kReplThreads / 32], swf[kReplThreads / 32];
    __shared__ int sbi[kReplThreads / 32], swi[kReplThreads / 32];
    long long bf = LLONG_MIN, wf = LLONG_MAX;
    int bi = INT_MAX, wi = INT_MAX;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const long long f = fit[lo + t];
        if (fitter(f, lo + t, bf, bi)) { bf = f; bi = lo + t; }
        if (f < wf || (f == wf && lo + t < wi)) { wf = f; wi = lo + t; }
    }
    warp_best(bf, bi);
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        const long long of = __shfl_xor_sync(kFull, wf, off);
        const int oi = __shfl_xor_sync(kFull, wi, off);
        if (of < wf || (of == wf && oi < wi)) { wf = of; wi = oi; }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { sbf[warp] = bf; sbi[warp] = bi; swf[warp] = wf; swi[warp] = wi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q) {
            if (fitter(sbf[q], sbi[q], sbf[0], sbi[0])) { sbf[0] = sbf[q]; sbi[0] = sbi[q]; }
            if (swf[q] < swf[0] || (swf[q] == swf[0] && swi[q] < swi[0])) { swf[0] = swf[q]; swi[0] = swi[q]; }
        }
    }
    __syncthreads();
    best = sbi[0];
    worst = swi[0];
    __syncthreads();
}

__device__ void copy_ind(int16_t *yd, int8_t *xd, const int16_t *ys, const int8_t *xs, int K) {
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        yd[k] = ys[k];
        xd[k] = xs[k];
    }
}

// E_max = 10^a, the smallest a >= 1 above every initial objective (Sec. 5); fitness Eq. (13).
__global__ void k_emax(ReplArgs a) {
    __shared__ long long smax[32];
    long long mx = 0;
    for (int i = threadIdx.x; i < a.P; i += blockDim.x) mx = max(mx, (long long)a.obj[0][i]);
#pragma unroll
    for (int off = 16; off; off >>= 1) mx = max(mx, __shfl_xor_sync(kFull, mx, off));
    if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q) mx = max(mx, smax[q]);
        long long e = 10;
        while (e <= mx) e *= 10;
        a.dev->emax = e;
        smax[0] = e;
    }
    __syncthreads();
    const long long e = smax[0];
    for (int i = threadIdx.x; i < a.P; i += blockDim.x) {
        const long long f = e - a.obj[0][i];
        a.fit[0][i] = f > 0 ? f : 0;
    }
}

// Generation 0: the best initial individual of every island becomes its best-ever.
__global__ void __launch_bounds__(kReplThreads) k_init_best(ReplArgs a) {
    const int isl = blockIdx.x, lo = isl * a.I, K = a.K;
    int best, worst;
    island_extremes(a.fit[0], lo, a.I, best, worst);
    copy_ind(a.bY + (size_t)isl * K, a.bX + (size_t)isl * K, a.Y[0] + (size_t)best * K, a.X[0] + (size_t)best * K, K);
    if (threadIdx.x == 0) {
        a.bobj[isl] = a.obj[0][best];
        a.bfit[isl] = a.fit[0][best];
    }
}

// Raises a kernel's dynamic shared memory limit once per (kernel, size); later calls,
// including those made while a stream is being captured, find it already set.
std::mutex g_attr_mu;
std::map<const void *, int> g_attr_smem;

template <typename KernelT>
cudaError_t prepare(KernelT kernel, int smem) {
    if (smem <= 48 * 1024) return cudaSuccess;
    std::lock_guard<std::mutex> lk(g_attr_mu);
    int &have = g_attr_smem[reinterpret_cast<const void *>(kernel)];
    if (have >= smem) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) have = smem;
    return e;
}

}  // namespace

#ifdef FFS_CHECKED
unsigned int bounds_faults_kernels() { return bounds_faults_take(); }
#endif

int cta_smem_bytes(const TabHeader &h, int Hcap, bool ga, bool global_profile, bool insert) {
    const WarpLayout L = warp_layout(h.N, h.M, h.K, global_profile ? 0 : Hcap, ga, insert && !global_profile ? h.maxo : 0);
    return 128 + ((h.bytes + 127) & ~127) + kWarpsPerBlock * L.bytes;
}

// Runs the body with O_/M_ bound to the (order, mach) pair of the enclosing scope.
// The machine mode of a public call (gene or earliest) and the instance's machine model
// (identical, or unrelated with per-gene p and q) give the kernel's machine mode.
#define FFS_CASE(O, M, ...)                                    \
    if (order == (O) && kmach == (M)) {                        \
        constexpr int O_ = (O), M_ = (M);                      \
        __VA_ARGS__;                                           \
    }
#define FFS_DISPATCH(...)                                                                  \
    do {                                                                                   \
        const int kmach = mach + (h.unrel ? 2 : 0);  /* mach carries kPlaceInsert */       \
        FFS_CASE(kOrderStage, kMachEarliest, __VA_ARGS__)                                  \
        else FFS_CASE(kOrderStage, kMachGene, __VA_ARGS__)                                 \
        else FFS_CASE(kOrderTopo, kMachEarliest, __VA_ARGS__)                              \
        else FFS_CASE(kOrderTopo, kMachGene, __VA_ARGS__)                                  \
        else FFS_CASE(kOrderStage, kMachEarliestU, __VA_ARGS__)                            \
        else FFS_CASE(kOrderStage, kMachGeneU, __VA_ARGS__)                                \
        else FFS_CASE(kOrderTopo, kMachEarliestU, __VA_ARGS__)                             \
        else FFS_CASE(kOrderTopo, kMachGeneU, __VA_ARGS__)                                 \
        else FFS_CASE(kOrderStage, kMachEarliest | kPlaceInsert, __VA_ARGS__)              \
        else FFS_CASE(kOrderStage, kMachGene | kPlaceInsert, __VA_ARGS__)                  \
        else FFS_CASE(kOrderStage, kMachEarliestU | kPlaceInsert, __VA_ARGS__)             \
        else FFS_CASE(kOrderStage, kMachGeneU | kPlaceInsert, __VA_ARGS__)                 \
        else e = cudaErrorInvalidValue;                                                    \
    } while (0)

cudaError_t launch_decode(int order, int mach, bool global_profile, const DecodeArgs &a,
                          const TabHeader &h, int grid, cudaStream_t st) {
    const int smem = cta_smem_bytes(h, a.Hcap, false, global_profile, mach_insert(mach));
    cudaError_t e = cudaSuccess;
    FFS_DISPATCH({
        if (global_profile) {
            e = prepare(k_decode<O_, M_, true>, smem);
            if (e == cudaSuccess) k_decode<O_, M_, true><<<grid, kWarpsPerBlock * 32, smem, st>>>(a);
        } else {
            e = prepare(k_decode<O_, M_, false>, smem);
            if (e == cudaSuccess) k_decode<O_, M_, false><<<grid, kWarpsPerBlock * 32, smem, st>>>(a);
        }
    });
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_ga_init(int order, int mach, const GenArgs &a, const TabHeader &h, int grid,
                           cudaStream_t st) {
    const int smem = cta_smem_bytes(h, a.Hcap, true, false, mach_insert(mach));
    cudaError_t e = cudaSuccess;
    FFS_DISPATCH({
        e = prepare(k_ga_init<O_, M_>, smem);
        if (e == cudaSuccess) k_ga_init<O_, M_><<<grid, kWarpsPerBlock * 32, smem, st>>>(a);
    });
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_ga_generation(int order, int mach, const GenArgs &a, const TabHeader &h,
                                 int grid, cudaStream_t st, bool overlap) {
    const int smem = cta_smem_bytes(h, a.Hcap, true, false, mach_insert(mach));
    cudaError_t e = cudaSuccess;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kWarpsPerBlock * 32);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = overlap ? 1 : 0;
    FFS_DISPATCH({
        e = prepare(k_ga_generation<O_, M_>, smem);
        if (e == cudaSuccess) e = cudaLaunchKernelEx(&cfg, k_ga_generation<O_, M_>, a);
    });
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t prepare_ga_generation(int order, int mach, const TabHeader &h, int Hcap) {
    const int smem = cta_smem_bytes(h, Hcap, true, false, mach_insert(mach));
    cudaError_t e = cudaSuccess;
    FFS_DISPATCH({ e = prepare(k_ga_generation<O_, M_>, smem); });
    return e;
}

cudaError_t prepare_candidates(int mach, const TabHeader &h) {
    const int smem = cta_smem_bytes(h, 0, true, false);
    return mach_gene(mach) ? prepare(k_candidates<kMachGene>, smem) : prepare(k_candidates<kMachEarliest>, smem);
}

cudaError_t launch_candidates(int mach, const GenArgs &a, const TabHeader &h, int grid, cudaStream_t st) {
    const int smem = cta_smem_bytes(h, 0, true, false);
    cudaError_t e;
    if (mach_gene(mach)) {
        e = prepare(k_candidates<kMachGene>, smem);
        if (e == cudaSuccess) k_candidates<kMachGene><<<grid, kWarpsPerBlock * 32, smem, st>>>(a);
    } else {
        e = prepare(k_candidates<kMachEarliest>, smem);
        if (e == cudaSuccess) k_candidates<kMachEarliest><<<grid, kWarpsPerBlock * 32, smem, st>>>(a);
    }
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_warm_remap(const WarmArgs &a, cudaStream_t st) {
    if (a.Ko > kMaxK || a.K > kMaxK) return cudaErrorInvalidValue;
    const int grid = a.P < 1216 ? a.P : 1216;
    k_warm_remap<<<grid, kRemapThreads, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_island_top(const float *score, const uint8_t *is_new, int P, int F, int I, int32_t *keep,
                              cudaStream_t st) {
    if (F < 1 || I < 1 || P % I || F * I > kTopMax) return cudaErrorInvalidValue;
    k_island_top<<<P / I, kTopThreads, 0, st>>>(score, is_new, P, F, I, keep);
    return cudaGetLastError();
}

cudaError_t launch_emax(const ReplArgs &a, cudaStream_t st) {
    k_emax<<<1, 1024, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_replace(const ReplArgs &a, cudaStream_t st) {
    k_init_best<<<a.P / a.I, kReplThreads, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace edffs
