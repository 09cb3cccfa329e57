// ffs_ga.cuh -- GA building blocks shared by the per-generation kernel and the batched
// persistent kernel: warp workspace views, child construction (Sec. 4.4: selection,
// neighbouring paired crossover with correction, mutation), generation-0 initialisation
// (Sec. 4.3) and warp-level elitist replacement and ring migration.
#pragma once
#include <stdint.h>

#include <climits>

#include "ffs_device.cuh"

namespace edffs {

struct WarpPtrs {
    uint16_t *h;
    int32_t *C, *mfree;
    int16_t *inv, *y;
    int8_t *x;
    uint32_t *bits;
};

// Views of one warp's slice `ws` laid out by warp_layout(..., Hcap, ga); with a global
// profile (`hg` non-null) the profile lives there instead.
__device__ __forceinline__ WarpPtrs warp_view(char *ws, const WarpLayout &L, uint16_t *hg) {
    WarpPtrs w;
    w.h = hg ? hg : reinterpret_cast<uint16_t *>(ws + L.off_h);
    w.C = reinterpret_cast<int32_t *>(ws + L.off_C);
    w.mfree = reinterpret_cast<int32_t *>(ws + L.off_mfree);
    w.inv = reinterpret_cast<int16_t *>(ws + L.off_inv);
    w.y = reinterpret_cast<int16_t *>(ws + L.off_y);
    w.x = reinterpret_cast<int8_t *>(ws + L.off_x);
    w.bits = reinterpret_cast<uint32_t *>(ws + L.off_bits);
    return w;
}

// Better individual: larger fitness, ties to the lower population index.
__device__ __forceinline__ bool fitter(long long f, int i, long long bf, int bi) {
    return f > bf || (f == bf && i < bi);
}

__device__ __forceinline__ void warp_best(long long &bf, int &bi) {
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        const long long of = __shfl_xor_sync(kFull, bf, off);
        const int oi = __shfl_xor_sync(kFull, bi, off);
        if (fitter(of, oi, bf, bi)) {
            bf = of;
            bi = oi;
        }
    }
}


constexpr int kRowU = 4;

// Copies a parent's y row (when ys is non-null) and the x row made of xa[0 .. cx) and
// xb[cx .. K) (when `with_x`) from global into shared memory; each lane loads its values
// of a chunk of 32 kRowU genes before it stores any.
__device__ __forceinline__ void rows_to_smem(int16_t *yd, int8_t *xd, const int16_t *ys, const int8_t *xa,
                                             const int8_t *xb, int cx, int K, bool with_x, int lane) {
    for (int k0 = lane; k0 < K; k0 += 32 * kRowU) {
        int16_t vy[kRowU];
        int8_t vx[kRowU];
#pragma unroll
        for (int u = 0; u < kRowU; ++u) {
            const int k = k0 + 32 * u;
            if (k < K) {
                if (ys) vy[u] = ys[k];
                if (with_x) vx[u] = k < cx ? xa[k] : xb[k];
            }
        }
#pragma unroll
        for (int u = 0; u < kRowU; ++u) {
            const int k = k0 + 32 * u;
            if (k < K) {
                if (ys) yd[k] = vy[u];
                if (with_x) xd[k] = vx[u];
            }
        }
    }
}

// Parent population and operator settings of one generation.
struct GASrc {
    const int16_t *Yc;   // [P][K] parents
    const int8_t *Xc;
    const int64_t *fc;   // [P] parents' fitness
    int P, I, K, tour_k, side;
    uint64_t pc_thr, pm_thr, seed;
    uint32_t iid;        // 24-bit instance id of the stream
    int F;               // children per population slot (1; more when over-generating for a surrogate)
};

// Builds child i of generation `gen` into the warp's w.y / w.x: both parents of its pair
// are selected from the counter-based stream, so the two children of a pair can be built
// by different warps.  With s.F > 1, child i = f P + j is candidate f of population slot
// j: it draws its parents from slot j's island (or neighbourhood), candidate f of slots
// 2q and 2q+1 are the two children of one pair, and candidate 0 is exactly the child a
// plain generation builds for slot j.
// Returns true if the child differs from a plain copy of a parent (crossover or mutation
// was applied).
template <int MACH>
__device__ __forceinline__ bool make_child(const Tabs &T, const WarpPtrs &w, const GASrc &s, int i, uint32_t gen,
                                           int lane) {
    const int K = s.K, I = s.I;
    const int pp = i >> 1;
    int parent[2];
    // Entrant e of slot 2 pp + t's tournament (the 5-cell neighbourhood with tour_k = 0).
    auto entrant = [&](int t, int e, long long &bf, int &bi) {
        const int slot = 2 * pp + t;
        if (s.tour_k > 0) {
            if (e < s.tour_k) {
                const int lo = ((s.F > 1 ? slot % s.P : slot) / I) * I;  // the island of the slot the child is for
                bi = lo + (int)below(draw(s.seed, kPSelect, s.iid, gen, (uint32_t)slot, (uint32_t)e), (uint32_t)I);
                bf = s.fc[bi];
            }
        } else if (e < 5) {  // the cell and its N, S, W, E neighbours on the torus
            const int sd = s.side, base = s.F > 1 ? slot % s.P : slot, r = base / sd, cc = base % sd;
            const int rr = e == 1 ? (r + sd - 1) % sd : e == 2 ? (r + 1) % sd : r;
            const int c2 = e == 3 ? (cc + sd - 1) % sd : e == 4 ? (cc + 1) % sd : cc;
            bi = rr * sd + c2;
            bf = s.fc[bi];
        }
    };
    if (s.tour_k <= 16) {  // both tournaments at once, one per half-warp
        long long bf = LLONG_MIN;
        int bi = INT_MAX;
        entrant(lane >> 4, lane & 15, bf, bi);
#pragma unroll
        for (int off = 8; off; off >>= 1) {
            const long long of = __shfl_xor_sync(kFull, bf, off);
            const int oi = __shfl_xor_sync(kFull, bi, off);
            if (fitter(of, oi, bf, bi)) {
                bf = of;
                bi = oi;
            }
        }
        parent[0] = __shfl_sync(kFull, bi, 0);
        parent[1] = __shfl_sync(kFull, bi, 16);
    } else {
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            long long bf = LLONG_MIN;
            int bi = INT_MAX;
            entrant(t, lane, bf, bi);
            warp_best(bf, bi);
            parent[t] = bi;
        }
    }
    const uint4 rc = stream_block(s.seed, kPCross, s.iid, gen, (uint32_t)pp, 0);
    const bool cross = K >= 2 && (uint64_t)rc.x < s.pc_thr;
    const int first = (i & 1) ? parent[1] : parent[0];
    const int second = (i & 1) ? parent[0] : parent[1];
    const int16_t *yf = s.Yc + (size_t)first * K, *yb = s.Yc + (size_t)second * K;
    if (!cross) {
        rows_to_smem(w.y, w.x, yf, s.Xc + (size_t)first * K, s.Xc + (size_t)first * K, K, K, mach_gene(MACH),
                     lane);
    } else {
        const int cx = 1 + (int)below(rc.y, (uint32_t)(K - 1));
        const int cy = 1 + (int)below(rc.z, (uint32_t)(K - 1));
        const int nw = (K + 32) / 32;  // bitmap words covering values 0..K
        for (int q = lane; q < nw; q += 32) w.bits[q] = 0;
        __syncwarp();
        // Parent reads: each lane loads its values of a chunk of 32 kRowU genes before it
        // uses any, so a chunk costs one round trip to L2.
        for (int k0 = lane; k0 < cy; k0 += 32 * kRowU) {
            int v[kRowU];
#pragma unroll
            for (int u = 0; u < kRowU; ++u) v[u] = k0 + 32 * u < cy ? yf[k0 + 32 * u] : 0;
#pragma unroll
            for (int u = 0; u < kRowU; ++u)
                if (k0 + 32 * u < cy) {
                    w.y[k0 + 32 * u] = (int16_t)v[u];
                    atomicOr(&w.bits[FFS_IX(v[u] >> 5, nw)], 1u << (v[u] & 31));
                }
        }
        __syncwarp();
        for (int k0 = cy + lane; k0 < K; k0 += 32 * kRowU) {  // tail values already in the head: duplicates
            int v[kRowU];
#pragma unroll
            for (int u = 0; u < kRowU; ++u) v[u] = k0 + 32 * u < K ? yb[k0 + 32 * u] : 0;
#pragma unroll
            for (int u = 0; u < kRowU; ++u)
                if (k0 + 32 * u < K) {
                    const bool dup = (w.bits[FFS_IX(v[u] >> 5, nw)] >> (v[u] & 31)) & 1u;
                    w.y[k0 + 32 * u] = dup ? (int16_t)0 : (int16_t)v[u];
                }
        }
        __syncwarp();
        for (int k = cy + lane; k < K; k += 32) {
            const int v = w.y[k];
            if (v) atomicOr(&w.bits[FFS_IX(v >> 5, nw)], 1u << (v & 31));
        }
        __syncwarp();
        // Missing values, ascending, into `miss`.
        int16_t *miss = w.inv;
        int base = 0;
        for (int q0 = 0; q0 < nw; q0 += 32) {
            const int q = q0 + lane;
            unsigned m = 0;
            if (q < nw) {
                m = ~w.bits[q];
                if (q == 0) m &= ~1u;
                const int hi = K - q * 32;  // highest valid bit
                if (hi < 31) m &= hi >= 0 ? ((2u << hi) - 1u) : 0u;
            }
            const int cnt = __popc(m);
            int incl = cnt;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int v = __shfl_up_sync(kFull, incl, off);
                if (lane >= off) incl += v;
            }
            int o = base + incl - cnt;
            while (m) {
                const int b = __ffs(m) - 1;
                m &= m - 1;
                miss[FFS_IX(o++, K)] = (int16_t)(q * 32 + b);
            }
            base += __shfl_sync(kFull, incl, 31);
        }
        __syncwarp();
        int rank = 0;
        for (int k0 = cy; k0 < K; k0 += 32) {  // the r-th duplicate takes the r-th missing value
            const int k = k0 + lane;
            const bool dup = k < K && w.y[k] == 0;
            const unsigned bm = __ballot_sync(kFull, dup);
            if (dup) w.y[k] = miss[FFS_IX(rank + __popc(bm & ((1u << lane) - 1u)), K)];
            rank += __popc(bm);
        }
        if (mach_gene(MACH))
            rows_to_smem(nullptr, w.x, nullptr, s.Xc + (size_t)first * K, s.Xc + (size_t)second * K, cx, K, true,
                         lane);
    }
    __syncwarp();
    const uint4 rm = stream_block(s.seed, kPMutate, s.iid, gen, (uint32_t)i, 0);
    if ((uint64_t)rm.x < s.pm_thr) {
        if (K >= 2 && lane == 0) {
            const int ma = (int)below(rm.y, (uint32_t)K);
            int mb = (int)below(rm.z, (uint32_t)(K - 1));
            mb += mb >= ma;
            const int16_t t = w.y[ma];
            w.y[ma] = w.y[mb];
            w.y[mb] = t;
        }
        if (mach_gene(MACH)) {
            for (int k = lane; k < K; k += 32) {
                const int o = T.o[T.gstg[k]];
                if (o >= 2) {
                    const uint32_t u = draw(s.seed, kPMutate, s.iid, gen, (uint32_t)i, (uint32_t)(3 + k));
                    const int r = (int)below(u, (uint32_t)(o - 1));
                    w.x[k] = (int8_t)(r + (r >= w.x[k]));
                }
            }
        }
    }
    __syncwarp();
    return cross || (uint64_t)rm.x < s.pm_thr;
}

// Generation 0 of individual i (Sec. 4.3): Y a Fisher-Yates permutation of 1..K, X uniform
// machines, into w.y / w.x.
template <int MACH>
__device__ __forceinline__ void make_initial(const Tabs &T, const WarpPtrs &w, uint64_t seed, uint32_t iid, int i,
                                             int lane) {
    const int K = T.K;
    // Fisher-Yates: step d swaps position K-1-d with a uniform position <= K-1-d.
    int16_t *target = w.inv;
    for (int d = lane; d < K - 1; d += 32) {
        const uint32_t u = draw(seed, kPInitY, iid, 0, (uint32_t)i, (uint32_t)d);
        target[d] = (int16_t)below(u, (uint32_t)(K - d));
    }
    for (int k = lane; k < K; k += 32) w.y[k] = (int16_t)(k + 1);
    __syncwarp();
    if (lane == 0) {
        for (int d = 0; d < K - 1; ++d) {
            const int pa = K - 1 - d, pb = target[d];
            const int16_t t = w.y[pa];
            w.y[pa] = w.y[pb];
            w.y[pb] = t;
        }
    }
    __syncwarp();
    if (mach_gene(MACH)) {
        for (int k = lane; k < K; k += 32) {
            const uint32_t u = draw(seed, kPInitX, iid, 0, (uint32_t)i, (uint32_t)k);
            w.x[k] = (int8_t)below(u, (uint32_t)T.o[T.gstg[k]]);
        }
    }
    __syncwarp();
}

// ---------------------------------------------------------------- GA: island bookkeeping
// Best (largest fitness, lowest index) and worst (smallest fitness, lowest index) of
// fit[lo .. lo+n) with one warp, and the best's fitness; reads bypass L1 because other SMs
// wrote the values.
__device__ __forceinline__ void warp_extremes(const int64_t *fit, int lo, int n, int lane, int &best, int &worst,
                                              long long &best_fit) {
    long long bf = LLONG_MIN, wf = LLONG_MAX;
    int bi = INT_MAX, wi = INT_MAX;
    for (int t = lane; t < n; t += 32) {
        const long long f = __ldcg(fit + lo + t);
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
    best = bi;
    worst = wi;
    best_fit = bf;
}

__device__ __forceinline__ void warp_extremes(const int64_t *fit, int lo, int n, int lane, int &best, int &worst) {
    long long bf;
    warp_extremes(fit, lo, n, lane, best, worst, bf);
}

// Copies one individual (K genes of y and x) to one or two destinations.  Each lane loads
// its share of a chunk of 32 U genes before it stores any of them, so a chunk costs one
// round trip to L2 rather than one per 32 genes.
template <int U = 4>
__device__ __forceinline__ void warp_copy_ind(int16_t *yd, int8_t *xd, const int16_t *ys, const int8_t *xs, int K,
                                              int lane, int16_t *yd2 = nullptr, int8_t *xd2 = nullptr,
                                              int16_t *yd3 = nullptr, int8_t *xd3 = nullptr) {
#pragma unroll 1
    for (int k0 = lane; k0 < K; k0 += 32 * U) {
        const int n = K - k0;  // genes left from this lane's first one
        uint32_t v[U];         // y in the low halfword, x in bits 16..23
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (32 * u < n)
                v[u] = (uint16_t)__ldcg(ys + k0 + 32 * u) | ((uint32_t)(uint8_t)__ldcg(xs + k0 + 32 * u) << 16);
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (32 * u < n) {
                yd[k0 + 32 * u] = (int16_t)(v[u] & 0xFFFFu);
                xd[k0 + 32 * u] = (int8_t)(v[u] >> 16);
                if (yd2) {
                    yd2[k0 + 32 * u] = (int16_t)(v[u] & 0xFFFFu);
                    xd2[k0 + 32 * u] = (int8_t)(v[u] >> 16);
                }
                if (yd3) {
                    yd3[k0 + 32 * u] = (int16_t)(v[u] & 0xFFFFu);
                    xd3[k0 + 32 * u] = (int8_t)(v[u] >> 16);
                }
            }
    }
}

// Best (largest fitness, lowest index) and worst (smallest fitness, lowest index) of an
// island of at most 64 held in registers: lane l has slots l (f0, o0) and l + 32 (f1, o1),
// lanes past the island LLONG_MIN / LLONG_MAX-free placeholders excluded by `h0`, `h1`.
// Returns the indices (island-relative) and the best's fitness and objective.
__device__ __forceinline__ void reg_extremes(long long f0, long long o0, bool h0, long long f1, long long o1, bool h1,
                                             int lane, int &best, int &worst, long long &bfit, long long &bobj) {
    long long bf = LLONG_MIN, wf = LLONG_MAX;
    int bi = INT_MAX, wi = INT_MAX;
    if (h0) { bf = f0; bi = lane; wf = f0; wi = lane; }
    if (h1) {
        if (fitter(f1, lane + 32, bf, bi)) { bf = f1; bi = lane + 32; }
        if (f1 < wf) { wf = f1; wi = lane + 32; }
    }
    warp_best(bf, bi);
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        const long long of = __shfl_xor_sync(kFull, wf, off);
        const int oi = __shfl_xor_sync(kFull, wi, off);
        if (of < wf || (of == wf && oi < wi)) { wf = of; wi = oi; }
    }
    best = bi;
    worst = wi;
    bfit = bf;
    // the best's objective from the lane that holds it
    const long long mine = (bi >> 5) ? o1 : o0;
    bobj = __shfl_sync(kFull, mine, bi & 31);
}

// Elitist replacement of island `isl` by one warp (Sec. 4.4): the best-ever individual is
// updated if a child is strictly fitter, then overwrites the worst child.  With `migrate`,
// the island's best and worst after replacement are recorded for the ring exchange.  U:
// genes per lane per copy chunk.  With REG (kernels with registers to spare), islands of
// up to 64 are read once (fitness, objectives and the best-ever record in one round trip)
// and the state after replacement is derived in registers.
template <int U = 4, bool REG = false>
__device__ __forceinline__ void island_replace(int16_t *Y, int8_t *X, int64_t *obj, int64_t *fit, int16_t *bY,
                                               int8_t *bX, int64_t *bobj, int64_t *bfit, int isl, int I, int K,
                                               bool migrate, int16_t *mY, int8_t *mX, int64_t *mobj, int64_t *mfit,
                                               int32_t *mw, int lane) {
    const int lo = isl * I;
    int16_t *bYi = bY + (size_t)isl * K;
    int8_t *bXi = bX + (size_t)isl * K;
    if (REG && I <= 64) {
        const bool h0 = lane < I, h1 = lane + 32 < I;
        long long f0 = 0, f1 = 0, o0 = 0, o1 = 0;
        if (h0) {
            f0 = __ldcg(fit + lo + lane);
            o0 = __ldcg(obj + lo + lane);
        }
        if (h1) {
            f1 = __ldcg(fit + lo + lane + 32);
            o1 = __ldcg(obj + lo + lane + 32);
        }
        const long long bf0 = __ldcg(bfit + isl), bo0 = __ldcg(bobj + isl);
        int best, worst;
        long long fb, ob;
        reg_extremes(f0, o0, h0, f1, o1, h1, lane, best, worst, fb, ob);
        const bool better = fb > bf0;
        const long long eobj = better ? ob : bo0, efit = better ? fb : bf0;
        const int16_t *ys = better ? Y + (size_t)(lo + best) * K : bYi;
        const int8_t *xs = better ? X + (size_t)(lo + best) * K : bXi;
        int16_t *yw = Y + (size_t)(lo + worst) * K;
        int8_t *xw = X + (size_t)(lo + worst) * K;
        // the island after replacement: the worst slot holds the elite, whose fitness is at
        // least every child's, so its best is the lower of `worst` and `best` when the two
        // fitnesses tie, else `worst`; its worst is the least of the other slots, unless
        // none is below the elite
        const int b2 = efit == fb ? min(worst, best) : worst;
        const bool same = b2 == worst || better;  // the migrant's row is the elite's
        if (migrate) {
            long long wf = LLONG_MAX;
            int wi = INT_MAX;
            if (h0 && lane != worst) { wf = f0; wi = lane; }
            if (h1 && lane + 32 != worst && f1 < wf) { wf = f1; wi = lane + 32; }
#pragma unroll
            for (int off = 16; off; off >>= 1) {
                const long long of = __shfl_xor_sync(kFull, wf, off);
                const int oi = __shfl_xor_sync(kFull, wi, off);
                if (of < wf || (of == wf && oi < wi)) { wf = of; wi = oi; }
            }
            const int w2 = wf < efit || (wf == efit && wi < worst) ? wi : worst;
            if (lane == 0) {
                mobj[isl] = b2 == worst ? eobj : ob;
                mfit[isl] = efit;
                mw[isl] = lo + w2;
            }
        }
        if (lane == 0) {
            if (better) {
                bobj[isl] = eobj;
                bfit[isl] = efit;
            }
            obj[lo + worst] = eobj;
            fit[lo + worst] = efit;
        }
        if (better)
            warp_copy_ind<U>(yw, xw, ys, xs, K, lane, bYi, bXi);
        else
            warp_copy_ind<U>(yw, xw, ys, xs, K, lane);
        if (migrate)  // the migrant: the elite's row, or a child tied with it at a lower index
            warp_copy_ind<U>(mY + (size_t)isl * K, mX + (size_t)isl * K, same ? ys : Y + (size_t)(lo + b2) * K,
                             same ? xs : X + (size_t)(lo + b2) * K, K, lane);
        __syncwarp();
        return;
    }
    int best, worst;
    long long fb;
    warp_extremes(fit, lo, I, lane, best, worst, fb);
    const long long bf0 = bfit[isl];
    const bool better = fb > bf0;
    // the elite after the update: the best child if strictly fitter, else the kept one;
    // it overwrites the worst child (and, when it is new, the island's best-ever record)
    long long eobj = 0;
    if (lane == 0) eobj = better ? __ldcg(obj + best) : bobj[isl];
    const long long efit = better ? fb : bf0;
    if (better)
        warp_copy_ind<U>(Y + (size_t)worst * K, X + (size_t)worst * K, Y + (size_t)best * K, X + (size_t)best * K,
                         K, lane, bYi, bXi);
    else
        warp_copy_ind<U>(Y + (size_t)worst * K, X + (size_t)worst * K, bYi, bXi, K, lane);
    if (lane == 0) {
        if (better) {
            bobj[isl] = eobj;
            bfit[isl] = efit;
        }
        obj[worst] = eobj;
        fit[worst] = efit;
    }
    __syncwarp();
    if (migrate) {
        warp_extremes(fit, lo, I, lane, best, worst, fb);
        long long mo = 0;
        if (lane == 0) mo = __ldcg(obj + best);
        warp_copy_ind<U>(mY + (size_t)isl * K, mX + (size_t)isl * K, Y + (size_t)best * K, X + (size_t)best * K, K,
                         lane);
        if (lane == 0) {
            mobj[isl] = mo;
            mfit[isl] = fb;
            mw[isl] = worst;
        }
    }
}

// Edge e of the single migration ring, by one warp: island e's recorded worst slot <-
// island e-1's migrant.
__device__ __forceinline__ void migrate_edge(int16_t *Y, int8_t *X, int64_t *obj, int64_t *fit, const int16_t *mY,
                                             const int8_t *mX, const int64_t *mobj, const int64_t *mfit,
                                             const int32_t *mw, int e, int nisl, int K, int lane) {
    const int src = (e + nisl - 1) % nisl, wslot = __ldcg(mw + e);
    long long o = 0, f = 0;
    if (lane == 0) {
        o = __ldcg(mobj + src);
        f = __ldcg(mfit + src);
    }
    warp_copy_ind(Y + (size_t)wslot * K, X + (size_t)wslot * K, mY + (size_t)src * K, mX + (size_t)src * K, K, lane);
    if (lane == 0) {
        obj[wslot] = o;
        fit[wslot] = f;
    }
}

// The whole single ring by one warp (island d's recorded worst slot <- island d-1's
// migrant, every d): lane l first reads the slot and migrant record of island 32 c + l, so
// each island then costs only the copy.
template <int U = 4>
__device__ __forceinline__ void ring_migrate(int16_t *Y, int8_t *X, int64_t *obj, int64_t *fit, const int16_t *mY,
                                             const int8_t *mX, const int64_t *mobj, const int64_t *mfit,
                                             const int32_t *mw, int nisl, int K, int lane) {
    for (int c = 0; c < nisl; c += 32) {
        const int d = c + lane, src = (d + nisl - 1) % nisl;
        int ws = 0;
        long long o = 0, f = 0;
        if (d < nisl) {
            ws = __ldcg(mw + d);
            o = __ldcg(mobj + src);
            f = __ldcg(mfit + src);
        }
        const int n = min(32, nisl - c);
#pragma unroll 1
        for (int l = 0; l < n; ++l) {
            const int wslot = __shfl_sync(kFull, ws, l), sl = (c + l + nisl - 1) % nisl;
            warp_copy_ind<U>(Y + (size_t)wslot * K, X + (size_t)wslot * K, mY + (size_t)sl * K, mX + (size_t)sl * K,
                             K, lane);
        }
        if (d < nisl) {
            obj[ws] = o;
            fit[ws] = f;
        }
    }
}

}  // namespace edffs
