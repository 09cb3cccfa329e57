// ffs_batch.cu -- many independent rescheduling instances in one persistent launch.
//
// The launch is a grid of thread-block clusters.  A cluster owns one instance at a time
// and takes the next one from a queue (instances sorted largest first) when it is done;
// CTA r of the cluster owns islands
// r, r + CS, ... of that instance.  Each CTA stages the instance's tables into its shared
// memory with a bulk copy and runs every requested generation for its islands: children
// (one warp each, several per warp), then elitist replacement per island.  Islands only
// interact through E_max at generation 0, ring migration every migrate_every generations
// and, for the 5-cell neighbourhood selection, every generation; those points are cluster
// barriers (hardware, no spinning), with data passed through global memory or the
// cluster's distributed shared memory.  Each warp's power profile slice is cut from the
// CTA's shared-memory budget for the instance at hand; schedules that outgrow it are
// redone in the warp's global slice.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <climits>
#include <mutex>

#include "ffs_device.cuh"
#include "ffs_ga.cuh"
#include "ffs_kernels.cuh"

namespace cg = cooperative_groups;

namespace edffs {

namespace {

// Bulk copy of one instance's tables; `phase` is the mbarrier parity to wait for.
__device__ __forceinline__ bool stage_again(char *dst, const char *src, int bytes, uint64_t *mbar, uint32_t phase,
                                            int32_t *err) {
    const uint32_t bar = smem_u32(mbar);
    if (threadIdx.x == 0) {
        // the previous instance's tables were read through the generic proxy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
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
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(phase)
            : "memory");
        done = ok != 0;
    }
    if (!done) atomicOr(err, kErrTimeout);
    return __syncthreads_and(done) != 0;
}

__device__ __forceinline__ void write_ind(int16_t *Y, int8_t *X, const WarpPtrs &w, int i, int K, bool gene, int lane) {
    int16_t *yo = Y + (size_t)i * K;
    for (int k = lane; k < K; k += 32) yo[k] = w.y[k];
    if (gene) {
        int8_t *xo = X + (size_t)i * K;
        for (int k = lane; k < K; k += 32) xo[k] = w.x[k];
    }
    __syncwarp();
}

// Decodes the warp's chromosome (already written to row i of Y) into obj/fit slot i.  The
// schedule is built in the warp's shared slice (filled with full headroom first) unless
// `gfirst`; one that outgrows the slice is redone in the warp's global slice from the row
// in global memory (the decode reuses w.y), and counted in *overflows.
template <int ORDER, int MACH>
__device__ __forceinline__ void decode_into(const Tabs &T, const WarpPtrs &w, int Hcap, uint16_t *hg, int H,
                                            bool gfirst, const int16_t *Y, int64_t *obj, int64_t *fit,
                                            long long emax, int i, int32_t *err, int *overflows, int lane) {
    DecodeOut r{0, 0, 1};
    if (!gfirst) {
        // many warps per scheduler here: the plain placement loop (fewer instructions per op)
        r = decode_warp<ORDER, MACH, true, false>(T, w.h, Hcap, w.C, w.mfree, w.inv, w.y, w.x, nullptr, nullptr, lane);
        if (r.status == 1) {
            if (lane == 0) atomicAdd(overflows, 1);
            const int16_t *row = Y + (size_t)i * T.K;
            for (int k = lane; k < T.K; k += 32) w.y[k] = row[k];
            __syncwarp();
        }
    }
    if (r.status == 1) r = decode_warp<ORDER, MACH, false, false>(T, hg, H, w.C, w.mfree, w.inv, w.y, w.x, nullptr, nullptr, lane);
    if (lane == 0) {
        if (r.status != 0) {
            atomicOr(err, r.status == 2 ? kErrBadChromosome : kErrOverflow);
        } else {
            const long long o = (long long)T.WT * r.tard + r.cmax;
            obj[i] = o;
            if (fit) fit[i] = emax - o > 0 ? emax - o : 0;
        }
    }
    __syncwarp();
}

// 128 registers: the whole register file for one CTA of 512 threads per SM (shared memory
// allows one), set explicitly so that no variant spills.
template <int ORDER, int MACH>
__global__ void __maxnreg__(128) k_batch(BatchArgs a) {
    extern __shared__ __align__(128) char smem[];
    __shared__ long long s_red[32];
    __shared__ int s_over;
    __shared__ int s_next;  // next of this CTA's children to build in the current generation
    __shared__ int s_item;  // rank 0: the instance its cluster took from the queue
    __shared__ int s_stop[2];  // rank 0: the stop word as read at a generation's start (by parity)
    cg::cluster_group cluster = cg::this_cluster();
    const int CS = (int)cluster.num_blocks(), rank = (int)cluster.block_rank();
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem);
    char *tab = smem + 128;
    const int W = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t phase = 0;
    uint16_t *hg = a.gscratch + (size_t)(blockIdx.x * W + warp) * (size_t)a.Hmax;
    const int P = a.P, I = a.I;
    const bool gene = mach_gene(MACH);
    // Every CTA of a cluster follows the same control flow, so the cluster barriers below
    // are reached by all of them.
    for (;;) {
        // rank 0 takes the cluster's next instance; every CTA reads it after the barrier
        // (and rank 0 overwrites it only after the barrier that ends the instance)
        if (rank == 0 && threadIdx.x == 0) s_item = atomicAdd(a.next, 1);
        cluster.sync();
        const int item = *cluster.map_shared_rank(&s_item, 0);
        if (item >= a.count) {
            cluster.sync();  // rank 0's shared memory stays until every CTA has read it
            break;
        }
        BatchInst *in = a.inst + a.order[item];
        const int K = in->K, nisl = in->nisl, H = in->H;
        const bool staged = stage_again(tab, in->blob, in->blob_bytes, mbar, phase, a.err);
        phase ^= 1u;
        const Tabs T = tabs_view(tab);
        const int fixed = warp_layout(T.N, T.M, K, 0, true).bytes;
        const int avail = (a.smem_bytes - 128 - ((in->blob_bytes + 127) & ~127)) / W - fixed;
        const int Hcap = avail >= 2 * kMinBatchSlots ? min(H, (avail / 2) & ~7) : 0;
        const WarpLayout L = warp_layout(T.N, T.M, K, Hcap, true);
        // the host rejects mappings where this cannot hold; the check keeps every CTA in step
        const bool fits = staged && 128 + ((in->blob_bytes + 127) & ~127) + W * L.bytes <= a.smem_bytes;
        if (!fits && threadIdx.x == 0) atomicOr(a.err, kErrOverflow);
        const WarpPtrs w = warp_view(tab + ((in->blob_bytes + 127) & ~127) + warp * L.bytes, L, nullptr);
        int gen = in->gen;
        long long emax = in->emax;
        // Profiles go to shared memory first; if more than a quarter of this CTA's first
        // round of decodes for the instance outgrows the slice, the rest go straight to
        // global memory (schedules, and so results, are the same either way).
        if (threadIdx.x == 0) {
            s_over = 0;
            s_next = 0;
        }
        __syncthreads();
        bool gfirst = Hcap == 0;
        bool probing = true;
        const int per_round = ((nisl - rank + CS - 1) / CS) * I;  // decodes per round in this CTA

        if (emax == 0) {  // generation 0
            long long mx = 0;
            if (fits) {
                for (int isl = rank; isl < nisl; isl += CS)
                    for (int c = warp; c < I; c += W) {
                        const int i = isl * I + c;
                        make_initial<MACH>(T, w, a.seed, in->iid, i, lane);
                        write_ind(in->Y[0], in->X[0], w, i, K, gene, lane);
                        decode_into<ORDER, MACH>(T, w, Hcap, hg, H, gfirst, in->Y[0], in->obj[0], nullptr, 0, i,
                                                 a.err, &s_over, lane);
                    }
                __syncthreads();
                gfirst = gfirst || 4 * s_over > per_round;
                probing = false;
                for (int isl = rank; isl < nisl; isl += CS)
                    for (int c = threadIdx.x; c < I; c += blockDim.x) mx = max(mx, (long long)in->obj[0][isl * I + c]);
            }
#pragma unroll
            for (int off = 16; off; off >>= 1) mx = max(mx, __shfl_xor_sync(kFull, mx, off));
            if (lane == 0) s_red[warp] = mx;
            __syncthreads();
            if (threadIdx.x == 0) {
                for (int q = 1; q < W; ++q) mx = max(mx, s_red[q]);
                s_red[0] = mx;
            }
            cluster.sync();  // every CTA's maximum is in its s_red[0]
            if (threadIdx.x == 0) {
                long long m = 0;
                for (int r = 0; r < CS; ++r) m = max(m, *cluster.map_shared_rank(&s_red[0], r));
                long long e = 10;  // E_max = 10^a, the smallest a >= 1 above every initial objective
                while (e <= m) e *= 10;
                s_red[1] = e;
            }
            cluster.sync();  // no CTA overwrites s_red[0] before every CTA has read it
            emax = s_red[1];
            if (fits) {
                for (int isl = rank; isl < nisl; isl += CS)
                    for (int c = threadIdx.x; c < I; c += blockDim.x) {
                        const long long f = emax - in->obj[0][isl * I + c];
                        in->fit[0][isl * I + c] = f > 0 ? f : 0;
                    }
                __syncthreads();
                for (int isl = rank + warp * CS; isl < nisl; isl += W * CS) {
                    int best, worst;
                    warp_extremes(in->fit[0], isl * I, I, lane, best, worst);
                    warp_copy_ind(in->bY + (size_t)isl * K, in->bX + (size_t)isl * K, in->Y[0] + (size_t)best * K,
                                  in->X[0] + (size_t)best * K, K, lane);
                    if (lane == 0) {
                        in->bobj[isl] = __ldcg(in->obj[0] + best);
                        in->bfit[isl] = __ldcg(in->fit[0] + best);
                    }
                }
            }
            __syncthreads();
        }

        bool stopped = false;
        for (int step = 0; step < a.generations; ++step) {
            if (a.stop) {  // a stop request ends the cluster at this generation boundary
                if (rank == 0 && threadIdx.x == 0) s_stop[step & 1] = *a.stop != 0;
                cluster.sync();  // every CTA acts on rank 0's reading
                if (*cluster.map_shared_rank(&s_stop[step & 1], 0)) {
                    stopped = true;
                    break;
                }
            }
            const int cur = gen & 1, nx = cur ^ 1;
            const uint32_t g1 = (uint32_t)gen + 1;
            const bool migrate = a.migrate_every > 0 && (int)g1 % a.migrate_every == 0 && nisl > 1;
            if (fits) {
                const GASrc src{in->Y[cur], in->X[cur], in->fit[cur], P, I, K, a.tour_k, a.side,
                                a.pc_thr, a.pm_thr, a.seed, in->iid, 1};
                // children t = 0 .. per_round-1 of this CTA's islands (rank, rank + CS, ...), taken
                // one at a time by whichever warp is free, so slow decodes do not pile up on one
                // warp (a child's result depends only on its index)
                for (;;) {
                    int t = 0;
                    if (lane == 0) t = atomicAdd(&s_next, 1);
                    t = __shfl_sync(kFull, t, 0);
                    if (t >= per_round) break;
                    const int i = (rank + (t / I) * CS) * I + t % I;
                    make_child<MACH>(T, w, src, i, g1, lane);
                    write_ind(in->Y[nx], in->X[nx], w, i, K, gene, lane);
                    decode_into<ORDER, MACH>(T, w, Hcap, hg, H, gfirst, in->Y[nx], in->obj[nx], in->fit[nx], emax,
                                             i, a.err, &s_over, lane);
                }
                __syncthreads();
                if (threadIdx.x == 0) s_next = 0;  // the next generation starts after another barrier
                if (probing) {
                    gfirst = gfirst || 4 * s_over > per_round;
                    probing = false;
                }
                for (int isl = rank + warp * CS; isl < nisl; isl += W * CS)
                    island_replace(in->Y[nx], in->X[nx], in->obj[nx], in->fit[nx], in->bY, in->bX, in->bobj,
                                   in->bfit, isl, I, K, migrate, in->mY, in->mX, in->mobj, in->mfit, in->mw, lane);
            }
            __threadfence();
            if (migrate) {
                cluster.sync();  // every island's migrant is recorded
                if (fits) {
                    for (int isl = rank + warp * CS; isl < nisl; isl += W * CS)
                        migrate_edge(in->Y[nx], in->X[nx], in->obj[nx], in->fit[nx], in->mY, in->mX, in->mobj,
                                     in->mfit, in->mw, isl, nisl, K, lane);
                }
                __threadfence();
            }
            if (migrate || a.tour_k == 0) cluster.sync();  // migrants read; neighbours' children ready
            else __syncthreads();
            gen = (int)g1;
        }
        if (rank == 0 && threadIdx.x == 0) {
            in->gen = gen;
            in->emax = emax;
            if (stopped) *a.stop = 2;
        }
        cluster.sync();
        if (stopped) break;  // no further instance (the whole cluster decided alike)
    }
}

// The maximum dynamic shared memory is a per-kernel setting shared by every batch in the
// process, so it is only ever raised.
template <typename KernelT>
cudaError_t raise_smem(KernelT kernel, int v, int smem_bytes) {
    static std::mutex mu;
    static int have[4] = {48 * 1024, 48 * 1024, 48 * 1024, 48 * 1024};
    std::lock_guard<std::mutex> lk(mu);
    if (smem_bytes <= have[v]) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if (e == cudaSuccess) have[v] = smem_bytes;
    return e;
}

template <typename Fn>
cudaError_t with_kernel(int order, int mach, Fn fn) {
    if (order == kOrderStage && mach == kMachEarliest) return fn(k_batch<kOrderStage, kMachEarliest>, 0);
    if (order == kOrderStage && mach == kMachGene) return fn(k_batch<kOrderStage, kMachGene>, 1);
    if (order == kOrderTopo && mach == kMachEarliest) return fn(k_batch<kOrderTopo, kMachEarliest>, 2);
    return fn(k_batch<kOrderTopo, kMachGene>, 3);
}

}  // namespace

#ifdef FFS_CHECKED
unsigned int bounds_faults_batch() { return bounds_faults_take(); }
#endif

cudaError_t prepare_batch(int order, int mach, int smem_bytes) {
    return with_kernel(order, mach, [&](auto kernel, int v) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
        return raise_smem(kernel, v, smem_bytes);
    });
}

cudaError_t batch_max_clusters(int order, int mach, int cluster, int warps, int smem_bytes, int *clusters) {
    return with_kernel(order, mach, [&](auto kernel, int) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cluster;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(cluster, 1, 1);
        cfg.blockDim = dim3(warps * 32, 1, 1);
        cfg.dynamicSmemBytes = smem_bytes;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaOccupancyMaxActiveClusters(clusters, kernel, &cfg);
    });
}

cudaError_t launch_batch(int order, int mach, const BatchArgs &a, int grid, int warps, int cluster,
                         cudaStream_t st) {
    cudaError_t e = with_kernel(order, mach, [&](auto kernel, int) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cluster;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(grid, 1, 1);
        cfg.blockDim = dim3(warps * 32, 1, 1);
        cfg.dynamicSmemBytes = a.smem_bytes;
        cfg.stream = st;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, kernel, a);
    });
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace edffs
