// ffs_umma.cu -- the surrogate's dense contractions on the fifth-generation tensor cores:
// C[M x N] = A[M x K] . B[N x K]^T, BF16 operands, FP32 accumulation in tensor memory.
//
// One CTA of four warps computes a 128 x BN tile (BN = 256, or 128 when N is not a
// multiple of 256):
//   - thread 0 streams 64-wide K slices of A and B into a four-stage shared-memory ring
//     with TMA (cp.async.bulk.tensor, 128-byte swizzle), paced by full/empty mbarriers;
//   - thread 32 issues tcgen05.mma (kind::f16, M = 128, N = BN, K = 16 per instruction)
//     into a 128 x BN FP32 accumulator in tensor memory, and tcgen05.commit releases each
//     stage once the instructions reading it have completed;
//   - after the last slice, warp w reads accumulator rows 32w .. 32w+31 (its TMEM lane
//     quadrant) with tcgen05.ld and applies the epilogue (FP32 store, or bias + ReLU to
//     BF16).
// Every wait has an iteration limit.  On a timeout the CTA records kErrTimeout, stops
// issuing, waits (again bounded) for the copies it started, frees its tensor memory and
// returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>

#include "ffs_device.cuh"
#include "ffs_mlp.cuh"

namespace edffs {

namespace {

constexpr int kTM = 128;           // tile rows (UMMA M)
constexpr int kTK = 64;            // K slice per stage: 64 BF16 = one 128-byte swizzle row
constexpr int kStages = 4;
constexpr int kThreads = 128;
constexpr int kABytes = kTM * kTK * 2;
constexpr int kWaitIters = 1 << 24;
// Failure injection for tests: operand loads skipped, and this short wait limit (nothing
// is then in flight when a wait runs out).
constexpr int kInjectWaitIters = 1 << 12;
std::atomic<int> g_inject_skip_loads{0};

__device__ int32_t g_gemm_err;  // sticky kErrTimeout from any GEMM launch

template <int BN>
struct Smem {
    static constexpr int kBBytes = BN * kTK * 2;
    static constexpr int kRing = kStages * (kABytes + kBBytes);
    // ring | full[S] empty[S] done | tmem slot | counters
    static constexpr int kBytes = 1024 + kRing + 8 * (2 * kStages + 1) + 16;
};

__device__ __forceinline__ bool wait_parity(uint32_t bar, uint32_t parity, int iters) {
    for (int it = 0; it < iters; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// Shared-memory matrix descriptor of a K-major operand tile written by TMA with the
// 128-byte swizzle: rows of 128 bytes, 8-row atoms of 1024 bytes (stride-dimension offset),
// descriptor version 1, layout type 2 (128-byte swizzle).  The leading-dimension offset is
// not used by swizzled K-major layouts.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both K-major.
template <int BN>
__device__ __forceinline__ uint32_t instr_desc() {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(kTM >> 4) << 24);
}

__device__ __forceinline__ void tma_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

template <int BN, int EPI>
__global__ void __launch_bounds__(kThreads, 1)
    k_umma(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB, int K, void *C, int ldc,
           const float *__restrict__ bias, int skip_loads, int iters) {
    using L = Smem<BN>;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    uint8_t *base = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    const uint32_t sA = smem_u32(base), sB = sA + kStages * kABytes;
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + L::kRing);
    const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * kStages, done = empty0 + 8 * kStages;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2 * kStages + 1);
    volatile int32_t *ctr = reinterpret_cast<volatile int32_t *>(tslot + 1);  // [0] abort [1] issued [2] consumed
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nk = K / kTK;
    const int m0 = blockIdx.y * kTM, n0 = blockIdx.x * BN;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(full0 + 8 * s) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(empty0 + 8 * s) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(done) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        ctr[0] = 0;
        ctr[1] = 0;
        ctr[2] = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    if (warp == 0) {
        if (lane == 0) {  // TMA producer
            int kb = 0;
            for (; kb < nk && !skip_loads; ++kb) {
                const int s = kb % kStages;
                if (kb >= kStages && !wait_parity(empty0 + 8 * s, ((kb / kStages) & 1) ^ 1, iters)) {
                    ctr[0] = 1;
                    break;
                }
                if (ctr[0]) break;
                const uint32_t fb = full0 + 8 * s;
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb),
                             "r"(kABytes + L::kBBytes)
                             : "memory");
                tma_2d(sA + s * kABytes, &tA, kb * kTK, m0, fb);
                tma_2d(sB + s * L::kBBytes, &tB, kb * kTK, n0, fb);
            }
            ctr[1] = kb;
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            const uint32_t idesc = instr_desc<BN>();
            int kb = 0;
            for (; kb < nk; ++kb) {
                const int s = kb % kStages;
                if (!wait_parity(full0 + 8 * s, (kb / kStages) & 1, iters)) {
                    ctr[0] = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                for (int kk = 0; kk < kTK / 16; ++kk) {
                    const uint64_t ad = sw128_desc(sA + s * kABytes + kk * 32);
                    const uint64_t bd = sw128_desc(sB + s * L::kBBytes + kk * 32);
                    const uint32_t acc = (kb | kk) ? 1u : 0u;
                    asm volatile(
                        "{\n\t.reg .pred p;\n\t"
                        "setp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                        : "memory");
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 empty0 + 8 * s)
                             : "memory");
            }
            ctr[2] = kb;
            // arrives once every MMA issued above has completed
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(done)
                         : "memory");
        }
        __syncwarp();
    }

    const bool ok = wait_parity(done, 0, iters) && !ctr[0];
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (__all_sync(kFull, ok)) {
        const int row = m0 + 32 * warp + lane;
        const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);
#pragma unroll 1
        for (int c = 0; c < BN; c += 32) {
            uint32_t r[32];
            tmem_ld32(trow + (uint32_t)c, r);
            if (EPI == kEpiF32) {
                float4 *out = reinterpret_cast<float4 *>(static_cast<float *>(C) + (size_t)row * ldc + n0 + c);
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    out[q] = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                                         __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
            } else {
                const float *b = bias + n0 + c;
                uint32_t pk[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const float v0 = fmaxf(__uint_as_float(r[2 * q]) + b[2 * q], 0.f);
                    const float v1 = fmaxf(__uint_as_float(r[2 * q + 1]) + b[2 * q + 1], 0.f);
                    const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
                    pk[q] = *reinterpret_cast<const uint32_t *>(&h);
                }
                uint4 *out =
                    reinterpret_cast<uint4 *>(static_cast<__nv_bfloat16 *>(C) + (size_t)row * ldc + n0 + c);
#pragma unroll
                for (int q = 0; q < 4; ++q) out[q] = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0 && (!ok || ctr[0])) {
        atomicOr(&g_gemm_err, kErrTimeout);
        // copies issued but never consumed may still be landing: wait for them (bounded)
        for (int kb = ctr[2]; kb < ctr[1]; ++kb) wait_parity(full0 + 8 * (kb % kStages), (kb / kStages) & 1, iters);
    }
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
    }
}

// ---------------------------------------------------------------- host side
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
    static EncodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    });
    return fn;
}

// Row-major [rows][K] BF16 matrix, boxes of box_rows x 64 with the 128-byte swizzle.
cudaError_t make_map(CUtensorMap *m, const void *ptr, int rows, int K, int box_rows) {
    EncodeTiled fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)K * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kTK, (cuuint32_t)box_rows};
    const cuuint32_t es[2] = {1, 1};
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int BN, int EPI>
cudaError_t launch(const CUtensorMap &a, const CUtensorMap &b, int M, int N, int K, void *C, int ldc,
                   const float *bias, cudaStream_t st) {
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(k_umma<BN, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem<BN>::kBytes);
    });
    if (attr != cudaSuccess) return attr;
    const int skip = g_inject_skip_loads.load();
    k_umma<BN, EPI><<<dim3(N / BN, M / kTM), kThreads, Smem<BN>::kBytes, st>>>(a, b, K, C, ldc, bias, skip,
                                                                               skip ? kInjectWaitIters : kWaitIters);
    return cudaGetLastError();
}

}  // namespace

cudaError_t mlp_gemm(int epi, const __nv_bfloat16 *A, const __nv_bfloat16 *B, int M, int N, int K, void *C, int ldc,
                     const float *bias, cudaStream_t st) {
    if (M <= 0 || N <= 0 || K <= 0 || M % kTM || N % 128 || K % kTK || ldc % 8 || ldc < N) return cudaErrorInvalidValue;
    if (epi == kEpiBiasReluBf16 && !bias) return cudaErrorInvalidValue;
    if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B) | reinterpret_cast<uintptr_t>(C)) & 15)
        return cudaErrorInvalidValue;
    const int BN = N % 256 == 0 ? 256 : 128;
    CUtensorMap ma, mb;
    cudaError_t e = make_map(&ma, A, M, K, kTM);
    if (e == cudaSuccess) e = make_map(&mb, B, N, K, BN);
    if (e != cudaSuccess) return e;
    if (BN == 256)
        return epi == kEpiF32 ? launch<256, kEpiF32>(ma, mb, M, N, K, C, ldc, bias, st)
                              : launch<256, kEpiBiasReluBf16>(ma, mb, M, N, K, C, ldc, bias, st);
    return epi == kEpiF32 ? launch<128, kEpiF32>(ma, mb, M, N, K, C, ldc, bias, st)
                          : launch<128, kEpiBiasReluBf16>(ma, mb, M, N, K, C, ldc, bias, st);
}

void mlp_gemm_inject_skip_loads(bool on) { g_inject_skip_loads.store(on ? 1 : 0); }

int32_t mlp_gemm_take_error() {
    int32_t e = 0;
    if (cudaMemcpyFromSymbol(&e, g_gemm_err, 4) != cudaSuccess) return kErrTimeout;
    if (e) {
        const int32_t z = 0;
        cudaMemcpyToSymbol(g_gemm_err, &z, 4);
    }
    return e;
}

}  // namespace edffs
