// ffs_mlp.cu -- kernels of the learned fitness surrogate: a 3-layer perceptron over a
// chromosome's priorities and its genes' features (H = 256 hidden units, BF16 weights and
// activations, FP32 accumulation), its backward pass and Adam.
//
// The input features are yh_k * (1, ph_k, dh_k) per gene (yh_k = 1 - r_k / n_s, the gene's
// rank among its stage's genes), so the first layer is applied as V yh with
// V[n, k] = W1[n, 3k] + ph_k W1[n, 3k+1] + dh_k W1[n, 3k+2]; its weight gradient is
// recovered exactly as dW1[n, 3k+f] = G[n, k] c_f(k) from G = dZ1^T Yh.  Every
// contraction is one tcgen05 GEMM (ffs_umma.cu), C = A B^T with both operands
// K-contiguous; the other kernels here are elementwise or reductions in a fixed order, so
// results are reproducible.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "ffs_device.cuh"
#include "ffs_mlp.cuh"

namespace edffs {

namespace {

// out[r] = w3 . h2[r] + b3 (BF16 operands, FP32 sum, fixed order), one warp per row.
__global__ void k_rowdot(const __nv_bfloat16 *__restrict__ h2, const __nv_bfloat16 *__restrict__ w3, const float *b3,
                         int rows, int H, float *out) {
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (r >= rows) return;
    float s = 0.f;
    for (int n = lane; n < H; n += 32) s += __bfloat162float(h2[(size_t)r * H + n]) * __bfloat162float(w3[n]);
#pragma unroll
    for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) out[r] = s + b3[0];
}

// V[n, k] = W1[n, 3k] + ph_k W1[n, 3k+1] + dh_k W1[n, 3k+2] (k < K), 0 up to Kpad.
__global__ void k_make_v(const float *__restrict__ W1, const float *__restrict__ ph, const float *__restrict__ dh,
                         int H, int K, int Kpad, __nv_bfloat16 *V) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= H * Kpad) return;
    const int n = i / Kpad, k = i % Kpad;
    float v = 0.f;
    if (k < K) {
        const float *w = W1 + (size_t)n * 3 * K + 3 * k;
        v = w[0] + ph[k] * w[1] + dh[k] * w[2];
    }
    V[i] = __float2bfloat16_rn(v);
}

// Model inputs of `rows` chromosomes (within-stage rank features), one warp per row, zero
// rows up to rows_pad; each warp uses K int16 of dynamic shared memory.
__global__ void k_stage_features(const int16_t *__restrict__ y, int rows, int rows_pad, int K, int Kpad,
                                 const int8_t *__restrict__ gstg, const int32_t *__restrict__ soff, int g,
                                 __nv_bfloat16 *Yh) {
    extern __shared__ int16_t s_inv[];
    const int wpb = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = blockIdx.x * wpb + warp;
    if (r >= rows_pad) return;
    uint16_t *row = reinterpret_cast<uint16_t *>(Yh) + (size_t)r * Kpad;
    if (r >= rows) {
        for (int k = lane; k < Kpad; k += 32) row[k] = 0;
        return;
    }
    stage_rank_row(y + (size_t)r * K, K, Kpad, gstg, soff, g, s_inv + (size_t)warp * K, row, lane);
}

// Tiled transpose of a BF16 [R x C] matrix (R, C multiples of 32) into [C x R].
__global__ void k_transpose(const __nv_bfloat16 *__restrict__ in, int R, int C, __nv_bfloat16 *out) {
    __shared__ __nv_bfloat16 t[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) t[dy][threadIdx.x] = in[(size_t)(r0 + dy) * C + c0 + threadIdx.x];
    __syncthreads();
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) out[(size_t)(c0 + dy) * R + r0 + threadIdx.x] = t[threadIdx.x][dy];
}

__global__ void k_f32_to_bf16(const float *__restrict__ in, size_t n, __nv_bfloat16 *out) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = __float2bfloat16_rn(in[i]);
}

// Normalised targets t = (obj - mean) / std over `rows` (one block, fixed order, FP64).
__global__ void k_targets(const int64_t *__restrict__ obj, int rows, float *t, int *step) {
    __shared__ double s1[32], s2[32];
    double a = 0, b = 0;
    for (int r = threadIdx.x; r < rows; r += blockDim.x) {
        const double v = (double)obj[r];
        a += v;
        b += v * v;
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, off);
        b += __shfl_xor_sync(0xffffffffu, b, off);
    }
    if (l == 0) {
        s1[w] = a;
        s2[w] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q) {
            s1[0] += s1[q];
            s2[0] += s2[q];
        }
        if (step) *step += 1;  // the Adam step that these targets feed
    }
    __syncthreads();
    const double mean = s1[0] / rows, var = s2[0] / rows - mean * mean;
    const double sd = var > 0 ? sqrt(var) : 1.0;
    for (int r = threadIdx.x; r < rows; r += blockDim.x) t[r] = (float)(((double)obj[r] - mean) / sd);
}

// dout = 2 (out - t) / rows (0 in padding rows); dZ2 = dout w3 * [h2 > 0], FP32 and BF16.
__global__ void k_dz2(const float *__restrict__ out, const float *__restrict__ t, int rows, int rows_pad,
                      const __nv_bfloat16 *__restrict__ h2, const __nv_bfloat16 *__restrict__ w3, int H, float *dout,
                      float *dz2, __nv_bfloat16 *dz2b) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)rows_pad * H) return;
    const int r = (int)(i / H), n = (int)(i % H);
    const float d = r < rows ? 2.f * (out[r] - t[r]) / (float)rows : 0.f;
    if (n == 0) dout[r] = d;
    const float v = __bfloat162float(h2[i]) > 0.f ? d * __bfloat162float(w3[n]) : 0.f;
    dz2[i] = v;
    dz2b[i] = __float2bfloat16_rn(v);
}

// dZ1 = dH1 * [h1 > 0], FP32 and BF16.
__global__ void k_dz1(const float *__restrict__ dh1, const __nv_bfloat16 *__restrict__ h1, size_t n, float *dz1,
                      __nv_bfloat16 *dz1b) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float v = __bfloat162float(h1[i]) > 0.f ? dh1[i] : 0.f;
    dz1[i] = v;
    dz1b[i] = __float2bfloat16_rn(v);
}

// Column sums over rows of an FP32 [rows x cols] matrix, one thread per column, in order.
__global__ void k_colsum(const float *__restrict__ m, int rows, int cols, float *out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float s = 0.f;
    for (int r = 0; r < rows; ++r) s += m[(size_t)r * cols + c];
    out[c] = s;
}

// gw3[n] = sum_r dout[r] h2[r, n]; gb3 = sum_r dout[r] (thread H), in order.
__global__ void k_grad_out(const float *__restrict__ dout, const __nv_bfloat16 *__restrict__ h2, int rows, int H,
                           float *gw3, float *gb3) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n > H) return;
    float s = 0.f;
    for (int r = 0; r < rows; ++r) s += dout[r] * (n < H ? __bfloat162float(h2[(size_t)r * H + n]) : 1.f);
    if (n < H) gw3[n] = s;
    else gb3[0] = s;
}

// dW1[n, 3k+f] = G[n, k] c_f(k), c = (1, ph, dh).
__global__ void k_grad_w1(const float *__restrict__ G, int Kpad, const float *__restrict__ ph,
                          const float *__restrict__ dh, int H, int K, float *gW1) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= H * K) return;
    const int n = i / K, k = i % K;
    const float g = G[(size_t)n * Kpad + k];
    float *o = gW1 + (size_t)n * 3 * K + 3 * k;
    o[0] = g;
    o[1] = g * ph[k];
    o[2] = g * dh[k];
}

// One Adam step on n FP32 parameters (Kingma & Ba 2015), step count *step >= 1.
__global__ void k_adam(float *p, const float *g, float *m, float *v, size_t n, float lr, float b1, float b2,
                       float eps, const int *step) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float t = (float)*step;
    const float bc1 = 1.f - powf(b1, t), bc2 = 1.f - powf(b2, t);
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi, vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

__global__ void k_obj_to_score(const int64_t *__restrict__ obj, int n, float *score) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) score[i] = (float)obj[i];
}

unsigned blocks(size_t n, unsigned t) { return (unsigned)((n + t - 1) / t); }

}  // namespace


cudaError_t mlp_rowdot(const __nv_bfloat16 *h2, const __nv_bfloat16 *w3, const float *b3, int rows, int H, float *out,
                       cudaStream_t st) {
    k_rowdot<<<blocks(rows, 8), 256, 0, st>>>(h2, w3, b3, rows, H, out);
    return cudaGetLastError();
}

cudaError_t mlp_make_v(const float *W1, const float *ph, const float *dh, int H, int K, int Kpad, __nv_bfloat16 *V,
                       cudaStream_t st) {
    k_make_v<<<blocks((size_t)H * Kpad, 256), 256, 0, st>>>(W1, ph, dh, H, K, Kpad, V);
    return cudaGetLastError();
}

cudaError_t mlp_stage_features(const int16_t *y, int rows, int rows_pad, int K, int Kpad, const int8_t *gstg,
                               const int32_t *soff, int g, __nv_bfloat16 *Yh, cudaStream_t st) {
    const int wpb = std::max(1, std::min(8, (40 * 1024) / (2 * K)));
    const int smem = wpb * 2 * K;
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(k_stage_features, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    k_stage_features<<<blocks(rows_pad, wpb), wpb * 32, smem, st>>>(y, rows, rows_pad, K, Kpad, gstg, soff, g, Yh);
    return cudaGetLastError();
}

cudaError_t mlp_transpose(const __nv_bfloat16 *in, int R, int C, __nv_bfloat16 *out, cudaStream_t st) {
    if (R % 32 || C % 32) return cudaErrorInvalidValue;
    k_transpose<<<dim3(C / 32, R / 32), dim3(32, 8), 0, st>>>(in, R, C, out);
    return cudaGetLastError();
}

cudaError_t mlp_to_bf16(const float *in, size_t n, __nv_bfloat16 *out, cudaStream_t st) {
    k_f32_to_bf16<<<blocks(n, 256), 256, 0, st>>>(in, n, out);
    return cudaGetLastError();
}

cudaError_t mlp_targets(const int64_t *obj, int rows, float *t, int *step, cudaStream_t st) {
    k_targets<<<1, 1024, 0, st>>>(obj, rows, t, step);
    return cudaGetLastError();
}

cudaError_t mlp_backward_out(const float *out, const float *t, int rows, int rows_pad, const __nv_bfloat16 *h2,
                             const __nv_bfloat16 *w3, int H, float *dout, float *dz2, __nv_bfloat16 *dz2b, float *gw3,
                             float *gb3, float *gb2, cudaStream_t st) {
    k_dz2<<<blocks((size_t)rows_pad * H, 256), 256, 0, st>>>(out, t, rows, rows_pad, h2, w3, H, dout, dz2, dz2b);
    k_grad_out<<<blocks(H + 1, 256), 256, 0, st>>>(dout, h2, rows_pad, H, gw3, gb3);
    k_colsum<<<blocks(H, 256), 256, 0, st>>>(dz2, rows_pad, H, gb2);
    return cudaGetLastError();
}

cudaError_t mlp_backward_hidden(const float *dh1, const __nv_bfloat16 *h1, int rows_pad, int H, float *dz1,
                                __nv_bfloat16 *dz1b, float *gb1, cudaStream_t st) {
    k_dz1<<<blocks((size_t)rows_pad * H, 256), 256, 0, st>>>(dh1, h1, (size_t)rows_pad * H, dz1, dz1b);
    k_colsum<<<blocks(H, 256), 256, 0, st>>>(dz1, rows_pad, H, gb1);
    return cudaGetLastError();
}

cudaError_t mlp_grad_w1(const float *G, int Kpad, const float *ph, const float *dh, int H, int K, float *gW1,
                        cudaStream_t st) {
    k_grad_w1<<<blocks((size_t)H * K, 256), 256, 0, st>>>(G, Kpad, ph, dh, H, K, gW1);
    return cudaGetLastError();
}

cudaError_t mlp_obj_to_score(const int64_t *obj, int n, float *score, cudaStream_t st) {
    k_obj_to_score<<<blocks(n, 256), 256, 0, st>>>(obj, n, score);
    return cudaGetLastError();
}

cudaError_t mlp_adam(float *p, const float *g, float *m, float *v, size_t n, float lr, float b1, float b2, float eps,
                     const int *step, cudaStream_t st) {
    k_adam<<<blocks(n, 256), 256, 0, st>>>(p, g, m, v, n, lr, b1, b2, eps, step);
    return cudaGetLastError();
}

}  // namespace edffs
