// ffs_mlp.cuh -- launch wrappers of the surrogate kernels (ffs_mlp.cu).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace edffs {

constexpr int kEpiF32 = 0;            // C = A B^T, FP32
constexpr int kEpiBiasReluBf16 = 1;   // C = relu(A B^T + bias), BF16

// C[M x N] = A[M x K] B[N x K]^T (BF16 operands, FP32 accumulation) on the tcgen05 tensor
// cores (ffs_umma.cu); M, N multiples of 128, K a multiple of 64; ldc in elements, a
// multiple of 8; A, B and C 16-byte aligned.
cudaError_t mlp_gemm(int epi, const __nv_bfloat16 *A, const __nv_bfloat16 *B, int M, int N, int K, void *C, int ldc,
                     const float *bias, cudaStream_t st);
// Error bits (kErrTimeout) that GEMM launches recorded since the last call, and clears
// them.  Synchronous.
int32_t mlp_gemm_take_error();
// score[i] = obj[i] as FP32 (exact scoring of candidates, a diagnostic).
cudaError_t mlp_obj_to_score(const int64_t *obj, int n, float *score, cudaStream_t st);
// Failure injection for tests: GEMM launches issue no operand loads (see ffs_debug_inject).
void mlp_gemm_inject_skip_loads(bool on);
cudaError_t mlp_rowdot(const __nv_bfloat16 *h2, const __nv_bfloat16 *w3, const float *b3, int rows, int H, float *out,
                       cudaStream_t st);
cudaError_t mlp_make_v(const float *W1, const float *ph, const float *dh, int H, int K, int Kpad, __nv_bfloat16 *V,
                       cudaStream_t st);
// Within-stage rank features of `rows` chromosomes y [rows][K] into Yh [rows_pad][Kpad].
cudaError_t mlp_stage_features(const int16_t *y, int rows, int rows_pad, int K, int Kpad, const int8_t *gstg,
                               const int32_t *soff, int g, __nv_bfloat16 *Yh, cudaStream_t st);
cudaError_t mlp_transpose(const __nv_bfloat16 *in, int R, int C, __nv_bfloat16 *out, cudaStream_t st);
cudaError_t mlp_to_bf16(const float *in, size_t n, __nv_bfloat16 *out, cudaStream_t st);
cudaError_t mlp_targets(const int64_t *obj, int rows, float *t, int *step, cudaStream_t st);
cudaError_t mlp_backward_out(const float *out, const float *t, int rows, int rows_pad, const __nv_bfloat16 *h2,
                             const __nv_bfloat16 *w3, int H, float *dout, float *dz2, __nv_bfloat16 *dz2b, float *gw3,
                             float *gb3, float *gb2, cudaStream_t st);
cudaError_t mlp_backward_hidden(const float *dh1, const __nv_bfloat16 *h1, int rows_pad, int H, float *dz1,
                                __nv_bfloat16 *dz1b, float *gb1, cudaStream_t st);
cudaError_t mlp_grad_w1(const float *G, int Kpad, const float *ph, const float *dh, int H, int K, float *gW1,
                        cudaStream_t st);
// Adam with the step count read from *step (bias corrections 1 - beta^step).
cudaError_t mlp_adam(float *p, const float *g, float *m, float *v, size_t n, float lr, float b1, float b2, float eps,
                     const int *step, cudaStream_t st);

}  // namespace edffs
