// ffs_surrogate.cu -- the learned fitness surrogate and surrogate-assisted GA generations.
//
// A surrogate belongs to one instance at its current rescheduling point.  Its input is, per
// gene, the gene's rank among its stage's genes (the order the stage-by-stage decoder
// follows), scaled to (0, 1], times (1, p / max p, D / max D).  Its parameters
// (W1 [H x 3K], b1 [H], W2 [H x H], b2 [H], w3 [H], b3, FP32 masters with BF16 copies for
// the tensor cores) are trained online by Adam on the exact objectives of the children the
// GA keeps.  With a surrogate attached, a generation over-generates F candidates per slot,
// scores all of them with one batched forward pass, decodes exactly only the best-scored
// candidate of each slot, and takes one training step on those exact results.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "ffs.h"
#include "ffs_internal.h"
#include "ffs_mlp.cuh"

using namespace edffs;
using namespace ffs_rt;

struct ffs_surrogate {
    ffs_instance *inst = nullptr;
    int version = 0;
    cudaStream_t st = nullptr;
    int H = 256, K = 0, Kpad = 0, rows_cap = 0;
    size_t n_params = 0, off_W1 = 0, off_b1 = 0, off_W2 = 0, off_b2 = 0, off_w3 = 0, off_b3 = 0;
    float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
    int *step = nullptr;
    float *ph = nullptr, *dh = nullptr;
    int8_t *gstg = nullptr;   // stage of every gene
    int32_t *soff = nullptr;  // [g+1] first gene of every stage in stage order
    int g = 0;
    __nv_bfloat16 *V = nullptr, *W2b = nullptr, *W2Tb = nullptr, *w3b = nullptr;
    __nv_bfloat16 *Yh = nullptr, *YhT = nullptr, *H1 = nullptr, *H2 = nullptr, *dz2b = nullptr, *dz2T = nullptr,
                  *H1T = nullptr, *dz1b = nullptr, *dz1T = nullptr;
    float *out = nullptr, *t = nullptr, *dout = nullptr, *dz2 = nullptr, *dh1 = nullptr, *dz1 = nullptr, *G = nullptr;
    // diagnostic: candidates scored by their exact objective instead of the network
    int exact = 0;
    int64_t *cand_obj = nullptr;
    size_t cand_obj_cap = 0;

    ~ffs_surrogate() {
        dfree(cand_obj);
        dfree(params); dfree(grads); dfree(m); dfree(v); dfree(step); dfree(ph); dfree(dh); dfree(gstg); dfree(soff);
        dfree(V); dfree(W2b); dfree(W2Tb); dfree(w3b);
        dfree(Yh); dfree(YhT); dfree(H1); dfree(H2); dfree(dz2b); dfree(dz2T); dfree(H1T); dfree(dz1b); dfree(dz1T);
        dfree(out); dfree(t); dfree(dout); dfree(dz2); dfree(dh1); dfree(dz1); dfree(G);
    }
};

namespace {

constexpr float kBeta1 = 0.9f, kBeta2 = 0.999f, kEps = 1e-8f;

int round_up(int x, int a) { return (x + a - 1) / a * a; }

// BF16 copies of the weights; V from W1 and the gene features.
int sync_weights(ffs_surrogate *s, cudaStream_t st) {
    FFS_CUDA(mlp_make_v(s->params + s->off_W1, s->ph, s->dh, s->H, s->K, s->Kpad, s->V, st));
    FFS_CUDA(mlp_to_bf16(s->params + s->off_W2, (size_t)s->H * s->H, s->W2b, st));
    FFS_CUDA(mlp_transpose(s->W2b, s->H, s->H, s->W2Tb, st));
    FFS_CUDA(mlp_to_bf16(s->params + s->off_w3, (size_t)s->H, s->w3b, st));
    return FFS_OK;
}

// out = w3 . relu(W2 relu(V yh + b1) + b2) + b3 for rows_pad rows of Yh.
int forward(ffs_surrogate *s, const __nv_bfloat16 *Yh, int rows_pad, __nv_bfloat16 *H1, __nv_bfloat16 *H2,
            float *out, cudaStream_t st) {
    FFS_CUDA(mlp_gemm(kEpiBiasReluBf16, Yh, s->V, rows_pad, s->H, s->Kpad, H1, s->H, s->params + s->off_b1, st));
    FFS_CUDA(mlp_gemm(kEpiBiasReluBf16, H1, s->W2b, rows_pad, s->H, s->H, H2, s->H, s->params + s->off_b2, st));
    FFS_CUDA(mlp_rowdot(H2, s->w3b, s->params + s->off_b3, rows_pad, s->H, out, st));
    return FFS_OK;
}

// Gradients of the mean squared error to the normalised objectives of the first `rows` of
// s->Yh (activations of the last forward on s->Yh in s->H1/H2/out); Adam if `update`.
int backward(ffs_surrogate *s, const int64_t *obj, int rows, int rows_pad, bool update, float lr, cudaStream_t st) {
    const int H = s->H;
    FFS_CUDA(mlp_targets(obj, rows, s->t, update ? s->step : nullptr, st));
    FFS_CUDA(mlp_backward_out(s->out, s->t, rows, rows_pad, s->H2, s->w3b, H, s->dout, s->dz2, s->dz2b,
                              s->grads + s->off_w3, s->grads + s->off_b3, s->grads + s->off_b2, st));
    FFS_CUDA(mlp_gemm(kEpiF32, s->dz2b, s->W2Tb, rows_pad, H, H, s->dh1, H, nullptr, st));  // dH1 = dZ2 W2
    FFS_CUDA(mlp_backward_hidden(s->dh1, s->H1, rows_pad, H, s->dz1, s->dz1b, s->grads + s->off_b1, st));
    FFS_CUDA(mlp_transpose(s->dz2b, rows_pad, H, s->dz2T, st));
    FFS_CUDA(mlp_transpose(s->H1, rows_pad, H, s->H1T, st));
    FFS_CUDA(mlp_transpose(s->dz1b, rows_pad, H, s->dz1T, st));
    FFS_CUDA(mlp_transpose(s->Yh, rows_pad, s->Kpad, s->YhT, st));
    FFS_CUDA(mlp_gemm(kEpiF32, s->dz2T, s->H1T, H, H, rows_pad, s->grads + s->off_W2, H, nullptr, st));  // dW2
    FFS_CUDA(mlp_gemm(kEpiF32, s->dz1T, s->YhT, H, s->Kpad, rows_pad, s->G, s->Kpad, nullptr, st));     // G
    FFS_CUDA(mlp_grad_w1(s->G, s->Kpad, s->ph, s->dh, H, s->K, s->grads + s->off_W1, st));
    if (update) FFS_CUDA(mlp_adam(s->params, s->grads, s->m, s->v, s->n_params, lr, kBeta1, kBeta2, kEps, s->step, st));
    return FFS_OK;
}

uint64_t splitmix(uint64_t &x) {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

int check_batch(ffs_surrogate *s, int count) {
    if (!s || count < 1 || count > s->rows_cap) return FFS_E_ARG;
    if (s->version != s->inst->version) return FFS_E_STATE;
    return FFS_OK;
}

// Loss on the host from the device outputs and targets of the first `rows` rows.
int host_loss(ffs_surrogate *s, int rows, float *loss) {
    std::vector<float> o(rows), t(rows);
    FFS_CUDA(cudaStreamSynchronize(s->st));
    FFS_TRY(ffs_rt::surrogate_status());
    FFS_CUDA(cudaMemcpy(o.data(), s->out, 4 * (size_t)rows, cudaMemcpyDeviceToHost));
    FFS_CUDA(cudaMemcpy(t.data(), s->t, 4 * (size_t)rows, cudaMemcpyDeviceToHost));
    double acc = 0;
    for (int r = 0; r < rows; ++r) acc += (double)(o[r] - t[r]) * (o[r] - t[r]);
    *loss = (float)(acc / rows);
    return FFS_OK;
}

}  // namespace

extern "C" {

int ffs_surrogate_create(ffs_instance *in, int32_t max_batch, uint64_t seed, void *stream, ffs_surrogate **out) {
    if (!in || !out || max_batch < 1 || in->K < 1) return FFS_E_ARG;
    *out = nullptr;
    ffs_surrogate *s = new (std::nothrow) ffs_surrogate();
    if (!s) return FFS_E_NOMEM;
    auto fail = [&](int rc) {
        delete s;
        return rc;
    };
    s->inst = in;
    s->version = in->version;
    s->st = static_cast<cudaStream_t>(stream);
    const int H = s->H, K = in->K;
    s->K = K;
    s->Kpad = round_up(K, 128);
    s->rows_cap = round_up(max_batch, 128);
    s->off_W1 = 0;
    s->off_b1 = s->off_W1 + (size_t)H * 3 * K;
    s->off_W2 = s->off_b1 + H;
    s->off_b2 = s->off_W2 + (size_t)H * H;
    s->off_w3 = s->off_b2 + H;
    s->off_b3 = s->off_w3 + H;
    s->n_params = s->off_b3 + 1;
    const size_t R = s->rows_cap, Kp = s->Kpad, NP = s->n_params;
    bool ok = dalloc(&s->params, NP) == cudaSuccess && dalloc(&s->grads, NP) == cudaSuccess &&
              dalloc(&s->m, NP) == cudaSuccess && dalloc(&s->v, NP) == cudaSuccess && dalloc(&s->step, 1) == cudaSuccess &&
              dalloc(&s->ph, (size_t)K) == cudaSuccess && dalloc(&s->dh, (size_t)K) == cudaSuccess &&
              dalloc(&s->gstg, (size_t)K) == cudaSuccess && dalloc(&s->soff, (size_t)in->g + 1) == cudaSuccess &&
              dalloc(&s->V, (size_t)H * Kp) == cudaSuccess && dalloc(&s->W2b, (size_t)H * H) == cudaSuccess &&
              dalloc(&s->W2Tb, (size_t)H * H) == cudaSuccess && dalloc(&s->w3b, (size_t)H) == cudaSuccess &&
              dalloc(&s->Yh, R * Kp) == cudaSuccess && dalloc(&s->YhT, Kp * R) == cudaSuccess &&
              dalloc(&s->H1, R * H) == cudaSuccess && dalloc(&s->H2, R * H) == cudaSuccess &&
              dalloc(&s->dz2b, R * H) == cudaSuccess && dalloc(&s->dz2T, R * H) == cudaSuccess &&
              dalloc(&s->H1T, R * H) == cudaSuccess && dalloc(&s->dz1b, R * H) == cudaSuccess &&
              dalloc(&s->dz1T, R * H) == cudaSuccess && dalloc(&s->out, R) == cudaSuccess &&
              dalloc(&s->t, R) == cudaSuccess && dalloc(&s->dout, R) == cudaSuccess &&
              dalloc(&s->dz2, R * H) == cudaSuccess && dalloc(&s->dh1, R * H) == cudaSuccess &&
              dalloc(&s->dz1, R * H) == cudaSuccess && dalloc(&s->G, (size_t)H * Kp) == cudaSuccess;
    if (!ok) return fail(FFS_E_NOMEM);
    // gene features: processing time over the largest, due date over the largest magnitude
    std::vector<double> pk(K), dk(K);
    double pmax = 1.0, dmax = 1.0;
    for (int k = 0; k < K; ++k) {
        const int j = in->gjob[k], st = in->gstg[k];
        pk[k] = in->p[j * in->g + st];
        dk[k] = in->D[j];
        pmax = std::max(pmax, pk[k]);
        dmax = std::max(dmax, std::fabs(dk[k]));
    }
    std::vector<float> phf(K), dhf(K);
    for (int k = 0; k < K; ++k) {
        phf[k] = (float)(pk[k] / pmax);
        dhf[k] = (float)(dk[k] / dmax);
    }
    // He-uniform hidden layers, small output layer, zero biases
    std::vector<float> p0(NP, 0.f);
    uint64_t x = seed;
    auto uni = [&](double lim) { return (float)(((splitmix(x) >> 11) * (1.0 / 9007199254740992.0) * 2 - 1) * lim); };
    for (size_t i = 0; i < (size_t)H * 3 * K; ++i) p0[s->off_W1 + i] = uni(std::sqrt(6.0 / (3.0 * K)));
    for (size_t i = 0; i < (size_t)H * H; ++i) p0[s->off_W2 + i] = uni(std::sqrt(6.0 / H));
    for (int i = 0; i < H; ++i) p0[s->off_w3 + i] = uni(1.0 / std::sqrt((double)H));
    s->g = in->g;
    std::vector<int8_t> gs(K);
    std::vector<int32_t> so(in->g + 1, 0);
    for (int k = 0; k < K; ++k) {
        gs[k] = (int8_t)in->gstg[k];
        so[in->gstg[k] + 1]++;
    }
    for (int q = 0; q < in->g; ++q) so[q + 1] += so[q];
    int rc = cuda_rc(cudaMemcpy(s->ph, phf.data(), 4 * (size_t)K, cudaMemcpyHostToDevice));
    if (rc == FFS_OK) rc = cuda_rc(cudaMemcpy(s->gstg, gs.data(), (size_t)K, cudaMemcpyHostToDevice));
    if (rc == FFS_OK) rc = cuda_rc(cudaMemcpy(s->soff, so.data(), 4 * ((size_t)in->g + 1), cudaMemcpyHostToDevice));
    if (rc == FFS_OK) rc = cuda_rc(cudaMemcpy(s->dh, dhf.data(), 4 * (size_t)K, cudaMemcpyHostToDevice));
    if (rc == FFS_OK) rc = ffs_surrogate_set_params(s, p0.data());
    if (rc != FFS_OK) return fail(rc);
    *out = s;
    return FFS_OK;
}

int ffs_surrogate_destroy(ffs_surrogate *s) {
    delete s;
    return FFS_OK;
}

int ffs_surrogate_param_count(const ffs_surrogate *s, int64_t *n) {
    if (!s || !n) return FFS_E_ARG;
    *n = (int64_t)s->n_params;
    return FFS_OK;
}

int ffs_surrogate_get_params(ffs_surrogate *s, float *host) {
    if (!s || !host) return FFS_E_ARG;
    FFS_CUDA(cudaStreamSynchronize(s->st));
    FFS_CUDA(cudaMemcpy(host, s->params, 4 * s->n_params, cudaMemcpyDeviceToHost));
    return FFS_OK;
}

int ffs_surrogate_set_params(ffs_surrogate *s, const float *host) {
    if (!s || !host) return FFS_E_ARG;
    FFS_CUDA(cudaStreamSynchronize(s->st));
    FFS_CUDA(cudaMemcpy(s->params, host, 4 * s->n_params, cudaMemcpyHostToDevice));
    FFS_CUDA(cudaMemset(s->m, 0, 4 * s->n_params));
    FFS_CUDA(cudaMemset(s->v, 0, 4 * s->n_params));
    FFS_CUDA(cudaMemset(s->step, 0, sizeof(int)));
    return FFS_OK;
}

int ffs_surrogate_predict(ffs_surrogate *s, const int16_t *y, int32_t count, float *out) {
    if (!s || !y || !out || count < 1) return FFS_E_ARG;
    if (s->version != s->inst->version) return FFS_E_STATE;
    FFS_TRY(sync_weights(s, s->st));
    for (int base = 0; base < count; base += s->rows_cap) {
        const int rows = std::min(s->rows_cap, count - base), rows_pad = round_up(rows, 128);
        FFS_CUDA(mlp_stage_features(y + (size_t)base * s->K, rows, rows_pad, s->K, s->Kpad, s->gstg, s->soff, s->g,
                                    s->Yh, s->st));
        FFS_TRY(forward(s, s->Yh, rows_pad, s->H1, s->H2, s->out, s->st));
        FFS_CUDA(cudaMemcpyAsync(out + base, s->out, 4 * (size_t)rows, cudaMemcpyDeviceToDevice, s->st));
    }
    ffs_rt::g_launches += 6;
    return FFS_OK;
}

int ffs_surrogate_gradients(ffs_surrogate *s, const int16_t *y, const int64_t *obj, int32_t count, float *grad_host,
                            float *loss_host) {
    FFS_TRY(check_batch(s, count));
    if (!y || !obj) return FFS_E_ARG;
    const int rows_pad = round_up(count, 128);
    FFS_TRY(sync_weights(s, s->st));
    FFS_CUDA(mlp_stage_features(y, count, rows_pad, s->K, s->Kpad, s->gstg, s->soff, s->g, s->Yh, s->st));
    FFS_TRY(forward(s, s->Yh, rows_pad, s->H1, s->H2, s->out, s->st));
    FFS_TRY(backward(s, obj, count, rows_pad, false, 0.f, s->st));
    if (loss_host) FFS_TRY(host_loss(s, count, loss_host));
    if (grad_host) {
        FFS_CUDA(cudaStreamSynchronize(s->st));
        FFS_TRY(ffs_rt::surrogate_status());
        FFS_CUDA(cudaMemcpy(grad_host, s->grads, 4 * s->n_params, cudaMemcpyDeviceToHost));
    }
    return FFS_OK;
}

int ffs_surrogate_train(ffs_surrogate *s, const int16_t *y, const int64_t *obj, int32_t count, float lr,
                        float *loss_host) {
    FFS_TRY(check_batch(s, count));
    if (!y || !obj || !(lr > 0.f)) return FFS_E_ARG;
    const int rows_pad = round_up(count, 128);
    FFS_TRY(sync_weights(s, s->st));
    FFS_CUDA(mlp_stage_features(y, count, rows_pad, s->K, s->Kpad, s->gstg, s->soff, s->g, s->Yh, s->st));
    FFS_TRY(forward(s, s->Yh, rows_pad, s->H1, s->H2, s->out, s->st));
    FFS_TRY(backward(s, obj, count, rows_pad, true, lr, s->st));
    // the targets exist once the backward pass has run; the outputs are the pre-step ones
    if (loss_host) FFS_TRY(host_loss(s, count, loss_host));
    return FFS_OK;
}

int ffs_surrogate_read_activations(ffs_surrogate *s, int32_t rows, uint16_t *h1, uint16_t *h2, float *out,
                                   float *t) {
    if (!s || rows < 0 || rows > s->rows_cap) return FFS_E_ARG;
    FFS_CUDA(cudaStreamSynchronize(s->st));
    FFS_TRY(ffs_rt::surrogate_status());
    const size_t n = (size_t)rows * s->H;
    if (h1) FFS_CUDA(cudaMemcpy(h1, s->H1, 2 * n, cudaMemcpyDeviceToHost));
    if (h2) FFS_CUDA(cudaMemcpy(h2, s->H2, 2 * n, cudaMemcpyDeviceToHost));
    if (out) FFS_CUDA(cudaMemcpy(out, s->out, 4 * (size_t)rows, cudaMemcpyDeviceToHost));
    if (t) FFS_CUDA(cudaMemcpy(t, s->t, 4 * (size_t)rows, cudaMemcpyDeviceToHost));
    return FFS_OK;
}

int ffs_tensor_gemm(const void *A, const void *B, int32_t M, int32_t N, int32_t K, const float *bias, void *C,
                    int32_t relu_bf16, int32_t synchronous, void *stream) {
    if (!A || !B || !C || (relu_bf16 && !bias)) return FFS_E_ARG;
    const cudaError_t e = mlp_gemm(relu_bf16 ? kEpiBiasReluBf16 : kEpiF32, static_cast<const __nv_bfloat16 *>(A),
                                   static_cast<const __nv_bfloat16 *>(B), M, N, K, C, N, bias,
                                   static_cast<cudaStream_t>(stream));
    if (e == cudaErrorInvalidValue) return FFS_E_ARG;
    FFS_CUDA(e);
    ffs_rt::g_launches += 1;
    if (!synchronous) return FFS_OK;
    FFS_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    return ffs_rt::surrogate_status();
}

int ga_population_attach_surrogate(ga_population *pp, ffs_surrogate *s, int32_t oversample, float lr,
                                   int32_t train_steps, int32_t screen_permille) {
    if (!pp) return FFS_E_ARG;
    if (!s) {  // detach
        pp->sur = nullptr;
        return FFS_OK;
    }
    if (s->inst != pp->inst || s->version != pp->version || oversample < 1 || oversample > 32 || !(lr > 0.f) ||
        train_steps < 0 || train_steps > 64 || screen_permille < 0 || screen_permille > 1000 ||
        (pp->P * oversample) % 128 || s->rows_cap < pp->P || pp->P % 128)
        return FFS_E_ARG;
    const size_t C = (size_t)pp->P * oversample;
    if (pp->F != oversample || !pp->cand_Y) {
        dfree(pp->cand_Y); dfree(pp->cand_X); dfree(pp->cand_Yh); dfree(pp->cand_H1); dfree(pp->cand_H2);
        dfree(pp->cand_out);
        dfree(pp->cand_new);
        if (dalloc(&pp->cand_new, C) != cudaSuccess || dalloc(&pp->cand_Y, C * pp->K) != cudaSuccess || dalloc(&pp->cand_X, C * pp->K) != cudaSuccess ||
            dalloc(&pp->cand_Yh, C * s->Kpad) != cudaSuccess || dalloc(&pp->cand_H1, C * s->H) != cudaSuccess ||
            dalloc(&pp->cand_H2, C * s->H) != cudaSuccess || dalloc(&pp->cand_out, C) != cudaSuccess)
            return FFS_E_NOMEM;
    }
    if (!pp->kept_obj && dalloc(&pp->kept_obj, (size_t)pp->P) != cudaSuccess) return FFS_E_NOMEM;
    if (!pp->cand_keep && dalloc(&pp->cand_keep, (size_t)pp->P) != cudaSuccess) return FFS_E_NOMEM;
    if (pp->keep_rule != FFS_KEEP_SLOT && oversample * pp->I > kTopMax) return FFS_E_ARG;
    pp->sur = s;
    pp->F = oversample;
    pp->lr = lr;
    pp->train_steps = train_steps;
    pp->screen_thr = (uint64_t)(uint32_t)screen_permille * ((uint64_t)1 << 32) / 1000u;
    if (pp->graph_sur) {
        cudaGraphExecDestroy(pp->graph_sur);
        pp->graph_sur = nullptr;
    }
    return FFS_OK;
}

int ffs_surrogate_score_exactly(ffs_surrogate *s, int32_t on) {
    if (!s) return FFS_E_ARG;
    s->exact = on != 0;
    return FFS_OK;
}

int ga_population_surrogate_keep(ga_population *pp, int32_t rule) {
    if (!pp || !pp->sur || (rule != FFS_KEEP_SLOT && rule != FFS_KEEP_ISLAND && rule != FFS_KEEP_ISLAND_OFFSPRING))
        return FFS_E_ARG;
    if (rule != FFS_KEEP_SLOT && pp->F * pp->I > kTopMax) {
        std::snprintf(ffs_rt::g_last_error, sizeof(ffs_rt::g_last_error),
                      "island keep rule: oversample x island = %d candidates per island, limit %d", pp->F * pp->I,
                      kTopMax);
        return FFS_E_ARG;
    }
    if (pp->keep_rule != rule && pp->graph_sur) {
        cudaGraphExecDestroy(pp->graph_sur);
        pp->graph_sur = nullptr;
    }
    pp->keep_rule = rule;
    return FFS_OK;
}

int ga_population_read_candidates(ga_population *pp, int16_t *Y, int8_t *X, float *score, int32_t *keep) {
    if (!pp || !pp->sur || !pp->cand_Y) return FFS_E_ARG;
    FFS_CUDA(cudaStreamSynchronize(pp->st));
    const size_t C = (size_t)pp->P * pp->F;
    if (Y) FFS_CUDA(cudaMemcpy(Y, pp->cand_Y, 2 * C * pp->K, cudaMemcpyDeviceToHost));
    if (X) FFS_CUDA(cudaMemcpy(X, pp->cand_X, C * pp->K, cudaMemcpyDeviceToHost));
    if (score) FFS_CUDA(cudaMemcpy(score, pp->cand_out, 4 * C, cudaMemcpyDeviceToHost));
    if (keep) FFS_CUDA(cudaMemcpy(keep, pp->cand_keep, 4 * (size_t)pp->P, cudaMemcpyDeviceToHost));
    return FFS_OK;
}

int ffs_surrogate_pretrain(ffs_surrogate *s, ga_population *pp, int32_t steps, float lr, float *loss) {
    if (!s || !pp || steps < 0 || !(lr > 0.f) || s->inst != pp->inst || s->version != pp->version ||
        pp->P > s->rows_cap)
        return FFS_E_ARG;
    FFS_CUDA(cudaStreamSynchronize(pp->st));
    GADev dv;
    FFS_CUDA(cudaMemcpy(&dv, pp->dev, sizeof(dv), cudaMemcpyDeviceToHost));
    const int b = dv.gen & 1, rows_pad = round_up(pp->P, 128);
    FFS_CUDA(mlp_stage_features(pp->Y[b], pp->P, rows_pad, s->K, s->Kpad, s->gstg, s->soff, s->g, s->Yh, s->st));
    for (int i = 0; i < steps; ++i) {
        FFS_TRY(sync_weights(s, s->st));
        FFS_TRY(forward(s, s->Yh, rows_pad, s->H1, s->H2, s->out, s->st));
        FFS_TRY(backward(s, pp->obj[b], pp->P, rows_pad, true, lr, s->st));
    }
    if (loss && steps > 0) FFS_TRY(host_loss(s, pp->P, loss));
    FFS_CUDA(cudaStreamSynchronize(s->st));
    return ffs_rt::surrogate_status();
}

}  // extern "C"

int ffs_rt::surrogate_status() { return mlp_gemm_take_error() ? FFS_E_TIMEOUT : FFS_OK; }

// One surrogate-assisted generation: candidates, their scores, the fused select + decode +
// replacement kernel, then one training step on the kept children's exact objectives.
int ffs_rt::surrogate_launches_per_generation(const ga_population *pp) {
    // exact scoring replaces the 7 launches of weight sync and forward pass with up to two
    // decode launches and one conversion
    return kSurrogateFixedLaunches + kSurrogateStepLaunches * pp->train_steps +
           (pp->keep_rule != FFS_KEEP_SLOT ? 1 : 0) - (pp->sur->exact ? 4 : 0);
}

bool ffs_rt::surrogate_is_exact(const ga_population *pp) { return pp->sur && pp->sur->exact; }

// With `phase` (six events), the phases are bracketed: candidates, scoring, keep rule,
// exact decode with replacement, training.
int ffs_rt::surrogate_enqueue_generation(ga_population *pp, cudaStream_t st, cudaEvent_t ev0, cudaEvent_t ev1,
                                         cudaEvent_t *phase) {
    ffs_surrogate *s = pp->sur;
    GenArgs a;
    ga_gen_args(pp, &a);
    a.F = pp->F;
    a.Kpad = s->Kpad;
    a.cand_Y = pp->cand_Y;
    a.cand_X = pp->cand_X;
    a.cand_Yh = pp->cand_Yh;
    a.cand_out = pp->cand_out;
    a.cand_new = pp->cand_new;
    a.kept_Yh = reinterpret_cast<uint16_t *>(s->Yh);
    a.kept_obj = pp->kept_obj;
    a.screen_thr = pp->screen_thr;
    const int C = pp->P * pp->F;
    const int grid_c = std::max(1, std::min((C + kWarpsPerBlock - 1) / kWarpsPerBlock, num_sms() * 8));
    auto mark = [&](int q) { return phase ? cuda_rc(cudaEventRecord(phase[q], st)) : FFS_OK; };
    FFS_TRY(mark(0));
    FFS_CUDA(launch_candidates(pp->par.machine_mode, a, pp->hdr, grid_c, st));
    FFS_TRY(mark(1));
    if (s->exact) {  // diagnostic: a perfect model, every candidate decoded exactly
        if ((size_t)C > s->cand_obj_cap) {
            dfree(s->cand_obj);
            FFS_CUDA(dalloc(&s->cand_obj, (size_t)C));
            s->cand_obj_cap = (size_t)C;
        }
        FFS_TRY(decode_impl(pp->inst, pp->par.order_mode, pp->par.machine_mode, pp->cand_Y, pp->cand_X, C, s->cand_obj,
                            nullptr, nullptr, nullptr, nullptr, st));
        FFS_CUDA(mlp_obj_to_score(s->cand_obj, C, pp->cand_out, st));
    } else {
        FFS_TRY(sync_weights(s, st));
        FFS_TRY(forward(s, reinterpret_cast<const __nv_bfloat16 *>(pp->cand_Yh), C,
                        reinterpret_cast<__nv_bfloat16 *>(pp->cand_H1),
                        reinterpret_cast<__nv_bfloat16 *>(pp->cand_H2), pp->cand_out, st));
    }
    FFS_TRY(mark(2));
    if (pp->keep_rule != FFS_KEEP_SLOT) {
        FFS_CUDA(launch_island_top(pp->cand_out, pp->keep_rule == FFS_KEEP_ISLAND_OFFSPRING ? pp->cand_new : nullptr,
                                   pp->P, pp->F, pp->I, pp->cand_keep, st));
        a.cand_keep = pp->cand_keep;
    }
    FFS_TRY(mark(3));
    if (ev0) FFS_CUDA(cudaEventRecord(ev0, st));
    FFS_CUDA(launch_ga_generation(pp->par.order_mode, pp->par.machine_mode, a, pp->hdr, pp->grid_gen, st));
    if (ev1) FFS_CUDA(cudaEventRecord(ev1, st));
    FFS_TRY(mark(4));
    // training steps on the kept children (inputs gathered into s->Yh, objectives in kept_obj)
    for (int step = 0; step < pp->train_steps; ++step) {
        if (step) FFS_TRY(sync_weights(s, st));
        FFS_TRY(forward(s, s->Yh, pp->P, s->H1, s->H2, s->out, st));
        FFS_TRY(backward(s, pp->kept_obj, pp->P, pp->P, true, pp->lr, st));
    }
    return mark(5);
}

int ffs_rt::prepare_surrogate_kernels(ga_population *pp) {
    FFS_CUDA(prepare_ga_generation(pp->par.order_mode, pp->par.machine_mode, pp->hdr, pp->Hcap));
    FFS_CUDA(prepare_candidates(pp->par.machine_mode, pp->hdr));
    return FFS_OK;
}
