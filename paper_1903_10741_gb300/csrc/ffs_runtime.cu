// ffs_runtime.cu -- host runtime behind the C ABI of include/ffs.h.
//
// An ffs_instance keeps the problem (Table 2), the committed plan and the classification
// of every operation at the current rescheduling point (Alg. 1), and mirrors them on the
// device as one table blob.  A ga_population keeps the GA state on the device; one
// generation is five kernels (fused selection/crossover/mutation/decode, overflow
// fallback decode, elitist replacement, migration, counter advance) captured once in a
// CUDA graph and replayed.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "ffs.h"
#include "ffs_internal.h"
#include "ffs_kernels.cuh"
#include "ffs_layout.h"
#include "ffs_mlp.cuh"

using namespace edffs;
using namespace ffs_rt;

namespace ffs_rt {

std::atomic<unsigned long long> g_launches{0};  // kernels issued by this library

constexpr int kSmemBudget = 112 * 1024;  // per CTA: two CTAs of four warps per SM
constexpr int kMinSmemSlots = 256;       // below this the shared-memory profile is not worth it
constexpr int kMaxN = 32767, kMaxG = 127, kMaxO = 31, kMaxM = 32767, kMaxP = 32767, kMaxQ = 32767;

int num_sms() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
    }
    return n;
}

}  // namespace

namespace ffs_rt {

thread_local char g_last_error[256] = "";

int cuda_rc(cudaError_t e) {
    if (e == cudaSuccess) return FFS_OK;
    std::snprintf(g_last_error, sizeof(g_last_error), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
    return FFS_E_CUDA;
}


int op_p(const ffs_instance *in, int j, int s, int m) {
    return in->unrel ? in->pm[(size_t)j * in->M + in->moff[s] + m] : in->p[j * in->g + s];
}

int op_q(const ffs_instance *in, int j, int s, int m) {
    return in->unrel ? in->qm[(size_t)j * in->M + in->moff[s] + m] : in->q[in->moff[s] + m];
}

// Rebuilds the gene map, the profile bound and the table blob, and uploads them.
int rebuild(ffs_instance *in) {
    const int N = in->N, g = in->g, M = in->M, RS = in->RS;
    in->gjob.clear();
    in->gstg.clear();
    std::vector<int16_t> gfirst(N, -1);
    std::vector<int8_t> gcnt(N, 0);
    std::vector<int32_t> C0(N, 0), mfree0(M, RS);
    long long base = RS, work = 0, exec_end = RS;
    for (int j = 0; j < N; ++j) {
        base = std::max<long long>(base, in->R[j]);
        for (int s = 0; s < g; ++s) {
            const int k = j * g + s;
            if (in->status[k] == kStFree) {
                if (gfirst[j] < 0) gfirst[j] = (int16_t)in->gjob.size();
                gcnt[j]++;
                in->gjob.push_back(j);
                in->gstg.push_back(s);
                int pmax = 0;  // the slowest of the op's machines
                for (int m = 0; m < in->o[s]; ++m) pmax = std::max(pmax, op_p(in, j, s, m));
                work += pmax;
            } else {
                const int end = in->S0[k] + op_p(in, j, s, in->M0[k]);
                C0[j] = end;  // frozen ops form a prefix of the job's stages
                if (in->status[k] == kStExec || in->status[k] == kStFixed) {  // draws power past RS
                    const int mg = in->moff[s] + in->M0[k];
                    mfree0[mg] = std::max(mfree0[mg], end);
                    exec_end = std::max<long long>(exec_end, end);
                }
            }
        }
    }
    base = std::max(base, exec_end);
    const long long H = ((base - RS + work + 1) + 7) / 8 * 8;
    // start times are packed with a 5-bit machine index into 32-bit keys
    if (H >= (1ll << 26) || (long long)RS + H > INT32_MAX) return FFS_E_ARG;
    in->K = (int)in->gjob.size();
    if (in->K > kMaxK) return FFS_E_ARG;
    in->Hfull = (int)H;
    const int E0 = (int)(exec_end - RS);
    std::vector<uint16_t> h0(E0, (uint16_t)in->Qmax);
    for (int j = 0; j < N; ++j)
        for (int s = 0; s < g; ++s) {
            const int k = j * g + s;
            if (in->status[k] != kStExec && in->status[k] != kStFixed) continue;
            const int q = op_q(in, j, s, in->M0[k]);
            for (int t = std::max(RS, in->S0[k]); t < in->S0[k] + op_p(in, j, s, in->M0[k]); ++t)
                h0[t - RS] = (uint16_t)(h0[t - RS] - q);
        }

    TabHeader h{};
    h.N = N; h.g = g; h.M = M; h.K = in->K;
    h.RS = RS; h.Qmax = in->Qmax; h.WT = in->WT; h.H = in->Hfull; h.E0 = E0; h.maxo = 0;
    for (int s = 0; s < g; ++s) h.maxo = std::max(h.maxo, in->o[s]);
    int off = align16((int)sizeof(TabHeader));
    auto take = [&](int32_t &field, int bytes) {
        field = off;
        off += align16(bytes);
    };
    take(h.off_o, 4 * g);
    take(h.off_moff, 4 * (g + 1));
    take(h.off_q, 4 * M);
    take(h.off_p, 2 * N * g);
    take(h.off_R, 4 * N);
    take(h.off_D, 4 * N);
    take(h.off_C0, 4 * N);
    take(h.off_mfree0, 4 * M);
    take(h.off_gjob, 2 * in->K);
    take(h.off_gstg, in->K);
    take(h.off_gfirst, 2 * N);
    take(h.off_gcnt, N);
    take(h.off_h0, 2 * E0);
    take(h.off_grec, 8 * in->K);
    take(h.off_soff, 4 * (g + 1));
    h.unrel = in->unrel ? 1 : 0;
    if (in->unrel) take(h.off_gm, 4 * in->K * h.maxo);
    h.bytes = off;
    in->hdr = h;
    in->blob.assign(off, 0);
    char *b = in->blob.data();
    std::memcpy(b, &h, sizeof(h));
    std::memcpy(b + h.off_o, in->o.data(), 4 * g);
    std::memcpy(b + h.off_moff, in->moff.data(), 4 * (g + 1));
    std::memcpy(b + h.off_q, in->q.data(), 4 * M);
    int16_t *pp = reinterpret_cast<int16_t *>(b + h.off_p);
    for (int i = 0; i < N * g; ++i) pp[i] = (int16_t)in->p[i];
    std::memcpy(b + h.off_R, in->R.data(), 4 * N);
    std::memcpy(b + h.off_D, in->D.data(), 4 * N);
    std::memcpy(b + h.off_C0, C0.data(), 4 * N);
    std::memcpy(b + h.off_mfree0, mfree0.data(), 4 * M);
    int16_t *gj = reinterpret_cast<int16_t *>(b + h.off_gjob);
    int8_t *gs = reinterpret_cast<int8_t *>(b + h.off_gstg);
    for (int k = 0; k < in->K; ++k) {
        gj[k] = (int16_t)in->gjob[k];
        gs[k] = (int8_t)in->gstg[k];
    }
    std::memcpy(b + h.off_gfirst, gfirst.data(), 2 * N);
    std::memcpy(b + h.off_gcnt, gcnt.data(), N);
    if (E0) std::memcpy(b + h.off_h0, h0.data(), 2 * E0);
    int32_t *soff = reinterpret_cast<int32_t *>(b + h.off_soff);
    for (int k = 0; k < in->K; ++k) soff[in->gstg[k] + 1]++;
    for (int s = 0; s < g; ++s) soff[s + 1] += soff[s];
    uint32_t *gr = reinterpret_cast<uint32_t *>(b + h.off_grec);
    for (int k = 0; k < in->K; ++k) {
        const int j = in->gjob[k], s = in->gstg[k];
        gr[2 * k] = (uint32_t)j | ((uint32_t)s << 16) | ((uint32_t)in->o[s] << 24);
        gr[2 * k + 1] = (uint32_t)in->p[j * g + s] | ((uint32_t)in->moff[s] << 16);
    }
    if (in->unrel) {
        uint32_t *gm = reinterpret_cast<uint32_t *>(b + h.off_gm);
        for (int k = 0; k < in->K; ++k) {
            const int j = in->gjob[k], s = in->gstg[k];
            for (int m = 0; m < in->o[s]; ++m)
                gm[(size_t)k * h.maxo + m] = (uint32_t)op_p(in, j, s, m) | ((uint32_t)op_q(in, j, s, m) << 16);
        }
    }

    in->dev_dirty = true;
    in->version++;
    return FFS_OK;
}

// Uploads the tables and the committed plan if the host copy changed since the last upload.
int sync_device(ffs_instance *in) {
    if (!in->dev_dirty) return FFS_OK;
    const NoArena plain;  // instance tables outlive any service arena
    const int off = in->hdr.bytes;
    if ((size_t)off > in->d_blob_cap) {
        dfree(in->d_blob);
        FFS_CUDA(dalloc(&in->d_blob, (size_t)off));
        in->d_blob_cap = off;
    }
    FFS_CUDA(cudaMemcpy(in->d_blob, in->blob.data(), off, cudaMemcpyHostToDevice));
    const size_t NG = (size_t)in->N * in->g;
    if (NG > in->d_plan_cap) {
        dfree(in->d_S0);
        dfree(in->d_M0);
        dfree(in->d_status);
        FFS_CUDA(dalloc(&in->d_S0, NG));
        FFS_CUDA(dalloc(&in->d_M0, NG));
        FFS_CUDA(dalloc(&in->d_status, NG));
        in->d_plan_cap = NG;
    }
    FFS_CUDA(cudaMemcpy(in->d_S0, in->S0.data(), 4 * NG, cudaMemcpyHostToDevice));
    FFS_CUDA(cudaMemcpy(in->d_M0, in->M0.data(), 4 * NG, cudaMemcpyHostToDevice));
    FFS_CUDA(cudaMemcpy(in->d_status, in->status.data(), 4 * NG, cudaMemcpyHostToDevice));
    if (!in->d_over_count) {
        FFS_CUDA(dalloc(&in->d_over_count, 1));
        FFS_CUDA(dalloc(&in->d_err, 1));
        FFS_CUDA(cudaMemset(in->d_err, 0, 4));
    }
    in->dev_dirty = false;
    return FFS_OK;
}

// Profile slots per warp that fit the shared-memory budget (0 if too few to be useful);
// with insertion each slot also needs a bit per machine of the widest stage.
int smem_slots(const TabHeader &h, bool ga, bool insert) {
    const int fixed = cta_smem_bytes(h, 0, ga, true);
    const int per_warp = (kSmemBudget - fixed) / kWarpsPerBlock;
    int slots = per_warp / 2 / 8 * 8;
    if (insert) {
        slots = (int)((long long)per_warp * 32 / (64 + 4 * h.maxo)) / 32 * 32;
        while (slots > 0 && profile_bytes(slots, h.maxo) > per_warp) slots -= 32;
    }
    if (slots < kMinSmemSlots) return 0;
    return std::min(slots, h.H);
}

int ensure_scratch(uint16_t **p, size_t *cap, size_t elems) {
    if (elems > *cap) {
        dfree(*p);
        FFS_CUDA(dalloc(p, elems));
        *cap = elems;
    }
    return FFS_OK;
}

int check_modes(int32_t order_mode, int32_t machine_mode) {
    const int mach = machine_mode & ~FFS_PLACE_INSERT;
    if ((order_mode != FFS_ORDER_TOPO && order_mode != FFS_ORDER_STAGE) ||
        (mach != FFS_MACH_GENE && mach != FFS_MACH_EARLIEST))
        return FFS_E_ARG;
    if ((machine_mode & FFS_PLACE_INSERT) && order_mode != FFS_ORDER_STAGE) {
        std::snprintf(g_last_error, sizeof(g_last_error), "insertion placement needs the stage-by-stage order");
        return FFS_E_ARG;
    }
    return FFS_OK;
}

// Failure injection for tests (ffs_debug_inject): decode launches skip the table copy.
std::atomic<int> g_inject_table_copy{0};
constexpr int kInjectWaitIters = 1 << 12;

int decode_impl(ffs_instance *in, int32_t order, int32_t mach, const int16_t *y, const int8_t *x,
                int32_t count, int64_t *obj, int64_t *tard, int32_t *cmax, int32_t *S, int32_t *Mo,
                cudaStream_t st) {
    FFS_TRY(check_modes(order, mach));
    if (count < 0 || (count > 0 && (!y || !obj)) || ((mach & 1) == FFS_MACH_GENE && count > 0 && !x))
        return FFS_E_ARG;
    const bool ins = (mach & FFS_PLACE_INSERT) != 0;
    if (count == 0) return FFS_OK;
    FFS_TRY(sync_device(in));
    const TabHeader &h = in->hdr;
    DecodeArgs a{};
    a.blob = in->d_blob;
    a.blob_bytes = h.bytes;
    a.Y[0] = a.Y[1] = y;
    a.X[0] = a.X[1] = x;
    a.count = count;
    a.obj[0] = a.obj[1] = obj;
    a.tard = tard;
    a.cmax = cmax;
    a.S = S;
    a.Mo = Mo;
    a.S0 = in->d_S0;
    a.M0 = in->d_M0;
    a.status = in->d_status;
    a.err = in->d_err;
    if (g_inject_table_copy.load()) {
        a.inject_skip = 1;
        a.wait_iters = kInjectWaitIters;
    }
    const int slots = smem_slots(h, false, ins);
    const int sms = num_sms();
    const NoArena plain;  // per-instance buffers outlive any service arena
    if (slots > 0) {
        if ((size_t)count > in->d_over_cap) {
            dfree(in->d_over);
            FFS_CUDA(dalloc(&in->d_over, (size_t)count));
            in->d_over_cap = count;
        }
        FFS_CUDA(cudaMemsetAsync(in->d_over_count, 0, 4, st));
        a.Hcap = slots;
        a.over_list = in->d_over;
        a.over_count = in->d_over_count;
        const int per_sm = std::max(1, (228 * 1024) / (cta_smem_bytes(h, slots, false, false, ins) + 1024));
        const int grid = std::max(1, std::min((count + kWarpsPerBlock - 1) / kWarpsPerBlock, sms * per_sm));
        FFS_CUDA(launch_decode(order, mach, false, a, h, grid, st));
        g_launches += 1;
        if (slots >= h.H) return FFS_OK;  // the profile bound fits: nothing can overflow
        a.list = in->d_over;
        a.list_count = in->d_over_count;
    }
    // Global-memory profiles: the whole bound per warp.
    const int grid = std::max(1, std::min((count + kWarpsPerBlock - 1) / kWarpsPerBlock, sms * 2));
    FFS_TRY(ensure_scratch(&in->d_scratch, &in->d_scratch_cap,
                           (size_t)grid * kWarpsPerBlock * gwork_stride(h.H, h.maxo, ins)));
    a.gscratch = in->d_scratch;
    a.Hcap = h.H;
    g_launches += 1;
    return cuda_rc(launch_decode(order, mach, true, a, h, grid, st));
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

const char *ffs_strerror(int code) {
    switch (code) {
        case FFS_OK: return "ok";
        case FFS_E_ARG: return "invalid argument";
        case FFS_E_INFEASIBLE: return "infeasible instance (machine power above the peak, or an empty stage)";
        case FFS_E_NOMEM: return "out of memory";
        case FFS_E_CUDA: return "CUDA error";
        case FFS_E_TIMEOUT: return "device wait timed out";
        case FFS_E_ADMISSION: return "request not admitted";
        case FFS_E_STATE: return "call not valid in the current state";
        case FFS_E_DEVICE: return "kernel reported an error";
        case FFS_E_STOPPED: return "batched run stopped early on request";
        default: return "unknown status";
    }
}

int ffs_instance_create(const ffs_problem *pr, ffs_instance **out) {
    if (!pr || !out) return FFS_E_ARG;
    *out = nullptr;
    const int N = pr->n_jobs, g = pr->n_stages;
    const bool unrel = pr->proc_machine != nullptr;
    if (N < 1 || N > kMaxN || g < 1 || g > kMaxG || !pr->machines_per_stage || (!unrel && (!pr->proc || !pr->power)) ||
        (unrel != (pr->power_machine != nullptr)) || !pr->release || !pr->due || pr->peak_power < 0 ||
        pr->peak_power > kMaxQ || pr->wt < 0)
        return FFS_E_ARG;
    int M = 0;
    for (int s = 0; s < g; ++s) {
        const int o = pr->machines_per_stage[s];
        if (o < 1) return FFS_E_INFEASIBLE;
        if (o > kMaxO) return FFS_E_ARG;
        M += o;
    }
    if (M > kMaxM) return FFS_E_ARG;
    if (unrel) {
        for (size_t i = 0; i < (size_t)N * M; ++i) {
            if (pr->proc_machine[i] < 0 || pr->proc_machine[i] > kMaxP || pr->power_machine[i] < 0) return FFS_E_ARG;
            if (pr->power_machine[i] > pr->peak_power) return FFS_E_INFEASIBLE;
        }
    } else {
        for (int i = 0; i < N * g; ++i)
            if (pr->proc[i] < 0 || pr->proc[i] > kMaxP) return FFS_E_ARG;
        for (int m = 0; m < M; ++m) {
            if (pr->power[m] < 0) return FFS_E_ARG;
            if (pr->power[m] > pr->peak_power) return FFS_E_INFEASIBLE;
        }
    }
    for (int j = 0; j < N; ++j)
        if (pr->release[j] < 0) return FFS_E_ARG;
    ffs_instance *in = new (std::nothrow) ffs_instance();
    if (!in) return FFS_E_NOMEM;
    in->N = N; in->g = g; in->M = M; in->Qmax = pr->peak_power; in->WT = pr->wt; in->RS = 0;
    in->o.assign(pr->machines_per_stage, pr->machines_per_stage + g);
    in->moff.assign(g + 1, 0);
    for (int s = 0; s < g; ++s) in->moff[s + 1] = in->moff[s] + in->o[s];
    if (unrel) {
        in->unrel = true;
        in->pm.assign(pr->proc_machine, pr->proc_machine + (size_t)N * M);
        in->qm.assign(pr->power_machine, pr->power_machine + (size_t)N * M);
        // per-op summary (gene records, surrogate features): the fastest machine's time;
        // per-machine summary: the largest power any job draws on it
        in->p.assign((size_t)N * g, 0);
        in->q.assign(M, 0);
        for (int j = 0; j < N; ++j)
            for (int s = 0; s < g; ++s) {
                int best = INT_MAX;
                for (int m = 0; m < in->o[s]; ++m) {
                    const int mg = in->moff[s] + m;
                    best = std::min(best, in->pm[(size_t)j * M + mg]);
                    in->q[mg] = std::max(in->q[mg], in->qm[(size_t)j * M + mg]);
                }
                in->p[j * g + s] = best;
            }
    } else {
        in->p.assign(pr->proc, pr->proc + N * g);
        in->q.assign(pr->power, pr->power + M);
    }
    in->R.assign(pr->release, pr->release + N);
    in->D.assign(pr->due, pr->due + N);
    in->status.assign(N * g, kStFree);
    in->S0.assign(N * g, 0);
    in->M0.assign(N * g, 0);
    const int rc = rebuild(in);
    if (rc != FFS_OK) {
        delete in;
        return rc;
    }
    *out = in;
    return FFS_OK;
}

int ffs_instance_destroy(ffs_instance *in) {
    delete in;
    return FFS_OK;
}

int ffs_instance_info(const ffs_instance *in, ffs_info *info) {
    if (!in || !info) return FFS_E_ARG;
    info->n_jobs = in->N;
    info->n_stages = in->g;
    info->n_machines = in->M;
    info->n_genes = in->K;
    info->rs = in->RS;
    info->horizon = in->Hfull;
    info->peak_power = in->Qmax;
    info->wt = in->WT;
    return FFS_OK;
}

int ffs_instance_genes(const ffs_instance *in, int32_t *gene_job, int32_t *gene_stage) {
    if (!in || (in->K > 0 && (!gene_job || !gene_stage))) return FFS_E_ARG;
    for (int k = 0; k < in->K; ++k) {
        gene_job[k] = in->gjob[k];
        gene_stage[k] = in->gstg[k];
    }
    return FFS_OK;
}

int ffs_instance_status(const ffs_instance *in, int32_t *status) {
    if (!in || !status) return FFS_E_ARG;
    std::memcpy(status, in->status.data(), sizeof(int32_t) * in->status.size());
    return FFS_OK;
}

int ffs_commit(ffs_instance *in, const int32_t *start, const int32_t *machine) {
    if (!in || !start || !machine) return FFS_E_ARG;
    const int NG = in->N * in->g;
    for (int i = 0; i < NG; ++i) {
        const int s = i % in->g;
        if (machine[i] < 0 || machine[i] >= in->o[s] || start[i] < 0) return FFS_E_ARG;
        if (in->status[i] != kStFree && (start[i] != in->S0[i] || machine[i] != in->M0[i])) return FFS_E_ARG;
        if (in->status[i] == kStFree && start[i] < in->RS) return FFS_E_ARG;
    }
    std::memcpy(in->S0.data(), start, 4 * (size_t)NG);
    std::memcpy(in->M0.data(), machine, 4 * (size_t)NG);
    in->has_plan = true;
    in->dev_dirty = true;
    return FFS_OK;
}

}  // extern "C"

namespace {

// Alg. 1 at t_now against the committed plan, then the new jobs appended.  static_plan:
// ops that have not started keep their start and machine (the traditional static
// approach) instead of becoming free.
int reschedule_impl(ffs_instance *in, const ffs_arrivals *arr, int32_t t_now, bool static_plan) {
    if (!in || t_now < in->RS) return FFS_E_ARG;
    const int n1 = arr ? arr->job_count : 0;
    if (n1 < 0 || in->N + n1 > kMaxN || (n1 > 0 && (!arr->release || !arr->due))) return FFS_E_ARG;
    if (n1 > 0 && (in->unrel ? (!arr->proc_machine || !arr->power_machine) : !arr->proc)) return FFS_E_ARG;
    if (in->unrel) {
        for (size_t i = 0; i < (size_t)n1 * in->M; ++i) {
            if (arr->proc_machine[i] < 0 || arr->proc_machine[i] > kMaxP || arr->power_machine[i] < 0) return FFS_E_ARG;
            if (arr->power_machine[i] > in->Qmax) return FFS_E_INFEASIBLE;
        }
    } else {
        for (int i = 0; i < n1 * in->g; ++i)
            if (arr->proc[i] < 0 || arr->proc[i] > kMaxP) return FFS_E_ARG;
    }
    for (int j = 0; j < n1; ++j)
        if (arr->release[j] < 0) return FFS_E_ARG;
    if (!in->has_plan && t_now != in->RS) return FFS_E_STATE;
    const int g = in->g;
    if (in->has_plan) {
        // Alg. 1: S + P <= RS completed, S < RS < S + P being executed, otherwise free
        // (or, in the static approach, fixed in the plan).
        const int later = static_plan ? kStFixed : kStFree;
        for (int i = 0; i < in->N * g; ++i) {
            const int st = in->S0[i], en = in->S0[i] + op_p(in, i / g, i % g, in->M0[i]);
            in->status[i] = en <= t_now ? kStDone : st < t_now ? kStExec : later;
        }
    }
    for (int j = 0; j < n1; ++j) {
        for (int s = 0; s < g; ++s) {
            int pv;
            if (in->unrel) {
                pv = INT_MAX;
                for (int m = 0; m < in->o[s]; ++m) {
                    const size_t i = (size_t)j * in->M + in->moff[s] + m;
                    pv = std::min(pv, arr->proc_machine[i]);
                    in->q[in->moff[s] + m] = std::max(in->q[in->moff[s] + m], arr->power_machine[i]);
                }
            } else {
                pv = arr->proc[j * g + s];
            }
            in->p.push_back(pv);
            in->status.push_back(kStFree);
            in->S0.push_back(0);
            in->M0.push_back(0);
        }
        in->R.push_back(arr->release[j]);
        in->D.push_back(arr->due[j]);
    }
    if (in->unrel) {
        in->pm.insert(in->pm.end(), arr ? arr->proc_machine : nullptr, arr ? arr->proc_machine + (size_t)n1 * in->M : nullptr);
        in->qm.insert(in->qm.end(), arr ? arr->power_machine : nullptr, arr ? arr->power_machine + (size_t)n1 * in->M : nullptr);
    }
    in->N += n1;
    in->RS = t_now;
    in->has_plan = false;
    return rebuild(in);
}

}  // namespace

extern "C" {

int ffs_reschedule(ffs_instance *in, const ffs_arrivals *arr, int32_t t_now) {
    return reschedule_impl(in, arr, t_now, false);
}

int ffs_reschedule_static(ffs_instance *in, const ffs_arrivals *arr, int32_t t_now) {
    return reschedule_impl(in, arr, t_now, true);
}

int ffs_decode(ffs_instance *in, int32_t order_mode, int32_t machine_mode, const int16_t *y,
               const int8_t *x, int32_t count, int64_t *obj, int64_t *tard, int32_t *cmax, void *stream) {
    if (!in) return FFS_E_ARG;
    return decode_impl(in, order_mode, machine_mode, y, x, count, obj, tard, cmax, nullptr, nullptr,
                       static_cast<cudaStream_t>(stream));
}

int ffs_decode_schedule(ffs_instance *in, int32_t order_mode, int32_t machine_mode, const int16_t *y,
                        const int8_t *x, int32_t count, int64_t *obj, int32_t *start, int32_t *machine,
                        void *stream) {
    if (!in || (count > 0 && (!start || !machine))) return FFS_E_ARG;
    return decode_impl(in, order_mode, machine_mode, y, x, count, obj, nullptr, nullptr, start, machine,
                       static_cast<cudaStream_t>(stream));
}

int ffs_decode_check(ffs_instance *in, void *stream) {
    if (!in) return FFS_E_ARG;
    FFS_TRY(sync_device(in));
    FFS_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    int32_t e = 0;
    FFS_CUDA(cudaMemcpy(&e, in->d_err, 4, cudaMemcpyDeviceToHost));
    FFS_CUDA(cudaMemset(in->d_err, 0, 4));
    if (e & kErrTimeout) return FFS_E_TIMEOUT;
    return e ? FFS_E_DEVICE : FFS_OK;
}

// ---------------------------------------------------------------- GA

static int ga_replace_args(ga_population *pp, ReplArgs *r, int init) {
    *r = ReplArgs{};
    for (int b = 0; b < 2; ++b) {
        r->Y[b] = pp->Y[b];
        r->X[b] = pp->X[b];
        r->obj[b] = pp->obj[b];
        r->fit[b] = pp->fit[b];
    }
    r->bY = pp->bY; r->bX = pp->bX; r->bobj = pp->bobj; r->bfit = pp->bfit;
    r->mY = pp->mY; r->mX = pp->mX; r->mobj = pp->mobj; r->mfit = pp->mfit; r->mw = pp->mw;
    r->dev = pp->dev;
    r->P = pp->P; r->I = pp->I; r->K = pp->K;
    r->migrate_every = pp->par.migrate_every;
    r->init = init;
    return FFS_OK;
}

}  // extern "C"

void ffs_rt::ga_gen_args(ga_population *pp, GenArgs *a) {
    *a = GenArgs{};
    a->blob = pp->d_blob;
    a->blob_bytes = pp->hdr.bytes;
    a->Hcap = pp->Hcap;
    for (int b = 0; b < 2; ++b) {
        a->Y[b] = pp->Y[b];
        a->X[b] = pp->X[b];
        a->obj[b] = pp->obj[b];
        a->fit[b] = pp->fit[b];
    }
    a->dev = pp->dev;
    a->P = pp->P;
    a->I = pp->I;
    a->K = pp->K;
    a->gen_ofs = 0;
    a->publish = 1;
    a->H = pp->hdr.H;
    a->gscratch = pp->scratch;
    a->isl_done = pp->isl_done;
    a->nisl = pp->nisl;
    a->migrate_every = pp->par.migrate_every;
    a->bY = pp->bY; a->bX = pp->bX; a->bobj = pp->bobj; a->bfit = pp->bfit;
    a->mY = pp->mY; a->mX = pp->mX; a->mobj = pp->mobj; a->mfit = pp->mfit; a->mw = pp->mw;
    a->tour_k = pp->par.tournament_k;
    a->side = pp->side;
    a->pc_thr = ((uint64_t)(uint32_t)pp->par.pc_num << 32) / (uint64_t)(uint32_t)pp->par.pc_den;
    a->pm_thr = ((uint64_t)(uint32_t)pp->par.pm_num << 32) / (uint64_t)(uint32_t)pp->par.pm_den;
    a->instance_id = (uint32_t)pp->par.instance_id & 0xFFFFFFu;
    a->seed = pp->par.seed;
    a->over_list = pp->over;
    a->err = pp->err;
}

extern "C" {

static void ga_fallback_args(ga_population *pp, DecodeArgs *d, bool ga_mode) {
    *d = DecodeArgs{};
    d->blob = pp->d_blob;
    d->blob_bytes = pp->hdr.bytes;
    d->Hcap = pp->hdr.H;
    for (int b = 0; b < 2; ++b) {
        d->Y[b] = pp->Y[b];
        d->X[b] = pp->X[b];
        d->obj[b] = pp->obj[b];
        d->fit[b] = pp->fit[b];
    }
    d->list = pp->over;
    d->list_count = &pp->dev->nover;
    d->gdev = ga_mode ? pp->dev : nullptr;
    d->gscratch = pp->scratch;
    d->err = pp->err;
}

// One generation is one kernel: selection, crossover, mutation and decoding per child,
// then (by the last warps to finish) elitist replacement, migration and the counter.
// With timing events, the kernel is bracketed by ev0/ev1 on the population's stream.
// With `overlap`, the kernel is launched as a programmatic dependent of the previous one on
// the stream: its CTAs are scheduled while that kernel drains and stage their tables, then
// wait until it has completed and its writes are visible.
// In a chain of generations launched together, generation `ofs` reads the counter as it
// stood when the chain began and only the last one (`publish`) advances it.
static int ga_enqueue_generation(ga_population *pp, cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr,
                                 bool overlap = false, int ofs = 0, bool publish = true) {
    GenArgs a;
    ga_gen_args(pp, &a);
    a.gen_ofs = ofs;
    a.publish = publish ? 1 : 0;
    if (ev0) FFS_CUDA(cudaEventRecord(ev0, pp->st));
    FFS_CUDA(launch_ga_generation(pp->par.order_mode, pp->par.machine_mode, a, pp->hdr, pp->grid_gen, pp->st,
                                  overlap));
    if (ev1) FFS_CUDA(cudaEventRecord(ev1, pp->st));
    return FFS_OK;
}

}  // extern "C"

namespace {

int check_ga_params(const ga_params *par, int *side) {
    FFS_TRY(check_modes(par->order_mode, par->machine_mode));
    const int P = par->pop, I = par->island;
    if (P < 2 || P % 2 || I < 2 || I % 2 || P % I || par->tournament_k < 0 || par->tournament_k > 32 ||
        par->pc_den <= 0 || par->pm_den <= 0 || par->pc_num < 0 || par->pm_num < 0 ||
        par->pc_num > par->pc_den || par->pm_num > par->pm_den || par->migrate_every < 0)
        return FFS_E_ARG;
    *side = 0;
    if (par->tournament_k == 0) {
        int s = 0;
        while (s * s < P) ++s;
        if (s * s != P) return FFS_E_ARG;
        *side = s;
    }
    return FFS_OK;
}

// Sizes of a population of `in` (no allocation).
void pop_shape(ga_population *pp, ffs_instance *in, const ga_params *par, int side) {
    pp->inst = in;
    pp->version = in->version;
    pp->par = *par;
    pp->st = static_cast<cudaStream_t>(par->cuda_stream);
    pp->P = par->pop;
    pp->I = par->island;
    pp->K = in->K;
    pp->nisl = pp->P / pp->I;
    pp->side = side;
    pp->hdr = in->hdr;
    pp->NG = in->N * in->g;
    const bool ins = (par->machine_mode & FFS_PLACE_INSERT) != 0;
    pp->Hcap = smem_slots(pp->hdr, true, ins);
    const int P = pp->P;
    pp->grid_gen = std::max(1, std::min((P + kWarpsPerBlock - 1) / kWarpsPerBlock,
                                        num_sms() * std::max(1, (228 * 1024) / (cta_smem_bytes(pp->hdr, pp->Hcap, true, false, ins) + 1024))));
    pp->grid_fb = std::max(1, std::min((P + kWarpsPerBlock - 1) / kWarpsPerBlock, num_sms() * 2));
}

// Every device buffer of a population, in allocation order: f(pointer, element count).
template <typename F>
void pop_buffers(ga_population *pp, F &&f) {
    const size_t PK = (size_t)pp->P * pp->K, NK = (size_t)pp->nisl * pp->K, nisl = pp->nisl;
    f(pp->d_blob, (size_t)pp->hdr.bytes);
    for (int b = 0; b < 2; ++b) {
        f(pp->Y[b], PK);
        f(pp->X[b], PK);
        f(pp->obj[b], (size_t)pp->P);
        f(pp->fit[b], (size_t)pp->P);
    }
    f(pp->bY, NK); f(pp->bX, NK); f(pp->bobj, nisl); f(pp->bfit, nisl);
    f(pp->mY, NK); f(pp->mX, NK); f(pp->mobj, nisl); f(pp->mfit, nisl); f(pp->mw, nisl);
    f(pp->over, (size_t)pp->P);
    f(pp->err, (size_t)1);
    f(pp->dev, (size_t)1);
    f(pp->isl_done, nisl);
    f(pp->scratch, (size_t)std::max(pp->grid_fb, pp->grid_gen) * kWarpsPerBlock *
                       gwork_stride(pp->hdr.H, pp->hdr.maxo, (pp->par.machine_mode & FFS_PLACE_INSERT) != 0));
    f(pp->r_obj, (size_t)1); f(pp->r_tard, (size_t)1); f(pp->r_cm, (size_t)1);
    f(pp->r_S, (size_t)pp->NG); f(pp->r_M, (size_t)pp->NG);
    f(pp->r_over, (size_t)1); f(pp->r_cnt, (size_t)1);
}

size_t pop_bytes(ga_population *pp) {
    size_t total = 0;
    pop_buffers(pp, [&](auto *&ptr, size_t n) {
        const size_t bytes = std::max<size_t>(n, 1) * sizeof(*ptr);
        total += (bytes + kArenaAlign - 1) / kArenaAlign * kArenaAlign;
    });
    return total;
}

// Creates a population; with `prev` (an earlier population of the same instance),
// generation 0 is prev's current population carried over to the present gene set.
int create_population(ffs_instance *in, const ga_params *par, ga_population *prev, ga_population **out) {
    if (!in || !par || !out) return FFS_E_ARG;
    *out = nullptr;
    int side = 0;
    FFS_TRY(check_ga_params(par, &side));
    if (in->K < 1) return FFS_E_STATE;
    if (prev && (prev->inst != in || prev->version > in->version || prev->profiling)) return FFS_E_ARG;
    FFS_TRY(sync_device(in));
    ga_population *pp = new (std::nothrow) ga_population();
    if (!pp) return FFS_E_NOMEM;
    auto fail = [&](int rc) {
        delete pp;
        return rc;
    };
    pop_shape(pp, in, par, side);
    bool ok = true;
    pop_buffers(pp, [&](auto *&ptr, size_t n) {
        if (ok) ok = dalloc(&ptr, n) == cudaSuccess;
    });
    if (!ok) return fail(FFS_E_NOMEM);
    pp->gkey.resize(pp->K);
    for (int k = 0; k < pp->K; ++k) pp->gkey[k] = (int64_t)in->gjob[k] * in->g + in->gstg[k];
    const size_t PK = (size_t)pp->P * pp->K;
    cudaStream_t st = pp->st;
    int rc = FFS_OK;
    auto step = [&](cudaError_t e) {
        if (rc == FFS_OK && e != cudaSuccess) rc = cuda_rc(e);
    };
    step(cudaMemcpyAsync(pp->d_blob, in->blob.data(), in->hdr.bytes, cudaMemcpyHostToDevice, st));
    for (int b = 0; b < 2; ++b) step(cudaMemsetAsync(pp->X[b], 0, PK, st));
    step(cudaMemsetAsync(pp->err, 0, 4, st));
    step(cudaMemsetAsync(pp->dev, 0, sizeof(GADev), st));
    step(cudaMemsetAsync(pp->isl_done, 0, 4 * (size_t)pp->nisl, st));
    int32_t *d_map = nullptr;
    if (prev && rc == FFS_OK) {
        // old gene -> new gene (or -1 once frozen); new genes with no old counterpart
        std::vector<int32_t> slot((size_t)in->N * in->g, -1), map(prev->K), fresh;
        for (int k = 0; k < pp->K; ++k) slot[pp->gkey[k]] = k;
        std::vector<char> seen(pp->K, 0);
        for (int k = 0; k < prev->K; ++k) {
            const int64_t key = prev->gkey[k];
            map[k] = key < (int64_t)slot.size() ? slot[key] : -1;
            if (map[k] >= 0) seen[map[k]] = 1;
        }
        for (int k = 0; k < pp->K; ++k)
            if (!seen[k]) fresh.push_back(k);
        if (dalloc(&d_map, (size_t)prev->K + fresh.size()) != cudaSuccess) return fail(FFS_E_NOMEM);
        // the old rows are read on this stream once prev's queued work is done
        cudaEvent_t ev = nullptr;
        step(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        if (rc == FFS_OK) {
            step(cudaEventRecord(ev, prev->st));
            step(cudaStreamWaitEvent(st, ev, 0));
            cudaEventDestroy(ev);
        }
        step(cudaMemcpyAsync(d_map, map.data(), 4 * map.size(), cudaMemcpyHostToDevice, st));
        if (!fresh.empty())
            step(cudaMemcpyAsync(d_map + prev->K, fresh.data(), 4 * fresh.size(), cudaMemcpyHostToDevice, st));
        WarmArgs w{};
        for (int b = 0; b < 2; ++b) {
            w.Yo[b] = prev->Y[b];
            w.Xo[b] = prev->X[b];
        }
        w.odev = prev->dev;
        w.Po = prev->P;
        w.Ko = prev->K;
        w.map = d_map;
        w.fresh = d_map + prev->K;
        w.n_new = (int)fresh.size();
        w.Y = pp->Y[0];
        w.X = pp->X[0];
        w.P = pp->P;
        w.K = pp->K;
        w.err = pp->err;
        step(launch_warm_remap(w, st));
        if (rc == FFS_OK) g_launches += 1;
        // pageable sources: the copies have been staged once cudaMemcpyAsync returned
    }
    GenArgs a;
    ga_gen_args(pp, &a);
    a.warm = prev ? 1 : 0;
    step(launch_ga_init(par->order_mode, par->machine_mode, a, pp->hdr, pp->grid_gen, st));
    DecodeArgs d;
    ga_fallback_args(pp, &d, false);
    step(launch_decode(par->order_mode, par->machine_mode, true, d, pp->hdr, pp->grid_fb, st));
    ReplArgs r;
    ga_replace_args(pp, &r, 1);
    step(launch_emax(r, st));
    step(launch_replace(r, st));
    step(cudaMemsetAsync(&pp->dev->nover, 0, 4, st));
    if (rc != FFS_OK) {
        cudaStreamSynchronize(st);
        dfree(d_map);
        return fail(rc);
    }
    g_launches += 4;  // init, fallback decode, E_max, island bests
    // Capture one generation once; ga_run replays it.
    if (prepare_ga_generation(par->order_mode, par->machine_mode, pp->hdr, pp->Hcap) != cudaSuccess) {
        cudaStreamSynchronize(st);
        dfree(d_map);
        return fail(FFS_E_CUDA);
    }
    // The caller's stream may be the legacy default stream, which cannot be captured: the
    // graph is recorded on a private stream and later launched on the caller's.
    cudaGraph_t graph = nullptr;
    cudaStream_t cap = nullptr;
    rc = cuda_rc(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    if (rc == FFS_OK) {
        cudaStream_t user = pp->st;
        pp->st = cap;
        rc = cuda_rc(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
        const int erc = rc == FFS_OK ? ga_enqueue_generation(pp) : rc;
        const int ce = rc == FFS_OK ? cuda_rc(cudaStreamEndCapture(cap, &graph)) : rc;
        rc = erc != FFS_OK ? erc : ce;
        if (rc == FFS_OK) rc = cuda_rc(cudaGraphInstantiate(&pp->graph, graph, 0));
        if (graph) cudaGraphDestroy(graph);
        graph = nullptr;
        // kGraphGens generations in one graph, each launched as a programmatic dependent of
        // the one before, which hides the launch gap between generations
        if (rc == FFS_OK) rc = cuda_rc(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
        int erc2 = FFS_OK;
        for (int g = 0; rc == FFS_OK && erc2 == FFS_OK && g < kGraphGens; ++g)
            erc2 = ga_enqueue_generation(pp, nullptr, nullptr, g > 0, g, g == kGraphGens - 1);
        const int ce2 = rc == FFS_OK ? cuda_rc(cudaStreamEndCapture(cap, &graph)) : rc;
        if (rc == FFS_OK) rc = erc2 != FFS_OK ? erc2 : ce2;
        if (rc == FFS_OK) rc = cuda_rc(cudaGraphInstantiate(&pp->graph_r, graph, 0));
        if (graph) cudaGraphDestroy(graph);
        pp->st = user;
        cudaStreamDestroy(cap);
    }
    const int sync_rc = cuda_rc(cudaStreamSynchronize(st));
    dfree(d_map);
    if (rc != FFS_OK) return fail(rc);
    if (sync_rc != FFS_OK) return fail(sync_rc);
    int32_t e = 0;
    if (cudaMemcpy(&e, pp->err, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return fail(FFS_E_CUDA);
    if (e) return fail(e & kErrTimeout ? FFS_E_TIMEOUT : FFS_E_DEVICE);
    *out = pp;
    return FFS_OK;
}

}  // namespace

int ffs_rt::population_footprint(ffs_instance *in, const ga_params *par, int64_t *bytes) {
    int side = 0;
    FFS_TRY(check_ga_params(par, &side));
    if (in->K < 1) return FFS_E_STATE;
    ga_population shape;
    pop_shape(&shape, in, par, side);
    *bytes = (int64_t)pop_bytes(&shape);
    return FFS_OK;
}

int ffs_rt::population_create(ffs_instance *in, const ga_params *par, ga_population *prev, ga_population **out) {
    return create_population(in, par, prev, out);
}

void ffs_rt::population_trim(ga_population *pp) {
    if (pp->graph) cudaGraphExecDestroy(pp->graph);
    if (pp->graph_sur) cudaGraphExecDestroy(pp->graph_sur);
    if (pp->graph_r) cudaGraphExecDestroy(pp->graph_r);
    pp->graph = pp->graph_sur = pp->graph_r = nullptr;
    dfree(pp->d_blob);
    for (int b = 0; b < 2; ++b) {
        dfree(pp->obj[b]);
        dfree(pp->fit[b]);
    }
    dfree(pp->bY); dfree(pp->bX); dfree(pp->bobj); dfree(pp->bfit);
    dfree(pp->mY); dfree(pp->mX); dfree(pp->mobj); dfree(pp->mfit); dfree(pp->mw);
    dfree(pp->over); dfree(pp->isl_done); dfree(pp->scratch);
    dfree(pp->r_obj); dfree(pp->r_tard); dfree(pp->r_cm); dfree(pp->r_S); dfree(pp->r_M);
    dfree(pp->r_over); dfree(pp->r_cnt);
    dfree(pp->cand_Y); dfree(pp->cand_X); dfree(pp->cand_Yh); dfree(pp->cand_H1); dfree(pp->cand_H2);
    dfree(pp->cand_out); dfree(pp->cand_new); dfree(pp->kept_obj); dfree(pp->cand_keep);
    pp->sur = nullptr;
}

extern "C" {

int ga_population_create(ffs_instance *in, const ga_params *par, ga_population **out) {
    return create_population(in, par, nullptr, out);
}

int ga_population_create_warm(ffs_instance *in, const ga_params *par, ga_population *prev, ga_population **out) {
    if (!prev) return FFS_E_ARG;
    return create_population(in, par, prev, out);
}

int ga_population_footprint(const ffs_instance *in, const ga_params *par, int64_t *bytes) {
    if (!in || !par || !bytes) return FFS_E_ARG;
    return population_footprint(const_cast<ffs_instance *>(in), par, bytes);
}

int ga_population_destroy(ga_population *pp) {
    delete pp;
    return FFS_OK;
}

int ga_population_read(ga_population *pp, int16_t *Y, int8_t *X, int64_t *obj, int64_t *fit, int16_t *bY,
                       int8_t *bX, int64_t *bobj, int64_t *bfit, int64_t *emax, int32_t *generation) {
    if (!pp) return FFS_E_ARG;
    FFS_CUDA(cudaStreamSynchronize(pp->st));
    GADev dv;
    FFS_CUDA(cudaMemcpy(&dv, pp->dev, sizeof(dv), cudaMemcpyDeviceToHost));
    const int b = dv.gen & 1;
    const size_t PK = (size_t)pp->P * pp->K, NK = (size_t)pp->nisl * pp->K;
    if (Y) FFS_CUDA(cudaMemcpy(Y, pp->Y[b], 2 * PK, cudaMemcpyDeviceToHost));
    if (X) FFS_CUDA(cudaMemcpy(X, pp->X[b], PK, cudaMemcpyDeviceToHost));
    if (obj) FFS_CUDA(cudaMemcpy(obj, pp->obj[b], 8 * (size_t)pp->P, cudaMemcpyDeviceToHost));
    if (fit) FFS_CUDA(cudaMemcpy(fit, pp->fit[b], 8 * (size_t)pp->P, cudaMemcpyDeviceToHost));
    if (bY) FFS_CUDA(cudaMemcpy(bY, pp->bY, 2 * NK, cudaMemcpyDeviceToHost));
    if (bX) FFS_CUDA(cudaMemcpy(bX, pp->bX, NK, cudaMemcpyDeviceToHost));
    if (bobj) FFS_CUDA(cudaMemcpy(bobj, pp->bobj, 8 * (size_t)pp->nisl, cudaMemcpyDeviceToHost));
    if (bfit) FFS_CUDA(cudaMemcpy(bfit, pp->bfit, 8 * (size_t)pp->nisl, cudaMemcpyDeviceToHost));
    if (emax) *emax = dv.emax;
    if (generation) *generation = dv.gen;
    return FFS_OK;
}

}  // extern "C"

int ffs_rt::ga_enqueue(ga_population *pp, int32_t generations, int *timed) {
    if (!pp || generations < 0) return FFS_E_ARG;
    if (timed) *timed = 0;
    ffs_instance *in = pp->inst;
    if (pp->version != in->version) return FFS_E_STATE;
    const unsigned long long per_gen = pp->sur ? (unsigned long long)surrogate_launches_per_generation(pp) : 1;
    if (pp->sur && !pp->graph_sur && pp->profiling != 1 && !surrogate_is_exact(pp)) {  // capture once
        FFS_TRY(prepare_surrogate_kernels(pp));
        cudaStream_t cap = nullptr;
        FFS_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        int rc = cuda_rc(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
        if (rc == FFS_OK) rc = surrogate_enqueue_generation(pp, cap, nullptr, nullptr);
        const int ce = cuda_rc(cudaStreamEndCapture(cap, &g));
        cudaStreamDestroy(cap);
        if (rc == FFS_OK) rc = ce;
        if (rc == FFS_OK) rc = cuda_rc(cudaGraphInstantiate(&pp->graph_sur, g, 0));
        if (g) cudaGraphDestroy(g);
        if (rc != FFS_OK) return rc;
    }
    if (pp->profiling == 1) return FFS_E_STATE;
    if (surrogate_is_exact(pp)) {  // decodes every candidate: launched directly
        FFS_TRY(prepare_surrogate_kernels(pp));
        for (int i = 0; i < generations; ++i) FFS_TRY(surrogate_enqueue_generation(pp, pp->st, nullptr, nullptr));
        g_launches += per_gen * (unsigned long long)generations;
        return FFS_OK;
    }
    cudaGraphExec_t gx = pp->sur ? pp->graph_sur : pp->graph;
    // profiling mode 2: events around every replay, in the launch mode of ga_run itself
    const bool time_it = pp->profiling == 2 && timed;
    const int pairs = time_it ? (pp->sur || !pp->graph_r ? generations
                                                          : generations / kGraphGens + generations % kGraphGens)
                              : 0;
    while ((int)pp->ev.size() < 2 * pairs) {
        cudaEvent_t e;
        FFS_CUDA(cudaEventCreate(&e));
        pp->ev.push_back(e);
    }
    int i = 0, q = 0;
    auto replay = [&](cudaGraphExec_t g) {
        if (time_it) FFS_CUDA(cudaEventRecord(pp->ev[2 * q], pp->st));
        FFS_CUDA(cudaGraphLaunch(g, pp->st));
        if (time_it) FFS_CUDA(cudaEventRecord(pp->ev[2 * q + 1], pp->st));
        ++q;
        return FFS_OK;
    };
    if (!pp->sur && pp->graph_r)
        for (; i + kGraphGens <= generations; i += kGraphGens) FFS_TRY(replay(pp->graph_r));
    for (; i < generations; ++i) FFS_TRY(replay(gx));
    g_launches += per_gen * (unsigned long long)generations;
    if (time_it) *timed = q;
    return FFS_OK;
}

int ffs_rt::ga_finish(ga_population *pp, ffs_result *best) {
    ffs_instance *in = pp->inst;
    FFS_CUDA(cudaStreamSynchronize(pp->st));
    if (pp->sur) FFS_TRY(surrogate_status());
    int32_t e = 0;
    FFS_CUDA(cudaMemcpy(&e, pp->err, 4, cudaMemcpyDeviceToHost));
    if (e) return e & kErrTimeout ? FFS_E_TIMEOUT : FFS_E_DEVICE;
    // best-ever island: largest fitness, lowest island index
    std::vector<int64_t> bfit(pp->nisl);
    FFS_CUDA(cudaMemcpy(bfit.data(), pp->bfit, 8 * (size_t)pp->nisl, cudaMemcpyDeviceToHost));
    int bi = 0;
    for (int i = 1; i < pp->nisl; ++i)
        if (bfit[i] > bfit[bi]) bi = i;
    // Decode it into the population's own buffers: shared-memory profile first, the
    // global-memory one (whole bound) if the schedule outgrows it.
    FFS_TRY(sync_device(in));  // frozen operations' plan
    const TabHeader &h = pp->hdr;
    DecodeArgs a{};
    a.blob = pp->d_blob;
    a.blob_bytes = h.bytes;
    a.Y[0] = a.Y[1] = pp->bY + (size_t)bi * pp->K;
    a.X[0] = a.X[1] = pp->bX + (size_t)bi * pp->K;
    a.count = 1;
    a.obj[0] = a.obj[1] = pp->r_obj;
    a.tard = pp->r_tard;
    a.cmax = pp->r_cm;
    a.S = pp->r_S;
    a.Mo = pp->r_M;
    a.S0 = in->d_S0;
    a.M0 = in->d_M0;
    a.status = in->d_status;
    a.err = pp->err;
    const int order = pp->par.order_mode, mach = pp->par.machine_mode;
    const int slots = smem_slots(h, false, (mach & FFS_PLACE_INSERT) != 0);
    if (slots > 0) {
        FFS_CUDA(cudaMemsetAsync(pp->r_cnt, 0, 4, pp->st));
        a.Hcap = slots;
        a.over_list = pp->r_over;
        a.over_count = pp->r_cnt;
        FFS_CUDA(launch_decode(order, mach, false, a, h, 1, pp->st));
        g_launches += 1;
        a.list = pp->r_over;
        a.list_count = pp->r_cnt;
    }
    if (slots < h.H) {
        a.gscratch = pp->scratch;
        a.Hcap = h.H;
        FFS_CUDA(launch_decode(order, mach, true, a, h, 1, pp->st));
        g_launches += 1;
    }
    FFS_CUDA(cudaStreamSynchronize(pp->st));
    FFS_CUDA(cudaMemcpy(&e, pp->err, 4, cudaMemcpyDeviceToHost));
    if (e) return e & kErrTimeout ? FFS_E_TIMEOUT : FFS_E_DEVICE;
    const size_t NG = (size_t)pp->NG;
    std::vector<int32_t> S(NG), M(NG);
    int64_t o = 0, t = 0;
    int32_t cm = 0;
    FFS_CUDA(cudaMemcpy(S.data(), pp->r_S, 4 * NG, cudaMemcpyDeviceToHost));
    FFS_CUDA(cudaMemcpy(M.data(), pp->r_M, 4 * NG, cudaMemcpyDeviceToHost));
    FFS_CUDA(cudaMemcpy(&o, pp->r_obj, 8, cudaMemcpyDeviceToHost));
    FFS_CUDA(cudaMemcpy(&t, pp->r_tard, 8, cudaMemcpyDeviceToHost));
    FFS_CUDA(cudaMemcpy(&cm, pp->r_cm, 4, cudaMemcpyDeviceToHost));
    FFS_TRY(ffs_commit(in, S.data(), M.data()));
    if (best) {
        best->objective = o;
        best->total_tardiness = t;
        best->makespan = cm;
        best->n_ops = (int32_t)NG;
        if (best->start) std::memcpy(best->start, S.data(), 4 * NG);
        if (best->machine) std::memcpy(best->machine, M.data(), 4 * NG);
    }
    return FFS_OK;
}


extern "C" {

int ga_run(ga_population *pp, int32_t generations, ffs_result *best) {
    if (!pp || generations < 0) return FFS_E_ARG;
    if (pp->version != pp->inst->version) return FFS_E_STATE;
    if (pp->profiling != 1) {
        int timed = 0;
        FFS_TRY(ga_enqueue(pp, generations, &timed));
        const int rc = ga_finish(pp, best);  // synchronises the stream first
        for (int q = 0; q < timed; ++q) {
            float ms = 0.f;
            FFS_CUDA(cudaEventElapsedTime(&ms, pp->ev[2 * q], pp->ev[2 * q + 1]));
            pp->prof_ms += ms;
        }
        if (timed) pp->prof_launches += generations;
        return rc;
    }
    // profiling: every generation launched eagerly between two events (surrogate generations:
    // six events bracketing their phases)
    const unsigned long long per_gen = pp->sur ? (unsigned long long)surrogate_launches_per_generation(pp) : 1;
    if (pp->sur) FFS_TRY(prepare_surrogate_kernels(pp));
    while ((int)pp->ev.size() < 2 * generations) {
        cudaEvent_t e;
        FFS_CUDA(cudaEventCreate(&e));
        pp->ev.push_back(e);
    }
    while (pp->sur && (int)pp->ev_sur.size() < 6 * generations) {
        cudaEvent_t e;
        FFS_CUDA(cudaEventCreate(&e));
        pp->ev_sur.push_back(e);
    }
    for (int i = 0; i < generations; ++i) {
        if (pp->sur)
            FFS_TRY(surrogate_enqueue_generation(pp, pp->st, pp->ev[2 * i], pp->ev[2 * i + 1], &pp->ev_sur[6 * i]));
        else FFS_TRY(ga_enqueue_generation(pp, pp->ev[2 * i], pp->ev[2 * i + 1]));
    }
    g_launches += per_gen * (unsigned long long)generations;
    FFS_CUDA(cudaStreamSynchronize(pp->st));
    for (int i = 0; i < generations; ++i) {
        float ms = 0.f;
        FFS_CUDA(cudaEventElapsedTime(&ms, pp->ev[2 * i], pp->ev[2 * i + 1]));
        pp->prof_ms += ms;
        for (int q = 0; pp->sur && q < 5; ++q) {
            FFS_CUDA(cudaEventElapsedTime(&ms, pp->ev_sur[6 * i + q], pp->ev_sur[6 * i + q + 1]));
            pp->phase_ms[q] += ms;
        }
    }
    pp->prof_launches += generations;
    return ga_finish(pp, best);
}

int ga_set_profiling(ga_population *pp, int32_t enable) {
    if (!pp) return FFS_E_ARG;
    if (enable < 0 || enable > 2) return FFS_E_ARG;
    pp->profiling = enable;
    pp->prof_ms = 0.0;
    pp->prof_launches = 0;
    for (double &v : pp->phase_ms) v = 0.0;
    return FFS_OK;
}

int ga_profile_read_phases(ga_population *pp, double *ms) {
    if (!pp || !ms) return FFS_E_ARG;
    for (int q = 0; q < 5; ++q) ms[q] = pp->phase_ms[q];
    return FFS_OK;
}

int ga_profile_read(ga_population *pp, double *kernel_ms, int64_t *launches) {
    if (!pp || !kernel_ms || !launches) return FFS_E_ARG;
    *kernel_ms = pp->prof_ms;
    *launches = pp->prof_launches;
    return FFS_OK;
}

const char *ffs_last_error(void) { return g_last_error; }

int ffs_debug_inject(int32_t mode) {
    if (mode & ~(FFS_INJECT_TABLE_COPY | FFS_INJECT_GEMM_LOADS)) return FFS_E_ARG;
    g_inject_table_copy.store((mode & FFS_INJECT_TABLE_COPY) ? 1 : 0);
    mlp_gemm_inject_skip_loads((mode & FFS_INJECT_GEMM_LOADS) != 0);
    return FFS_OK;
}

int ffs_debug_bounds_faults(uint32_t *count) {
    if (!count) return FFS_E_ARG;
#ifdef FFS_CHECKED
    const unsigned int a = bounds_faults_kernels(), b = bounds_faults_batch();
    if (a == ~0u || b == ~0u) return FFS_E_CUDA;
    *count = a + b;
    return FFS_OK;
#else
    *count = 0;
    return FFS_E_STATE;  // an ordinary build does not check
#endif
}

int ffs_kernel_launches(uint64_t *count) {
    if (!count) return FFS_E_ARG;
    *count = g_launches.load();
    return FFS_OK;
}

struct CkptHeader {
    uint32_t magic, version;
    int32_t P, K, nisl, gen;
    int64_t emax;
};

int ga_checkpoint(ga_population *pp, void *buf, size_t *len) {
    if (!pp || !len) return FFS_E_ARG;
    const size_t PK = (size_t)pp->P * pp->K, NK = (size_t)pp->nisl * pp->K;
    const size_t need = sizeof(CkptHeader) + 3 * PK + 16 * (size_t)pp->P + 3 * NK + 16 * (size_t)pp->nisl;
    if (!buf) {
        *len = need;
        return FFS_OK;
    }
    if (*len < need) return FFS_E_ARG;
    char *b = static_cast<char *>(buf);
    CkptHeader h{0x47534646u, 1u, pp->P, pp->K, pp->nisl, 0, 0};
    char *p = b + sizeof(h);
    int16_t *Y = reinterpret_cast<int16_t *>(p); p += 2 * PK;
    int8_t *X = reinterpret_cast<int8_t *>(p); p += PK;
    int64_t *obj = reinterpret_cast<int64_t *>(p); p += 8 * (size_t)pp->P;
    int64_t *fit = reinterpret_cast<int64_t *>(p); p += 8 * (size_t)pp->P;
    int16_t *bY = reinterpret_cast<int16_t *>(p); p += 2 * NK;
    int8_t *bX = reinterpret_cast<int8_t *>(p); p += NK;
    int64_t *bobj = reinterpret_cast<int64_t *>(p); p += 8 * (size_t)pp->nisl;
    int64_t *bfit = reinterpret_cast<int64_t *>(p);
    FFS_TRY(ga_population_read(pp, Y, X, obj, fit, bY, bX, bobj, bfit, &h.emax, &h.gen));
    std::memcpy(b, &h, sizeof(h));
    *len = need;
    return FFS_OK;
}

int ga_restore(ga_population *pp, const void *buf, size_t len) {
    if (!pp || !buf || len < sizeof(CkptHeader)) return FFS_E_ARG;
    CkptHeader h;
    std::memcpy(&h, buf, sizeof(h));
    const size_t PK = (size_t)pp->P * pp->K, NK = (size_t)pp->nisl * pp->K;
    const size_t need = sizeof(CkptHeader) + 3 * PK + 16 * (size_t)pp->P + 3 * NK + 16 * (size_t)pp->nisl;
    if (h.magic != 0x47534646u || h.version != 1u || h.P != pp->P || h.K != pp->K || h.nisl != pp->nisl ||
        len < need || h.gen < 0)
        return FFS_E_ARG;
    const char *p = static_cast<const char *>(buf) + sizeof(h);
    const int b = h.gen & 1;
    {   // every chromosome must be a permutation of 1..K with machines in range
        const int K = pp->K;
        const int16_t *Y = reinterpret_cast<const int16_t *>(p);
        const int8_t *X = reinterpret_cast<const int8_t *>(p + 2 * PK);
        const char *q2 = p + 3 * PK + 16 * (size_t)pp->P;
        const int16_t *bY = reinterpret_cast<const int16_t *>(q2);
        const int8_t *bX = reinterpret_cast<const int8_t *>(q2 + 2 * NK);
        std::vector<char> seen(K + 1);
        auto valid = [&](const int16_t *y, const int8_t *x) {
            std::fill(seen.begin(), seen.end(), 0);
            for (int k = 0; k < K; ++k) {
                if (y[k] < 1 || y[k] > K || seen[y[k]]) return false;
                seen[y[k]] = 1;
                if (x[k] < 0 || x[k] >= pp->inst->o[pp->inst->gstg[k]]) return false;
            }
            return true;
        };
        if (pp->version != pp->inst->version) return FFS_E_STATE;
        for (int i = 0; i < pp->P; ++i)
            if (!valid(Y + (size_t)i * K, X + (size_t)i * K)) return FFS_E_ARG;
        for (int i = 0; i < pp->nisl; ++i)
            if (!valid(bY + (size_t)i * K, bX + (size_t)i * K)) return FFS_E_ARG;
    }
    FFS_CUDA(cudaStreamSynchronize(pp->st));
    FFS_CUDA(cudaMemcpy(pp->Y[b], p, 2 * PK, cudaMemcpyHostToDevice)); p += 2 * PK;
    FFS_CUDA(cudaMemcpy(pp->X[b], p, PK, cudaMemcpyHostToDevice)); p += PK;
    FFS_CUDA(cudaMemcpy(pp->obj[b], p, 8 * (size_t)pp->P, cudaMemcpyHostToDevice)); p += 8 * (size_t)pp->P;
    FFS_CUDA(cudaMemcpy(pp->fit[b], p, 8 * (size_t)pp->P, cudaMemcpyHostToDevice)); p += 8 * (size_t)pp->P;
    FFS_CUDA(cudaMemcpy(pp->bY, p, 2 * NK, cudaMemcpyHostToDevice)); p += 2 * NK;
    FFS_CUDA(cudaMemcpy(pp->bX, p, NK, cudaMemcpyHostToDevice)); p += NK;
    FFS_CUDA(cudaMemcpy(pp->bobj, p, 8 * (size_t)pp->nisl, cudaMemcpyHostToDevice)); p += 8 * (size_t)pp->nisl;
    FFS_CUDA(cudaMemcpy(pp->bfit, p, 8 * (size_t)pp->nisl, cudaMemcpyHostToDevice));
    GADev dv{};
    dv.gen = h.gen;
    dv.emax = h.emax;
    FFS_CUDA(cudaMemcpy(pp->dev, &dv, sizeof(dv), cudaMemcpyHostToDevice));
    return FFS_OK;
}

}  // extern "C"

// ====================================================================== allocation-free decode
//
// Some callers cannot allocate device memory: hosts that hand the library a fixed memory
// budget and forbid growth after start-up, frameworks whose own caching allocator owns the
// device memory, and real-time loops that must not block on the allocator (cudaMalloc can
// block; cudaFree synchronises the device).  ffs_decode_noalloc serves them.  It runs the global-profile decode kernel
// with every piece of scratch it needs placed in one file-scope device array, so it
// allocates nothing.
//
// The array is kNoAllocBytes, reserved on every GPU that loads the library until the
// process exits.  Its layout is: [0, 256) the kernel's error word; [256, 256 + 1 MiB)
// the instance tables; the rest per-warp power profiles.
namespace {

constexpr size_t kNoAllocBytes = 16u << 20;
constexpr size_t kNoAllocTableOff = 256, kNoAllocTableCap = 1u << 20;
constexpr size_t kNoAllocProfileOff = kNoAllocTableOff + kNoAllocTableCap;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kNoAllocMaxDevices] = {};  // device address of the array, per device

// Looks up the array's device address for the current device once.  In host code the
// array's name is only a host-side stand-in, so the kernel must get this address.
int noalloc_scratch(void **out) {
    int dev = 0;
    FFS_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) return FFS_E_ARG;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        FFS_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return FFS_OK;
}

}  // namespace

extern "C" int ffs_decode_noalloc(ffs_instance *in, int32_t order_mode, int32_t machine_mode,
                                  const int16_t *y, const int8_t *x, int32_t count, int64_t *obj,
                                  int64_t *tard, int32_t *cmax, void *stream) {
    if (!in) return FFS_E_ARG;
    FFS_TRY(check_modes(order_mode, machine_mode));
    if (count < 0 || (count > 0 && (!y || !obj)) || ((machine_mode & 1) == FFS_MACH_GENE && count > 0 && !x))
        return FFS_E_ARG;
    if (count == 0) return FFS_OK;
    const TabHeader &h = in->hdr;
    const size_t per_cta =
        (size_t)kWarpsPerBlock * gwork_stride(h.H, h.maxo, (machine_mode & FFS_PLACE_INSERT) != 0) * sizeof(uint16_t);
    const size_t profile_bytes = kNoAllocBytes - kNoAllocProfileOff;
    if ((size_t)h.bytes > kNoAllocTableCap || per_cta > profile_bytes) {
        std::snprintf(g_last_error, sizeof(g_last_error),
                      "ffs_decode_noalloc: instance needs %d table bytes (limit %zu) and %zu profile bytes per "
                      "4 warps (limit %zu); use ffs_decode",
                      h.bytes, kNoAllocTableCap, per_cta, profile_bytes);
        return FFS_E_ARG;
    }
    void *base = nullptr;
    FFS_TRY(noalloc_scratch(&base));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *b = static_cast<char *>(base);
    int32_t *err = reinterpret_cast<int32_t *>(b);
    char *blob = b + kNoAllocTableOff;
    uint16_t *prof = reinterpret_cast<uint16_t *>(b + kNoAllocProfileOff);
    // The array keeps the previous call's contents: the error word must start at zero.
    // The tables are rewritten and every profile slice is initialised by the kernel.
    FFS_CUDA(cudaMemsetAsync(err, 0, sizeof(int32_t), st));
    FFS_CUDA(cudaMemcpyAsync(blob, in->blob.data(), (size_t)h.bytes, cudaMemcpyHostToDevice, st));
    const int fit = (int)std::min<size_t>(profile_bytes / per_cta, (size_t)INT32_MAX);
    const int grid = std::max(1, std::min({(count + kWarpsPerBlock - 1) / kWarpsPerBlock, num_sms() * 4, fit}));
    DecodeArgs a{};
    a.blob = blob;
    a.blob_bytes = h.bytes;
    a.Hcap = h.H;
    a.Y[0] = a.Y[1] = y;
    a.X[0] = a.X[1] = x;
    a.count = count;
    a.obj[0] = a.obj[1] = obj;
    a.tard = tard;
    a.cmax = cmax;
    a.gscratch = prof;
    a.err = err;
    FFS_CUDA(launch_decode(order_mode, machine_mode, true, a, h, grid, st));
    g_launches += 1;
    // The host copy of the tables must outlive the copy, and the error word is read here:
    // the call returns after the stream has finished its work.
    FFS_CUDA(cudaStreamSynchronize(st));
    int32_t e = 0;
    FFS_CUDA(cudaMemcpy(&e, err, sizeof(e), cudaMemcpyDeviceToHost));
    if (e & kErrTimeout) return FFS_E_TIMEOUT;
    return e ? FFS_E_DEVICE : FFS_OK;
}

// ====================================================================== batched GA
//
// Many instances' GAs in one persistent kernel (see ffs_batch.cu).  All device state of a
// batch lives in one arena so that the autotuner can snapshot and restore it with one
// copy.
struct ga_batch {
    std::vector<ffs_instance *> insts;
    std::vector<int> versions;
    ga_params par{};
    cudaStream_t st = nullptr;
    int count = 0, P = 0, I = 0, nisl = 0, side = 0, Hmax = 0;
    char *arena = nullptr, *shadow = nullptr;
    size_t arena_bytes = 0;
    BatchInst *d_inst = nullptr;
    std::vector<BatchInst> h_inst;
    int32_t *d_order = nullptr, *d_next = nullptr, *d_err = nullptr;
    uint16_t *gscratch = nullptr;
    size_t gscratch_elems = 0;
    int warps = 8, smem = 112 * 1024, grid = 1, cluster = 1;
    cudaGraphExec_t graph = nullptr;
    int graph_gens = -1;
    float tuned_ms = 0.f;
    // stop word in host-mapped memory (ga_batch_stop writes 1; a launch that ended early 2)
    volatile int32_t *stop_host = nullptr;
    int32_t *stop_dev = nullptr;

    ~ga_batch() {
        if (graph) cudaGraphExecDestroy(graph);
        if (stop_host) cudaFreeHost(const_cast<int32_t *>(stop_host));
        dfree(arena);
        dfree(shadow);
        dfree(d_inst);
        dfree(d_order);
        dfree(d_next);
        dfree(d_err);
        dfree(gscratch);
    }
};

namespace {

// Persistent grid: as many clusters as can be resident, at most one per instance.
int batch_grid(ga_batch *b, int warps, int smem, int *grid) {
    int clusters = 0;
    FFS_CUDA(batch_max_clusters(b->par.order_mode, b->par.machine_mode, b->cluster, warps, smem, &clusters));
    if (clusters < 1) return FFS_E_ARG;  // this shape cannot run
    *grid = b->cluster * std::max(1, std::min(b->count, clusters));
    return FFS_OK;
}

int batch_config(ga_batch *b, int warps, int smem, int cluster) {
    if (warps < 1 || warps > 16 || smem < 16 * 1024 || smem > 227 * 1024 || cluster < 1 || cluster > 8 ||
        cluster > b->nisl)
        return FFS_E_ARG;
    // every instance's tables and its warps' fixed workspace must fit the CTA's budget
    for (const ffs_instance *in : b->insts) {
        const TabHeader &h = in->hdr;
        if (128 + ((h.bytes + 127) & ~127) + warps * warp_layout(h.N, h.M, h.K, 0, true).bytes > smem) return FFS_E_ARG;
    }
    FFS_CUDA(prepare_batch(b->par.order_mode, b->par.machine_mode, smem));
    const int old_cluster = b->cluster;
    b->cluster = cluster;
    int grid = 0;
    const int grc = batch_grid(b, warps, smem, &grid);
    if (grc != FFS_OK) {
        b->cluster = old_cluster;
        return grc;
    }
    b->warps = warps;
    b->smem = smem;
    b->grid = grid;
    const size_t need = (size_t)b->grid * warps * (size_t)b->Hmax;
    if (need > b->gscratch_elems) {
        dfree(b->gscratch);
        FFS_CUDA(dalloc(&b->gscratch, need));
        b->gscratch_elems = need;
    }
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
        b->graph_gens = -1;
    }
    return FFS_OK;
}

// stoppable: the launch reads the stop word (runs); generation 0 and tuner trials do not.
BatchArgs batch_args(ga_batch *b, int generations, bool stoppable) {
    BatchArgs a{};
    a.inst = b->d_inst;
    a.count = b->count;
    a.order = b->d_order;
    a.next = b->d_next;
    a.generations = generations;
    a.P = b->P;
    a.I = b->I;
    a.tour_k = b->par.tournament_k;
    a.side = b->side;
    a.migrate_every = b->par.migrate_every;
    a.pc_thr = ((uint64_t)(uint32_t)b->par.pc_num << 32) / (uint64_t)(uint32_t)b->par.pc_den;
    a.pm_thr = ((uint64_t)(uint32_t)b->par.pm_num << 32) / (uint64_t)(uint32_t)b->par.pm_den;
    a.seed = b->par.seed;
    a.smem_bytes = b->smem;
    a.gscratch = b->gscratch;
    a.Hmax = b->Hmax;
    a.err = b->d_err;
    a.stop = stoppable ? b->stop_dev : nullptr;
    return a;
}

// Enqueues one persistent launch: reset the work queue, then every instance runs
// `generations` generations (after generation 0 where it has not run yet).
int batch_enqueue(ga_batch *b, int generations, cudaStream_t st, bool stoppable = false) {
    FFS_CUDA(cudaMemsetAsync(b->d_next, 0, sizeof(int32_t), st));
    FFS_CUDA(launch_batch(b->par.order_mode, b->par.machine_mode, batch_args(b, generations, stoppable), b->grid, b->warps,
                          b->cluster, st));
    g_launches += 1;
    return FFS_OK;
}

int batch_check(ga_batch *b) {
    FFS_CUDA(cudaStreamSynchronize(b->st));
    int32_t e = 0;
    FFS_CUDA(cudaMemcpy(&e, b->d_err, 4, cudaMemcpyDeviceToHost));
    if (e & kErrTimeout) return FFS_E_TIMEOUT;
    return e ? FFS_E_DEVICE : FFS_OK;
}

}  // namespace

extern "C" {

int ga_batch_create(ffs_instance *const *insts, int32_t count, const ga_params *par, ga_batch **out) {
    if (!insts || !par || !out || count < 1) return FFS_E_ARG;
    *out = nullptr;
    for (int i = 0; i < count; ++i)
        if (insts[i] && insts[i]->unrel) {
            std::snprintf(ffs_rt::g_last_error, sizeof(ffs_rt::g_last_error),
                          "batched runs take identical-machine instances only");
            return FFS_E_ARG;
        }
    FFS_TRY(check_modes(par->order_mode, par->machine_mode));
    if (par->machine_mode & FFS_PLACE_INSERT) {
        std::snprintf(ffs_rt::g_last_error, sizeof(ffs_rt::g_last_error), "batched runs use append placement only");
        return FFS_E_ARG;
    }
    const int P = par->pop, I = par->island;
    if (P < 2 || P % 2 || I < 2 || I % 2 || P % I || par->tournament_k < 0 || par->tournament_k > 32 ||
        par->pc_den <= 0 || par->pm_den <= 0 || par->pc_num < 0 || par->pm_num < 0 || par->pc_num > par->pc_den ||
        par->pm_num > par->pm_den || par->migrate_every < 0 || (long long)par->instance_id + count > (1 << 24))
        return FFS_E_ARG;
    int side = 0;
    if (par->tournament_k == 0) {
        while (side * side < P) ++side;
        if (side * side != P) return FFS_E_ARG;
    }
    for (int i = 0; i < count; ++i)
        if (!insts[i] || insts[i]->K < 1) return FFS_E_ARG;
    ga_batch *b = new (std::nothrow) ga_batch();
    if (!b) return FFS_E_NOMEM;
    auto fail = [&](int rc) {
        delete b;
        return rc;
    };
    b->insts.assign(insts, insts + count);
    for (int i = 0; i < count; ++i) b->versions.push_back(insts[i]->version);
    b->par = *par;
    b->st = static_cast<cudaStream_t>(par->cuda_stream);
    b->count = count;
    b->P = P;
    b->I = I;
    b->nisl = P / I;
    b->side = side;
    b->cluster = std::min(b->nisl, 8);  // one CTA per island, up to the portable cluster size
    // arena layout, 256-byte aligned pieces
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    std::vector<size_t> base(count);
    size_t off = 0;
    for (int i = 0; i < count; ++i) {
        const ffs_instance *in = insts[i];
        const size_t PK = (size_t)P * in->K, NK = (size_t)b->nisl * in->K;
        base[i] = off;
        off += al(in->hdr.bytes) + 2 * (al(2 * PK) + al(PK) + 2 * al(8 * (size_t)P)) + 2 * (al(2 * NK) + al(NK)) +
               4 * al(8 * (size_t)b->nisl) + al(4 * (size_t)b->nisl);
        b->Hmax = std::max(b->Hmax, in->hdr.H);
    }
    b->arena_bytes = off;
    if (dalloc(&b->arena, off) != cudaSuccess || dalloc(&b->d_inst, (size_t)count) != cudaSuccess ||
        dalloc(&b->d_order, (size_t)count) != cudaSuccess || dalloc(&b->d_next, 1) != cudaSuccess ||
        dalloc(&b->d_err, 1) != cudaSuccess)
        return fail(FFS_E_NOMEM);
    {
        void *hp = nullptr;
        if (cudaHostAlloc(&hp, sizeof(int32_t), cudaHostAllocMapped) != cudaSuccess) return fail(FFS_E_NOMEM);
        b->stop_host = static_cast<volatile int32_t *>(hp);
        *b->stop_host = 0;
        void *dp = nullptr;
        const int mrc = cuda_rc(cudaHostGetDevicePointer(&dp, hp, 0));
        if (mrc != FFS_OK) return fail(mrc);
        b->stop_dev = static_cast<int32_t *>(dp);
    }
    b->h_inst.resize(count);
    std::vector<std::pair<long long, int>> work(count);
    int rc = FFS_OK;
    for (int i = 0; i < count && rc == FFS_OK; ++i) {
        const ffs_instance *in = insts[i];
        const size_t PK = (size_t)P * in->K, NK = (size_t)b->nisl * in->K;
        char *p = b->arena + base[i];
        auto take = [&](size_t bytes) {
            char *q = p;
            p += al(bytes);
            return q;
        };
        BatchInst &h = b->h_inst[i];
        h = BatchInst{};
        char *blob = take(in->hdr.bytes);
        h.blob = blob;
        h.blob_bytes = in->hdr.bytes;
        h.N = in->N;
        h.M = in->M;
        h.K = in->K;
        h.H = in->hdr.H;
        h.nisl = b->nisl;
        h.gen = 0;
        h.iid = (uint32_t)(par->instance_id + i) & 0xFFFFFFu;
        h.emax = 0;
        for (int s = 0; s < 2; ++s) {
            h.Y[s] = reinterpret_cast<int16_t *>(take(2 * PK));
            h.X[s] = reinterpret_cast<int8_t *>(take(PK));
            h.obj[s] = reinterpret_cast<int64_t *>(take(8 * (size_t)P));
            h.fit[s] = reinterpret_cast<int64_t *>(take(8 * (size_t)P));
        }
        h.bY = reinterpret_cast<int16_t *>(take(2 * NK));
        h.mY = reinterpret_cast<int16_t *>(take(2 * NK));
        h.bX = reinterpret_cast<int8_t *>(take(NK));
        h.mX = reinterpret_cast<int8_t *>(take(NK));
        h.bobj = reinterpret_cast<int64_t *>(take(8 * (size_t)b->nisl));
        h.bfit = reinterpret_cast<int64_t *>(take(8 * (size_t)b->nisl));
        h.mobj = reinterpret_cast<int64_t *>(take(8 * (size_t)b->nisl));
        h.mfit = reinterpret_cast<int64_t *>(take(8 * (size_t)b->nisl));
        h.mw = reinterpret_cast<int32_t *>(take(4 * (size_t)b->nisl));
        work[i] = {-(long long)in->K * (in->N + in->hdr.H / 64), i};  // largest first
    }
    if (rc != FFS_OK) return fail(rc);
    std::sort(work.begin(), work.end());
    std::vector<int32_t> order(count);
    for (int i = 0; i < count; ++i) order[i] = work[i].second;
    if ((rc = cuda_rc(cudaMemset(b->arena, 0, b->arena_bytes))) != FFS_OK) return fail(rc);
    for (int i = 0; i < count && rc == FFS_OK; ++i) {  // tables again: the memset cleared them
        rc = cuda_rc(cudaMemcpy(const_cast<char *>(b->h_inst[i].blob), insts[i]->blob.data(), insts[i]->hdr.bytes,
                                cudaMemcpyHostToDevice));
    }
    if (rc == FFS_OK) rc = cuda_rc(cudaMemcpy(b->d_inst, b->h_inst.data(), sizeof(BatchInst) * count, cudaMemcpyHostToDevice));
    if (rc == FFS_OK) rc = cuda_rc(cudaMemcpy(b->d_order, order.data(), 4 * (size_t)count, cudaMemcpyHostToDevice));
    if (rc == FFS_OK) rc = cuda_rc(cudaMemset(b->d_err, 0, 4));
    if (rc == FFS_OK) {  // default mapping: the widest of these that every instance fits
        rc = FFS_E_ARG;
        const int def[][2] = {{8, 112 * 1024}, {4, 112 * 1024}, {4, 225 * 1024}, {1, 225 * 1024}};
        for (const auto &d : def)
            if ((rc = batch_config(b, d[0], d[1], b->cluster)) == FFS_OK) break;
    }
    if (rc == FFS_OK) rc = batch_enqueue(b, 0, b->st);  // generation 0 of every instance
    if (rc == FFS_OK) rc = batch_check(b);
    if (rc != FFS_OK) return fail(rc);
    *out = b;
    return FFS_OK;
}

int ga_batch_destroy(ga_batch *b) {
    delete b;
    return FFS_OK;
}

int ga_batch_stop(ga_batch *b) {
    if (!b || !b->stop_host) return FFS_E_ARG;
    *b->stop_host = 1;
    return FFS_OK;
}

int ga_batch_set_config(ga_batch *b, const ga_batch_config *cfg) {
    if (!b || !cfg) return FFS_E_ARG;
    return batch_config(b, cfg->warps_per_cta, cfg->smem_bytes, cfg->cluster > 0 ? cfg->cluster : b->cluster);
}

int ga_batch_get_config(const ga_batch *b, ga_batch_config *cfg) {
    if (!b || !cfg) return FFS_E_ARG;
    cfg->warps_per_cta = b->warps;
    cfg->smem_bytes = b->smem;
    cfg->ctas = b->grid;
    cfg->cluster = b->cluster;
    cfg->ms_per_generation = b->tuned_ms;
    return FFS_OK;
}

int ga_batch_run(ga_batch *b, int32_t generations, ffs_result *best) {
    if (!b || generations < 0) return FFS_E_ARG;
    for (int i = 0; i < b->count; ++i)
        if (b->insts[i]->version != b->versions[i]) return FFS_E_STATE;
    if (b->graph_gens != generations) {  // capture the launch once per generation count
        if (b->graph) cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
        cudaStream_t cap = nullptr;
        FFS_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        int rc = cuda_rc(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
        if (rc == FFS_OK) rc = batch_enqueue(b, generations, cap, true);
        const int ce = cuda_rc(cudaStreamEndCapture(cap, &g));
        cudaStreamDestroy(cap);
        if (rc == FFS_OK) rc = ce;
        if (rc == FFS_OK) rc = cuda_rc(cudaGraphInstantiate(&b->graph, g, 0));
        if (g) cudaGraphDestroy(g);
        if (rc != FFS_OK) return rc;
        b->graph_gens = generations;
        g_launches -= 1;  // counted at replay
    }
    *b->stop_host = 0;  // a request made before this run has no effect on it
    FFS_CUDA(cudaGraphLaunch(b->graph, b->st));
    g_launches += 1;
    FFS_TRY(batch_check(b));
    if (*b->stop_host == 2) return FFS_E_STOPPED;
    if (!best) return FFS_OK;
    // best-ever island of every instance, decoded and committed
    for (int i = 0; i < b->count; ++i) {
        const BatchInst &h = b->h_inst[i];
        std::vector<int64_t> bfit(b->nisl);
        FFS_CUDA(cudaMemcpy(bfit.data(), h.bfit, 8 * (size_t)b->nisl, cudaMemcpyDeviceToHost));
        int bi = 0;
        for (int q = 1; q < b->nisl; ++q)
            if (bfit[q] > bfit[bi]) bi = q;
        ffs_instance *in = b->insts[i];
        const size_t NG = (size_t)in->N * in->g;
        int64_t *d_o = nullptr, *d_t = nullptr;
        int32_t *d_c = nullptr, *d_S = nullptr, *d_M = nullptr;
        int rc = FFS_OK;
        if (dalloc(&d_o, 1) != cudaSuccess || dalloc(&d_t, 1) != cudaSuccess || dalloc(&d_c, 1) != cudaSuccess ||
            dalloc(&d_S, NG) != cudaSuccess || dalloc(&d_M, NG) != cudaSuccess)
            rc = FFS_E_NOMEM;
        if (rc == FFS_OK)
            rc = decode_impl(in, b->par.order_mode, b->par.machine_mode, h.bY + (size_t)bi * in->K,
                             h.bX + (size_t)bi * in->K, 1, d_o, d_t, d_c, d_S, d_M, b->st);
        if (rc == FFS_OK) rc = ffs_decode_check(in, b->st);
        std::vector<int32_t> S(NG), M(NG);
        int64_t o = 0, t = 0;
        int32_t cm = 0;
        if (rc == FFS_OK) rc = cuda_rc(cudaMemcpy(S.data(), d_S, 4 * NG, cudaMemcpyDeviceToHost));
        if (rc == FFS_OK) rc = cuda_rc(cudaMemcpy(M.data(), d_M, 4 * NG, cudaMemcpyDeviceToHost));
        if (rc == FFS_OK) rc = cuda_rc(cudaMemcpy(&o, d_o, 8, cudaMemcpyDeviceToHost));
        if (rc == FFS_OK) rc = cuda_rc(cudaMemcpy(&t, d_t, 8, cudaMemcpyDeviceToHost));
        if (rc == FFS_OK) rc = cuda_rc(cudaMemcpy(&cm, d_c, 4, cudaMemcpyDeviceToHost));
        dfree(d_o); dfree(d_t); dfree(d_c); dfree(d_S); dfree(d_M);
        if (rc != FFS_OK) return rc;
        FFS_TRY(ffs_commit(in, S.data(), M.data()));
        b->versions[i] = in->version;
        best[i].objective = o;
        best[i].total_tardiness = t;
        best[i].makespan = cm;
        best[i].n_ops = (int32_t)NG;
        if (best[i].start) std::memcpy(best[i].start, S.data(), 4 * NG);
        if (best[i].machine) std::memcpy(best[i].machine, M.data(), 4 * NG);
    }
    return FFS_OK;
}

int ga_batch_read(ga_batch *b, int32_t index, int16_t *Y, int8_t *X, int64_t *obj, int64_t *fit, int16_t *bY,
                  int8_t *bX, int64_t *bobj, int64_t *bfit, int64_t *emax, int32_t *generation) {
    if (!b || index < 0 || index >= b->count) return FFS_E_ARG;
    FFS_CUDA(cudaStreamSynchronize(b->st));
    BatchInst h;
    FFS_CUDA(cudaMemcpy(&h, b->d_inst + index, sizeof(h), cudaMemcpyDeviceToHost));
    const int s = h.gen & 1;
    const size_t PK = (size_t)b->P * h.K, NK = (size_t)b->nisl * h.K;
    if (Y) FFS_CUDA(cudaMemcpy(Y, h.Y[s], 2 * PK, cudaMemcpyDeviceToHost));
    if (X) FFS_CUDA(cudaMemcpy(X, h.X[s], PK, cudaMemcpyDeviceToHost));
    if (obj) FFS_CUDA(cudaMemcpy(obj, h.obj[s], 8 * (size_t)b->P, cudaMemcpyDeviceToHost));
    if (fit) FFS_CUDA(cudaMemcpy(fit, h.fit[s], 8 * (size_t)b->P, cudaMemcpyDeviceToHost));
    if (bY) FFS_CUDA(cudaMemcpy(bY, h.bY, 2 * NK, cudaMemcpyDeviceToHost));
    if (bX) FFS_CUDA(cudaMemcpy(bX, h.bX, NK, cudaMemcpyDeviceToHost));
    if (bobj) FFS_CUDA(cudaMemcpy(bobj, h.bobj, 8 * (size_t)b->nisl, cudaMemcpyDeviceToHost));
    if (bfit) FFS_CUDA(cudaMemcpy(bfit, h.bfit, 8 * (size_t)b->nisl, cudaMemcpyDeviceToHost));
    if (emax) *emax = h.emax;
    if (generation) *generation = h.gen;
    return FFS_OK;
}

int ga_batch_tune(ga_batch *b, int32_t generations, ga_batch_config *chosen) {
    if (!b || generations < 1) return FFS_E_ARG;
    if (!b->shadow) FFS_CUDA(dalloc(&b->shadow, b->arena_bytes));
    std::vector<BatchInst> saved(b->count);
    FFS_CUDA(cudaStreamSynchronize(b->st));
    FFS_CUDA(cudaMemcpy(saved.data(), b->d_inst, sizeof(BatchInst) * b->count, cudaMemcpyDeviceToHost));
    FFS_CUDA(cudaMemcpy(b->shadow, b->arena, b->arena_bytes, cudaMemcpyDeviceToDevice));
    cudaEvent_t e0, e1;
    FFS_CUDA(cudaEventCreate(&e0));
    FFS_CUDA(cudaEventCreate(&e1));
    const int warps_c[] = {4, 8, 16};
    const int smem_c[] = {56 * 1024, 75 * 1024, 112 * 1024, 225 * 1024};
    const int cluster_c[] = {8, 4, 2};
    float best_ms = 1e30f;
    int bw = b->warps, bs = b->smem, bc = b->cluster, rc = FFS_OK;
    for (int ci = 0; ci < 3 && rc == FFS_OK; ++ci) {
        for (int wi = 0; wi < 3 && rc == FFS_OK; ++wi) {
            for (int si = 0; si < 4 && rc == FFS_OK; ++si) {
                // skip mappings that do not fit every instance or cannot be resident
                if (batch_config(b, warps_c[wi], smem_c[si], cluster_c[ci]) != FFS_OK) continue;
                rc = cuda_rc(cudaEventRecord(e0, b->st));
                if (rc == FFS_OK) rc = batch_enqueue(b, generations, b->st);
                if (rc == FFS_OK) rc = cuda_rc(cudaEventRecord(e1, b->st));
                if (rc == FFS_OK) rc = batch_check(b);
                float ms = 0.f;
                if (rc == FFS_OK) rc = cuda_rc(cudaEventElapsedTime(&ms, e0, e1));
                if (rc == FFS_OK && ms < best_ms) {
                    best_ms = ms;
                    bw = warps_c[wi];
                    bs = smem_c[si];
                    bc = cluster_c[ci];
                }
                // restore the state the trial advanced
                if (rc == FFS_OK)
                    rc = cuda_rc(cudaMemcpy(b->arena, b->shadow, b->arena_bytes, cudaMemcpyDeviceToDevice));
                if (rc == FFS_OK)
                    rc = cuda_rc(cudaMemcpy(b->d_inst, saved.data(), sizeof(BatchInst) * b->count,
                                            cudaMemcpyHostToDevice));
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != FFS_OK) return rc;
    FFS_TRY(batch_config(b, bw, bs, bc));
    b->tuned_ms = best_ms / (float)generations;
    if (chosen) FFS_TRY(ga_batch_get_config(b, chosen));
    return FFS_OK;
}

}  // extern "C"
