// ffs_internal.h -- host-side internals shared by the library's translation units: the
// instance and population objects behind the opaque C handles, allocation helpers and
// the error conventions.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <vector>

#include "ffs.h"
#include "ffs_kernels.cuh"
#include "ffs_layout.h"

namespace ffs_rt {

extern std::atomic<unsigned long long> g_launches;  // kernels issued by this library
extern thread_local char g_last_error[256];

int num_sms();
int cuda_rc(cudaError_t e);  // FFS_OK, or FFS_E_CUDA with the error text kept

// Device memory comes from cudaMalloc, or, while a thread has an arena set (a service
// allocating inside its fixed budget), from that arena; a block is returned to whichever
// arena holds it, without the device-wide synchronisation of cudaFree.
struct Arena;
extern thread_local Arena *t_arena;
constexpr size_t kArenaAlign = 256;
cudaError_t raw_alloc(void **p, size_t bytes);
void raw_free(void *p);

// Suspends the thread's arena for the guard's lifetime.
struct NoArena {
    Arena *saved;
    NoArena() : saved(t_arena) { t_arena = nullptr; }
    ~NoArena() { t_arena = saved; }
    NoArena(const NoArena &) = delete;
    NoArena &operator=(const NoArena &) = delete;
};

template <typename T>
cudaError_t dalloc(T **p, size_t n) {
    *p = nullptr;
    if (n == 0) n = 1;
    return raw_alloc(reinterpret_cast<void **>(p), n * sizeof(T));
}

template <typename T>
void dfree(T *&p) {
    if (p) raw_free(p);
    p = nullptr;
}

#define FFS_TRY(expr)                  \
    do {                               \
        const int rc_ = (expr);        \
        if (rc_ != FFS_OK) return rc_; \
    } while (0)
#define FFS_CUDA(expr) FFS_TRY(ffs_rt::cuda_rc(expr))

}  // namespace ffs_rt

using ffs_rt::dalloc;
using ffs_rt::dfree;

struct ffs_instance;
namespace ffs_rt {
// P_jsm and Q_jsm (Table 2) of job j's op at stage s on stage-local machine m.
int op_p(const ffs_instance *in, int j, int s, int m);
int op_q(const ffs_instance *in, int j, int s, int m);
}  // namespace ffs_rt

struct ffs_instance {
    int N = 0, g = 0, M = 0, Qmax = 0, WT = 0, RS = 0;
    std::vector<int32_t> o, moff, p, q, R, D;   // problem
    bool unrel = false;                         // unrelated machines: P_jsm, Q_jsm per job and machine
    std::vector<int32_t> pm, qm;                // [N][M] when unrel
    std::vector<int32_t> status, S0, M0;       // plan and classification, [N*g]
    bool has_plan = false;
    bool dev_dirty = true;  // host tables or plan changed since the last upload
    int K = 0, Hfull = 0;
    std::vector<int32_t> gjob, gstg;
    edffs::TabHeader hdr{};
    std::vector<char> blob;
    int version = 0;
    // device mirrors
    char *d_blob = nullptr;
    size_t d_blob_cap = 0;
    int32_t *d_S0 = nullptr, *d_M0 = nullptr, *d_status = nullptr;
    size_t d_plan_cap = 0;
    uint16_t *d_scratch = nullptr;  // global power profiles for the fallback decode
    size_t d_scratch_cap = 0;
    int32_t *d_over = nullptr;
    size_t d_over_cap = 0;
    int32_t *d_over_count = nullptr, *d_err = nullptr;

    ~ffs_instance() {
        dfree(d_blob);
        dfree(d_S0);
        dfree(d_M0);
        dfree(d_status);
        dfree(d_scratch);
        dfree(d_over);
        dfree(d_over_count);
        dfree(d_err);
    }
};

struct ga_population {
    ffs_instance *inst = nullptr;
    int version = 0;
    ga_params par{};
    cudaStream_t st = nullptr;
    int P = 0, I = 0, K = 0, nisl = 0, side = 0;
    int Hcap = 0, grid_gen = 0, grid_fb = 0;
    edffs::TabHeader hdr{};
    char *d_blob = nullptr;  // private copy of the instance tables at creation
    int16_t *Y[2] = {nullptr, nullptr};
    int8_t *X[2] = {nullptr, nullptr};
    int64_t *obj[2] = {nullptr, nullptr}, *fit[2] = {nullptr, nullptr};
    int16_t *bY = nullptr, *mY = nullptr;
    int8_t *bX = nullptr, *mX = nullptr;
    int64_t *bobj = nullptr, *bfit = nullptr, *mobj = nullptr, *mfit = nullptr;
    int32_t *mw = nullptr, *over = nullptr, *err = nullptr, *isl_done = nullptr;
    edffs::GADev *dev = nullptr;
    uint16_t *scratch = nullptr;
    cudaGraphExec_t graph = nullptr;
    std::vector<int64_t> gkey;              // job * g + stage of each gene at creation
    // decode of the best-ever individual (ga_finish)
    int64_t *r_obj = nullptr, *r_tard = nullptr;
    int32_t *r_cm = nullptr, *r_S = nullptr, *r_M = nullptr, *r_over = nullptr, *r_cnt = nullptr;
    int NG = 0;
    // surrogate-assisted generations (see ffs_surrogate.cu)
    struct ffs_surrogate *sur = nullptr;
    int F = 1;
    float lr = 0.f;
    int16_t *cand_Y = nullptr;
    int8_t *cand_X = nullptr;
    uint16_t *cand_Yh = nullptr, *cand_H1 = nullptr, *cand_H2 = nullptr;
    float *cand_out = nullptr;
    uint8_t *cand_new = nullptr;
    int64_t *kept_obj = nullptr;
    int train_steps = 1;
    uint64_t screen_thr = (uint64_t)1 << 32;  // floor(screen probability * 2^32)
    int keep_rule = 0;                      // FFS_KEEP_SLOT or FFS_KEEP_ISLAND
    int32_t *cand_keep = nullptr;           // [P] kept candidate of each slot (island rule)
    std::vector<cudaEvent_t> ev_sur;        // profiling: phase events of surrogate generations
    double phase_ms[5] = {0, 0, 0, 0, 0};   // candidates, scoring, keep rule, exact decode, training
    cudaGraphExec_t graph_sur = nullptr;
    cudaGraphExec_t graph_r = nullptr;      // kGraphGens generations, each launched as the previous one drains
    int profiling = 0;                      // 1: eager launches with timed generation kernels;
                                            // 2: graph replays, each bracketed by events
    std::vector<cudaEvent_t> ev;            // event pairs, reused across ga_run calls
    double prof_ms = 0.0;
    int64_t prof_launches = 0;

    ~ga_population() {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        if (graph) cudaGraphExecDestroy(graph);
        if (graph_sur) cudaGraphExecDestroy(graph_sur);
        if (graph_r) cudaGraphExecDestroy(graph_r);
        dfree(cand_Y);
        dfree(cand_X);
        dfree(cand_Yh);
        dfree(cand_H1);
        dfree(cand_H2);
        dfree(cand_out);
        dfree(cand_new);
        dfree(kept_obj);
        dfree(cand_keep);
        for (cudaEvent_t e : ev_sur) cudaEventDestroy(e);
        dfree(d_blob);
        for (int b = 0; b < 2; ++b) {
            dfree(Y[b]);
            dfree(X[b]);
            dfree(obj[b]);
            dfree(fit[b]);
        }
        dfree(bY); dfree(bX); dfree(bobj); dfree(bfit);
        dfree(mY); dfree(mX); dfree(mobj); dfree(mfit); dfree(mw);
        dfree(over); dfree(err); dfree(dev); dfree(scratch); dfree(isl_done);
        dfree(r_obj); dfree(r_tard); dfree(r_cm); dfree(r_S); dfree(r_M); dfree(r_over); dfree(r_cnt);
    }
};


namespace ffs_rt {

int check_modes(int32_t order_mode, int32_t machine_mode);
int sync_device(ffs_instance *in);
int decode_impl(ffs_instance *in, int32_t order, int32_t mach, const int16_t *y, const int8_t *x, int32_t count,
                int64_t *obj, int64_t *tard, int32_t *cmax, int32_t *S, int32_t *Mo, cudaStream_t st);
void ga_gen_args(ga_population *pp, edffs::GenArgs *a);
// Enqueues `generations` generations on the population's stream without waiting.  In
// profiling mode 2 each graph replay is bracketed by an event pair (pp->ev) and *timed
// gets the number of pairs.
int ga_enqueue(ga_population *pp, int32_t generations, int *timed = nullptr);
// Waits for the population's stream, then decodes, commits and returns the best-ever schedule.
int ga_finish(ga_population *pp, ffs_result *best);
// Device bytes a population of `in` with `par` holds (each buffer rounded to kArenaAlign).
int population_footprint(ffs_instance *in, const ga_params *par, int64_t *bytes);
// ga_population_create / ga_population_create_warm (prev may be null).
int population_create(ffs_instance *in, const ga_params *par, ga_population *prev, ga_population **out);
// Frees everything but the chromosomes (both buffers) and the generation counter: what a
// warm start reads.  The population can then only be a warm start's source or destroyed.
void population_trim(ga_population *pp);
// One surrogate-assisted generation on `st` (ffs_surrogate.cu); with events, the fused
// generation kernel is bracketed by ev0/ev1.  Kernels launched per generation:
constexpr int kSurrogateFixedLaunches = 12, kSurrogateStepLaunches = 18;
// ... plus one with the island keep rule.
int surrogate_launches_per_generation(const ga_population *pp);
// The attached surrogate scores candidates by their exact objectives (a diagnostic); such
// generations are launched directly, not from a captured graph.
bool surrogate_is_exact(const ga_population *pp);
// FFS_E_TIMEOUT if a tensor-core GEMM recorded a wait timeout since the last call (and
// clears it).  Synchronous.
int surrogate_status();
int surrogate_enqueue_generation(ga_population *pp, cudaStream_t st, cudaEvent_t ev0, cudaEvent_t ev1,
                                 cudaEvent_t *phase = nullptr);
// Raises the shared-memory limits of the kernels a surrogate generation launches, so that
// the generation can be captured.
int prepare_surrogate_kernels(ga_population *pp);

}  // namespace ffs_rt
