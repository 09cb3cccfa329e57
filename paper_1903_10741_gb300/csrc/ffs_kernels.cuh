// ffs_kernels.cuh -- kernel argument blocks and launch wrappers (host-visible).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "ffs_layout.h"

namespace edffs {

constexpr int kWarpsPerBlock = 4;

struct DecodeArgs {
    const char *blob;
    int blob_bytes;
    int Hcap;                   // profile slots per warp (shared or global)
    const int16_t *Y[2];        // [.][K] chromosomes; GA mode picks the child buffer
    const int8_t *X[2];
    int count;                  // number of chromosomes (when list == nullptr)
    const int32_t *list;        // optional indirection (fallback after overflow)
    const int32_t *list_count;  // device count for `list`
    int64_t *obj[2];
    int64_t *tard;
    int32_t *cmax;
    int64_t *fit[2];            // GA mode: fitness = max(E_max - obj, 0)
    const GADev *gdev;          // non-null: GA mode, buffer (gen + 1) & 1
    int32_t *S;                 // optional schedule output [count][N*g]
    int32_t *Mo;
    const int32_t *S0;          // committed plan (frozen ops), [N*g]
    const int32_t *M0;
    const int32_t *status;      // [N*g]
    uint16_t *gscratch;         // global-profile variant: Hcap slots per resident warp
    int32_t *over_list;         // shared-profile variant: chromosomes that overflowed
    int32_t *over_count;
    int32_t *err;
    // failure injection for tests: skip the table copy and wait only this many iterations
    // (0: the default limit); no copy is then in flight when the wait runs out
    int inject_skip, wait_iters;
};

struct GenArgs {
    const char *blob;
    int blob_bytes;
    int Hcap;                   // shared-memory profile slots per warp
    int H;                      // full profile bound: slots per warp of gscratch
    uint16_t *gscratch;         // global profiles for children that outgrow Hcap
    int16_t *Y[2];
    int8_t *X[2];
    int64_t *obj[2];
    int64_t *fit[2];
    GADev *dev;
    int P, I, K, tour_k, side;  // side: torus side for 5-neighbourhood selection
    // Generation gen_ofs of a chain launched together (the counter is read as it stood when
    // the chain began); only a chain's last generation (publish) advances the counter.
    int gen_ofs, publish;
    uint64_t pc_thr, pm_thr;    // floor(p * 2^32)
    uint32_t instance_id;
    uint64_t seed;
    int32_t *over_list;
    int32_t *err;
    // island bookkeeping, done by the last warp to finish each island
    int32_t *isl_done;          // [n_isl] children finished this generation
    int nisl, migrate_every;
    int16_t *bY;                // best-ever individual per island
    int8_t *bX;
    int64_t *bobj, *bfit;
    int16_t *mY;                // migrants (island bests after replacement)
    int8_t *mX;
    int64_t *mobj, *mfit;
    int32_t *mw;                // worst slot of each island at migration time
    // surrogate-assisted generations (null cand_Y: plain generations)
    int F;                      // candidates per slot
    int Kpad;                   // row length of the BF16 model inputs
    int16_t *cand_Y;            // [P*F][K] candidates
    int8_t *cand_X;
    uint16_t *cand_Yh;          // [P*F][Kpad] BF16 within-stage rank features (zero padded)
    const float *cand_out;      // [P*F] surrogate scores, lower is better
    uint8_t *cand_new;          // [P*F] 1 if the candidate is an offspring, 0 if a parent's copy
    uint16_t *kept_Yh;          // [P][Kpad] inputs of the kept candidates, for training
    int64_t *kept_obj;          // [P] their exact objectives (before replacement)
    uint64_t screen_thr;        // an offspring slot takes the model's pick iff its draw < this
    const int32_t *cand_keep;   // [P] candidate kept for each slot (island top rule), or null
    int warm;                   // generation 0 decodes the rows already in Y[0] / X[0]
};

// Warm start: the rows of an earlier population of the same instance, carried over to
// the gene set of a later rescheduling point (see k_warm_remap).
struct WarmArgs {
    const int16_t *Yo[2];       // old population, both buffers; the current one is odev->gen & 1
    const int8_t *Xo[2];
    const GADev *odev;
    int Po, Ko;
    const int32_t *map;         // [Ko] new gene index of old gene k, or -1 if it froze
    const int32_t *fresh;       // [n_new] genes with no old counterpart, ascending
    int n_new;
    int16_t *Y;                 // [P][K] generation-0 rows
    int8_t *X;
    int P, K;
    int32_t *err;
};

struct ReplArgs {
    int16_t *Y[2];
    int8_t *X[2];
    int64_t *obj[2];
    int64_t *fit[2];
    int16_t *bY;
    int8_t *bX;
    int64_t *bobj, *bfit;
    int16_t *mY;                // migrant buffer [n_isl][K]
    int8_t *mX;
    int64_t *mobj, *mfit;
    int32_t *mw;                // worst slot of each island at migration time
    GADev *dev;
    int P, I, K, migrate_every;
    int init;                   // 1: generation 0 (set E_max, fitness, best-ever)
};

// One instance of a batch: its tables and device-resident GA state.
struct BatchInst {
    const char *blob;
    int blob_bytes, N, M, K, H, nisl;
    int gen;                    // generations completed
    uint32_t iid;               // 24-bit stream id
    long long emax;             // 0 until generation 0 has run
    int16_t *Y[2];
    int8_t *X[2];
    int64_t *obj[2], *fit[2];
    int16_t *bY, *mY;
    int8_t *bX, *mX;
    int64_t *bobj, *bfit, *mobj, *mfit;
    int32_t *mw;
};

struct BatchArgs {
    BatchInst *inst;
    int count;
    const int32_t *order;       // instances, largest work first
    int32_t *next;              // instance queue head: zeroed before each launch
    int generations;
    int P, I, tour_k, side, migrate_every;
    uint64_t pc_thr, pm_thr, seed;
    int smem_bytes;             // dynamic shared memory of a CTA
    uint16_t *gscratch;         // Hmax slots per (CTA, warp)
    int Hmax;
    int32_t *err;
    // host-mapped stop word: nonzero asks the launch to end at a generation boundary; a
    // cluster that ends early sets it to 2
    volatile int32_t *stop;
};

#ifdef FFS_CHECKED
// Bounds-checked builds: index faults counted since the last call in the decode and GA
// kernels' and in the batched kernel's translation units (read and cleared).
unsigned int bounds_faults_kernels();
unsigned int bounds_faults_batch();
#endif

cudaError_t prepare_batch(int order, int mach, int smem_bytes);
// Clusters of `cluster` CTAs of the given shape that can be resident at once.
cudaError_t batch_max_clusters(int order, int mach, int cluster, int warps, int smem_bytes, int *clusters);
cudaError_t launch_batch(int order, int mach, const BatchArgs &a, int grid, int warps, int cluster,
                         cudaStream_t st);

// Shared memory needed by one CTA of the decode / GA kernels.
int cta_smem_bytes(const TabHeader &h, int Hcap, bool ga, bool global_profile, bool insert = false);

cudaError_t launch_decode(int order, int mach, bool global_profile, const DecodeArgs &a,
                          const TabHeader &h, int grid, cudaStream_t st);
cudaError_t launch_ga_init(int order, int mach, const GenArgs &a, const TabHeader &h, int grid,
                           cudaStream_t st);
// overlap: launched as a programmatic dependent of the stream's previous kernel.
cudaError_t launch_ga_generation(int order, int mach, const GenArgs &a, const TabHeader &h,
                                 int grid, cudaStream_t st, bool overlap = false);
// Generations per graph of generations launched back to back.
constexpr int kGraphGens = 8;
cudaError_t prepare_ga_generation(int order, int mach, const TabHeader &h, int Hcap);
// Over-generation for the surrogate: P*F candidates (no decoding).
cudaError_t launch_candidates(int mach, const GenArgs &a, const TabHeader &h, int grid, cudaStream_t st);
cudaError_t prepare_candidates(int mach, const TabHeader &h);
cudaError_t launch_warm_remap(const WarmArgs &a, cudaStream_t st);
// Island top rule of surrogate screening: of the F * I candidates of each island (candidate
// f of slot j is row f P + j), the I best-scored (lowest score, ties to the lower row; an
// undefined score ranks last) are kept, and slot lo + r takes the r-th kept row in row
// order.  With is_new (offspring only): slots whose first candidate is a parent's plain
// copy keep it, and only offspring compete for the other places.  F * I <= kTopMax.
constexpr int kTopMax = 4096;
cudaError_t launch_island_top(const float *score, const uint8_t *is_new, int P, int F, int I, int32_t *keep,
                              cudaStream_t st);
cudaError_t launch_emax(const ReplArgs &a, cudaStream_t st);
cudaError_t launch_replace(const ReplArgs &a, cudaStream_t st);

}  // namespace edffs
