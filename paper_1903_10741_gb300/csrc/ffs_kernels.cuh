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

// Shared memory needed by one CTA of the decode / GA kernels.
int cta_smem_bytes(const TabHeader &h, int Hcap, bool ga, bool global_profile);

cudaError_t launch_decode(int order, int mach, bool global_profile, const DecodeArgs &a,
                          const TabHeader &h, int grid, cudaStream_t st);
cudaError_t launch_ga_init(int order, int mach, const GenArgs &a, const TabHeader &h, int grid,
                           cudaStream_t st);
cudaError_t launch_ga_generation(int order, int mach, const GenArgs &a, const TabHeader &h,
                                 int grid, cudaStream_t st);
cudaError_t prepare_ga_generation(int order, int mach, const TabHeader &h, int Hcap);
cudaError_t launch_emax(const ReplArgs &a, cudaStream_t st);
cudaError_t launch_replace(const ReplArgs &a, cudaStream_t st);

}  // namespace edffs
