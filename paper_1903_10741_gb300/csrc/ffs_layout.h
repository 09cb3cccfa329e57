// ffs_layout.h -- device-resident layout of an EDFFS instance and of the per-warp decode
// workspace.  Shared by the host runtime (which builds the tables) and the kernels (which
// stage them into shared memory with one bulk copy).  Internal to the library.
#pragma once
#include <stdint.h>
#ifndef __CUDACC__
struct uint2 { unsigned int x, y; };
#else
#include <vector_types.h>
#endif

#ifdef __CUDACC__
#define FFS_HD __host__ __device__ __forceinline__
#else
#define FFS_HD inline
#endif

namespace edffs {

constexpr int kStFree = 0, kStExec = 1, kStDone = 2;  // Alg. 1 classification
constexpr int kStFixed = 3;  // static approach: a planned op kept at its start and machine

// Header at the start of the table blob.  Offsets are bytes from the blob start, each a
// multiple of 16 so the whole blob is one cp.async.bulk copy.
struct TabHeader {
    int32_t N, g, M, K;           // jobs, stages, machines, genes
    int32_t RS, Qmax, WT, H;      // rescheduling point, peak, weight, profile bound (slots past RS)
    int32_t E0, bytes, maxo, unrel;// slots of initial profile (executing ops), blob size, max o_s,
                                   // 1 for unrelated machines (per-gene, per-machine p and q)
    int32_t off_o, off_moff, off_q, off_p;
    int32_t off_R, off_D, off_C0, off_mfree0;
    int32_t off_gjob, off_gstg, off_gfirst, off_gcnt;
    int32_t off_h0, off_grec, off_soff, off_gm;
};
static_assert(sizeof(TabHeader) == 112, "header layout");

FFS_HD int align16(int x) { return (x + 15) & ~15; }

// Views into a staged blob.
struct Tabs {
    int N, g, M, K, RS, Qmax, WT, H, E0;
    const int32_t *o, *moff, *q, *R, *D, *C0, *mfree0;
    const int16_t *p, *gjob, *gfirst;
    const int8_t *gstg, *gcnt;
    const uint16_t *h0;
    // Per gene, packed: x = job | stage << 16 | o_stage << 24, y = p | first machine << 16.
    const uint2 *grec;
    const int32_t *soff;  // [g+1] first gene index of each stage in the stage-major order
    // Unrelated machines: [K][maxo] p | q << 16 of gene k on stage-local machine m (P_jsm,
    // Q_jsm of Table 2); null for identical machines.
    int maxo;
    const uint32_t *gm;
};

FFS_HD Tabs tabs_view(const char *base) {
    const TabHeader *h = reinterpret_cast<const TabHeader *>(base);
    Tabs t;
    t.N = h->N; t.g = h->g; t.M = h->M; t.K = h->K;
    t.RS = h->RS; t.Qmax = h->Qmax; t.WT = h->WT; t.H = h->H; t.E0 = h->E0;
    t.o = reinterpret_cast<const int32_t *>(base + h->off_o);
    t.moff = reinterpret_cast<const int32_t *>(base + h->off_moff);
    t.q = reinterpret_cast<const int32_t *>(base + h->off_q);
    t.p = reinterpret_cast<const int16_t *>(base + h->off_p);
    t.R = reinterpret_cast<const int32_t *>(base + h->off_R);
    t.D = reinterpret_cast<const int32_t *>(base + h->off_D);
    t.C0 = reinterpret_cast<const int32_t *>(base + h->off_C0);
    t.mfree0 = reinterpret_cast<const int32_t *>(base + h->off_mfree0);
    t.gjob = reinterpret_cast<const int16_t *>(base + h->off_gjob);
    t.gstg = reinterpret_cast<const int8_t *>(base + h->off_gstg);
    t.gfirst = reinterpret_cast<const int16_t *>(base + h->off_gfirst);
    t.gcnt = reinterpret_cast<const int8_t *>(base + h->off_gcnt);
    t.h0 = reinterpret_cast<const uint16_t *>(base + h->off_h0);
    t.grec = reinterpret_cast<const uint2 *>(base + h->off_grec);
    t.soff = reinterpret_cast<const int32_t *>(base + h->off_soff);
    t.maxo = h->maxo;
    t.gm = h->unrel ? reinterpret_cast<const uint32_t *>(base + h->off_gm) : nullptr;
    return t;
}

// Per-warp decode workspace in shared memory.
//   h     uint16 [Hcap]   power headroom Qmax - Q_t for t = RS + i (Eq. 7-8); Hcap is a
//                         multiple of 8 and the slice is read and written 4 slots at a time
//   C     int32  [N]      completion of each job's last assigned stage
//   mfree int32  [M]      end of the last op assigned to each machine
//   inv   int16  [K + N]  gene by priority rank, then the next gene of every job (Alg. 1)
//   y     int16  [K], x int8 [K]   the chromosome being decoded (y becomes the stage order)
//   bits  uint32 [K/32+1] value bitmap for the crossover correction (GA kernels only)
struct WarpLayout {
    int off_h, off_C, off_mfree, off_inv, off_y, off_x, off_bits, bytes;
};

// Insertion placement keeps, after the Hcap profile slots, one occupancy bitmap of
// busy_words(Hcap) words for each machine of the current stage (nmach of them).
FFS_HD int busy_words(int Hcap) { return (Hcap + 31) / 32; }
FFS_HD int profile_bytes(int Hcap, int nmach) { return align16(Hcap * 2 + nmach * 4 * busy_words(Hcap)); }
// Global-memory workspace of one warp in uint16 units: the profile bound H and, with
// insertion, the occupancy bitmaps of up to maxo machines.
FFS_HD size_t gwork_stride(int H, int maxo, bool insert) {
    const size_t words = insert ? (size_t)maxo * (size_t)((H + 31) / 32) : 0;
    return ((size_t)H * 2 + words * 4 + 15) / 16 * 8;
}

FFS_HD WarpLayout warp_layout(int N, int M, int K, int Hcap, bool ga, int nmach = 0) {
    WarpLayout L;
    int o = 0;
    L.off_h = o;     o += profile_bytes(Hcap, nmach);
    L.off_C = o;     o += align16(N * 4);
    L.off_mfree = o; o += align16(M * 4);
    L.off_inv = o;   o += align16((K + N) * 2);
    L.off_y = o;     o += align16(K * 2);
    L.off_x = o;     o += align16(K);
    L.off_bits = o;  o += ga ? align16(((K + 32) / 32) * 4) : 0;
    L.bytes = o;
    return L;
}

// Device-side GA bookkeeping (one per population).
struct GADev {
    int32_t gen;     // generations completed; population lives in buffer gen & 1
    int32_t nover;   // children whose profile outgrew shared memory this generation
    int32_t err;     // sticky error bits (1 bad chromosome, 2 profile overflow, 4 wait timeout)
    int32_t islands_done;  // islands whose replacement finished this generation
    int64_t emax;    // E_max of Eq. (13)
};

constexpr int kErrBadChromosome = 1, kErrOverflow = 2, kErrTimeout = 4;
constexpr int kMaxK = 32767;  // genes per chromosome: priorities are int16

// Below this many profile slots per warp a shared-memory slice is not worth keeping.
constexpr int kMinBatchSlots = 256;

// Philox stream purposes.
constexpr uint32_t kPInitY = 1, kPInitX = 2, kPSelect = 3, kPCross = 4, kPMutate = 5;
constexpr uint32_t kPScreen = 6;  // surrogate: whether an offspring slot takes the model's pick

}  // namespace edffs
