/*
 * ffs.h -- C ABI of the GB300 EDFFS library: decoding of priority chromosomes into
 * energy-efficient flexible-flow-shop schedules and the priority-based hybrid parallel GA
 * with predictive-reactive complete rescheduling, after Luo, Fujimura & El Baz,
 * "GPU based Parallel Genetic Algorithm for Solving an Energy Efficient Dynamic Flexible
 * Flow Shop Scheduling Problem" (arXiv 1903.10741).
 *
 * Conventions
 *   - Every function returns FFS_OK (0) or a negative FFS_E_* code; ffs_strerror() names it.
 *   - Times, processing times and powers are int32 >= 0; objectives are int64.
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA global memory of
 *     the current device.  Inputs are copied at the call; the caller keeps ownership of
 *     every array it passes.  Opaque handles are owned by the library until destroyed.
 *   - A handle must not be used by two threads at once.
 *   - Stream arguments are cudaStream_t values passed as void* (NULL = legacy stream).
 *   - Matrices are row-major: op (j, s) of job j at stage s sits at index j * g + s.
 *   - Machines are numbered per stage (0 .. o_s - 1); "global" machine numbers are
 *     stage-major (stage 0's machines first).
 *   - Genes are the free operations at the current rescheduling point, numbered job-major
 *     then by stage (the row-major order of the X/Y matrices of Eq. (10)-(11) with their
 *     -1 cells removed).  K is their count.
 *
 * Size limits (checked, FFS_E_ARG beyond them): jobs and genes <= 32767, stages <= 127,
 * machines per stage <= 31, total machines <= 32767, processing time <= 32767, peak
 * power <= 32767, and the schedule horizon past the rescheduling point (the latest
 * release or executing end plus the total free processing time) below 2^26.
 */
#ifndef FFS_H
#define FFS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes */
#define FFS_OK            0
#define FFS_E_ARG        -1   /* invalid argument or size limit exceeded                 */
#define FFS_E_INFEASIBLE -2   /* some machine's power exceeds the peak, or a stage has no machine */
#define FFS_E_NOMEM      -3   /* device or host allocation failed                        */
#define FFS_E_CUDA       -4   /* a CUDA call failed                                      */
#define FFS_E_TIMEOUT    -5   /* a bounded device-side wait ran out                      */
#define FFS_E_ADMISSION  -6   /* the service cannot admit the request                    */
#define FFS_E_STATE      -7   /* call not valid in the handle's current state            */
#define FFS_E_DEVICE     -8   /* a kernel reported an internal error (bad chromosome, overflow) */
#define FFS_E_STOPPED    -9   /* a batched run ended early on a stop request (ga_batch_stop)  */

/* ---- decoding modes (Sec. 4.3) */
#define FFS_ORDER_TOPO      0  /* Alg. 1: largest y among the next free op of every job   */
#define FFS_ORDER_STAGE     1  /* stage by stage, y descending within a stage            */
#define FFS_MACH_GENE       0  /* machine of op (j, s) is x_js, Eq. (10)                 */
#define FFS_MACH_EARLIEST   1  /* machine with the earliest power-feasible start (completion,
                                  with unrelated machines)                                 */
/* Or-ed into a machine mode: idle-gap insertion placement (an option; the paper's Alg. 2
 * appends each op after the op last assigned to its machine).  An op may start in any
 * idle gap of its machine after the machine's frozen ops, with the same power check
 * (Eq. 7).  Only with FFS_ORDER_STAGE, and not in batched runs. */
#define FFS_PLACE_INSERT    4

typedef struct ffs_instance ffs_instance;      /* opaque: problem + rescheduling state    */
typedef struct ga_population ga_population;    /* opaque: device-resident GA state        */

/* An EDFFS instance, Table 2 of the paper.  All arrays are host memory.
 * Identical parallel machines: proc and power give P_js and each machine's Q, and
 * proc_machine / power_machine are NULL.  Unrelated machines (Table 2's P_jsm and Q_jsm):
 * proc_machine and power_machine give every job's processing time and power on every
 * machine, [n][sum o_s] with machines stage-major; proc and power are then ignored (may be
 * NULL).  With unrelated machines, FFS_MACH_EARLIEST picks the machine with the earliest
 * power-feasible completion (with identical machines that is the earliest start), and a
 * machine gene's op takes that machine's time and power. */
typedef struct {
    int32_t n_jobs;                      /* n                                           */
    int32_t n_stages;                    /* g                                           */
    const int32_t *machines_per_stage;   /* [g]  o_s >= 1 parallel machines              */
    const int32_t *proc;                 /* [n][g] P_js (the same on every machine of s) */
    const int32_t *power;                /* [sum o_s] Q of each machine, stage-major     */
    const int32_t *release;              /* [n]  R_j                                    */
    const int32_t *due;                  /* [n]  D_j                                    */
    int32_t peak_power;                  /* Q_max, Eq. (7)                              */
    int32_t wt;                          /* WT, Eq. (1)                                 */
    const int32_t *proc_machine;         /* [n][sum o_s] P_jsm, or NULL                  */
    const int32_t *power_machine;        /* [n][sum o_s] Q_jsm, or NULL                  */
} ffs_problem;

/* New jobs J' arriving at a rescheduling point (Sec. 4.1).  Host arrays.  For an
 * instance with unrelated machines proc_machine / power_machine are required and proc is
 * ignored; otherwise proc is required and they are ignored. */
typedef struct {
    int32_t job_count;                   /* n'                                          */
    const int32_t *proc;                 /* [n'][g]                                     */
    const int32_t *release;              /* [n']                                        */
    const int32_t *due;                  /* [n']                                        */
    const int32_t *proc_machine;         /* [n'][sum o_s] P_jsm, or NULL                 */
    const int32_t *power_machine;        /* [n'][sum o_s] Q_jsm, or NULL                 */
} ffs_arrivals;

/* GA settings (Sec. 4.2, 4.4). */
typedef struct {
    int32_t pop;            /* population size P, even, a multiple of `island`         */
    int32_t island;         /* island size (individuals per island), even              */
    int32_t tournament_k;   /* tournament size within the island; 0 = best of the 5-cell
                               neighbourhood on the sqrt(P) x sqrt(P) torus (P square)   */
    int32_t pc_num, pc_den; /* crossover probability per pair                          */
    int32_t pm_num, pm_den; /* mutation probability per individual                     */
    int32_t order_mode;     /* FFS_ORDER_*                                             */
    int32_t machine_mode;   /* FFS_MACH_*                                              */
    int32_t migrate_every;  /* ring migration period in generations; 0 = none          */
    int32_t instance_id;    /* 24-bit id mixed into every random stream                */
    uint64_t seed;          /* Philox4x32-10 key                                       */
    void *cuda_stream;      /* stream for every launch of this population              */
} ga_params;

/* Best schedule returned by ga_run. */
typedef struct {
    int64_t objective;        /* WT * sum_j T_j + C_max, Eq. (1)                      */
    int64_t total_tardiness;  /* sum_j T_j, Eq. (2)                                   */
    int32_t makespan;         /* C_max, Eq. (3)                                       */
    int32_t n_ops;            /* n_jobs * n_stages of the current instance            */
    int32_t *start;           /* host [n][g] S_js, or NULL; caller-allocated          */
    int32_t *machine;         /* host [n][g] M_js (stage-local), or NULL              */
} ffs_result;

/* Sizes of an instance at its current rescheduling point. */
typedef struct {
    int32_t n_jobs, n_stages, n_machines, n_genes;  /* N, g, sum o_s, K              */
    int32_t rs;                                     /* current rescheduling point     */
    int32_t horizon;        /* length of the power profile past RS that bounds any schedule */
    int32_t peak_power, wt;
} ffs_info;

/* ---------------------------------------------------------------- instances */

/* Creates an instance from the problem statement of Sec. 3.2 (Table 2), with RS = 0 and
 * every operation free.  Copies all inputs.  FFS_E_INFEASIBLE if some machine's power
 * exceeds peak_power (no schedule can satisfy Eq. 7) or some stage has no machine. */
int ffs_instance_create(const ffs_problem *problem, ffs_instance **out);

/* Frees an instance and its device tables.  NULL is accepted. */
int ffs_instance_destroy(ffs_instance *inst);

/* Sizes of the instance at its current rescheduling point. */
int ffs_instance_info(const ffs_instance *inst, ffs_info *info);

/* Gene numbering: host arrays [K] receive the job and the stage of every free op. */
int ffs_instance_genes(const ffs_instance *inst, int32_t *gene_job, int32_t *gene_stage);

/* Per-op status at the current rescheduling point: host [n][g], 0 free, 1 being executed,
 * 2 completed (Alg. 1, first branch), 3 fixed in the kept plan (ffs_reschedule_static). */
int ffs_instance_status(const ffs_instance *inst, int32_t *status);

/* Makes (start, machine) -- host [n][g], stage-local machines -- the plan being executed.
 * Frozen ops must keep their committed values.  ga_run commits its best schedule itself. */
int ffs_commit(ffs_instance *inst, const int32_t *start, const int32_t *machine);

/* Predictive-reactive complete rescheduling (Sec. 4.1, Alg. 1): at t_now, every op of the
 * committed plan with S + P <= t_now is completed, S < t_now < S + P is being executed
 * (keeps its machine and power until it ends), S >= t_now is free again; the arriving
 * jobs are appended with all stages free; genes are renumbered.  t_now must not precede
 * the previous rescheduling point (FFS_E_ARG); a plan must have been committed unless
 * every op is still free at t_now (FFS_E_STATE). */
int ffs_reschedule(ffs_instance *inst, const ffs_arrivals *arrivals, int32_t t_now);

/* The traditional static approach of Sec. 4.1 (Fig. 7) and Sec. 5.3 (Table 10), as the
 * comparison for ffs_reschedule: at t_now, ops of the committed plan that completed are
 * done and those running are being executed, as in Alg. 1; every other op of the plan is
 * fixed (status 3): it keeps its planned start and machine and draws its power over
 * [S, S + P).  Only the new jobs are genes, and each of their ops starts after the last
 * planned op of its machine.  Arguments and errors as ffs_reschedule. */
int ffs_reschedule_static(ffs_instance *inst, const ffs_arrivals *arrivals, int32_t t_now);

/* ---------------------------------------------------------------- decoding */

/* Decodes `count` chromosomes (Sec. 4.3, Alg. 1-2) and writes their objectives.
 *   y    device [count][K] int16, each row a permutation of 1..K (larger = higher priority)
 *   x    device [count][K] int8 stage-local machines (FFS_MACH_GENE), or NULL
 *   obj  device [count] int64 Eq. (1);  tard device [count] int64 or NULL;
 *   cmax device [count] int32 or NULL.
 * Asynchronous on `stream`; FFS_E_DEVICE is reported by a later synchronising call if a
 * row was not a permutation.  The kernel uses a device scratch buffer owned by the instance
 * for chromosomes whose schedule outgrows shared memory. */
int ffs_decode(ffs_instance *inst, int32_t order_mode, int32_t machine_mode,
               const int16_t *y, const int8_t *x, int32_t count,
               int64_t *obj, int64_t *tard, int32_t *cmax, void *stream);

/* As ffs_decode, and also writes every schedule: start, machine device [count][n][g]
 * (frozen ops carry their committed values). */
int ffs_decode_schedule(ffs_instance *inst, int32_t order_mode, int32_t machine_mode,
                        const int16_t *y, const int8_t *x, int32_t count,
                        int64_t *obj, int32_t *start, int32_t *machine, void *stream);

/* ---------------------------------------------------------------- batched GA */

/* Many independent instances, each with its own population, advanced together by one
 * persistent kernel launch (captured in a CUDA graph and replayed): a thread-block
 * cluster per instance, one CTA per island (up to 8 per cluster).  Not in the paper: it
 * serves many concurrent rescheduling requests with the GA of Sec. 4.4. */
typedef struct ga_batch ga_batch;

/* Launch mapping of a batch: warps per CTA, dynamic shared memory per CTA (tables plus
 * each warp's power profile slice), the resulting number of persistent CTAs, the cluster
 * size (a cluster owns one instance at a time and its CTAs share the islands), and the
 * milliseconds per generation the tuner measured (0 if not tuned). */
typedef struct {
    int32_t warps_per_cta;
    int32_t smem_bytes;
    int32_t ctas;
    int32_t cluster;          /* CTAs per instance (islands are dealt to them), 1..8 */
    float ms_per_generation;
} ga_batch_config;

/* Copies the `count` instances' current tables and runs generation 0 of every one.  All
 * share `params` (pop, island, operators, modes, seed, stream); instance i draws from
 * stream id params->instance_id + i, so its run equals ga_population_create + ga_run
 * with that id.  The instances must not be rescheduled while the batch is used. * Instances with unrelated machines are refused (FFS_E_ARG). FFS_PLACE_INSERT is refused too. */
int ga_batch_create(ffs_instance *const *insts, int32_t count, const ga_params *params, ga_batch **out);

/* Frees a batch.  NULL is accepted. */
int ga_batch_destroy(ga_batch *batch);

/* Advances every instance by `generations` generations in one launch.  With `best` (an
 * array of `count` results, caller-allocated, start/machine optional), each instance's
 * best-ever schedule is decoded, returned and committed to its instance. */
int ga_batch_run(ga_batch *batch, int32_t generations, ffs_result *best);

/* Asks a ga_batch_run in progress on `batch` (called from another host thread) to end
 * early, for a caller that must take the GPU back before a long persistent launch would
 * finish (a deadline, a shutdown).  The paper has no counterpart.  The request is one word
 * of host-mapped memory that each cluster of the launch reads at the start of every
 * generation; a cluster that sees it finishes no further generation and takes no further
 * instance.  Every instance is therefore left after a whole number of generations, in the
 * state a run of exactly that many generations gives (ga_batch_read returns each one's
 * count; instances may differ).  The run then returns FFS_E_STOPPED without decoding best
 * schedules.  A request made while no run is in progress, or one that arrives after every
 * cluster has finished, has no effect: each ga_batch_run clears it when it starts, and
 * ga_batch_tune's trials do not read it.  FFS_E_ARG for a NULL batch. */
int ga_batch_stop(ga_batch *batch);

/* As ga_population_read, for instance `index` of the batch. */
int ga_batch_read(ga_batch *batch, int32_t index, int16_t *Y, int8_t *X, int64_t *obj, int64_t *fit,
                  int16_t *bY, int8_t *bX, int64_t *bobj, int64_t *bfit, int64_t *emax,
                  int32_t *generation);

/* Autotuner: times `generations` generations under each candidate mapping (clusters of
 * 8/4/2 CTAs x 4/8/16 warps per CTA x 56/75/112/225 KB of shared memory per CTA) that fits
 * every instance,
 * restoring the batch state after every trial, and keeps the fastest.  Results never
 * depend on the mapping. */
int ga_batch_tune(ga_batch *batch, int32_t generations, ga_batch_config *chosen);

/* Reads or sets the mapping (warps 1..16, shared memory 16..227 KB, cluster 1..8 and at
 * most the island count; 0 keeps the current cluster size).  Setting a mapping that some
 * instance does not fit returns FFS_E_ARG. */
int ga_batch_get_config(const ga_batch *batch, ga_batch_config *config);
int ga_batch_set_config(ga_batch *batch, const ga_batch_config *config);

/* ---------------------------------------------------------------- learned surrogate */

/* A learned fitness surrogate for one instance at its current rescheduling point.  Not in
 * the paper: it lets the GA screen over-generated offspring before the exact decoder
 * (Sec. 4.3) evaluates the kept ones.  Model: with yh_k = 1 - r_k / n_s (r_k the rank of
 * gene k by y among the n_s genes of its stage, 0 for the highest) and per-gene features
 * ph = p_js / max p and dh = D_j / max |D|, the input is x = [yh_k, yh_k ph_k, yh_k dh_k]
 * (3K values); h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2) with 256 units each, and
 * out = w3 . h2 + b3 predicts the objective normalised over a batch (lower is better).
 * BF16 weights and activations on the tensor cores, FP32 accumulation and FP32 master
 * weights; training is Adam on the mean squared error to (obj - mean) / std.
 * Parameters are one FP32 vector: W1 [256][3K] (row-major), b1 [256], W2 [256][256],
 * b2 [256], w3 [256], b3 [1]. */
typedef struct ffs_surrogate ffs_surrogate;

/* Creates a surrogate for the instance's current genes, with batches of up to `max_batch`
 * chromosomes (training) and weights drawn from `seed`. */
int ffs_surrogate_create(ffs_instance *inst, int32_t max_batch, uint64_t seed, void *stream, ffs_surrogate **out);
int ffs_surrogate_destroy(ffs_surrogate *sur);
int ffs_surrogate_param_count(const ffs_surrogate *sur, int64_t *count);
/* Host copies of the FP32 parameter vector; setting it also resets the Adam state. */
int ffs_surrogate_get_params(ffs_surrogate *sur, float *params);
int ffs_surrogate_set_params(ffs_surrogate *sur, const float *params);
/* Scores `count` device chromosomes y [count][K] into device out [count]. */
int ffs_surrogate_predict(ffs_surrogate *sur, const int16_t *y, int32_t count, float *out);
/* Gradient of the loss on a device batch (y [count][K], exact objectives obj [count],
 * count <= max_batch) into host grad [param count]; host *loss if not NULL.  No update. */
int ffs_surrogate_gradients(ffs_surrogate *sur, const int16_t *y, const int64_t *obj, int32_t count, float *grad,
                            float *loss);
/* One Adam step (betas 0.9 / 0.999, eps 1e-8, learning rate lr) on a device batch; host
 * *loss (before the step) if not NULL. */
int ffs_surrogate_train(ffs_surrogate *sur, const int16_t *y, const int64_t *obj, int32_t count, float lr,
                        float *loss);
/* For verification (not in the paper): copies to host the first `rows` rows of the
 * surrogate's last forward pass over its own batch -- the one made by ffs_surrogate_predict
 * (with count <= max_batch), ffs_surrogate_gradients or ffs_surrogate_train: the stored
 * hidden activations h1, h2 host [rows][256] as BF16 bit patterns, the outputs host [rows]
 * FP32 and, after a gradient or training call, the normalised targets t host [rows] FP32.
 * Any pointer may be NULL.  rows <= the batch rows (FFS_E_ARG beyond); synchronises. */
int ffs_surrogate_read_activations(ffs_surrogate *sur, int32_t rows, uint16_t *h1, uint16_t *h2, float *out,
                                   float *t);

/* Surrogate-assisted generations for a population of the same instance: each generation
 * builds `oversample` candidates per slot with the Sec. 4.4 operators and scores them all.
 * A slot whose first candidate is a parent's plain copy keeps it, as a plain generation
 * would.  Otherwise the slot is screened with probability screen_permille / 1000 (a
 * Philox draw, purpose 6, per slot and generation) and then keeps the best-scored
 * offspring among its candidates (ties to the lower candidate); an unscreened slot keeps
 * its first candidate.  Only the kept children are decoded exactly; the surrogate then
 * takes `train_steps` Adam steps on their exact objectives.  P and P * oversample must be
 * multiples of 128, max_batch >= P, 0 <= screen_permille <= 1000.  NULL detaches. */
int ga_population_attach_surrogate(ga_population *pop, ffs_surrogate *sur, int32_t oversample, float lr,
                                   int32_t train_steps, int32_t screen_permille);

/* Keep rule of surrogate-assisted generations (after ga_population_attach_surrogate):
 *   FFS_KEEP_SLOT    (default) per-slot screening as described above;
 *   FFS_KEEP_ISLAND  each island ranks all oversample x island candidates of its slots by
 *                    the surrogate's score (ties to the lower candidate row, an undefined
 *                    score last) and keeps the best `island` of them, 1/oversample of the
 *                    pool -- with oversample 8 the top 12.5 % -- in candidate-row order,
 *                    one per slot; screen_permille is then unused.  Ranking within each
 *                    island keeps one island's candidates from crowding out another's.
 *   FFS_KEEP_ISLAND_OFFSPRING  as FFS_KEEP_ISLAND, except that a slot whose first candidate
 *                    is a parent's plain copy keeps that copy (the plain GA's copy rate) and
 *                    only offspring (crossover or mutation applied) compete for the island's
 *                    other places.
 * Island rules require oversample x island <= 4096 (FFS_E_ARG otherwise).  With a constant
 * score they keep every slot's first candidate, which is the plain generation's child. */
#define FFS_KEEP_SLOT    0
#define FFS_KEEP_ISLAND  1
#define FFS_KEEP_ISLAND_OFFSPRING  2
int ga_population_surrogate_keep(ga_population *pop, int32_t rule);

/* Diagnostic (not in the paper): with on != 0 the surrogate scores candidates by their exact
 * objectives (every candidate decoded) instead of the network -- a perfect model, to
 * measure what a keep rule itself gives.  Such generations are launched directly rather
 * than replayed from a graph; training still runs as configured. */
int ffs_surrogate_score_exactly(ffs_surrogate *sur, int32_t on);

/* For verification (not in the paper): host copies of the last surrogate-assisted
 * generation's candidates -- Y, X [P * oversample][K] (row f P + j is candidate f of slot
 * j), their scores [P * oversample] -- and, under an island rule, the row kept for each
 * slot, keep [P].  Any pointer may be NULL.  FFS_E_ARG without an attached surrogate or
 * before the first such generation's buffers exist; synchronises. */
int ga_population_read_candidates(ga_population *pop, int16_t *Y, int8_t *X, float *score, int32_t *keep);

/* `steps` Adam steps on the population's current members and their exact objectives (for
 * example generation 0, before surrogate-assisted generations begin); host *loss after
 * the last step's forward pass if not NULL. */
int ffs_surrogate_pretrain(ffs_surrogate *sur, ga_population *pop, int32_t steps, float lr, float *loss);

/* Allocation-free variant of ffs_decode, for callers that cannot allocate device memory:
 * hosts that fix the process's device memory at start-up and hand each library a budget
 * it may not grow, frameworks whose own caching allocator owns the device memory, and
 * real-time loops that must not wait on the allocator (cudaMalloc can block, and
 * cudaFree synchronises the whole device).  The paper has no counterpart; it is a
 * deployment aid.  Arguments and results are those of ffs_decode; the caller still
 * provides the chromosomes and the output arrays.  It allocates nothing: its scratch (error
 * word, instance tables, per-warp power profiles) is one 16 MiB device array inside the
 * library, reserved on every GPU that loads it until the process exits.
 *   - Limits: instance tables up to 1 MiB, and 4 warps' profiles (4 * 2 bytes per slot of
 *     ffs_info.horizon) within the remaining ~15 MiB; beyond them it returns FFS_E_ARG
 *     and ffs_last_error() explains.  ffs_decode has no such limit.
 *   - The first call on each device looks up the array's device address; make that
 *     first call before any stream capture begins.
 *   - Every call shares the one array, which keeps the last call's contents (the error
 *     word is cleared at each call): calls whose work overlaps on the GPU (other streams,
 *     other threads) race and must be serialised by the caller.
 *   - Synchronous: copies the tables from host memory, waits for `stream` to finish and
 *     returns FFS_E_DEVICE if a row was not a permutation of 1..K. */
int ffs_decode_noalloc(ffs_instance *inst, int32_t order_mode, int32_t machine_mode,
                       const int16_t *y, const int8_t *x, int32_t count,
                       int64_t *obj, int64_t *tard, int32_t *cmax, void *stream);

/* Synchronises `stream` and returns FFS_E_DEVICE if a decode since the last check met a
 * malformed chromosome, FFS_OK otherwise (and clears the flag). */
int ffs_decode_check(ffs_instance *inst, void *stream);

/* ---------------------------------------------------------------- GA */

/* Allocates the device-resident population for the instance's current genes and runs
 * generation 0: random X (uniform machine) and Y (Fisher-Yates permutation) drawn from
 * Philox4x32-10, decoding, E_max = 10^a above every initial objective (Sec. 5), fitness
 * (Eq. 13) and the best-ever individual of every island. */
int ga_population_create(ffs_instance *inst, const ga_params *params, ga_population **out);

/* Warm start (an addition to the paper, whose GA restarts from random at every
 * rescheduling point, Sec. 4.1).  Like ga_population_create, except that generation 0 is
 * `prev`'s current population carried over to the instance's present gene set: row r
 * comes from prev's row r mod prev's pop; a gene (job j, stage s) present in both keeps
 * its machine gene and the surviving genes keep their relative priority order, taking
 * priorities n_new+1 .. K; the n_new genes of newly arrived jobs take n_new .. 1 in gene
 * order (gene = free operation, job-major), with machine gene 0.  prev must be a
 * population of the same instance (created before or at its current rescheduling
 * point), not in profiling mode; it is read on prev's stream order and left unchanged.
 * Synchronises the new population's stream. */
int ga_population_create_warm(ffs_instance *inst, const ga_params *params, ga_population *prev,
                              ga_population **out);

/* Device bytes a population of the instance (at its current rescheduling point) with
 * `params` holds: both generation buffers (Y int16 and X int8 per gene, objective and
 * fitness per individual), island bests and migrants, tables, global profile scratch and
 * the best-schedule buffers, each rounded up to 256 bytes. */
int ga_population_footprint(const ffs_instance *inst, const ga_params *params, int64_t *bytes);

/* Frees a population.  NULL is accepted. */
int ga_population_destroy(ga_population *pop);

/* Runs `generations` generations (Sec. 4.4: selection, paired crossover with correction,
 * mutation, decoding, elitist replacement per island, ring migration every
 * migrate_every), continuing the generation counter, so two calls equal one longer call.
 * Writes the best-ever schedule into *best (if not NULL) and commits it to the instance.
 * Synchronises the population's stream. */
int ga_run(ga_population *pop, int32_t generations, ffs_result *best);

/* Copies the population state to host arrays (any may be NULL): Y [P][K], X [P][K],
 * objective and fitness [P], island best-ever bY [P/island][K], bX, bobj, bfit
 * [P/island], E_max and the generation counter. */
int ga_population_read(ga_population *pop, int16_t *Y, int8_t *X, int64_t *obj, int64_t *fit,
                       int16_t *bY, int8_t *bX, int64_t *bobj, int64_t *bfit,
                       int64_t *emax, int32_t *generation);

/* Serialises the full GA state.  With buf == NULL, stores the required size in *len. */
int ga_checkpoint(ga_population *pop, void *buf, size_t *len);

/* Restores a state written by ga_checkpoint for the same instance and parameters.
 * FFS_E_ARG if the buffer does not match or holds a chromosome that is not a permutation
 * of 1..K with machines in range; FFS_E_STATE if the instance was rescheduled since the
 * population was created. */
int ga_restore(ga_population *pop, const void *buf, size_t len);

/* Measurement modes of ga_run.  enable = 0 (default): replays of the captured generation
 * graphs, untimed.  enable = 1: each generation's kernels are launched directly, with a
 * CUDA event pair on the population's stream around the fused
 * selection/crossover/mutation/decode kernel, whose durations are summed.  enable = 2: the
 * same graph replays as mode 0 (chains of 8 generations, each launched as a programmatic
 * dependent of the one before), each replay bracketed by an event pair; the summed
 * durations cover the generations in the launch mode ga_run normally uses.  Results are
 * identical in every mode.  Resets the sums; FFS_E_ARG for other values. */
int ga_set_profiling(ga_population *pop, int32_t enable);

/* Summed duration (milliseconds) and number of generations measured since profiling was
 * enabled (mode 1: of the fused generation kernel's launches; mode 2: of the graph replays). */
int ga_profile_read(ga_population *pop, double *kernel_ms, int64_t *launches);

/* Summed durations (milliseconds) of the phases of surrogate-assisted generations run in
 * profiling mode since it was enabled: ms[0] over-generation of the candidates, ms[1]
 * scoring by the surrogate, ms[2] the keep rule (island ranking; 0 for per-slot screening,
 * which runs inside the next phase), ms[3] selection of the kept children, exact decoding
 * and replacement, ms[4] training. */
int ga_profile_read_phases(ga_population *pop, double *ms);

/* The surrogate's dense contraction, exposed for verification (not in the paper):
 * C = A . B^T with A [M][K] and B [N][K] row-major BF16 device matrices, accumulated in
 * FP32 on the tcgen05 tensor cores.  relu_bf16 = 0: C is [M][N] FP32; relu_bf16 = 1:
 * C = relu(A . B^T + bias) rounded to BF16, bias [N] FP32.  M and N multiples of 128, K a
 * multiple of 64, pointers 16-byte aligned, else FFS_E_ARG.  Asynchronous on `stream`;
 * FFS_E_TIMEOUT (at the next synchronising call of the surrogate, or here when
 * synchronous = 1) if a bounded wait inside the kernel ran out. */
int ffs_tensor_gemm(const void *A, const void *B, int32_t M, int32_t N, int32_t K, const float *bias, void *C,
                    int32_t relu_bf16, int32_t synchronous, void *stream);

/* ---------------------------------------------------------------- rescheduling service
 *
 * Continuous batching of rescheduling requests on one GPU (an addition to the paper,
 * which solves one rescheduling point at a time, Sec. 4.1).  A request names an instance,
 * the jobs that arrived and the rescheduling point t_now: the service applies
 * ffs_reschedule (Alg. 1 freeze, new jobs appended), runs `generations` generations of
 * the GA and commits the best schedule to the instance, exactly as ffs_reschedule +
 * ga_population_create(_warm) + ga_run would.  A worker thread owned by the service
 *   - admits queued requests first come first served while fewer than max_active are on
 *     the device and the request's population (ga_population_footprint) fits in the
 *     service's memory; a request whose instance already has one queued ahead or running
 *     waits for it, and later requests of other instances may pass it;
 *   - gives each admitted request its own stream, so the generations of all active
 *     requests overlap on the GPU; finished requests are retired as their streams drain,
 *     and their slots and memory go to the next requests;
 *   - keeps each instance's last population on the device and starts the instance's next
 *     request from it (ga_population_create_warm); a kept population holds only its
 *     chromosomes (2 x P x K x 3 bytes) and its generation counter.  Kept populations are
 *     dropped, least recently used first, when an admission needs their memory, and the
 *     request then starts cold (ffs_request_info.warm = 0).
 * Every request of an instance draws from Philox stream id ga.instance_id + (the number
 * of the instance's earlier requests in this service), so its result depends only on the
 * instance, the request and whether it started warm: not on the other requests, their
 * timing or max_active.
 * The caller must not use an instance (nor destroy it) between submitting a request for
 * it and that request's completion; ffs_service_forget releases an idle instance. */
typedef struct ffs_service ffs_service;

typedef struct {
    int32_t max_active;       /* requests on the device at once, >= 1                      */
    int32_t pad;
    int64_t memory_bytes;     /* device memory for populations, reserved at creation, > 0 */
    ga_params ga;             /* GA settings of every request; cuda_stream and
                                 instance_id are taken as described above            */
} ffs_service_config;

#define FFS_REQ_QUEUED  0
#define FFS_REQ_ACTIVE  1
#define FFS_REQ_DONE    2
#define FFS_REQ_FAILED  3

typedef struct {
    int32_t state;            /* FFS_REQ_*                                                */
    int32_t status;           /* FFS_OK, or the failed request's error code             */
    int32_t warm;             /* 1 if generation 0 came from the instance's last population */
    int32_t generations;      /* generations run: as requested, fewer if it was stopped     */
    int64_t submit_ns, admit_ns, done_ns;  /* steady-clock times (ns) of the three events  */
    int64_t footprint;        /* device bytes of the request's population                */
    int32_t n_ops;            /* N * g of the instance after this request's arrivals      */
    int32_t pad;
} ffs_request_info;

typedef struct {
    int32_t active, queued, warm;   /* requests on the device, waiting; kept populations   */
    int32_t pad;
    int64_t completed, failed;
    int64_t memory_bytes, used_bytes, peak_bytes;  /* arena size, in use now, high-water mark */
} ffs_service_stats;

/* Reserves cfg->memory_bytes of device memory on the current device, creates
 * cfg->max_active streams and starts the worker thread.  FFS_E_ARG for invalid settings
 * (as ga_population_create), FFS_E_NOMEM if the reservation fails. */
int ffs_service_create(const ffs_service_config *cfg, ffs_service **out);

/* Stops admitting, waits for the active requests, fails the queued ones (FFS_E_STATE),
 * stops the worker and frees every population, stream and the reserved memory.  NULL is
 * accepted.  Results of finished requests are lost. */
int ffs_service_destroy(ffs_service *svc);

/* Queues a request; copies `arrivals` (may be NULL: no new jobs).  The arguments are
 * checked when the request is admitted (ffs_reschedule's rules), and a request that fails
 * there finishes in state FFS_REQ_FAILED.  generations >= 0.  *ticket identifies it. */
int ffs_service_submit(ffs_service *svc, ffs_instance *inst, const ffs_arrivals *arrivals, int32_t t_now,
                       int32_t generations, int64_t *ticket);

/* Waits up to timeout_ms (0: just look; < 0: no limit) for a request to finish and fills
 * *info (if not NULL).  When it has finished, fills *best like ga_run: best->start and
 * best->machine (if not NULL) must hold info->n_ops entries.  Returns FFS_OK once the
 * request is done, the request's error code if it failed (ffs_last_error() then gives
 * the worker's CUDA error text, if any), FFS_E_TIMEOUT if it is still queued or active,
 * FFS_E_ARG for an unknown ticket. */
int ffs_service_wait(ffs_service *svc, int64_t ticket, int32_t timeout_ms, ffs_request_info *info,
                     ffs_result *best);

/* Ends a request early, for a caller whose request has gone stale (a newer event for the
 * instance) or who needs an answer now; the paper has no counterpart.  The worker enqueues
 * an admitted request's generations 64 at a time, and checks for a stop between chunks:
 *   - an admitted request ends after the chunk in flight and finishes FFS_REQ_DONE with
 *     the best schedule found so far (committed to its instance, and its population kept
 *     for the instance's next request, as for a full run); info.generations then says how
 *     many generations ran, and the result equals a request for exactly that many;
 *   - a queued request whose rescheduling has not yet been applied is dropped without
 *     touching its instance and finishes FFS_REQ_FAILED with status FFS_E_STOPPED (it
 *     does not count as one of the instance's requests for stream ids);
 *   - a queued request whose rescheduling was already applied (it waited for memory) is
 *     admitted and ends after generation 0.
 * Results of a stopped request depend on when the stop arrived.  FFS_OK for a finished
 * request (no effect), FFS_E_ARG for an unknown ticket. */
int ffs_service_stop_request(ffs_service *svc, int64_t ticket);

/* Drops the instance's kept population and its request count.  FFS_E_STATE while a
 * request of the instance is queued or active. */
int ffs_service_forget(ffs_service *svc, ffs_instance *inst);

int ffs_service_stats_read(ffs_service *svc, ffs_service_stats *stats);

/* Bounds-checked builds, for tests (the paper has no counterpart; compute-sanitizer is not
 * available where the library is tested).  A library built with FFS_CHECKED checks the
 * device indices of the decoder's shared-memory profile windows, schedule records and job
 * completion times, its stage-order list, and the crossover's bitmap and missing-value
 * list: an index outside its buffer is counted and replaced by 0, so nothing is accessed
 * out of range and control flow does not change.  *count = the indices found out of range
 * since the last call (the count is then cleared).  An ordinary build checks nothing: it
 * sets *count = 0 and returns FFS_E_STATE. */
int ffs_debug_bounds_faults(uint32_t *count);

/* Failure injection, for tests of the library's bounded device waits (not in the paper;
 * not for production use).  Process-wide; mode is an or of:
 *   FFS_INJECT_TABLE_COPY  every later ffs_decode launch skips the copy of the instance
 *                          tables into shared memory, so each CTA's bounded wait for them
 *                          runs out (a short limit: no copy is in flight), the CTA records
 *                          a timeout and returns, and ffs_decode_check reports
 *                          FFS_E_TIMEOUT;
 *   FFS_INJECT_GEMM_LOADS  every later ffs_tensor_gemm launch issues no operand loads, so
 *                          the tensor-core issuer's bounded wait runs out (short limit, no
 *                          copy in flight), the CTA frees its tensor memory and the call
 *                          reports FFS_E_TIMEOUT.
 * FFS_INJECT_NONE restores normal operation.  FFS_E_ARG for unknown bits. */
#define FFS_INJECT_NONE        0
#define FFS_INJECT_TABLE_COPY  1
#define FFS_INJECT_GEMM_LOADS  2
int ffs_debug_inject(int32_t mode);

/* Number of kernels this library has launched in the process so far (graph replays count
 * each kernel node).  For benchmark accounting. */
int ffs_kernel_launches(uint64_t *count);

/* Text of the last CUDA error this thread's calls met (empty if none).  The pointer stays
 * valid until the thread's next library call. */
const char *ffs_last_error(void);

/* Human-readable name of a status code. */
const char *ffs_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* FFS_H */
