/*
 * ffs_oracle.c -- CPU oracle for the EDFFS decoder and the priority-based hybrid GA of
 * Luo, Fujimura & El Baz, "GPU based Parallel Genetic Algorithm for Solving an Energy
 * Efficient Dynamic Flexible Flow Shop Scheduling Problem" (arXiv 1903.10741).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, single-threaded, deliberately slow
 * statement of what the library computes.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load it.  It shares no code, header, table or constant
 * generator with the CUDA library, and the library never calls it.
 *
 * Everything is int32/int64: times, powers, objective.  Parity pins (tests/):
 *   - Philox4x32-10 known-answer vectors (Salmon et al., SC'11).
 *   - Worked example of Sec. 4.3 (Table 4, X/Y/Z matrices, delay narrative, Fig. 8 C_max).
 *   - Schedule invariants Eq. (4)-(10) checked on a literal per-instant Q_t array.
 *   - Greedy-earliest property of every placement, checked by brute force.
 *   - Closed forms: single machine (sum of p), power never binding (list scheduling).
 *   - Brute force over all priority orders on tiny instances.
 *   - Fig. 11 crossover/correction and Fig. 12 mutation examples.
 *   - Table 11 objective arithmetic (Eq. 1).
 *   - Hand-worked selection (tournament ties, the 5-cell torus), elitist replacement and
 *     ring migration cases, the operator order of a generation, and the Z order of both
 *     readings of Alg. 1 on the Sec. 4.3 example, position by position.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- constants */

enum { ST_FREE = 0, ST_EXEC = 1, ST_DONE = 2, ST_FIXED = 3 };  /* Alg. 1 classification; FIXED: static approach */
enum { ORDER_TOPO = 0, ORDER_STAGE = 1, ORDER_GIVEN = 2 };  /* how Z is built         */
enum { MACH_GENE = 0, MACH_EARLIEST = 1 };                  /* how M_js is chosen     */
enum { PLACE_INSERT = 4 };  /* flag on the machine mode: back-fill machine idle gaps */
enum { P_INIT_Y = 1, P_INIT_X = 2, P_SELECT = 3, P_CROSS = 4, P_MUTATE = 5 };

/* ---------------------------------------------------------------- Philox4x32-10 */
/* Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11:
 * ten rounds of  (c0,c1,c2,c3) -> (hi(M1*c2)^c1^k0, lo(M1*c2), hi(M0*c0)^c3^k1, lo(M0*c0))
 * with M0 = 0xD2511F53, M1 = 0xCD9E8D57; the key is bumped by the Weyl constants
 * (0x9E3779B9, 0xBB67AE85) before every round but the first. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* One 32-bit draw of the library's stream: counter = (d/4, slot, generation,
 * purpose<<24 | instance), key = seed, word d%4. */
uint32_t orc_draw(uint64_t seed, uint32_t purpose, uint32_t instance, uint32_t gen,
                  uint32_t slot, uint32_t d)
{
    uint32_t ctr[4] = { d >> 2, slot, gen, (purpose << 24) | (instance & 0xFFFFFFu) };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[d & 3u];
}

/* Integer in [0, n) from a 32-bit draw: floor(u * n / 2^32). */
static uint32_t below(uint32_t u, uint32_t n)
{
    return (uint32_t)(((uint64_t)u * (uint64_t)n) >> 32);
}

/* Bernoulli(num/den): u < floor(num * 2^32 / den). */
static int chance(uint32_t u, int32_t num, int32_t den)
{
    uint64_t thr = ((uint64_t)(uint32_t)num << 32) / (uint64_t)(uint32_t)den;
    return (uint64_t)u < thr;
}

/* ---------------------------------------------------------------- instance */

/* An instance at a rescheduling point RS.  Ops (j, s) index j*g+s.  For frozen ops
 * (status EXEC or DONE) S0/M0 hold the start and stage-local machine of the plan being
 * executed; free ops are the genes, numbered job-major then stage (row-major over the
 * (n+n') x g matrices of Eq. (10)-(11) with the -1 cells removed). */
typedef struct {
    int32_t N, g, Qmax, WT, RS;
    const int32_t *o;       /* [g]      machines per stage                        */
    const int32_t *p;       /* [N*g]    processing time (identical machines)      */
    const int32_t *q;       /* [sum o]  power of each machine, stage-major        */
    const int32_t *R, *D;   /* [N]      release and due times                     */
    const int32_t *status;  /* [N*g]    ST_FREE / ST_EXEC / ST_DONE / ST_FIXED    */
    const int32_t *S0;      /* [N*g]    committed start of frozen ops             */
    const int32_t *M0;      /* [N*g]    committed stage-local machine of frozen ops */
    const int32_t *pm;      /* [N][sum o] P_jsm on every machine (unrelated machines), or NULL */
    const int32_t *qm;      /* [N][sum o] Q_jsm on every machine, or NULL               */
} orc_inst;

/* Processing time and power of job j's op at stage s on global machine mg (Table 2:
 * P_jsm and Q_jsm); without the per-machine tables, p of the op and q of the machine. */
static int32_t op_p(const orc_inst *in, int32_t j, int32_t s, int32_t mg, int32_t Mtot)
{
    return in->pm ? in->pm[(size_t)j * Mtot + mg] : in->p[j * in->g + s];
}

static int32_t op_q(const orc_inst *in, int32_t j, int32_t mg, int32_t Mtot)
{
    return in->qm ? in->qm[(size_t)j * Mtot + mg] : in->q[mg];
}

typedef struct {
    int64_t obj;      /* WT * sum T_j + C_max, Eq. (1)                 */
    int64_t tard;     /* sum_j T_j, Eq. (2)                            */
    int32_t cmax;     /* Eq. (3)                                       */
    int32_t err;      /* 0 ok, <0 invalid input                        */
    int64_t probes;   /* time slots examined by the Eq. (7) checks     */
    int64_t span;     /* sum over ops of (start - t0 + p) on the chosen machine */
    int64_t slots;    /* algorithmic work: for every op, sum over the machines tried of
                         (earliest feasible start - earliest availability + p), plus p for
                         the profile update: the instants an exact Eq. (7) check must read */
} orc_eval;

/* Alg. 1, first branch: classify every op of the executed plan at RS.
 * S + P <= RS: completed; S < RS < S + P: being executed; S >= RS: free. */
void orc_classify(int32_t N, int32_t g, const int32_t *p, const int32_t *S, int32_t RS,
                  int32_t *status_out)
{
    for (int32_t j = 0; j < N; j++) {
        for (int32_t s = 0; s < g; s++) {
            int32_t k = j * g + s;
            int32_t st = S[k], en = S[k] + p[k];
            if (en <= RS)
                status_out[k] = ST_DONE;
            else if (st < RS)
                status_out[k] = ST_EXEC;
            else
                status_out[k] = ST_FREE;
        }
    }
}

/* The traditional static approach (Sec. 4.1, Fig. 7; Sec. 5.3): the executed plan is kept.
 * S + P <= RS: completed; S < RS < S + P: being executed; S >= RS: fixed, i.e. it keeps its
 * planned start and machine and draws power over [S, S + P).  Only new jobs are free. */
void orc_classify_static(int32_t N, int32_t g, const int32_t *p, const int32_t *S, int32_t RS,
                         int32_t *status_out)
{
    orc_classify(N, g, p, S, RS, status_out);
    for (int32_t k = 0; k < N * g; k++)
        if (status_out[k] == ST_FREE)
            status_out[k] = ST_FIXED;
}

/* Number of free ops (genes) K = g(n+n') - r, Sec. 4.3. */
int32_t orc_gene_count(const orc_inst *in)
{
    int32_t K = 0;
    for (int32_t k = 0; k < in->N * in->g; k++)
        K += (in->status[k] == ST_FREE);
    return K;
}

/* gene -> (job, stage), row-major over the job x stage matrix. */
void orc_gene_map(const orc_inst *in, int32_t *gene_job, int32_t *gene_stage)
{
    int32_t K = 0;
    for (int32_t j = 0; j < in->N; j++)
        for (int32_t s = 0; s < in->g; s++)
            if (in->status[j * in->g + s] == ST_FREE) {
                gene_job[K] = j;
                gene_stage[K] = s;
                K++;
            }
}

static int32_t max32(int32_t a, int32_t b) { return a > b ? a : b; }

/* ---------------------------------------------------------------- decoder */

/* Z, the assignment order of the K free ops (Alg. 1), into order[0..K):
 *   ORDER_TOPO  -- repeatedly the next unassigned free op of some job: among those heads,
 *                  the one with the largest y (y values are distinct).
 *   ORDER_STAGE -- stage s = 0..g-1 in turn, each stage's free ops by y descending.
 *   ORDER_GIVEN -- `given` as it is.
 * gene_at[j*g+s] is the gene of op (j, s), or -1 for a frozen op. */
static void fill_order(int32_t N, int32_t g, int32_t K, const int32_t *gstg, const int32_t *gene_at,
                       int32_t order_mode, const int16_t *y, const int32_t *given, int32_t *order)
{
    if (order_mode == ORDER_TOPO) {
        int32_t *head = (int32_t *)calloc((size_t)N + 1, sizeof(int32_t)); /* next stage of j */
        for (int32_t j = 0; j < N; j++) {
            head[j] = 0;
            while (head[j] < g && gene_at[j * g + head[j]] < 0) head[j]++;
        }
        for (int32_t n = 0; n < K; n++) {
            int32_t bestj = -1, besty = -1;
            for (int32_t j = 0; j < N; j++) {
                if (head[j] >= g) continue;
                int32_t k = gene_at[j * g + head[j]];
                if (y[k] > besty) { besty = y[k]; bestj = j; }
            }
            order[n] = gene_at[bestj * g + head[bestj]];
            head[bestj]++;
        }
        free(head);
    } else if (order_mode == ORDER_STAGE) {
        int32_t n = 0;
        for (int32_t s = 0; s < g; s++) {
            int32_t first = n;
            for (int32_t k = 0; k < K; k++)
                if (gstg[k] == s) order[n++] = k;
            /* insertion sort of this stage's genes by y, descending */
            for (int32_t a = first + 1; a < n; a++) {
                int32_t v = order[a], b = a - 1;
                while (b >= first && y[order[b]] < y[v]) { order[b + 1] = order[b]; b--; }
                order[b + 1] = v;
            }
        }
    } else {
        for (int32_t n = 0; n < K; n++) order[n] = given[n];
    }
}

/*
 * Decode one chromosome (Sec. 4.3, Alg. 1 and Alg. 2) into a schedule and its objective.
 *
 * Order of assignment (matrix Z):
 *   ORDER_TOPO  -- Alg. 1 read as a topological order: repeatedly take, among the next
 *                  unassigned free op of every job, the one with the largest y.
 *   ORDER_STAGE -- stage by stage (s = 0..g-1), the free ops of each stage by y descending.
 *   ORDER_GIVEN -- the gene order passed in `given` (used for the printed Z of Sec. 4.3).
 * Machine:
 *   MACH_GENE     -- M_js = x_js (Eq. 10).
 *   MACH_EARLIEST -- the machine of the stage with the earliest power-feasible start,
 *                    ties to the lowest machine index.
 * Placement (Alg. 2): an op becomes available at est = max(RS, R_j, C_{j,s-1}); on
 * machine m it cannot start before the end of the op last assigned to m (ops are
 * appended to machines in assignment order).  It starts at the smallest integer t from
 * there on such that, for every instant tau in [t, t+p), the power already drawn Q_tau
 * (Eq. 8-9) plus its own power stays within Qmax (Eq. 7).  Otherwise it is delayed.
 * With PLACE_INSERT or-ed into the machine mode (an option, not the paper's Alg. 2), an
 * op may instead fill an idle gap: on machine m it starts at the smallest integer
 * t >= max(est, end of m's frozen ops) such that m is idle at every instant of [t, t+p)
 * (no op assigned before it overlaps) and the power check holds.
 *
 * The power profile is a literal per-instant array Q_tau over [RS, RS+H), with H an upper
 * bound on the makespan (all free ops run back to back after the latest release or
 * executing end).
 */
int32_t orc_decode(const orc_inst *in, int32_t order_mode, int32_t mach_mode,
                   const int16_t *y, const int8_t *x, const int32_t *given,
                   int32_t *S_out, int32_t *M_out, orc_eval *ev)
{
    const int32_t N = in->N, g = in->g, RS = in->RS, Qmax = in->Qmax;
    const int insert = (mach_mode & PLACE_INSERT) != 0;
    mach_mode &= 1;
    memset(ev, 0, sizeof(*ev));

    int32_t *moff = (int32_t *)calloc((size_t)g + 1, sizeof(int32_t));
    for (int32_t s = 0; s < g; s++)
        moff[s + 1] = moff[s] + in->o[s];
    const int32_t Mtot = moff[g];

    const int32_t K = orc_gene_count(in);
    int32_t *gjob = (int32_t *)calloc((size_t)K + 1, sizeof(int32_t));
    int32_t *gstg = (int32_t *)calloc((size_t)K + 1, sizeof(int32_t));
    orc_gene_map(in, gjob, gstg);

    /* validate the chromosome: Y a permutation of 1..K; X machines in range */
    int32_t *seen = (int32_t *)calloc((size_t)K + 2, sizeof(int32_t));
    for (int32_t k = 0; k < K; k++) {
        int32_t v = y[k];
        if (v < 1 || v > K || seen[v]) {
            ev->err = -1;
            break;
        }
        seen[v] = 1;
        if ((mach_mode & 1) == MACH_GENE && (x[k] < 0 || x[k] >= in->o[gstg[k]])) {
            ev->err = -2;
            break;
        }
    }
    free(seen);
    if (ev->err) {
        free(moff); free(gjob); free(gstg);
        return ev->err;
    }

    /* horizon bound and per-instant power array */
    int64_t base = RS, work = 0;
    for (int32_t j = 0; j < N; j++) {
        if (in->R[j] > base) base = in->R[j];
        for (int32_t s = 0; s < g; s++) {
            int32_t k = j * g + s;
            if (in->status[k] == ST_EXEC || in->status[k] == ST_FIXED) {
                int32_t e = in->S0[k] + op_p(in, j, s, moff[s] + in->M0[k], Mtot);
                if (e > base) base = e;
            }
            if (in->status[k] == ST_FREE) {  /* the longest of its machines */
                int32_t pmax = 0;
                for (int32_t m = 0; m < in->o[s]; m++) {
                    int32_t v = op_p(in, j, s, moff[s] + m, Mtot);
                    if (v > pmax) pmax = v;
                }
                work += pmax;
            }
        }
    }
    const int64_t H = base - RS + work + 1;
    int32_t *Qt = (int32_t *)calloc((size_t)H, sizeof(int32_t));     /* Q_tau - at RS+i */
    int32_t *mfree = (int32_t *)calloc((size_t)Mtot, sizeof(int32_t)); /* end of last op on m */
    int32_t *C = (int32_t *)calloc((size_t)N + 1, sizeof(int32_t));   /* C_{j, last placed} */
    /* insertion: instants at which each machine runs an op placed by this decode */
    uint8_t *busy = insert ? (uint8_t *)calloc((size_t)Mtot * (size_t)H, 1) : NULL;

    for (int32_t m = 0; m < Mtot; m++)
        mfree[m] = RS;
    for (int32_t j = 0; j < N; j++) {
        C[j] = 0;
        for (int32_t s = 0; s < g; s++) {
            int32_t k = j * g + s;
            if (in->status[k] == ST_FREE)
                continue;
            int32_t end = in->S0[k] + op_p(in, j, s, moff[s] + in->M0[k], Mtot);
            C[j] = end;                                   /* frozen ops are a prefix */
            S_out[k] = in->S0[k];
            M_out[k] = in->M0[k];
            if (in->status[k] == ST_EXEC || in->status[k] == ST_FIXED) {  /* draws power past RS */
                int32_t mg = moff[s] + in->M0[k];
                if (end > mfree[mg]) mfree[mg] = end;
                int32_t from = in->S0[k] > RS ? in->S0[k] : RS;
                int32_t qv = op_q(in, j, mg, Mtot);
                for (int32_t t = from; t < end; t++)
                    Qt[t - RS] += qv;
            }
        }
    }

    /* ---- Z: the assignment order of the free ops */
    int32_t *order = (int32_t *)calloc((size_t)K + 1, sizeof(int32_t));
    int32_t *gene_at = (int32_t *)malloc(sizeof(int32_t) * (size_t)N * (size_t)g);
    for (int32_t i = 0; i < N * g; i++) gene_at[i] = -1;
    for (int32_t k = 0; k < K; k++) gene_at[gjob[k] * g + gstg[k]] = k;
    fill_order(N, g, K, gstg, gene_at, order_mode, y, given, order);

    /* ---- Alg. 2: assign in Z order */
    int32_t *placed = (int32_t *)calloc((size_t)K + 1, sizeof(int32_t));
    for (int32_t n = 0; n < K && !ev->err; n++) {
        int32_t k = order[n];
        if (k < 0 || k >= K || placed[k]) { ev->err = -3; break; }
        int32_t j = gjob[k], s = gstg[k];
        if (s > 0 && in->status[j * g + s - 1] == ST_FREE && !placed[gene_at[j * g + s - 1]]) {
            ev->err = -4;                                /* order breaks stage precedence */
            break;
        }
        int32_t est = max32(RS, max32(in->R[j], C[j]));
        int32_t mlo = 0, mhi = in->o[s];
        if (mach_mode == MACH_GENE) { mlo = x[k]; mhi = x[k] + 1; }

        /* the machine with the earliest completion (with identical machines: the earliest
         * start), ties to the lowest machine */
        int32_t best_t = -1, best_m = -1, best_t0 = 0, best_p = 0;
        for (int32_t m = mlo; m < mhi; m++) {
            int32_t mg = moff[s] + m, qm = op_q(in, j, mg, Mtot), pj = op_p(in, j, s, mg, Mtot);
            int32_t t0 = max32(est, mfree[mg]);
            int32_t t = t0;
            for (;;) {
                /* last instant of [t, t+p) at which adding qm would exceed Qmax */
                int32_t bad = -1;
                for (int32_t tau = t; tau < t + pj; tau++) {
                    ev->probes++;
                    if (Qt[tau - RS] + qm > Qmax) bad = tau;
                    if (insert && busy[(size_t)mg * H + (tau - RS)]) bad = tau;
                }
                if (bad < 0) break;
                t = bad + 1;                             /* delayed past the violation */
            }
            ev->slots += (int64_t)(t - t0) + pj;
            if (best_m < 0 || t + pj < best_t + best_p) { best_t = t; best_m = m; best_t0 = t0; best_p = pj; }
        }
        int32_t mg = moff[s] + best_m, pj = best_p, qb = op_q(in, j, mg, Mtot);
        for (int32_t tau = best_t; tau < best_t + pj; tau++)
            Qt[tau - RS] += qb;
        if (insert) {
            for (int32_t tau = best_t; tau < best_t + pj; tau++) busy[(size_t)mg * H + (tau - RS)] = 1;
        } else {
            mfree[mg] = best_t + pj;
        }
        C[j] = best_t + pj;
        S_out[j * g + s] = best_t;
        M_out[j * g + s] = best_m;
        ev->span += (int64_t)(best_t - best_t0) + pj;
        ev->slots += pj;
        placed[k] = 1;
    }

    if (!ev->err) {
        /* Eq. (1)-(3): tardiness and makespan over all jobs J u J' */
        int64_t tard = 0;
        int32_t cmax = 0;
        for (int32_t j = 0; j < N; j++) {
            int32_t cj = C[j];
            if (cj - in->D[j] > 0) tard += cj - in->D[j];
            if (cj > cmax) cmax = cj;
        }
        ev->tard = tard;
        ev->cmax = cmax;
        ev->obj = (int64_t)in->WT * tard + cmax;
    }

    free(placed); free(order); free(gene_at); free(Qt); free(mfree); free(C); free(busy);
    free(moff); free(gjob); free(gstg);
    return ev->err;
}

/* The assignment order Z that orc_decode uses for chromosome y (Alg. 1): order_out[n] is
 * the gene placed n-th.  y must be a permutation of 1..K (not checked here). */
void orc_order(const orc_inst *in, int32_t order_mode, const int16_t *y, const int32_t *given,
               int32_t *order_out)
{
    const int32_t N = in->N, g = in->g, K = orc_gene_count(in);
    int32_t *gjob = (int32_t *)calloc((size_t)K + 1, sizeof(int32_t));
    int32_t *gstg = (int32_t *)calloc((size_t)K + 1, sizeof(int32_t));
    orc_gene_map(in, gjob, gstg);
    int32_t *gene_at = (int32_t *)malloc(sizeof(int32_t) * (size_t)N * (size_t)g);
    for (int32_t i = 0; i < N * g; i++) gene_at[i] = -1;
    for (int32_t k = 0; k < K; k++) gene_at[gjob[k] * g + gstg[k]] = k;
    fill_order(N, g, K, gstg, gene_at, order_mode, y, given, order_out);
    free(gene_at); free(gjob); free(gstg);
}

/* Objective of Eq. (1) from per-job completion times (Table 11 arithmetic). */
int64_t orc_objective(int32_t N, const int32_t *Cj, const int32_t *D, int32_t WT,
                      int64_t *tard_out, int32_t *cmax_out)
{
    int64_t tard = 0;
    int32_t cmax = 0;
    for (int32_t j = 0; j < N; j++) {
        if (Cj[j] - D[j] > 0) tard += Cj[j] - D[j];
        if (Cj[j] > cmax) cmax = Cj[j];
    }
    *tard_out = tard;
    *cmax_out = cmax;
    return (int64_t)WT * tard + cmax;
}

/* ---------------------------------------------------------------- GA operators */

/* Correction after crossover (Sec. 4.4, Fig. 11): scanning the genes in row-major order,
 * the first occurrence of a value stays; each later duplicate, in scan order, takes the
 * next missing value of 1..K in ascending order. */
void orc_correct(int32_t K, int16_t *y)
{
    int32_t *seen = (int32_t *)calloc((size_t)K + 2, sizeof(int32_t));
    int32_t *dup = (int32_t *)calloc((size_t)K + 1, sizeof(int32_t));
    int32_t nd = 0;
    for (int32_t k = 0; k < K; k++) {
        if (seen[y[k]]) dup[nd++] = k;
        else seen[y[k]] = 1;
    }
    int32_t next = 0;
    for (int32_t v = 1; v <= K && next < nd; v++)
        if (!seen[v]) y[dup[next++]] = (int16_t)v;
    free(seen);
    free(dup);
}

/* Neighbouring paired single-point crossover (Sec. 4.4, Fig. 10-11) with explicit cuts:
 * the first cy genes of Y (cx of X) come from one parent, the rest from the other;
 * child0 = head(a) + tail(b), child1 = head(b) + tail(a); then Y is corrected. */
void orc_crossover(int32_t K, const int16_t *ya, const int8_t *xa, const int16_t *yb,
                   const int8_t *xb, int32_t cx, int32_t cy, int16_t *y0, int8_t *x0,
                   int16_t *y1, int8_t *x1)
{
    for (int32_t k = 0; k < K; k++) {
        y0[k] = k < cy ? ya[k] : yb[k];
        y1[k] = k < cy ? yb[k] : ya[k];
        if (xa && xb) {
            x0[k] = k < cx ? xa[k] : xb[k];
            x1[k] = k < cx ? xb[k] : xa[k];
        }
    }
    orc_correct(K, y0);
    orc_correct(K, y1);
}

/* Mutation (Sec. 4.4, Fig. 12) with explicit draws: every x moves to another machine of
 * its stage (r in [0, o-1) skips the current one), and y[a] <-> y[b] with a != b. */
void orc_mutate(int32_t K, const int32_t *gene_o, int16_t *y, int8_t *x,
                const uint32_t *xr, int32_t a, int32_t b)
{
    if (x) {
        for (int32_t k = 0; k < K; k++) {
            if (gene_o[k] < 2) continue;
            int32_t r = (int32_t)xr[k];
            x[k] = (int8_t)(r + (r >= x[k]));
        }
    }
    if (K >= 2) {
        int16_t t = y[a];
        y[a] = y[b];
        y[b] = t;
    }
}

/* ---------------------------------------------------------------- GA */

typedef struct {
    int32_t P;               /* population size                                    */
    int32_t I;               /* island size (even, divides P)                      */
    int32_t tour_k;          /* tournament size; 0 = local 5-neighbourhood on a torus */
    int32_t pc_num, pc_den;  /* crossover probability                              */
    int32_t pm_num, pm_den;  /* mutation probability                               */
    int32_t order_mode, mach_mode;
    int32_t migrate_every;   /* ring migration period in generations (0 = none)    */
    int32_t instance_id;     /* 24-bit stream id                                   */
    int32_t pad;
    uint64_t seed;
} orc_ga_params;

typedef struct {
    int16_t *Y;    int8_t *X;     /* [P*K] current population                 */
    int64_t *obj;  int64_t *fit;  /* [P]                                      */
    int16_t *bY;   int8_t *bX;    /* [n_isl*K] best-ever individual per island */
    int64_t *bobj; int64_t *bfit; /* [n_isl]                                  */
    int64_t emax;
    int32_t gen;
    int32_t K;
} orc_ga_state;

static int32_t decode_one(const orc_inst *in, const orc_ga_params *par, const int16_t *y,
                          const int8_t *x, int64_t *obj)
{
    int32_t NG = in->N * in->g;
    int32_t *S = (int32_t *)calloc((size_t)NG, sizeof(int32_t));
    int32_t *M = (int32_t *)calloc((size_t)NG, sizeof(int32_t));
    orc_eval ev;
    int32_t rc = orc_decode(in, par->order_mode, par->mach_mode, y, x, NULL, S, M, &ev);
    *obj = ev.obj;
    free(S);
    free(M);
    return rc;
}

/* Fitness, Eq. (13): max(E_max - objective, 0). */
static int64_t fitness(int64_t emax, int64_t obj)
{
    return emax - obj > 0 ? emax - obj : 0;
}

/* Best (largest fitness) and worst (smallest fitness) of fit[lo..hi), each the lowest
 * index among equals. */
void orc_island_best_worst(const int64_t *fit, int32_t lo, int32_t hi, int32_t *best, int32_t *worst)
{
    int32_t b = lo, w = lo;
    for (int32_t i = lo + 1; i < hi; i++) {
        if (fit[i] > fit[b]) b = i;
        if (fit[i] < fit[w]) w = i;
    }
    *best = b;
    *worst = w;
}

/* Winner among the n entrants cand[0..n) (population indices, repeats allowed): the
 * largest fitness, ties to the lowest index (Sec. 4.4 selection). */
int32_t orc_tournament(const int64_t *fit, const int32_t *cand, int32_t n)
{
    int32_t best = -1;
    for (int32_t t = 0; t < n; t++) {
        int32_t c = cand[t];
        if (best < 0 || fit[c] > fit[best] || (fit[c] == fit[best] && c < best))
            best = c;
    }
    return best;
}

/* The 5-cell neighbourhood of cell i on the side x side torus of the population grid
 * (Sec. 4.4, Fig. 9: the cell, then N, S, W, E), side * side = P, cells row-major. */
void orc_l5_cells(int32_t P, int32_t i, int32_t out[5])
{
    int32_t side = 1;
    while (side * side < P) side++;
    int32_t r = i / side, c = i % side;
    out[0] = i;
    out[1] = ((r + side - 1) % side) * side + c;
    out[2] = ((r + 1) % side) * side + c;
    out[3] = r * side + (c + side - 1) % side;
    out[4] = r * side + (c + 1) % side;
}

/* Parent drawn with the selection stream of row `v` from the island (or torus
 * neighbourhood) of population slot `home`: with tour_k > 0 the winner of k entrants drawn
 * uniformly from the island (entrant t = island start + floor(u_t * I / 2^32), u_t = draw t
 * of row v's selection stream); with tour_k = 0 the winner of the 5-cell neighbourhood. */
static int32_t select_parent(const int64_t *fit, int32_t P, int32_t I, int32_t tour_k, uint64_t seed,
                             int32_t iid, int32_t gen, int32_t v, int32_t home)
{
    int32_t cand[64];
    int32_t n;
    if (tour_k > 0) {
        int32_t lo = (home / I) * I;
        n = tour_k < 64 ? tour_k : 64;
        for (int32_t t = 0; t < n; t++)
            cand[t] = lo + (int32_t)below(orc_draw(seed, P_SELECT, (uint32_t)iid, (uint32_t)gen, (uint32_t)v,
                                                   (uint32_t)t), (uint32_t)I);
    } else {
        orc_l5_cells(P, home, cand);
        n = 5;
    }
    return orc_tournament(fit, cand, n);
}

/* Parent of population slot i at generation gen (Sec. 4.4 selection). */
int32_t orc_select(const int64_t *fit, int32_t P, int32_t I, int32_t tour_k, uint64_t seed,
                   int32_t iid, int32_t gen, int32_t i)
{
    return select_parent(fit, P, I, tour_k, seed, iid, gen, i, i);
}

/* Elitist replacement of one island (Sec. 4.4): the children cY/cX/cobj/cfit of slots
 * lo..lo+I; b* is the island's best-ever record.  If the best child (lowest index among
 * equals) is strictly fitter than the record, it becomes the record; then the record
 * overwrites the worst child (lowest index among equals). */
void orc_island_replace(int32_t K, int32_t lo, int32_t I, int16_t *cY, int8_t *cX, int64_t *cobj,
                        int64_t *cfit, int16_t *bY, int8_t *bX, int64_t *bobj, int64_t *bfit)
{
    int32_t b, w;
    orc_island_best_worst(cfit, lo, lo + I, &b, &w);
    if (cfit[b] > *bfit) {
        memcpy(bY, cY + (size_t)b * K, sizeof(int16_t) * (size_t)K);
        memcpy(bX, cX + (size_t)b * K, (size_t)K);
        *bobj = cobj[b];
        *bfit = cfit[b];
    }
    memcpy(cY + (size_t)w * K, bY, sizeof(int16_t) * (size_t)K);
    memcpy(cX + (size_t)w * K, bX, (size_t)K);
    cobj[w] = *bobj;
    cfit[w] = *bfit;
}

/* Single-ring migration over nisl islands of I slots (Sec. 4.4): from a snapshot of every
 * island's best and worst (after replacement), island i's worst slot takes island
 * (i - 1 mod nisl)'s best individual. */
void orc_migrate(int32_t K, int32_t I, int32_t nisl, int16_t *cY, int8_t *cX, int64_t *cobj, int64_t *cfit)
{
    int32_t *bi = (int32_t *)calloc((size_t)nisl, sizeof(int32_t));
    int32_t *wi = (int32_t *)calloc((size_t)nisl, sizeof(int32_t));
    int16_t *mY = (int16_t *)calloc((size_t)nisl * K, sizeof(int16_t));
    int8_t *mX = (int8_t *)calloc((size_t)nisl * K, 1);
    int64_t *mo = (int64_t *)calloc((size_t)nisl, sizeof(int64_t));
    int64_t *mf = (int64_t *)calloc((size_t)nisl, sizeof(int64_t));
    for (int32_t isl = 0; isl < nisl; isl++) {
        orc_island_best_worst(cfit, isl * I, isl * I + I, &bi[isl], &wi[isl]);
        memcpy(mY + (size_t)isl * K, cY + (size_t)bi[isl] * K, sizeof(int16_t) * (size_t)K);
        memcpy(mX + (size_t)isl * K, cX + (size_t)bi[isl] * K, (size_t)K);
        mo[isl] = cobj[bi[isl]];
        mf[isl] = cfit[bi[isl]];
    }
    for (int32_t isl = 0; isl < nisl; isl++) {
        int32_t src = (isl + nisl - 1) % nisl, w = wi[isl];
        memcpy(cY + (size_t)w * K, mY + (size_t)src * K, sizeof(int16_t) * (size_t)K);
        memcpy(cX + (size_t)w * K, mX + (size_t)src * K, (size_t)K);
        cobj[w] = mo[src];
        cfit[w] = mf[src];
    }
    free(bi); free(wi); free(mY); free(mX); free(mo); free(mf);
}

/* Generation-0 bookkeeping over the rows already in st->Y / st->X: decode every row,
 * E_max = 10^a for the smallest a >= 1 above every initial objective (Sec. 5), fitness
 * (Eq. 13), and the best-ever individual of each island (largest fitness, lowest index). */
int32_t orc_ga_init_from(const orc_inst *in, const orc_ga_params *par, orc_ga_state *st)
{
    const int32_t P = par->P, K = st->K, I = par->I;
    int32_t rc = 0;
    for (int32_t i = 0; i < P; i++)
        rc |= decode_one(in, par, st->Y + (size_t)i * K, st->X + (size_t)i * K, &st->obj[i]);
    int64_t mx = 0;
    for (int32_t i = 0; i < P; i++) if (st->obj[i] > mx) mx = st->obj[i];
    int64_t e = 10;
    while (e <= mx) e *= 10;
    st->emax = e;
    for (int32_t i = 0; i < P; i++) st->fit[i] = fitness(e, st->obj[i]);
    for (int32_t isl = 0; isl < P / I; isl++) {
        int32_t b, w;
        orc_island_best_worst(st->fit, isl * I, isl * I + I, &b, &w);
        memcpy(st->bY + (size_t)isl * K, st->Y + (size_t)b * K, sizeof(int16_t) * (size_t)K);
        memcpy(st->bX + (size_t)isl * K, st->X + (size_t)b * K, (size_t)K);
        st->bobj[isl] = st->obj[b];
        st->bfit[isl] = st->fit[b];
    }
    st->gen = 0;
    return rc;
}

/* Generation 0: random X and a Fisher-Yates permutation Y per individual (Sec. 4.3), then
 * the bookkeeping of orc_ga_init_from. */
int32_t orc_ga_init(const orc_inst *in, const orc_ga_params *par, orc_ga_state *st)
{
    const int32_t P = par->P, K = st->K;
    int32_t *gstg = (int32_t *)calloc((size_t)K + 1, sizeof(int32_t));
    int32_t *gjob = (int32_t *)calloc((size_t)K + 1, sizeof(int32_t));
    orc_gene_map(in, gjob, gstg);
    for (int32_t i = 0; i < P; i++) {
        int16_t *y = st->Y + (size_t)i * K;
        int8_t *x = st->X + (size_t)i * K;
        for (int32_t k = 0; k < K; k++) y[k] = (int16_t)(k + 1);
        for (int32_t a = K - 1; a >= 1; a--) {
            uint32_t u = orc_draw(par->seed, P_INIT_Y, par->instance_id, 0, i, K - 1 - a);
            int32_t b = (int32_t)below(u, (uint32_t)a + 1);
            int16_t t = y[a]; y[a] = y[b]; y[b] = t;
        }
        for (int32_t k = 0; k < K; k++) {
            if ((par->mach_mode & 1) == MACH_GENE) {
                uint32_t u = orc_draw(par->seed, P_INIT_X, par->instance_id, 0, i, k);
                x[k] = (int8_t)below(u, (uint32_t)in->o[gstg[k]]);
            } else {
                x[k] = 0;
            }
        }
    }
    free(gstg);
    free(gjob);
    return orc_ga_init_from(in, par, st);
}

/* The offspring of generation st->gen + 1 built from the population st with the Sec. 4.4
 * operators, F per slot (F > 1: candidates of a surrogate-assisted generation, not in the
 * paper): row v = f P + j is candidate f of slot j.  Row v's parent comes from slot j's
 * island (or torus neighbourhood) with row v's selection stream; rows 2q and 2q+1 are the
 * two children of pair q (crossover stream of pair q: head of the first parent, corrected
 * tail of the second); row v is then mutated with its own mutation stream.  With F = 1 the
 * rows are the children of orc_ga_step.  cnew (may be NULL) gets 1 for a row that
 * crossover or mutation changed from a parent's copy. */
int32_t orc_candidates(const orc_inst *in, const orc_ga_params *par, const orc_ga_state *st, int32_t F,
                       int16_t *cY, int8_t *cX, uint8_t *cnew)
{
    const int32_t P = par->P, K = st->K, I = par->I, R = P * F;
    const int32_t gen = st->gen + 1;
    const uint64_t seed = par->seed;
    const int32_t iid = par->instance_id;
    const int gene_mode = (par->mach_mode & 1) == MACH_GENE;

    int32_t *gstg = (int32_t *)calloc((size_t)K + 1, sizeof(int32_t));
    int32_t *gjob = (int32_t *)calloc((size_t)K + 1, sizeof(int32_t));
    int32_t *gene_o = (int32_t *)calloc((size_t)K + 1, sizeof(int32_t));
    orc_gene_map(in, gjob, gstg);
    for (int32_t k = 0; k < K; k++) gene_o[k] = in->o[gstg[k]];

    /* selection: one parent per row */
    int32_t *parent = (int32_t *)calloc((size_t)R, sizeof(int32_t));
    for (int32_t v = 0; v < R; v++)
        parent[v] = select_parent(st->fit, P, I, par->tour_k, seed, iid, gen, v, v % P);

    /* crossover on neighbouring pairs, then mutation of each row */
    uint32_t *xr = (uint32_t *)calloc((size_t)K + 1, sizeof(uint32_t));
    for (int32_t pp = 0; pp < R / 2; pp++) {
        int32_t a = parent[2 * pp], b = parent[2 * pp + 1];
        int16_t *y0 = cY + (size_t)(2 * pp) * K, *y1 = cY + (size_t)(2 * pp + 1) * K;
        int8_t *x0 = cX + (size_t)(2 * pp) * K, *x1 = cX + (size_t)(2 * pp + 1) * K;
        int cross = K >= 2 && chance(orc_draw(seed, P_CROSS, iid, gen, pp, 0), par->pc_num, par->pc_den);
        if (cross) {
            int32_t cx = 1 + (int32_t)below(orc_draw(seed, P_CROSS, iid, gen, pp, 1), (uint32_t)K - 1);
            int32_t cy = 1 + (int32_t)below(orc_draw(seed, P_CROSS, iid, gen, pp, 2), (uint32_t)K - 1);
            orc_crossover(K, st->Y + (size_t)a * K, st->X + (size_t)a * K, st->Y + (size_t)b * K,
                          st->X + (size_t)b * K, cx, cy, y0, x0, y1, x1);
            if (!gene_mode) { memset(x0, 0, (size_t)K); memset(x1, 0, (size_t)K); }
        } else {
            memcpy(y0, st->Y + (size_t)a * K, sizeof(int16_t) * (size_t)K);
            memcpy(y1, st->Y + (size_t)b * K, sizeof(int16_t) * (size_t)K);
            memcpy(x0, st->X + (size_t)a * K, (size_t)K);
            memcpy(x1, st->X + (size_t)b * K, (size_t)K);
        }
        if (cnew) cnew[2 * pp] = cnew[2 * pp + 1] = (uint8_t)cross;
    }
    for (int32_t i = 0; i < R; i++) {
        if (!chance(orc_draw(seed, P_MUTATE, iid, gen, i, 0), par->pm_num, par->pm_den))
            continue;
        int32_t ma = 0, mb = 0;
        if (K >= 2) {
            ma = (int32_t)below(orc_draw(seed, P_MUTATE, iid, gen, i, 1), (uint32_t)K);
            mb = (int32_t)below(orc_draw(seed, P_MUTATE, iid, gen, i, 2), (uint32_t)K - 1);
            mb += (mb >= ma);
        }
        for (int32_t k = 0; k < K; k++)
            xr[k] = gene_o[k] >= 2
                ? below(orc_draw(seed, P_MUTATE, iid, gen, i, 3 + k), (uint32_t)gene_o[k] - 1) : 0;
        orc_mutate(K, gene_o, cY + (size_t)i * K, gene_mode ? cX + (size_t)i * K : NULL, xr, ma, mb);
        if (cnew) cnew[i] = 1;
    }
    free(parent); free(xr); free(gstg); free(gjob); free(gene_o);
    return 0;
}

/* One generation (Sec. 4.4): selection -> paired crossover + correction -> mutation ->
 * decode -> elitist replacement per island -> ring migration every `migrate_every`. */
int32_t orc_ga_step(const orc_inst *in, const orc_ga_params *par, orc_ga_state *st)
{
    const int32_t P = par->P, K = st->K, I = par->I, nisl = P / I;
    const int32_t gen = st->gen + 1;

    /* selection, crossover on neighbouring pairs, mutation */
    int16_t *cY = (int16_t *)calloc((size_t)P * K + 1, sizeof(int16_t));
    int8_t *cX = (int8_t *)calloc((size_t)P * K + 1, 1);
    int64_t *cobj = (int64_t *)calloc((size_t)P, sizeof(int64_t));
    int64_t *cfit = (int64_t *)calloc((size_t)P, sizeof(int64_t));
    orc_candidates(in, par, st, 1, cY, cX, NULL);

    /* fitness of the children */
    int32_t rc = 0;
    for (int32_t i = 0; i < P; i++) {
        rc |= decode_one(in, par, cY + (size_t)i * K, cX + (size_t)i * K, &cobj[i]);
        cfit[i] = fitness(st->emax, cobj[i]);
    }

    /* elitist replacement: the island's best-ever overwrites its worst child */
    for (int32_t isl = 0; isl < nisl; isl++)
        orc_island_replace(K, isl * I, I, cY, cX, cobj, cfit, st->bY + (size_t)isl * K, st->bX + (size_t)isl * K,
                           &st->bobj[isl], &st->bfit[isl]);

    /* single-ring migration: island i's worst <- island (i-1)'s best, from a snapshot */
    if (par->migrate_every > 0 && gen % par->migrate_every == 0 && nisl > 1)
        orc_migrate(K, I, nisl, cY, cX, cobj, cfit);

    memcpy(st->Y, cY, sizeof(int16_t) * (size_t)P * K);
    memcpy(st->X, cX, (size_t)P * K);
    memcpy(st->obj, cobj, sizeof(int64_t) * (size_t)P);
    memcpy(st->fit, cfit, sizeof(int64_t) * (size_t)P);
    st->gen = gen;

    free(cY); free(cX); free(cobj); free(cfit);
    return rc;
}
