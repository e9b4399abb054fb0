/*
 * pa.h -- C ABI of the GB300 population-annealing engine (libpa.so).
 *
 * Population annealing (PA) anneals a population of R replicas of an Ising
 * model through an inverse-temperature schedule beta_0 = 0 < beta_1 < ... ;
 * at each step it reweights every replica by exp(-(beta_i - beta_{i-1}) H),
 * resamples the population, equilibrates it with theta Metropolis sweeps and
 * measures observables (arXiv:2207.05535, Sec. II.B, steps (i)-(vi); Eqs.
 * tauBoltz, QBoltz).  Results of M independent runs are combined with the
 * free-energy weights of Sec. IV (Eqs. appropriateWeight, simpleWeight).
 *
 * Conventions for every entry point:
 *  - Every call returns a pa_status; nothing else crosses the ABI on error.
 *  - Pointers named host_* or documented as "host" are host memory owned by
 *    the caller; the engine copies what it needs and keeps no reference.
 *  - The engine owns all device memory it allocates (from cudaMalloc, or from
 *    the allocator installed by pa_set_allocator) and frees it in
 *    pa_destroy.  Work is enqueued asynchronously on the engine's CUDA stream;
 *    device-side run errors (capacity overflow, extinction) are latched in
 *    a device status word and returned by pa_sync and pa_weighted_average_runs;
 *    pa_anneal_step refuses to continue once one is latched.  The read calls
 *    (pa_records, pa_measure, pa_population) report CUDA errors only, so the
 *    record of a run that stopped (its `status` field) stays readable.
 *  - An engine is not thread safe: serialise calls on one engine.
 *  - Randomness is counter-based Philox4x32-10 keyed by (seed, run_id) and the
 *    counters listed in the engine's documentation, so a run's result does not
 *    depend on which other runs share the engine.
 */
#ifndef PA_H
#define PA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PA_OK = 0,
    PA_ERR_INVALID_ARG = 1, /* a descriptor or argument is out of range */
    PA_ERR_OOM = 2,         /* device or host allocation failed */
    PA_ERR_CAPACITY = 3,    /* a run's population exceeded its capacity R_cap */
    PA_ERR_EXTINCT = 4,     /* a run's population became empty */
    PA_ERR_CUDA = 5,        /* a CUDA runtime call failed */
    PA_ERR_TIMEOUT = 6,     /* reserved for a bounded device-side wait that gave up.  No CTA of
                               this engine spins on another: CTAs of one run meet only at
                               cluster barriers, or the last to finish takes over by a ticket,
                               so no call returns it */
    PA_ERR_STATE = 7,       /* call not valid in the engine's current state */
    PA_ERR_BUSY = 8         /* no room to admit another run */
} pa_status;

enum { PA_FERRO = 0, PA_EA_PMJ = 1 };          /* Eq. H_ferro (J = 1), Eq. H_SG (J = +-1) */
enum { PA_NEAREST = 0, PA_MULTINOMIAL = 1 };   /* resampling of Sec. II.B step (iii) / Sec. IV.C */
/* Overlap pairs of Sec. III.D (bit flags): index shift j <-> j + floor(R_i/2);
 * j <-> j with the paired population; Wang et al.'s pairing (k, pi*_k) from random
 * permutations with a random search pattern, no pair within one family (needs
 * R_cap <= PA_WANG_MAX_RCAP; skipped at a step where no such pairing is found). */
enum { PA_Q_NONE = 0, PA_Q_SHIFT = 1, PA_Q_PAIR = 2, PA_Q_WANG = 4 };
#define PA_WANG_MAX_RCAP 8192u
enum { PA_WEIGHT_FULL = 0, PA_WEIGHT_SIMPLE = 1 };     /* Eq. appropriateWeight / Eq. simpleWeight */

/* theta = PA_THETA_INF: the theta -> infinity limit of Sec. V.B.  Step (iv)'s
 * Metropolis sweeps are replaced by simple sampling of the exact energy
 * distribution P_beta(E) = g(E) exp(-beta E) / Z(beta) from the density of
 * states the descriptor supplies (log_g); every replica gets a fresh energy at
 * each temperature (and at beta_0).  Spins are not represented (all -1 in
 * pa_population) and M = 0; overlaps are not available. */
#define PA_THETA_INF 0xFFFFFFFFu

/* One PA run (Sec. II.B): caller-owned, copied by pa_create. */
typedef struct pa_run_desc {
    uint32_t L;           /* linear lattice size, even, 4 <= L <= 256; N = L*L sites, periodic */
    uint32_t model;       /* PA_FERRO or PA_EA_PMJ */
    uint32_t R;           /* target population size R (Sec. II.B step (i)), >= 1 */
    uint32_t R_cap;       /* capacity (>= R); 0 = R + 8 ceil(sqrt R) + 64 (R for multinomial) */
    uint32_t theta;       /* Metropolis sweeps per temperature (Sec. V.A.1), <= 2^22, or PA_THETA_INF */
    uint32_t n_beta;      /* number of temperatures, >= 1 */
    const double *beta;   /* host, n_beta entries, non-decreasing; beta[0] = 0 gives absolute F */
    uint32_t seed;        /* Philox key word 0 */
    uint32_t run_id;      /* Philox key word 1 (replica randomness) */
    uint32_t disorder_id; /* Philox key word 1 for the +-J couplings */
    uint32_t resample;    /* PA_NEAREST or PA_MULTINOMIAL */
    uint32_t overlap;     /* PA_Q_* flags */
    int32_t paired;       /* with PA_Q_PAIR: index (in this pa_create call) of the partner run, else -1 */
    uint32_t reserved;    /* must be 0 */
    const double *log_g;  /* theta = PA_THETA_INF: host, 2N+1 entries, ln g(E) of the exact density of
                             states at E = 2u - 2N, u = 0..2N (-INFINITY where g(E) = 0; no NaN or
                             +INFINITY; the finite entries all at even u or all at odd u, as the
                             energies of one lattice's states differ by multiples of 4); read at
                             admission.  Ignored (may be NULL) otherwise. */
} pa_run_desc;

/* Per-temperature record of one run (Sec. III.B-D, Eq. rho_t).  Integer sums
 * are exact; ln Q_i and -beta_i F_i are FP64. */
typedef struct pa_step_record {
    double beta;          /* beta_i */
    double lnQ;           /* ln Q_i (Eq. QBoltz); 0 at i = 0 */
    double minus_betaF;   /* -beta_i F_i = N ln 2 + ln Q_1 + ... + ln Q_i (Eq. F), summed in step order */
    int64_t sumE, sumE2;  /* sum_j H_j, sum_j H_j^2 over the R_i replicas */
    int64_t sumAbsM, sumM2; /* sum_j |M_j|, sum_j M_j^2, M_j = sum_n s_n */
    int64_t sum_c2;       /* sum over families of (family size)^2; rho_t = sum_c2 / R_i */
    int64_t sum_absq;     /* sum over index-shift pairs of |N - 2 d| (N |q|) */
    int64_t sum_absq_pair;/* same over pairs with the partner population */
    uint32_t R;           /* R_i */
    uint32_t R_target;    /* R */
    uint32_t n_fam;       /* number of surviving families */
    uint32_t max_fam;     /* largest family */
    uint32_t n_q;         /* number of index-shift pairs, floor(R_i / 2) */
    uint32_t n_q_pair;    /* number of pairs with the partner, min(R_i, R_i') */
    uint32_t N;           /* number of spins */
    uint32_t status;      /* 0, or the pa_status that stopped this run */
    /* Higher powers for the central-moment and Binder estimators (Sec. IV.E):
     * exact sums as 128-bit two's-complement integers, word 0 the low 64 bits
     * (a single H_j^4 exceeds int64 at L = 256). */
    uint64_t sumE3[2];    /* sum_j H_j^3 */
    uint64_t sumE4[2];    /* sum_j H_j^4 */
    uint64_t sumAbsM3[2]; /* sum_j |M_j|^3 */
    uint64_t sumM4[2];    /* sum_j M_j^4 */
    int64_t sum_absq_wang; /* sum over the Wang pairs (k, pi*_k), k < R_i, of |N - 2 d| */
    uint32_t n_q_wang;    /* R_i, or 0 when no pairing without a shared family was found */
    uint32_t wang_swaps;  /* transpositions made by the pairing search */
} pa_step_record;

/* Weighted averages at one temperature over M runs (Sec. IV). */
typedef struct pa_wavg {
    double beta;
    double W_e, W_e2, W_m, W_m2; /* Eq. W_conf applied to e, e^2, |m|, m^2 */
    double Wvar_c, Wvar_chi;     /* Eqs. Wvar_C, Wvar_Chi */
    double W_c, W_chi;           /* Eq. W_conf applied to c and chi (lower bound, Eq. Wvar_bound) */
    double W_minus_betaF;        /* Eq. W_F: -beta_i W[F_i] */
    double W_absq, W_absq_pair;  /* Eq. W_conf applied to |q| */
    double w_max;                /* largest weight */
    double sum_w;                /* sum of the weights */
    double W_e3, W_e4, W_m3, W_m4; /* Eq. W_conf applied to e^3, e^4, |m|^3, m^4 */
    double Wk3_e, Wk4_e;         /* Eq. W_k: central moments of order 3 and 4 of e,
                                    sum_l C(k,l) (-1)^(k-l) W[e]^(k-l) W[e^l], W[e^0] = 1 */
    double Wk3_m, Wk4_m;         /* the same for |m| */
    double W_U4;                 /* Binder cumulant from weighted moments, 1 - W[m^4] / (3 W[m^2]^2) */
    double W_U4_conf;            /* Eq. W_conf applied to each run's 1 - m^4 / (3 (m^2)^2); NaN when a
                                    run's population has M = 0 in every replica */
    double W_absq_wang;          /* Eq. W_conf applied to |q| over the Wang pairs */
} pa_wavg;

typedef struct pa_engine pa_engine;

/* Device memory allocator.  By default an engine takes its device memory from
 * cudaMalloc; pa_set_allocator installs callbacks that every engine created
 * afterwards (and every pa_weighted_average call) uses instead, for example a
 * framework's caching allocator, so that the engine's pools come from the same
 * memory as the caller's tensors.  alloc returns a device pointer to at least
 * `bytes` bytes (256-byte aligned) usable on `stream` of `device`, or NULL when
 * it cannot, which the engine reports as PA_ERR_OOM after releasing what it
 * already holds.  free_ receives every block back with the size it was asked
 * for, when the engine no longer uses it (pa_destroy, or a growing scratch
 * buffer after its work finished).  An engine keeps the allocator it was created
 * with until it is destroyed.  pa_set_allocator(NULL, NULL, NULL) restores
 * cudaMalloc.  The engine allocates only in pa_create, pa_server_create and
 * the first calls of pa_weighted_average_runs / pa_step_records with a larger
 * batch than before; never during an anneal step.  PA_ERR_INVALID_ARG if only
 * one of the two callbacks is given. */
typedef void *(*pa_alloc_fn)(size_t bytes, int device, void *stream, void *ctx);
typedef void (*pa_free_fn)(void *ptr, size_t bytes, int device, void *stream, void *ctx);
pa_status pa_set_allocator(pa_alloc_fn alloc, pa_free_fn free_, void *ctx);

/* Create an engine holding n_runs runs, allocate their device memory, draw the
 * beta_0 = 0 populations (Sec. II.B step (i): uniform states), the couplings
 * (Eq. H_SG) and measure step 0.  cuda_stream: a cudaStream_t to enqueue on,
 * or NULL for a private non-blocking stream.  *out receives the engine.
 * Errors: PA_ERR_INVALID_ARG (descriptor out of range; paired runs must share
 * L, model, disorder_id and n_beta), PA_ERR_OOM, PA_ERR_CUDA. */
pa_status pa_create(const pa_run_desc *runs, uint32_t n_runs, void *cuda_stream, pa_engine **out);

/* pa_create with options (bit flags):
 *   PA_CREATE_GENERIC_SWEEP keeps every lattice size on the general byte-plane
 *     sweep kernel instead of the bit-sliced kernels (rows tiling 32-bit words
 *     when L/2 is a power of two, otherwise rows repacked without padding or
 *     padded rows, whichever the autotuner finds faster); all give identical
 *     results, and the option exists to check that;
 *   PA_CREATE_NO_AUTOTUNE skips timing the bit-sliced kernels' launch shapes on
 *     the first anneal steps and uses the default shape;
 *   PA_CREATE_SEPARATE_KERNELS keeps small runs on the per-stage kernels.
 * Without it, a small run (L = 8, 16 or 32, nearest-integer resampling, no
 * overlaps, R_cap <= 8192) is annealed by one launch per step when its lattice
 * size's runs can each have a cluster of CTAs on SMs of their own (few runs,
 * populations of a few thousand at most): the cluster resamples, sweeps and
 * measures it (when every resident run is
 * small, pa_anneal_step(n) is one launch per lattice size for all n steps, and
 * at L = 8 and 16 the cluster draws each next temperature's random numbers
 * while it measures the current one).
 * Both paths give identical results; PA_CREATE_GENERIC_SWEEP implies the
 * per-stage kernels.
 * Without it, the first anneal steps of a lattice size time every candidate shape
 * on the steps' real sweeps (pa_tuning_pending) and keep the fastest; the
 * choice is shared with every later engine of the process on the same device,
 * which then skips the timing for that size.
 * Results never depend on the launch shape. */
enum { PA_CREATE_GENERIC_SWEEP = 1, PA_CREATE_NO_AUTOTUNE = 2, PA_CREATE_SEPARATE_KERNELS = 4 };
pa_status pa_create_ex(const pa_run_desc *runs, uint32_t n_runs, void *cuda_stream, uint32_t flags,
                       pa_engine **out);

/* ---- Serving: continuous batching of PA jobs ----------------------------
 * A server engine owns fixed device pools sized by this configuration (all
 * counts, not bytes; a word is 4 bytes except where 64-bit words are named).
 * A run takes from each pool what its descriptor implies, in the units below,
 * where a colour plane holds P(L) = ceil(L * pitch / 32) words, the pitch is
 * L/2 when that is a power of two, else the smallest of 4, 8, 16, 32 that is
 * >= L/2 with L * pitch a multiple of 32 (L/2 < 32), else L/2 rounded up to a
 * multiple of 32, and a replica's spin stride is S(L) = 2 P(L) rounded up to
 * a multiple of 4.  Jobs (runs) are admitted and
 * retired between anneal steps; every pa_anneal_step advances all resident,
 * unfinished runs by one temperature in shared launches, each at its own
 * temperature index.  A run's results do not depend on which other runs were
 * resident (its randomness is keyed by its own seed and ids). */
typedef struct pa_server_config {
    uint32_t max_runs;          /* slots */
    uint32_t reserved;          /* must be 0 */
    uint64_t replica_capacity;  /* sum over resident runs of R_cap */
    uint64_t spin_words;        /* sum of R_cap * S(L) */
    uint64_t record_capacity;   /* sum of n_beta */
    uint64_t qhist_words;       /* sum over overlap runs of n_beta (L^2 + 1) */
    uint64_t scratch_words;     /* 64-bit words, per run 3 floor((L^2 + 2) / 2) + L^2 + 5
                                   + max(floor((R_cap + 1) / 2), 128, 4 ceil(R_cap / 16384)) */
    uint64_t coupling_words;    /* per run 2 S(L) + 8 P(L) */
    uint64_t table_doubles;     /* cache of weight tables, (L^2 + 1) per distinct (L, dbeta) */
} pa_server_config;

/* The pools that hold these n_runs runs at once (the sizes pa_create gives an
 * engine for them): *out receives, per pool, the sum of the runs' needs in the
 * units above, max_runs = n_runs, and table_doubles for their distinct
 * (L^2, beta_i - beta_{i-1}) weight tables plus, for theta = PA_THETA_INF runs,
 * n_beta (2 L^2 + 2) per distinct (log_g, schedule).  A server created with it
 * admits exactly these runs (a server's tables are a cache that keeps every
 * distinct table it has built, so a long-lived server needs table space for
 * every distinct one it will meet).  Sums of several calls size a server for a
 * mix.  Host only: no device work, usable without a GPU.  Errors:
 * PA_ERR_INVALID_ARG (as pa_create for the descriptors, or out NULL). */
pa_status pa_pool_sizes(const pa_run_desc *runs, uint32_t n_runs, pa_server_config *out);

/* Create an empty server engine (flags as for pa_create_ex).  Serving has no
 * counterpart in the paper: each admitted run is the PA run of Sec. II.B,
 * unchanged by which other runs share the server.  Errors:
 * PA_ERR_INVALID_ARG, PA_ERR_OOM, PA_ERR_CUDA. */
pa_status pa_server_create(const pa_server_config *cfg, void *cuda_stream, uint32_t flags, pa_engine **out);

/* Admit n_runs runs (pair indices relative to this call; a pair is admitted
 * together) into free slots; *slots_out receives their slot numbers, which
 * every per-run call takes in place of a run index.  All or nothing: returns
 * PA_ERR_BUSY (nothing admitted) when slots, pool space or table space are
 * short.  Their beta_0 populations are drawn with the next enqueued work. */
pa_status pa_admit(pa_engine *e, const pa_run_desc *runs, uint32_t n_runs, uint32_t *slots_out);

/* Release a slot and its pool ranges (after reading its records).  Waits for
 * the engine's queued work.  A retired run's partner continues without
 * two-population overlaps. */
pa_status pa_retire(pa_engine *e, uint32_t slot);

/* Slots whose runs have reached their last temperature (host bookkeeping, no
 * synchronisation): writes up to cap slots, *n_out = how many there are. */
pa_status pa_finished(const pa_engine *e, uint32_t *slots_out, uint32_t cap, uint32_t *n_out);

/* Device state of a slot: temperature index, population size and status
 * (0 or the pa_status that stopped it).  Synchronises. */
pa_status pa_run_state(pa_engine *e, uint32_t slot, uint32_t *step, uint32_t *R, uint32_t *status);

/* Return every run of the engine to its beta_0 population (Sec. II.B step
 * (i); same descriptors, same randomness, so the next anneal repeats the first
 * one bit for bit) without reallocating: clears records, histograms and
 * statuses, redraws the couplings and populations and measures step 0.
 * Asynchronous. */
pa_status pa_reset(pa_engine *e);

/* Advance every unfinished run by up to n_steps temperatures (fewer when every
 * run reaches its last temperature first): resampling
 * (Eqs. tauBoltz, QBoltz and step (iii)), theta checkerboard Metropolis sweeps
 * at beta_i (step (iv)) and measurements (step (v)).  Asynchronous.  With
 * use_graph != 0 the per-step launch sequence is captured once as a CUDA graph
 * and replayed.  Errors surface at the next synchronising call. */
pa_status pa_anneal_step(pa_engine *e, uint32_t n_steps, int use_graph);

/* Block until the engine's queued work is done; returns the latched status. */
pa_status pa_sync(pa_engine *e);

/* Copy the records of run `run` (index in pa_create order) for steps
 * 0..n_beta-1 into host_out[n_beta] (the population sums, ln Q_i and -beta_i F_i
 * of Sec. III.B-D; steps not reached yet are zero), and the
 * overlap histograms over d = 0..N (d = Hamming distance, q = 1 - 2d/N) into
 * host_qhist[n_beta][N+1] / host_qhist_pair[n_beta][N+1] / host_qhist_wang[n_beta][N+1]
 * (index shift, paired population, Wang pairs) when non-NULL.  Synchronises. */
pa_status pa_records(pa_engine *e, uint32_t run, pa_step_record *host_out, uint32_t *host_qhist,
                     uint32_t *host_qhist_pair, uint32_t *host_qhist_wang);

/* The record of each run in runs[0..n_runs) at the temperature it has reached
 * (its current temperature index) into host_out[n_runs]: one gather on the
 * device and one copy back, for streaming a batch's or a server's results
 * after every anneal step.  Synchronises.  PA_ERR_INVALID_ARG for a run that
 * is not resident. */
pa_status pa_step_records(pa_engine *e, const uint32_t *runs, uint32_t n_runs, pa_step_record *host_out);

/* Copy the record of one run at one step (Sec. III.B-D; and optional overlap
 * histograms, N+1 entries each).  Synchronises. */
pa_status pa_measure(pa_engine *e, uint32_t run, uint32_t step, pa_step_record *host_out, uint32_t *host_qhist,
                     uint32_t *host_qhist_pair, uint32_t *host_qhist_wang);

/* Copy the current population of run `run` (the R_i replicas of Sec. II.B at
 * the temperature reached): host_spins[R_i][N] as int8 +-1
 * (site n = y*L + x), energies, magnetisations and family ids (index of the
 * beta_0 ancestor), each R_i entries, caller-sized to at least R_cap; *R_out = R_i;
 * *step_out = current temperature index.  Any pointer may be NULL.  Synchronises. */
pa_status pa_population(pa_engine *e, uint32_t run, int8_t *host_spins, int32_t *host_E, int32_t *host_M,
                        uint32_t *host_fam, uint32_t *R_out, uint32_t *step_out);

/* The same for replicas first .. first+count-1 only (clipped to R_i): the
 * outputs hold min(count, R_i - first) entries (spins [that][N]).  For sampling
 * replicas of populations too large to copy whole.  Synchronises. */
pa_status pa_population_slice(pa_engine *e, uint32_t run, uint32_t first, uint32_t count, int8_t *host_spins,
                              int32_t *host_E, int32_t *host_M, uint32_t *host_fam, uint32_t *R_out,
                              uint32_t *step_out);

/* Checkpoint and resume of one run between anneal steps.  The state after
 * temperature i of Sec. II.B is everything the rest of the anneal reads: the
 * population at beta_i (spins, E, M, family ids), the records of steps 0..i
 * (with ln Q and -beta F), the overlap histograms, the couplings, and the
 * next resampling's level tables.  Counter-based randomness needs no
 * generator state, so a resumed run continues exactly as if never stopped.
 *
 * pa_checkpoint copies run `run`'s state into host_buf.  *bytes: capacity of
 * host_buf on entry, bytes written (or needed) on return; host_buf NULL asks
 * for the size only.  PA_ERR_INVALID_ARG if the buffer is too small (*bytes
 * then holds the size), PA_ERR_STATE if the run stopped with an error status.
 * Synchronous (waits for the work queued before it).
 *
 * pa_restore overwrites run `run` of any engine with a checkpoint.  The run
 * must have been admitted with the same descriptor (L, model, R, R_cap, theta,
 * schedule, seed, run_id, disorder_id, resample, overlap, and for theta =
 * PA_THETA_INF the same ln g); otherwise, or if the buffer is not a whole
 * checkpoint, PA_ERR_INVALID_ARG and nothing is changed.  Paired runs
 * (PA_Q_PAIR) are restored together, from checkpoints of the same step.  When
 * no resident run is left stopped afterwards, the engine's latched error
 * (capacity, extinction) is cleared, so a run that failed can be resumed from
 * an earlier checkpoint.  Synchronous; host_buf may be reused on return. */
pa_status pa_checkpoint(pa_engine *e, uint32_t run, void *host_buf, size_t *bytes);
pa_status pa_restore(pa_engine *e, uint32_t run, const void *host_buf, size_t bytes);

/* Weighted averages (Sec. IV) over groups of runs resident in the engine:
 * group g holds runs run_idx[g*M .. g*M+M-1] (same N and n_beta).  Writes
 * host_out[g][n_beta] and, when non-NULL, the weighted overlap distributions
 * host_Pq[g][n_beta][N+1] / host_Pq_pair / host_Pq_wang (Eq. W_conf_q).  weight_kind is
 * PA_WEIGHT_FULL or PA_WEIGHT_SIMPLE.  Runs in FP64 on the device.  Synchronises. */
pa_status pa_weighted_average_runs(pa_engine *e, const uint32_t *run_idx, uint32_t n_groups, uint32_t M,
                                   uint32_t weight_kind, pa_wavg *host_out, double *host_Pq,
                                   double *host_Pq_pair, double *host_Pq_wang);

/* Weighted averages (Sec. IV; Eqs. appropriateWeight or simpleWeight, W_conf,
 * W_F, Wvar_C, Wvar_Chi, W_conf_q, W_k) from host records: recs[m*n_steps + i] for M runs of N spins,
 * optional histograms qhist[(m*n_steps + i)*(N+1) + d] (likewise qhist_pair,
 * qhist_wang).  Writes out[n_steps] and Pq / Pq_pair / Pq_wang [n_steps][N+1]
 * when non-NULL.  Computes on the device of the current CUDA context (stream:
 * cudaStream_t or NULL); blocking. */
pa_status pa_weighted_average(const pa_step_record *recs, const uint32_t *qhist, const uint32_t *qhist_pair,
                              const uint32_t *qhist_wang, uint32_t M, uint32_t n_steps, uint32_t N,
                              uint32_t weight_kind, pa_wavg *out, double *Pq, double *Pq_pair, double *Pq_wang,
                              void *cuda_stream);

/* Limits of pa_weighted_average_noalloc's fixed scratch. */
#define PA_NOALLOC_MAX_RUNS 4096u      /* M */
#define PA_NOALLOC_MAX_WEIGHTS 65536u  /* M * n_steps */

/* Weighted averages (Sec. IV, the same arithmetic as pa_weighted_average, no
 * overlap distributions) for callers that cannot allocate device memory: serving
 * loops that reserve all device memory up front and must not call into the
 * allocator in the steady state (cudaMalloc can synchronise the device and
 * stall the other streams), or processes whose device memory belongs to
 * another allocator (a framework's caching allocator or a pre-sized arena).
 * The paper has no counterpart; this is a deployment variant.
 *   d_recs: device pointer, M * n_steps records laid out [m][i] (run m, step i);
 *   d_out:  device pointer, n_steps results; N: spins per run.
 * Nothing is allocated or freed.  The scratch (record offsets and weights) is
 * one fixed array of about 544 KiB in device memory that every GPU loading
 * libpa.so holds until the process exits; M > PA_NOALLOC_MAX_RUNS or
 * M * n_steps > PA_NOALLOC_MAX_WEIGHTS is rejected with PA_ERR_INVALID_ARG
 * (and a message on stderr).  The first call on each device looks up the
 * array's device address (with that device current) and keeps it for the
 * life of the process.  A cudaDeviceReset of that device makes the kept
 * address stale: do not call this entry point on a device after resetting
 * it.  The work is enqueued on cuda_stream (a
 * cudaStream_t or NULL) and the call returns without waiting.  Every call
 * shares the one array: calls whose work overlaps on the GPU (other streams,
 * or other host threads) race and must be serialised by the caller. */
pa_status pa_weighted_average_noalloc(const pa_step_record *d_recs, uint32_t M, uint32_t n_steps, uint32_t N,
                                      uint32_t weight_kind, pa_wavg *d_out, void *cuda_stream);

/* Number of kernels this engine has launched (graph replays count each node). */
uint64_t pa_launch_count(const pa_engine *e);

/* Launch shape of the sweep for lattice-size group `group` (groups in order of
 * first appearance of each L): words of a colour plane per thread (0 for the
 * byte-plane kernel), threads per CTA, and whether it was chosen by timing. */
pa_status pa_sweep_shape(const pa_engine *e, uint32_t group, uint32_t *L, uint32_t *words_per_thread,
                         uint32_t *block, uint32_t *tuned);

/* Number of lattice sizes whose sweep launch shape is still being chosen: the
 * first anneal steps after a size appears run each candidate shape on the
 * step's real sweep (one warm-up step, then two steps per candidate, timed)
 * eagerly, before graph replay takes over.  Host bookkeeping; no
 * synchronisation. */
pa_status pa_tuning_pending(const pa_engine *e, uint32_t *n);

/* Kernel classes timed by the profiling mode. */
enum { PA_K_RESAMPLE = 0, PA_K_SWEEP = 1, PA_K_OVERLAP = 2, PA_K_MEASURE = 3, PA_K_INIT = 4, PA_K_WAVG = 5,
       PA_K_SMALL = 6, PA_K_COUNT = 7 };  /* PA_K_SMALL: the one-launch-per-step path of small runs */

/* Profiling mode: with on != 0 every kernel launch is bracketed by CUDA events
 * on the engine's stream and pa_anneal_step launches eagerly (no graph). */
pa_status pa_set_profiling(pa_engine *e, int on);

/* Synchronise and return, per kernel class, the summed device time in ms and
 * the number of launches timed since the previous call (arrays of PA_K_COUNT). */
pa_status pa_kernel_times(pa_engine *e, double *ms_out, uint64_t *launches_out);

/* Bytes this engine has copied host->device and device->host so far. */
pa_status pa_transfer_bytes(const pa_engine *e, uint64_t *h2d, uint64_t *d2h);

/* Throughput of Philox4x32-10 (Salmon et al., SC'11; the generator behind every
 * random decision of the engine) alone on the current device, in calls per second:
 * a loop of independent calls (8 per thread, 2432 CTAs of 128 threads, 64
 * iterations), timed with CUDA events after one warm-up launch, best of `reps`.
 * wide = 0 writes each 32x32->64 multiply as separate high and low halves, 1 as
 * one 64-bit product.  It measures the integer-multiplier roof that the sweep
 * kernels are compared against (40 multiply-add slots per call).  Allocates and
 * frees a small device buffer; runs on `cuda_stream` (cudaStream_t or NULL);
 * blocking. */
pa_status pa_calibrate_philox(uint32_t wide, uint32_t reps, void *cuda_stream, double *calls_per_s);

/* Free all device memory of the engine.  Synchronises first. */
pa_status pa_destroy(pa_engine *e);

/* Static description of a status code. */
const char *pa_status_string(pa_status s);

#ifdef __cplusplus
}
#endif

#endif /* PA_H */
