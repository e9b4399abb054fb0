// Internal layout shared by the engine's host code and its kernels.
//
// Device memory layout (one pool per engine, every run at its own offsets):
//   spins[b]  uint32 [sum R_cap wstride]    replica j of a run at word spin_off + j wstride:
//                                           colour plane 0 in words [0, PW), plane 1 in
//                                           [PW, 2 PW); site n = y L + x has colour (x + y) & 1
//                                           and sits in row y of its plane at bit position
//                                           y * pitch + (x >> 1) (rows padded to the pitch,
//                                           padding bits 0); bit 1 = spin +1; buffer b = step & 1
//   E[b], M[b], fam[b]   [sum R_cap]        energy, magnetisation, beta_0 ancestor
//   parent, cnt          [sum R_cap]        parent map of the children, copy numbers r_j
//   rec                  [sum n_beta]       per-temperature records (pa_step_record)
//   qh, qhp, qhw         [sum n_beta (N+1)] overlap histograms over d (shift / pair / Wang)
//   beta, thr                               schedule and Metropolis thresholds per step
//   wt, wtoff                               weight tables exp(-4 n dbeta) shared by every run
//                                           and step with the same (N, dbeta); wtoff[wt_off + i]
//                                           = offset of step i's table in wt.  Runs with
//                                           theta = PA_THETA_INF also keep per step the
//                                           cumulative level weights of P_beta_i over
//                                           u = 0..2N and, in entry 2N + 1, the last level
//                                           with a positive weight (as a double)
//   J                    per run: site-order "J = -1" bits of right / down bonds
//                        (2 wstride words), then per colour plane word the four bond
//                        masks (same, rotated, up, down neighbour) [2][4][PW]
//   scratch              per run: energy and magnetisation histograms (N+1 u32 each),
//                        level CDF or thresholds (N+1 f64 / u64), level fill counters or
//                        floors (N+1 u32), then members (R_cap u32) / per-CTA totals /
//                        per-CTA family statistics
#pragma once

#include <cstdint>
#include <vector>

#include "pa.h"

namespace pa {

constexpr uint32_t TAG_INIT = 1u, TAG_SWEEP = 2u, TAG_RESAMPLE = 3u, TAG_MULTINOMIAL = 4u, TAG_DISORDER = 5u,
                   TAG_DOS = 6u, TAG_WANG = 7u;
constexpr uint32_t WANG_IDX_BITS = 13u;  // PA_WANG_MAX_RCAP = 2^13

// status bits in the engine-wide device status word
constexpr uint32_t ST_CAPACITY = 1u << PA_ERR_CAPACITY;
constexpr uint32_t ST_EXTINCT = 1u << PA_ERR_EXTINCT;
constexpr uint32_t ST_TIMEOUT = 1u << PA_ERR_TIMEOUT;

struct RunDev {
    uint32_t L, N, Lh, wstride;  // wstride: words per replica, a multiple of 4
    uint32_t model, R, R_cap, theta;
    uint32_t n_beta, seed, run_id, disorder_id;
    uint32_t resample, overlap;
    int32_t paired;
    uint32_t pitch;  // bits per row in a colour plane (>= L/2; see row_pitch)
    uint32_t pw;     // words per colour plane = ceil(L pitch / 32)
    uint32_t pad0;
    uint64_t rep_off;   // first replica slot (E, M, fam, parent, cnt)
    uint64_t spin_off;  // first spin word (runs of different L have different wstride)
    uint64_t rec_off, qh_off, beta_off, wt_off, thr_off, J_off, scr_off;
    double ln2N;  // N ln 2 = ln Z(beta_0 = 0)
    uint64_t dos_off;  // theta = PA_THETA_INF: step i's energy CDF at wt[dos_off + i (2N + 2)]
};

struct RunState {
    uint32_t step;   // temperature index of the population held
    uint32_t R_cur;  // R_step
    uint32_t R_new;  // population size produced by the resampling in flight
    uint32_t status; // 0 or a pa_status that stopped the run
    double lnQ;      // ln Q of the resampling in flight
    uint32_t ticket;   // CTAs of the run done in the launch in flight (0 between launches)
    int32_t Emin;      // nearest-integer resampling in flight: lowest energy of the population
    uint32_t n_levels; // and its number of energy levels (Emax - Emin) / 4 + 1
    uint32_t pad;
};

// Kernels that split one population over several CTAs give each CTA about
// CTA_REPLICAS replicas, at most MAX_RUN_CTAS CTAs per run.
constexpr uint32_t CTA_REPLICAS = 16384, MAX_RUN_CTAS = 256;
__host__ __device__ inline uint32_t run_ctas(uint32_t R_cap)
{
    const uint32_t c = (R_cap + CTA_REPLICAS - 1) / CTA_REPLICAS;
    return c < 1 ? 1 : (c > MAX_RUN_CTAS ? MAX_RUN_CTAS : c);
}

struct Pool {
    const RunDev *runs;
    RunState *st;
    uint32_t *spins[2];
    int32_t *E[2];
    int32_t *M[2];
    uint32_t *fam[2];
    uint32_t *parent;
    uint32_t *cnt;
    pa_step_record *rec;
    uint32_t *qh;
    uint32_t *qhp;
    uint32_t *qhw;
    const double *beta;
    const double *wt;                  // weight tables exp(-4 n dbeta), (N + 1) doubles each
    const unsigned long long *wtoff;   // per run and step: offset of its table in wt
    const unsigned long long *thr;
    uint32_t *J;
    unsigned long long *scratch;
    uint32_t *status;
};

// Sweep launch shape for one lattice size.
struct SweepCfg {
    uint32_t fast;   // 0: byte planes; 1: bit-sliced (L/2 a power of two); 2: bit-sliced, padded rows;
                     // 3: bit-sliced, rows repacked without padding in shared memory
    uint32_t block;  // threads per CTA
    uint32_t TPR;    // threads per replica (power of two; bit-sliced kernels: words per plane / WPT)
    uint32_t RPC;    // replicas per CTA
    uint32_t G;      // Philox groups per colour = ceil(N / 8)
    uint32_t PS;     // bytes per colour plane = 4 G (byte planes); the row pitch (padded or compact rows)
    uint32_t smem;   // dynamic shared memory bytes
    uint32_t WPT;    // fast kernel: plane words per thread
};

// Row pitch of a colour plane: L/2 when that is a power of two; else the
// smallest power of two >= L/2 that makes L * pitch a multiple of 32 (rows then
// tile 32-bit words, so the bit-sliced sweep applies) for L/2 < 32, and L/2
// rounded up to a multiple of 32 beyond.
inline uint32_t row_pitch(uint32_t L)
{
    const uint32_t Lh = L / 2;
    if ((Lh & (Lh - 1)) == 0) return Lh;
    if (Lh < 32)
        for (uint32_t P = 4; P <= 32; P <<= 1)
            if (P >= Lh && (L * P) % 32 == 0) return P;
    return (Lh + 31) / 32 * 32;
}

inline uint32_t plane_words_of(uint32_t L) { return (L * row_pitch(L) + 31) / 32; }

// Scratch of one run, in 64-bit words from scr_off: the energy and the
// magnetisation histograms of the measurement (N + 1 u32 each, left cleared
// between steps), a per-level f64 / u64 table (N + 1), a per-level u32 table
// (N + 1), then a tail used by one kernel at a time: the multinomial member
// list (R_cap u32), or the per-CTA replica totals of the resampling
// (MAX_RUN_CTAS u32), or the measurement's per-CTA family statistics
// (MEASURE_PART_WORDS each).
constexpr uint64_t MEASURE_PART_WORDS = 4;
__host__ __device__ inline uint64_t scr_hist_words(uint32_t N) { return (uint64_t(N) + 2) / 2; }
__host__ __device__ inline uint64_t scr_mhist_off(uint32_t N) { return scr_hist_words(N); }
__host__ __device__ inline uint64_t scr_table_off(uint32_t N) { return 2 * scr_hist_words(N); }
__host__ __device__ inline uint64_t scr_level_off(uint32_t N) { return scr_table_off(N) + N + 1; }
__host__ __device__ inline uint64_t scr_tail_off(uint32_t N) { return scr_level_off(N) + scr_hist_words(N); }
inline uint64_t scratch_words(uint32_t N, uint32_t R_cap)
{
    const uint64_t members = (uint64_t(R_cap) + 1) / 2;
    const uint64_t totals = MAX_RUN_CTAS / 2, parts = MEASURE_PART_WORDS * run_ctas(R_cap);
    uint64_t tail = members > totals ? members : totals;
    tail = tail > parts ? tail : parts;
    return scr_tail_off(N) + tail + 4;
}

// Small populations annealed by one launch per step (anneal_small_kernel): one
// thread-block cluster per run, cluster size small_cluster().
constexpr uint32_t SMALL_MAX_RCAP = 8192;
inline bool small_eligible(const RunDev &x)
{
    return (x.L == 8 || x.L == 16 || x.L == 32) && x.theta != PA_THETA_INF && x.resample == PA_NEAREST &&
           x.overlap == 0 && x.R_cap <= SMALL_MAX_RCAP;
}
// Lanes that share one colour-plane word in the small-population kernel's
// sweeps (each draws 8 / LPW of the word's Philox groups); the fastest
// measured for 20 runs of a few hundred replicas: 8 at L = 8, 2 at L = 16,
// 1 and 2 alike at L = 32.
#ifndef SMALL_LPW_L8
#define SMALL_LPW_L8 8
#endif
#ifndef SMALL_LPW_L16
#define SMALL_LPW_L16 2
#endif
#ifndef SMALL_LPW_L32
#define SMALL_LPW_L32 2
#endif

// Launch wrappers implemented in pa_kernels.cu (all asynchronous on `s`).
// `runs`: device list of the indices of the runs to process (the two
// initialisation launches also take NULL for runs 0..n_runs-1).
void launch_init_couplings(const Pool &P, const uint32_t *runs, uint32_t n_runs, cudaStream_t s);
// Work lists: tile_off = prefix of per-run tile counts (n + 1 entries).
void launch_init_population(const Pool &P, const uint32_t *tile_off, const uint32_t *runs, uint32_t n_runs,
                            uint32_t n_tiles, uint32_t max_pw, cudaStream_t s);
// Resampling of runs with PA_MULTINOMIAL, one CTA per run.  max_Rcap: the
// largest R_cap among the runs (sets the energies staged in shared memory).
void launch_resample_multinomial(const Pool &P, const uint32_t *runs, uint32_t n_runs, uint32_t max_Rcap,
                                 cudaStream_t s);
// Nearest-integer resampling (PA_NEAREST) from the tables the measurement of
// the previous step prepared, run_ctas(R_cap) CTAs per run, in
// resample_nearest_launches(max_Rcap) kernel launches (one when every
// population fits one CTA).
inline uint32_t resample_nearest_launches(uint32_t max_Rcap) { return run_ctas(max_Rcap) == 1 ? 1u : 2u; }
void launch_resample_nearest(const Pool &P, const uint32_t *runs, uint32_t n_runs, uint32_t max_Rcap, cudaStream_t s);
// Launch shapes to try for lattice size L (first = default); one entry unless
// the bit-sliced kernel applies.
std::vector<SweepCfg> sweep_candidates(uint32_t L, int allow_fast);
void launch_sweep(const Pool &P, const uint32_t *group_runs, const uint32_t *tile_off, uint32_t n_group_runs,
                  uint32_t n_tiles, const SweepCfg &cfg, int any_glass, cudaStream_t s);
void launch_overlap(const Pool &P, const uint32_t *q_runs, uint32_t n_q_runs, uint32_t max_Rcap, int init,
                    cudaStream_t s);
// run_ctas(R_cap) CTAs per run (at most run_ctas(max_Rcap)); also prepares the
// next nearest-integer resampling of each run.
void launch_measure(const Pool &P, const uint32_t *runs, uint32_t n_runs, uint32_t max_Rcap, int init,
                    cudaStream_t s);
// theta = PA_THETA_INF runs: fresh energies from the exact distribution for
// the population of the step in flight (init: the beta_0 population).
void launch_dos_sample(const Pool &P, const uint32_t *runs, uint32_t n_runs, uint32_t max_R, int init,
                       cudaStream_t s);
// Wang et al.'s pairing and its overlaps for the runs in `runs` (init: step 0);
// max_Rcap: the largest R_cap among them (sets the shared memory).
void launch_wang(const Pool &P, const uint32_t *runs, uint32_t n_runs, uint32_t max_Rcap, int init, cudaStream_t s);
size_t wang_smem_bytes(uint32_t max_Rcap);
void launch_wavg_wang(const pa_step_record *recs, const unsigned long long *rec_off, const uint32_t *qh,
                      const uint32_t *qhp, const uint32_t *qhw, const unsigned long long *qh_off, uint32_t n_groups,
                      uint32_t M, uint32_t n_steps, uint32_t N, uint32_t kind, pa_wavg *out, double *w, double *Pq,
                      double *Pqp, double *Pqw, cudaStream_t s);
void launch_wavg(const pa_step_record *recs, const unsigned long long *rec_off, const uint32_t *qh,
                 const uint32_t *qhp, const unsigned long long *qh_off, uint32_t n_groups, uint32_t M,
                 uint32_t n_steps, uint32_t N, uint32_t kind, pa_wavg *out, double *w, double *Pq, double *Pqp,
                 cudaStream_t s);
// Copies the record of each listed run at the temperature it has reached to out[k].
void launch_gather_records(const Pool &P, const uint32_t *runs, uint32_t n_runs, pa_step_record *out,
                           cudaStream_t s);
// n_steps temperatures of the small runs `runs` (all of lattice size L), cs
// CTAs (a cluster) per run.
// Launch shape of the small-run kernel: CTAs per cluster (one cluster per run),
// threads per CTA, the compiled variant (0: 512 threads two CTAs per SM; 1 / 2:
// up to 512 / 768 threads one CTA per SM; 3 / 4: the same with 4 lanes per word
// at L = 8), the half-sweeps whose comparison bits are drawn ahead (0: none)
// and the dynamic shared memory they take.
struct SmallShape {
    uint32_t cs, block, variant, H, smem;
};
SmallShape small_shape(uint32_t L, int any_glass, uint32_t n_runs, uint32_t R_max, uint32_t R_cap_max);
SmallShape small_shape_ahead(uint32_t L, int any_glass, uint32_t n_runs, uint32_t R_max, uint32_t theta_max);
void launch_anneal_small(const Pool &P, const uint32_t *runs, uint32_t n_runs, uint32_t L, const SmallShape &sh,
                         int any_glass, uint32_t n_steps, cudaStream_t s);
cudaError_t prepare_kernels();
// Philox-only calibration loop: blocks x threads threads, iters x 8 calls each.
void launch_philox_calibration(uint32_t *out, uint32_t blocks, uint32_t threads, uint32_t iters, bool wide,
                               cudaStream_t s);

}  // namespace pa
