/*
 * Plain CPU oracle for population annealing (PA) of the 2D Ising ferromagnet and
 * the 2D +-J Edwards-Anderson spin glass, with free-energy-weighted averages.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library.  It shares no code, header, table or
 * constant generator with the CUDA engine; it is deliberately slow and follows the
 * paper step by step:
 *   - the generic PA loop, steps (i)-(vi) of Sec. II.B, in its canonical form
 *     (Eqs. tauBoltz, QBoltz) with nearest-integer resampling,
 *   - the Hamiltonians of Sec. III.A (Eqs. H_ferro, H_SG), periodic L x L lattice,
 *   - the population estimators of Sec. III.B (Eqs. PopAvrg, e, m, c, chi),
 *   - the free-energy estimator of Sec. III.C (Eq. F with ln Z(0) = N ln 2),
 *   - the overlap q and index-shift pairs of Sec. III.D,
 *   - the mean-square family size rho_t of Sec. V.A.4 (Eq. rho_t),
 *   - the weighted averages of Sec. IV (Eqs. appropriateWeight, simpleWeight,
 *     W_conf, W_F, Wvar_C, Wvar_Chi, W_conf_q), and the central-moment estimators
 *     W_k of Sec. IV.E for k = 3, 4 with the Binder cumulant built the same way,
 * plus exact reference solvers used only to pin this oracle: brute-force
 * enumeration, Kaufman's finite-lattice partition function (Sec. V.A.3 names it as
 * the exact FM reference) and a transfer-matrix density of states.
 *
 * Randomness is counter-based Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel
 * random numbers: as easy as 1, 2, 3", SC'11), written here from that definition.
 * The keying (which counter feeds which decision) is the normative contract that
 * the CUDA engine implements independently:
 *   key = (seed, run_id)           [couplings: key = (seed, disorder_id)]
 *   counter word 3 = tag << 24 | extra
 *   init spin i of replica j       : ctr (i>>2, j, 0, INIT<<24),            word i&3, bit 31 => s=+1
 *   coupling right/down of site i  : ctr (i>>2, 0, 0, DISORDER<<24),        word i&3, bit31/bit30 => J=+1
 *   nearest-int draw, replica j    : ctr (j, 0, step, RESAMPLE<<24),        word 0
 *   multinomial draw d             : ctr (d, 0, step, MULTINOMIAL<<24),     words 0,1 (level), 2 (member)
 *   Metropolis at site with sublattice index k, child j, sweep t, colour c:
 *                                    ctr (k>>2, j, step, SWEEP<<24 | t<<1 | c), word k&3
 *   energy draw of replica j (theta = infinity, Sec. V.B):
 *                                    ctr (j, 0, step, DOS<<24),               words 0,1
 *   permutation keys of replica j (Wang pairing, Sec. III.D):
 *                                    ctr (j, 0, step, WANG<<24),              words 0,1 (pi), 2,3 (sigma)
 * Build with -ffp-contract=off: no fused multiply-add anywhere in the FP64 paths.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_TAG_INIT 1u
#define OR_TAG_SWEEP 2u
#define OR_TAG_RESAMPLE 3u
#define OR_TAG_MULTINOMIAL 4u
#define OR_TAG_DISORDER 5u
#define OR_TAG_DOS 6u
#define OR_TAG_WANG 7u
#define OR_WANG_IDX_BITS 13u     /* Wang pairing: R_cap <= 2^13 */
#define OR_THETA_INF 0xFFFFFFFFu /* theta = infinity: simple sampling of the exact energy distribution */

#define OR_OK 0
#define OR_ERR_INVALID 1
#define OR_ERR_OOM 2
#define OR_ERR_CAPACITY 3
#define OR_ERR_EXTINCT 4
#define OR_ERR_STATE 7

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon et al., SC'11): 10 rounds of the 4x32 Philox S-box,  */
/* multipliers 0xD2511F53 / 0xCD9E8D57, Weyl key increments 0x9E3779B9 /     */
/* 0xBB67AE85 between rounds.                                                */
/* ------------------------------------------------------------------------- */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k0;
        uint32_t n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
    out[0] = c[0];
    out[1] = c[1];
    out[2] = c[2];
    out[3] = c[3];
}

static uint32_t philox_word(uint32_t seed, uint32_t keyid, uint32_t c0, uint32_t c1, uint32_t c2,
                            uint32_t c3, unsigned word)
{
    uint32_t ctr[4] = {c0, c1, c2, c3}, key[2] = {seed, keyid}, out[4];
    or_philox4x32_10(ctr, key, out);
    return out[word];
}

/* ------------------------------------------------------------------------- */
/* Run description (mirrors the caller's descriptor; defined here on its own) */
/* ------------------------------------------------------------------------- */
typedef struct {
    uint32_t L;            /* even, >= 4 */
    uint32_t model;        /* 0 = ferromagnet (J=1), 1 = +-J EA glass */
    uint32_t R;            /* target population size */
    uint32_t R_cap;        /* capacity: R_i > R_cap is an error */
    uint32_t theta;        /* Metropolis sweeps per temperature */
    uint32_t n_beta;       /* number of temperatures beta_0..beta_{n-1} */
    const double *beta;    /* schedule, non-decreasing */
    uint32_t seed, run_id, disorder_id;
    uint32_t resample;     /* 0 = nearest integer, 1 = multinomial */
    uint32_t overlap;      /* bit 0: index-shift q; bit 1: q against a paired run; bit 2: Wang pairing */
    const double *log_g;   /* theta = OR_THETA_INF: ln g(E) at E = 2u - 2N, u = 0..2N (-INFINITY where g = 0) */
} or_desc;

/* Per-temperature record (one per step i = 0..n_beta-1). */
typedef struct {
    double beta;           /* beta_i */
    double lnQ;            /* ln Q_i, Eq. QBoltz (0 at i = 0) */
    double minus_betaF;    /* -beta_i F_i = N ln 2 + sum_{k<=i} ln Q_k, Eq. F */
    int64_t sumE, sumE2, sumAbsM, sumM2;
    int64_t sum_c2;        /* sum over families of (family size)^2 */
    int64_t sum_absq;      /* sum over index-shift pairs of |N - 2 d| */
    int64_t sum_absq_pair; /* same for pairs with the paired run */
    uint32_t R;            /* R_i */
    uint32_t R_target;     /* R */
    uint32_t n_fam, max_fam;
    uint32_t n_q, n_q_pair;
    uint32_t N;
    uint32_t status;
    /* Sec. IV.E central moments need higher powers: exact sums as 128-bit two's
     * complement integers, word 0 the low 64 bits (sum_j H_j^4 exceeds int64
     * once L reaches 256). */
    uint64_t sumE3[2];     /* sum_j H_j^3 */
    uint64_t sumE4[2];     /* sum_j H_j^4 */
    uint64_t sumAbsM3[2];  /* sum_j |M_j|^3 */
    uint64_t sumM4[2];     /* sum_j M_j^4 */
    int64_t sum_absq_wang; /* sum over the R_i Wang pairs (k, pi*_k) of |N - 2 d| */
    uint32_t n_q_wang;     /* R_i, or 0 when no pairing without a shared family was found */
    uint32_t wang_swaps;   /* transpositions made by the pairing search */
} or_record;

static void put_i128(uint64_t w[2], __int128 v)
{
    unsigned __int128 u = (unsigned __int128)v;
    w[0] = (uint64_t)u;
    w[1] = (uint64_t)(u >> 64);
}

static __int128 get_i128(const uint64_t w[2])
{
    return (__int128)(((unsigned __int128)w[1] << 64) | (unsigned __int128)w[0]);
}

typedef struct {
    or_desc d;
    double *beta;
    uint32_t L, N;
    int8_t *s;             /* [R_cap][N] spins +1/-1 */
    int8_t *s_tmp;
    int32_t *E, *M, *E_tmp, *M_tmp;
    uint32_t *fam, *fam_tmp;
    uint32_t *r;           /* copy counts of the last resampling */
    int8_t *Jr, *Jd;       /* couplings to the right / lower neighbour */
    uint32_t R_cur;
    uint32_t step;
    uint32_t status;
    or_record *rec;        /* [n_beta] */
    uint32_t *qhist;       /* [n_beta][N+1] index-shift overlap histogram over d */
    uint32_t *qhist_pair;  /* [n_beta][N+1] */
    uint32_t *qhist_wang;  /* [n_beta][N+1] Wang-pairing overlap histogram */
} or_run;

/* ------------------------------------------------------------------------- */
/* Lattice and Hamiltonian, Sec. III.A.  Site i = y*L + x, periodic.         */
/* ------------------------------------------------------------------------- */
static uint32_t site(uint32_t L, int x, int y)
{
    int Li = (int)L;
    x = ((x % Li) + Li) % Li;
    y = ((y % Li) + Li) % Li;
    return (uint32_t)(y * Li + x);
}

/* H = - sum_<mn> J_mn s_m s_n, every bond counted once via (right, down). */
int64_t or_energy(uint32_t L, const int8_t *s, const int8_t *Jr, const int8_t *Jd)
{
    int64_t H = 0;
    for (uint32_t y = 0; y < L; ++y)
        for (uint32_t x = 0; x < L; ++x) {
            uint32_t i = y * L + x;
            H -= (int64_t)Jr[i] * s[i] * s[site(L, (int)x + 1, (int)y)];
            H -= (int64_t)Jd[i] * s[i] * s[site(L, (int)x, (int)y + 1)];
        }
    return H;
}

int64_t or_magnetisation(uint32_t N, const int8_t *s)
{
    int64_t m = 0;
    for (uint32_t i = 0; i < N; ++i) m += s[i];
    return m;
}

/* Couplings: ferromagnet J = +1 everywhere; EA glass J = +-1 equiprobable. */
void or_couplings(uint32_t L, uint32_t model, uint32_t seed, uint32_t disorder_id, int8_t *Jr, int8_t *Jd)
{
    uint32_t N = L * L;
    for (uint32_t i = 0; i < N; ++i) {
        if (model == 0) {
            Jr[i] = 1;
            Jd[i] = 1;
        } else {
            uint32_t w = philox_word(seed, disorder_id, i >> 2, 0, 0, OR_TAG_DISORDER << 24, i & 3);
            Jr[i] = (w >> 31) & 1u ? 1 : -1;
            Jd[i] = (w >> 30) & 1u ? 1 : -1;
        }
    }
}

/* Energy change of flipping site (x, y): dE = 2 s_i sum_nbr J s_nbr. */
static int32_t flip_dE(uint32_t L, const int8_t *s, const int8_t *Jr, const int8_t *Jd, uint32_t x, uint32_t y)
{
    uint32_t i = site(L, (int)x, (int)y);
    uint32_t r = site(L, (int)x + 1, (int)y), l = site(L, (int)x - 1, (int)y);
    uint32_t d = site(L, (int)x, (int)y + 1), u = site(L, (int)x, (int)y - 1);
    int32_t h = Jr[i] * s[r] + Jr[l] * s[l] + Jd[i] * s[d] + Jd[u] * s[u];
    return 2 * s[i] * h;
}

/* ------------------------------------------------------------------------- */
/* Metropolis thresholds: accept a move with dE > 0 iff u < T[dE/4], where    */
/* u is a uniform 32-bit integer and T[m] = floor(exp(-4 m beta) * 2^32)      */
/* (capped at 2^32).  Moves with dE <= 0 are always accepted.  This is the    */
/* Metropolis rule min(1, exp(-beta dE)) quantised to 2^-32.                  */
/* ------------------------------------------------------------------------- */
uint64_t or_metropolis_threshold(double beta, int m)
{
    double p = exp(-(double)(4 * m) * beta);
    if (p >= 1.0) return (uint64_t)1 << 32;
    return (uint64_t)(p * 4294967296.0);
}

/* theta checkerboard sweeps of one lattice s (child replica j of run `run_id`)
 * at temperature index `step` with inverse temperature beta (Sec. V.A.1:
 * single-spin-flip Metropolis; colour 0 = sites with x+y even, then colour 1).
 * E and M are updated incrementally. */
void or_sweep_lattice(uint32_t L, int8_t *s, const int8_t *Jr, const int8_t *Jd, double beta, uint32_t theta,
                      uint32_t seed, uint32_t run_id, uint32_t j, uint32_t step, int32_t *E, int32_t *M)
{
    uint64_t T[3];
    T[0] = (uint64_t)1 << 32;
    T[1] = or_metropolis_threshold(beta, 1);
    T[2] = or_metropolis_threshold(beta, 2);
    for (uint32_t t = 0; t < theta; ++t)
        for (uint32_t colour = 0; colour < 2; ++colour)
            for (uint32_t y = 0; y < L; ++y)
                for (uint32_t x = 0; x < L; ++x) {
                    if (((x + y) & 1u) != colour) continue;
                    uint32_t i = y * L + x;
                    uint32_t k = i >> 1; /* index within the colour's sublattice */
                    int32_t dE = flip_dE(L, s, Jr, Jd, x, y);
                    uint32_t u = philox_word(seed, run_id, k >> 2, j, step, (OR_TAG_SWEEP << 24) | (t << 1) | colour,
                                             k & 3);
                    int accept = (dE <= 0) || ((uint64_t)u < T[dE / 4]);
                    if (accept) {
                        *M -= 2 * s[i];
                        s[i] = (int8_t)(-s[i]);
                        *E += dE;
                    }
                }
}

static void sweep_replica(or_run *a, uint32_t j, uint32_t step)
{
    or_sweep_lattice(a->L, a->s + (size_t)j * a->N, a->Jr, a->Jd, a->beta[step], a->d.theta, a->d.seed,
                     a->d.run_id, j, step, &a->E[j], &a->M[j]);
}

/* ------------------------------------------------------------------------- */
/* Measurement at beta_i, Sec. III.B-D and Eq. rho_t.                         */
/* ------------------------------------------------------------------------- */
static uint32_t hamming(const int8_t *a, const int8_t *b, uint32_t N)
{
    uint32_t d = 0;
    for (uint32_t n = 0; n < N; ++n) d += (a[n] != b[n]);
    return d;
}

/* Independent pairings from permutations (Sec. III.D, the method of Wang et al.
 * with the random search pattern sigma).  A random permutation of 0..R-1 lists
 * the replica indices j in ascending order of 64-bit keys drawn per replica, the
 * low 13 bits of each key replaced by j (so no two keys tie). */
static int cmp_u64(const void *x, const void *y)
{
    uint64_t u = *(const uint64_t *)x, v = *(const uint64_t *)y;
    return u < v ? -1 : u > v ? 1 : 0;
}

static void wang_permutation(uint32_t seed, uint32_t run_id, uint32_t step, uint32_t R, int which, uint32_t *out,
                             uint64_t *tmp)
{
    const uint64_t mask = ((uint64_t)1 << OR_WANG_IDX_BITS) - 1;
    for (uint32_t j = 0; j < R; ++j) {
        uint32_t ctr[4] = {j, 0, step, OR_TAG_WANG << 24}, key[2] = {seed, run_id}, o[4];
        or_philox4x32_10(ctr, key, o);
        uint64_t k = which ? ((uint64_t)o[2] << 32 | o[3]) : ((uint64_t)o[0] << 32 | o[1]);
        tmp[j] = (k & ~mask) | j;
    }
    qsort(tmp, R, sizeof(uint64_t), cmp_u64);
    for (uint32_t k = 0; k < R; ++k) out[k] = (uint32_t)(tmp[k] & mask);
}

/* Starting from a random permutation pi, visit the positions k = sigma_0,
 * sigma_1, ... (sigma a second random permutation); where replica k and pi_k
 * share a family, try the positions p = sigma_{i+1}, sigma_{i+2}, ... (indices
 * mod R) until pi_p is not in k's family and pi_k is not in p's family, then
 * swap pi_k and pi_p.  A swap leaves both positions without a shared family and
 * changes no other, so one pass suffices.  Returns 1 with pi = pi*, or 0 if a
 * search tried all R - 1 positions in vain (possible once a family holds more
 * than R/2 replicas); *swaps counts the swaps made.  f: family of each replica;
 * the keys come from (seed, run_id) at temperature index `step`. */
int or_wang_pairing(uint32_t seed, uint32_t run_id, uint32_t step, uint32_t R, const uint32_t *f, uint32_t *pi,
                    uint32_t *swaps)
{
    if (R > (1u << OR_WANG_IDX_BITS)) return 0;
    uint32_t *sigma = (uint32_t *)malloc(sizeof(uint32_t) * R);
    uint64_t *tmp = (uint64_t *)malloc(sizeof(uint64_t) * R);
    int ok = sigma && tmp;
    *swaps = 0;
    if (ok) {
        wang_permutation(seed, run_id, step, R, 0, pi, tmp);
        wang_permutation(seed, run_id, step, R, 1, sigma, tmp);
        for (uint32_t i = 0; i < R && ok; ++i) {
            uint32_t k = sigma[i];
            if (f[pi[k]] != f[k]) continue;
            int found = 0;
            for (uint32_t l = 1; l < R; ++l) {
                uint32_t p = sigma[(i + l) % R];
                if (f[pi[p]] != f[k] && f[pi[k]] != f[p]) {
                    uint32_t t = pi[k];
                    pi[k] = pi[p];
                    pi[p] = t;
                    *swaps += 1;
                    found = 1;
                    break;
                }
            }
            ok = found;
        }
    }
    free(sigma);
    free(tmp);
    return ok;
}

static void measure(or_run *a, uint32_t step)
{
    or_record *rc = &a->rec[step];
    uint32_t N = a->N, R = a->R_cur;
    rc->beta = a->beta[step];
    rc->R = R;
    rc->R_target = a->d.R;
    rc->N = N;
    rc->sumE = rc->sumE2 = rc->sumAbsM = rc->sumM2 = 0;
    __int128 sE3 = 0, sE4 = 0, sAM3 = 0, sM4 = 0;
    for (uint32_t j = 0; j < R; ++j) {
        int64_t e = a->E[j], m = a->M[j];
        int64_t am = m < 0 ? -m : m;
        rc->sumE += e;
        rc->sumE2 += e * e;
        rc->sumAbsM += am;
        rc->sumM2 += m * m;
        __int128 E = e, A = am;
        sE3 += E * E * E;
        sE4 += E * E * E * E;
        sAM3 += A * A * A;
        sM4 += A * A * A * A;
    }
    put_i128(rc->sumE3, sE3);
    put_i128(rc->sumE4, sE4);
    put_i128(rc->sumAbsM3, sAM3);
    put_i128(rc->sumM4, sM4);
    /* families: runs of equal ancestor id (copies are placed contiguously) */
    rc->sum_c2 = 0;
    rc->n_fam = 0;
    rc->max_fam = 0;
    uint32_t j = 0;
    while (j < R) {
        uint32_t e = j;
        while (e < R && a->fam[e] == a->fam[j]) ++e;
        uint64_t c = e - j;
        rc->sum_c2 += (int64_t)(c * c);
        rc->n_fam += 1;
        if (c > rc->max_fam) rc->max_fam = (uint32_t)c;
        j = e;
    }
    /* index-shift pairs j <-> j + floor(R/2), Sec. III.D */
    rc->n_q = 0;
    rc->sum_absq = 0;
    if (a->d.overlap & 1u) {
        uint32_t *hist = a->qhist + (size_t)step * (N + 1);
        memset(hist, 0, sizeof(uint32_t) * (N + 1));
        uint32_t h = R / 2;
        for (uint32_t p = 0; p < h; ++p) {
            uint32_t dd = hamming(a->s + (size_t)p * N, a->s + (size_t)(p + h) * N, N);
            hist[dd] += 1;
            int64_t qn = (int64_t)N - 2 * (int64_t)dd;
            rc->sum_absq += qn < 0 ? -qn : qn;
        }
        rc->n_q = h;
    }
    /* Wang pairs (k, pi*_k), k = 0..R-1: every replica used twice */
    rc->n_q_wang = 0;
    rc->sum_absq_wang = 0;
    rc->wang_swaps = 0;
    if (a->d.overlap & 4u) {
        uint32_t *hist = a->qhist_wang + (size_t)step * (N + 1);
        memset(hist, 0, sizeof(uint32_t) * (N + 1));
        uint32_t *pi = (uint32_t *)malloc(sizeof(uint32_t) * (R ? R : 1));
        if (pi && or_wang_pairing(a->d.seed, a->d.run_id, step, R, a->fam, pi, &rc->wang_swaps)) {
            for (uint32_t k = 0; k < R; ++k) {
                uint32_t dd = hamming(a->s + (size_t)k * N, a->s + (size_t)pi[k] * N, N);
                hist[dd] += 1;
                int64_t qn = (int64_t)N - 2 * (int64_t)dd;
                rc->sum_absq_wang += qn < 0 ? -qn : qn;
            }
            rc->n_q_wang = R;
        }
        free(pi);
    }
}

/* Overlaps between two independent populations of the same disorder sample:
 * pairs A_j <-> B_j for j < min(R_A, R_B).  Recorded in both runs. */
int or_measure_pair(or_run *a, or_run *b)
{
    if (a->step != b->step || a->N != b->N) return OR_ERR_STATE;
    uint32_t N = a->N, step = a->step;
    uint32_t n = a->R_cur < b->R_cur ? a->R_cur : b->R_cur;
    uint32_t *ha = a->qhist_pair + (size_t)step * (N + 1);
    uint32_t *hb = b->qhist_pair + (size_t)step * (N + 1);
    memset(ha, 0, sizeof(uint32_t) * (N + 1));
    int64_t sum = 0;
    for (uint32_t p = 0; p < n; ++p) {
        uint32_t dd = hamming(a->s + (size_t)p * N, b->s + (size_t)p * N, N);
        ha[dd] += 1;
        int64_t qn = (int64_t)N - 2 * (int64_t)dd;
        sum += qn < 0 ? -qn : qn;
    }
    memcpy(hb, ha, sizeof(uint32_t) * (N + 1));
    a->rec[step].sum_absq_pair = b->rec[step].sum_absq_pair = sum;
    a->rec[step].n_q_pair = b->rec[step].n_q_pair = n;
    return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* Step (i): R_0 = R replicas drawn uniformly (beta_0 = 0 => uniform on      */
/* Gamma), Sec. II.A/II.B.                                                   */
/* ------------------------------------------------------------------------- */
static void free_run(or_run *a)
{
    if (!a) return;
    free(a->beta);
    free(a->s);
    free(a->s_tmp);
    free(a->E);
    free(a->M);
    free(a->E_tmp);
    free(a->M_tmp);
    free(a->fam);
    free(a->fam_tmp);
    free(a->r);
    free(a->Jr);
    free(a->Jd);
    free(a->rec);
    free(a->qhist);
    free(a->qhist_pair);
    free(a->qhist_wang);
    free(a);
}

void or_destroy(or_run *a) { free_run(a); }

/* ------------------------------------------------------------------------- */
/* theta = infinity (Sec. V.B): step (iv) replaced by simple sampling of the  */
/* exact energy distribution P_beta(E) = g(E) exp(-beta E) / Z(beta).         */
/* ------------------------------------------------------------------------- */
/* Cumulative weights over the levels u = 0..2N (E = 2u - 2N) in ascending order,
 *   C[u] = sum_{v <= u} exp(ln g(v) - beta E(v) - c),  c = max_v (ln g(v) - beta E(v)),
 * with exp(-inf) = 0 where g = 0.  Returns the last level with a positive weight. */
static uint32_t dos_cdf(const or_run *a, double beta, double *C)
{
    uint32_t U = 2 * a->N;
    double c = -INFINITY;
    for (uint32_t u = 0; u <= U; ++u)
        if (a->d.log_g[u] > -INFINITY) {
            double l = a->d.log_g[u] - beta * (double)(2 * (int64_t)u - 2 * (int64_t)a->N);
            if (l > c) c = l;
        }
    double acc = 0.0;
    uint32_t last = 0;
    for (uint32_t u = 0; u <= U; ++u) {
        double p = 0.0;
        if (a->d.log_g[u] > -INFINITY) {
            double l = a->d.log_g[u] - beta * (double)(2 * (int64_t)u - 2 * (int64_t)a->N);
            p = exp(l - c);
        }
        acc = acc + p;
        C[u] = acc;
        if (p > 0.0) last = u;
    }
    return last;
}

/* One energy from P_beta: the first level u with x < C[u], x a 53-bit uniform
 * (words 0 and 1 of the replica's draw) times C[2N]; the last positive level if x
 * rounds up to C[2N]. */
static int32_t dos_draw(const or_run *a, const double *C, uint32_t last, uint32_t step, uint32_t j)
{
    uint32_t U = 2 * a->N;
    uint32_t ctr[4] = {j, 0, step, OR_TAG_DOS << 24}, key[2] = {a->d.seed, a->d.run_id}, o[4];
    or_philox4x32_10(ctr, key, o);
    uint64_t u53 = ((uint64_t)(o[0] >> 5) << 26) | (uint64_t)(o[1] >> 6);
    double x = (double)u53 * (1.0 / 9007199254740992.0) * C[U];
    uint32_t lev = last;
    for (uint32_t u = 0; u <= U; ++u)
        if (x < C[u]) {
            lev = u;
            break;
        }
    return (int32_t)(2 * (int64_t)lev - 2 * (int64_t)a->N);
}

/* Fresh energies for replicas 0..R-1 at beta_step; their spins are not
 * represented (left at -1) and M = 0. */
static int dos_resample_energies(or_run *a, uint32_t step, uint32_t R)
{
    double *C = (double *)malloc(sizeof(double) * (2 * a->N + 1));
    if (!C) return OR_ERR_OOM;
    uint32_t last = dos_cdf(a, a->beta[step], C);
    for (uint32_t j = 0; j < R; ++j) {
        a->E[j] = dos_draw(a, C, last, step, j);
        a->M[j] = 0;
    }
    free(C);
    return OR_OK;
}

or_run *or_create(const or_desc *d, int *status)
{
    *status = OR_ERR_INVALID;
    if (d->L < 4 || (d->L & 1u) || d->R < 1 || d->R_cap < d->R || d->n_beta < 1 || !d->beta) return NULL;
    if (d->theta == OR_THETA_INF && (!d->log_g || d->overlap)) return NULL;
    if ((d->overlap & 4u) && d->R_cap > (1u << OR_WANG_IDX_BITS)) return NULL;
    for (uint32_t i = 1; i < d->n_beta; ++i)
        if (!(d->beta[i] >= d->beta[i - 1])) return NULL;
    or_run *a = (or_run *)calloc(1, sizeof(or_run));
    if (!a) {
        *status = OR_ERR_OOM;
        return NULL;
    }
    a->d = *d;
    a->L = d->L;
    a->N = d->L * d->L;
    uint32_t N = a->N, C = d->R_cap;
    a->beta = (double *)malloc(sizeof(double) * d->n_beta);
    a->s = (int8_t *)malloc((size_t)C * N);
    a->s_tmp = (int8_t *)malloc((size_t)C * N);
    a->E = (int32_t *)malloc(sizeof(int32_t) * C);
    a->M = (int32_t *)malloc(sizeof(int32_t) * C);
    a->E_tmp = (int32_t *)malloc(sizeof(int32_t) * C);
    a->M_tmp = (int32_t *)malloc(sizeof(int32_t) * C);
    a->fam = (uint32_t *)malloc(sizeof(uint32_t) * C);
    a->fam_tmp = (uint32_t *)malloc(sizeof(uint32_t) * C);
    a->r = (uint32_t *)calloc(C, sizeof(uint32_t));
    a->Jr = (int8_t *)malloc(N);
    a->Jd = (int8_t *)malloc(N);
    a->rec = (or_record *)calloc(d->n_beta, sizeof(or_record));
    a->qhist = (uint32_t *)calloc((size_t)d->n_beta * (N + 1), sizeof(uint32_t));
    a->qhist_pair = (uint32_t *)calloc((size_t)d->n_beta * (N + 1), sizeof(uint32_t));
    a->qhist_wang = (uint32_t *)calloc((size_t)d->n_beta * (N + 1), sizeof(uint32_t));
    if (!a->beta || !a->s || !a->s_tmp || !a->E || !a->M || !a->E_tmp || !a->M_tmp || !a->fam ||
        !a->fam_tmp || !a->r || !a->Jr || !a->Jd || !a->rec || !a->qhist || !a->qhist_pair ||
        !a->qhist_wang) {
        free_run(a);
        *status = OR_ERR_OOM;
        return NULL;
    }
    memcpy(a->beta, d->beta, sizeof(double) * d->n_beta);
    a->d.beta = a->beta;
    or_couplings(a->L, d->model, d->seed, d->disorder_id, a->Jr, a->Jd);
    if (d->theta == OR_THETA_INF) {
        /* beta_0 = 0 population as energies drawn from g(E) / 2^N */
        memset(a->s, -1, (size_t)C * N);
        memset(a->s_tmp, -1, (size_t)C * N);
        if (dos_resample_energies(a, 0, d->R) != OR_OK) {
            free_run(a);
            *status = OR_ERR_OOM;
            return NULL;
        }
        for (uint32_t j = 0; j < d->R; ++j) a->fam[j] = j;
    }
    for (uint32_t j = 0; j < d->R && d->theta != OR_THETA_INF; ++j) {
        int8_t *s = a->s + (size_t)j * N;
        for (uint32_t i = 0; i < N; ++i) {
            uint32_t w = philox_word(d->seed, d->run_id, i >> 2, j, 0, OR_TAG_INIT << 24, i & 3);
            s[i] = (w >> 31) ? 1 : -1;
        }
        a->E[j] = (int32_t)or_energy(a->L, s, a->Jr, a->Jd);
        a->M[j] = (int32_t)or_magnetisation(N, s);
        a->fam[j] = j;
    }
    a->R_cur = d->R;
    a->step = 0;
    a->rec[0].lnQ = 0.0;
    a->rec[0].minus_betaF = (double)N * log(2.0); /* ln Z(beta_0 = 0) = N ln 2 */
    measure(a, 0);
    *status = OR_OK;
    return a;
}

/* ------------------------------------------------------------------------- */
/* Steps (ii)-(v) for one temperature, canonical form (Eqs. tauBoltz, QBoltz)*/
/* ------------------------------------------------------------------------- */
int or_step(or_run *a)
{
    if (a->status != OR_OK) return (int)a->status;
    if (a->step + 1 >= a->d.n_beta) return OR_ERR_STATE;
    uint32_t i = a->step + 1, N = a->N, Rprev = a->R_cur;
    double dbeta = a->beta[i] - a->beta[i - 1];

    /* energies relative to the lowest one: level n_j = (E_j - E_min)/4, so that
     * exp(-dbeta E_j) = exp(-dbeta E_min) * w[n_j] with w[n] = exp(-4 n dbeta). */
    int32_t Emin = a->E[0];
    for (uint32_t j = 1; j < Rprev; ++j)
        if (a->E[j] < Emin) Emin = a->E[j];
    uint32_t *h = (uint32_t *)calloc(N + 1, sizeof(uint32_t));
    double *w = (double *)malloc(sizeof(double) * (N + 1));
    if (!h || !w) {
        free(h);
        free(w);
        return OR_ERR_OOM;
    }
    for (uint32_t n = 0; n <= N; ++n) w[n] = exp(-(double)(4 * n) * dbeta);
    for (uint32_t j = 0; j < Rprev; ++j) {
        int32_t diff = a->E[j] - Emin;
        if (diff % 4 != 0) {
            free(h);
            free(w);
            return OR_ERR_STATE;
        }
        h[diff / 4] += 1;
    }
    /* S = sum_j exp(-dbeta (E_j - E_min)), summed level by level in ascending order */
    double S = 0.0;
    for (uint32_t n = 0; n <= N; ++n) S = S + (double)h[n] * w[n];
    /* Eq. QBoltz: Q_i = (1/R_{i-1}) sum_j exp(-dbeta E_j) */
    double lnQ = -dbeta * (double)Emin + log(S) - log((double)Rprev);

    /* Step (iii): copy numbers r_j with mean tau_j (Eq. tauBoltz):
     * tau_j = (R/R_{i-1}) (1/Q_i) exp(-dbeta E_j) = R w[n_j] / S. */
    uint32_t Rnew = 0;
    if (a->d.resample == 0) {
        /* nearest-integer resampling: ceil(tau) with probability tau - floor(tau) */
        for (uint32_t j = 0; j < Rprev; ++j) {
            double tau = ((double)a->d.R * w[(a->E[j] - Emin) / 4]) / S;
            double fl = floor(tau);
            uint32_t u = philox_word(a->d.seed, a->d.run_id, j, 0, i, OR_TAG_RESAMPLE << 24, 0);
            double uf = (double)u * (1.0 / 4294967296.0);
            a->r[j] = (uint32_t)fl + (uf < tau - fl ? 1u : 0u);
            Rnew += a->r[j];
        }
    } else {
        /* multinomial resampling: R independent draws with probability
         * proportional to exp(-dbeta E_j); each draw picks an energy level from
         * the cumulative level weights (ascending order), then a member of that
         * level uniformly, members ordered by replica index. */
        double *cdf = (double *)malloc(sizeof(double) * (N + 1));
        uint32_t *first = (uint32_t *)malloc(sizeof(uint32_t) * (N + 1));
        uint32_t *members = (uint32_t *)malloc(sizeof(uint32_t) * (Rprev ? Rprev : 1));
        if (!cdf || !first || !members) {
            free(cdf);
            free(first);
            free(members);
            free(h);
            free(w);
            return OR_ERR_OOM;
        }
        double acc = 0.0;
        uint32_t pos = 0;
        for (uint32_t n = 0; n <= N; ++n) {
            acc = acc + (double)h[n] * w[n];
            cdf[n] = acc;
            first[n] = pos;
            pos += h[n];
        }
        /* stable list of replicas by level */
        uint32_t *fill = (uint32_t *)calloc(N + 1, sizeof(uint32_t));
        for (uint32_t j = 0; j < Rprev; ++j) {
            uint32_t n = (uint32_t)((a->E[j] - Emin) / 4);
            members[first[n] + fill[n]] = j;
            fill[n] += 1;
        }
        free(fill);
        for (uint32_t j = 0; j < Rprev; ++j) a->r[j] = 0;
        uint32_t last_level = 0;
        for (uint32_t n = 0; n <= N; ++n)
            if (h[n]) last_level = n;
        for (uint32_t dd = 0; dd < a->d.R; ++dd) {
            uint32_t ctr[4] = {dd, 0, i, OR_TAG_MULTINOMIAL << 24}, key[2] = {a->d.seed, a->d.run_id}, o[4];
            or_philox4x32_10(ctr, key, o);
            uint64_t u53 = ((uint64_t)(o[0] >> 5) << 26) | (uint64_t)(o[1] >> 6);
            double x = (double)u53 * (1.0 / 9007199254740992.0) * S;
            uint32_t lev = last_level;
            for (uint32_t n = 0; n <= N; ++n)
                if (h[n] && x < cdf[n]) {
                    lev = n;
                    break;
                }
            uint32_t idx = (uint32_t)(((uint64_t)o[2] * (uint64_t)h[lev]) >> 32);
            a->r[members[first[lev] + idx]] += 1;
        }
        Rnew = a->d.R;
        free(cdf);
        free(first);
        free(members);
    }
    free(h);
    free(w);
    if (Rnew == 0) {
        a->status = OR_ERR_EXTINCT;
        return OR_ERR_EXTINCT;
    }
    if (Rnew > a->d.R_cap) {
        a->status = OR_ERR_CAPACITY;
        return OR_ERR_CAPACITY;
    }
    /* copies of the same ancestor are placed next to each other (Sec. V.A.1) */
    uint32_t k = 0;
    for (uint32_t j = 0; j < Rprev; ++j)
        for (uint32_t c = 0; c < a->r[j]; ++c, ++k) {
            memcpy(a->s_tmp + (size_t)k * N, a->s + (size_t)j * N, N);
            a->E_tmp[k] = a->E[j];
            a->M_tmp[k] = a->M[j];
            a->fam_tmp[k] = a->fam[j];
        }
    int8_t *ts = a->s;
    a->s = a->s_tmp;
    a->s_tmp = ts;
    int32_t *tE = a->E;
    a->E = a->E_tmp;
    a->E_tmp = tE;
    int32_t *tM = a->M;
    a->M = a->M_tmp;
    a->M_tmp = tM;
    uint32_t *tf = a->fam;
    a->fam = a->fam_tmp;
    a->fam_tmp = tf;
    a->R_cur = Rnew;
    a->step = i;

    /* Step (iv): theta Metropolis sweeps at beta_i for every replica, or at
     * theta = infinity fresh energies from the exact distribution at beta_i */
    if (a->d.theta == OR_THETA_INF) {
        if (dos_resample_energies(a, i, Rnew) != OR_OK) return OR_ERR_OOM;
    } else {
        for (uint32_t j = 0; j < Rnew; ++j) sweep_replica(a, j, i);
    }

    /* Step (v): measurements at beta_i */
    a->rec[i].lnQ = lnQ;
    a->rec[i].minus_betaF = a->rec[i - 1].minus_betaF + lnQ; /* Eq. F, running sum */
    measure(a, i);
    return OR_OK;
}

/* Accessors for the tests. */
uint32_t or_current_step(const or_run *a) { return a->step; }
uint32_t or_current_R(const or_run *a) { return a->R_cur; }
void or_get_record(const or_run *a, uint32_t step, or_record *out) { *out = a->rec[step]; }
void or_get_qhist(const or_run *a, uint32_t step, uint32_t *out, uint32_t *out_pair, uint32_t *out_wang)
{
    size_t n = a->N + 1;
    if (out) memcpy(out, a->qhist + (size_t)step * n, sizeof(uint32_t) * n);
    if (out_pair) memcpy(out_pair, a->qhist_pair + (size_t)step * n, sizeof(uint32_t) * n);
    if (out_wang) memcpy(out_wang, a->qhist_wang + (size_t)step * n, sizeof(uint32_t) * n);
}
void or_get_counts(const or_run *a, uint32_t *r, uint32_t n) { memcpy(r, a->r, sizeof(uint32_t) * n); }
void or_get_population(const or_run *a, int8_t *s, int32_t *E, int32_t *M, uint32_t *fam)
{
    uint32_t R = a->R_cur;
    if (s) memcpy(s, a->s, (size_t)R * a->N);
    if (E) memcpy(E, a->E, sizeof(int32_t) * R);
    if (M) memcpy(M, a->M, sizeof(int32_t) * R);
    if (fam) memcpy(fam, a->fam, sizeof(uint32_t) * R);
}
void or_get_couplings(const or_run *a, int8_t *Jr, int8_t *Jd)
{
    memcpy(Jr, a->Jr, a->N);
    memcpy(Jd, a->Jd, a->N);
}

/* ------------------------------------------------------------------------- */
/* Weighted averages over M independent runs, Sec. IV.                        */
/* recs[m * n_steps + i], qh[(m * n_steps + i) * (N+1)] (optional; likewise  */
/* qh_pair and qh_wang, with Pq, Pq_pair, Pq_wang [n_steps][N+1] out).        */
/* kind 0: free-energy weight w (Eq. appropriateWeight);                      */
/* kind 1: simplified weight (Eq. simpleWeight, read with beta = beta_i).     */
/* ------------------------------------------------------------------------- */
typedef struct {
    double beta;
    double W_e, W_e2, W_m, W_m2;     /* Eq. W_conf applied to e, e^2, m, m^2 */
    double Wvar_c, Wvar_chi;         /* Eqs. Wvar_C, Wvar_Chi */
    double W_c, W_chi;               /* Eq. W_conf applied to c and chi */
    double W_minus_betaF;            /* Eq. W_F */
    double W_absq, W_absq_pair;      /* Eq. W_conf applied to |q| */
    double w_max;                    /* largest weight */
    double sum_w;                    /* sum of the weights (1 up to rounding) */
    double W_e3, W_e4, W_m3, W_m4;   /* Eq. W_conf applied to e^3, e^4, |m|^3, m^4 */
    double Wk3_e, Wk4_e;             /* Eq. W_k, k = 3, 4, for O = e */
    double Wk3_m, Wk4_m;             /* Eq. W_k, k = 3, 4, for O = |m| */
    double W_U4;                     /* Binder cumulant 1 - W[m^4] / (3 W[m^2]^2) */
    double W_U4_conf;                /* Eq. W_conf applied to each run's 1 - m^4 / (3 (m^2)^2) */
    double W_absq_wang;              /* Eq. W_conf applied to |q| over the Wang pairs */
} or_wavg;

/* Eq. W_k (Sec. IV.E): the k-th central moment from the weighted raw moments
 * Wl[l] = W[O^l], l = 0..k, Wl[0] = 1 (mu'_0 = 1), by the binomial expansion
 *   sum_{l=0}^{k} C(k, l) (-1)^{k-l} W[O]^{k-l} W[O^l],  terms in order l = 0..k. */
static double central_moment(int k, const double *Wl)
{
    double sum = 0.0;
    for (int l = 0; l <= k; ++l) {
        double binom = 1.0;
        for (int t = 0; t < l; ++t) binom = binom * (double)(k - t) / (double)(t + 1);
        double pw = 1.0;
        for (int t = 0; t < k - l; ++t) pw = pw * Wl[1];
        double sign = ((k - l) & 1) ? -1.0 : 1.0;
        sum = sum + sign * binom * pw * Wl[l];
    }
    return sum;
}

static double log_weight(const or_record *recs, uint32_t n_steps, uint32_t m, uint32_t i, uint32_t kind)
{
    const or_record *r = recs + (size_t)m * n_steps;
    double lam = log((double)r[i].R) + r[i].minus_betaF;
    if (kind == 0)
        for (uint32_t k = 1; k <= i; ++k) lam += log((double)r[k - 1].R / (double)r[k].R_target);
    return lam;
}

/* The exponent that or_weighted_average normalises (run m, step i), for the tests. */
double or_log_weight(const or_record *recs, uint32_t n_steps, uint32_t m, uint32_t i, uint32_t kind)
{
    return log_weight(recs, n_steps, m, i, kind);
}

int or_weighted_average(const or_record *recs, const uint32_t *qh, const uint32_t *qh_pair, const uint32_t *qh_wang,
                        uint32_t M, uint32_t n_steps, uint32_t N, uint32_t kind, or_wavg *out, double *Pq,
                        double *Pq_pair, double *Pq_wang, double *w_out /* [n_steps][M] or NULL */)
{
    if (M == 0 || n_steps == 0 || N == 0 || kind > 1) return OR_ERR_INVALID;
    double *w = (double *)malloc(sizeof(double) * M);
    double *wprev = (double *)malloc(sizeof(double) * M);
    if (!w || !wprev) {
        free(w);
        free(wprev);
        return OR_ERR_OOM;
    }
    double Nd = (double)N;
    double WF = Nd * log(2.0);
    for (uint32_t i = 0; i < n_steps; ++i) {
        /* free-energy weights at beta_i (normalised log-sum-exp over m in order) */
        double lmax = -INFINITY;
        for (uint32_t m = 0; m < M; ++m) {
            double l = log_weight(recs, n_steps, m, i, kind);
            w[m] = l;
            if (l > lmax) lmax = l;
        }
        double z = 0.0;
        for (uint32_t m = 0; m < M; ++m) {
            w[m] = exp(w[m] - lmax);
            z = z + w[m];
        }
        for (uint32_t m = 0; m < M; ++m) w[m] = w[m] / z;
        if (w_out)
            for (uint32_t m = 0; m < M; ++m) w_out[(size_t)i * M + m] = w[m];

        or_wavg *o = &out[i];
        memset(o, 0, sizeof *o);
        o->beta = recs[i].beta;
        double beta = o->beta;
        for (uint32_t m = 0; m < M; ++m) {
            const or_record *r = &recs[(size_t)m * n_steps + i];
            double Ri = (double)r->R;
            double e = (double)r->sumE / (Nd * Ri);
            double e2 = (double)r->sumE2 / (Nd * Nd * Ri);
            double mm = (double)r->sumAbsM / (Nd * Ri);
            double m2 = (double)r->sumM2 / (Nd * Nd * Ri);
            double c = beta * beta * Nd * (e2 - e * e); /* Eq. c */
            double chi = beta * Nd * (m2 - mm * mm);    /* Eq. chi */
            o->W_e += w[m] * e;
            o->W_e2 += w[m] * e2;
            o->W_m += w[m] * mm;
            o->W_m2 += w[m] * m2;
            o->W_c += w[m] * c;
            o->W_chi += w[m] * chi;
            double e3 = (double)get_i128(r->sumE3) / (Nd * Nd * Nd * Ri);
            double e4 = (double)get_i128(r->sumE4) / (Nd * Nd * Nd * Nd * Ri);
            double m3 = (double)get_i128(r->sumAbsM3) / (Nd * Nd * Nd * Ri);
            double m4 = (double)get_i128(r->sumM4) / (Nd * Nd * Nd * Nd * Ri);
            o->W_e3 += w[m] * e3;
            o->W_e4 += w[m] * e4;
            o->W_m3 += w[m] * m3;
            o->W_m4 += w[m] * m4;
            o->W_U4_conf += w[m] * (1.0 - m4 / (3.0 * m2 * m2)); /* NaN if a run has M = 0 throughout */
            if (r->n_q) o->W_absq += w[m] * ((double)r->sum_absq / (Nd * (double)r->n_q));
            if (r->n_q_pair) o->W_absq_pair += w[m] * ((double)r->sum_absq_pair / (Nd * (double)r->n_q_pair));
            if (r->n_q_wang) o->W_absq_wang += w[m] * ((double)r->sum_absq_wang / (Nd * (double)r->n_q_wang));
            o->sum_w += w[m];
            if (w[m] > o->w_max) o->w_max = w[m];
        }
        o->Wvar_c = beta * beta * Nd * (o->W_e2 - o->W_e * o->W_e);
        o->Wvar_chi = beta * Nd * (o->W_m2 - o->W_m * o->W_m);
        {
            double We[5] = {1.0, o->W_e, o->W_e2, o->W_e3, o->W_e4};
            double Wm[5] = {1.0, o->W_m, o->W_m2, o->W_m3, o->W_m4};
            o->Wk3_e = central_moment(3, We);
            o->Wk4_e = central_moment(4, We);
            o->Wk3_m = central_moment(3, Wm);
            o->Wk4_m = central_moment(4, Wm);
            o->W_U4 = 1.0 - o->W_m4 / (3.0 * o->W_m2 * o->W_m2);
        }
        /* Eq. W_F: -beta_i W[F_i] = sum_{k<=i} ln W[Q_k] + ln Z(0), W[Q_k] = sum_m w_{k-1} Q_k */
        if (i > 0) {
            double lm = -INFINITY;
            for (uint32_t m = 0; m < M; ++m) {
                double l = log(wprev[m]) + recs[(size_t)m * n_steps + i].lnQ;
                if (l > lm) lm = l;
            }
            double zz = 0.0;
            for (uint32_t m = 0; m < M; ++m) zz = zz + exp(log(wprev[m]) + recs[(size_t)m * n_steps + i].lnQ - lm);
            WF = WF + (lm + log(zz));
        }
        o->W_minus_betaF = WF;
        /* Eq. W_conf_q: weighted overlap distribution over d = N(1-q)/2 */
        if (Pq && qh) {
            double *P = Pq + (size_t)i * (N + 1);
            for (uint32_t dd = 0; dd <= N; ++dd) P[dd] = 0.0;
            for (uint32_t m = 0; m < M; ++m) {
                const or_record *r = &recs[(size_t)m * n_steps + i];
                if (!r->n_q) continue;
                const uint32_t *hq = qh + ((size_t)m * n_steps + i) * (N + 1);
                for (uint32_t dd = 0; dd <= N; ++dd) P[dd] += w[m] * ((double)hq[dd] / (double)r->n_q);
            }
        }
        if (Pq_pair && qh_pair) {
            double *P = Pq_pair + (size_t)i * (N + 1);
            for (uint32_t dd = 0; dd <= N; ++dd) P[dd] = 0.0;
            for (uint32_t m = 0; m < M; ++m) {
                const or_record *r = &recs[(size_t)m * n_steps + i];
                if (!r->n_q_pair) continue;
                const uint32_t *hq = qh_pair + ((size_t)m * n_steps + i) * (N + 1);
                for (uint32_t dd = 0; dd <= N; ++dd) P[dd] += w[m] * ((double)hq[dd] / (double)r->n_q_pair);
            }
        }
        if (Pq_wang && qh_wang) {
            double *P = Pq_wang + (size_t)i * (N + 1);
            for (uint32_t dd = 0; dd <= N; ++dd) P[dd] = 0.0;
            for (uint32_t m = 0; m < M; ++m) {
                const or_record *r = &recs[(size_t)m * n_steps + i];
                if (!r->n_q_wang) continue;
                const uint32_t *hq = qh_wang + ((size_t)m * n_steps + i) * (N + 1);
                for (uint32_t dd = 0; dd <= N; ++dd) P[dd] += w[m] * ((double)hq[dd] / (double)r->n_q_wang);
            }
        }
        for (uint32_t m = 0; m < M; ++m) wprev[m] = w[m];
    }
    free(w);
    free(wprev);
    return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* Exact solvers (pins).                                                     */
/* ------------------------------------------------------------------------- */

/* Brute-force enumeration over all 2^N states (N <= 24): ln Z, <e>, c, <|m|>,
 * chi (Eqs. e, m, c, chi with ensemble averages) and the exact energy
 * distribution.  Returns OR_ERR_INVALID if N > 24. */
int or_bruteforce(uint32_t L, const int8_t *Jr, const int8_t *Jd, double beta, double *lnZ, double *e_avg,
                  double *c, double *absm_avg, double *chi, double *pE /* [N+1] by level (E+2N)/4 or NULL */)
{
    uint32_t N = L * L;
    if (N > 24) return OR_ERR_INVALID;
    int8_t s[24];
    long double Emin = 0;
    /* first pass: minimum energy for a stable log-sum-exp */
    int64_t Elo = INT64_MAX;
    for (uint64_t st = 0; st < ((uint64_t)1 << N); ++st) {
        for (uint32_t i = 0; i < N; ++i) s[i] = (st >> i) & 1u ? 1 : -1;
        int64_t E = or_energy(L, s, Jr, Jd);
        if (E < Elo) Elo = E;
    }
    Emin = (long double)Elo;
    long double Z = 0, sE = 0, sE2 = 0, sM = 0, sM2 = 0;
    if (pE)
        for (uint32_t n = 0; n <= N; ++n) pE[n] = 0;
    long double *pl = (long double *)calloc(N + 1, sizeof(long double));
    for (uint64_t st = 0; st < ((uint64_t)1 << N); ++st) {
        for (uint32_t i = 0; i < N; ++i) s[i] = (st >> i) & 1u ? 1 : -1;
        int64_t E = or_energy(L, s, Jr, Jd);
        int64_t Mg = or_magnetisation(N, s);
        long double b = expl(-(long double)beta * ((long double)E - Emin));
        Z += b;
        sE += b * (long double)E;
        sE2 += b * (long double)E * (long double)E;
        long double am = (long double)(Mg < 0 ? -Mg : Mg);
        sM += b * am;
        sM2 += b * am * am;
        if (pl) pl[(uint32_t)((E + 2 * (int64_t)N) / 4)] += b;
    }
    long double Nl = (long double)N;
    long double e1 = sE / Z / Nl, e2 = sE2 / Z / (Nl * Nl);
    long double m1 = sM / Z / Nl, m2 = sM2 / Z / (Nl * Nl);
    *lnZ = (double)(logl(Z) - (long double)beta * Emin);
    *e_avg = (double)e1;
    *c = (double)((long double)beta * beta * Nl * (e2 - e1 * e1));
    *absm_avg = (double)m1;
    *chi = (double)((long double)beta * Nl * (m2 - m1 * m1));
    if (pE && pl)
        for (uint32_t n = 0; n <= N; ++n) pE[n] = (double)(pl[n] / Z);
    free(pl);
    return OR_OK;
}

/* Brute-force enumeration of the Boltzmann moments that the central-moment and
 * Binder estimators of Sec. IV.E target: out[k-1] = <e^k>, out[3+k] = <|m|^k>
 * for k = 1..4 (e = H/N, m = M/N), in long double.  N <= 24. */
int or_bruteforce_moments(uint32_t L, const int8_t *Jr, const int8_t *Jd, double beta, double out[8])
{
    uint32_t N = L * L;
    if (N > 24) return OR_ERR_INVALID;
    int8_t s[24];
    int64_t Elo = INT64_MAX;
    for (uint64_t st = 0; st < ((uint64_t)1 << N); ++st) {
        for (uint32_t i = 0; i < N; ++i) s[i] = (st >> i) & 1u ? 1 : -1;
        int64_t E = or_energy(L, s, Jr, Jd);
        if (E < Elo) Elo = E;
    }
    long double Z = 0, se[4] = {0, 0, 0, 0}, sm[4] = {0, 0, 0, 0};
    long double Nl = (long double)N;
    for (uint64_t st = 0; st < ((uint64_t)1 << N); ++st) {
        for (uint32_t i = 0; i < N; ++i) s[i] = (st >> i) & 1u ? 1 : -1;
        int64_t E = or_energy(L, s, Jr, Jd);
        int64_t Mg = or_magnetisation(N, s);
        long double b = expl(-(long double)beta * (long double)(E - Elo));
        long double e = (long double)E / Nl, am = (long double)(Mg < 0 ? -Mg : Mg) / Nl;
        long double pe = 1, pm = 1;
        Z += b;
        for (int k = 0; k < 4; ++k) {
            pe *= e;
            pm *= am;
            se[k] += b * pe;
            sm[k] += b * pm;
        }
    }
    for (int k = 0; k < 4; ++k) {
        out[k] = (double)(se[k] / Z);
        out[4 + k] = (double)(sm[k] / Z);
    }
    return OR_OK;
}

/* Kaufman's exact partition function of the L x L periodic Ising ferromagnet
 * (B. Kaufman, Phys. Rev. 76, 1232 (1949)):
 *   Z = 1/2 (2 sinh 2K)^{N/2} (Z1 + Z2 + Z3 + Z4),
 *   Z1 = prod_{r=0}^{L-1} 2 cosh(L g_{2r+1}/2),  Z2 = prod 2 sinh(L g_{2r+1}/2),
 *   Z3 = prod_{r=0}^{L-1} 2 cosh(L g_{2r}/2),    Z4 = prod 2 sinh(L g_{2r}/2),
 *   cosh g_k = cosh 2K coth 2K - cos(pi k / L) (k >= 1),  g_0 = 2K + ln tanh K.
 * Evaluated in long double with signed logarithms.  Returns ln Z. */
double or_kaufman_lnZ(uint32_t L, double Kd)
{
    long double K = (long double)Kd;
    long double pi = 3.141592653589793238462643383279502884L;
    long double c2 = coshl(2 * K) / tanhl(2 * K);
    long double l1 = 0, l2 = 0, l3 = 0, l4 = 0; /* log |Z_l| */
    int sg4 = 1;
    for (uint32_t r = 0; r < L; ++r) {
        long double go = acoshl(c2 - cosl(pi * (long double)(2 * r + 1) / (long double)L));
        long double ge;
        if (r == 0)
            ge = 2 * K + logl(tanhl(K));
        else
            ge = acoshl(c2 - cosl(pi * (long double)(2 * r) / (long double)L));
        long double xo = (long double)L * go / 2, xe = (long double)L * ge / 2;
        l1 += logl(2 * coshl(xo));
        l2 += logl(2 * sinhl(xo));
        l3 += logl(2 * coshl(xe));
        long double s4 = 2 * sinhl(xe);
        if (s4 < 0) {
            sg4 = -sg4;
            s4 = -s4;
        }
        l4 += logl(s4);
    }
    long double top = l1;
    if (l2 > top) top = l2;
    if (l3 > top) top = l3;
    if (l4 > top) top = l4;
    long double sum = expl(l1 - top) + expl(l2 - top) + expl(l3 - top) + (long double)sg4 * expl(l4 - top);
    long double lnZ = -logl(2.0L) + ((long double)(L * L) / 2) * logl(2 * sinhl(2 * K)) + top + logl(sum);
    return (double)lnZ;
}

/* Transfer-matrix density of states g(E) of the L x L periodic lattice with
 * couplings (Jr, Jd), built row by row for every fixed first row (L <= 10).
 * E = -2N + 4 n for the FM; in general out[n] counts states with
 * (E + 2N)/2 = n (levels of 2, n in [0, 2N]).  Exact in unsigned 128-bit
 * integers; returned as pairs (low 64 bits, high 64 bits). */
int or_dos_transfer(uint32_t L, const int8_t *Jr, const int8_t *Jd, uint64_t *out_lo, uint64_t *out_hi)
{
    if (L < 2 || L > 10) return OR_ERR_INVALID;
    uint32_t N = L * L, S = 1u << L, NE = 2 * N + 1; /* index (E + 2N)/2 */
    typedef unsigned __int128 u128;
    u128 *cur = (u128 *)calloc((size_t)S * NE, sizeof(u128));
    u128 *nxt = (u128 *)calloc((size_t)S * NE, sizeof(u128));
    u128 *tot = (u128 *)calloc(NE, sizeof(u128));
    if (!cur || !nxt || !tot) {
        free(cur);
        free(nxt);
        free(tot);
        return OR_ERR_OOM;
    }
    /* energy of horizontal bonds inside row y for row state a, and of vertical
     * bonds between row y (state a) and row y+1 (state b) */
#define SPIN(st, x) (((st) >> (x)) & 1u ? 1 : -1)
    for (uint32_t f = 0; f < S; ++f) {
        memset(cur, 0, sizeof(u128) * (size_t)S * NE);
        int Eh = 0;
        for (uint32_t x = 0; x < L; ++x) Eh -= Jr[x] * SPIN(f, x) * SPIN(f, (x + 1) % L);
        cur[(size_t)f * NE + (uint32_t)((Eh + 2 * (int)N) / 2)] = 1;
        for (uint32_t y = 0; y + 1 < L; ++y) {
            memset(nxt, 0, sizeof(u128) * (size_t)S * NE);
            for (uint32_t a = 0; a < S; ++a)
                for (uint32_t b = 0; b < S; ++b) {
                    int dE = 0;
                    for (uint32_t x = 0; x < L; ++x) {
                        dE -= Jd[y * L + x] * SPIN(a, x) * SPIN(b, x);
                        dE -= Jr[(y + 1) * L + x] * SPIN(b, x) * SPIN(b, (x + 1) % L);
                    }
                    u128 *src = cur + (size_t)a * NE;
                    u128 *dst = nxt + (size_t)b * NE;
                    for (uint32_t n = 0; n < NE; ++n) {
                        if (!src[n]) continue;
                        int m = (int)n + dE / 2;
                        if (m >= 0 && m < (int)NE) dst[m] += src[n];
                    }
                }
            u128 *t = cur;
            cur = nxt;
            nxt = t;
        }
        /* close the torus: vertical bonds between the last row and row 0 */
        for (uint32_t b = 0; b < S; ++b) {
            int dE = 0;
            for (uint32_t x = 0; x < L; ++x) dE -= Jd[(L - 1) * L + x] * SPIN(b, x) * SPIN(f, x);
            u128 *src = cur + (size_t)b * NE;
            for (uint32_t n = 0; n < NE; ++n) {
                if (!src[n]) continue;
                int m = (int)n + dE / 2;
                if (m >= 0 && m < (int)NE) tot[m] += src[n];
            }
        }
    }
#undef SPIN
    for (uint32_t n = 0; n < NE; ++n) {
        out_lo[n] = (uint64_t)tot[n];
        out_hi[n] = (uint64_t)(tot[n] >> 64);
    }
    free(cur);
    free(nxt);
    free(tot);
    return OR_OK;
}

uint32_t or_sizeof_record(void) { return (uint32_t)sizeof(or_record); }
uint32_t or_sizeof_wavg(void) { return (uint32_t)sizeof(or_wavg); }
uint32_t or_sizeof_desc(void) { return (uint32_t)sizeof(or_desc); }
