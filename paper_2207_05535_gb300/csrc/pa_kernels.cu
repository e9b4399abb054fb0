// Kernels of the population-annealing hot path for sm_103a (GB300).
//
// One anneal step (arXiv:2207.05535, Sec. II.B steps (ii)-(v)) runs over every
// run of the engine in a handful of launches:
//   resample_counts_kernel / resample_parents_kernel
//                    nearest-integer resampling, a population split over several
//                    CTAs: copy numbers r_j from the per-level tables the previous
//                    measurement prepared, then the exclusive scan and the parent
//                    map that places copies of one ancestor next to each other
//                    (Sec. V.A.1); one launch when every population fits one CTA
//   resample_multinomial_kernel
//                    multinomial resampling, one CTA per run (level histogram,
//                    Q_i of Eq. QBoltz, R draws, scan, parent map)
//   sweep_pow2_kernel / sweep_compact_kernel / sweep_pad_kernel / sweep_kernel
//                    per lattice size: each replica is gathered from its parent
//                    (the resampling copy) and swept theta times with Philox
//                    thresholds (Sec. V.A.1), bit-sliced: rows tiling words (L/2 a
//                    power of two), rows repacked without padding in shared memory,
//                    or padded rows; byte planes as the cross-check
//   anneal_small_kernel
//                    small runs (L = 8, 16, 32, nearest-integer, no overlaps): one
//                    thread-block cluster per run resamples, sweeps and measures,
//                    several temperatures per launch
//   dos_sample_kernel
//                    theta = infinity runs (Sec. V.B): fresh energies from the exact
//                    distribution instead of sweeps
//   overlap_kernel / wang_kernel
//                    overlaps of index-shift pairs, partner populations and Wang
//                    et al.'s pairings (Sec. III.D)
//   measure_kernel   moments of E and |M| (k <= 4, exact integers) from per-level
//                    histograms, family statistics (Eq. rho_t), the free-energy
//                    running sum (Eq. F), and the next nearest-integer resampling's
//                    E_min, Q_{i+1} and per-level tables
// The weighted averages of Sec. IV run after the anneal (wavg_*_kernel).
// Nothing here allocates memory; no spin-wait exists in any kernel.
//
// Randomness: Philox4x32-10 (Salmon et al., SC'11), key (seed, run_id):
//   init spin n of replica j   ctr (n>>2, j, 0, INIT<<24)                word n&3, bit 31
//   coupling of site n         ctr (n>>2, 0, 0, DISORDER<<24), key (seed, disorder_id)
//                              word n&3: bit 31 -> J_right = +1, bit 30 -> J_down = +1
//   nearest-integer draw of j  ctr (j, 0, i, RESAMPLE<<24)               word 0
//   multinomial draw d         ctr (d, 0, i, MULTINOMIAL<<24)            words 0,1 level; word 2 member
//   Metropolis, sublattice k   ctr (k>>2, child, i, SWEEP<<24|t<<1|c)     word k&3
//   theta = infinity draw of j ctr (j, 0, i, DOS<<24)                    words 0,1 (53-bit uniform)
//   Wang keys of replica j     ctr (j, 0, i, WANG<<24)                   words 0,1 pi, words 2,3 sigma
// FP64 arithmetic that decides an integer uses explicit round-to-nearest
// intrinsics (no contraction), in the same order as the plain definition.
#include <cooperative_groups.h>
#include <cmath>
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "pa_internal.cuh"

namespace pa {

namespace cg = cooperative_groups;

namespace {

constexpr unsigned FULL = 0xffffffffu;
#ifndef PA_PACK_MODE
#define PA_PACK_MODE 0  // packing of the comparison bits: 0 compare + predicated or (integer ALU), 1 shifted adds
#endif
constexpr uint32_t SMEM_BINS = 4096;

__device__ __forceinline__ uint4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                               uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return make_uint4(c0, c1, c2, c3);
}

// acc |= bit where u < t: a compare and a predicated or, both on the integer
// ALU, which leaves the multiplier pipe to Philox (the sweeps' binding unit).
__device__ __forceinline__ void or_if_below(uint32_t &acc, uint32_t u, uint32_t t, uint32_t bit)
{
    asm("{\n\t.reg .pred p;\n\tsetp.lt.u32 p, %1, %2;\n\t@p or.b32 %0, %0, %3;\n\t}" : "+r"(acc) : "r"(u), "r"(t), "r"(bit));
}

// The comparison bits of one Philox group g (uniforms u) against t1 and t2 into
// bits 4g..4g+3 of B1 and B2.
__device__ __forceinline__ void pack_group(uint32_t &B1, uint32_t &B2, const uint4 &u, uint32_t g, uint32_t t1,
                                           uint32_t t2)
{
#if PA_PACK_MODE == 1
    B1 += ((uint32_t)(u.x < t1) << (4 * g)) + ((uint32_t)(u.y < t1) << (4 * g + 1)) +
          ((uint32_t)(u.z < t1) << (4 * g + 2)) + ((uint32_t)(u.w < t1) << (4 * g + 3));
    B2 += ((uint32_t)(u.x < t2) << (4 * g)) + ((uint32_t)(u.y < t2) << (4 * g + 1)) +
          ((uint32_t)(u.z < t2) << (4 * g + 2)) + ((uint32_t)(u.w < t2) << (4 * g + 3));
#else
    or_if_below(B1, u.x, t1, 1u << (4 * g));
    or_if_below(B1, u.y, t1, 2u << (4 * g));
    or_if_below(B1, u.z, t1, 4u << (4 * g));
    or_if_below(B1, u.w, t1, 8u << (4 * g));
    or_if_below(B2, u.x, t2, 1u << (4 * g));
    or_if_below(B2, u.y, t2, 2u << (4 * g));
    or_if_below(B2, u.z, t2, 4u << (4 * g));
    or_if_below(B2, u.w, t2, 8u << (4 * g));
#endif
}

__device__ __forceinline__ uint32_t pick(const uint4 &u, uint32_t q)
{
    return q == 0 ? u.x : q == 1 ? u.y : q == 2 ? u.z : u.w;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_max(T v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        T w = __shfl_xor_sync(FULL, v, o);
        v = w > v ? w : v;
    }
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_min(T v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        T w = __shfl_xor_sync(FULL, v, o);
        v = w < v ? w : v;
    }
    return v;
}

// Block-wide sum broadcast to every thread.  sh: >= 32 elements.
template <typename T>
__device__ T block_sum(T v, T *sh)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    T r = lane < nw ? sh[lane] : T(0);
    r = warp_sum(r);
    __syncthreads();
    return r;
}

template <typename T>
__device__ T block_max(T v, T *sh, T ident)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_max(v);
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    T r = lane < nw ? sh[lane] : ident;
    r = warp_max(r);
    __syncthreads();
    return r;
}

template <typename T>
__device__ T block_min(T v, T *sh, T ident)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_min(v);
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    T r = lane < nw ? sh[lane] : ident;
    r = warp_min(r);
    __syncthreads();
    return r;
}

// Exclusive prefix sum over the block (blockDim a multiple of 32); total to all.
__device__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *sh, uint32_t &total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t s = lane < nw ? sh[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(FULL, s, o);
            if (lane >= o) s += y;
        }
        sh[lane] = s;
    }
    __syncthreads();
    const uint32_t base = wid ? sh[wid - 1] : 0u;
    total = sh[nw - 1];
    __syncthreads();
    return base + x - v;
}

// Inclusive max-scan over the block.
__device__ uint32_t block_inclusive_max(uint32_t v, uint32_t *sh)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x = y > x ? y : x;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t s = lane < nw ? sh[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(FULL, s, o);
            if (lane >= o) s = y > s ? y : s;
        }
        sh[lane] = s;
    }
    __syncthreads();
    const uint32_t base = wid ? sh[wid - 1] : 0u;
    __syncthreads();
    return base > x ? base : x;
}

__device__ __forceinline__ uint32_t get_bit(const uint32_t *w, uint32_t n) { return (w[n >> 5] >> (n & 31)) & 1u; }

// Work list: tile_off[g] = first tile of run slot g (prefix of per-run tile
// counts, tile_off[n] = total).  Returns the slot holding tile t.
__device__ __forceinline__ uint32_t locate_slot(const uint32_t *tile_off, uint32_t n, uint32_t t)
{
    uint32_t a = 0, b = n;  // invariant: tile_off[a] <= t < tile_off[b]
    while (b - a > 1) {
        const uint32_t m = (a + b) >> 1;
        if (tile_off[m] <= t)
            a = m;
        else
            b = m;
    }
    return a;
}

__device__ __forceinline__ void set_status(const Pool &P, uint32_t run, uint32_t code)
{
    P.st[run].status = code;
    atomicOr(P.status, 1u << code);
}

// --------------------------------------------------------------------------
// Spin layout of a replica (HBM and the bit-sliced sweeps' shared memory): two
// colour planes, plane c holding the sites of colour c = (x + y) & 1, row y of
// the plane at bit positions [y P, y P + L/2) with P = rd.pitch >= L/2 (padding
// bits 0), position y P + (x >> 1) for site n = y L + x; bit pos & 31 of word
// pos >> 5, bit 1 = spin +1.  Plane 0 occupies words [0, PW), plane 1
// [PW, 2 PW), PW = rd.pw.  Philox counters use the compact sublattice index
// k = n >> 1 = y L/2 + (x >> 1) whatever the pitch.
// --------------------------------------------------------------------------
__device__ __forceinline__ uint32_t spin_bit(const uint32_t *planes, uint32_t PW, uint32_t L, uint32_t pitch,
                                             uint32_t n)
{
    const uint32_t x = n % L, y = n / L, c = (x + y) & 1u, pos = y * pitch + (x >> 1);
    return (planes[c * PW + (pos >> 5)] >> (pos & 31)) & 1u;
}

// Neighbour masks of word w of colour plane c (L a power of two, 8..256), read
// from the other plane O (HW words): the spin at the same sublattice index,
// at the index rotated by one within the row (k - 1 on rows with (c + y) even,
// k + 1 on odd rows), in the row above and in the row below.
__device__ __forceinline__ void plane_neighbours(const uint32_t *O, uint32_t HW, uint32_t Lh, uint32_t c, uint32_t w,
                                                 uint32_t &same, uint32_t &rot, uint32_t &up, uint32_t &dn)
{
    if (Lh < 32) {  // several rows per word
        const uint32_t LOW = Lh == 4 ? 0x11111111u : Lh == 8 ? 0x01010101u : 0x00010001u;
        const uint32_t HIGH = LOW << (Lh - 1);
        const uint32_t EVEN = Lh == 4 ? 0x0F0F0F0Fu : Lh == 8 ? 0x00FF00FFu : 0x0000FFFFu;  // rows 0, 2, ...
        const uint32_t o = O[w], op = O[(w - 1) & (HW - 1)], on = O[(w + 1) & (HW - 1)];
        same = o;
        up = __funnelshift_l(op, o, Lh);  // bit k <- k - Lh
        dn = __funnelshift_r(o, on, Lh);  // bit k <- k + Lh
        const uint32_t rl = ((o << 1) & ~LOW) | ((o >> (Lh - 1)) & LOW);   // bit k <- k - 1 in the row
        const uint32_t rr = ((o >> 1) & ~HIGH) | ((o << (Lh - 1)) & HIGH); // bit k <- k + 1 in the row
        rot = c == 0 ? ((rl & EVEN) | (rr & ~EVEN)) : ((rr & EVEN) | (rl & ~EVEN));
    } else {  // WR words per row
        const uint32_t WR = Lh >> 5;
        const uint32_t o = O[w];
        same = o;
        up = O[(w - WR) & (HW - 1)];
        dn = O[(w + WR) & (HW - 1)];
        const uint32_t y = w / WR, base = y * WR, q = w - base;
        if (((c + y) & 1u) == 0)
            rot = (o << 1) | (O[base + ((q - 1) & (WR - 1))] >> 31);
        else
            rot = (o >> 1) | (O[base + ((q + 1) & (WR - 1))] << 31);
    }
}

// --------------------------------------------------------------------------
// Initialisation (Sec. II.B step (i) at beta_0 = 0; couplings of Eq. H_SG).
// Couplings are kept twice: site order (bit n of Jr / Jd: the right / down
// bond of site n is J = -1) and, for the fast sweep, per colour plane word the
// four bond masks of its sites: bond to the same-index neighbour, to the
// rotated neighbour (index k -+ 1 within the row), up and down.
// --------------------------------------------------------------------------
__global__ void init_couplings_kernel(Pool P, const uint32_t *runs)
{
    const RunDev rd = P.runs[runs ? runs[blockIdx.x] : blockIdx.x];
    const uint32_t SW = rd.wstride;          // site-order words (>= ceil(N/32))
    const uint32_t PW = rd.pw;               // plane words
    uint32_t *Jr = P.J + rd.J_off, *Jd = Jr + SW, *Jp = Jd + SW;  // Jp: [c][4][PW]
    for (uint32_t w = threadIdx.x; w < SW; w += blockDim.x) {
        uint32_t wr = 0, wd = 0;
        if (rd.model == PA_EA_PMJ) {
            for (uint32_t g = 0; g < 8; ++g) {
                const uint32_t n0 = 32 * w + 4 * g;
                if (n0 >= rd.N) break;
                const uint4 u = philox4x32_10(n0 >> 2, 0, 0, TAG_DISORDER << 24, rd.seed, rd.disorder_id);
                for (uint32_t q = 0; q < 4; ++q) {
                    if (n0 + q >= rd.N) break;
                    const uint32_t v = pick(u, q);
                    wr |= ((~v >> 31) & 1u) << (4 * g + q);  // bit set where J_right = -1
                    wd |= ((~v >> 30) & 1u) << (4 * g + q);  // bit set where J_down = -1
                }
            }
        }
        Jr[w] = wr;
        Jd[w] = wd;
    }
    __syncthreads();
    const uint32_t L = rd.L, Lh = rd.Lh, Pt = rd.pitch;
    for (uint32_t cw = threadIdx.x; cw < 2 * PW; cw += blockDim.x) {
        const uint32_t c = cw / PW, w = cw - c * PW;
        uint32_t js = 0, jr = 0, ju = 0, jd = 0;
        for (uint32_t b = 0; b < 32; ++b) {
            const uint32_t pos = 32 * w + b, y = pos / Pt, xp = pos - y * Pt;
            if (y >= L || xp >= Lh) continue;  // row padding
            const uint32_t x = 2 * xp + ((c + y) & 1u), n = y * L + x;
            const uint32_t p = (c + y) & 1u;
            const uint32_t right = get_bit(Jr, n), left = get_bit(Jr, y * L + (x == 0 ? L - 1 : x - 1));
            const uint32_t down = get_bit(Jd, n), up = get_bit(Jd, (y == 0 ? L - 1 : y - 1) * L + x);
            js |= (p ? left : right) << b;
            jr |= (p ? right : left) << b;
            ju |= up << b;
            jd |= down << b;
        }
        uint32_t *o = Jp + c * 4 * PW;
        o[w] = js;
        o[PW + w] = jr;
        o[2 * PW + w] = ju;
        o[3 * PW + w] = jd;
    }
}

// One warp per replica (4 per CTA, CTAs from the work list over all runs):
// uniform spins from Philox (one call per four consecutive sites), then E and
// M exactly.  Power-of-two L uses word-wide neighbour masks for E.
__global__ void __launch_bounds__(128)
    init_population_kernel(Pool P, const uint32_t *tile_off, const uint32_t *runs, uint32_t n_runs)
{
    extern __shared__ __align__(16) uint32_t sw[];  // per warp: 2 PW plane words
    const uint32_t slot = locate_slot(tile_off, n_runs, blockIdx.x);
    const RunDev rd = P.runs[runs ? runs[slot] : slot];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t j = (blockIdx.x - tile_off[slot]) * (blockDim.x >> 5) + warp;
    if (j >= rd.R) return;  // warp-uniform; no block barrier below
    const uint32_t L = rd.L, N = rd.N, PW = rd.pw, Pt = rd.pitch;
    uint32_t *pl = sw + warp * 2 * PW;
    for (uint32_t cw = lane; cw < 2 * PW; cw += 32) pl[cw] = 0;
    __syncwarp();
    for (uint32_t g = lane; 4 * g < N; g += 32) {
        const uint4 u = philox4x32_10(g, j, 0, TAG_INIT << 24, rd.seed, rd.run_id);
        for (uint32_t q = 0; q < 4; ++q) {
            const uint32_t n = 4 * g + q;
            if (n >= N) break;
            const uint32_t x = n % L, y = n / L, c = (x + y) & 1u, pos = y * Pt + (x >> 1);
            if (pick(u, q) >> 31) atomicOr(&pl[c * PW + (pos >> 5)], 1u << (pos & 31));
        }
    }
    __syncwarp();
    uint32_t *s = P.spins[0] + rd.spin_off + (uint64_t)j * rd.wstride;
    for (uint32_t cw = lane; cw < rd.wstride; cw += 32) s[cw] = cw < 2 * PW ? pl[cw] : 0u;  // padding cleared
    int32_t unsat = 0, up = 0;
    for (uint32_t cw = lane; cw < 2 * PW; cw += 32) up += __popc(pl[cw]);
    const bool pow2 = L >= 8 && Pt == rd.Lh;  // L/2 a power of two: rows fill the words
    if (pow2) {
        const uint32_t *Jp = P.J + rd.J_off + 2 * rd.wstride;  // [c][4][PW] bond masks
        for (uint32_t w = lane; w < PW; w += 32) {
            uint32_t same, rot, upn, dn;
            plane_neighbours(pl + PW, PW, rd.Lh, 0, w, same, rot, upn, dn);
            const uint32_t S = pl[w];
            unsat += __popc(S ^ same ^ Jp[w]) + __popc(S ^ rot ^ Jp[PW + w]) + __popc(S ^ upn ^ Jp[2 * PW + w]) +
                     __popc(S ^ dn ^ Jp[3 * PW + w]);
        }
    } else {
        const uint32_t *Jr = P.J + rd.J_off, *Jd = Jr + rd.wstride;
        for (uint32_t n = lane; n < N; n += 32) {
            const uint32_t x = n % L, y = n / L;
            const uint32_t b = spin_bit(pl, PW, L, Pt, n);
            const uint32_t br = spin_bit(pl, PW, L, Pt, y * L + (x + 1 == L ? 0 : x + 1));
            const uint32_t bd = spin_bit(pl, PW, L, Pt, (y + 1 == L ? 0 : y + 1) * L + x);
            unsat += (int32_t)((b ^ br ^ get_bit(Jr, n)) + (b ^ bd ^ get_bit(Jd, n)));
        }
    }
    unsat = warp_sum(unsat);
    up = warp_sum(up);
    if (lane == 0) {
        P.E[0][rd.rep_off + j] = 2 * unsat - 2 * (int32_t)N;  // H = (#unsatisfied) - (#satisfied)
        P.M[0][rd.rep_off + j] = 2 * up - (int32_t)N;
        P.fam[0][rd.rep_off + j] = j;
    }
}

// --------------------------------------------------------------------------
// Resampling (Sec. II.B steps (ii)-(iii), Eqs. tauBoltz and QBoltz).
//
// Both schemes share the normalisation: the population's energies are counted
// per level n = (E - E_min) / 4 (energies of one population differ by
// multiples of 4: a spin flip changes E by 0, +-4 or +-8), and
// S = sum_j exp(-dbeta (E_j - E_min)) is summed level by level in ascending
// order with the shared table w[n] = exp(-4 n dbeta); Q = exp(-dbeta E_min) S / R.
// --------------------------------------------------------------------------
// Populations of up to this many replicas have their energies staged in shared memory.
constexpr uint32_t RESAMPLE_STAGE_MAX = 24576;  // 96 KB

// Multinomial resampling (PA_MULTINOMIAL), one CTA per run: R draws, each
// picking a level from the cumulative weights and a member of that level
// uniformly; then the copy numbers' scan and the parent map as below.
__global__ void __launch_bounds__(512) resample_multinomial_kernel(Pool P, const uint32_t *runs, uint32_t stage)
{
    extern __shared__ int32_t sE[];  // [stage]
    __shared__ uint32_t sh_hist[SMEM_BINS];
    __shared__ int32_t sh_i[32];
    __shared__ uint32_t sh_u[33];
    __shared__ double sh_S;
    __shared__ uint32_t sh_carry;

    const uint32_t run = runs[blockIdx.x];
    const RunDev rd = P.runs[run];
    RunState *st = &P.st[run];
    if (st->status) return;
    const uint32_t i = st->step + 1;
    if (i >= rd.n_beta) return;
    const uint32_t Rprev = st->R_cur;
    const int32_t *E = P.E[(i - 1) & 1] + rd.rep_off;
    const uint32_t tid = threadIdx.x, nt = blockDim.x;

    // energy range of the population at beta_{i-1}; the energies are read once from
    // global memory and, when they fit, kept in shared memory for the later passes
    const bool staged = Rprev <= stage;
    int32_t lo = INT32_MAX, hi = INT32_MIN;
    for (uint32_t j = tid; j < Rprev; j += nt) {
        const int32_t e = E[j];
        if (staged) sE[j] = e;
        lo = e < lo ? e : lo;
        hi = e > hi ? e : hi;
    }
    const int32_t *Ev = staged ? sE : E;
    const int32_t Emin = block_min(lo, sh_i, INT32_MAX);
    const int32_t Emax = block_max(hi, sh_i, INT32_MIN);
    const uint32_t nb = (uint32_t)(Emax - Emin) / 4u + 1u;

    unsigned long long *scr = P.scratch + rd.scr_off;
    uint32_t *g_hist = reinterpret_cast<uint32_t *>(scr);
    double *cdf = reinterpret_cast<double *>(scr + scr_table_off(rd.N));
    uint32_t *fill = reinterpret_cast<uint32_t *>(scr + scr_level_off(rd.N));
    uint32_t *members = reinterpret_cast<uint32_t *>(scr + scr_tail_off(rd.N));
    uint32_t *h = nb <= SMEM_BINS ? sh_hist : g_hist;
    for (uint32_t n = tid; n < nb; n += nt) h[n] = 0;
    __syncthreads();
    for (uint32_t j = tid; j < Rprev; j += nt) atomicAdd(&h[(uint32_t)(Ev[j] - Emin) >> 2], 1u);
    __syncthreads();

    const double dbeta = P.beta[rd.beta_off + i] - P.beta[rd.beta_off + i - 1];
    const double *w = P.wt + P.wtoff[rd.wt_off + i];  // w[n] = exp(-4 n dbeta_i), shared table
    if (tid == 0) {
        double S = 0.0;
        for (uint32_t n = 0; n < nb; ++n) {
            S = __dadd_rn(S, __dmul_rn((double)h[n], w[n]));
            cdf[n] = S;
        }
        sh_S = S;
        st->lnQ = (-dbeta) * (double)Emin + log(S) - log((double)Rprev);
    }
    __syncthreads();
    const double S = sh_S;
    uint32_t *cnt = P.cnt + rd.rep_off;

    // stable list of replicas by level: members[first(n) + rank]
    if (tid < 32) {
        uint32_t acc = 0;
        for (uint32_t base = 0; base < nb; base += 32) {  // fill[n] = first(n)
            const uint32_t n = base + tid;
            const uint32_t v = n < nb ? h[n] : 0u;
            uint32_t x = v;
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(FULL, x, o);
                if ((int)tid >= o) x += y;
            }
            if (n < nb) fill[n] = acc + x - v;
            acc += __shfl_sync(FULL, x, 31);
        }
        __syncwarp();
        for (uint32_t base = 0; base < Rprev; base += 32) {
            const uint32_t j = base + tid;
            const bool ok = j < Rprev;
            const uint32_t n = ok ? (uint32_t)(Ev[j] - Emin) >> 2 : 0xffffffffu;
            const unsigned peers = __match_any_sync(FULL, n);
            const uint32_t rank = __popc(peers & ((1u << tid) - 1u));
            uint32_t pos = 0;
            if (ok) pos = fill[n] + rank;
            __syncwarp();
            if (ok) {
                members[pos] = j;
                if (rank == 0) fill[n] += __popc(peers);
            }
            __syncwarp();
        }
    }
    for (uint32_t j = tid; j < Rprev; j += nt) cnt[j] = 0;
    __syncthreads();
    const uint32_t last = nb - 1;
    for (uint32_t d = tid; d < rd.R; d += nt) {
        const uint4 o = philox4x32_10(d, 0, i, TAG_MULTINOMIAL << 24, rd.seed, rd.run_id);
        const unsigned long long u53 = ((unsigned long long)(o.x >> 5) << 26) | (unsigned long long)(o.y >> 6);
        const double x = __dmul_rn(__dmul_rn((double)u53, 1.0 / 9007199254740992.0), S);
        uint32_t a = 0, b = nb;  // first n with cdf[n] > x
        while (a < b) {
            const uint32_t m = (a + b) >> 1;
            if (cdf[m] > x)
                b = m;
            else
                a = m + 1;
        }
        const uint32_t lev = a < nb ? a : last;
        const uint32_t idx = (uint32_t)(((unsigned long long)o.z * (unsigned long long)h[lev]) >> 32);
        const uint32_t first = fill[lev] - h[lev];
        atomicAdd(&cnt[members[first + idx]], 1u);
    }
    __syncthreads();
    if (h == g_hist)  // leave the measurement's histogram cleared
        for (uint32_t n = tid; n < nb; n += nt) g_hist[n] = 0u;

    // the copy numbers' exclusive scan and the parent map (contiguous families).
    // Each warp takes a contiguous chunk of the replicas; one barrier joins the chunks.
    uint32_t *parent = P.parent + rd.rep_off;
    const uint32_t lane = tid & 31u, wid = tid >> 5, nwarp = nt >> 5;
    const uint32_t chunk = (Rprev + nwarp - 1) / nwarp;
    const uint32_t c_lo = min(Rprev, wid * chunk), c_hi = min(Rprev, c_lo + chunk);
    uint32_t wsum = 0;
    for (uint32_t j = c_lo + lane; j < c_hi; j += 32) wsum += cnt[j];
    wsum = warp_sum(wsum);
    if (lane == 0) sh_u[wid] = wsum;
    __syncthreads();
    if (tid == 0) {
        uint32_t acc = 0;
        for (uint32_t k = 0; k < nwarp; ++k) {
            const uint32_t v = sh_u[k];
            sh_u[k] = acc;
            acc += v;
        }
        sh_carry = acc;
    }
    __syncthreads();
    uint32_t carry = sh_u[wid];
    for (uint32_t base = c_lo; base < c_hi; base += 32) {
        const uint32_t j = base + lane;
        const uint32_t r = j < c_hi ? cnt[j] : 0u;
        uint32_t x = r;  // inclusive scan over the lanes
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, x, o);
            if ((int)lane >= o) x += y;
        }
        const uint32_t o = carry + x - r;
        for (uint32_t c = 0; c < r; ++c)
            if (o + c < rd.R_cap) parent[o + c] = j;
        carry += __shfl_sync(FULL, x, 31);
    }
    if (tid == 0) {
        const uint32_t Rn = sh_carry;
        st->R_new = Rn;
        if (Rn == 0)
            set_status(P, run, PA_ERR_EXTINCT);
        else if (Rn > rd.R_cap)
            set_status(P, run, PA_ERR_CAPACITY);
        if (Rn == 0 || Rn > rd.R_cap) P.rec[rd.rec_off + i].status = st->status;
    }
}

// Nearest-integer resampling (PA_NEAREST): r_j = floor(tau) + [u 2^-32 < tau - floor(tau)],
// tau = R w[n_j] / S.  tau depends on the level only, so per level the floor and
// the integer threshold ceil(frac 2^32) are tabulated once (u 2^-32 < frac <=>
// u < frac 2^32 exactly: scaling by 2^32 is exact and u is an integer).  The
// measurement of the previous step, which counts the population per energy
// level anyway, finds E_min, sums S and Q and writes these tables.
//
// A run's population is split over nc = run_ctas(R_cap) CTAs (CTA c of the
// run: blockIdx.y = c, replicas [c ceil(R/nc), (c+1) ceil(R/nc))), in two
// launches:
//   resample_counts_kernel   r_j of every replica and each CTA's total
//   resample_parents_kernel  offsets (earlier CTAs' totals plus a scan inside
//                            the CTA) and the parent map
constexpr uint32_t RESAMPLE_THREADS = 512;
constexpr uint32_t COUNTS_SMEM_LEVELS = 2048;  // level tables staged in shared memory (L <= 45)
constexpr uint32_t COUNTS_BATCH = 4;           // replicas per thread in flight
constexpr uint32_t PARENT_BATCH = 8;           // rows of 32 copy numbers a warp loads at once

struct RunChunk {
    uint32_t lo, hi;  // this CTA's replicas
};

__device__ __forceinline__ RunChunk cta_chunk(uint32_t R, uint32_t nc, uint32_t c)
{
    const uint32_t chunk = (R + nc - 1) / nc;
    const uint32_t lo = min(R, c * chunk);
    return {lo, min(R, lo + chunk)};
}

// The parent map of one CTA's chunk (copy numbers in cnt, written before a
// barrier): exclusive offsets from `off` (the earlier CTAs' copies) plus a scan
// per warp chunk; the CTA holding the run's first chunk records the new size
// R_new = total and the capacity or extinction status.
__device__ __forceinline__ void parents_pass(const Pool &P, uint32_t run, const RunDev &rd, RunState *st, uint32_t i,
                                             RunChunk ch, uint32_t off, uint32_t total, bool first_cta,
                                             uint32_t *sh_u)
{
    const uint32_t tid = threadIdx.x, lane = tid & 31u, wid = tid >> 5, nwarp = blockDim.x >> 5;
    const uint32_t *cnt = P.cnt + rd.rep_off;
    uint32_t *parent = P.parent + rd.rep_off;
    // each warp takes a contiguous piece of the CTA's chunk, PARENT_BATCH rows of
    // 32 at a time; the first batch stays in registers between the two passes
    const uint32_t wchunk = (ch.hi - ch.lo + nwarp - 1) / nwarp;
    const uint32_t w_lo = min(ch.hi, ch.lo + wid * wchunk), w_hi = min(ch.hi, w_lo + wchunk);
    uint32_t wsum = 0, cq[PARENT_BATCH];
    for (uint32_t b0 = w_lo; b0 < w_hi; b0 += 32 * PARENT_BATCH) {
        uint32_t t[PARENT_BATCH];
#pragma unroll
        for (uint32_t r = 0; r < PARENT_BATCH; ++r) {
            const uint32_t j = b0 + 32 * r + lane;
            t[r] = j < w_hi ? cnt[j] : 0u;
            wsum += t[r];
        }
        if (b0 == w_lo)
#pragma unroll
            for (uint32_t r = 0; r < PARENT_BATCH; ++r) cq[r] = t[r];
    }
    wsum = warp_sum(wsum);
    if (lane == 0) sh_u[wid] = wsum;
    __syncthreads();
    if (tid == 0) {
        uint32_t acc = off;
        for (uint32_t k = 0; k < nwarp; ++k) {
            const uint32_t v = sh_u[k];
            sh_u[k] = acc;
            acc += v;
        }
    }
    __syncthreads();
    uint32_t carry = sh_u[wid];
    for (uint32_t b0 = w_lo; b0 < w_hi; b0 += 32 * PARENT_BATCH) {
        uint32_t t[PARENT_BATCH];
#pragma unroll
        for (uint32_t r = 0; r < PARENT_BATCH; ++r) {
            const uint32_t j = b0 + 32 * r + lane;
            t[r] = b0 == w_lo ? cq[r] : (j < w_hi ? cnt[j] : 0u);
        }
#pragma unroll
        for (uint32_t q = 0; q < PARENT_BATCH; ++q) {
            if (b0 + 32 * q >= w_hi) break;  // uniform over the warp
            const uint32_t j = b0 + 32 * q + lane, r = t[q];
            uint32_t x = r;  // inclusive scan over the lanes
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(FULL, x, o);
                if ((int)lane >= o) x += y;
            }
            const uint32_t o = carry + x - r;
            for (uint32_t c = 0; c < r; ++c)
                if (o + c < rd.R_cap) parent[o + c] = j;
            carry += __shfl_sync(FULL, x, 31);
        }
    }
    if (first_cta && tid == 0) {
        const uint32_t Rn = total;
        st->R_new = Rn;
        if (Rn == 0)
            set_status(P, run, PA_ERR_EXTINCT);
        else if (Rn > rd.R_cap)
            set_status(P, run, PA_ERR_CAPACITY);
        if (Rn == 0 || Rn > rd.R_cap) P.rec[rd.rec_off + i].status = st->status;
    }
}

// FUSED (every run in one CTA): the parent map follows in the same CTA.
template <bool FUSED>
__global__ void __launch_bounds__(RESAMPLE_THREADS, 2) resample_counts_kernel(Pool P, const uint32_t *runs)
{
    __shared__ unsigned long long s_thr[COUNTS_SMEM_LEVELS];
    __shared__ uint32_t s_flo[COUNTS_SMEM_LEVELS];
    __shared__ uint32_t sh_r[32];
    __shared__ uint32_t sh_u[RESAMPLE_THREADS / 32];
    const uint32_t run = runs[blockIdx.x];
    const RunDev rd = P.runs[run];
    RunState *st = &P.st[run];
    if (st->status) return;
    const uint32_t i = st->step + 1;
    if (i >= rd.n_beta) return;
    const uint32_t nc = min(gridDim.y, run_ctas(rd.R_cap));
    if (blockIdx.y >= nc) return;
    const RunChunk ch = cta_chunk(st->R_cur, nc, blockIdx.y);
    const int32_t *E = P.E[(i - 1) & 1] + rd.rep_off;
    const int32_t Emin = st->Emin;
    const uint32_t nb = st->n_levels, tid = threadIdx.x, nt = blockDim.x;
    const unsigned long long *scr = P.scratch + rd.scr_off;
    const unsigned long long *thr = scr + scr_table_off(rd.N);
    const uint32_t *flo = reinterpret_cast<const uint32_t *>(scr + scr_level_off(rd.N));
    // the first batch's energies and uniforms are requested before the tables are staged
    int32_t e[COUNTS_BATCH];
    uint32_t u[COUNTS_BATCH];
    const uint32_t j_first = ch.lo + tid;
#pragma unroll
    for (uint32_t r = 0; r < COUNTS_BATCH; ++r) {
        const uint32_t j = j_first + r * nt;
        e[r] = j < ch.hi ? E[j] : Emin;
        u[r] = philox4x32_10(j, 0, i, TAG_RESAMPLE << 24, rd.seed, rd.run_id).x;
    }
    if (nb <= COUNTS_SMEM_LEVELS) {
        for (uint32_t n = tid; n < nb; n += nt) {
            s_thr[n] = thr[n];
            s_flo[n] = flo[n];
        }
        __syncthreads();
        thr = s_thr;
        flo = s_flo;
    }
    uint32_t *cnt = P.cnt + rd.rep_off;
    uint32_t sum = 0;
    for (uint32_t j0 = j_first; j0 < ch.hi; j0 += COUNTS_BATCH * nt) {
        if (j0 != j_first) {
#pragma unroll
            for (uint32_t r = 0; r < COUNTS_BATCH; ++r) e[r] = j0 + r * nt < ch.hi ? E[j0 + r * nt] : Emin;
#pragma unroll
            for (uint32_t r = 0; r < COUNTS_BATCH; ++r)
                u[r] = philox4x32_10(j0 + r * nt, 0, i, TAG_RESAMPLE << 24, rd.seed, rd.run_id).x;
        }
#pragma unroll
        for (uint32_t r = 0; r < COUNTS_BATCH; ++r) {
            const uint32_t j = j0 + r * nt;
            if (j >= ch.hi) break;
            const uint32_t n = (uint32_t)(e[r] - Emin) >> 2;
            const uint32_t c = flo[n] + ((unsigned long long)u[r] < thr[n] ? 1u : 0u);
            cnt[j] = c;
            sum += c;
        }
    }
    sum = block_sum(sum, sh_r);  // ends with a barrier: this CTA's copy numbers are visible
    if (FUSED)
        parents_pass(P, run, rd, st, i, ch, 0u, sum, true, sh_u);
    else if (tid == 0)
        reinterpret_cast<uint32_t *>(P.scratch + rd.scr_off + scr_tail_off(rd.N))[blockIdx.y] = sum;
}

__global__ void __launch_bounds__(RESAMPLE_THREADS) resample_parents_kernel(Pool P, const uint32_t *runs)
{
    __shared__ uint32_t sh_u[RESAMPLE_THREADS / 32];
    __shared__ uint32_t sh_off, sh_total;
    const uint32_t run = runs[blockIdx.x];
    const RunDev rd = P.runs[run];
    RunState *st = &P.st[run];
    if (st->status) return;
    const uint32_t i = st->step + 1;
    if (i >= rd.n_beta) return;
    const uint32_t nc = min(gridDim.y, run_ctas(rd.R_cap));
    if (blockIdx.y >= nc) return;
    const RunChunk ch = cta_chunk(st->R_cur, nc, blockIdx.y);
    const uint32_t *cta_tot = reinterpret_cast<const uint32_t *>(P.scratch + rd.scr_off + scr_tail_off(rd.N));
    if (threadIdx.x < 32) {  // the earlier CTAs' totals (this CTA's offset) and the new size
        const uint32_t lane = threadIdx.x;
        uint32_t before = 0, all = 0;
        for (uint32_t k = lane; k < nc; k += 32) {
            const uint32_t v = cta_tot[k];
            before += k < blockIdx.y ? v : 0u;
            all += v;
        }
        before = warp_sum(before);
        all = warp_sum(all);
        if (lane == 0) {
            sh_off = before;
            sh_total = all;
        }
    }
    __syncthreads();
    parents_pass(P, run, rd, st, i, ch, sh_off, sh_total, blockIdx.y == 0, sh_u);
}

// --------------------------------------------------------------------------
// Fused gather + theta checkerboard Metropolis sweeps (Sec. V.A.1), any even L.
// Shared memory per replica: the two colour planes unpacked to one byte per
// site.  Every thread owns Philox groups g (sublattice sites 4g..4g+3 of a
// colour): one Philox call gives the four uniforms of a group.  A shared
// "bond mask" plane holds per site the J = -1 bits of its right, left, down
// and up bonds.
// --------------------------------------------------------------------------
template <bool HOIST, int MAXT>
__global__ void __launch_bounds__(MAXT) sweep_kernel(Pool P, const uint32_t *group_runs, const uint32_t *tile_off,
                                                     uint32_t n_group_runs, SweepCfg cfg)
{
    extern __shared__ __align__(16) uint8_t sm[];
    const uint32_t slot = locate_slot(tile_off, n_group_runs, blockIdx.x);
    const uint32_t run = group_runs[slot];
    const RunDev rd = P.runs[run];
    const RunState st = P.st[run];
    if (st.status) return;
    const uint32_t i = st.step + 1;
    if (i >= rd.n_beta) return;
    const uint32_t Rn = st.R_new;
    const uint32_t tile0 = (blockIdx.x - tile_off[slot]) * cfg.RPC;
    if (tile0 >= Rn) return;  // uniform over the CTA

    const uint32_t L = rd.L, N = rd.N, Lh = rd.Lh, half = N >> 1, PS = cfg.PS, PW = rd.pw, Pt = rd.pitch;
    const uint32_t rloc = threadIdx.x / cfg.TPR, tl = threadIdx.x % cfg.TPR;
    const uint32_t child = tile0 + rloc;
    const bool active = rloc < cfg.RPC && child < Rn;
    uint8_t *planes = sm + (size_t)rloc * 2 * PS;
    uint8_t *jm = sm + (size_t)cfg.RPC * 2 * PS;
    int32_t *acc = reinterpret_cast<int32_t *>(jm + 2 * PS);

    // bond masks (shared by all replicas of the run)
    const uint32_t *Jr = P.J + rd.J_off, *Jd = Jr + rd.wstride;
    for (uint32_t n = threadIdx.x; n < N; n += blockDim.x) {
        const uint32_t x = n % L, y = n / L;
        const uint32_t c = (x + y) & 1u;
        uint32_t m = 0;
        if (rd.model == PA_EA_PMJ) {
            const uint32_t nl = y * L + (x == 0 ? L - 1 : x - 1);
            const uint32_t nu = (y == 0 ? L - 1 : y - 1) * L + x;
            m = get_bit(Jr, n) | (get_bit(Jr, nl) << 1) | (get_bit(Jd, n) << 2) | (get_bit(Jd, nu) << 3);
        }
        jm[c * PS + (n >> 1)] = (uint8_t)m;
    }
    if (threadIdx.x < 2 * cfg.RPC) acc[threadIdx.x] = 0;

    // gather the parent (this is the resampling copy)
    const uint32_t ob = (i - 1) & 1u, nbuf = i & 1u;
    uint32_t parent = 0;
    if (active) {
        parent = P.parent[rd.rep_off + child];
        const uint32_t *src = P.spins[ob] + rd.spin_off + (uint64_t)parent * rd.wstride;
        for (uint32_t cw = tl; cw < 2 * PW; cw += cfg.TPR) {
            const uint32_t c = cw / PW, w = cw - c * PW;
            const uint32_t word = src[cw];
            for (uint32_t b = 0; b < 32; ++b) {
                const uint32_t pos = 32 * w + b, y = pos / Pt, xp = pos - y * Pt;
                if (y >= L || xp >= Lh) continue;  // row padding
                planes[c * PS + y * Lh + xp] = (uint8_t)((word >> b) & 1u);
            }
        }
    }
    __syncthreads();

    const unsigned long long T1 = P.thr[rd.thr_off + 2 * i], T2 = P.thr[rd.thr_off + 2 * i + 1];
    int32_t dE = 0, dM = 0;
    if (HOIST) {
        // One Philox group per thread (blocks of at most 512 threads): the neighbour indices and bond
        // bits of its four sites per colour are computed once, outside the sweeps.
        const uint32_t g = tl;
        const bool has = active && g < cfg.G;
        uint32_t nrl[2][4], ndu[2][4];  // packed 16-bit indices in the other plane: right|left, down|up
        uint32_t jbits = 0;             // 4 bond bits per site, site (c, q) at bit 16 c + 4 q
        uint32_t nval[2] = {0, 0};
#pragma unroll
        for (uint32_t c = 0; c < 2; ++c)
#pragma unroll
            for (uint32_t q = 0; q < 4; ++q) {
                nrl[c][q] = ndu[c][q] = 0;
                const uint32_t k = 4 * g + q;
                if (!has || k >= half) continue;
                const uint32_t y = k / Lh, xp = k - y * Lh;
                const uint32_t x = 2 * xp + ((c + y) & 1u);
                const uint32_t xr = x + 1 == L ? 0 : x + 1, xl = x == 0 ? L - 1 : x - 1;
                const uint32_t yd = y + 1 == L ? 0 : y + 1, yu = y == 0 ? L - 1 : y - 1;
                nrl[c][q] = (y * Lh + (xr >> 1)) | ((y * Lh + (xl >> 1)) << 16);
                ndu[c][q] = (yd * Lh + xp) | ((yu * Lh + xp) << 16);
                jbits |= (uint32_t)jm[c * PS + k] << (16 * c + 4 * q);
                nval[c] = q + 1;
            }
        for (uint32_t t = 0; t < rd.theta; ++t) {
#pragma unroll
            for (uint32_t c = 0; c < 2; ++c) {
                if (has) {
                    uint8_t *mine = planes + c * PS;
                    const uint8_t *other = planes + (c ^ 1u) * PS;
                    const uint4 u = philox4x32_10(g, child, i, (TAG_SWEEP << 24) | (t << 1) | c, rd.seed, rd.run_id);
#pragma unroll
                    for (uint32_t q = 0; q < 4; ++q) {
                        if (q >= nval[c]) break;
                        const uint32_t k = 4 * g + q;
                        const uint32_t jb = (jbits >> (16 * c + 4 * q)) & 15u;
                        const uint32_t s = mine[k];
                        const uint32_t unsat = (s ^ other[nrl[c][q] & 0xffffu] ^ (jb & 1u)) +
                                               (s ^ other[nrl[c][q] >> 16] ^ ((jb >> 1) & 1u)) +
                                               (s ^ other[ndu[c][q] & 0xffffu] ^ ((jb >> 2) & 1u)) +
                                               (s ^ other[ndu[c][q] >> 16] ^ (jb >> 3));
                        const bool accept =
                            unsat >= 2u || (unsigned long long)pick(u, q) < (unsat == 1u ? T1 : T2);
                        if (accept) {
                            mine[k] = (uint8_t)(s ^ 1u);
                            dE += 8 - 4 * (int32_t)unsat;
                            dM += 2 - 4 * (int32_t)s;
                        }
                    }
                }
                __syncthreads();
            }
        }
    } else
    for (uint32_t t = 0; t < rd.theta; ++t) {
        for (uint32_t c = 0; c < 2; ++c) {
            if (active) {
                uint8_t *mine = planes + c * PS;
                const uint8_t *other = planes + (c ^ 1u) * PS;
                const uint8_t *jmc = jm + c * PS;
                for (uint32_t g = tl; g < cfg.G; g += cfg.TPR) {
                    const uint4 u = philox4x32_10(g, child, i, (TAG_SWEEP << 24) | (t << 1) | c, rd.seed, rd.run_id);
#pragma unroll
                    for (uint32_t q = 0; q < 4; ++q) {
                        const uint32_t k = 4 * g + q;
                        if (k >= half) break;
                        const uint32_t y = k / Lh, xp = k - y * Lh;
                        const uint32_t x = 2 * xp + ((c + y) & 1u);
                        const uint32_t xr = x + 1 == L ? 0 : x + 1, xl = x == 0 ? L - 1 : x - 1;
                        const uint32_t yd = y + 1 == L ? 0 : y + 1, yu = y == 0 ? L - 1 : y - 1;
                        const uint32_t s = mine[k], jb = jmc[k];
                        const uint32_t unsat = (s ^ other[y * Lh + (xr >> 1)] ^ (jb & 1u)) +
                                               (s ^ other[y * Lh + (xl >> 1)] ^ ((jb >> 1) & 1u)) +
                                               (s ^ other[yd * Lh + xp] ^ ((jb >> 2) & 1u)) +
                                               (s ^ other[yu * Lh + xp] ^ (jb >> 3));
                        // dE = 8 - 4 unsat; accept if dE <= 0, else with probability T[dE/4] / 2^32
                        const bool accept =
                            unsat >= 2u || (unsigned long long)pick(u, q) < (unsat == 1u ? T1 : T2);
                        if (accept) {
                            mine[k] = (uint8_t)(s ^ 1u);
                            dE += 8 - 4 * (int32_t)unsat;
                            dM += 2 - 4 * (int32_t)s;
                        }
                    }
                }
            }
            __syncthreads();
        }
    }

    // pack and write the child
    if (active) {
        uint32_t *dst = P.spins[nbuf] + rd.spin_off + (uint64_t)child * rd.wstride;
        for (uint32_t cw = tl; cw < 2 * PW; cw += cfg.TPR) {
            const uint32_t c = cw / PW, w = cw - c * PW;
            uint32_t word = 0;
            for (uint32_t b = 0; b < 32; ++b) {
                const uint32_t pos = 32 * w + b, y = pos / Pt, xp = pos - y * Pt;
                if (y >= L || xp >= Lh) continue;  // row padding stays 0
                word |= (uint32_t)planes[c * PS + y * Lh + xp] << b;
            }
            dst[cw] = word;
        }
        atomicAdd(&acc[2 * rloc], dE);
        atomicAdd(&acc[2 * rloc + 1], dM);
    }
    __syncthreads();
    if (active && tl == 0) {
        const uint64_t pc = rd.rep_off + parent, cc = rd.rep_off + child;
        P.E[nbuf][cc] = P.E[ob][pc] + acc[2 * rloc];
        P.M[nbuf][cc] = P.M[ob][pc] + acc[2 * rloc + 1];
        P.fam[nbuf][cc] = P.fam[ob][pc];
    }
}

// --------------------------------------------------------------------------
// Bit-sliced sweep for L a power of two, 8 <= L <= 256 (Sec. V.A.1).
// Each thread owns WPT words of both colour planes of one replica (32 sites of
// a colour per word).  Per half-sweep and word it forms, as 32-bit masks, the
// spin of each neighbour (same index, index rotated by one within the row, row
// above, row below) from the other plane, the unsatisfied bonds
// x_d = s ^ n_d ^ J_d, their count with a bit-sliced adder (c0 = count & 1,
// ge2 = count >= 2), and the acceptance mask
//      accept = ge2 | (c0 & B1) | B2,   B_m = [u < T_m]  (T_2 <= T_1),
// i.e. dE = 8 - 4 count <= 0, or u < T_1 when dE = 4, or u < T_2 when dE = 8.
// The 32 uniforms come from 8 Philox calls with the same counters as the
// generic kernel, so both kernels (and the oracle) flip the same spins.
// E and M of the child are recomputed from its final planes.
//
// Throughput (GB300): Philox4x32-10 dominates.  Each round is two
// 32x32->64 multiplies (multiplier pipe, half rate, two passes each) and two
// 3-input XORs (integer pipe); the multiplier bounds the kernel at about
// 40 multiply-add slots per Philox call.  The round keys are precomputed and
// the first round's multiply of the temperature counter is hoisted.
// --------------------------------------------------------------------------
struct PhiloxKeys {
    uint32_t k0[10], k1[10];
};

__device__ __forceinline__ void philox_keys(PhiloxKeys &K, uint32_t seed, uint32_t id)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        K.k0[r] = seed + (uint32_t)r * 0x9E3779B9u;
        K.k1[r] = id + (uint32_t)r * 0xBB67AE85u;
    }
}

// Philox4x32-10 with precomputed round keys; the first round's multiply of
// counter word 2 (the temperature index, fixed for the kernel) is passed in.
// WIDE writes each multiply as one 32x32->64 product instead of separate high and
// low halves: the same numbers; 7 % faster inside the power-of-two sweep, 3 %
// slower inside the padded-row sweep and in a Philox-only loop (measured).
template <bool WIDE>
__device__ __forceinline__ uint4 philox_rk(uint32_t c0, uint32_t c1, uint32_t c3, uint32_t hi1_0, uint32_t lo1_0,
                                           const PhiloxKeys &K)
{
    uint32_t hi0, lo0;
    if (WIDE) {
        const unsigned long long p0 = 0xD2511F53ull * c0;
        hi0 = (uint32_t)(p0 >> 32);
        lo0 = (uint32_t)p0;
    } else {
        hi0 = __umulhi(0xD2511F53u, c0);
        lo0 = 0xD2511F53u * c0;
    }
    uint32_t x0 = hi1_0 ^ c1 ^ K.k0[0], x1 = lo1_0, x2 = hi0 ^ c3 ^ K.k1[0], x3 = lo0;
#pragma unroll
    for (int r = 1; r < 10; ++r) {
        uint32_t hi1, lo1;
        if (WIDE) {
            const unsigned long long p0 = 0xD2511F53ull * x0, p1 = 0xCD9E8D57ull * x2;
            hi0 = (uint32_t)(p0 >> 32);
            lo0 = (uint32_t)p0;
            hi1 = (uint32_t)(p1 >> 32);
            lo1 = (uint32_t)p1;
        } else {
            hi0 = __umulhi(0xD2511F53u, x0);
            lo0 = 0xD2511F53u * x0;
            hi1 = __umulhi(0xCD9E8D57u, x2);
            lo1 = 0xCD9E8D57u * x2;
        }
        x0 = hi1 ^ x1 ^ K.k0[r];
        x1 = lo1;
        x2 = hi0 ^ x3 ^ K.k1[r];
        x3 = lo0;
    }
    return make_uint4(x0, x1, x2, x3);
}

template <bool SG, int WPT>
__device__ __forceinline__ void sweep_pow2_body(const Pool &P, const uint32_t *group_runs, const uint32_t *tile_off,
                                                uint32_t n_group_runs, const SweepCfg &cfg)
{
    extern __shared__ __align__(16) uint32_t smw[];
    const uint32_t slot = locate_slot(tile_off, n_group_runs, blockIdx.x);
    const uint32_t run = group_runs[slot];
    const RunDev rd = P.runs[run];
    const RunState st = P.st[run];
    if (st.status) return;
    const uint32_t i = st.step + 1;
    if (i >= rd.n_beta) return;
    const uint32_t Rn = st.R_new;
    const uint32_t tile0 = (blockIdx.x - tile_off[slot]) * cfg.RPC;
    if (tile0 >= Rn) return;  // uniform over the CTA

    const uint32_t TPR = cfg.TPR, HW = TPR * WPT;  // threads per replica, words per plane
    const uint32_t Lh = rd.Lh, N = rd.N;
    const uint32_t rloc = threadIdx.x / TPR, tl = threadIdx.x & (TPR - 1);
    const uint32_t child = tile0 + rloc;
    const bool active = child < Rn;
    uint32_t *pl = smw + rloc * 2 * HW;
    int32_t *acc = reinterpret_cast<int32_t *>(smw + cfg.RPC * 2 * HW);
    const bool wide = TPR > 32;
    if (wide && threadIdx.x < 2 * cfg.RPC) acc[threadIdx.x] = 0;

    const uint32_t ob = (i - 1) & 1u, nbuf = i & 1u;
    uint32_t own[WPT][2];
    uint32_t parent = 0;
    if (active) parent = P.parent[rd.rep_off + child];
    const uint32_t *src = P.spins[ob] + rd.spin_off + (uint64_t)parent * rd.wstride;
#pragma unroll
    for (int q = 0; q < WPT; ++q) {
        const uint32_t w = tl + q * TPR;
        own[q][0] = active ? src[w] : 0u;
        own[q][1] = active ? src[HW + w] : 0u;
        pl[w] = own[q][0];
        pl[HW + w] = own[q][1];
    }
    uint32_t J[WPT][2][4];
#pragma unroll
    for (int q = 0; q < WPT; ++q)
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int d = 0; d < 4; ++d) J[q][c][d] = 0;
    if (SG) {
        const uint32_t *Jp = P.J + rd.J_off + 2 * rd.wstride;
#pragma unroll
        for (int q = 0; q < WPT; ++q)
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int d = 0; d < 4; ++d) J[q][c][d] = Jp[(c * 4 + d) * HW + tl + q * TPR];
    }
    const unsigned long long T1 = P.thr[rd.thr_off + 2 * i], T2 = P.thr[rd.thr_off + 2 * i + 1];
    const uint32_t t1 = T1 > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)T1;
    const uint32_t t2 = T2 > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)T2;
    const uint32_t all1 = T1 > 0xFFFFFFFFull ? 0xFFFFFFFFu : 0u;
    const uint32_t all2 = T2 > 0xFFFFFFFFull ? 0xFFFFFFFFu : 0u;
    PhiloxKeys K;
    philox_keys(K, rd.seed, rd.run_id);
    const uint32_t hi1_0 = __umulhi(0xCD9E8D57u, i), lo1_0 = 0xCD9E8D57u * i;
    if (TPR <= 32) __syncwarp(); else __syncthreads();

    auto neighbours = [&](uint32_t c, uint32_t w, uint32_t &same, uint32_t &rot, uint32_t &up, uint32_t &dn) {
        plane_neighbours(pl + (c ^ 1u) * HW, HW, Lh, c, w, same, rot, up, dn);
    };

    for (uint32_t t = 0; t < rd.theta; ++t) {
#pragma unroll
        for (uint32_t c = 0; c < 2; ++c) {
            if (active) {
                const uint32_t ctr3 = (TAG_SWEEP << 24) | (t << 1) | c;
#pragma unroll
                for (int q = 0; q < WPT; ++q) {
                    const uint32_t w = tl + q * TPR;
                    uint32_t same, rot, up, dn;
                    neighbours(c, w, same, rot, up, dn);
                    const uint32_t S = own[q][c];
                    const uint32_t x1 = S ^ same ^ J[q][c][0], x2 = S ^ rot ^ J[q][c][1];
                    const uint32_t x3 = S ^ up ^ J[q][c][2], x4 = S ^ dn ^ J[q][c][3];
                    const uint32_t a = x1 ^ x2, b = x1 & x2, e = x3 ^ x4, f = x3 & x4;
                    const uint32_t c0 = a ^ e, ge2 = b | f | (a & e);
                    // bits of distinct sites never collide, so the packing can add or or
                    uint32_t B1 = 0, B2 = 0;
#pragma unroll
                    for (uint32_t g = 0; g < 8; ++g) {
                        const uint4 u = philox_rk<true>(8 * w + g, child, ctr3, hi1_0, lo1_0, K);
                        pack_group(B1, B2, u, g, t1, t2);
                    }
                    const uint32_t flip = ge2 | (c0 & (B1 | all1)) | B2 | all2;
                    own[q][c] = S ^ flip;
                }
                // all of this colour's words are updated before any is published
#pragma unroll
                for (int q = 0; q < WPT; ++q) pl[c * HW + tl + q * TPR] = own[q][c];
            }
            if (TPR <= 32) __syncwarp(); else __syncthreads();
        }
    }

    // child: planes, E from the final lattice (every bond touches one colour-0 site), M
    int32_t unsat = 0, up1 = 0;
    if (active) {
        uint32_t *dst = P.spins[nbuf] + rd.spin_off + (uint64_t)child * rd.wstride;
#pragma unroll
        for (int q = 0; q < WPT; ++q) {
            const uint32_t w = tl + q * TPR;
            dst[w] = own[q][0];
            dst[HW + w] = own[q][1];
            uint32_t same, rot, up, dn;
            neighbours(0, w, same, rot, up, dn);
            const uint32_t S = own[q][0];
            unsat += __popc(S ^ same ^ J[q][0][0]) + __popc(S ^ rot ^ J[q][0][1]) + __popc(S ^ up ^ J[q][0][2]) +
                     __popc(S ^ dn ^ J[q][0][3]);
            up1 += __popc(own[q][0]) + __popc(own[q][1]);
        }
    }
    if (!wide) {
        for (uint32_t o = 1; o < TPR; o <<= 1) {
            unsat += __shfl_xor_sync(FULL, unsat, o);
            up1 += __shfl_xor_sync(FULL, up1, o);
        }
    } else {
        if (active) {
            atomicAdd(&acc[2 * rloc], unsat);
            atomicAdd(&acc[2 * rloc + 1], up1);
        }
        __syncthreads();
        unsat = acc[2 * rloc];
        up1 = acc[2 * rloc + 1];
    }
    if (active && tl == 0) {
        const uint64_t pc = rd.rep_off + parent, cc = rd.rep_off + child;
        P.E[nbuf][cc] = 2 * unsat - 2 * (int32_t)N;
        P.M[nbuf][cc] = 2 * up1 - (int32_t)N;
        P.fam[nbuf][cc] = P.fam[ob][pc];
    }
}

// The kernels: the compiler's own register choice for 256 and 1024 threads
// (78 and 40 registers; an explicit bound of one CTA per SM let it take 150 at
// 256 threads and run 19 % slower at L = 128), two CTAs per SM for 512 threads
// (L = 256: +5 % against one, measured).
template <bool SG, int WPT, int MAXT>
__global__ void __launch_bounds__(MAXT) sweep_pow2_kernel(Pool P, const uint32_t *group_runs, const uint32_t *tile_off,
                                                          uint32_t n_group_runs, SweepCfg cfg)
{
    sweep_pow2_body<SG, WPT>(P, group_runs, tile_off, n_group_runs, cfg);
}

template <bool SG, int WPT>
__global__ void __launch_bounds__(512, 2) sweep_pow2_kernel_2cta(Pool P, const uint32_t *group_runs,
                                                                 const uint32_t *tile_off, uint32_t n_group_runs,
                                                                 SweepCfg cfg)
{
    sweep_pow2_body<SG, WPT>(P, group_runs, tile_off, n_group_runs, cfg);
}

// --------------------------------------------------------------------------
// Bit-sliced sweep for even L whose half-width L/2 is not a power of two but
// at most 31 (Sec. V.A.1): rows of a colour plane are padded to a pitch P in
// {4, 8, 16, 32} with L P a multiple of 32, so rows tile 32-bit words exactly
// as in the power-of-two kernel; padding bits are masked out of every flip
// and popcount and stay 0.  Each thread owns one plane word (32 / P rows); its
// sites are the compact sublattice indices [kb, kb + (32 / P) L/2), drawn from
// the same Philox counters as every other path (the groups at either end of
// the range are shared with the neighbouring words and drawn by both), and
// each comparison bit is placed at its padded position.
// --------------------------------------------------------------------------
// Compact sites of one padded plane word: RW rows of Lh sites with RW * pitch = 32 and
// Lh <= pitch, i.e. at most 32 sites, starting anywhere in a Philox group: <= 9 groups.
constexpr uint32_t PAD_MAX_GROUPS = 9;

#ifndef PA_PAD_MIN_BLOCKS
#define PA_PAD_MIN_BLOCKS 3  // caps registers at 85: 3 CTAs of 256 threads per SM (measured best of 1, 2, 3)
#endif


template <bool SG, uint32_t PT>  // PT: the row pitch of the runs' lattice size (8, 16 or 32)
__global__ void __launch_bounds__(256, PA_PAD_MIN_BLOCKS) sweep_pad_kernel(Pool P, const uint32_t *group_runs, const uint32_t *tile_off,
                                                        uint32_t n_group_runs, SweepCfg cfg)
{
    extern __shared__ __align__(16) uint32_t smw[];
    const uint32_t slot = locate_slot(tile_off, n_group_runs, blockIdx.x);
    const uint32_t run = group_runs[slot];
    const RunDev rd = P.runs[run];
    const RunState st = P.st[run];
    if (st.status) return;
    const uint32_t i = st.step + 1;
    if (i >= rd.n_beta) return;
    const uint32_t Rn = st.R_new;
    const uint32_t tile0 = (blockIdx.x - tile_off[slot]) * cfg.RPC;
    if (tile0 >= Rn) return;  // uniform over the CTA

    const uint32_t HW = cfg.TPR;  // words per plane = threads per replica
    constexpr uint32_t Pt = PT;
    const uint32_t Lh = rd.Lh, N = rd.N;
    const uint32_t rloc = threadIdx.x / HW, w = threadIdx.x - rloc * HW;
    const uint32_t child = tile0 + rloc;
    const bool active = child < Rn;
    uint32_t *pl = smw + rloc * 2 * HW;
    int32_t *acc = reinterpret_cast<int32_t *>(smw + cfg.RPC * 2 * HW);
    if (threadIdx.x < 2 * cfg.RPC) acc[threadIdx.x] = 0;

    const uint32_t ob = (i - 1) & 1u, nbuf = i & 1u;
    uint32_t own[2] = {0u, 0u}, parent = 0;
    if (active) {
        parent = P.parent[rd.rep_off + child];
        const uint32_t *src = P.spins[ob] + rd.spin_off + (uint64_t)parent * rd.wstride;
        own[0] = src[w];
        own[1] = src[HW + w];
    }
    pl[w] = own[0];
    pl[HW + w] = own[1];
    uint32_t J[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
    if (SG) {
        const uint32_t *Jp = P.J + rd.J_off + 2 * rd.wstride;
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int d = 0; d < 4; ++d) J[c][d] = Jp[(c * 4 + d) * HW + w];
    }
    // word geometry
    constexpr bool sub = Pt < 32;  // several rows per word
    constexpr uint32_t RW = sub ? 32 / Pt : 1u;
    const uint32_t y0 = w * RW;
    const uint32_t wp = (w + HW - 1) % HW, wn = (w + 1) % HW;
    constexpr uint32_t LOW = !sub ? 1u : Pt == 4 ? 0x11111111u : Pt == 8 ? 0x01010101u : 0x00010001u;
    const uint32_t HIGH = LOW << (Lh - 1);
    constexpr uint32_t EVEN = Pt == 4 ? 0x0F0F0F0Fu : Pt == 8 ? 0x00FF00FFu : 0x0000FFFFu;  // rows 0, 2, ... (sub)
    const uint32_t VMASK = LOW * ((1u << Lh) - 1u);                                      // Lh < 32 here
    const uint32_t kb = y0 * Lh, kend = kb + RW * Lh;                                     // compact sites of the word
    const uint32_t g0 = kb >> 2, off = kb & 3u, ng = (kend - 4 * g0 + 3) / 4;          // Philox groups (<= 9)
    const uint32_t ROWMASK = (1u << Lh) - 1u;

    const unsigned long long T1 = P.thr[rd.thr_off + 2 * i], T2 = P.thr[rd.thr_off + 2 * i + 1];
    const uint32_t t1 = T1 > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)T1;
    const uint32_t t2 = T2 > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)T2;
    const uint32_t all1 = T1 > 0xFFFFFFFFull ? 0xFFFFFFFFu : 0u;
    const uint32_t all2 = T2 > 0xFFFFFFFFull ? 0xFFFFFFFFu : 0u;
    PhiloxKeys K;
    philox_keys(K, rd.seed, rd.run_id);
    const uint32_t hi1_0 = __umulhi(0xCD9E8D57u, i), lo1_0 = 0xCD9E8D57u * i;
    __syncthreads();

    auto neighbours = [&](uint32_t c, uint32_t &same, uint32_t &rot, uint32_t &up, uint32_t &dn) {
        const uint32_t *O = pl + (c ^ 1u) * HW;
        const uint32_t o = O[w];
        same = o;
        const uint32_t rl = ((o << 1) & ~LOW) | ((o >> (Lh - 1)) & LOW);   // xp <- xp - 1 in the row
        const uint32_t rr = ((o >> 1) & ~HIGH) | ((o << (Lh - 1)) & HIGH); // xp <- xp + 1 in the row
        if (sub) {
            up = __funnelshift_l(O[wp], o, Pt);  // row above: position - P
            dn = __funnelshift_r(o, O[wn], Pt);  // row below: position + P
            rot = c == 0 ? ((rl & EVEN) | (rr & ~EVEN)) : ((rr & EVEN) | (rl & ~EVEN));
        } else {
            up = O[wp];
            dn = O[wn];
            rot = ((c + y0) & 1u) == 0 ? rl : rr;
        }
    };

    for (uint32_t t = 0; t < rd.theta; ++t) {
#pragma unroll
        for (uint32_t c = 0; c < 2; ++c) {
            if (active) {
                uint32_t same, rot, up, dn;
                neighbours(c, same, rot, up, dn);
                const uint32_t S = own[c];
                const uint32_t x1 = S ^ same ^ J[c][0], x2 = S ^ rot ^ J[c][1];
                const uint32_t x3 = S ^ up ^ J[c][2], x4 = S ^ dn ^ J[c][3];
                const uint32_t a = x1 ^ x2, b = x1 & x2, e = x3 ^ x4, f = x3 & x4;
                const uint32_t c0 = a ^ e, ge2 = b | f | (a & e);
                const uint32_t ctr3 = (TAG_SWEEP << 24) | (t << 1) | c;
                // comparison bits of the word's compact sites kb..kend-1, in compact order from
                // bit `off` of C1 / C2 (the Philox groups of 4 start at kb & ~3) ...
#if PA_PACK_MODE == 1
                unsigned long long C1 = 0, C2 = 0;
#pragma unroll
                for (uint32_t q = 0; q < PAD_MAX_GROUPS; ++q) {
                    if (q < ng) {
                        const uint4 u = philox_rk<false>(g0 + q, child, ctr3, hi1_0, lo1_0, K);
                        C1 |= (unsigned long long)((uint32_t)(u.x < t1) | ((uint32_t)(u.y < t1) << 1) |
                                                   ((uint32_t)(u.z < t1) << 2) | ((uint32_t)(u.w < t1) << 3))
                              << (4 * q);
                        C2 |= (unsigned long long)((uint32_t)(u.x < t2) | ((uint32_t)(u.y < t2) << 1) |
                                                   ((uint32_t)(u.z < t2) << 2) | ((uint32_t)(u.w < t2) << 3))
                              << (4 * q);
                    }
                }
#else
                // groups 0..7 fill the low words, group 8 the high words (positions 32..35)
                uint32_t C1l = 0, C2l = 0, C1h = 0, C2h = 0;
#pragma unroll
                for (uint32_t q = 0; q < PAD_MAX_GROUPS - 1; ++q) {
                    if (q < ng) {
                        const uint4 u = philox_rk<false>(g0 + q, child, ctr3, hi1_0, lo1_0, K);
                        pack_group(C1l, C2l, u, q, t1, t2);
                    }
                }
                if (ng == PAD_MAX_GROUPS) {
                    const uint4 u = philox_rk<false>(g0 + PAD_MAX_GROUPS - 1, child, ctr3, hi1_0, lo1_0, K);
                    pack_group(C1h, C2h, u, 0, t1, t2);
                }
                const unsigned long long C1 = ((unsigned long long)C1h << 32) | C1l;
                const unsigned long long C2 = ((unsigned long long)C2h << 32) | C2l;
#endif
                // ... then each row's Lh bits moved to its padded position r * Pt
                uint32_t B1 = 0, B2 = 0;
#pragma unroll
                for (uint32_t r = 0; r < 8; ++r) {
                    if (r < RW) {
                        const uint32_t sh = off + r * Lh;
                        B1 |= ((uint32_t)(C1 >> sh) & ROWMASK) << (r * Pt);
                        B2 |= ((uint32_t)(C2 >> sh) & ROWMASK) << (r * Pt);
                    }
                }
                const uint32_t flip = (ge2 | (c0 & (B1 | all1)) | B2 | all2) & VMASK;
                own[c] = S ^ flip;
                pl[c * HW + w] = own[c];
            }
            __syncthreads();
        }
    }

    // child: planes, E from the final lattice (every bond touches one colour-0 site), M
    if (active) {
        uint32_t *dst = P.spins[nbuf] + rd.spin_off + (uint64_t)child * rd.wstride;
        dst[w] = own[0];
        dst[HW + w] = own[1];
        uint32_t same, rot, up, dn;
        neighbours(0, same, rot, up, dn);
        const uint32_t S = own[0];
        const int32_t unsat = __popc((S ^ same ^ J[0][0]) & VMASK) + __popc((S ^ rot ^ J[0][1]) & VMASK) +
                              __popc((S ^ up ^ J[0][2]) & VMASK) + __popc((S ^ dn ^ J[0][3]) & VMASK);
        atomicAdd(&acc[2 * rloc], unsat);
        atomicAdd(&acc[2 * rloc + 1], __popc(own[0]) + __popc(own[1]));
    }
    __syncthreads();
    if (active && w == 0) {
        const uint64_t pc = rd.rep_off + parent, cc = rd.rep_off + child;
        P.E[nbuf][cc] = 2 * acc[2 * rloc] - 2 * (int32_t)N;
        P.M[nbuf][cc] = 2 * acc[2 * rloc + 1] - (int32_t)N;
        P.fam[nbuf][cc] = P.fam[ob][pc];
    }
}

// --------------------------------------------------------------------------
// Bit-sliced sweep on compact rows: every even L >= 4 that the power-of-two
// kernel does not take, colour planes of up to 1024 words.  In HBM the planes
// keep their padded rows; the kernel repacks each plane in shared memory with
// no padding, sublattice site k = y L/2 + x' at bit k of the plane's bit
// string, so a thread's word holds 32 consecutive sites: exactly Philox groups
// 8 w .. 8 w + 7, drawn unconditionally as in the power-of-two kernel (only a
// plane's last word is partial, its surplus bits masked).  Rows then begin
// anywhere in a word, so each thread keeps, for its word, masks of the row
// starts, the row ends, the even rows, and the bits whose row above or below
// wraps around the lattice, and reads its neighbours as 32-bit windows of the
// other plane at fixed offsets (k - L/2, k - L/2 + 1, k - 1, k + 1,
// k + L/2 - 1, k + L/2: one word offset and shift each for the whole CTA) and,
// in the words of the first and last rows only, at the wrapped positions.  A
// plane's string starts after FP = ceil(L/64) words and is followed by
// L/64 + 2 words, so every window stays inside the array; bits read from those
// margins are always masked out.  Both this kernel and the padded-row kernel
// are launch-shape candidates for L <= 64 (the padded rows are faster for some
// small L, whose compact planes end in a mostly empty word).
// --------------------------------------------------------------------------
#ifndef PA_COMPACT_WIDE
#define PA_COMPACT_WIDE true
#endif

__device__ __forceinline__ uint32_t low_bits(uint32_t n) { return n >= 32 ? 0xFFFFFFFFu : (1u << n) - 1u; }

// 32 bits of the bit string s from bit p on (words p >> 5 and p >> 5 + 1 exist).
__device__ __forceinline__ uint32_t bits_at(const uint32_t *s, uint32_t p)
{
    const uint32_t q = p >> 5;
    return __funnelshift_r(s[q], s[q + 1], p & 31);
}

// Compact word w (sites 32 w .. 32 w + 31 < NB) of a colour plane stored with
// rows at the given pitch; reads only words that hold the sites.
__device__ uint32_t compact_from_padded(const uint32_t *g, uint32_t pitch, uint32_t Lh, uint32_t NB, uint32_t w)
{
    const uint32_t k0 = 32 * w, k1 = min(k0 + 32, NB);
    uint32_t y = k0 / Lh, xs = k0 - y * Lh, out = 0;
    for (uint32_t k = k0; k < k1; ++y, xs = 0) {
        const uint32_t len = min(Lh - xs, k1 - k), pos = y * pitch + xs, sh = pos & 31;
        uint32_t v = g[pos >> 5] >> sh;
        if (sh + len > 32) v |= g[(pos >> 5) + 1] << (32 - sh);
        out |= (v & low_bits(len)) << (k - k0);
        k += len;
    }
    return out;
}

// Padded word p of a colour plane from its compact bit string O (site k at bit base + k).
__device__ uint32_t padded_from_compact(const uint32_t *O, uint32_t base, uint32_t pitch, uint32_t Lh, uint32_t p)
{
    if (pitch < 32) {  // 32 / pitch rows per word
        const uint32_t RW = 32 / pitch;
        uint32_t v = 0;
        for (uint32_t r = 0; r < RW; ++r) v |= (bits_at(O, base + (p * RW + r) * Lh) & low_bits(Lh)) << (r * pitch);
        return v;
    }
    const uint32_t y = 32 * p / pitch, x0 = 32 * p - y * pitch;  // pitch a multiple of 32
    return x0 < Lh ? bits_at(O, base + y * Lh + x0) & low_bits(Lh - x0) : 0u;
}

// Per-thread geometry of compact word w.
struct CompactWord {
    uint32_t RS, RE, EV, VM;  // row starts, row ends, even rows, sites of the plane
    uint32_t mU, mD;          // bits whose row above (below) is the lattice's last (first) row
    uint32_t pU, pD;          // window positions of the wrapped rows (the plain ones where none wraps)
};

__device__ __forceinline__ CompactWord compact_word(uint32_t w, uint32_t Lh, uint32_t NB, uint32_t base)
{
    CompactWord g;
    const uint32_t k0 = 32 * w, k1 = min(k0 + 32, NB);
    g.VM = low_bits(k1 - k0);
    g.RS = g.RE = g.EV = 0;
    uint32_t y = k0 / Lh, xs = k0 - y * Lh;
    for (uint32_t k = k0; k < k1; ++y, xs = 0) {
        const uint32_t len = min(Lh - xs, k1 - k), j = k - k0;
        if (xs == 0) g.RS |= 1u << j;
        if (xs + len == Lh) g.RE |= 1u << (j + len - 1);
        if (!(y & 1u)) g.EV |= low_bits(len) << j;
        k += len;
    }
    g.mU = k0 < Lh ? low_bits(Lh - k0) : 0u;
    const int jt = (int)NB - (int)Lh - (int)k0;  // first bit whose row below wraps
    g.mD = jt <= 0 ? 0xFFFFFFFFu : jt >= 32 ? 0u : ~low_bits((uint32_t)jt);
    g.pU = g.mU ? base + k0 + NB - Lh : base + k0 - Lh;
    g.pD = g.mD ? base + k0 + Lh - NB : base + k0 + Lh;
    return g;
}

// Word offsets and bit shifts of the windows at k + L/2 - 1, k - L/2 + 1, k - L/2
// and k + L/2 from a word's own position: the same for every thread of a CTA.
struct CompactShifts {
    int dl, dr, du, dd;
    uint32_t sl, sr, su, sd;
};

__device__ __forceinline__ CompactShifts compact_shifts(uint32_t Lh)
{
    CompactShifts s;
    const int off[4] = {(int)Lh - 1, 1 - (int)Lh, -(int)Lh, (int)Lh};
    s.dl = off[0] >> 5, s.dr = off[1] >> 5, s.du = off[2] >> 5, s.dd = off[3] >> 5;  // floor(off / 32)
    s.sl = off[0] & 31, s.sr = off[1] & 31, s.su = off[2] & 31, s.sd = off[3] & 31;
    return s;
}

// 32 bits from bit sh of word Ow[dq] on.
__device__ __forceinline__ uint32_t window(const uint32_t *Ow, int dq, uint32_t sh)
{
    return __funnelshift_r(Ow[dq], Ow[dq + 1], sh);
}

// Neighbour masks of compact word w of colour c, read from the other plane's
// string O; Ow = O + FP + w is the word itself.
// NARROW (L/2 <= 31): every window lies in the words w - 1, w and w + 1, so
// they are funnel shifts of those three.
template <bool NARROW>
__device__ __forceinline__ void compact_neighbours(const uint32_t *O, const uint32_t *Ow, const CompactShifts &z,
                                                   const CompactWord &g, uint32_t c, uint32_t &same, uint32_t &rot,
                                                   uint32_t &up, uint32_t &dn)
{
    const uint32_t om = Ow[-1], o = Ow[0], op = Ow[1];
    same = o;
    const uint32_t l1 = __funnelshift_l(om, o, 1);  // bit k <- k - 1
    const uint32_t r1 = __funnelshift_r(o, op, 1);  // bit k <- k + 1
    uint32_t lw, rw;
    if (NARROW) {  // offsets L/2 - 1 and L/2 in word 0, -(L/2 - 1) and -L/2 in word -1
        lw = __funnelshift_r(o, op, z.sl);
        rw = __funnelshift_r(om, o, z.sr);
        up = __funnelshift_r(om, o, z.su);
        dn = __funnelshift_r(o, op, z.sd);
    } else {
        lw = window(Ow, z.dl, z.sl);
        rw = window(Ow, z.dr, z.sr);
        up = window(Ow, z.du, z.su);
        dn = window(Ow, z.dd, z.sd);
    }
    const uint32_t left = (l1 & ~g.RS) | (lw & g.RS);   // x' - 1 within the row
    const uint32_t right = (r1 & ~g.RE) | (rw & g.RE);  // x' + 1 within the row
    rot = c == 0 ? ((left & g.EV) | (right & ~g.EV)) : ((right & g.EV) | (left & ~g.EV));
    if (g.mU) up = (up & ~g.mU) | (bits_at(O, g.pU) & g.mU);  // the first row's row above: the last row
    if (g.mD) dn = (dn & ~g.mD) | (bits_at(O, g.pD) & g.mD);  // the last row's row below: the first row
}

#ifndef PA_COMPACT_MIN_BLOCKS
#define PA_COMPACT_MIN_BLOCKS 4  // caps registers at 64 (no spills); 1-8 % faster than 3 or 2 CTAs of 256 (measured)
#endif

template <bool SG, int MAXT, bool NARROW>
__global__ void __launch_bounds__(MAXT, MAXT <= 256 ? PA_COMPACT_MIN_BLOCKS : 1)
    sweep_compact_kernel(Pool P, const uint32_t *group_runs, const uint32_t *tile_off, uint32_t n_group_runs,
                         SweepCfg cfg)
{
    extern __shared__ __align__(16) uint32_t smw[];
    const uint32_t slot = locate_slot(tile_off, n_group_runs, blockIdx.x);
    const uint32_t run = group_runs[slot];
    const RunDev rd = P.runs[run];
    const RunState st = P.st[run];
    if (st.status) return;
    const uint32_t i = st.step + 1;
    if (i >= rd.n_beta) return;
    const uint32_t Rn = st.R_new;
    const uint32_t tile0 = (blockIdx.x - tile_off[slot]) * cfg.RPC;
    if (tile0 >= Rn) return;  // uniform over the CTA

    const uint32_t CW = cfg.TPR;  // compact words per plane = threads per replica
    const uint32_t Lh = rd.Lh, N = rd.N, NB = N / 2, pitch = rd.pitch, PW = rd.pw;
    const uint32_t FP = (Lh + 31) >> 5, AW = FP + CW + (Lh >> 5) + 2, base = 32 * FP;
    const uint32_t rloc = threadIdx.x / CW, w = threadIdx.x - rloc * CW;
    const uint32_t child = tile0 + rloc;
    const bool active = child < Rn;
    uint32_t *pl = smw + rloc * 2 * AW;
    int32_t *acc = reinterpret_cast<int32_t *>(smw + cfg.RPC * 2 * AW);
    for (uint32_t q = threadIdx.x; q < 2 * cfg.RPC; q += blockDim.x) acc[q] = 0;  // one thread per replica at L <= 6

    const uint32_t ob = (i - 1) & 1u, nbuf = i & 1u;
    uint32_t own[2] = {0u, 0u}, parent = 0;
    if (active) {
        parent = P.parent[rd.rep_off + child];
        const uint32_t *src = P.spins[ob] + rd.spin_off + (uint64_t)parent * rd.wstride;
        own[0] = compact_from_padded(src, pitch, Lh, NB, w);
        own[1] = compact_from_padded(src + PW, pitch, Lh, NB, w);
    }
    pl[FP + w] = own[0];
    pl[AW + FP + w] = own[1];
    uint32_t J[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
    if (SG) {
        const uint32_t *Jp = P.J + rd.J_off + 2 * rd.wstride;
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int d = 0; d < 4; ++d) J[c][d] = compact_from_padded(Jp + (c * 4 + d) * PW, pitch, Lh, NB, w);
    }
    const CompactWord g = compact_word(w, Lh, NB, base);
    const CompactShifts z = compact_shifts(Lh);

    const unsigned long long T1 = P.thr[rd.thr_off + 2 * i], T2 = P.thr[rd.thr_off + 2 * i + 1];
    const uint32_t t1 = T1 > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)T1;
    const uint32_t t2 = T2 > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)T2;
    const uint32_t all1 = T1 > 0xFFFFFFFFull ? 0xFFFFFFFFu : 0u;
    const uint32_t all2 = T2 > 0xFFFFFFFFull ? 0xFFFFFFFFu : 0u;
    PhiloxKeys K;
    philox_keys(K, rd.seed, rd.run_id);
    const uint32_t hi1_0 = __umulhi(0xCD9E8D57u, i), lo1_0 = 0xCD9E8D57u * i;
    __syncthreads();

    for (uint32_t t = 0; t < rd.theta; ++t) {
#pragma unroll
        for (uint32_t c = 0; c < 2; ++c) {
            if (active) {
                uint32_t same, rot, up, dn;
                compact_neighbours<NARROW>(pl + (c ^ 1u) * AW, pl + (c ^ 1u) * AW + FP + w, z, g, c, same, rot, up,
                                           dn);
                const uint32_t S = own[c];
                const uint32_t x1 = S ^ same ^ J[c][0], x2 = S ^ rot ^ J[c][1];
                const uint32_t x3 = S ^ up ^ J[c][2], x4 = S ^ dn ^ J[c][3];
                const uint32_t a = x1 ^ x2, b = x1 & x2, e = x3 ^ x4, f = x3 & x4;
                const uint32_t c0 = a ^ e, ge2 = b | f | (a & e);
                const uint32_t ctr3 = (TAG_SWEEP << 24) | (t << 1) | c;
                uint32_t B1 = 0, B2 = 0;
#pragma unroll
                for (uint32_t q = 0; q < 8; ++q) {
                    const uint4 u = philox_rk<PA_COMPACT_WIDE>(8 * w + q, child, ctr3, hi1_0, lo1_0, K);
                    pack_group(B1, B2, u, q, t1, t2);
                }
                const uint32_t flip = (ge2 | (c0 & (B1 | all1)) | B2 | all2) & g.VM;
                own[c] = S ^ flip;
                pl[c * AW + FP + w] = own[c];
            }
            __syncthreads();
        }
    }

    // child: planes back in their padded rows, E from the final lattice (every bond
    // touches one colour-0 site), M
    if (active) {
        uint32_t *dst = P.spins[nbuf] + rd.spin_off + (uint64_t)child * rd.wstride;
        for (uint32_t p = w; p < PW; p += CW) {
            dst[p] = padded_from_compact(pl, base, pitch, Lh, p);
            dst[PW + p] = padded_from_compact(pl + AW, base, pitch, Lh, p);
        }
        uint32_t same, rot, up, dn;
        compact_neighbours<NARROW>(pl + AW, pl + AW + FP + w, z, g, 0, same, rot, up, dn);
        const uint32_t S = own[0];
        const int32_t unsat = __popc((S ^ same ^ J[0][0]) & g.VM) + __popc((S ^ rot ^ J[0][1]) & g.VM) +
                              __popc((S ^ up ^ J[0][2]) & g.VM) + __popc((S ^ dn ^ J[0][3]) & g.VM);
        atomicAdd(&acc[2 * rloc], unsat);
        atomicAdd(&acc[2 * rloc + 1], __popc(own[0]) + __popc(own[1]));
    }
    __syncthreads();
    if (active && w == 0) {
        const uint64_t pc = rd.rep_off + parent, cc = rd.rep_off + child;
        P.E[nbuf][cc] = 2 * acc[2 * rloc] - 2 * (int32_t)N;
        P.M[nbuf][cc] = 2 * acc[2 * rloc + 1] - (int32_t)N;
        P.fam[nbuf][cc] = P.fam[ob][pc];
    }
}

// --------------------------------------------------------------------------
// Overlaps (Sec. III.D): d = popcount(s XOR s') over the packed spins.
// --------------------------------------------------------------------------
// Hamming distance of two replicas' colour planes (nw words; 16-byte loads
// when nw is a multiple of 4: replica slots are 16-byte aligned).
__device__ __forceinline__ uint32_t plane_distance(const uint32_t *a, const uint32_t *b, uint32_t nw)
{
    uint32_t d = 0;
    if ((nw & 3u) == 0) {
        const uint4 *a4 = reinterpret_cast<const uint4 *>(a), *b4 = reinterpret_cast<const uint4 *>(b);
        for (uint32_t q = 0; q < nw / 4; ++q) {
            const uint4 x = a4[q], y = b4[q];
            d += __popc(x.x ^ y.x) + __popc(x.y ^ y.y) + __popc(x.z ^ y.z) + __popc(x.w ^ y.w);
        }
    } else {
        for (uint32_t q = 0; q < nw; ++q) d += __popc(a[q] ^ b[q]);
    }
    return d;
}

// Histograms up to this many bins are accumulated in shared memory per CTA.
constexpr uint32_t OVERLAP_SMEM_BINS = 4097;  // L <= 64

__global__ void __launch_bounds__(256) overlap_kernel(Pool P, const uint32_t *q_runs, int init)
{
    __shared__ long long sh_l[32];
    __shared__ uint32_t hs[2][OVERLAP_SMEM_BINS];
    const uint32_t run = q_runs[blockIdx.y];
    const RunDev rd = P.runs[run];
    const RunState st = P.st[run];
    if (st.status) return;
    const uint32_t i = init ? 0u : st.step + 1;
    if (i >= rd.n_beta) return;
    const uint32_t R = init ? rd.R : st.R_new;
    const uint32_t buf = i & 1u;
    const uint32_t N = rd.N, ws = rd.wstride;
    const uint32_t nw = 2 * rd.pw;  // plane words; the stride's padding is never compared
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    const bool smem_hist = N + 1 <= OVERLAP_SMEM_BINS;
    pa_step_record *rec = P.rec + rd.rec_off + i;
    const uint32_t *S = P.spins[buf] + rd.spin_off;

    const bool shift = (rd.overlap & PA_Q_SHIFT) && blockIdx.x * blockDim.x < R / 2;
    int32_t pr = -1;
    uint32_t n_pair = 0;
    const uint32_t *Sb = nullptr;
    uint32_t *hb = nullptr;
    pa_step_record *rb_rec = nullptr;
    if ((rd.overlap & PA_Q_PAIR) && rd.paired > (int32_t)run) {
        const RunDev rb = P.runs[(uint32_t)rd.paired];
        const RunState sb = P.st[(uint32_t)rd.paired];
        if (!sb.status) {
            const uint32_t Rb = init ? rb.R : sb.R_new;
            n_pair = R < Rb ? R : Rb;
            if (blockIdx.x * blockDim.x < n_pair) {
                pr = rd.paired;
                Sb = P.spins[buf] + rb.spin_off;
                hb = P.qhp + rb.qh_off + (uint64_t)i * (N + 1);
                rb_rec = P.rec + rb.rec_off + i;
            }
        }
    }
    if (!shift && pr < 0) return;  // uniform over the CTA
    if (smem_hist) {
        for (uint32_t d = threadIdx.x; d <= N; d += blockDim.x) {
            hs[0][d] = 0;
            hs[1][d] = 0;
        }
        __syncthreads();
    }
    uint32_t *ha = P.qh + rd.qh_off + (uint64_t)i * (N + 1);
    uint32_t *hp = P.qhp + rd.qh_off + (uint64_t)i * (N + 1);
    long long v = 0, vp = 0;
    if (shift) {
        const uint32_t h = R / 2;
        if (p < h) {
            const uint32_t d = plane_distance(S + (uint64_t)p * ws, S + (uint64_t)(p + h) * ws, nw);
            if (smem_hist) atomicAdd(&hs[0][d], 1u);
            else atomicAdd(&ha[d], 1u);
            const long long qn = (long long)N - 2 * (long long)d;
            v = qn < 0 ? -qn : qn;
        }
    }
    if (pr >= 0 && p < n_pair) {
        const uint32_t d = plane_distance(S + (uint64_t)p * ws, Sb + (uint64_t)p * ws, nw);
        if (smem_hist) {
            atomicAdd(&hs[1][d], 1u);
        } else {
            atomicAdd(&hp[d], 1u);
            atomicAdd(&hb[d], 1u);
        }
        const long long qn = (long long)N - 2 * (long long)d;
        vp = qn < 0 ? -qn : qn;
    }
    v = block_sum(v, sh_l);
    vp = block_sum(vp, sh_l);
    if (smem_hist) {  // one global add per non-empty bin of this CTA
        for (uint32_t d = threadIdx.x; d <= N; d += blockDim.x) {
            if (hs[0][d]) atomicAdd(&ha[d], hs[0][d]);
            if (hs[1][d]) {
                atomicAdd(&hp[d], hs[1][d]);
                atomicAdd(&hb[d], hs[1][d]);
            }
        }
    }
    if (threadIdx.x == 0) {
        if (shift) {
            atomicAdd(reinterpret_cast<unsigned long long *>(&rec->sum_absq), (unsigned long long)v);
            if (blockIdx.x == 0) rec->n_q = R / 2;
        }
        if (pr >= 0) {
            atomicAdd(reinterpret_cast<unsigned long long *>(&rec->sum_absq_pair), (unsigned long long)vp);
            atomicAdd(reinterpret_cast<unsigned long long *>(&rb_rec->sum_absq_pair), (unsigned long long)vp);
            if (blockIdx.x == 0) {
                rec->n_q_pair = n_pair;
                rb_rec->n_q_pair = n_pair;
            }
        }
    }
}

// --------------------------------------------------------------------------
// Independent pairings from permutations (Sec. III.D, Wang et al., with the
// random search pattern sigma).  One CTA per run, everything in shared memory:
//   1. pi and sigma: replica indices in ascending order of per-replica 64-bit
//      Philox keys whose low 13 bits are replaced by the index (bitonic sort);
//   2. warp 0 visits positions k = sigma_0, sigma_1, ...; where replica k and
//      pi_k share a family it tests the positions sigma_{i+1}, sigma_{i+2}, ...
//      (mod R) 32 at a time with a ballot and swaps pi_k with the first pi_p
//      outside k's family whose position p is outside pi_k's family.  A swap
//      fixes both positions and breaks no other, so one pass in sigma order
//      equals the serial algorithm; a search that exhausts its R - 1 positions
//      skips the measurement at this step;
//   3. every thread takes pairs (k, pi*_k): Hamming distance of the colour
//      planes, histogram, sum |N - 2d|.
// --------------------------------------------------------------------------
constexpr uint32_t WANG_BUCKET_BITS = 12, WANG_BUCKETS = 1u << WANG_BUCKET_BITS;

// Replica indices 0..R-1 in ascending order of their (distinct) 64-bit keys,
// written to dst: a counting sort on the top 12 key bits (the keys are uniform,
// so a bucket holds R / 4096 < 2 keys on average), then an insertion sort of
// each bucket by the whole key.  cnt: WANG_BUCKETS counters in shared memory.
__device__ void sort_by_key(const unsigned long long *key, uint32_t R, uint32_t *dst, uint32_t *cnt,
                            uint32_t *sh_scan)
{
    const uint32_t tid = threadIdx.x, nt = blockDim.x;  // nt * 4 == WANG_BUCKETS
    for (uint32_t q = tid; q < WANG_BUCKETS; q += nt) cnt[q] = 0;
    __syncthreads();
    for (uint32_t j = tid; j < R; j += nt) atomicAdd(&cnt[key[j] >> (64 - WANG_BUCKET_BITS)], 1u);
    __syncthreads();
    uint32_t c[4], sum = 0;  // exclusive scan: each thread owns 4 consecutive buckets
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        c[q] = cnt[4 * tid + q];
        sum += c[q];
    }
    uint32_t total;
    uint32_t run = block_exclusive_scan(sum, sh_scan, total);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        cnt[4 * tid + q] = run;
        run += c[q];
    }
    __syncthreads();
    for (uint32_t j = tid; j < R; j += nt) dst[atomicAdd(&cnt[key[j] >> (64 - WANG_BUCKET_BITS)], 1u)] = j;
    __syncthreads();  // cnt[q] is now the end of bucket q
    for (uint32_t q = tid; q < WANG_BUCKETS; q += nt) {
        const uint32_t lo = q ? cnt[q - 1] : 0u, hi = cnt[q];
        for (uint32_t x = lo + 1; x < hi; ++x) {  // insertion sort of a few entries
            const uint32_t v = dst[x];
            const unsigned long long kv = key[v];
            uint32_t y = x;
            while (y > lo && key[dst[y - 1]] > kv) {
                dst[y] = dst[y - 1];
                --y;
            }
            dst[y] = v;
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(1024) wang_kernel(Pool P, const uint32_t *runs, int init, uint32_t cap)
{
    extern __shared__ __align__(16) unsigned long long wsm[];
    __shared__ long long sh_l[32];
    __shared__ uint32_t sh_scan[33];
    __shared__ uint32_t s_ok, s_swaps;
    const uint32_t run = runs[blockIdx.x];
    const RunDev rd = P.runs[run];
    const RunState st = P.st[run];
    if (st.status) return;
    const uint32_t i = init ? 0u : st.step + 1;
    if (i >= rd.n_beta) return;
    const uint32_t R = init ? rd.R : st.R_new;
    const uint32_t b = i & 1u, tid = threadIdx.x, nt = blockDim.x, lane = tid & 31u;
    unsigned long long *key = wsm;                                // [cap] sort keys, then the families
    uint32_t *fam = reinterpret_cast<uint32_t *>(wsm);            // [cap], over the keys once sorted
    uint32_t *pi = reinterpret_cast<uint32_t *>(wsm + cap);       // [cap]
    uint32_t *sg = pi + cap;                                      // [cap]
    uint32_t *cnt = sg + cap;                                     // [WANG_BUCKETS]
    const unsigned long long mask = (1ull << WANG_IDX_BITS) - 1;
    for (int which = 0; which < 2; ++which) {
        for (uint32_t j = tid; j < R; j += nt) {  // low 13 bits replaced by the index: no ties
            const uint4 o = philox4x32_10(j, 0u, i, TAG_WANG << 24, rd.seed, rd.run_id);
            const unsigned long long k = which ? ((unsigned long long)o.z << 32 | o.w)
                                               : ((unsigned long long)o.x << 32 | o.y);
            key[j] = (k & ~mask) | j;
        }
        __syncthreads();
        sort_by_key(key, R, which ? sg : pi, cnt, sh_scan);
    }
    for (uint32_t j = tid; j < R; j += nt) fam[j] = P.fam[b][rd.rep_off + j];
    __syncthreads();
    if (tid < 32) {
        uint32_t swaps = 0;
        bool ok = true;
        for (uint32_t base = 0; base < R && ok; base += 32) {
            int last = -1;
            for (;;) {  // mismatches of this chunk in sigma order; at most 32 rounds
                const uint32_t ii = base + lane;
                bool mis = false;
                if (ii < R && (int)lane > last) {
                    const uint32_t k = sg[ii];
                    mis = fam[pi[k]] == fam[k];
                }
                const unsigned bal = __ballot_sync(FULL, mis);
                if (!bal) break;
                const int t = __ffs(bal) - 1;
                const uint32_t i0 = base + t, k = sg[i0];
                const uint32_t fk = fam[k], fpk = fam[pi[k]];
                uint32_t found = 0xFFFFFFFFu;
                for (uint32_t l0 = 1; l0 < R; l0 += 32) {  // at most R - 1 positions
                    const uint32_t l = l0 + lane;
                    bool c = false;
                    uint32_t p = 0;
                    if (l < R) {
                        uint32_t q = i0 + l;
                        if (q >= R) q -= R;
                        p = sg[q];
                        c = fam[pi[p]] != fk && fpk != fam[p];
                    }
                    const unsigned bc = __ballot_sync(FULL, c);
                    if (bc) {
                        found = __shfl_sync(FULL, p, __ffs(bc) - 1);
                        break;
                    }
                }
                if (found == 0xFFFFFFFFu) {
                    ok = false;
                    break;
                }
                if (lane == 0) {
                    const uint32_t tmp = pi[k];
                    pi[k] = pi[found];
                    pi[found] = tmp;
                }
                __syncwarp();
                ++swaps;
                last = t;
            }
        }
        if (lane == 0) {
            s_ok = ok ? 1u : 0u;
            s_swaps = swaps;
        }
    }
    __syncthreads();
    pa_step_record *rec = P.rec + rd.rec_off + i;
    if (!s_ok) {
        if (tid == 0) {
            rec->n_q_wang = 0;
            rec->sum_absq_wang = 0;
            rec->wang_swaps = s_swaps;
        }
        return;  // uniform over the CTA
    }
    const uint32_t N = rd.N, ws = rd.wstride, nw = 2 * rd.pw;
    const uint32_t *S = P.spins[b] + rd.spin_off;
    long long v = 0;
    for (uint32_t k = tid; k < R; k += nt) {
        const uint32_t *x = S + (uint64_t)k * ws, *y = S + (uint64_t)pi[k] * ws;
        uint32_t d = 0;
        for (uint32_t q = 0; q < nw; ++q) d += __popc(x[q] ^ y[q]);
        atomicAdd(&P.qhw[rd.qh_off + (uint64_t)i * (N + 1) + d], 1u);
        const long long qn = (long long)N - 2 * (long long)d;
        v += qn < 0 ? -qn : qn;
    }
    v = block_sum(v, sh_l);
    if (tid == 0) {
        rec->sum_absq_wang = v;
        rec->n_q_wang = R;
        rec->wang_swaps = s_swaps;
    }
}

// --------------------------------------------------------------------------
// theta = infinity (Sec. V.B): step (iv) replaced by simple sampling of the
// exact energy distribution.  One thread per child: a 53-bit uniform from
// Philox (words 0, 1), x = u * C[2N], the first level u with x < C[u] by
// binary search over the host-built cumulative weights (the last positive
// level if x rounds up to C[2N]); E = 2u - 2N, M = 0, family from the parent.
// Configurations are not represented: the spin planes of both buffers are
// cleared once, when the population is drawn at beta_0, and nothing writes
// them afterwards.
//
// GB300 issues double-precision instructions at a small fraction of the
// integer rate, so the draw uses one: u 2^-53 is assembled exactly from its
// IEEE-754 fields, and since C and x are non-negative and never NaN, x < C[u]
// is decided on the bit patterns as unsigned integers (the order of
// non-negative doubles is the order of their encodings).
// --------------------------------------------------------------------------
constexpr uint32_t DOS_SMEM_LEVELS = 4096;  // tables of L <= 44 are staged in shared memory
constexpr uint32_t DOS_THREADS = 256, DOS_PER_THREAD = 4;  // replicas k0 + r DOS_THREADS + threadIdx.x

// u 2^-53 as a double, exactly, for 0 <= u < 2^53: the leading bit p of u sets
// the exponent p - 53, the 52 bits below it the fraction.
__device__ __forceinline__ double unit_from_u53(unsigned long long u)
{
    if (u == 0) return 0.0;
    const uint32_t p = 63u - (uint32_t)__clzll((long long)u);
    const unsigned long long frac = (u << (52u - p)) & ((1ull << 52) - 1ull);
    return __longlong_as_double((long long)(((unsigned long long)(p + 1023u - 53u) << 52) | frac));
}

// The DOS_PER_THREAD draws of one thread: the first level u with x < C[u],
// x = u53 2^-53 C[U], found by a branch-free binary search on the encodings Cb
// of C whose ceil(log2(U + 1)) steps are the same for every replica, so the
// searches interleave; the last positive level (stored in C[U + 1]) if x
// rounds up to C[U].  The level is unique because C is non-decreasing.
__device__ __forceinline__ void dos_levels(const unsigned long long *Cb, uint32_t U, const unsigned long long *u53,
                                           uint32_t *lev)
{
    const double top = __longlong_as_double((long long)Cb[U]);
    unsigned long long xb[DOS_PER_THREAD];
    uint32_t base[DOS_PER_THREAD];
#pragma unroll
    for (uint32_t r = 0; r < DOS_PER_THREAD; ++r) {
        xb[r] = (unsigned long long)__double_as_longlong(__dmul_rn(unit_from_u53(u53[r]), top));
        base[r] = 0;
    }
    // invariant: the answer lies in [base, base + len], indices read stay <= U
    for (uint32_t len = U + 1; len > 1;) {
        const uint32_t half = len >> 1;
#pragma unroll
        for (uint32_t r = 0; r < DOS_PER_THREAD; ++r) base[r] += Cb[base[r] + half] <= xb[r] ? half : 0u;
        len -= half;
    }
    const uint32_t last = (uint32_t)__longlong_as_double((long long)Cb[U + 1]);
#pragma unroll
    for (uint32_t r = 0; r < DOS_PER_THREAD; ++r) {
        const uint32_t u = base[r] + (Cb[base[r]] <= xb[r] ? 1u : 0u);
        lev[r] = u <= U ? u : last;
    }
}

__global__ void __launch_bounds__(DOS_THREADS) dos_sample_kernel(Pool P, const uint32_t *runs, int init)
{
    __shared__ unsigned long long sC[DOS_SMEM_LEVELS];
    const uint32_t run = runs[blockIdx.y];
    const RunDev rd = P.runs[run];
    const RunState *st = &P.st[run];
    if (st->status) return;
    const uint32_t i = init ? 0u : st->step + 1;
    if (i >= rd.n_beta) return;
    const uint32_t R = init ? rd.R : st->R_new;
    const uint32_t span = DOS_THREADS * DOS_PER_THREAD;
    const uint32_t k0 = blockIdx.x * span;
    if (k0 >= (init ? rd.R_cap : R)) return;  // uniform over the CTA
    if (init) {  // clear both buffers' planes of replicas k0 .. k0 + span - 1 (coalesced)
        const uint32_t k1 = min(rd.R_cap, k0 + span);
        const uint64_t w0 = rd.spin_off + (uint64_t)k0 * rd.wstride, nw = (uint64_t)(k1 - k0) * rd.wstride;
        for (uint64_t w = threadIdx.x; w < nw; w += blockDim.x) {
            P.spins[0][w0 + w] = 0u;
            P.spins[1][w0 + w] = 0u;
        }
        if (k0 >= R) return;
    }
    const uint32_t U = 2 * rd.N, b = i & 1u;
    const unsigned long long *C =
        reinterpret_cast<const unsigned long long *>(P.wt + rd.dos_off + (uint64_t)i * (U + 2));
    const bool staged = U + 2 <= DOS_SMEM_LEVELS;
    if (staged) {
        for (uint32_t u = threadIdx.x; u < U + 2; u += blockDim.x) sC[u] = C[u];
        __syncthreads();
    }
    // parents first (their families are gathered after the draws), then the draws
    uint32_t par[DOS_PER_THREAD];
    unsigned long long u53[DOS_PER_THREAD];
#pragma unroll
    for (uint32_t r = 0; r < DOS_PER_THREAD; ++r) {
        const uint32_t k = k0 + r * DOS_THREADS + threadIdx.x;
        par[r] = !init && k < R ? P.parent[rd.rep_off + k] : 0u;
    }
    PhiloxKeys K;  // counters (k, 0, i, TAG_DOS << 24): key schedule and first product of i shared
    philox_keys(K, rd.seed, rd.run_id);
    const uint32_t hi1_0 = __umulhi(0xCD9E8D57u, i), lo1_0 = 0xCD9E8D57u * i;
#pragma unroll
    for (uint32_t r = 0; r < DOS_PER_THREAD; ++r) {
        const uint4 o = philox_rk<true>(k0 + r * DOS_THREADS + threadIdx.x, 0u, TAG_DOS << 24, hi1_0, lo1_0, K);
        u53[r] = ((unsigned long long)(o.x >> 5) << 26) | (unsigned long long)(o.y >> 6);
    }
    uint32_t f[DOS_PER_THREAD];
#pragma unroll
    for (uint32_t r = 0; r < DOS_PER_THREAD; ++r) {
        const uint32_t k = k0 + r * DOS_THREADS + threadIdx.x;
        f[r] = init ? k : (k < R ? P.fam[b ^ 1u][rd.rep_off + par[r]] : 0u);
    }
    uint32_t lev[DOS_PER_THREAD];
    dos_levels(staged ? sC : C, U, u53, lev);
#pragma unroll
    for (uint32_t r = 0; r < DOS_PER_THREAD; ++r) {
        const uint32_t k = k0 + r * DOS_THREADS + threadIdx.x;
        if (k >= R) continue;
        const uint64_t slot = rd.rep_off + k;
        P.E[b][slot] = (int32_t)(2 * (int64_t)lev[r] - 2 * (int64_t)rd.N);
        P.M[b][slot] = 0;
        P.fam[b][slot] = f[r];
    }
}

// --------------------------------------------------------------------------
// Measurement (Sec. III.B, Eqs. e, m, c, chi through exact integer sums;
// Eq. F running sum; Eq. rho_t through family run lengths).  Finishes the step.
// --------------------------------------------------------------------------
// 128-bit two's-complement integer, lo the low 64 bits: exact sums of the
// third and fourth powers of energies and magnetisations (Sec. IV.E).
struct I128 {
    unsigned long long lo;
    long long hi;
};

__device__ __forceinline__ void add128(I128 &a, unsigned long long lo, long long hi)
{
    const unsigned long long s = a.lo + lo;
    a.hi += hi + (s < lo ? 1ll : 0ll);
    a.lo = s;
}

__device__ __forceinline__ void add128(I128 &a, const I128 &b) { add128(a, b.lo, b.hi); }

// The full product of two unsigned 64-bit integers.
__device__ __forceinline__ I128 mul_u64(unsigned long long a, unsigned long long b)
{
    return {a * b, (long long)__umul64hi(a, b)};
}

// a b for a >= 0 and a b < 2^127.
__device__ __forceinline__ I128 mul_128_u64(const I128 &a, unsigned long long b)
{
    I128 r = mul_u64(a.lo, b);
    r.hi += (long long)((unsigned long long)a.hi * b);
    return r;
}

__device__ __forceinline__ I128 neg128(const I128 &a)
{
    const unsigned long long lo = ~a.lo + 1ull;
    return {lo, ~a.hi + (lo == 0ull ? 1ll : 0ll)};
}

__device__ __forceinline__ I128 warp_sum128(I128 v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const unsigned long long lo = __shfl_xor_sync(FULL, v.lo, o);
        const long long hi = __shfl_xor_sync(FULL, v.hi, o);
        add128(v, lo, hi);
    }
    return v;
}

// Family run statistics of one contiguous chunk of replicas (a warp's, a
// CTA's).  lead: the replicas at the chunk's start that continue the family
// open before it; trail: the length of the chunk's last run (counted from the
// chunk's start when the chunk has no family start).
struct FamPart {
    long long c2;  // sum over the chunk's runs of length^2
    uint32_t nfam, cmax, lead, trail, len, pad;
};
static_assert(sizeof(FamPart) == MEASURE_PART_WORDS * 8, "FamPart fills its scratch words");

// Appends chunk q (the next one in replica order) to t.  A family open at the
// end of t that continues into q was counted as pieces a and b, a^2 + b^2: the
// join adds 2ab.
__device__ __forceinline__ void join_part(FamPart &t, const FamPart &q)
{
    if (q.len == 0) return;
    if (t.len == 0) {
        t = q;
        return;
    }
    t.c2 += q.c2;
    t.nfam += q.nfam;
    t.cmax = q.cmax > t.cmax ? q.cmax : t.cmax;
    if (q.lead > 0) {
        t.c2 += 2 * (long long)t.trail * q.lead;
        const uint32_t merged = t.trail + q.lead;
        t.cmax = merged > t.cmax ? merged : t.cmax;
        if (t.lead == t.len) t.lead += q.lead;
        t.trail = q.lead == q.len ? merged : q.trail;
    } else {
        t.trail = q.trail;
    }
    t.len += q.len;
}

__device__ __forceinline__ void store_part_cg(FamPart *dst, const FamPart &v)
{
    const unsigned long long *a = reinterpret_cast<const unsigned long long *>(&v);
    unsigned long long *b = reinterpret_cast<unsigned long long *>(dst);
#pragma unroll
    for (int k = 0; k < (int)MEASURE_PART_WORDS; ++k) __stcg(b + k, a[k]);
}

__device__ __forceinline__ FamPart load_part_cg(const FamPart *src)
{
    FamPart v;
    unsigned long long *a = reinterpret_cast<unsigned long long *>(&v);
    const unsigned long long *b = reinterpret_cast<const unsigned long long *>(src);
#pragma unroll
    for (int k = 0; k < (int)MEASURE_PART_WORDS; ++k) a[k] = __ldcg(b + k);
    return v;
}

// Sums of E^k and |M|^k, k = 1..4.
struct Moments {
    long long sE, sE2, sAM, sM2;
    I128 sE3, sE4, sAM3, sM4;
};

// Measurement of a run's population at beta_i, split over nc = run_ctas(R_cap)
// CTAs (blockIdx.y) and each CTA's chunk over its warps.
//  - Moments: energies and magnetisations take N + 1 values each, E = b + 4n
//    with b = -2N + ((E_0 + 2N) mod 4) (every energy of a population is
//    congruent to E_0 mod 4: a spin flip changes E by 0, +-4 or +-8; |E| <= 2N)
//    and M = 2n - N.  Every CTA counts its replicas per value (a per-lane
//    run-length cache in front of the shared-memory counters) and adds its
//    counts into the run's histograms; the sums of E^k and |M|^k (k <= 4,
//    128-bit for k >= 3) are exact integer sums over the histograms.
//  - Families are contiguous runs of equal ancestor id.  Within a warp the run
//    starts are a ballot and a replica's run start is the highest start at or
//    below it (the chunk's first replica counts as a start); chunks are then
//    joined in order (join_part): a CTA's warps by its thread 0, the CTAs by
//    the last CTA of the run to finish (a ticket in the run state).
// The last CTA writes the step record and, for a nearest-integer run with a
// next temperature, prepares that resampling (Sec. II.B, Eqs. tauBoltz and
// QBoltz): E_min from the histogram, S = sum_j exp(-dbeta (E_j - E_min))
// summed level by level in ascending order with the table w[n] =
// exp(-4 n dbeta_{i+1}), ln Q_{i+1} = -dbeta E_min + ln S - ln R_i, and per
// level floor(tau) and the draw threshold ceil(frac 2^32).  It leaves the
// histograms cleared.
#ifndef PA_MEASURE_THREADS
#define PA_MEASURE_THREADS 512
#endif
#ifndef PA_MEASURE_MIN_BLOCKS
#define PA_MEASURE_MIN_BLOCKS 2  // two CTAs per SM: at most 64 registers
#endif
constexpr uint32_t MEASURE_SMEM_BINS = 4097;  // L <= 64: counts in shared memory
constexpr uint32_t MEASURE_BATCH = 4;         // rows of 32 replicas a warp loads at once
constexpr uint32_t MEASURE_SMEM_TERMS = MEASURE_SMEM_BINS;  // doubles that fit in the counters' space

// The shared memory of a run's measurement tail (CTAs of up to 1024 threads).
struct TailSmem {
    Moments mom[32];
    uint32_t wlo[32], whi[32], lohi[2];
    double S, logS, logR;
};

// The tail of a run's measurement at beta_i, by the one CTA that finishes the run
// once every CTA's counts are in the run's histograms gE, gM (levels from the
// energy base eb) and the family statistics are joined in *fam: the moments, the
// step record, and for a nearest-integer run with a next temperature that
// resampling's E_min, ln Q_{i+1} and per-level tables; the histograms are left
// cleared.  terms: shared memory for n_terms doubles (the terms h_n w[n]).
// Needs at least three warps.
__device__ void run_tail(const Pool &P, const RunDev &rd, RunState *st, uint32_t i, int init, uint32_t R, int32_t eb,
                         uint32_t *gE, uint32_t *gM, unsigned long long *scr, const FamPart *fam, double *terms,
                         uint32_t n_terms, TailSmem &ts)
{
    // The run's tail.  Every thread forms partial moments and the occupied levels
    // over its share of the N + 1 histogram entries; then warp 1 joins the levels
    // and forms the terms h_n w[n], their ascending sum S and ln S (the chain the
    // next resampling waits for) while warp 2 takes ln R and warp 0 joins the
    // moments and writes the record; then the tables of floor(tau) and draw thresholds.
    const uint32_t tid = threadIdx.x, nt = blockDim.x, lane = tid & 31u, wid = tid >> 5, nw = nt >> 5;
    const uint32_t N = rd.N, n1 = N + 1;
    const bool prep = rd.resample != PA_MULTINOMIAL && i + 1 < rd.n_beta;
    const double lnQ_i = init ? 0.0 : st->lnQ;  // read before it is replaced by ln Q_{i+1}
    {
        Moments mo = {0, 0, 0, 0, {0ull, 0ll}, {0ull, 0ll}, {0ull, 0ll}, {0ull, 0ll}};
        uint32_t elo = 0xffffffffu, ehi = 0u;
        for (uint32_t n = tid; n < n1; n += nt) {
            const uint32_t he = __ldcg(&gE[n]), hm = __ldcg(&gM[n]);
            if (he) {
                elo = n < elo ? n : elo;
                ehi = n > ehi ? n : ehi;
                const long long e = (long long)eb + 4ll * n;
                const unsigned long long ae = (unsigned long long)(e < 0 ? -e : e), e2 = ae * ae;  // |E| <= 2^17
                mo.sE += (long long)he * e;
                mo.sE2 += (long long)((unsigned long long)he * e2);
                const I128 t3 = mul_u64(he, ae * e2);
                add128(mo.sE3, e < 0 ? neg128(t3) : t3);
                add128(mo.sE4, mul_128_u64(mul_u64(he, e2), e2));
            }
            if (hm) {
                const long long m = 2ll * n - (long long)N;
                const unsigned long long am = (unsigned long long)(m < 0 ? -m : m), m2 = am * am;  // |M| <= 2^16
                mo.sAM += (long long)((unsigned long long)hm * am);
                mo.sM2 += (long long)((unsigned long long)hm * m2);
                add128(mo.sAM3, mul_u64(hm, am * m2));
                add128(mo.sM4, mul_128_u64(mul_u64(hm, m2), m2));
            }
        }
        mo.sE = warp_sum(mo.sE);
        mo.sE2 = warp_sum(mo.sE2);
        mo.sAM = warp_sum(mo.sAM);
        mo.sM2 = warp_sum(mo.sM2);
        mo.sE3 = warp_sum128(mo.sE3);
        mo.sE4 = warp_sum128(mo.sE4);
        mo.sAM3 = warp_sum128(mo.sAM3);
        mo.sM4 = warp_sum128(mo.sM4);
        elo = warp_min(elo);
        ehi = warp_max(ehi);
        if (lane == 0) {
            ts.mom[wid] = mo;
            ts.wlo[wid] = elo;
            ts.whi[wid] = ehi;
        }
    }
    __syncthreads();
    if (wid == 1) {
        const uint32_t l = warp_min(lane < nw ? ts.wlo[lane] : 0xffffffffu);
        const uint32_t h = warp_max(lane < nw ? ts.whi[lane] : 0u);
        if (lane == 0) {
            ts.lohi[0] = l;
            ts.lohi[1] = h;
        }
        if (prep) {
            const uint32_t nb = h - l + 1;
            const double *wt = P.wt + P.wtoff[rd.wt_off + i + 1];  // exp(-4 n dbeta_{i+1})
            const bool staged = nb <= n_terms;
            if (staged) {
                for (uint32_t n = lane; n < nb; n += 32) terms[n] = __dmul_rn((double)__ldcg(&gE[l + n]), wt[n]);
                __syncwarp();
            }
            if (lane == 0) {
                double S = 0.0;
                if (staged)
                    for (uint32_t n = 0; n < nb; ++n) S = __dadd_rn(S, terms[n]);
                else
                    for (uint32_t n = 0; n < nb; ++n) S = __dadd_rn(S, __dmul_rn((double)__ldcg(&gE[l + n]), wt[n]));
                ts.S = S;
                ts.logS = log(S);
            }
        }
    } else if (wid == 2) {
        if (prep && lane == 0) ts.logR = log((double)R);
    } else if (wid == 0) {  // the warps' partial moments joined, the record
        const bool has = lane < nw;
        const long long sE = warp_sum(has ? ts.mom[lane].sE : 0ll), sE2 = warp_sum(has ? ts.mom[lane].sE2 : 0ll);
        const long long sAM = warp_sum(has ? ts.mom[lane].sAM : 0ll), sM2 = warp_sum(has ? ts.mom[lane].sM2 : 0ll);
        const I128 z = {0ull, 0ll};
        const I128 sE3 = warp_sum128(has ? ts.mom[lane].sE3 : z), sE4 = warp_sum128(has ? ts.mom[lane].sE4 : z);
        const I128 sAM3 = warp_sum128(has ? ts.mom[lane].sAM3 : z), sM4 = warp_sum128(has ? ts.mom[lane].sM4 : z);
        if (lane == 0) {
            const FamPart f = *fam;
            pa_step_record *rec = P.rec + rd.rec_off + i;
            rec->beta = P.beta[rd.beta_off + i];
            rec->lnQ = lnQ_i;
            rec->minus_betaF = init ? rd.ln2N : P.rec[rd.rec_off + i - 1].minus_betaF + lnQ_i;
            rec->sumE = sE;
            rec->sumE2 = sE2;
            rec->sumAbsM = sAM;
            rec->sumM2 = sM2;
            rec->sum_c2 = f.c2;
            rec->sumE3[0] = sE3.lo;
            rec->sumE3[1] = (unsigned long long)sE3.hi;
            rec->sumE4[0] = sE4.lo;
            rec->sumE4[1] = (unsigned long long)sE4.hi;
            rec->sumAbsM3[0] = sAM3.lo;
            rec->sumAbsM3[1] = (unsigned long long)sAM3.hi;
            rec->sumM4[0] = sM4.lo;
            rec->sumM4[1] = (unsigned long long)sM4.hi;
            rec->R = R;
            rec->R_target = rd.R;
            rec->n_fam = f.nfam;
            rec->max_fam = f.cmax;
            rec->N = rd.N;
            rec->status = 0;
            st->step = i;
            st->R_cur = R;
            st->R_new = R;
        }
    }
    __syncthreads();
    if (prep) {  // ln Q_{i+1}, E_min, and per level floor(tau) and the draw threshold, tau = R_target w[n] / S
        const uint32_t l = ts.lohi[0], nb = ts.lohi[1] - l + 1;
        const double *wt = P.wt + P.wtoff[rd.wt_off + i + 1];
        if (tid == 32) {
            const int32_t Emin = eb + 4 * (int32_t)l;
            const double dbeta = P.beta[rd.beta_off + i + 1] - P.beta[rd.beta_off + i];
            st->lnQ = (-dbeta) * (double)Emin + ts.logS - ts.logR;
            st->Emin = Emin;
            st->n_levels = nb;
        }
        const double S = ts.S;
        unsigned long long *thr = scr + scr_table_off(N);
        uint32_t *flo = reinterpret_cast<uint32_t *>(scr + scr_level_off(N));
        for (uint32_t n = tid; n < nb; n += nt) {
            const double tau = __ddiv_rn(__dmul_rn((double)rd.R, wt[n]), S);
            const double fl = floor(tau);
            flo[n] = (uint32_t)fl;
            thr[n] = (unsigned long long)ceil(__dmul_rn(__dsub_rn(tau, fl), 4294967296.0));
        }
    }
    for (uint32_t n = tid; n < n1; n += nt) {  // cleared for the next step (every read of them is done)
        gE[n] = 0u;
        gM[n] = 0u;
    }
}

__global__ void __launch_bounds__(PA_MEASURE_THREADS, PA_MEASURE_MIN_BLOCKS) measure_kernel(Pool P, const uint32_t *runs,
                                                                                           int init)
{
    __shared__ __align__(16) uint32_t sh_h[2][MEASURE_SMEM_BINS];
    __shared__ FamPart part[32];
    __shared__ TailSmem ts;
    __shared__ uint32_t sh_last;
    const uint32_t run = runs[blockIdx.x];
    const RunDev rd = P.runs[run];
    RunState *st = &P.st[run];
    if (st->status) return;
    const uint32_t i = init ? 0u : st->step + 1;
    if (i >= rd.n_beta) return;
    const uint32_t nc = min(gridDim.y, run_ctas(rd.R_cap));
    if (blockIdx.y >= nc) return;
    const uint32_t R = init ? rd.R : st->R_new;
    const uint32_t b = i & 1u;
    const int32_t *E = P.E[b] + rd.rep_off;
    const int32_t *M = P.M[b] + rd.rep_off;
    const uint32_t *fam = P.fam[b] + rd.rep_off;
    const uint32_t tid = threadIdx.x, nt = blockDim.x, lane = tid & 31u, wid = tid >> 5, nw = nt >> 5;
    const uint32_t N = rd.N, n1 = N + 1;
    const int32_t twoN = 2 * (int32_t)N;
    const int32_t eb = -twoN + ((E[0] + twoN) & 3);
    unsigned long long *scr = P.scratch + rd.scr_off;
    uint32_t *gE = reinterpret_cast<uint32_t *>(scr);
    uint32_t *gM = reinterpret_cast<uint32_t *>(scr + scr_mhist_off(N));
    const bool smem = n1 <= MEASURE_SMEM_BINS;
    uint32_t *hE = smem ? sh_h[0] : gE, *hM = smem ? sh_h[1] : gM;
    if (smem) {
        for (uint32_t n = tid; n < n1; n += nt) {
            sh_h[0][n] = 0u;
            sh_h[1][n] = 0u;
        }
        __syncthreads();
    }

    const uint32_t cchunk = (R + nc - 1) / nc;
    const uint32_t c_lo = min(R, blockIdx.y * cchunk), c_hi = min(R, c_lo + cchunk);
    const uint32_t chunk = (c_hi - c_lo + nw - 1) / nw;
    const uint32_t lo = min(c_hi, c_lo + wid * chunk), hi = min(c_hi, lo + chunk);

    uint32_t e_bin = 0, e_cnt = 0, m_bin = 0, m_cnt = 0;  // per-lane run-length caches of the counts
    long long c2 = 0;
    uint32_t nfam = 0, cmax = 0, first = hi, open = lo;  // nfam, first, open: warp-uniform
    uint32_t f_prev = lo > 0 && lo < hi ? fam[lo - 1] : 0u;  // family before the chunk (lane 0's left)
    // rows of 32 replicas in batches of MEASURE_BATCH: the next batch's loads are
    // issued before the current batch is walked row by row; fam[j - 1] comes from
    // the neighbouring lane
    int32_t eq[MEASURE_BATCH], mq[MEASURE_BATCH];
    uint32_t fq[MEASURE_BATCH];
#pragma unroll
    for (uint32_t r = 0; r < MEASURE_BATCH; ++r) {
        const uint32_t j = lo + 32 * r + lane;
        eq[r] = j < hi ? E[j] : 0;
        mq[r] = j < hi ? M[j] : 0;
        fq[r] = j < hi ? fam[j] : 0u;
    }
    for (uint32_t b0 = lo; b0 < hi; b0 += 32 * MEASURE_BATCH) {
        int32_t en[MEASURE_BATCH], mn[MEASURE_BATCH];
        uint32_t fn[MEASURE_BATCH];
#pragma unroll
        for (uint32_t r = 0; r < MEASURE_BATCH; ++r) {
            const uint32_t j = b0 + 32 * (MEASURE_BATCH + r) + lane;
            en[r] = j < hi ? E[j] : 0;
            mn[r] = j < hi ? M[j] : 0;
            fn[r] = j < hi ? fam[j] : 0u;
        }
#pragma unroll
        for (uint32_t r = 0; r < MEASURE_BATCH; ++r) {
            const uint32_t base = b0 + 32 * r;
            if (base >= hi) break;  // uniform over the warp
            const uint32_t j = base + lane;
            const bool ok = j < hi;
            const uint32_t f_cur = fq[r];
            uint32_t f_left = __shfl_up_sync(FULL, f_cur, 1);
            if (lane == 0) f_left = f_prev;
            f_prev = __shfl_sync(FULL, f_cur, 31);
            if (ok) {
                const uint32_t ne = (uint32_t)(eq[r] - eb) >> 2, nm = (uint32_t)(mq[r] + (int32_t)N) >> 1;
                if (ne != e_bin) {
                    if (e_cnt) atomicAdd(&hE[e_bin], e_cnt);
                    e_bin = ne;
                    e_cnt = 0;
                }
                ++e_cnt;
                if (nm != m_bin) {
                    if (m_cnt) atomicAdd(&hM[m_bin], m_cnt);
                    m_bin = nm;
                    m_cnt = 0;
                }
                ++m_cnt;
            }
            const bool start = ok && (j == 0 || f_cur != f_left);
            const uint32_t smask = __ballot_sync(FULL, start);
            const uint32_t fmask = __ballot_sync(FULL, start || (ok && j == lo));
            const uint32_t below = fmask & (0xffffffffu >> (31u - lane));
            const uint32_t sj = below ? base + 31u - (uint32_t)__clz(below) : open;
            if (ok) {
                c2 += 2 * (long long)(j - sj) + 1;  // sum over a run of (2r + 1) = length^2
                cmax = j - sj + 1 > cmax ? j - sj + 1 : cmax;
            }
            nfam += (uint32_t)__popc(smask);
            if (smask && first == hi) first = base + (uint32_t)__ffs(smask) - 1u;
            if (fmask) open = base + 31u - (uint32_t)__clz(fmask);
        }
#pragma unroll
        for (uint32_t r = 0; r < MEASURE_BATCH; ++r) {
            eq[r] = en[r];
            mq[r] = mn[r];
            fq[r] = fn[r];
        }
    }
    if (e_cnt) atomicAdd(&hE[e_bin], e_cnt);
    if (m_cnt) atomicAdd(&hM[m_bin], m_cnt);
    FamPart w;
    w.c2 = warp_sum(c2);
    w.cmax = warp_max(cmax);
    w.nfam = nfam;
    w.lead = first - lo;  // replicas continuing the previous chunk's family
    w.trail = hi - open;  // length of the chunk's last run
    w.len = hi - lo;
    w.pad = 0;
    if (lane == 0) part[wid] = w;
    __syncthreads();
    if (smem)  // this CTA's counts into the run's histograms
        for (uint32_t n = tid; n < n1; n += nt) {
            if (sh_h[0][n]) atomicAdd(&gE[n], sh_h[0][n]);
            if (sh_h[1][n]) atomicAdd(&gM[n], sh_h[1][n]);
        }
    FamPart *gp = reinterpret_cast<FamPart *>(scr + scr_tail_off(N));
    if (tid == 0) {
        FamPart t = part[0];
        for (uint32_t k = 1; k < nw; ++k) join_part(t, part[k]);
        if (nc > 1) store_part_cg(gp + blockIdx.y, t);
        else part[0] = t;
    }
    if (nc > 1) {  // the last CTA of the run to finish goes on
        __threadfence();
        __syncthreads();
        if (tid == 0) sh_last = atomicAdd(&st->ticket, 1u) == nc - 1 ? 1u : 0u;
        __syncthreads();
        if (!sh_last) return;
        __threadfence();
        if (wid == 0) {  // the CTAs' family statistics, joined in order, 32 loaded at a time
            FamPart t;
            t.len = 0;
            for (uint32_t k0 = 0; k0 < nc; k0 += 32) {
                if (k0 + lane < nc) part[lane] = load_part_cg(gp + k0 + lane);
                __syncwarp();
                if (lane == 0)
                    for (uint32_t k = 0; k < 32 && k0 + k < nc; ++k) join_part(t, part[k]);
                __syncwarp();
            }
            if (lane == 0) {
                part[0] = t;
                st->ticket = 0u;
            }
        }
    }
    __syncthreads();

    run_tail(P, rd, st, i, init, R, eb, gE, gM, scr, &part[0], reinterpret_cast<double *>(&sh_h[0][0]),
             MEASURE_SMEM_TERMS, ts);
}

// A record's 128-bit sum as a double: sign and magnitude, then hi 2^64 + lo
// (hi < 2^53, so at most two roundings).
__device__ __forceinline__ double i128_to_double(const uint64_t *w)
{
    unsigned long long lo = w[0], hi = w[1];
    const bool neg = (long long)hi < 0;
    if (neg) {
        lo = ~lo + 1ull;
        hi = ~hi + (lo == 0ull ? 1ull : 0ull);
    }
    const double v = (double)hi * 18446744073709551616.0 + (double)lo;
    return neg ? -v : v;
}

// Eq. W_k (Sec. IV.E): k-th central moment from weighted raw moments
// raw[l] = W[O^l] (raw[0] = 1) by the binomial expansion, terms l = 0..k.
__device__ __forceinline__ double central_from_raw(int k, const double *raw)
{
    double acc = 0.0, binom = 1.0;
    for (int l = 0; l <= k; ++l) {
        double p = 1.0;
        for (int t = l; t < k; ++t) p = p * raw[1];
        const double term = binom * p * raw[l];
        acc = acc + (((k - l) & 1) ? -term : term);
        binom = binom * (double)(k - l) / (double)(l + 1);
    }
    return acc;
}

// --------------------------------------------------------------------------
// Weighted averages (Sec. IV, Eqs. appropriateWeight / simpleWeight, W_conf,
// W_F, Wvar_C, Wvar_Chi) in FP64: one warp per group, lanes over the runs m,
// temperatures in order.  w receives the weights [group][step][m].
// --------------------------------------------------------------------------
// pass 1, one warp per (group, run m): log weights over the temperatures,
// lambda(i, m) = ln R_i + (-beta_i F_i) [+ sum_{k<=i} ln(R_{k-1} / R)], into w[g][i][m].
// The lanes take the logarithms of 32 temperatures at once (FP64 logarithms are
// long dependent chains); the running sum then adds the terms in temperature
// order, each broadcast to every lane, so every lane holds the sum up to its own
// temperature: the same additions in the same order as a sequential loop.
__global__ void __launch_bounds__(128) wavg_lambda_kernel(const pa_step_record *recs,
                                                          const unsigned long long *rec_off, uint32_t n_groups,
                                                          uint32_t M, uint32_t n_steps, uint32_t kind, double *w)
{
    const uint64_t t = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t lane = threadIdx.x & 31u;
    if (t >= (uint64_t)n_groups * M) return;  // warp-uniform
    const uint32_t g = (uint32_t)(t / M), m = (uint32_t)(t % M);
    const pa_step_record *r = recs + rec_off[t];
    double *wg = w + (uint64_t)g * n_steps * M;
    double lsum = 0.0;
    for (uint32_t i0 = 0; i0 < n_steps; i0 += 32) {
        const uint32_t i = i0 + lane;
        double a = 0.0, b = 0.0;
        if (i < n_steps) {
            a = log((double)r[i].R) + r[i].minus_betaF;
            if (kind == PA_WEIGHT_FULL && i > 0) b = log((double)r[i - 1].R / (double)r[i].R_target);
        }
        double mine = 0.0;
        const uint32_t nk = n_steps - i0 < 32 ? n_steps - i0 : 32u;
        for (uint32_t k = 0; k < nk; ++k) {
            lsum += __shfl_sync(FULL, b, k);
            if (k == lane) mine = lsum;
        }
        if (i < n_steps) wg[(uint64_t)i * M + m] = a + mine;
    }
}

// max and sum of exp(lambda - max) over the M runs of one temperature (warp-wide)
__device__ __forceinline__ void weight_norm(const double *li, uint32_t M, uint32_t lane, double &lmax, double &z)
{
    lmax = -INFINITY;
    for (uint32_t m = lane; m < M; m += 32) lmax = li[m] > lmax ? li[m] : lmax;
    lmax = warp_max(lmax);
    z = 0.0;
    for (uint32_t m = lane; m < M; m += 32) z += exp(li[m] - lmax);
    z = warp_sum(z);
}

// pass 2, one warp per (group, temperature): the weights w = exp(lambda - max) / z
// and every weighted average; W_minus_betaF temporarily holds ln W[Q_i] (Eq. W_F).
__global__ void __launch_bounds__(128) wavg_step_kernel(const pa_step_record *recs, const unsigned long long *rec_off,
                                                        uint32_t n_groups, uint32_t M, uint32_t n_steps, uint32_t N,
                                                        pa_wavg *out, const double *w)
{
    const uint32_t i = blockIdx.y * (blockDim.x >> 5) + (threadIdx.x >> 5), g = blockIdx.x, lane = threadIdx.x & 31;
    if (i >= n_steps) return;  // warp-uniform
    const unsigned long long *off = rec_off + (uint64_t)g * M;
    const double *li = w + ((uint64_t)g * n_steps + i) * M;
    const double Nd = (double)N;
    double lmax, z;
    weight_norm(li, M, lane, lmax, z);
    const double beta = recs[off[0] + i].beta;
    double se = 0.0, se2 = 0.0, sm = 0.0, sm2 = 0.0, sc = 0.0, schi = 0.0, sq = 0.0, sqp = 0.0, sw = 0.0,
           wmax = 0.0, se3 = 0.0, se4 = 0.0, sm3 = 0.0, sm4 = 0.0, su4 = 0.0, sqw = 0.0;
    const double N3 = Nd * Nd * Nd, N4 = N3 * Nd;
    for (uint32_t m = lane; m < M; m += 32) {
        const double wm = exp(li[m] - lmax) / z;
        const pa_step_record *r = recs + off[m] + i;
        const double Ri = (double)r->R;
        const double e = (double)r->sumE / (Nd * Ri);
        const double e2 = (double)r->sumE2 / (Nd * Nd * Ri);
        const double mm = (double)r->sumAbsM / (Nd * Ri);
        const double m2 = (double)r->sumM2 / (Nd * Nd * Ri);
        const double c = beta * beta * Nd * (e2 - e * e);  // Eq. c
        const double chi = beta * Nd * (m2 - mm * mm);     // Eq. chi
        se += wm * e;
        se2 += wm * e2;
        sm += wm * mm;
        sm2 += wm * m2;
        sc += wm * c;
        schi += wm * chi;
        if (r->n_q) sq += wm * ((double)r->sum_absq / (Nd * (double)r->n_q));
        if (r->n_q_pair) sqp += wm * ((double)r->sum_absq_pair / (Nd * (double)r->n_q_pair));
        if (r->n_q_wang) sqw += wm * ((double)r->sum_absq_wang / (Nd * (double)r->n_q_wang));
        const double e3 = i128_to_double(r->sumE3) / (N3 * Ri);
        const double e4 = i128_to_double(r->sumE4) / (N4 * Ri);
        const double m3 = i128_to_double(r->sumAbsM3) / (N3 * Ri);
        const double m4 = i128_to_double(r->sumM4) / (N4 * Ri);
        se3 += wm * e3;
        se4 += wm * e4;
        sm3 += wm * m3;
        sm4 += wm * m4;
        su4 += wm * (1.0 - m4 / (3.0 * m2 * m2));  // per-run Binder cumulant
        sw += wm;
        wmax = wm > wmax ? wm : wmax;
    }
    pa_wavg o;
    o.beta = beta;
    o.W_e = warp_sum(se);
    o.W_e2 = warp_sum(se2);
    o.W_m = warp_sum(sm);
    o.W_m2 = warp_sum(sm2);
    o.W_c = warp_sum(sc);
    o.W_chi = warp_sum(schi);
    o.W_absq = warp_sum(sq);
    o.W_absq_pair = warp_sum(sqp);
    o.sum_w = warp_sum(sw);
    o.w_max = warp_max(wmax);
    o.Wvar_c = beta * beta * Nd * (o.W_e2 - o.W_e * o.W_e);
    o.Wvar_chi = beta * Nd * (o.W_m2 - o.W_m * o.W_m);
    o.W_e3 = warp_sum(se3);
    o.W_e4 = warp_sum(se4);
    o.W_m3 = warp_sum(sm3);
    o.W_m4 = warp_sum(sm4);
    o.W_U4_conf = warp_sum(su4);
    o.W_absq_wang = warp_sum(sqw);
    {
        const double re[5] = {1.0, o.W_e, o.W_e2, o.W_e3, o.W_e4};
        const double rm[5] = {1.0, o.W_m, o.W_m2, o.W_m3, o.W_m4};
        o.Wk3_e = central_from_raw(3, re);
        o.Wk4_e = central_from_raw(4, re);
        o.Wk3_m = central_from_raw(3, rm);
        o.Wk4_m = central_from_raw(4, rm);
        o.W_U4 = 1.0 - o.W_m4 / (3.0 * o.W_m2 * o.W_m2);
    }
    double dF = 0.0;
    if (i > 0) {  // Eq. W_F: ln W[Q_i] = ln sum_m w_{i-1} Q_i as a log-sum-exp, ln w_{i-1} = lambda - max - ln z
        const double *lp = li - M;
        double pmax, pz;
        weight_norm(lp, M, lane, pmax, pz);
        const double lpz = pmax + log(pz);
        double lm = -INFINITY;
        for (uint32_t m = lane; m < M; m += 32) {
            const double l = lp[m] - lpz + recs[off[m] + i].lnQ;
            lm = l > lm ? l : lm;
        }
        lm = warp_max(lm);
        double zz = 0.0;
        for (uint32_t m = lane; m < M; m += 32) zz += exp(lp[m] - lpz + recs[off[m] + i].lnQ - lm);
        zz = warp_sum(zz);
        dF = lm + log(zz);
    }
    o.W_minus_betaF = dF;
    if (lane == 0) out[(uint64_t)g * n_steps + i] = o;
}

// pass 3: the weights normalised in place (for the overlap distributions) and,
// per group in temperature order, -beta_i W[F_i] = N ln 2 + sum_{k<=i} ln W[Q_k].
__global__ void __launch_bounds__(128) wavg_finish_kernel(uint32_t n_groups, uint32_t M, uint32_t n_steps,
                                                          uint32_t N, pa_wavg *out, double *w)
{
    const uint32_t i = blockIdx.y * (blockDim.x >> 5) + (threadIdx.x >> 5), g = blockIdx.x, lane = threadIdx.x & 31;
    if (i < n_steps) {
        double *li = w + ((uint64_t)g * n_steps + i) * M;
        double lmax, z;
        weight_norm(li, M, lane, lmax, z);
        for (uint32_t m = lane; m < M; m += 32) li[m] = exp(li[m] - lmax) / z;
    }
    if (blockIdx.y == 0 && threadIdx.x == 0) {
        pa_wavg *og = out + (uint64_t)g * n_steps;
        double WF = (double)N * log(2.0);
        for (uint32_t k = 0; k < n_steps; ++k) {
            if (k > 0) WF = WF + og[k].W_minus_betaF;
            og[k].W_minus_betaF = WF;
        }
    }
}

// Weighted overlap distributions (Eq. W_conf_q): grid (steps, groups).
__global__ void wavg_q_kernel(const pa_step_record *recs, const unsigned long long *rec_off, const uint32_t *qh,
                              const uint32_t *qhp, const uint32_t *qhw, const unsigned long long *qh_off, uint32_t M,
                              uint32_t n_steps, uint32_t N, const double *w, double *Pq, double *Pqp, double *Pqw)
{
    const uint32_t i = blockIdx.y, g = blockIdx.x;
    const double *wi = w + ((uint64_t)g * n_steps + i) * M;
    const unsigned long long *ro = rec_off + (uint64_t)g * M, *qo = qh_off + (uint64_t)g * M;
    for (uint32_t d = threadIdx.x; d <= N; d += blockDim.x) {
        double a = 0.0, b = 0.0, c = 0.0;
        for (uint32_t m = 0; m < M; ++m) {
            const pa_step_record *r = recs + ro[m] + i;
            const uint64_t q = qo[m] + (uint64_t)i * (N + 1) + d;
            if (Pq && r->n_q) a += wi[m] * ((double)qh[q] / (double)r->n_q);
            if (Pqp && r->n_q_pair) b += wi[m] * ((double)qhp[q] / (double)r->n_q_pair);
            if (Pqw && r->n_q_wang) c += wi[m] * ((double)qhw[q] / (double)r->n_q_wang);
        }
        const uint64_t o = ((uint64_t)g * n_steps + i) * (N + 1) + d;
        if (Pq) Pq[o] = a;
        if (Pqp) Pqp[o] = b;
        if (Pqw) Pqw[o] = c;
    }
}

// --------------------------------------------------------------------------
// Small populations: one launch per anneal step, or per whole anneal (Sec. II.B
// steps (ii)-(v)).  A run with nearest-integer resampling, no overlap pairs,
// L/2 a power of two with 8 <= L <= 32 and R_cap <= SMALL_MAX_RCAP is annealed
// by one thread-block cluster of CS CTAs (CS = gridDim.x / number of runs, set
// by the launch).  Per temperature:
//   CTA 0       copy numbers, their scan and the parent map (as
//               resample_counts_kernel with one CTA per run);
//   every CTA   its share of the children: the resampling copy and theta
//               sweeps, each plane word's 8 Philox groups spread over LPW lanes
//               whose comparison bits are joined by shuffles, so that even a
//               few hundred replicas fill the SMs of the cluster;
//   CTA 0       the measurement of the new population and the next
//               resampling's tables (as measure_kernel with one CTA per run).
// With drawing ahead (H > 0, launches of several temperatures at L = 8, 16) CTA 0
// sweeps no children, and while it measures and resamples the other CTAs draw the
// next temperature's comparison bits for their slices into shared memory.
// The phases are separated by two cluster barriers per temperature
// (barrier.cluster arrive with release and wait with acquire semantics at cluster
// scope, so each phase sees the global memory the previous one wrote): after
// the resampling and after the sweeps.  Every CTA of a cluster reads the same
// run state after the same barrier, so all of them take the same number of
// barriers.  The arithmetic, the Philox counters and the device state left
// behind (records, scratch tables, run state) are those of the multi-kernel
// path, so a run can move between the two paths at any step.
// --------------------------------------------------------------------------
constexpr uint32_t SMALL_MAX_N = 1024;  // L <= 32

// HW: words of a colour plane (L = 8: 1, 16: 4, 32: 16); LPW lanes per word; NT the
// largest block (a multiple of 32, at least 128) and MINB the CTAs per SM it is
// compiled for: 512 threads two per SM (64 registers), or 512 / 768 threads one
// per SM (the compiler's register choice up to 128 / 85).
template <bool SG, uint32_t HW, uint32_t LPW, uint32_t NT, uint32_t MINB>
__global__ void __launch_bounds__(NT, MINB) anneal_small_kernel(Pool P, const uint32_t *runs, uint32_t n_steps,
                                                                uint32_t H)
{
    constexpr uint32_t GPL = 8u / LPW;             // Philox groups per lane and word
    constexpr uint32_t LPR = HW * LPW;             // lanes per replica (divides 32)
    constexpr uint32_t TR = NT / LPR;              // replicas per tile at the largest block
    static_assert(LPR <= 32 && 32 % LPR == 0, "a replica's lanes lie in one warp");
    constexpr bool AHEAD = LPR == 4 && MINB == 1;  // the variants launched with H > 0 (L = 8 and 16)
    constexpr int AHEAD_UNROLL = HW == 1 ? 2 : 4;  // half-sweeps drawn at once ahead (measured best: L=8 2, L=16 4)
    __shared__ uint32_t s_pl[TR][2 * HW];
    __shared__ __align__(16) uint32_t s_cnt[SMALL_MAX_RCAP];  // copy numbers; the measurement's terms h_n w[n]
    __shared__ uint32_t s_hE[SMALL_MAX_N + 1], s_hM[SMALL_MAX_N + 1];
    double *s_terms = reinterpret_cast<double *>(s_cnt);  // N + 1 <= 1025 doubles, used after the resampling
    static_assert(sizeof(double) * (SMALL_MAX_N + 1) <= sizeof(uint32_t) * SMALL_MAX_RCAP, "terms fit");
    __shared__ uint32_t sh_u[32];
    __shared__ long long sh_ll[32];
    __shared__ uint32_t sh_u2[32];
    __shared__ Moments mom[NT / 32];
    __shared__ uint32_t sh_lvl[2];  // the lowest and highest occupied energy level
    __shared__ double sh_S, sh_logS, sh_logR;
    __shared__ uint32_t sh_carry, sh_first;
    __shared__ FamPart s_part[8];  // CTA 0: the family statistics of each CTA's chunk of children
    __shared__ int32_t sh_eb;      // CTA 0: base of the energy levels of the new population
    __shared__ uint32_t sh_pre_step;  // the temperature whose comparison bits s_pre holds
    extern __shared__ uint2 s_pre[];  // H > 0: [half-sweep][replica of the tile][word] (B1, B2)

    cg::cluster_group cl = cg::this_cluster();
    const uint32_t CS = cl.num_blocks(), rank = cl.block_rank();
    const uint32_t run = runs[blockIdx.x / CS];
    const RunDev rd = P.runs[run];
    RunState *st = &P.st[run];
    const uint32_t tid = threadIdx.x, nt = blockDim.x, lane = tid & 31u, wid = tid >> 5, nw = nt >> 5;
    const uint32_t N = rd.N, n1 = N + 1, Lh = rd.Lh;
    const uint32_t rl = tid / LPR, ll = tid % LPR, w = ll / LPW, sub = ll % LPW;
    unsigned long long *scr = P.scratch + rd.scr_off;
    unsigned long long *thr_tab = scr + scr_table_off(N);
    uint32_t *flo_tab = reinterpret_cast<uint32_t *>(scr + scr_level_off(N));
    uint32_t *parent = P.parent + rd.rep_off;
    PhiloxKeys K;
    philox_keys(K, rd.seed, rd.run_id);
    // With H > 0 (and CS >= 2) CTA 0 sweeps no children: it resamples and measures, while
    // the other CTAs sweep fixed slices of Wc children (from R + 3 sqrt(R), beyond the
    // nearest-integer resampling's spread; the last slice also takes any child beyond) and,
    // while CTA 0 measures, draw the next temperature's comparison bits of their slice for
    // its first H half-sweeps into s_pre.  The bits depend only on the Philox counters, so
    // the sweeps flip the same spins either way.
    uint32_t Wc = 0;
    if (!AHEAD) H = 0;
    if (H) {
        uint32_t q = (uint32_t)sqrtf((float)rd.R);  // floor(sqrt(R)), corrected
        while (q * q > rd.R) --q;
        while ((q + 1) * (q + 1) <= rd.R) ++q;
        Wc = (rd.R + 3 * q + 1 + CS - 2) / (CS - 1);
    }
    if (tid == 0) sh_pre_step = 0xffffffffu;
    uint32_t J[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
    if (SG) {  // the bond masks of this lane's plane word, both colours
        const uint32_t *Jp = P.J + rd.J_off + 2 * rd.wstride;
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int d = 0; d < 4; ++d) J[c][d] = Jp[(c * 4 + d) * HW + w];
    }

    // Every CTA decides from values that no CTA writes between the barriers
    // around the read, so all of them leave the loop at the same point: the
    // status and the temperature index before any barrier of this launch (each
    // CTA then counts the temperatures itself), and the status after the
    // resampling (between its first and second barrier).  A step has two cluster
    // barriers: the other CTAs need nothing from the measurement that the next
    // step's first barrier does not order (CTA 0 measures, then resamples, then
    // arrives there), and they touch CTA 0's shared memory only between the
    // first and second barrier of a step.
    if (st->status) return;
    const uint32_t i0 = st->step + 1;
    for (uint32_t s = 0; s < n_steps; ++s) {
        const uint32_t i = i0 + s;
        if (i >= rd.n_beta) break;
        const uint32_t ob = (i - 1) & 1u, nb = i & 1u;

        // ---- CTA 0: copy numbers r_j = floor(tau) + [u < threshold] per level, scan, parent map;
        // its histograms, which every CTA fills during the sweeps, start cleared
        if (rank == 0) {
            for (uint32_t n = tid; n < n1; n += nt) {
                s_hE[n] = 0u;
                s_hM[n] = 0u;
            }
            const uint32_t Rc = st->R_cur;
            const int32_t *E = P.E[ob] + rd.rep_off;
            const int32_t Emin = st->Emin;
            for (uint32_t j = tid; j < Rc; j += nt) {
                const uint32_t n = min((uint32_t)(E[j] - Emin) >> 2, N);  // <= N for any population; bounds the tables
                const uint32_t u = philox4x32_10(j, 0, i, TAG_RESAMPLE << 24, rd.seed, rd.run_id).x;
                s_cnt[j] = flo_tab[n] + ((unsigned long long)u < thr_tab[n] ? 1u : 0u);
            }
            __syncthreads();
            uint32_t carry = 0;
            for (uint32_t base = 0; base < Rc; base += nt) {
                const uint32_t j = base + tid, r = j < Rc ? s_cnt[j] : 0u;
                uint32_t tot;
                const uint32_t o = carry + block_exclusive_scan(r, sh_u, tot);
                for (uint32_t c = 0; c < r; ++c)
                    if (o + c < rd.R_cap) parent[o + c] = j;
                carry += tot;
            }
            if (tid == 0) {
                st->R_new = carry;
                if (carry == 0)
                    set_status(P, run, PA_ERR_EXTINCT);
                else if (carry > rd.R_cap)
                    set_status(P, run, PA_ERR_CAPACITY);
                if (carry == 0 || carry > rd.R_cap) P.rec[rd.rec_off + i].status = st->status;
            }
        }
        cl.sync();
        if (st->status) break;

        // ---- every CTA: its children, gathered from their parents and swept theta times
        {
            const uint32_t Rn = st->R_new;
            uint32_t c_lo, c_hi;
            if (H) {
                c_lo = min(Rn, rank == 0 ? 0u : (rank - 1) * Wc);
                c_hi = min(Rn, rank == 0 ? 0u : rank + 1 == CS ? 0xffffffffu : rank * Wc);
            } else {
                const uint32_t chunk = (Rn + CS - 1) / CS;
                c_lo = min(Rn, rank * chunk);
                c_hi = min(Rn, c_lo + chunk);
            }
            const unsigned long long T1 = P.thr[rd.thr_off + 2 * i], T2 = P.thr[rd.thr_off + 2 * i + 1];
            const uint32_t t1 = T1 > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)T1;
            const uint32_t t2 = T2 > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)T2;
            const uint32_t all1 = T1 > 0xFFFFFFFFull ? 0xFFFFFFFFu : 0u;
            const uint32_t all2 = T2 > 0xFFFFFFFFull ? 0xFFFFFFFFu : 0u;
            const uint32_t hi1_0 = __umulhi(0xCD9E8D57u, i), lo1_0 = 0xCD9E8D57u * i;
            uint32_t *pl = s_pl[rl];
            for (uint32_t tile0 = c_lo; tile0 < c_hi; tile0 += nt / LPR) {
                const uint32_t child = tile0 + rl;
                const bool active = child < c_hi;
                const uint32_t par = active ? parent[child] : 0u;
                const uint32_t *src = P.spins[ob] + rd.spin_off + (uint64_t)par * rd.wstride;
                uint32_t own[2];
                own[0] = active ? src[w] : 0u;
                own[1] = active ? src[HW + w] : 0u;
                if (sub == 0) {
                    pl[w] = own[0];
                    pl[HW + w] = own[1];
                }
                __syncwarp();
                // The comparison bits of half-sweep h = 2 t + c depend only on the Philox counters,
                // not on the spins: each step draws (and joins over the word's lanes) those of the
                // next half-sweep while it applies the current one, which keeps the Philox chains
                // off the dependent path of spin updates.
                // the first tile of a slice may find its bits drawn already
                const bool pre = AHEAD && H && tile0 == c_lo && rank != 0 && sh_pre_step == i;
                const uint32_t Hh = min(H, 2 * rd.theta);
                auto draw = [&](uint32_t h, uint32_t &B1, uint32_t &B2) {
                    if (AHEAD && pre && h < Hh) {
                        const uint2 v = s_pre[(h * (nt / LPR) + rl) * HW + w];
                        B1 = v.x;
                        B2 = v.y;
                        return;
                    }
                    const uint32_t ctr3 = (TAG_SWEEP << 24) | h;
                    B1 = 0;
                    B2 = 0;
#pragma unroll
                    for (uint32_t q = 0; q < GPL; ++q) {
                        const uint32_t g = sub * GPL + q;
                        const uint4 u = philox_rk<true>(8 * w + g, child, ctr3, hi1_0, lo1_0, K);
                        pack_group(B1, B2, u, g, t1, t2);
                    }
#pragma unroll
                    for (uint32_t o = 1; o < LPW; o <<= 1) {  // the word's lanes are adjacent
                        B1 |= __shfl_xor_sync(FULL, B1, o);
                        B2 |= __shfl_xor_sync(FULL, B2, o);
                    }
                };
                auto apply = [&](uint32_t c, uint32_t B1, uint32_t B2) {
                    uint32_t same, rot, up, dn;
                    plane_neighbours(pl + (c ^ 1u) * HW, HW, Lh, c, w, same, rot, up, dn);
                    const uint32_t S = own[c];
                    const uint32_t x1 = S ^ same ^ J[c][0], x2 = S ^ rot ^ J[c][1];
                    const uint32_t x3 = S ^ up ^ J[c][2], x4 = S ^ dn ^ J[c][3];
                    const uint32_t a = x1 ^ x2, b = x1 & x2, e = x3 ^ x4, f = x3 & x4;
                    const uint32_t c0 = a ^ e, ge2 = b | f | (a & e);
                    own[c] = S ^ (ge2 | (c0 & (B1 | all1)) | B2 | all2);
                    if (sub == 0) pl[c * HW + w] = own[c];
                    __syncwarp();
                };
                if (rd.theta > 0) {
                    uint32_t B1, B2, N1, N2;
                    draw(0, B1, B2);
                    for (uint32_t t = 0; t + 1 < rd.theta; ++t) {
                        draw(2 * t + 1, N1, N2);
                        apply(0, B1, B2);
                        draw(2 * t + 2, B1, B2);
                        apply(1, N1, N2);
                    }
                    draw(2 * rd.theta - 1, N1, N2);
                    apply(0, B1, B2);
                    apply(1, N1, N2);
                }
                // the child: planes, E from the final lattice (every bond touches one colour-0 site), M
                int32_t unsat = 0, up1 = 0;
                if (sub == 0) {
                    uint32_t same, rot, up, dn;
                    plane_neighbours(pl + HW, HW, Lh, 0, w, same, rot, up, dn);
                    const uint32_t S = own[0];
                    unsat = __popc(S ^ same ^ J[0][0]) + __popc(S ^ rot ^ J[0][1]) + __popc(S ^ up ^ J[0][2]) +
                            __popc(S ^ dn ^ J[0][3]);
                    up1 = __popc(own[0]) + __popc(own[1]);
                    if (active) {
                        uint32_t *dst = P.spins[nb] + rd.spin_off + (uint64_t)child * rd.wstride;
                        dst[w] = own[0];
                        dst[HW + w] = own[1];
                    }
                }
#pragma unroll
                for (uint32_t o = LPW; o < LPR; o <<= 1) {
                    unsat += __shfl_xor_sync(FULL, unsat, o);
                    up1 += __shfl_xor_sync(FULL, up1, o);
                }
                if (active && ll == 0) {
                    const uint64_t cc = rd.rep_off + child;
                    const int32_t Ec = 2 * unsat - 2 * (int32_t)N, Mc = 2 * up1 - (int32_t)N;
                    P.E[nb][cc] = Ec;
                    P.M[nb][cc] = Mc;
                    P.fam[nb][cc] = P.fam[ob][rd.rep_off + par];
                    // counts per energy and magnetisation value into CTA 0's histograms; every
                    // energy of the population has the residue of E_0 mod 4, so any child gives the base
                    const int32_t eb = -2 * (int32_t)N + ((Ec + 2 * (int32_t)N) & 3);
                    if (child == 0) *cl.map_shared_rank(&sh_eb, 0) = eb;  // child 0 may be another CTA's
                    atomicAdd(cl.map_shared_rank(&s_hE[(uint32_t)(Ec - eb) >> 2], 0), 1u);
                    atomicAdd(cl.map_shared_rank(&s_hM[(uint32_t)(Mc + (int32_t)N) >> 1], 0), 1u);
                }
                __syncwarp();
            }
            // the family statistics of this CTA's chunk (Eq. rho_t): runs of equal ancestor id; a
            // replica's run starts at the last start at or below it, the chunk's first counting as one.
            // A child's family is its parent's, read through the parent map (the neighbouring CTAs'
            // children may not be written yet)
            const uint32_t *fam_old = P.fam[ob] + rd.rep_off;
            long long c2 = 0;
            uint32_t nfam = 0, cmax = 0;
            if (tid == 0) {
                sh_carry = c_lo;
                sh_first = c_hi;
            }
            __syncthreads();
            for (uint32_t base = c_lo; base < c_hi; base += nt) {
                const uint32_t j = base + tid;
                const bool ok = j < c_hi;
                const bool start = ok && (j == 0 || fam_old[parent[j]] != fam_old[parent[j - 1]]);
                const uint32_t before = sh_carry;
                uint32_t sj = block_inclusive_max(start || (ok && j == c_lo) ? j : 0u, sh_u);
                sj = sj > before ? sj : before;
                if (ok) {
                    c2 += 2 * (long long)(j - sj) + 1;  // sum over a run of (2r + 1) = length^2
                    cmax = j - sj + 1 > cmax ? j - sj + 1 : cmax;
                    nfam += start ? 1u : 0u;
                    if (start) atomicMin(&sh_first, j);
                }
                __syncthreads();
                if (tid == nt - 1) sh_carry = sj;
                __syncthreads();
            }
            c2 = warp_sum(c2);  // the three totals in one pass over the warps
            nfam = warp_sum(nfam);
            cmax = warp_max(cmax);
            if (lane == 0) {
                sh_ll[wid] = c2;
                sh_u[wid] = nfam;
                sh_u2[wid] = cmax;
            }
            __syncthreads();
            if (tid == 0) {
                FamPart f;
                f.c2 = 0;
                f.nfam = 0;
                f.cmax = 0;
                for (uint32_t k = 0; k < nw; ++k) {
                    f.c2 += sh_ll[k];
                    f.nfam += sh_u[k];
                    f.cmax = sh_u2[k] > f.cmax ? sh_u2[k] : f.cmax;
                }
                f.lead = sh_first - c_lo;  // replicas continuing the family open before the chunk
                f.trail = c_hi - sh_carry; // length of the chunk's last run
                f.len = c_hi - c_lo;
                f.pad = 0;
                *cl.map_shared_rank(&s_part[rank], 0) = f;
            }
        }
        cl.sync();

        // ---- the other CTAs, while CTA 0 measures and resamples: the next temperature's
        // comparison bits of their slice (every lane draws, so the shuffles see full warps)
        if (AHEAD && H && rank != 0 && s + 1 < n_steps && i + 1 < rd.n_beta) {
            const uint32_t i2 = i + 1, lo_k = (rank - 1) * Wc;
            const uint32_t cnt = rd.R_cap > lo_k ? min(Wc, rd.R_cap - lo_k) : 0u;
            const unsigned long long U1 = P.thr[rd.thr_off + 2 * i2], U2 = P.thr[rd.thr_off + 2 * i2 + 1];
            const uint32_t u1 = U1 > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)U1;
            const uint32_t u2 = U2 > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)U2;
            const uint32_t g1 = __umulhi(0xCD9E8D57u, i2), g0 = 0xCD9E8D57u * i2;
            const uint32_t child = lo_k + rl, Hh = min(H, 2 * rd.theta), tr = nt / LPR;
#pragma unroll AHEAD_UNROLL
            for (uint32_t h = 0; h < Hh; ++h) {
                const uint32_t ctr3 = (TAG_SWEEP << 24) | h;
                uint32_t B1 = 0, B2 = 0;
#pragma unroll
                for (uint32_t q = 0; q < GPL; ++q) {
                    const uint32_t g = sub * GPL + q;
                    const uint4 u = philox_rk<true>(8 * w + g, child, ctr3, g1, g0, K);
                    pack_group(B1, B2, u, g, u1, u2);
                }
#pragma unroll
                for (uint32_t o = 1; o < LPW; o <<= 1) {
                    B1 |= __shfl_xor_sync(FULL, B1, o);
                    B2 |= __shfl_xor_sync(FULL, B2, o);
                }
                if (sub == 0 && rl < cnt) s_pre[(h * tr + rl) * HW + w] = make_uint2(B1, B2);
            }
            if (tid == 0) sh_pre_step = i2;
        }

        // ---- CTA 0: measurement at beta_i (from the histograms and chunk statistics every CTA
        // left in its shared memory) and the next resampling's tables.  The serial chain that the
        // next step waits for (occupied levels, terms h_n w[n], their ascending sum S and ln S)
        // runs on warp 1 while warp 2 takes ln R and the other warps form the moments; then warp 0
        // writes the record beside the tables of floor(tau) and draw thresholds.
        if (rank == 0) {
            const uint32_t R = st->R_new;
            const int32_t eb = sh_eb;
            const double lnQ_i = st->lnQ;  // read before it is replaced by ln Q_{i+1}
            const bool prep = i + 1 < rd.n_beta;
            if (wid == 1) {
                uint32_t lo = 0xffffffffu, hi = 0u;
                for (uint32_t n0 = 0; n0 < n1; n0 += 32) {
                    const uint32_t n = n0 + lane;
                    const uint32_t m = __ballot_sync(FULL, n < n1 && s_hE[n] != 0u);
                    if (m) {
                        lo = lo == 0xffffffffu ? n0 + __ffs(m) - 1 : lo;
                        hi = n0 + 31 - __clz(m);
                    }
                }
                if (lane == 0) {
                    sh_lvl[0] = lo;
                    sh_lvl[1] = hi;
                }
                if (prep) {
                    const double *wt = P.wt + P.wtoff[rd.wt_off + i + 1];
                    const uint32_t nb_l = hi - lo + 1;
                    for (uint32_t n = lane; n < nb_l; n += 32) s_terms[n] = __dmul_rn((double)s_hE[lo + n], wt[n]);
                    __syncwarp();
                    if (lane == 0) {
                        double S = 0.0;
                        for (uint32_t n = 0; n < nb_l; ++n) S = __dadd_rn(S, s_terms[n]);
                        sh_S = S;
                        sh_logS = log(S);
                    }
                }
            } else if (wid == 2) {
                if (prep && lane == 0) sh_logR = log((double)R);
            } else {  // warps 0 and 3.. : the moments' partial sums over the levels, energy then
                      // magnetisation (half the accumulators live at a time)
                const uint32_t mt = wid == 0 ? lane : tid - 64, nmt = nt - 64;
                long long s1 = 0, s2 = 0;
                I128 s3 = {0ull, 0ll}, s4 = {0ull, 0ll};
                for (uint32_t n = mt; n < n1; n += nmt) {
                    const uint32_t he = s_hE[n];
                    if (he) {
                        const long long e = (long long)eb + 4ll * n;
                        const unsigned long long ae = (unsigned long long)(e < 0 ? -e : e), e2 = ae * ae;
                        s1 += (long long)he * e;
                        s2 += (long long)((unsigned long long)he * e2);
                        const I128 t3 = mul_u64(he, ae * e2);
                        add128(s3, e < 0 ? neg128(t3) : t3);
                        add128(s4, mul_128_u64(mul_u64(he, e2), e2));
                    }
                }
                s1 = warp_sum(s1);
                s2 = warp_sum(s2);
                s3 = warp_sum128(s3);
                s4 = warp_sum128(s4);
                if (lane == 0) {
                    mom[wid].sE = s1;
                    mom[wid].sE2 = s2;
                    mom[wid].sE3 = s3;
                    mom[wid].sE4 = s4;
                }
                s1 = s2 = 0;
                s3 = s4 = I128{0ull, 0ll};
                for (uint32_t n = mt; n < n1; n += nmt) {
                    const uint32_t hm = s_hM[n];
                    if (hm) {
                        const long long m = 2ll * n - (long long)N;
                        const unsigned long long am = (unsigned long long)(m < 0 ? -m : m), m2 = am * am;
                        s1 += (long long)((unsigned long long)hm * am);
                        s2 += (long long)((unsigned long long)hm * m2);
                        add128(s3, mul_u64(hm, am * m2));
                        add128(s4, mul_128_u64(mul_u64(hm, m2), m2));
                    }
                }
                s1 = warp_sum(s1);
                s2 = warp_sum(s2);
                s3 = warp_sum128(s3);
                s4 = warp_sum128(s4);
                if (lane == 0) {
                    mom[wid].sAM = s1;
                    mom[wid].sM2 = s2;
                    mom[wid].sAM3 = s3;
                    mom[wid].sM4 = s4;
                }
            }
            __syncthreads();
            const uint32_t lvl_lo = sh_lvl[0], nb_l = sh_lvl[1] - lvl_lo + 1;
            if (wid == 0) {  // the warps' partial sums joined, the record
                const bool has = lane < nw && lane != 1 && lane != 2;
                const long long sE = warp_sum(has ? mom[lane].sE : 0ll), sE2 = warp_sum(has ? mom[lane].sE2 : 0ll);
                const long long sAM = warp_sum(has ? mom[lane].sAM : 0ll), sM2 = warp_sum(has ? mom[lane].sM2 : 0ll);
                const I128 z = {0ull, 0ll};
                const I128 sE3 = warp_sum128(has ? mom[lane].sE3 : z), sE4 = warp_sum128(has ? mom[lane].sE4 : z);
                const I128 sAM3 = warp_sum128(has ? mom[lane].sAM3 : z), sM4 = warp_sum128(has ? mom[lane].sM4 : z);
                if (lane == 0) {
                    FamPart f = s_part[0];  // the chunks' family statistics, joined in order
                    for (uint32_t k = 1; k < CS; ++k) join_part(f, s_part[k]);
                    pa_step_record *rec = P.rec + rd.rec_off + i;
                    rec->beta = P.beta[rd.beta_off + i];
                    rec->lnQ = lnQ_i;
                    rec->minus_betaF = P.rec[rd.rec_off + i - 1].minus_betaF + lnQ_i;
                    rec->sumE = sE;
                    rec->sumE2 = sE2;
                    rec->sumAbsM = sAM;
                    rec->sumM2 = sM2;
                    rec->sum_c2 = f.c2;
                    rec->sumE3[0] = sE3.lo;
                    rec->sumE3[1] = (unsigned long long)sE3.hi;
                    rec->sumE4[0] = sE4.lo;
                    rec->sumE4[1] = (unsigned long long)sE4.hi;
                    rec->sumAbsM3[0] = sAM3.lo;
                    rec->sumAbsM3[1] = (unsigned long long)sAM3.hi;
                    rec->sumM4[0] = sM4.lo;
                    rec->sumM4[1] = (unsigned long long)sM4.hi;
                    rec->R = R;
                    rec->R_target = rd.R;
                    rec->n_fam = f.nfam;
                    rec->max_fam = f.cmax;
                    rec->N = N;
                    rec->status = 0;
                    st->step = i;
                    st->R_cur = R;
                    st->R_new = R;
                }
            } else if (prep) {  // ln Q_{i+1}, E_min, and per level floor(tau) and the draw threshold,
                                // tau = R_target w[n] / S
                if (tid == 32) {
                    const int32_t Emin = eb + 4 * (int32_t)lvl_lo;
                    const double dbeta = P.beta[rd.beta_off + i + 1] - P.beta[rd.beta_off + i];
                    st->lnQ = (-dbeta) * (double)Emin + sh_logS - sh_logR;
                    st->Emin = Emin;
                    st->n_levels = nb_l;
                }
                const double *wt = P.wt + P.wtoff[rd.wt_off + i + 1];
                const double S = sh_S;
                for (uint32_t n = tid - 32; n < nb_l; n += nt - 32) {
                    const double tau = __ddiv_rn(__dmul_rn((double)rd.R, wt[n]), S);
                    const double fl = floor(tau);
                    flo_tab[n] = (uint32_t)fl;
                    thr_tab[n] = (unsigned long long)ceil(__dmul_rn(__dsub_rn(tau, fl), 4294967296.0));
                }
            }
            __syncthreads();  // the tables and the run state, before the next resampling reads them
        }
    }
}

// --------------------------------------------------------------------------
// Calibration of the integer-multiplier roof: independent Philox4x32-10 calls
// (8 per thread and iteration), results folded into one word per thread.
// --------------------------------------------------------------------------
template <bool WIDE>
__global__ void __launch_bounds__(128) philox_calibration_kernel(uint32_t *out, uint32_t iters)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    PhiloxKeys K;
    philox_keys(K, 12345u, 678u);
    const uint32_t hi1_0 = __umulhi(0xCD9E8D57u, 7u), lo1_0 = 0xCD9E8D57u * 7u;
    uint32_t acc = 0;
    for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
        for (uint32_t g = 0; g < 8; ++g) {
            const uint4 u = philox_rk<WIDE>(t * 8 + g, it, 1u, hi1_0, lo1_0, K);
            acc ^= u.x ^ u.y ^ u.z ^ u.w;
        }
    }
    out[t] = acc;
}

// The record of each listed run at the temperature it has reached (a gather
// for pa_step_records: one copy back to the host for a whole batch).
__global__ void gather_records_kernel(Pool P, const uint32_t *runs, uint32_t n, pa_step_record *out)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const uint32_t run = runs[t];
    out[t] = P.rec[P.runs[run].rec_off + P.st[run].step];
}

}  // namespace

// ------------------------------------------------------------------ launchers
// The small-run kernel for (L, glass, variant): variant 0 = 512 threads, two
// CTAs per SM; 1 = up to 512 threads, one per SM; 2 = up to 768, one per SM;
// 3 and 4 = as 1 and 2 with 4 lanes per replica (L = 8: 4 per word; L = 16: 1 per
// word), launched with the comparison bits drawn ahead.
template <bool SG, uint32_t HW, uint32_t LPW>
static void *small_kernel_v(uint32_t variant)
{
    return variant == 0   ? (void *)anneal_small_kernel<SG, HW, LPW, 512, 2>
           : variant == 1 ? (void *)anneal_small_kernel<SG, HW, LPW, 512, 1>
                          : (void *)anneal_small_kernel<SG, HW, LPW, 768, 1>;
}

static void *small_kernel(uint32_t L, int sg, uint32_t variant)
{
    if (L == 8 && variant >= 3)
        return sg ? small_kernel_v<true, 1, 4>(variant - 2) : small_kernel_v<false, 1, 4>(variant - 2);
    if (L == 16 && variant >= 3)
        return sg ? small_kernel_v<true, 4, 1>(variant - 2) : small_kernel_v<false, 4, 1>(variant - 2);
    if (L == 8) return sg ? small_kernel_v<true, 1, SMALL_LPW_L8>(variant) : small_kernel_v<false, 1, SMALL_LPW_L8>(variant);
    if (L == 16)
        return sg ? small_kernel_v<true, 4, SMALL_LPW_L16>(variant) : small_kernel_v<false, 4, SMALL_LPW_L16>(variant);
    return sg ? small_kernel_v<true, 16, SMALL_LPW_L32>(variant) : small_kernel_v<false, 16, SMALL_LPW_L32>(variant);
}

constexpr uint32_t SMALL_PRE_BYTES = 96 * 1024;  // shared memory for precomputed comparison bits

static cudaLaunchConfig_t small_launch_config(uint32_t n_clusters, const SmallShape &sh, cudaStream_t s,
                                              cudaLaunchAttribute *at)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(n_clusters * sh.cs);
    cfg.blockDim = dim3(sh.block);
    cfg.dynamicSmemBytes = sh.smem;
    cfg.stream = s;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = sh.cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cfg;
}

static int small_fit(uint32_t L, int any_glass, const SmallShape &sh)
{
    cudaLaunchAttribute at[1];
    cudaLaunchConfig_t cfg = small_launch_config(1, sh, 0, at);
    int fit = 0;
    if (cudaOccupancyMaxActiveClusters(&fit, small_kernel(L, any_glass, sh.variant), &cfg) != cudaSuccess) {
        (void)cudaGetLastError();
        fit = 0;
    }
    return fit;
}

// floor(sqrt(R)), the same integer the kernel computes
static uint32_t isqrt_u32(uint32_t R)
{
    uint32_t q = (uint32_t)std::sqrt((float)R);
    while (q * q > R) --q;
    while ((q + 1) * (q + 1) <= R) ++q;
    return q;
}

// Launch shapes of the small-run kernel for n runs of lattice size L.  A run's
// steps are a chain of cluster barriers, so a run whose CTAs share SMs with
// another run's is slower by the sharing, and the launch lasts as long as its
// slowest run: every shape here keeps all clusters on SMs of their own (asked
// of the occupancy calculator), the largest cluster first (at most 8 CTAs).
// small_shape: a block covering a CTA's equal share of R + 3 sqrt(R) + 1
// children (beyond the nearest-integer resampling's spread); without one,
// 512-thread CTAs two per SM, about two CTAs per SM over all the runs, the
// cluster at most the tiles of the largest capacity.
SmallShape small_shape(uint32_t L, int any_glass, uint32_t n_runs, uint32_t R_max, uint32_t R_cap_max)
{
    const uint32_t hw = L * L / 64;
    const uint32_t lpr = hw * (L == 8 ? SMALL_LPW_L8 : L == 16 ? SMALL_LPW_L16 : SMALL_LPW_L32);
    const uint32_t R_est = R_max + 3 * isqrt_u32(R_max) + 1;
    for (uint32_t cs = 8; cs >= 1; --cs) {
        const uint32_t chunk = (R_est + cs - 1) / cs;
        uint32_t block = (chunk * lpr + 31) / 32 * 32;
        block = block < 128 ? 128 : block;
        if (block > 768) break;  // smaller clusters only need larger blocks
        const SmallShape sh = {cs, block, block <= 512 ? 1u : 2u, 0u, 0u};
        if (small_fit(L, any_glass, sh) >= (int)n_runs) return sh;
    }
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        (void)cudaGetLastError();
        sms = 152;
    }
    const uint32_t tiles = (R_cap_max + 512 / lpr - 1) / (512 / lpr);
    SmallShape sh = {1, 512, 0, 0, 0};
    while (sh.cs < 8 && 2 * sh.cs * n_runs <= 2u * (uint32_t)sms && 2 * sh.cs <= tiles) sh.cs *= 2;
    return sh;
}

// small_shape_ahead, for launches that cover several temperatures (L = 8, 16):
// CTA 0 resamples and measures while the others sweep slices of
// (R + 3 sqrt(R) + 1) / (CS - 1) children in one tile, 4 lanes per replica,
// drawing the next temperature's comparison bits while CTA 0 measures.  cs = 0
// when none fits.
SmallShape small_shape_ahead(uint32_t L, int any_glass, uint32_t n_runs, uint32_t R_max, uint32_t theta_max)
{
    const SmallShape none = {0, 0, 0, 0, 0};
    if ((L != 8 && L != 16) || theta_max == 0) return none;
    const uint32_t hw = L * L / 64, lpr4 = 4;
    const uint32_t R_est = R_max + 3 * isqrt_u32(R_max) + 1;
    for (uint32_t cs = 8; cs >= 2; --cs) {
        const uint32_t Wc = (R_est + cs - 2) / (cs - 1);
        uint32_t block = (Wc * lpr4 + 31) / 32 * 32;
        block = block < 128 ? 128 : block;
        if (block > 768) break;
        const uint32_t per_h = (block / lpr4) * hw * 8;  // bytes of one half-sweep's bits
        uint32_t H = SMALL_PRE_BYTES / per_h;
        H = H < 2 * theta_max ? H : 2 * theta_max;
        const SmallShape sh = {cs, block, block <= 512 ? 3u : 4u, H, H * per_h};
        if (small_fit(L, any_glass, sh) >= (int)n_runs) return sh;
    }
    return none;
}

void launch_anneal_small(const Pool &P, const uint32_t *runs, uint32_t n_runs, uint32_t L, const SmallShape &sh,
                         int any_glass, uint32_t n_steps, cudaStream_t s)
{
    if (n_runs == 0 || n_steps == 0) return;
    cudaLaunchAttribute at[1];
    const cudaLaunchConfig_t cfg = small_launch_config(n_runs, sh, s, at);
    uint32_t H = sh.H;
    void *args[] = {(void *)&P, (void *)&runs, (void *)&n_steps, (void *)&H};
    cudaLaunchKernelExC(&cfg, small_kernel(L, any_glass, sh.variant), args);
}

void launch_gather_records(const Pool &P, const uint32_t *runs, uint32_t n_runs, pa_step_record *out, cudaStream_t s)
{
    gather_records_kernel<<<(n_runs + 127) / 128, 128, 0, s>>>(P, runs, n_runs, out);
}

cudaError_t prepare_kernels()
{
    for (uint32_t L : {8u, 16u, 32u})
        for (int sg = 0; sg < 2; ++sg)
            for (uint32_t v = 1; v <= (L == 32 ? 2u : 4u); ++v) {
                const cudaError_t e = cudaFuncSetAttribute(small_kernel(L, sg, v),
                                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                           (int)SMALL_PRE_BYTES);
                if (e != cudaSuccess) return e;
            }
    cudaError_t e = cudaFuncSetAttribute(sweep_kernel<false, 1024>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         200 * 1024);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sweep_kernel<true, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(resample_multinomial_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 RESAMPLE_STAGE_MAX * sizeof(int32_t));
    if (e == cudaSuccess)  // Wang pairing with R_cap up to 8192: 144 KB
        e = cudaFuncSetAttribute(wang_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    return e;
}

void launch_init_couplings(const Pool &P, const uint32_t *runs, uint32_t n_runs, cudaStream_t s)
{
    init_couplings_kernel<<<n_runs, 256, 0, s>>>(P, runs);
}

void launch_init_population(const Pool &P, const uint32_t *tile_off, const uint32_t *runs, uint32_t n_runs,
                            uint32_t n_tiles, uint32_t max_pw, cudaStream_t s)
{
    init_population_kernel<<<n_tiles, 128, 4 * 2 * max_pw * sizeof(uint32_t), s>>>(P, tile_off, runs, n_runs);
}

void launch_dos_sample(const Pool &P, const uint32_t *runs, uint32_t n_runs, uint32_t max_R, int init,
                       cudaStream_t s)
{
    if (n_runs == 0 || max_R == 0) return;
    const uint32_t span = DOS_THREADS * DOS_PER_THREAD;
    dos_sample_kernel<<<dim3((max_R + span - 1) / span, n_runs), DOS_THREADS, 0, s>>>(P, runs, init);
}

void launch_resample_multinomial(const Pool &P, const uint32_t *runs, uint32_t n_runs, uint32_t max_Rcap,
                                 cudaStream_t s)
{
    if (n_runs == 0) return;
    const uint32_t stage = max_Rcap < RESAMPLE_STAGE_MAX ? max_Rcap : RESAMPLE_STAGE_MAX;
    resample_multinomial_kernel<<<n_runs, 512, stage * sizeof(int32_t), s>>>(P, runs, stage);
}

void launch_resample_nearest(const Pool &P, const uint32_t *runs, uint32_t n_runs, uint32_t max_Rcap, cudaStream_t s)
{
    if (n_runs == 0) return;
    const dim3 grid(n_runs, run_ctas(max_Rcap));
    if (grid.y == 1) {  // every population in one CTA: one launch
        resample_counts_kernel<true><<<grid, RESAMPLE_THREADS, 0, s>>>(P, runs);
        return;
    }
    resample_counts_kernel<false><<<grid, RESAMPLE_THREADS, 0, s>>>(P, runs);
    resample_parents_kernel<<<grid, RESAMPLE_THREADS, 0, s>>>(P, runs);
}

// Launch shapes of the bit-sliced kernel: WPT plane words per thread and
// `block` threads per CTA (a multiple of the threads per replica, HW / WPT).
SweepCfg sweep_fast_config(uint32_t L, uint32_t WPT, uint32_t block)
{
    SweepCfg c{};
    const uint32_t N = L * L, HW = N / 64;
    c.fast = 1;
    c.WPT = WPT;
    c.TPR = HW / WPT;
    c.block = block;
    c.RPC = block / c.TPR;
    c.G = N / 8;
    c.PS = 0;
    c.smem = c.RPC * 2 * HW * 4 + 8 * c.RPC;
    return c;
}

std::vector<SweepCfg> sweep_candidates(uint32_t L, int allow_fast)
{
    std::vector<SweepCfg> v;
    const uint32_t N = L * L;
    const bool pow2 = L >= 8 && L <= 256 && (L & (L - 1)) == 0;
    if (pow2 && allow_fast) {
        const uint32_t HW = N / 64;
        if (HW <= 128) {
            v.push_back(sweep_fast_config(L, 1, 128));
            v.push_back(sweep_fast_config(L, 1, 256));
        } else if (HW == 256) {
            v.push_back(sweep_fast_config(L, 1, 256));
            v.push_back(sweep_fast_config(L, 2, 128));
        } else {  // L = 256
            v.push_back(sweep_fast_config(L, 4, 256));
            v.push_back(sweep_fast_config(L, 2, 512));
            v.push_back(sweep_fast_config(L, 1, 1024));
        }
        return v;
    }
    const uint32_t Pt = row_pitch(L), Lh = L / 2, CW = (L * Lh + 31) / 32;
    if (allow_fast && CW <= 1024) {  // compact rows
        for (uint32_t target : {256u, 128u}) {
            SweepCfg c{};
            c.fast = 3;
            c.WPT = 1;
            c.TPR = CW;
            c.RPC = target / CW > 0 ? target / CW : 1;
            c.block = c.RPC * CW;
            c.G = (N + 7) / 8;
            c.PS = Pt;
            c.smem = c.RPC * 2 * ((Lh + 31) / 32 + CW + Lh / 32 + 2) * 4 + 8 * c.RPC;
            if (v.empty() || v.back().block != c.block) v.push_back(c);
        }
    }
    if (allow_fast && L >= 6 && Pt <= 32 && Pt != L / 2) {  // padded rows
        const uint32_t HW = L * Pt / 32;
        for (uint32_t target : {128u, 256u}) {
            SweepCfg c{};
            c.fast = 2;
            c.WPT = 1;
            c.TPR = HW;
            c.RPC = target / HW > 0 ? target / HW : 1;
            c.block = c.RPC * HW;
            c.G = (N + 7) / 8;
            c.PS = Pt;  // the row pitch selects the kernel instantiation
            c.smem = c.RPC * 2 * HW * 4 + 8 * c.RPC;
            v.push_back(c);
        }
    }
    if (!v.empty()) return v;
    SweepCfg c{};
    c.fast = 0;
    c.WPT = 1;
    c.G = (N + 7) / 8;
    uint32_t tpr = 1;
    while (tpr < c.G) tpr <<= 1;
    if (tpr <= 128) {
        c.block = 128;
        c.TPR = tpr;
        c.RPC = 128 / tpr;
    } else {
        c.TPR = tpr < 1024 ? tpr : 1024;
        c.block = c.TPR;
        c.RPC = 1;
    }
    c.PS = 4 * c.G;
    c.smem = c.RPC * 2 * c.PS + 2 * c.PS + 8 * c.RPC;
    v.push_back(c);
    return v;
}

void launch_sweep(const Pool &P, const uint32_t *group_runs, const uint32_t *tile_off, uint32_t n_group_runs,
                  uint32_t n_tiles, const SweepCfg &cfg, int any_glass, cudaStream_t s)
{
    const dim3 grid(n_tiles);
#define PA_SWEEP_FAST(SG, WPT, MAXT) \
    sweep_pow2_kernel<SG, WPT, MAXT><<<grid, cfg.block, cfg.smem, s>>>(P, group_runs, tile_off, n_group_runs, cfg)
#define PA_SWEEP_FAST2(SG, WPT) \
    sweep_pow2_kernel_2cta<SG, WPT><<<grid, cfg.block, cfg.smem, s>>>(P, group_runs, tile_off, n_group_runs, cfg)
    if (cfg.fast == 3) {  // compact rows; the row pitch is at most 32 exactly when L/2 <= 31
#define PA_SWEEP_COMPACT(MAXT, NARROW)                                                                            \
    (any_glass ? sweep_compact_kernel<true, MAXT, NARROW><<<grid, cfg.block, cfg.smem, s>>>(P, group_runs, tile_off, \
                                                                                          n_group_runs, cfg)      \
               : sweep_compact_kernel<false, MAXT, NARROW><<<grid, cfg.block, cfg.smem, s>>>(P, group_runs,         \
                                                                                           tile_off, n_group_runs, cfg))
        if (cfg.block <= 256 && cfg.PS <= 32)
            PA_SWEEP_COMPACT(256, true);
        else if (cfg.block <= 256)
            PA_SWEEP_COMPACT(256, false);
        else
            PA_SWEEP_COMPACT(1024, false);
#undef PA_SWEEP_COMPACT
    } else if (cfg.fast == 2) {  // padded rows: cfg.PS holds the row pitch
#define PA_SWEEP_PAD(PT)                                                                                 \
    (any_glass ? sweep_pad_kernel<true, PT><<<grid, cfg.block, cfg.smem, s>>>(P, group_runs, tile_off, \
                                                                               n_group_runs, cfg)      \
               : sweep_pad_kernel<false, PT><<<grid, cfg.block, cfg.smem, s>>>(P, group_runs, tile_off, \
                                                                                n_group_runs, cfg))
        if (cfg.PS == 8)
            PA_SWEEP_PAD(8);
        else if (cfg.PS == 16)
            PA_SWEEP_PAD(16);
        else
            PA_SWEEP_PAD(32);
#undef PA_SWEEP_PAD
    } else if (!cfg.fast && cfg.G <= cfg.TPR && cfg.block <= 512)
        sweep_kernel<true, 512><<<grid, cfg.block, cfg.smem, s>>>(P, group_runs, tile_off, n_group_runs, cfg);
    else if (!cfg.fast)
        sweep_kernel<false, 1024><<<grid, cfg.block, cfg.smem, s>>>(P, group_runs, tile_off, n_group_runs, cfg);
    else if (cfg.WPT == 1 && cfg.block <= 256)
        any_glass ? PA_SWEEP_FAST(true, 1, 256) : PA_SWEEP_FAST(false, 1, 256);
    else if (cfg.WPT == 1)
        any_glass ? PA_SWEEP_FAST(true, 1, 1024) : PA_SWEEP_FAST(false, 1, 1024);
    else if (cfg.WPT == 2)
        any_glass ? PA_SWEEP_FAST2(true, 2) : PA_SWEEP_FAST2(false, 2);
    else
        any_glass ? PA_SWEEP_FAST(true, 4, 256) : PA_SWEEP_FAST(false, 4, 256);
#undef PA_SWEEP_FAST
#undef PA_SWEEP_FAST2
}

void launch_overlap(const Pool &P, const uint32_t *q_runs, uint32_t n_q_runs, uint32_t max_Rcap, int init,
                    cudaStream_t s)
{
    dim3 grid((max_Rcap + 255) / 256, n_q_runs);
    overlap_kernel<<<grid, 256, 0, s>>>(P, q_runs, init);
}

void launch_measure(const Pool &P, const uint32_t *runs, uint32_t n_runs, uint32_t max_Rcap, int init,
                    cudaStream_t s)
{
    if (n_runs == 0) return;
    measure_kernel<<<dim3(n_runs, run_ctas(max_Rcap)), PA_MEASURE_THREADS, 0, s>>>(P, runs, init);
}

void launch_philox_calibration(uint32_t *out, uint32_t blocks, uint32_t threads, uint32_t iters, bool wide,
                               cudaStream_t s)
{
    if (wide)
        philox_calibration_kernel<true><<<blocks, threads, 0, s>>>(out, iters);
    else
        philox_calibration_kernel<false><<<blocks, threads, 0, s>>>(out, iters);
}

void launch_wavg_wang(const pa_step_record *recs, const unsigned long long *rec_off, const uint32_t *qh,
                      const uint32_t *qhp, const uint32_t *qhw, const unsigned long long *qh_off, uint32_t n_groups,
                      uint32_t M, uint32_t n_steps, uint32_t N, uint32_t kind, pa_wavg *out, double *w, double *Pq,
                      double *Pqp, double *Pqw, cudaStream_t s)
{
    const uint64_t nGM = (uint64_t)n_groups * M;
    wavg_lambda_kernel<<<(unsigned)((32 * nGM + 127) / 128), 128, 0, s>>>(recs, rec_off, n_groups, M, n_steps, kind, w);
    // groups on x (up to 2^31 - 1 of them), temperatures on y
    const dim3 grid(n_groups, (n_steps + 3) / 4);  // one warp per (group, temperature)
    wavg_step_kernel<<<grid, 128, 0, s>>>(recs, rec_off, n_groups, M, n_steps, N, out, w);
    wavg_finish_kernel<<<grid, 128, 0, s>>>(n_groups, M, n_steps, N, out, w);
    if (Pq || Pqp || Pqw) {
        dim3 grid(n_groups, n_steps);
        wavg_q_kernel<<<grid, 256, 0, s>>>(recs, rec_off, qh, qhp, qhw, qh_off, M, n_steps, N, w, Pq, Pqp, Pqw);
    }
}

void launch_wavg(const pa_step_record *recs, const unsigned long long *rec_off, const uint32_t *qh,
                 const uint32_t *qhp, const unsigned long long *qh_off, uint32_t n_groups, uint32_t M,
                 uint32_t n_steps, uint32_t N, uint32_t kind, pa_wavg *out, double *w, double *Pq, double *Pqp,
                 cudaStream_t s)
{
    launch_wavg_wang(recs, rec_off, qh, qhp, nullptr, qh_off, n_groups, M, n_steps, N, kind, out, w, Pq, Pqp, nullptr,
                     s);
}

// keys (8 R_cap bytes, reused for the families) + pi and sigma (4 R_cap bytes each)
// + the bucket counters: about 104 KB at R_cap = 5630, so two CTAs fit on an SM
size_t wang_smem_bytes(uint32_t max_Rcap)
{
    const uint32_t cap = (max_Rcap + 3) / 4 * 4;
    return (size_t)cap * 16 + (size_t)WANG_BUCKETS * 4;
}

void launch_wang(const Pool &P, const uint32_t *runs, uint32_t n_runs, uint32_t max_Rcap, int init, cudaStream_t s)
{
    if (n_runs == 0) return;
    const uint32_t cap = (max_Rcap + 3) / 4 * 4;
    wang_kernel<<<n_runs, 1024, wang_smem_bytes(max_Rcap), s>>>(P, runs, init, cap);  // 1024 * 4 = WANG_BUCKETS
}

}  // namespace pa
