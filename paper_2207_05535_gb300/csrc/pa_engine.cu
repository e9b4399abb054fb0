// Host side of the population-annealing engine: the C ABI declared in pa.h.
//
// An engine owns fixed device pools (replica slots, spin words, records,
// overlap histograms, per-run tables, scratch) and a set of resident runs,
// each at its own offsets (pa_internal.cuh).  Runs enter by admission: the
// engine carves their ranges from free lists, uploads their descriptor and
// tables, and with the next enqueued work draws their beta_0 populations and
// measures step 0.  Every anneal step then advances all resident, unfinished
// runs by one temperature in shared launches: resample (all runs), sweep (one
// launch per lattice size over a work list of (run, tile)), overlaps and
// measurement.  Kernels read each run's temperature index from device state,
// so runs at different temperatures share launches and one captured graph
// serves every step while the resident set is unchanged.
//
// pa_create sizes the pools to exactly its runs and admits them all (batch
// form); pa_server_create sizes them from a configuration and runs enter and
// leave with pa_admit / pa_retire between steps (continuous batching).
//
// Host tables: the resampling weights exp(-4 n dbeta) for n = 0..N are built
// with libm once per distinct (N, dbeta) and shared by every run and step that
// uses them; the Metropolis thresholds floor(exp(-4 m beta_i) 2^32) per step.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "pa_internal.cuh"

using namespace pa;

namespace {

// First-fit free list over [0, cap) in arbitrary units.
struct FreeList {
    uint64_t cap = 0;
    std::map<uint64_t, uint64_t> free_;  // offset -> size
    void init(uint64_t c)
    {
        cap = c;
        free_.clear();
        if (c) free_[0] = c;
    }
    bool alloc(uint64_t n, uint64_t &off)
    {
        if (n == 0) {
            off = 0;
            return true;
        }
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (it->second >= n) {
                off = it->first;
                const uint64_t rest = it->second - n;
                free_.erase(it);
                if (rest) free_[off + n] = rest;
                return true;
            }
        return false;
    }
    void release(uint64_t off, uint64_t n)
    {
        if (n == 0) return;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct Tuning {
    std::vector<SweepCfg> candidates;
    uint32_t pick = 0;
    bool tuned = false;
    float ms = 0.f;
    uint32_t round = 0;       // tuning steps taken so far
    std::vector<float> best;  // per candidate: its fastest timed step (ms), 0 = not timed yet
};

// Launch shapes chosen by timing are shared by every engine of the process on the
// same device: a new engine reuses the choice for a lattice size instead of timing
// the candidates again.  Key: (device, L, bit-sliced kernels allowed).
std::mutex g_tune_mu;
std::map<std::tuple<int, uint32_t, int>, uint32_t> g_tuned;

std::tuple<int, uint32_t, int> tune_key(uint32_t L, uint32_t flags)
{
    int dev = 0;
    cudaGetDevice(&dev);
    return std::make_tuple(dev, L, (flags & PA_CREATE_GENERIC_SWEEP) ? 0 : 1);
}

// Device allocator: cudaMalloc / cudaFree unless the caller installed callbacks
// with pa_set_allocator.  An engine keeps the allocator it was created with, so
// every block is freed by the allocator that made it.
struct Allocator {
    pa_alloc_fn alloc = nullptr;
    pa_free_fn free_ = nullptr;
    void *ctx = nullptr;
};
std::mutex g_alloc_mu;
Allocator g_alloc;

Allocator current_allocator()
{
    std::lock_guard<std::mutex> lock(g_alloc_mu);
    return g_alloc;
}

// One block from allocator `a` on `stream`; nullptr when it is refused.
void *device_alloc(const Allocator &a, size_t bytes, cudaStream_t stream)
{
    if (bytes == 0) bytes = 16;
    if (a.alloc) {
        int dev = 0;
        cudaGetDevice(&dev);
        return a.alloc(bytes, dev, stream, a.ctx);
    }
    void *q = nullptr;
    if (cudaMalloc(&q, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return q;
}

void device_free(const Allocator &a, void *p, size_t bytes, cudaStream_t stream)
{
    if (!p) return;
    if (bytes == 0) bytes = 16;
    if (a.free_) {
        int dev = 0;
        cudaGetDevice(&dev);
        a.free_(p, bytes, dev, stream, a.ctx);
    } else {
        cudaFree(p);
    }
}

struct SmallGroup {  // small runs of one lattice size, annealed by anneal_small_kernel
    uint32_t L = 0;
    int any_glass = 0;
    std::vector<uint32_t> runs;
    uint64_t runs_off = 0;  // in d_meta
    uint32_t R_max = 0, R_cap_max = 0, theta_max = 0;
    SmallShape shape = {1, 512, 0, 0, 0};  // one temperature per launch
    SmallShape ahead = {0, 0, 0, 0, 0};     // several temperatures per launch (cs = 0: none)
};

struct SweepGroup {  // runs of one lattice size among the resident runs
    uint32_t L = 0;
    int any_glass = 0;
    std::vector<uint32_t> runs;
    uint64_t runs_off = 0;               // in d_meta
    std::vector<uint64_t> tile_map_off;  // per candidate, in d_meta (n + 1 entries)
    std::vector<uint32_t> n_tiles;       // per candidate
};

// Offsets of one run in each pool (units of that pool).
struct Ranges {
    uint64_t rep = 0, spin = 0, rec = 0, qh = 0, scr = 0, J = 0, beta = 0, thr = 0, wto = 0;
};

struct RunHost {  // host view of a resident run
    bool used = false;
    pa_run_desc d{};
    Ranges g;
    uint32_t steps_done = 0;  // temperature index reached (mirrors the device while no error)
    uint64_t dos_hash = 0;    // theta = PA_THETA_INF: hash of ln g (a checkpoint must come from the same one)
};

// FNV-1a over the bytes of ln g(E), 2N + 1 doubles (0 when the run has none).
uint64_t dos_hash_of(const pa_run_desc &d)
{
    if (d.theta != PA_THETA_INF || !d.log_g) return 0;
    uint64_t h = 1469598103934665603ull;
    const unsigned char *b = reinterpret_cast<const unsigned char *>(d.log_g);
    for (size_t k = 0; k < sizeof(double) * (2ull * d.L * d.L + 1); ++k) h = (h ^ b[k]) * 1099511628211ull;
    return h;
}

}  // namespace

struct pa_engine {
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    uint32_t flags = 0;
    bool server = false;
    // slots
    uint32_t S = 0;
    std::vector<RunDev> rd;
    std::vector<RunHost> rh;
    std::vector<uint32_t> active;   // resident slots, admission order
    std::vector<uint32_t> pending;  // admitted, beta_0 not drawn yet
    // pools and their free lists
    Pool P{};
    RunDev *d_runs = nullptr;
    double *d_beta = nullptr, *d_wt = nullptr;
    unsigned long long *d_thr = nullptr, *d_wtoff = nullptr;
    FreeList fl_rep, fl_spin, fl_rec, fl_qh, fl_scr, fl_J, fl_beta, fl_thr, fl_wto;
    uint64_t wt_cap = 0, wt_used = 0;
    std::map<std::pair<uint32_t, uint64_t>, uint64_t> wt_cache;  // (N, dbeta bits) -> offset
    std::map<std::vector<double>, uint64_t> dos_cache;            // (ln g, schedule, N) -> offset
    // device metadata (lists and work lists), rebuilt when the resident set changes
    uint32_t *d_meta = nullptr;
    uint64_t meta_cap = 0;
    std::vector<uint32_t> h_meta;
    bool dirty = true;
    uint64_t active_off = 0, q_off = 0, init_runs_off = 0, init_tiles_off = 0, init_q_off = 0;
    uint32_t init_q_n = 0;
    std::vector<uint32_t> q_runs;
    uint32_t init_n = 0, init_tiles = 0;
    std::vector<uint32_t> inf_runs;  // resident theta = PA_THETA_INF runs
    std::vector<uint32_t> near_runs, multi_runs;  // resident runs by resampling scheme
    uint64_t near_off = 0, multi_off = 0;
    uint32_t near_maxcap = 0, multi_maxcap = 0;
    std::vector<uint32_t> wang_runs;  // resident runs with PA_Q_WANG
    uint64_t wang_off = 0, init_wang_off = 0;
    uint32_t wang_maxcap = 0, init_wang_n = 0, init_wang_maxcap = 0;
    uint64_t inf_off = 0, init_inf_off = 0;
    uint32_t inf_maxR = 0, init_inf_n = 0, init_inf_maxR = 0;
    std::vector<SweepGroup> groups;
    std::vector<SmallGroup> small;     // runs on the one-launch-per-step path
    std::vector<uint32_t> big;         // the other resident runs (per-stage kernels)
    uint64_t big_off = 0;
    std::map<uint32_t, Tuning> tuning;  // per lattice size
    uint32_t max_Rcap_active = 0, max_pw = 1;
    // execution
    uint64_t launches = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    uint64_t graph_tick_launches = 0;  // kernel launches in one replay of the graph
    pa_status latched = PA_OK;
    bool profiling = false;
    std::vector<cudaEvent_t> ev_free;
    struct Timed {
        int kind;
        cudaEvent_t a, b;
    };
    std::vector<Timed> timed;
    uint64_t h2d = 0, d2h = 0;
    Allocator alloc;                                   // the allocator of every block below
    void *wa_buf = nullptr;                            // weighted averages of resident runs
    size_t wa_bytes = 0;
    void *sr_buf = nullptr;                            // pa_step_records staging
    size_t sr_bytes = 0;
    std::vector<std::pair<void *, size_t>> allocs;     // pools
};

namespace {

pa_status cuda_fail(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return PA_OK;
    std::fprintf(stderr, "libpa: %s: %s\n", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? PA_ERR_OOM : PA_ERR_CUDA;
}

#define PA_CUDA(call)                                       \
    do {                                                    \
        cudaError_t _e = (call);                            \
        if (_e != cudaSuccess) return cuda_fail(_e, #call); \
    } while (0)

#define PA_TRY(expr)                \
    do {                            \
        pa_status _s = (expr);      \
        if (_s != PA_OK) return _s; \
    } while (0)

template <typename T>
pa_status dalloc(pa_engine *e, T **p, size_t count)
{
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = 16;
    void *q = device_alloc(e->alloc, bytes, e->stream);
    if (!q) return PA_ERR_OOM;
    e->allocs.emplace_back(q, bytes);
    *p = static_cast<T *>(q);
    return PA_OK;
}

// A growable engine-owned buffer (the old contents are not kept).
pa_status ensure_buffer(pa_engine *e, void **buf, size_t *have, size_t bytes)
{
    if (*have >= bytes) return PA_OK;
    if (*buf) {
        cudaStreamSynchronize(e->stream);  // no queued work may still use it
        device_free(e->alloc, *buf, *have, e->stream);
    }
    *buf = nullptr;
    *have = 0;
    void *q = device_alloc(e->alloc, bytes, e->stream);
    if (!q) return PA_ERR_OOM;
    *buf = q;
    *have = bytes;
    return PA_OK;
}

uint32_t cap_of(const pa_run_desc &d)
{
    if (d.R_cap) return d.R_cap;
    if (d.resample == PA_MULTINOMIAL) return d.R;
    return d.R + 8u * (uint32_t)std::ceil(std::sqrt((double)d.R)) + 64u;
}

uint32_t plane_words(uint32_t L) { return plane_words_of(L); }
uint32_t stride_words(uint32_t L) { return (2 * plane_words(L) + 3) / 4 * 4; }

Ranges sizes_of(const pa_run_desc &d)
{
    const uint32_t N = d.L * d.L, cap = cap_of(d);
    Ranges z;
    z.rep = cap;
    z.spin = (uint64_t)cap * stride_words(d.L);
    z.rec = d.n_beta;
    z.qh = d.overlap ? (uint64_t)d.n_beta * (N + 1) : 0;
    z.scr = scratch_words(N, cap);
    z.J = 2ull * stride_words(d.L) + 8ull * plane_words(d.L);
    z.beta = d.n_beta;
    z.thr = 2ull * d.n_beta;
    z.wto = d.n_beta;
    return z;
}

// Validate runs[0..n) as one admission (pair indices relative to the batch).
pa_status validate(const pa_run_desc *runs, uint32_t n)
{
    if (!runs || n == 0) return PA_ERR_INVALID_ARG;
    for (uint32_t r = 0; r < n; ++r) {
        const pa_run_desc &d = runs[r];
        if (d.L < 4 || d.L > 256 || (d.L & 1u)) return PA_ERR_INVALID_ARG;
        if (d.model > PA_EA_PMJ || d.resample > PA_MULTINOMIAL || d.overlap > 7u || d.reserved)
            return PA_ERR_INVALID_ARG;
        if ((d.overlap & PA_Q_WANG) && cap_of(d) > PA_WANG_MAX_RCAP) return PA_ERR_INVALID_ARG;
        if (d.R < 1 || d.n_beta < 1 || !d.beta) return PA_ERR_INVALID_ARG;
        if (d.theta == PA_THETA_INF) {  // needs a density of states; no configurations, so no overlaps
            if (!d.log_g || d.overlap) return PA_ERR_INVALID_ARG;
            int parity = -1;  // energies of a lattice's states differ by multiples of 4: u of one parity
            for (uint32_t u = 0; u <= 2 * d.L * d.L; ++u) {
                const double v = d.log_g[u];
                if (std::isnan(v) || v == INFINITY) return PA_ERR_INVALID_ARG;
                if (v > -INFINITY) {
                    if (parity >= 0 && (int)(u & 1u) != parity) return PA_ERR_INVALID_ARG;
                    parity = (int)(u & 1u);
                }
            }
            if (parity < 0) return PA_ERR_INVALID_ARG;
        } else if (d.theta > (1u << 22)) {
            return PA_ERR_INVALID_ARG;
        }
        if (cap_of(d) < d.R) return PA_ERR_INVALID_ARG;
        for (uint32_t i = 1; i < d.n_beta; ++i)
            if (!(d.beta[i] >= d.beta[i - 1])) return PA_ERR_INVALID_ARG;
        if (!std::isfinite(d.beta[0]) || !std::isfinite(d.beta[d.n_beta - 1])) return PA_ERR_INVALID_ARG;
        if (d.overlap & PA_Q_PAIR) {
            if (d.paired < 0 || (uint32_t)d.paired >= n || (uint32_t)d.paired == r) return PA_ERR_INVALID_ARG;
            const pa_run_desc &o = runs[d.paired];
            if (o.paired != (int32_t)r || !(o.overlap & PA_Q_PAIR) || o.L != d.L || o.n_beta != d.n_beta)
                return PA_ERR_INVALID_ARG;
        }
    }
    return PA_OK;
}

// Metropolis threshold: floor(exp(-4 m beta) * 2^32), capped at 2^32.
unsigned long long threshold(double beta, int m)
{
    const double p = std::exp(-(double)(4 * m) * beta);
    if (p >= 1.0) return 1ull << 32;
    return (unsigned long long)(p * 4294967296.0);
}

pa_status alloc_pools(pa_engine *e, const pa_server_config &c)
{
    e->S = c.max_runs;
    e->rd.assign(e->S, RunDev{});
    e->rh.assign(e->S, RunHost{});
    PA_TRY(dalloc(e, &e->d_runs, e->S));
    PA_TRY(dalloc(e, &e->P.st, e->S));
    for (int b = 0; b < 2; ++b) {
        PA_TRY(dalloc(e, &e->P.spins[b], c.spin_words));
        PA_TRY(dalloc(e, &e->P.E[b], c.replica_capacity));
        PA_TRY(dalloc(e, &e->P.M[b], c.replica_capacity));
        PA_TRY(dalloc(e, &e->P.fam[b], c.replica_capacity));
        PA_CUDA(cudaMemsetAsync(e->P.spins[b], 0, sizeof(uint32_t) * std::max<uint64_t>(c.spin_words, 1), e->stream));
    }
    PA_TRY(dalloc(e, &e->P.parent, c.replica_capacity));
    PA_TRY(dalloc(e, &e->P.cnt, c.replica_capacity));
    PA_TRY(dalloc(e, &e->P.rec, c.record_capacity));
    PA_TRY(dalloc(e, &e->P.qh, c.qhist_words));
    PA_TRY(dalloc(e, &e->P.qhp, c.qhist_words));
    PA_TRY(dalloc(e, &e->P.qhw, c.qhist_words));
    PA_TRY(dalloc(e, &e->P.J, c.coupling_words));
    PA_TRY(dalloc(e, &e->P.scratch, c.scratch_words));
    PA_TRY(dalloc(e, &e->P.status, 1));
    PA_TRY(dalloc(e, &e->d_beta, c.record_capacity));
    PA_TRY(dalloc(e, &e->d_thr, 2 * c.record_capacity));
    PA_TRY(dalloc(e, &e->d_wtoff, c.record_capacity));
    PA_TRY(dalloc(e, &e->d_wt, c.table_doubles));
    e->meta_cap = 20ull * e->S + 3ull * 128 + 1024;  // every work list of rebuild() (up to 16 per run slot)
    PA_TRY(dalloc(e, &e->d_meta, e->meta_cap));
    PA_CUDA(cudaMemsetAsync(e->P.status, 0, sizeof(uint32_t), e->stream));
    e->P.runs = e->d_runs;
    e->P.beta = e->d_beta;
    e->P.wt = e->d_wt;
    e->P.wtoff = e->d_wtoff;
    e->P.thr = e->d_thr;
    e->fl_rep.init(c.replica_capacity);
    e->fl_spin.init(c.spin_words);
    e->fl_rec.init(c.record_capacity);
    e->fl_qh.init(c.qhist_words);
    e->fl_scr.init(c.scratch_words);
    e->fl_J.init(c.coupling_words);
    e->fl_beta.init(c.record_capacity);
    e->fl_thr.init(2 * c.record_capacity);
    e->fl_wto.init(c.record_capacity);
    e->wt_cap = c.table_doubles;
    return PA_OK;
}

// Weight table exp(-4 n dbeta), n = 0..N, from the cache or built now.
pa_status weight_table(pa_engine *e, uint32_t N, double dbeta, uint64_t &off)
{
    uint64_t bits;
    std::memcpy(&bits, &dbeta, sizeof bits);
    auto key = std::make_pair(N, bits);
    auto it = e->wt_cache.find(key);
    if (it != e->wt_cache.end()) {
        off = it->second;
        return PA_OK;
    }
    if (e->wt_used + N + 1 > e->wt_cap) return PA_ERR_BUSY;
    std::vector<double> t(N + 1);
    for (uint32_t n = 0; n <= N; ++n) t[n] = std::exp(-(double)(4 * n) * dbeta);
    PA_CUDA(cudaMemcpyAsync(e->d_wt + e->wt_used, t.data(), sizeof(double) * t.size(), cudaMemcpyHostToDevice,
                            e->stream));
    PA_CUDA(cudaStreamSynchronize(e->stream));  // t must outlive the copy
    e->h2d += sizeof(double) * t.size();
    off = e->wt_used;
    e->wt_used += N + 1;
    e->wt_cache.emplace(key, off);
    return PA_OK;
}

// theta = PA_THETA_INF: per step i the cumulative weights of the exact energy
// distribution over the levels u = 0..2N (E = 2u - 2N), ascending,
//   C[u] = sum_{v<=u} exp(ln g(v) - beta_i E(v) - c),  c = max_v (ln g(v) - beta_i E(v)),
// then the last level with a positive weight; (2N + 2) doubles per step, built
// with libm on the host and shared by runs with the same (ln g, schedule).
pa_status dos_table(pa_engine *e, const pa_run_desc &d, uint64_t &off)
{
    const uint32_t N = d.L * d.L, U = 2 * N;
    std::vector<double> key(d.log_g, d.log_g + U + 1);
    key.insert(key.end(), d.beta, d.beta + d.n_beta);
    key.push_back((double)N);
    auto it = e->dos_cache.find(key);
    if (it != e->dos_cache.end()) {
        off = it->second;
        return PA_OK;
    }
    const uint64_t n = (uint64_t)d.n_beta * (U + 2);
    if (e->wt_used + n > e->wt_cap) return PA_ERR_BUSY;
    std::vector<double> t(n);
    for (uint32_t i = 0; i < d.n_beta; ++i) {
        double *C = t.data() + (uint64_t)i * (U + 2);
        const double beta = d.beta[i];
        double c = -INFINITY;
        for (uint32_t u = 0; u <= U; ++u)
            if (d.log_g[u] > -INFINITY) {
                const double l = d.log_g[u] - beta * (double)(2 * (int64_t)u - 2 * (int64_t)N);
                if (l > c) c = l;
            }
        double acc = 0.0;
        uint32_t last = 0;
        for (uint32_t u = 0; u <= U; ++u) {
            double p = 0.0;
            if (d.log_g[u] > -INFINITY) {
                const double l = d.log_g[u] - beta * (double)(2 * (int64_t)u - 2 * (int64_t)N);
                p = std::exp(l - c);
            }
            acc = acc + p;
            C[u] = acc;
            if (p > 0.0) last = u;
        }
        C[U + 1] = (double)last;
    }
    PA_CUDA(cudaMemcpyAsync(e->d_wt + e->wt_used, t.data(), sizeof(double) * n, cudaMemcpyHostToDevice, e->stream));
    PA_CUDA(cudaStreamSynchronize(e->stream));  // t must outlive the copy
    e->h2d += sizeof(double) * n;
    off = e->wt_used;
    e->wt_used += n;
    e->dos_cache.emplace(std::move(key), off);
    return PA_OK;
}

// Reserve every pool range of one run (all or nothing).
bool reserve(pa_engine *e, const pa_run_desc &d, Ranges &g)
{
    const Ranges z = sizes_of(d);
    FreeList *fl[9] = {&e->fl_rep, &e->fl_spin, &e->fl_rec, &e->fl_qh, &e->fl_scr,
                       &e->fl_J, &e->fl_beta, &e->fl_thr, &e->fl_wto};
    const uint64_t n[9] = {z.rep, z.spin, z.rec, z.qh, z.scr, z.J, z.beta, z.thr, z.wto};
    uint64_t *o[9] = {&g.rep, &g.spin, &g.rec, &g.qh, &g.scr, &g.J, &g.beta, &g.thr, &g.wto};
    for (int k = 0; k < 9; ++k)
        if (!fl[k]->alloc(n[k], *o[k])) {
            for (int q = 0; q < k; ++q) fl[q]->release(*o[q], n[q]);
            return false;
        }
    return true;
}

void unreserve(pa_engine *e, const pa_run_desc &d, const Ranges &g)
{
    const Ranges z = sizes_of(d);
    e->fl_rep.release(g.rep, z.rep);
    e->fl_spin.release(g.spin, z.spin);
    e->fl_rec.release(g.rec, z.rec);
    e->fl_qh.release(g.qh, z.qh);
    e->fl_scr.release(g.scr, z.scr);
    e->fl_J.release(g.J, z.J);
    e->fl_beta.release(g.beta, z.beta);
    e->fl_thr.release(g.thr, z.thr);
    e->fl_wto.release(g.wto, z.wto);
}

// Admit runs[0..n): reserve slots and ranges and table references (all or
// nothing), upload the descriptors and tables; the beta_0 draw is enqueued
// with the next work.
pa_status admit(pa_engine *e, const pa_run_desc *runs, uint32_t n, uint32_t *slots)
{
    PA_TRY(validate(runs, n));
    std::vector<uint32_t> got;
    for (uint32_t s = 0; s < e->S && got.size() < n; ++s)
        if (!e->rh[s].used) got.push_back(s);
    if (got.size() < n) return PA_ERR_BUSY;
    std::vector<Ranges> gs(n);
    std::vector<std::vector<unsigned long long>> wtos(n);
    std::vector<uint64_t> dos_offs(n, 0);
    uint32_t k = 0;
    pa_status st = PA_OK;
    for (; k < n; ++k) {
        if (!reserve(e, runs[k], gs[k])) {
            st = PA_ERR_BUSY;
            break;
        }
        const pa_run_desc &d = runs[k];
        wtos[k].assign(d.n_beta, 0ull);
        for (uint32_t i = 1; i < d.n_beta && st == PA_OK; ++i) {
            uint64_t off = 0;
            st = weight_table(e, d.L * d.L, d.beta[i] - d.beta[i - 1], off);
            wtos[k][i] = off;
        }
        if (st == PA_OK && d.theta == PA_THETA_INF) st = dos_table(e, d, dos_offs[k]);
        if (st != PA_OK) {
            unreserve(e, runs[k], gs[k]);
            break;
        }
    }
    if (st != PA_OK) {  // roll back the runs reserved so far (cached tables stay)
        for (uint32_t q = 0; q < k; ++q) unreserve(e, runs[q], gs[q]);
        return st;
    }
    for (uint32_t r = 0; r < n; ++r) {
        const pa_run_desc &d = runs[r];
        const uint32_t N = d.L * d.L, s = got[r];
        const Ranges &g = gs[r];
        std::vector<unsigned long long> thr(2 * d.n_beta);
        for (uint32_t i = 0; i < d.n_beta; ++i) {
            thr[2 * i] = threshold(d.beta[i], 1);
            thr[2 * i + 1] = threshold(d.beta[i], 2);
        }
        RunDev x;
        std::memset(&x, 0, sizeof x);
        x.L = d.L;
        x.N = N;
        x.Lh = d.L / 2;
        x.wstride = stride_words(d.L);
        x.model = d.model;
        x.R = d.R;
        x.R_cap = cap_of(d);
        x.theta = d.theta;
        x.n_beta = d.n_beta;
        x.seed = d.seed;
        x.run_id = d.run_id;
        x.disorder_id = d.disorder_id;
        x.resample = d.resample;
        x.overlap = d.overlap;
        x.paired = (d.overlap & PA_Q_PAIR) ? (int32_t)got[d.paired] : -1;
        x.pitch = row_pitch(d.L);
        x.pw = plane_words(d.L);
        x.rep_off = g.rep;
        x.spin_off = g.spin;
        x.rec_off = g.rec;
        x.qh_off = g.qh;
        x.beta_off = g.beta;
        x.wt_off = g.wto;
        x.thr_off = g.thr;
        x.J_off = g.J;
        x.scr_off = g.scr;
        x.ln2N = (double)N * std::log(2.0);
        x.dos_off = dos_offs[r];
        e->rd[s] = x;
        RunState rs;
        rs.step = 0;
        rs.R_cur = d.R;
        rs.R_new = d.R;
        rs.status = 0;
        rs.lnQ = 0.0;
        rs.ticket = 0;
        rs.Emin = 0;
        rs.n_levels = 0;
        rs.pad = 0;
        const uint64_t nq = sizes_of(d).qh;
        cudaError_t err = cudaMemcpyAsync(e->d_runs + s, &e->rd[s], sizeof(RunDev), cudaMemcpyHostToDevice, e->stream);
        if (!err) err = cudaMemcpyAsync(e->P.st + s, &rs, sizeof rs, cudaMemcpyHostToDevice, e->stream);
        if (!err)
            err = cudaMemcpyAsync(e->d_beta + g.beta, d.beta, sizeof(double) * d.n_beta, cudaMemcpyHostToDevice,
                                  e->stream);
        if (!err)
            err = cudaMemcpyAsync(e->d_thr + g.thr, thr.data(), sizeof(unsigned long long) * thr.size(),
                                  cudaMemcpyHostToDevice, e->stream);
        if (!err)
            err = cudaMemcpyAsync(e->d_wtoff + g.wto, wtos[r].data(), sizeof(unsigned long long) * d.n_beta,
                                  cudaMemcpyHostToDevice, e->stream);
        if (!err) err = cudaMemsetAsync(e->P.rec + g.rec, 0, sizeof(pa_step_record) * d.n_beta, e->stream);
        if (!err && nq) err = cudaMemsetAsync(e->P.qh + g.qh, 0, sizeof(uint32_t) * nq, e->stream);
        if (!err && nq) err = cudaMemsetAsync(e->P.qhp + g.qh, 0, sizeof(uint32_t) * nq, e->stream);
        if (!err && nq) err = cudaMemsetAsync(e->P.qhw + g.qh, 0, sizeof(uint32_t) * nq, e->stream);
        // the measurement's histograms start (and every step leaves them) cleared
        if (!err) err = cudaMemsetAsync(e->P.scratch + g.scr, 0, 8 * scr_table_off(N), e->stream);
        if (!err) err = cudaStreamSynchronize(e->stream);  // host buffers must outlive the copies
        if (err) return cuda_fail(err, "admit upload");
        e->h2d += sizeof(RunDev) + sizeof rs + sizeof(double) * d.n_beta +
                  sizeof(unsigned long long) * (thr.size() + d.n_beta);
        RunHost &h = e->rh[s];
        h.used = true;
        h.d = d;
        h.dos_hash = dos_hash_of(d);
        h.d.beta = nullptr;  // not kept: the caller owns it
        h.d.log_g = nullptr;
        h.g = g;
        h.steps_done = 0;
        e->active.push_back(s);
        e->pending.push_back(s);
        if (slots) slots[r] = s;
        e->max_pw = std::max(e->max_pw, plane_words(d.L));
    }
    e->dirty = true;
    return PA_OK;
}

// Rebuild the device lists (resident runs, overlap runs, per-size work lists,
// the pending-draw list) after the resident set changed.
pa_status rebuild(pa_engine *e)
{
    PA_CUDA(cudaStreamSynchronize(e->stream));  // nothing in flight reads d_meta
    std::vector<uint32_t> &m = e->h_meta;
    m.clear();
    e->active_off = m.size();
    m.insert(m.end(), e->active.begin(), e->active.end());
    // small runs (one launch per step) and the others
    e->small.clear();
    e->big.clear();
    const bool fuse = !(e->flags & (PA_CREATE_SEPARATE_KERNELS | PA_CREATE_GENERIC_SWEEP));
    for (uint32_t s : e->active) {
        const RunDev &x = e->rd[s];
        if (!fuse || !small_eligible(x)) {
            e->big.push_back(s);
            continue;
        }
        size_t k = 0;
        while (k < e->small.size() && e->small[k].L != x.L) ++k;
        if (k == e->small.size()) {
            e->small.emplace_back();
            e->small[k].L = x.L;
        }
        e->small[k].runs.push_back(s);
        if (x.model == PA_EA_PMJ) e->small[k].any_glass = 1;
        e->small[k].R_max = std::max(e->small[k].R_max, x.R);
        e->small[k].R_cap_max = std::max(e->small[k].R_cap_max, x.R_cap);
        e->small[k].theta_max = std::max(e->small[k].theta_max, x.theta);
    }
    // Each lattice size is its own launch, with the GPU to itself.  A size for which
    // neither launch shape keeps every run's cluster on SMs of its own (many runs, or
    // populations that need several tiles per CTA) goes to the per-stage kernels,
    // which batch all its runs per launch: 20 runs of L = 32 at R = 300 (2000) ran at
    // 413 (555) updates/ns on the one-launch path against 691 (1368) per stage.
    for (size_t k = 0; k < e->small.size();) {
        SmallGroup &g = e->small[k];
        g.shape = small_shape(g.L, g.any_glass, (uint32_t)g.runs.size(), g.R_max, g.R_cap_max);
        g.ahead = small_shape_ahead(g.L, g.any_glass, (uint32_t)g.runs.size(), g.R_max, g.theta_max);
        if (g.shape.variant == 0 && g.ahead.cs == 0) {
            e->big.insert(e->big.end(), g.runs.begin(), g.runs.end());
            e->small.erase(e->small.begin() + k);
            continue;
        }
        g.runs_off = m.size();
        m.insert(m.end(), g.runs.begin(), g.runs.end());
        ++k;
    }
    e->big_off = m.size();
    m.insert(m.end(), e->big.begin(), e->big.end());
    e->q_runs.clear();
    e->max_Rcap_active = 0;
    for (uint32_t s : e->active) {
        if (e->rd[s].overlap) e->q_runs.push_back(s);  // small runs have none
        e->max_Rcap_active = std::max(e->max_Rcap_active, e->rd[s].R_cap);
    }
    e->q_off = m.size();
    m.insert(m.end(), e->q_runs.begin(), e->q_runs.end());
    e->near_runs.clear();
    e->multi_runs.clear();
    e->near_maxcap = e->multi_maxcap = 0;
    for (uint32_t s : e->big) {
        const bool multi = e->rd[s].resample == PA_MULTINOMIAL;
        (multi ? e->multi_runs : e->near_runs).push_back(s);
        uint32_t &cap = multi ? e->multi_maxcap : e->near_maxcap;
        cap = std::max(cap, e->rd[s].R_cap);
    }
    e->near_off = m.size();
    m.insert(m.end(), e->near_runs.begin(), e->near_runs.end());
    e->multi_off = m.size();
    m.insert(m.end(), e->multi_runs.begin(), e->multi_runs.end());
    e->wang_runs.clear();
    e->wang_maxcap = 0;
    for (uint32_t s : e->active)
        if (e->rd[s].overlap & PA_Q_WANG) {
            e->wang_runs.push_back(s);
            e->wang_maxcap = std::max(e->wang_maxcap, e->rd[s].R_cap);
        }
    e->wang_off = m.size();
    m.insert(m.end(), e->wang_runs.begin(), e->wang_runs.end());
    e->groups.clear();
    std::map<uint32_t, size_t> gi;  // lattice size -> group, in order of first appearance
    e->inf_runs.clear();
    e->inf_maxR = 0;
    for (uint32_t s : e->big) {
        if (e->rd[s].theta == PA_THETA_INF) {  // sampled from the density of states, no sweep
            e->inf_runs.push_back(s);
            e->inf_maxR = std::max(e->inf_maxR, e->rd[s].R_cap);
            continue;
        }
        const uint32_t L = e->rd[s].L;
        auto it = gi.find(L);
        if (it == gi.end()) {
            it = gi.emplace(L, e->groups.size()).first;
            SweepGroup g;
            g.L = L;
            e->groups.push_back(g);
            if (!e->tuning.count(L)) {
                Tuning t;
                t.candidates = sweep_candidates(L, (e->flags & PA_CREATE_GENERIC_SWEEP) ? 0 : 1);
                t.tuned = t.candidates.size() < 2 || (e->flags & PA_CREATE_NO_AUTOTUNE);
                if (!t.tuned) {
                    std::lock_guard<std::mutex> lock(g_tune_mu);
                    auto c = g_tuned.find(tune_key(L, e->flags));
                    if (c != g_tuned.end() && c->second < t.candidates.size()) {
                        t.pick = c->second;
                        t.tuned = true;
                    }
                }
                e->tuning[L] = t;
            }
        }
        SweepGroup &g = e->groups[it->second];
        g.runs.push_back(s);
        if (e->rd[s].model == PA_EA_PMJ) g.any_glass = 1;
    }
    for (auto &g : e->groups) {
        const Tuning &t = e->tuning[g.L];
        g.runs_off = m.size();
        m.insert(m.end(), g.runs.begin(), g.runs.end());
        for (const SweepCfg &c : t.candidates) {
            g.tile_map_off.push_back(m.size());
            uint64_t acc = 0;
            m.push_back(0u);
            for (uint32_t s : g.runs) {
                acc += (e->rd[s].R_cap + c.RPC - 1) / c.RPC;
                if (acc > 0x7fffffffull) return PA_ERR_INVALID_ARG;  // beyond one launch's grid
                m.push_back((uint32_t)acc);
            }
            g.n_tiles.push_back((uint32_t)acc);
        }
    }
    e->inf_off = m.size();
    m.insert(m.end(), e->inf_runs.begin(), e->inf_runs.end());
    e->init_runs_off = m.size();
    m.insert(m.end(), e->pending.begin(), e->pending.end());
    e->init_tiles_off = m.size();
    uint64_t acc = 0;
    m.push_back(0u);
    for (uint32_t s : e->pending) {  // 4 replicas per CTA; none for theta = PA_THETA_INF runs
        acc += e->rd[s].theta == PA_THETA_INF ? 0u : (e->rd[s].R + 3) / 4;
        if (acc > 0x7fffffffull) return PA_ERR_INVALID_ARG;
        m.push_back((uint32_t)acc);
    }
    e->init_n = (uint32_t)e->pending.size();
    e->init_tiles = (uint32_t)acc;
    e->init_inf_off = m.size();
    e->init_inf_n = 0;
    e->init_inf_maxR = 0;
    for (uint32_t s : e->pending)
        if (e->rd[s].theta == PA_THETA_INF) {
            m.push_back(s);
            ++e->init_inf_n;
            // the beta_0 draw also clears the planes of all R_cap slots
            e->init_inf_maxR = std::max(e->init_inf_maxR, e->rd[s].R_cap);
        }
    e->init_wang_off = m.size();
    e->init_wang_n = 0;
    e->init_wang_maxcap = 0;
    for (uint32_t s : e->pending)
        if (e->rd[s].overlap & PA_Q_WANG) {
            m.push_back(s);
            ++e->init_wang_n;
            e->init_wang_maxcap = std::max(e->init_wang_maxcap, e->rd[s].R_cap);
        }
    e->init_q_off = m.size();  // pending runs with overlaps: their step-0 overlaps only
    e->init_q_n = 0;
    for (uint32_t s : e->pending)
        if (e->rd[s].overlap) {
            m.push_back(s);
            ++e->init_q_n;
        }
    if (m.size() > e->meta_cap) return PA_ERR_INVALID_ARG;
    PA_CUDA(cudaMemcpyAsync(e->d_meta, m.data(), sizeof(uint32_t) * m.size(), cudaMemcpyHostToDevice, e->stream));
    PA_CUDA(cudaStreamSynchronize(e->stream));
    e->h2d += sizeof(uint32_t) * m.size();
    e->dirty = false;
    if (e->graph_exec) {
        cudaGraphExecDestroy(e->graph_exec);
        e->graph_exec = nullptr;
    }
    if (e->graph) {
        cudaGraphDestroy(e->graph);
        e->graph = nullptr;
    }
    return PA_OK;
}

cudaEvent_t take_event(pa_engine *e)
{
    if (!e->ev_free.empty()) {
        cudaEvent_t ev = e->ev_free.back();
        e->ev_free.pop_back();
        return ev;
    }
    cudaEvent_t ev = nullptr;
    cudaEventCreate(&ev);
    return ev;
}

// Run `launch` (one kernel on e->stream), bracketed by events in profiling mode.
template <typename F>
void timed_launch(pa_engine *e, int kind, F &&launch)
{
    e->launches += 1;
    if (!e->profiling) {
        launch();
        return;
    }
    pa_engine::Timed t{kind, take_event(e), take_event(e)};
    cudaEventRecord(t.a, e->stream);
    launch();
    cudaEventRecord(t.b, e->stream);
    e->timed.push_back(t);
}

const uint32_t *meta(pa_engine *e, uint64_t off) { return e->d_meta + off; }

void launch_group_sweep(pa_engine *e, const SweepGroup &g, uint32_t c)
{
    const Tuning &t = e->tuning[g.L];
    launch_sweep(e->P, meta(e, g.runs_off), meta(e, g.tile_map_off[c]), (uint32_t)g.runs.size(), g.n_tiles[c],
                 t.candidates[c], g.any_glass, e->stream);
}

// beta_0 draws of the pending runs (Sec. II.B step (i)) and their step-0 measurement.
pa_status enqueue_pending(pa_engine *e)
{
    if (e->pending.empty()) return PA_OK;
    const uint32_t *runs = meta(e, e->init_runs_off);
    timed_launch(e, PA_K_INIT, [&] { launch_init_couplings(e->P, runs, e->init_n, e->stream); });
    if (e->init_tiles)
        timed_launch(e, PA_K_INIT, [&] {
            launch_init_population(e->P, meta(e, e->init_tiles_off), runs, e->init_n, e->init_tiles, e->max_pw,
                                   e->stream);
        });
    if (e->init_inf_n)
        timed_launch(e, PA_K_INIT, [&] {
            launch_dos_sample(e->P, meta(e, e->init_inf_off), e->init_inf_n, e->init_inf_maxR, 1, e->stream);
        });
    if (e->init_q_n)  // step-0 overlaps of the pending runs (pairs are admitted together)
        timed_launch(e, PA_K_OVERLAP, [&] {
            launch_overlap(e->P, meta(e, e->init_q_off), e->init_q_n, e->max_Rcap_active, 1, e->stream);
        });
    if (e->init_wang_n)
        timed_launch(e, PA_K_OVERLAP, [&] {
            launch_wang(e->P, meta(e, e->init_wang_off), e->init_wang_n, e->init_wang_maxcap, 1, e->stream);
        });
    timed_launch(e, PA_K_MEASURE,
                 [&] { launch_measure(e->P, runs, e->init_n, e->max_Rcap_active, 1, e->stream); });
    e->pending.clear();
    e->dirty = true;  // the pending list is consumed
    PA_CUDA(cudaGetLastError());
    return PA_OK;
}

// Wang pairings of the runs that measure them (after the sweeps, like the overlaps).
void enqueue_wang(pa_engine *e)
{
    if (e->wang_runs.empty()) return;
    timed_launch(e, PA_K_OVERLAP, [&] {
        launch_wang(e->P, meta(e, e->wang_off), (uint32_t)e->wang_runs.size(), e->wang_maxcap, 0, e->stream);
    });
}

// Resampling of every resident run: the nearest-integer runs split over
// several CTAs each (two launches; one when every population fits one CTA),
// the multinomial runs one CTA each.
void enqueue_resample(pa_engine *e)
{
    if (!e->near_runs.empty()) {
        timed_launch(e, PA_K_RESAMPLE, [&] {
            launch_resample_nearest(e->P, meta(e, e->near_off), (uint32_t)e->near_runs.size(), e->near_maxcap,
                                    e->stream);
        });
        e->launches += resample_nearest_launches(e->near_maxcap) - 1;
    }
    if (!e->multi_runs.empty())
        timed_launch(e, PA_K_RESAMPLE, [&] {
            launch_resample_multinomial(e->P, meta(e, e->multi_off), (uint32_t)e->multi_runs.size(),
                                        e->multi_maxcap, e->stream);
        });
}

// Fresh energies for the theta = PA_THETA_INF runs (in place of their sweeps).
void enqueue_dos_sample(pa_engine *e)
{
    if (e->inf_runs.empty()) return;
    timed_launch(e, PA_K_SWEEP, [&] {
        launch_dos_sample(e->P, meta(e, e->inf_off), (uint32_t)e->inf_runs.size(), e->inf_maxR, 0, e->stream);
    });
}

// n_steps temperatures of every small run, one launch per lattice size.
void enqueue_small(pa_engine *e, uint32_t n_steps)
{
    for (auto &g : e->small)
        timed_launch(e, PA_K_SMALL, [&] {
            launch_anneal_small(e->P, meta(e, g.runs_off), (uint32_t)g.runs.size(), g.L,
                                n_steps > 1 && g.ahead.cs ? g.ahead : g.shape, g.any_glass,
                                n_steps, e->stream);
        });
}

void enqueue_tick(pa_engine *e)
{
    enqueue_small(e, 1);
    if (e->big.empty()) return;
    const uint32_t *act = meta(e, e->big_off);
    const uint32_t na = (uint32_t)e->big.size();
    enqueue_resample(e);
    for (auto &g : e->groups) timed_launch(e, PA_K_SWEEP, [&] { launch_group_sweep(e, g, e->tuning[g.L].pick); });
    enqueue_dos_sample(e);
    if (!e->q_runs.empty())
        timed_launch(e, PA_K_OVERLAP, [&] {
            launch_overlap(e->P, meta(e, e->q_off), (uint32_t)e->q_runs.size(), e->max_Rcap_active, 0, e->stream);
        });
    enqueue_wang(e);
    timed_launch(e, PA_K_MEASURE, [&] { launch_measure(e->P, act, na, e->max_Rcap_active, 0, e->stream); });
}

// One eager step of tuning.  A lattice size whose sweep shape is not chosen yet
// runs this step's real sweep with one of its candidate shapes, in rotation, timed
// with events: the first tuning step only warms up, then every candidate sweeps
// two steps, and its faster step counts.  Candidates read the same parents and
// write identical children, so any of them may do a step's work; timing them on
// the anneal's own steps measures the steady state without extra launches (one
// extra launch per candidate on the first step, timed back to back, favoured the
// shapes that were fastest on the freshly drawn population, not later on).
pa_status enqueue_tuning_tick(pa_engine *e)
{
    enqueue_small(e, 1);
    const uint32_t *act = meta(e, e->big_off);
    const uint32_t na = (uint32_t)e->big.size();
    enqueue_resample(e);
    struct Timing {
        SweepGroup *g;
        uint32_t c;
        cudaEvent_t a, b;
    };
    std::vector<Timing> timing;
    for (auto &g : e->groups) {
        Tuning &t = e->tuning[g.L];
        if (t.tuned) {
            timed_launch(e, PA_K_SWEEP, [&] { launch_group_sweep(e, g, t.pick); });
            continue;
        }
        bool live = false;  // a run of this size still has a temperature to go
        for (uint32_t r : g.runs) live |= e->rh[r].steps_done + 1 < e->rh[r].d.n_beta;
        if (!live) {
            timed_launch(e, PA_K_SWEEP, [&] { launch_group_sweep(e, g, t.pick); });
            continue;
        }
        const uint32_t nc = (uint32_t)t.candidates.size();
        const uint32_t c = t.round == 0 ? 0u : (t.round - 1) % nc;
        Timing x{&g, c, nullptr, nullptr};
        PA_CUDA(cudaEventCreate(&x.a));
        PA_CUDA(cudaEventCreate(&x.b));
        PA_CUDA(cudaEventRecord(x.a, e->stream));
        launch_group_sweep(e, g, c);
        PA_CUDA(cudaEventRecord(x.b, e->stream));
        e->launches += 1;
        timing.push_back(x);
    }
    enqueue_dos_sample(e);
    if (!e->q_runs.empty())
        timed_launch(e, PA_K_OVERLAP, [&] {
            launch_overlap(e->P, meta(e, e->q_off), (uint32_t)e->q_runs.size(), e->max_Rcap_active, 0, e->stream);
        });
    enqueue_wang(e);
    if (na) timed_launch(e, PA_K_MEASURE, [&] { launch_measure(e->P, act, na, e->max_Rcap_active, 0, e->stream); });
    PA_CUDA(cudaGetLastError());
    if (timing.empty()) return PA_OK;
    PA_CUDA(cudaStreamSynchronize(e->stream));
    for (auto &x : timing) {
        Tuning &t = e->tuning[x.g->L];
        const uint32_t nc = (uint32_t)t.candidates.size();
        float ms = 0.f;
        PA_CUDA(cudaEventElapsedTime(&ms, x.a, x.b));
        cudaEventDestroy(x.a);
        cudaEventDestroy(x.b);
        if (t.best.size() != nc) t.best.assign(nc, 0.f);
        if (t.round > 0 && (t.best[x.c] == 0.f || ms < t.best[x.c])) t.best[x.c] = ms;
        t.round += 1;
        if (t.round == 1 + 2 * nc) {  // every candidate timed on two steps
            t.pick = 0;
            for (uint32_t c = 1; c < nc; ++c)
                if (t.best[c] < t.best[t.pick]) t.pick = c;
            t.tuned = true;
            t.ms = t.best[t.pick];
            std::lock_guard<std::mutex> lock(g_tune_mu);
            g_tuned[tune_key(x.g->L, e->flags)] = t.pick;
        }
    }
    return PA_OK;
}

// Bring the device lists up to date and draw pending populations.
pa_status prepare(pa_engine *e)
{
    if (e->dirty) PA_TRY(rebuild(e));
    if (!e->pending.empty()) {
        PA_TRY(enqueue_pending(e));
        PA_TRY(rebuild(e));  // drop the consumed pending list
    }
    return PA_OK;
}

void advance_host_steps(pa_engine *e, uint32_t n)
{
    for (uint32_t s : e->active) {
        RunHost &h = e->rh[s];
        const uint32_t last = h.d.n_beta - 1;
        h.steps_done = std::min<uint32_t>(last, h.steps_done + n);
    }
}

// Synchronise for a read: CUDA errors only (a run that stopped is readable).
pa_status sync_read(pa_engine *e)
{
    PA_CUDA(cudaStreamSynchronize(e->stream));
    PA_CUDA(cudaGetLastError());
    return PA_OK;
}

pa_status latch_device_status(pa_engine *e)
{
    uint32_t word = 0;
    PA_CUDA(cudaMemcpyAsync(&word, e->P.status, sizeof word, cudaMemcpyDeviceToHost, e->stream));
    PA_CUDA(cudaStreamSynchronize(e->stream));
    if (e->latched == PA_OK && word) {
        for (uint32_t c = 1; c < 32; ++c)
            if (word & (1u << c)) {
                e->latched = (pa_status)c;
                break;
            }
    }
    return e->latched;
}

pa_status engine_new(void *cuda_stream, uint32_t flags, pa_engine **out)
{
    if (flags & ~(uint32_t)(PA_CREATE_GENERIC_SWEEP | PA_CREATE_NO_AUTOTUNE | PA_CREATE_SEPARATE_KERNELS))
        return PA_ERR_INVALID_ARG;
    PA_CUDA(prepare_kernels());
    pa_engine *e = new (std::nothrow) pa_engine();
    if (!e) return PA_ERR_OOM;
    e->flags = flags;
    e->alloc = current_allocator();
    if (cuda_stream) {
        e->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        cudaError_t err = cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking);
        if (err != cudaSuccess) {
            delete e;
            return cuda_fail(err, "cudaStreamCreate");
        }
        e->own_stream = true;
    }
    *out = e;
    return PA_OK;
}

bool slot_ok(const pa_engine *e, uint32_t s) { return e && s < e->S && e->rh[s].used; }

// Checkpoint of one run: a fixed header, the run state, the schedule, then the
// device sections below in this order.
constexpr char CKPT_MAGIC[8] = {'P', 'A', 'C', 'K', 'P', 'T', '0', '1'};
struct CkptHeader {
    char magic[8];
    uint32_t L, model, R, R_cap, theta, n_beta, seed, run_id, disorder_id, resample, overlap;
    uint32_t steps_done, R_cur, buffer, wstride, pad;
    uint64_t scratch_words, J_words, total_bytes;
    uint64_t dos_hash;  // theta = PA_THETA_INF: hash of the run's ln g (0 otherwise)
};

struct CkptSection {
    void *dev;      // device address
    size_t bytes;
};

// The run's device sections, given its state (population of buffer st.step & 1).
std::vector<CkptSection> ckpt_sections(pa_engine *e, uint32_t run, const RunState &st)
{
    const RunDev &x = e->rd[run];
    const uint32_t b = st.step & 1u;
    const uint64_t nq = (uint64_t)x.n_beta * (x.N + 1);
    std::vector<CkptSection> v = {
        {e->P.spins[b] + x.spin_off, sizeof(uint32_t) * (size_t)st.R_cur * x.wstride},
        {e->P.E[b] + x.rep_off, sizeof(int32_t) * (size_t)st.R_cur},
        {e->P.M[b] + x.rep_off, sizeof(int32_t) * (size_t)st.R_cur},
        {e->P.fam[b] + x.rep_off, sizeof(uint32_t) * (size_t)st.R_cur},
        {e->P.rec + x.rec_off, sizeof(pa_step_record) * (size_t)x.n_beta},
        {e->P.scratch + x.scr_off, sizeof(unsigned long long) * (size_t)scratch_words(x.N, x.R_cap)},
        {e->P.J + x.J_off, sizeof(uint32_t) * (size_t)sizes_of(e->rh[run].d).J},
    };
    if (x.overlap) {
        v.push_back({e->P.qh + x.qh_off, sizeof(uint32_t) * (size_t)nq});
        v.push_back({e->P.qhp + x.qh_off, sizeof(uint32_t) * (size_t)nq});
        v.push_back({e->P.qhw + x.qh_off, sizeof(uint32_t) * (size_t)nq});
    }
    return v;
}

size_t ckpt_bytes(const RunDev &x, const std::vector<CkptSection> &v)
{
    size_t n = sizeof(CkptHeader) + sizeof(RunState) + sizeof(double) * x.n_beta;
    for (const auto &c : v) n += c.bytes;
    return n;
}

// Pools sized exactly for these (validated) runs: each run's ranges, and weight
// tables for their distinct (N, dbeta) plus the theta = infinity CDF tables of
// their distinct (density of states, schedule).
void pool_sizes(const pa_run_desc *runs, uint32_t n_runs, pa_server_config &c)
{
    c = pa_server_config{};
    c.max_runs = n_runs;
    std::map<std::pair<uint32_t, uint64_t>, int> keys;
    std::map<std::vector<double>, int> dos_keys;
    for (uint32_t r = 0; r < n_runs; ++r) {
        const Ranges z = sizes_of(runs[r]);
        c.replica_capacity += z.rep;
        c.spin_words += z.spin;
        c.record_capacity += z.rec;
        c.qhist_words += z.qh;
        c.scratch_words += z.scr;
        c.coupling_words += z.J;
        const uint32_t N = runs[r].L * runs[r].L;
        for (uint32_t i = 1; i < runs[r].n_beta; ++i) {
            const double db = runs[r].beta[i] - runs[r].beta[i - 1];
            uint64_t bits;
            std::memcpy(&bits, &db, sizeof bits);
            if (keys.emplace(std::make_pair(N, bits), 0).second) c.table_doubles += N + 1;
        }
        if (runs[r].theta == PA_THETA_INF) {
            std::vector<double> key(runs[r].log_g, runs[r].log_g + 2 * N + 1);
            key.insert(key.end(), runs[r].beta, runs[r].beta + runs[r].n_beta);
            key.push_back((double)N);
            if (dos_keys.emplace(std::move(key), 0).second) c.table_doubles += (uint64_t)runs[r].n_beta * (2 * N + 2);
        }
    }
}

}  // namespace

extern "C" {

const char *pa_status_string(pa_status s)
{
    switch (s) {
    case PA_OK: return "ok";
    case PA_ERR_INVALID_ARG: return "invalid argument";
    case PA_ERR_OOM: return "out of memory";
    case PA_ERR_CAPACITY: return "population exceeded its capacity R_cap";
    case PA_ERR_EXTINCT: return "population became empty";
    case PA_ERR_CUDA: return "CUDA error";
    case PA_ERR_TIMEOUT: return "device wait timed out";
    case PA_ERR_STATE: return "invalid state";
    case PA_ERR_BUSY: return "no room to admit the run";
    }
    return "unknown status";
}

pa_status pa_destroy(pa_engine *e)
{
    if (!e) return PA_ERR_INVALID_ARG;
    if (e->stream) cudaStreamSynchronize(e->stream);
    if (e->graph_exec) cudaGraphExecDestroy(e->graph_exec);
    if (e->graph) cudaGraphDestroy(e->graph);
    for (auto &b : e->allocs) device_free(e->alloc, b.first, b.second, e->stream);
    device_free(e->alloc, e->wa_buf, e->wa_bytes, e->stream);
    device_free(e->alloc, e->sr_buf, e->sr_bytes, e->stream);
    for (auto &t : e->timed) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    for (auto ev : e->ev_free) cudaEventDestroy(ev);
    if (e->own_stream && e->stream) cudaStreamDestroy(e->stream);
    delete e;
    return PA_OK;
}

pa_status pa_create(const pa_run_desc *runs, uint32_t n_runs, void *cuda_stream, pa_engine **out)
{
    return pa_create_ex(runs, n_runs, cuda_stream, 0u, out);
}

pa_status pa_pool_sizes(const pa_run_desc *runs, uint32_t n_runs, pa_server_config *out)
{
    if (!out) return PA_ERR_INVALID_ARG;
    PA_TRY(validate(runs, n_runs));
    pool_sizes(runs, n_runs, *out);
    return PA_OK;
}

pa_status pa_create_ex(const pa_run_desc *runs, uint32_t n_runs, void *cuda_stream, uint32_t flags, pa_engine **out)
{
    if (!out) return PA_ERR_INVALID_ARG;
    *out = nullptr;
    PA_TRY(validate(runs, n_runs));
    pa_server_config c;
    pool_sizes(runs, n_runs, c);
    pa_engine *e = nullptr;
    PA_TRY(engine_new(cuda_stream, flags, &e));
    pa_status s = alloc_pools(e, c);
    if (s == PA_OK) s = admit(e, runs, n_runs, nullptr);
    if (s == PA_OK) s = prepare(e);
    if (s != PA_OK) {
        pa_destroy(e);
        return s;
    }
    *out = e;
    return PA_OK;
}

pa_status pa_server_create(const pa_server_config *cfg, void *cuda_stream, uint32_t flags, pa_engine **out)
{
    if (!out || !cfg || cfg->max_runs == 0 || cfg->max_runs > (1u << 20)) return PA_ERR_INVALID_ARG;
    *out = nullptr;
    pa_engine *e = nullptr;
    PA_TRY(engine_new(cuda_stream, flags, &e));
    e->server = true;
    pa_status s = alloc_pools(e, *cfg);
    if (s != PA_OK) {
        pa_destroy(e);
        return s;
    }
    *out = e;
    return PA_OK;
}

pa_status pa_admit(pa_engine *e, const pa_run_desc *runs, uint32_t n_runs, uint32_t *slots_out)
{
    if (!e || !slots_out) return PA_ERR_INVALID_ARG;
    if (e->latched != PA_OK) return e->latched;
    return admit(e, runs, n_runs, slots_out);
}

pa_status pa_retire(pa_engine *e, uint32_t slot)
{
    if (!slot_ok(e, slot)) return PA_ERR_INVALID_ARG;
    PA_CUDA(cudaStreamSynchronize(e->stream));  // no queued work may still use its ranges
    const int32_t partner = e->rd[slot].paired;
    if (partner >= 0 && slot_ok(e, (uint32_t)partner) && e->rd[(uint32_t)partner].paired == (int32_t)slot) {
        // the partner keeps running without two-population overlaps
        RunDev &p = e->rd[(uint32_t)partner];
        p.paired = -1;
        p.overlap &= ~(uint32_t)PA_Q_PAIR;
        PA_CUDA(cudaMemcpyAsync(e->d_runs + partner, &p, sizeof(RunDev), cudaMemcpyHostToDevice, e->stream));
        PA_CUDA(cudaStreamSynchronize(e->stream));
    }
    unreserve(e, e->rh[slot].d, e->rh[slot].g);
    e->rh[slot] = RunHost{};
    e->active.erase(std::remove(e->active.begin(), e->active.end(), slot), e->active.end());
    e->pending.erase(std::remove(e->pending.begin(), e->pending.end(), slot), e->pending.end());
    e->dirty = true;
    return PA_OK;
}

pa_status pa_run_state(pa_engine *e, uint32_t slot, uint32_t *step, uint32_t *R, uint32_t *status)
{
    if (!slot_ok(e, slot)) return PA_ERR_INVALID_ARG;
    PA_TRY(prepare(e));
    RunState st;
    PA_CUDA(cudaMemcpyAsync(&st, e->P.st + slot, sizeof st, cudaMemcpyDeviceToHost, e->stream));
    PA_CUDA(cudaStreamSynchronize(e->stream));
    if (step) *step = st.step;
    if (R) *R = st.R_cur;
    if (status) *status = st.status;
    return PA_OK;
}

pa_status pa_finished(const pa_engine *e, uint32_t *slots_out, uint32_t cap, uint32_t *n_out)
{
    if (!e || !n_out) return PA_ERR_INVALID_ARG;
    uint32_t n = 0;
    for (uint32_t s : e->active) {
        const RunHost &h = e->rh[s];
        if (h.steps_done + 1 >= h.d.n_beta) {
            if (slots_out && n < cap) slots_out[n] = s;
            ++n;
        }
    }
    *n_out = n;
    return PA_OK;
}

pa_status pa_reset(pa_engine *e)
{
    if (!e) return PA_ERR_INVALID_ARG;
    PA_CUDA(cudaStreamSynchronize(e->stream));
    std::vector<RunState> st(e->active.size());
    for (size_t k = 0; k < e->active.size(); ++k) {
        const uint32_t s = e->active[k];
        const RunDev &x = e->rd[s];
        st[k].step = 0;
        st[k].R_cur = x.R;
        st[k].R_new = x.R;
        st[k].status = 0;
        st[k].lnQ = 0.0;
        st[k].ticket = 0;
        st[k].Emin = 0;
        st[k].n_levels = 0;
        st[k].pad = 0;
        PA_CUDA(cudaMemcpyAsync(e->P.st + s, &st[k], sizeof(RunState), cudaMemcpyHostToDevice, e->stream));
        PA_CUDA(cudaMemsetAsync(e->P.rec + x.rec_off, 0, sizeof(pa_step_record) * x.n_beta, e->stream));
        PA_CUDA(cudaMemsetAsync(e->P.scratch + x.scr_off, 0, 8 * scr_table_off(x.N), e->stream));
        if (x.overlap) {
            const uint64_t nq = (uint64_t)x.n_beta * (x.N + 1);
            PA_CUDA(cudaMemsetAsync(e->P.qh + x.qh_off, 0, sizeof(uint32_t) * nq, e->stream));
            PA_CUDA(cudaMemsetAsync(e->P.qhp + x.qh_off, 0, sizeof(uint32_t) * nq, e->stream));
            PA_CUDA(cudaMemsetAsync(e->P.qhw + x.qh_off, 0, sizeof(uint32_t) * nq, e->stream));
        }
        e->rh[s].steps_done = 0;
        if (std::find(e->pending.begin(), e->pending.end(), s) == e->pending.end()) e->pending.push_back(s);
    }
    PA_CUDA(cudaMemsetAsync(e->P.status, 0, sizeof(uint32_t), e->stream));
    PA_CUDA(cudaStreamSynchronize(e->stream));  // st must outlive the copies
    e->latched = PA_OK;
    e->h2d += sizeof(RunState) * e->active.size();
    e->dirty = true;
    return prepare(e);
}

pa_status pa_anneal_step(pa_engine *e, uint32_t n_steps, int use_graph)
{
    if (!e) return PA_ERR_INVALID_ARG;
    if (e->latched != PA_OK) return e->latched;
    PA_TRY(prepare(e));
    uint32_t left = 0;  // temperatures any resident run still has to go
    for (uint32_t s : e->active) left = std::max(left, e->rh[s].d.n_beta - 1 - e->rh[s].steps_done);
    n_steps = std::min(n_steps, left);
    if (n_steps == 0 || e->active.empty()) return PA_OK;
    for (;;) {  // eager tuning steps while a lattice size's sweep shape is not chosen yet
        bool untuned = false;
        for (auto &g : e->groups) untuned |= !e->tuning[g.L].tuned;
        if (!untuned) break;
        PA_TRY(enqueue_tuning_tick(e));
        advance_host_steps(e, 1);
        if (--n_steps == 0) return PA_OK;
    }
    if (e->big.empty()) {  // every run on the small path: n temperatures in one launch per lattice size
        enqueue_small(e, n_steps);
        PA_CUDA(cudaGetLastError());
        advance_host_steps(e, n_steps);
        return PA_OK;
    }
    if (use_graph && !e->profiling) {
        if (!e->graph_exec) {
            const uint64_t l0 = e->launches;
            PA_CUDA(cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal));
            enqueue_tick(e);
            PA_CUDA(cudaStreamEndCapture(e->stream, &e->graph));
            PA_CUDA(cudaGraphInstantiate(&e->graph_exec, e->graph, 0));
            e->graph_tick_launches = e->launches - l0;  // the kernels one replay launches
            e->launches = l0;                            // capturing launched nothing
        }
        for (uint32_t k = 0; k < n_steps; ++k) PA_CUDA(cudaGraphLaunch(e->graph_exec, e->stream));
        e->launches += e->graph_tick_launches * n_steps;
    } else {
        for (uint32_t k = 0; k < n_steps; ++k) enqueue_tick(e);
        PA_CUDA(cudaGetLastError());
    }
    advance_host_steps(e, n_steps);
    return PA_OK;
}

pa_status pa_sync(pa_engine *e)
{
    if (!e) return PA_ERR_INVALID_ARG;
    PA_TRY(prepare(e));
    PA_CUDA(cudaStreamSynchronize(e->stream));
    PA_CUDA(cudaGetLastError());
    return latch_device_status(e);
}

uint64_t pa_launch_count(const pa_engine *e) { return e ? e->launches : 0; }

pa_status pa_tuning_pending(const pa_engine *e, uint32_t *n)
{
    if (!e || !n) return PA_ERR_INVALID_ARG;
    uint32_t k = 0;
    for (const auto &g : e->groups) k += e->tuning.at(g.L).tuned ? 0u : 1u;
    *n = k;
    return PA_OK;
}

pa_status pa_sweep_shape(const pa_engine *e, uint32_t group, uint32_t *L, uint32_t *words_per_thread,
                         uint32_t *block, uint32_t *tuned)
{
    if (!e || group >= e->groups.size() || !L || !words_per_thread || !block || !tuned) return PA_ERR_INVALID_ARG;
    const SweepGroup &g = e->groups[group];
    const Tuning &t = e->tuning.at(g.L);
    const SweepCfg &c = t.candidates[t.pick];
    *L = g.L;
    *words_per_thread = c.fast ? c.WPT : 0;
    *block = c.block;
    *tuned = (t.tuned && t.candidates.size() > 1) ? 1u : 0u;
    return PA_OK;
}

pa_status pa_set_profiling(pa_engine *e, int on)
{
    if (!e) return PA_ERR_INVALID_ARG;
    e->profiling = on != 0;
    return PA_OK;
}

pa_status pa_kernel_times(pa_engine *e, double *ms_out, uint64_t *launches_out)
{
    if (!e || !ms_out || !launches_out) return PA_ERR_INVALID_ARG;
    PA_CUDA(cudaStreamSynchronize(e->stream));
    for (int k = 0; k < PA_K_COUNT; ++k) {
        ms_out[k] = 0.0;
        launches_out[k] = 0;
    }
    for (auto &t : e->timed) {
        float ms = 0.f;
        PA_CUDA(cudaEventElapsedTime(&ms, t.a, t.b));
        ms_out[t.kind] += ms;
        launches_out[t.kind] += 1;
        e->ev_free.push_back(t.a);
        e->ev_free.push_back(t.b);
    }
    e->timed.clear();
    return PA_OK;
}

pa_status pa_transfer_bytes(const pa_engine *e, uint64_t *h2d, uint64_t *d2h)
{
    if (!e || !h2d || !d2h) return PA_ERR_INVALID_ARG;
    *h2d = e->h2d;
    *d2h = e->d2h;
    return PA_OK;
}

pa_status pa_calibrate_philox(uint32_t wide, uint32_t reps, void *cuda_stream, double *calls_per_s)
{
    if (!calls_per_s || reps == 0 || reps > 1000) return PA_ERR_INVALID_ARG;
    const uint32_t blocks = 2432, threads = 128, iters = 64;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    uint32_t *out = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    double best = 0.0;
    cudaError_t err = cudaMalloc(&out, sizeof(uint32_t) * blocks * threads);
    if (!err) err = cudaEventCreate(&a);
    if (!err) err = cudaEventCreate(&b);
    for (uint32_t r = 0; r <= reps && !err; ++r) {  // launch 0 warms up
        err = cudaEventRecord(a, s);
        if (!err) launch_philox_calibration(out, blocks, threads, iters, wide != 0, s);
        if (!err) err = cudaGetLastError();
        if (!err) err = cudaEventRecord(b, s);
        if (!err) err = cudaEventSynchronize(b);
        float ms = 0.f;
        if (!err) err = cudaEventElapsedTime(&ms, a, b);
        if (!err && r > 0 && ms > 0.f) {
            const double v = (double)blocks * threads * iters * 8 / (ms * 1e-3);
            best = v > best ? v : best;
        }
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (out) cudaFree(out);
    if (err) return cuda_fail(err, "pa_calibrate_philox");
    *calls_per_s = best;
    return PA_OK;
}

pa_status pa_records(pa_engine *e, uint32_t run, pa_step_record *host_out, uint32_t *host_qhist,
                     uint32_t *host_qhist_pair, uint32_t *host_qhist_wang)
{
    if (!slot_ok(e, run) || !host_out) return PA_ERR_INVALID_ARG;
    const RunDev &x = e->rd[run];
    if ((host_qhist || host_qhist_pair || host_qhist_wang) && !x.overlap) return PA_ERR_INVALID_ARG;
    PA_TRY(prepare(e));
    PA_CUDA(cudaMemcpyAsync(host_out, e->P.rec + x.rec_off, sizeof(pa_step_record) * x.n_beta,
                            cudaMemcpyDeviceToHost, e->stream));
    const size_t nq = (size_t)x.n_beta * (x.N + 1);
    e->d2h += sizeof(pa_step_record) * x.n_beta +
              sizeof(uint32_t) * nq * ((host_qhist ? 1 : 0) + (host_qhist_pair ? 1 : 0) + (host_qhist_wang ? 1 : 0));
    if (host_qhist)
        PA_CUDA(cudaMemcpyAsync(host_qhist, e->P.qh + x.qh_off, sizeof(uint32_t) * nq, cudaMemcpyDeviceToHost, e->stream));
    if (host_qhist_pair)
        PA_CUDA(cudaMemcpyAsync(host_qhist_pair, e->P.qhp + x.qh_off, sizeof(uint32_t) * nq, cudaMemcpyDeviceToHost,
                                e->stream));
    if (host_qhist_wang)
        PA_CUDA(cudaMemcpyAsync(host_qhist_wang, e->P.qhw + x.qh_off, sizeof(uint32_t) * nq, cudaMemcpyDeviceToHost,
                                e->stream));
    return sync_read(e);
}

pa_status pa_measure(pa_engine *e, uint32_t run, uint32_t step, pa_step_record *host_out, uint32_t *host_qhist,
                     uint32_t *host_qhist_pair, uint32_t *host_qhist_wang)
{
    if (!slot_ok(e, run) || !host_out) return PA_ERR_INVALID_ARG;
    const RunDev &x = e->rd[run];
    if (step >= x.n_beta) return PA_ERR_INVALID_ARG;
    PA_TRY(prepare(e));
    if ((host_qhist || host_qhist_pair || host_qhist_wang) && !x.overlap) return PA_ERR_INVALID_ARG;
    PA_CUDA(cudaMemcpyAsync(host_out, e->P.rec + x.rec_off + step, sizeof(pa_step_record), cudaMemcpyDeviceToHost,
                            e->stream));
    const size_t n1 = x.N + 1;
    if (host_qhist)
        PA_CUDA(cudaMemcpyAsync(host_qhist, e->P.qh + x.qh_off + step * n1, sizeof(uint32_t) * n1,
                                cudaMemcpyDeviceToHost, e->stream));
    if (host_qhist_pair)
        PA_CUDA(cudaMemcpyAsync(host_qhist_pair, e->P.qhp + x.qh_off + step * n1, sizeof(uint32_t) * n1,
                                cudaMemcpyDeviceToHost, e->stream));
    if (host_qhist_wang)
        PA_CUDA(cudaMemcpyAsync(host_qhist_wang, e->P.qhw + x.qh_off + step * n1, sizeof(uint32_t) * n1,
                                cudaMemcpyDeviceToHost, e->stream));
    return sync_read(e);
}

pa_status pa_population_slice(pa_engine *e, uint32_t run, uint32_t first, uint32_t count, int8_t *host_spins,
                              int32_t *host_E, int32_t *host_M, uint32_t *host_fam, uint32_t *R_out,
                              uint32_t *step_out)
{
    if (!slot_ok(e, run)) return PA_ERR_INVALID_ARG;
    PA_TRY(prepare(e));
    const RunDev &x = e->rd[run];
    RunState st;
    PA_CUDA(cudaMemcpyAsync(&st, e->P.st + run, sizeof st, cudaMemcpyDeviceToHost, e->stream));
    PA_CUDA(cudaStreamSynchronize(e->stream));
    const uint32_t b = st.step & 1u, R = st.R_cur;
    if (R_out) *R_out = R;
    if (step_out) *step_out = st.step;
    const uint32_t lo = std::min(first, R), n = std::min<uint64_t>(count, (uint64_t)R - lo);
    if (host_spins && n) {
        std::vector<uint32_t> words((size_t)n * x.wstride);
        PA_CUDA(cudaMemcpyAsync(words.data(), e->P.spins[b] + x.spin_off + (uint64_t)lo * x.wstride,
                                sizeof(uint32_t) * words.size(), cudaMemcpyDeviceToHost, e->stream));
        PA_CUDA(cudaStreamSynchronize(e->stream));
        e->d2h += sizeof(uint32_t) * words.size();
        for (uint32_t j = 0; j < n; ++j)
            for (uint32_t q = 0; q < x.N; ++q) {
                const uint32_t xx = q % x.L, y = q / x.L, c = (xx + y) & 1u, pos = y * x.pitch + (xx >> 1);
                const uint32_t word = words[(size_t)j * x.wstride + c * x.pw + (pos >> 5)];
                host_spins[(size_t)j * x.N + q] = ((word >> (pos & 31)) & 1u) ? (int8_t)1 : (int8_t)-1;
            }
    }
    if (host_E && n)
        PA_CUDA(cudaMemcpyAsync(host_E, e->P.E[b] + x.rep_off + lo, sizeof(int32_t) * n, cudaMemcpyDeviceToHost,
                                e->stream));
    if (host_M && n)
        PA_CUDA(cudaMemcpyAsync(host_M, e->P.M[b] + x.rep_off + lo, sizeof(int32_t) * n, cudaMemcpyDeviceToHost,
                                e->stream));
    if (host_fam && n)
        PA_CUDA(cudaMemcpyAsync(host_fam, e->P.fam[b] + x.rep_off + lo, sizeof(uint32_t) * n,
                                cudaMemcpyDeviceToHost, e->stream));
    return sync_read(e);
}

pa_status pa_population(pa_engine *e, uint32_t run, int8_t *host_spins, int32_t *host_E, int32_t *host_M,
                        uint32_t *host_fam, uint32_t *R_out, uint32_t *step_out)
{
    return pa_population_slice(e, run, 0u, 0xFFFFFFFFu, host_spins, host_E, host_M, host_fam, R_out, step_out);
}

static pa_status ensure_wa(pa_engine *e, size_t bytes) { return ensure_buffer(e, &e->wa_buf, &e->wa_bytes, bytes); }

static size_t align256(size_t x) { return (x + 255) / 256 * 256; }

pa_status pa_set_allocator(pa_alloc_fn alloc, pa_free_fn free_, void *ctx)
{
    if ((alloc == nullptr) != (free_ == nullptr)) return PA_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_alloc_mu);
    g_alloc.alloc = alloc;
    g_alloc.free_ = free_;
    g_alloc.ctx = alloc ? ctx : nullptr;
    return PA_OK;
}

pa_status pa_step_records(pa_engine *e, const uint32_t *runs, uint32_t n_runs, pa_step_record *host_out)
{
    if (!e || !runs || !n_runs || !host_out) return PA_ERR_INVALID_ARG;
    for (uint32_t k = 0; k < n_runs; ++k)
        if (!slot_ok(e, runs[k])) return PA_ERR_INVALID_ARG;
    PA_TRY(prepare(e));
    const size_t b_rec = align256(sizeof(uint32_t) * n_runs);
    PA_TRY(ensure_buffer(e, &e->sr_buf, &e->sr_bytes, b_rec + sizeof(pa_step_record) * n_runs));
    auto *d_runs = static_cast<uint32_t *>(e->sr_buf);
    auto *d_out = reinterpret_cast<pa_step_record *>(static_cast<char *>(e->sr_buf) + b_rec);
    PA_CUDA(cudaMemcpyAsync(d_runs, runs, sizeof(uint32_t) * n_runs, cudaMemcpyHostToDevice, e->stream));
    e->launches += 1;
    launch_gather_records(e->P, d_runs, n_runs, d_out, e->stream);
    PA_CUDA(cudaGetLastError());
    PA_CUDA(cudaMemcpyAsync(host_out, d_out, sizeof(pa_step_record) * n_runs, cudaMemcpyDeviceToHost, e->stream));
    e->h2d += sizeof(uint32_t) * n_runs;
    e->d2h += sizeof(pa_step_record) * n_runs;
    return sync_read(e);
}

pa_status pa_weighted_average_runs(pa_engine *e, const uint32_t *run_idx, uint32_t n_groups, uint32_t M,
                                   uint32_t weight_kind, pa_wavg *host_out, double *host_Pq, double *host_Pq_pair,
                                   double *host_Pq_wang)
{
    if (!e || !run_idx || !n_groups || !M || !host_out || weight_kind > PA_WEIGHT_SIMPLE) return PA_ERR_INVALID_ARG;
    if (!slot_ok(e, run_idx[0])) return PA_ERR_INVALID_ARG;
    PA_TRY(prepare(e));
    const RunDev &r0 = e->rd[run_idx[0]];
    const uint32_t n_steps = r0.n_beta, N = r0.N;
    std::vector<unsigned long long> rec_off((size_t)n_groups * M), qh_off((size_t)n_groups * M);
    for (size_t k = 0; k < rec_off.size(); ++k) {
        if (!slot_ok(e, run_idx[k])) return PA_ERR_INVALID_ARG;
        const RunDev &x = e->rd[run_idx[k]];
        if (x.n_beta != n_steps || x.N != N) return PA_ERR_INVALID_ARG;
        if ((host_Pq || host_Pq_pair || host_Pq_wang) && !x.overlap) return PA_ERR_INVALID_ARG;
        rec_off[k] = x.rec_off;
        qh_off[k] = x.qh_off;
    }
    const size_t nGM = (size_t)n_groups * M, nP = (size_t)n_groups * n_steps * (N + 1);
    const size_t b_off = align256(sizeof(unsigned long long) * nGM);
    const size_t b_qoff = b_off + align256(sizeof(unsigned long long) * nGM);
    const size_t b_out = b_qoff + align256(sizeof(pa_wavg) * n_groups * n_steps);
    const size_t b_w = b_out + align256(sizeof(double) * n_groups * n_steps * M);
    const size_t b_pq = b_w + align256(host_Pq ? sizeof(double) * nP : 0);
    const size_t b_pqp = b_pq + align256(host_Pq_pair ? sizeof(double) * nP : 0);
    const size_t total = b_pqp + align256(host_Pq_wang ? sizeof(double) * nP : 0);
    pa_status s = ensure_wa(e, total);
    if (s != PA_OK) return s;
    char *base = static_cast<char *>(e->wa_buf);
    auto *d_roff = reinterpret_cast<unsigned long long *>(base);
    auto *d_qoff = reinterpret_cast<unsigned long long *>(base + b_off);
    auto *d_out = reinterpret_cast<pa_wavg *>(base + b_qoff);
    auto *d_w = reinterpret_cast<double *>(base + b_out);
    double *d_pq = host_Pq ? reinterpret_cast<double *>(base + b_w) : nullptr;
    double *d_pqp = host_Pq_pair ? reinterpret_cast<double *>(base + b_pq) : nullptr;
    double *d_pqw = host_Pq_wang ? reinterpret_cast<double *>(base + b_pqp) : nullptr;
    PA_CUDA(cudaMemcpyAsync(d_roff, rec_off.data(), sizeof(unsigned long long) * nGM, cudaMemcpyHostToDevice, e->stream));
    PA_CUDA(cudaMemcpyAsync(d_qoff, qh_off.data(), sizeof(unsigned long long) * nGM, cudaMemcpyHostToDevice, e->stream));
    timed_launch(e, PA_K_WAVG, [&] {
        launch_wavg_wang(e->P.rec, d_roff, e->P.qh, e->P.qhp, e->P.qhw, d_qoff, n_groups, M, n_steps, N, weight_kind,
                         d_out, d_w, d_pq, d_pqp, d_pqw, e->stream);
    });
    e->launches += 2 + ((d_pq || d_pqp || d_pqw) ? 1 : 0);  // with the one counted above: 3 passes + histograms
    e->h2d += 2 * sizeof(unsigned long long) * nGM;
    e->d2h += sizeof(pa_wavg) * n_groups * n_steps +
              sizeof(double) * nP * ((host_Pq ? 1 : 0) + (host_Pq_pair ? 1 : 0) + (host_Pq_wang ? 1 : 0));
    PA_CUDA(cudaGetLastError());
    PA_CUDA(cudaMemcpyAsync(host_out, d_out, sizeof(pa_wavg) * n_groups * n_steps, cudaMemcpyDeviceToHost, e->stream));
    if (host_Pq) PA_CUDA(cudaMemcpyAsync(host_Pq, d_pq, sizeof(double) * nP, cudaMemcpyDeviceToHost, e->stream));
    if (host_Pq_pair)
        PA_CUDA(cudaMemcpyAsync(host_Pq_pair, d_pqp, sizeof(double) * nP, cudaMemcpyDeviceToHost, e->stream));
    if (host_Pq_wang)
        PA_CUDA(cudaMemcpyAsync(host_Pq_wang, d_pqw, sizeof(double) * nP, cudaMemcpyDeviceToHost, e->stream));
    return pa_sync(e);
}

pa_status pa_weighted_average(const pa_step_record *recs, const uint32_t *qhist, const uint32_t *qhist_pair,
                              const uint32_t *qhist_wang, uint32_t M, uint32_t n_steps, uint32_t N,
                              uint32_t weight_kind, pa_wavg *out, double *Pq, double *Pq_pair, double *Pq_wang,
                              void *cuda_stream)
{
    if (!recs || !M || !n_steps || !N || !out || weight_kind > PA_WEIGHT_SIMPLE) return PA_ERR_INVALID_ARG;
    if ((Pq && !qhist) || (Pq_pair && !qhist_pair) || (Pq_wang && !qhist_wang)) return PA_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const size_t nr = (size_t)M * n_steps, nq = nr * (N + 1), nP = (size_t)n_steps * (N + 1);
    const size_t b_rec = align256(sizeof(pa_step_record) * nr);
    const size_t b_qh = b_rec + align256(qhist ? sizeof(uint32_t) * nq : 0);
    const size_t b_qhp = b_qh + align256(qhist_pair ? sizeof(uint32_t) * nq : 0);
    const size_t b_qhw = b_qhp + align256(qhist_wang ? sizeof(uint32_t) * nq : 0);
    const size_t b_off = b_qhw + align256(sizeof(unsigned long long) * M);
    const size_t b_qoff = b_off + align256(sizeof(unsigned long long) * M);
    const size_t b_out = b_qoff + align256(sizeof(pa_wavg) * n_steps);
    const size_t b_w = b_out + align256(sizeof(double) * n_steps * M);
    const size_t b_pq = b_w + align256(Pq ? sizeof(double) * nP : 0);
    const size_t b_pqp = b_pq + align256(Pq_pair ? sizeof(double) * nP : 0);
    const size_t total = b_pqp + align256(Pq_wang ? sizeof(double) * nP : 0);
    const Allocator alloc = current_allocator();
    char *base = static_cast<char *>(device_alloc(alloc, total, st));
    if (!base) return PA_ERR_OOM;
    cudaError_t err = cudaSuccess;
    pa_status s = PA_OK;
    std::vector<unsigned long long> roff(M), qoff(M);
    for (uint32_t m = 0; m < M; ++m) {
        roff[m] = (unsigned long long)m * n_steps;
        qoff[m] = (unsigned long long)m * n_steps * (N + 1);
    }
    auto *d_rec = reinterpret_cast<pa_step_record *>(base);
    auto *d_qh = qhist ? reinterpret_cast<uint32_t *>(base + b_rec) : nullptr;
    auto *d_qhp = qhist_pair ? reinterpret_cast<uint32_t *>(base + b_qh) : nullptr;
    auto *d_qhw = qhist_wang ? reinterpret_cast<uint32_t *>(base + b_qhp) : nullptr;
    auto *d_roff = reinterpret_cast<unsigned long long *>(base + b_qhw);
    auto *d_qoff = reinterpret_cast<unsigned long long *>(base + b_off);
    auto *d_out = reinterpret_cast<pa_wavg *>(base + b_qoff);
    auto *d_w = reinterpret_cast<double *>(base + b_out);
    double *d_pq = Pq ? reinterpret_cast<double *>(base + b_w) : nullptr;
    double *d_pqp = Pq_pair ? reinterpret_cast<double *>(base + b_pq) : nullptr;
    double *d_pqw = Pq_wang ? reinterpret_cast<double *>(base + b_pqp) : nullptr;
    do {
        if ((err = cudaMemcpyAsync(d_rec, recs, sizeof(pa_step_record) * nr, cudaMemcpyHostToDevice, st))) break;
        if (qhist && (err = cudaMemcpyAsync(d_qh, qhist, sizeof(uint32_t) * nq, cudaMemcpyHostToDevice, st))) break;
        if (qhist_pair && (err = cudaMemcpyAsync(d_qhp, qhist_pair, sizeof(uint32_t) * nq, cudaMemcpyHostToDevice, st)))
            break;
        if (qhist_wang && (err = cudaMemcpyAsync(d_qhw, qhist_wang, sizeof(uint32_t) * nq, cudaMemcpyHostToDevice, st)))
            break;
        if ((err = cudaMemcpyAsync(d_roff, roff.data(), sizeof(unsigned long long) * M, cudaMemcpyHostToDevice, st))) break;
        if ((err = cudaMemcpyAsync(d_qoff, qoff.data(), sizeof(unsigned long long) * M, cudaMemcpyHostToDevice, st))) break;
        launch_wavg_wang(d_rec, d_roff, d_qh, d_qhp, d_qhw, d_qoff, 1, M, n_steps, N, weight_kind, d_out, d_w, d_pq,
                         d_pqp, d_pqw, st);
        if ((err = cudaGetLastError())) break;
        if ((err = cudaMemcpyAsync(out, d_out, sizeof(pa_wavg) * n_steps, cudaMemcpyDeviceToHost, st))) break;
        if (Pq && (err = cudaMemcpyAsync(Pq, d_pq, sizeof(double) * nP, cudaMemcpyDeviceToHost, st))) break;
        if (Pq_pair && (err = cudaMemcpyAsync(Pq_pair, d_pqp, sizeof(double) * nP, cudaMemcpyDeviceToHost, st))) break;
        if (Pq_wang && (err = cudaMemcpyAsync(Pq_wang, d_pqw, sizeof(double) * nP, cudaMemcpyDeviceToHost, st))) break;
        err = cudaStreamSynchronize(st);
    } while (0);
    if (err != cudaSuccess) s = cuda_fail(err, "pa_weighted_average");
    device_free(alloc, base, total, st);
    return s;
}

pa_status pa_checkpoint(pa_engine *e, uint32_t run, void *host_buf, size_t *bytes)
{
    if (!slot_ok(e, run) || !bytes) return PA_ERR_INVALID_ARG;
    PA_TRY(prepare(e));
    const RunDev &x = e->rd[run];
    RunState st;
    PA_CUDA(cudaMemcpyAsync(&st, e->P.st + run, sizeof st, cudaMemcpyDeviceToHost, e->stream));
    PA_CUDA(cudaStreamSynchronize(e->stream));
    if (st.status) return PA_ERR_STATE;  // a stopped run is inspected, not resumed
    const std::vector<CkptSection> sec = ckpt_sections(e, run, st);
    const size_t need = ckpt_bytes(x, sec);
    if (!host_buf) {
        *bytes = need;
        return PA_OK;
    }
    if (*bytes < need) {
        *bytes = need;
        return PA_ERR_INVALID_ARG;
    }
    const pa_run_desc &d = e->rh[run].d;
    CkptHeader h{};
    std::memcpy(h.magic, CKPT_MAGIC, sizeof h.magic);
    h.L = d.L;
    h.model = d.model;
    h.R = d.R;
    h.R_cap = x.R_cap;
    h.theta = d.theta;
    h.n_beta = d.n_beta;
    h.seed = d.seed;
    h.run_id = d.run_id;
    h.disorder_id = d.disorder_id;
    h.resample = d.resample;
    h.overlap = d.overlap;
    h.steps_done = e->rh[run].steps_done;
    h.R_cur = st.R_cur;
    h.buffer = st.step & 1u;
    h.wstride = x.wstride;
    h.scratch_words = scratch_words(x.N, x.R_cap);
    h.J_words = sizes_of(d).J;
    h.total_bytes = need;
    h.dos_hash = e->rh[run].dos_hash;
    char *out = static_cast<char *>(host_buf);
    std::memcpy(out, &h, sizeof h);
    size_t o = sizeof h;
    std::memcpy(out + o, &st, sizeof st);
    o += sizeof st;
    PA_CUDA(cudaMemcpyAsync(out + o, e->d_beta + x.beta_off, sizeof(double) * x.n_beta, cudaMemcpyDeviceToHost,
                            e->stream));
    o += sizeof(double) * x.n_beta;
    for (const auto &c : sec) {
        if (c.bytes) PA_CUDA(cudaMemcpyAsync(out + o, c.dev, c.bytes, cudaMemcpyDeviceToHost, e->stream));
        o += c.bytes;
    }
    e->d2h += need;
    *bytes = need;
    return sync_read(e);
}

pa_status pa_restore(pa_engine *e, uint32_t run, const void *host_buf, size_t bytes)
{
    if (!slot_ok(e, run) || !host_buf || bytes < sizeof(CkptHeader) + sizeof(RunState)) return PA_ERR_INVALID_ARG;
    PA_TRY(prepare(e));  // the slot's beta_0 draw, if pending, must not run after the restore
    PA_CUDA(cudaStreamSynchronize(e->stream));
    const RunDev &x = e->rd[run];
    const pa_run_desc &d = e->rh[run].d;
    CkptHeader h;
    std::memcpy(&h, host_buf, sizeof h);
    if (std::memcmp(h.magic, CKPT_MAGIC, sizeof h.magic) != 0 || h.total_bytes != bytes) return PA_ERR_INVALID_ARG;
    if (h.L != d.L || h.model != d.model || h.R != d.R || h.R_cap != x.R_cap || h.theta != d.theta ||
        h.n_beta != d.n_beta || h.seed != d.seed || h.run_id != d.run_id || h.disorder_id != d.disorder_id ||
        h.resample != d.resample || h.overlap != d.overlap || h.wstride != x.wstride ||
        h.scratch_words != scratch_words(x.N, x.R_cap) || h.J_words != sizes_of(d).J ||
        h.dos_hash != e->rh[run].dos_hash)
        return PA_ERR_INVALID_ARG;
    const char *in = static_cast<const char *>(host_buf);
    RunState st;
    std::memcpy(&st, in + sizeof h, sizeof st);
    if (st.R_cur != h.R_cur || (st.step & 1u) != h.buffer || st.R_cur > x.R_cap || st.step >= d.n_beta ||
        h.steps_done != st.step)
        return PA_ERR_INVALID_ARG;
    std::vector<double> beta(x.n_beta);
    PA_CUDA(cudaMemcpyAsync(beta.data(), e->d_beta + x.beta_off, sizeof(double) * x.n_beta, cudaMemcpyDeviceToHost,
                            e->stream));
    PA_CUDA(cudaStreamSynchronize(e->stream));
    if (std::memcmp(beta.data(), in + sizeof h + sizeof st, sizeof(double) * x.n_beta) != 0)
        return PA_ERR_INVALID_ARG;  // another schedule
    const std::vector<CkptSection> sec = ckpt_sections(e, run, st);
    if (ckpt_bytes(x, sec) != bytes) return PA_ERR_INVALID_ARG;
    st.ticket = 0;
    size_t o = sizeof h + sizeof st + sizeof(double) * x.n_beta;
    for (const auto &c : sec) {
        if (c.bytes) PA_CUDA(cudaMemcpyAsync(c.dev, in + o, c.bytes, cudaMemcpyHostToDevice, e->stream));
        o += c.bytes;
    }
    PA_CUDA(cudaMemcpyAsync(e->P.st + run, &st, sizeof st, cudaMemcpyHostToDevice, e->stream));
    PA_CUDA(cudaStreamSynchronize(e->stream));  // the caller's buffer and st must outlive the copies
    e->h2d += bytes;
    e->rh[run].steps_done = h.steps_done;
    e->dirty = true;
    // An engine-level error (capacity, extinction) is cleared once no resident run is stopped any
    // more, so that restoring the run that failed from an earlier checkpoint lets the anneal go on.
    std::vector<RunState> all(e->S);
    PA_CUDA(cudaMemcpyAsync(all.data(), e->P.st, sizeof(RunState) * e->S, cudaMemcpyDeviceToHost, e->stream));
    PA_CUDA(cudaStreamSynchronize(e->stream));
    bool stopped = false;
    for (uint32_t s : e->active) stopped |= all[s].status != 0;
    if (!stopped) {
        PA_CUDA(cudaMemsetAsync(e->P.status, 0, sizeof(uint32_t), e->stream));
        PA_CUDA(cudaStreamSynchronize(e->stream));
        e->latched = PA_OK;
    }
    return PA_OK;
}

}  // extern "C"

