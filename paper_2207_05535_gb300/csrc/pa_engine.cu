// Host side of the population-annealing engine: the C ABI declared in pa.h.
//
// pa_create lays out one device pool for all runs (offsets per run, see
// pa_internal.cuh), builds the per-step tables on the host (weights
// exp(-4 n dbeta_i) for the resampling normalisation and the Metropolis
// thresholds floor(exp(-4 m beta_i) 2^32)), draws the beta_0 populations and
// measures step 0.  pa_anneal_step enqueues one anneal step per call for all
// runs: resample (all runs), sweep (one launch per lattice size), overlaps and
// measurement; the sequence can be captured once as a CUDA graph and
// replayed because every kernel reads its temperature index from device state.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "pa_internal.cuh"

using namespace pa;

struct SweepGroup {
    uint32_t L;
    int any_glass = 0;
    SweepCfg cfg;                     // chosen launch shape
    std::vector<SweepCfg> candidates; // timed on the first anneal step when more than one
    bool tuned = false;
    float tuned_ms = 0.f;
    uint32_t max_Rcap;
    std::vector<uint32_t> runs;
    std::vector<uint32_t> n_tiles;   // per candidate: total tiles (prefix of ceil(R_cap / RPC))
    uint32_t *d_runs = nullptr;      // run indices, then per candidate its tile map (n + 1 entries)
    uint32_t pick = 0;               // chosen candidate
    const uint32_t *tile_map(uint32_t c) const { return d_runs + runs.size() + (size_t)c * (runs.size() + 1); }
};

struct pa_engine {
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    uint32_t n_runs = 0;
    std::vector<RunDev> rd;
    std::vector<SweepGroup> groups;
    std::vector<uint32_t> q_runs;
    uint32_t *d_q_runs = nullptr;
    uint32_t *d_init_tiles = nullptr;  // prefix of ceil(R / 4) over all runs
    uint32_t init_tiles = 0;
    uint32_t max_pw = 1;  // largest colour-plane word count of any run
    uint32_t max_Rcap = 0, max_R = 0, max_nbeta = 0;
    Pool P{};
    std::vector<void *> allocs;
    uint64_t launches = 0;
    uint64_t rec_count = 0, qh_count = 0;
    uint64_t launches_per_tick = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    pa_status latched = PA_OK;
    // profiling: event pairs per launch, summed by pa_kernel_times
    bool profiling = false;
    std::vector<cudaEvent_t> ev_free;
    struct Timed {
        int kind;
        cudaEvent_t a, b;
    };
    std::vector<Timed> timed;
    uint64_t h2d = 0, d2h = 0;
    // scratch for weighted averages (grown on demand)
    void *wa_buf = nullptr;
    size_t wa_bytes = 0;
};

namespace {

pa_status cuda_fail(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return PA_OK;
    std::fprintf(stderr, "libpa: %s: %s\n", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? PA_ERR_OOM : PA_ERR_CUDA;
}

#define PA_CUDA(call)                                             \
    do {                                                          \
        cudaError_t _e = (call);                                  \
        if (_e != cudaSuccess) return cuda_fail(_e, #call);       \
    } while (0)

template <typename T>
pa_status dalloc(pa_engine *e, T **p, size_t count)
{
    void *q = nullptr;
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = 16;
    cudaError_t err = cudaMalloc(&q, bytes);
    if (err != cudaSuccess) {
        cudaGetLastError();
        return err == cudaErrorMemoryAllocation ? PA_ERR_OOM : cuda_fail(err, "cudaMalloc");
    }
    e->allocs.push_back(q);
    *p = static_cast<T *>(q);
    return PA_OK;
}

uint32_t default_cap(const pa_run_desc &d)
{
    if (d.R_cap) return d.R_cap;
    if (d.resample == PA_MULTINOMIAL) return d.R;
    return d.R + 8u * (uint32_t)std::ceil(std::sqrt((double)d.R)) + 64u;
}

pa_status validate(const pa_run_desc *runs, uint32_t n)
{
    if (!runs || n == 0) return PA_ERR_INVALID_ARG;
    for (uint32_t r = 0; r < n; ++r) {
        const pa_run_desc &d = runs[r];
        if (d.L < 4 || d.L > 256 || (d.L & 1u)) return PA_ERR_INVALID_ARG;
        if (d.model > PA_EA_PMJ || d.resample > PA_MULTINOMIAL || d.overlap > 3u || d.reserved) return PA_ERR_INVALID_ARG;
        if (d.R < 1 || d.n_beta < 1 || !d.beta || d.theta > (1u << 22)) return PA_ERR_INVALID_ARG;
        const uint32_t cap = default_cap(d);
        if (cap < d.R) return PA_ERR_INVALID_ARG;
        if (d.resample == PA_MULTINOMIAL && cap < d.R) return PA_ERR_INVALID_ARG;
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

std::string key_of(const double *b, uint32_t n, uint32_t N)
{
    std::string k(reinterpret_cast<const char *>(&N), sizeof N);
    k.append(reinterpret_cast<const char *>(b), sizeof(double) * n);
    return k;
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

pa_status upload_tile_maps(pa_engine *e, SweepGroup &g)
{
    std::vector<uint32_t> h(g.runs);
    g.n_tiles.clear();
    for (const SweepCfg &c : g.candidates) {
        uint64_t acc = 0;
        h.push_back(0u);
        for (uint32_t r : g.runs) {
            acc += (e->rd[r].R_cap + c.RPC - 1) / c.RPC;
            if (acc > 0x7fffffffull) return PA_ERR_INVALID_ARG;  // beyond one launch's grid
            h.push_back((uint32_t)acc);
        }
        g.n_tiles.push_back((uint32_t)acc);
    }
    cudaError_t err = cudaMemcpy(g.d_runs, h.data(), sizeof(uint32_t) * h.size(), cudaMemcpyHostToDevice);
    if (err != cudaSuccess) return cuda_fail(err, "tile maps");
    e->h2d += sizeof(uint32_t) * h.size();
    return PA_OK;
}

// One eager anneal step that times every candidate sweep shape of the groups
// not tuned yet on the real data and keeps the fastest.  Each candidate reads
// the same parents and writes the same children, so running several is
// harmless; the last launch leaves the children in place.
pa_status enqueue_tuning_tick(pa_engine *e)
{
    launch_resample(e->P, e->n_runs, e->stream);
    e->launches += 1;
    for (auto &g : e->groups) {
        if (g.tuned) {
            launch_sweep(e->P, g.d_runs, g.tile_map(g.pick), (uint32_t)g.runs.size(), g.n_tiles[g.pick], g.cfg,
                         g.any_glass, e->stream);
            e->launches += 1;
            continue;
        }
        std::vector<cudaEvent_t> ev(2 * g.candidates.size());
        for (auto &x : ev) PA_CUDA(cudaEventCreate(&x));
        for (uint32_t c = 0; c < g.candidates.size(); ++c) {
            PA_CUDA(cudaEventRecord(ev[2 * c], e->stream));
            launch_sweep(e->P, g.d_runs, g.tile_map(c), (uint32_t)g.runs.size(), g.n_tiles[c], g.candidates[c],
                         g.any_glass, e->stream);
            PA_CUDA(cudaEventRecord(ev[2 * c + 1], e->stream));
            e->launches += 1;
        }
        PA_CUDA(cudaStreamSynchronize(e->stream));
        PA_CUDA(cudaGetLastError());
        float best = 0.f;
        for (uint32_t c = 0; c < g.candidates.size(); ++c) {
            float ms = 0.f;
            PA_CUDA(cudaEventElapsedTime(&ms, ev[2 * c], ev[2 * c + 1]));
            if (c == 0 || ms < best) {
                best = ms;
                g.pick = c;
            }
        }
        for (auto &x : ev) cudaEventDestroy(x);
        g.cfg = g.candidates[g.pick];
        g.tuned = true;
        g.tuned_ms = best;
    }
    if (!e->q_runs.empty()) {
        launch_overlap(e->P, e->d_q_runs, (uint32_t)e->q_runs.size(), e->max_Rcap, 0, e->stream);
        e->launches += 1;
    }
    launch_measure(e->P, e->n_runs, 0, e->stream);
    e->launches += 1;
    PA_CUDA(cudaGetLastError());
    return PA_OK;
}

void enqueue_tick(pa_engine *e)
{
    timed_launch(e, PA_K_RESAMPLE, [&] { launch_resample(e->P, e->n_runs, e->stream); });
    for (auto &g : e->groups)
        timed_launch(e, PA_K_SWEEP, [&] {
            launch_sweep(e->P, g.d_runs, g.tile_map(g.pick), (uint32_t)g.runs.size(), g.n_tiles[g.pick], g.cfg,
                         g.any_glass, e->stream);
        });
    if (!e->q_runs.empty())
        timed_launch(e, PA_K_OVERLAP, [&] {
            launch_overlap(e->P, e->d_q_runs, (uint32_t)e->q_runs.size(), e->max_Rcap, 0, e->stream);
        });
    timed_launch(e, PA_K_MEASURE, [&] { launch_measure(e->P, e->n_runs, 0, e->stream); });
}

// beta_0: couplings, uniform populations, step-0 measurement (Sec. II.B step (i)).
pa_status enqueue_init(pa_engine *e)
{
    std::vector<RunState> h_st(e->n_runs);
    for (uint32_t r = 0; r < e->n_runs; ++r) {
        h_st[r].step = 0;
        h_st[r].R_cur = e->rd[r].R;
        h_st[r].R_new = e->rd[r].R;
        h_st[r].status = 0;
        h_st[r].lnQ = 0.0;
    }
    cudaError_t err = cudaMemcpyAsync(e->P.st, h_st.data(), sizeof(RunState) * e->n_runs, cudaMemcpyHostToDevice,
                                      e->stream);
    if (!err) err = cudaMemsetAsync(e->P.rec, 0, sizeof(pa_step_record) * (e->rec_count ? e->rec_count : 1), e->stream);
    if (!err) err = cudaMemsetAsync(e->P.qh, 0, sizeof(uint32_t) * (e->qh_count ? e->qh_count : 1), e->stream);
    if (!err) err = cudaMemsetAsync(e->P.qhp, 0, sizeof(uint32_t) * (e->qh_count ? e->qh_count : 1), e->stream);
    if (!err) err = cudaMemsetAsync(e->P.status, 0, sizeof(uint32_t), e->stream);
    if (!err) err = cudaStreamSynchronize(e->stream);  // h_st must outlive the copy
    if (err) return cuda_fail(err, "reset state");
    e->h2d += sizeof(RunState) * e->n_runs;
    timed_launch(e, PA_K_INIT, [&] { launch_init_couplings(e->P, e->n_runs, e->stream); });
    timed_launch(e, PA_K_INIT,
                 [&] { launch_init_population(e->P, e->d_init_tiles, e->n_runs, e->init_tiles, e->max_pw, e->stream); });
    if (!e->q_runs.empty())
        timed_launch(e, PA_K_OVERLAP, [&] {
            launch_overlap(e->P, e->d_q_runs, (uint32_t)e->q_runs.size(), e->max_Rcap, 1, e->stream);
        });
    timed_launch(e, PA_K_MEASURE, [&] { launch_measure(e->P, e->n_runs, 1, e->stream); });
    e->launches += 3 + (e->q_runs.empty() ? 0 : 1);
    e->latched = PA_OK;
    err = cudaGetLastError();
    return err ? cuda_fail(err, "init launch") : PA_OK;
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
    for (void *p : e->allocs) cudaFree(p);
    if (e->wa_buf) cudaFree(e->wa_buf);
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

pa_status pa_create_ex(const pa_run_desc *runs, uint32_t n_runs, void *cuda_stream, uint32_t flags, pa_engine **out)
{
    if (!out || (flags & ~(uint32_t)(PA_CREATE_GENERIC_SWEEP | PA_CREATE_NO_AUTOTUNE))) return PA_ERR_INVALID_ARG;
    *out = nullptr;
    pa_status vs = validate(runs, n_runs);
    if (vs != PA_OK) return vs;
    PA_CUDA(prepare_kernels());

    pa_engine *e = new (std::nothrow) pa_engine();
    if (!e) return PA_ERR_OOM;
    cudaGetDevice(&e->device);
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
    e->n_runs = n_runs;
    e->rd.resize(n_runs);

    // ---- layout
    uint64_t rep = 0, spinw = 0, rec = 0, qh = 0, J = 0, scr = 0;
    std::map<std::string, uint64_t> beta_tab, wt_tab, thr_tab;
    std::vector<double> h_beta, h_wt;
    std::vector<unsigned long long> h_thr;
    std::map<uint32_t, size_t> group_of_L;
    for (uint32_t r = 0; r < n_runs; ++r) {
        const pa_run_desc &d = runs[r];
        RunDev &x = e->rd[r];
        std::memset(&x, 0, sizeof x);
        x.L = d.L;
        x.N = d.L * d.L;
        x.Lh = d.L / 2;
        const uint32_t pw = (x.N + 63) / 64;  // words per colour plane
        x.wstride = (2 * pw + 3) / 4 * 4;
        e->max_pw = pw > e->max_pw ? pw : e->max_pw;
        x.model = d.model;
        x.R = d.R;
        x.R_cap = default_cap(d);
        x.theta = d.theta;
        x.n_beta = d.n_beta;
        x.seed = d.seed;
        x.run_id = d.run_id;
        x.disorder_id = d.disorder_id;
        x.resample = d.resample;
        x.overlap = d.overlap;
        x.paired = (d.overlap & PA_Q_PAIR) ? d.paired : -1;
        x.rep_off = rep;
        rep += x.R_cap;
        x.spin_off = spinw;
        spinw += (uint64_t)x.R_cap * x.wstride;
        x.rec_off = rec;
        rec += d.n_beta;
        x.qh_off = qh;
        if (d.overlap) qh += (uint64_t)d.n_beta * (x.N + 1);
        x.J_off = J;
        J += 2ull * x.wstride + 8ull * pw;
        x.scr_off = scr;
        scr += scratch_words(x.N, x.R_cap);
        x.ln2N = (double)x.N * std::log(2.0);
        // schedule and tables, shared by runs with equal (N, schedule)
        std::string kb = key_of(d.beta, d.n_beta, 0);
        auto itb = beta_tab.find(kb);
        if (itb == beta_tab.end()) {
            itb = beta_tab.emplace(kb, h_beta.size()).first;
            h_beta.insert(h_beta.end(), d.beta, d.beta + d.n_beta);
            thr_tab[kb] = h_thr.size();
            for (uint32_t i = 0; i < d.n_beta; ++i) {
                h_thr.push_back(threshold(d.beta[i], 1));
                h_thr.push_back(threshold(d.beta[i], 2));
            }
        }
        x.beta_off = itb->second;
        x.thr_off = thr_tab[kb];
        std::string kw = key_of(d.beta, d.n_beta, x.N);
        auto itw = wt_tab.find(kw);
        if (itw == wt_tab.end()) {
            itw = wt_tab.emplace(kw, h_wt.size()).first;
            const uint32_t n1 = x.N + 1;
            size_t base = h_wt.size();
            h_wt.resize(base + (size_t)d.n_beta * n1, 0.0);
            for (uint32_t i = 1; i < d.n_beta; ++i) {
                const double dbeta = d.beta[i] - d.beta[i - 1];
                for (uint32_t n = 0; n < n1; ++n) h_wt[base + (size_t)i * n1 + n] = std::exp(-(double)(4 * n) * dbeta);
            }
        }
        x.wt_off = itw->second;
        e->max_Rcap = x.R_cap > e->max_Rcap ? x.R_cap : e->max_Rcap;
        e->max_R = x.R > e->max_R ? x.R : e->max_R;
        e->max_nbeta = d.n_beta > e->max_nbeta ? d.n_beta : e->max_nbeta;
        auto g = group_of_L.find(d.L);
        if (g == group_of_L.end()) {
            g = group_of_L.emplace(d.L, e->groups.size()).first;
            SweepGroup sg;
            sg.L = d.L;
            sg.candidates = sweep_candidates(d.L, (flags & PA_CREATE_GENERIC_SWEEP) ? 0 : 1);
            sg.cfg = sg.candidates[0];
            sg.tuned = sg.candidates.size() < 2 || (flags & PA_CREATE_NO_AUTOTUNE);
            sg.max_Rcap = 0;
            e->groups.push_back(sg);
        }
        SweepGroup &sg = e->groups[g->second];
        sg.runs.push_back(r);
        if (d.model == PA_EA_PMJ) sg.any_glass = 1;
        sg.max_Rcap = x.R_cap > sg.max_Rcap ? x.R_cap : sg.max_Rcap;
        if (d.overlap) e->q_runs.push_back(r);
    }

    // ---- allocation
    pa_status s = PA_OK;
    RunDev *d_runs = nullptr;
    unsigned long long *d_thr = nullptr;
    double *d_beta = nullptr, *d_wt = nullptr;
    uint32_t wmax = 0;
    for (auto &x : e->rd) wmax = x.wstride > wmax ? x.wstride : wmax;
    uint64_t spin_words = 0;
    for (auto &x : e->rd) spin_words += (uint64_t)x.R_cap * x.wstride;
#define TRY(expr)                      \
    do {                               \
        s = (expr);                    \
        if (s != PA_OK) goto fail;     \
    } while (0)
    TRY(dalloc(e, &d_runs, n_runs));
    TRY(dalloc(e, &e->P.st, n_runs));
    for (int b = 0; b < 2; ++b) {
        TRY(dalloc(e, &e->P.spins[b], spin_words));
        TRY(dalloc(e, &e->P.E[b], rep));
        TRY(dalloc(e, &e->P.M[b], rep));
        TRY(dalloc(e, &e->P.fam[b], rep));
    }
    TRY(dalloc(e, &e->P.parent, rep));
    TRY(dalloc(e, &e->P.cnt, rep));
    TRY(dalloc(e, &e->P.rec, rec));
    TRY(dalloc(e, &e->P.qh, qh));
    TRY(dalloc(e, &e->P.qhp, qh));
    TRY(dalloc(e, &d_beta, h_beta.size()));
    TRY(dalloc(e, &d_wt, h_wt.size()));
    TRY(dalloc(e, &d_thr, h_thr.size()));
    TRY(dalloc(e, &e->P.J, J));
    TRY(dalloc(e, &e->P.scratch, scr));
    TRY(dalloc(e, &e->P.status, 1));
    e->P.runs = d_runs;
    e->P.beta = d_beta;
    e->P.wt = d_wt;
    e->P.thr = d_thr;
    for (auto &g : e->groups) {
        // run indices, then one tile map per candidate shape (each n + 1 entries)
        TRY(dalloc(e, &g.d_runs, g.runs.size() * (1 + g.candidates.size()) + g.candidates.size()));
        TRY(upload_tile_maps(e, g));
    }
    {
        std::vector<uint32_t> h(1, 0u);
        for (uint32_t r = 0; r < n_runs; ++r) {
            const uint64_t next = (uint64_t)h.back() + (e->rd[r].R + 3) / 4;
            if (next > 0x7fffffffull) TRY(PA_ERR_INVALID_ARG);
            h.push_back((uint32_t)next);
        }
        e->init_tiles = h.back();
        TRY(dalloc(e, &e->d_init_tiles, h.size()));
        if (cudaMemcpy(e->d_init_tiles, h.data(), sizeof(uint32_t) * h.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            TRY(PA_ERR_CUDA);
        e->h2d += sizeof(uint32_t) * h.size();
    }
    if (!e->q_runs.empty()) {
        TRY(dalloc(e, &e->d_q_runs, e->q_runs.size()));
        if (cudaMemcpyAsync(e->d_q_runs, e->q_runs.data(), sizeof(uint32_t) * e->q_runs.size(),
                            cudaMemcpyHostToDevice, e->stream) != cudaSuccess)
            TRY(PA_ERR_CUDA);
    }
    {
        cudaError_t err = cudaSuccess;
        err = err ? err : cudaMemcpyAsync(d_runs, e->rd.data(), sizeof(RunDev) * n_runs, cudaMemcpyHostToDevice, e->stream);
        err = err ? err : cudaMemcpyAsync(d_beta, h_beta.data(), sizeof(double) * h_beta.size(), cudaMemcpyHostToDevice, e->stream);
        err = err ? err : cudaMemcpyAsync(d_wt, h_wt.data(), sizeof(double) * h_wt.size(), cudaMemcpyHostToDevice, e->stream);
        err = err ? err : cudaMemcpyAsync(d_thr, h_thr.data(), sizeof(unsigned long long) * h_thr.size(), cudaMemcpyHostToDevice, e->stream);
        for (int b = 0; b < 2 && err == cudaSuccess; ++b)
            err = cudaMemsetAsync(e->P.spins[b], 0, sizeof(uint32_t) * (spin_words ? spin_words : 1), e->stream);
        if (err != cudaSuccess) TRY(cuda_fail(err, "upload"));
        e->h2d += sizeof(RunDev) * n_runs + sizeof(double) * (h_beta.size() + h_wt.size()) +
                  sizeof(unsigned long long) * h_thr.size();
        // host tables must outlive the asynchronous copies
        err = cudaStreamSynchronize(e->stream);
        if (err != cudaSuccess) TRY(cuda_fail(err, "upload sync"));
    }
    e->rec_count = rec;
    e->qh_count = qh;
    e->launches_per_tick = 2 + e->groups.size() + (e->q_runs.empty() ? 0 : 1);
    TRY(enqueue_init(e));
    *out = e;
    return PA_OK;
fail:
#undef TRY
    pa_destroy(e);
    return s;
}

pa_status pa_reset(pa_engine *e)
{
    if (!e) return PA_ERR_INVALID_ARG;
    PA_CUDA(cudaStreamSynchronize(e->stream));
    return enqueue_init(e);
}

pa_status pa_anneal_step(pa_engine *e, uint32_t n_steps, int use_graph)
{
    if (!e) return PA_ERR_INVALID_ARG;
    if (e->latched != PA_OK) return e->latched;
    if (n_steps == 0) return PA_OK;
    bool untuned = false;
    for (auto &g : e->groups) untuned |= !g.tuned;
    if (untuned) {
        pa_status s = enqueue_tuning_tick(e);
        if (s != PA_OK) return s;
        if (--n_steps == 0) return PA_OK;
    }
    if (use_graph && !e->profiling) {
        if (!e->graph_exec) {
            PA_CUDA(cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal));
            enqueue_tick(e);
            PA_CUDA(cudaStreamEndCapture(e->stream, &e->graph));
            PA_CUDA(cudaGraphInstantiate(&e->graph_exec, e->graph, 0));
        }
        for (uint32_t k = 0; k < n_steps; ++k) PA_CUDA(cudaGraphLaunch(e->graph_exec, e->stream));
    } else {
        for (uint32_t k = 0; k < n_steps; ++k) enqueue_tick(e);
        PA_CUDA(cudaGetLastError());
    }
    e->launches += e->launches_per_tick * n_steps;
    return PA_OK;
}

pa_status pa_sync(pa_engine *e)
{
    if (!e) return PA_ERR_INVALID_ARG;
    PA_CUDA(cudaStreamSynchronize(e->stream));
    PA_CUDA(cudaGetLastError());
    return latch_device_status(e);
}

uint64_t pa_launch_count(const pa_engine *e) { return e ? e->launches : 0; }

pa_status pa_sweep_shape(const pa_engine *e, uint32_t group, uint32_t *L, uint32_t *words_per_thread,
                         uint32_t *block, uint32_t *tuned)
{
    if (!e || group >= e->groups.size() || !L || !words_per_thread || !block || !tuned) return PA_ERR_INVALID_ARG;
    const SweepGroup &g = e->groups[group];
    *L = g.L;
    *words_per_thread = g.cfg.fast ? g.cfg.WPT : 0;
    *block = g.cfg.block;
    *tuned = (g.tuned && g.candidates.size() > 1) ? 1u : 0u;
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

pa_status pa_records(pa_engine *e, uint32_t run, pa_step_record *host_out, uint32_t *host_qhist,
                     uint32_t *host_qhist_pair)
{
    if (!e || run >= e->n_runs || !host_out) return PA_ERR_INVALID_ARG;
    const RunDev &x = e->rd[run];
    if ((host_qhist || host_qhist_pair) && !x.overlap) return PA_ERR_INVALID_ARG;
    PA_CUDA(cudaMemcpyAsync(host_out, e->P.rec + x.rec_off, sizeof(pa_step_record) * x.n_beta,
                            cudaMemcpyDeviceToHost, e->stream));
    const size_t nq = (size_t)x.n_beta * (x.N + 1);
    e->d2h += sizeof(pa_step_record) * x.n_beta + sizeof(uint32_t) * nq * ((host_qhist ? 1 : 0) + (host_qhist_pair ? 1 : 0));
    if (host_qhist)
        PA_CUDA(cudaMemcpyAsync(host_qhist, e->P.qh + x.qh_off, sizeof(uint32_t) * nq, cudaMemcpyDeviceToHost, e->stream));
    if (host_qhist_pair)
        PA_CUDA(cudaMemcpyAsync(host_qhist_pair, e->P.qhp + x.qh_off, sizeof(uint32_t) * nq, cudaMemcpyDeviceToHost,
                                e->stream));
    return sync_read(e);
}

pa_status pa_measure(pa_engine *e, uint32_t run, uint32_t step, pa_step_record *host_out, uint32_t *host_qhist,
                     uint32_t *host_qhist_pair)
{
    if (!e || run >= e->n_runs || !host_out) return PA_ERR_INVALID_ARG;
    const RunDev &x = e->rd[run];
    if (step >= x.n_beta) return PA_ERR_INVALID_ARG;
    if ((host_qhist || host_qhist_pair) && !x.overlap) return PA_ERR_INVALID_ARG;
    PA_CUDA(cudaMemcpyAsync(host_out, e->P.rec + x.rec_off + step, sizeof(pa_step_record), cudaMemcpyDeviceToHost,
                            e->stream));
    const size_t n1 = x.N + 1;
    if (host_qhist)
        PA_CUDA(cudaMemcpyAsync(host_qhist, e->P.qh + x.qh_off + step * n1, sizeof(uint32_t) * n1,
                                cudaMemcpyDeviceToHost, e->stream));
    if (host_qhist_pair)
        PA_CUDA(cudaMemcpyAsync(host_qhist_pair, e->P.qhp + x.qh_off + step * n1, sizeof(uint32_t) * n1,
                                cudaMemcpyDeviceToHost, e->stream));
    return sync_read(e);
}

pa_status pa_population(pa_engine *e, uint32_t run, int8_t *host_spins, int32_t *host_E, int32_t *host_M,
                        uint32_t *host_fam, uint32_t *R_out, uint32_t *step_out)
{
    if (!e || run >= e->n_runs) return PA_ERR_INVALID_ARG;
    const RunDev &x = e->rd[run];
    RunState st;
    PA_CUDA(cudaMemcpyAsync(&st, e->P.st + run, sizeof st, cudaMemcpyDeviceToHost, e->stream));
    PA_CUDA(cudaStreamSynchronize(e->stream));
    const uint32_t b = st.step & 1u, R = st.R_cur;
    if (R_out) *R_out = R;
    if (step_out) *step_out = st.step;
    if (host_spins && R) {
        std::vector<uint32_t> words((size_t)R * x.wstride);
        PA_CUDA(cudaMemcpyAsync(words.data(), e->P.spins[b] + x.spin_off, sizeof(uint32_t) * words.size(),
                                cudaMemcpyDeviceToHost, e->stream));
        PA_CUDA(cudaStreamSynchronize(e->stream));
        const uint32_t pw = (x.N + 63) / 64;
        for (uint32_t j = 0; j < R; ++j)
            for (uint32_t n = 0; n < x.N; ++n) {
                const uint32_t c = ((n % x.L) + (n / x.L)) & 1u, k = n >> 1;
                const uint32_t word = words[(size_t)j * x.wstride + c * pw + (k >> 5)];
                host_spins[(size_t)j * x.N + n] = ((word >> (k & 31)) & 1u) ? (int8_t)1 : (int8_t)-1;
            }
    }
    if (host_E && R)
        PA_CUDA(cudaMemcpyAsync(host_E, e->P.E[b] + x.rep_off, sizeof(int32_t) * R, cudaMemcpyDeviceToHost, e->stream));
    if (host_M && R)
        PA_CUDA(cudaMemcpyAsync(host_M, e->P.M[b] + x.rep_off, sizeof(int32_t) * R, cudaMemcpyDeviceToHost, e->stream));
    if (host_fam && R)
        PA_CUDA(cudaMemcpyAsync(host_fam, e->P.fam[b] + x.rep_off, sizeof(uint32_t) * R, cudaMemcpyDeviceToHost,
                                e->stream));
    return sync_read(e);
}

static pa_status ensure_wa(pa_engine *e, size_t bytes)
{
    if (e->wa_bytes >= bytes) return PA_OK;
    if (e->wa_buf) cudaFree(e->wa_buf);
    e->wa_buf = nullptr;
    e->wa_bytes = 0;
    cudaError_t err = cudaMalloc(&e->wa_buf, bytes);
    if (err != cudaSuccess) {
        cudaGetLastError();
        return PA_ERR_OOM;
    }
    e->wa_bytes = bytes;
    return PA_OK;
}

static size_t align256(size_t x) { return (x + 255) / 256 * 256; }

pa_status pa_weighted_average_runs(pa_engine *e, const uint32_t *run_idx, uint32_t n_groups, uint32_t M,
                                   uint32_t weight_kind, pa_wavg *host_out, double *host_Pq, double *host_Pq_pair)
{
    if (!e || !run_idx || !n_groups || !M || !host_out || weight_kind > PA_WEIGHT_SIMPLE) return PA_ERR_INVALID_ARG;
    const RunDev &r0 = e->rd[run_idx[0] < e->n_runs ? run_idx[0] : 0];
    const uint32_t n_steps = r0.n_beta, N = r0.N;
    std::vector<unsigned long long> rec_off((size_t)n_groups * M), qh_off((size_t)n_groups * M);
    for (size_t k = 0; k < rec_off.size(); ++k) {
        if (run_idx[k] >= e->n_runs) return PA_ERR_INVALID_ARG;
        const RunDev &x = e->rd[run_idx[k]];
        if (x.n_beta != n_steps || x.N != N) return PA_ERR_INVALID_ARG;
        if ((host_Pq || host_Pq_pair) && !x.overlap) return PA_ERR_INVALID_ARG;
        rec_off[k] = x.rec_off;
        qh_off[k] = x.qh_off;
    }
    const size_t nGM = (size_t)n_groups * M, nP = (size_t)n_groups * n_steps * (N + 1);
    const size_t b_off = align256(sizeof(unsigned long long) * nGM);
    const size_t b_qoff = b_off + align256(sizeof(unsigned long long) * nGM);
    const size_t b_out = b_qoff + align256(sizeof(pa_wavg) * n_groups * n_steps);
    const size_t b_w = b_out + align256(sizeof(double) * n_groups * n_steps * M);
    const size_t b_pq = b_w + align256(host_Pq ? sizeof(double) * nP : 0);
    const size_t total = b_pq + align256(host_Pq_pair ? sizeof(double) * nP : 0);
    pa_status s = ensure_wa(e, total);
    if (s != PA_OK) return s;
    char *base = static_cast<char *>(e->wa_buf);
    auto *d_roff = reinterpret_cast<unsigned long long *>(base);
    auto *d_qoff = reinterpret_cast<unsigned long long *>(base + b_off);
    auto *d_out = reinterpret_cast<pa_wavg *>(base + b_qoff);
    auto *d_w = reinterpret_cast<double *>(base + b_out);
    double *d_pq = host_Pq ? reinterpret_cast<double *>(base + b_w) : nullptr;
    double *d_pqp = host_Pq_pair ? reinterpret_cast<double *>(base + b_pq) : nullptr;
    PA_CUDA(cudaMemcpyAsync(d_roff, rec_off.data(), sizeof(unsigned long long) * nGM, cudaMemcpyHostToDevice, e->stream));
    PA_CUDA(cudaMemcpyAsync(d_qoff, qh_off.data(), sizeof(unsigned long long) * nGM, cudaMemcpyHostToDevice, e->stream));
    timed_launch(e, PA_K_WAVG, [&] {
        launch_wavg(e->P.rec, d_roff, e->P.qh, e->P.qhp, d_qoff, n_groups, M, n_steps, N, weight_kind, d_out, d_w,
                    d_pq, d_pqp, e->stream);
    });
    e->launches += 1 + ((d_pq || d_pqp) ? 1 : 0);
    e->h2d += 2 * sizeof(unsigned long long) * nGM;
    e->d2h += sizeof(pa_wavg) * n_groups * n_steps + sizeof(double) * nP * ((host_Pq ? 1 : 0) + (host_Pq_pair ? 1 : 0));
    PA_CUDA(cudaGetLastError());
    PA_CUDA(cudaMemcpyAsync(host_out, d_out, sizeof(pa_wavg) * n_groups * n_steps, cudaMemcpyDeviceToHost, e->stream));
    if (host_Pq) PA_CUDA(cudaMemcpyAsync(host_Pq, d_pq, sizeof(double) * nP, cudaMemcpyDeviceToHost, e->stream));
    if (host_Pq_pair)
        PA_CUDA(cudaMemcpyAsync(host_Pq_pair, d_pqp, sizeof(double) * nP, cudaMemcpyDeviceToHost, e->stream));
    return pa_sync(e);
}

pa_status pa_weighted_average(const pa_step_record *recs, const uint32_t *qhist, const uint32_t *qhist_pair,
                              uint32_t M, uint32_t n_steps, uint32_t N, uint32_t weight_kind, pa_wavg *out,
                              double *Pq, double *Pq_pair, void *cuda_stream)
{
    if (!recs || !M || !n_steps || !N || !out || weight_kind > PA_WEIGHT_SIMPLE) return PA_ERR_INVALID_ARG;
    if ((Pq && !qhist) || (Pq_pair && !qhist_pair)) return PA_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const size_t nr = (size_t)M * n_steps, nq = nr * (N + 1), nP = (size_t)n_steps * (N + 1);
    const size_t b_rec = align256(sizeof(pa_step_record) * nr);
    const size_t b_qh = b_rec + align256(qhist ? sizeof(uint32_t) * nq : 0);
    const size_t b_qhp = b_qh + align256(qhist_pair ? sizeof(uint32_t) * nq : 0);
    const size_t b_off = b_qhp + align256(sizeof(unsigned long long) * M);
    const size_t b_qoff = b_off + align256(sizeof(unsigned long long) * M);
    const size_t b_out = b_qoff + align256(sizeof(pa_wavg) * n_steps);
    const size_t b_w = b_out + align256(sizeof(double) * n_steps * M);
    const size_t b_pq = b_w + align256(Pq ? sizeof(double) * nP : 0);
    const size_t total = b_pq + align256(Pq_pair ? sizeof(double) * nP : 0);
    char *base = nullptr;
    cudaError_t err = cudaMalloc(&base, total);
    if (err != cudaSuccess) {
        cudaGetLastError();
        return PA_ERR_OOM;
    }
    pa_status s = PA_OK;
    std::vector<unsigned long long> roff(M), qoff(M);
    for (uint32_t m = 0; m < M; ++m) {
        roff[m] = (unsigned long long)m * n_steps;
        qoff[m] = (unsigned long long)m * n_steps * (N + 1);
    }
    auto *d_rec = reinterpret_cast<pa_step_record *>(base);
    auto *d_qh = qhist ? reinterpret_cast<uint32_t *>(base + b_rec) : nullptr;
    auto *d_qhp = qhist_pair ? reinterpret_cast<uint32_t *>(base + b_qh) : nullptr;
    auto *d_roff = reinterpret_cast<unsigned long long *>(base + b_qhp);
    auto *d_qoff = reinterpret_cast<unsigned long long *>(base + b_off);
    auto *d_out = reinterpret_cast<pa_wavg *>(base + b_qoff);
    auto *d_w = reinterpret_cast<double *>(base + b_out);
    double *d_pq = Pq ? reinterpret_cast<double *>(base + b_w) : nullptr;
    double *d_pqp = Pq_pair ? reinterpret_cast<double *>(base + b_pq) : nullptr;
    do {
        if ((err = cudaMemcpyAsync(d_rec, recs, sizeof(pa_step_record) * nr, cudaMemcpyHostToDevice, st))) break;
        if (qhist && (err = cudaMemcpyAsync(d_qh, qhist, sizeof(uint32_t) * nq, cudaMemcpyHostToDevice, st))) break;
        if (qhist_pair && (err = cudaMemcpyAsync(d_qhp, qhist_pair, sizeof(uint32_t) * nq, cudaMemcpyHostToDevice, st)))
            break;
        if ((err = cudaMemcpyAsync(d_roff, roff.data(), sizeof(unsigned long long) * M, cudaMemcpyHostToDevice, st))) break;
        if ((err = cudaMemcpyAsync(d_qoff, qoff.data(), sizeof(unsigned long long) * M, cudaMemcpyHostToDevice, st))) break;
        launch_wavg(d_rec, d_roff, d_qh, d_qhp, d_qoff, 1, M, n_steps, N, weight_kind, d_out, d_w, d_pq, d_pqp, st);
        if ((err = cudaGetLastError())) break;
        if ((err = cudaMemcpyAsync(out, d_out, sizeof(pa_wavg) * n_steps, cudaMemcpyDeviceToHost, st))) break;
        if (Pq && (err = cudaMemcpyAsync(Pq, d_pq, sizeof(double) * nP, cudaMemcpyDeviceToHost, st))) break;
        if (Pq_pair && (err = cudaMemcpyAsync(Pq_pair, d_pqp, sizeof(double) * nP, cudaMemcpyDeviceToHost, st))) break;
        err = cudaStreamSynchronize(st);
    } while (0);
    if (err != cudaSuccess) s = cuda_fail(err, "pa_weighted_average");
    cudaFree(base);
    return s;
}

}  // extern "C"
