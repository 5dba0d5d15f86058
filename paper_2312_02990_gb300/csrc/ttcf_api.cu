// ttcf_api.cu -- host implementation of the C ABI declared in ttcf.h.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <functional>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "ttcf_confined.h"
#include "ttcf_cv.h"
#include "ttcf_internal.h"

using namespace ttcf;

namespace {

constexpr double RC_WCA = 1.1224620483093730;   // 2^(1/6)

thread_local std::string g_create_error;

struct BatchHost {
    int N = 0, M = 0, G = 0, S = 0;
    int n_obs = 1;                        // observables per sample
    bool confined = false;                // Example 2 batch (ttcf_confined.cu)
    bool elong = false;                   // planar elongational flow (ttcf_elong.cu)
    int ncmax[3] = {0, 0, 0};             // elongational list-cell bound per axis
    double eskin = 0.0;                   // elongational Verlet skin
    int maps[MAX_MAPS] = {};
    double L[3] = {0, 0, 0};
    double V = 0, Q = 0, gT = 0;
    int nc[3] = {0, 0, 0}, ncell = 0;     // list cells, width >= r_c + skin
    int snc[3] = {0, 0, 0}, sncell = 0;   // spawn cells, width >= r_c
    long long d0 = 0;
    int variant = 0, threads = 256;
    double skin = DEFAULT_SKIN;
    std::vector<double> gamma;
    unsigned long long *mothers = nullptr;
    double *m_alpha = nullptr, *gamma_d = nullptr, *B = nullptr, *Omega = nullptr;
    int *status = nullptr;
    unsigned long long *pairs = nullptr;
    unsigned int *rebuilds = nullptr;
    double *scal = nullptr;
    unsigned long long *state = nullptr;
    double *feat = nullptr;
    // confined system
    int *types = nullptr;
    double *lattice = nullptr;
    double A = 0, rc = 0, k_tether = 0, c_ff = 0, c_wf = 0, c_ww = 0, half_h = 0;
    int ww_on = 0;
    double inner_y[2] = {0, 0};          // inner wall layers (see ConfBatchDev)
    int n_inner[2] = {0, 0};              // atoms in each inner wall layer
    // reduction
    bool reduced = false;
    double *Y = nullptr, *Dg = nullptr, *J = nullptr, *Og = nullptr, *valid = nullptr, *out = nullptr;
    long long D() const { return (long long)G * M; }
};

}  // namespace

struct TunedEntry { int N; int variant; double skin; double cell_frac; };

// Default cell width of the bulk list build, in units of r_c + skin
// (measured fastest for N = 2048 among r_l/2, 2r_l/3 and r_l).
constexpr double DEFAULT_CELL_FRAC = 2.0 / 3.0;

// The trained control-variate network (device buffers owned by the context).
struct CvModel {
    bool trained = false;
    float *w = nullptr, *m = nullptr, *v = nullptr;
    __nv_bfloat16 *wb = nullptr;
    double *fstats = nullptr;   // [CV_NF][2]
    double *zstats = nullptr;   // [2]
    double c = 0.0;
    int N = 0;
    double L[3] = {0, 0, 0};
};

struct ttcf_ctx {
    ttcf_config cfg;
    std::string err;
    cudaStream_t st = nullptr;
    int device = 0, nsm = 0, smem_optin = 0, smem_per_sm = 0;
    double skin = DEFAULT_SKIN;
    std::vector<BatchHost> batches;
    std::vector<TunedEntry> tuned;   // autotuner results per atom count
    CvModel cv;
    std::vector<void *> allocs;
    long long total_d = 0;
    int steps_done = 0;
    bool ran = false;
    int *h_abort = nullptr, *d_abort = nullptr;
    cudaStream_t cap_st = nullptr;   // private stream for CUDA-graph capture
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    double ms_spawn_pending = 0.0;   // spawn-kernel time not yet reported by a ttcf_run
    ttcf_stats stats;
    // launch tables, rebuilt when batches change
    bool tables_ok = false;
    BatchDev *d_batches = nullptr;
    int *d_dbatch = nullptr, *d_work = nullptr, *d_queue = nullptr;

};

namespace {

ttcf_status fail(ttcf_ctx *c, ttcf_status s, const std::string &msg) {
    if (c) c->err = msg; else g_create_error = msg;
    return s;
}

ttcf_status cuda_fail(ttcf_ctx *c, cudaError_t e, const char *where) {
    cudaGetLastError();   // clear a non-sticky error so later launch checks are not confused
    return fail(c, TTCF_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// An event that must be waited on or timed after a graph launch: inside a
// stream capture it has to become an external event-record node.
cudaError_t record_event(cudaEvent_t ev, cudaStream_t st, bool capturing) {
    return capturing ? cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal)
                     : cudaEventRecord(ev, st);
}

#define CK(call)                                                     \
    do {                                                             \
        cudaError_t _e = (call);                                     \
        if (_e != cudaSuccess) return cuda_fail(ctx, _e, #call);     \
    } while (0)

void *dev_alloc_raw(ttcf_ctx *ctx, size_t bytes) {
    if (bytes == 0) bytes = 16;
    void *p = nullptr;
    if (ctx->cfg.dev_alloc) {
        p = ctx->cfg.dev_alloc(bytes, ctx->cfg.stream, ctx->cfg.alloc_user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    return p;
}

void dev_free_raw(ttcf_ctx *ctx, void *p) {
    if (!p) return;
    if (ctx->cfg.dev_free) ctx->cfg.dev_free(p, ctx->cfg.stream, ctx->cfg.alloc_user);
    else cudaFree(p);
}

// Scoped set of device allocations; `keep` hands them to the context.
struct Pool {
    ttcf_ctx *ctx;
    std::vector<void *> ptrs;
    bool oom = false;
    explicit Pool(ttcf_ctx *c) : ctx(c) {}
    template <class T> T *get(size_t count) {
        void *p = dev_alloc_raw(ctx, count * sizeof(T));
        if (!p) { oom = true; return nullptr; }
        ptrs.push_back(p);
        return (T *)p;
    }
    void keep() { ctx->allocs.insert(ctx->allocs.end(), ptrs.begin(), ptrs.end()); ptrs.clear(); }
    ~Pool() {
        if (!ptrs.empty()) cudaStreamSynchronize(ctx->st);
        for (void *p : ptrs) dev_free_raw(ctx, p);
    }
};


// Launch variant, block size and Verlet skin for a daughter of N atoms:
// explicit configuration first, then the autotuner's result for this N,
// then the default table.
ttcf_status choose_class(ttcf_ctx *ctx, int N, int force_variant, double force_skin,
                         int &variant, int &threads, double &skin) {
    const ttcf_config &cf = ctx->cfg;
    const TunedEntry *tu = nullptr;
    for (auto &e : ctx->tuned) if (e.N == N) tu = &e;
    if (force_variant >= 0) variant = force_variant;
    else if (cf.kernel_variant > 0) variant = cf.kernel_variant - 1;
    else if (tu) variant = tu->variant;
    else variant = default_variant(N);
    if (force_skin > 0) skin = force_skin;
    else if (cf.skin > 0) skin = cf.skin;
    else if (tu) skin = tu->skin;
    else skin = DEFAULT_SKIN;
    if (variant < 0 || variant >= N_VARIANTS) return fail(ctx, TTCF_E_INVALID, "kernel_variant out of range");
    const Variant v = variant_of(variant);
    int t = cf.block_threads > 0 ? cf.block_threads : (N + v.apt - 1) / v.apt;
    t = (t + 31) / 32 * 32;
    if (t > v.maxt || t * v.apt < N)
        return fail(ctx, TTCF_E_INVALID, "kernel_variant/block_threads cannot hold n_atoms");
    threads = t;
    return TTCF_OK;
}

// Cells of the neighbour build: width `frac` r_l (finer cells: fewer
// candidates but more, shorter and more divergent rows per atom), or the
// next coarser of {2r_l/3, r_l} whose shared memory still lets the variant
// reach its target number of resident CTAs per SM.
void pick_cells(ttcf_ctx *ctx, BatchHost &b, double rl, double frac) {
    const bool mixed = ctx->cfg.precision == TTCF_MIXED;
    const Variant v = variant_of(b.variant);
    const double fracs[3] = {frac, std::max(frac, 2.0 / 3.0), 1.0};
    for (int f = 0; f < 3; f++) {
        int nc[3];
        for (int k = 0; k < 3; k++) nc[k] = std::max(3, (int)floor(b.L[k] / (rl * fracs[f])));
        const int ncell = nc[0] * nc[1] * nc[2];
        const size_t sm = daughter_smem_bytes(mixed, b.N, ncell, false, !plo_global(mixed, b.variant));
        if (f == 2 || (size_t)v.minb * (sm + 1024) <= (size_t)ctx->smem_per_sm) {
            for (int k = 0; k < 3; k++) b.nc[k] = nc[k];
            b.ncell = ncell;
            return;
        }
    }
}

// Allocate a batch, copy its mothers and run the spawn kernel.
ttcf_status make_batch(ttcf_ctx *ctx, Pool &pool, BatchHost &b, int N, const double box[3], int G,
                       const double *soa, const double *alpha, const double *gamma,
                       int is_dev, const int *maps, int M, int S, double delta0,
                       int force_variant = -1, double force_skin = -1.0,
                       double force_frac = -1.0) {
    const ttcf_config &cf = ctx->cfg;
    if (N < 4 || N > 4096) return fail(ctx, TTCF_E_INVALID, "n_atoms must be in [4, 4096]");
    if (G <= 0) return fail(ctx, TTCF_E_INVALID, "n_mothers must be positive");
    if (!soa) return fail(ctx, TTCF_E_INVALID, "mother_soa is NULL");
    {
        ttcf_status cs = choose_class(ctx, N, force_variant, force_skin, b.variant, b.threads, b.skin);
        if (cs != TTCF_OK) return cs;
    }
    const double rl = RC_WCA + b.skin;
    for (int k = 0; k < 3; k++) {
        if (!(box[k] > 0) || !isfinite(box[k])) return fail(ctx, TTCF_E_INVALID, "box edges must be positive");
        if (box[k] < 3.0 * rl)
            return fail(ctx, TTCF_E_INVALID, "box edge shorter than 3*(r_c+skin): system too small");
    }
    for (int k = 0; k < M; k++)
        if (map_swaps_xz(maps[k]) && !(fabs(box[0] - box[2]) <= 1e-12 * box[0]))
            return fail(ctx, TTCF_E_INVALID, "the x <-> z exchange mappings need L_x = L_z");
    b.N = N; b.G = G; b.M = M; b.S = S;
    for (int k = 0; k < M; k++) b.maps[k] = maps[k];
    b.V = box[0] * box[1] * box[2];
    for (int k = 0; k < 3; k++) {
        b.L[k] = box[k];
        b.snc[k] = (int)floor(box[k] / RC_WCA);
    }
    {
        double frac = DEFAULT_CELL_FRAC;
        for (auto &e : ctx->tuned) if (e.N == N) frac = e.cell_frac;
        if (cf.cell_frac > 0) frac = cf.cell_frac;
        if (force_frac > 0) frac = force_frac;
        pick_cells(ctx, b, rl, frac);
    }
    b.sncell = b.snc[0] * b.snc[1] * b.snc[2];
    const double g = cf.dof_mode == 1 ? 3.0 * N - 3.0 : 3.0 * N;
    b.Q = g * cf.T * cf.tau_T * cf.tau_T;
    b.gT = g * cf.T;

    // host copies of gamma (needed for viscosity) and the device arrays
    b.gamma.resize(G);
    std::vector<double> alpha_h(G, 0.0);
    if (is_dev) {
        if (gamma) CK(cudaMemcpy(b.gamma.data(), gamma, sizeof(double) * G, cudaMemcpyDeviceToHost));
        else std::fill(b.gamma.begin(), b.gamma.end(), 0.0);
        if (alpha) CK(cudaMemcpy(alpha_h.data(), alpha, sizeof(double) * G, cudaMemcpyDeviceToHost));
    } else {
        for (int k = 0; k < G; k++) b.gamma[k] = gamma ? gamma[k] : 0.0;
        if (alpha) for (int k = 0; k < G; k++) alpha_h[k] = alpha[k];
    }
    for (int k = 0; k < G; k++)
        if (!isfinite(b.gamma[k]) || !isfinite(alpha_h[k]))
            return fail(ctx, TTCF_E_INVALID, "non-finite shear rate or alpha");
    const long long D = b.D();
    const size_t slots = (size_t)G * 6 * N;
    b.mothers = pool.get<unsigned long long>(slots);
    b.m_alpha = pool.get<double>(G);
    b.gamma_d = pool.get<double>(G);
    b.B = pool.get<double>((size_t)D * S);
    b.Omega = pool.get<double>(D);
    b.status = pool.get<int>(D);
    b.pairs = pool.get<unsigned long long>(D);
    b.rebuilds = pool.get<unsigned int>(D);
    b.scal = pool.get<double>((size_t)D * 4);
    b.feat = pool.get<double>((size_t)G * FEAT_RAW);
    if (pool.oom) return fail(ctx, TTCF_E_OOM, "device allocation failed (batch)");
    cudaStream_t st = ctx->st;
    CK(cudaMemcpyAsync(b.m_alpha, alpha_h.data(), sizeof(double) * G, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(b.gamma_d, b.gamma.data(), sizeof(double) * G, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(b.B, 0, sizeof(double) * D * S, st));
    CK(cudaMemsetAsync(b.status, 0, sizeof(int) * D, st));
    CK(cudaMemsetAsync(b.pairs, 0, sizeof(unsigned long long) * D, st));
    CK(cudaMemsetAsync(b.rebuilds, 0, sizeof(unsigned int) * D, st));
    CK(cudaMemsetAsync(b.scal, 0, sizeof(double) * D * 4, st));

    // the FP64 mother states on the device (temporary)
    Pool tmp(ctx);
    const double *src = soa;
    if (!is_dev) {
        double *s = tmp.get<double>(slots);
        if (tmp.oom) return fail(ctx, TTCF_E_OOM, "device allocation failed (mother copy)");
        CK(cudaMemcpyAsync(s, soa, sizeof(double) * slots, cudaMemcpyHostToDevice, st));
        src = s;
    }
    SpawnArgs sa;
    memset(&sa, 0, sizeof(sa));
    sa.N = N; sa.M = M; sa.G = G;
    for (int k = 0; k < MAX_MAPS; k++) sa.maps[k] = b.maps[k];
    for (int k = 0; k < 3; k++) { sa.nc[k] = b.snc[k]; sa.L[k] = b.L[k]; }
    sa.ncell = b.sncell;
    sa.V = b.V; sa.T = cf.T;
    sa.mixed = cf.precision == TTCF_MIXED;
    sa.src = src; sa.gamma = b.gamma_d; sa.mothers = b.mothers;
    sa.B = b.B; sa.S = S; sa.Omega = b.Omega; sa.feat = b.feat; sa.delta = delta0;
    sa.elong = b.elong ? 1 : 0;
    CK(cudaEventRecord(ctx->ev[2], st));
    CK(launch_spawn(sa, st));
    CK(cudaEventRecord(ctx->ev[3], st));
    CK(cudaStreamSynchronize(st));   // before the temporary copy is released
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev[2], ctx->ev[3]);
    ctx->ms_spawn_pending += ms;
    return TTCF_OK;
}

BatchDev to_dev(const BatchHost &b) {
    BatchDev d;
    memset(&d, 0, sizeof(d));
    d.N = b.N; d.M = b.M; d.G = b.G; d.S = b.S;
    for (int k = 0; k < MAX_MAPS; k++) d.maps[k] = b.maps[k];
    for (int k = 0; k < 3; k++) { d.nc[k] = b.nc[k]; d.L[k] = b.L[k]; }
    d.ncell = b.ncell;
    d.V = b.V; d.Q = b.Q; d.gT = b.gT; d.d0 = b.d0;
    d.skin = (float)b.skin;
    d.mothers = b.mothers; d.m_alpha = b.m_alpha; d.gamma = b.gamma_d;
    d.B = b.B; d.Omega = b.Omega; d.status = b.status; d.pairs = b.pairs;
    d.rebuilds = b.rebuilds; d.scal = b.scal; d.state = b.state;
    return d;
}

struct ClassLaunch {
    int variant, threads, nmax, ncellmax, grid, cpos;
    size_t smem;
    std::vector<int> work;
};

// Group the batches' daughters by launch class (apt, threads).
std::vector<ClassLaunch> plan_classes(ttcf_ctx *ctx, std::vector<BatchHost *> &bs) {
    std::vector<ClassLaunch> cls;
    for (BatchHost *b : bs) {
        ClassLaunch *c = nullptr;
        for (auto &x : cls) if (x.variant == b->variant && x.threads == b->threads) c = &x;
        if (!c) { cls.push_back({b->variant, b->threads, 0, 0, 0, 0, 0, {}}); c = &cls.back(); }
        c->nmax = std::max(c->nmax, b->N);
        c->ncellmax = std::max(c->ncellmax, b->ncell);
        for (long long k = 0; k < b->D(); k++) c->work.push_back((int)(b->d0 + k));
    }
    const bool mixed = ctx->cfg.precision == TTCF_MIXED;
    for (auto &c : cls) {
        const bool plo_smem = !plo_global(mixed, c.variant);
        c.smem = daughter_smem_bytes(mixed, c.nmax, c.ncellmax, false, plo_smem);
        c.grid = 0;
        c.cpos = 0;
        if (c.smem > (size_t)ctx->smem_optin) continue;   // rejected by the caller
        int nb = daughter_occupancy(mixed, c.variant, c.threads, c.smem);
        {   // the cell-ordered list build where its larger shared memory keeps
            // the variant's resident CTAs per SM
            const size_t s2 = daughter_smem_bytes(mixed, c.nmax, c.ncellmax, true, plo_smem);
            if (s2 <= (size_t)ctx->smem_optin) {
                const int nb2 = daughter_occupancy(mixed, c.variant, c.threads, s2);
                if (nb2 >= 1 && nb2 >= std::min(nb, variant_of(c.variant).minb)) {
                    c.cpos = 1; c.smem = s2; nb = nb2;
                }
            }
        }
        if (nb < 1) nb = 1;
        c.grid = (int)std::min<long long>((long long)c.work.size(), (long long)nb * ctx->nsm);
        if (c.grid < 1) c.grid = 1;
    }
    return cls;
}

// One persistent launch per class over the given batches (device tables
// built in `pool`).  `proto` carries the run-wide fields.
ttcf_status launch_batches(ttcf_ctx *ctx, Pool &pool, std::vector<BatchHost *> &bs,
                           RunArgs proto, int &launches, cudaEvent_t ev_begin = nullptr,
                           cudaEvent_t ev_end = nullptr,
                           const std::function<ttcf_status()> &tail = nullptr) {
    const bool mixed = ctx->cfg.precision == TTCF_MIXED;
    if (bs.empty()) return TTCF_OK;
    long long dmax = 0;
    for (BatchHost *b : bs) dmax = std::max(dmax, b->d0 + b->D());
    std::vector<BatchDev> hb;
    std::vector<int> dbatch((size_t)dmax, 0);
    for (size_t k = 0; k < bs.size(); k++) {
        hb.push_back(to_dev(*bs[k]));
        for (long long d = 0; d < bs[k]->D(); d++) dbatch[(size_t)(bs[k]->d0 + d)] = (int)k;
    }
    std::vector<ClassLaunch> cls = plan_classes(ctx, bs);
    for (auto &c : cls)
        if (c.grid == 0)
            return fail(ctx, TTCF_E_INVALID, "a daughter needs more shared memory than a CTA has "
                                             "(n_atoms too large for this skin)");
    BatchDev *d_b = pool.get<BatchDev>(hb.size());
    int *d_db = pool.get<int>(dbatch.size());
    int *d_q = pool.get<int>(cls.size());
    if (pool.oom) return fail(ctx, TTCF_E_OOM, "device allocation failed (tables)");
    cudaStream_t st = ctx->st;
    CK(cudaMemcpyAsync(d_b, hb.data(), sizeof(BatchDev) * hb.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_db, dbatch.data(), sizeof(int) * dbatch.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(d_q, 0, sizeof(int) * cls.size(), st));
    std::vector<int *> d_work(cls.size());
    std::vector<unsigned int *> d_nbr(cls.size());
    std::vector<float4 *> d_plo(cls.size(), nullptr);
    const bool mixed_run = ctx->cfg.precision == TTCF_MIXED;
    for (size_t k = 0; k < cls.size(); k++) {
        d_work[k] = pool.get<int>(cls[k].work.size());
        d_nbr[k] = pool.get<unsigned int>((size_t)cls[k].grid * NBR_WORDS * cls[k].nmax);
        if (plo_global(mixed_run, cls[k].variant))
            d_plo[k] = pool.get<float4>((size_t)cls[k].grid * cls[k].nmax);
        if (pool.oom) return fail(ctx, TTCF_E_OOM, "device allocation failed (work lists)");
        CK(cudaMemcpyAsync(d_work[k], cls[k].work.data(), sizeof(int) * cls[k].work.size(),
                           cudaMemcpyHostToDevice, st));
    }
    // classes run concurrently on forked streams joined back into st; with
    // use_graph the whole fork/join (and `tail`, e.g. the reductions) is
    // captured once and launched as one CUDA graph
    std::vector<cudaStream_t> side(cls.size(), st);
    std::vector<cudaEvent_t> done(cls.size(), nullptr);
    cudaEvent_t fork = nullptr;
    if (cls.size() > 1) {
        CK(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
        for (size_t k = 1; k < cls.size(); k++) {
            CK(cudaStreamCreateWithFlags(&side[k], cudaStreamNonBlocking));
            CK(cudaEventCreateWithFlags(&done[k], cudaEventDisableTiming));
        }
    }
    std::vector<cudaStream_t> owned(side.begin() + (side.empty() ? 0 : 1), side.end());
    auto cleanup = [&]() {
        for (auto e : done) if (e) cudaEventDestroy(e);
        if (fork) cudaEventDestroy(fork);
        for (cudaStream_t x : owned) if (x) cudaStreamDestroy(x);
        owned.clear();
    };
    // The caller's stream may be the legacy default stream, which cannot be
    // captured: capture on the context's own stream, launch on the caller's.
    const bool graph = ctx->cfg.use_graph != 0;
    const cudaStream_t user_st = st;
    cudaGraph_t g = nullptr;
    if (graph) {
        if (!ctx->cap_st) CK(cudaStreamCreateWithFlags(&ctx->cap_st, cudaStreamNonBlocking));
        st = ctx->cap_st;
        for (size_t k = 0; k < side.size(); k++) if (k == 0 || side[k] == user_st) side[k] = st;
        ctx->st = st;   // work issued by `tail` goes into the capture too
        cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            ctx->st = user_st;
            cleanup();
            return cuda_fail(ctx, e, "cudaStreamBeginCapture");
        }
    }
    auto body = [&]() -> ttcf_status {
        if (ev_begin) CK(record_event(ev_begin, st, graph));
        if (fork) {
            CK(cudaEventRecord(fork, st));
            for (size_t k = 1; k < cls.size(); k++) CK(cudaStreamWaitEvent(side[k], fork, 0));
        }
        for (size_t k = 0; k < cls.size(); k++) {
            RunArgs a = proto;
            a.batches = d_b; a.dbatch = d_db; a.work = d_work[k];
            a.n_work = (int)cls[k].work.size();
            a.queue = d_q + k;
            a.nbr = d_nbr[k]; a.nmax = cls[k].nmax; a.ncellmax = cls[k].ncellmax;
            a.plo_g = d_plo[k];
            a.cpos = cls[k].cpos;
            CK(launch_daughters(mixed, cls[k].variant, a, cls[k].threads, cls[k].grid, cls[k].smem, side[k]));
            launches++;
            ctx->stats.block_threads = std::max(ctx->stats.block_threads, cls[k].threads);
        }
        for (size_t k = 1; k < cls.size(); k++) {
            CK(cudaEventRecord(done[k], side[k]));
            CK(cudaStreamWaitEvent(st, done[k], 0));
        }
        if (ev_end) CK(record_event(ev_end, st, graph));
        if (tail) {
            ttcf_status ts = tail();
            if (ts != TTCF_OK) return ts;
        }
        return TTCF_OK;
    };
    ttcf_status bs_ = body();
    if (graph) {
        cudaError_t e = cudaStreamEndCapture(st, &g);
        ctx->st = user_st;
        st = user_st;
        if (bs_ == TTCF_OK && e != cudaSuccess) bs_ = cuda_fail(ctx, e, "cudaStreamEndCapture");
        if (bs_ == TTCF_OK) {
            cudaGraphExec_t ex = nullptr;
            e = cudaGraphInstantiate(&ex, g, 0);
            if (e == cudaSuccess) e = cudaGraphLaunch(ex, user_st);
            if (ex) cudaGraphExecDestroy(ex);   // freed once the launch completes
            if (e != cudaSuccess) bs_ = cuda_fail(ctx, e, "CUDA graph launch");
        }
        if (g) cudaGraphDestroy(g);
    }
    if (bs_ != TTCF_OK) { cudaStreamSynchronize(st); cleanup(); return bs_; }
    // without a graph the side streams and events are released once st has
    // passed them; a captured graph no longer refers to them
    if (fork && !graph) CK(cudaStreamSynchronize(st));
    cleanup();
    return TTCF_OK;
}

// Wait for the stream with the context's wall-clock limit.
ttcf_status wait_with_timeout(ttcf_ctx *ctx, cudaEvent_t ev) {
    const double lim = ctx->cfg.timeout_s;
    if (lim <= 0) { CK(cudaEventSynchronize(ev)); return TTCF_OK; }
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t q = cudaEventQuery(ev);
        if (q == cudaSuccess) return TTCF_OK;
        if (q != cudaErrorNotReady) return cuda_fail(ctx, q, "cudaEventQuery");
        double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > lim) {
            *(volatile int *)ctx->h_abort = 1;   // daughters stop within 64 steps
            CK(cudaEventSynchronize(ev));
            return fail(ctx, TTCF_E_TIMEOUT, "ttcf_run exceeded timeout_s; daughters aborted");
        }
        std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
}

ttcf_status ensure_reduce_buffers(ttcf_ctx *ctx, BatchHost &b) {
    if (b.out) return TTCF_OK;
    Pool p(ctx);
    b.Y = p.get<double>((size_t)b.n_obs * b.G * b.S);
    b.Dg = p.get<double>((size_t)b.n_obs * b.G * b.S);
    b.J = p.get<double>((size_t)b.n_obs * b.G * b.S);
    b.Og = p.get<double>(b.G + 2);   // + <Omega(0)> and the valid-group count
    b.valid = p.get<double>(b.G);
    b.out = p.get<double>((size_t)9 * b.n_obs * b.S);
    if (p.oom) return fail(ctx, TTCF_E_OOM, "device allocation failed (reduction)");
    p.keep();
    return TTCF_OK;
}

ttcf_status reduce_batch(ttcf_ctx *ctx, BatchHost &b) {
    if (b.reduced) return TTCF_OK;
    ttcf_status rs = ensure_reduce_buffers(ctx, b);
    if (rs != TTCF_OK) return rs;
    ReduceArgs r;
    r.M = b.M; r.G = b.G; r.S = b.S; r.n_obs = b.n_obs;
    r.B = b.B; r.Omega = b.Omega; r.status = b.status;
    r.ds = ctx->cfg.sample_every * ctx->cfg.dt;
    r.Y = b.Y; r.Dg = b.Dg; r.J = b.J; r.Og = b.Og; r.valid = b.valid; r.out = b.out;
    CK(launch_reduce(r, ctx->st));
    b.reduced = true;
    return TTCF_OK;
}

}  // namespace

void ttcf::set_global_error(const char *msg) { g_create_error = msg; }

namespace {

BatchHost *get_batch(ttcf_ctx *ctx, int id) {
    if (!ctx || id < 0 || id >= (int)ctx->batches.size()) return nullptr;
    return &ctx->batches[id];
}

}  // namespace

// ======================================================= confined system ==
namespace {

// Cells of the confined list build: the finest width in {r_l/2, 2r_l/3, r_l}
// whose shared memory still fits one CTA (one daughter per SM).
bool conf_pick_cells(ttcf_ctx *ctx, BatchHost &b, double rl) {
    const double fracs[3] = {0.5, 2.0 / 3.0, 1.0};
    for (int f = 0; f < 3; f++) {
        int nc[3];
        for (int k = 0; k < 3; k++) nc[k] = std::max(1, (int)floor(b.L[k] / (rl * fracs[f])));
        const int ncell = nc[0] * nc[1] * nc[2];
        if (conf_smem_bytes(b.N, ncell) <= (size_t)ctx->smem_optin) {
            for (int k = 0; k < 3; k++) b.nc[k] = nc[k];
            b.ncell = ncell;
            return true;
        }
    }
    return false;
}

// Allocate a confined batch, copy its inputs and run the spawn kernel.
ttcf_status make_conf_batch(ttcf_ctx *ctx, Pool &pool, BatchHost &b, int N, const double box[3],
                            const int *types, const double *lattice,
                            const ttcf_confined_params &p, int G, const double *soa,
                            const double *alpha, const double *gamma, int is_dev,
                            const int *maps, int M, int S) {
    const ttcf_config &cf = ctx->cfg;
    if (N < 4 || N > CONF_NMAX) return fail(ctx, TTCF_E_INVALID, "n_atoms must be in [4, 12288]");
    if (G <= 0) return fail(ctx, TTCF_E_INVALID, "n_mothers must be positive");
    if (!soa || !types || !lattice) return fail(ctx, TTCF_E_INVALID, "NULL array");
    if (!(p.rc > 0) || !(p.k >= 0) || !(p.h > 0) || !isfinite(p.rc) || !isfinite(p.k) ||
        !isfinite(p.h) || !isfinite(p.c_ff) || !isfinite(p.c_wf) || !isfinite(p.c_ww) ||
        (p.ww_on != 0 && p.ww_on != 1))
        return fail(ctx, TTCF_E_INVALID, "bad confined parameters");
    b.confined = true;
    b.n_obs = CONF_NOBS;
    b.skin = cf.skin > 0 ? cf.skin : CONF_DEFAULT_SKIN;
    const double rl = p.rc + b.skin;
    for (int k = 0; k < 3; k++)
        if (!(box[k] > 0) || !isfinite(box[k])) return fail(ctx, TTCF_E_INVALID, "box edges must be positive");
    if (box[0] < 3.0 * rl || box[2] < 3.0 * rl)
        return fail(ctx, TTCF_E_INVALID, "Lx and Lz must be >= 3*(r_c+skin)");
    b.N = N; b.G = G; b.M = M; b.S = S;
    for (int k = 0; k < M; k++) b.maps[k] = maps[k];
    for (int k = 0; k < 3; k++) b.L[k] = box[k];
    b.V = box[0] * box[1] * box[2];
    b.A = box[0] * box[2];
    b.rc = p.rc; b.k_tether = p.k; b.c_ff = p.c_ff; b.c_wf = p.c_wf; b.c_ww = p.c_ww;
    b.ww_on = p.ww_on; b.half_h = 0.5 * p.h;
    if (!conf_pick_cells(ctx, b, rl))
        return fail(ctx, TTCF_E_INVALID, "n_atoms too large for one CTA's shared memory");
    for (int k = 0; k < 3; k++) b.snc[k] = std::max(1, (int)floor(box[k] / p.rc));
    b.sncell = b.snc[0] * b.snc[1] * b.snc[2];
    if (conf_spawn_smem_bytes(N, b.sncell) > (size_t)ctx->smem_optin)
        return fail(ctx, TTCF_E_INVALID, "too many spawn cells");

    // host copies: types (wall count), gamma, alpha
    std::vector<int> types_h(N);
    b.gamma.resize(G);
    std::vector<double> alpha_h(G, 0.0);
    if (is_dev) {
        CK(cudaMemcpy(types_h.data(), types, sizeof(int) * N, cudaMemcpyDeviceToHost));
        if (gamma) CK(cudaMemcpy(b.gamma.data(), gamma, sizeof(double) * G, cudaMemcpyDeviceToHost));
        else std::fill(b.gamma.begin(), b.gamma.end(), 0.0);
        if (alpha) CK(cudaMemcpy(alpha_h.data(), alpha, sizeof(double) * G, cudaMemcpyDeviceToHost));
    } else {
        std::copy(types, types + N, types_h.begin());
        for (int k = 0; k < G; k++) b.gamma[k] = gamma ? gamma[k] : 0.0;
        if (alpha) for (int k = 0; k < G; k++) alpha_h[k] = alpha[k];
    }
    int n_wall = 0;
    for (int t : types_h) {
        if (t < 0 || t > 2) return fail(ctx, TTCF_E_INVALID, "types must be 0, 1 or 2");
        n_wall += t != 0;
    }
    if (n_wall == 0) return fail(ctx, TTCF_E_INVALID, "no wall atoms");
    {   // the innermost layer of each wall: sites within CONF_LAYER_TOL in y of
        // the wall's site plane nearest the channel
        std::vector<double> ys(N);
        if (is_dev) CK(cudaMemcpy(ys.data(), lattice + N, sizeof(double) * N, cudaMemcpyDeviceToHost));
        else std::copy(lattice + N, lattice + 2 * (size_t)N, ys.begin());
        double ybot = -INFINITY, ytop = INFINITY;
        for (int i = 0; i < N; i++) {
            if (!isfinite(ys[i])) return fail(ctx, TTCF_E_INVALID, "non-finite tether site");
            if (types_h[i] == 1) ybot = std::max(ybot, ys[i]);
            if (types_h[i] == 2) ytop = std::min(ytop, ys[i]);
        }
        b.inner_y[0] = ybot - CONF_LAYER_TOL;
        b.inner_y[1] = ytop + CONF_LAYER_TOL;
        b.n_inner[0] = b.n_inner[1] = 0;
        for (int i = 0; i < N; i++) {
            if (types_h[i] == 1 && ys[i] >= b.inner_y[0]) b.n_inner[0]++;
            if (types_h[i] == 2 && ys[i] <= b.inner_y[1]) b.n_inner[1]++;
        }
    }
    for (int k = 0; k < G; k++)
        if (!isfinite(b.gamma[k]) || !isfinite(alpha_h[k]))
            return fail(ctx, TTCF_E_INVALID, "non-finite shear rate or alpha");
    const double g = 3.0 * n_wall;
    b.Q = g * cf.T * cf.tau_T * cf.tau_T;
    b.gT = g * cf.T;

    const long long D = b.D();
    const size_t slots = (size_t)G * 6 * N;
    b.mothers = pool.get<unsigned long long>(slots);
    b.m_alpha = pool.get<double>(G);
    b.gamma_d = pool.get<double>(G);
    b.B = pool.get<double>((size_t)D * b.n_obs * S);
    b.Omega = pool.get<double>(D);
    b.status = pool.get<int>(D);
    b.pairs = pool.get<unsigned long long>(D);
    b.rebuilds = pool.get<unsigned int>(D);
    b.types = pool.get<int>(N);
    b.lattice = pool.get<double>((size_t)3 * N);
    if (pool.oom) return fail(ctx, TTCF_E_OOM, "device allocation failed (batch)");
    cudaStream_t st = ctx->st;
    const cudaMemcpyKind kind = is_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaMemcpyAsync(b.m_alpha, alpha_h.data(), sizeof(double) * G, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(b.gamma_d, b.gamma.data(), sizeof(double) * G, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(b.types, types_h.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(b.lattice, lattice, sizeof(double) * 3 * N, kind, st));
    CK(cudaMemsetAsync(b.B, 0, sizeof(double) * D * b.n_obs * S, st));
    CK(cudaMemsetAsync(b.status, 0, sizeof(int) * D, st));
    CK(cudaMemsetAsync(b.pairs, 0, sizeof(unsigned long long) * D, st));
    CK(cudaMemsetAsync(b.rebuilds, 0, sizeof(unsigned int) * D, st));

    Pool tmp(ctx);
    const double *src = soa;
    if (!is_dev) {
        double *s = tmp.get<double>(slots);
        if (tmp.oom) return fail(ctx, TTCF_E_OOM, "device allocation failed (mother copy)");
        CK(cudaMemcpyAsync(s, soa, sizeof(double) * slots, cudaMemcpyHostToDevice, st));
        src = s;
    }
    ConfSpawnArgs sa;
    memset(&sa, 0, sizeof(sa));
    sa.N = N; sa.M = M; sa.G = G; sa.S = S; sa.n_obs = b.n_obs;
    for (int k = 0; k < 4; k++) sa.maps[k] = b.maps[k];
    for (int k = 0; k < 3; k++) { sa.nc[k] = b.snc[k]; sa.L[k] = b.L[k]; }
    sa.ncell = b.sncell;
    sa.A = b.A; sa.Tw = cf.T; sa.rc = b.rc; sa.k = b.k_tether; sa.c_wf = b.c_wf; sa.half_h = b.half_h;
    sa.inner_y[0] = b.inner_y[0]; sa.inner_y[1] = b.inner_y[1];
    sa.src = src; sa.gamma = b.gamma_d; sa.types = b.types; sa.lattice = b.lattice;
    sa.mothers = b.mothers; sa.B = b.B; sa.Omega = b.Omega;
    CK(cudaEventRecord(ctx->ev[2], st));
    CK(launch_conf_spawn(sa, st));
    CK(cudaEventRecord(ctx->ev[3], st));
    CK(cudaStreamSynchronize(st));   // before the temporary copy is released
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev[2], ctx->ev[3]);
    ctx->ms_spawn_pending += ms;
    return TTCF_OK;
}

ConfBatchDev conf_to_dev(const BatchHost &b) {
    ConfBatchDev d;
    memset(&d, 0, sizeof(d));
    d.N = b.N; d.M = b.M; d.G = b.G; d.S = b.S; d.n_obs = b.n_obs;
    for (int k = 0; k < 4; k++) d.maps[k] = b.maps[k];
    for (int k = 0; k < 3; k++) { d.nc[k] = b.nc[k]; d.L[k] = b.L[k]; }
    d.ncell = b.ncell;
    d.A = b.A; d.Q = b.Q; d.gT = b.gT;
    d.rc = b.rc; d.k = b.k_tether; d.c_ff = b.c_ff; d.c_wf = b.c_wf; d.c_ww = b.c_ww;
    d.ww_on = b.ww_on; d.half_h = b.half_h;
    d.inner_y[0] = b.inner_y[0]; d.inner_y[1] = b.inner_y[1];
    d.skin = (float)b.skin;
    d.d0 = b.d0;
    d.mothers = b.mothers; d.m_alpha = b.m_alpha; d.gamma = b.gamma_d;
    d.types = b.types; d.lattice = b.lattice;
    d.B = b.B; d.Omega = b.Omega; d.status = b.status; d.pairs = b.pairs; d.rebuilds = b.rebuilds;
    return d;
}

// One persistent launch over every daughter of the given confined batches
// (one CTA per SM, work queue), timed by ev0/ev1 on the context's stream.
ttcf_status launch_conf_batches(ttcf_ctx *ctx, Pool &pool, std::vector<BatchHost *> &bs,
                                ConfRunArgs proto, int &launches, cudaEvent_t ev0 = nullptr,
                                cudaEvent_t ev1 = nullptr) {
    long long dmax = 0;
    int nmax = 0, ncellmax = 0;
    std::vector<ConfBatchDev> hb;
    for (BatchHost *b : bs) {
        dmax = std::max(dmax, b->d0 + b->D());
        nmax = std::max(nmax, b->N);
        ncellmax = std::max(ncellmax, b->ncell);
        hb.push_back(conf_to_dev(*b));
    }
    std::vector<int> dbatch((size_t)dmax, 0), work;
    for (size_t k = 0; k < bs.size(); k++)
        for (long long d = 0; d < bs[k]->D(); d++) {
            dbatch[(size_t)(bs[k]->d0 + d)] = (int)k;
            work.push_back((int)(bs[k]->d0 + d));
        }
    const size_t smem = conf_smem_bytes(nmax, ncellmax);
    if (smem > (size_t)ctx->smem_optin)
        return fail(ctx, TTCF_E_INVALID, "confined batches need more shared memory than a CTA has");
    const int grid = (int)std::max<long long>(1, std::min<long long>((long long)work.size(), ctx->nsm));
    ConfBatchDev *d_b = pool.get<ConfBatchDev>(hb.size());
    int *d_db = pool.get<int>(dbatch.size());
    int *d_work = pool.get<int>(work.size());
    int *d_q = pool.get<int>(1);
    float4 *scratch = pool.get<float4>((size_t)grid * CONF_SCRATCH_F4 * nmax);
    uint4 *nbr = pool.get<uint4>((size_t)grid * CONF_GROUPS * nmax);
    int *ncnt = pool.get<int>((size_t)grid * nmax);
    if (pool.oom) return fail(ctx, TTCF_E_OOM, "device allocation failed (confined tables)");
    cudaStream_t st = ctx->st;
    CK(cudaMemcpyAsync(d_b, hb.data(), sizeof(ConfBatchDev) * hb.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_db, dbatch.data(), sizeof(int) * dbatch.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_work, work.data(), sizeof(int) * work.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(d_q, 0, sizeof(int), st));
    ConfRunArgs a = proto;
    a.batches = d_b; a.dbatch = d_db; a.work = d_work; a.n_work = (int)work.size();
    a.queue = d_q; a.scratch = scratch; a.nbr = nbr; a.ncnt = ncnt;
    a.nmax = nmax; a.ncellmax = ncellmax;
    if (ev0) CK(cudaEventRecord(ev0, st));
    CK(launch_confined(a, grid, smem, st));
    launches++;
    if (ev1) CK(cudaEventRecord(ev1, st));
    ctx->stats.block_threads = CONF_THREADS;
    return TTCF_OK;
}

ttcf_status run_confined(ttcf_ctx *ctx, int n_steps) {
    const ttcf_config &cf = ctx->cfg;
    if (ctx->steps_done >= cf.n_steps) return TTCF_OK;
    if (n_steps > 0 && n_steps < cf.n_steps)
        return fail(ctx, TTCF_E_INVALID, "confined daughters run all n_steps in one ttcf_run");
    ctx->ran = true;
    *(volatile int *)ctx->h_abort = 0;
    memset(&ctx->stats, 0, sizeof(ctx->stats));
    ctx->stats.ms_spawn = ctx->ms_spawn_pending;
    ctx->ms_spawn_pending = 0.0;
    for (auto &b : ctx->batches) {
        ttcf_status r = ensure_reduce_buffers(ctx, b);
        if (r != TTCF_OK) return r;
    }
    ConfRunArgs a;
    memset(&a, 0, sizeof(a));
    a.n_steps = cf.n_steps;
    a.sample_every = cf.sample_every;
    a.reset_alpha = cf.reset_alpha;
    a.dt = cf.dt;
    a.abort_flag = ctx->d_abort;
    std::vector<BatchHost *> bs;
    for (auto &b : ctx->batches) bs.push_back(&b);
    Pool pool(ctx);
    int launches = 0;
    ttcf_status s = launch_conf_batches(ctx, pool, bs, a, launches, ctx->ev[0], ctx->ev[1]);
    if (s != TTCF_OK) return s;
    CK(cudaEventRecord(ctx->ev[2], ctx->st));
    for (auto &b : ctx->batches) {
        b.reduced = false;
        s = reduce_batch(ctx, b);
        if (s != TTCF_OK) return s;
        launches += 3;
    }
    CK(cudaEventRecord(ctx->ev[3], ctx->st));
    s = wait_with_timeout(ctx, ctx->ev[3]);
    if (s != TTCF_OK && s != TTCF_E_TIMEOUT) return s;
    const bool timed_out = s == TTCF_E_TIMEOUT;
    float ms = 0.f, msr = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]);
    cudaEventElapsedTime(&msr, ctx->ev[2], ctx->ev[3]);
    ctx->stats.ms_run = ms;
    ctx->stats.ms_reduce = msr;
    ctx->stats.skin = ctx->batches[0].skin;
    ctx->steps_done = cf.n_steps;
    bool any_fail = false;
    for (auto &b : ctx->batches) {
        std::vector<int> stv(b.D());
        std::vector<unsigned long long> pr(b.D());
        std::vector<unsigned int> rb(b.D());
        CK(cudaMemcpy(stv.data(), b.status, sizeof(int) * b.D(), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(pr.data(), b.pairs, sizeof(unsigned long long) * b.D(), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(rb.data(), b.rebuilds, sizeof(unsigned int) * b.D(), cudaMemcpyDeviceToHost));
        for (long long d = 0; d < b.D(); d++) {
            any_fail |= stv[d] != 0;
            ctx->stats.pairs_interacting += (double)pr[d];
            ctx->stats.rebuilds += (double)rb[d];
        }
        ctx->stats.atom_steps += (double)b.D() * b.N * cf.n_steps;
    }
    ctx->stats.launches = launches;
    if (timed_out) return fail(ctx, TTCF_E_TIMEOUT, "ttcf_run exceeded timeout_s; daughters aborted");
    if (any_fail) return fail(ctx, TTCF_E_NUMERIC, "some daughters failed; see ttcf_group_status");
    return TTCF_OK;
}

ttcf_confined_params conf_params_or_default(const ttcf_confined_params *p) {
    ttcf_confined_params q;
    if (p) return *p;
    memset(&q, 0, sizeof(q));
    q.k = 150.0; q.rc = 2.5; q.c_ff = 1.2; q.c_wf = 0.6325; q.c_ww = 1.0; q.h = 10.0; q.ww_on = 1;
    return q;
}

// ======================================================= elongational flow ==
// Checks an elongational batch against the daughter length and sizes its
// Verlet lists and their cell grid: the box deforms as Lx(t) = Lx e^{eps t},
// Lz(t) = Lz e^{-eps t}, and the minimum image of a listed pair is unique
// while every edge stays above 2 r_l, r_l = r_c + skin; the skin is
// ELONG_SKIN, or less where the most compressed edge of the run needs it
// (at least 0.05).  The grid (cells at least r_l (1 + 1e-4) wide) is
// bounded per axis by the largest edge the run reaches.
ttcf_status elong_plan(ttcf_ctx *ctx, int N, const double box[3], const std::vector<double> &rates,
                       BatchHost &b) {
    const ttcf_config &cf = ctx->cfg;
    const double t_end = cf.n_steps * cf.dt;
    double emax = 0.0, emin = 0.0;
    for (double r : rates) {
        if (!isfinite(r)) return fail(ctx, TTCF_E_INVALID, "non-finite elongation rate");
        emax = std::max(emax, r);
        emin = std::min(emin, r);
    }
    const double lo = std::min({box[0] * exp(emin * t_end), box[1], box[2] * exp(-emax * t_end)});
    const double skin = std::min(ELONG_SKIN, 0.5 * lo - RC_WCA - 0.01);
    if (!(skin >= 0.05))
        return fail(ctx, TTCF_E_INVALID, "elongation too strong for the daughter length: a compressed "
                                         "box edge would fall below 2 (r_c + 0.06)");
    const double w = (RC_WCA + skin) * (1.0 + 1e-4);
    const double hi[3] = {box[0] * exp(emax * t_end), box[1], box[2] * exp(-emin * t_end)};
    for (int k = 0; k < 3; k++) {
        const double n = floor(hi[k] / w) + 1.0;
        if (!(n >= 1.0 && n <= 40.0)) return fail(ctx, TTCF_E_INVALID, "elongational box too large");
        b.ncmax[k] = (int)n;
    }
    const size_t smem = elong_smem_bytes(cf.precision == TTCF_MIXED, N,
                                         b.ncmax[0] * b.ncmax[1] * b.ncmax[2]);
    if (smem > (size_t)ctx->smem_optin)
        return fail(ctx, TTCF_E_INVALID, "n_atoms too large for an elongational daughter in one CTA's "
                                         "shared memory");
    b.eskin = skin;
    b.elong = true;
    return TTCF_OK;
}

// One persistent launch per elongational batch, then the reductions.
ttcf_status run_elong(ttcf_ctx *ctx, int n_steps) {
    const ttcf_config &cf = ctx->cfg;
    const int step0 = ctx->steps_done;
    if (step0 >= cf.n_steps) return TTCF_OK;
    const int step1 = (n_steps <= 0 || step0 + n_steps > cf.n_steps) ? cf.n_steps : step0 + n_steps;
    const bool save = step1 < cf.n_steps || cf.keep_state;
    if (save) {
        for (auto &b : ctx->batches) {
            if (b.state) continue;
            Pool p(ctx);
            b.state = p.get<unsigned long long>((size_t)b.D() * 6 * b.N);
            if (p.oom) return fail(ctx, TTCF_E_OOM, "device allocation failed (state)");
            p.keep();
        }
    }
    if (step0 > 0)
        for (auto &b : ctx->batches)
            if (!b.state) return fail(ctx, TTCF_E_STATE, "resume without saved state");
    const bool finishing = step1 >= cf.n_steps;
    if (finishing) {
        for (auto &b : ctx->batches) {
            ttcf_status r = ensure_reduce_buffers(ctx, b);
            if (r != TTCF_OK) return r;
        }
    }
    ctx->ran = true;
    *(volatile int *)ctx->h_abort = 0;
    memset(&ctx->stats, 0, sizeof(ctx->stats));
    ctx->stats.ms_spawn = ctx->ms_spawn_pending;
    ctx->ms_spawn_pending = 0.0;
    const bool mixed = cf.precision == TTCF_MIXED;
    int launches = 0;
    Pool scratch(ctx);
    std::vector<int> grids;
    std::vector<unsigned short *> lists;
    for (auto &b : ctx->batches) {   // Verlet list scratch of each launch
        const int g = elong_grid(mixed, b.N, b.ncmax[0] * b.ncmax[1] * b.ncmax[2], ctx->nsm, b.D());
        if (g <= 0) return fail(ctx, TTCF_E_INVALID, "an elongational daughter does not fit one CTA");
        grids.push_back(g);
        lists.push_back(scratch.get<unsigned short>((size_t)g * ELONG_CAP * b.N));
        if (scratch.oom) return fail(ctx, TTCF_E_OOM, "device allocation failed (Verlet lists)");
    }
    CK(cudaEventRecord(ctx->ev[0], ctx->st));
    for (size_t q = 0; q < ctx->batches.size(); q++) {
        BatchHost &b = ctx->batches[q];
        ElongArgs a;
        memset(&a, 0, sizeof(a));
        a.b = to_dev(b);
        a.skin = (float)b.eskin;
        a.nbr = lists[q];
        a.step0 = step0; a.step1 = step1;
        a.sample_every = cf.sample_every;
        a.fresh = step0 == 0;
        a.save_state = save ? 1 : 0;
        a.reset_alpha = cf.reset_alpha;
        for (int k = 0; k < 3; k++) a.ncmax[k] = b.ncmax[k];
        a.dt = cf.dt;
        a.abort_flag = ctx->d_abort;
        CK(launch_elong(mixed, a, grids[q], ctx->st));
        launches++;
        ctx->stats.block_threads = std::max(ctx->stats.block_threads, elong_threads(b.N));
    }
    CK(cudaEventRecord(ctx->ev[1], ctx->st));
    if (finishing) {
        CK(cudaEventRecord(ctx->ev[2], ctx->st));
        for (auto &b : ctx->batches) {
            b.reduced = false;
            ttcf_status r = reduce_batch(ctx, b);
            if (r != TTCF_OK) return r;
            launches += 3;
        }
        CK(cudaEventRecord(ctx->ev[3], ctx->st));
    }
    ttcf_status s = wait_with_timeout(ctx, finishing ? ctx->ev[3] : ctx->ev[1]);
    if (s != TTCF_OK && s != TTCF_E_TIMEOUT) return s;
    const bool timed_out = s == TTCF_E_TIMEOUT;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]);
    ctx->stats.ms_run = ms;
    ctx->stats.skin = ctx->batches[0].eskin;
    if (finishing) {
        float msr = 0.f;
        cudaEventElapsedTime(&msr, ctx->ev[2], ctx->ev[3]);
        ctx->stats.ms_reduce = msr;
    }
    ctx->steps_done = step1;
    bool any_fail = false;
    for (auto &b : ctx->batches) {
        std::vector<int> stv(b.D());
        std::vector<unsigned long long> pr(b.D());
        std::vector<unsigned int> rb(b.D());
        CK(cudaMemcpy(stv.data(), b.status, sizeof(int) * b.D(), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(pr.data(), b.pairs, sizeof(unsigned long long) * b.D(), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(rb.data(), b.rebuilds, sizeof(unsigned int) * b.D(), cudaMemcpyDeviceToHost));
        for (long long d = 0; d < b.D(); d++) {
            any_fail |= stv[d] != 0;
            ctx->stats.pairs_interacting += (double)pr[d];
            ctx->stats.rebuilds += (double)rb[d];
        }
        ctx->stats.atom_steps += (double)b.D() * b.N * (step1 - step0);
        CK(cudaMemsetAsync(b.pairs, 0, sizeof(unsigned long long) * b.D(), ctx->st));
        CK(cudaMemsetAsync(b.rebuilds, 0, sizeof(unsigned int) * b.D(), ctx->st));
    }
    ctx->stats.launches = launches;
    if (timed_out) return fail(ctx, TTCF_E_TIMEOUT, "ttcf_run exceeded timeout_s; daughters aborted");
    if (any_fail) return fail(ctx, TTCF_E_NUMERIC, "some daughters failed; see ttcf_group_status");
    return TTCF_OK;
}

}  // namespace

// =================================================================== ABI ==
extern "C" {

void ttcf_config_default(ttcf_config *c) {
    if (!c) return;
    memset(c, 0, sizeof(*c));
    c->system = TTCF_BULK_WCA;
    c->precision = TTCF_MIXED;
    c->dt = 0.0025;
    c->T = 0.722;
    c->tau_T = 0.25;
    c->dof_mode = 0;
    c->n_steps = 1000;
    c->sample_every = 1;
    c->mapping_mask = 0xF;
    c->reset_alpha = 0;
    c->keep_state = 0;
    c->skin = 0.0;
    c->block_threads = 0;
    c->kernel_variant = 0;
    c->use_graph = 1;
    c->timeout_s = 0.0;
}

const char *ttcf_version(void) { return "ttcf-gb300 1.0 (sm_103a)"; }

const char *ttcf_last_error(const ttcf_ctx *ctx) {
    return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

ttcf_status ttcf_create(const ttcf_config *cfg, ttcf_ctx **out) {
    if (!cfg || !out) return fail(nullptr, TTCF_E_INVALID, "NULL argument");
    *out = nullptr;
    const ttcf_config &c = *cfg;
    if (c.system != TTCF_BULK_WCA && c.system != TTCF_CONFINED_LJ && c.system != TTCF_BULK_WCA_ELONG)
        return fail(nullptr, TTCF_E_INVALID, "unknown system");
    if (c.system == TTCF_CONFINED_LJ && c.precision != TTCF_MIXED)
        return fail(nullptr, TTCF_E_INVALID, "the confined system runs in TTCF_MIXED precision only");
    if (c.precision != TTCF_FP64 && c.precision != TTCF_MIXED)
        return fail(nullptr, TTCF_E_INVALID, "precision must be TTCF_FP64 or TTCF_MIXED");
    if (!(c.dt > 0) || !(c.T > 0) || !(c.tau_T > 0))
        return fail(nullptr, TTCF_E_INVALID, "dt, T and tau_T must be positive");
    if (c.n_steps < 1 || c.sample_every < 1 || c.n_steps % c.sample_every)
        return fail(nullptr, TTCF_E_INVALID, "n_steps must be a positive multiple of sample_every");
    if (c.mapping_mask == 0)
        return fail(nullptr, TTCF_E_INVALID, "mapping_mask must select at least one mapping");
    if (c.system == TTCF_CONFINED_LJ && (c.mapping_mask & ~0xFu))
        return fail(nullptr, TTCF_E_INVALID, "the confined system takes the mappings 0..3 of Eq. 3 only");
    if (c.block_threads < 0 || c.block_threads % 32 || c.block_threads > 1024)
        return fail(nullptr, TTCF_E_INVALID, "block_threads must be 0 or a multiple of 32 <= 1024");
    if (c.kernel_variant < 0 || c.kernel_variant > N_VARIANTS)
        return fail(nullptr, TTCF_E_INVALID, "kernel_variant out of range");
    if (c.skin > 1.0) return fail(nullptr, TTCF_E_INVALID, "skin must be <= 1");
    if (c.cell_frac != 0.0 && !(c.cell_frac >= 0.4 && c.cell_frac <= 1.0))
        return fail(nullptr, TTCF_E_INVALID, "cell_frac must be 0 or in [0.4, 1]");
    if ((c.dev_alloc == nullptr) != (c.dev_free == nullptr))
        return fail(nullptr, TTCF_E_INVALID, "dev_alloc and dev_free must be set together");
    ttcf_ctx *ctx = new (std::nothrow) ttcf_ctx();
    if (!ctx) return fail(nullptr, TTCF_E_OOM, "host allocation failed");
    ctx->cfg = c;
    memset(&ctx->stats, 0, sizeof(ctx->stats));
    ctx->st = (cudaStream_t)c.stream;
    ctx->skin = c.skin > 0 ? c.skin : DEFAULT_SKIN;
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&ctx->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&ctx->smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, ctx->device);
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&ctx->h_abort, sizeof(int), cudaHostAllocMapped);
    if (e == cudaSuccess) { *ctx->h_abort = 0; e = cudaHostGetDevicePointer((void **)&ctx->d_abort, ctx->h_abort, 0); }
    for (int k = 0; k < 4 && e == cudaSuccess; k++) e = cudaEventCreate(&ctx->ev[k]);
    if (e != cudaSuccess) {
        g_create_error = std::string("CUDA initialisation failed: ") + cudaGetErrorString(e);
        cudaGetLastError();
        ttcf_destroy(ctx);
        return TTCF_E_CUDA;
    }
    *out = ctx;
    return TTCF_OK;
}

void ttcf_destroy(ttcf_ctx *ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->st);
    for (void *p : ctx->allocs) dev_free_raw(ctx, p);
    for (int k = 0; k < 4; k++) if (ctx->ev[k]) cudaEventDestroy(ctx->ev[k]);
    if (ctx->cap_st) cudaStreamDestroy(ctx->cap_st);
    if (ctx->h_abort) cudaFreeHost(ctx->h_abort);
    delete ctx;
}

ttcf_status ttcf_spawn_daughters(ttcf_ctx *ctx, int n_atoms, const double box[3], int n_mothers,
                                 const double *mother_soa, const double *mother_alpha,
                                 const double *shear_rates, int ptr_is_device, int *batch_id) {
    if (!ctx || !box) return fail(ctx, TTCF_E_INVALID, "NULL argument");
    if (ctx->cfg.system != TTCF_BULK_WCA && ctx->cfg.system != TTCF_BULK_WCA_ELONG)
        return fail(ctx, TTCF_E_INVALID, "ttcf_spawn_daughters needs a bulk (TTCF_BULK_WCA or "
                                         "TTCF_BULK_WCA_ELONG) context");
    if (ctx->ran) return fail(ctx, TTCF_E_STATE, "ttcf_spawn_daughters after ttcf_run");
    int maps[MAX_MAPS], M = 0;
    for (int m = 0; m < MAX_MAPS; m++) if (ctx->cfg.mapping_mask & (1u << m)) maps[M++] = m;
    const int S = ctx->cfg.n_steps / ctx->cfg.sample_every + 1;
    BatchHost b;
    if (ctx->cfg.system == TTCF_BULK_WCA_ELONG) {   // checked before any work is queued
        if (n_mothers <= 0 || !shear_rates)
            return fail(ctx, TTCF_E_INVALID, "an elongational batch needs its elongation rates");
        if (n_atoms < 4 || n_atoms > 4096) return fail(ctx, TTCF_E_INVALID, "n_atoms must be in [4, 4096]");
        std::vector<double> rates(n_mothers);
        if (ptr_is_device)
            CK(cudaMemcpy(rates.data(), shear_rates, sizeof(double) * n_mothers, cudaMemcpyDeviceToHost));
        else
            for (int k = 0; k < n_mothers; k++) rates[k] = shear_rates[k];
        ttcf_status ps = elong_plan(ctx, n_atoms, box, rates, b);
        if (ps != TTCF_OK) return ps;
    }
    Pool pool(ctx);
    ttcf_status s = make_batch(ctx, pool, b, n_atoms, box, n_mothers, mother_soa, mother_alpha,
                               shear_rates, ptr_is_device, maps, M, S, 0.0);
    if (s != TTCF_OK) return s;
    if (ctx->total_d + b.D() > 2000000000LL) return fail(ctx, TTCF_E_INVALID, "too many daughters");
    b.d0 = ctx->total_d;
    ctx->total_d += b.D();
    pool.keep();
    ctx->batches.push_back(b);
    ctx->tables_ok = false;
    if (batch_id) *batch_id = (int)ctx->batches.size() - 1;
    return TTCF_OK;
}

ttcf_status ttcf_run(ttcf_ctx *ctx, int n_steps) {
    if (!ctx) return fail(ctx, TTCF_E_INVALID, "NULL context");
    if (ctx->batches.empty()) return fail(ctx, TTCF_E_STATE, "ttcf_run before ttcf_spawn_daughters");
    if (ctx->cfg.system == TTCF_CONFINED_LJ) return run_confined(ctx, n_steps);
    if (ctx->cfg.system == TTCF_BULK_WCA_ELONG) return run_elong(ctx, n_steps);
    const ttcf_config &cf = ctx->cfg;
    const int step0 = ctx->steps_done;
    if (step0 >= cf.n_steps) return TTCF_OK;
    const int step1 = (n_steps <= 0 || step0 + n_steps > cf.n_steps) ? cf.n_steps : step0 + n_steps;
    const bool save = step1 < cf.n_steps || cf.keep_state;
    if (save) {
        for (auto &b : ctx->batches) {
            if (b.state) continue;
            Pool p(ctx);
            b.state = p.get<unsigned long long>((size_t)b.D() * 6 * b.N);
            if (p.oom) return fail(ctx, TTCF_E_OOM, "device allocation failed (state)");
            p.keep();
        }
    }
    if (step0 > 0)
        for (auto &b : ctx->batches)
            if (!b.state) return fail(ctx, TTCF_E_STATE, "resume without saved state");
    ctx->ran = true;
    *(volatile int *)ctx->h_abort = 0;
    memset(&ctx->stats, 0, sizeof(ctx->stats));
    ctx->stats.ms_spawn = ctx->ms_spawn_pending;   // the spawns this run is the first to cover
    ctx->ms_spawn_pending = 0.0;

    RunArgs a;
    memset(&a, 0, sizeof(a));
    a.step0 = step0; a.step1 = step1;
    a.sample_every = cf.sample_every;
    a.fresh = step0 == 0;
    a.save_state = save ? 1 : 0;
    a.reset_alpha = cf.reset_alpha;
    a.dt = cf.dt;
    a.delta0 = 0.0;
    a.abort_flag = ctx->d_abort;

    std::vector<BatchHost *> bs;
    for (auto &b : ctx->batches) bs.push_back(&b);
    Pool pool(ctx);
    int launches = 0;
    const bool finishing = step1 >= cf.n_steps;
    if (finishing) {   // reduction buffers exist before a graph is captured
        for (auto &b : ctx->batches) {
            ttcf_status r = ensure_reduce_buffers(ctx, b);
            if (r != TTCF_OK) return r;
        }
    }
    const bool capturing = cf.use_graph != 0;
    auto tail = [&]() -> ttcf_status {
        if (!finishing) return TTCF_OK;
        CK(record_event(ctx->ev[2], ctx->st, capturing));
        for (auto &b : ctx->batches) {
            b.reduced = false;
            ttcf_status r = reduce_batch(ctx, b);
            if (r != TTCF_OK) return r;
            launches += 3;
        }
        CK(record_event(ctx->ev[3], ctx->st, capturing));
        return TTCF_OK;
    };
    ttcf_status s = launch_batches(ctx, pool, bs, a, launches, ctx->ev[0], ctx->ev[1], tail);
    if (s != TTCF_OK) return s;
    s = wait_with_timeout(ctx, finishing ? ctx->ev[3] : ctx->ev[1]);
    if (s != TTCF_OK && s != TTCF_E_TIMEOUT) return s;
    const bool timed_out = s == TTCF_E_TIMEOUT;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]);
    ctx->stats.ms_run = ms;
    ctx->stats.skin = ctx->batches.empty() ? ctx->skin : ctx->batches[0].skin;
    ctx->steps_done = step1;
    if (finishing) {
        float msr = 0.f;
        cudaEventElapsedTime(&msr, ctx->ev[2], ctx->ev[3]);
        ctx->stats.ms_reduce = msr;
    }

    // counters and failures
    bool any_fail = false;
    for (auto &b : ctx->batches) {
        std::vector<int> stv(b.D());
        std::vector<unsigned long long> pr(b.D());
        std::vector<unsigned int> rb(b.D());
        CK(cudaMemcpy(stv.data(), b.status, sizeof(int) * b.D(), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(pr.data(), b.pairs, sizeof(unsigned long long) * b.D(), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(rb.data(), b.rebuilds, sizeof(unsigned int) * b.D(), cudaMemcpyDeviceToHost));
        for (long long d = 0; d < b.D(); d++) {
            any_fail |= stv[d] != 0;
            ctx->stats.pairs_interacting += (double)pr[d];
            ctx->stats.rebuilds += (double)rb[d];
        }
        ctx->stats.atom_steps += (double)b.D() * b.N * (step1 - step0);
        // counters are per run
        CK(cudaMemsetAsync(b.pairs, 0, sizeof(unsigned long long) * b.D(), ctx->st));
        CK(cudaMemsetAsync(b.rebuilds, 0, sizeof(unsigned int) * b.D(), ctx->st));
    }
    ctx->stats.launches = launches;
    if (timed_out) return fail(ctx, TTCF_E_TIMEOUT, "ttcf_run exceeded timeout_s; daughters aborted");
    if (any_fail) return fail(ctx, TTCF_E_NUMERIC, "some daughters failed; see ttcf_group_status");
    return TTCF_OK;
}

ttcf_status ttcf_response_obs(ttcf_ctx *ctx, int batch_id, int observable, int corrected,
                              double *t, double *dav, double *dav_se, double *corr,
                              double *corr_se, double *ttcf, double *ttcf_se, int capacity,
                              int *n_samples) {
    BatchHost *b = get_batch(ctx, batch_id);
    if (!b) return fail(ctx, TTCF_E_INVALID, "bad batch id");
    if (observable < 0 || observable >= b->n_obs) return fail(ctx, TTCF_E_INVALID, "bad observable index");
    if (!b->reduced) return fail(ctx, TTCF_E_STATE, "run not finished");
    if (n_samples) *n_samples = b->S;
    if (capacity < b->S) return fail(ctx, TTCF_E_INVALID, "capacity smaller than the sample count");
    const int S = b->S;
    std::vector<double> h((size_t)9 * S);
    CK(cudaMemcpyAsync(h.data(), b->out + (size_t)observable * 9 * S, sizeof(double) * h.size(),
                       cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    const double ds = ctx->cfg.sample_every * ctx->cfg.dt;
    for (int s = 0; s < S; s++) {
        if (t) t[s] = s * ds;
        if (corr) corr[s] = corrected ? h[6 * S + s] : h[s];
        if (corr_se) corr_se[s] = h[S + s];
        if (dav) dav[s] = h[2 * S + s];
        if (dav_se) dav_se[s] = h[3 * S + s];
        if (ttcf) ttcf[s] = corrected ? h[7 * S + s] : h[4 * S + s];
        if (ttcf_se) ttcf_se[s] = h[5 * S + s];
    }
    return TTCF_OK;
}

ttcf_status ttcf_response(ttcf_ctx *ctx, int batch_id, int corrected, double *t, double *dav,
                          double *dav_se, double *corr, double *corr_se, double *ttcf,
                          double *ttcf_se, int capacity, int *n_samples) {
    return ttcf_response_obs(ctx, batch_id, 0, corrected, t, dav, dav_se, corr, corr_se, ttcf,
                             ttcf_se, capacity, n_samples);
}

ttcf_status ttcf_viscosity(ttcf_ctx *ctx, int batch_id, double *t, double *eta_ttcf,
                           double *eta_ttcf_se, double *eta_dav, double *eta_dav_se, int capacity,
                           int *n_samples) {
    BatchHost *b = get_batch(ctx, batch_id);
    if (!b) return fail(ctx, TTCF_E_INVALID, "bad batch id");
    if (b->confined) return fail(ctx, TTCF_E_INVALID, "viscosity of a confined batch is not defined");
    const double g = b->gamma.empty() ? 0.0 : b->gamma[0];
    for (double x : b->gamma)
        if (x != g) return fail(ctx, TTCF_E_INVALID, "shear rate differs between groups");
    if (g == 0.0) return fail(ctx, TTCF_E_INVALID, "zero shear rate");
    std::vector<double> tt(b->S), dv(b->S), dse(b->S), tc(b->S), tse(b->S);
    ttcf_status s = ttcf_response(ctx, batch_id, 0, tt.data(), dv.data(), dse.data(), nullptr,
                                  nullptr, tc.data(), tse.data(), (int)b->S, n_samples);
    if (s != TTCF_OK) return s;
    if (capacity < b->S) return fail(ctx, TTCF_E_INVALID, "capacity smaller than the sample count");
    // shear: eta = -P_xy / gamma; planar elongation: eta_1 = -(P_xx - P_zz) / (4 eps)
    const double sc = b->elong ? 4.0 * g : g;
    for (int k = 0; k < b->S; k++) {
        if (t) t[k] = tt[k];
        if (eta_ttcf) eta_ttcf[k] = -tc[k] / sc;
        if (eta_ttcf_se) eta_ttcf_se[k] = tse[k] / fabs(sc);
        if (eta_dav) eta_dav[k] = -dv[k] / sc;
        if (eta_dav_se) eta_dav_se[k] = dse[k] / fabs(sc);
    }
    return TTCF_OK;
}

ttcf_status ttcf_omega_mean(ttcf_ctx *ctx, int batch_id, double *omega_mean, double *n_valid) {
    BatchHost *b = get_batch(ctx, batch_id);
    if (!b) return fail(ctx, TTCF_E_INVALID, "bad batch id");
    if (!b->reduced) return fail(ctx, TTCF_E_STATE, "run not finished");
    double h[2];
    CK(cudaMemcpyAsync(h, b->Og + b->G, sizeof(h), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    if (omega_mean) *omega_mean = h[0];
    if (n_valid) *n_valid = h[1];
    return TTCF_OK;
}

ttcf_status ttcf_daughter_series(ttcf_ctx *ctx, int batch_id, double *B, double *Omega,
                                 size_t capacity_B) {
    BatchHost *b = get_batch(ctx, batch_id);
    if (!b) return fail(ctx, TTCF_E_INVALID, "bad batch id");
    const size_t n = (size_t)b->D() * b->n_obs * b->S;
    if (B && capacity_B < n) return fail(ctx, TTCF_E_INVALID, "capacity_B too small");
    CK(cudaStreamSynchronize(ctx->st));
    if (B) CK(cudaMemcpy(B, b->B, sizeof(double) * n, cudaMemcpyDeviceToHost));
    if (Omega) CK(cudaMemcpy(Omega, b->Omega, sizeof(double) * b->D(), cudaMemcpyDeviceToHost));
    return TTCF_OK;
}

ttcf_status ttcf_group_status(ttcf_ctx *ctx, int batch_id, int *status, int capacity) {
    BatchHost *b = get_batch(ctx, batch_id);
    if (!b) return fail(ctx, TTCF_E_INVALID, "bad batch id");
    if (!status || capacity < b->G) return fail(ctx, TTCF_E_INVALID, "capacity smaller than n_mothers");
    std::vector<int> st(b->D());
    CK(cudaStreamSynchronize(ctx->st));
    CK(cudaMemcpy(st.data(), b->status, sizeof(int) * b->D(), cudaMemcpyDeviceToHost));
    for (int g = 0; g < b->G; g++) {
        int v = 0;
        for (int k = 0; k < b->M; k++) v |= st[(size_t)g * b->M + k];
        status[g] = v;
    }
    return TTCF_OK;
}

ttcf_status ttcf_get_state(ttcf_ctx *ctx, int batch_id, int daughter, double *soa, double *alpha,
                           double *delta) {
    BatchHost *b = get_batch(ctx, batch_id);
    if (!b) return fail(ctx, TTCF_E_INVALID, "bad batch id");
    if (!b->state) return fail(ctx, TTCF_E_STATE, "no saved state (set keep_state = 1)");
    if (daughter < 0 || daughter >= b->D()) return fail(ctx, TTCF_E_INVALID, "bad daughter index");
    const int N = b->N;
    std::vector<unsigned long long> sl((size_t)6 * N);
    double sc[4];
    CK(cudaStreamSynchronize(ctx->st));
    CK(cudaMemcpy(sl.data(), b->state + (size_t)daughter * 6 * N, sizeof(unsigned long long) * 6 * N,
                  cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(sc, b->scal + (size_t)daughter * 4, sizeof(sc), cudaMemcpyDeviceToHost));
    const bool mixed = ctx->cfg.precision == TTCF_MIXED;
    if (mixed)   // alpha, K2, e1, delta kept as float pairs in MIXED mode
        for (int k = 0; k < 4; k++) { float2 v; memcpy(&v, &sc[k], 8); sc[k] = (double)v.x + (double)v.y; }
    auto val = [&](size_t k) {
        if (mixed) { float2 v; memcpy(&v, &sl[k], 8); return (double)v.x + (double)v.y; }
        double v; memcpy(&v, &sl[k], 8); return v;
    };
    if (b->elong) {   // wrapped into the box of the last step; alpha, Lx, Lz kept
        for (int e = 0; e < 6 * N && soa; e++) soa[e] = val(e);
        if (alpha) *alpha = sc[0];
        if (delta) *delta = 0.0;
        return TTCF_OK;
    }
    const double f = 1.0 + sc[2];
    const double dl = sc[3];
    for (int i = 0; i < N; i++) {
        double x = val(i), y = val(N + i), z = val(2 * N + i);
        const double ny = rint(y / b->L[1]);
        y -= ny * b->L[1]; x -= ny * dl;
        x -= b->L[0] * rint(x / b->L[0]);
        z -= b->L[2] * rint(z / b->L[2]);
        if (x >= 0.5 * b->L[0]) x -= b->L[0];
        if (y >= 0.5 * b->L[1]) y -= b->L[1];
        if (z >= 0.5 * b->L[2]) z -= b->L[2];
        if (soa) {
            soa[i] = x; soa[N + i] = y; soa[2 * N + i] = z;
            soa[3 * N + i] = f * val(3 * N + i);
            soa[4 * N + i] = f * val(4 * N + i);
            soa[5 * N + i] = f * val(5 * N + i);
        }
    }
    if (alpha) *alpha = sc[0];
    if (delta) *delta = dl;
    return TTCF_OK;
}

ttcf_status ttcf_get_stats(ttcf_ctx *ctx, ttcf_stats *out) {
    if (!ctx || !out) return fail(ctx, TTCF_E_INVALID, "NULL argument");
    *out = ctx->stats;
    return TTCF_OK;
}

ttcf_status ttcf_sample_mothers(ttcf_ctx *ctx, int n_atoms, const double box[3], int n_init,
                                const double *init_soa, int n_eq, int n_states, int spacing,
                                double *out_soa, double *out_alpha) {
    if (!ctx || !box || !init_soa || !out_soa) return fail(ctx, TTCF_E_INVALID, "NULL argument");
    if (ctx->cfg.system != TTCF_BULK_WCA && ctx->cfg.system != TTCF_BULK_WCA_ELONG)
        return fail(ctx, TTCF_E_INVALID, "ttcf_sample_mothers needs a bulk context");
    if (n_eq < 0 || n_states < 1 || spacing < 1) return fail(ctx, TTCF_E_INVALID, "bad sampling schedule");
    const long long total = (long long)n_eq + (long long)n_states * spacing;
    if (total > 2000000000LL) return fail(ctx, TTCF_E_INVALID, "trajectory too long");
    const int maps[1] = {0};
    BatchHost b;
    Pool pool(ctx);
    ttcf_status s = make_batch(ctx, pool, b, n_atoms, box, n_init, init_soa, nullptr, nullptr, 0,
                               maps, 1, 1, 0.0);
    if (s != TTCF_OK) return s;
    b.d0 = 0;
    const int N = n_atoms;
    double *snap = pool.get<double>((size_t)n_init * n_states * 6 * N);
    double *snap_a = pool.get<double>((size_t)n_init * n_states);
    if (pool.oom) return fail(ctx, TTCF_E_OOM, "device allocation failed (mother snapshots)");
    RunArgs a;
    memset(&a, 0, sizeof(a));
    a.step0 = 0; a.step1 = (int)total;
    a.sample_every = (int)total + 1;
    a.fresh = 1; a.dt = ctx->cfg.dt;
    a.reset_alpha = 1;
    a.abort_flag = nullptr;
    a.snap = snap; a.snap_alpha = snap_a;
    a.snap_first = n_eq + spacing; a.snap_every = spacing; a.n_snap = n_states;
    std::vector<BatchHost *> bs = {&b};
    int launches = 0;
    s = launch_batches(ctx, pool, bs, a, launches);
    if (s != TTCF_OK) return s;
    CK(cudaStreamSynchronize(ctx->st));
    std::vector<int> stv(b.D());
    CK(cudaMemcpy(stv.data(), b.status, sizeof(int) * b.D(), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(out_soa, snap, sizeof(double) * (size_t)n_init * n_states * 6 * N, cudaMemcpyDeviceToHost));
    if (out_alpha)
        CK(cudaMemcpy(out_alpha, snap_a, sizeof(double) * (size_t)n_init * n_states, cudaMemcpyDeviceToHost));
    for (int v : stv)
        if (v) return fail(ctx, TTCF_E_NUMERIC, "a mother trajectory failed");
    return TTCF_OK;
}

// Copies of one phase point with small random momentum kicks (see
// ttcf_kick.cu); host or device buffers.
ttcf_status ttcf_kick_states(ttcf_ctx *ctx, int n_atoms, const double *state_soa, const int *types,
                             int n_copies, double kick, unsigned long long seed, int keep_energy,
                             double *out_soa, int is_dev) {
    if (!ctx || !state_soa || !out_soa) return fail(ctx, TTCF_E_INVALID, "NULL argument");
    if (n_atoms < 1 || n_copies < 1) return fail(ctx, TTCF_E_INVALID, "n_atoms and n_copies must be positive");
    if (!(kick >= 0.0) || !isfinite(kick)) return fail(ctx, TTCF_E_INVALID, "kick must be finite and >= 0");
    const int N = n_atoms;
    std::vector<int> th;
    if (types) {   // groups must be 0, 1 or 2
        th.resize(N);
        if (is_dev) CK(cudaMemcpy(th.data(), types, sizeof(int) * N, cudaMemcpyDeviceToHost));
        else memcpy(th.data(), types, sizeof(int) * N);
        for (int t : th)
            if (t < 0 || t > 2) return fail(ctx, TTCF_E_INVALID, "types must be 0, 1 or 2");
    }
    Pool pool(ctx);
    const double *d_src = state_soa;
    const int *d_types = types;
    double *d_out = out_soa;
    if (!is_dev) {
        double *s = pool.get<double>((size_t)6 * N);
        int *t = types ? pool.get<int>(N) : nullptr;
        d_out = pool.get<double>((size_t)n_copies * 6 * N);
        if (pool.oom) return fail(ctx, TTCF_E_OOM, "device allocation failed (kicks)");
        CK(cudaMemcpyAsync(s, state_soa, sizeof(double) * 6 * N, cudaMemcpyHostToDevice, ctx->st));
        if (t) CK(cudaMemcpyAsync(t, th.data(), sizeof(int) * N, cudaMemcpyHostToDevice, ctx->st));
        d_src = s;
        d_types = t;
    }
    KickArgs ka;
    ka.N = N;
    ka.keep_energy = keep_energy ? 1 : 0;
    ka.ks = kick * sqrt(ctx->cfg.T);
    ka.seed = seed;
    ka.src = d_src;
    ka.types = d_types;
    ka.out = d_out;
    CK(launch_kick(ka, n_copies, ctx->st));
    if (!is_dev)
        CK(cudaMemcpyAsync(out_soa, d_out, sizeof(double) * (size_t)n_copies * 6 * N, cudaMemcpyDeviceToHost,
                           ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return TTCF_OK;
}

ttcf_status ttcf_mother_acf(ttcf_ctx *ctx, int n_atoms, const double box[3], int n_init,
                            const double *init_soa, int n_eq, int n_steps, int max_lag,
                            double *acf_pxy, double *acf_pxy2, double *eta_gk, double *series) {
    if (!ctx || !box || !init_soa) return fail(ctx, TTCF_E_INVALID, "NULL argument");
    if (ctx->cfg.system != TTCF_BULK_WCA && ctx->cfg.system != TTCF_BULK_WCA_ELONG)
        return fail(ctx, TTCF_E_INVALID, "ttcf_mother_acf needs a bulk context");
    if (n_eq < 0 || n_steps < 2 || max_lag < 0 || max_lag >= n_steps || n_init < 1 ||
        (long long)n_eq + n_steps > 2000000000LL)
        return fail(ctx, TTCF_E_INVALID, "bad correlation schedule");
    const int maps[1] = {0};
    const int S = n_steps + 1;
    BatchHost b;
    Pool pool(ctx);
    ttcf_status s = make_batch(ctx, pool, b, n_atoms, box, n_init, init_soa, nullptr, nullptr, 0,
                               maps, 1, S, 0.0);
    if (s != TTCF_OK) return s;
    b.d0 = 0;
    b.state = pool.get<unsigned long long>((size_t)n_init * 6 * n_atoms);
    double *acf = pool.get<double>((size_t)max_lag + 1), *acf2 = pool.get<double>((size_t)max_lag + 1);
    double *m2 = pool.get<double>(1);
    if (pool.oom) return fail(ctx, TTCF_E_OOM, "device allocation failed (correlations)");
    std::vector<BatchHost *> bs = {&b};
    int launches = 0;
    RunArgs a;
    memset(&a, 0, sizeof(a));
    a.dt = ctx->cfg.dt;
    a.reset_alpha = 1;
    if (n_eq > 0) {   // thermalisation, no samples, state kept
        a.step0 = 0; a.step1 = n_eq; a.sample_every = n_eq + 1; a.fresh = 1; a.save_state = 1;
        s = launch_batches(ctx, pool, bs, a, launches);
        if (s != TTCF_OK) return s;
    }
    // production: B(s) = P_xy(s) every step, s = 1 .. n_steps (row index s)
    a.step0 = 0; a.step1 = n_steps; a.sample_every = 1; a.fresh = n_eq > 0 ? 0 : 1; a.save_state = 0;
    s = launch_batches(ctx, pool, bs, a, launches);
    if (s != TTCF_OK) return s;
    CK(launch_acf(b.B, n_init, S, 1, n_steps, max_lag, acf, acf2, m2, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    std::vector<int> stv(n_init);
    CK(cudaMemcpy(stv.data(), b.status, sizeof(int) * n_init, cudaMemcpyDeviceToHost));
    for (int v : stv)
        if (v) return fail(ctx, TTCF_E_NUMERIC, "a mother trajectory failed");
    std::vector<double> h((size_t)max_lag + 1);
    CK(cudaMemcpy(h.data(), acf, sizeof(double) * h.size(), cudaMemcpyDeviceToHost));
    if (acf_pxy) memcpy(acf_pxy, h.data(), sizeof(double) * h.size());
    if (acf_pxy2) CK(cudaMemcpy(acf_pxy2, acf2, sizeof(double) * h.size(), cudaMemcpyDeviceToHost));
    if (eta_gk) {   // Green-Kubo running integral (V/T) int_0^t C(s) ds, trapezoid
        const double f = b.V / ctx->cfg.T;
        double run = 0.0;
        eta_gk[0] = 0.0;
        for (int k = 1; k <= max_lag; k++) {
            run += 0.5 * ctx->cfg.dt * (h[k - 1] + h[k]);
            eta_gk[k] = f * run;
        }
    }
    if (series)
        for (int g = 0; g < n_init; g++)
            CK(cudaMemcpy(series + (size_t)g * n_steps, b.B + (size_t)g * S + 1, sizeof(double) * n_steps,
                          cudaMemcpyDeviceToHost));
    return TTCF_OK;
}

ttcf_status ttcf_forces(ttcf_ctx *ctx, int n_atoms, const double box[3], int n_states,
                        double delta, const double *soa, double *F, double *W, double *U) {
    if (!ctx || !box || !soa) return fail(ctx, TTCF_E_INVALID, "NULL argument");
    if (ctx->cfg.system != TTCF_BULK_WCA && ctx->cfg.system != TTCF_BULK_WCA_ELONG)
        return fail(ctx, TTCF_E_INVALID, "ttcf_forces needs a bulk context");
    const int maps[1] = {0};
    BatchHost b;
    Pool pool(ctx);
    ttcf_status s = make_batch(ctx, pool, b, n_atoms, box, n_states, soa, nullptr, nullptr, 0,
                               maps, 1, 1, delta);
    if (s != TTCF_OK) return s;
    b.d0 = 0;
    const int N = n_atoms;
    double *fo = pool.get<double>((size_t)n_states * 3 * N);
    double *wo = pool.get<double>(n_states);
    if (pool.oom) return fail(ctx, TTCF_E_OOM, "device allocation failed (forces)");
    RunArgs a;
    memset(&a, 0, sizeof(a));
    a.step0 = 0; a.step1 = 0; a.sample_every = 1; a.fresh = 1;
    a.dt = ctx->cfg.dt; a.delta0 = delta;
    a.force_out = fo; a.wxy_out = wo;
    std::vector<BatchHost *> bs = {&b};
    int launches = 0;
    s = launch_batches(ctx, pool, bs, a, launches);
    if (s != TTCF_OK) return s;
    CK(cudaStreamSynchronize(ctx->st));
    std::vector<double> wxy(n_states), feat((size_t)n_states * FEAT_RAW);
    if (F) CK(cudaMemcpy(F, fo, sizeof(double) * (size_t)n_states * 3 * N, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(wxy.data(), wo, sizeof(double) * n_states, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(feat.data(), b.feat, sizeof(double) * feat.size(), cudaMemcpyDeviceToHost));
    for (int k = 0; k < n_states; k++) {
        if (W) {
            // xy from the kernel under test; the other components from the
            // double-precision spawn pass (virial part only)
            for (int c = 0; c < 6; c++) W[6 * k + c] = feat[(size_t)FEAT_RAW * k + 6 + c];
            W[6 * k + 3] = wxy[k];
        }
        if (U) U[k] = feat[(size_t)FEAT_RAW * k + 12];
    }
    return TTCF_OK;
}

ttcf_status ttcf_autotune(ttcf_ctx *ctx, int n_atoms, const double box[3], int n_states,
                          const double *soa, double shear_rate, int n_steps, int *best_variant,
                          double *best_skin, double *best_cell_frac, double *best_ms) {
    if (!ctx || !box || !soa || n_states < 1 || n_steps < 1)
        return fail(ctx, TTCF_E_INVALID, "bad autotune arguments");
    if (ctx->cfg.system != TTCF_BULK_WCA)
        return fail(ctx, TTCF_E_INVALID, "ttcf_autotune needs a TTCF_BULK_WCA context");
    const double skins[5] = {0.3, 0.35, 0.4, 0.5, 0.6};
    const int maps[4] = {0, 1, 2, 3};
    std::vector<double> gam(n_states, shear_rate);
    double best = 1e300;
    int bv = -1;
    double bskin = DEFAULT_SKIN, bfrac = DEFAULT_CELL_FRAC;
    const double fracs[3] = {0.5, 2.0 / 3.0, 1.0};
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    for (int v = 0; v < N_VARIANTS; v++) {
        const Variant var = variant_of(v);
        if (var.apt * var.maxt < n_atoms) continue;
        if (var.apt > 1 && (n_atoms + var.apt - 1) / var.apt < 64) continue;   // too few threads
        for (double sk : skins)
        for (double fr : fracs) {
            if (3.0 * (RC_WCA + sk) > std::min(box[0], std::min(box[1], box[2]))) continue;
            BatchHost b;
            Pool pool(ctx);
            ttcf_status s = make_batch(ctx, pool, b, n_atoms, box, n_states, soa, nullptr, gam.data(),
                                       0, maps, 4, n_steps + 1, 0.0, v, sk, fr);
            if (s != TTCF_OK) continue;   // e.g. shared memory exceeded
            b.d0 = 0;
            RunArgs a;
            memset(&a, 0, sizeof(a));
            a.step0 = 0; a.step1 = n_steps; a.sample_every = 1; a.fresh = 1;
            a.dt = ctx->cfg.dt; a.reset_alpha = ctx->cfg.reset_alpha;
            std::vector<BatchHost *> bs = {&b};
            int launches = 0;
            s = launch_batches(ctx, pool, bs, a, launches, e0, e1);
            if (s != TTCF_OK) { ctx->err.clear(); continue; }
            CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) { best = ms; bv = v; bskin = sk; bfrac = fr; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (bv < 0) return fail(ctx, TTCF_E_INVALID, "no launch variant can run this system");
    bool found = false;
    for (auto &e : ctx->tuned)
        if (e.N == n_atoms) { e.variant = bv; e.skin = bskin; e.cell_frac = bfrac; found = true; }
    if (!found) ctx->tuned.push_back({n_atoms, bv, bskin, bfrac});
    if (best_variant) *best_variant = bv + 1;
    if (best_skin) *best_skin = bskin;
    if (best_cell_frac) *best_cell_frac = bfrac;
    if (best_ms) *best_ms = best;
    return TTCF_OK;
}


void ttcf_confined_params_default(ttcf_confined_params *p) {
    if (p) *p = conf_params_or_default(nullptr);
}

ttcf_status ttcf_spawn_confined(ttcf_ctx *ctx, int n_atoms, const double box[3], const int *types,
                                const double *lattice, const ttcf_confined_params *params,
                                int n_mothers, const double *mother_soa,
                                const double *mother_alpha, const double *shear_rates,
                                int ptr_is_device, int *batch_id) {
    if (!ctx || !box) return fail(ctx, TTCF_E_INVALID, "NULL argument");
    if (ctx->cfg.system != TTCF_CONFINED_LJ)
        return fail(ctx, TTCF_E_INVALID, "ttcf_spawn_confined needs a TTCF_CONFINED_LJ context");
    if (ctx->ran) return fail(ctx, TTCF_E_STATE, "ttcf_spawn_confined after ttcf_run");
    int maps[4], M = 0;
    for (int m = 0; m < 4; m++) if (ctx->cfg.mapping_mask & (1u << m)) maps[M++] = m;
    const int S = ctx->cfg.n_steps / ctx->cfg.sample_every + 1;
    BatchHost b;
    Pool pool(ctx);
    ttcf_status s = make_conf_batch(ctx, pool, b, n_atoms, box, types, lattice,
                                    conf_params_or_default(params), n_mothers, mother_soa,
                                    mother_alpha, shear_rates, ptr_is_device, maps, M, S);
    if (s != TTCF_OK) return s;
    if (ctx->total_d + b.D() > 2000000000LL) return fail(ctx, TTCF_E_INVALID, "too many daughters");
    b.d0 = ctx->total_d;
    ctx->total_d += b.D();
    pool.keep();
    ctx->batches.push_back(b);
    if (batch_id) *batch_id = (int)ctx->batches.size() - 1;
    return TTCF_OK;
}

ttcf_status ttcf_sample_mothers_confined(ttcf_ctx *ctx, int n_atoms, const double box[3],
                                         const int *types, const double *lattice,
                                         const ttcf_confined_params *params, int n_init,
                                         const double *init_soa, int n_eq, int n_states,
                                         int spacing, double *out_soa, double *out_alpha,
                                         int *chain_status) {
    if (!ctx || !box || !init_soa || !out_soa) return fail(ctx, TTCF_E_INVALID, "NULL argument");
    if (ctx->cfg.system != TTCF_CONFINED_LJ)
        return fail(ctx, TTCF_E_INVALID, "ttcf_sample_mothers_confined needs a TTCF_CONFINED_LJ context");
    if (n_eq < 0 || n_states < 1 || spacing < 1) return fail(ctx, TTCF_E_INVALID, "bad sampling schedule");
    const long long total = (long long)n_eq + (long long)n_states * spacing;
    if (total > 2000000000LL) return fail(ctx, TTCF_E_INVALID, "trajectory too long");
    const int maps[1] = {0};
    BatchHost b;
    Pool pool(ctx);
    ttcf_status s = make_conf_batch(ctx, pool, b, n_atoms, box, types, lattice,
                                    conf_params_or_default(params), n_init, init_soa, nullptr,
                                    nullptr, 0, maps, 1, 1);
    if (s != TTCF_OK) return s;
    b.d0 = 0;
    const int N = n_atoms;
    double *snap = pool.get<double>((size_t)n_init * n_states * 6 * N);
    double *snap_a = pool.get<double>((size_t)n_init * n_states);
    if (pool.oom) return fail(ctx, TTCF_E_OOM, "device allocation failed (mother snapshots)");
    CK(cudaMemsetAsync(snap, 0, sizeof(double) * (size_t)n_init * n_states * 6 * N, ctx->st));
    CK(cudaMemsetAsync(snap_a, 0, sizeof(double) * (size_t)n_init * n_states, ctx->st));
    ConfRunArgs a;
    memset(&a, 0, sizeof(a));
    a.n_steps = (int)total;
    a.sample_every = (int)total + 1;
    a.reset_alpha = 1;
    a.dt = ctx->cfg.dt;
    a.snap = snap; a.snap_alpha = snap_a;
    a.snap_first = n_eq + spacing; a.snap_every = spacing; a.n_snap = n_states;
    std::vector<BatchHost *> bs = {&b};
    int launches = 0;
    s = launch_conf_batches(ctx, pool, bs, a, launches);
    if (s != TTCF_OK) return s;
    CK(cudaStreamSynchronize(ctx->st));
    std::vector<int> stv(b.D());
    CK(cudaMemcpy(stv.data(), b.status, sizeof(int) * b.D(), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(out_soa, snap, sizeof(double) * (size_t)n_init * n_states * 6 * N, cudaMemcpyDeviceToHost));
    if (out_alpha)
        CK(cudaMemcpy(out_alpha, snap_a, sizeof(double) * (size_t)n_init * n_states, cudaMemcpyDeviceToHost));
    if (chain_status) for (int k = 0; k < n_init; k++) chain_status[k] = stv[k];
    for (int v : stv)
        if (v) return fail(ctx, TTCF_E_NUMERIC, "a mother chain failed; see chain_status");
    return TTCF_OK;
}


extern "C++" {
namespace {
// Slabs adjacent to a wall (0 bottom, 1 top): centres within 1 sigma of its
// innermost layer, on the fluid side (the outermost fluid layer).
std::vector<int> adjacent_slabs(const BatchHost &b, int wall) {
    const double Ly = b.L[1], w = Ly / CONF_NSLAB, hh = b.half_h;
    std::vector<int> ks;
    for (int k = 0; k < CONF_NSLAB; k++) {
        const double c = -0.5 * Ly + (k + 0.5) * w;
        if (wall == 1 ? (c > hh - 1.0 && c < hh) : (c < -hh + 1.0 && c > -hh)) ks.push_back(k);
    }
    return ks;
}
}  // namespace
}  // extern "C++"

ttcf_status ttcf_friction(ttcf_ctx *ctx, int batch_id, int wall, double *t, double *slip_ttcf,
                          double *slip_dav, double *xi_ttcf, double *xi_dav, int capacity,
                          int *n_samples) {
    BatchHost *b = get_batch(ctx, batch_id);
    if (!b) return fail(ctx, TTCF_E_INVALID, "bad batch id");
    if (!b->confined) return fail(ctx, TTCF_E_INVALID, "friction needs a confined batch");
    if (wall != 0 && wall != 1) return fail(ctx, TTCF_E_INVALID, "wall must be 0 or 1");
    const double g = b->gamma.empty() ? 0.0 : b->gamma[0];
    for (double x : b->gamma)
        if (x != g) return fail(ctx, TTCF_E_INVALID, "shear rate differs between groups");
    if (!b->reduced) return fail(ctx, TTCF_E_STATE, "run not finished");
    const int S = b->S;
    if (n_samples) *n_samples = S;
    if (capacity < S) return fail(ctx, TTCF_E_INVALID, "capacity smaller than the sample count");
    const std::vector<int> ks = adjacent_slabs(*b, wall);
    if (ks.empty()) return fail(ctx, TTCF_E_INVALID, "no slab lies next to the wall");
    std::vector<double> h((size_t)b->n_obs * 9 * S);
    CK(cudaMemcpyAsync(h.data(), b->out, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    if (b->n_inner[wall] <= 0) return fail(ctx, TTCF_E_INVALID, "the wall has no inner layer");
    auto col = [&](int o, int q, int s) { return h[((size_t)o * 9 + q) * S + s]; };   // q: 2 dav, 4 ttcf
    const double ds = ctx->cfg.sample_every * ctx->cfg.dt;
    const int o_wall = 2 + 2 * CONF_NSLAB + wall;   // sum of p_x over the inner wall layer
    for (int s = 0; s < S; s++) {
        double sl[2], sg[2];
        for (int e = 0; e < 2; e++) {
            const int q = e == 0 ? 4 : 2;
            double P = 0.0, n = 0.0;
            for (int k : ks) { P += col(2 + k, q, s); n += col(2 + CONF_NSLAB + k, q, s); }
            sl[e] = col(o_wall, q, s) / b->n_inner[wall] - P / n;
            sg[e] = col(wall, q, s);
        }
        if (t) t[s] = s * ds;
        if (slip_ttcf) slip_ttcf[s] = sl[0];
        if (slip_dav) slip_dav[s] = sl[1];
        if (xi_ttcf) xi_ttcf[s] = -sg[0] / sl[0];
        if (xi_dav) xi_dav[s] = -sg[1] / sl[1];
    }
    return TTCF_OK;
}

ttcf_status ttcf_friction_equilibrium(ttcf_ctx *ctx, int batch_id, int wall, int max_lag, int n_s,
                                      const double *s_grid, double out[4], double *c_dvf,
                                      double *c_dvdv, double *zeta_s) {
    BatchHost *b = get_batch(ctx, batch_id);
    if (!b) return fail(ctx, TTCF_E_INVALID, "bad batch id");
    if (!b->confined) return fail(ctx, TTCF_E_INVALID, "friction needs a confined batch");
    if (wall != 0 && wall != 1) return fail(ctx, TTCF_E_INVALID, "wall must be 0 or 1");
    for (double x : b->gamma)
        if (x != 0.0) return fail(ctx, TTCF_E_INVALID, "the equilibrium method needs a zero-shear batch");
    if (!b->reduced) return fail(ctx, TTCF_E_STATE, "run not finished");
    const int S = b->S;
    if (max_lag < 1 || max_lag > S - 2) return fail(ctx, TTCF_E_INVALID, "max_lag must be in [1, samples - 2]");
    if (n_s < 2 || !s_grid || !out) return fail(ctx, TTCF_E_INVALID, "need >= 2 Laplace variables and out");
    for (int j = 0; j < n_s; j++)
        if (!(s_grid[j] >= 0.0) || !isfinite(s_grid[j])) return fail(ctx, TTCF_E_INVALID, "bad Laplace variable");
    if (b->n_inner[wall] <= 0) return fail(ctx, TTCF_E_INVALID, "the wall has no inner layer");
    const std::vector<int> ks = adjacent_slabs(*b, wall);
    if (ks.empty() || ks.size() > (size_t)SLIP_MAX_SLABS)
        return fail(ctx, TTCF_E_INVALID, "no (or too many) slabs next to the wall");
    Pool pool(ctx);
    const long long D = b->D();
    double *dv = pool.get<double>((size_t)D * S), *F = pool.get<double>((size_t)D * S);
    double *cf = pool.get<double>((size_t)max_lag + 1), *cv = pool.get<double>((size_t)max_lag + 1);
    if (pool.oom) return fail(ctx, TTCF_E_OOM, "device allocation failed (friction)");
    SlipArgs a;
    memset(&a, 0, sizeof(a));
    a.B = b->B; a.status = b->status;
    a.D = (int)D; a.n_obs = b->n_obs; a.S = S; a.nslab = CONF_NSLAB; a.wall = wall;
    a.n_slabs = (int)ks.size();
    for (size_t j = 0; j < ks.size(); j++) a.slabs[j] = ks[j];
    a.n_layer = (double)b->n_inner[wall];
    a.area = b->A;
    a.dv = dv; a.F = F;
    CK(launch_slip_correlations(a, max_lag, cf, cv, ctx->st));
    std::vector<double> hf((size_t)max_lag + 1), hv((size_t)max_lag + 1);
    CK(cudaMemcpyAsync(hf.data(), cf, sizeof(double) * hf.size(), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaMemcpyAsync(hv.data(), cv, sizeof(double) * hv.size(), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    if (c_dvf) memcpy(c_dvf, hf.data(), sizeof(double) * hf.size());
    if (c_dvdv) memcpy(c_dvdv, hv.data(), sizeof(double) * hv.size());
    // Laplace transforms on the lag grid (trapezoid), zeta~(s) = C~_dvF / C~_dvdv,
    // and the least-squares line 1/zeta~(s) = i + m s of the Maxwell kernel
    const double ds = ctx->cfg.sample_every * ctx->cfg.dt;
    auto lap = [&](const std::vector<double> &c, double sv) {
        double acc = 0.0;
        for (int k = 0; k <= max_lag; k++) acc += exp(-sv * k * ds) * c[k];
        const double f0 = c[0], fl = exp(-sv * max_lag * ds) * c[max_lag];
        return ds * (acc - 0.5 * (f0 + fl));
    };
    double sx = 0, sy = 0, sxx = 0, sxy = 0;
    for (int j = 0; j < n_s; j++) {
        const double z = lap(hf, s_grid[j]) / lap(hv, s_grid[j]);
        if (zeta_s) zeta_s[j] = z;
        const double x = s_grid[j], y = 1.0 / z;
        sx += x; sy += y; sxx += x * x; sxy += x * y;
    }
    const double den = n_s * sxx - sx * sx;
    if (!(den != 0.0)) return fail(ctx, TTCF_E_INVALID, "the Laplace variables must differ");
    const double slope = (n_s * sxy - sx * sy) / den, icpt = (sy - slope * sx) / n_s;
    const double z0 = 1.0 / icpt;
    out[0] = z0 / b->A;                               // xi_0
    out[1] = z0;                                      // zeta_0
    out[2] = slope / icpt;                            // tau_M
    out[3] = lap(hf, 0.0) / lap(hv, 0.0) / b->A;      // ratio of the integrals / A
    return TTCF_OK;
}

// ============================================================ checkpoints ==
extern "C++" {
namespace {

constexpr char CKPT_MAGIC[8] = {'T', 'T', 'C', 'F', 'C', 'K', 'P', '1'};
constexpr int CKPT_VERSION = 3;   // 2: MIXED per-daughter scalars as float pairs; 3: 32 mapping codes, inner wall layers

struct FileW {
    FILE *f;
    bool ok = true;
    template <class T> void put(const T &v) { ok = ok && fwrite(&v, sizeof(T), 1, f) == 1; }
    void bytes(const void *p, size_t n) { ok = ok && (n == 0 || fwrite(p, 1, n, f) == n); }
};
struct FileR {
    FILE *f;
    bool ok = true;
    template <class T> void get(T &v) { ok = ok && fread(&v, sizeof(T), 1, f) == 1; }
    void bytes(void *p, size_t n) { ok = ok && (n == 0 || fread(p, 1, n, f) == n); }
};

// The configuration fields that define the daughters' dynamics and samples.
bool same_dynamics(const ttcf_config &a, const ttcf_config &b) {
    return a.system == b.system && a.precision == b.precision && a.dt == b.dt && a.T == b.T &&
           a.tau_T == b.tau_T && a.dof_mode == b.dof_mode && a.n_steps == b.n_steps &&
           a.sample_every == b.sample_every && a.mapping_mask == b.mapping_mask &&
           a.reset_alpha == b.reset_alpha;
}

// One device array: its element count, then the bytes (0 = absent).
ttcf_status save_dev(ttcf_ctx *ctx, FileW &w, const void *d, size_t bytes) {
    unsigned long long n = d ? bytes : 0ull;
    w.put(n);
    if (!n) return TTCF_OK;
    std::vector<unsigned char> h(bytes);
    CK(cudaMemcpy(h.data(), d, bytes, cudaMemcpyDeviceToHost));
    w.bytes(h.data(), bytes);
    return TTCF_OK;
}

template <class T>
ttcf_status load_dev(ttcf_ctx *ctx, FileR &r, Pool &pool, T *&d, size_t expect_bytes, bool optional) {
    unsigned long long n = 0;
    r.get(n);
    if (!r.ok) return fail(ctx, TTCF_E_INVALID, "checkpoint truncated");
    if (n == 0) {
        d = nullptr;
        if (!optional) return fail(ctx, TTCF_E_INVALID, "checkpoint misses a required array");
        return TTCF_OK;
    }
    if (n != expect_bytes) return fail(ctx, TTCF_E_INVALID, "checkpoint array of unexpected size");
    std::vector<unsigned char> h(n);
    r.bytes(h.data(), n);
    if (!r.ok) return fail(ctx, TTCF_E_INVALID, "checkpoint truncated");
    d = pool.get<T>(n / sizeof(T));
    if (pool.oom) return fail(ctx, TTCF_E_OOM, "device allocation failed (checkpoint)");
    CK(cudaMemcpy(d, h.data(), n, cudaMemcpyHostToDevice));
    return TTCF_OK;
}

}  // namespace
}  // extern "C++"

ttcf_status ttcf_save(ttcf_ctx *ctx, const char *path) {
    if (!ctx || !path) return fail(ctx, TTCF_E_INVALID, "NULL argument");
    CK(cudaStreamSynchronize(ctx->st));
    FILE *f = fopen(path, "wb");
    if (!f) return fail(ctx, TTCF_E_INVALID, std::string("cannot open ") + path + " for writing");
    FileW w{f};
    w.bytes(CKPT_MAGIC, 8);
    w.put(CKPT_VERSION);
    ttcf_config c = ctx->cfg;
    c.stream = nullptr; c.dev_alloc = nullptr; c.dev_free = nullptr; c.alloc_user = nullptr;
    w.put(c);
    w.put(ctx->steps_done);
    w.put(ctx->total_d);
    const int nb = (int)ctx->batches.size();
    w.put(nb);
    ttcf_status st = TTCF_OK;
    for (const BatchHost &b : ctx->batches) {
        if (st != TTCF_OK) break;
        w.put(b.N); w.put(b.M); w.put(b.G); w.put(b.S); w.put(b.n_obs);
        const int conf = b.confined ? 1 : 0;
        w.put(conf);
        w.bytes(b.maps, sizeof(b.maps)); w.bytes(b.L, sizeof(b.L));
        w.put(b.V); w.put(b.Q); w.put(b.gT);
        w.bytes(b.nc, sizeof(b.nc)); w.put(b.ncell); w.bytes(b.snc, sizeof(b.snc)); w.put(b.sncell);
        w.put(b.d0); w.put(b.variant); w.put(b.threads); w.put(b.skin);
        w.bytes(b.gamma.data(), sizeof(double) * b.G);
        w.put(b.A); w.put(b.rc); w.put(b.k_tether); w.put(b.c_ff); w.put(b.c_wf); w.put(b.c_ww);
        w.put(b.ww_on); w.put(b.half_h);
        w.bytes(b.inner_y, sizeof(b.inner_y)); w.bytes(b.n_inner, sizeof(b.n_inner));
        const size_t D = (size_t)b.D();
        if ((st = save_dev(ctx, w, b.mothers, sizeof(unsigned long long) * b.G * 6 * b.N)) != TTCF_OK) break;
        if ((st = save_dev(ctx, w, b.m_alpha, sizeof(double) * b.G)) != TTCF_OK) break;
        if ((st = save_dev(ctx, w, b.gamma_d, sizeof(double) * b.G)) != TTCF_OK) break;
        if ((st = save_dev(ctx, w, b.B, sizeof(double) * D * b.n_obs * b.S)) != TTCF_OK) break;
        if ((st = save_dev(ctx, w, b.Omega, sizeof(double) * D)) != TTCF_OK) break;
        if ((st = save_dev(ctx, w, b.status, sizeof(int) * D)) != TTCF_OK) break;
        if ((st = save_dev(ctx, w, b.scal, sizeof(double) * D * 4)) != TTCF_OK) break;
        if ((st = save_dev(ctx, w, b.state, sizeof(unsigned long long) * D * 6 * b.N)) != TTCF_OK) break;
        if ((st = save_dev(ctx, w, b.feat, sizeof(double) * b.G * FEAT_RAW)) != TTCF_OK) break;
        if ((st = save_dev(ctx, w, b.types, sizeof(int) * b.N)) != TTCF_OK) break;
        if ((st = save_dev(ctx, w, b.lattice, sizeof(double) * 3 * b.N)) != TTCF_OK) break;
    }
    const bool ok = w.ok;
    if (fclose(f) != 0 || !ok) {
        if (st == TTCF_OK) st = fail(ctx, TTCF_E_INVALID, std::string("write to ") + path + " failed");
    }
    return st;
}

ttcf_status ttcf_load(ttcf_ctx *ctx, const char *path) {
    if (!ctx || !path) return fail(ctx, TTCF_E_INVALID, "NULL argument");
    if (!ctx->batches.empty() || ctx->ran)
        return fail(ctx, TTCF_E_STATE, "ttcf_load needs a freshly created context");
    FILE *f = fopen(path, "rb");
    if (!f) return fail(ctx, TTCF_E_INVALID, std::string("cannot open ") + path);
    FileR r{f};
    char magic[8];
    int ver = 0;
    r.bytes(magic, 8);
    r.get(ver);
    ttcf_config c;
    r.get(c);
    int steps_done = 0, nb = 0;
    long long total_d = 0;
    r.get(steps_done); r.get(total_d); r.get(nb);
    auto bad = [&](ttcf_status s, const char *msg) { fclose(f); return fail(ctx, s, msg); };
    if (!r.ok || memcmp(magic, CKPT_MAGIC, 8) != 0 || ver != CKPT_VERSION)
        return bad(TTCF_E_INVALID, "not a ttcf checkpoint (or another version)");
    if (!same_dynamics(c, ctx->cfg))
        return bad(TTCF_E_INVALID, "checkpoint was written under another configuration");
    if (nb < 0 || nb > 1 << 20 || steps_done < 0 || steps_done > c.n_steps || total_d < 0)
        return bad(TTCF_E_INVALID, "checkpoint header out of range");
    std::vector<BatchHost> loaded;
    Pool pool(ctx);
    for (int k = 0; k < nb; k++) {
        BatchHost b;
        int conf = 0;
        r.get(b.N); r.get(b.M); r.get(b.G); r.get(b.S); r.get(b.n_obs); r.get(conf);
        r.bytes(b.maps, sizeof(b.maps)); r.bytes(b.L, sizeof(b.L));
        r.get(b.V); r.get(b.Q); r.get(b.gT);
        r.bytes(b.nc, sizeof(b.nc)); r.get(b.ncell); r.bytes(b.snc, sizeof(b.snc)); r.get(b.sncell);
        r.get(b.d0); r.get(b.variant); r.get(b.threads); r.get(b.skin);
        b.confined = conf != 0;
        // the kernels index shared arrays with these numbers: check that they
        // are the ones the spawn calls would have chosen
        bool okh = r.ok && b.M >= 1 && b.M <= MAX_MAPS && b.G >= 1 && b.S == c.n_steps / c.sample_every + 1 &&
                   b.d0 >= 0 && b.skin > 0 && b.skin <= 1.0 &&
                   b.n_obs == (b.confined ? CONF_NOBS : 1) && b.confined == (c.system == TTCF_CONFINED_LJ) &&
                   b.N >= 4 && b.N <= (b.confined ? CONF_NMAX : 4096);
        for (int k = 0; k < 3 && okh; k++)
            okh = isfinite(b.L[k]) && b.L[k] > 0 && b.nc[k] >= (b.confined ? 1 : 3) && b.nc[k] <= 4096 &&
                  b.snc[k] >= 1 && b.snc[k] <= 4096;
        okh = okh && b.ncell == b.nc[0] * b.nc[1] * b.nc[2] && b.sncell == b.snc[0] * b.snc[1] * b.snc[2];
        for (int k = 0; k < b.M && okh; k++)
            okh = b.maps[k] >= 0 && b.maps[k] < (b.confined ? 4 : MAX_MAPS);
        if (okh && !b.confined) {
            okh = b.variant >= 0 && b.variant < N_VARIANTS;
            if (okh) {
                const Variant v = variant_of(b.variant);
                okh = b.threads >= 32 && b.threads % 32 == 0 && b.threads <= v.maxt && b.threads * v.apt >= b.N;
            }
        }
        if (!okh) return bad(TTCF_E_INVALID, "checkpoint batch header out of range");
        b.gamma.resize(b.G);
        r.bytes(b.gamma.data(), sizeof(double) * b.G);
        r.get(b.A); r.get(b.rc); r.get(b.k_tether); r.get(b.c_ff); r.get(b.c_wf); r.get(b.c_ww);
        r.get(b.ww_on); r.get(b.half_h);
        r.bytes(b.inner_y, sizeof(b.inner_y)); r.bytes(b.n_inner, sizeof(b.n_inner));
        if (!r.ok) return bad(TTCF_E_INVALID, "checkpoint truncated");
        if (b.n_inner[0] < 0 || b.n_inner[1] < 0 || b.n_inner[0] + b.n_inner[1] > b.N)
            return bad(TTCF_E_INVALID, "checkpoint batch header out of range");
        const size_t D = (size_t)b.D();
        ttcf_status s;
        if ((s = load_dev(ctx, r, pool, b.mothers, sizeof(unsigned long long) * b.G * 6 * b.N, false)) ||
            (s = load_dev(ctx, r, pool, b.m_alpha, sizeof(double) * b.G, false)) ||
            (s = load_dev(ctx, r, pool, b.gamma_d, sizeof(double) * b.G, false)) ||
            (s = load_dev(ctx, r, pool, b.B, sizeof(double) * D * b.n_obs * b.S, false)) ||
            (s = load_dev(ctx, r, pool, b.Omega, sizeof(double) * D, false)) ||
            (s = load_dev(ctx, r, pool, b.status, sizeof(int) * D, false)) ||
            (s = load_dev(ctx, r, pool, b.scal, sizeof(double) * D * 4, true)) ||
            (s = load_dev(ctx, r, pool, b.state, sizeof(unsigned long long) * D * 6 * b.N, true)) ||
            (s = load_dev(ctx, r, pool, b.feat, sizeof(double) * b.G * FEAT_RAW, true)) ||
            (s = load_dev(ctx, r, pool, b.types, sizeof(int) * b.N, true)) ||
            (s = load_dev(ctx, r, pool, b.lattice, sizeof(double) * 3 * b.N, true))) {
            fclose(f);
            return s;
        }
        if (b.confined != (b.types != nullptr) || (b.confined && !b.lattice))
            return bad(TTCF_E_INVALID, "checkpoint batch is inconsistent");
        if (steps_done > 0 && steps_done < c.n_steps && !b.confined && !b.state)
            return bad(TTCF_E_INVALID, "checkpoint of a partial run lacks the loop state");
        if (c.system == TTCF_BULK_WCA_ELONG) {   // the grid bound, as the spawn planned it
            ttcf_status ps = elong_plan(ctx, b.N, b.L, b.gamma, b);
            if (ps != TTCF_OK) { fclose(f); return ps; }
        }
        b.pairs = pool.get<unsigned long long>(D);
        b.rebuilds = pool.get<unsigned int>(D);
        if (pool.oom) return bad(TTCF_E_OOM, "device allocation failed (checkpoint)");
        CK(cudaMemsetAsync(b.pairs, 0, sizeof(unsigned long long) * D, ctx->st));
        CK(cudaMemsetAsync(b.rebuilds, 0, sizeof(unsigned int) * D, ctx->st));
        loaded.push_back(b);
    }
    fclose(f);
    pool.keep();
    ctx->batches = loaded;
    ctx->steps_done = steps_done;
    ctx->total_d = total_d;
    ctx->ran = steps_done > 0;
    ctx->tables_ok = false;
    if (steps_done >= c.n_steps) {   // a finished run: its reductions again
        for (auto &b : ctx->batches) {
            ttcf_status s = reduce_batch(ctx, b);
            if (s != TTCF_OK) return s;
        }
        CK(cudaStreamSynchronize(ctx->st));
    }
    return TTCF_OK;
}

// ======================================================= control variate ==
namespace {

uint64_t splitmix64(uint64_t &x) {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
double uniform01(uint64_t &x) { return (double)(splitmix64(x) >> 11) * (1.0 / 9007199254740992.0); }

bool batch_finished(ttcf_ctx *ctx, BatchHost *b) { return b && b->reduced; }

// Features X [D][32] (device, unstandardised) and targets z [D] (device).
// The network's forward pass (tensor cores) with its bounded waits checked.
ttcf_status cv_predict(ttcf_ctx *ctx, const __nv_bfloat16 *wb, const float *X, long long n, float *out,
                       cudaStream_t st) {
    CK(cv_tc_reset(st));
    CK(cv_launch_predict(wb, X, n, out, ctx->nsm, st));
    int failed = 0;
    CK(cv_tc_failed(st, &failed));
    if (failed) return fail(ctx, TTCF_E_TIMEOUT, "tensor-core forward pass: a wait on the MMAs timed out");
    return TTCF_OK;
}

// Raw features of G states of batch b's system from src ([G][6][N]: IEEE
// doubles, kind 0, or float-pair slots, kind 1) with the FP32 features kernel.
cudaError_t cv_raw_features(ttcf_ctx *ctx, const void *src, int kind, const BatchHost &b, int G, double *raw) {
    CvRawArgs ra;
    memset(&ra, 0, sizeof(ra));
    ra.src = src; ra.kind = kind; ra.N = b.N; ra.G = G; ra.raw = raw;
    for (int k = 0; k < 3; k++) {
        ra.L[k] = b.L[k];
        ra.nc[k] = std::max(3, (int)floor(b.L[k] / RC_WCA));
    }
    ra.ncell = ra.nc[0] * ra.nc[1] * ra.nc[2];
    if (cv_raw_smem_bytes(b.N, ra.ncell) > (size_t)ctx->smem_optin) return cudaErrorInvalidValue;
    return cv_launch_raw_features(ra, ctx->st);
}

ttcf_status cv_batch_data(ttcf_ctx *ctx, Pool &pool, BatchHost &b, float *&X, double *&z) {
    if (b.confined || b.elong || !b.feat)
        return fail(ctx, TTCF_E_INVALID, "the control variate needs a sheared bulk batch");
    for (int k = 0; k < b.M; k++)
        if (b.maps[k] > 3) return fail(ctx, TTCF_E_INVALID, "the control variate takes the mappings 0..3 of Eq. 3 only");
    const long long D = b.D();
    X = pool.get<float>((size_t)D * CV_NF);
    z = pool.get<double>((size_t)D);
    double *raw = pool.get<double>((size_t)b.G * FEAT_RAW);
    if (pool.oom) return fail(ctx, TTCF_E_OOM, "device allocation failed (cv data)");
    // the network's inputs come from the FP32 features kernel for every set
    // of states (training, evaluation, auxiliary): one function on all sides
    CK(cv_raw_features(ctx, b.mothers, ctx->cfg.precision == TTCF_MIXED ? 1 : 0, b, b.G, raw));
    CvFeatArgs fa;
    memset(&fa, 0, sizeof(fa));
    fa.raw = raw; fa.alpha = b.m_alpha; fa.reset_alpha = ctx->cfg.reset_alpha;
    fa.M = b.M; for (int k = 0; k < 4; k++) fa.maps[k] = b.maps[k];
    fa.D = D; fa.N = b.N; fa.V = b.V; fa.X = X;
    CK(cv_launch_features(fa, ctx->st));
    CK(cv_launch_targets(b.B, b.Omega, b.gamma_d, b.M, D, b.S,
                         ctx->cfg.sample_every * ctx->cfg.dt, z, ctx->st));
    return TTCF_OK;
}

std::vector<int> valid_groups(ttcf_ctx *ctx, BatchHost &b, ttcf_status &st) {
    std::vector<int> stv(b.D()), out;
    st = TTCF_OK;
    if (cudaMemcpy(stv.data(), b.status, sizeof(int) * b.D(), cudaMemcpyDeviceToHost) != cudaSuccess) {
        st = fail(ctx, TTCF_E_CUDA, "status read failed");
        return out;
    }
    for (int g = 0; g < b.G; g++) {
        int v = 0;
        for (int k = 0; k < b.M; k++) v |= stv[(size_t)g * b.M + k];
        if (v == 0) out.push_back(g);
    }
    return out;
}

}  // namespace

void ttcf_cv_config_default(ttcf_cv_config *c) {
    if (!c) return;
    c->epochs = 40;
    c->batch = 256;
    c->lr = 1e-3f; c->beta1 = 0.9f; c->beta2 = 0.999f; c->eps = 1e-8f;
    c->holdout = 0.2f;
    c->seed = 20231205ull;
}

ttcf_status ttcf_cv_data(ttcf_ctx *ctx, int batch_id, float *X, double *z, size_t capacity) {
    BatchHost *b = get_batch(ctx, batch_id);
    if (!b) return fail(ctx, TTCF_E_INVALID, "bad batch id");
    if (!batch_finished(ctx, b)) return fail(ctx, TTCF_E_STATE, "run not finished");
    if (capacity < (size_t)b->D()) return fail(ctx, TTCF_E_INVALID, "capacity smaller than the daughter count");
    Pool pool(ctx);
    float *dX; double *dz;
    ttcf_status s = cv_batch_data(ctx, pool, *b, dX, dz);
    if (s != TTCF_OK) return s;
    CK(cudaStreamSynchronize(ctx->st));
    if (X) CK(cudaMemcpy(X, dX, sizeof(float) * CV_NF * b->D(), cudaMemcpyDeviceToHost));
    if (z) CK(cudaMemcpy(z, dz, sizeof(double) * b->D(), cudaMemcpyDeviceToHost));
    return TTCF_OK;
}

ttcf_status ttcf_cv_train(ttcf_ctx *ctx, int batch_id, const ttcf_cv_config *cfg, double *loss_curve,
                          int capacity) {
    BatchHost *b = get_batch(ctx, batch_id);
    if (!b || !cfg) return fail(ctx, TTCF_E_INVALID, "bad batch id or NULL config");
    if (!batch_finished(ctx, b)) return fail(ctx, TTCF_E_STATE, "run not finished");
    if (cfg->epochs < 1 || cfg->batch < 32 || cfg->batch % 32 || !(cfg->lr > 0) ||
        !(cfg->holdout >= 0 && cfg->holdout < 1))
        return fail(ctx, TTCF_E_INVALID, "bad control-variate configuration");
    for (double g : b->gamma)
        if (g == 0.0) return fail(ctx, TTCF_E_INVALID, "training needs a nonzero shear rate");
    ttcf_status st;
    std::vector<int> groups = valid_groups(ctx, *b, st);
    if (st != TTCF_OK) return st;
    const int ng = (int)groups.size();
    const int nhold = std::max(2, (int)(cfg->holdout * ng));
    const int ntrain_g = ng - nhold;
    if (ntrain_g < 2) return fail(ctx, TTCF_E_INVALID, "too few valid groups to train");
    Pool tmp(ctx);
    float *X; double *z;
    ttcf_status s = cv_batch_data(ctx, tmp, *b, X, z);
    if (s != TTCF_OK) return s;
    const long long D = b->D();
    std::vector<int> rows;
    for (int k = 0; k < ntrain_g; k++)
        for (int m = 0; m < b->M; m++) rows.push_back(groups[k] * b->M + m);
    const int nrows = (int)rows.size();
    std::vector<int> hold(groups.begin() + ntrain_g, groups.end());
    float *zf = tmp.get<float>(D), *y = tmp.get<float>(D), *f = tmp.get<float>(D);
    int *d_rows = tmp.get<int>(nrows), *d_idx = tmp.get<int>(nrows), *d_hold = tmp.get<int>(nhold);
    int *d_step = tmp.get<int>(1);
    const int tiles = cfg->batch / 32;
    float *part = tmp.get<float>((size_t)tiles * CV_NP);
    double *lpart = tmp.get<double>(tiles), *loss = tmp.get<double>(1);
    double *yg = tmp.get<double>(nhold), *hg = tmp.get<double>(nhold), *est = tmp.get<double>(8);
    float *wbest = tmp.get<float>(CV_NP);
    CvModel &cvm = ctx->cv;
    if (!cvm.w) {
        Pool keep(ctx);
        cvm.w = keep.get<float>(CV_NP); cvm.m = keep.get<float>(CV_NP); cvm.v = keep.get<float>(CV_NP);
        cvm.wb = keep.get<__nv_bfloat16>(CV_NP);
        cvm.fstats = keep.get<double>(2 * CV_NF); cvm.zstats = keep.get<double>(2);
        if (keep.oom) return fail(ctx, TTCF_E_OOM, "device allocation failed (cv model)");
        keep.keep();
    }
    if (tmp.oom) return fail(ctx, TTCF_E_OOM, "device allocation failed (cv training)");
    cudaStream_t sm = ctx->st;
    CK(cudaMemcpyAsync(d_rows, rows.data(), sizeof(int) * nrows, cudaMemcpyHostToDevice, sm));
    CK(cudaMemcpyAsync(d_hold, hold.data(), sizeof(int) * nhold, cudaMemcpyHostToDevice, sm));
    // standardisation from the training rows
    CK(cv_launch_colstats(X, CV_NF, d_rows, nrows, CV_NF, cvm.fstats, sm));
    {
        std::vector<double> zh(D);
        CK(cudaStreamSynchronize(sm));
        CK(cudaMemcpy(zh.data(), z, sizeof(double) * D, cudaMemcpyDeviceToHost));
        std::vector<float> zfh(D);
        for (long long d = 0; d < D; d++) zfh[d] = (float)zh[d];
        CK(cudaMemcpy(zf, zfh.data(), sizeof(float) * D, cudaMemcpyHostToDevice));
    }
    CK(cv_launch_colstats(zf, 1, d_rows, nrows, 1, cvm.zstats, sm));
    CK(cv_launch_standardize(X, D, cvm.fstats, y, cvm.zstats, z, sm));
    // Xavier-uniform initialisation, zero biases (seeded splitmix64)
    {
        std::vector<float> w(CV_NP, 0.f);
        uint64_t sd = cfg->seed;
        auto fill = [&](int off, int fan_out, int fan_in) {
            const double a = sqrt(6.0 / (fan_in + fan_out));
            for (int k = 0; k < fan_out * fan_in; k++) w[off + k] = (float)((2.0 * uniform01(sd) - 1.0) * a);
        };
        fill(0, CV_H, CV_NF);
        fill(CV_H * CV_NF + CV_H, CV_H, CV_H);
        fill(CV_H * CV_NF + CV_H + CV_H * CV_H + CV_H, 1, CV_H);
        CK(cudaMemcpyAsync(cvm.w, w.data(), sizeof(float) * CV_NP, cudaMemcpyHostToDevice, sm));
        CK(cudaMemsetAsync(cvm.m, 0, sizeof(float) * CV_NP, sm));
        CK(cudaMemsetAsync(cvm.v, 0, sizeof(float) * CV_NP, sm));
        CK(cudaMemsetAsync(d_step, 0, sizeof(int), sm));
        CK(cv_launch_to_bf16(cvm.w, cvm.wb, sm));
        CK(cudaStreamSynchronize(sm));
    }
    // epochs over shuffled training rows (Fisher-Yates, splitmix64)
    const int nb = nrows / cfg->batch;   // full minibatches only
    if (nb < 1) return fail(ctx, TTCF_E_INVALID, "fewer training daughters than one minibatch");
    std::vector<int> perm(rows);
    uint64_t sh = cfg->seed ^ 0xA5A5A5A5A5A5A5A5ull;
    double best_gain = 0.0;
    for (int ep = 0; ep < cfg->epochs; ep++) {
        for (int k = nrows - 1; k > 0; k--) {
            const int j = (int)(splitmix64(sh) % (uint64_t)(k + 1));
            std::swap(perm[k], perm[j]);
        }
        CK(cudaMemcpyAsync(d_idx, perm.data(), sizeof(int) * nrows, cudaMemcpyHostToDevice, sm));
        CK(cudaMemsetAsync(loss, 0, sizeof(double), sm));
        for (int k = 0; k < nb; k++) {
            CK(cv_launch_grad(cvm.wb, X, y, d_idx, (long long)k * cfg->batch, cfg->batch, part, lpart,
                              d_step, sm));
            CK(cv_launch_adam(part, tiles, lpart, nullptr, loss, cvm.w, cvm.m, cvm.v, cvm.wb, d_step,
                              cfg->lr, cfg->beta1, cfg->beta2, cfg->eps, sm));
        }
        double l = 0.0;
        CK(cudaMemcpyAsync(&l, loss, sizeof(double), cudaMemcpyDeviceToHost, sm));
        // early stopping: the variance reduction 1/(1 - rho^2) of the group
        // control variate on the held-out groups; the best epoch's weights
        // are kept (the per-daughter target is mostly noise, and later
        // epochs fit it)
        { const ttcf_status ps = cv_predict(ctx, cvm.wb, X, D, f, sm); if (ps != TTCF_OK) return ps; }
        CK(cv_launch_group(z, f, cvm.zstats, b->M, d_hold, nhold, yg, hg, sm));
        CK(cv_launch_estimate(yg, hg, nhold, nullptr, 0, 1, 0.0, est, sm));
        double eh[8];
        CK(cudaMemcpyAsync(eh, est, sizeof(eh), cudaMemcpyDeviceToHost, sm));
        CK(cudaStreamSynchronize(sm));
        if (loss_curve && ep < capacity) loss_curve[ep] = l / nb;
        if (ep == 0 || eh[5] > best_gain) {
            best_gain = eh[5];
            CK(cudaMemcpyAsync(wbest, cvm.w, sizeof(float) * CV_NP, cudaMemcpyDeviceToDevice, sm));
        }
    }
    CK(cudaMemcpyAsync(cvm.w, wbest, sizeof(float) * CV_NP, cudaMemcpyDeviceToDevice, sm));
    CK(cv_launch_to_bf16(cvm.w, cvm.wb, sm));
    // c from the held-out groups
    { const ttcf_status ps = cv_predict(ctx, cvm.wb, X, D, f, sm); if (ps != TTCF_OK) return ps; }
    CK(cv_launch_group(z, f, cvm.zstats, b->M, d_hold, nhold, yg, hg, sm));
    CK(cv_launch_estimate(yg, hg, nhold, nullptr, 0, 1, 0.0, est, sm));
    double eh[8];
    CK(cudaMemcpyAsync(eh, est, sizeof(eh), cudaMemcpyDeviceToHost, sm));
    CK(cudaStreamSynchronize(sm));
    cvm.c = eh[4];
    cvm.trained = true;
    cvm.N = b->N;
    for (int k = 0; k < 3; k++) cvm.L[k] = b->L[k];
    return TTCF_OK;
}

ttcf_status ttcf_cv_apply(ttcf_ctx *ctx, int batch_id, int n_aux, const double *aux_soa,
                          const double *aux_alpha, double out[8]) {
    BatchHost *b = get_batch(ctx, batch_id);
    if (!b || !out) return fail(ctx, TTCF_E_INVALID, "bad batch id or NULL output");
    if (!ctx->cv.trained) return fail(ctx, TTCF_E_STATE, "control variate not trained");
    if (!batch_finished(ctx, b)) return fail(ctx, TTCF_E_STATE, "run not finished");
    if (b->N != ctx->cv.N) return fail(ctx, TTCF_E_INVALID, "evaluation batch N differs from training");
    for (int k = 0; k < b->M; k++)
        if (b->maps[k] > 3) return fail(ctx, TTCF_E_INVALID, "the control variate takes the mappings 0..3 of Eq. 3 only");
    if (n_aux < 2 || !aux_soa) return fail(ctx, TTCF_E_INVALID, "need >= 2 auxiliary mother states");
    for (double g : b->gamma)
        if (g == 0.0) return fail(ctx, TTCF_E_INVALID, "evaluation needs a nonzero shear rate");
    ttcf_status st;
    std::vector<int> groups = valid_groups(ctx, *b, st);
    if (st != TTCF_OK) return st;
    const int ng = (int)groups.size();
    if (ng < 2) return fail(ctx, TTCF_E_INVALID, "too few valid groups");
    Pool tmp(ctx);
    float *X; double *z;
    ttcf_status s = cv_batch_data(ctx, tmp, *b, X, z);
    if (s != TTCF_OK) return s;
    const long long D = b->D();
    CvModel &cvm = ctx->cv;
    cudaStream_t sm = ctx->st;
    float *f = tmp.get<float>(D);
    int *d_g = tmp.get<int>(ng);
    double *yg = tmp.get<double>(ng), *hg = tmp.get<double>(ng), *est = tmp.get<double>(8);
    if (tmp.oom) return fail(ctx, TTCF_E_OOM, "device allocation failed (cv apply)");
    CK(cudaMemcpyAsync(d_g, groups.data(), sizeof(int) * ng, cudaMemcpyHostToDevice, sm));
    CK(cv_launch_standardize(X, D, cvm.fstats, nullptr, nullptr, nullptr, sm));
    { const ttcf_status ps = cv_predict(ctx, cvm.wb, X, D, f, sm); if (ps != TTCF_OK) return ps; }
    CK(cv_launch_group(z, f, cvm.zstats, b->M, d_g, ng, yg, hg, sm));
    // auxiliary mothers: features (FP32 kernel, no daughters), mapped
    // features, predictions; host or device arrays (both pointers of one kind)
    int aux_dev = 0;
    {
        cudaPointerAttributes pa;
        if (cudaPointerGetAttributes(&pa, aux_soa) == cudaSuccess &&
            (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged))
            aux_dev = 1;
        cudaGetLastError();
    }
    // the auxiliary states need features only: no daughters are spawned
    const long long DA = (long long)n_aux * b->M;
    const size_t aslots = (size_t)n_aux * 6 * b->N;
    float *XA = tmp.get<float>((size_t)DA * CV_NF);
    float *fA = tmp.get<float>(DA);
    int *d_ga = tmp.get<int>(n_aux);
    double *hA = tmp.get<double>(n_aux);
    double *rawA = tmp.get<double>((size_t)n_aux * FEAT_RAW);
    double *alA = tmp.get<double>(n_aux);
    const double *srcA = aux_soa;
    if (!aux_dev) {
        double *d = tmp.get<double>(aslots);
        if (d) CK(cudaMemcpyAsync(d, aux_soa, sizeof(double) * aslots, cudaMemcpyHostToDevice, sm));
        srcA = d;
    }
    if (tmp.oom) return fail(ctx, TTCF_E_OOM, "device allocation failed (cv auxiliary)");
    if (aux_alpha)
        CK(cudaMemcpyAsync(alA, aux_alpha, sizeof(double) * n_aux,
                           aux_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, sm));
    else
        CK(cudaMemsetAsync(alA, 0, sizeof(double) * n_aux, sm));
    CK(cv_raw_features(ctx, srcA, 0, *b, n_aux, rawA));
    CvFeatArgs fa;
    memset(&fa, 0, sizeof(fa));
    fa.raw = rawA; fa.alpha = alA; fa.reset_alpha = ctx->cfg.reset_alpha;
    fa.M = b->M; for (int k = 0; k < 4; k++) fa.maps[k] = b->maps[k];
    fa.D = DA; fa.N = b->N; fa.V = b->V; fa.X = XA;
    CK(cv_launch_features(fa, sm));
    CK(cv_launch_standardize(XA, DA, cvm.fstats, nullptr, nullptr, nullptr, sm));
    { const ttcf_status ps = cv_predict(ctx, cvm.wb, XA, DA, fA, sm); if (ps != TTCF_OK) return ps; }
    {
        std::vector<int> ga(n_aux);
        for (int k = 0; k < n_aux; k++) ga[k] = k;
        CK(cudaMemcpyAsync(d_ga, ga.data(), sizeof(int) * n_aux, cudaMemcpyHostToDevice, sm));
        CK(cv_launch_group(nullptr, fA, cvm.zstats, b->M, d_ga, n_aux, nullptr, hA, sm));
        CK(cv_launch_estimate(yg, hg, ng, hA, n_aux, 0, cvm.c, est, sm));
        CK(cudaMemcpyAsync(out, est, sizeof(double) * 8, cudaMemcpyDeviceToHost, sm));
        CK(cudaStreamSynchronize(sm));
    }
    return TTCF_OK;
}

ttcf_status ttcf_cv_get_model(ttcf_ctx *ctx, float *params, double *feat_stats, double *z_stats,
                              double *c) {
    if (!ctx) return fail(ctx, TTCF_E_INVALID, "NULL context");
    if (!ctx->cv.trained) return fail(ctx, TTCF_E_STATE, "control variate not trained");
    CK(cudaStreamSynchronize(ctx->st));
    if (params) CK(cudaMemcpy(params, ctx->cv.w, sizeof(float) * CV_NP, cudaMemcpyDeviceToHost));
    if (feat_stats) CK(cudaMemcpy(feat_stats, ctx->cv.fstats, sizeof(double) * 2 * CV_NF, cudaMemcpyDeviceToHost));
    if (z_stats) CK(cudaMemcpy(z_stats, ctx->cv.zstats, sizeof(double) * 2, cudaMemcpyDeviceToHost));
    if (c) *c = ctx->cv.c;
    return TTCF_OK;
}

static ttcf_status cv_upload_params(ttcf_ctx *ctx, Pool &tmp, const float *params, __nv_bfloat16 *&wb) {
    float *w = tmp.get<float>(CV_NP);
    wb = tmp.get<__nv_bfloat16>(CV_NP);
    if (tmp.oom) return fail(ctx, TTCF_E_OOM, "device allocation failed (params)");
    CK(cudaMemcpyAsync(w, params, sizeof(float) * CV_NP, cudaMemcpyHostToDevice, ctx->st));
    CK(cv_launch_to_bf16(w, wb, ctx->st));
    return TTCF_OK;
}

ttcf_status ttcf_cv_forward(ttcf_ctx *ctx, const float *params, int n, const float *X, float *out) {
    if (!ctx || !params || !X || !out || n < 1) return fail(ctx, TTCF_E_INVALID, "bad arguments");
    Pool tmp(ctx);
    __nv_bfloat16 *wb;
    ttcf_status s = cv_upload_params(ctx, tmp, params, wb);
    if (s != TTCF_OK) return s;
    float *dX = tmp.get<float>((size_t)n * CV_NF), *df = tmp.get<float>(n);
    if (tmp.oom) return fail(ctx, TTCF_E_OOM, "device allocation failed (forward)");
    CK(cudaMemcpyAsync(dX, X, sizeof(float) * n * CV_NF, cudaMemcpyHostToDevice, ctx->st));
    { const ttcf_status ps = cv_predict(ctx, wb, dX, n, df, ctx->st); if (ps != TTCF_OK) return ps; }
    CK(cudaMemcpyAsync(out, df, sizeof(float) * n, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return TTCF_OK;
}

ttcf_status ttcf_cv_gradient(ttcf_ctx *ctx, const float *params, int n, const float *X,
                             const float *y, float *grad, double *loss) {
    if (!ctx || !params || !X || !y || n < 1 || n > 65536) return fail(ctx, TTCF_E_INVALID, "bad arguments");
    Pool tmp(ctx);
    __nv_bfloat16 *wb;
    ttcf_status s = cv_upload_params(ctx, tmp, params, wb);
    if (s != TTCF_OK) return s;
    const int tiles = (n + 31) / 32;
    float *dX = tmp.get<float>((size_t)n * CV_NF), *dy = tmp.get<float>(n);
    float *part = tmp.get<float>((size_t)tiles * CV_NP), *dg = tmp.get<float>(CV_NP);
    double *lpart = tmp.get<double>(tiles), *dl = tmp.get<double>(1);
    if (tmp.oom) return fail(ctx, TTCF_E_OOM, "device allocation failed (gradient)");
    CK(cudaMemcpyAsync(dX, X, sizeof(float) * n * CV_NF, cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(dy, y, sizeof(float) * n, cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemsetAsync(dl, 0, sizeof(double), ctx->st));
    CK(cv_launch_grad(wb, dX, dy, nullptr, 0, n, part, lpart, nullptr, ctx->st));
    CK(cv_launch_adam(part, tiles, lpart, dg, dl, nullptr, nullptr, nullptr, nullptr, nullptr, 0.f,
                      0.f, 0.f, 0.f, ctx->st));
    if (grad) CK(cudaMemcpyAsync(grad, dg, sizeof(float) * CV_NP, cudaMemcpyDeviceToHost, ctx->st));
    double l = 0.0;
    CK(cudaMemcpyAsync(&l, dl, sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    if (loss) *loss = l;
    return TTCF_OK;
}

}  // extern "C"
