// C ABI of the RVE block (see include/fe2.h): context, RVE registry with
// HBM-budget admission, id-list cache, transient workspace, and the launch
// sequences of the assemble / reduce / condense / macro-step calls.
#include <algorithm>
#include <cmath>
#include <chrono>
#include <cstdarg>
#include <deque>
#include <unordered_set>
#include <cstdio>
#include <cstring>
#include <map>
#include <set>
#include <string>
#include <vector>

#include "fe2_internal.cuh"

using namespace fe2;

namespace {

struct HostRve {
    bool active = false;
    bool all_linear = true;
    int chunk = -1;       // allocation chunk
    std::vector<double> mat;
    // RVEs defined by fe2_rve_define hold device state only while resident (in a slot)
    bool deferred = false;
    bool resident = true;
    char* slot = nullptr;
    std::vector<uint8_t> phase;  // host definition
    std::vector<double> w;       // w~ (folded order) while not resident
    bool w_zero = true;
    unsigned long long last_use = 0;
};

struct Chunk {
    void* dev = nullptr;
    int refs = 0;
};

struct IdList {
    std::vector<int> ids;
    int* dev = nullptr;
    int* pinned = nullptr;
    unsigned long long last = 0;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

struct fe2_ctx {
    fe2_config cfg{};
    cudaStream_t stream = nullptr;
    std::string err;
    int max_smem = 0;
    // registry
    std::vector<RveDev> mirror;
    std::vector<HostRve> host;
    std::vector<int> free_ids;
    std::vector<Chunk> chunks;
    RveDev* d_tab = nullptr;
    int tab_cap = 0;
    size_t persistent_bytes = 0;
    // transient buffers
    char* ws = nullptr;
    size_t ws_bytes = 0;
    double* elem = nullptr;
    size_t elem_bytes = 0;
    std::vector<int> elem_ids;     // ids whose element data is in `elem`
    int* d_status_tmp = nullptr;
    size_t status_tmp_n = 0;
    int* d_redo = nullptr;          // per-slot "refine again" flags of the mixed path
    size_t redo_n = 0;
    double* d_tol = nullptr;        // device copy of cfg.refine_tol
    // id-list cache
    std::vector<IdList> idcache;
    unsigned long long tick = 0;
    long long launches = 0;
    std::map<int, int> kd_cache;
    std::map<int, int*> nbr_tabs;   // N -> device table [N^d][3^d]
    // per-kernel event timing
    bool prof = false;
    struct Pending {
        std::string name;
        cudaEvent_t a, b;
    };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> evpool;
    std::map<std::string, std::pair<double, long long>> totals;
    // macro problem
    bool macro_ready = false;
    MacroDev macro{};
    std::vector<double> macro_X;    // reference nodal positions [nnode][d] (host copy)
    std::vector<void*> macro_bufs;  // device buffers owned by the macro problem
    // slots of the RVEs defined by fe2_rve_define (uniform size, allocated in slabs)
    size_t slot_bytes = 0;
    std::vector<void*> slabs;
    std::vector<char*> free_slots;
    size_t extra_bytes = 0;         // device bytes counted against the budget by a server (lanes)
    std::set<std::pair<unsigned long long, int>> lru;  // resident defined RVEs by last use
    int def_maxN = 0;                                  // largest defined mesh size
    long long n_admitted = 0, n_evicted = 0;
    int* d_macro_status = nullptr;
};

static fe2_status fail(fe2_ctx* c, fe2_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return s;
}

#define CK(call)                                                                                       \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) return fail(ctx, FE2_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// ------------------------------------------------------------------ sizes
static int nodes_of(int N, int d) { return d == 2 ? N * N : N * N * N; }

static int compute_kd(fe2_ctx* ctx, int N, int d) {
    auto it = ctx->kd_cache.find(N * 4 + d);
    if (it != ctx->kd_cache.end()) return it->second;
    int kd = 0;
    const int nn = nodes_of(N, d);
    if (d == 2) {
        for (int q = 1; q < nn; ++q) {
            const int i = unfold_pos(q % N, N), j = unfold_pos(q / N, N);
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int qn = fold_pos((i + dx + N) % N, N) + N * fold_pos((j + dy + N) % N, N);
                    if (qn == 0) continue;
                    kd = std::max(kd, 2 * std::abs(qn - q) + 1);
                }
        }
    } else {
        for (int q = 1; q < nn; ++q) {
            const int i = unfold_pos(q % N, N), j = unfold_pos((q / N) % N, N), k = unfold_pos(q / (N * N), N);
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int qn = fold_pos((i + dx + N) % N, N) + N * fold_pos((j + dy + N) % N, N) +
                                       N * N * fold_pos((k + dz + N) % N, N);
                        if (qn == 0) continue;
                        kd = std::max(kd, 3 * std::abs(qn - q) + 2);
                    }
        }
    }
    // the factorisation window needs kd >= NB (a panel must lie inside the band
    // storage); for small meshes the extra band rows are structural zeros
    kd = std::max(kd, NB);
    ctx->kd_cache[N * 4 + d] = kd;
    return kd;
}

static const int* nbr_table(fe2_ctx* ctx, int N, int d) {
    auto it = ctx->nbr_tabs.find(N * 4 + d);
    if (it != ctx->nbr_tabs.end()) return it->second;
    const int nn = nodes_of(N, d), ns = d == 2 ? 9 : 27;
    std::vector<int> t((size_t)nn * ns);
    for (int q = 0; q < nn; ++q) {
        int c[3] = {0, 0, 0};
        int qq = q;
        for (int k = 0; k < d; ++k) {
            c[k] = unfold_pos(qq % N, N);
            qq /= N;
        }
        for (int off = 0; off < ns; ++off) {
            int o = off, qn = 0, mul = 1;
            for (int k = 0; k < d; ++k) {
                const int dk = o % 3 - 1;
                o /= 3;
                const int v = (c[k] + dk + N) % N;
                qn += fold_pos(v, N) * mul;
                mul *= N;
            }
            t[(size_t)q * ns + off] = qn;
        }
    }
    int* dptr = nullptr;
    if (cudaMalloc(&dptr, sizeof(int) * t.size()) != cudaSuccess) return nullptr;
    if (cudaMemcpy(dptr, t.data(), sizeof(int) * t.size(), cudaMemcpyHostToDevice) != cudaSuccess) return nullptr;
    ctx->nbr_tabs[N * 4 + d] = dptr;
    return dptr;
}

static size_t persistent_bytes_of(int N, int d, int nphase, int nq = 1) {
    const int nn = nodes_of(N, d), nm = d * (nn - 1), nr = d * d * nq + 1;
    const int nst = (d == 2 ? 9 : 27) * d * d;
    size_t b = 0;
    b += align256(nn);                               // phase
    b += align256((size_t)nphase * 4 * 8);           // mat
    b += align256((size_t)nm * 8);                   // w
    b += align256((size_t)nst * nn * 8);             // stencil
    b += 2 * align256((size_t)nr * nm * 8);          // rhs, X
    b += align256((size_t)(d * d * d * d + d * d) * nq * 8);  // KMM, Pint per macro Gauss point
    return b;
}

// Device pointers of one RVE's persistent state inside `base` (the layout that
// persistent_bytes_of counts); r.d, nn, nm, nr and nphase must be set.
static void place_rve(RveDev& r, char* base, int nst, int nq) {
    const int d = r.d, nn = r.nn, nm = r.nm, nr = r.nr;
    size_t o = 0;
    r.phase = (const uint8_t*)(base + o);
    o += align256(nn);
    r.mat = (const double*)(base + o);
    o += align256((size_t)r.nphase * 4 * 8);
    r.w = (double*)(base + o);
    o += align256((size_t)nm * 8);
    r.stencil = (double*)(base + o);
    o += align256((size_t)nst * nn * 8);
    r.rhs = (double*)(base + o);
    o += align256((size_t)nr * nm * 8);
    r.X = (double*)(base + o);
    o += align256((size_t)nr * nm * 8);
    r.KMM = (double*)(base + o);  // [nq][d^4], then Pint [nq][d^2]
    r.Pint = r.KMM + d * d * d * d * nq;
}

// macro Gauss points per RVE: 1 (Dirac basis) or 4 (element RVE, piecewise-constant basis)
static int nq_of(const fe2_ctx* ctx) { return ctx->cfg.macro_basis == FE2_BASIS_CONST ? MAX_NQ : 1; }

struct WsLayout {
    size_t offY, offR, offD, offWin, stride;
    bool gw;  // wide band: the factor window lives in global memory
};

// The shared-memory band factor serves bands whose window fits one CTA; wider
// bands (3D) use the global-window kernel.
static bool use_smem_factor(int kd, int nr, bool fp64, int max_smem, int d) {
    return d == 2 && kd + nr + 32 <= FACT_THREADS && (int)factor_smem_bytes(kd, nr, fp64) <= max_smem;
}

// Mixed path: the tensor-core FP32 factor when the context asks for it and
// the band fits it; the CUDA-core kernel otherwise (and by default).
static bool use_tc_factor(const fe2_ctx* ctx, int maxkd, int maxnr) {
    return ctx->cfg.factor_kernel == FE2_FACTOR_TENSOR_CORE &&
           (factor_tc2_eligible(maxkd, maxnr, ctx->cfg.dim, ctx->max_smem) ||
            factor_tc_eligible(maxkd, maxnr, ctx->cfg.dim, ctx->max_smem));
}

// The tensor-core factor: two RVEs per SM where the band allows it, else one.
static cudaError_t launch_tc_factor(const fe2_ctx* ctx, const RveDev* tab, const int* ids, int n, Workspace ws,
                                    int* st, int maxkd, int maxnr, cudaStream_t s) {
    if (factor_tc2_eligible(maxkd, maxnr, ctx->cfg.dim, ctx->max_smem))
        return launch_factor_tc2(tab, ids, n, ws, st, maxkd, maxnr, s);
    return launch_factor_tc(tab, ids, n, ws, st, maxkd, maxnr, s);
}

// The pipelined band factor when the context asks for it and the band fits it.
static bool use_la_factor(const fe2_ctx* ctx, int maxkd, int maxnr, bool fp64) {
    return ctx->cfg.factor_kernel == FE2_FACTOR_CUDA_CORE_PIPELINED && ctx->cfg.dim == 2 &&
           factor_la_eligible(maxkd, maxnr, fp64, ctx->max_smem);
}

static WsLayout ws_layout(int maxkd, int maxnr, int maxnm, int maxnmp, bool fp64, int max_smem, int d) {
    const size_t es = fp64 ? 8 : 4;
    WsLayout l;
    l.gw = !use_smem_factor(maxkd, maxnr, fp64, max_smem, d);
    size_t o = align256((size_t)maxnmp * (maxkd + 1) * es);
    l.offY = o;
    o += align256((size_t)maxnr * maxnmp * es);
    l.offR = o;
    o += align256((size_t)maxnr * maxnm * 8);
    l.offD = o;
    o += align256((size_t)maxnmp * es);
    l.offWin = o;  // unused: the wide-band factor works in L itself
    l.stride = o;
    return l;
}

static fe2_status free_ws(fe2_ctx* ctx) {
    if (!ctx->ws) return FE2_OK;
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaFree(ctx->ws));
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
    return FE2_OK;
}

// Make the transient workspace hold `bytes`; a workspace larger than `limit`
// (what the budget leaves) is released first.
static fe2_status ensure_ws(fe2_ctx* ctx, size_t bytes, size_t limit = (size_t)-1) {
    if (ctx->ws_bytes > limit) {
        fe2_status st = free_ws(ctx);
        if (st != FE2_OK) return st;
    }
    if (bytes <= ctx->ws_bytes) return FE2_OK;
    CK(cudaStreamSynchronize(ctx->stream));
    if (ctx->ws) CK(cudaFree(ctx->ws));
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
    CK(cudaMalloc(&ctx->ws, bytes));
    ctx->ws_bytes = bytes;
    return FE2_OK;
}

// device bytes held against the HBM budget (a server's lane buffers included)
static size_t used_bytes(const fe2_ctx* c) {
    return c->persistent_bytes + c->ws_bytes + c->elem_bytes + c->extra_bytes;
}

// ------------------------------------------------------------------ id lists
static fe2_status get_ids(fe2_ctx* ctx, int n, const int* ids, const int** dev) {
    if (n <= 0 || !ids) return fail(ctx, FE2_ERR_ARG, "empty id list");
    for (int k = 0; k < n; ++k) {
        const int id = ids[k];
        if (id < 0 || id >= (int)ctx->host.size() || !ctx->host[id].active)
            return fail(ctx, FE2_ERR_ARG, "rve id %d is not registered", id);
        if (!ctx->host[id].resident)
            return fail(ctx, FE2_ERR_ARG, "rve %d is not resident (fe2_rve_admit it first)", id);
    }
    ++ctx->tick;
    for (auto& e : ctx->idcache) {
        if ((int)e.ids.size() == n && std::memcmp(e.ids.data(), ids, sizeof(int) * n) == 0) {
            e.last = ctx->tick;
            *dev = e.dev;
            return FE2_OK;
        }
    }
    {  // duplicates would race inside a launch
        std::vector<int> s(ids, ids + n);
        std::sort(s.begin(), s.end());
        if (std::adjacent_find(s.begin(), s.end()) != s.end())
            return fail(ctx, FE2_ERR_ARG, "duplicate rve id in one call");
    }
    if (ctx->idcache.size() >= 16) {
        auto lru = std::min_element(ctx->idcache.begin(), ctx->idcache.end(),
                                    [](const IdList& a, const IdList& b) { return a.last < b.last; });
        CK(cudaStreamSynchronize(ctx->stream));
        cudaFree(lru->dev);
        cudaFreeHost(lru->pinned);
        ctx->idcache.erase(lru);
    }
    IdList e;
    e.ids.assign(ids, ids + n);
    CK(cudaMalloc(&e.dev, sizeof(int) * n));
    CK(cudaMallocHost(&e.pinned, sizeof(int) * n));
    std::memcpy(e.pinned, ids, sizeof(int) * n);
    CK(cudaMemcpyAsync(e.dev, e.pinned, sizeof(int) * n, cudaMemcpyHostToDevice, ctx->stream));
    e.last = ctx->tick;
    ctx->idcache.push_back(e);
    *dev = ctx->idcache.back().dev;
    return FE2_OK;
}

static void drop_cached_lists_with(fe2_ctx* ctx, const std::vector<int>& released) {
    if (ctx->idcache.empty()) return;
    std::vector<char> mark(ctx->host.size(), 0);
    for (int id : released) mark[id] = 1;
    bool synced = false;
    for (size_t k = 0; k < ctx->idcache.size();) {
        bool hit = false;
        for (int id : ctx->idcache[k].ids) hit |= mark[id] != 0;
        if (hit) {
            if (!synced) {
                cudaStreamSynchronize(ctx->stream);
                synced = true;
            }
            cudaFree(ctx->idcache[k].dev);
            cudaFreeHost(ctx->idcache[k].pinned);
            ctx->idcache.erase(ctx->idcache.begin() + k);
        } else {
            ++k;
        }
    }
}

struct BatchInfo {
    int maxN = 0, maxkd = 0, maxnr = 0, maxnm = 0, maxnmp = 0, maxnn = 0, maxnphase = 0;
    bool all_linear = true;
    // assembly kernel selector: 0 general, 1 linear, 2 linear with node rows tabulated
    // by phase combination (at most 3 phases per RVE)
    int linear_mode() const { return all_linear ? (maxnphase <= 3 ? 2 : 1) : 0; }
};

static BatchInfo batch_info(const fe2_ctx* ctx, int n, const int* ids) {
    BatchInfo b;
    for (int k = 0; k < n; ++k) {
        const RveDev& r = ctx->mirror[ids[k]];
        b.maxN = std::max(b.maxN, r.N);
        b.maxkd = std::max(b.maxkd, r.kd);
        b.maxnphase = std::max(b.maxnphase, r.nphase);
        b.maxnr = std::max(b.maxnr, r.nr);
        b.maxnm = std::max(b.maxnm, r.nm);
        b.maxnmp = std::max(b.maxnmp, r.nm_pad);
        b.maxnn = std::max(b.maxnn, r.nn);
        b.all_linear &= ctx->host[ids[k]].all_linear;
    }
    return b;
}

static fe2_status upload_desc(fe2_ctx* ctx, int id) {
    // the source lives in a std::vector that may move: complete the copy now
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaMemcpy(ctx->d_tab + id, &ctx->mirror[id], sizeof(RveDev), cudaMemcpyHostToDevice));
    return FE2_OK;
}

static fe2_status upload_all(fe2_ctx* ctx) {
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaMemcpy(ctx->d_tab, ctx->mirror.data(), sizeof(RveDev) * ctx->mirror.size(), cudaMemcpyHostToDevice));
    return FE2_OK;
}

// ------------------------------------------------------------------ timing
static cudaEvent_t take_event(fe2_ctx* ctx) {
    if (!ctx->evpool.empty()) {
        cudaEvent_t e = ctx->evpool.back();
        ctx->evpool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

struct KTimer {
    fe2_ctx* ctx;
    const char* name;
    cudaEvent_t a = nullptr;
    KTimer(fe2_ctx* c, const char* n) : ctx(c), name(n) {
        ++ctx->launches;
        if (ctx->prof) {
            a = take_event(ctx);
            cudaEventRecord(a, ctx->stream);
        }
    }
    ~KTimer() {
        if (ctx->prof) {
            cudaEvent_t b = take_event(ctx);
            cudaEventRecord(b, ctx->stream);
            ctx->pending.push_back({name, a, b});
        }
    }
};

static void drain_timing(fe2_ctx* ctx) {
    if (ctx->pending.empty()) return;
    cudaStreamSynchronize(ctx->stream);
    for (auto& p : ctx->pending) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, p.a, p.b);
        auto& t = ctx->totals[p.name];
        t.first += ms;
        t.second += 1;
        ctx->evpool.push_back(p.a);
        ctx->evpool.push_back(p.b);
    }
    ctx->pending.clear();
}

#define TIMED(name, call)                     \
    do {                                      \
        KTimer kt_(ctx, name);                \
        CK(call);                             \
    } while (0)

// ------------------------------------------------------------------ condensation
static fe2_status condense_impl(fe2_ctx* ctx, int n, const int* ids, const int* d_ids, double* sigma,
                                double* Cbar, int* status, double* err, bool reset_status) {
    const BatchInfo b = batch_info(ctx, n, ids);
    const bool fp64 = ctx->cfg.precision == FE2_PREC_FP64;
    const WsLayout l = ws_layout(b.maxkd, b.maxnr, b.maxnm, b.maxnmp, fp64, ctx->max_smem, ctx->cfg.dim);
    // chunk the batch so that its workspace fits the budget
    int cap = n;
    size_t limit = (size_t)-1;
    if (ctx->cfg.hbm_budget_bytes) {
        const size_t used = ctx->persistent_bytes + ctx->elem_bytes;
        limit = ctx->cfg.hbm_budget_bytes > used ? ctx->cfg.hbm_budget_bytes - used : 0;
        cap = (int)std::min<size_t>((size_t)n, limit / l.stride);
        if (cap < 1) return fail(ctx, FE2_ERR_BUDGET, "no room for one RVE of workspace within the HBM budget");
    }
    fe2_status st = ensure_ws(ctx, l.stride * (size_t)cap, limit);
    if (st != FE2_OK) return st;
    if (reset_status) CK(cudaMemsetAsync(status, 0, sizeof(int) * n, ctx->stream));
    Workspace ws{ctx->ws, l.stride, l.offY, l.offR, l.offD, l.offWin};
    // per-RVE output sizes: sigma [nq][d^2], Cbar [nq d^2][nq d^2]
    const int dd = ctx->cfg.dim * ctx->cfg.dim * nq_of(ctx);
    const bool d3 = ctx->cfg.dim == 3, elem = nq_of(ctx) > 1;
    auto residual = [&](const int* di, int m, const int* active) {
        return d3     ? launch_residual3(ctx->d_tab, di, m, ws, b.maxnn, active, ctx->stream)
               : elem ? launch_residual_elem(ctx->d_tab, di, m, ws, b.maxnn, active, ctx->stream)
                      : launch_residual(ctx->d_tab, di, m, ws, b.maxnn, active, ctx->stream);
    };
    auto schur = [&](const int* di, int m, int corrected, double* sg, double* cb, int* stp, double* er,
                     const double* tol, int* redo, int sweep) {
        return d3     ? launch_schur3(ctx->d_tab, di, m, ws, corrected, sg, cb, stp, er, tol, redo, ctx->stream, sweep)
               : elem ? launch_schur_elem(ctx->d_tab, di, m, ws, corrected, sg, cb, stp, er, tol, redo, ctx->stream,
                                          sweep)
                      : launch_schur(ctx->d_tab, di, m, ws, corrected, sg, cb, stp, er, tol, redo, ctx->stream, sweep);
    };
    for (int c0 = 0; c0 < n; c0 += cap) {
        const int m = std::min(cap, n - c0);
        const int* di = d_ids + c0;
        int* stp = status + c0;
        double* sg = sigma + (size_t)c0 * dd;
        double* cb = Cbar + (size_t)c0 * dd * dd;
        double* er = err ? err + c0 : nullptr;
        if (fp64) {
            if (l.gw)
                TIMED("band_factor_fp64_gw", launch_factor_gw<double>(ctx->d_tab, di, m, ws, stp, b.maxkd, b.maxnr, ctx->stream));
            else if (use_la_factor(ctx, b.maxkd, b.maxnr, true))
                TIMED("band_factor_fp64_pipelined", launch_factor_la<double>(ctx->d_tab, di, m, ws, stp, b.maxkd, b.maxnr, ctx->stream));
            else
                TIMED("band_factor_fp64", launch_factor<double>(ctx->d_tab, di, m, ws, stp, b.maxkd, b.maxnr, ctx->stream));
            TIMED("band_backward_fp64",
                  launch_backward<double>(ctx->d_tab, di, m, ws, 0, b.maxkd, b.maxnr, b.maxnmp, stp, ctx->stream));
            TIMED("schur", schur(di, m, 0, sg, cb, stp, er, nullptr, nullptr, 0));
        } else {
            // FP32 factor, one FP64 residual and the residual-corrected Schur complement;
            // RVEs whose error estimate exceeds refine_tol get up to max_refine sweeps
            // of FP64-residual refinement (the others skip the launches' work)
            if ((size_t)cap > ctx->redo_n) {
                CK(cudaStreamSynchronize(ctx->stream));
                cudaFree(ctx->d_redo);
                ctx->d_redo = nullptr;
                CK(cudaMalloc(&ctx->d_redo, sizeof(int) * cap));
                ctx->redo_n = cap;
            }
            int* redo = ctx->cfg.max_refine > 0 ? ctx->d_redo : nullptr;
            if (l.gw)
                TIMED("band_factor_fp32_gw", launch_factor_gw<float>(ctx->d_tab, di, m, ws, stp, b.maxkd, b.maxnr, ctx->stream));
            else if (use_tc_factor(ctx, b.maxkd, b.maxnr))
                TIMED("band_factor_tc", launch_tc_factor(ctx, ctx->d_tab, di, m, ws, stp, b.maxkd, b.maxnr, ctx->stream));
            else if (use_la_factor(ctx, b.maxkd, b.maxnr, false))
                TIMED("band_factor_fp32_pipelined", launch_factor_la<float>(ctx->d_tab, di, m, ws, stp, b.maxkd, b.maxnr, ctx->stream));
            else
                TIMED("band_factor_fp32", launch_factor<float>(ctx->d_tab, di, m, ws, stp, b.maxkd, b.maxnr, ctx->stream));
            TIMED("band_backward_fp32",
                  launch_backward<float>(ctx->d_tab, di, m, ws, 0, b.maxkd, b.maxnr, b.maxnmp, stp, ctx->stream));
            TIMED("residual_fp64", residual(di, m, nullptr));
            // Dirac-basis RVEs: every RVE gets the correction dx from the FP32 factor
            // and the second-order corrected Schur complement; further sweeps, and every
            // sweep of element RVEs, go to the RVEs whose estimate exceeds refine_tol
            int it0 = 0;
            if (!elem && ctx->cfg.max_refine > 0) {
                TIMED("band_correct_fp32", launch_solve_correct<float>(ctx->d_tab, di, m, ws, b.maxkd, b.maxnr,
                                                                       b.maxnmp, stp, nullptr, ctx->stream, 1));
                TIMED("schur", schur(di, m, 2, sg, cb, stp, er, ctx->d_tol, redo, ctx->cfg.max_refine > 1 ? 0 : 3));
                it0 = 1;
            } else {
                TIMED("schur", schur(di, m, 1, sg, cb, stp, er, ctx->d_tol, redo, ctx->cfg.max_refine > 0 ? 0 : 3));
            }
            for (int it = it0; it < ctx->cfg.max_refine; ++it) {
                const bool last = it + 1 == ctx->cfg.max_refine;
                // after the second-order pass X has advanced: its residual first
                if (it0) TIMED("residual_fp64_refine", residual(di, m, ctx->d_redo));
                TIMED("band_refine_fp32", launch_solve_correct<float>(ctx->d_tab, di, m, ws, b.maxkd, b.maxnr, b.maxnmp,
                                                                      stp, ctx->d_redo, ctx->stream));
                TIMED("residual_fp64_refine", residual(di, m, ctx->d_redo));
                TIMED("schur_refine", schur(di, m, 1, sg, cb, stp, er, ctx->d_tol, ctx->d_redo, last ? 2 : 1));
            }
        }
    }
    return FE2_OK;
}

template <typename V>
static fe2_status upload_vec(fe2_ctx* ctx, const std::vector<V>& h, V** out) {
    V* d = nullptr;
    CK(cudaMalloc(&d, sizeof(V) * std::max<size_t>(h.size(), 1)));
    ctx->macro_bufs.push_back(d);
    if (!h.empty()) CK(cudaMemcpy(d, h.data(), sizeof(V) * h.size(), cudaMemcpyHostToDevice));
    *out = d;
    return FE2_OK;
}

// ================================================================== C ABI
extern "C" {

fe2_status fe2_create(const fe2_config* cfg, fe2_ctx** out) {
    fe2_ctx* ctx = nullptr;
    if (!cfg || !out) return FE2_ERR_ARG;
    *out = nullptr;
    if (cfg->dim != 2 && cfg->dim != 3) return FE2_ERR_ARG;
    if ((cfg->dim == 2) != (cfg->elem == FE2_ELEM_Q4)) return FE2_ERR_ARG;
    if (cfg->precision != FE2_PREC_FP64 && cfg->precision != FE2_PREC_MIXED) return FE2_ERR_ARG;
    if (cfg->max_refine < 0 || cfg->max_refine > 16) return FE2_ERR_ARG;
    if (cfg->factor_kernel < FE2_FACTOR_AUTO || cfg->factor_kernel > FE2_FACTOR_CUDA_CORE_PIPELINED) return FE2_ERR_ARG;
    if (cfg->macro_basis != FE2_BASIS_DIRAC && cfg->macro_basis != FE2_BASIS_CONST) return FE2_ERR_ARG;
    if (cfg->macro_basis == FE2_BASIS_CONST && cfg->dim != 2) return FE2_ERR_ARG;
    ctx = new fe2_ctx();
    ctx->cfg = *cfg;
    if (!(ctx->cfg.refine_tol > 0.0)) ctx->cfg.refine_tol = 1e-10;
    ctx->stream = (cudaStream_t)cfg->cuda_stream;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_tol, sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(ctx->d_tol, &ctx->cfg.refine_tol, sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        delete ctx;
        return FE2_ERR_CUDA;
    }
    *out = ctx;
    return FE2_OK;
}

void fe2_destroy(fe2_ctx* ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    for (auto& c : ctx->chunks)
        if (c.dev) cudaFree(c.dev);
    for (void* p : ctx->slabs) cudaFree(p);
    for (auto& e : ctx->idcache) {
        cudaFree(e.dev);
        cudaFreeHost(e.pinned);
    }
    cudaFree(ctx->d_tab);
    cudaFree(ctx->ws);
    cudaFree(ctx->elem);
    cudaFree(ctx->d_status_tmp);
    cudaFree(ctx->d_redo);
    cudaFree(ctx->d_tol);
    for (void* p : ctx->macro_bufs) cudaFree(p);
    cudaFree(ctx->d_macro_status);
    for (auto& t : ctx->nbr_tabs) cudaFree(t.second);
    drain_timing(ctx);
    for (auto e : ctx->evpool) cudaEventDestroy(e);
    delete ctx;
}

const char* fe2_last_error(const fe2_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

fe2_status fe2_sync(fe2_ctx* ctx) {
    if (!ctx) return FE2_ERR_ARG;
    CK(cudaStreamSynchronize(ctx->stream));
    return FE2_OK;
}

long long fe2_launch_count(const fe2_ctx* ctx) { return ctx ? ctx->launches : -1; }

fe2_status fe2_selftest_wait_timeout(fe2_ctx* ctx, int* status) {
    if (!ctx || !status) return FE2_ERR_ARG;
    CK(launch_selftest_wait(status, ctx->stream));
    return FE2_OK;
}

fe2_status fe2_profile(fe2_ctx* ctx, int enable) {
    if (!ctx) return FE2_ERR_ARG;
    drain_timing(ctx);
    ctx->totals.clear();
    ctx->prof = enable != 0;
    return FE2_OK;
}

int fe2_profile_read(fe2_ctx* ctx, int max, char* names, double* ms, long long* count) {
    if (!ctx || max < 0) return -1;
    drain_timing(ctx);
    int k = 0;
    for (auto& t : ctx->totals) {
        if (k >= max) break;
        if (names) {
            std::strncpy(names + 48 * k, t.first.c_str(), 47);
            names[48 * k + 47] = 0;
        }
        if (ms) ms[k] = t.second.first;
        if (count) count[k] = t.second.second;
        ++k;
    }
    return (int)ctx->totals.size();
}

size_t fe2_rve_bytes(const fe2_ctx* ctx, int N) {
    if (!ctx || N < 2) return 0;
    const int d = ctx->cfg.dim;
    const int kd = compute_kd(const_cast<fe2_ctx*>(ctx), N, d);
    const int nn = nodes_of(N, d), nm = d * (nn - 1), nmp = (nm + NB - 1) / NB * NB;
    const int nq = nq_of(ctx);
    const WsLayout l = ws_layout(kd, d * d * nq + 1, nm, nmp, ctx->cfg.precision == FE2_PREC_FP64, ctx->max_smem, d);
    return persistent_bytes_of(N, d, 2, nq) + l.stride;
}

// ids for nrve new RVEs (released ids first); the device descriptor table grows
// to hold them
static fe2_status new_ids(fe2_ctx* ctx, int nrve, std::vector<int>& ids) {
    ids.assign(nrve, -1);
    for (int k = 0; k < nrve; ++k) {
        if (!ctx->free_ids.empty()) {
            ids[k] = ctx->free_ids.back();
            ctx->free_ids.pop_back();
        } else {
            ids[k] = (int)ctx->host.size();
            ctx->host.emplace_back();
            ctx->mirror.emplace_back();
        }
    }
    const int need_cap = (int)ctx->host.size();
    if (need_cap > ctx->tab_cap) {
        int cap = std::max(need_cap, std::max(64, ctx->tab_cap * 2));
        RveDev* nt = nullptr;
        CK(cudaStreamSynchronize(ctx->stream));
        CK(cudaMalloc(&nt, sizeof(RveDev) * cap));
        if (ctx->d_tab) {
            CK(cudaMemcpy(nt, ctx->d_tab, sizeof(RveDev) * ctx->tab_cap, cudaMemcpyDeviceToDevice));
            CK(cudaFree(ctx->d_tab));
        }
        ctx->d_tab = nt;
        ctx->tab_cap = cap;
    }
    return FE2_OK;
}

fe2_status fe2_rve_register(fe2_ctx* ctx, int nrve, const int* N, const uint8_t* phase, int nphase,
                            const double* mat, int* rve_ids_out) {
    if (!ctx) return FE2_ERR_ARG;
    if (nrve <= 0 || !N || !phase || !mat || !rve_ids_out) return fail(ctx, FE2_ERR_ARG, "bad register arguments");
    if (nphase < 1 || nphase > MAX_PHASES) return fail(ctx, FE2_ERR_ARG, "nphase must be in [1, %d]", MAX_PHASES);
    const int d = ctx->cfg.dim;
    const bool fp64 = ctx->cfg.precision == FE2_PREC_FP64;
    size_t total = 0, ws_need = 0;
    std::vector<size_t> offs(nrve);
    size_t phase_off = 0;
    for (int k = 0; k < nrve; ++k) {
        if (N[k] < 3 || N[k] > 256) return fail(ctx, FE2_ERR_ARG, "mesh size N=%d out of range (N >= 3)", N[k]);
        const int kd = compute_kd(ctx, N[k], d);
        const int nr = d * d * nq_of(ctx) + 1;
        if (nr > MAX_NR) return fail(ctx, FE2_ERR_ARG, "%d right-hand sides exceed the solver limit %d", nr, MAX_NR);
        {
            // the FP64 path never runs the refinement solve (which keeps y in shared memory)
            const int nmk = d * (nodes_of(N[k], d) - 1), nmpk = (nmk + NB - 1) / NB * NB;
            if ((!use_smem_factor(kd, nr, fp64, ctx->max_smem, d) &&
                 (int)factor_gw_smem_bytes(kd, nr, fp64) > ctx->max_smem) ||
                (int)solve_smem_bytes(kd, nr, fp64 ? 0 : nmpk, fp64) > ctx->max_smem)
                return fail(ctx, FE2_ERR_ARG, "N=%d: band of half width %d is too wide for the %s path", N[k], kd,
                            fp64 ? "FP64" : "mixed");
        }
        const int nn = nodes_of(N[k], d);
        for (int p = 0; p < nphase; ++p) {
            const double* m = mat + ((size_t)k * nphase + p) * 4;
            const int model = (int)m[0];
            if (model != FE2_MODEL_LINEAR && model != FE2_MODEL_NEOHOOKE && model != FE2_MODEL_MOONEY_RIVLIN)
                return fail(ctx, FE2_ERR_ARG, "rve %d phase %d: unknown material model %g", k, p, m[0]);
            if (model == FE2_MODEL_MOONEY_RIVLIN && d != 2)
                return fail(ctx, FE2_ERR_ARG, "rve %d phase %d: the Mooney-Rivlin model is 2D only", k, p);
        }
        for (int e = 0; e < nn; ++e)
            if (phase[phase_off + e] >= nphase) return fail(ctx, FE2_ERR_ARG, "rve %d: phase index out of range", k);
        phase_off += nn;
        offs[k] = total;
        total += persistent_bytes_of(N[k], d, nphase, nq_of(ctx));
        const int nm = d * (nn - 1), nmp = (nm + NB - 1) / NB * NB;
        ws_need = std::max(ws_need, ws_layout(kd, nr, nm, nmp, fp64, ctx->max_smem, d).stride);
    }
    if (ctx->cfg.hbm_budget_bytes) {
        // persistent state of everything registered plus one workspace slot must fit;
        // the transient workspace is reclaimed (and re-grown by the next condensation)
        const size_t keep = ctx->persistent_bytes + ctx->elem_bytes;
        if (keep + total + ws_need > ctx->cfg.hbm_budget_bytes)
            return fail(ctx, FE2_ERR_BUDGET,
                        "admission refused: %zu B registered + %zu B requested exceeds budget %zu B", keep,
                        total + ws_need, ctx->cfg.hbm_budget_bytes);
        if (keep + total + ctx->ws_bytes > ctx->cfg.hbm_budget_bytes) {
            fe2_status st = free_ws(ctx);
            if (st != FE2_OK) return st;
        }
    }
    std::vector<int> ids;
    {
        fe2_status st = new_ids(ctx, nrve, ids);
        if (st != FE2_OK) return st;
    }
    Chunk ch;
    CK(cudaMalloc(&ch.dev, total));
    CK(cudaMemsetAsync(ch.dev, 0, total, ctx->stream));
    ch.refs = nrve;
    int chunk_id = -1;
    for (size_t c = 0; c < ctx->chunks.size(); ++c)
        if (!ctx->chunks[c].dev) {
            chunk_id = (int)c;
            break;
        }
    if (chunk_id < 0) {
        chunk_id = (int)ctx->chunks.size();
        ctx->chunks.push_back(ch);
    } else {
        ctx->chunks[chunk_id] = ch;
    }
    ctx->persistent_bytes += total;
    // stage phase + mat for all RVEs of the chunk with one host buffer
    std::vector<unsigned char> stage(total, 0);
    phase_off = 0;
    for (int k = 0; k < nrve; ++k) {
        const int nq = nq_of(ctx);
        const int nn = nodes_of(N[k], d), nm = d * (nn - 1), nr = d * d * nq + 1;
        const int nst = (d == 2 ? 9 : 27) * d * d;
        char* base = (char*)ch.dev + offs[k];
        unsigned char* hb = stage.data() + offs[k];
        RveDev r{};
        r.N = N[k];
        r.d = d;
        r.nm = nm;
        r.kd = compute_kd(ctx, N[k], d);
        r.nn = nn;
        r.nphase = nphase;
        r.nm_pad = (nm + NB - 1) / NB * NB;
        r.nr = nr;
        place_rve(r, base, nst, nq);
        std::memcpy(hb + ((const char*)r.phase - base), phase + phase_off, nn);
        std::memcpy(hb + ((const char*)r.mat - base), mat + (size_t)k * nphase * 4, (size_t)nphase * 4 * 8);
        r.nq = nq;
        for (int g = 0; g < MAX_NQ; ++g) r.wq[g] = g < nq ? 1.0 / nq : 0.0;
        r.elem = nullptr;
        r.nbr = nbr_table(ctx, N[k], d);
        if (!r.nbr) return fail(ctx, FE2_ERR_CUDA, "neighbour table allocation failed");
        r.zero_w = 1;
        phase_off += nn;
        const int id = ids[k];
        ctx->mirror[id] = r;
        HostRve& h = ctx->host[id];
        h = HostRve();
        h.active = true;
        h.chunk = chunk_id;
        h.mat.assign(mat + (size_t)k * nphase * 4, mat + (size_t)(k + 1) * nphase * 4);
        h.all_linear = true;
        for (int p = 0; p < nphase; ++p) h.all_linear &= (int)h.mat[4 * p] == FE2_MODEL_LINEAR;
        rve_ids_out[k] = id;
    }
    CK(cudaMemcpyAsync(ch.dev, stage.data(), total, cudaMemcpyHostToDevice, ctx->stream));
    // descriptors (contiguous runs are common; upload one by one for simplicity)
    std::vector<RveDev> tmp(nrve);
    for (int k = 0; k < nrve; ++k) tmp[k] = ctx->mirror[ids[k]];
    for (int k = 0; k < nrve; ++k)
        CK(cudaMemcpyAsync(ctx->d_tab + ids[k], &tmp[k], sizeof(RveDev), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return FE2_OK;
}

fe2_status fe2_rve_release(fe2_ctx* ctx, int n, const int* rve_ids) {
    if (!ctx) return FE2_ERR_ARG;
    if (n < 0 || (n > 0 && !rve_ids)) return fail(ctx, FE2_ERR_ARG, "bad release arguments");
    std::vector<int> rel;
    for (int k = 0; k < n; ++k) {
        const int id = rve_ids[k];
        if (id < 0 || id >= (int)ctx->host.size() || !ctx->host[id].active)
            return fail(ctx, FE2_ERR_ARG, "rve id %d is not registered", id);
        rel.push_back(id);
    }
    drop_cached_lists_with(ctx, rel);
    CK(cudaStreamSynchronize(ctx->stream));
    for (int id : rel) {
        HostRve& h = ctx->host[id];
        if (!h.active) continue;
        h.active = false;
        if (h.deferred) {  // its slot (if any) goes back to the pool
            if (h.resident && h.slot) ctx->free_slots.push_back(h.slot);
            ctx->lru.erase({h.last_use, id});
            h = HostRve();
            ctx->free_ids.push_back(id);
            continue;
        }
        const RveDev& r = ctx->mirror[id];
        ctx->persistent_bytes -= persistent_bytes_of(r.N, r.d, r.nphase, r.nq > 0 ? r.nq : 1);
        Chunk& c = ctx->chunks[h.chunk];
        if (--c.refs == 0) {
            CK(cudaFree(c.dev));
            c.dev = nullptr;
        }
        h.chunk = -1;
        ctx->free_ids.push_back(id);
    }
    return FE2_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ defined RVEs
// RVEs defined by fe2_rve_define keep their definition (mesh size, phases,
// materials) and, while not resident, their fluctuation w~ on the host; their
// device state lives in uniform slots (the largest defined RVE's persistent
// bytes), carved from slabs allocated within the HBM budget and recycled, not
// freed, when an RVE is evicted.

static void touch(fe2_ctx* ctx, int id) {
    HostRve& h = ctx->host[id];
    ctx->lru.erase({h.last_use, id});
    h.last_use = ++ctx->tick;
    ctx->lru.insert({h.last_use, id});
}

// Move w~ of an idle resident defined RVE to the host and give back its slot.
static fe2_status evict_one(fe2_ctx* ctx, int id) {
    HostRve& h = ctx->host[id];
    if (!h.deferred || !h.resident) return FE2_OK;
    RveDev& r = ctx->mirror[id];
    CK(cudaStreamSynchronize(ctx->stream));
    h.w_zero = r.zero_w != 0;
    if (!h.w_zero) {
        h.w.resize(r.nm);
        CK(cudaMemcpy(h.w.data(), r.w, sizeof(double) * r.nm, cudaMemcpyDeviceToHost));
    }
    ctx->free_slots.push_back(h.slot);
    ctx->lru.erase({h.last_use, id});
    h.slot = nullptr;
    h.resident = false;
    ++ctx->n_evicted;
    return FE2_OK;
}

// Make a defined RVE resident, its state copied in on stream s.  *ok = false
// (nothing changed) when no slot is free, no slab fits the budget and no
// evictable RVE is left; `busy(id)` marks RVEs that must not be evicted.
template <typename Busy>
static fe2_status admit_one(fe2_ctx* ctx, int id, cudaStream_t s, bool* ok, Busy busy) {
    HostRve& h = ctx->host[id];
    *ok = true;
    if (h.resident) {
        if (h.deferred) touch(ctx, id);
        return FE2_OK;
    }
    if (ctx->free_slots.empty()) {
        const size_t budget = ctx->cfg.hbm_budget_bytes;
        int per = 16;
        if (budget) {
            const size_t used = used_bytes(ctx);
            const size_t room = budget > used ? budget - used : 0;
            per = std::min<size_t>(per, room / ctx->slot_bytes);
        }
        if (per >= 1) {
            void* p = nullptr;
            CK(cudaMalloc(&p, ctx->slot_bytes * per));
            ctx->slabs.push_back(p);
            ctx->persistent_bytes += ctx->slot_bytes * per;
            for (int k = 0; k < per; ++k) ctx->free_slots.push_back((char*)p + ctx->slot_bytes * k);
        } else {
            for (auto it = ctx->lru.begin(); it != ctx->lru.end(); ++it)
                if (it->second != id && !busy(it->second)) {
                    fe2_status st = evict_one(ctx, it->second);
                    if (st != FE2_OK) return st;
                    break;
                }
        }
        if (ctx->free_slots.empty()) {
            *ok = false;
            return FE2_OK;
        }
    }
    char* slot = ctx->free_slots.back();
    ctx->free_slots.pop_back();
    RveDev& r = ctx->mirror[id];
    const int nst = (r.d == 2 ? 9 : 27) * r.d * r.d;
    place_rve(r, slot, nst, 1);
    r.zero_w = h.w_zero ? 1 : 0;
    CK(cudaMemcpyAsync((void*)r.phase, h.phase.data(), h.phase.size(), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync((void*)r.mat, h.mat.data(), sizeof(double) * h.mat.size(), cudaMemcpyHostToDevice, s));
    if (h.w_zero)
        CK(cudaMemsetAsync(r.w, 0, sizeof(double) * r.nm, s));
    else
        CK(cudaMemcpyAsync(r.w, h.w.data(), sizeof(double) * r.nm, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->d_tab + id, &r, sizeof(RveDev), cudaMemcpyHostToDevice, s));
    h.slot = slot;
    h.resident = true;
    touch(ctx, id);
    ++ctx->n_admitted;
    return FE2_OK;
}

extern "C" {

fe2_status fe2_rve_define(fe2_ctx* ctx, int nrve, const int* N, const uint8_t* phase, int nphase,
                          const double* mat, int* rve_ids_out) {
    if (!ctx) return FE2_ERR_ARG;
    if (nrve <= 0 || !N || !phase || !mat || !rve_ids_out) return fail(ctx, FE2_ERR_ARG, "bad define arguments");
    if (nphase < 1 || nphase > MAX_PHASES) return fail(ctx, FE2_ERR_ARG, "nphase must be in [1, %d]", MAX_PHASES);
    if (nq_of(ctx) > 1) return fail(ctx, FE2_ERR_ARG, "defined RVEs take the Dirac basis");
    const int d = ctx->cfg.dim;
    const bool fp64 = ctx->cfg.precision == FE2_PREC_FP64;
    size_t need = 0, phase_off = 0;
    for (int k = 0; k < nrve; ++k) {
        if (N[k] < 3 || N[k] > 256) return fail(ctx, FE2_ERR_ARG, "mesh size N=%d out of range (N >= 3)", N[k]);
        const int kd = compute_kd(ctx, N[k], d), nr = d * d + 1;
        const int nmk = d * (nodes_of(N[k], d) - 1), nmpk = (nmk + NB - 1) / NB * NB;
        if ((!use_smem_factor(kd, nr, fp64, ctx->max_smem, d) && (int)factor_gw_smem_bytes(kd, nr, fp64) > ctx->max_smem) ||
            (int)solve_smem_bytes(kd, nr, fp64 ? 0 : nmpk, fp64) > ctx->max_smem)
            return fail(ctx, FE2_ERR_ARG, "N=%d: band of half width %d is too wide", N[k], kd);
        for (int p = 0; p < nphase; ++p) {
            const int model = (int)mat[((size_t)k * nphase + p) * 4];
            if (model != FE2_MODEL_LINEAR && model != FE2_MODEL_NEOHOOKE && model != FE2_MODEL_MOONEY_RIVLIN)
                return fail(ctx, FE2_ERR_ARG, "rve %d phase %d: unknown material model", k, p);
            if (model == FE2_MODEL_MOONEY_RIVLIN && d != 2)
                return fail(ctx, FE2_ERR_ARG, "rve %d phase %d: the Mooney-Rivlin model is 2D only", k, p);
        }
        const int nn = nodes_of(N[k], d);
        for (int e = 0; e < nn; ++e)
            if (phase[phase_off + e] >= nphase) return fail(ctx, FE2_ERR_ARG, "rve %d: phase index out of range", k);
        phase_off += nn;
        need = std::max(need, persistent_bytes_of(N[k], d, nphase, 1));
    }
    if (ctx->slot_bytes == 0) ctx->slot_bytes = need;
    for (int k = 0; k < nrve; ++k) ctx->def_maxN = std::max(ctx->def_maxN, N[k]);
    if (need > ctx->slot_bytes)
        return fail(ctx, FE2_ERR_ARG, "defined RVEs need %zu B slots, the pool has %zu B (define the largest first)",
                    need, ctx->slot_bytes);
    std::vector<int> ids;
    fe2_status st = new_ids(ctx, nrve, ids);
    if (st != FE2_OK) return st;
    phase_off = 0;
    for (int k = 0; k < nrve; ++k) {
        const int nn = nodes_of(N[k], d), nm = d * (nn - 1);
        RveDev r{};
        r.N = N[k];
        r.d = d;
        r.nm = nm;
        r.kd = compute_kd(ctx, N[k], d);
        r.nn = nn;
        r.nphase = nphase;
        r.nm_pad = (nm + NB - 1) / NB * NB;
        r.nr = d * d + 1;
        r.nq = 1;
        r.wq[0] = 1.0;
        r.nbr = nbr_table(ctx, N[k], d);
        if (!r.nbr) return fail(ctx, FE2_ERR_CUDA, "neighbour table allocation failed");
        r.zero_w = 1;
        const int id = ids[k];
        ctx->mirror[id] = r;
        HostRve& h = ctx->host[id];
        h = HostRve();
        h.active = true;
        h.deferred = true;
        h.resident = false;
        h.mat.assign(mat + (size_t)k * nphase * 4, mat + (size_t)(k + 1) * nphase * 4);
        h.all_linear = true;
        for (int p = 0; p < nphase; ++p) h.all_linear &= (int)h.mat[4 * p] == FE2_MODEL_LINEAR;
        h.phase.assign(phase + phase_off, phase + phase_off + nn);
        phase_off += nn;
        rve_ids_out[k] = id;
    }
    return FE2_OK;
}

fe2_status fe2_rve_admit(fe2_ctx* ctx, int n, const int* rve_ids) {
    if (!ctx) return FE2_ERR_ARG;
    if (n < 0 || (n > 0 && !rve_ids)) return fail(ctx, FE2_ERR_ARG, "bad admit arguments");
    std::unordered_set<int> keep;
    for (int k = 0; k < n; ++k) {
        const int id = rve_ids[k];
        if (id < 0 || id >= (int)ctx->host.size() || !ctx->host[id].active)
            return fail(ctx, FE2_ERR_ARG, "rve id %d is not registered", id);
        keep.insert(id);
    }
    CK(cudaStreamSynchronize(ctx->stream));
    for (int k = 0; k < n; ++k) {
        bool ok = true;
        fe2_status st = admit_one(ctx, rve_ids[k], ctx->stream, &ok, [&](int x) { return keep.count(x) > 0; });
        if (st != FE2_OK) return st;
        if (!ok) return fail(ctx, FE2_ERR_BUDGET, "no room for rve %d within the HBM budget", rve_ids[k]);
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return FE2_OK;
}

fe2_status fe2_rve_evict(fe2_ctx* ctx, int n, const int* rve_ids) {
    if (!ctx) return FE2_ERR_ARG;
    if (n < 0 || (n > 0 && !rve_ids)) return fail(ctx, FE2_ERR_ARG, "bad evict arguments");
    for (int k = 0; k < n; ++k) {
        const int id = rve_ids[k];
        if (id < 0 || id >= (int)ctx->host.size() || !ctx->host[id].active)
            return fail(ctx, FE2_ERR_ARG, "rve id %d is not registered", id);
        if (!ctx->host[id].deferred) return fail(ctx, FE2_ERR_ARG, "rve %d was registered, not defined", id);
        fe2_status st = evict_one(ctx, id);
        if (st != FE2_OK) return st;
    }
    return FE2_OK;
}

int fe2_rve_resident(const fe2_ctx* ctx, int rve_id) {
    if (!ctx || rve_id < 0 || rve_id >= (int)ctx->host.size() || !ctx->host[rve_id].active) return -1;
    return ctx->host[rve_id].resident ? 1 : 0;
}

fe2_status fe2_micro_assemble(fe2_ctx* ctx, int n, const int* rve_ids, const double* Fbar) {
    if (!ctx) return FE2_ERR_ARG;
    if (ctx->cfg.macro_basis == FE2_BASIS_CONST)
        return fail(ctx, FE2_ERR_ARG, "element RVEs (piecewise-constant basis) use the fused fe2_rve_solve");
    if (!Fbar) return fail(ctx, FE2_ERR_ARG, "Fbar is NULL");
    const int* d_ids = nullptr;
    fe2_status st = get_ids(ctx, n, rve_ids, &d_ids);
    if (st != FE2_OK) return st;
    const BatchInfo b = batch_info(ctx, n, rve_ids);
    const int d = ctx->cfg.dim;
    const size_t per = (size_t)b.maxnn * elem_comps(d) * 8;
    const size_t need = per * n;
    if (need > ctx->elem_bytes) {
        if (ctx->cfg.hbm_budget_bytes && used_bytes(ctx) - ctx->elem_bytes + need > ctx->cfg.hbm_budget_bytes)
            return fail(ctx, FE2_ERR_BUDGET, "element workspace of %zu B exceeds the HBM budget", need);
        CK(cudaStreamSynchronize(ctx->stream));
        if (ctx->elem) CK(cudaFree(ctx->elem));
        ctx->elem = nullptr;
        ctx->elem_bytes = 0;
        CK(cudaMalloc(&ctx->elem, need));
        ctx->elem_bytes = need;
    }
    for (int id : ctx->elem_ids)
        if (id < (int)ctx->mirror.size()) ctx->mirror[id].elem = nullptr;
    ctx->elem_ids.assign(rve_ids, rve_ids + n);
    for (int k = 0; k < n; ++k) ctx->mirror[rve_ids[k]].elem = (double*)((char*)ctx->elem + per * k);
    st = upload_all(ctx);
    if (st != FE2_OK) return st;
    if (d == 3)
        TIMED("assemble_elems_hex8", launch_assemble_elems3(ctx->d_tab, d_ids, n, Fbar, b.maxN, ctx->stream));
    else
        TIMED("assemble_elems", launch_assemble_elems(ctx->d_tab, d_ids, n, Fbar, d, b.maxN, ctx->stream));
    return FE2_OK;
}

fe2_status fe2_nullspace_reduce(fe2_ctx* ctx, int n, const int* rve_ids) {
    if (!ctx) return FE2_ERR_ARG;
    if (ctx->cfg.macro_basis == FE2_BASIS_CONST)
        return fail(ctx, FE2_ERR_ARG, "element RVEs (piecewise-constant basis) use the fused fe2_rve_solve");
    const int* d_ids = nullptr;
    fe2_status st = get_ids(ctx, n, rve_ids, &d_ids);
    if (st != FE2_OK) return st;
    for (int k = 0; k < n; ++k)
        if (!ctx->mirror[rve_ids[k]].elem)
            return fail(ctx, FE2_ERR_ARG, "rve %d has no element data: call fe2_micro_assemble first", rve_ids[k]);
    const BatchInfo b = batch_info(ctx, n, rve_ids);
    if (ctx->cfg.dim == 3)
        TIMED("nullspace_reduce_hex8", launch_reduce3(ctx->d_tab, d_ids, n, ctx->stream));
    else
        TIMED("nullspace_reduce", launch_reduce(ctx->d_tab, d_ids, n, ctx->cfg.dim, b.maxN, ctx->stream));
    return FE2_OK;
}

fe2_status fe2_condense(fe2_ctx* ctx, int n, const int* rve_ids, double* sigma_eff, double* Cbar, int* rve_status,
                        double* err_est) {
    if (!ctx) return FE2_ERR_ARG;
    if (!sigma_eff || !Cbar || !rve_status) return fail(ctx, FE2_ERR_ARG, "output pointer is NULL");
    const int* d_ids = nullptr;
    fe2_status st = get_ids(ctx, n, rve_ids, &d_ids);
    if (st != FE2_OK) return st;
    return condense_impl(ctx, n, rve_ids, d_ids, sigma_eff, Cbar, rve_status, err_est, true);
}

fe2_status fe2_rve_solve(fe2_ctx* ctx, int n, const int* rve_ids, const double* Fbar, double* sigma_eff,
                         double* Cbar, int* rve_status, double* err_est) {
    if (!ctx) return FE2_ERR_ARG;
    if (!Fbar || !sigma_eff || !Cbar || !rve_status) return fail(ctx, FE2_ERR_ARG, "NULL pointer argument");
    const int* d_ids = nullptr;
    fe2_status st = get_ids(ctx, n, rve_ids, &d_ids);
    if (st != FE2_OK) return st;
    const BatchInfo b = batch_info(ctx, n, rve_ids);
    if (ctx->cfg.dim == 3) {
        // Hex8: element rows to the element workspace, then the node-row gather
        TIMED("check_fbar", launch_check_fbar(Fbar, n, ctx->cfg.dim, rve_status, ctx->stream));
        st = fe2_micro_assemble(ctx, n, rve_ids, Fbar);
        if (st != FE2_OK) return st;
        st = fe2_nullspace_reduce(ctx, n, rve_ids);
        if (st != FE2_OK) return st;
        return condense_impl(ctx, n, rve_ids, d_ids, sigma_eff, Cbar, rve_status, err_est, false);
    }
    if (nq_of(ctx) > 1) {
        TIMED("check_fbar", launch_check_fbar_dd(Fbar, n, 4 * nq_of(ctx), rve_status, ctx->stream));
        TIMED("assemble_reduce_elem", launch_assemble_fused_elem(ctx->d_tab, d_ids, n, Fbar, b.maxN, ctx->stream));
        return condense_impl(ctx, n, rve_ids, d_ids, sigma_eff, Cbar, rve_status, err_est, false);
    }
    TIMED("check_fbar", launch_check_fbar(Fbar, n, ctx->cfg.dim, rve_status, ctx->stream));
    TIMED(b.all_linear ? "assemble_reduce_linear" : "assemble_reduce_general",
          launch_assemble_fused(ctx->d_tab, d_ids, n, Fbar, ctx->cfg.dim, b.maxN, b.linear_mode(), ctx->stream));
    return condense_impl(ctx, n, rve_ids, d_ids, sigma_eff, Cbar, rve_status, err_est, false);
}

fe2_status fe2_macro_step(fe2_ctx* ctx, int n, const int* rve_ids, const double* dFbar) {
    if (!ctx) return FE2_ERR_ARG;
    if (!dFbar) return fail(ctx, FE2_ERR_ARG, "dFbar is NULL");
    const int* d_ids = nullptr;
    fe2_status st = get_ids(ctx, n, rve_ids, &d_ids);
    if (st != FE2_OK) return st;
    const BatchInfo b = batch_info(ctx, n, rve_ids);
    if (nq_of(ctx) > 1)
        TIMED("macro_update", launch_macro_update_elem(ctx->d_tab, d_ids, n, dFbar, b.maxnm, ctx->stream));
    else
        TIMED("macro_update", launch_macro_update(ctx->d_tab, d_ids, n, dFbar, b.maxnm, ctx->stream));
    for (int k = 0; k < n; ++k) ctx->mirror[rve_ids[k]].zero_w = 0;
    return FE2_OK;
}

fe2_status fe2_rve_w_copy(fe2_ctx* ctx, int n, const int* rve_ids, double* buf, int ld, int to_buf) {
    if (!ctx) return FE2_ERR_ARG;
    if (!buf) return fail(ctx, FE2_ERR_ARG, "buf is NULL");
    const int* d_ids = nullptr;
    fe2_status st = get_ids(ctx, n, rve_ids, &d_ids);
    if (st != FE2_OK) return st;
    const BatchInfo b = batch_info(ctx, n, rve_ids);
    if (ld < b.maxnm) return fail(ctx, FE2_ERR_ARG, "row length %d below the largest n_m %d", ld, b.maxnm);
    TIMED("w_copy", launch_w_copy(ctx->d_tab, d_ids, n, buf, ld, b.maxnm, to_buf ? 1 : 0, ctx->stream));
    if (!to_buf)
        for (int k = 0; k < n; ++k) ctx->mirror[rve_ids[k]].zero_w = 0;
    return FE2_OK;
}

// folded index of natural node p = i + N j (+ N^2 k) of a 2D or 3D RVE
static int fold_node(int p, int N, int d) {
    const int i = p % N, j = (p / N) % N;
    int q = fold_pos(i, N) + N * fold_pos(j, N);
    if (d == 3) q += N * N * fold_pos(p / (N * N), N);
    return q;
}

fe2_status fe2_rve_set_w(fe2_ctx* ctx, int rve_id, const double* host_w) {
    if (!ctx) return FE2_ERR_ARG;
    if (rve_id < 0 || rve_id >= (int)ctx->host.size() || !ctx->host[rve_id].active || !host_w)
        return fail(ctx, FE2_ERR_ARG, "bad rve id or NULL w");
    RveDev& r = ctx->mirror[rve_id];
    const int N = r.N, d = r.d;
    std::vector<double> wf(r.nm);
    for (int p = 1; p < r.nn; ++p) {
        const int q = fold_node(p, N, d);
        for (int c = 0; c < d; ++c) wf[d * (q - 1) + c] = host_w[d * (p - 1) + c];
    }
    HostRve& h = ctx->host[rve_id];
    if (!h.resident) {  // a defined RVE held on the host: its w~ is copied in when admitted
        h.w = wf;
        h.w_zero = false;
        return FE2_OK;
    }
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaMemcpy(r.w, wf.data(), sizeof(double) * r.nm, cudaMemcpyHostToDevice));
    r.zero_w = 0;
    return upload_desc(ctx, rve_id);
}

fe2_status fe2_rve_export(fe2_ctx* ctx, int rve_id, int what, double* out) {
    if (!ctx) return FE2_ERR_ARG;
    if (rve_id < 0 || rve_id >= (int)ctx->host.size() || !ctx->host[rve_id].active || !out)
        return fail(ctx, FE2_ERR_ARG, "bad rve id or NULL output");
    if (!ctx->host[rve_id].resident) return fail(ctx, FE2_ERR_ARG, "rve %d is not resident", rve_id);
    CK(cudaStreamSynchronize(ctx->stream));
    const RveDev& r = ctx->mirror[rve_id];
    const int N = r.N, d = r.d, nm = r.nm, nn = r.nn, dd = d * d;
    if (d != 2 && what == 0) return fail(ctx, FE2_ERR_ARG, "the dense K_mm export is 2D only");
    std::vector<int> q2p(nn);
    for (int p = 0; p < nn; ++p) q2p[fold_node(p, N, d)] = p;
    auto nat = [&](int fdof) { return d * (q2p[fdof / d + 1] - 1) + fdof % d; };
    if (what == 0) {
        std::vector<double> st((size_t)9 * 4 * nn);
        CK(cudaMemcpy(st.data(), r.stencil, sizeof(double) * st.size(), cudaMemcpyDeviceToHost));
        std::memset(out, 0, sizeof(double) * (size_t)nm * nm);
        for (int q = 1; q < nn; ++q) {
            const int p = q2p[q], i = p % N, j = p / N;
            for (int off = 0; off < 9; ++off) {
                const int dx = off % 3 - 1, dy = off / 3 - 1;
                const int pn = (i + dx + N) % N + N * ((j + dy + N) % N);
                if (pn == 0) continue;
                for (int c = 0; c < 2; ++c)
                    for (int c2 = 0; c2 < 2; ++c2)
                        out[(size_t)(2 * (p - 1) + c) * nm + 2 * (pn - 1) + c2] +=
                            st[(size_t)((off * 2 + c) * 2 + c2) * nn + q];
            }
        }
    } else if (what == 1 || what == 2) {
        std::vector<double> rhs((size_t)r.nr * nm);
        CK(cudaMemcpy(rhs.data(), r.rhs, sizeof(double) * rhs.size(), cudaMemcpyDeviceToHost));
        for (int m = 0; m < nm; ++m) {
            if (what == 1)
                out[nat(m)] = rhs[(size_t)dd * nm + m];
            else
                for (int kL = 0; kL < dd; ++kL) out[(size_t)nat(m) * dd + kL] = rhs[(size_t)kL * nm + m];
        }
    } else if (what == 3) {
        std::vector<double> w(nm);
        CK(cudaMemcpy(w.data(), r.w, sizeof(double) * nm, cudaMemcpyDeviceToHost));
        for (int m = 0; m < nm; ++m) out[nat(m)] = r.zero_w ? 0.0 : w[m];
    } else if (what == 4) {
        CK(cudaMemcpy(out, r.KMM, sizeof(double) * (dd * dd + dd), cudaMemcpyDeviceToHost));
    } else {
        return fail(ctx, FE2_ERR_ARG, "unknown export selector %d", what);
    }
    return FE2_OK;
}

fe2_status fe2_macro_setup(fe2_ctx* ctx, int nnode, const double* X, int nelem, const int* conn,
                           const uint8_t* fixed) {
    if (!ctx) return FE2_ERR_ARG;
    const int d = ctx->cfg.dim, nen = 1 << d;
    if (d == 3 && nq_of(ctx) > 1) return fail(ctx, FE2_ERR_ARG, "element RVEs are 2D");
    if (nnode <= 0 || nelem <= 0 || !X || !conn || !fixed) return fail(ctx, FE2_ERR_ARG, "bad macro mesh");
    CK(cudaStreamSynchronize(ctx->stream));
    for (void* p : ctx->macro_bufs) cudaFree(p);
    ctx->macro_bufs.clear();
    ctx->macro_ready = false;
    const int ngp = nen * nelem;
    std::vector<int> cn(conn, conn + (size_t)nen * nelem);
    for (int v : cn)
        if (v < 0 || v >= nnode) return fail(ctx, FE2_ERR_ARG, "connectivity references node %d", v);
    ctx->macro_X.assign(X, X + (size_t)d * nnode);
    // free DOFs in natural order; band width from the element couplings
    std::vector<int> d2f((size_t)d * nnode, -1);
    int nfree = 0;
    for (int t = 0; t < d * nnode; ++t)
        if (!fixed[t]) d2f[t] = nfree++;
    if (nfree == 0) return fail(ctx, FE2_ERR_ARG, "no free macro DOFs");
    int kd = 0;
    for (int e = 0; e < nelem; ++e)
        for (int a = 0; a < nen; ++a)
            for (int b = 0; b < nen; ++b)
                for (int c = 0; c < d; ++c)
                    for (int k = 0; k < d; ++k) {
                        const int i = d2f[d * cn[nen * e + a] + c], j = d2f[d * cn[nen * e + b] + k];
                        if (i >= 0 && j >= 0) kd = std::max(kd, std::abs(i - j));
                    }
    // Gauss-point gradients and weights (2^d Gauss points on the isoparametric
    // Q4 / Hex8): N_a = prod_k (1 + s_ak xi_k) / 2, s_ak = +-1 from the bits of a
    std::vector<double> grads((size_t)ngp * nen * d), eta(ngp);
    const double g = 0.57735026918962576451;
    for (int e = 0; e < nelem; ++e)
        for (int q = 0; q < nen; ++q) {
            double xi[3], dN[8][3], Jm[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
            for (int k = 0; k < d; ++k) xi[k] = ((q >> k) & 1) ? g : -g;
            for (int a = 0; a < nen; ++a) {
                double sgn[3], fac[3];
                for (int k = 0; k < d; ++k) {
                    sgn[k] = ((a >> k) & 1) ? 1.0 : -1.0;
                    fac[k] = 0.5 * (1.0 + sgn[k] * xi[k]);
                }
                for (int J = 0; J < d; ++J) {
                    double v = 0.5 * sgn[J];
                    for (int k = 0; k < d; ++k)
                        if (k != J) v *= fac[k];
                    dN[a][J] = v;
                }
                for (int i = 0; i < d; ++i)
                    for (int k = 0; k < d; ++k) Jm[i][k] += X[(size_t)d * cn[nen * e + a] + i] * dN[a][k];
            }
            double inv[3][3], det;
            if (d == 2) {
                det = Jm[0][0] * Jm[1][1] - Jm[0][1] * Jm[1][0];
                inv[0][0] = Jm[1][1] / det;
                inv[0][1] = -Jm[0][1] / det;
                inv[1][0] = -Jm[1][0] / det;
                inv[1][1] = Jm[0][0] / det;
            } else {
                // inverse by cofactors: inv[k][i] = cof[i][k] / det
                double cof[3][3];
                for (int i = 0; i < 3; ++i)
                    for (int k = 0; k < 3; ++k) {
                        const int i1 = (i + 1) % 3, i2 = (i + 2) % 3, k1 = (k + 1) % 3, k2 = (k + 2) % 3;
                        cof[i][k] = Jm[i1][k1] * Jm[i2][k2] - Jm[i1][k2] * Jm[i2][k1];
                    }
                det = Jm[0][0] * cof[0][0] + Jm[0][1] * cof[0][1] + Jm[0][2] * cof[0][2];
                for (int i = 0; i < 3; ++i)
                    for (int k = 0; k < 3; ++k) inv[k][i] = cof[i][k] / det;
            }
            if (!(det > 0.0)) return fail(ctx, FE2_ERR_ARG, "macro element %d is inverted", e);
            const int b = nen * e + q;
            // grad N_a = dN/dxi (dX/dxi)^-1
            for (int a = 0; a < nen; ++a)
                for (int J = 0; J < d; ++J) {
                    double v = 0.0;
                    for (int k = 0; k < d; ++k) v += dN[a][k] * inv[k][J];
                    grads[((size_t)b * nen + a) * d + J] = v;
                }
            eta[b] = det;
        }
    std::vector<int> adj_ptr(nnode + 1, 0), adj;
    for (int e = 0; e < nelem; ++e)
        for (int a = 0; a < nen; ++a) ++adj_ptr[cn[nen * e + a] + 1];
    for (int n = 0; n < nnode; ++n) adj_ptr[n + 1] += adj_ptr[n];
    adj.assign(adj_ptr[nnode], 0);
    std::vector<int> fill(adj_ptr.begin(), adj_ptr.end() - 1);
    for (int e = 0; e < nelem; ++e)
        for (int a = 0; a < nen; ++a) adj[fill[cn[nen * e + a]]++] = nen * e + a;
    MacroDev M{};
    M.d = d;
    M.nnode = nnode;
    M.nelem = nelem;
    M.nfree = nfree;
    M.kd = kd;
    M.ngp = ngp;
    fe2_status st;
    int *dconn, *dd2f, *dadjp, *dadj;
    double *dgr, *deta, *dq, *dK, *dR, *ddq;
    if ((st = upload_vec(ctx, cn, &dconn)) || (st = upload_vec(ctx, d2f, &dd2f)) ||
        (st = upload_vec(ctx, grads, &dgr)) || (st = upload_vec(ctx, eta, &deta)) ||
        (st = upload_vec(ctx, adj_ptr, &dadjp)) || (st = upload_vec(ctx, adj, &dadj)))
        return st;
    std::vector<double> q0(X, X + (size_t)d * nnode);
    if ((st = upload_vec(ctx, q0, &dq))) return st;
    if ((st = upload_vec(ctx, std::vector<double>((size_t)nfree * (kd + 1)), &dK))) return st;
    if ((st = upload_vec(ctx, std::vector<double>(nfree), &dR))) return st;
    if ((st = upload_vec(ctx, std::vector<double>((size_t)d * nnode), &ddq))) return st;
    double* dfext;
    if ((st = upload_vec(ctx, std::vector<double>((size_t)d * nnode), &dfext))) return st;
    M.fext = dfext;
    M.conn = dconn;
    M.dof2free = dd2f;
    M.grads = dgr;
    M.eta = deta;
    M.adj_ptr = dadjp;
    M.adj = dadj;
    M.q = dq;
    M.K = dK;
    M.R = dR;
    M.dq = ddq;
    if (!ctx->d_macro_status) CK(cudaMalloc(&ctx->d_macro_status, sizeof(int)));
    ctx->macro = M;
    ctx->macro_ready = true;
    return FE2_OK;
}

fe2_status fe2_macro_set_positions(fe2_ctx* ctx, const double* q_host, const uint8_t* which) {
    if (!ctx) return FE2_ERR_ARG;
    if (!ctx->macro_ready || !q_host) return fail(ctx, FE2_ERR_ARG, "no macro problem / NULL positions");
    const int nd = ctx->macro.d * ctx->macro.nnode;
    std::vector<double> q(nd);
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaMemcpy(q.data(), ctx->macro.q, sizeof(double) * nd, cudaMemcpyDeviceToHost));
    for (int t = 0; t < nd; ++t)
        if (!which || which[t]) q[t] = q_host[t];
    CK(cudaMemcpy(ctx->macro.q, q.data(), sizeof(double) * nd, cudaMemcpyHostToDevice));
    return FE2_OK;
}

fe2_status fe2_macro_set_load(fe2_ctx* ctx, const double* fext_host) {
    if (!ctx) return FE2_ERR_ARG;
    if (!ctx->macro_ready) return fail(ctx, FE2_ERR_ARG, "no macro problem");
    const int nd = ctx->macro.d * ctx->macro.nnode;
    std::vector<double> f(nd, 0.0);
    if (fext_host) f.assign(fext_host, fext_host + nd);
    for (int t = 0; t < nd; ++t)
        if (!std::isfinite(f[t])) return fail(ctx, FE2_ERR_NAN, "external force %d is not finite", t);
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaMemcpy(const_cast<double*>(ctx->macro.fext), f.data(), sizeof(double) * nd, cudaMemcpyHostToDevice));
    return FE2_OK;
}

fe2_status fe2_macro_set_edge_load(fe2_ctx* ctx, int n, const int* nodes, const double* T, double scale) {
    if (!ctx) return FE2_ERR_ARG;
    if (!ctx->macro_ready) return fail(ctx, FE2_ERR_ARG, "no macro problem");
    if (ctx->macro.d != 2) return fail(ctx, FE2_ERR_ARG, "edge loads are 2D (Q4 macro meshes)");
    if (n < 2 || !nodes || !T) return fail(ctx, FE2_ERR_ARG, "an edge load needs >= 2 nodes and a traction");
    const int nnode = ctx->macro.nnode;
    for (int k = 0; k < n; ++k)
        if (nodes[k] < 0 || nodes[k] >= nnode) return fail(ctx, FE2_ERR_ARG, "edge node %d out of range", nodes[k]);
    if (!std::isfinite(T[0]) || !std::isfinite(T[1]) || !std::isfinite(scale))
        return fail(ctx, FE2_ERR_NAN, "traction or scale not finite");
    // Neumann term of Eq. (weakMech) for a constant traction on straight
    // bilinear edges: each segment of length l gives T l / 2 to both end nodes
    std::vector<double> f((size_t)2 * nnode, 0.0);
    const std::vector<double>& X = ctx->macro_X;
    for (int k = 0; k + 1 < n; ++k) {
        const int a = nodes[k], b = nodes[k + 1];
        const double l = std::hypot(X[2 * b] - X[2 * a], X[2 * b + 1] - X[2 * a + 1]);
        for (int c = 0; c < 2; ++c) {
            f[2 * a + c] += 0.5 * l * T[c] * scale;
            f[2 * b + c] += 0.5 * l * T[c] * scale;
        }
    }
    return fe2_macro_set_load(ctx, f.data());
}

fe2_status fe2_macro_get_positions(fe2_ctx* ctx, double* q_host) {
    if (!ctx) return FE2_ERR_ARG;
    if (!ctx->macro_ready || !q_host) return fail(ctx, FE2_ERR_ARG, "no macro problem / NULL output");
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaMemcpy(q_host, ctx->macro.q, sizeof(double) * ctx->macro.d * ctx->macro.nnode, cudaMemcpyDeviceToHost));
    return FE2_OK;
}

fe2_status fe2_macro_gradients(fe2_ctx* ctx, double* Fbar, double* eta) {
    if (!ctx) return FE2_ERR_ARG;
    if (!ctx->macro_ready || !Fbar) return fail(ctx, FE2_ERR_ARG, "no macro problem / NULL output");
    TIMED("macro_gradients", launch_macro_gradients(ctx->macro, Fbar, eta, ctx->stream));
    return FE2_OK;
}

fe2_status fe2_macro_residual(fe2_ctx* ctx, const double* stress, double* rnorm) {
    if (!ctx) return FE2_ERR_ARG;
    if (!ctx->macro_ready || !stress || !rnorm) return fail(ctx, FE2_ERR_ARG, "no macro problem / NULL pointer");
    TIMED("macro_residual", launch_macro_residual(ctx->macro, stress, rnorm, ctx->stream));
    ctx->launches += 2;  // assembly of R, its norm
    return FE2_OK;
}

fe2_status fe2_macro_solve(fe2_ctx* ctx, const double* sigma, const double* Cbar, double* dFbar, double* rnorm,
                           int* status) {
    if (!ctx) return FE2_ERR_ARG;
    if (!ctx->macro_ready || !sigma || !Cbar || !dFbar || !rnorm)
        return fail(ctx, FE2_ERR_ARG, "no macro problem / NULL pointer");
    int nl = 0;
    if (nq_of(ctx) > 1)
        TIMED("macro_solve", launch_macro_solve_elem(ctx->macro, sigma, Cbar, dFbar, rnorm,
                                                     status ? status : ctx->d_macro_status, ctx->stream, &nl));
    else
        TIMED("macro_solve", launch_macro_solve(ctx->macro, sigma, Cbar, dFbar, rnorm,
                                                status ? status : ctx->d_macro_status, ctx->stream, &nl));
    ctx->launches += nl;
    return FE2_OK;
}

fe2_status fe2_macro_system_size(const fe2_ctx* ctx, int* nfree, int* kd) {
    if (!ctx || !ctx->macro_ready || !nfree || !kd) return FE2_ERR_ARG;
    *nfree = ctx->macro.nfree;
    *kd = ctx->macro.kd;
    return FE2_OK;
}

fe2_status fe2_macro_assemble(fe2_ctx* ctx, const double* sigma, const double* Cbar, double* K, double* R) {
    if (!ctx) return FE2_ERR_ARG;
    if (!ctx->macro_ready || !sigma || !R || (Cbar && !K))
        return fail(ctx, FE2_ERR_ARG, "no macro problem / NULL pointer");
    MacroDev M = ctx->macro;
    M.K = K;
    M.R = R;
    TIMED("macro_assemble", launch_macro_assemble_only(M, sigma, Cbar, nq_of(ctx) > 1, ctx->stream));
    ctx->launches += 1;
    return FE2_OK;
}

fe2_status fe2_macro_norm(fe2_ctx* ctx, const double* R, double* rnorm) {
    if (!ctx) return FE2_ERR_ARG;
    if (!ctx->macro_ready || !R || !rnorm) return fail(ctx, FE2_ERR_ARG, "no macro problem / NULL pointer");
    MacroDev M = ctx->macro;
    M.R = const_cast<double*>(R);
    TIMED("macro_norm", launch_macro_norm(M, rnorm, ctx->stream));
    ctx->launches += 1;
    return FE2_OK;
}

fe2_status fe2_macro_solve_assembled(fe2_ctx* ctx, double* K, double* R, double* dFbar, double* rnorm,
                                     int* status) {
    if (!ctx) return FE2_ERR_ARG;
    if (!ctx->macro_ready || !K || !R || !dFbar || !rnorm)
        return fail(ctx, FE2_ERR_ARG, "no macro problem / NULL pointer");
    MacroDev M = ctx->macro;
    M.K = K;
    M.R = R;
    int nl = 0;
    TIMED("macro_solve", launch_macro_factor_apply(M, dFbar, rnorm, status ? status : ctx->d_macro_status,
                                                   ctx->stream, &nl));
    ctx->launches += nl;
    return FE2_OK;
}

fe2_status fe2_rve_average_stress(fe2_ctx* ctx, int n, const int* rve_ids, double* Pbar) {
    if (!ctx) return FE2_ERR_ARG;
    if (!Pbar) return fail(ctx, FE2_ERR_ARG, "Pbar is NULL");
    const int* d_ids = nullptr;
    fe2_status st = get_ids(ctx, n, rve_ids, &d_ids);
    if (st != FE2_OK) return st;
    if (nq_of(ctx) > 1)
        TIMED("rve_average_stress", launch_rve_avg_stress_elem(ctx->d_tab, d_ids, n, Pbar, ctx->stream));
    else
        TIMED("rve_average_stress", launch_rve_avg_stress(ctx->d_tab, d_ids, n, Pbar, ctx->stream));
    return FE2_OK;
}

fe2_status fe2_rve_set_quad_weights(fe2_ctx* ctx, int n, const int* rve_ids, const double* wq) {
    if (!ctx) return FE2_ERR_ARG;
    if (nq_of(ctx) == 1) return fail(ctx, FE2_ERR_ARG, "quadrature weights belong to element RVEs (FE2_BASIS_CONST)");
    if (n < 0 || (n > 0 && (!rve_ids || !wq))) return fail(ctx, FE2_ERR_ARG, "bad weight arguments");
    const int nq = nq_of(ctx);
    for (int k = 0; k < n; ++k) {
        const int id = rve_ids[k];
        if (id < 0 || id >= (int)ctx->host.size() || !ctx->host[id].active)
            return fail(ctx, FE2_ERR_ARG, "rve id %d is not registered", id);
        for (int g = 0; g < nq; ++g)
            if (!(wq[(size_t)k * nq + g] > 0.0)) return fail(ctx, FE2_ERR_ARG, "weight %d of rve %d is not positive", g, id);
    }
    for (int k = 0; k < n; ++k)
        for (int g = 0; g < nq; ++g) ctx->mirror[rve_ids[k]].wq[g] = wq[(size_t)k * nq + g];
    return upload_all(ctx);
}

fe2_status fe2_rve_residual_norm(fe2_ctx* ctx, int n, const int* rve_ids, double* rnorm) {
    if (!ctx) return FE2_ERR_ARG;
    if (!rnorm) return fail(ctx, FE2_ERR_ARG, "rnorm is NULL");
    const int* d_ids = nullptr;
    fe2_status st = get_ids(ctx, n, rve_ids, &d_ids);
    if (st != FE2_OK) return st;
    TIMED("rve_residual_norm", launch_rve_rnorm(ctx->d_tab, d_ids, n, rnorm, ctx->stream));
    return FE2_OK;
}

}  // extern "C"

// ================================================================== serving
// Continuous batching over execution lanes.  Each lane owns a CUDA stream, a
// factorisation workspace, device/pinned staging and a completion event, so a
// batch formed while another is running is launched at once and overlaps it on
// the device.  A batch takes queued requests of one mesh size (the oldest
// request's) whose RVE is not already in flight; RVE state stays resident.
namespace {

struct ServeReq {
    long long ticket;
    int rve;
    double F[9];
    std::chrono::steady_clock::time_point t0;
};

struct ServeDone {
    long long ticket;
    double sigma[9];
    double C[81];
    int status;
    double lat_ms;
};

// What a lane's launch sequence depends on besides the contents of its buffers:
// a captured graph is replayed only for an equal key.
struct GraphKey {
    int n, maxN, maxkd, maxnr, maxnm, maxnmp, maxnn, lin, tc;
    const void* tab;
    const void* ws;
    bool operator<(const GraphKey& o) const {
        const int a[9] = {n, maxN, maxkd, maxnr, maxnm, maxnmp, maxnn, lin, tc};
        const int b[9] = {o.n, o.maxN, o.maxkd, o.maxnr, o.maxnm, o.maxnmp, o.maxnn, o.lin, o.tc};
        for (int k = 0; k < 9; ++k)
            if (a[k] != b[k]) return a[k] < b[k];
        if (tab != o.tab) return tab < o.tab;
        return ws < o.ws;
    }
};

struct Lane {
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    bool busy = false;
    char* ws = nullptr;
    size_t ws_bytes = 0;
    int *d_ids = nullptr, *h_ids = nullptr, *d_st = nullptr, *h_st = nullptr, *d_redo = nullptr;
    double *d_F = nullptr, *h_F = nullptr, *d_sig = nullptr, *h_sig = nullptr, *d_C = nullptr, *h_C = nullptr;
    double *d_err = nullptr;
    std::vector<ServeReq> batch;
    std::map<GraphKey, cudaGraphExec_t> graphs;  // launch sequences captured per batch shape
    std::deque<GraphKey> graph_order;            // insertion order, for eviction
};

constexpr int kMaxLaneGraphs = 64;

}  // namespace

struct fe2_server {
    fe2_ctx* ctx = nullptr;
    int max_batch = 0;
    bool use_graphs = true;
    long long graph_captures = 0, graph_replays = 0;
    std::vector<Lane> lanes;
    std::deque<ServeReq> queue;
    std::deque<ServeDone> done;
    std::unordered_set<int> inflight;
    long long next_ticket = 1;
    bool bucket = true;                 // batch sizes rounded down to powers of two (graph reuse)
    bool mixed = false;                 // batches may mix mesh sizes (one launch of uneven RVEs)
    long long n_deferred = 0;           // requests passed over for lack of device memory
};

// device bytes of the lanes counted against the budget: their buffers, and their
// workspaces at the size a full batch of the largest defined RVE needs (so that
// admissions leave room for the workspace a lane grows to later)
static size_t lanes_bytes(const fe2_server* srv) {
    fe2_ctx* ctx = srv->ctx;
    const int d = ctx->cfg.dim, dd = d * d;
    size_t wsmax = 0;
    if (ctx->def_maxN) {
        const int N = ctx->def_maxN, kd = compute_kd(ctx, N, d), nm = d * (nodes_of(N, d) - 1);
        const int nmp = (nm + NB - 1) / NB * NB;
        wsmax = (size_t)srv->max_batch * ws_layout(kd, dd + 1, nm, nmp, ctx->cfg.precision == FE2_PREC_FP64,
                                                   ctx->max_smem, d).stride;
    }
    size_t b = 0;
    for (auto& L : srv->lanes)
        b += std::max(L.ws_bytes, wsmax) +
             (size_t)srv->max_batch * (3 * sizeof(int) + sizeof(double) * (dd + dd + dd * dd + 1));
    return b;
}

static fe2_status lane_enqueue(fe2_server* srv, Lane& L, int n, const BatchInfo& b, const WsLayout& l, bool tc,
                               bool record = true);

static fe2_status lane_launch(fe2_server* srv, Lane& L) {
    fe2_ctx* ctx = srv->ctx;
    const int n = (int)L.batch.size();
    const int d = ctx->cfg.dim, dd = d * d;
    std::vector<int> ids(n);
    for (int k = 0; k < n; ++k) {
        ids[k] = L.batch[k].rve;
        L.h_ids[k] = ids[k];
        std::memcpy(L.h_F + (size_t)k * dd, L.batch[k].F, sizeof(double) * dd);
    }
    const BatchInfo b = batch_info(ctx, n, ids.data());
    const bool fp64 = ctx->cfg.precision == FE2_PREC_FP64;
    const WsLayout l = ws_layout(b.maxkd, b.maxnr, b.maxnm, b.maxnmp, fp64, ctx->max_smem, d);
    if (l.stride * (size_t)n > L.ws_bytes) {
        CK(cudaStreamSynchronize(L.s));
        if (L.ws) CK(cudaFree(L.ws));
        L.ws = nullptr;
        L.ws_bytes = 0;
        CK(cudaMalloc(&L.ws, l.stride * (size_t)n));
        L.ws_bytes = l.stride * (size_t)n;
        ctx->extra_bytes = lanes_bytes(srv);
    }
    cudaStream_t s = L.s;
    const bool tc = !fp64 && !l.gw && use_tc_factor(ctx, b.maxkd, b.maxnr);
    if (!srv->use_graphs) return lane_enqueue(srv, L, n, b, l, tc);
    const GraphKey key{n, b.maxN, b.maxkd, b.maxnr, b.maxnm, b.maxnmp, b.maxnn, b.linear_mode(), tc ? 1 : 0,
                       ctx->d_tab, L.ws};
    auto it = L.graphs.find(key);
    if (it == L.graphs.end()) {
        // capture the sequence once for this batch shape (the kernels read ids and Fbar
        // from the lane's fixed buffers, so the graph serves every batch of the shape)
        if ((int)L.graphs.size() >= kMaxLaneGraphs) {
            auto old = L.graphs.find(L.graph_order.front());
            if (old != L.graphs.end()) {
                CK(cudaStreamSynchronize(s));
                cudaGraphExecDestroy(old->second);
                L.graphs.erase(old);
            }
            L.graph_order.pop_front();
        }
        CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
        const fe2_status st = lane_enqueue(srv, L, n, b, l, tc, false);
        cudaGraph_t g = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(s, &g);
        if (st != FE2_OK || ec != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            return st != FE2_OK ? st : fail(ctx, FE2_ERR_CUDA, "lane graph capture: %s", cudaGetErrorString(ec));
        }
        cudaGraphExec_t x = nullptr;
        const cudaError_t ei = cudaGraphInstantiate(&x, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) return fail(ctx, FE2_ERR_CUDA, "lane graph instantiate: %s", cudaGetErrorString(ei));
        it = L.graphs.emplace(key, x).first;
        L.graph_order.push_back(key);
        ++srv->graph_captures;
    } else {
        ++srv->graph_replays;
    }
    CK(cudaGraphLaunch(it->second, s));
    ctx->launches += fp64 ? 5 : 6 + (ctx->cfg.max_refine > 0 ? 1 : 0) + 4 * std::max(0, ctx->cfg.max_refine - 1);
    CK(cudaEventRecord(L.ev, s));
    L.busy = true;
    return FE2_OK;
}

// The lane's launch sequence: inputs in, S1 - S6, results out (and, unless it is
// being captured into a graph, the completion event).
static fe2_status lane_enqueue(fe2_server* srv, Lane& L, int n, const BatchInfo& b, const WsLayout& l, bool tc,
                               bool record) {
    fe2_ctx* ctx = srv->ctx;
    const int d = ctx->cfg.dim, dd = d * d;
    const bool fp64 = ctx->cfg.precision == FE2_PREC_FP64;
    cudaStream_t s = L.s;
    CK(cudaMemcpyAsync(L.d_ids, L.h_ids, sizeof(int) * n, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(L.d_F, L.h_F, sizeof(double) * dd * n, cudaMemcpyHostToDevice, s));
    Workspace ws{L.ws, l.stride, l.offY, l.offR, l.offD, l.offWin};
    CK(launch_check_fbar(L.d_F, n, d, L.d_st, s));
    CK(launch_assemble_fused(ctx->d_tab, L.d_ids, n, L.d_F, d, b.maxN, b.linear_mode(), s));
    if (fp64) {
        if (l.gw)
            CK(launch_factor_gw<double>(ctx->d_tab, L.d_ids, n, ws, L.d_st, b.maxkd, b.maxnr, s));
        else if (use_la_factor(ctx, b.maxkd, b.maxnr, true))
            CK(launch_factor_la<double>(ctx->d_tab, L.d_ids, n, ws, L.d_st, b.maxkd, b.maxnr, s));
        else
            CK(launch_factor<double>(ctx->d_tab, L.d_ids, n, ws, L.d_st, b.maxkd, b.maxnr, s));
        CK(launch_backward<double>(ctx->d_tab, L.d_ids, n, ws, 0, b.maxkd, b.maxnr, b.maxnmp, L.d_st, s));
        CK(launch_schur(ctx->d_tab, L.d_ids, n, ws, 0, L.d_sig, L.d_C, L.d_st, L.d_err, nullptr, nullptr, s));
        if (record) ctx->launches += 5;
    } else {
        if (l.gw)
            CK(launch_factor_gw<float>(ctx->d_tab, L.d_ids, n, ws, L.d_st, b.maxkd, b.maxnr, s));
        else if (tc)
            CK(launch_tc_factor(ctx, ctx->d_tab, L.d_ids, n, ws, L.d_st, b.maxkd, b.maxnr, s));
        else if (use_la_factor(ctx, b.maxkd, b.maxnr, false))
            CK(launch_factor_la<float>(ctx->d_tab, L.d_ids, n, ws, L.d_st, b.maxkd, b.maxnr, s));
        else
            CK(launch_factor<float>(ctx->d_tab, L.d_ids, n, ws, L.d_st, b.maxkd, b.maxnr, s));
        CK(launch_backward<float>(ctx->d_tab, L.d_ids, n, ws, 0, b.maxkd, b.maxnr, b.maxnmp, L.d_st, s));
        CK(launch_residual(ctx->d_tab, L.d_ids, n, ws, b.maxnn, nullptr, s));
        int* redo = ctx->cfg.max_refine > 0 ? L.d_redo : nullptr;
        int it0 = 0;
        if (ctx->cfg.max_refine > 0) {  // second-order pass over every RVE, as in fe2_condense
            CK(launch_solve_correct<float>(ctx->d_tab, L.d_ids, n, ws, b.maxkd, b.maxnr, b.maxnmp, L.d_st, nullptr, s,
                                           1));
            CK(launch_schur(ctx->d_tab, L.d_ids, n, ws, 2, L.d_sig, L.d_C, L.d_st, L.d_err, ctx->d_tol, redo, s,
                            ctx->cfg.max_refine > 1 ? 0 : 3));
            it0 = 1;
        } else {
            CK(launch_schur(ctx->d_tab, L.d_ids, n, ws, 1, L.d_sig, L.d_C, L.d_st, L.d_err, ctx->d_tol, redo, s, 3));
        }
        for (int it = it0; it < ctx->cfg.max_refine; ++it) {
            CK(launch_residual(ctx->d_tab, L.d_ids, n, ws, b.maxnn, L.d_redo, s));
            CK(launch_solve_correct<float>(ctx->d_tab, L.d_ids, n, ws, b.maxkd, b.maxnr, b.maxnmp, L.d_st, L.d_redo, s));
            CK(launch_residual(ctx->d_tab, L.d_ids, n, ws, b.maxnn, L.d_redo, s));
            CK(launch_schur(ctx->d_tab, L.d_ids, n, ws, 1, L.d_sig, L.d_C, L.d_st, L.d_err, ctx->d_tol, L.d_redo, s,
                            it + 1 == ctx->cfg.max_refine ? 2 : 1));
        }
        if (record) ctx->launches += 6 + (ctx->cfg.max_refine > 0 ? 1 : 0) + 4 * std::max(0, ctx->cfg.max_refine - 1);
    }
    CK(cudaMemcpyAsync(L.h_sig, L.d_sig, sizeof(double) * dd * n, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(L.h_C, L.d_C, sizeof(double) * dd * dd * n, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(L.h_st, L.d_st, sizeof(int) * n, cudaMemcpyDeviceToHost, s));
    if (record) {
        CK(cudaEventRecord(L.ev, s));
        L.busy = true;
    }
    return FE2_OK;
}

extern "C" {

fe2_status fe2_server_create(fe2_ctx* ctx, int max_batch, int nlanes, fe2_server** out) {
    if (!ctx || !out) return FE2_ERR_ARG;
    *out = nullptr;
    if (max_batch < 1 || nlanes < 1 || nlanes > 8) return fail(ctx, FE2_ERR_ARG, "bad server sizes");
    if (ctx->cfg.dim != 2) return fail(ctx, FE2_ERR_ARG, "the server batches 2D (Q4) RVEs");
    if (nq_of(ctx) > 1) return fail(ctx, FE2_ERR_ARG, "the server batches Dirac-basis RVEs");
    fe2_server* srv = new fe2_server();
    srv->ctx = ctx;
    srv->max_batch = max_batch;
    srv->lanes.resize(nlanes);
    const int dd = ctx->cfg.dim * ctx->cfg.dim;
    for (auto& L : srv->lanes) {
        cudaError_t e = cudaStreamCreateWithFlags(&L.s, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L.ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMalloc(&L.d_ids, sizeof(int) * max_batch);
        if (e == cudaSuccess) e = cudaMalloc(&L.d_st, sizeof(int) * max_batch);
        if (e == cudaSuccess) e = cudaMalloc(&L.d_redo, sizeof(int) * max_batch);
        if (e == cudaSuccess) e = cudaMalloc(&L.d_F, sizeof(double) * dd * max_batch);
        if (e == cudaSuccess) e = cudaMalloc(&L.d_sig, sizeof(double) * dd * max_batch);
        if (e == cudaSuccess) e = cudaMalloc(&L.d_C, sizeof(double) * dd * dd * max_batch);
        if (e == cudaSuccess) e = cudaMalloc(&L.d_err, sizeof(double) * max_batch);
        if (e == cudaSuccess) e = cudaMallocHost(&L.h_ids, sizeof(int) * max_batch);
        if (e == cudaSuccess) e = cudaMallocHost(&L.h_st, sizeof(int) * max_batch);
        if (e == cudaSuccess) e = cudaMallocHost(&L.h_F, sizeof(double) * dd * max_batch);
        if (e == cudaSuccess) e = cudaMallocHost(&L.h_sig, sizeof(double) * dd * max_batch);
        if (e == cudaSuccess) e = cudaMallocHost(&L.h_C, sizeof(double) * dd * dd * max_batch);
        if (e != cudaSuccess) {
            fe2_server_destroy(srv);
            return fail(ctx, FE2_ERR_CUDA, "server lane allocation: %s", cudaGetErrorString(e));
        }
    }
    ctx->extra_bytes = lanes_bytes(srv);
    *out = srv;
    return FE2_OK;
}

void fe2_server_destroy(fe2_server* srv) {
    if (!srv) return;
    srv->ctx->extra_bytes = 0;
    for (auto& L : srv->lanes) {
        if (L.s) cudaStreamSynchronize(L.s);
        for (auto& g : L.graphs) cudaGraphExecDestroy(g.second);
        cudaFree(L.ws);
        cudaFree(L.d_ids);
        cudaFree(L.d_st);
        cudaFree(L.d_redo);
        cudaFree(L.d_F);
        cudaFree(L.d_sig);
        cudaFree(L.d_C);
        cudaFree(L.d_err);
        cudaFreeHost(L.h_ids);
        cudaFreeHost(L.h_st);
        cudaFreeHost(L.h_F);
        cudaFreeHost(L.h_sig);
        cudaFreeHost(L.h_C);
        if (L.ev) cudaEventDestroy(L.ev);
        if (L.s) cudaStreamDestroy(L.s);
    }
    delete srv;
}

fe2_status fe2_server_submit(fe2_server* srv, int n, const int* rve_ids, const double* Fbar, long long* tickets) {
    if (!srv) return FE2_ERR_ARG;
    fe2_ctx* ctx = srv->ctx;
    if (n < 0 || (n > 0 && (!rve_ids || !Fbar))) return fail(ctx, FE2_ERR_ARG, "bad submit arguments");
    const int dd = ctx->cfg.dim * ctx->cfg.dim;
    const auto now = std::chrono::steady_clock::now();
    for (int k = 0; k < n; ++k) {
        const int id = rve_ids[k];
        if (id < 0 || id >= (int)ctx->host.size() || !ctx->host[id].active)
            return fail(ctx, FE2_ERR_ARG, "rve id %d is not registered", id);
        ServeReq r;
        r.ticket = srv->next_ticket++;
        r.rve = id;
        std::memcpy(r.F, Fbar + (size_t)k * dd, sizeof(double) * dd);
        r.t0 = now;
        srv->queue.push_back(r);
        if (tickets) tickets[k] = r.ticket;
    }
    return FE2_OK;
}

fe2_status fe2_server_pump(fe2_server* srv, int* busy_lanes) {
    if (!srv) return FE2_ERR_ARG;
    fe2_ctx* ctx = srv->ctx;
    const int dd = ctx->cfg.dim * ctx->cfg.dim;
    // harvest finished lanes
    for (auto& L : srv->lanes) {
        if (!L.busy) continue;
        const cudaError_t q = cudaEventQuery(L.ev);
        if (q == cudaErrorNotReady) continue;
        CK(q);
        const auto now = std::chrono::steady_clock::now();
        for (size_t k = 0; k < L.batch.size(); ++k) {
            ServeDone dn;
            dn.ticket = L.batch[k].ticket;
            std::memcpy(dn.sigma, L.h_sig + k * dd, sizeof(double) * dd);
            std::memcpy(dn.C, L.h_C + k * dd * dd, sizeof(double) * dd * dd);
            dn.status = L.h_st[k];
            dn.lat_ms = std::chrono::duration<double, std::milli>(now - L.batch[k].t0).count();
            srv->done.push_back(dn);
            srv->inflight.erase(L.batch[k].rve);
        }
        L.batch.clear();
        L.busy = false;
    }
    // launch new batches on idle lanes
    ctx->extra_bytes = lanes_bytes(srv);
    for (auto& L : srv->lanes) {
        if (L.busy || srv->queue.empty()) continue;
        int Nsel = -1;
        std::unordered_set<int> taken;
        for (auto it = srv->queue.begin(); it != srv->queue.end() && (int)L.batch.size() < srv->max_batch;) {
            const int id = it->rve;
            if (srv->inflight.count(id) || taken.count(id)) {
                ++it;
                continue;
            }
            const int N = ctx->mirror[id].N;
            if (Nsel < 0) Nsel = N;
            if (N != Nsel && !srv->mixed) {
                ++it;
                continue;
            }
            if (!ctx->host[id].resident) {  // admission by HBM budget; idle RVEs may be evicted
                bool ok = true;
                fe2_status st = admit_one(ctx, id, L.s, &ok,
                                          [&](int x) { return srv->inflight.count(x) > 0 || taken.count(x) > 0; });
                if (st != FE2_OK) return st;
                if (!ok) {
                    ++srv->n_deferred;
                    ++it;
                    continue;
                }
            } else if (ctx->host[id].deferred) {
                touch(ctx, id);
            }
            taken.insert(id);
            L.batch.push_back(*it);
            it = srv->queue.erase(it);
        }
        if (srv->bucket && srv->use_graphs && L.batch.size() > 1) {
            // a batch size from a short list, so that lanes replay their captured graphs; the
            // rest go back to the head of the queue in their order (their admission copies,
            // queued on this lane's idle stream, complete first: another lane may take them)
            // sizes 1, 2, 3, 4, 6, 8, 12, 16, 24, ...: powers of two and 1.5 times them, so at
            // most a third of the batch waits for the next one
            size_t m = 1;
            for (size_t p = 1; p <= L.batch.size(); p *= 2) {
                m = p;
                if (p + p / 2 <= L.batch.size() && p >= 2) m = p + p / 2;
            }
            if (m < L.batch.size()) CK(cudaStreamSynchronize(L.s));
            for (size_t k = L.batch.size(); k-- > m;) {
                taken.erase(L.batch[k].rve);
                srv->queue.push_front(L.batch[k]);
            }
            L.batch.resize(m);
        }
        if (L.batch.empty()) continue;
        for (int id : taken) srv->inflight.insert(id);
        fe2_status st = lane_launch(srv, L);
        if (st != FE2_OK) return st;
    }
    if (busy_lanes) {
        int b = 0;
        for (auto& L : srv->lanes) b += L.busy;
        *busy_lanes = b;
    }
    return FE2_OK;
}

int fe2_server_take(fe2_server* srv, int max, long long* tickets, double* sigma, double* Cbar, int* status,
                    double* latency_ms) {
    if (!srv || max < 0) return -1;
    const int dd = srv->ctx->cfg.dim * srv->ctx->cfg.dim;
    int k = 0;
    while (k < max && !srv->done.empty()) {
        const ServeDone& dn = srv->done.front();
        if (tickets) tickets[k] = dn.ticket;
        if (sigma) std::memcpy(sigma + (size_t)k * dd, dn.sigma, sizeof(double) * dd);
        if (Cbar) std::memcpy(Cbar + (size_t)k * dd * dd, dn.C, sizeof(double) * dd * dd);
        if (status) status[k] = dn.status;
        if (latency_ms) latency_ms[k] = dn.lat_ms;
        srv->done.pop_front();
        ++k;
    }
    return k;
}

fe2_status fe2_server_use_graphs(fe2_server* srv, int enable) {
    if (!srv) return FE2_ERR_ARG;
    srv->use_graphs = enable != 0;
    return FE2_OK;
}

fe2_status fe2_server_mixed_sizes(fe2_server* srv, int enable) {
    if (!srv) return FE2_ERR_ARG;
    srv->mixed = enable != 0;
    return FE2_OK;
}

fe2_status fe2_server_bucket(fe2_server* srv, int enable) {
    if (!srv) return FE2_ERR_ARG;
    srv->bucket = enable != 0;
    return FE2_OK;
}

fe2_status fe2_server_memory_stats(const fe2_server* srv, long long* admitted, long long* evicted,
                                   long long* deferred, size_t* device_bytes) {
    if (!srv) return FE2_ERR_ARG;
    if (admitted) *admitted = srv->ctx->n_admitted;
    if (evicted) *evicted = srv->ctx->n_evicted;
    if (deferred) *deferred = srv->n_deferred;
    if (device_bytes) *device_bytes = used_bytes(srv->ctx);
    return FE2_OK;
}

fe2_status fe2_server_graph_stats(const fe2_server* srv, long long* captures, long long* replays) {
    if (!srv) return FE2_ERR_ARG;
    if (captures) *captures = srv->graph_captures;
    if (replays) *replays = srv->graph_replays;
    return FE2_OK;
}

int fe2_server_pending(const fe2_server* srv) {
    if (!srv) return -1;
    int b = 0;
    for (auto& L : srv->lanes) b += (int)L.batch.size();
    return (int)srv->queue.size() + b;
}

}  // extern "C"
