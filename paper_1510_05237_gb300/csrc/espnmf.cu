// espnmf.cu -- the C ABI declared in include/espnmf.h: context set-up, the
// alternating update of Alg. 2, the Sec. 3.1 measures, factor export,
// options, profiling and CUDA-graph replay of whole sweeps.
//
// One sweep (update_V then update_U) enqueues, per half:
//   gram_inverse(other factor's Gram) on the auxiliary stream, concurrently with
//   spmm (+ combine for split rows) on the main stream, then
//   solve+project -> select -> emit -> gram_reduce (+ measures for U).
// The inverse of a factor's Gram only feeds the *next* half-step's solve,
// so it is deferred to the start of that half and runs beside its SpMM.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "../../include/espnmf.h"
#include "common.cuh"
#include "host_layout.cuh"

using namespace espnmf;

namespace espnmf {
const char* kernel_name(int kind)
{
    static const char* names[K_COUNT] = {"spmm_AV", "spmm_AtU", "spmm_combine", "solve_project",
                                         "select_topt", "emit", "gram_reduce",
                                         "gram_inverse", "to_colmajor", "norm2", "ell_dot",
                                         "scatter", "grad", "lambda_max", "pg_apply",
                                         "spmm_freq_AV", "spmm_freq_AtU", "gram_table", "refine",
                                         "spmm_freq2_AV", "spmm_freq2_AtU"};
    return kind >= 0 && kind < K_COUNT ? names[kind] : "?";
}
}  // namespace espnmf

namespace {

thread_local std::string g_init_error;

}  // namespace

void espnmf::set_thread_error(const char* msg) { g_init_error = msg ? msg : ""; }

namespace {

struct Factor {
    int64_t rows = 0;
    EllDev buf[2];
    int cur = 0;
    double* G = nullptr;       // k x k FP64 Gram of the current factor
    double* Ginv64 = nullptr;  // k x k FP64 inverse
    void* GinvT = nullptr;     // k x k inverse in T
    float* Lf = nullptr;       // FP32 form, k <= 64: Cholesky factor (L, L^T, 1/diag)
    void* sel_hint = nullptr;  // FP32 form: each column's last selection threshold (k keys, 0: none)
    bool chol_pending = true;
    bool valid = false;        // holds a value (V is empty until the first update)
};

struct ProfRec {
    int kind;
    cudaEvent_t a, b;
    double bytes;
};

struct Stat {
    int64_t launches = 0;
    double ms = 0.0;
    double bytes = 0.0;
};

}  // namespace

// Alg. 3 (sequential ALS): the converged topics held densely (rows x ld1,
// first k1 columns valid) while a k = k2 context finds the next block.
struct Deflation {
    bool active = false;   // espnmf_sequential's context: the hook runs in every half-step
    void* U1 = nullptr;
    void* V1 = nullptr;
    int ld1 = 0;
    int k1_max = 0;        // the most converged topics a block has (k - k2)
    int* k1 = nullptr;     // device: the converged topics of the current block
    double* g = nullptr;
};

struct espnmf_ctx {
    int device = 0;
    int sm_count = 0;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;

    int64_t n = 0, m = 0, nnz = 0;
    int k = 0;
    int64_t t_u = 0, t_v = 0;
    int mode = 0;
    espnmf_dtype dt = ESPNMF_F32;
    size_t esz = 4;

    SellDev sA;   // rows of A   -> Y = A V
    SellDev sAt;  // rows of A^T -> Y = A^T U
    Factor U, V;

    void* Y = nullptr;
    int64_t ldy = 0;
    void* Xt = nullptr;
    int64_t ldx = 0;

    int fin_blocks = 0;
    double* gram_part = nullptr;
    double* scal_part = nullptr;
    double* scal = nullptr;
    unsigned* gram_counter = nullptr;
    double* A2 = nullptr;
    double* norm_part = nullptr;
    double* met = nullptr;      // [0] R, [1] E, [2] f, [3] trace
    double* dot = nullptr;      // scratch scalar
    double* pg = nullptr;       // [0] projected-gradient step eta, [1] lambda_max
    void* tau = nullptr;        // selector thresholds (k keys of 8 bytes)
    uint32_t* cut = nullptr;    // selector tie cut-offs (k)
    double* hist_R = nullptr;
    double* hist_E = nullptr;
    int* hist_counter = nullptr;
    int hist_cap = 0;
    unsigned* status_d = nullptr;
    unsigned* status_h = nullptr;
    // FP32 form, column mode: the selector marks the survivors (rowbits,
    // ceil(k/32) words per row of the larger factor, kept zero between
    // updates) and writes the Gram diagonal (diag_part, k x cluster size)
    uint32_t* rowbits = nullptr;
    unsigned long long* sel_counts = nullptr;   // FP32: column selections [warm, full search]
    Deflation defl;                             // espnmf_sequential only
    double* diag_part = nullptr;

    bool have_R = false;
    bool Y_is_AV = false;
    bool met_valid = false;
    int64_t sweeps = 0;   // completed U updates (Alg. 2 sweeps) since init or load
    bool refine = false;  // FP32 form (Cholesky path): one refinement step of each solve

    bool use_graph = true;
    // FP32 sparse-product launch shapes, [0] A V (rows of A), [1] A^T U
    SpmmConfig spmm_cfg[2];
    bool spmm_tune = true;
    bool spmm_tuned = false;
    cudaGraphExec_t gexec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};

    bool profile = false;
    std::vector<ProfRec> pending;
    std::vector<cudaEvent_t> ev_pool;
    Stat stats[K_COUNT];
    int launches_this = 0;
    int64_t wait_limit = 1ll << 26;

    std::vector<void*> allocs;
    std::string err;
};

namespace {

espnmf_status set_err(espnmf_ctx* c, espnmf_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    else g_init_error = buf;
    return s;
}

#define CU(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return set_err(ctx, ESPNMF_ERR_CUDA, "%s:%d %s: %s", __FILE__, __LINE__,    \
                           #call, cudaGetErrorString(e_));                              \
    } while (0)

#define TRY(expr)                                \
    do {                                         \
        espnmf_status s_ = (expr);               \
        if (s_ != ESPNMF_OK) return s_;          \
    } while (0)

template <typename P>
espnmf_status dmalloc(espnmf_ctx* ctx, P** p, size_t bytes)
{
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_err(ctx, ESPNMF_ERR_OOM, "cudaMalloc(%zu bytes): %s", bytes,
                       cudaGetErrorString(e));
    }
    ctx->allocs.push_back(q);
    *p = static_cast<P*>(q);
    return ESPNMF_OK;
}

template <typename P>
espnmf_status dupload(espnmf_ctx* ctx, P** p, const void* src, size_t bytes)
{
    TRY(dmalloc(ctx, p, bytes));
    if (bytes) CU(cudaMemcpyAsync(*p, src, bytes, cudaMemcpyHostToDevice, ctx->st));
    return ESPNMF_OK;
}

// --- kernel launches with optional event timing ------------------------------

cudaEvent_t pool_event(espnmf_ctx* ctx)
{
    if (!ctx->ev_pool.empty()) {
        cudaEvent_t e = ctx->ev_pool.back();
        ctx->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

template <typename F>
espnmf_status run(espnmf_ctx* ctx, int kind, double bytes, cudaStream_t s, F&& launch)
{
    cudaEvent_t a = nullptr, b = nullptr;
    if (ctx->profile) {
        a = pool_event(ctx);
        b = pool_event(ctx);
        CU(cudaEventRecord(a, s));
    }
    cudaError_t e = launch();
    if (e != cudaSuccess)
        return set_err(ctx, ESPNMF_ERR_CUDA, "launch of %s failed: %s", kernel_name(kind),
                       cudaGetErrorString(e));
    ctx->launches_this++;
    if (ctx->profile) {
        CU(cudaEventRecord(b, s));
        ctx->pending.push_back({kind, a, b, bytes});
    }
    return ESPNMF_OK;
}

espnmf_status collect_profile(espnmf_ctx* ctx)
{
    for (auto& r : ctx->pending) {
        CU(cudaEventSynchronize(r.b));
        float ms = 0.f;
        CU(cudaEventElapsedTime(&ms, r.a, r.b));
        Stat& s = ctx->stats[r.kind];
        s.launches++;
        s.ms += ms;
        s.bytes += r.bytes;
        ctx->ev_pool.push_back(r.a);
        ctx->ev_pool.push_back(r.b);
    }
    ctx->pending.clear();
    return ESPNMF_OK;
}

// --- device status -------------------------------------------------------------

espnmf_status check_status(espnmf_ctx* ctx)
{
    CU(cudaMemcpyAsync(ctx->status_h, ctx->status_d, sizeof(unsigned), cudaMemcpyDeviceToHost,
                       ctx->st));
    CU(cudaStreamSynchronize(ctx->st));
    CU(cudaGetLastError());
    const unsigned s = *ctx->status_h;
    if (s == 0) return ESPNMF_OK;
    CU(cudaMemsetAsync(ctx->status_d, 0, sizeof(unsigned), ctx->st));
    CU(cudaStreamSynchronize(ctx->st));
    if (s & ST_SINGULAR)
        return set_err(ctx, ESPNMF_ERR_SINGULAR,
                       "a Gram matrix (U^T U or V^T V) is singular beyond its zero columns");
    if (s & ST_NONFINITE) return set_err(ctx, ESPNMF_ERR_NONFINITE, "non-finite value in an iterate");
    if (s & ST_BADINPUT) return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "negative entry in a factor");
    if (s & ST_TIMEOUT) return set_err(ctx, ESPNMF_ERR_TIMEOUT, "a bounded device wait gave up");
    if (s & ST_OVERFLOW) return set_err(ctx, ESPNMF_ERR_CUDA, "internal: factor row overflow");
    return set_err(ctx, ESPNMF_ERR_CUDA, "unknown device status 0x%x", s);
}

using namespace espnmf::layout;

espnmf_status upload_tier(espnmf_ctx* ctx, const FreqTierHost& H, FreqTierDev& D)
{
    D.nnz = H.nnz;
    D.nent = (int64_t)H.ent.size();
    D.nrows = (int)H.rows.size();
    D.nchunks = (int)H.chunk.size() - 1;
    TRY(dupload(ctx, &D.ent, H.ent.data(), H.ent.size() * sizeof(uint2)));
    TRY(dupload(ctx, &D.rows, H.rows.data(), H.rows.size() * sizeof(int2)));
    TRY(dupload(ctx, &D.chunk, H.chunk.data(), H.chunk.size() * 4));
    TRY(dmalloc(ctx, &D.counter, sizeof(int)));
    return ESPNMF_OK;
}

espnmf_status upload_frequent(espnmf_ctx* ctx, const FreqHost& H, SellDev& D)
{
    D.h = H.h;
    D.h1 = H.h1;
    TRY(dupload(ctx, &D.slot_of, H.slot_of.data(), H.slot_of.size() * 4));
    TRY(upload_tier(ctx, H.t[0], D.ft[0]));
    if (H.h > H.h1) TRY(upload_tier(ctx, H.t[1], D.ft[1]));
    CU(cudaStreamSynchronize(ctx->st));
    return ESPNMF_OK;
}

template <typename T>
espnmf_status upload_sell(espnmf_ctx* ctx, const SellHost<T>& H, SellDev& D)
{
    D.rows = H.rows;
    D.nseg = H.nseg;
    D.nslices = H.nslices;
    D.total = H.total;
    D.nnz = H.nnz;
    D.nsplit = (int64_t)H.split_row.size();
    D.npart = H.npart;
    TRY(dupload(ctx, &D.slice_ptr, H.slice_ptr.data(), H.slice_ptr.size() * 8));
    TRY(dupload(ctx, &D.slice_len, H.slice_len.data(), H.slice_len.size() * 4));
    TRY(dupload(ctx, &D.idx, H.idx.data(), H.idx.size() * 4));
    TRY(dupload(ctx, &D.val, H.val.data(), H.val.size() * sizeof(T)));
    TRY(dupload(ctx, &D.seg_row, H.seg_row.data(), H.seg_row.size() * 4));
    TRY(dupload(ctx, &D.seg_part, H.seg_part.data(), H.seg_part.size() * 4));
    TRY(dupload(ctx, &D.seg_grp, H.seg_grp.data(), H.seg_grp.size() * 4));
    TRY(dupload(ctx, &D.split_row, H.split_row.data(), H.split_row.size() * 4));
    TRY(dupload(ctx, &D.split_first, H.split_first.data(), H.split_first.size() * 4));
    TRY(dupload(ctx, &D.split_count, H.split_count.data(), H.split_count.size() * 4));
    TRY(dmalloc(ctx, &D.partials, (size_t)H.npart * factor_ld(ctx->k) * sizeof(T)));
    // host vectors die with H: make sure the copies are done
    CU(cudaStreamSynchronize(ctx->st));
    return ESPNMF_OK;
}

// --- per-dtype dispatch ------------------------------------------------------------

bool is_f64(const espnmf_ctx* ctx) { return ctx->dt == ESPNMF_F64; }

espnmf_status do_spmm(espnmf_ctx* ctx, bool transA, const EllDev& F)
{
    const SellDev& S = transA ? ctx->sAt : ctx->sA;
    // the SELL part: its entries (index + value), slice pointers, Y written
    const double bytes = (double)S.nnz * (4.0 + ctx->esz) +
                         (double)(S.nslices + 1) * 8.0 + (double)S.rows * ctx->ldy * ctx->esz;
    TRY(run(ctx, transA ? K_SPMM_T : K_SPMM, bytes, ctx->st, [&] {
        const SpmmConfig cfg = ctx->spmm_cfg[transA ? 1 : 0];
        return is_f64(ctx) ? launch_spmm<double>(S, F, ctx->k, (double*)ctx->Y, ctx->ldy, cfg,
                                                 ctx->st, ctx->sm_count)
                           : launch_spmm<float>(S, F, ctx->k, (float*)ctx->Y, ctx->ldy, cfg,
                                                ctx->st, ctx->sm_count);
    }));
    if (S.nsplit > 0) {
        const double cb = (double)S.npart * ctx->ldy * ctx->esz;
        TRY(run(ctx, K_COMBINE, cb, ctx->st, [&] {
            return is_f64(ctx) ? launch_spmm_combine<double>(S, (int)ctx->ldy, (double*)ctx->Y, ctx->ldy, ctx->st)
                               : launch_spmm_combine<float>(S, (int)ctx->ldy, (float*)ctx->Y, ctx->ldy, ctx->st);
        }));
    }
    for (int tier = 1; tier <= 2; ++tier) {
        const FreqTierDev& T = S.ft[tier - 1];
        if (S.h == 0 || T.nrows == 0 || (tier == 2 && S.h <= S.h1)) continue;
        // entries (table row offset + value, padding included), row list,
        // Y read and written back for the rows with entries
        const double hb = (double)T.nent * 8.0 + (double)T.nrows * 8.0 +
                          2.0 * (double)T.nrows * ctx->ldy * 4.0;
        const KernelKind kind = tier == 1 ? (transA ? K_SPMM_H_T : K_SPMM_H)
                                          : (transA ? K_SPMM_H2_T : K_SPMM_H2);
        TRY(run(ctx, kind, hb, ctx->st, [&] {
            return launch_spmm_h(S, F, (float*)ctx->Y, ctx->sm_count, ctx->status_d,
                                 ctx->wait_limit, ctx->st, tier);
        }));
    }
    return ESPNMF_OK;
}

void drop_graphs(espnmf_ctx* ctx);

// Times every FP32 launch shape of both sparse products on the current
// factors (each shape gives bitwise the same Y) and keeps the fastest.
// Leaves Y = A V, as the last U update did.
// The tuner's picks, kept for the process and keyed by the product's shape
// class (the factor width, log2 of the output rows and of the entries per
// row, whether the product has a frequent part and whether the bitmask can
// be staged), so that contexts of the same class skip the timing.
struct TuneKey {
    int ld, lrows, ldens, freq, smask;
    bool operator<(const TuneKey& o) const
    {
        return std::tie(ld, lrows, ldens, freq, smask) < std::tie(o.ld, o.lrows, o.ldens, o.freq, o.smask);
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, SpmmConfig> g_tune_cache;

TuneKey tune_key(const espnmf_ctx* ctx, int o)
{
    const SellDev& S = o ? ctx->sAt : ctx->sA;
    const int64_t rows = std::max<int64_t>(S.rows, 1);
    auto lg = [](double x) { return x < 1.0 ? 0 : (int)std::floor(std::log2(x)); };
    const int64_t gathered = o ? ctx->n : ctx->m;
    return {(int)ctx->ldy, lg((double)rows), lg(4.0 * (double)ctx->nnz / (double)rows),
            S.h > 0 ? 1 : 0, gathered > 32ll * kSellSmemMaskWords ? 0 : 1};
}

espnmf_status tune_spmm(espnmf_ctx* ctx)
{
    ctx->spmm_tuned = true;
    if (is_f64(ctx)) return ESPNMF_OK;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto a = g_tune_cache.find(tune_key(ctx, 0)), b = g_tune_cache.find(tune_key(ctx, 1));
        if (a != g_tune_cache.end() && b != g_tune_cache.end()) {
            ctx->spmm_cfg[0] = a->second;
            ctx->spmm_cfg[1] = b->second;
            drop_graphs(ctx);
            return ESPNMF_OK;
        }
    }
    std::vector<SpmmConfig> cands;
    for (int sp : {1, 2, 4}) {
        if (sp > 1 && ctx->ldy < 16) continue;
        for (int cv : {100, 75, 50})
            for (int mk : {0, 1, 2}) {
                if (mk == 2 && std::max(ctx->n, ctx->m) > 32ll * kSellSmemMaskWords) continue;
                SpmmConfig c;
                c.split = sp;
                c.carveout = cv;
                c.mask = mk;
                cands.push_back(c);
            }
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    espnmf_status st = ESPNMF_OK;
    for (int o = 1; o >= 0 && st == ESPNMF_OK; --o) {
        const SellDev& S = o ? ctx->sAt : ctx->sA;
        const EllDev& F = o ? ctx->U.buf[ctx->U.cur] : ctx->V.buf[ctx->V.cur];
        float best = 1e30f;
        SpmmConfig pick = ctx->spmm_cfg[o];
        for (const SpmmConfig& c : cands) {
            cudaError_t e = launch_spmm<float>(S, F, ctx->k, (float*)ctx->Y, ctx->ldy, c, ctx->st,
                                               ctx->sm_count);
            if (e == cudaSuccess) e = cudaEventRecord(e0, ctx->st);
            for (int r = 0; r < 3 && e == cudaSuccess; ++r)
                e = launch_spmm<float>(S, F, ctx->k, (float*)ctx->Y, ctx->ldy, c, ctx->st,
                                       ctx->sm_count);
            if (e == cudaSuccess) e = cudaEventRecord(e1, ctx->st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) {
                st = set_err(ctx, ESPNMF_ERR_CUDA, "spmm tuning: %s", cudaGetErrorString(e));
                break;
            }
            if (ms < best) {
                best = ms;
                pick = c;
            }
        }
        ctx->spmm_cfg[o] = pick;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    TRY(st);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[tune_key(ctx, 0)] = ctx->spmm_cfg[0];
        g_tune_cache[tune_key(ctx, 1)] = ctx->spmm_cfg[1];
    }
    drop_graphs(ctx);
    TRY(do_spmm(ctx, false, ctx->V.buf[ctx->V.cur]));
    ctx->Y_is_AV = true;
    return ESPNMF_OK;
}

bool use_cholesky(const espnmf_ctx* ctx) { return !is_f64(ctx) && ctx->ldy <= 64; }

espnmf_status do_gram_inverse(espnmf_ctx* ctx, Factor& F, cudaStream_t s)
{
    if (use_cholesky(ctx)) {
        const int KP = (int)ctx->ldy;
        return run(ctx, K_INVERSE, (double)ctx->k * ctx->k * 8.0 + 2.0 * KP * KP * 4.0, s, [&] {
            float* gh = F.Lf + 2 * KP * KP + KP;   // G as an FP32 pair, for the refinement
            return launch_cholesky(F.G, ctx->k, KP, F.Lf, F.Lf + KP * KP, F.Lf + 2 * KP * KP,
                                   ctx->status_d, s, gh, gh + KP * KP);
        });
    }
    const double bytes = (double)ctx->k * ctx->k * (8.0 + 8.0 + ctx->esz);
    return run(ctx, K_INVERSE, bytes, s, [&] {
        return is_f64(ctx) ? launch_gram_inverse<double>(F.G, ctx->k, F.Ginv64, (double*)F.GinvT,
                                                     ctx->status_d, s)
                           : launch_gram_inverse<float>(F.G, ctx->k, F.Ginv64, (float*)F.GinvT,
                                                    ctx->status_d, s);
    });
}

// Writes factor F's next buffer from the projected candidate in Xt and the
// selector's thresholds (tau/cut), zeroes the current buffer's counts, and
// reduces the new Gram matrix (with R and E when `metrics`).  The buffers
// are swapped afterwards.
espnmf_status do_emit(espnmf_ctx* ctx, Factor& F, bool residual, const void* Y, bool metrics,
                      int mode)
{
    EllDev& nxt = F.buf[F.cur ^ 1];
    EllDev& cur = F.buf[F.cur];
    const double bytes = (double)F.rows * ctx->k * ctx->esz + (double)F.rows * 8.0 +
                         (double)ctx->fin_blocks * ctx->k * ctx->k * 8.0;
    TRY(run(ctx, K_EMIT, bytes, ctx->st, [&] {
        return is_f64(ctx)
                   ? launch_emit<double>((const double*)ctx->Xt, ctx->ldx, F.rows, ctx->k, mode,
                                         ctx->tau, ctx->cut, nxt, cur, residual, (const double*)Y,
                                         ctx->ldy, ctx->gram_part, ctx->scal_part,
                                         ctx->fin_blocks, ctx->st)
                   : launch_emit<float>((const float*)ctx->Xt, ctx->ldx, F.rows, ctx->k, mode,
                                        ctx->tau, ctx->cut, nxt, cur, residual, (const float*)Y,
                                        ctx->ldy, ctx->gram_part, ctx->scal_part,
                                        ctx->fin_blocks, ctx->st);
    }));
    MetricsArgs ma;
    if (metrics) {
        ma.enabled = true;
        ma.G_other = ctx->V.G;
        ma.A2 = ctx->A2;
        ma.out = ctx->met;
        ma.hist_R = ctx->hist_R;
        ma.hist_E = ctx->hist_E;
        ma.hist_counter = ctx->hist_counter;
        ma.hist_cap = ctx->hist_cap;
    }
    const double rb = (double)ctx->fin_blocks * ctx->k * (ctx->k + 1) / 2 * 8.0;
    TRY(run(ctx, K_GRAM_REDUCE, rb, ctx->st, [&] {
        return launch_gram_reduce(ctx->gram_part, ctx->scal_part, ctx->fin_blocks,
                                  ctx->fin_blocks, ctx->k, nullptr, 0, false, F.G, ctx->scal,
                                  ctx->gram_counter, ma, ctx->st);
    }));
    F.cur ^= 1;
    F.chol_pending = true;
    return ESPNMF_OK;
}

espnmf_status do_select(espnmf_ctx* ctx, int64_t rows, int64_t t, bool mark, void* hint)
{
    return run(ctx, K_SELECT, (double)rows * ctx->k * ctx->esz, ctx->st, [&] {
        return is_f64(ctx) ? launch_select<double>((const double*)ctx->Xt, ctx->ldx, rows, ctx->k,
                                                   t, ctx->mode, ctx->tau, ctx->cut, ctx->st,
                                                   ctx->sm_count, nullptr, nullptr)
                           : launch_select<float>((const float*)ctx->Xt, ctx->ldx, rows, ctx->k,
                                                  t, ctx->mode, ctx->tau, ctx->cut, ctx->st,
                                                  ctx->sm_count, mark ? ctx->rowbits : nullptr,
                                                  mark ? ctx->diag_part : nullptr,
                                                  mark ? hint : nullptr,
                                                  mark ? ctx->sel_counts : nullptr);
    });
}

// The half-step's survivors were marked by the selector (FP32 form, column
// mode): writes factor F's next buffer from them, the Gram of the frequent
// rows from the table, and reduces the Gram (and R, E with `metrics`).
espnmf_status do_emit_survivors(espnmf_ctx* ctx, Factor& F, bool residual, const void* Y,
                                bool metrics)
{
    EllDev& nxt = F.buf[F.cur ^ 1];
    EllDev& cur = F.buf[F.cur];
    const int Pe = ctx->fin_blocks;
    const bool tab = nxt.h > 0;
    const int P = Pe + (tab ? ctx->sm_count : 0);
    const int ntri = ctx->k * (ctx->k + 1) / 2;
    // the rows' survivor bits and counts, the survivors' values and pairs
    const double bytes = (double)F.rows * (4.0 * ((ctx->k + 31) / 32) + 4.0 + 16.0) +
                         (double)Pe * ntri * 8.0;
    TRY(run(ctx, K_EMIT, bytes, ctx->st, [&] {
        return launch_emit_s((const float*)ctx->Xt, ctx->ldx, F.rows, ctx->k, ctx->rowbits, nxt,
                             cur, residual, (const float*)Y, ctx->ldy, ctx->gram_part,
                             ctx->scal_part, Pe, P, ctx->st);
    }));
    if (tab)
        TRY(run(ctx, K_GRAM_TABLE, (double)nxt.h * nxt.ld * 4.0, ctx->st, [&] {
            return launch_gram_table(nxt, ctx->k, ctx->gram_part, P, Pe, ctx->sm_count, ctx->st);
        }));
    MetricsArgs ma;
    if (metrics) {
        ma.enabled = true;
        ma.G_other = ctx->V.G;
        ma.A2 = ctx->A2;
        ma.out = ctx->met;
        ma.hist_R = ctx->hist_R;
        ma.hist_E = ctx->hist_E;
        ma.hist_counter = ctx->hist_counter;
        ma.hist_cap = ctx->hist_cap;
    }
    const int Cd = select_cluster(F.rows, ctx->k, TOPT_COLUMN, ctx->sm_count);
    TRY(run(ctx, K_GRAM_REDUCE, (double)P * ntri * 8.0, ctx->st, [&] {
        return launch_gram_reduce(ctx->gram_part, ctx->scal_part, P, Pe, ctx->k, ctx->diag_part,
                                  Cd, true, F.G, ctx->scal, ctx->gram_counter, ma, ctx->st);
    }));
    F.cur ^= 1;
    F.chol_pending = true;
    return ESPNMF_OK;
}

bool survivor_path(const espnmf_ctx* ctx) { return ctx->rowbits != nullptr && ctx->mode == TOPT_COLUMN; }

// Alg. 2 steps 1-2 (updV) or 3-4.
espnmf_status half_update(espnmf_ctx* ctx, bool updV)
{
    Factor& F = updV ? ctx->V : ctx->U;
    Factor& O = updV ? ctx->U : ctx->V;
    const int64_t rows = F.rows;
    // The other factor's Gram inverse runs beside the SpMM.
    CU(cudaEventRecord(ctx->ev_fork, ctx->st));
    CU(cudaStreamWaitEvent(ctx->aux, ctx->ev_fork, 0));
    TRY(do_gram_inverse(ctx, O, ctx->aux));
    CU(cudaEventRecord(ctx->ev_join, ctx->aux));
    O.chol_pending = false;

    TRY(do_spmm(ctx, updV, O.buf[O.cur]));
    if (ctx->defl.active) {
        // Alg. 3: subtract the converged topics' part (Eq. 7 / Eq. 8); the
        // number of converged topics is read on the device
        const Deflation& d = ctx->defl;
        const EllDev& f = O.buf[O.cur];
        const void* G1 = updV ? d.U1 : d.V1;
        void* H1 = updV ? d.V1 : d.U1;
        CU(is_f64(ctx) ? launch_seq_deflate<double>(O.rows, (const double*)G1, rows, (const double*)H1,
                                                    d.ld1, d.k1_max, d.k1, ctx->k, f.cnt, f.col,
                                                    (const double*)f.val, f.ld, d.g,
                                                    (double*)ctx->Y, ctx->ldy, ctx->st)
                       : launch_seq_deflate<float>(O.rows, (const float*)G1, rows, (const float*)H1,
                                                   d.ld1, d.k1_max, d.k1, ctx->k, f.cnt, f.col,
                                                   (const float*)f.val, f.ld, d.g,
                                                   (float*)ctx->Y, ctx->ldy, ctx->st));
    }
    CU(cudaStreamWaitEvent(ctx->st, ctx->ev_join, 0));

    const double sb = (double)rows * ctx->k * ctx->esz * 2.0;
    TRY(run(ctx, K_SOLVE, sb, ctx->st, [&] {
        if (use_cholesky(ctx)) {
            const int KP = (int)ctx->ldy;
            return launch_solve_chol((const float*)ctx->Y, ctx->ldy, rows, ctx->k, KP, O.Lf,
                                     O.Lf + KP * KP, O.Lf + 2 * KP * KP, (float*)ctx->Xt,
                                     ctx->ldx, ctx->status_d, ctx->st, ctx->sm_count,
                                     !ctx->refine);
        }
        return is_f64(ctx) ? launch_solve<double>((const double*)ctx->Y, ctx->ldy, rows, ctx->k,
                                                  (const double*)O.GinvT, (double*)ctx->Xt,
                                                  ctx->ldx, ctx->status_d, ctx->st, ctx->sm_count)
                           : launch_solve<float>((const float*)ctx->Y, ctx->ldy, rows, ctx->k,
                                                 (const float*)O.GinvT, (float*)ctx->Xt, ctx->ldx,
                                                 ctx->status_d, ctx->st, ctx->sm_count);
    }));
    if (use_cholesky(ctx) && ctx->refine) {
        // one step of iterative refinement of the solve (projects at the end)
        const int KP = (int)ctx->ldy;
        const float* gh = O.Lf + 2 * KP * KP + KP;
        TRY(run(ctx, K_REFINE, (double)rows * ctx->k * ctx->esz * 3.0, ctx->st, [&] {
            return launch_refine((const float*)ctx->Y, ctx->ldy, nullptr, 0, rows, ctx->k, KP, O.Lf,
                                 O.Lf + 2 * KP * KP, gh, gh + KP * KP, (float*)ctx->Xt, ctx->ldx,
                                 nullptr, 0, false, true, ctx->status_d, ctx->st, ctx->sm_count);
        }));
    }
    const int64_t t = updV ? ctx->t_v : ctx->t_u;
    if (survivor_path(ctx)) {
        TRY(do_select(ctx, rows, t, true, F.sel_hint));
        TRY(do_emit_survivors(ctx, F, !updV && F.valid, updV ? nullptr : ctx->Y, !updV));
    } else {
        TRY(do_select(ctx, rows, t, false, nullptr));
        TRY(do_emit(ctx, F, !updV && F.valid, updV ? nullptr : ctx->Y, !updV, ctx->mode));
    }
    F.valid = true;
    if (updV) {
        ctx->Y_is_AV = false;
        ctx->met_valid = false;
    } else {
        ctx->Y_is_AV = true;
        ctx->met_valid = true;
        ctx->have_R = true;
        ++ctx->sweeps;
    }
    return ESPNMF_OK;
}

espnmf_status enqueue_sweep(espnmf_ctx* ctx)
{
    TRY(half_update(ctx, true));
    TRY(half_update(ctx, false));
    return ESPNMF_OK;
}

struct HostState {
    int ucur, vcur;
    bool upend, vpend, uvalid, vvalid, have_R, Y_is_AV, met_valid;
    int64_t sweeps;
};

HostState save_state(const espnmf_ctx* c)
{
    return {c->U.cur, c->V.cur, c->U.chol_pending, c->V.chol_pending, c->U.valid, c->V.valid,
            c->have_R, c->Y_is_AV, c->met_valid, c->sweeps};
}

void restore_state(espnmf_ctx* c, const HostState& s)
{
    c->U.cur = s.ucur;
    c->V.cur = s.vcur;
    c->U.chol_pending = s.upend;
    c->V.chol_pending = s.vpend;
    c->U.valid = s.uvalid;
    c->V.valid = s.vvalid;
    c->have_R = s.have_R;
    c->Y_is_AV = s.Y_is_AV;
    c->met_valid = s.met_valid;
    c->sweeps = s.sweeps;
}

void drop_graphs(espnmf_ctx* ctx)
{
    for (auto& row : ctx->gexec)
        for (auto& g : row)
            if (g) {
                cudaGraphExecDestroy(g);
                g = nullptr;
            }
}

espnmf_status sweep_graph(espnmf_ctx* ctx, cudaGraphExec_t* out)
{
    const HostState s0 = save_state(ctx);
    // the graph is captured once V exists; a sweep always has it afterwards
    CU(cudaStreamBeginCapture(ctx->st, cudaStreamCaptureModeThreadLocal));
    espnmf_status st = enqueue_sweep(ctx);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(ctx->st, &g);
    restore_state(ctx, s0);
    if (st != ESPNMF_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return set_err(ctx, ESPNMF_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return set_err(ctx, ESPNMF_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    return ESPNMF_OK;
}

void after_sweep_state(espnmf_ctx* c)
{
    c->U.cur ^= 1;
    c->V.cur ^= 1;
    c->U.chol_pending = true;
    c->V.chol_pending = true;
    c->U.valid = c->V.valid = true;
    c->have_R = c->Y_is_AV = c->met_valid = true;
    ++c->sweeps;
}

espnmf_status ensure_hist(espnmf_ctx* ctx, int need)
{
    if (need <= ctx->hist_cap) return ESPNMF_OK;
    int cap = std::max(need, std::max(64, ctx->hist_cap * 2));
    double *r = nullptr, *e = nullptr;
    TRY(dmalloc(ctx, &r, sizeof(double) * cap));
    TRY(dmalloc(ctx, &e, sizeof(double) * cap));
    ctx->hist_R = r;
    ctx->hist_E = e;
    ctx->hist_cap = cap;
    drop_graphs(ctx);   // the captured sweeps point at the old arrays
    return ESPNMF_OK;
}

espnmf_status enter(espnmf_ctx* ctx)
{
    if (!ctx) return ESPNMF_ERR_INVALID_ARG;
    ctx->err.clear();
    CU(cudaSetDevice(ctx->device));
    return ESPNMF_OK;
}

// Replaces factor F by a dense rows x k matrix (host or device).
espnmf_status set_factor_impl(espnmf_ctx* ctx, Factor& F, const void* src, espnmf_dtype dtype,
                              int on_device)
{
    if (!src) return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "factor pointer is NULL");
    if (dtype != ESPNMF_F64 && dtype != ESPNMF_F32 && dtype != ESPNMF_BF16)
        return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "factor dtype must be F64, F32 or BF16");
    const size_t es = dtype == ESPNMF_F64 ? 8 : dtype == ESPNMF_F32 ? 4 : 2;
    const size_t bytes = (size_t)F.rows * ctx->k * es;
    const void* dptr = src;
    void* tmp = nullptr;
    void* tmp32 = nullptr;
    if (!on_device) {
        CU(cudaMallocAsync(&tmp, bytes ? bytes : 16, ctx->st));
        CU(cudaMemcpyAsync(tmp, src, bytes, cudaMemcpyHostToDevice, ctx->st));
        dptr = tmp;
    }
    if (dtype == ESPNMF_BF16) {
        // widened to FP32 (exact), then handled as an FP32 factor
        const int64_t count = F.rows * (int64_t)ctx->k;
        CU(cudaMallocAsync(&tmp32, count ? (size_t)count * 4 : 16, ctx->st));
        CU(launch_bf16_to_f32(static_cast<const uint16_t*>(dptr), count, static_cast<float*>(tmp32),
                              ctx->st));
        dptr = tmp32;
        dtype = ESPNMF_F32;
    }
    const double cb = (double)F.rows * ctx->k * (es + ctx->esz);
    espnmf_status s = run(ctx, K_TO_COLMAJOR, cb, ctx->st, [&] {
        if (dtype == ESPNMF_F64)
            return is_f64(ctx) ? launch_dense_to_colmajor<double, double>(
                                     (const double*)dptr, F.rows, ctx->k, ctx->k, (double*)ctx->Xt,
                                     ctx->ldx, ctx->status_d, true, ctx->st)
                               : launch_dense_to_colmajor<double, float>(
                                     (const double*)dptr, F.rows, ctx->k, ctx->k, (float*)ctx->Xt,
                                     ctx->ldx, ctx->status_d, true, ctx->st);
        return is_f64(ctx) ? launch_dense_to_colmajor<float, double>(
                                 (const float*)dptr, F.rows, ctx->k, ctx->k, (double*)ctx->Xt,
                                 ctx->ldx, ctx->status_d, true, ctx->st)
                           : launch_dense_to_colmajor<float, float>(
                                 (const float*)dptr, F.rows, ctx->k, ctx->k, (float*)ctx->Xt,
                                 ctx->ldx, ctx->status_d, true, ctx->st);
    });
    if (tmp) CU(cudaFreeAsync(tmp, ctx->st));
    if (tmp32) CU(cudaFreeAsync(tmp32, ctx->st));
    TRY(s);
    TRY(check_status(ctx));
    // thresholds that keep every positive entry (U0 is not enforced)
    CU(cudaMemsetAsync(ctx->tau, 0, 8 * (size_t)ctx->k, ctx->st));
    CU(cudaMemsetAsync(ctx->cut, 0xff, 4 * (size_t)ctx->k, ctx->st));
    TRY(do_emit(ctx, F, false, nullptr, false, TOPT_COLUMN));
    F.valid = true;
    return ESPNMF_OK;
}

espnmf_status fail_init(espnmf_ctx* ctx, espnmf_status s)
{
    g_init_error = ctx->err;
    espnmf_destroy(ctx);
    return s;
}

// R/E/f of the current U, V: ||A||^2 - 2 <U, A V> + <U^T U, V^T V>, with
// A V from the last U update when it is still current.
espnmf_status ensure_metrics(espnmf_ctx* ctx)
{
    if (ctx->met_valid) return ESPNMF_OK;
    if (!ctx->Y_is_AV) {
        TRY(do_spmm(ctx, false, ctx->V.buf[ctx->V.cur]));
        ctx->Y_is_AV = true;
    }
    EllDev& u = ctx->U.buf[ctx->U.cur];
    TRY(run(ctx, K_DOT, (double)ctx->n * 4, ctx->st, [&] {
        return is_f64(ctx) ? launch_ell_dot<double>(ctx->n, ctx->k, u, (const double*)ctx->Y, ctx->ldy,
                                                    ctx->norm_part, ctx->sm_count, ctx->dot, ctx->st)
                           : launch_ell_dot<float>(ctx->n, ctx->k, u, (const float*)ctx->Y, ctx->ldy,
                                                   ctx->norm_part, ctx->sm_count, ctx->dot, ctx->st);
    }));
    TRY(run(ctx, K_DOT, 0.0, ctx->st, [&] {
        return launch_error_metrics(ctx->U.G, ctx->V.G, ctx->k, ctx->A2, ctx->dot, ctx->met,
                                    ctx->st);
    }));
    ctx->met_valid = true;
    return ESPNMF_OK;
}

// Y = A V (for U) or A^T U (for V), the sparse product a gradient needs.
espnmf_status ensure_product_for(espnmf_ctx* ctx, espnmf_which which)
{
    if (which == ESPNMF_U) {
        if (!ctx->Y_is_AV) {
            TRY(do_spmm(ctx, false, ctx->V.buf[ctx->V.cur]));
            ctx->Y_is_AV = true;
        }
    } else {
        TRY(do_spmm(ctx, true, ctx->U.buf[ctx->U.cur]));
        ctx->Y_is_AV = false;
    }
    return ESPNMF_OK;
}

// --- checkpoints -------------------------------------------------------------------

// File layout (little-endian): the 8-byte magic, then the header fields in
// the order of CkptHeader, the factors U (n x k) and V (m x k) dense
// row-major in the context's arithmetic, the FP64 Gram matrices U^T U and
// V^T V (k x k each), each factor's last selection thresholds (k 8-byte
// keys each; they decide how the selector groups the Gram diagonal's
// partial sums, so the resumed sums round alike), and an FNV-1a 64-bit
// checksum of everything before it.
constexpr char kCkptMagic[8] = {'E', 'S', 'P', 'N', 'M', 'F', 'C', 'K'};
constexpr uint32_t kCkptVersion = 1;

struct CkptHeader {
    uint32_t version;
    uint32_t dtype;     // ESPNMF_F64 or ESPNMF_F32
    int64_t n, m;
    int32_t k, mode;
    int64_t t_u, t_v;
    int64_t sweeps;
    uint64_t tag;
    uint32_t v_valid;   // V holds a value (at least one V update ran)
    uint32_t reserved;
};

uint64_t fnv1a(uint64_t h, const void* p, size_t bytes)
{
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < bytes; ++i) {
        h ^= b[i];
        h *= 0x100000001b3ull;
    }
    return h;
}

// Factor F as dense row-major bytes in the context's arithmetic (values as
// stored, zeros included).
espnmf_status factor_dense_host(espnmf_ctx* ctx, const Factor& F, std::vector<unsigned char>& out)
{
    const EllDev& E = F.buf[F.cur];
    const int64_t rows = F.rows;
    const int k = ctx->k, ld = E.ld;
    const size_t es = ctx->esz;
    std::vector<int32_t> cnt(rows), col((size_t)rows * ld);
    std::vector<unsigned char> v((size_t)rows * ld * es);
    CU(cudaMemcpy(cnt.data(), E.cnt, 4 * rows, cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(col.data(), E.col, 4 * (size_t)rows * ld, cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(v.data(), E.val, es * (size_t)rows * ld, cudaMemcpyDeviceToHost));
    out.assign((size_t)rows * k * es, 0);
    for (int64_t r = 0; r < rows; ++r)
        for (int q = 0; q < cnt[r]; ++q)
            memcpy(&out[((size_t)r * k + col[(size_t)r * ld + q]) * es], &v[((size_t)r * ld + q) * es], es);
    return ESPNMF_OK;
}

}  // namespace

// =================================================================================
// Public entry points

extern "C" {

const char* espnmf_status_string(espnmf_status s)
{
    switch (s) {
    case ESPNMF_OK: return "ESPNMF_OK";
    case ESPNMF_ERR_INVALID_ARG: return "ESPNMF_ERR_INVALID_ARG";
    case ESPNMF_ERR_BAD_MATRIX: return "ESPNMF_ERR_BAD_MATRIX";
    case ESPNMF_ERR_SINGULAR: return "ESPNMF_ERR_SINGULAR";
    case ESPNMF_ERR_NONFINITE: return "ESPNMF_ERR_NONFINITE";
    case ESPNMF_ERR_OOM: return "ESPNMF_ERR_OOM";
    case ESPNMF_ERR_CUDA: return "ESPNMF_ERR_CUDA";
    case ESPNMF_ERR_TIMEOUT: return "ESPNMF_ERR_TIMEOUT";
    case ESPNMF_ERR_UNSUPPORTED: return "ESPNMF_ERR_UNSUPPORTED";
    }
    return "ESPNMF_ERR_UNKNOWN";
}

const char* espnmf_last_error(const espnmf_ctx* ctx)
{
    return ctx ? ctx->err.c_str() : g_init_error.c_str();
}

espnmf_status espnmf_init(espnmf_ctx** out, const espnmf_csr* A, int32_t k, int64_t t_u,
                          int64_t t_v, espnmf_topt_mode mode, espnmf_dtype compute,
                          const void* U0, espnmf_dtype U0_dtype, int32_t U0_on_device,
                          void* stream)
{
    g_init_error.clear();
    if (!out) return set_err(nullptr, ESPNMF_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!A || !U0) return set_err(nullptr, ESPNMF_ERR_INVALID_ARG, "A or U0 is NULL");
    if (compute == ESPNMF_BF16)
        return set_err(nullptr, ESPNMF_ERR_UNSUPPORTED, "BF16 compute is not implemented");
    if (compute != ESPNMF_F64 && compute != ESPNMF_F32)
        return set_err(nullptr, ESPNMF_ERR_INVALID_ARG, "compute must be F64 or F32");
    if (A->n < 1 || A->m < 1 || A->nnz < 0)
        return set_err(nullptr, ESPNMF_ERR_INVALID_ARG, "A must have n >= 1, m >= 1, nnz >= 0");
    if (A->n >= (1ll << 31) || A->m >= (1ll << 31))
        return set_err(nullptr, ESPNMF_ERR_INVALID_ARG, "n and m must be < 2^31");
    if (k < 1 || k > 128 || k > A->n || k > A->m)
        return set_err(nullptr, ESPNMF_ERR_INVALID_ARG, "k must satisfy 1 <= k <= min(n, m, 128)");
    if (t_u < 0 || t_v < 0) return set_err(nullptr, ESPNMF_ERR_INVALID_ARG, "t must be >= 0");
    if (mode != ESPNMF_TOPT_COLUMN && mode != ESPNMF_TOPT_MATRIX && mode != ESPNMF_TOPT_NONE)
        return set_err(nullptr, ESPNMF_ERR_INVALID_ARG, "unknown enforcement mode");
    if (mode == ESPNMF_TOPT_MATRIX &&
        ((int64_t)k * A->n >= (1ll << 31) || (int64_t)k * A->m >= (1ll << 31)))
        return set_err(nullptr, ESPNMF_ERR_INVALID_ARG, "matrix mode needs rows*k < 2^31");
    if (A->vdtype != ESPNMF_F64 && A->vdtype != ESPNMF_F32 && A->vdtype != ESPNMF_BF16)
        return set_err(nullptr, ESPNMF_ERR_INVALID_ARG, "A values must be F64, F32 or BF16");
    if (U0_dtype != ESPNMF_F64 && U0_dtype != ESPNMF_F32 && U0_dtype != ESPNMF_BF16)
        return set_err(nullptr, ESPNMF_ERR_INVALID_ARG, "U0 dtype must be F64, F32 or BF16");
    if (A->nnz > 0 && (!A->rowptr || !A->colidx || !A->values))
        return set_err(nullptr, ESPNMF_ERR_INVALID_ARG, "A arrays are NULL");

    espnmf_ctx* ctx = new (std::nothrow) espnmf_ctx();
    if (!ctx) return set_err(nullptr, ESPNMF_ERR_OOM, "host allocation failed");
    ctx->n = A->n;
    ctx->m = A->m;
    ctx->nnz = A->nnz;
    ctx->k = k;
    ctx->t_u = t_u;
    ctx->t_v = t_v;
    ctx->mode = (int)mode;
    ctx->dt = compute;
    ctx->esz = compute == ESPNMF_F64 ? 8 : 4;
    {
        cudaError_t e = cudaGetDevice(&ctx->device);
        if (e == cudaSuccess)
            e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, ctx->device);
        if (e != cudaSuccess) {
            set_err(ctx, ESPNMF_ERR_CUDA, "no usable CUDA device: %s", cudaGetErrorString(e));
            cudaGetLastError();
            return fail_init(ctx, ESPNMF_ERR_CUDA);
        }
    }
    // ESPNMF_TRACE_INIT set: the host time of each phase of the set-up on
    // stderr (the device work of a phase is not waited for)
    const bool trace = std::getenv("ESPNMF_TRACE_INIT") != nullptr;
    auto t_last = std::chrono::steady_clock::now();
    auto phase = [&](const char* what) {
        if (!trace) return;
        const auto now = std::chrono::steady_clock::now();
        std::fprintf(stderr, "espnmf_init: %-28s %8.2f ms\n", what,
                     std::chrono::duration<double, std::milli>(now - t_last).count());
        t_last = now;
    };
    espnmf_status s = [&]() -> espnmf_status {
        if (stream) {
            ctx->st = (cudaStream_t)stream;
        } else {
            CU(cudaStreamCreateWithFlags(&ctx->st, cudaStreamNonBlocking));
            ctx->own_stream = true;
        }
        // the Gram inverse on the auxiliary stream must not queue behind the
        // concurrent SpMM's blocks: give the stream the highest priority
        int prio_lo = 0, prio_hi = 0;
        CU(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
        CU(cudaStreamCreateWithPriority(&ctx->aux, cudaStreamNonBlocking, prio_hi));
        CU(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
        CU(cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming));
        CU(setup_spmm());
        CU(setup_solve());
        CU(setup_select());
        CU(setup_factor());
        CU(setup_chol());

        phase("streams, kernel attributes");
        // ---- A: validate and build both layouts on host threads.  A on the
        // device is first copied to the host; host arrays are read in place.
        const int64_t n = A->n, m = A->m, nnz = A->nnz;
        const size_t vsz = A->vdtype == ESPNMF_F64 ? 8 : A->vdtype == ESPNMF_F32 ? 4 : 2;
        std::vector<int64_t> rp_h;
        hvec<int32_t> ci_h;
        hvec<unsigned char> vraw_h;
        const int64_t* rp = nullptr;
        const int32_t* ci = nullptr;
        const unsigned char* vraw = nullptr;
        if (A->on_device) {
            rp_h.resize(n + 1);
            ci_h.resize(nnz);
            vraw_h.resize(nnz * vsz);
            CU(cudaMemcpy(rp_h.data(), A->rowptr, (n + 1) * 8, cudaMemcpyDeviceToHost));
            if (nnz) {
                CU(cudaMemcpy(ci_h.data(), A->colidx, nnz * 4, cudaMemcpyDeviceToHost));
                CU(cudaMemcpy(vraw_h.data(), A->values, nnz * vsz, cudaMemcpyDeviceToHost));
            }
            rp = rp_h.data();
            ci = ci_h.data();
            vraw = vraw_h.data();
        } else {
            if (!A->rowptr) return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "rowptr is NULL");
            rp = A->rowptr;
            ci = A->colidx;
            vraw = static_cast<const unsigned char*>(A->values);
        }
        // A's values: in the FP32 form FP32 or BF16 ones are kept in FP32
        // (FP32 ones read in place), otherwise they are widened to FP64;
        // both exact, and every layout rounds them the same way
        const bool vals32 = compute != ESPNMF_F64 && vsz <= 4;
        hvec<double> vv;
        hvec<float> vf_h;
        const float* vf = nullptr;
        if (vals32 && vsz == 4 && reinterpret_cast<uintptr_t>(vraw) % alignof(float) == 0) {
            vf = reinterpret_cast<const float*>(vraw);
        } else if (vals32) {
            vf_h.resize(nnz);
            parallel_chunks(nnz, [&](int64_t p0, int64_t p1) {
                for (int64_t p = p0; p < p1; ++p) {
                    float f;
                    if (vsz == 4) {
                        memcpy(&f, vraw + p * 4, 4);
                    } else {
                        // BF16: the high half of the FP32 word
                        uint16_t b;
                        memcpy(&b, vraw + p * 2, 2);
                        const uint32_t w = (uint32_t)b << 16;
                        memcpy(&f, &w, 4);
                    }
                    vf_h[p] = f;
                }
            });
            vf = vf_h.data();
        } else {
            vv.resize(nnz);
            parallel_chunks(nnz, [&](int64_t p0, int64_t p1) {
                for (int64_t p = p0; p < p1; ++p) {
                    double x;
                    if (vsz == 8) {
                        memcpy(&x, vraw + p * 8, 8);
                    } else if (vsz == 4) {
                        float f;
                        memcpy(&f, vraw + p * 4, 4);
                        x = f;
                    } else {
                        // BF16: the high half of the FP32 word (exact)
                        uint16_t b;
                        memcpy(&b, vraw + p * 2, 2);
                        const uint32_t w = (uint32_t)b << 16;
                        float f;
                        memcpy(&f, &w, 4);
                        x = f;
                    }
                    vv[p] = x;
                }
            });
        }
        if (rp[0] != 0 || rp[n] != nnz)
            return set_err(ctx, ESPNMF_ERR_BAD_MATRIX, "rowptr must run from 0 to nnz");
        for (int64_t r = 0; r < n; ++r)
            if (rp[r + 1] < rp[r]) return set_err(ctx, ESPNMF_ERR_BAD_MATRIX, "rowptr decreases at row %lld", (long long)r);
        {
            // rows checked in chunks on host threads; the first bad row
            // (lowest index) is reported
            std::mutex bad_mu;
            int64_t bad_row = n;
            int bad_kind = 0;
            auto check = [&](const auto* vals) {
                parallel_weighted(n, rp, [&](int64_t r0, int64_t r1) {
                    for (int64_t r = r0; r < r1; ++r) {
                        int kind = 0;
                        for (int64_t p = rp[r]; p < rp[r + 1] && !kind; ++p) {
                            const double x = (double)vals[p];
                            if (ci[p] < 0 || ci[p] >= m) kind = 1;
                            else if (p > rp[r] && ci[p] <= ci[p - 1]) kind = 2;
                            else if (!std::isfinite(x)) kind = 3;
                            else if (x < 0.0) kind = 4;
                        }
                        if (kind) {
                            std::lock_guard<std::mutex> lock(bad_mu);
                            if (r < bad_row) {
                                bad_row = r;
                                bad_kind = kind;
                            }
                            return;
                        }
                    }
                });
            };
            if (vf) check(vf);
            else check(vv.data());
            static const char* what[] = {"", "column index out of range", "column indices not strictly increasing",
                                         "non-finite value", "negative value (A >= 0 is required)"};
            if (bad_kind)
                return set_err(ctx, ESPNMF_ERR_BAD_MATRIX, "%s in row %lld", what[bad_kind], (long long)bad_row);
        }
        phase("copy, convert, validate A");
        // CSC (= CSR of A^T), rows ascending inside each column
        std::vector<int64_t> cp;
        hvec<int32_t> ri;
        hvec<double> cv;     // FP64 form
        hvec<float> cv32;    // FP32 form: the values as its layouts store them
        if (compute == ESPNMF_F64) transpose_csr(n, m, rp, ci, vv.data(), cp, ri, cv);
        else if (vf) transpose_csr(n, m, rp, ci, vf, cp, ri, cv32);
        else transpose_csr(n, m, rp, ci, vv.data(), cp, ri, cv32);
        phase("transpose");
        // The two orientations are laid out on two host threads; the uploads
        // follow on this thread.
        if (compute == ESPNMF_F64) {
            SellHost<double> h1, h2;
            std::thread th([&] {
                t_share = 2;
                build_sell(m, cp.data(), ri.data(), cv.data(), h2);
            });
            t_share = 2;
            build_sell(n, rp, ci, vv.data(), h1);
            t_share = 1;
            th.join();
            TRY(upload_sell(ctx, h1, ctx->sA));
            TRY(upload_sell(ctx, h2, ctx->sAt));
        } else {
            const int ld = factor_ld(k);
            // chunks of the frequent part's rows: four per warp of spmm_freq
            const int nchunks = 4 * ctx->sm_count * (kHThreads / 32);
            const bool col_mode = mode == ESPNMF_TOPT_COLUMN;
            const int64_t tu = col_mode ? t_u : 0, tv = col_mode ? t_v : 0;
            auto upload_f32 = [&](const BuiltF32& B, SellDev& D) -> espnmf_status {
                TRY(upload_sell(ctx, B.h, D));
                if (B.F.h > 0) TRY(upload_frequent(ctx, B.F, D));
                return ESPNMF_OK;
            };
            BuiltF32 ba, bat;
            if (vf)
                build_layouts_f32(n, m, rp, ci, vf, cp.data(), ri.data(), cv32.data(), ld, nchunks,
                                  tu, tv, ba, bat);
            else
                build_layouts_f32(n, m, rp, ci, vv.data(), cp.data(), ri.data(), cv32.data(), ld,
                                  nchunks, tu, tv, ba, bat);
            phase("layouts built");
            TRY(upload_f32(ba, ctx->sA));
            TRY(upload_f32(bat, ctx->sAt));
        }

        phase("layouts uploaded");
        // ---- work buffers
        const int64_t rmax = std::max(n, m);
        ctx->ldy = factor_ld(k);
        ctx->ldx = (rmax + 31) / 32 * 32;
        TRY(dmalloc(ctx, &ctx->Y, (size_t)rmax * ctx->ldy * ctx->esz));
        TRY(dmalloc(ctx, &ctx->Xt, (size_t)k * ctx->ldx * ctx->esz));
        CU(cudaMemsetAsync(ctx->Xt, 0, (size_t)k * ctx->ldx * ctx->esz, ctx->st));
        ctx->fin_blocks = 2 * ctx->sm_count;
        {
            // partials: emit blocks (and the frequent table's), upper triangle
            const size_t ntri = (size_t)k * (k + 1) / 2;
            const size_t parts = std::max((size_t)ctx->fin_blocks * k * k,
                                          (size_t)(ctx->fin_blocks + ctx->sm_count) * ntri);
            TRY(dmalloc(ctx, &ctx->gram_part, sizeof(double) * parts));
        }
        if (!is_f64(ctx)) {
            const size_t words = (size_t)rmax * ((k + 31) / 32);
            TRY(dmalloc(ctx, &ctx->rowbits, 4 * words));
            CU(cudaMemsetAsync(ctx->rowbits, 0, 4 * words, ctx->st));
            TRY(dmalloc(ctx, &ctx->sel_counts, 2 * sizeof(unsigned long long)));
            CU(cudaMemsetAsync(ctx->sel_counts, 0, 2 * sizeof(unsigned long long), ctx->st));
            TRY(dmalloc(ctx, &ctx->diag_part, sizeof(double) * k * 8));
        }
        TRY(dmalloc(ctx, &ctx->scal_part, sizeof(double) * ctx->fin_blocks * 4));
        TRY(dmalloc(ctx, &ctx->scal, sizeof(double) * 4));
        TRY(dmalloc(ctx, &ctx->gram_counter, sizeof(unsigned)));
        CU(cudaMemsetAsync(ctx->gram_counter, 0, sizeof(unsigned), ctx->st));
        TRY(dmalloc(ctx, &ctx->A2, sizeof(double)));
        TRY(dmalloc(ctx, &ctx->norm_part, sizeof(double) * ctx->sm_count));
        TRY(dmalloc(ctx, &ctx->met, sizeof(double) * 4));
        CU(cudaMemsetAsync(ctx->met, 0, sizeof(double) * 4, ctx->st));
        TRY(dmalloc(ctx, &ctx->dot, sizeof(double)));
        TRY(dmalloc(ctx, &ctx->pg, 2 * sizeof(double)));
        TRY(dmalloc(ctx, &ctx->tau, 8 * (size_t)k));
        TRY(dmalloc(ctx, &ctx->cut, 4 * (size_t)k));
        TRY(dmalloc(ctx, &ctx->hist_counter, sizeof(int)));
        CU(cudaMemsetAsync(ctx->hist_counter, 0, sizeof(int), ctx->st));
        TRY(ensure_hist(ctx, 64));
        TRY(dmalloc(ctx, &ctx->status_d, sizeof(unsigned)));
        CU(cudaMemsetAsync(ctx->status_d, 0, sizeof(unsigned), ctx->st));
        CU(cudaMallocHost(&ctx->status_h, sizeof(unsigned)));

        phase("work buffers");
        for (Factor* F : {&ctx->U, &ctx->V}) {
            F->rows = F == &ctx->U ? n : m;
            const int ld = factor_ld(k);
            const int dld = dense_ld(ld);
            void* dense = nullptr;
            TRY(dmalloc(ctx, &dense, ctx->esz * F->rows * dld));
            // one dense copy and one record array per factor, rewritten by
            // each emit (the emit writes every row's record)
            uint4* rec = nullptr;
            uint32_t* nzmask = nullptr;
            void* htab = nullptr;
            uint8_t* hnz = nullptr;
            // the product that gathers this factor: A^T U gathers U, A V gathers V
            const SellDev& Gp = F == &ctx->U ? ctx->sAt : ctx->sA;
            if (!is_f64(ctx)) {
                TRY(dmalloc(ctx, &F->sel_hint, 8 * (size_t)k));
                CU(cudaMemsetAsync(F->sel_hint, 0, 8 * (size_t)k, ctx->st));
                TRY(dmalloc(ctx, &rec, 2 * sizeof(uint4) * F->rows));
                CU(cudaMemsetAsync(rec, 0, 2 * sizeof(uint4) * F->rows, ctx->st));
                const size_t words = (size_t)(F->rows + 31) / 32;
                TRY(dmalloc(ctx, &nzmask, 4 * words));
                CU(cudaMemsetAsync(nzmask, 0, 4 * words, ctx->st));
                if (Gp.h > 0) {
                    // the h table rows and a zero row (read by the second tier)
                    TRY(dmalloc(ctx, &htab, ((size_t)Gp.h + 1) * ld * 4));
                    CU(cudaMemsetAsync(htab, 0, ((size_t)Gp.h + 1) * ld * 4, ctx->st));
                    TRY(dmalloc(ctx, &hnz, (size_t)Gp.h));
                    CU(cudaMemsetAsync(hnz, 0, (size_t)Gp.h, ctx->st));
                }
            }
            for (int b = 0; b < 2; ++b) {
                TRY(dmalloc(ctx, &F->buf[b].cnt, sizeof(int32_t) * F->rows));
                TRY(dmalloc(ctx, &F->buf[b].col, sizeof(int32_t) * F->rows * ld));
                TRY(dmalloc(ctx, &F->buf[b].val, ctx->esz * F->rows * ld));
                CU(cudaMemsetAsync(F->buf[b].cnt, 0, sizeof(int32_t) * F->rows, ctx->st));
                F->buf[b].dense = dense;
                F->buf[b].rec = rec;
                F->buf[b].nzmask = nzmask;
                F->buf[b].hslot = Gp.h > 0 ? Gp.slot_of : nullptr;
                F->buf[b].htab = htab;
                F->buf[b].hnz = hnz;
                F->buf[b].h = htab ? Gp.h : 0;
                F->buf[b].ld = ld;
                F->buf[b].rows = F->rows;
                F->buf[b].dld = dld;
                F->buf[b].heavy = heavy_threshold(ld);
            }
            TRY(dmalloc(ctx, &F->G, sizeof(double) * k * k));
            CU(cudaMemsetAsync(F->G, 0, sizeof(double) * k * k, ctx->st));
            TRY(dmalloc(ctx, &F->Ginv64, sizeof(double) * k * k));
            TRY(dmalloc(ctx, &F->GinvT, ctx->esz * k * k));
            if (use_cholesky(ctx)) {
                // L, L^T, 1 / diag, then G's FP32 pair (hi, lo)
                const size_t lf = (size_t)4 * ctx->ldy * ctx->ldy + ctx->ldy;
                TRY(dmalloc(ctx, &F->Lf, sizeof(float) * lf));
                CU(cudaMemsetAsync(F->Lf, 0, sizeof(float) * lf, ctx->st));
            }
        }

        phase("factor buffers");
        // ---- ||A||^2 from the values the kernels use
        if (is_f64(ctx))
            TRY(run(ctx, K_NORM2, (double)ctx->sA.total * 8, ctx->st, [&] {
                return launch_norm2<double>((const double*)ctx->sA.val, ctx->sA.total, nullptr, 0,
                                            nullptr, 0, ctx->norm_part, ctx->sm_count, ctx->A2,
                                            ctx->st);
            }));
        else
            TRY(run(ctx, K_NORM2, (double)ctx->sA.total * 4, ctx->st, [&] {
                // the SELL part's values and both tiers of the frequent part
                return launch_norm2<float>((const float*)ctx->sA.val, ctx->sA.total,
                                           ctx->sA.ft[0].ent, ctx->sA.ft[0].nent,
                                           ctx->sA.ft[1].ent, ctx->sA.ft[1].nent,
                                           ctx->norm_part, ctx->sm_count, ctx->A2, ctx->st);
            }));

        // ---- U = U0 (Alg. 2 START; not enforced)
        TRY(set_factor_impl(ctx, ctx->U, U0, U0_dtype, U0_on_device));
        TRY(check_status(ctx));
        phase("norm, U0, synchronise");
        return ESPNMF_OK;
    }();
    if (s != ESPNMF_OK) return fail_init(ctx, s);
    *out = ctx;
    return ESPNMF_OK;
}

espnmf_status espnmf_destroy(espnmf_ctx* ctx)
{
    if (!ctx) return ESPNMF_OK;
    cudaSetDevice(ctx->device);
    if (ctx->st) cudaStreamSynchronize(ctx->st);
    if (ctx->aux) cudaStreamSynchronize(ctx->aux);
    drop_graphs(ctx);
    for (auto& r : ctx->pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : ctx->ev_pool) cudaEventDestroy(e);
    for (void* p : ctx->allocs) cudaFree(p);
    if (ctx->status_h) cudaFreeHost(ctx->status_h);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    if (ctx->aux) cudaStreamDestroy(ctx->aux);
    if (ctx->own_stream && ctx->st) cudaStreamDestroy(ctx->st);
    cudaGetLastError();
    delete ctx;
    return ESPNMF_OK;
}

espnmf_status espnmf_als_update_V(espnmf_ctx* ctx)
{
    TRY(enter(ctx));
    ctx->launches_this = 0;
    return half_update(ctx, true);
}

espnmf_status espnmf_als_update_U(espnmf_ctx* ctx)
{
    TRY(enter(ctx));
    if (!ctx->V.valid)
        return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "V has no value yet: update V (or set it) first");
    ctx->launches_this = 0;
    return half_update(ctx, false);
}

espnmf_status espnmf_iterate(espnmf_ctx* ctx, int32_t iters, double* R_out, double* E_out)
{
    TRY(enter(ctx));
    if (iters < 0) return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "iters must be >= 0");
    if (iters == 0) return ESPNMF_OK;
    TRY(ensure_hist(ctx, iters));
    CU(cudaMemsetAsync(ctx->hist_counter, 0, sizeof(int), ctx->st));
    int it = 0;
    // the first sweep from U0 runs eagerly: V does not exist before it
    if (!ctx->V.valid || !ctx->use_graph || ctx->profile) {
        TRY(enqueue_sweep(ctx));
        ++it;
    }
    if (ctx->use_graph && !ctx->profile) {
        if (it < iters && ctx->spmm_tune && !ctx->spmm_tuned) TRY(tune_spmm(ctx));
        for (; it < iters; ++it) {
            cudaGraphExec_t& g = ctx->gexec[ctx->U.cur][ctx->V.cur];
            if (!g) TRY(sweep_graph(ctx, &g));
            CU(cudaGraphLaunch(g, ctx->st));
            after_sweep_state(ctx);
        }
    } else {
        for (; it < iters; ++it) TRY(enqueue_sweep(ctx));
    }
    if (R_out || E_out) {
        TRY(check_status(ctx));
        if (R_out) CU(cudaMemcpy(R_out, ctx->hist_R, sizeof(double) * iters, cudaMemcpyDeviceToHost));
        if (E_out) CU(cudaMemcpy(E_out, ctx->hist_E, sizeof(double) * iters, cudaMemcpyDeviceToHost));
    }
    return ESPNMF_OK;
}

espnmf_status espnmf_enforce_topt(espnmf_ctx* ctx, espnmf_which which, int64_t t)
{
    TRY(enter(ctx));
    if (which != ESPNMF_U && which != ESPNMF_V) return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "which");
    if (t < 0) return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "t must be >= 0");
    Factor& F = which == ESPNMF_U ? ctx->U : ctx->V;
    if (!F.valid) return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "factor has no value yet");
    EllDev& cur = F.buf[F.cur];
    TRY(run(ctx, K_SCATTER, (double)F.rows * ctx->k * ctx->esz, ctx->st, [&] {
        return is_f64(ctx) ? launch_ell_to_colmajor<double>(F.rows, ctx->k, cur, (double*)ctx->Xt, ctx->ldx, ctx->st)
                           : launch_ell_to_colmajor<float>(F.rows, ctx->k, cur, (float*)ctx->Xt, ctx->ldx, ctx->st);
    }));
    TRY(do_select(ctx, F.rows, t, false, nullptr));
    TRY(do_emit(ctx, F, false, nullptr, false, ctx->mode));
    ctx->met_valid = false;
    if (which == ESPNMF_V) ctx->Y_is_AV = false;
    return check_status(ctx);
}

espnmf_status espnmf_set_factor(espnmf_ctx* ctx, espnmf_which which, const void* F,
                                espnmf_dtype dtype, int32_t on_device)
{
    TRY(enter(ctx));
    if (which != ESPNMF_U && which != ESPNMF_V) return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "which");
    Factor& Fa = which == ESPNMF_U ? ctx->U : ctx->V;
    TRY(set_factor_impl(ctx, Fa, F, dtype, on_device));
    ctx->met_valid = false;
    if (which == ESPNMF_V) ctx->Y_is_AV = false;
    else ctx->have_R = false;
    return check_status(ctx);
}

espnmf_status espnmf_save(espnmf_ctx* ctx, const char* path, uint64_t tag)
{
    TRY(enter(ctx));
    if (!path) return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "path is NULL");
    if (!ctx->U.valid) return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "U has no value");
    TRY(check_status(ctx));
    CkptHeader h = {};
    h.version = kCkptVersion;
    h.dtype = (uint32_t)ctx->dt;
    h.n = ctx->n;
    h.m = ctx->m;
    h.k = ctx->k;
    h.mode = ctx->mode;
    h.t_u = ctx->t_u;
    h.t_v = ctx->t_v;
    h.sweeps = ctx->sweeps;
    h.tag = tag;
    h.v_valid = ctx->V.valid ? 1u : 0u;
    std::vector<unsigned char> Ub, Vb;
    TRY(factor_dense_host(ctx, ctx->U, Ub));
    if (ctx->V.valid) TRY(factor_dense_host(ctx, ctx->V, Vb));
    else Vb.assign((size_t)ctx->m * ctx->k * ctx->esz, 0);
    const size_t kk = (size_t)ctx->k * ctx->k;
    std::vector<double> GU(kk), GV(kk, 0.0);
    CU(cudaMemcpy(GU.data(), ctx->U.G, 8 * kk, cudaMemcpyDeviceToHost));
    if (ctx->V.valid) CU(cudaMemcpy(GV.data(), ctx->V.G, 8 * kk, cudaMemcpyDeviceToHost));
    std::vector<uint64_t> HU(ctx->k, 0), HV(ctx->k, 0);
    if (ctx->U.sel_hint) CU(cudaMemcpy(HU.data(), ctx->U.sel_hint, 8 * (size_t)ctx->k, cudaMemcpyDeviceToHost));
    if (ctx->V.sel_hint) CU(cudaMemcpy(HV.data(), ctx->V.sel_hint, 8 * (size_t)ctx->k, cudaMemcpyDeviceToHost));
    uint64_t sum = 0xcbf29ce484222325ull;
    sum = fnv1a(sum, kCkptMagic, sizeof kCkptMagic);
    sum = fnv1a(sum, &h, sizeof h);
    sum = fnv1a(sum, Ub.data(), Ub.size());
    sum = fnv1a(sum, Vb.data(), Vb.size());
    sum = fnv1a(sum, GU.data(), 8 * kk);
    sum = fnv1a(sum, GV.data(), 8 * kk);
    sum = fnv1a(sum, HU.data(), 8 * HU.size());
    sum = fnv1a(sum, HV.data(), 8 * HV.size());
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = fopen(tmp.c_str(), "wb");
    if (!f) return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "cannot open %s for writing", tmp.c_str());
    bool ok = fwrite(kCkptMagic, sizeof kCkptMagic, 1, f) == 1 && fwrite(&h, sizeof h, 1, f) == 1 &&
              fwrite(Ub.data(), 1, Ub.size(), f) == Ub.size() &&
              fwrite(Vb.data(), 1, Vb.size(), f) == Vb.size() &&
              fwrite(GU.data(), 8, kk, f) == kk && fwrite(GV.data(), 8, kk, f) == kk &&
              fwrite(HU.data(), 8, HU.size(), f) == HU.size() &&
              fwrite(HV.data(), 8, HV.size(), f) == HV.size() &&
              fwrite(&sum, sizeof sum, 1, f) == 1;
    ok = (fclose(f) == 0) && ok;
    if (!ok || rename(tmp.c_str(), path) != 0) {
        remove(tmp.c_str());
        return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "writing %s failed", path);
    }
    return ESPNMF_OK;
}

espnmf_status espnmf_load(espnmf_ctx* ctx, const char* path, uint64_t* tag, int64_t* sweeps)
{
    TRY(enter(ctx));
    if (!path) return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "path is NULL");
    FILE* f = fopen(path, "rb");
    if (!f) return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "cannot open %s", path);
    char magic[8] = {};
    CkptHeader h = {};
    const bool head_ok = fread(magic, sizeof magic, 1, f) == 1 && fread(&h, sizeof h, 1, f) == 1 &&
                         memcmp(magic, kCkptMagic, sizeof magic) == 0;
    auto bad = [&](const char* why) {
        fclose(f);
        return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "%s: %s", path, why);
    };
    if (!head_ok) return bad("not a checkpoint of this library");
    if (h.version != kCkptVersion) return bad("unsupported checkpoint version");
    if (h.dtype != (uint32_t)ctx->dt || h.n != ctx->n || h.m != ctx->m || h.k != ctx->k ||
        h.mode != ctx->mode || h.t_u != ctx->t_u || h.t_v != ctx->t_v)
        return bad("saved by a context of another shape, mode, t or arithmetic");
    const size_t es = ctx->esz, kk = (size_t)ctx->k * ctx->k;
    std::vector<unsigned char> Ub((size_t)h.n * h.k * es), Vb((size_t)h.m * h.k * es);
    std::vector<double> GU(kk), GV(kk);
    std::vector<uint64_t> HU(ctx->k), HV(ctx->k);
    uint64_t stored = 0;
    const bool body_ok = fread(Ub.data(), 1, Ub.size(), f) == Ub.size() &&
                         fread(Vb.data(), 1, Vb.size(), f) == Vb.size() &&
                         fread(GU.data(), 8, kk, f) == kk && fread(GV.data(), 8, kk, f) == kk &&
                         fread(HU.data(), 8, HU.size(), f) == HU.size() &&
                         fread(HV.data(), 8, HV.size(), f) == HV.size() &&
                         fread(&stored, sizeof stored, 1, f) == 1;
    if (!body_ok) return bad("truncated");
    fclose(f);
    uint64_t sum = 0xcbf29ce484222325ull;
    sum = fnv1a(sum, kCkptMagic, sizeof kCkptMagic);
    sum = fnv1a(sum, &h, sizeof h);
    sum = fnv1a(sum, Ub.data(), Ub.size());
    sum = fnv1a(sum, Vb.data(), Vb.size());
    sum = fnv1a(sum, GU.data(), 8 * kk);
    sum = fnv1a(sum, GV.data(), 8 * kk);
    sum = fnv1a(sum, HU.data(), 8 * HU.size());
    sum = fnv1a(sum, HV.data(), 8 * HV.size());
    if (sum != stored) return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "%s: checksum mismatch", path);
    // the factors as stored (their Grams are then replaced by the saved
    // ones, so that the next sweep repeats the uninterrupted run exactly)
    drop_graphs(ctx);
    TRY(set_factor_impl(ctx, ctx->U, Ub.data(), ctx->dt, 0));
    if (h.v_valid) TRY(set_factor_impl(ctx, ctx->V, Vb.data(), ctx->dt, 0));
    CU(cudaMemcpyAsync(ctx->U.G, GU.data(), 8 * kk, cudaMemcpyHostToDevice, ctx->st));
    if (h.v_valid) CU(cudaMemcpyAsync(ctx->V.G, GV.data(), 8 * kk, cudaMemcpyHostToDevice, ctx->st));
    if (ctx->U.sel_hint)
        CU(cudaMemcpyAsync(ctx->U.sel_hint, HU.data(), 8 * HU.size(), cudaMemcpyHostToDevice, ctx->st));
    if (ctx->V.sel_hint)
        CU(cudaMemcpyAsync(ctx->V.sel_hint, HV.data(), 8 * HV.size(), cudaMemcpyHostToDevice, ctx->st));
    CU(cudaStreamSynchronize(ctx->st));
    ctx->V.valid = h.v_valid != 0;
    ctx->met_valid = false;
    ctx->Y_is_AV = false;
    ctx->have_R = false;
    ctx->sweeps = h.sweeps;
    if (tag) *tag = h.tag;
    if (sweeps) *sweeps = h.sweeps;
    return check_status(ctx);
}

espnmf_status espnmf_topic_accuracy(espnmf_ctx* ctx, espnmf_which which, const int32_t* labels,
                                    int32_t n_classes, int32_t on_device, double* acc)
{
    TRY(enter(ctx));
    if (which != ESPNMF_U && which != ESPNMF_V) return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "which");
    if (!labels || !acc || n_classes < 1)
        return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "labels/acc NULL or n_classes < 1");
    Factor& F = which == ESPNMF_U ? ctx->U : ctx->V;
    if (!F.valid) return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "factor has no value yet");
    TRY(check_status(ctx));
    const size_t bl = ((size_t)F.rows * 4 + 255) & ~(size_t)255;
    const size_t bh = ((size_t)ctx->k * n_classes * 4 + 255) & ~(size_t)255;
    unsigned char* ws = nullptr;
    CU(cudaMallocAsync((void**)&ws, bl + bh + 8 * (size_t)ctx->k + 256, ctx->st));
    const int32_t* lab = labels;
    cudaError_t e = cudaSuccess;
    if (!on_device) {
        e = cudaMemcpyAsync(ws, labels, 4 * (size_t)F.rows, cudaMemcpyHostToDevice, ctx->st);
        lab = reinterpret_cast<const int32_t*>(ws);
    }
    double* acc_d = reinterpret_cast<double*>(ws + bl + bh);
    if (e == cudaSuccess)
        e = launch_topic_accuracy(F.buf[F.cur], ctx->k, lab, n_classes,
                                  reinterpret_cast<unsigned*>(ws + bl), acc_d, ctx->status_d,
                                  ctx->sm_count, ctx->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(acc, acc_d, 8 * (size_t)ctx->k, cudaMemcpyDeviceToHost, ctx->st);
    cudaError_t e2 = cudaFreeAsync(ws, ctx->st);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_err(ctx, ESPNMF_ERR_CUDA, "topic accuracy: %s", cudaGetErrorString(e));
    }
    unsigned hs = 0;
    CU(cudaMemcpy(&hs, ctx->status_d, sizeof hs, cudaMemcpyDeviceToHost));
    if (hs & ST_BADINPUT) {
        CU(cudaMemset(ctx->status_d, 0, sizeof(unsigned)));
        return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "a member row's label is outside [0, n_classes)");
    }
    return check_status(ctx);
}

espnmf_status espnmf_sweeps_done(espnmf_ctx* ctx, int64_t* sweeps)
{
    TRY(enter(ctx));
    if (sweeps) *sweeps = ctx->sweeps;
    return ESPNMF_OK;
}

espnmf_status espnmf_residual(espnmf_ctx* ctx, double* R)
{
    TRY(enter(ctx));
    if (!R) return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "R is NULL");
    if (!ctx->have_R) return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "no U update has run");
    TRY(check_status(ctx));
    CU(cudaMemcpy(R, ctx->met, sizeof(double), cudaMemcpyDeviceToHost));
    return ESPNMF_OK;
}

espnmf_status espnmf_error(espnmf_ctx* ctx, double* E)
{
    TRY(enter(ctx));
    if (!E) return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "E is NULL");
    if (!ctx->V.valid) return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "V has no value yet");
    TRY(ensure_metrics(ctx));
    TRY(check_status(ctx));
    CU(cudaMemcpy(E, ctx->met + 1, sizeof(double), cudaMemcpyDeviceToHost));
    return ESPNMF_OK;
}

espnmf_status espnmf_loss(espnmf_ctx* ctx, double* f)
{
    TRY(enter(ctx));
    if (!f) return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "f is NULL");
    if (!ctx->V.valid) return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "V has no value yet");
    TRY(ensure_metrics(ctx));
    TRY(check_status(ctx));
    CU(cudaMemcpy(f, ctx->met + 2, sizeof(double), cudaMemcpyDeviceToHost));
    return ESPNMF_OK;
}

espnmf_status espnmf_grad(espnmf_ctx* ctx, espnmf_which which, void* out, espnmf_dtype dtype,
                          int32_t on_device)
{
    TRY(enter(ctx));
    if (which != ESPNMF_U && which != ESPNMF_V) return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "which");
    if (!out) return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "out is NULL");
    if (dtype != ESPNMF_F64 && dtype != ESPNMF_F32)
        return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "dtype must be F64 or F32");
    if (!ctx->U.valid || !ctx->V.valid)
        return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "U and V need values");
    Factor& F = which == ESPNMF_U ? ctx->U : ctx->V;
    Factor& O = which == ESPNMF_U ? ctx->V : ctx->U;
    TRY(ensure_product_for(ctx, which));
    const size_t es = dtype == ESPNMF_F64 ? 8 : 4;
    const size_t bytes = (size_t)F.rows * ctx->k * es;
    void* dst = out;
    if (!on_device) CU(cudaMallocAsync(&dst, bytes ? bytes : 16, ctx->st));
    const EllDev& fe = F.buf[F.cur];
    const espnmf_status s = run(ctx, K_GRAD, (double)bytes + (double)F.rows * ctx->ldy * ctx->esz,
                                ctx->st, [&]() -> cudaError_t {
        if (is_f64(ctx))
            return dtype == ESPNMF_F64
                       ? launch_grad<double, double>(F.rows, ctx->k, fe, O.G, (const double*)ctx->Y,
                                                     ctx->ldy, (double*)dst, ctx->st)
                       : launch_grad<double, float>(F.rows, ctx->k, fe, O.G, (const double*)ctx->Y,
                                                    ctx->ldy, (float*)dst, ctx->st);
        return dtype == ESPNMF_F64
                   ? launch_grad<float, double>(F.rows, ctx->k, fe, O.G, (const float*)ctx->Y,
                                                ctx->ldy, (double*)dst, ctx->st)
                   : launch_grad<float, float>(F.rows, ctx->k, fe, O.G, (const float*)ctx->Y,
                                               ctx->ldy, (float*)dst, ctx->st);
    });
    if (!on_device) {
        cudaError_t e = s == ESPNMF_OK ? cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, ctx->st)
                                       : cudaSuccess;
        cudaError_t e2 = cudaFreeAsync(dst, ctx->st);
        TRY(s);
        CU(e);
        CU(e2);
    }
    TRY(s);
    return check_status(ctx);
}

espnmf_status espnmf_pg_step(espnmf_ctx* ctx, espnmf_which which, double eta, double* eta_used)
{
    TRY(enter(ctx));
    if (which != ESPNMF_U && which != ESPNMF_V) return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "which");
    if (!(eta <= 0.0 || std::isfinite(eta))) return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "eta");
    if (!ctx->U.valid || !ctx->V.valid)
        return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "U and V need values");
    Factor& F = which == ESPNMF_U ? ctx->U : ctx->V;
    Factor& O = which == ESPNMF_U ? ctx->V : ctx->U;
    TRY(ensure_product_for(ctx, which));
    if (eta > 0.0) {
        CU(cudaMemcpyAsync(ctx->pg, &eta, sizeof(double), cudaMemcpyHostToDevice, ctx->st));
    } else {
        TRY(run(ctx, K_LAMBDA, (double)ctx->k * ctx->k * 8, ctx->st, [&] {
            return launch_lambda_max(O.G, ctx->k, ctx->pg, ctx->pg + 1, ctx->st);
        }));
    }
    const EllDev& fe = F.buf[F.cur];
    TRY(run(ctx, K_PG, (double)F.rows * ctx->k * ctx->esz * 2, ctx->st, [&] {
        return is_f64(ctx) ? launch_pg_apply<double>(F.rows, ctx->k, fe, O.G, (const double*)ctx->Y,
                                                     ctx->ldy, ctx->pg, (double*)ctx->Xt, ctx->ldx,
                                                     ctx->st)
                           : launch_pg_apply<float>(F.rows, ctx->k, fe, O.G, (const float*)ctx->Y,
                                                    ctx->ldy, ctx->pg, (float*)ctx->Xt, ctx->ldx,
                                                    ctx->st);
    }));
    // keep every positive entry of the candidate (the support only shrinks)
    CU(cudaMemsetAsync(ctx->tau, 0, 8 * (size_t)ctx->k, ctx->st));
    CU(cudaMemsetAsync(ctx->cut, 0xff, 4 * (size_t)ctx->k, ctx->st));
    if (which == ESPNMF_U) {
        // Y = A V is current: the emit also forms R (old vs new U) and E
        TRY(do_emit(ctx, F, true, ctx->Y, false, TOPT_COLUMN));
        ctx->met_valid = false;
        ctx->have_R = false;
    } else {
        TRY(do_emit(ctx, F, false, nullptr, false, TOPT_COLUMN));
        ctx->met_valid = false;
    }
    if (eta_used) CU(cudaMemcpyAsync(eta_used, ctx->pg, sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    CU(cudaStreamSynchronize(ctx->st));
    return check_status(ctx);
}

espnmf_status espnmf_factor_nnz(espnmf_ctx* ctx, espnmf_which which, int64_t* nnz)
{
    TRY(enter(ctx));
    if (!nnz) return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "nnz is NULL");
    Factor& F = which == ESPNMF_U ? ctx->U : ctx->V;
    TRY(check_status(ctx));
    std::vector<int32_t> cnt(F.rows);
    CU(cudaMemcpy(cnt.data(), F.buf[F.cur].cnt, 4 * F.rows, cudaMemcpyDeviceToHost));
    int64_t s = 0;
    for (auto c : cnt) s += c;
    *nnz = s;
    return ESPNMF_OK;
}

espnmf_status espnmf_get_factor(espnmf_ctx* ctx, espnmf_which which, espnmf_layout layout,
                                int64_t* ptr, int32_t* idx, void* val, espnmf_dtype dtype,
                                int32_t on_device)
{
    TRY(enter(ctx));
    if (which != ESPNMF_U && which != ESPNMF_V) return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "which");
    if (dtype != ESPNMF_F64 && dtype != ESPNMF_F32)
        return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "dtype must be F64 or F32");
    if (!val) return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "val is NULL");
    if (layout != ESPNMF_DENSE_ROWMAJOR && (!ptr || !idx))
        return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "ptr/idx are NULL");
    Factor& F = which == ESPNMF_U ? ctx->U : ctx->V;
    TRY(check_status(ctx));
    const int64_t rows = F.rows;
    const int k = ctx->k;
    const EllDev& E = F.buf[F.cur];
    const int ld = E.ld;
    if (layout != ESPNMF_DENSE_ROWMAJOR && layout != ESPNMF_CSR && layout != ESPNMF_CSC)
        return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "unknown layout");
    // the row-packed arrays, copied into uninitialised host buffers; the
    // values are read in the compute type
    hvec<int32_t> cnt(rows), col((size_t)rows * ld);
    CU(cudaMemcpy(cnt.data(), E.cnt, 4 * rows, cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(col.data(), E.col, 4 * rows * ld, cudaMemcpyDeviceToHost));
    const size_t es = dtype == ESPNMF_F64 ? 8 : 4;
    std::vector<unsigned char> vo;
    std::vector<int64_t> po;
    std::vector<int32_t> io;
    if (is_f64(ctx)) {
        hvec<double> v((size_t)rows * ld);
        CU(cudaMemcpy(v.data(), E.val, 8 * rows * ld, cudaMemcpyDeviceToHost));
        pack_factor(rows, k, ld, cnt.data(), col.data(), v.data(), layout, es, vo, po, io);
    } else {
        hvec<float> v((size_t)rows * ld);
        CU(cudaMemcpy(v.data(), E.val, 4 * rows * ld, cudaMemcpyDeviceToHost));
        pack_factor(rows, k, ld, cnt.data(), col.data(), v.data(), layout, es, vo, po, io);
    }
    const cudaMemcpyKind kind = on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
    if (!vo.empty()) CU(cudaMemcpy(val, vo.data(), vo.size(), kind));
    if (!po.empty()) CU(cudaMemcpy(ptr, po.data(), po.size() * 8, kind));
    if (!io.empty()) CU(cudaMemcpy(idx, io.data(), io.size() * 4, kind));
    return ESPNMF_OK;
}

espnmf_status espnmf_set_option(espnmf_ctx* ctx, espnmf_option opt, int64_t value)
{
    TRY(enter(ctx));
    switch (opt) {
    case ESPNMF_OPT_USE_GRAPH: ctx->use_graph = value != 0; return ESPNMF_OK;
    case ESPNMF_OPT_PROFILE: ctx->profile = value != 0; return ESPNMF_OK;
    case ESPNMF_OPT_WAIT_LIMIT:
        if (value < 1) return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "wait limit must be >= 1");
        ctx->wait_limit = value;
        return ESPNMF_OK;
    case ESPNMF_OPT_SPMM_TUNE:
        ctx->spmm_tune = value != 0;
        if (ctx->spmm_tune) ctx->spmm_tuned = false;
        return ESPNMF_OK;
    case ESPNMF_OPT_SPMM_SPLIT:
        if (value != 1 && value != 2 && value != 4)
            return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "split is 1, 2 or 4");
        ctx->spmm_cfg[0].split = ctx->spmm_cfg[1].split = (int)value;
        ctx->spmm_tune = false;
        drop_graphs(ctx);
        return ESPNMF_OK;
    case ESPNMF_OPT_SPMM_CARVEOUT:
        if (value < -1 || value > 100) return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "carveout in -1..100");
        ctx->spmm_cfg[0].carveout = ctx->spmm_cfg[1].carveout = (int)value;
        ctx->spmm_tune = false;
        drop_graphs(ctx);
        return ESPNMF_OK;
    case ESPNMF_OPT_REFINE:
        if (value != 0 && value != 1) return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "refine is 0 or 1");
        ctx->refine = value != 0;
        drop_graphs(ctx);
        return ESPNMF_OK;
    case ESPNMF_OPT_SPMM_MASK:
        if (value < 0 || value > 2) return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "mask is 0, 1 or 2");
        for (int o = 0; o < 2; ++o) {
            // the product that gathers U (A^T U, o = 1) or V (A V, o = 0)
            const int64_t rows = o ? ctx->n : ctx->m;
            ctx->spmm_cfg[o].mask = (value == 2 && rows > 32ll * kSellSmemMaskWords) ? 1 : (int)value;
        }
        ctx->spmm_tune = false;
        drop_graphs(ctx);
        return ESPNMF_OK;
    }
    return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "unknown option");
}

espnmf_status espnmf_spmm_frequent(espnmf_ctx* ctx, int32_t product, int32_t* h, int64_t* hnnz)
{
    TRY(enter(ctx));
    if (!h || !hnnz || product < 0 || product > 1)
        return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "product must be 0 or 1, outputs non-NULL");
    const SellDev& S = product == 0 ? ctx->sA : ctx->sAt;
    *h = S.h;
    *hnnz = S.ft[0].nnz + S.ft[1].nnz;
    return ESPNMF_OK;
}

espnmf_status espnmf_select_stats(espnmf_ctx* ctx, int64_t* warm, int64_t* full)
{
    TRY(enter(ctx));
    if (!warm || !full) return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "outputs must be non-NULL");
    *warm = 0;
    *full = 0;
    if (!ctx->sel_counts) return ESPNMF_OK;
    unsigned long long h[2] = {0, 0};
    CU(cudaMemcpyAsync(h, ctx->sel_counts, sizeof(h), cudaMemcpyDeviceToHost, ctx->st));
    CU(cudaStreamSynchronize(ctx->st));
    *warm = (int64_t)h[0];
    *full = (int64_t)h[1];
    return ESPNMF_OK;
}

espnmf_status espnmf_kernel_stat_count(espnmf_ctx* ctx, int32_t* count)
{
    TRY(enter(ctx));
    if (!count) return ESPNMF_ERR_INVALID_ARG;
    *count = K_COUNT;
    return ESPNMF_OK;
}

espnmf_status espnmf_kernel_stat(espnmf_ctx* ctx, int32_t i, const char** name,
                                 int64_t* launches, double* total_ms, double* bytes)
{
    TRY(enter(ctx));
    if (i < 0 || i >= K_COUNT) return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "kernel index");
    TRY(collect_profile(ctx));
    if (name) *name = kernel_name(i);
    if (launches) *launches = ctx->stats[i].launches;
    if (total_ms) *total_ms = ctx->stats[i].ms;
    if (bytes) *bytes = ctx->stats[i].bytes;
    return ESPNMF_OK;
}

espnmf_status espnmf_kernel_stats_reset(espnmf_ctx* ctx)
{
    TRY(enter(ctx));
    TRY(collect_profile(ctx));
    for (auto& s : ctx->stats) s = Stat();
    return ESPNMF_OK;
}

espnmf_status espnmf_launches_per_sweep(espnmf_ctx* ctx, int32_t* count)
{
    TRY(enter(ctx));
    if (!count) return ESPNMF_ERR_INVALID_ARG;
    // U update: A V (+ combine, + frequent part), solve, select, emit,
    // (+ U's table Gram), reduce; the V update likewise with A^T U
    const bool sv = survivor_path(ctx);
    auto freq_launches = [](const SellDev& S) {
        return (S.h > 0 && S.ft[0].nrows > 0 ? 1 : 0) + (S.h > S.h1 && S.ft[1].nrows > 0 ? 1 : 0);
    };
    int per_half_A = 5 + (ctx->sA.nsplit > 0 ? 1 : 0) + freq_launches(ctx->sA) +
                     (sv && ctx->sAt.h > 0 ? 1 : 0);
    int per_half_At = 5 + (ctx->sAt.nsplit > 0 ? 1 : 0) + freq_launches(ctx->sAt) +
                      (sv && ctx->sA.h > 0 ? 1 : 0);
    *count = per_half_A + per_half_At + 2;   // + the two Gram inverse launches
    return ESPNMF_OK;
}

espnmf_status espnmf_sync(espnmf_ctx* ctx)
{
    TRY(enter(ctx));
    return check_status(ctx);
}

espnmf_status espnmf_solve_gram(const void* Y, int64_t rows, int32_t k, int64_t ldy,
                                const double* G, void* X, int64_t ldx, int32_t refine,
                                void* stream)
{
    g_init_error.clear();
    if (!Y || !G || !X || rows < 0 || k < 1 || k > 64 || ldy < k || ldx < k)
        return set_err(nullptr, ESPNMF_ERR_INVALID_ARG, "bad Y/G/X/rows/k/ld");
    if (rows >= (1ll << 31)) return set_err(nullptr, ESPNMF_ERR_INVALID_ARG, "too many rows");
    if (rows == 0) return ESPNMF_OK;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    auto cuerr = [&](cudaError_t e, const char* what) {
        cudaGetLastError();
        return set_err(nullptr, ESPNMF_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    };
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuerr(e, "device");
    {
        static std::mutex setup_mu;
        static bool setup_done[64] = {};
        std::lock_guard<std::mutex> lock(setup_mu);
        if (dev >= 64 || !setup_done[dev]) {
            if ((e = setup_chol()) != cudaSuccess) return cuerr(e, "setup");
            if (dev < 64) setup_done[dev] = true;
        }
    }
    const int KP = factor_ld(k);
    const int64_t ldt = (rows + 31) / 32 * 32;
    auto a256 = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t bl = a256(sizeof(float) * (4 * (size_t)KP * KP + KP));
    const size_t by = a256(sizeof(float) * (size_t)rows * KP);
    const size_t bt = a256(sizeof(float) * (size_t)k * ldt);
    unsigned char* ws = nullptr;
    e = cudaMallocAsync((void**)&ws, bl + by + bt + 256, st);
    if (e != cudaSuccess) return cuerr(e, "cudaMallocAsync");
    float* Lf = (float*)ws;
    float* Yp = (float*)(ws + bl);
    float* Xt = (float*)(ws + bl + by);
    unsigned* status = (unsigned*)(ws + bl + by + bt);
    float* gh = Lf + 2 * KP * KP + KP;
    e = cudaMemsetAsync(status, 0, sizeof(unsigned), st);
    // Y padded to KP columns (rows 16-byte aligned for the solve's loads)
    if (e == cudaSuccess) e = cudaMemsetAsync(Yp, 0, sizeof(float) * (size_t)rows * KP, st);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(Yp, sizeof(float) * KP, Y, sizeof(float) * ldy, sizeof(float) * k,
                              (size_t)rows, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = launch_cholesky(G, k, KP, Lf, Lf + KP * KP, Lf + 2 * KP * KP, status, st, gh, gh + KP * KP);
    if (e == cudaSuccess)
        e = launch_solve_chol(Yp, KP, rows, k, KP, Lf, Lf + KP * KP, Lf + 2 * KP * KP, Xt, ldt,
                              status, st, sms, false);
    if (e == cudaSuccess)
        e = launch_refine(Yp, KP, nullptr, 0, rows, k, KP, Lf, Lf + 2 * KP * KP, gh, gh + KP * KP,
                          Xt, ldt, (float*)X, ldx, true, refine != 0, status, st, sms);
    unsigned hstat = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hstat, status, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    cudaError_t e2 = cudaFreeAsync(ws, st);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuerr(e, "solve_gram");
    // a singular G is the cause of the non-finite X it leads to: report it first
    if (hstat & ST_SINGULAR) return set_err(nullptr, ESPNMF_ERR_SINGULAR, "G is singular beyond its zero columns");
    if (hstat & ST_NONFINITE) return set_err(nullptr, ESPNMF_ERR_NONFINITE, "non-finite value in G or X");
    return ESPNMF_OK;
}

espnmf_status espnmf_enforce_topt_buffer(void* X, int64_t rows, int32_t k, int64_t ld,
                                         espnmf_dtype dtype, int64_t t, espnmf_topt_mode mode,
                                         void* stream)
{
    g_init_error.clear();
    if (!X || rows < 0 || k < 1 || k > 128 || ld < k || t < 0)
        return set_err(nullptr, ESPNMF_ERR_INVALID_ARG, "bad X/rows/k/ld/t");
    if (dtype != ESPNMF_F64 && dtype != ESPNMF_F32)
        return set_err(nullptr, ESPNMF_ERR_INVALID_ARG, "dtype must be F64 or F32");
    if (mode != ESPNMF_TOPT_COLUMN && mode != ESPNMF_TOPT_MATRIX && mode != ESPNMF_TOPT_NONE)
        return set_err(nullptr, ESPNMF_ERR_INVALID_ARG, "unknown enforcement mode");
    if (rows >= (1ll << 31) || (mode == ESPNMF_TOPT_MATRIX && rows * k >= (1ll << 31)))
        return set_err(nullptr, ESPNMF_ERR_INVALID_ARG, "too many rows");
    if (rows == 0) return ESPNMF_OK;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    auto cuerr = [&](cudaError_t e, const char* what) {
        cudaGetLastError();
        return set_err(nullptr, ESPNMF_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    };
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuerr(e, "device");
    {
        // per-device kernel attribute set-up, once, under a lock (callers
        // may come from several host threads)
        static std::mutex setup_mu;
        static bool setup_done[64] = {};
        std::lock_guard<std::mutex> lock(setup_mu);
        if (dev >= 64 || !setup_done[dev]) {
            if ((e = setup_select()) != cudaSuccess) return cuerr(e, "setup");
            if (dev < 64) setup_done[dev] = true;
        }
    }
    const size_t es = dtype == ESPNMF_F64 ? 8 : 4;
    const int64_t ldx = (rows + 31) / 32 * 32;
    auto a256 = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t bx = a256((size_t)k * ldx * es), bt = a256((size_t)k * 8), bc = a256((size_t)k * 4);
    unsigned char* ws = nullptr;
    e = cudaMallocAsync((void**)&ws, bx + bt + bc + 256, st);
    if (e != cudaSuccess) return cuerr(e, "cudaMallocAsync");
    void* tau = ws + bx;
    uint32_t* cut = (uint32_t*)(ws + bx + bt);
    unsigned* status = (unsigned*)(ws + bx + bt + bc);
    e = cudaMemsetAsync(status, 0, sizeof(unsigned), st);
    if (e == cudaSuccess)
        e = dtype == ESPNMF_F64
                ? launch_dense_to_colmajor<double, double>((const double*)X, rows, k, ld, (double*)ws, ldx, status, false, st)
                : launch_dense_to_colmajor<float, float>((const float*)X, rows, k, ld, (float*)ws, ldx, status, false, st);
    if (e == cudaSuccess)
        e = dtype == ESPNMF_F64
                ? launch_select<double>((const double*)ws, ldx, rows, k, t, (int)mode, tau, cut, st, sms, nullptr, nullptr)
                : launch_select<float>((const float*)ws, ldx, rows, k, t, (int)mode, tau, cut, st, sms, nullptr, nullptr);
    if (e == cudaSuccess)
        e = dtype == ESPNMF_F64 ? launch_apply_thresholds<double>((double*)X, rows, k, ld, (int)mode, tau, cut, status, st)
                                : launch_apply_thresholds<float>((float*)X, rows, k, ld, (int)mode, tau, cut, status, st);
    unsigned hstat = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hstat, status, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    cudaError_t e2 = cudaFreeAsync(ws, st);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuerr(e, "enforce_topt_buffer");
    if (hstat & ST_NONFINITE) return set_err(nullptr, ESPNMF_ERR_NONFINITE, "non-finite value in X");
    return ESPNMF_OK;
}

}  // extern "C"

extern "C" espnmf_status espnmf_spmm_config(espnmf_ctx* ctx, int32_t product, int32_t* split,
                                            int32_t* carveout, int32_t* mask)
{
    TRY(enter(ctx));
    if (product != 0 && product != 1) return set_err(ctx, ESPNMF_ERR_INVALID_ARG, "product is 0 or 1");
    const SpmmConfig& c = ctx->spmm_cfg[product];
    if (split) *split = (is_f64(ctx) || ctx->ldy < 16) ? 1 : c.split;
    if (carveout) *carveout = c.carveout;
    if (mask) *mask = is_f64(ctx) ? 0 : c.mask;
    return ESPNMF_OK;
}

// =================================================================================
// Batched sweeps: many independent problems, one captured CUDA graph per sweep

struct espnmf_batch {
    int device = 0;
    std::vector<espnmf_ctx*> ctxs;
    std::vector<cudaStream_t> pool;   // problem i runs on pool[i % pool.size()]
    cudaStream_t st = nullptr;        // graph launches
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;    // one per pool stream
    cudaGraphExec_t gexec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    bool use_graph = true;
};

namespace {

espnmf_status batch_fail(espnmf_status s, const std::string& msg)
{
    espnmf::set_thread_error(msg.c_str());
    return s;
}

// st waits for everything enqueued on the pool streams so far
cudaError_t pool_to_main(espnmf_batch* b)
{
    for (size_t s = 0; s < b->pool.size(); ++s) {
        cudaError_t e = cudaEventRecord(b->join[s], b->pool[s]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->st, b->join[s], 0);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// every pool stream waits for everything enqueued on st so far
cudaError_t main_to_pool(espnmf_batch* b)
{
    cudaError_t e = cudaEventRecord(b->fork, b->st);
    for (size_t s = 0; e == cudaSuccess && s < b->pool.size(); ++s)
        e = cudaStreamWaitEvent(b->pool[s], b->fork, 0);
    return e;
}

// One sweep of every problem, captured from the pool streams into one graph.
espnmf_status batch_graph(espnmf_batch* b, cudaGraphExec_t* out)
{
    std::vector<HostState> saved;
    for (auto* c : b->ctxs) saved.push_back(save_state(c));
    cudaError_t e = cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return batch_fail(ESPNMF_ERR_CUDA, std::string("batch capture: ") + cudaGetErrorString(e));
    e = main_to_pool(b);
    espnmf_status st = e == cudaSuccess ? ESPNMF_OK : ESPNMF_ERR_CUDA;
    for (size_t i = 0; st == ESPNMF_OK && i < b->ctxs.size(); ++i) st = enqueue_sweep(b->ctxs[i]);
    if (st == ESPNMF_OK && pool_to_main(b) != cudaSuccess) st = ESPNMF_ERR_CUDA;
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->st, &g);
    for (size_t i = 0; i < b->ctxs.size(); ++i) restore_state(b->ctxs[i], saved[i]);
    if (st != ESPNMF_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return batch_fail(ESPNMF_ERR_CUDA, "batch capture failed");
    }
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return batch_fail(ESPNMF_ERR_CUDA, std::string("batch graph: ") + cudaGetErrorString(e));
    return ESPNMF_OK;
}

}  // namespace

extern "C" {

espnmf_status espnmf_batch_init(espnmf_batch** out, int32_t nprob, const espnmf_csr* As,
                                const int32_t* ks, const int64_t* t_us, const int64_t* t_vs,
                                espnmf_topt_mode mode, espnmf_dtype compute,
                                const void* const* U0s, espnmf_dtype U0_dtype,
                                int32_t U0_on_device, int32_t streams)
{
    espnmf::set_thread_error("");
    if (!out) return batch_fail(ESPNMF_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (nprob < 1 || !As || !ks || !t_us || !t_vs || !U0s)
        return batch_fail(ESPNMF_ERR_INVALID_ARG, "need nprob >= 1 and non-NULL arrays");
    auto* b = new espnmf_batch();
    auto fail = [&](espnmf_status s, const std::string& m) {
        espnmf_batch_destroy(b);
        return batch_fail(s, m);
    };
    cudaError_t e = cudaGetDevice(&b->device);
    const int S = std::max(1, std::min<int>(nprob, streams > 0 ? streams : 16));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    for (int s = 0; e == cudaSuccess && s < S; ++s) {
        cudaStream_t ps = nullptr;
        cudaEvent_t ev = nullptr;
        e = cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking);
        if (e == cudaSuccess) b->pool.push_back(ps);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) b->join.push_back(ev);
    }
    if (e != cudaSuccess) return fail(ESPNMF_ERR_CUDA, std::string("batch streams: ") + cudaGetErrorString(e));
    for (int i = 0; i < nprob; ++i) {
        espnmf_ctx* c = nullptr;
        const espnmf_status s = espnmf_init(&c, &As[i], ks[i], t_us[i], t_vs[i], mode, compute,
                                            U0s[i], U0_dtype, U0_on_device, b->pool[i % S]);
        if (s != ESPNMF_OK) {
            const std::string why = espnmf_last_error(nullptr);
            return fail(s, "problem " + std::to_string(i) + ": " + why);
        }
        b->ctxs.push_back(c);
    }
    *out = b;
    return ESPNMF_OK;
}

espnmf_status espnmf_batch_destroy(espnmf_batch* b)
{
    if (!b) return ESPNMF_OK;
    cudaSetDevice(b->device);
    if (b->st) cudaStreamSynchronize(b->st);
    for (auto& row : b->gexec)
        for (auto& g : row)
            if (g) cudaGraphExecDestroy(g);
    for (auto* c : b->ctxs) espnmf_destroy(c);
    for (auto s : b->pool) cudaStreamDestroy(s);
    for (auto ev : b->join) cudaEventDestroy(ev);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->st) cudaStreamDestroy(b->st);
    delete b;
    return ESPNMF_OK;
}

espnmf_status espnmf_batch_ctx(espnmf_batch* b, int32_t i, espnmf_ctx** out)
{
    if (!b || !out || i < 0 || i >= (int32_t)b->ctxs.size())
        return batch_fail(ESPNMF_ERR_INVALID_ARG, "bad batch, index or out");
    *out = b->ctxs[i];
    return ESPNMF_OK;
}

espnmf_status espnmf_batch_set_option(espnmf_batch* b, espnmf_option opt, int64_t value)
{
    if (!b) return batch_fail(ESPNMF_ERR_INVALID_ARG, "batch is NULL");
    if (opt != ESPNMF_OPT_USE_GRAPH) return batch_fail(ESPNMF_ERR_INVALID_ARG, "unsupported batch option");
    b->use_graph = value != 0;
    return ESPNMF_OK;
}

espnmf_status espnmf_batch_iterate(espnmf_batch* b, int32_t iters, espnmf_status* status_out,
                                   double* R_out, double* E_out)
{
    espnmf::set_thread_error("");
    if (!b) return batch_fail(ESPNMF_ERR_INVALID_ARG, "batch is NULL");
    if (iters < 0) return batch_fail(ESPNMF_ERR_INVALID_ARG, "iters must be >= 0");
    cudaError_t e = cudaSetDevice(b->device);
    if (e != cudaSuccess) return batch_fail(ESPNMF_ERR_CUDA, cudaGetErrorString(e));
    const int n = (int)b->ctxs.size();
    for (auto* c : b->ctxs) {
        c->err.clear();
        espnmf_status s = ensure_hist(c, std::max(iters, 1));
        if (s == ESPNMF_OK && cudaMemsetAsync(c->hist_counter, 0, sizeof(int), c->st) != cudaSuccess)
            s = ESPNMF_ERR_CUDA;
        if (s != ESPNMF_OK) return batch_fail(s, "batch history buffers");
    }
    int it = 0;
    // the problems sweep in lockstep; a graph needs them all in one state
    auto lockstep = [&]() {
        for (auto* c : b->ctxs)
            if (!c->V.valid || c->U.cur != b->ctxs[0]->U.cur || c->V.cur != b->ctxs[0]->V.cur)
                return false;
        return true;
    };
    espnmf_status st = ESPNMF_OK;
    for (; st == ESPNMF_OK && it < iters; ++it) {
        if (!b->use_graph || !lockstep()) {
            for (int i = 0; st == ESPNMF_OK && i < n; ++i) st = enqueue_sweep(b->ctxs[i]);
            continue;
        }
        cudaGraphExec_t& g = b->gexec[b->ctxs[0]->U.cur][b->ctxs[0]->V.cur];
        if (!g) st = batch_graph(b, &g);
        if (st != ESPNMF_OK) break;
        if (pool_to_main(b) != cudaSuccess || cudaGraphLaunch(g, b->st) != cudaSuccess ||
            main_to_pool(b) != cudaSuccess) {
            st = batch_fail(ESPNMF_ERR_CUDA, "batch graph launch");
            break;
        }
        for (auto* c : b->ctxs) after_sweep_state(c);
    }
    if (st != ESPNMF_OK) return st;
    // per-problem status and measures
    espnmf_status worst = ESPNMF_OK;
    for (int i = 0; i < n; ++i) {
        espnmf_ctx* c = b->ctxs[i];
        espnmf_status s = check_status(c);
        if (s == ESPNMF_OK && iters > 0) {
            if (R_out && cudaMemcpy(R_out + (size_t)i * iters, c->hist_R, sizeof(double) * iters,
                                    cudaMemcpyDeviceToHost) != cudaSuccess)
                s = ESPNMF_ERR_CUDA;
            if (E_out && cudaMemcpy(E_out + (size_t)i * iters, c->hist_E, sizeof(double) * iters,
                                    cudaMemcpyDeviceToHost) != cudaSuccess)
                s = ESPNMF_ERR_CUDA;
        }
        if (status_out) status_out[i] = s;
        if (s != ESPNMF_OK && worst == ESPNMF_OK) worst = s;
    }
    if (worst != ESPNMF_OK)
        espnmf::set_thread_error("one or more problems failed: see the status array");
    return worst;
}

// Alg. 3 (sequential ALS, Sec. 4) on one k = k2 context: for each block of
// k2 topics the context's U is reset to U0, `iters` sweeps run (graph
// replays after the first, as espnmf_iterate runs them) with the converged
// topics subtracted after each sparse product (the deflation hook of
// half_update, which reads the number of converged topics on the device;
// none for the first block, which is Alg. 2 itself), and the block is
// appended to the dense U1, V1.
espnmf_status espnmf_sequential(const espnmf_csr* A, int32_t k, int32_t k2, int64_t t_u,
                                int64_t t_v, int32_t iters, espnmf_dtype compute, const void* U0,
                                espnmf_dtype u0_dtype, int32_t u0_on_device, void* U_out,
                                void* V_out, double* seconds_out, void* stream)
{
    espnmf::set_thread_error("");
    if (!A || !U0 || !U_out || !V_out)
        return batch_fail(ESPNMF_ERR_INVALID_ARG, "A, U0, U_out and V_out must be non-NULL");
    if (k < 1 || k2 < 1 || iters < 1)
        return batch_fail(ESPNMF_ERR_INVALID_ARG, "need k >= 1, k2 >= 1 and iters >= 1");
    if (k % k2 != 0)
        return batch_fail(ESPNMF_ERR_INVALID_ARG, "k must be a multiple of k2");
    if (k > A->n || k > A->m)
        return batch_fail(ESPNMF_ERR_INVALID_ARG, "k must be <= min(n, m)");
    espnmf_ctx* c = nullptr;
    espnmf_status st = espnmf_init(&c, A, k2, t_u, t_v, ESPNMF_TOPT_COLUMN, compute, U0, u0_dtype,
                                   u0_on_device, stream);
    if (st != ESPNMF_OK) return st;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    auto fail = [&](espnmf_status s) {
        const std::string msg = c->err;
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
        espnmf_destroy(c);
        return batch_fail(s, msg.empty() ? "sequential ALS failed" : msg);
    };
    if (seconds_out &&
        (cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess))
        return fail(set_err(c, ESPNMF_ERR_CUDA, "sequential: event"));
    const bool f64 = is_f64(c);
    const size_t es = c->esz;
    const int64_t n = c->n, m = c->m;
    Deflation& d = c->defl;
    if ((st = dmalloc(c, &d.U1, es * (size_t)n * k)) != ESPNMF_OK) return fail(st);
    if ((st = dmalloc(c, &d.V1, es * (size_t)m * k)) != ESPNMF_OK) return fail(st);
    if ((st = dmalloc(c, &d.g, sizeof(double) * (size_t)k * k2)) != ESPNMF_OK) return fail(st);
    if (cudaMemsetAsync(d.U1, 0, es * (size_t)n * k, c->st) != cudaSuccess ||
        cudaMemsetAsync(d.V1, 0, es * (size_t)m * k, c->st) != cudaSuccess)
        return fail(set_err(c, ESPNMF_ERR_CUDA, "sequential: memset"));
    d.ld1 = k;
    // the converged topics of block b, b * k2, copied on the stream into the
    // device word the deflation reads before the block's sweeps
    const int nblocks = k / k2;
    int* kvals = nullptr;
    {
        std::vector<int> kv(nblocks);
        for (int b = 0; b < nblocks; ++b) kv[b] = b * k2;
        if ((st = dupload(c, &kvals, kv.data(), sizeof(int) * (size_t)nblocks)) != ESPNMF_OK)
            return fail(st);
    }
    if ((st = dmalloc(c, &d.k1, sizeof(int))) != ESPNMF_OK) return fail(st);
    d.k1_max = k - k2;
    d.active = true;
    if (ev[0] && cudaEventRecord(ev[0], c->st) != cudaSuccess)
        return fail(set_err(c, ESPNMF_ERR_CUDA, "sequential: event"));
    for (int b = 0; b < nblocks; ++b) {
        const int j0 = b * k2;
        if (j0 > 0 && (st = espnmf_set_factor(c, ESPNMF_U, U0, u0_dtype, u0_on_device)) != ESPNMF_OK)
            return fail(st);
        if (cudaMemcpyAsync(d.k1, kvals + b, sizeof(int), cudaMemcpyDeviceToDevice, c->st) != cudaSuccess)
            return fail(set_err(c, ESPNMF_ERR_CUDA, "sequential: block start"));
        // the block's sweeps: the first eagerly (the first block's V does not
        // exist yet), the rest replayed from the context's captured sweeps
        if ((st = espnmf_iterate(c, iters, nullptr, nullptr)) != ESPNMF_OK) return fail(st);
        const EllDev& fu = c->U.buf[c->U.cur];
        const EllDev& fv = c->V.buf[c->V.cur];
        cudaError_t e = f64 ? launch_seq_append<double>(n, fu.cnt, fu.col, (const double*)fu.val,
                                                        fu.ld, k2, (double*)d.U1, k, j0, c->st)
                            : launch_seq_append<float>(n, fu.cnt, fu.col, (const float*)fu.val,
                                                       fu.ld, k2, (float*)d.U1, k, j0, c->st);
        if (e == cudaSuccess)
            e = f64 ? launch_seq_append<double>(m, fv.cnt, fv.col, (const double*)fv.val, fv.ld, k2,
                                                (double*)d.V1, k, j0, c->st)
                    : launch_seq_append<float>(m, fv.cnt, fv.col, (const float*)fv.val, fv.ld, k2,
                                               (float*)d.V1, k, j0, c->st);
        if (e != cudaSuccess)
            return fail(set_err(c, ESPNMF_ERR_CUDA, "sequential: %s", cudaGetErrorString(e)));
    }
    if (ev[1] && cudaEventRecord(ev[1], c->st) != cudaSuccess)
        return fail(set_err(c, ESPNMF_ERR_CUDA, "sequential: event"));
    if (cudaMemcpyAsync(U_out, d.U1, es * (size_t)n * k, cudaMemcpyDeviceToDevice, c->st) != cudaSuccess ||
        cudaMemcpyAsync(V_out, d.V1, es * (size_t)m * k, cudaMemcpyDeviceToDevice, c->st) != cudaSuccess)
        return fail(set_err(c, ESPNMF_ERR_CUDA, "sequential: copy-out"));
    if ((st = check_status(c)) != ESPNMF_OK) return fail(st);
    if (cudaStreamSynchronize(c->st) != cudaSuccess)
        return fail(set_err(c, ESPNMF_ERR_CUDA, "sequential: synchronize"));
    if (seconds_out) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ev[0], ev[1]) != cudaSuccess)
            return fail(set_err(c, ESPNMF_ERR_CUDA, "sequential: event time"));
        *seconds_out = ms / 1000.0;
        cudaEventDestroy(ev[0]);
        cudaEventDestroy(ev[1]);
    }
    espnmf_destroy(c);
    return ESPNMF_OK;
}

espnmf_status espnmf_checked_flags(uint32_t* flags)
{
    if (!flags) return batch_fail(ESPNMF_ERR_INVALID_ARG, "flags is NULL");
#ifdef ESPNMF_CHECKED
    const unsigned part[4] = {check_flags_spmm(), check_flags_select(), check_flags_factor(),
                              check_flags_seq()};
    *flags = 0;
    for (unsigned v : part) {
        if (v == 0xffffffffu)
            return batch_fail(ESPNMF_ERR_CUDA, "could not read the check flags (no usable CUDA device)");
        *flags |= v;
    }
    espnmf::set_thread_error("");
    return ESPNMF_OK;
#else
    *flags = 0;
    return batch_fail(ESPNMF_ERR_UNSUPPORTED, "not a checked build (compile with -DESPNMF_CHECKED)");
#endif
}

}  // extern "C"
