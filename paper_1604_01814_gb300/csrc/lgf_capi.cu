// C ABI of the library: argument checking, context life cycle, plan and
// spectrum caches, the batched path and its CUDA-graph cache.
#include <algorithm>
#include <array>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <set>
#include <string>
#include <vector>

#include "lgf_internal.cuh"
#include "lgf_tune.h"

namespace lgf {

lgf_status fail(lgf_ctx *ctx, lgf_status st, const std::string &msg)
{
    if (ctx) ctx->last_error = msg;
    return st;
}

lgf_status cuda_fail(lgf_ctx *ctx, cudaError_t e, const char *what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    if (e == cudaErrorMemoryAllocation) return fail(ctx, LGF_ENOMEM, m);
    return fail(ctx, LGF_ECUDA, m);
}

void invalidate_graphs(lgf_ctx *ctx)
{
    ctx->graphs.invalidate([](cudaGraphExec_t g) { cudaGraphExecDestroy(g); }, &ctx->counters);
}

void before_evict(lgf_ctx *ctx)
{
    invalidate_graphs(ctx);
    cudaDeviceSynchronize();
}

lgf_status ensure_scratch(lgf_ctx *ctx, void **p, size_t *have, size_t need)
{
    if (need <= *have) return LGF_OK;
    // a cached graph may hold the old buffer's address: drop them all
    if (ctx) {
        invalidate_graphs(ctx);
        ++ctx->counters.scratch_reallocs;
    }
    if (*p) {
        cudaError_t e = cudaFree(*p);
        *p = nullptr;
        *have = 0;
        if (e != cudaSuccess) return cuda_fail(ctx, e, "scratch release");
    }
    const size_t bytes = need + need / 8 + 256;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(ctx, LGF_ENOMEM, "scratch allocation of " + std::to_string(bytes) + " bytes failed");
    }
    *have = bytes;
    return LGF_OK;
}

lgf_status check_blockset(lgf_ctx *ctx, const lgf_blockset *bs, const char *name)
{
    if (!bs) return fail(ctx, LGF_EINVAL, std::string(name) + ": null block set");
    if (bs->nblocks < 0) return fail(ctx, LGF_EINVAL, std::string(name) + ": negative block count");
    if (bs->nblocks > 0 && !bs->coords) return fail(ctx, LGF_EINVAL, std::string(name) + ": null coordinates");
    const int b = bs->b;
    if (b != 4 && b != 8 && b != 16 && b != 32 && b != 64)
        return fail(ctx, LGF_EINVAL, std::string(name) + ": block edge must be 4, 8, 16, 32 or 64");
    for (int i = 0; i < 3 * bs->nblocks; ++i)
        if (bs->coords[i] < -(1 << 19) || bs->coords[i] >= (1 << 19))
            return fail(ctx, LGF_EINVAL, std::string(name) + ": block coordinate out of range");
    return LGF_OK;
}

int prof_begin(lgf_ctx *ctx, cudaStream_t s, const char *name)
{
    if (!ctx->prof) return -1;
    int id = -1;
    for (size_t i = 0; i < ctx->prof_names.size(); ++i)
        if (ctx->prof_names[i] == name) id = (int)i;
    if (id < 0) {
        id = (int)ctx->prof_names.size();
        ctx->prof_names.push_back(name);
        ctx->prof_launches.push_back(0);
        ctx->prof_ms.push_back(0.0);
    }
    cudaEvent_t ev[2];
    for (int k = 0; k < 2; ++k) {
        if (!ctx->ev_pool.empty()) {
            ev[k] = ctx->ev_pool.back();
            ctx->ev_pool.pop_back();
        } else if (cudaEventCreate(&ev[k]) != cudaSuccess) {
            return -1;
        }
    }
    cudaEventRecord(ev[0], s);
    ctx->prof_pending.push_back({id, ev[0], ev[1]});
    return (int)ctx->prof_pending.size() - 1;
}

void prof_end(lgf_ctx *ctx, cudaStream_t s, int handle)
{
    if (handle < 0 || !ctx->prof) return;
    cudaEventRecord(ctx->prof_pending[handle].b, s);
}

}  // namespace lgf

using namespace lgf;

namespace {

lgf_status enter(lgf_ctx *ctx)
{
    if (!ctx) return LGF_EINVAL;
    ctx->last_error.clear();
    ctx->cur = &ctx->scr[0];
    ++ctx->counters.epoch;   // cache entries stamped with this call are kept until it returns
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    return LGF_OK;
}

lgf_status check_fields(lgf_ctx *ctx, const void *f, void *u, int ncomp, int nrhs, int nsrc, int ntgt)
{
    if (ncomp < 1 || nrhs < 1) return fail(ctx, LGF_EINVAL, "ncomp and nrhs must be >= 1");
    if (ntgt > 0 && !u) return fail(ctx, LGF_EINVAL, "null output pointer");
    if (nsrc > 0 && ntgt > 0 && !f) return fail(ctx, LGF_EINVAL, "null input pointer");
    return LGF_OK;
}

size_t elem_size(const lgf_ctx *ctx) { return ctx->prec == LGF_F64 ? 8 : 4; }

// Everything an apply needs before any kernel is enqueued (allocations,
// synchronous set-up); also used to make batch capture allocation-free.
struct PreparedPoisson {
    PoissonPlan *plan = nullptr;
    Spectrum *spec = nullptr;
};

// kalpha = 0: the kernel G_L; kalpha > 0: G_K(kalpha).
lgf_status prepare_poisson(lgf_ctx *ctx, const lgf_blockset *src, const lgf_blockset *tgt, int nfields,
                           double kalpha, cudaStream_t s, PreparedPoisson *pp)
{
    if (ctx->table_dev == nullptr) return fail(ctx, LGF_ENOTABLE, "lgf_table_build has not been called");
    lgf_status st = poisson_plan(ctx, src, tgt, &pp->plan);
    if (st != LGF_OK) return st;
    if ((st = tune_poisson(ctx, pp->plan, nfields, kalpha, s)) != LGF_OK) return st;
    st = poisson_spectrum(ctx, pp->plan->g, kalpha, &pp->spec, s);
    if (st != LGF_OK) return st;
    st = poisson_prepare_scratch(ctx, pp->plan, nfields);
    if (st != LGF_OK) return st;
    for (int d = 0; d < 3; ++d) {
        twiddles(ctx, pp->plan->g.M[d], ctx->prec == LGF_F64, &st);
        if (st != LGF_OK) return st;
    }
    return LGF_OK;
}

struct PreparedIntf {
    IntfPlan *plan = nullptr;
    IntfWeights *w = nullptr;
};

lgf_status prepare_intf(lgf_ctx *ctx, double alpha, const lgf_blockset *src, const lgf_blockset *tgt, int nfields,
                        cudaStream_t s, PreparedIntf *pi)
{
    lgf_status st = intf_weights(ctx, alpha, &pi->w, s);
    if (st != LGF_OK) return st;
    st = intf_plan(ctx, src, tgt, pi->w->R, &pi->plan);
    if (st != LGF_OK) return st;
    return intf_prepare_scratch(ctx, pi->plan, nfields, 1);
}

}  // namespace

extern "C" {

int32_t lgf_version(void) { return 10000; }

const char *lgf_status_string(lgf_status s)
{
    switch (s) {
    case LGF_OK: return "success";
    case LGF_EINVAL: return "invalid argument";
    case LGF_ENOMEM: return "out of memory";
    case LGF_ECUDA: return "CUDA error";
    case LGF_ETIMEOUT: return "device-side wait timed out";
    case LGF_EUNSUPPORTED: return "unsupported size";
    case LGF_ENOTABLE: return "G_L table not built";
    }
    return "unknown status";
}

const char *lgf_last_error(lgf_ctx *ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

lgf_status lgf_ctx_create(lgf_ctx **out, const lgf_options *opt)
{
    if (!out) return LGF_EINVAL;
    *out = nullptr;
    lgf_options o{};
    if (opt) o = *opt;
    if (o.prec != LGF_F32 && o.prec != LGF_F64) return LGF_EINVAL;
    if (!(o.tol >= 0.0) || !std::isfinite(o.tol) || o.tol >= 1.0) return LGF_EINVAL;
    if (o.table_radius != 0 && (o.table_radius < 8 || o.table_radius > 96)) return LGF_EINVAL;
    if (o.stencil_radius < 0 || o.stencil_radius > 128 || o.device < 0) return LGF_EINVAL;
    for (int i = 0; i < 3; ++i)
        if (o.reserved[i] != 0) return LGF_EINVAL;
    if ((o.flags & ~(LGF_FLAG_BULK_STAGING | LGF_FLAG_BATCH_RAGGED | LGF_FLAG_BATCH_PER_PROBLEM)) != 0 ||
        ((o.flags & LGF_FLAG_BATCH_RAGGED) && (o.flags & LGF_FLAG_BATCH_PER_PROBLEM)))
        return LGF_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || o.device >= ndev) {
        cudaGetLastError();
        return LGF_ECUDA;
    }
    if (cudaSetDevice(o.device) != cudaSuccess) return LGF_ECUDA;
    lgf_ctx *ctx = new (std::nothrow) lgf_ctx;
    if (!ctx) return LGF_ENOMEM;
    ctx->opt = o;
    ctx->opt_bulk = (o.flags & LGF_FLAG_BULK_STAGING) != 0;
    ctx->opt_rag = (o.flags & LGF_FLAG_BATCH_RAGGED) != 0;
    ctx->opt_units = (o.flags & LGF_FLAG_BATCH_PER_PROBLEM) != 0;
    ctx->device = o.device;
    ctx->prec = o.prec;
    ctx->tol = o.tol > 0.0 ? o.tol : (o.prec == LGF_F64 ? 1e-13 : 1e-7);
    if (ctx->opt.table_radius == 0) ctx->opt.table_radius = 48;
    if (cudaMalloc(&ctx->red_dev, 16 * sizeof(double)) != cudaSuccess) {
        delete ctx;
        return LGF_ENOMEM;
    }
    if (cudaMalloc(&ctx->err_dev, sizeof(int)) != cudaSuccess || cudaMemset(ctx->err_dev, 0, sizeof(int)) != cudaSuccess) {
        cudaFree(ctx->red_dev);
        cudaFree(ctx->err_dev);
        delete ctx;
        return LGF_ENOMEM;
    }
    *out = ctx;
    return LGF_OK;
}

lgf_status lgf_ctx_destroy(lgf_ctx *ctx)
{
    if (!ctx) return LGF_EINVAL;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    invalidate_graphs(ctx);
    ctx->pplans.clear();
    ctx->iplans.clear();
    ctx->cplans.clear();
    ctx->ibplans.clear();
    ctx->spectra.clear();
    for (auto &kv : ctx->gk_tables) cudaFree(kv.second);
    for (auto &kv : ctx->tw32) cudaFree(kv.second);
    for (auto &kv : ctx->tw64) cudaFree(kv.second);
    for (auto &w : ctx->weights) {
        cudaFree(w->w64);
        cudaFree(w->w32);
    }
    cudaFree(ctx->table_dev);
    for (auto &sc : ctx->scr) {
        cudaFree(sc.A);
        cudaFree(sc.B);
        cudaFree(sc.C);
        cudaFree(sc.D);
        cudaFree(sc.E);
        cudaFree(sc.F);
        cudaFree(sc.G);
    }
    for (int b = 0; b < kBranches; ++b) {
        if (ctx->br[b]) cudaStreamDestroy(ctx->br[b]);
        if (ctx->ev_join[b]) cudaEventDestroy(ctx->ev_join[b]);
    }
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    cudaFree(ctx->red_dev);
    cudaFree(ctx->err_dev);
    cudaFree(ctx->tune_f);
    cudaFree(ctx->tune_u);
    for (auto &r : ctx->prof_pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : ctx->ev_pool) cudaEventDestroy(e);
    delete ctx;
    return LGF_OK;
}

lgf_status lgf_table_build(lgf_ctx *ctx, int32_t max_offset, void *stream)
{
    lgf_status st = enter(ctx);
    if (st != LGF_OK) return st;
    if (max_offset < 0) return fail(ctx, LGF_EINVAL, "table_build: max_offset < 0");
    const int R = std::min(ctx->opt.table_radius, std::max<int>(max_offset, kMinTableRadius));
    if (ctx->table_dev && ctx->table_radius >= R) return LGF_OK;
    st = table_build(ctx, R, (cudaStream_t)stream);
    if (st != LGF_OK) return st;
    // spectra and G_K tables built from an older table are stale (the graphs
    // that read them go first)
    before_evict(ctx);
    ctx->spectra.clear();
    for (auto &kv : ctx->gk_tables) cudaFree(kv.second);
    ctx->gk_tables.clear();
    return LGF_OK;
}

lgf_status lgf_table_info(lgf_ctx *ctx, int32_t *table_radius, double *shell_mismatch)
{
    if (!ctx) return LGF_EINVAL;
    if (!ctx->table_dev) return fail(ctx, LGF_ENOTABLE, "table not built");
    if (table_radius) *table_radius = ctx->table_radius;
    if (shell_mismatch) *shell_mismatch = ctx->shell_mismatch;
    return LGF_OK;
}

lgf_status lgf_table_lookup(lgf_ctx *ctx, const int32_t *offsets_dev, int64_t n, double *out_dev, void *stream)
{
    lgf_status st = enter(ctx);
    if (st != LGF_OK) return st;
    if (!ctx->table_dev) return fail(ctx, LGF_ENOTABLE, "table not built");
    if (n < 0 || (n > 0 && (!offsets_dev || !out_dev))) return fail(ctx, LGF_EINVAL, "table_lookup: bad arguments");
    return table_lookup(ctx, ctx->table_dev, offsets_dev, n, out_dev, (cudaStream_t)stream);
}

lgf_status lgf_kinv_lookup(lgf_ctx *ctx, double alpha, const int32_t *offsets_dev, int64_t n, double *out_dev,
                           void *stream)
{
    lgf_status st = enter(ctx);
    if (st != LGF_OK) return st;
    if (!ctx->table_dev) return fail(ctx, LGF_ENOTABLE, "table not built");
    if (!(alpha >= 0.0) || !std::isfinite(alpha)) return fail(ctx, LGF_EINVAL, "alpha must be >= 0 and finite");
    if (n < 0 || (n > 0 && (!offsets_dev || !out_dev))) return fail(ctx, LGF_EINVAL, "kinv_lookup: bad arguments");
    const double *table = nullptr;
    if ((st = gk_table(ctx, alpha, &table, (cudaStream_t)stream)) != LGF_OK) return st;
    return table_lookup(ctx, table, offsets_dev, n, out_dev, (cudaStream_t)stream);
}

}  // extern "C"

namespace {
lgf_status kernel_apply(lgf_ctx *ctx, double kalpha, const lgf_blockset *src, const lgf_blockset *tgt,
                        const void *f_dev, void *u_dev, int32_t ncomp, int32_t nrhs, double dx, void *stream)
{
    lgf_status st = enter(ctx);
    if (st != LGF_OK) return st;
    if (!(kalpha >= 0.0) || !std::isfinite(kalpha)) return fail(ctx, LGF_EINVAL, "alpha must be >= 0 and finite");
    if ((st = check_blockset(ctx, src, "source")) != LGF_OK) return st;
    if ((st = check_blockset(ctx, tgt, "target")) != LGF_OK) return st;
    if (src->b != tgt->b) return fail(ctx, LGF_EINVAL, "source and target block edges differ");
    if (!(dx > 0.0) || !std::isfinite(dx)) return fail(ctx, LGF_EINVAL, "dx must be positive and finite");
    if ((st = check_fields(ctx, f_dev, u_dev, ncomp, nrhs, src->nblocks, tgt->nblocks)) != LGF_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int nf = ncomp * nrhs;
    const size_t b3 = (size_t)src->b * src->b * src->b;
    if (tgt->nblocks == 0) return LGF_OK;
    if (src->nblocks == 0) {
        LGF_CUDA(ctx, cudaMemsetAsync(u_dev, 0, (size_t)tgt->nblocks * b3 * nf * elem_size(ctx), s));
        return LGF_OK;
    }
    PreparedPoisson pp;
    if ((st = prepare_poisson(ctx, src, tgt, nf, kalpha, s, &pp)) != LGF_OK) return st;
    return poisson_run(ctx, pp.plan, pp.spec, f_dev, u_dev, nf, dx, s);
}
}  // namespace

extern "C" {

lgf_status lgf_poisson_apply(lgf_ctx *ctx, const lgf_blockset *src, const lgf_blockset *tgt, const void *f_dev,
                             void *u_dev, int32_t ncomp, int32_t nrhs, double dx, void *stream)
{
    return kernel_apply(ctx, 0.0, src, tgt, f_dev, u_dev, ncomp, nrhs, dx, stream);
}

lgf_status lgf_kinv_apply(lgf_ctx *ctx, double alpha, const lgf_blockset *src, const lgf_blockset *tgt,
                          const void *f_dev, void *u_dev, int32_t ncomp, int32_t nrhs, double dx, void *stream)
{
    return kernel_apply(ctx, alpha, src, tgt, f_dev, u_dev, ncomp, nrhs, dx, stream);
}

}  // extern "C"

namespace {
lgf_status curl_apply(lgf_ctx *ctx, int dir, const lgf_blockset *src, const lgf_blockset *tgt, const void *in_dev,
                      void *out_dev, int32_t nrhs, double dx, void *stream)
{
    lgf_status st = enter(ctx);
    if (st != LGF_OK) return st;
    if ((st = check_blockset(ctx, src, "source")) != LGF_OK) return st;
    if ((st = check_blockset(ctx, tgt, "target")) != LGF_OK) return st;
    if (src->b != tgt->b) return fail(ctx, LGF_EINVAL, "source and target block edges differ");
    if (!(dx > 0.0) || !std::isfinite(dx)) return fail(ctx, LGF_EINVAL, "dx must be positive and finite");
    if ((st = check_fields(ctx, in_dev, out_dev, 3, nrhs, src->nblocks, tgt->nblocks)) != LGF_OK) return st;
    if (tgt->nblocks == 0) return LGF_OK;
    CurlPlan *pl = nullptr;
    if ((st = curl_plan(ctx, src, tgt, dir, &pl)) != LGF_OK) return st;
    return curl_run(ctx, pl, in_dev, out_dev, nrhs, dir < 0 ? 1.0 / dx : -1.0 / dx, (cudaStream_t)stream);
}
}  // namespace

extern "C" {

lgf_status lgf_curl(lgf_ctx *ctx, const lgf_blockset *src, const lgf_blockset *tgt, const void *u_dev, void *w_dev,
                    int32_t nrhs, double dx, void *stream)
{
    return curl_apply(ctx, -1, src, tgt, u_dev, w_dev, nrhs, dx, stream);
}

lgf_status lgf_curl_adjoint(lgf_ctx *ctx, const lgf_blockset *src, const lgf_blockset *tgt, const void *w_dev,
                            void *u_dev, int32_t nrhs, double dx, void *stream)
{
    return curl_apply(ctx, 1, src, tgt, w_dev, u_dev, nrhs, dx, stream);
}

lgf_status lgf_velocity_refresh(lgf_ctx *ctx, const lgf_blockset *src, const lgf_blockset *tgt, const void *u_dev,
                                void *u_out_dev, int32_t nrhs, double dx, void *stream)
{
    lgf_status st = enter(ctx);
    if (st != LGF_OK) return st;
    if ((st = check_blockset(ctx, src, "source")) != LGF_OK) return st;
    if ((st = check_blockset(ctx, tgt, "target")) != LGF_OK) return st;
    if (src->b != tgt->b) return fail(ctx, LGF_EINVAL, "source and target block edges differ");
    if (!(dx > 0.0) || !std::isfinite(dx)) return fail(ctx, LGF_EINVAL, "dx must be positive and finite");
    if ((st = check_fields(ctx, u_dev, u_out_dev, 3, nrhs, src->nblocks, tgt->nblocks)) != LGF_OK) return st;
    if (ctx->table_dev == nullptr) return fail(ctx, LGF_ENOTABLE, "lgf_table_build has not been called");
    cudaStream_t s = (cudaStream_t)stream;
    const int b = src->b;
    const size_t b3 = (size_t)b * b * b;
    if (tgt->nblocks == 0) return LGF_OK;
    if (src->nblocks == 0) {
        LGF_CUDA(ctx, cudaMemsetAsync(u_out_dev, 0, (size_t)tgt->nblocks * b3 * 3 * nrhs * elem_size(ctx), s));
        return LGF_OK;
    }
    const std::vector<int32_t> grown = grown_forward(tgt);
    const lgf_blockset tp{b, (int32_t)(grown.size() / 3), grown.data()};
    CurlPlan *pc = nullptr, *pa = nullptr;
    if ((st = curl_plan(ctx, src, src, -1, &pc)) != LGF_OK) return st;
    if ((st = curl_plan(ctx, &tp, tgt, 1, &pa)) != LGF_OK) return st;
    PreparedPoisson pp;
    if ((st = prepare_poisson(ctx, src, &tp, 3 * nrhs, 0.0, s, &pp)) != LGF_OK) return st;
    Scratch &sc = ctx->scr[0];
    const size_t esz = elem_size(ctx);
    if ((st = ensure_scratch(ctx, &sc.E, &sc.e, (size_t)nrhs * 3 * src->nblocks * b3 * esz)) != LGF_OK) return st;
    if ((st = ensure_scratch(ctx, &sc.F, &sc.f, (size_t)nrhs * 3 * tp.nblocks * b3 * esz)) != LGF_OK) return st;
    // w = C u on the source blocks; s = dx^2 G_L * w on the grown targets;
    // u = -C^dagger s on the targets
    if ((st = curl_run(ctx, pc, u_dev, sc.E, nrhs, 1.0 / dx, s)) != LGF_OK) return st;
    if ((st = poisson_run(ctx, pp.plan, pp.spec, sc.E, sc.F, 3 * nrhs, dx, s)) != LGF_OK) return st;
    return curl_run(ctx, pa, sc.F, u_out_dev, nrhs, 1.0 / dx, s);
}

}  // extern "C"

namespace {
// D followed by the blocks at -x, -y, -z of D that are not in D (sorted): the
// cells the gradient on the faces of D reads.
std::vector<int32_t> grown_backward(const lgf_blockset *D)
{
    std::set<std::array<int, 3>> have, extra;
    for (int t = 0; t < D->nblocks; ++t) have.insert({D->coords[3 * t], D->coords[3 * t + 1], D->coords[3 * t + 2]});
    for (auto &c : have)
        for (int k = 0; k < 3; ++k) {
            std::array<int, 3> m = c;
            --m[k];
            if (!have.count(m)) extra.insert(m);
        }
    std::vector<int32_t> v(D->coords, D->coords + 3 * (size_t)D->nblocks);
    for (auto &c : extra) v.insert(v.end(), c.begin(), c.end());
    return v;
}
}  // namespace

extern "C" {

lgf_status lgf_nested_projection_stage(lgf_ctx *ctx, const lgf_stage *st, void *stream)
{
    lgf_status rc = enter(ctx);
    if (rc != LGF_OK) return rc;
    if (!st) return fail(ctx, LGF_EINVAL, "stage: null description");
    const lgf_blockset *D = &st->flow;
    if ((rc = check_blockset(ctx, D, "stage flow set")) != LGF_OK) return rc;
    for (int i = 0; i < 4; ++i)
        if (st->reserved[i] != 0) return fail(ctx, LGF_EINVAL, "stage: reserved fields must be zero");
    if (!(st->dx > 0.0) || !std::isfinite(st->dx)) return fail(ctx, LGF_EINVAL, "dx must be positive and finite");
    if (!(st->alpha >= 0.0) || !std::isfinite(st->alpha)) return fail(ctx, LGF_EINVAL, "alpha must be >= 0 and finite");
    const int64_t nm = st->nmarkers;
    if (nm < 0 || 3 * nm > INT32_MAX) return fail(ctx, LGF_EINVAL, "stage: bad marker count");
    if (nm > 0 && (!st->X_dev || !st->X_prev_dev || !st->ub_dev || !st->W1_dev))
        return fail(ctx, LGF_EINVAL, "stage: null marker array or force factor");
    if (D->nblocks == 0) {
        if (nm > 0 && st->f_dev)
            LGF_CUDA(ctx, cudaMemsetAsync(st->f_dev, 0, (size_t)3 * nm * elem_size(ctx), (cudaStream_t)stream));
        return LGF_OK;
    }
    if (!st->r_dev || !st->u_dev) return fail(ctx, LGF_EINVAL, "stage: null r or u");
    if (ctx->table_dev == nullptr) return fail(ctx, LGF_ENOTABLE, "lgf_table_build has not been called");
    cudaStream_t s = (cudaStream_t)stream;
    const int b = D->b;
    const size_t b3 = (size_t)b * b * b, nD = (size_t)D->nblocks;
    const std::vector<int32_t> dm = grown_backward(D);
    const lgf_blockset Dm{b, (int32_t)(dm.size() / 3), dm.data()};
    // plans: Dbar on D (dir +1), G from the cells of Dm to the faces of D
    // (dir -1), L^{-1} from D to Dm, H = E(alpha) on D, the IB operators on D
    CurlPlan *pdiv = nullptr, *pgrad = nullptr;
    if ((rc = curl_plan(ctx, D, D, 1, &pdiv)) != LGF_OK) return rc;
    if ((rc = curl_plan(ctx, &Dm, D, -1, &pgrad)) != LGF_OK) return rc;
    PreparedPoisson pp;
    if ((rc = prepare_poisson(ctx, D, &Dm, 1, 0.0, s, &pp)) != LGF_OK) return rc;
    PreparedIntf pi;
    if ((rc = prepare_intf(ctx, st->alpha, D, D, 3, s, &pi)) != LGF_OK) return rc;
    IBPlan *pib = nullptr;
    if (nm > 0 && (rc = ib_plan(ctx, D, &pib)) != LGF_OK) return rc;
    // stage buffers: q (cells of D), dd (cells of Dm), v, w, g (faces of D),
    // U, rhs, y, fh (3 nm each), each 256-byte aligned
    const size_t esz = elem_size(ctx);
    auto al = [](size_t n) { return (n + 255) & ~size_t(255); };
    const size_t n_q = al(nD * b3 * esz), n_d = al(Dm.nblocks * b3 * esz), n_v = al(3 * nD * b3 * esz),
                 n_m = al((size_t)3 * nm * esz + 1);
    Scratch &sc = ctx->scr[0];
    if ((rc = ensure_scratch(ctx, &sc.G, &sc.g, n_q + n_d + 3 * n_v + 4 * n_m)) != LGF_OK) return rc;
    unsigned char *base = (unsigned char *)sc.G;
    void *q = base, *dd = base + n_q, *v = base + n_q + n_d, *w = base + n_q + n_d + n_v,
         *g = base + n_q + n_d + 2 * n_v;
    unsigned char *mk = base + n_q + n_d + 3 * n_v;
    void *U = mk, *rhs = mk + n_m, *y = mk + 2 * n_m, *fh = mk + 3 * n_m;
    const double dx = st->dx;
    // ip (Eq. nested_proj-ip): L_C d* = -G^dagger r = Dbar r
    if ((rc = stage_div(ctx, pdiv, st->r_dev, nullptr, q, dx, s)) != LGF_OK) return rc;
    if ((rc = poisson_run(ctx, pp.plan, pp.spec, q, dd, 1, dx, s)) != LGF_OK) return rc;
    const void *gforce = nullptr;
    if (nm > 0) {
        // f (Eq. nested_proj-f): C f_hat = I^i H [r - G d*] - u_Gamma, f_hat = W2 (W1 rhs)
        if ((rc = stage_grad(ctx, pgrad, dd, st->r_dev, nullptr, v, dx, s)) != LGF_OK) return rc;
        if ((rc = intf_run(ctx, pi.plan, pi.w, v, w, 3, s)) != LGF_OK) return rc;
        if ((rc = ib_run(ctx, pib, false, nm, st->X_dev, w, U, 1, 1.0, s)) != LGF_OK) return rc;
        if ((rc = stage_force(ctx, U, st->ub_dev, st->W1_dev, st->W2_dev, rhs, y, fh, (int)(3 * nm), s)) != LGF_OK)
            return rc;
        // (I^{i-1})^dagger f_hat = dx^3 R f_hat: the bare kernel sum (R at dx = 1)
        if ((rc = ib_run(ctx, pib, true, nm, st->X_prev_dev, fh, g, 1, 1.0, s)) != LGF_OK) return rc;
        gforce = g;
        // pc (Eq. nested_proj-pc): d_hat = d* + L_C^{-1} G^dagger g = L_C^{-1} Dbar (r - g)
        // (one Poisson apply of the summed source, by linearity)
        if ((rc = stage_div(ctx, pdiv, st->r_dev, g, q, dx, s)) != LGF_OK) return rc;
        if ((rc = poisson_run(ctx, pp.plan, pp.spec, q, dd, 1, dx, s)) != LGF_OK) return rc;
        if (st->f_dev) LGF_CUDA(ctx, cudaMemcpyAsync(st->f_dev, fh, 3 * nm * esz, cudaMemcpyDeviceToDevice, s));
    }
    // vc (Eq. nested_proj-vc): u = H [r - G d_hat - g]
    if ((rc = stage_grad(ctx, pgrad, dd, st->r_dev, gforce, v, dx, s)) != LGF_OK) return rc;
    if ((rc = intf_run(ctx, pi.plan, pi.w, v, st->u_dev, 3, s)) != LGF_OK) return rc;
    if (st->d_dev) LGF_CUDA(ctx, cudaMemcpyAsync(st->d_dev, dd, nD * b3 * esz, cudaMemcpyDeviceToDevice, s));
    return LGF_OK;
}

}  // extern "C"

namespace {
lgf_status ib_apply(lgf_ctx *ctx, bool spread, const lgf_blockset *set, int64_t nmarkers, const double *X_dev,
                    const void *in_dev, void *out_dev, int32_t nrhs, double dx, void *stream)
{
    lgf_status st = enter(ctx);
    if (st != LGF_OK) return st;
    if ((st = check_blockset(ctx, set, "block set")) != LGF_OK) return st;
    if (nrhs < 1) return fail(ctx, LGF_EINVAL, "nrhs must be >= 1");
    if (nmarkers < 0 || (nmarkers > 0 && !X_dev)) return fail(ctx, LGF_EINVAL, "IB: bad marker arrays");
    if (!(dx > 0.0) || !std::isfinite(dx)) return fail(ctx, LGF_EINVAL, "dx must be positive and finite");
    const bool has_out = spread ? set->nblocks > 0 : nmarkers > 0;
    if (has_out && !out_dev) return fail(ctx, LGF_EINVAL, "null output pointer");
    const bool reads_in = spread ? nmarkers > 0 : (set->nblocks > 0 && nmarkers > 0);
    if (reads_in && !in_dev) return fail(ctx, LGF_EINVAL, "null input pointer");
    cudaStream_t s = (cudaStream_t)stream;
    if (set->nblocks == 0) {
        if (!spread && nmarkers > 0)
            LGF_CUDA(ctx, cudaMemsetAsync(out_dev, 0, (size_t)nrhs * 3 * nmarkers * elem_size(ctx), s));
        return LGF_OK;
    }
    IBPlan *pl = nullptr;
    if ((st = ib_plan(ctx, set, &pl)) != LGF_OK) return st;
    return ib_run(ctx, pl, spread, nmarkers, X_dev, in_dev, out_dev, nrhs, dx, s);
}
}  // namespace

extern "C" {

lgf_status lgf_ib_spread(lgf_ctx *ctx, const lgf_blockset *set, int64_t nmarkers, const double *X_dev,
                         const void *g_dev, void *f_dev, int32_t nrhs, double dx, void *stream)
{
    return ib_apply(ctx, true, set, nmarkers, X_dev, g_dev, f_dev, nrhs, dx, stream);
}

lgf_status lgf_ib_interp(lgf_ctx *ctx, const lgf_blockset *set, int64_t nmarkers, const double *X_dev,
                         const void *v_dev, void *U_dev, int32_t nrhs, void *stream)
{
    return ib_apply(ctx, false, set, nmarkers, X_dev, v_dev, U_dev, nrhs, 1.0, stream);
}

lgf_status lgf_intfactor_weights(lgf_ctx *ctx, double alpha, double *w_dev, int32_t cap, int32_t *radius,
                                 void *stream)
{
    lgf_status st = enter(ctx);
    if (st != LGF_OK) return st;
    if (!(alpha >= 0.0) || !std::isfinite(alpha)) return fail(ctx, LGF_EINVAL, "alpha must be >= 0 and finite");
    IntfWeights *w = nullptr;
    if ((st = intf_weights(ctx, alpha, &w, (cudaStream_t)stream)) != LGF_OK) return st;
    if (radius) *radius = w->R;
    if (w_dev) {
        if (cap <= w->R) return fail(ctx, LGF_EINVAL, "intfactor_weights: cap must exceed the radius");
        LGF_CUDA(ctx, cudaMemcpyAsync(w_dev, w->w64, (w->R + 1) * sizeof(double), cudaMemcpyDeviceToDevice,
                                      (cudaStream_t)stream));
    }
    return LGF_OK;
}

lgf_status lgf_intfactor_apply(lgf_ctx *ctx, double alpha, const lgf_blockset *src, const lgf_blockset *tgt,
                               const void *f_dev, void *u_dev, int32_t ncomp, int32_t nrhs, void *stream)
{
    lgf_status st = enter(ctx);
    if (st != LGF_OK) return st;
    if (!(alpha >= 0.0) || !std::isfinite(alpha)) return fail(ctx, LGF_EINVAL, "alpha must be >= 0 and finite");
    if ((st = check_blockset(ctx, src, "source")) != LGF_OK) return st;
    if ((st = check_blockset(ctx, tgt, "target")) != LGF_OK) return st;
    if (src->b != tgt->b) return fail(ctx, LGF_EINVAL, "source and target block edges differ");
    if ((st = check_fields(ctx, f_dev, u_dev, ncomp, nrhs, src->nblocks, tgt->nblocks)) != LGF_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int nf = ncomp * nrhs;
    const size_t b3 = (size_t)src->b * src->b * src->b;
    if (tgt->nblocks == 0) return LGF_OK;
    if (src->nblocks == 0) {
        LGF_CUDA(ctx, cudaMemsetAsync(u_dev, 0, (size_t)tgt->nblocks * b3 * nf * elem_size(ctx), s));
        return LGF_OK;
    }
    PreparedIntf pi;
    if ((st = prepare_intf(ctx, alpha, src, tgt, nf, s, &pi)) != LGF_OK) return st;
    return intf_run(ctx, pi.plan, pi.w, f_dev, u_dev, nf, s);
}

lgf_status lgf_residual(lgf_ctx *ctx, const lgf_blockset *set, const void *u_dev, const void *f_dev, double dx,
                        double *r_dev, double *max_abs, double *max_f, void *stream)
{
    lgf_status st = enter(ctx);
    if (st != LGF_OK) return st;
    if ((st = check_blockset(ctx, set, "set")) != LGF_OK) return st;
    if (!(dx > 0.0) || !std::isfinite(dx)) return fail(ctx, LGF_EINVAL, "dx must be positive and finite");
    if (set->nblocks > 0 && (!u_dev || !f_dev || !r_dev)) return fail(ctx, LGF_EINVAL, "null field pointer");
    return residual_run(ctx, set, u_dev, f_dev, dx, r_dev, max_abs, max_f, (cudaStream_t)stream);
}

lgf_status lgf_profile_enable(lgf_ctx *ctx, int32_t enable)
{
    lgf_status st = enter(ctx);
    if (st != LGF_OK) return st;
    LGF_CUDA(ctx, cudaDeviceSynchronize());
    for (auto &r : ctx->prof_pending) {
        ctx->ev_pool.push_back(r.a);
        ctx->ev_pool.push_back(r.b);
    }
    ctx->prof_pending.clear();
    ctx->prof_names.clear();
    ctx->prof_launches.clear();
    ctx->prof_ms.clear();
    ctx->prof = enable != 0;
    return LGF_OK;
}

lgf_status lgf_profile_read(lgf_ctx *ctx, lgf_kernel_stat *out, int32_t cap, int32_t *n)
{
    lgf_status st = enter(ctx);
    if (st != LGF_OK) return st;
    if (cap < 0 || (cap > 0 && !out) || !n) return fail(ctx, LGF_EINVAL, "profile_read: bad arguments");
    LGF_CUDA(ctx, cudaDeviceSynchronize());
    for (auto &r : ctx->prof_pending) {
        float ms = 0.f;
        LGF_CUDA(ctx, cudaEventElapsedTime(&ms, r.a, r.b));
        ctx->prof_launches[r.name] += 1;
        ctx->prof_ms[r.name] += ms;
        ctx->ev_pool.push_back(r.a);
        ctx->ev_pool.push_back(r.b);
    }
    ctx->prof_pending.clear();
    const int k = (int)ctx->prof_names.size();
    *n = k;
    for (int i = 0; i < k && i < cap; ++i) {
        memset(&out[i], 0, sizeof(out[i]));
        strncpy(out[i].name, ctx->prof_names[i].c_str(), sizeof(out[i].name) - 1);
        out[i].launches = ctx->prof_launches[i];
        out[i].total_ms = ctx->prof_ms[i];
    }
    for (int i = 0; i < k; ++i) {
        ctx->prof_launches[i] = 0;
        ctx->prof_ms[i] = 0.0;
    }
    return LGF_OK;
}

lgf_status lgf_batch_apply(lgf_ctx *ctx, const lgf_problem *probs, int32_t nprob, void *stream)
{
    lgf_status st = enter(ctx);
    if (st != LGF_OK) return st;
    if (nprob < 0 || (nprob > 0 && !probs)) return fail(ctx, LGF_EINVAL, "batch: bad problem list");
    cudaStream_t s = (cudaStream_t)stream;
    // 1. validate and build a key of everything that shapes the work
    std::vector<unsigned char> key, shape;   // shape: the key without buffers and stream
    auto put = [&](const void *p, size_t n) {
        const unsigned char *c = (const unsigned char *)p;
        key.insert(key.end(), c, c + n);
    };
    auto put_shape = [&](const void *p, size_t n) {
        const unsigned char *c = (const unsigned char *)p;
        shape.insert(shape.end(), c, c + n);
    };
    for (int i = 0; i < nprob; ++i) {
        const lgf_problem &p = probs[i];
        if ((st = check_blockset(ctx, &p.src, "batch source")) != LGF_OK) return st;
        if ((st = check_blockset(ctx, &p.tgt, "batch target")) != LGF_OK) return st;
        if (p.src.b != p.tgt.b) return fail(ctx, LGF_EINVAL, "batch: block edges differ");
        if (p.op < LGF_OP_POISSON || p.op > LGF_OP_KINV || p.reserved != 0)
            return fail(ctx, LGF_EINVAL, "batch: unknown operation");
        if (p.op != LGF_OP_POISSON && (!(p.alpha >= 0.0) || !std::isfinite(p.alpha)))
            return fail(ctx, LGF_EINVAL, "batch: alpha must be >= 0 and finite");
        if (p.op != LGF_OP_INTFACTOR && (!(p.dx > 0.0) || !std::isfinite(p.dx)))
            return fail(ctx, LGF_EINVAL, "batch: dx must be positive and finite");
        if ((st = check_fields(ctx, p.f_dev, p.u_dev, p.ncomp, p.nrhs, p.src.nblocks, p.tgt.nblocks)) != LGF_OK)
            return st;
        put(&p.src.b, sizeof(int32_t));
        put(&p.src.nblocks, sizeof(int32_t));
        put(p.src.coords, 3 * sizeof(int32_t) * (size_t)p.src.nblocks);
        put(&p.tgt.nblocks, sizeof(int32_t));
        put(p.tgt.coords, 3 * sizeof(int32_t) * (size_t)p.tgt.nblocks);
        put(&p.f_dev, sizeof(void *));
        put(&p.u_dev, sizeof(void *));
        put(&p.ncomp, 4 * sizeof(int32_t));
        put(&p.alpha, 2 * sizeof(double));
        put_shape(&p.src.b, sizeof(int32_t));
        put_shape(&p.src.nblocks, sizeof(int32_t));
        put_shape(p.src.coords, 3 * sizeof(int32_t) * (size_t)p.src.nblocks);
        put_shape(&p.tgt.nblocks, sizeof(int32_t));
        put_shape(p.tgt.coords, 3 * sizeof(int32_t) * (size_t)p.tgt.nblocks);
        put_shape(&p.ncomp, 4 * sizeof(int32_t));
        put_shape(&p.alpha, 2 * sizeof(double));
    }
    put(&s, sizeof(s));
    // 2. prepare every plan, spectrum, weight set and the largest scratch;
    //    integrating factors on the same block sets (and field count) form one
    //    group that runs as one launch per pass
    std::vector<PreparedPoisson> pois(nprob);
    struct Group {
        IntfPlan *plan;
        int nf;
        bool after_poisson;   // reads outputs of the batch's Poisson parts
        std::vector<IntfJob> jobs;
        std::vector<int> prob;    // problem of each job
    };
    std::vector<Group> groups;
    for (int i = 0; i < nprob; ++i) {
        const lgf_problem &p = probs[i];
        const int nf = p.ncomp * p.nrhs;
        if (p.tgt.nblocks == 0 || p.src.nblocks == 0) continue;
        if (p.op != LGF_OP_INTFACTOR) {
            const double kalpha = p.op == LGF_OP_KINV ? p.alpha : 0.0;
            if ((st = prepare_poisson(ctx, &p.src, &p.tgt, nf, kalpha, s, &pois[i])) != LGF_OK) return st;
        }
        if (p.op == LGF_OP_POISSON || p.op == LGF_OP_KINV) continue;
        PreparedIntf pi;
        const lgf_blockset *isrc = p.op == LGF_OP_INTFACTOR ? &p.src : &p.tgt;
        if ((st = prepare_intf(ctx, p.alpha, isrc, &p.tgt, nf, s, &pi)) != LGF_OK) return st;
        const void *in = p.op == LGF_OP_INTFACTOR ? p.f_dev : p.u_dev;
        const bool after = p.op == LGF_OP_POISSON_THEN_INTFACTOR;
        Group *g = nullptr;
        for (auto &q : groups)
            if (q.plan == pi.plan && q.nf == nf && q.after_poisson == after) g = &q;
        if (!g) {
            groups.push_back(Group{pi.plan, nf, after, {}, {}});
            g = &groups.back();
        }
        g->jobs.push_back(IntfJob{pi.w, in, p.u_dev});
        g->prob.push_back(i);
    }
    // 3. units of concurrent work: every Poisson part (with its dependent
    //    integrating factor when no other problem shares that group) and every
    //    integrating-factor group that reads only batch inputs.  Dependent
    //    groups of several problems run after the join.  Units go to up to
    //    kBranches branches (longest first onto the least loaded), each branch
    //    with its own stream and scratch.
    struct Unit {
        int prob = -1, grp = -1, dep = -1, branch = 0;
        double cost = 0.0;
    };
    std::vector<Unit> units;
    std::vector<int> prob_unit(nprob, -1), post;
    auto grp_cost = [&](const Group &g) {
        const double b3 = (double)g.plan->b * g.plan->b * g.plan->b;
        return 8.0 * g.jobs.size() * g.nf * b3 * ((double)g.plan->n2 + (double)g.plan->tgt.size() / 3);
    };
    for (int i = 0; i < nprob; ++i) {
        if (!pois[i].plan) continue;
        const int *M = pois[i].plan->g.M;
        Unit u;
        u.prob = i;
        u.cost = 3.0 * (double)M[0] * M[1] * M[2] * probs[i].ncomp * probs[i].nrhs;
        prob_unit[i] = (int)units.size();
        units.push_back(u);
    }
    for (size_t k = 0; k < groups.size(); ++k) {
        const Group &g = groups[k];
        if (!g.after_poisson) {
            Unit u;
            u.grp = (int)k;
            u.cost = grp_cost(g);
            units.push_back(u);
        } else if (g.jobs.size() == 1 && prob_unit[g.prob[0]] >= 0) {
            Unit &u = units[prob_unit[g.prob[0]]];
            u.dep = (int)k;
            u.cost += grp_cost(g);
        } else {
            post.push_back((int)k);
        }
    }
    const int nb_max = std::min<int>(kBranches, std::max<int>(1, (int)units.size()));
    int nb = ctx->prof ? 1 : std::min(nb_max, kDefaultBranches);
    // Ragged mode: all Poisson parts together, one launch per pass and
    // transform length (poisson_run_ragged), then every integrating-factor
    // group, the groups spread over the branches.
    std::vector<RagPart> parts;
    for (int i = 0; i < nprob; ++i)
        if (pois[i].plan)
            parts.push_back(RagPart{pois[i].plan, pois[i].spec, probs[i].f_dev, probs[i].u_dev,
                                    probs[i].ncomp * probs[i].nrhs, probs[i].dx});
    // (the default for batches of several Poisson parts, or on request)
    bool rag = !ctx->opt_units && ((ctx->opt_rag && !parts.empty()) || parts.size() >= 2);
    // (the ragged mode's length groups of a pass on 2 branches by default:
    // on the 64-plate batch 2 branches ran 1.7 % faster than 4, 8 and 1 slower)
    constexpr int kRagBranches = 2;
    if (rag && !ctx->prof) nb = kRagBranches;
    // integrating-factor groups of the ragged mode: those that read the
    // batch's Poisson results (after the Poisson passes, scratch of branch 0)
    // and those that read only batch inputs (alongside the Poisson passes on
    // the last branch, with its scratch)
    std::vector<IntfGroupRef> grefs_dep, grefs_ind;
    for (auto &g : groups)
        (g.after_poisson ? grefs_dep : grefs_ind)
            .push_back(IntfGroupRef{g.plan, g.jobs.data(), (int)g.jobs.size(), g.nf});
    Scratch *const scr_ind = &ctx->scr[kBranches - 1];
    auto make_branches = [&](int nbv) -> lgf_status {
        if (nbv > 1) {
            if (!ctx->ev_fork) LGF_CUDA(ctx, cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
            for (int b = 0; b < nbv; ++b) {
                if (!ctx->br[b]) LGF_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->br[b], cudaStreamNonBlocking));
                if (!ctx->ev_join[b])
                    LGF_CUDA(ctx, cudaEventCreateWithFlags(&ctx->ev_join[b], cudaEventDisableTiming));
            }
        }
        return LGF_OK;
    };
    auto setup_rag = [&](int nbv) -> lgf_status {
        lgf_status e2 = poisson_ragged_scratch(ctx, parts.data(), (int)parts.size());
        if (e2 == LGF_OK) e2 = intf_ragged_scratch(ctx, grefs_dep.data(), (int)grefs_dep.size(), &ctx->scr[0]);
        if (e2 == LGF_OK) e2 = intf_ragged_scratch(ctx, grefs_ind.data(), (int)grefs_ind.size(), scr_ind);
        if (e2 != LGF_OK) return e2;
        return make_branches(grefs_ind.empty() ? nbv : kBranches);
    };
    // units onto nbv branches (longest first onto the least loaded), each
    // branch's scratch grown for its units, its stream and events made
    auto setup = [&](int nbv) -> lgf_status {
        if (rag) return setup_rag(nbv);
        std::vector<int> order(units.size());
        for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
        std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return units[a].cost > units[c].cost; });
        double load[kBranches] = {};
        for (int i : order) {
            int best = 0;
            for (int b = 1; b < nbv; ++b)
                if (load[b] < load[best]) best = b;
            units[i].branch = best;
            load[best] += units[i].cost;
        }
        lgf_status e2 = LGF_OK;
        for (auto &u : units) {
            ctx->cur = &ctx->scr[u.branch];
            const int i = u.prob;
            if (i >= 0 && (e2 = poisson_prepare_scratch(ctx, pois[i].plan, probs[i].ncomp * probs[i].nrhs)) != LGF_OK)
                break;
            for (int k : {u.grp, u.dep}) {
                if (k < 0 || e2 != LGF_OK) continue;
                const Group &g = groups[k];
                e2 = intf_prepare_scratch(ctx, g.plan, g.nf, (int)g.jobs.size());
            }
            if (e2 != LGF_OK) break;
        }
        ctx->cur = &ctx->scr[0];
        if (e2 != LGF_OK) return e2;
        for (int k : post)
            if ((e2 = intf_prepare_scratch(ctx, groups[k].plan, groups[k].nf, (int)groups[k].jobs.size())) != LGF_OK)
                return e2;
        return make_branches(nbv);
    };
    if ((st = setup(nb)) != LGF_OK) return st;
    auto enqueue = [&]() -> lgf_status {
        // problems with no source blocks: zero output
        for (int i = 0; i < nprob; ++i) {
            const lgf_problem &p = probs[i];
            const size_t b3 = (size_t)p.src.b * p.src.b * p.src.b;
            if (p.tgt.nblocks > 0 && p.src.nblocks == 0)
                LGF_CUDA(ctx, cudaMemsetAsync(p.u_dev, 0,
                                              (size_t)p.tgt.nblocks * b3 * p.ncomp * p.nrhs * elem_size(ctx), s));
        }
        if (rag) {
            const bool side = !grefs_ind.empty() && !parts.empty() && nb > 1;
            cudaStream_t si = side ? ctx->br[kBranches - 1] : s;
            if (side) {
                LGF_CUDA(ctx, cudaEventRecord(ctx->ev_fork, s));
                LGF_CUDA(ctx, cudaStreamWaitEvent(si, ctx->ev_fork, 0));
            }
            lgf_status e2 = intf_run_ragged(ctx, grefs_ind.data(), (int)grefs_ind.size(), si, scr_ind);
            if (e2 == LGF_OK) e2 = poisson_run_ragged(ctx, parts.data(), (int)parts.size(), s, nb);
            if (e2 == LGF_OK) e2 = intf_run_ragged(ctx, grefs_dep.data(), (int)grefs_dep.size(), s, &ctx->scr[0]);
            if (e2 != LGF_OK) return e2;
            if (side) {
                LGF_CUDA(ctx, cudaEventRecord(ctx->ev_join[kBranches - 1], si));
                LGF_CUDA(ctx, cudaStreamWaitEvent(s, ctx->ev_join[kBranches - 1], 0));
            }
            return LGF_OK;
        }
        if (nb > 1) {
            LGF_CUDA(ctx, cudaEventRecord(ctx->ev_fork, s));
            for (int b = 0; b < nb; ++b) LGF_CUDA(ctx, cudaStreamWaitEvent(ctx->br[b], ctx->ev_fork, 0));
        }
        for (auto &u : units) {
            cudaStream_t us = nb > 1 ? ctx->br[u.branch] : s;
            ctx->cur = &ctx->scr[u.branch];
            lgf_status e2 = LGF_OK;
            if (u.prob >= 0) {
                const lgf_problem &p = probs[u.prob];
                e2 = poisson_run(ctx, pois[u.prob].plan, pois[u.prob].spec, p.f_dev, p.u_dev, p.ncomp * p.nrhs, p.dx,
                                 us);
            }
            for (int k : {u.dep, u.grp}) {
                if (e2 != LGF_OK || k < 0) continue;
                const Group &g = groups[k];
                e2 = intf_run_jobs(ctx, g.plan, g.jobs.data(), (int)g.jobs.size(), g.nf, us);
            }
            if (e2 != LGF_OK) {
                ctx->cur = &ctx->scr[0];
                return e2;
            }
        }
        ctx->cur = &ctx->scr[0];
        if (nb > 1)
            for (int b = 0; b < nb; ++b) {
                LGF_CUDA(ctx, cudaEventRecord(ctx->ev_join[b], ctx->br[b]));
                LGF_CUDA(ctx, cudaStreamWaitEvent(s, ctx->ev_join[b], 0));
            }
        for (int k : post) {
            const Group &g = groups[k];
            lgf_status e2 = intf_run_jobs(ctx, g.plan, g.jobs.data(), (int)g.jobs.size(), g.nf, s);
            if (e2 != LGF_OK) return e2;
        }
        return LGF_OK;
    };
    // 4. the execution of this batch shape: the persisted choice, or (tuning
    //    on, a new shape) the fastest of 1, 2, 4 and 8 branches of per-problem
    //    launches and of the ragged mode on 2 or 4 branches, timed with direct
    //    launches on the caller's stream (the default first: the others must
    //    win by 3 %)
    if (ctx->tune_mode != LGF_TUNE_OFF && !ctx->prof && s != nullptr && nb_max > 1) {
        const std::string tk = tune_batch_key(ctx->prec == LGF_F64, tune_hash(shape.data(), shape.size()));
        auto it = ctx->tune_db.find(tk);
        int pick = 0;
        if (it != ctx->tune_db.end() && std::sscanf(it->second.c_str(), "nb%d", &pick) == 1 && pick >= 1 &&
            pick <= nb_max) {
            nb = pick;
            rag = false;
        } else if (it != ctx->tune_db.end() && std::sscanf(it->second.c_str(), "rg%d", &pick) == 1 && pick >= 1 &&
                   pick <= kBranches) {
            rag = true;
            nb = pick;
        } else if (ctx->tune_mode == LGF_TUNE_ON) {
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            LGF_CUDA(ctx, cudaEventCreate(&e0));
            LGF_CUDA(ctx, cudaEventCreate(&e1));
            float tbest = 0.f;
            int best = nb;
            bool best_rag = false;
            // the default first: the others must beat it by 3 %
            struct Cand {
                bool rag;
                int nb;
            };
            static constexpr Cand kRagFirst[6] = {{true, kRagBranches}, {true, 4}, {false, 4},
                                                  {false, 8}, {false, 2}, {false, 1}};
            static constexpr Cand kUnitsFirst[6] = {{false, 4}, {false, 8}, {false, 2},
                                                    {false, 1}, {true, kRagBranches}, {true, 4}};
            const Cand *cands = rag ? kRagFirst : kUnitsFirst;
            for (int ci = 0; ci < 6; ++ci) {
                const bool crag = cands[ci].rag;
                const int cand = cands[ci].nb;
                if (!crag && cand > nb_max) continue;
                if (crag && parts.empty()) continue;
                rag = crag;
                if ((st = setup(cand)) != LGF_OK) break;
                nb = cand;
                std::vector<float> t;
                for (int r = 0; r < 3 && st == LGF_OK; ++r) {
                    cudaEventRecord(e0, s);
                    st = enqueue();
                    cudaEventRecord(e1, s);
                    float v = 0.f;
                    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&v, e0, e1) != cudaSuccess)
                        st = fail(ctx, LGF_ECUDA, "batch: branch timing");
                    if (r > 0) t.push_back(v);
                }
                if (st != LGF_OK) break;
                const float tm = std::min(t[0], t[1]);
                ctx->tune_candidates++;
                if (tbest == 0.f || tm < 0.97f * tbest) {   // later candidates must win by 3 %
                    tbest = tm;
                    best = cand;
                    best_rag = crag;
                }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if (st != LGF_OK) return st;
            nb = best;
            rag = best_rag;
            ++ctx->tune_batches;
            tune_record(ctx, tk, (rag ? "rg" : "nb") + std::to_string(nb));
        }
        if ((st = setup(nb)) != LGF_OK) return st;
    }
    ctx->tune_last_branches = nb;
    ctx->tune_last_ragged = rag ? 1 : 0;
    // 5. the legacy default stream cannot be captured, and per-kernel timing
    //    needs direct launches: run without a graph
    //    (and so does a context whose graph cache is switched off)
    if (s == nullptr || ctx->prof || ctx->graphs.cap() == 0) return enqueue();
    // every buffer the batch needs has its final address now (the prepare
    // step above grew the scratch, which dropped any graph holding an older
    // address), so a cached graph of this key is safe to replay
    if (cudaGraphExec_t *g = ctx->graphs.find(key, ++ctx->graph_clock)) {
        LGF_CUDA(ctx, cudaGraphLaunch(*g, s));
        return LGF_OK;
    }
    ctx->graphs.make_room([](cudaGraphExec_t g) { cudaGraphExecDestroy(g); }, &ctx->counters);
    LGF_CUDA(ctx, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    lgf_status est = enqueue();
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &graph);
    if (est != LGF_OK) {
        if (graph) cudaGraphDestroy(graph);
        return est;
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batch: stream capture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batch: graph instantiation");
    ctx->graphs.add(std::move(key), exec, ++ctx->graph_clock);
    LGF_CUDA(ctx, cudaGraphLaunch(exec, s));
    return LGF_OK;
}

lgf_status lgf_poisson_error_estimate(lgf_ctx *ctx, const lgf_blockset *src, const lgf_blockset *tgt,
                                      const void *f_dev, const void *u_dev, int32_t ncomp, int32_t nrhs, double dx,
                                      int32_t nsample, double *max_rel_err, void *stream)
{
    lgf_status st = enter(ctx);
    if (st != LGF_OK) return st;
    if ((st = check_blockset(ctx, src, "source")) != LGF_OK) return st;
    if ((st = check_blockset(ctx, tgt, "target")) != LGF_OK) return st;
    if (src->b != tgt->b) return fail(ctx, LGF_EINVAL, "source and target block edges differ");
    if (!(dx > 0.0) || !std::isfinite(dx)) return fail(ctx, LGF_EINVAL, "dx must be positive and finite");
    if ((st = check_fields(ctx, f_dev, const_cast<void *>(u_dev), ncomp, nrhs, src->nblocks, tgt->nblocks)) !=
        LGF_OK)
        return st;
    if (nsample < 1 || nsample > 65536 || !max_rel_err) return fail(ctx, LGF_EINVAL, "error estimate: nsample 1..65536");
    if (!ctx->table_dev) return fail(ctx, LGF_ENOTABLE, "lgf_table_build has not been called");
    *max_rel_err = 0.0;
    if (tgt->nblocks == 0 || src->nblocks == 0) return LGF_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int b = tgt->b;
    const int64_t b3 = (int64_t)b * b * b, ntot = (int64_t)tgt->nblocks * b3;
    const int n = (int)std::min<int64_t>(nsample, ntot);
    // evenly spread target points, in the field's element order
    std::vector<int64_t> idx(n);
    std::vector<int32_t> pts(3 * (size_t)n);
    for (int k = 0; k < n; ++k) {
        const int64_t i = std::min<int64_t>(ntot - 1, (int64_t)(((double)k + 0.5) * (double)ntot / n));
        idx[k] = i;
        const int64_t blk = i / b3, loc = i % b3;
        pts[3 * k] = tgt->coords[3 * blk] * b + (int)(loc % b);
        pts[3 * k + 1] = tgt->coords[3 * blk + 1] * b + (int)((loc / b) % b);
        pts[3 * k + 2] = tgt->coords[3 * blk + 2] * b + (int)(loc / ((int64_t)b * b));
    }
    const size_t esz = elem_size(ctx);
    std::vector<double> ref(n), got(n);
    double worst = 0.0;
    for (int fld = 0; fld < ncomp * nrhs; ++fld) {
        const void *ff = (const unsigned char *)f_dev + (size_t)fld * src->nblocks * b3 * esz;
        const void *uf = (const unsigned char *)u_dev + (size_t)fld * ntot * esz;
        if ((st = direct_samples(ctx, src, ff, pts.data(), n, dx, ref.data(), s)) != LGF_OK) return st;
        if ((st = gather_values(ctx, uf, idx.data(), n, got.data(), s)) != LGF_OK) return st;
        double num = 0.0, den = 0.0;
        for (int k = 0; k < n; ++k) {
            num = std::max(num, std::fabs(got[k] - ref[k]));
            den = std::max(den, std::fabs(ref[k]));
        }
        if (den > 0.0) worst = std::max(worst, num / den);
    }
    *max_rel_err = worst;
    return LGF_OK;
}

lgf_status lgf_table_save(lgf_ctx *ctx, const char *path)
{
    lgf_status st = enter(ctx);
    if (st != LGF_OK) return st;
    if (!path) return fail(ctx, LGF_EINVAL, "table_save: null path");
    if (!ctx->table_dev) return fail(ctx, LGF_ENOTABLE, "table not built");
    return table_save(ctx, path);
}

lgf_status lgf_table_load(lgf_ctx *ctx, const char *path)
{
    lgf_status st = enter(ctx);
    if (st != LGF_OK) return st;
    if (!path) return fail(ctx, LGF_EINVAL, "table_load: null path");
    before_evict(ctx);   // spectra, G_K tables and graphs built from the old table go
    if ((st = table_load(ctx, path)) != LGF_OK) return st;
    ctx->spectra.clear();
    for (auto &kv : ctx->gk_tables) cudaFree(kv.second);
    ctx->gk_tables.clear();
    return LGF_OK;
}

lgf_status lgf_device_status(lgf_ctx *ctx, int32_t *word)
{
    lgf_status st = enter(ctx);
    if (st != LGF_OK) return st;
    LGF_CUDA(ctx, cudaDeviceSynchronize());
    int w = 0;
    LGF_CUDA(ctx, cudaMemcpy(&w, ctx->err_dev, sizeof(int), cudaMemcpyDeviceToHost));
    LGF_CUDA(ctx, cudaMemset(ctx->err_dev, 0, sizeof(int)));
    if (word) *word = w;
    if (w != 0) return fail(ctx, LGF_ETIMEOUT, "a bounded device-side wait ran out (error word " + std::to_string(w) + ")");
    return LGF_OK;
}

lgf_status lgf_wait_selftest(lgf_ctx *ctx, int64_t cycles, void *stream)
{
    lgf_status st = enter(ctx);
    if (st != LGF_OK) return st;
    if (cycles < 1 || cycles > 4000000000LL) return fail(ctx, LGF_EINVAL, "wait_selftest: cycles in [1, 4e9]");
    return wait_selftest(ctx, cycles, (cudaStream_t)stream);
}

lgf_status lgf_autotune(lgf_ctx *ctx, int32_t mode, const char *cache_path)
{
    lgf_status st = enter(ctx);
    if (st != LGF_OK) return st;
    if (mode != LGF_TUNE_OFF && mode != LGF_TUNE_ON && mode != LGF_TUNE_CACHED)
        return fail(ctx, LGF_EINVAL, "autotune: mode must be LGF_TUNE_OFF, LGF_TUNE_ON or LGF_TUNE_CACHED");
    ctx->tune_mode = mode;
    const char *path = cache_path ? cache_path : std::getenv("LGF_TUNE_CACHE");
    ctx->tune_path = path ? path : "";
    if (!ctx->tune_path.empty()) {
        if (FILE *f = std::fopen(ctx->tune_path.c_str(), "r")) {
            std::string text;
            char buf[4096];
            size_t n;
            while ((n = std::fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, n);
            std::fclose(f);
            tune_parse(text, &ctx->tune_db);
        }
    }
    return LGF_OK;
}

lgf_status lgf_tune_report(lgf_ctx *ctx, lgf_tune_info *out)
{
    if (!ctx || !out) return LGF_EINVAL;
    memset(out, 0, sizeof(*out));
    out->plans_tuned = ctx->tune_plans;
    out->plans_from_cache = ctx->tune_plans_cached;
    out->candidates_timed = ctx->tune_candidates;
    out->batches_tuned = ctx->tune_batches;
    out->last_branches = ctx->tune_last_branches;
    out->last_ragged = ctx->tune_last_ragged;
    out->tune_ms = ctx->tune_ms;
    for (auto &p : ctx->pplans.items()) {
        out->shifted_x += p->choice.shift[0];
        out->shifted_y += p->choice.shift[1];
        out->longer_x += p->choice.bump[0] > 0;
        out->longer_y += p->choice.bump[1] > 0;
        out->longer_z += p->choice.bump[2] > 0;
        out->z_variant += p->choice.zvar;
        int rpb = 0;
        out->fused_inverse += ctx->prec == LGF_F32 && poisson_fused_ncl(p->g, &rpb) > 0;
    }
    return LGF_OK;
}

lgf_status lgf_ctx_stats(lgf_ctx *ctx, lgf_stats *out)
{
    if (!ctx || !out) return LGF_EINVAL;
    memset(out, 0, sizeof(*out));
    out->graphs_cached = (int64_t)ctx->graphs.size();
    out->poisson_plans = (int64_t)ctx->pplans.size();
    out->intfactor_plans = (int64_t)ctx->iplans.size();
    out->curl_plans = (int64_t)ctx->cplans.size();
    out->ib_plans = (int64_t)ctx->ibplans.size();
    out->spectra = (int64_t)ctx->spectra.size();
    out->generation = (int64_t)ctx->counters.generation;
    out->graphs_dropped = (int64_t)ctx->counters.graphs_dropped;
    out->evictions = (int64_t)ctx->counters.plans_evicted;
    out->scratch_reallocs = (int64_t)ctx->counters.scratch_reallocs;
    int64_t bytes = 0;
    for (const auto &sc : ctx->scr) bytes += (int64_t)(sc.a + sc.b + sc.c + sc.d + sc.e + sc.f + sc.g);
    out->scratch_bytes = bytes;
    return LGF_OK;
}

lgf_status lgf_cache_limits(lgf_ctx *ctx, int32_t max_plans, int32_t max_spectra, int32_t max_graphs)
{
    lgf_status st = enter(ctx);
    if (st != LGF_OK) return st;
    if (max_plans == 0 || max_plans < -1 || max_spectra == 0 || max_spectra < -1 || max_graphs < -1)
        return fail(ctx, LGF_EINVAL, "cache_limits: plans and spectra >= 1, graphs >= 0, or -1 to keep");
    if (max_plans > 0) {
        ctx->pplans.set_cap((size_t)max_plans);
        ctx->iplans.set_cap((size_t)max_plans);
        ctx->cplans.set_cap((size_t)max_plans);
        ctx->ibplans.set_cap((size_t)max_plans);
    }
    if (max_spectra > 0) ctx->spectra.set_cap((size_t)max_spectra);
    if (max_graphs >= 0 && (size_t)max_graphs != ctx->graphs.cap()) {
        invalidate_graphs(ctx);
        ctx->graphs.set_cap((size_t)max_graphs);
    }
    return LGF_OK;
}

}  // extern "C"
