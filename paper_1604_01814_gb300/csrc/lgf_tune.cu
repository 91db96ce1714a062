// Autotuner of the Poisson engine's free choices.
//
// A Poisson plan's geometry has knobs that the method leaves open and whose
// best setting depends on the block sets, the field count and the GPU: the
// embedding along x and along y (the even circular embedding or the shifted
// window), the transform length along each axis (the smallest supported
// length that holds the convolution, or the next one, whose radix plan may
// run faster), and the register variant of the z pass.  (Whether the y and x
// inverses run as one cluster kernel is a persisted choice only.)  On a plan's first
// use with tuning on, the tuner times candidates by coordinate descent from
// the default choice: it changes one knob at a time, keeps a change that
// cuts the median of the timed repetitions by at least 3 %, and stops after
// one sweep.  Each candidate runs the plan's five passes on the caller's
// stream with CUDA events around them (two untimed runs first); the kernel
// spectra built for candidates that lost are freed again.  The choice is
// kept in the plan, in the context's table and, when a file is set, in a
// text file read back by later contexts (lgf_tune.h), so a solver tunes once
// per geometry.  The batch's branch count is tuned in lgf_batch_apply.
#include <algorithm>
#include <cstdio>
#include <set>

#include "lgf_internal.cuh"
#include "lgf_tune.h"

namespace lgf {

void tune_record(lgf_ctx *ctx, const std::string &key, const std::string &value)
{
    ctx->tune_db[key] = value;
    if (ctx->tune_path.empty()) return;
    if (FILE *f = std::fopen(ctx->tune_path.c_str(), "a")) {
        const std::string line = tune_line(key, value);
        std::fwrite(line.data(), 1, line.size(), f);
        std::fclose(f);
    }
}

namespace {

std::string plan_key(const lgf_ctx *ctx, const PoissonPlan &pl, int nf)
{
    int nbs[3], nbt[3], off[3];
    for (int d = 0; d < 3; ++d) {
        nbs[d] = pl.shi[d] - pl.slo[d] + 1;
        nbt[d] = pl.thi[d] - pl.tlo[d] + 1;
        off[d] = pl.tlo[d] - pl.slo[d];
    }
    return tune_plan_key(ctx->prec == LGF_F64, pl.b, nbs, nbt, off, nf);
}

TuneChoiceText to_text(const PoissonChoice &c)
{
    TuneChoiceText t;
    for (int d = 0; d < 2; ++d) t.shift[d] = c.shift[d];
    for (int d = 0; d < 3; ++d) t.bump[d] = c.bump[d];
    t.zvar = c.zvar;
    t.fuse = c.fuse;
    return t;
}

PoissonChoice from_text(const TuneChoiceText &t)
{
    PoissonChoice c;
    for (int d = 0; d < 2; ++d) c.shift[d] = t.shift[d];
    for (int d = 0; d < 3; ++d) c.bump[d] = t.bump[d];
    c.zvar = t.zvar;
    c.fuse = t.fuse;
    return c;
}

}  // namespace

lgf_status tune_poisson(lgf_ctx *ctx, PoissonPlan *pl, int nf, double kalpha, cudaStream_t s)
{
    if (ctx->tune_mode == LGF_TUNE_OFF || pl->tuned_nf != 0) return LGF_OK;
    const std::string key = plan_key(ctx, *pl, nf);
    auto it = ctx->tune_db.find(key);
    if (it != ctx->tune_db.end()) {
        TuneChoiceText t;
        PoissonGeom g = pl->g;
        int64_t A, B;
        if (tune_parse_plan_value(it->second, &t) && poisson_geometry(*pl, from_text(t), &g, &A, &B)) {
            poisson_set_choice(pl, from_text(t));
            pl->tuned_nf = nf;
            ++ctx->tune_plans_cached;
            return LGF_OK;
        }
    }
    if (ctx->tune_mode != LGF_TUNE_ON) {   // cached choices only: keep the default
        pl->tuned_nf = nf;
        return LGF_OK;
    }
    // spectra present before tuning stay; those built for losing candidates go
    std::set<const Spectrum *> before;
    for (auto &sp : ctx->spectra.items()) before.insert(sp.get());
    PoissonChoice best = pl->choice;
    float tbest = 0.f;
    struct Wall {   // wall time of the whole tuning, destroyed on every return
        cudaEvent_t a = nullptr, b = nullptr;
        ~Wall()
        {
            if (a) cudaEventDestroy(a);
            if (b) cudaEventDestroy(b);
        }
    } wall;
    const bool timed = cudaEventCreate(&wall.a) == cudaSuccess && cudaEventCreate(&wall.b) == cudaSuccess;
    if (timed) cudaEventRecord(wall.a, s);
    lgf_status st = poisson_time_choice(ctx, pl, best, nf, kalpha, s, &tbest);
    if (st != LGF_OK) return st;
    ++ctx->tune_candidates;
    const bool f32 = ctx->prec == LGF_F32;
    // (the fused y+x inverse is not searched: timed alone it won on some plate
    // plans by a few per cent, inside the batch it lost; a persisted choice
    // "f1" selects it)
    for (int knob = 0; knob < 6; ++knob) {
        PoissonChoice c = best;
        if (knob < 2) c.shift[knob] ^= 1;                 // the other embedding along x, y
        else if (knob < 5) c.bump[knob - 2] = 1;          // a longer transform along x, y, z
        else if (f32) c.zvar ^= 1;                        // the other z-pass register cap
        if (c == best) continue;
        PoissonGeom g = pl->g;
        int64_t A, B;
        if (!poisson_geometry(*pl, c, &g, &A, &B)) continue;
        float t = 0.f;
        st = poisson_time_choice(ctx, pl, c, nf, kalpha, s, &t);
        if (st == LGF_EUNSUPPORTED || st == LGF_ENOMEM) {   // e.g. too large: not a candidate
            cudaGetLastError();
            continue;
        }
        if (st != LGF_OK) return st;
        ++ctx->tune_candidates;
        if (t < 0.97f * tbest) {
            tbest = t;
            best = c;
        }
    }
    poisson_set_choice(pl, best);
    pl->tuned_nf = nf;
    ++ctx->tune_plans;
    // free the spectra of the losing candidates (synchronised: the timing runs
    // waited on their events; no graph was captured with them)
    const PoissonGeom &gw = pl->g;
    ctx->spectra.erase_if([&](const Spectrum &q) {
        if (before.count(&q)) return false;
        const bool winner = q.M == std::array<int, 3>{gw.M[0], gw.M[1], gw.M[2]} && q.alpha == kalpha &&
                            q.xasym == gw.xasym && q.xc == gw.xc && q.xP == gw.xP && q.yasym == gw.yasym &&
                            q.yc == gw.yc && q.yP == gw.yP;
        return !winner;
    });
    if (timed) {
        cudaEventRecord(wall.b, s);
        float ms = 0.f;
        if (cudaEventSynchronize(wall.b) == cudaSuccess && cudaEventElapsedTime(&ms, wall.a, wall.b) == cudaSuccess)
            ctx->tune_ms += ms;
    }
    tune_record(ctx, key, tune_plan_value(to_text(best)));
    return LGF_OK;
}

}  // namespace lgf
