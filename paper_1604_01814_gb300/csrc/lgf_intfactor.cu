// Integrating factor u = E(alpha) f on block sets (Sec. 2.3 footnote; App. A,
// Eq. lgf_intfac).  The kernel E_alpha(n) = prod_i w(|n_i|), w(k) =
// e^{-2 alpha} I_k(2 alpha), is separable, so the apply is three one-dimensional
// passes (x, then y, then z), each a symmetric (2R+1)-tap stencil truncated at
// the radius R where w(R) < tol/8 w(0).  Sources outside the source blocks are
// zero (the truncation of Table 1).  Every pass maps a block set to a block
// set; a pass's output block reads its own position and the nr = ceil(R/b)
// neighbours on each side along the pass axis (missing blocks read as zero):
//
//   pass x : S  -> X1 = {blocks within nr in x of S} that some target needs
//   pass y : X1 -> Y2 = {blocks within nr in y of X1} that some target needs
//   pass z : Y2 -> T
//
// One CTA handles one output block, one slab of lines and one field; it
// stages the slab plus its halo in shared memory.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <tuple>
#include <unordered_map>
#include <unordered_set>

#include "lgf_intfactor_win.cuh"

namespace lgf {

// Register-window passes: templates in lgf_intfactor_win.cuh, instantiated
// per precision in lgf_intfactor_win_f32.cu / lgf_intfactor_win_f64.cu.
extern template lgf_status launch_sep_window<float>(lgf_ctx *, int, int, int, const SepJobs<float> &, cudaStream_t,
                                                    const int *, int, bool *);
extern template lgf_status launch_sep_window<double>(lgf_ctx *, int, int, int, const SepJobs<double> &, cudaStream_t,
                                                     const int *, int, bool *);
extern template lgf_status launch_sep_xy<float>(lgf_ctx *, int, int, const SepJobs<float> &, cudaStream_t, const int *,
                                                const int *, int, bool *);
extern template lgf_status launch_sep_xy<double>(lgf_ctx *, int, int, const SepJobs<double> &, cudaStream_t,
                                                 const int *, const int *, int, bool *);
extern template lgf_status launch_sep_rag<float>(lgf_ctx *, bool, int, int, SepRagJob<float> *, int, cudaStream_t);
extern template lgf_status launch_sep_rag<double>(lgf_ctx *, bool, int, int, SepRagJob<double> *, int, cudaStream_t);

IntfPlan::~IntfPlan()
{
    for (auto &p : pass) cudaFree(p.nbr_dev);
    cudaFree(nbr_xy_dev);
    cudaFree(xy_items_dev);
}

namespace {

constexpr int kThreads = 256;
constexpr int kSlabElems = 12288;   // staged elements per CTA

inline int64_t pack(int x, int y, int z)
{
    return (((int64_t)(x + (1 << 20))) << 42) | (((int64_t)(y + (1 << 20))) << 21) | (int64_t)(z + (1 << 20));
}

// Vectorised pass (block edge and axis fixed at compile time).  The staged
// region covers the output slab plus a halo of HL >= R points along the
// axis, HL a multiple of 4, read with 16-byte loads from the neighbour
// blocks; every thread produces VEC consecutive x outputs with one 16-byte
// store.  Region layouts (x fastest):
//   AX 0: [ns][b][E]   AX 1: [ns][E][b]   AX 2: [E][ns][b],   E = b + 2 HL.
template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
    using V = float4;
    static constexpr int N = 4;
};
template <>
struct Vec16<double> {
    using V = double2;
    static constexpr int N = 2;
};

template <typename T, int LB, int AX>
__global__ void __launch_bounds__(kThreads) k_sep_vec(const T *__restrict__ in, T *__restrict__ out,
                                                       const int *__restrict__ nbr, const T *__restrict__ wg, int R,
                                                       int HL, int nr, int slab, int64_t in_stride, int64_t out_stride)
{
    constexpr int b = 1 << LB, bm = b - 1;
    using V = typename Vec16<T>::V;
    constexpr int NV = Vec16<T>::N;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *w = reinterpret_cast<T *>(smem_raw);
    T *s = w + ((R + 1 + 3) & ~3);
    for (int i = threadIdx.x; i <= R; i += blockDim.x) w[i] = wg[i];
    const int o = blockIdx.x;
    const int s0 = blockIdx.y * slab;
    const int ns = min(slab, b - s0);
    const int E = b + 2 * HL;
    const int nd = 2 * nr + 1;
    const int *nb = nbr + (int64_t)o * nd;
    const T *inf = in + blockIdx.z * in_stride;
    T *outf = out + blockIdx.z * out_stride;
    // ---- stage the region with 16-byte loads ----
    const int rowlen = AX == 0 ? E : b;              // elements per staged row
    const int nrows = AX == 0 ? ns * b : ns * E;
    const int vpr = rowlen / NV;
    const int total = nrows * vpr;
    constexpr int U = 4;
    for (int base = threadIdx.x; base < total; base += U * blockDim.x) {
        V v[U];
        int dst[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int it = base + u * blockDim.x;
            dst[u] = -1;
            v[u] = V{};
            if (it >= total) continue;
            const int row = it / vpr, cv = it - row * vpr;
            int x, y, z, e;
            if (AX == 0) {
                e = cv * NV - HL;
                y = row & bm;
                z = s0 + (row >> LB);
                x = e & bm;
            } else if (AX == 1) {
                x = cv * NV;
                e = row % E - HL;
                z = s0 + row / E;
                y = e & bm;
            } else {
                x = cv * NV;
                y = s0 + row % ns;
                e = row / ns - HL;
                z = e & bm;
            }
            dst[u] = it * NV;
            const int bi = nb[(e + nr * b) >> LB];
            if (bi >= 0)
                v[u] = *reinterpret_cast<const V *>(inf + ((int64_t)bi << (3 * LB)) + (((z << LB) + y) << LB) + x);
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (dst[u] >= 0) *reinterpret_cast<V *>(s + dst[u]) = v[u];
    }
    __syncthreads();
    // ---- stencil: NV consecutive x outputs per thread ----
    const int nout = ns * b * (b / NV);
    for (int it = threadIdx.x; it < nout; it += blockDim.x) {
        const int xv = it % (b / NV), rest = it / (b / NV);
        const int x = xv * NV;
        const int y2 = rest & bm;          // y for AX 0/1, z for AX 2
        const int sl = rest >> LB;         // slab-local coordinate
        int c, st, X = x, Y, Z;
        if (AX == 0) {
            Y = y2; Z = s0 + sl;
            c = (sl * b + Y) * E + (X + HL);
            st = 1;
        } else if (AX == 1) {
            Y = y2; Z = s0 + sl;
            c = (sl * E + (Y + HL)) * b + X;
            st = b;
        } else {
            Z = y2; Y = s0 + sl;
            c = ((Z + HL) * ns + sl) * b + X;
            st = ns * b;
        }
        T acc[NV];
        const T w0 = w[0];
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] = w0 * s[c + v];
        for (int k = 1; k <= R; ++k) {
            const T wk = w[k];
            if (AX == 0) {
#pragma unroll
                for (int v = 0; v < NV; ++v) acc[v] += wk * (s[c + v - k] + s[c + v + k]);
            } else {
                const V lo = *reinterpret_cast<const V *>(s + c - k * st);
                const V hi = *reinterpret_cast<const V *>(s + c + k * st);
                const T *l = reinterpret_cast<const T *>(&lo);
                const T *h = reinterpret_cast<const T *>(&hi);
#pragma unroll
                for (int v = 0; v < NV; ++v) acc[v] += wk * (l[v] + h[v]);
            }
        }
        V r;
        T *rr = reinterpret_cast<T *>(&r);
#pragma unroll
        for (int v = 0; v < NV; ++v) rr[v] = acc[v];
        *reinterpret_cast<V *>(outf + ((int64_t)o << (3 * LB)) + (((Z << LB) + Y) << LB) + X) = r;
    }
}

__global__ void k_to_float(const double *a, float *b, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

}  // namespace

lgf_status intf_weights(lgf_ctx *ctx, double alpha, IntfWeights **out, cudaStream_t s)
{
    for (auto &w : ctx->weights)
        if (w->alpha == alpha) {
            *out = w.get();
            return LGF_OK;
        }
    const int cap = 128;
    double *dw = nullptr;
    if (cudaMalloc(&dw, (cap + 1) * sizeof(double)) != cudaSuccess)
        return fail(ctx, LGF_ENOMEM, "intfactor: weight allocation failed");
    lgf_status st = bessel_weights(ctx, 2.0 * alpha, cap, dw, s);
    std::vector<double> hw(cap + 1);
    if (st == LGF_OK) {
        cudaError_t e = cudaMemcpyAsync(hw.data(), dw, hw.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(ctx, e, "intfactor weights");
    }
    if (st != LGF_OK) {
        cudaFree(dw);
        return st;
    }
    int R;
    if (ctx->opt.stencil_radius > 0) {
        R = std::min(ctx->opt.stencil_radius, cap);
    } else {
        R = 0;
        const double thr = ctx->tol / 8.0 * hw[0];
        while (R < cap && hw[R] >= thr) ++R;
        if (alpha == 0.0) R = 0;
    }
    if (ctx->opt.stencil_radius == 0 && alpha > 0.0 && hw[cap] >= ctx->tol / 8.0 * hw[0]) {
        cudaFree(dw);
        return fail(ctx, LGF_EUNSUPPORTED, "intfactor: alpha needs a stencil radius above 128");
    }
    auto w = std::make_unique<IntfWeights>();
    w->alpha = alpha;
    w->R = R;
    w->w64 = dw;
    if (cudaMalloc(&w->w32, (R + 1) * sizeof(float)) != cudaSuccess) {
        cudaFree(dw);
        return fail(ctx, LGF_ENOMEM, "intfactor: weight allocation failed");
    }
    k_to_float<<<1, 256, 0, s>>>(dw, w->w32, R + 1);
    LGF_CHECK_LAUNCH(ctx, "intfactor weights");
    LGF_CUDA(ctx, cudaStreamSynchronize(s));
    ctx->weights.push_back(std::move(w));
    *out = ctx->weights.back().get();
    return LGF_OK;
}

lgf_status intf_plan(lgf_ctx *ctx, const lgf_blockset *src, const lgf_blockset *tgt, int R, IntfPlan **out)
{
    const int b = src->b;
    const int nr = R == 0 ? 0 : (R + b - 1) / b;
    const std::vector<int32_t> sv(src->coords, src->coords + 3 * (size_t)src->nblocks);
    const std::vector<int32_t> tv(tgt->coords, tgt->coords + 3 * (size_t)tgt->nblocks);
    if (IntfPlan *hit = ctx->iplans.find(
            [&](const IntfPlan &p) { return p.b == b && p.nr == nr && p.src == sv && p.tgt == tv; },
            ctx->counters.epoch)) {
        *out = hit;
        return LGF_OK;
    }
    std::unordered_map<int64_t, int> S, T;
    for (int i = 0; i < src->nblocks; ++i)
        if (!S.emplace(pack(sv[3 * i], sv[3 * i + 1], sv[3 * i + 2]), i).second)
            return fail(ctx, LGF_EINVAL, "intfactor: duplicate block in the source set");
    for (int i = 0; i < tgt->nblocks; ++i)
        if (!T.emplace(pack(tv[3 * i], tv[3 * i + 1], tv[3 * i + 2]), i).second)
            return fail(ctx, LGF_EINVAL, "intfactor: duplicate block in the target set");
    // candidate intermediate sets
    std::unordered_set<int64_t> y2cand;
    for (int i = 0; i < tgt->nblocks; ++i)
        for (int dz = -nr; dz <= nr; ++dz) y2cand.insert(pack(tv[3 * i], tv[3 * i + 1], tv[3 * i + 2] + dz));
    std::vector<std::array<int, 3>> x1;
    std::unordered_map<int64_t, int> X1;
    {
        std::unordered_set<int64_t> seen;
        for (int i = 0; i < src->nblocks; ++i)
            for (int dx = -nr; dx <= nr; ++dx) {
                const int x = sv[3 * i] + dx, y = sv[3 * i + 1], z = sv[3 * i + 2];
                const int64_t k = pack(x, y, z);
                if (seen.count(k)) continue;
                seen.insert(k);
                bool need = false;
                for (int dy = -nr; dy <= nr && !need; ++dy) need = y2cand.count(pack(x, y + dy, z)) > 0;
                if (need) {
                    X1.emplace(k, (int)x1.size());
                    x1.push_back({x, y, z});
                }
            }
    }
    std::vector<std::array<int, 3>> y2;
    std::unordered_map<int64_t, int> Y2;
    for (int64_t k : y2cand) {
        const int x = (int)((k >> 42) & ((1 << 21) - 1)) - (1 << 20);
        const int y = (int)((k >> 21) & ((1 << 21) - 1)) - (1 << 20);
        const int z = (int)(k & ((1 << 21) - 1)) - (1 << 20);
        bool need = false;
        for (int dy = -nr; dy <= nr && !need; ++dy) need = X1.count(pack(x, y + dy, z)) > 0;
        if (need) {
            Y2.emplace(k, (int)y2.size());
            y2.push_back({x, y, z});
        }
    }
    auto plan = std::make_unique<IntfPlan>();
    plan->b = b;
    plan->nr = nr;
    plan->src = sv;
    plan->tgt = tv;
    plan->n1 = (int)x1.size();
    plan->n2 = (int)y2.size();
    const int nd = 2 * nr + 1;
    auto build = [&](int pi, const std::vector<std::array<int, 3>> &outs, const std::unordered_map<int64_t, int> &in,
                     int ax) -> lgf_status {
        std::vector<int> nbr((size_t)outs.size() * nd, -1);
        for (size_t o = 0; o < outs.size(); ++o)
            for (int d = -nr; d <= nr; ++d) {
                std::array<int, 3> c = outs[o];
                c[ax] += d;
                auto it = in.find(pack(c[0], c[1], c[2]));
                if (it != in.end()) nbr[o * nd + d + nr] = it->second;
            }
        plan->pass[pi].nout = (int)outs.size();
        if (!nbr.empty()) {
            if (cudaMalloc(&plan->pass[pi].nbr_dev, nbr.size() * sizeof(int)) != cudaSuccess)
                return fail(ctx, LGF_ENOMEM, "intfactor: neighbour table allocation failed");
            LGF_CUDA(ctx, cudaMemcpy(plan->pass[pi].nbr_dev, nbr.data(), nbr.size() * sizeof(int),
                                     cudaMemcpyHostToDevice));
        }
        return LGF_OK;
    };
    std::vector<std::array<int, 3>> touts(tgt->nblocks);
    for (int i = 0; i < tgt->nblocks; ++i) touts[i] = {tv[3 * i], tv[3 * i + 1], tv[3 * i + 2]};
    lgf_status st;
    if ((st = build(0, x1, S, 0)) != LGF_OK) return st;
    if ((st = build(1, y2, X1, 1)) != LGF_OK) return st;
    if ((st = build(2, touts, Y2, 2)) != LGF_OK) return st;
    {   // fused x+y pass: the source block at each xy offset of every Y2 block
        const int nd2 = nd * nd;
        std::vector<int> nxy((size_t)y2.size() * nd2, -1);
        for (size_t o = 0; o < y2.size(); ++o)
            for (int dy = -nr; dy <= nr; ++dy)
                for (int dx = -nr; dx <= nr; ++dx) {
                    auto it = S.find(pack(y2[o][0] + dx, y2[o][1] + dy, y2[o][2]));
                    if (it != S.end()) nxy[o * nd2 + (dy + nr) * nd + (dx + nr)] = it->second;
                }
        if (!nxy.empty()) {
            if (cudaMalloc(&plan->nbr_xy_dev, nxy.size() * sizeof(int)) != cudaSuccess)
                return fail(ctx, LGF_ENOMEM, "intfactor: neighbour table allocation failed");
            LGF_CUDA(ctx, cudaMemcpy(plan->nbr_xy_dev, nxy.data(), nxy.size() * sizeof(int), cudaMemcpyHostToDevice));
        }
        // work items of the fused pass: Y2 blocks paired with their +y
        // neighbour in Y2 where it exists (walking every (x, z) column upwards)
        std::vector<int> order(y2.size());
        for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
        std::sort(order.begin(), order.end(), [&](int a, int c) {
            return std::make_tuple(y2[a][2], y2[a][0], y2[a][1]) < std::make_tuple(y2[c][2], y2[c][0], y2[c][1]);
        });
        std::vector<char> used(y2.size(), 0);
        std::vector<int> items;
        for (int o : order) {
            if (used[o]) continue;
            used[o] = 1;
            int o2 = -1;
            auto it = Y2.find(pack(y2[o][0], y2[o][1] + 1, y2[o][2]));
            if (it != Y2.end() && !used[it->second]) {
                o2 = it->second;
                used[o2] = 1;
            }
            items.push_back(o);
            items.push_back(o2);
        }
        plan->n_xy_items = (int)(items.size() / 2);
        if (!items.empty()) {
            if (cudaMalloc(&plan->xy_items_dev, items.size() * sizeof(int)) != cudaSuccess)
                return fail(ctx, LGF_ENOMEM, "intfactor: work item allocation failed");
            LGF_CUDA(ctx,
                     cudaMemcpy(plan->xy_items_dev, items.data(), items.size() * sizeof(int), cudaMemcpyHostToDevice));
        }
    }
    *out = ctx->iplans.insert(std::move(plan), ctx->counters.epoch, [&] { before_evict(ctx); },
                              &ctx->counters.plans_evicted);
    return LGF_OK;
}

lgf_status intf_prepare_scratch(lgf_ctx *ctx, const IntfPlan *pl, int nfields, int njobs)
{
    const size_t esz = ctx->prec == LGF_F64 ? 8 : 4;
    const size_t b3 = (size_t)pl->b * pl->b * pl->b;
    lgf_status st = ensure_scratch(ctx, &ctx->cur->C, &ctx->cur->c, std::max<size_t>(1, pl->n1) * b3 * nfields * esz);
    if (st != LGF_OK) return st;
    return ensure_scratch(ctx, &ctx->cur->D, &ctx->cur->d,
                          std::max<size_t>(1, pl->n2) * b3 * nfields * esz * (size_t)std::max(1, njobs));
}

// Region staging parameters shared by both launch paths.
struct SepGeom {
    int HL;      // halo, a multiple of 4 and >= R (<= nr * b)
    int slab;    // slab extent (planes of the slab axis per CTA)
    int nslab;
};

SepGeom sep_geom(int b, int R, int nr)
{
    SepGeom g;
    g.HL = std::min(((R + 3) / 4) * 4, nr * b);
    const int E = b + 2 * g.HL;
    g.slab = std::max(1, std::min(b, kSlabElems / (b * E)));
    g.nslab = (b + g.slab - 1) / g.slab;
    return g;
}

template <typename T, int LB, int AX>
lgf_status launch_sep_lb(lgf_ctx *ctx, dim3 grid, size_t smem, cudaStream_t s, const T *in, T *out, const int *nbr,
                         const T *w, int R, int HL, int nr, int slab, int64_t istr, int64_t ostr)
{
    auto kern = k_sep_vec<T, LB, AX>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaFuncSetAttribute");
    }
    kern<<<grid, kThreads, smem, s>>>(in, out, nbr, w, R, HL, nr, slab, istr, ostr);
    return LGF_OK;
}

template <typename T, int AX>
lgf_status launch_sep_ax(lgf_ctx *ctx, int b, dim3 grid, size_t smem, cudaStream_t s, const T *in, T *out,
                         const int *nbr, const T *w, int R, int HL, int nr, int slab, int64_t istr, int64_t ostr)
{
    switch (b) {
    case 4: return launch_sep_lb<T, 2, AX>(ctx, grid, smem, s, in, out, nbr, w, R, HL, nr, slab, istr, ostr);
    case 8: return launch_sep_lb<T, 3, AX>(ctx, grid, smem, s, in, out, nbr, w, R, HL, nr, slab, istr, ostr);
    case 16: return launch_sep_lb<T, 4, AX>(ctx, grid, smem, s, in, out, nbr, w, R, HL, nr, slab, istr, ostr);
    case 32: return launch_sep_lb<T, 5, AX>(ctx, grid, smem, s, in, out, nbr, w, R, HL, nr, slab, istr, ostr);
    default: return launch_sep_lb<T, 6, AX>(ctx, grid, smem, s, in, out, nbr, w, R, HL, nr, slab, istr, ostr);
    }
}

// One separable pass along axis `ax` for `nout` output blocks.
template <typename T>
lgf_status launch_sep(lgf_ctx *ctx, int ax, int b, int nout, int nfields, cudaStream_t s, const T *in, T *out,
                      const int *nbr, const T *w, int R, int nr, int64_t istr, int64_t ostr)
{
    bool done = false;
    SepJobs<T> jobs{};
    jobs.n = 1;
    jobs.nf = nfields;
    jobs.j[0] = SepJob<T>{in, out, w, R, 0, istr, ostr};
    lgf_status wst = launch_sep_window<T>(ctx, ax, b, nout, jobs, s, nbr, nr, &done);
    if (wst != LGF_OK) return wst;
    if (done) {
        LGF_CHECK_LAUNCH(ctx, "intfactor pass");
        return LGF_OK;
    }
    const SepGeom sg = sep_geom(b, R, nr);
    const size_t smem = sizeof(T) * (((R + 1 + 3) & ~3) + (size_t)sg.slab * b * (b + 2 * sg.HL));
    dim3 grid(nout, sg.nslab, nfields);
    lgf_status st;
    if (ax == 0) st = launch_sep_ax<T, 0>(ctx, b, grid, smem, s, in, out, nbr, w, R, sg.HL, nr, sg.slab, istr, ostr);
    else if (ax == 1) st = launch_sep_ax<T, 1>(ctx, b, grid, smem, s, in, out, nbr, w, R, sg.HL, nr, sg.slab, istr, ostr);
    else st = launch_sep_ax<T, 2>(ctx, b, grid, smem, s, in, out, nbr, w, R, sg.HL, nr, sg.slab, istr, ostr);
    if (st != LGF_OK) return st;
    LGF_CHECK_LAUNCH(ctx, "intfactor pass");
    return LGF_OK;
}

// All jobs of one plan: fused x+y then z launches over the whole job list
// (chunks of kMaxSepJobs) when the window kernels apply, else the three
// generic passes job by job.
template <typename T>
static lgf_status run_sep_jobs(lgf_ctx *ctx, IntfPlan *pl, const IntfJob *jobs, int njobs, int nfields,
                               cudaStream_t s)
{
    const int b = pl->b, nr = pl->nr;
    const int64_t b3 = (int64_t)b * b * b;
    const int nsrc = (int)(pl->src.size() / 3), ntgt = (int)(pl->tgt.size() / 3);
    const int64_t y2f = (int64_t)pl->n2 * b3;                       // Y2 elements per field
    T *X1 = (T *)ctx->cur->C, *Y2all = (T *)ctx->cur->D;
    auto wptr = [](const IntfJob &j) -> const T * {
        return sizeof(T) == 8 ? (const T *)(const void *)j.w->w64 : (const T *)(const void *)j.w->w32;
    };
    // jobs in order of their window class, so that a launch never pays for a
    // larger radius than its own jobs need
    std::vector<int> order(njobs);
    for (int i = 0; i < njobs; ++i) order[i] = i;
    auto cls_key = [&](int i) { const int c = window_class(jobs[i].w->R); return c == 0 ? 1 << 20 : c; };
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cls_key(a) < cls_key(c); });
    int first_generic = 0;
    if (pl->n2 > 0 && pl->pass[2].nout > 0) {
        first_generic = njobs;
        for (int c0 = 0; c0 < njobs;) {
            int cn = 0;
            const int cls = window_class(jobs[order[c0]].w->R);
            while (c0 + cn < njobs && cn < kMaxSepJobs && window_class(jobs[order[c0 + cn]].w->R) == cls) ++cn;
            SepJobs<T> jx{}, jz{};
            jx.n = jz.n = cn;
            jx.nf = jz.nf = nfields;
            for (int i = 0; i < cn; ++i) {
                const IntfJob &J = jobs[order[c0 + i]];
                T *y2 = Y2all + (int64_t)(c0 + i) * y2f * nfields;
                jx.j[i] = SepJob<T>{(const T *)J.f, y2, wptr(J), J.w->R, 0, nsrc * b3, y2f};
                jz.j[i] = SepJob<T>{y2, (T *)J.u, wptr(J), J.w->R, 0, y2f, ntgt * b3};
            }
            const int ph = prof_begin(ctx, s, "intfactor_pass_xy");
            bool done = false;
            lgf_status st = launch_sep_xy<T>(ctx, b, pl->n_xy_items, jx, s, pl->nbr_xy_dev, pl->xy_items_dev, nr,
                                             &done);
            if (st != LGF_OK) return st;
            if (!done) {
                prof_end(ctx, s, ph);
                first_generic = c0;   // (classes only grow: every later chunk falls back too)
                break;
            }
            LGF_CHECK_LAUNCH(ctx, "intfactor xy pass");
            prof_end(ctx, s, ph);
            const int pz = prof_begin(ctx, s, "intfactor_pass_z");
            st = launch_sep_window<T>(ctx, 2, b, ntgt, jz, s, pl->pass[2].nbr_dev, nr, &done);
            if (st != LGF_OK) return st;
            if (!done) return fail(ctx, LGF_ECUDA, "intfactor: z window pass unavailable after the xy pass");
            LGF_CHECK_LAUNCH(ctx, "intfactor z pass");
            prof_end(ctx, s, pz);
            c0 += cn;
        }
    }
    static const char *names[3] = {"intfactor_pass_x", "intfactor_pass_y", "intfactor_pass_z"};
    for (int jo = first_generic; jo < njobs; ++jo) {
        const IntfJob &J = jobs[order[jo]];
        T *Y2 = Y2all;
        const T *ins[3] = {(const T *)J.f, X1, Y2};
        T *outs[3] = {X1, Y2, (T *)J.u};
        const int64_t istr[3] = {nsrc * b3, pl->n1 * b3, pl->n2 * b3};
        const int64_t ostr[3] = {pl->n1 * b3, pl->n2 * b3, ntgt * b3};
        for (int p = 0; p < 3; ++p) {
            if (pl->pass[p].nout == 0) continue;
            const int ph = prof_begin(ctx, s, names[p]);
            lgf_status st = launch_sep<T>(ctx, p, b, pl->pass[p].nout, nfields, s, ins[p], outs[p],
                                          pl->pass[p].nbr_dev, wptr(J), J.w->R, nr, istr[p], ostr[p]);
            if (st != LGF_OK) return st;
            prof_end(ctx, s, ph);
        }
    }
    return LGF_OK;
}

lgf_status intf_run_jobs(lgf_ctx *ctx, IntfPlan *pl, const IntfJob *jobs, int njobs, int nfields, cudaStream_t s)
{
    // the stencil kernels move 16-byte vectors (block and field strides keep
    // the alignment of the base pointers)
    for (int j = 0; j < njobs; ++j)
        if ((reinterpret_cast<uintptr_t>(jobs[j].f) | reinterpret_cast<uintptr_t>(jobs[j].u)) % 16 != 0)
            return fail(ctx, LGF_EINVAL, "integrating factor: f and u must be 16-byte aligned");
    lgf_status st = intf_prepare_scratch(ctx, pl, nfields, njobs);
    if (st != LGF_OK) return st;
    const int ntgt = (int)(pl->tgt.size() / 3);
    const size_t esz = ctx->prec == LGF_F64 ? 8 : 4;
    const size_t b3 = (size_t)pl->b * pl->b * pl->b;
    if (pl->pass[2].nout > 0 && pl->n2 == 0) {
        // no source reaches any target: the results are zero
        for (int j = 0; j < njobs; ++j)
            LGF_CUDA(ctx, cudaMemsetAsync(jobs[j].u, 0, (size_t)ntgt * b3 * nfields * esz, s));
        return LGF_OK;
    }
    if (ctx->prec == LGF_F64) return run_sep_jobs<double>(ctx, pl, jobs, njobs, nfields, s);
    return run_sep_jobs<float>(ctx, pl, jobs, njobs, nfields, s);
}

namespace {

// Window bound of a job on a plan, 0 where the window kernels do not cover it.
int rag_rmax(const IntfPlan *pl, const IntfJob &j)
{
    const int c = window_class(j.w->R);
    if (c == 0 || c > pl->nr * pl->b || (pl->b != 8 && pl->b != 16 && pl->b != 32)) return 0;
    return c;
}

// Groups of the ragged launches: every job of a group has a window bound and
// the plan a z pass with sources.
bool rag_group(const IntfGroupRef &g)
{
    if (g.plan->n2 == 0 || g.plan->pass[2].nout == 0) return false;
    for (int j = 0; j < g.njobs; ++j)
        if (rag_rmax(g.plan, g.jobs[j]) == 0) return false;
    return true;
}

template <typename T>
lgf_status run_ragged_t(lgf_ctx *ctx, const IntfGroupRef *gs, int n, cudaStream_t s)
{
    const size_t esz = sizeof(T);
    T *Y2all = (T *)ctx->cur->D;
    int64_t y2off = 0;
    // (block edge, window bound) -> the jobs of the x+y pass and of the z pass
    std::vector<std::array<int, 2>> keys;
    std::vector<std::vector<SepRagJob<T>>> xy, zz;
    for (int gi = 0; gi < n; ++gi) {
        const IntfGroupRef &g = gs[gi];
        if (!rag_group(g)) continue;
        const IntfPlan *pl = g.plan;
        const int64_t b3 = (int64_t)pl->b * pl->b * pl->b;
        const int64_t y2f = (int64_t)pl->n2 * b3;
        const int nsrc = (int)(pl->src.size() / 3), ntgt = (int)(pl->tgt.size() / 3);
        for (int j = 0; j < g.njobs; ++j) {
            const IntfJob &J = g.jobs[j];
            if ((reinterpret_cast<uintptr_t>(J.f) | reinterpret_cast<uintptr_t>(J.u)) % 16 != 0)
                return fail(ctx, LGF_EINVAL, "integrating factor: f and u must be 16-byte aligned");
            const T *w = sizeof(T) == 8 ? (const T *)(const void *)J.w->w64 : (const T *)(const void *)J.w->w32;
            T *y2 = Y2all + y2off;
            y2off += y2f * g.nf;
            const std::array<int, 2> key{pl->b, rag_rmax(pl, J)};
            size_t k = 0;
            while (k < keys.size() && keys[k] != key) ++k;
            if (k == keys.size()) {
                keys.push_back(key);
                xy.emplace_back();
                zz.emplace_back();
            }
            SepRagJob<T> a{};
            a.job = SepJob<T>{(const T *)J.f, y2, w, J.w->R, 0, nsrc * b3, y2f};
            a.nbr = pl->nbr_xy_dev;
            a.items = pl->xy_items_dev;
            a.nr = pl->nr;
            a.nitems = pl->n_xy_items;
            a.nf = g.nf;
            xy[k].push_back(a);
            SepRagJob<T> z{};
            z.job = SepJob<T>{y2, (T *)J.u, w, J.w->R, 0, y2f, ntgt * b3};
            z.nbr = pl->pass[2].nbr_dev;
            z.items = nullptr;
            z.nr = pl->nr;
            z.nitems = ntgt;
            z.nf = g.nf;
            zz[k].push_back(z);
        }
    }
    if ((size_t)y2off * esz > ctx->cur->d) return fail(ctx, LGF_EINVAL, "ragged integrating factor: scratch not prepared");
    for (size_t k = 0; k < keys.size(); ++k) {
        const int ph = prof_begin(ctx, s, "intfactor_pass_xy");
        lgf_status st = launch_sep_rag<T>(ctx, true, keys[k][0], keys[k][1], xy[k].data(), (int)xy[k].size(), s);
        if (st != LGF_OK) return st;
        LGF_CHECK_LAUNCH(ctx, "intfactor xy pass");
        prof_end(ctx, s, ph);
        const int pz = prof_begin(ctx, s, "intfactor_pass_z");
        if ((st = launch_sep_rag<T>(ctx, false, keys[k][0], keys[k][1], zz[k].data(), (int)zz[k].size(), s)) !=
            LGF_OK)
            return st;
        LGF_CHECK_LAUNCH(ctx, "intfactor z pass");
        prof_end(ctx, s, pz);
    }
    // the rest, group by group
    for (int gi = 0; gi < n; ++gi)
        if (!rag_group(gs[gi])) {
            lgf_status st = intf_run_jobs(ctx, gs[gi].plan, gs[gi].jobs, gs[gi].njobs, gs[gi].nf, s);
            if (st != LGF_OK) return st;
        }
    return LGF_OK;
}

}  // namespace

lgf_status intf_ragged_scratch(lgf_ctx *ctx, const IntfGroupRef *gs, int n, Scratch *sc)
{
    const size_t esz = ctx->prec == LGF_F64 ? 8 : 4;
    size_t d = 0;
    Scratch *keep = ctx->cur;
    ctx->cur = sc;
    lgf_status st = LGF_OK;
    for (int gi = 0; gi < n && st == LGF_OK; ++gi) {
        const IntfPlan *pl = gs[gi].plan;
        if (rag_group(gs[gi]))
            d += (size_t)pl->n2 * pl->b * pl->b * pl->b * gs[gi].nf * esz * gs[gi].njobs;
        else
            st = intf_prepare_scratch(ctx, pl, gs[gi].nf, gs[gi].njobs);
    }
    if (st == LGF_OK) st = ensure_scratch(ctx, &sc->D, &sc->d, std::max<size_t>(d, 1));
    ctx->cur = keep;
    return st;
}

lgf_status intf_run_ragged(lgf_ctx *ctx, const IntfGroupRef *gs, int n, cudaStream_t s, Scratch *sc)
{
    Scratch *keep = ctx->cur;
    ctx->cur = sc;
    const lgf_status st =
        ctx->prec == LGF_F64 ? run_ragged_t<double>(ctx, gs, n, s) : run_ragged_t<float>(ctx, gs, n, s);
    ctx->cur = keep;
    return st;
}

lgf_status intf_run(lgf_ctx *ctx, IntfPlan *pl, const IntfWeights *w, const void *f, void *u, int nfields,
                    cudaStream_t s)
{
    const IntfJob job{w, f, u};
    return intf_run_jobs(ctx, pl, &job, 1, nfields, s);
}

}  // namespace lgf

// ---------------------------------------------------------------------------
// Allocation-free variant of the integrating-factor apply.
//
// For callers that must not allocate device memory while they run (a solver
// loop whose device memory is reserved up front by another allocator, such as
// a framework's caching allocator, where a cudaMalloc could fail or stall the
// whole device).  The intermediate block arrays of the three passes, the
// neighbour tables and the weights live in one file-scope __device__ array of
// kNoAllocBytes; planning uses fixed-size host arrays.  The array's device
// address is taken with cudaGetSymbolAddress on the first call on each device.
// Every call reuses the same array, so calls that overlap on the GPU race.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocBytes = size_t(32) << 20;   // device scratch, held by every GPU that loads the library
constexpr int kNoAllocMaxBlocks = 1024;              // per source or target set
constexpr int kNoAllocMaxInter = 8192;               // per intermediate set
constexpr int kNoAllocGrid = 64;                     // block-lookup box edge (blocks)
constexpr int kNoAllocMaxDevices = 64;
constexpr int kNoAllocWeightCap = 128;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

void *g_noalloc_base[kNoAllocMaxDevices];
int32_t h_gS[kNoAllocGrid * kNoAllocGrid * kNoAllocGrid];
int32_t h_gX[kNoAllocGrid * kNoAllocGrid * kNoAllocGrid];
int32_t h_gY[kNoAllocGrid * kNoAllocGrid * kNoAllocGrid];
unsigned char h_gC[kNoAllocGrid * kNoAllocGrid * kNoAllocGrid];
int32_t h_x1[3 * kNoAllocMaxInter], h_y2[3 * kNoAllocMaxInter];
int32_t h_nbr[3 * kNoAllocMaxInter * 33];
double h_w[kNoAllocWeightCap + 1];

lgf_status noalloc_err(char *msg, int cap, lgf_status st, const char *text)
{
    if (msg && cap > 0) {
        strncpy(msg, text, (size_t)cap - 1);
        msg[cap - 1] = '\0';
    }
    return st;
}

}  // namespace

extern "C" LGF_API lgf_status lgf_intfactor_apply_noalloc(int32_t prec, double tol, double alpha,
                                                          const lgf_blockset *src, const lgf_blockset *tgt,
                                                          const void *f_dev, void *u_dev, int32_t ncomp,
                                                          int32_t nrhs, void *stream, char *err_msg,
                                                          int32_t err_cap)
{
    using namespace lgf;
    cudaStream_t s = (cudaStream_t)stream;
    auto err = [&](lgf_status st, const char *t) { return noalloc_err(err_msg, err_cap, st, t); };
    if (err_msg && err_cap > 0) err_msg[0] = '\0';
    if (prec != LGF_F32 && prec != LGF_F64) return err(LGF_EINVAL, "prec must be LGF_F32 or LGF_F64");
    if (!(tol >= 0.0) || !(tol < 1.0)) return err(LGF_EINVAL, "tol must be in [0, 1)");
    if (!(alpha >= 0.0) || !std::isfinite(alpha)) return err(LGF_EINVAL, "alpha must be >= 0 and finite");
    if (!src || !tgt) return err(LGF_EINVAL, "null block set");
    if (check_blockset(nullptr, src, "source") != LGF_OK || check_blockset(nullptr, tgt, "target") != LGF_OK)
        return err(LGF_EINVAL, "bad block set (edge 4..64, non-negative count, coordinates present)");
    if (src->b != tgt->b) return err(LGF_EINVAL, "source and target block edges differ");
    if (ncomp < 1 || nrhs < 1) return err(LGF_EINVAL, "ncomp and nrhs must be >= 1");
    if (src->nblocks > kNoAllocMaxBlocks || tgt->nblocks > kNoAllocMaxBlocks)
        return err(LGF_EUNSUPPORTED, "more than 1024 blocks in the source or target set");
    if (tgt->nblocks > 0 && !u_dev) return err(LGF_EINVAL, "null output pointer");
    if (src->nblocks > 0 && tgt->nblocks > 0 && !f_dev) return err(LGF_EINVAL, "null input pointer");
    if ((reinterpret_cast<uintptr_t>(f_dev) | reinterpret_cast<uintptr_t>(u_dev)) % 16 != 0)
        return err(LGF_EINVAL, "f and u must be 16-byte aligned");
    const int b = src->b, nf = ncomp * nrhs;
    const size_t esz = prec == LGF_F64 ? 8 : 4;
    const size_t b3 = (size_t)b * b * b;
    if (tgt->nblocks == 0) return LGF_OK;
    if (src->nblocks == 0) {
        if (cudaMemsetAsync(u_dev, 0, (size_t)tgt->nblocks * b3 * nf * esz, s) != cudaSuccess)
            return err(LGF_ECUDA, "cudaMemsetAsync failed");
        return LGF_OK;
    }
    // set-up, once per device: the device address of the static scratch
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return err(LGF_ECUDA, "cudaGetDevice failed");
    if (dev >= kNoAllocMaxDevices) return err(LGF_EUNSUPPORTED, "device ordinal 64 or above");
    if (!g_noalloc_base[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p)
            return err(LGF_ECUDA, "cudaGetSymbolAddress of the scratch array failed");
        g_noalloc_base[dev] = p;
    }
    unsigned char *base = (unsigned char *)g_noalloc_base[dev];
    double *w64 = (double *)base;
    float *w32 = (float *)(base + 2048);
    int32_t *nbr_dev = (int32_t *)(base + 4096);

    // weights on the GPU, radius chosen on the host
    const double thr_tol = tol > 0.0 ? tol : (prec == LGF_F64 ? 1e-13 : 1e-7);
    if (bessel_weights(nullptr, 2.0 * alpha, kNoAllocWeightCap, w64, s) != LGF_OK)
        return err(LGF_ECUDA, "weight kernel launch failed");
    if (cudaMemcpyAsync(h_w, w64, sizeof(h_w), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return err(LGF_ECUDA, "weight copy failed");
    int R = 0;
    const double thr = thr_tol / 8.0 * h_w[0];
    while (R < kNoAllocWeightCap && h_w[R] >= thr) ++R;
    if (alpha == 0.0) R = 0;
    if (alpha > 0.0 && h_w[kNoAllocWeightCap] >= thr) return err(LGF_EUNSUPPORTED, "alpha needs a radius above 128");
    const int nr = R == 0 ? 0 : (R + b - 1) / b;
    const int nd = 2 * nr + 1;
    if (nd > 33) return err(LGF_EUNSUPPORTED, "stencil reaches more than 16 blocks");
    k_to_float<<<1, 256, 0, s>>>(w64, w32, R + 1);

    // block-lookup box: sources and targets grown by nr blocks
    int lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
        lo[d] = INT32_MAX;
        hi[d] = INT32_MIN;
    }
    for (const lgf_blockset *bs : {src, tgt})
        for (int i = 0; i < bs->nblocks; ++i)
            for (int d = 0; d < 3; ++d) {
                lo[d] = std::min(lo[d], bs->coords[3 * i + d] - nr);
                hi[d] = std::max(hi[d], bs->coords[3 * i + d] + nr);
            }
    for (int d = 0; d < 3; ++d)
        if (hi[d] - lo[d] + 1 > kNoAllocGrid) return err(LGF_EUNSUPPORTED, "block sets span more than 64 blocks");
    const size_t ncell = (size_t)kNoAllocGrid * kNoAllocGrid * kNoAllocGrid;
    memset(h_gS, 0, ncell * sizeof(int32_t));
    memset(h_gX, 0, ncell * sizeof(int32_t));
    memset(h_gY, 0, ncell * sizeof(int32_t));
    memset(h_gC, 0, ncell);
    auto cell = [&](int x, int y, int z) -> long {
        x -= lo[0];
        y -= lo[1];
        z -= lo[2];
        if (x < 0 || y < 0 || z < 0 || x >= kNoAllocGrid || y >= kNoAllocGrid || z >= kNoAllocGrid) return -1;
        return ((long)z * kNoAllocGrid + y) * kNoAllocGrid + x;
    };
    for (int i = 0; i < src->nblocks; ++i) {
        const long c = cell(src->coords[3 * i], src->coords[3 * i + 1], src->coords[3 * i + 2]);
        if (h_gS[c]) return err(LGF_EINVAL, "duplicate block in the source set");
        h_gS[c] = i + 1;
    }
    for (int i = 0; i < tgt->nblocks; ++i) {
        const int *t = tgt->coords + 3 * i;
        const long c = cell(t[0], t[1], t[2]);
        if (h_gC[c] & 2) return err(LGF_EINVAL, "duplicate block in the target set");
        h_gC[c] |= 2;
        for (int dz = -nr; dz <= nr; ++dz) h_gC[cell(t[0], t[1], t[2] + dz)] |= 1;   // y-pass candidates
    }
    int n1 = 0, n2 = 0;
    for (int i = 0; i < src->nblocks; ++i)
        for (int dx = -nr; dx <= nr; ++dx) {
            const int x = src->coords[3 * i] + dx, y = src->coords[3 * i + 1], z = src->coords[3 * i + 2];
            const long c = cell(x, y, z);
            if (h_gX[c]) continue;
            bool need = false;
            for (int dy = -nr; dy <= nr && !need; ++dy) {
                const long q = cell(x, y + dy, z);
                need = q >= 0 && (h_gC[q] & 1);
            }
            if (!need) continue;
            if (n1 >= kNoAllocMaxInter) return err(LGF_EUNSUPPORTED, "more than 8192 blocks after the x pass");
            h_x1[3 * n1] = x;
            h_x1[3 * n1 + 1] = y;
            h_x1[3 * n1 + 2] = z;
            h_gX[c] = ++n1;
        }
    for (int i = 0; i < tgt->nblocks; ++i)
        for (int dz = -nr; dz <= nr; ++dz) {
            const int x = tgt->coords[3 * i], y = tgt->coords[3 * i + 1], z = tgt->coords[3 * i + 2] + dz;
            const long c = cell(x, y, z);
            if (h_gY[c]) continue;
            bool need = false;
            for (int dy = -nr; dy <= nr && !need; ++dy) {
                const long q = cell(x, y + dy, z);
                need = q >= 0 && h_gX[q] > 0;
            }
            if (!need) continue;
            if (n2 >= kNoAllocMaxInter) return err(LGF_EUNSUPPORTED, "more than 8192 blocks after the y pass");
            h_y2[3 * n2] = x;
            h_y2[3 * n2 + 1] = y;
            h_y2[3 * n2 + 2] = z;
            h_gY[c] = ++n2;
        }
    if (n2 == 0) {
        if (cudaMemsetAsync(u_dev, 0, (size_t)tgt->nblocks * b3 * nf * esz, s) != cudaSuccess)
            return err(LGF_ECUDA, "cudaMemsetAsync failed");
        return LGF_OK;
    }
    // neighbour tables of the three passes, one after the other
    const int nout[3] = {n1, n2, tgt->nblocks};
    const int32_t *outs[3] = {h_x1, h_y2, tgt->coords};
    const int32_t *grids[3] = {h_gS, h_gX, h_gY};
    size_t off[3], nn = 0;
    for (int p = 0; p < 3; ++p) {
        off[p] = nn;
        for (int o = 0; o < nout[p]; ++o)
            for (int d = -nr; d <= nr; ++d) {
                int c[3] = {outs[p][3 * o], outs[p][3 * o + 1], outs[p][3 * o + 2]};
                c[p] += d;
                const long q = cell(c[0], c[1], c[2]);
                h_nbr[nn++] = q >= 0 ? grids[p][q] - 1 : -1;
            }
    }
    const size_t nbr_bytes = nn * sizeof(int32_t);
    const size_t x1_off = (4096 + nbr_bytes + 255) & ~size_t(255);
    const size_t x1_bytes = (size_t)n1 * b3 * nf * esz;
    const size_t y2_off = (x1_off + x1_bytes + 255) & ~size_t(255);
    const size_t y2_bytes = (size_t)n2 * b3 * nf * esz;
    if (y2_off + y2_bytes > kNoAllocBytes)
        return err(LGF_EUNSUPPORTED, "intermediate fields exceed the 32 MiB scratch array");
    if (cudaMemcpyAsync(nbr_dev, h_nbr, nbr_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return err(LGF_ECUDA, "neighbour table copy failed");
    const int ntgt = tgt->nblocks, nsrc = src->nblocks;
    const int64_t istr[3] = {(int64_t)nsrc * (int64_t)b3, (int64_t)n1 * (int64_t)b3, (int64_t)n2 * (int64_t)b3};
    const int64_t ostr[3] = {(int64_t)n1 * (int64_t)b3, (int64_t)n2 * (int64_t)b3, (int64_t)ntgt * (int64_t)b3};
    for (int p = 0; p < 3; ++p) {
        if (nout[p] == 0) continue;
        lgf_status st;
        if (prec == LGF_F64) {
            const double *in = p == 0 ? (const double *)f_dev : (const double *)(base + (p == 1 ? x1_off : y2_off));
            double *o = p == 2 ? (double *)u_dev : (double *)(base + (p == 0 ? x1_off : y2_off));
            st = launch_sep<double>(nullptr, p, b, nout[p], nf, s, in, o, nbr_dev + off[p], w64, R, nr, istr[p],
                                    ostr[p]);
        } else {
            const float *in = p == 0 ? (const float *)f_dev : (const float *)(base + (p == 1 ? x1_off : y2_off));
            float *o = p == 2 ? (float *)u_dev : (float *)(base + (p == 0 ? x1_off : y2_off));
            st = launch_sep<float>(nullptr, p, b, nout[p], nf, s, in, o, nbr_dev + off[p], w32, R, nr, istr[p],
                                   ostr[p]);
        }
        if (st != LGF_OK) return err(LGF_ECUDA, "pass kernel launch failed");
    }
    return LGF_OK;
}
