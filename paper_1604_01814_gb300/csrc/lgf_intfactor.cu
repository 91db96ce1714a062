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
#include <unordered_map>
#include <unordered_set>

#include "lgf_internal.cuh"

namespace lgf {

IntfPlan::~IntfPlan()
{
    for (auto &p : pass) cudaFree(p.nbr_dev);
}

namespace {

constexpr int kThreads = 256;
constexpr int kSlabElems = 12288;   // staged elements per CTA

inline int64_t pack(int x, int y, int z)
{
    return (((int64_t)(x + (1 << 20))) << 42) | (((int64_t)(y + (1 << 20))) << 21) | (int64_t)(z + (1 << 20));
}

// One pass along `ax`.  in/out are field arrays on block sets (stride
// in_stride / out_stride elements per field).  nbr[o][d] (d = 0..2nr) is the
// input block at offset d - nr along ax from output block o, or -1.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_sep_pass(const T *__restrict__ in, T *__restrict__ out,
                                                        const int *__restrict__ nbr, const T *__restrict__ wg, int R,
                                                        int nr, int b, int lb, int ax, int slab, int64_t in_stride,
                                                        int64_t out_stride)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *w = reinterpret_cast<T *>(smem_raw);
    T *s = w + ((R + 1 + 3) & ~3);
    for (int i = threadIdx.x; i <= R; i += blockDim.x) w[i] = wg[i];
    const int o = blockIdx.x;
    const int s0 = blockIdx.y * slab;            // first slab coordinate
    const int ns = min(slab, b - s0);
    const int ext = b + 2 * R;
    const int nd = 2 * nr + 1;
    const int *nb = nbr + (int64_t)o * nd;
    const T *inf = in + blockIdx.z * in_stride;
    T *outf = out + blockIdx.z * out_stride;
    const int bm = b - 1;
    // Staged region, x fastest:
    //   ax 0: [ns][b][ext]   (slab over z, lines along x)
    //   ax 1: [ns][ext][b]   (slab over z, lines along y)
    //   ax 2: [ext][ns][b]   (slab over y, lines along z)
    const int total = ns * b * ext;
    for (int it = threadIdx.x; it < total; it += blockDim.x) {
        int x, y, z, e;  // e: extended coordinate along ax, in [-R, b + R)
        if (ax == 0) {
            e = it % ext - R;
            y = (it / ext) % b;
            z = s0 + it / (ext * b);
            x = e;
        } else if (ax == 1) {
            x = it % b;
            e = (it / b) % ext - R;
            z = s0 + it / (b * ext);
            y = e;
        } else {
            x = it % b;
            y = s0 + (it / b) % ns;
            e = it / (b * ns) - R;
            z = e;
        }
        const int d = (e + nr * b) >> lb;        // neighbour slot 0..2nr
        const int bi = nb[d];
        T v = T(0);
        if (bi >= 0) {
            const int xl = ax == 0 ? (e & bm) : x;
            const int yl = ax == 1 ? (e & bm) : y;
            const int zl = ax == 2 ? (e & bm) : z;
            v = inf[((int64_t)bi << (3 * lb)) + (((zl << lb) + yl) << lb) + xl];
        }
        s[it] = v;
    }
    __syncthreads();
    const int nout = ns * b * b;
    for (int it = threadIdx.x; it < nout; it += blockDim.x) {
        const int x = it & bm;
        const int y2 = (it >> lb) & bm;          // second fastest output coordinate
        const int sl = it >> (2 * lb);           // slab-local coordinate
        int c, st;                               // centre index in s, stride along ax
        int X, Y, Z;
        if (ax == 0) {
            X = x; Y = y2; Z = s0 + sl;
            c = (sl * b + Y) * ext + (X + R);
            st = 1;
        } else if (ax == 1) {
            X = x; Y = y2; Z = s0 + sl;
            c = (sl * ext + (Y + R)) * b + X;
            st = b;
        } else {
            // slab over y: it -> (x, z, y_local)
            X = x; Z = y2; Y = s0 + sl;
            c = ((Z + R) * ns + sl) * b + X;
            st = ns * b;
        }
        T acc = w[0] * s[c];
        for (int k = 1; k <= R; ++k) acc += w[k] * (s[c - k * st] + s[c + k * st]);
        outf[((int64_t)o << (3 * lb)) + (((Z << lb) + Y) << lb) + X] = acc;
    }
}

__global__ void k_to_float(const double *a, float *b, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

int log2i(int v)
{
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

int slab_for(int b, int R)
{
    const int per = b * (b + 2 * R);
    return std::max(1, std::min(b, kSlabElems / per));
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
    for (auto &p : ctx->iplans)
        if (p->b == b && p->nr == nr && p->src == sv && p->tgt == tv) {
            *out = p.get();
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
        ctx->iplans.push_back(std::move(plan));
    *out = ctx->iplans.back().get();
    return LGF_OK;
}

lgf_status intf_prepare_scratch(lgf_ctx *ctx, const IntfPlan *pl, int nfields)
{
    const size_t esz = ctx->prec == LGF_F64 ? 8 : 4;
    const size_t b3 = (size_t)pl->b * pl->b * pl->b;
    lgf_status st = ensure_scratch(ctx, &ctx->scrA, &ctx->scrA_bytes, std::max<size_t>(1, pl->n1) * b3 * nfields * esz);
    if (st != LGF_OK) return st;
    return ensure_scratch(ctx, &ctx->scrB, &ctx->scrB_bytes, std::max<size_t>(1, pl->n2) * b3 * nfields * esz);
}

template <typename T>
static lgf_status run_sep(lgf_ctx *ctx, IntfPlan *pl, const T *w, int R, const T *f, T *u, int nfields,
                          cudaStream_t s)
{
    static bool attr = false;
    if (!attr) {
        LGF_CUDA(ctx, cudaFuncSetAttribute(k_sep_pass<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        attr = true;
    }
    const int b = pl->b, lb = log2i(b), nr = pl->nr;
    const int64_t b3 = (int64_t)b * b * b;
    const int slab = slab_for(b, R);
    const int nslab = (b + slab - 1) / slab;
    const size_t smem = sizeof(T) * (((R + 1 + 3) & ~3) + (size_t)slab * b * (b + 2 * R));
    const int nsrc = (int)(pl->src.size() / 3), ntgt = (int)(pl->tgt.size() / 3);
    T *X1 = (T *)ctx->scrA, *Y2 = (T *)ctx->scrB;
    const T *ins[3] = {f, X1, Y2};
    T *outs[3] = {X1, Y2, u};
    const int64_t istr[3] = {nsrc * b3, pl->n1 * b3, pl->n2 * b3};
    const int64_t ostr[3] = {pl->n1 * b3, pl->n2 * b3, ntgt * b3};
    for (int p = 0; p < 3; ++p) {
        if (pl->pass[p].nout == 0) continue;
        dim3 grid(pl->pass[p].nout, nslab, nfields);
        static const char *names[3] = {"intfactor_pass_x", "intfactor_pass_y", "intfactor_pass_z"};
        const int ph = prof_begin(ctx, s, names[p]);
        k_sep_pass<T><<<grid, kThreads, smem, s>>>(ins[p], outs[p], pl->pass[p].nbr_dev, w, R, nr, b, lb, p, slab,
                                                   istr[p], ostr[p]);
        LGF_CHECK_LAUNCH(ctx, "intfactor pass");
        prof_end(ctx, s, ph);
    }
    return LGF_OK;
}

lgf_status intf_run(lgf_ctx *ctx, IntfPlan *pl, const IntfWeights *w, const void *f, void *u, int nfields,
                    cudaStream_t s)
{
    lgf_status st = intf_prepare_scratch(ctx, pl, nfields);
    if (st != LGF_OK) return st;
    const int ntgt = (int)(pl->tgt.size() / 3);
    const size_t esz = ctx->prec == LGF_F64 ? 8 : 4;
    const size_t b3 = (size_t)pl->b * pl->b * pl->b;
    if (pl->pass[2].nout > 0 && pl->n2 == 0) {
        // no source reaches any target: the result is zero
        LGF_CUDA(ctx, cudaMemsetAsync(u, 0, (size_t)ntgt * b3 * nfields * esz, s));
        return LGF_OK;
    }
    if (ctx->prec == LGF_F64)
        return run_sep<double>(ctx, pl, w->w64, w->R, (const double *)f, (double *)u, nfields, s);
    return run_sep<float>(ctx, pl, w->w32, w->R, (const float *)f, (float *)u, nfields, s);
}

}  // namespace lgf
