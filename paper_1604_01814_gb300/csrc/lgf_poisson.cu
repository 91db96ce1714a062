// LGF Poisson apply: u = dx^2 G_L * f on block sets (Sec. 2.2, Eq. dpoisson_conv).
//
// One problem's source and target block sets are placed in the bounding box of
// their union (extent L per axis).  G_L is even in every axis, so its circular
// embedding h[m] = G_L(min(m, M - m)) on a box of M >= 2L - 1 points per axis
// reproduces every source-target offset exactly, and the spectrum of h is real
// and even: only (Mx/2+1)(My/2+1)(Mz/2+1) reals are stored, computed once per
// box shape from the FP64 table (the pre-processing of App. A) and shared by
// every problem and field with that shape.  The apply is the exact lattice
// convolution (no far-field approximation) in five pruned passes:
//
//   X  : R2C along x of the source rows (two real rows per complex FFT),
//        gathered from the block layout              f   -> A [z][y][kx]
//   Y  : along y over the source z-planes            A   -> B [z][ky][kx]
//   Z  : along z, times the kernel spectrum, inverse along z, keeping the
//        target z-planes (in place)                  B   -> B [z'][ky][kx]
//   Yi : inverse along y, keeping the target rows    B   -> A [z'][y'][kx]
//   Xi : C2R along x, keeping the target points, times dx^2, scattered to the
//        target block layout                         A   -> u
//
// Zero rows, planes and columns outside the source region are never loaded
// from memory; outputs outside the target region are never stored.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <unordered_map>

#include "lgf_poisson_fused.cuh"

namespace lgf {
// The pass launchers are instantiated in lgf_poisson_{f32,f64}_{rows,cols,
// conv,conv_x,conv_y}.cu, which compile in parallel; this unit only calls them.
#define LGF_EXTERN_PASSES(T)                                                                                      \
    extern template lgf_status launch_row_forward<T>(lgf_ctx *, const PoissonGeom &, const T *, Cx<T> *,        \
                                                     const Cx<T> *, int, int, int, cudaStream_t);                \
    extern template lgf_status launch_row_inverse<T>(lgf_ctx *, const PoissonGeom &, const Cx<T> *, T *,        \
                                                     const Cx<T> *, int, int, cudaStream_t);                     \
    extern template lgf_status launch_col_forward<T>(lgf_ctx *, int, int, int, int, const Cx<T> *, Cx<T> *, int, \
                                                     int, int64_t, int64_t, int64_t, int64_t, int64_t, int64_t,   \
                                                     const Cx<T> *, pk::RowFlags, cudaStream_t, const char *);   \
    extern template lgf_status launch_col_inverse<T>(lgf_ctx *, int, int, int, int, const Cx<T> *, Cx<T> *, int, \
                                                     int, int64_t, int64_t, int64_t, int64_t, int64_t, int64_t,   \
                                                     const Cx<T> *, cudaStream_t, const char *);                 \
    extern template lgf_status launch_col_convolve<T, 0>(lgf_ctx *, const PoissonGeom &, Cx<T> *, const T *,   \
                                                         const Cx<T> *, int, cudaStream_t);                      \
    extern template lgf_status launch_col_convolve<T, 1>(lgf_ctx *, const PoissonGeom &, Cx<T> *, const T *,   \
                                                         const Cx<T> *, int, cudaStream_t);                      \
    extern template lgf_status launch_col_convolve<T, 2>(lgf_ctx *, const PoissonGeom &, Cx<T> *, const T *,   \
                                                         const Cx<T> *, int, cudaStream_t);                      \
    extern template lgf_status launch_row_forward_rag<T>(lgf_ctx *, int, pk::RowJob<T> *, int, cudaStream_t);    \
    extern template lgf_status launch_row_inverse_rag<T>(lgf_ctx *, int, bool, pk::RowJob<T> *, int,             \
                                                         cudaStream_t);                                          \
    extern template lgf_status launch_col_forward_rag<T>(lgf_ctx *, int, pk::ColJob<T> *, int, cudaStream_t);    \
    extern template lgf_status launch_col_inverse_rag<T>(lgf_ctx *, int, bool, pk::ColJob<T> *, int,             \
                                                         cudaStream_t);                                          \
    extern template lgf_status launch_col_convolve_rag<T, 0>(lgf_ctx *, int, int, pk::ConvJob<T> *, int,         \
                                                             cudaStream_t);                                      \
    extern template lgf_status launch_col_convolve_rag<T, 1>(lgf_ctx *, int, int, pk::ConvJob<T> *, int,         \
                                                             cudaStream_t);                                      \
    extern template lgf_status launch_col_convolve_rag<T, 2>(lgf_ctx *, int, int, pk::ConvJob<T> *, int,         \
                                                             cudaStream_t);
LGF_EXTERN_PASSES(float)
LGF_EXTERN_PASSES(double)
#undef LGF_EXTERN_PASSES
// the fused y+x inverse: lgf_poisson_f32_fused_<My>_<part>.cu
namespace pk {
#define LGF_EXTERN_YX(MYV)                                                                                     \
    extern template lgf_status yx_launch_my<MYV, 0>(lgf_ctx *, int, int, YXJob *, int, cudaStream_t);         \
    extern template lgf_status yx_launch_my<MYV, 1>(lgf_ctx *, int, int, YXJob *, int, cudaStream_t);
LGF_EXTERN_YX(64)
LGF_EXTERN_YX(80)
LGF_EXTERN_YX(96)
LGF_EXTERN_YX(128)
#undef LGF_EXTERN_YX
}  // namespace pk
}  // namespace lgf

namespace lgf {

namespace {
// 2^k, 3 * 2^k and 5 * 2^k: the box pays at most 1.34x its extent per axis
const int kFftSizes[] = {32,  64,  80,  96,   128,  160,  192,  256,  320,  384,
                         512, 640, 768, 1024, 1280, 1536, 2048, 2560, 3072, 4096};
constexpr int kNumFftSizes = sizeof(kFftSizes) / sizeof(kFftSizes[0]);

// The bump-th supported length above the smallest one >= n (2 kMaxFft if none).
int fft_size_bumped(int n, int bump)
{
    for (int i = 0; i < kNumFftSizes; ++i)
        if (kFftSizes[i] >= n) return i + bump < kNumFftSizes ? kFftSizes[i + bump] : 2 * kMaxFft;
    return 2 * kMaxFft;
}
}  // namespace

int next_fft_size(int n) { return fft_size_bumped(n, 0); }

bool poisson_geometry(const PoissonPlan &pl, const PoissonChoice &ch, PoissonGeom *gp, int64_t *A, int64_t *B)
{
    PoissonGeom &g = *gp;
    const int b = pl.b;
    g.b = b;
    for (int d = 0; d < 3; ++d) {
        const int lo = std::min(pl.slo[d], pl.tlo[d]), hi = std::max(pl.shi[d], pl.thi[d]);
        const int64_t L = ((int64_t)hi - lo + 1) * b;
        g.Ls[d] = (pl.shi[d] - pl.slo[d] + 1) * b;
        g.Lt[d] = (pl.thi[d] - pl.tlo[d] + 1) * b;
        g.nbs[d] = pl.shi[d] - pl.slo[d] + 1;
        g.nbt[d] = pl.thi[d] - pl.tlo[d] + 1;
        const bool shift = d < 2 && ch.shift[d];
        if (!shift) {
            // even embedding on the union extent: every offset within +-(L - 1)
            if (L > kMaxFft / 2) return false;
            g.M[d] = fft_size_bumped((int)(2 * L - 1), ch.bump[d]);
            g.s0[d] = (pl.slo[d] - lo) * b;
            g.t0[d] = (pl.tlo[d] - lo) * b;
        } else {
            // shifted window: the Ls + Lt - 1 distinct offsets, source and
            // target both at 0; the forward pass keeps its half-zero inputs
            g.M[d] = fft_size_bumped(g.Ls[d] + g.Lt[d] - 1, ch.bump[d]);
            if (2 * g.Ls[d] > g.M[d]) return false;
            g.s0[d] = 0;
            g.t0[d] = 0;
        }
        if (g.M[d] > kMaxFft) return false;
    }
    g.xasym = ch.shift[0];
    g.xc = ch.shift[0] ? (pl.tlo[0] - pl.slo[0]) * b : 0;
    g.xP = ch.shift[0] ? g.Lt[0] + (g.M[0] - g.Ls[0] + 1 - g.Lt[0]) / 2 : g.M[0] / 2;
    g.yasym = ch.shift[1];
    g.yc = ch.shift[1] ? (pl.tlo[1] - pl.slo[1]) * b : 0;
    g.yP = ch.shift[1] ? g.Lt[1] + (g.M[1] - g.Ls[1] + 1 - g.Lt[1]) / 2 : g.M[1] / 2;
    g.zvar = ch.zvar;
    g.fuse = ch.fuse;
    g.Kx = g.M[0] / 2 + 1;
    g.ldA_y = std::max(g.Ls[1], g.Lt[1]);
    *A = (int64_t)std::max(g.Ls[2], g.Lt[2]) * g.ldA_y * g.Kx;
    *B = (int64_t)std::max(g.Ls[2], g.Lt[2]) * g.M[1] * g.Kx;
    return true;
}

PoissonChoice poisson_default_choice(const PoissonPlan &pl, bool allow_shift)
{
    PoissonChoice ch;
    if (!allow_shift) return ch;
    // the shifted window along x and y where it gives a shorter transform
    // (it pays where source and target extents differ: a small body and its
    // long wake)
    for (int d = 0; d < 2; ++d) {
        PoissonChoice e = ch, s = ch;
        s.shift[d] = 1;
        PoissonGeom ge{}, gs{};
        int64_t a, bb;
        if (poisson_geometry(pl, s, &gs, &a, &bb) && poisson_geometry(pl, e, &ge, &a, &bb) && gs.M[d] < ge.M[d])
            ch.shift[d] = 1;
    }
    return ch;
}

void poisson_set_choice(PoissonPlan *pl, const PoissonChoice &ch)
{
    PoissonGeom g = pl->g;   // keeps the device maps and strides
    int64_t A = 0, B = 0;
    poisson_geometry(*pl, ch, &g, &A, &B);
    pl->g = g;
    pl->choice = ch;
    pl->A_elems = A;
    pl->B_elems = B;
}

Spectrum::~Spectrum() { cudaFree(dev); }

PoissonPlan::~PoissonPlan()
{
    cudaFree(srcmap_dev);
    cudaFree(tgtmap_dev);
    cudaFree(srcrow_dev);
    cudaFree(tgtrow_dev);
}

namespace {

__global__ void k_twiddles(int M, void *out, int dbl)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    double s, c;
    sincospi(-2.0 * m / M, &s, &c);
    if (dbl) {
        ((Cx<double> *)out)[m] = {c, s};
    } else {
        ((Cx<float> *)out)[m] = {(float)c, (float)s};
    }
}

// Spectrum of a shifted window: the complex forward transform at
// kx <= Mx/2, ky < nky (My/2 + 1 when the window is even in y, My when it
// is shifted in y), kz <= Mz/2 (even in z), scaled by 1/(Mx My Mz).
template <typename T>
__global__ void k_extract_c(const Cx<double> *__restrict__ B, Cx<T> *__restrict__ spec, int Mx, int My, int Mz,
                            int nky)
{
    const int K = Mx / 2 + 1, Khy = nky, Khz = Mz / 2 + 1;
    const int64_t n = (int64_t)K * Khy * Khz;
    const double sc = 1.0 / ((double)Mx * My * Mz);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int kx = (int)(i % K);
        const int ky = (int)((i / K) % Khy);
        const int kz = (int)(i / ((int64_t)K * Khy));
        const Cx<double> v = B[((int64_t)kz * My + ky) * K + kx];
        spec[i] = Cx<T>{T(v.x * sc), T(v.y * sc)};
    }
}

// Spectrum extraction: real part of the forward transform of the embedded
// kernel at kx <= Mx/2, ky <= My/2, kz <= Mz/2, scaled by 1/(Mx My Mz).
template <typename T>
__global__ void k_extract(const Cx<double> *__restrict__ B, T *__restrict__ spec, int Mx, int My, int Mz)
{
    const int K = Mx / 2 + 1, Khy = My / 2 + 1, Khz = Mz / 2 + 1;
    const int64_t n = (int64_t)K * Khy * Khz;
    const double sc = 1.0 / ((double)Mx * My * Mz);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int kx = (int)(i % K);
        const int ky = (int)((i / K) % Khy);
        const int kz = (int)(i / ((int64_t)K * Khy));
        spec[i] = T(B[((int64_t)kz * My + ky) * K + kx].x * sc);
    }
}

int log2i(int v)
{
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

constexpr size_t kFusedSmemMax = 200 * 1024;   // shared memory of one fused CTA, at most

bool yx_info(int My, int Mx, size_t *work, int *lpc)
{
    switch (My) {
    case 64: return pk::yx_info_my<64>(Mx, work, lpc);
    case 80: return pk::yx_info_my<80>(Mx, work, lpc);
    case 96: return pk::yx_info_my<96>(Mx, work, lpc);
    case 128: return pk::yx_info_my<128>(Mx, work, lpc);
    default: return false;
    }
}

lgf_status yx_launch(lgf_ctx *ctx, int My, int Mx, int ncl, pk::YXJob *jobs, int n, cudaStream_t s)
{
    switch (My) {
    case 64: return pk::yx_part(Mx) ? pk::yx_launch_my<64, 1>(ctx, Mx, ncl, jobs, n, s)
                                    : pk::yx_launch_my<64, 0>(ctx, Mx, ncl, jobs, n, s);
    case 80: return pk::yx_part(Mx) ? pk::yx_launch_my<80, 1>(ctx, Mx, ncl, jobs, n, s)
                                    : pk::yx_launch_my<80, 0>(ctx, Mx, ncl, jobs, n, s);
    case 96: return pk::yx_part(Mx) ? pk::yx_launch_my<96, 1>(ctx, Mx, ncl, jobs, n, s)
                                    : pk::yx_launch_my<96, 0>(ctx, Mx, ncl, jobs, n, s);
    case 128: return pk::yx_part(Mx) ? pk::yx_launch_my<128, 1>(ctx, Mx, ncl, jobs, n, s)
                                     : pk::yx_launch_my<128, 0>(ctx, Mx, ncl, jobs, n, s);
    default: return fail(ctx, LGF_EUNSUPPORTED, "fused inverse: length along y not instantiated");
    }
}

pk::YXJob yx_job(const PoissonGeom &g, const Cx<float> *B, float *u, const Cx<float> *twy, const Cx<float> *twx,
                 int nf, int rpb)
{
    pk::YXJob j{};
    j.g = g;
    j.B = B;
    j.u = u;
    j.twy = twy;
    j.twx = twx;
    j.nf = nf;
    j.lb = log2i(g.b);
    j.rpb = rpb;
    return j;
}

// The five passes of one problem (all fields in each launch); in spectrum
// mode only the forward transform of a dense box (x, y, then z in place).
template <typename T>
lgf_status run_passes(lgf_ctx *ctx, const PoissonGeom &g, const T *f, T *u, Cx<T> *A, Cx<T> *B, const T *spec,
                      int nf, int dense_ld, bool spectrum_mode, cudaStream_t s)
{
    const bool dbl = sizeof(T) == 8;
    lgf_status st = LGF_OK;
    const Cx<T> *twx = (const Cx<T> *)twiddles(ctx, g.M[0], dbl, &st);
    if (st != LGF_OK) return st;
    const Cx<T> *twy = (const Cx<T> *)twiddles(ctx, g.M[1], dbl, &st);
    if (st != LGF_OK) return st;
    const Cx<T> *twz = (const Cx<T> *)twiddles(ctx, g.M[2], dbl, &st);
    if (st != LGF_OK) return st;
    const int lb = log2i(g.b);
    const int K = g.Kx, My = g.M[1], Mz = g.M[2];
    const int64_t planeA = (int64_t)g.ldA_y * K, planeB = (int64_t)My * K;
    if ((st = launch_row_forward<T>(ctx, g, f, A, twx, nf, lb, dense_ld, s)) != LGF_OK) return st;
    const pk::RowFlags fsrc{spectrum_mode ? nullptr : g.srcrow, lb};
    if ((st = launch_col_forward<T>(ctx, My, K, g.Ls[2], nf, A, B, g.s0[1], g.Ls[1], K, K, planeA, planeB, g.Astride,
                                    g.Bstride, twy, fsrc, s,
                                    spectrum_mode ? "spectrum_y_forward" : "poisson_y_forward")) != LGF_OK)
        return st;
    if (spectrum_mode)
        return launch_col_forward<T>(ctx, Mz, K, My, nf, B, B, 0, Mz, planeB, planeB, K, K, g.Bstride, g.Bstride, twz,
                                     pk::RowFlags{}, s, "spectrum_z_forward");
    // the z pass for the spectrum's layout (even, shifted x, shifted y)
    st = g.yasym ? launch_col_convolve<T, 2>(ctx, g, B, spec, twz, nf, s)
       : g.xasym ? launch_col_convolve<T, 1>(ctx, g, B, spec, twz, nf, s)
                 : launch_col_convolve<T, 0>(ctx, g, B, spec, twz, nf, s);
    if (st != LGF_OK) return st;
    if constexpr (sizeof(T) == 4) {
        int rpb = 0;
        const int ncl = poisson_fused_ncl(g, &rpb);
        if (ncl > 0) {
            pk::YXJob j = yx_job(g, B, u, twy, twx, nf, rpb);
            return yx_launch(ctx, My, g.M[0], ncl, &j, 1, s);
        }
    }
    if ((st = launch_col_inverse<T>(ctx, My, K, g.Lt[2], nf, B, A, g.t0[1], g.Lt[1], K, K, planeB, planeA, g.Bstride,
                                    g.Astride, twy, s, "poisson_y_inverse")) != LGF_OK)
        return st;
    return launch_row_inverse<T>(ctx, g, A, u, twx, nf, lb, s);
}

}  // namespace

int poisson_fused_ncl(const PoissonGeom &g, int *rpb)
{
    size_t work = 0;
    int lpc = 0;
    if (!g.fuse || !yx_info(g.M[1], g.M[0], &work, &lpc) || g.Lt[1] < 2) return 0;
    // the smallest cluster whose CTAs hold their rows in one batch of line
    // pairs and in shared memory
    for (int ncl : {1, 2, 4}) {
        int r = (g.Lt[1] + ncl - 1) / ncl;
        r += r & 1;
        if (r <= 2 * lpc && (size_t)r * g.Kx * sizeof(Cx<float>) + work <= kFusedSmemMax) {
            *rpb = r;
            return ncl;
        }
    }
    return 0;
}

const void *twiddles(lgf_ctx *ctx, int M, bool dbl, lgf_status *st)
{
    auto &tab = dbl ? ctx->tw64 : ctx->tw32;
    auto it = tab.find(M);
    if (it != tab.end()) return it->second;
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, (size_t)M * (dbl ? 16 : 8));
    if (e != cudaSuccess) {
        *st = fail(ctx, LGF_ENOMEM, "twiddle table allocation failed");
        return nullptr;
    }
    k_twiddles<<<(M + 255) / 256, 256>>>(M, p, dbl ? 1 : 0);
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaFree(p);
        *st = cuda_fail(ctx, e, "twiddle kernel");
        return nullptr;
    }
    tab[M] = p;
    return p;
}

lgf_status poisson_plan(lgf_ctx *ctx, const lgf_blockset *src, const lgf_blockset *tgt, PoissonPlan **out)
{
    const int b = src->b;
    const std::vector<int32_t> sv(src->coords, src->coords + 3 * (size_t)src->nblocks);
    const std::vector<int32_t> tv(tgt->coords, tgt->coords + 3 * (size_t)tgt->nblocks);
    if (PoissonPlan *hit = ctx->pplans.find(
            [&](const PoissonPlan &p) { return p.b == b && p.src == sv && p.tgt == tv; }, ctx->counters.epoch)) {
        *out = hit;
        return LGF_OK;
    }
    int slo[3], shi[3], tlo[3], thi[3], lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
        slo[d] = tlo[d] = INT32_MAX;
        shi[d] = thi[d] = INT32_MIN;
    }
    for (int i = 0; i < src->nblocks; ++i)
        for (int d = 0; d < 3; ++d) {
            slo[d] = std::min(slo[d], sv[3 * i + d]);
            shi[d] = std::max(shi[d], sv[3 * i + d]);
        }
    for (int i = 0; i < tgt->nblocks; ++i)
        for (int d = 0; d < 3; ++d) {
            tlo[d] = std::min(tlo[d], tv[3 * i + d]);
            thi[d] = std::max(thi[d], tv[3 * i + d]);
        }
    auto plan = std::make_unique<PoissonPlan>();
    plan->b = b;
    plan->src = sv;
    plan->tgt = tv;
    for (int d = 0; d < 3; ++d) {
        plan->slo[d] = slo[d];
        plan->shi[d] = shi[d];
        plan->tlo[d] = tlo[d];
        plan->thi[d] = thi[d];
        lo[d] = std::min(slo[d], tlo[d]);
        hi[d] = std::max(shi[d], thi[d]);
        if (((int64_t)hi[d] - lo[d] + 1) * b > kMaxFft / 2)
            return fail(ctx, LGF_EUNSUPPORTED, "poisson: union of source and target spans more than 2048 points");
    }
    PoissonGeom &g = plan->g;
    const PoissonChoice ch = poisson_default_choice(*plan, ctx->opt_xshift);
    if (!poisson_geometry(*plan, ch, &g, &plan->A_elems, &plan->B_elems))
        return fail(ctx, LGF_EUNSUPPORTED, "poisson: no supported transform length for the block sets");
    plan->choice = ch;
    std::vector<int> smap((size_t)g.nbs[0] * g.nbs[1] * g.nbs[2], -1);
    std::vector<int> tmap((size_t)g.nbt[0] * g.nbt[1] * g.nbt[2], -1);
    for (int i = 0; i < src->nblocks; ++i) {
        const size_t k = ((size_t)(sv[3 * i + 2] - slo[2]) * g.nbs[1] + (sv[3 * i + 1] - slo[1])) * g.nbs[0] +
                         (sv[3 * i] - slo[0]);
        if (smap[k] >= 0) return fail(ctx, LGF_EINVAL, "poisson: duplicate block in the source set");
        smap[k] = i;
    }
    for (int i = 0; i < tgt->nblocks; ++i) {
        const size_t k = ((size_t)(tv[3 * i + 2] - tlo[2]) * g.nbt[1] + (tv[3 * i + 1] - tlo[1])) * g.nbt[0] +
                         (tv[3 * i] - tlo[0]);
        if (tmap[k] >= 0) return fail(ctx, LGF_EINVAL, "poisson: duplicate block in the target set");
        tmap[k] = i;
    }
    if (cudaMalloc(&plan->srcmap_dev, smap.size() * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&plan->tgtmap_dev, tmap.size() * sizeof(int)) != cudaSuccess)
        return fail(ctx, LGF_ENOMEM, "poisson: block map allocation failed");
    LGF_CUDA(ctx, cudaMemcpy(plan->srcmap_dev, smap.data(), smap.size() * sizeof(int), cudaMemcpyHostToDevice));
    LGF_CUDA(ctx, cudaMemcpy(plan->tgtmap_dev, tmap.data(), tmap.size() * sizeof(int), cudaMemcpyHostToDevice));
    g.srcmap = plan->srcmap_dev;
    g.tgtmap = plan->tgtmap_dev;
    // row blocks (y, z) with no block along x: the x passes skip them and the
    // y-forward pass does not read their rows
    auto row_flags = [&](const std::vector<int> &map, const int nb[3], unsigned long long **dev,
                         const unsigned long long **out) -> lgf_status {
        *out = nullptr;
        if (nb[1] > 64) return LGF_OK;
        std::vector<unsigned long long> f((size_t)nb[2], 0ull);
        bool all = true;
        for (int z = 0; z < nb[2]; ++z)
            for (int y = 0; y < nb[1]; ++y) {
                bool any = false;
                for (int x = 0; x < nb[0]; ++x) any = any || map[((size_t)z * nb[1] + y) * nb[0] + x] >= 0;
                if (any)
                    f[z] |= 1ull << y;
                else
                    all = false;
            }
        if (all) return LGF_OK;
        if (cudaMalloc(dev, f.size() * sizeof(unsigned long long)) != cudaSuccess)
            return fail(ctx, LGF_ENOMEM, "poisson: row flag allocation failed");
        LGF_CUDA(ctx, cudaMemcpy(*dev, f.data(), f.size() * sizeof(unsigned long long), cudaMemcpyHostToDevice));
        *out = *dev;
        return LGF_OK;
    };
    lgf_status rst = row_flags(smap, g.nbs, &plan->srcrow_dev, &g.srcrow);
    if (rst == LGF_OK) rst = row_flags(tmap, g.nbt, &plan->tgtrow_dev, &g.tgtrow);
    if (rst != LGF_OK) return rst;
    g.fstride = (int64_t)src->nblocks * b * b * b;
    g.ustride = (int64_t)tgt->nblocks * b * b * b;
    *out = ctx->pplans.insert(std::move(plan), ctx->counters.epoch, [&] { before_evict(ctx); },
                              &ctx->counters.plans_evicted);
    return LGF_OK;
}

lgf_status poisson_spectrum(lgf_ctx *ctx, const PoissonGeom &pg, double alpha, Spectrum **out, cudaStream_t s)
{
    const int *M = pg.M;
    const std::array<int, 3> shape{M[0], M[1], M[2]};
    if (Spectrum *hit = ctx->spectra.find(
            [&](const Spectrum &q) {
                return q.M == shape && q.alpha == alpha && q.xasym == pg.xasym && q.xc == pg.xc && q.xP == pg.xP &&
                       q.yasym == pg.yasym && q.yc == pg.yc && q.yP == pg.yP;
            },
            ctx->counters.epoch)) {
        *out = hit;
        return LGF_OK;
    }
    if (ctx->table_dev == nullptr) return fail(ctx, LGF_ENOTABLE, "poisson: lgf_table_build has not been called");
    const double *table = nullptr;
    lgf_status tst = gk_table(ctx, alpha, &table, s);
    if (tst != LGF_OK) return tst;
    PoissonGeom g{};
    for (int d = 0; d < 3; ++d) {
        g.M[d] = M[d];
        g.s0[d] = 0;
        g.Ls[d] = M[d];
        g.t0[d] = 0;
        g.Lt[d] = M[d];
        g.nbs[d] = g.nbt[d] = 1;
    }
    g.b = 1;
    g.Kx = M[0] / 2 + 1;
    g.ldA_y = M[1];
    const int64_t nbox = (int64_t)M[0] * M[1] * M[2];
    const int64_t nA = (int64_t)M[2] * M[1] * g.Kx;
    g.fstride = nbox;
    g.Astride = nA;
    g.Bstride = nA;
    double *box = nullptr;
    Cx<double> *A = nullptr, *B = nullptr;
    void *spec = nullptr;
    // layouts: even x and y: reals [kz][ky <= My/2][kx]; shifted x: complex,
    // same shape; shifted y: complex [kz][ky < My][kx] (no symmetry in ky)
    const int nky = pg.yasym ? M[1] : M[1] / 2 + 1;
    const bool cplx = pg.xasym || pg.yasym;
    const size_t spec_elems = (size_t)g.Kx * nky * (M[2] / 2 + 1) * (cplx ? 2 : 1);
    const size_t esz = ctx->prec == LGF_F64 ? 8 : 4;
    auto cleanup = [&]() {
        cudaFree(box);
        cudaFree(A);
        cudaFree(B);
    };
    if (cudaMalloc(&box, nbox * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&A, nA * sizeof(Cx<double>)) != cudaSuccess ||
        cudaMalloc(&B, nA * sizeof(Cx<double>)) != cudaSuccess || cudaMalloc(&spec, spec_elems * esz) != cudaSuccess) {
        cleanup();
        cudaFree(spec);
        return fail(ctx, LGF_ENOMEM, "poisson: kernel spectrum scratch allocation failed");
    }
    lgf_status st = kernel_window(ctx, table, M, pg.xc, pg.xP, pg.yc, pg.yP, box, s);
    if (st == LGF_OK)
        st = run_passes<double>(ctx, g, box, nullptr, A, B, nullptr, 1, M[0], true, s);
    if (st == LGF_OK) {
        if (cplx) {
            if (esz == 8)
                k_extract_c<double><<<152 * 4, 256, 0, s>>>(B, (Cx<double> *)spec, M[0], M[1], M[2], nky);
            else
                k_extract_c<float><<<152 * 4, 256, 0, s>>>(B, (Cx<float> *)spec, M[0], M[1], M[2], nky);
        } else if (esz == 8) {
            k_extract<double><<<152 * 4, 256, 0, s>>>(B, (double *)spec, M[0], M[1], M[2]);
        } else {
            k_extract<float><<<152 * 4, 256, 0, s>>>(B, (float *)spec, M[0], M[1], M[2]);
        }
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(ctx, e, "poisson: kernel spectrum");
    }
    cleanup();
    if (st != LGF_OK) {
        cudaFree(spec);
        return st;
    }
    auto sp = std::make_unique<Spectrum>();
    sp->M = shape;
    sp->alpha = alpha;
    sp->xasym = pg.xasym;
    sp->xc = pg.xc;
    sp->xP = pg.xP;
    sp->yasym = pg.yasym;
    sp->yc = pg.yc;
    sp->yP = pg.yP;
    sp->dev = spec;
    *out = ctx->spectra.insert(std::move(sp), ctx->counters.epoch, [&] { before_evict(ctx); },
                               &ctx->counters.plans_evicted);
    return LGF_OK;
}

lgf_status poisson_prepare_scratch(lgf_ctx *ctx, const PoissonPlan *pl, int nfields)
{
    const size_t csz = ctx->prec == LGF_F64 ? 16 : 8;
    lgf_status st = ensure_scratch(ctx, &ctx->cur->A, &ctx->cur->a, (size_t)pl->A_elems * nfields * csz);
    if (st != LGF_OK) return st;
    return ensure_scratch(ctx, &ctx->cur->B, &ctx->cur->b, (size_t)pl->B_elems * nfields * csz);
}

lgf_status poisson_run(lgf_ctx *ctx, PoissonPlan *pl, const Spectrum *sp, const void *f, void *u, int nfields,
                       double dx, cudaStream_t s)
{
    lgf_status st = poisson_prepare_scratch(ctx, pl, nfields);
    if (st != LGF_OK) return st;
    PoissonGeom g = pl->g;
    g.Astride = pl->A_elems;
    g.Bstride = pl->B_elems;
    g.scale = dx * dx;
    if (ctx->prec == LGF_F64)
        return run_passes<double>(ctx, g, (const double *)f, (double *)u, (Cx<double> *)ctx->cur->A,
                                  (Cx<double> *)ctx->cur->B, (const double *)sp->dev, nfields, 0, false, s);
    return run_passes<float>(ctx, g, (const float *)f, (float *)u, (Cx<float> *)ctx->cur->A, (Cx<float> *)ctx->cur->B,
                             (const float *)sp->dev, nfields, 0, false, s);
}

namespace {

// Scratch slices of the ragged run: part i's A at a[i], B at b[i] (complex
// elements), each rounded up to 32 elements (256-byte aligned for FP32).
void ragged_offsets(const RagPart *parts, int n, std::vector<int64_t> *a, std::vector<int64_t> *b, int64_t *atot,
                    int64_t *btot)
{
    a->assign(n, 0);
    b->assign(n, 0);
    int64_t ta = 0, tb = 0;
    for (int i = 0; i < n; ++i) {
        (*a)[i] = ta;
        (*b)[i] = tb;
        ta += (parts[i].plan->A_elems * parts[i].nf + 31) / 32 * 32;
        tb += (parts[i].plan->B_elems * parts[i].nf + 31) / 32 * 32;
    }
    *atot = ta;
    *btot = tb;
}

// Launches of one pass: the groups (one transform length and variant each)
// go round-robin to the branch streams, which fork from s and join it again.
template <class Launch>
lgf_status ragged_pass(lgf_ctx *ctx, cudaStream_t s, int nbr, int ngroups, Launch launch)
{
    const int nb = std::min(nbr, ngroups);
    if (nb <= 1) {
        for (int k = 0; k < ngroups; ++k) {
            lgf_status st = launch(k, s);
            if (st != LGF_OK) return st;
        }
        return LGF_OK;
    }
    LGF_CUDA(ctx, cudaEventRecord(ctx->ev_fork, s));
    for (int b = 0; b < nb; ++b) LGF_CUDA(ctx, cudaStreamWaitEvent(ctx->br[b], ctx->ev_fork, 0));
    for (int k = 0; k < ngroups; ++k) {
        lgf_status st = launch(k, ctx->br[k % nb]);
        if (st != LGF_OK) return st;
    }
    for (int b = 0; b < nb; ++b) {
        LGF_CUDA(ctx, cudaEventRecord(ctx->ev_join[b], ctx->br[b]));
        LGF_CUDA(ctx, cudaStreamWaitEvent(s, ctx->ev_join[b], 0));
    }
    return LGF_OK;
}

// Jobs grouped by a key (the transform length and the compile-time variant),
// groups in order of first appearance.
template <class Job>
struct JobGroups {
    std::vector<std::array<int, 3>> keys;
    std::vector<std::vector<Job>> jobs;
    void add(const std::array<int, 3> &k, const Job &j)
    {
        for (size_t i = 0; i < keys.size(); ++i)
            if (keys[i] == k) {
                jobs[i].push_back(j);
                return;
            }
        keys.push_back(k);
        jobs.push_back({j});
    }
};

template <typename T>
lgf_status run_ragged(lgf_ctx *ctx, const RagPart *parts, int n, cudaStream_t s, int nbr)
{
    const bool dbl = sizeof(T) == 8;
    std::vector<int64_t> ao, bo;
    int64_t at = 0, bt = 0;
    ragged_offsets(parts, n, &ao, &bo, &at, &bt);
    const size_t csz = sizeof(Cx<T>);
    if ((size_t)at * csz > ctx->scr[0].a || (size_t)bt * csz > ctx->scr[0].b)
        return fail(ctx, LGF_EINVAL, "ragged Poisson run: scratch not prepared");
    Cx<T> *A0 = (Cx<T> *)ctx->scr[0].A, *B0 = (Cx<T> *)ctx->scr[0].B;
    JobGroups<pk::RowJob<T>> xf, xi;
    JobGroups<pk::ColJob<T>> yf, yi;
    JobGroups<pk::ConvJob<T>> zc;
    JobGroups<pk::YXJob> yx;
    lgf_status st = LGF_OK;
    for (int i = 0; i < n; ++i) {
        const RagPart &q = parts[i];
        PoissonGeom g = q.plan->g;
        g.Astride = q.plan->A_elems;
        g.Bstride = q.plan->B_elems;
        g.scale = q.dx * q.dx;
        const Cx<T> *tw[3];
        for (int d = 0; d < 3; ++d) {
            tw[d] = (const Cx<T> *)twiddles(ctx, g.M[d], dbl, &st);
            if (st != LGF_OK) return st;
        }
        const int lb = log2i(g.b);
        const int K = g.Kx, My = g.M[1];
        const int64_t planeA = (int64_t)g.ldA_y * K, planeB = (int64_t)My * K;
        Cx<T> *A = A0 + ao[i], *B = B0 + bo[i];
        pk::RowJob<T> r{};
        r.g = g;
        r.in = q.f;
        r.out = A;
        r.tw = tw[0];
        r.npairs = (g.Ls[1] / 2) * g.Ls[2];
        r.lb = lb;
        r.nf = q.nf;
        xf.add({g.M[0], 0, 0}, r);
        pk::ColJob<T> c{};
        c.in = A;
        c.out = B;
        c.tw = tw[1];
        c.rf = pk::RowFlags{g.srcrow, lb};
        c.rs = c.os = K;
        c.in_plane = planeA;
        c.out_plane = planeB;
        c.in_field = g.Astride;
        c.out_field = g.Bstride;
        c.K = K;
        c.nplanes = g.Ls[2];
        c.lo = g.s0[1];
        c.n = g.Ls[1];
        c.nf = q.nf;
        yf.add({My, 0, 0}, c);
        pk::ConvJob<T> z{};
        z.B = B;
        z.spec = q.sp->dev;
        z.tw = tw[2];
        z.field = g.Bstride;
        z.K = K;
        z.My = My;
        z.s0 = g.s0[2];
        z.ns = g.Ls[2];
        z.t0 = g.t0[2];
        z.nt = g.Lt[2];
        z.nf = q.nf;
        const int spec = g.yasym ? 2 : g.xasym ? 1 : 0;
        zc.add({g.M[2], spec, sizeof(T) == 4 ? g.zvar : 0}, z);
        if constexpr (sizeof(T) == 4) {   // the fused y+x inverse where it applies
            int rpb = 0;
            const int ncl = poisson_fused_ncl(g, &rpb);
            if (ncl > 0) {
                yx.add({My, g.M[0], ncl}, yx_job(g, B, (float *)q.u, tw[1], tw[0], q.nf, rpb));
                continue;
            }
        }
        pk::ColJob<T> c2{};
        c2.in = B;
        c2.out = A;
        c2.tw = tw[1];
        c2.rs = c2.os = K;
        c2.in_plane = planeB;
        c2.out_plane = planeA;
        c2.in_field = g.Bstride;
        c2.out_field = g.Astride;
        c2.K = K;
        c2.nplanes = g.Lt[2];
        c2.lo = g.t0[1];
        c2.n = g.Lt[1];
        c2.nf = q.nf;
        yi.add({My, g.t0[1] + g.Lt[1] <= My / 2 ? 1 : 0, 0}, c2);
        pk::RowJob<T> r2{};
        r2.g = g;
        r2.in = A;
        r2.out = q.u;
        r2.tw = tw[0];
        r2.npairs = (g.Lt[1] / 2) * g.Lt[2];
        r2.lb = lb;
        r2.nf = q.nf;
        xi.add({g.M[0], 2 * (g.t0[0] + g.Lt[0]) <= g.M[0] ? 1 : 0, 0}, r2);
    }
    if ((st = ragged_pass(ctx, s, nbr, (int)xf.keys.size(), [&](int k, cudaStream_t bs) {
             return launch_row_forward_rag<T>(ctx, xf.keys[k][0], xf.jobs[k].data(), (int)xf.jobs[k].size(), bs);
         })) != LGF_OK)
        return st;
    if ((st = ragged_pass(ctx, s, nbr, (int)yf.keys.size(), [&](int k, cudaStream_t bs) {
             return launch_col_forward_rag<T>(ctx, yf.keys[k][0], yf.jobs[k].data(), (int)yf.jobs[k].size(), bs);
         })) != LGF_OK)
        return st;
    if ((st = ragged_pass(ctx, s, nbr, (int)zc.keys.size(), [&](int k, cudaStream_t bs) {
             const auto &key = zc.keys[k];
             pk::ConvJob<T> *j = zc.jobs[k].data();
             const int nj = (int)zc.jobs[k].size();
             return key[1] == 2   ? launch_col_convolve_rag<T, 2>(ctx, key[0], key[2], j, nj, bs)
                    : key[1] == 1 ? launch_col_convolve_rag<T, 1>(ctx, key[0], key[2], j, nj, bs)
                                  : launch_col_convolve_rag<T, 0>(ctx, key[0], key[2], j, nj, bs);
         })) != LGF_OK)
        return st;
    // the fused inverses go with the y inverses (both read B)
    const int nyi = (int)yi.keys.size();
    if ((st = ragged_pass(ctx, s, nbr, nyi + (int)yx.keys.size(), [&](int k, cudaStream_t bs) {
             if (k >= nyi) {
                 const auto &key = yx.keys[k - nyi];
                 auto &j = yx.jobs[k - nyi];
                 return yx_launch(ctx, key[0], key[1], key[2], j.data(), (int)j.size(), bs);
             }
             return launch_col_inverse_rag<T>(ctx, yi.keys[k][0], yi.keys[k][1] != 0, yi.jobs[k].data(),
                                              (int)yi.jobs[k].size(), bs);
         })) != LGF_OK)
        return st;
    return ragged_pass(ctx, s, nbr, (int)xi.keys.size(), [&](int k, cudaStream_t bs) {
        return launch_row_inverse_rag<T>(ctx, xi.keys[k][0], xi.keys[k][1] != 0, xi.jobs[k].data(),
                                         (int)xi.jobs[k].size(), bs);
    });
}

}  // namespace

lgf_status poisson_ragged_scratch(lgf_ctx *ctx, const RagPart *parts, int n)
{
    std::vector<int64_t> ao, bo;
    int64_t at = 0, bt = 0;
    ragged_offsets(parts, n, &ao, &bo, &at, &bt);
    const size_t csz = ctx->prec == LGF_F64 ? 16 : 8;
    lgf_status st = ensure_scratch(ctx, &ctx->scr[0].A, &ctx->scr[0].a, (size_t)at * csz);
    if (st != LGF_OK) return st;
    return ensure_scratch(ctx, &ctx->scr[0].B, &ctx->scr[0].b, (size_t)bt * csz);
}

lgf_status poisson_run_ragged(lgf_ctx *ctx, const RagPart *parts, int n, cudaStream_t s, int nbr)
{
    if (n == 0) return LGF_OK;
    if (ctx->prec == LGF_F64) return run_ragged<double>(ctx, parts, n, s, nbr);
    return run_ragged<float>(ctx, parts, n, s, nbr);
}

lgf_status poisson_time_choice(lgf_ctx *ctx, PoissonPlan *pl, const PoissonChoice &ch, int nf, double kalpha,
                               cudaStream_t s, float *ms)
{
    PoissonGeom g = pl->g;
    int64_t A = 0, B = 0;
    if (!poisson_geometry(*pl, ch, &g, &A, &B)) return LGF_EUNSUPPORTED;
    Spectrum *sp = nullptr;
    lgf_status st = poisson_spectrum(ctx, g, kalpha, &sp, s);
    if (st != LGF_OK) return st;
    const bool dbl = ctx->prec == LGF_F64;
    const size_t csz = dbl ? 16 : 8, esz = dbl ? 8 : 4;
    if ((st = ensure_scratch(ctx, &ctx->cur->A, &ctx->cur->a, (size_t)A * nf * csz)) != LGF_OK) return st;
    if ((st = ensure_scratch(ctx, &ctx->cur->B, &ctx->cur->b, (size_t)B * nf * csz)) != LGF_OK) return st;
    // timing inputs and outputs (zeros: the passes' work does not depend on
    // the values); not captured by any graph, so growth drops none
    const size_t fb = (size_t)g.fstride * nf * esz, ub = (size_t)g.ustride * nf * esz;
    const bool fresh = fb > ctx->tune_fb;
    if ((st = ensure_scratch(nullptr, &ctx->tune_f, &ctx->tune_fb, fb)) != LGF_OK) return st;
    if ((st = ensure_scratch(nullptr, &ctx->tune_u, &ctx->tune_ub, ub)) != LGF_OK) return st;
    if (fresh) LGF_CUDA(ctx, cudaMemsetAsync(ctx->tune_f, 0, ctx->tune_fb, s));
    for (int d = 0; d < 3; ++d) {
        twiddles(ctx, g.M[d], dbl, &st);
        if (st != LGF_OK) return st;
    }
    g.Astride = A;
    g.Bstride = B;
    g.scale = 1.0;
    auto run = [&]() -> lgf_status {
        if (dbl)
            return run_passes<double>(ctx, g, (const double *)ctx->tune_f, (double *)ctx->tune_u,
                                      (Cx<double> *)ctx->cur->A, (Cx<double> *)ctx->cur->B, (const double *)sp->dev,
                                      nf, 0, false, s);
        return run_passes<float>(ctx, g, (const float *)ctx->tune_f, (float *)ctx->tune_u, (Cx<float> *)ctx->cur->A,
                                 (Cx<float> *)ctx->cur->B, (const float *)sp->dev, nf, 0, false, s);
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    LGF_CUDA(ctx, cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(ctx, LGF_ECUDA, "tune: event creation failed");
    }
    std::vector<float> t;
    for (int r = 0; r < 2 + ctx->tune_reps && st == LGF_OK; ++r) {
        cudaEventRecord(e0, s);
        st = run();
        cudaEventRecord(e1, s);
        cudaError_t e = cudaEventSynchronize(e1);
        float v = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&v, e0, e1);
        if (e != cudaSuccess && st == LGF_OK) st = cuda_fail(ctx, e, "tune: timing");
        if (r >= 2) t.push_back(v);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != LGF_OK) return st;
    std::sort(t.begin(), t.end());
    *ms = t[t.size() / 2];
    return LGF_OK;
}

}  // namespace lgf
