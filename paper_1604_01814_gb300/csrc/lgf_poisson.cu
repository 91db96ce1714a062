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

#include "lgf_internal.cuh"

namespace lgf {

FftShape make_fft_shape(int M)
{
    FftShape sh{};
    sh.M = M;
    int l = 0;
    while ((1 << l) < M) ++l;
    sh.logM = l;
    sh.nst = 0;
    int rem = l;
    while (rem > 0) {
        const int r = rem >= 4 ? 4 : rem;
        sh.lg[sh.nst++] = r;
        rem -= r;
    }
    return sh;
}

int next_fft_size(int n)
{
    int m = 32;
    while (m < n) m *= 2;
    return m;
}

PoissonPlan::~PoissonPlan()
{
    cudaFree(srcmap_dev);
    cudaFree(tgtmap_dev);
}

namespace {

constexpr int kThreads = 256;

// Elements (complex) a CTA keeps in shared memory for its lines.
constexpr int kElemsPerCta = 4096;

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

template <typename T>
__device__ __forceinline__ T fetch_src(const T *__restrict__ f, const PoissonGeom &g, int lb, int x, int y, int z,
                                       int dense_ld)
{
    if (dense_ld) return f[((int64_t)z * g.M[1] + y) * dense_ld + x];
    const int xr = x - g.s0[0], yr = y - g.s0[1], zr = z - g.s0[2];
    const int bi = g.srcmap[((zr >> lb) * g.nbs[1] + (yr >> lb)) * g.nbs[0] + (xr >> lb)];
    if (bi < 0) return T(0);
    const int m = g.b - 1;
    return f[((int64_t)bi << (3 * lb)) + ((((zr & m) << lb) + (yr & m)) << lb) + (xr & m)];
}

// X forward: rows (y, y+1) of plane z packed as one complex line of length Mx.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_xfwd(const T *__restrict__ f, Cx<T> *__restrict__ A, PoissonGeom g,
                                                    FftShape sh, const Cx<T> *__restrict__ twg, int lines,
                                                    int npairs, int lb, int dense_ld)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx<T> *tw = reinterpret_cast<Cx<T> *>(smem_raw);
    Cx<T> *s = tw + sh.M;
    const int M = sh.M;
    for (int i = threadIdx.x; i < M; i += blockDim.x) tw[i] = twg[i];
    const T *ff = f + blockIdx.y * g.fstride;
    Cx<T> *AA = A + blockIdx.y * g.Astride;
    const int pair0 = blockIdx.x * lines;
    const int nl = min(lines, npairs - pair0);
    const RowAddr ad{M + M / 16};
    const int hp = g.Ls[1] >> 1;
    for (int it = threadIdx.x; it < lines * M; it += blockDim.x) {
        const int l = it / M, x = it - l * M;
        Cx<T> v{T(0), T(0)};
        if (l < nl && x >= g.s0[0] && x < g.s0[0] + g.Ls[0]) {
            const int p = pair0 + l, zi = p / hp, yi = 2 * (p - zi * hp);
            const int y = g.s0[1] + yi, z = g.s0[2] + zi;
            v.x = fetch_src(ff, g, lb, x, y, z, dense_ld);
            v.y = fetch_src(ff, g, lb, x, y + 1, z, dense_ld);
        }
        s[ad(l, x)] = v;
    }
    __syncthreads();
    fft_forward<false>(s, ad, lines, sh, tw);
    const int K = g.Kx;
    for (int it = threadIdx.x; it < nl * K; it += blockDim.x) {
        const int l = it / K, k = it - l * K;
        const Cx<T> zk = s[ad(l, pos_of_freq(k, sh))];
        const Cx<T> zm = s[ad(l, pos_of_freq((M - k) & (M - 1), sh))];
        // rows y and y+1: (Z[k] + conj Z[M-k]) / 2 and (Z[k] - conj Z[M-k]) / 2i
        const Cx<T> f1{T(0.5) * (zk.x + zm.x), T(0.5) * (zk.y - zm.y)};
        const Cx<T> f2{T(0.5) * (zk.y + zm.y), T(-0.5) * (zk.x - zm.x)};
        const int p = pair0 + l, zi = p / hp, yi = 2 * (p - zi * hp);
        Cx<T> *row = AA + ((int64_t)zi * g.ldA_y + yi) * K;
        row[k] = f1;
        row[K + k] = f2;
    }
}

// Y forward over the source z-planes, W columns of kx per CTA.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_yfwd(const Cx<T> *__restrict__ A, Cx<T> *__restrict__ B, PoissonGeom g,
                                                    FftShape sh, const Cx<T> *__restrict__ twg, int W)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx<T> *tw = reinterpret_cast<Cx<T> *>(smem_raw);
    Cx<T> *s = tw + sh.M;
    const int M = sh.M;
    for (int i = threadIdx.x; i < M; i += blockDim.x) tw[i] = twg[i];
    const int zi = blockIdx.y;
    const int kx0 = blockIdx.x * W;
    const int K = g.Kx;
    const Cx<T> *AA = A + blockIdx.z * g.Astride + (int64_t)zi * g.ldA_y * K;
    Cx<T> *BB = B + blockIdx.z * g.Bstride + (int64_t)zi * M * K;
    const ColAddr ad{W};
    for (int it = threadIdx.x; it < W * M; it += blockDim.x) {
        const int m = it / W, w = it - m * W;
        const int kx = kx0 + w;
        Cx<T> v{T(0), T(0)};
        if (kx < K && m >= g.s0[1] && m < g.s0[1] + g.Ls[1]) v = AA[(int64_t)(m - g.s0[1]) * K + kx];
        s[ad(w, m)] = v;
    }
    __syncthreads();
    fft_forward<true>(s, ad, W, sh, tw);
    for (int it = threadIdx.x; it < W * M; it += blockDim.x) {
        const int ky = it / W, w = it - ky * W;
        const int kx = kx0 + w;
        if (kx < K) BB[(int64_t)ky * K + kx] = s[ad(w, pos_of_freq(ky, sh))];
    }
}

// Z: forward along z, times the real even kernel spectrum, inverse along z.
// mode 0: keep target planes (in place).  mode 1: spectrum build -- forward
// only, every plane stored in natural order.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_zconv(Cx<T> *__restrict__ B, PoissonGeom g, FftShape sh,
                                                     const Cx<T> *__restrict__ twg, const T *__restrict__ spec,
                                                     int W, int mode)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx<T> *tw = reinterpret_cast<Cx<T> *>(smem_raw);
    Cx<T> *s = tw + sh.M;
    const int M = sh.M;
    for (int i = threadIdx.x; i < M; i += blockDim.x) tw[i] = twg[i];
    const int ky = blockIdx.y;
    const int kx0 = blockIdx.x * W;
    const int K = g.Kx;
    const int My = g.M[1];
    const int64_t plane = (int64_t)My * K;
    Cx<T> *BB = B + blockIdx.z * g.Bstride + (int64_t)ky * K;
    const ColAddr ad{W};
    for (int it = threadIdx.x; it < W * M; it += blockDim.x) {
        const int m = it / W, w = it - m * W;
        const int kx = kx0 + w;
        Cx<T> v{T(0), T(0)};
        if (kx < K && m >= g.s0[2] && m < g.s0[2] + g.Ls[2]) v = BB[(int64_t)(m - g.s0[2]) * plane + kx];
        s[ad(w, m)] = v;
    }
    __syncthreads();
    fft_forward<true>(s, ad, W, sh, tw);
    if (mode == 1) {
        for (int it = threadIdx.x; it < W * M; it += blockDim.x) {
            const int kz = it / W, w = it - kz * W;
            const int kx = kx0 + w;
            if (kx < K) BB[(int64_t)kz * plane + kx] = s[ad(w, pos_of_freq(kz, sh))];
        }
        return;
    }
    const int kyr = min(ky, My - ky);
    const int Khy = My / 2 + 1, Khz = M / 2 + 1;
    for (int it = threadIdx.x; it < W * M; it += blockDim.x) {
        const int P = it / W, w = it - P * W;
        const int kx = kx0 + w;
        const int kz = freq_of_pos(P, sh);
        const int kzr = min(kz, M - kz);
        const T gk = (kx < K) ? spec[((int64_t)kzr * Khy + kyr) * K + kx] : T(0);
        Cx<T> v = s[ad(w, P)];
        v.x *= gk;
        v.y *= gk;
        s[ad(w, P)] = v;
    }
    (void)Khz;
    __syncthreads();
    fft_inverse<true>(s, ad, W, sh, tw);
    for (int it = threadIdx.x; it < W * g.Lt[2]; it += blockDim.x) {
        const int zi = it / W, w = it - zi * W;
        const int kx = kx0 + w;
        if (kx < K) BB[(int64_t)zi * plane + kx] = s[ad(w, g.t0[2] + zi)];
    }
}

// Y inverse over the target z-planes, keeping the target rows.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_yinv(const Cx<T> *__restrict__ B, Cx<T> *__restrict__ A, PoissonGeom g,
                                                    FftShape sh, const Cx<T> *__restrict__ twg, int W)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx<T> *tw = reinterpret_cast<Cx<T> *>(smem_raw);
    Cx<T> *s = tw + sh.M;
    const int M = sh.M;
    for (int i = threadIdx.x; i < M; i += blockDim.x) tw[i] = twg[i];
    const int zi = blockIdx.y;
    const int kx0 = blockIdx.x * W;
    const int K = g.Kx;
    const Cx<T> *BB = B + blockIdx.z * g.Bstride + (int64_t)zi * M * K;
    Cx<T> *AA = A + blockIdx.z * g.Astride + (int64_t)zi * g.ldA_y * K;
    const ColAddr ad{W};
    for (int it = threadIdx.x; it < W * M; it += blockDim.x) {
        const int ky = it / W, w = it - ky * W;
        const int kx = kx0 + w;
        Cx<T> v{T(0), T(0)};
        if (kx < K) v = BB[(int64_t)ky * K + kx];
        s[ad(w, pos_of_freq(ky, sh))] = v;
    }
    __syncthreads();
    fft_inverse<true>(s, ad, W, sh, tw);
    for (int it = threadIdx.x; it < W * g.Lt[1]; it += blockDim.x) {
        const int yi = it / W, w = it - yi * W;
        const int kx = kx0 + w;
        if (kx < K) AA[(int64_t)yi * K + kx] = s[ad(w, g.t0[1] + yi)];
    }
}

// X inverse (C2R): rows (y, y+1) of the target region from one complex line.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_xinv(const Cx<T> *__restrict__ A, T *__restrict__ u, PoissonGeom g,
                                                    FftShape sh, const Cx<T> *__restrict__ twg, int lines,
                                                    int npairs, int lb)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx<T> *tw = reinterpret_cast<Cx<T> *>(smem_raw);
    Cx<T> *s = tw + sh.M;
    const int M = sh.M;
    for (int i = threadIdx.x; i < M; i += blockDim.x) tw[i] = twg[i];
    const int K = g.Kx;
    const Cx<T> *AA = A + blockIdx.y * g.Astride;
    T *uu = u + blockIdx.y * g.ustride;
    const int pair0 = blockIdx.x * lines;
    const int nl = min(lines, npairs - pair0);
    const RowAddr ad{M + M / 16};
    const int hp = g.Lt[1] >> 1;
    for (int it = threadIdx.x; it < lines * M; it += blockDim.x) {
        const int l = it / M, k = it - l * M;
        Cx<T> v{T(0), T(0)};
        if (l < nl) {
            const int p = pair0 + l, zi = p / hp, yi = 2 * (p - zi * hp);
            const Cx<T> *row = AA + ((int64_t)zi * g.ldA_y + yi) * K;
            if (k <= M / 2) {
                Cx<T> g1 = row[k], g2 = row[K + k];
                if (k == 0 || k == M / 2) {
                    g1.y = T(0);
                    g2.y = T(0);
                }
                v = {g1.x - g2.y, g1.y + g2.x};
            } else {
                const Cx<T> g1 = row[M - k], g2 = row[K + M - k];
                v = {g1.x + g2.y, g2.x - g1.y};
            }
        }
        s[ad(l, pos_of_freq(k, sh))] = v;
    }
    __syncthreads();
    fft_inverse<false>(s, ad, lines, sh, tw);
    const T sc = T(g.scale);
    const int Lx = g.Lt[0];
    const int m = g.b - 1;
    for (int it = threadIdx.x; it < nl * 2 * Lx; it += blockDim.x) {
        const int l = it / (2 * Lx), r = it - l * 2 * Lx;
        const int half = r / Lx, xi = r - half * Lx;
        const int p = pair0 + l, zi = p / hp, yi = 2 * (p - zi * hp) + half;
        const int bi = g.tgtmap[((zi >> lb) * g.nbt[1] + (yi >> lb)) * g.nbt[0] + (xi >> lb)];
        if (bi < 0) continue;
        const Cx<T> v = s[ad(l, g.t0[0] + xi)];
        uu[((int64_t)bi << (3 * lb)) + ((((zi & m) << lb) + (yi & m)) << lb) + (xi & m)] = sc * (half ? v.y : v.x);
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

struct LaunchCfg {
    int lines_x;   // row lines per CTA (X passes)
    int W;         // columns per CTA (Y, Z passes)
};

LaunchCfg cfg_for(int M)
{
    LaunchCfg c;
    c.lines_x = std::max(1, kElemsPerCta / M);
    c.W = std::min(16, std::max(4, kElemsPerCta / M));
    return c;
}

template <typename T>
size_t smem_rows(int M, int lines) { return sizeof(Cx<T>) * ((size_t)M + (size_t)lines * (M + M / 16)); }
template <typename T>
size_t smem_cols(int M, int W) { return sizeof(Cx<T>) * ((size_t)M + (size_t)W * M); }

template <typename T>
lgf_status set_smem_limits(lgf_ctx *ctx)
{
    static bool done = false;
    if (done) return LGF_OK;
    const int big = 200 * 1024;
    LGF_CUDA(ctx, cudaFuncSetAttribute(k_xfwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    LGF_CUDA(ctx, cudaFuncSetAttribute(k_yfwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    LGF_CUDA(ctx, cudaFuncSetAttribute(k_zconv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    LGF_CUDA(ctx, cudaFuncSetAttribute(k_yinv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    LGF_CUDA(ctx, cudaFuncSetAttribute(k_xinv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    done = true;
    return LGF_OK;
}

// Launch the five passes for `nfields` fields of one problem.
template <typename T>
lgf_status run_passes(lgf_ctx *ctx, const PoissonGeom &g, const T *f, T *u, Cx<T> *A, Cx<T> *B, const T *spec,
                      int nfields, int dense_ld, bool spectrum_mode, cudaStream_t s)
{
    lgf_status st = set_smem_limits<T>(ctx);
    if (st != LGF_OK) return st;
    const bool dbl = sizeof(T) == 8;
    const FftShape shx = make_fft_shape(g.M[0]), shy = make_fft_shape(g.M[1]), shz = make_fft_shape(g.M[2]);
    const Cx<T> *twx = (const Cx<T> *)twiddles(ctx, g.M[0], dbl, &st);
    if (st != LGF_OK) return st;
    const Cx<T> *twy = (const Cx<T> *)twiddles(ctx, g.M[1], dbl, &st);
    if (st != LGF_OK) return st;
    const Cx<T> *twz = (const Cx<T> *)twiddles(ctx, g.M[2], dbl, &st);
    if (st != LGF_OK) return st;
    const int lb = log2i(g.b);
    const LaunchCfg cx = cfg_for(g.M[0]), cy = cfg_for(g.M[1]), cz = cfg_for(g.M[2]);
    const int K = g.Kx;

    // X forward
    {
        const int npairs = (g.Ls[1] / 2) * g.Ls[2];
        dim3 grid((npairs + cx.lines_x - 1) / cx.lines_x, nfields);
        const int ph = prof_begin(ctx, s, "poisson_x_forward");
        k_xfwd<T><<<grid, kThreads, smem_rows<T>(g.M[0], cx.lines_x), s>>>(f, A, g, shx, twx, cx.lines_x, npairs, lb,
                                                                          dense_ld);
        LGF_CHECK_LAUNCH(ctx, "poisson x-forward");
        prof_end(ctx, s, ph);
    }
    // Y forward
    {
        dim3 grid((K + cy.W - 1) / cy.W, g.Ls[2], nfields);
        const int ph = prof_begin(ctx, s, "poisson_y_forward");
        k_yfwd<T><<<grid, kThreads, smem_cols<T>(g.M[1], cy.W), s>>>(A, B, g, shy, twy, cy.W);
        LGF_CHECK_LAUNCH(ctx, "poisson y-forward");
        prof_end(ctx, s, ph);
    }
    // Z forward, multiply, inverse
    {
        dim3 grid((K + cz.W - 1) / cz.W, g.M[1], nfields);
        const int ph = prof_begin(ctx, s, spectrum_mode ? "spectrum_z_forward" : "poisson_z_convolve");
        k_zconv<T><<<grid, kThreads, smem_cols<T>(g.M[2], cz.W), s>>>(B, g, shz, twz, spec, cz.W,
                                                                      spectrum_mode ? 1 : 0);
        LGF_CHECK_LAUNCH(ctx, "poisson z-convolve");
        prof_end(ctx, s, ph);
    }
    if (spectrum_mode) return LGF_OK;
    // Y inverse
    {
        dim3 grid((K + cy.W - 1) / cy.W, g.Lt[2], nfields);
        const int ph = prof_begin(ctx, s, "poisson_y_inverse");
        k_yinv<T><<<grid, kThreads, smem_cols<T>(g.M[1], cy.W), s>>>(B, A, g, shy, twy, cy.W);
        LGF_CHECK_LAUNCH(ctx, "poisson y-inverse");
        prof_end(ctx, s, ph);
    }
    // X inverse
    {
        const int npairs = (g.Lt[1] / 2) * g.Lt[2];
        dim3 grid((npairs + cx.lines_x - 1) / cx.lines_x, nfields);
        const int ph = prof_begin(ctx, s, "poisson_x_inverse");
        k_xinv<T><<<grid, kThreads, smem_rows<T>(g.M[0], cx.lines_x), s>>>(A, u, g, shx, twx, cx.lines_x, npairs, lb);
        LGF_CHECK_LAUNCH(ctx, "poisson x-inverse");
        prof_end(ctx, s, ph);
    }
    return LGF_OK;
}

}  // namespace

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
    for (auto &p : ctx->pplans) {
        if (p->b == b && p->src == sv && p->tgt == tv) {
            *out = p.get();
            return LGF_OK;
        }
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
    PoissonGeom &g = plan->g;
    g.b = b;
    for (int d = 0; d < 3; ++d) {
        lo[d] = std::min(slo[d], tlo[d]);
        hi[d] = std::max(shi[d], thi[d]);
        const int64_t L = ((int64_t)hi[d] - lo[d] + 1) * b;
        if (L > kMaxFft / 2)
            return fail(ctx, LGF_EUNSUPPORTED, "poisson: union of source and target spans more than 2048 points");
        g.M[d] = next_fft_size((int)(2 * L - 1));
        g.s0[d] = (slo[d] - lo[d]) * b;
        g.Ls[d] = (shi[d] - slo[d] + 1) * b;
        g.t0[d] = (tlo[d] - lo[d]) * b;
        g.Lt[d] = (thi[d] - tlo[d] + 1) * b;
        g.nbs[d] = shi[d] - slo[d] + 1;
        g.nbt[d] = thi[d] - tlo[d] + 1;
    }
    g.Kx = g.M[0] / 2 + 1;
    g.ldA_y = std::max(g.Ls[1], g.Lt[1]);
    plan->A_elems = (int64_t)std::max(g.Ls[2], g.Lt[2]) * g.ldA_y * g.Kx;
    plan->B_elems = (int64_t)std::max(g.Ls[2], g.Lt[2]) * g.M[1] * g.Kx;
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
    g.fstride = (int64_t)src->nblocks * b * b * b;
    g.ustride = (int64_t)tgt->nblocks * b * b * b;
        ctx->pplans.push_back(std::move(plan));
    *out = ctx->pplans.back().get();
    return LGF_OK;
}

lgf_status poisson_spectrum(lgf_ctx *ctx, const int M[3], Spectrum **out, cudaStream_t s)
{
    const std::array<int, 3> key{M[0], M[1], M[2]};
    auto it = ctx->spectra.find(key);
    if (it != ctx->spectra.end()) {
        *out = &it->second;
        return LGF_OK;
    }
    if (ctx->table_dev == nullptr) return fail(ctx, LGF_ENOTABLE, "poisson: lgf_table_build has not been called");
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
    const size_t spec_elems = (size_t)g.Kx * (M[1] / 2 + 1) * (M[2] / 2 + 1);
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
    lgf_status st = kernel_window(ctx, M, box, s);
    if (st == LGF_OK)
        st = run_passes<double>(ctx, g, box, nullptr, A, B, nullptr, 1, M[0], true, s);
    if (st == LGF_OK) {
        if (esz == 8)
            k_extract<double><<<152 * 4, 256, 0, s>>>(B, (double *)spec, M[0], M[1], M[2]);
        else
            k_extract<float><<<152 * 4, 256, 0, s>>>(B, (float *)spec, M[0], M[1], M[2]);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(ctx, e, "poisson: kernel spectrum");
    }
    cleanup();
    if (st != LGF_OK) {
        cudaFree(spec);
        return st;
    }
    Spectrum sp;
    sp.M = key;
    sp.dev = spec;
    auto ins = ctx->spectra.emplace(key, sp);
    *out = &ins.first->second;
    return LGF_OK;
}

lgf_status poisson_prepare_scratch(lgf_ctx *ctx, const PoissonPlan *pl, int nfields)
{
    const size_t csz = ctx->prec == LGF_F64 ? 16 : 8;
    lgf_status st = ensure_scratch(ctx, &ctx->scrA, &ctx->scrA_bytes, (size_t)pl->A_elems * nfields * csz);
    if (st != LGF_OK) return st;
    return ensure_scratch(ctx, &ctx->scrB, &ctx->scrB_bytes, (size_t)pl->B_elems * nfields * csz);
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
        return run_passes<double>(ctx, g, (const double *)f, (double *)u, (Cx<double> *)ctx->scrA,
                                  (Cx<double> *)ctx->scrB, (const double *)sp->dev, nfields, 0, false, s);
    return run_passes<float>(ctx, g, (const float *)f, (float *)u, (Cx<float> *)ctx->scrA, (Cx<float> *)ctx->scrB,
                             (const float *)sp->dev, nfields, 0, false, s);
}

}  // namespace lgf
