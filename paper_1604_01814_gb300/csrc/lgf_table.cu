// G_L table builder and look-up (FP64 on the GPU).
//
// G_L(n) = -int_0^inf prod_i e^{-2t} I_{|n_i|}(2t) dt      (App. A, Eq. lgf_lap)
//
// All table entries share one quadrature grid on [0, T]: 32-point
// Gauss-Legendre panels on [0, 1/4] and then on panels growing by 3/2.  For each
// node one thread evaluates e^{-2t} I_k(2t) for every order k the table needs
// (Miller's algorithm in ratio form), and one thread per table entry then sums
// the three-way products.  Past T the three Bessel factors follow their
// large-argument series; with t = T / s^2 the tail becomes a smooth integral
// over s in (0, 1] that the same Gauss-Legendre rule evaluates.
//
// G_K(alpha) (App. A, Eq. lgf_iflap) is built on top of the G_L table as
// G_L + R(alpha), R(alpha)(n) = int_0^alpha prod_i e^{-2t} I_{|n_i|}(2t) dt,
// with the same Gauss-Legendre rule on panels of width <= 1/2 of [0, alpha]
// (the integrand is smooth and bounded by 1 there).  Beyond the table radius
// G_K takes the G_L expansion; the builder requires R(alpha) on the outer
// shell to be negligible (the footnote of Sec. 2.2: R decays faster than any
// exponential), else the table must grow.
//
// Beyond the table radius G_L is taken from its far-field expansion
// -1/(4 pi r) + T3 + T5 + T7 (terms of order r^-3, r^-5, r^-7; Sec. 2.2 and
// the App. A footnote give the leading term), whose terms follow from
// expanding 1/sigma(xi) about xi = 0.  The builder checks the expansion
// against the quadrature on the outer shell of the table.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "lgf_internal.cuh"

namespace lgf {

namespace {

constexpr int kGL = 32;  // Gauss-Legendre points per panel

// e^{-z} I_k(z) for k = 0..nmax: ratios r_k = I_k / I_{k-1} from the backward
// recurrence r_k = 1 / (2k/z + r_{k+1}), normalised with
// e^{-z} (I_0 + 2 sum_k I_k) = 1.  No overflow: every ratio is <= 1.
__device__ void ive_ratio(double z, int nmax, double *out)
{
    if (z <= 0.0) {
        for (int k = 0; k <= nmax; ++k) out[k] = (k == 0) ? 1.0 : 0.0;
        return;
    }
    const int N = nmax + 40 + (int)(10.0 * sqrt(z));
    double r = 0.0, acc = 0.0;
    const double inv = 2.0 / z;
    for (int k = N; k >= 1; --k) {
        r = 1.0 / (k * inv + r);
        acc = r * (1.0 + acc);
        if (k <= nmax) out[k] = r;
    }
    out[0] = 1.0 / (1.0 + 2.0 * acc);
    for (int k = 1; k <= nmax; ++k) out[k] *= out[k - 1];
}

// Gauss-Legendre nodes/weights on [-1, 1] by Newton's method on P_n.
__global__ void k_gauss_legendre(int n, double *x, double *w)
{
    const int i = threadIdx.x;
    if (i >= n) return;
    const double pi = 3.14159265358979323846;
    double xi = cos(pi * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = xi;
        for (int k = 2; k <= n; ++k) {
            const double p2 = ((2.0 * k - 1.0) * xi * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (xi * p1 - p0) / (xi * xi - 1.0);
        const double dx = p1 / dp;
        xi -= dx;
        if (fabs(dx) < 1e-17) break;
    }
    {
        double p0 = 1.0, p1 = xi;
        for (int k = 2; k <= n; ++k) {
            const double p2 = ((2.0 * k - 1.0) * xi * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (xi * p1 - p0) / (xi * xi - 1.0);
    }
    x[i] = xi;
    w[i] = 2.0 / ((1.0 - xi * xi) * dp * dp);
}

// Quadrature nodes on [0, T]: panel p spans [edge[p], edge[p+1]].
__global__ void k_nodes(const double *edge, int npanel, const double *glx, const double *glw, double *t, double *wt)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npanel * kGL) return;
    const int p = i / kGL, q = i % kGL;
    const double a = edge[p], b = edge[p + 1];
    t[i] = 0.5 * (a + b) + 0.5 * (b - a) * glx[q];
    wt[i] = 0.5 * (b - a) * glw[q];
}

// Bessel factors at every node: B[i][k] = e^{-2 t_i} I_k(2 t_i), k <= R.
__global__ void k_bessel_nodes(const double *t, int nnodes, int R, double *B)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nnodes) return;
    ive_ratio(2.0 * t[i], R, B + (size_t)i * (R + 1));
}

// Large-argument series of e^{-z} I_n(z) * sqrt(2 pi z): sum_k c_k z^{-k},
// c_k = c_{k-1} * -(4n^2 - (2k-1)^2) / (8k).
__device__ double ive_series_scaled(int n, double z)
{
    const double mu = 4.0 * n * (double)n;
    double c = 1.0, s = 1.0, zk = 1.0;
    for (int k = 1; k <= 14; ++k) {
        const double f = mu - (2.0 * k - 1.0) * (2.0 * k - 1.0);
        c *= -f / (8.0 * k);
        zk /= z;
        s += c * zk;
    }
    return s;
}

}  // namespace

// Far-field expansion of G_L with the normalised invariants e2' = e2 / r^4 and
// e3' = e3 / r^6 of the squared offsets (e2 = XY + YZ + ZX, e3 = XYZ).
__device__ double lgf_far(double a, double b, double c)
{
    const double X = a * a, Y = b * b, Z = c * c;
    const double r2 = X + Y + Z, r = sqrt(r2);
    const double e2 = (X * Y + Y * Z + Z * X) / (r2 * r2);
    const double e3 = X * Y * Z / (r2 * r2 * r2);
    const double pi = 3.14159265358979323846;
    const double ir = 1.0 / r, ir2 = ir * ir;
    const double t1 = -0.25 / pi;
    const double t3 = (-1.0 + 5.0 * e2) / (16.0 * pi);
    const double t5 = (-23.0 + 336.0 * e2 + 1134.0 * e3 - 1155.0 * e2 * e2) / (128.0 * pi);
    const double t7 = (-647.0 + 20301.0 * e2 + 208494.0 * e3 - 178035.0 * e2 * e2 - 810810.0 * e2 * e3
                       + 425425.0 * e2 * e2 * e2) / (512.0 * pi);
    return ir * (t1 + ir2 * (t3 + ir2 * (t5 + ir2 * t7)));
}

__device__ __forceinline__ int64_t tab_index(int a, int b, int c)
{
    return (int64_t)a * (a + 1) * (a + 2) / 6 + (int64_t)b * (b + 1) / 2 + c;
}

__device__ double lgf_value(const double *table, int R, int n1, int n2, int n3)
{
    int a = abs(n1), b = abs(n2), c = abs(n3), t;
    if (a < b) { t = a; a = b; b = t; }
    if (b < c) { t = b; b = c; c = t; }
    if (a < b) { t = a; a = b; b = t; }
    if (a <= R) return table[tab_index(a, b, c)];
    return lgf_far(a, b, c);
}

namespace {

__global__ void k_table(const int *abc, int64_t n, const double *B, const double *wt, int nnodes, int R, double T,
                        const double *sx, const double *sw, int shell_lo, double *table,
                        unsigned long long *mismatch)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int a = abc[3 * i], b = abc[3 * i + 1], c = abc[3 * i + 2];
    const int ld = R + 1;
    double s = 0.0;
    for (int j = 0; j < nnodes; ++j) {
        const double *bj = B + (size_t)j * ld;
        s += wt[j] * (bj[a] * bj[b] * bj[c]);
    }
    // tail: int_0^1 (4 pi T)^{-3/2} 2T prod_i S_{n_i}(2T/s^2) ds
    double tail = 0.0;
    for (int q = 0; q < kGL; ++q) {
        const double sq = 0.5 + 0.5 * sx[q];
        const double z = 2.0 * T / (sq * sq);
        tail += 0.5 * sw[q] * ive_series_scaled(a, z) * ive_series_scaled(b, z) * ive_series_scaled(c, z);
    }
    const double pi = 3.14159265358979323846;
    tail *= 2.0 * T * pow(4.0 * pi * T, -1.5);
    const double g = -(s + tail);
    table[i] = g;
    if (a >= shell_lo && a > 0) {
        const double rel = fabs(lgf_far(a, b, c) - g) / fabs(g);
        atomicMax(mismatch, (unsigned long long)__double_as_longlong(rel));
    }
}

// G_K(alpha) = G_L + R(alpha) per sorted offset; the largest |R| on the
// outer shell a = R goes to *shell.
__global__ void k_rtable(const int *abc, int64_t n, const double *B, const double *wt, int nnodes, int R,
                         const double *gl, double *gk, unsigned long long *shell)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int a = abc[3 * i], b = abc[3 * i + 1], c = abc[3 * i + 2];
    const int ld = R + 1;
    double r = 0.0;
    for (int j = 0; j < nnodes; ++j) {
        const double *bj = B + (size_t)j * ld;
        r += wt[j] * (bj[a] * bj[b] * bj[c]);
    }
    gk[i] = gl[i] + r;
    if (a == R) atomicMax(shell, (unsigned long long)__double_as_longlong(fabs(r)));
}

__global__ void k_lookup(const double *table, int R, const int32_t *off, int64_t n, double *out)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = lgf_value(table, R, off[3 * i], off[3 * i + 1], off[3 * i + 2]);
}

// Even circular embedding of G_L on an Mx x My x Mz box:
// box[z][y][x] = G_L(min(x, Mx-x), min(y, My-y), min(z, Mz-z)).
// Circular embedding of G_L on an Mx x My x Mz box: even along z
// (h[m] = G_L(min(m, M - m))); along x and y the window h[m] = G_L(m + c) for
// m < P and G_L(m - M + c) above (c = 0, P = M/2 is the even one).
__global__ void k_window(const double *table, int R, int Mx, int My, int Mz, int xc, int xP, int yc, int yP,
                         double *box)
{
    const int64_t n = (int64_t)Mx * My * Mz;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % Mx);
        const int y = (int)((i / Mx) % My);
        const int z = (int)(i / ((int64_t)Mx * My));
        const int dxo = x < xP ? x + xc : x - Mx + xc;
        const int dyo = y < yP ? y + yc : y - My + yc;
        box[i] = lgf_value(table, R, abs(dxo), abs(dyo), min(z, Mz - z));
    }
}

__global__ void k_bessel_one(double z, int nmax, double *out) { ive_ratio(z, nmax, out); }

}  // namespace

namespace {
// Sorted offsets a >= b >= c >= 0, a <= R, in table order.
std::vector<int> sorted_offsets(int R)
{
    const int64_t n = (int64_t)(R + 1) * (R + 2) * (R + 3) / 6;
    std::vector<int> abc(3 * n);
    for (int a = 0; a <= R; ++a)
        for (int b = 0; b <= a; ++b)
            for (int c = 0; c <= b; ++c) {
                const int64_t i = (int64_t)a * (a + 1) * (a + 2) / 6 + (int64_t)b * (b + 1) / 2 + c;
                abc[3 * i] = a;
                abc[3 * i + 1] = b;
                abc[3 * i + 2] = c;
            }
    return abc;
}
}  // namespace

lgf_status table_build(lgf_ctx *ctx, int R, cudaStream_t s)
{
    const double T = 24.0 * R * (double)R + 200.0;
    std::vector<double> edge{0.0, 0.25};
    while (edge.back() < T) edge.push_back(std::min(T, edge.back() * 1.5));
    const int npanel = (int)edge.size() - 1;
    const int nnodes = npanel * kGL;
    const int64_t n = (int64_t)(R + 1) * (R + 2) * (R + 3) / 6;
    const std::vector<int> abc = sorted_offsets(R);

    double *glx = nullptr, *glw = nullptr, *dedge = nullptr, *t = nullptr, *wt = nullptr, *B = nullptr;
    double *table = nullptr;
    int *dabc = nullptr;
    unsigned long long *mism = nullptr;
    auto cleanup = [&]() {
        cudaFree(glx); cudaFree(glw); cudaFree(dedge); cudaFree(t); cudaFree(wt); cudaFree(B);
        cudaFree(dabc); cudaFree(mism);
    };
    cudaError_t e = cudaSuccess;
    if ((e = cudaMalloc(&glx, kGL * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&glw, kGL * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&dedge, edge.size() * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&t, nnodes * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&wt, nnodes * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&B, (size_t)nnodes * (R + 1) * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&dabc, abc.size() * sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc(&mism, sizeof(unsigned long long))) != cudaSuccess ||
        (e = cudaMalloc(&table, n * sizeof(double))) != cudaSuccess) {
        cleanup();
        cudaFree(table);
        return fail(ctx, LGF_ENOMEM, std::string("table_build: cudaMalloc: ") + cudaGetErrorString(e));
    }
    cudaMemcpyAsync(dedge, edge.data(), edge.size() * sizeof(double), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(dabc, abc.data(), abc.size() * sizeof(int), cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(mism, 0, sizeof(unsigned long long), s);
    k_gauss_legendre<<<1, kGL, 0, s>>>(kGL, glx, glw);
    k_nodes<<<(nnodes + 127) / 128, 128, 0, s>>>(dedge, npanel, glx, glw, t, wt);
    k_bessel_nodes<<<(nnodes + 63) / 64, 64, 0, s>>>(t, nnodes, R, B);
    const int shell_lo = R >= 8 ? R - 3 : R + 1;
    k_table<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(dabc, n, B, wt, nnodes, R, T, glx, glw, shell_lo, table,
                                                         mism);
    unsigned long long mh = 0;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&mh, mism, sizeof(mh), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cleanup();
    if (e != cudaSuccess) {
        cudaFree(table);
        return cuda_fail(ctx, e, "table_build");
    }
    double mm;
    memcpy(&mm, &mh, sizeof(mm));
    if (ctx->table_dev) cudaFree(ctx->table_dev);
    ctx->table_dev = table;
    ctx->table_radius = R;
    ctx->shell_mismatch = mm;
    return LGF_OK;
}

lgf_status gk_table(lgf_ctx *ctx, double alpha, const double **out, cudaStream_t s)
{
    if (ctx->table_dev == nullptr) return fail(ctx, LGF_ENOTABLE, "lgf_table_build has not been called");
    if (alpha == 0.0) {
        *out = ctx->table_dev;
        return LGF_OK;
    }
    if (!(alpha > 0.0) || !(alpha <= 64.0))
        return fail(ctx, LGF_EUNSUPPORTED, "G_K: alpha must lie in [0, 64]");
    auto it = ctx->gk_tables.find(alpha);
    if (it != ctx->gk_tables.end()) {
        *out = it->second;
        return LGF_OK;
    }
    const int R = ctx->table_radius;
    const int npanel = std::max(1, (int)std::ceil(alpha / 0.5));
    std::vector<double> edge(npanel + 1);
    for (int p = 0; p <= npanel; ++p) edge[p] = alpha * p / npanel;
    const int nnodes = npanel * kGL;
    const int64_t n = (int64_t)(R + 1) * (R + 2) * (R + 3) / 6;
    const std::vector<int> abc = sorted_offsets(R);
    double *glx = nullptr, *glw = nullptr, *dedge = nullptr, *t = nullptr, *wt = nullptr, *B = nullptr;
    double *table = nullptr;
    int *dabc = nullptr;
    unsigned long long *shell = nullptr;
    auto cleanup = [&]() {
        cudaFree(glx); cudaFree(glw); cudaFree(dedge); cudaFree(t); cudaFree(wt); cudaFree(B);
        cudaFree(dabc); cudaFree(shell);
    };
    cudaError_t e = cudaSuccess;
    if ((e = cudaMalloc(&glx, kGL * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&glw, kGL * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&dedge, edge.size() * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&t, nnodes * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&wt, nnodes * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&B, (size_t)nnodes * (R + 1) * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&dabc, abc.size() * sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc(&shell, sizeof(unsigned long long))) != cudaSuccess ||
        (e = cudaMalloc(&table, n * sizeof(double))) != cudaSuccess) {
        cleanup();
        cudaFree(table);
        return fail(ctx, LGF_ENOMEM, std::string("G_K table: cudaMalloc: ") + cudaGetErrorString(e));
    }
    cudaMemcpyAsync(dedge, edge.data(), edge.size() * sizeof(double), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(dabc, abc.data(), abc.size() * sizeof(int), cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(shell, 0, sizeof(unsigned long long), s);
    k_gauss_legendre<<<1, kGL, 0, s>>>(kGL, glx, glw);
    k_nodes<<<(nnodes + 127) / 128, 128, 0, s>>>(dedge, npanel, glx, glw, t, wt);
    k_bessel_nodes<<<(nnodes + 63) / 64, 64, 0, s>>>(t, nnodes, R, B);
    k_rtable<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(dabc, n, B, wt, nnodes, R, ctx->table_dev, table, shell);
    unsigned long long sh = 0;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&sh, shell, sizeof(sh), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cleanup();
    if (e != cudaSuccess) {
        cudaFree(table);
        return cuda_fail(ctx, e, "G_K table");
    }
    double shell_r;
    memcpy(&shell_r, &sh, sizeof(shell_r));
    // |G_L(0)| = 0.2527...: R(alpha) past the table must be negligible
    if (!(shell_r <= 1e-15 * 0.25)) {
        cudaFree(table);
        char msg[160];
        snprintf(msg, sizeof msg, "G_K: R(alpha=%g) is %.3g on the table's outer shell; build a larger table", alpha,
                 shell_r);
        return fail(ctx, LGF_EUNSUPPORTED, msg);
    }
    ctx->gk_tables[alpha] = table;
    *out = table;
    return LGF_OK;
}

// File form of the G_L table: magic "LGFTAB01", int32 radius, int64 count,
// double shell mismatch, the count FP64 values, then their 64-bit FNV-1a
// hash (little-endian host; the file is rejected unless all of it checks).
lgf_status table_save(lgf_ctx *ctx, const char *path)
{
    const int64_t n = (int64_t)(ctx->table_radius + 1) * (ctx->table_radius + 2) * (ctx->table_radius + 3) / 6;
    std::vector<double> h((size_t)n);
    LGF_CUDA(ctx, cudaMemcpy(h.data(), ctx->table_dev, n * sizeof(double), cudaMemcpyDeviceToHost));
    unsigned long long hash = 1469598103934665603ull;
    const unsigned char *bytes = (const unsigned char *)h.data();
    for (size_t i = 0; i < h.size() * sizeof(double); ++i) hash = (hash ^ bytes[i]) * 1099511628211ull;
    FILE *f = std::fopen(path, "wb");
    if (!f) return fail(ctx, LGF_EINVAL, std::string("table_save: cannot open ") + path);
    const char magic[8] = {'L', 'G', 'F', 'T', 'A', 'B', '0', '1'};
    const int32_t R = ctx->table_radius;
    bool ok = std::fwrite(magic, 1, 8, f) == 8 && std::fwrite(&R, 4, 1, f) == 1 && std::fwrite(&n, 8, 1, f) == 1 &&
              std::fwrite(&ctx->shell_mismatch, 8, 1, f) == 1 &&
              std::fwrite(h.data(), sizeof(double), h.size(), f) == h.size() && std::fwrite(&hash, 8, 1, f) == 1;
    ok = (std::fclose(f) == 0) && ok;
    return ok ? LGF_OK : fail(ctx, LGF_EINVAL, std::string("table_save: write failed: ") + path);
}

lgf_status table_load(lgf_ctx *ctx, const char *path)
{
    FILE *f = std::fopen(path, "rb");
    if (!f) return fail(ctx, LGF_EINVAL, std::string("table_load: cannot open ") + path);
    char magic[8];
    int32_t R = 0;
    int64_t n = 0;
    double mm = 0.0;
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "LGFTAB01", 8) == 0 &&
              std::fread(&R, 4, 1, f) == 1 && std::fread(&n, 8, 1, f) == 1 && std::fread(&mm, 8, 1, f) == 1 &&
              R >= 8 && R <= 96 && n == (int64_t)(R + 1) * (R + 2) * (R + 3) / 6;
    std::vector<double> h(ok ? (size_t)n : 0);
    unsigned long long hash = 0, want = 1469598103934665603ull;
    if (ok) ok = std::fread(h.data(), sizeof(double), h.size(), f) == h.size() && std::fread(&hash, 8, 1, f) == 1;
    std::fclose(f);
    if (ok) {
        const unsigned char *bytes = (const unsigned char *)h.data();
        for (size_t i = 0; i < h.size() * sizeof(double); ++i) want = (want ^ bytes[i]) * 1099511628211ull;
        ok = hash == want;
    }
    if (!ok) return fail(ctx, LGF_EINVAL, std::string("table_load: not a valid G_L table file: ") + path);
    double *dev = nullptr;
    if (cudaMalloc(&dev, n * sizeof(double)) != cudaSuccess)
        return fail(ctx, LGF_ENOMEM, "table_load: allocation failed");
    cudaError_t e = cudaMemcpy(dev, h.data(), n * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(dev);
        return cuda_fail(ctx, e, "table_load: copy");
    }
    cudaFree(ctx->table_dev);
    ctx->table_dev = dev;
    ctx->table_radius = R;
    ctx->shell_mismatch = mm;
    return LGF_OK;
}

lgf_status table_lookup(lgf_ctx *ctx, const double *table, const int32_t *off, int64_t n, double *out,
                        cudaStream_t s)
{
    if (n == 0) return LGF_OK;
    k_lookup<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(table, ctx->table_radius, off, n, out);
    LGF_CHECK_LAUNCH(ctx, "lookup kernel");
    return LGF_OK;
}

namespace {
// The exact sum u(t) = dx^2 sum_m G_L(t - m) f(m) at one sampled target per
// CTA, in FP64 (G_L from the table and its expansion, as the apply uses it):
// the reference values of the a-posteriori error estimate.
template <typename T>
__global__ void __launch_bounds__(256) k_direct_sample(const double *table, int R, const int *src, int nsrc, int lb,
                                                       const T *f, const int *pts, double dx2, double *out)
{
    const int *tp = pts + 3 * blockIdx.x;
    const int tx = tp[0], ty = tp[1], tz = tp[2];
    const int b = 1 << lb, b3 = b * b * b;
    const int64_t n = (int64_t)nsrc * b3;
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const T v = f[i];
        if (v == T(0)) continue;
        const int blk = (int)(i >> (3 * lb)), loc = (int)(i & (b3 - 1));
        const int mx = src[3 * blk] * b + (loc & (b - 1));
        const int my = src[3 * blk + 1] * b + ((loc >> lb) & (b - 1));
        const int mz = src[3 * blk + 2] * b + (loc >> (2 * lb));
        acc += lgf_value(table, R, tx - mx, ty - my, tz - mz) * (double)v;
    }
    __shared__ double red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = dx2 * red[0];
}
}  // namespace

namespace {
template <typename T>
__global__ void k_gather(const T *field, const int64_t *idx, int n, double *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (double)field[idx[i]];
}
}  // namespace

lgf_status gather_values(lgf_ctx *ctx, const void *field, const int64_t *idx_host, int n, double *out_host,
                         cudaStream_t s)
{
    if (n <= 0) return LGF_OK;
    int64_t *didx = nullptr;
    double *dout = nullptr;
    if (cudaMalloc(&didx, sizeof(int64_t) * n) != cudaSuccess || cudaMalloc(&dout, sizeof(double) * n) != cudaSuccess) {
        cudaFree(didx);
        return fail(ctx, LGF_ENOMEM, "error estimate: allocation failed");
    }
    cudaError_t e = cudaMemcpyAsync(didx, idx_host, sizeof(int64_t) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        if (ctx->prec == LGF_F64)
            k_gather<double><<<(n + 255) / 256, 256, 0, s>>>((const double *)field, didx, n, dout);
        else
            k_gather<float><<<(n + 255) / 256, 256, 0, s>>>((const float *)field, didx, n, dout);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(out_host, dout, sizeof(double) * n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(didx);
    cudaFree(dout);
    return e == cudaSuccess ? LGF_OK : cuda_fail(ctx, e, "error estimate: gather");
}

lgf_status direct_samples(lgf_ctx *ctx, const lgf_blockset *src, const void *f_field, const int32_t *pts_host,
                          int npts, double dx, double *out_host, cudaStream_t s)
{
    if (npts <= 0) return LGF_OK;
    int lb = 0;
    while ((1 << lb) < src->b) ++lb;
    int *dsrc = nullptr, *dpts = nullptr;
    double *dout = nullptr;
    auto cleanup = [&]() {
        cudaFree(dsrc);
        cudaFree(dpts);
        cudaFree(dout);
    };
    if (cudaMalloc(&dsrc, 3 * sizeof(int) * (size_t)std::max(1, src->nblocks)) != cudaSuccess ||
        cudaMalloc(&dpts, 3 * sizeof(int) * (size_t)npts) != cudaSuccess ||
        cudaMalloc(&dout, sizeof(double) * (size_t)npts) != cudaSuccess) {
        cleanup();
        return fail(ctx, LGF_ENOMEM, "error estimate: allocation failed");
    }
    cudaError_t e = cudaMemcpyAsync(dsrc, src->coords, 3 * sizeof(int) * (size_t)src->nblocks,
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dpts, pts_host, 3 * sizeof(int) * (size_t)npts, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        if (ctx->prec == LGF_F64)
            k_direct_sample<double><<<npts, 256, 0, s>>>(ctx->table_dev, ctx->table_radius, dsrc, src->nblocks, lb,
                                                         (const double *)f_field, dpts, dx * dx, dout);
        else
            k_direct_sample<float><<<npts, 256, 0, s>>>(ctx->table_dev, ctx->table_radius, dsrc, src->nblocks, lb,
                                                        (const float *)f_field, dpts, dx * dx, dout);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(out_host, dout, sizeof(double) * (size_t)npts, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cleanup();
    return e == cudaSuccess ? LGF_OK : cuda_fail(ctx, e, "error estimate: direct samples");
}

lgf_status kernel_window(lgf_ctx *ctx, const double *table, const int M[3], int xc, int xP, int yc, int yP,
                         double *box, cudaStream_t s)
{
    k_window<<<152 * 8, 256, 0, s>>>(table, ctx->table_radius, M[0], M[1], M[2], xc, xP, yc, yP, box);
    LGF_CHECK_LAUNCH(ctx, "window kernel");
    return LGF_OK;
}

lgf_status bessel_weights(lgf_ctx *ctx, double z, int nmax, double *out_dev, cudaStream_t s)
{
    k_bessel_one<<<1, 1, 0, s>>>(z, nmax, out_dev);
    LGF_CHECK_LAUNCH(ctx, "bessel kernel");
    return LGF_OK;
}

}  // namespace lgf
