// FP64 residual of the discrete Poisson problem (Sec. 2.2, Eq. dpoisson):
// r(n) = (sum_{+-e_i} u(n +- e_i) - 6 u(n)) / dx^2 - f(n) at every point of a
// block set whose six lattice neighbours are in the set.
#include <algorithm>
#include <cstring>
#include <unordered_map>
#include <vector>

#include "lgf_internal.cuh"

namespace lgf {

namespace {

template <typename T>
__global__ void k_residual(const T *__restrict__ u, const T *__restrict__ f, const int *__restrict__ nb6, int nblk,
                           int lb, double inv_dx2, double *__restrict__ r, unsigned long long *red)
{
    const int b = 1 << lb, bm = b - 1;
    const int64_t b3 = (int64_t)1 << (3 * lb);
    const int64_t n = nblk * b3;
    double rmax = 0.0, fm = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int blk = (int)(i >> (3 * lb));
        const int loc = (int)(i & (b3 - 1));
        const int x = loc & bm, y = (loc >> lb) & bm, z = loc >> (2 * lb);
        const int c[3] = {x, y, z};
        double sum = 0.0;
        bool ok = true;
        for (int ax = 0; ax < 3 && ok; ++ax)
            for (int sgn = -1; sgn <= 1 && ok; sgn += 2) {
                int q[3] = {c[0], c[1], c[2]};
                q[ax] += sgn;
                int bb = blk;
                if (q[ax] < 0 || q[ax] > bm) {
                    bb = nb6[blk * 6 + 2 * ax + (sgn > 0 ? 1 : 0)];
                    if (bb < 0) {
                        ok = false;
                        break;
                    }
                    q[ax] &= bm;
                }
                sum += (double)u[((int64_t)bb << (3 * lb)) + (((q[2] << lb) + q[1]) << lb) + q[0]];
            }
        double rv = 0.0;
        if (ok) {
            rv = (sum - 6.0 * (double)u[i]) * inv_dx2 - (double)f[i];
            rmax = fmax(rmax, fabs(rv));
            fm = fmax(fm, fabs((double)f[i]));
        }
        r[i] = rv;
    }
    atomicMax(&red[0], (unsigned long long)__double_as_longlong(rmax));
    atomicMax(&red[1], (unsigned long long)__double_as_longlong(fm));
}

}  // namespace

lgf_status residual_run(lgf_ctx *ctx, const lgf_blockset *set, const void *u, const void *f, double dx, double *r,
                        double *max_abs, double *max_f, cudaStream_t s)
{
    const int n = set->nblocks, b = set->b;
    int lb = 0;
    while ((1 << lb) < b) ++lb;
    std::unordered_map<int64_t, int> idx;
    auto key = [](int x, int y, int z) {
        return (((int64_t)(x + (1 << 20))) << 42) | (((int64_t)(y + (1 << 20))) << 21) | (int64_t)(z + (1 << 20));
    };
    for (int i = 0; i < n; ++i)
        if (!idx.emplace(key(set->coords[3 * i], set->coords[3 * i + 1], set->coords[3 * i + 2]), i).second)
            return fail(ctx, LGF_EINVAL, "residual: duplicate block");
    std::vector<int> nb6((size_t)n * 6, -1);
    for (int i = 0; i < n; ++i)
        for (int ax = 0; ax < 3; ++ax)
            for (int sg = 0; sg < 2; ++sg) {
                int c[3] = {set->coords[3 * i], set->coords[3 * i + 1], set->coords[3 * i + 2]};
                c[ax] += sg ? 1 : -1;
                auto it = idx.find(key(c[0], c[1], c[2]));
                if (it != idx.end()) nb6[i * 6 + 2 * ax + sg] = it->second;
            }
    int *dnb = nullptr;
    if (cudaMalloc(&dnb, nb6.size() * sizeof(int) + 4) != cudaSuccess)
        return fail(ctx, LGF_ENOMEM, "residual: allocation failed");
    cudaError_t e = cudaMemcpyAsync(dnb, nb6.data(), nb6.size() * sizeof(int), cudaMemcpyHostToDevice, s);
    unsigned long long *red = (unsigned long long *)ctx->red_dev;
    if (e == cudaSuccess) e = cudaMemsetAsync(red, 0, 2 * sizeof(unsigned long long), s);
    if (e == cudaSuccess && n > 0) {
        if (ctx->prec == LGF_F64)
            k_residual<double><<<152 * 4, 256, 0, s>>>((const double *)u, (const double *)f, dnb, n, lb, 1.0 / (dx * dx),
                                                       r, red);
        else
            k_residual<float><<<152 * 4, 256, 0, s>>>((const float *)u, (const float *)f, dnb, n, lb, 1.0 / (dx * dx),
                                                      r, red);
        e = cudaGetLastError();
    }
    unsigned long long h[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, red, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(dnb);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "residual");
    double v[2];
    memcpy(v, h, sizeof(v));
    if (max_abs) *max_abs = v[0];
    if (max_f) *max_f = v[1];
    return LGF_OK;
}

}  // namespace lgf
