// Kernels of the nested-projection stage (Sec. 3.1, Eq. nested_proj): the
// staggered divergence and gradient of Sec. 2.1 on block sets, the marker
// residual and the two dense products with the factors of the force Schur
// complement's inverse (Sec. 3.2).  The stage itself is composed in
// lgf_capi.cu from these and the Poisson, integrating-factor and IB passes.
//
// Cell n holds face k at (n + (1 - e_k)/2) dx, so
//   (Dbar u)(n) = sum_k [u_k(n + e_k) - u_k(n)] / dx     faces -> cells
//   (G q)_k(n)  = [q(n) - q(n - e_k)] / dx               cells -> faces
// and G^dagger = -Dbar.  Both read the block itself and, where the shift
// leaves it, the neighbour block of a CurlPlan (dir +1 for Dbar, -1 for G);
// values outside the input block set are zero.  One thread per output cell.
#include "lgf_async.cuh"
#include "lgf_internal.cuh"

namespace lgf {
namespace {

// out(n) = scale * sum_k [(a - c)_k(n + e_k) - (a - c)_k(n)]   (c may be null)
template <typename T, int LB>
__global__ void __launch_bounds__(256) k_div(const T *__restrict__ a, const T *__restrict__ c, T *__restrict__ out,
                                             const int *__restrict__ nbr, int64_t ncell, int64_t in_c, T scale)
{
    const int64_t idx = blockIdx.x * 256LL + threadIdx.x;
    if (idx >= ncell) return;
    constexpr int b = 1 << LB, bm = b - 1;
    const int o = (int)(idx >> (3 * LB));
    const int loc = (int)(idx & ((1LL << (3 * LB)) - 1));
    const int cc[3] = {loc & bm, (loc >> LB) & bm, loc >> (2 * LB)};
    const int *nb = nbr + 4 * (int64_t)o;
    auto val = [&](int k, int blk, int l) -> T {
        if (blk < 0) return T(0);
        const int64_t i = k * in_c + ((int64_t)blk << (3 * LB)) + l;
        return c ? a[i] - c[i] : a[i];
    };
    T s = T(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        int q[3] = {cc[0], cc[1], cc[2]};
        int blk = nb[0];
        if (++q[k] > bm) {
            q[k] = 0;
            blk = nb[1 + k];
        }
        s += val(k, blk, (((q[2] << LB) + q[1]) << LB) + q[0]) - val(k, nb[0], loc);
    }
    out[idx] = scale * s;
}

// out_k(n) = a_k(n) - inv_dx * [d(n) - d(n - e_k)] - c_k(n)   (c may be null);
// d on the plan's source blocks, a, c, out on its target blocks.
template <typename T, int LB>
__global__ void __launch_bounds__(256) k_grad_combine(const T *__restrict__ d, const T *__restrict__ a,
                                                      const T *__restrict__ c, T *__restrict__ out,
                                                      const int *__restrict__ nbr, int64_t ncell, T inv_dx)
{
    const int64_t idx = blockIdx.x * 256LL + threadIdx.x;
    if (idx >= ncell) return;
    constexpr int b = 1 << LB, bm = b - 1;
    const int o = (int)(idx >> (3 * LB));
    const int loc = (int)(idx & ((1LL << (3 * LB)) - 1));
    const int cc[3] = {loc & bm, (loc >> LB) & bm, loc >> (2 * LB)};
    const int *nb = nbr + 4 * (int64_t)o;
    const T dn = nb[0] >= 0 ? d[((int64_t)nb[0] << (3 * LB)) + loc] : T(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        int q[3] = {cc[0], cc[1], cc[2]};
        int blk = nb[0];
        if (--q[k] < 0) {
            q[k] = bm;
            blk = nb[1 + k];
        }
        const T dm = blk >= 0 ? d[((int64_t)blk << (3 * LB)) + (((q[2] << LB) + q[1]) << LB) + q[0]] : T(0);
        const int64_t i = k * ncell + idx;
        T v = a[i] - inv_dx * (dn - dm);
        if (c) v -= c[i];
        out[i] = v;
    }
}

template <typename T>
__global__ void k_sub(const T *__restrict__ x, const T *__restrict__ y, T *__restrict__ out, int64_t n)
{
    const int64_t i = blockIdx.x * 256LL + threadIdx.x;
    if (i < n) out[i] = x[i] - y[i];
}

// y = W x, W row-major n x n: one warp per row, lanes stride the row
// (coalesced), shuffle reduction.
template <typename T>
__global__ void __launch_bounds__(256) k_gemv_n(const T *__restrict__ W, const T *__restrict__ x, T *__restrict__ y,
                                                int n)
{
    const int row = blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    const T *w = W + (int64_t)row * n;
    T s = T(0);
    for (int j = lane; j < n; j += 32) s += w[j] * x[j];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (lane == 0) y[row] = s;
}

// y = W^T x: a CTA owns 32 columns; its 8 warps sum rows i = g (mod 8) with
// lane = column (each warp reads 32 contiguous values of a row), then the 8
// partial sums are added in shared memory.
template <typename T>
__global__ void __launch_bounds__(256) k_gemv_t(const T *__restrict__ W, const T *__restrict__ x, T *__restrict__ y,
                                                int n)
{
    __shared__ T part[8][32];
    const int col = blockIdx.x * 32 + (threadIdx.x & 31);
    const int g = threadIdx.x >> 5;
    T s = T(0);
    if (col < n)
        for (int i = g; i < n; i += 8) s += W[(int64_t)i * n + col] * x[i];
    part[g][threadIdx.x & 31] = s;
    __syncthreads();
    if (g == 0 && col < n) {
        T t = T(0);
#pragma unroll
        for (int q = 0; q < 8; ++q) t += part[q][threadIdx.x];
        y[col] = t;
    }
}

template <typename T, int LB>
void launch_div_lb(dim3 grid, cudaStream_t s, const T *a, const T *c, T *out, const int *nbr, int64_t ncell,
                   int64_t in_c, T scale)
{
    k_div<T, LB><<<grid, 256, 0, s>>>(a, c, out, nbr, ncell, in_c, scale);
}

template <typename T, int LB>
void launch_grad_lb(dim3 grid, cudaStream_t s, const T *d, const T *a, const T *c, T *out, const int *nbr,
                    int64_t ncell, T inv_dx)
{
    k_grad_combine<T, LB><<<grid, 256, 0, s>>>(d, a, c, out, nbr, ncell, inv_dx);
}

template <typename T>
lgf_status div_t(lgf_ctx *ctx, int lb, const T *a, const T *c, T *out, const int *nbr, int64_t ncell, int64_t in_c,
                 T scale, cudaStream_t s)
{
    dim3 grid((unsigned)((ncell + 255) / 256));
    const int ph = prof_begin(ctx, s, "stage_div");
    switch (lb) {
    case 2: launch_div_lb<T, 2>(grid, s, a, c, out, nbr, ncell, in_c, scale); break;
    case 3: launch_div_lb<T, 3>(grid, s, a, c, out, nbr, ncell, in_c, scale); break;
    case 4: launch_div_lb<T, 4>(grid, s, a, c, out, nbr, ncell, in_c, scale); break;
    case 5: launch_div_lb<T, 5>(grid, s, a, c, out, nbr, ncell, in_c, scale); break;
    case 6: launch_div_lb<T, 6>(grid, s, a, c, out, nbr, ncell, in_c, scale); break;
    default: return fail(ctx, LGF_EINVAL, "stage: block edge must be 4..64");
    }
    LGF_CHECK_LAUNCH(ctx, "stage divergence");
    prof_end(ctx, s, ph);
    return LGF_OK;
}

template <typename T>
lgf_status grad_t(lgf_ctx *ctx, int lb, const T *d, const T *a, const T *c, T *out, const int *nbr, int64_t ncell,
                  T inv_dx, cudaStream_t s)
{
    dim3 grid((unsigned)((ncell + 255) / 256));
    const int ph = prof_begin(ctx, s, "stage_grad");
    switch (lb) {
    case 2: launch_grad_lb<T, 2>(grid, s, d, a, c, out, nbr, ncell, inv_dx); break;
    case 3: launch_grad_lb<T, 3>(grid, s, d, a, c, out, nbr, ncell, inv_dx); break;
    case 4: launch_grad_lb<T, 4>(grid, s, d, a, c, out, nbr, ncell, inv_dx); break;
    case 5: launch_grad_lb<T, 5>(grid, s, d, a, c, out, nbr, ncell, inv_dx); break;
    case 6: launch_grad_lb<T, 6>(grid, s, d, a, c, out, nbr, ncell, inv_dx); break;
    default: return fail(ctx, LGF_EINVAL, "stage: block edge must be 4..64");
    }
    LGF_CHECK_LAUNCH(ctx, "stage gradient");
    prof_end(ctx, s, ph);
    return LGF_OK;
}

// The timeout path of the bounded waits: an mbarrier expecting one arrival
// that never comes (no thread arrives, no copy is issued), so the wait runs
// out after `cycles` and sets the error word.
__global__ void k_wait_selftest(int *err, long long cycles)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) async::mbar_init(&bar);
    __syncthreads();
    async::mbar_wait(&bar, 0, err, cycles);
}

int lb_of(int b)
{
    int l = 0;
    while ((1 << l) < b) ++l;
    return (1 << l) == b ? l : -1;
}

}  // namespace

// out = (1/dx) Dbar (a - c) on the plan's target blocks (plan dir +1; a, c on
// its source blocks, c may be null).
lgf_status stage_div(lgf_ctx *ctx, const CurlPlan *pl, const void *a, const void *c, void *out, double dx,
                     cudaStream_t s)
{
    const int64_t b3 = (int64_t)pl->b * pl->b * pl->b;
    const int64_t ncell = (int64_t)(pl->tgt.size() / 3) * b3, in_c = (int64_t)(pl->src.size() / 3) * b3;
    if (ncell == 0) return LGF_OK;
    if (ctx->prec == LGF_F64)
        return div_t<double>(ctx, lb_of(pl->b), (const double *)a, (const double *)c, (double *)out, pl->nbr_dev,
                             ncell, in_c, 1.0 / dx, s);
    return div_t<float>(ctx, lb_of(pl->b), (const float *)a, (const float *)c, (float *)out, pl->nbr_dev, ncell, in_c,
                        (float)(1.0 / dx), s);
}

// out = a - G d - c on the plan's target blocks (plan dir -1; d on its source
// blocks; a, c, out three components on its target blocks, c may be null).
lgf_status stage_grad(lgf_ctx *ctx, const CurlPlan *pl, const void *d, const void *a, const void *c, void *out,
                      double dx, cudaStream_t s)
{
    const int64_t b3 = (int64_t)pl->b * pl->b * pl->b;
    const int64_t ncell = (int64_t)(pl->tgt.size() / 3) * b3;
    if (ncell == 0) return LGF_OK;
    if (ctx->prec == LGF_F64)
        return grad_t<double>(ctx, lb_of(pl->b), (const double *)d, (const double *)a, (const double *)c,
                              (double *)out, pl->nbr_dev, ncell, 1.0 / dx, s);
    return grad_t<float>(ctx, lb_of(pl->b), (const float *)d, (const float *)a, (const float *)c, (float *)out,
                         pl->nbr_dev, ncell, (float)(1.0 / dx), s);
}

lgf_status wait_selftest(lgf_ctx *ctx, long long cycles, cudaStream_t s)
{
    k_wait_selftest<<<1, 32, 0, s>>>(ctx->err_dev, cycles);
    LGF_CHECK_LAUNCH(ctx, "wait self-test");
    return LGF_OK;
}

// rhs = U - ub; y = W1 rhs; fh = W2 y (W2 null: W1^T y).  Vectors of n values.
lgf_status stage_force(lgf_ctx *ctx, const void *U, const void *ub, const void *W1, const void *W2, void *rhs, void *y,
                       void *fh, int n, cudaStream_t s)
{
    if (n == 0) return LGF_OK;
    const unsigned gv = (unsigned)((n + 255) / 256), gn = (unsigned)((n + 7) / 8), gt = (unsigned)((n + 31) / 32);
    const int ph = prof_begin(ctx, s, "stage_force");
    if (ctx->prec == LGF_F64) {
        k_sub<double><<<gv, 256, 0, s>>>((const double *)U, (const double *)ub, (double *)rhs, n);
        k_gemv_n<double><<<gn, 256, 0, s>>>((const double *)W1, (const double *)rhs, (double *)y, n);
        if (W2)
            k_gemv_n<double><<<gn, 256, 0, s>>>((const double *)W2, (const double *)y, (double *)fh, n);
        else
            k_gemv_t<double><<<gt, 256, 0, s>>>((const double *)W1, (const double *)y, (double *)fh, n);
    } else {
        k_sub<float><<<gv, 256, 0, s>>>((const float *)U, (const float *)ub, (float *)rhs, n);
        k_gemv_n<float><<<gn, 256, 0, s>>>((const float *)W1, (const float *)rhs, (float *)y, n);
        if (W2)
            k_gemv_n<float><<<gn, 256, 0, s>>>((const float *)W2, (const float *)y, (float *)fh, n);
        else
            k_gemv_t<float><<<gt, 256, 0, s>>>((const float *)W1, (const float *)y, (float *)fh, n);
    }
    LGF_CHECK_LAUNCH(ctx, "stage force solve");
    prof_end(ctx, s, ph);
    return LGF_OK;
}

}  // namespace lgf
