// Immersed-boundary regularisation R and interpolation I (Sec. 2.1):
//   (R g)^k(n) = sum_i g^k(i) delta_dx(x_F^k(n) - X_i),
//   (I v)^k(i) = dx^3 sum_n v^k(n) delta_dx(x_F^k(n) - X_i),
// with face k of cell n at x_F^k(n) = (n + (1 - e_k)/2) dx and
// delta_h(x) = h^-3 prod_d phi(x_d / h).  phi is the three-point kernel
// (1 + sqrt(1 - 3 r^2)) / 3 for |r| <= 1/2, (5 - 3|r| - sqrt(1 - 3 (1 - |r|)^2))
// / 6 for 1/2 <= |r| <= 3/2, zero beyond: for marker coordinate t along an
// axis (in lattice-index units) exactly the three points floor(t - 1/2) + 0, 1,
// 2 can carry weight.
//
// One warp per (marker, component): nine lanes form the axis weights, 27
// lanes own one face point each.  Interpolation sums the lanes with shuffles,
// in a fixed order; regularisation adds into the points with atomics (the
// order of the additions, hence the last bits of the result, varies from run
// to run).  A dense look-up table over the bounding box of the block set maps
// a lattice point's block to its index.  GB300's FP64 rate is low, so only
// the nine positions are FP64; the kernel weights are evaluated and summed in
// the context precision.
#include <algorithm>
#include <cmath>

#include "lgf_internal.cuh"

namespace lgf {

IBPlan::~IBPlan() { cudaFree(lut_dev); }

namespace {

template <typename W>
__device__ __forceinline__ W phi3(W r)
{
    const W a = fabs(r);
    if (a <= W(0.5)) return (W(1) + sqrt(W(1) - W(3) * a * a)) / W(3);
    if (a <= W(1.5)) {
        const W d = W(1) - a;
        return (W(5) - W(3) * a - sqrt(fmax(W(0), W(1) - W(3) * d * d))) / W(6);
    }
    return W(0);
}

struct IBGeom {
    int lb, lo[3], ext[3];
    const int *lut;   // [ext_z][ext_y][ext_x] -> block index or -1
};

// Element offset of lattice point n in the block layout, or -1 if its block is absent.
__device__ __forceinline__ int64_t cell_offset(const IBGeom &g, int x, int y, int z)
{
    const int bx = (x >> g.lb) - g.lo[0], by = (y >> g.lb) - g.lo[1], bz = (z >> g.lb) - g.lo[2];
    if ((unsigned)bx >= (unsigned)g.ext[0] || (unsigned)by >= (unsigned)g.ext[1] || (unsigned)bz >= (unsigned)g.ext[2])
        return -1;
    const int blk = g.lut[((int64_t)bz * g.ext[1] + by) * g.ext[0] + bx];
    if (blk < 0) return -1;
    const int m = (1 << g.lb) - 1;
    return ((int64_t)blk << (3 * g.lb)) + ((((z & m) << g.lb) + (y & m)) << g.lb) + (x & m);
}

// One warp per (marker, component).  Lanes 3d + j (d, j < 3) form the axis
// weight phi(n0_d + j - t_d) in the context precision (t_d - n0_d - j is formed
// in FP64 from the FP64 position, so only phi itself is rounded to the
// context precision); lane l < 27 then owns support point (l % 3, l / 3 % 3,
// l / 9) and takes its three factors by shuffles.
template <typename W>
__device__ __forceinline__ bool lane_point(const IBGeom &g, const double *X, int k, int lane, W &wt, int64_t &off)
{
    const int d = lane < 9 ? lane / 3 : 0, j = lane < 9 ? lane % 3 : 0;
    const double t = X[d] - (d == k ? 0.0 : 0.5);
    const int n0 = (int)floor(t - 0.5);
    const W w = phi3<W>((W)((double)(n0 + j) - t));
    const int dx = lane % 3, dy = (lane / 3) % 3, dz = (lane / 9) % 3;
    const W wx = __shfl_sync(0xffffffffu, w, dx), wy = __shfl_sync(0xffffffffu, w, 3 + dy),
            wz = __shfl_sync(0xffffffffu, w, 6 + dz);
    const int nx = __shfl_sync(0xffffffffu, n0, 0), ny = __shfl_sync(0xffffffffu, n0, 3),
              nz = __shfl_sync(0xffffffffu, n0, 6);
    if (lane >= 27) return false;
    wt = wx * wy * wz;
    if (wt == W(0)) return false;
    off = cell_offset(g, nx + dx, ny + dy, nz + dz);
    return off >= 0;
}

template <typename T>
__global__ void __launch_bounds__(256) k_ib_spread(IBGeom g, const double *__restrict__ X,
                                                   const T *__restrict__ gin, T *__restrict__ f, int64_t nm, int nrhs,
                                                   int64_t fcomp, double scale)
{
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= 3 * nm) return;
    const int k = (int)(wid / nm);
    const int64_t i = wid - k * nm;
    const double Xi[3] = {X[3 * i], X[3 * i + 1], X[3 * i + 2]};
    T wt;
    int64_t off;
    if (!lane_point<T>(g, Xi, k, lane, wt, off)) return;
    wt *= (T)scale;
    for (int r = 0; r < nrhs; ++r) {
        const T gv = gin[((int64_t)r * 3 + k) * nm + i];
        atomicAdd(f + ((int64_t)r * 3 + k) * fcomp + off, wt * gv);
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_ib_interp(IBGeom g, const double *__restrict__ X, const T *__restrict__ v,
                                                   T *__restrict__ U, int64_t nm, int nrhs, int64_t vcomp)
{
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= 3 * nm) return;   // whole warps leave together
    const int k = (int)(wid / nm);
    const int64_t i = wid - k * nm;
    const double Xi[3] = {X[3 * i], X[3 * i + 1], X[3 * i + 2]};
    T wt = T(0);
    int64_t off = 0;
    const bool on = lane_point<T>(g, Xi, k, lane, wt, off);
    for (int r = 0; r < nrhs; ++r) {
        T acc = on ? wt * v[((int64_t)r * 3 + k) * vcomp + off] : T(0);
#pragma unroll
        for (int sh = 16; sh > 0; sh >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, sh);
        if (lane == 0) U[((int64_t)r * 3 + k) * nm + i] = (T)acc;
    }
}

}  // namespace

lgf_status ib_plan(lgf_ctx *ctx, const lgf_blockset *set, IBPlan **out)
{
    if (IBPlan *hit = ctx->ibplans.find(
            [&](const IBPlan &p) {
                return p.b == set->b && (int)p.coords.size() == 3 * set->nblocks &&
                       std::equal(p.coords.begin(), p.coords.end(), set->coords);
            },
            ctx->counters.epoch)) {
        *out = hit;
        return LGF_OK;
    }
    auto p = std::make_unique<IBPlan>();
    p->b = set->b;
    p->coords.assign(set->coords, set->coords + 3 * (size_t)set->nblocks);
    int hi[3];
    for (int d = 0; d < 3; ++d) {
        p->lo[d] = set->nblocks ? set->coords[d] : 0;
        hi[d] = p->lo[d];
    }
    for (int i = 0; i < set->nblocks; ++i)
        for (int d = 0; d < 3; ++d) {
            p->lo[d] = std::min(p->lo[d], (int)set->coords[3 * i + d]);
            hi[d] = std::max(hi[d], (int)set->coords[3 * i + d]);
        }
    int64_t n = 1;
    for (int d = 0; d < 3; ++d) {
        p->ext[d] = set->nblocks ? hi[d] - p->lo[d] + 1 : 1;
        n *= p->ext[d];
    }
    if (n > (int64_t)1 << 26) return fail(ctx, LGF_EUNSUPPORTED, "IB: block set's bounding box exceeds 2^26 blocks");
    std::vector<int> lut((size_t)n, -1);
    for (int i = 0; i < set->nblocks; ++i) {
        const int x = set->coords[3 * i] - p->lo[0], y = set->coords[3 * i + 1] - p->lo[1],
                  z = set->coords[3 * i + 2] - p->lo[2];
        lut[((size_t)z * p->ext[1] + y) * p->ext[0] + x] = i;
    }
    if (cudaMalloc(&p->lut_dev, lut.size() * sizeof(int)) != cudaSuccess)
        return fail(ctx, LGF_ENOMEM, "IB plan: cudaMalloc");
    cudaError_t e = cudaMemcpy(p->lut_dev, lut.data(), lut.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "IB plan: copy");
    *out = ctx->ibplans.insert(std::move(p), ctx->counters.epoch, [&] { before_evict(ctx); },
                               &ctx->counters.plans_evicted);
    return LGF_OK;
}

lgf_status ib_run(lgf_ctx *ctx, const IBPlan *pl, bool spread, int64_t nm, const double *X, const void *in, void *out,
                  int nrhs, double dx, cudaStream_t s)
{
    IBGeom g{};
    g.lb = 0;
    while ((1 << g.lb) < pl->b) ++g.lb;
    for (int d = 0; d < 3; ++d) {
        g.lo[d] = pl->lo[d];
        g.ext[d] = pl->ext[d];
    }
    g.lut = pl->lut_dev;
    const int64_t comp = (int64_t)(pl->coords.size() / 3) << (3 * g.lb);
    const size_t esz = ctx->prec == LGF_F64 ? 8 : 4;
    if (spread) LGF_CUDA(ctx, cudaMemsetAsync(out, 0, (size_t)nrhs * 3 * comp * esz, s));
    if (nm == 0) return LGF_OK;
    const unsigned grid = (unsigned)((3 * nm * 32 + 255) / 256);
    const int ph = prof_begin(ctx, s, spread ? "ib_spread" : "ib_interp");
    const double scale = 1.0 / (dx * dx * dx);
    if (ctx->prec == LGF_F64) {
        if (spread)
            k_ib_spread<double><<<grid, 256, 0, s>>>(g, X, (const double *)in, (double *)out, nm, nrhs, comp, scale);
        else
            k_ib_interp<double><<<grid, 256, 0, s>>>(g, X, (const double *)in, (double *)out, nm, nrhs, comp);
    } else {
        if (spread)
            k_ib_spread<float><<<grid, 256, 0, s>>>(g, X, (const float *)in, (float *)out, nm, nrhs, comp, scale);
        else
            k_ib_interp<float><<<grid, 256, 0, s>>>(g, X, (const float *)in, (float *)out, nm, nrhs, comp);
    }
    LGF_CHECK_LAUNCH(ctx, spread ? "IB spread" : "IB interpolation");
    prof_end(ctx, s, ph);
    return LGF_OK;
}

}  // namespace lgf
