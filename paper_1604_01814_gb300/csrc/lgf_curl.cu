// Staggered-grid curl C (faces -> edges), its adjoint C^dagger (edges ->
// faces) and the velocity refresh of Sec. 4.1, Eq. vel_refresh.
//
// Cell n holds face k at (n + (1 - e_k)/2) dx and edge k at (n + e_k/2) dx;
// a vector field is [nrhs][3][nblocks][b^3] with component k of cell n in
// the cell's slot.  With (k, i, j) the cyclic triples,
//   (C u)_k(n)         =  ([u_j(n) - u_j(n - e_i)] - [u_i(n) - u_i(n - e_j)]) / dx
//   (C^dagger w)_k(n)  = -([w_j(n) - w_j(n + e_i)] - [w_i(n) - w_i(n + e_j)]) / dx,
// one formula with the shift direction D = -1 or +1 and a sign.  Values
// outside the input block set are zero.  Each thread forms the three
// components of one output cell: three loads at the cell itself and six
// shifted ones (the shifted rows of the same block are the neighbouring
// threads' loads and come from L1), plus a neighbour-block load where the
// shift leaves the block.
//
// The refresh runs w = C u on the source blocks, s = L^{-1} w = dx^2 G_L * w
// (the Poisson engine, three scalar fields per right-hand side) on the
// target blocks and their +x, +y, +z neighbours, and u = -C^dagger s on the
// target blocks.  The minus sign makes the composition return a
// divergence-free u unchanged (L_F = -G G^dagger - C^dagger C, Sec. 2.1).
#include <algorithm>
#include <cmath>
#include <set>

#include "lgf_internal.cuh"

namespace lgf {

CurlPlan::~CurlPlan() { cudaFree(nbr_dev); }

namespace {

template <typename T, int LB, int D>
__global__ void __launch_bounds__(256) k_curl(const T *__restrict__ in, T *__restrict__ out,
                                              const int *__restrict__ nbr, int64_t ncell, int64_t in_c,
                                              int64_t out_c, T scale)
{
    const int64_t idx = blockIdx.x * 256LL + threadIdx.x;
    if (idx >= ncell) return;
    constexpr int b = 1 << LB, bm = b - 1;
    const int o = (int)(idx >> (3 * LB));
    const int loc = (int)(idx & ((1LL << (3 * LB)) - 1));
    const int c[3] = {loc & bm, (loc >> LB) & bm, loc >> (2 * LB)};
    const int *nb = nbr + 4 * (int64_t)o;
    const int self = nb[0];
    const T *inr = in + blockIdx.y * 3 * in_c;
    T *outr = out + blockIdx.y * 3 * out_c + ((int64_t)o << (3 * LB)) + loc;
    T v[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) v[k] = self >= 0 ? inr[k * in_c + ((int64_t)self << (3 * LB)) + loc] : T(0);
    // component comp at n + D e_a
    auto shifted = [&](int comp, int a) -> T {
        int cc[3] = {c[0], c[1], c[2]};
        cc[a] += D;
        int blk = self;
        if (cc[a] < 0 || cc[a] > bm) {
            blk = nb[1 + a];
            cc[a] &= bm;
        }
        if (blk < 0) return T(0);
        return inr[comp * in_c + ((int64_t)blk << (3 * LB)) + (((cc[2] << LB) + cc[1]) << LB) + cc[0]];
    };
    // (k, i, j) = (0, 1, 2), (1, 2, 0), (2, 0, 1)
    outr[0] = scale * ((v[2] - shifted(2, 1)) - (v[1] - shifted(1, 2)));
    outr[out_c] = scale * ((v[0] - shifted(0, 2)) - (v[2] - shifted(2, 0)));
    outr[2 * out_c] = scale * ((v[1] - shifted(1, 0)) - (v[0] - shifted(0, 1)));
}

template <typename T, int D>
lgf_status launch_curl_t(lgf_ctx *ctx, int lb, const T *in, T *out, const int *nbr, int64_t ncell, int64_t in_c,
                         int64_t out_c, int nrhs, T scale, cudaStream_t s)
{
    dim3 grid((unsigned)((ncell + 255) / 256), nrhs);
    const int ph = prof_begin(ctx, s, D < 0 ? "curl" : "curl_adjoint");
    switch (lb) {
    case 2: k_curl<T, 2, D><<<grid, 256, 0, s>>>(in, out, nbr, ncell, in_c, out_c, scale); break;
    case 3: k_curl<T, 3, D><<<grid, 256, 0, s>>>(in, out, nbr, ncell, in_c, out_c, scale); break;
    case 4: k_curl<T, 4, D><<<grid, 256, 0, s>>>(in, out, nbr, ncell, in_c, out_c, scale); break;
    case 5: k_curl<T, 5, D><<<grid, 256, 0, s>>>(in, out, nbr, ncell, in_c, out_c, scale); break;
    case 6: k_curl<T, 6, D><<<grid, 256, 0, s>>>(in, out, nbr, ncell, in_c, out_c, scale); break;
    default: return fail(ctx, LGF_EINVAL, "curl: block edge must be 4..64");
    }
    LGF_CHECK_LAUNCH(ctx, "curl kernel");
    prof_end(ctx, s, ph);
    return LGF_OK;
}

int log2_exact(int b)
{
    int l = 0;
    while ((1 << l) < b) ++l;
    return (1 << l) == b ? l : -1;
}

}  // namespace

lgf_status curl_plan(lgf_ctx *ctx, const lgf_blockset *src, const lgf_blockset *tgt, int dir, CurlPlan **out)
{
    const int b = src->b;
    if (CurlPlan *hit = ctx->cplans.find(
            [&](const CurlPlan &p) {
                return p.b == b && p.dir == dir && (int)p.src.size() == 3 * src->nblocks &&
                       (int)p.tgt.size() == 3 * tgt->nblocks && std::equal(p.src.begin(), p.src.end(), src->coords) &&
                       std::equal(p.tgt.begin(), p.tgt.end(), tgt->coords);
            },
            ctx->counters.epoch)) {
        *out = hit;
        return LGF_OK;
    }
    std::map<std::array<int, 3>, int> idx;
    for (int i = 0; i < src->nblocks; ++i)
        idx[{src->coords[3 * i], src->coords[3 * i + 1], src->coords[3 * i + 2]}] = i;
    auto find = [&](int x, int y, int z) {
        auto it = idx.find({x, y, z});
        return it == idx.end() ? -1 : it->second;
    };
    std::vector<int> nbr(4 * (size_t)tgt->nblocks);
    for (int t = 0; t < tgt->nblocks; ++t) {
        const int x = tgt->coords[3 * t], y = tgt->coords[3 * t + 1], z = tgt->coords[3 * t + 2];
        nbr[4 * t] = find(x, y, z);
        nbr[4 * t + 1] = find(x + dir, y, z);
        nbr[4 * t + 2] = find(x, y + dir, z);
        nbr[4 * t + 3] = find(x, y, z + dir);
    }
    auto p = std::make_unique<CurlPlan>();
    p->b = b;
    p->dir = dir;
    p->src.assign(src->coords, src->coords + 3 * (size_t)src->nblocks);
    p->tgt.assign(tgt->coords, tgt->coords + 3 * (size_t)tgt->nblocks);
    if (!nbr.empty()) {
        if (cudaMalloc(&p->nbr_dev, nbr.size() * sizeof(int)) != cudaSuccess)
            return fail(ctx, LGF_ENOMEM, "curl plan: cudaMalloc");
        cudaError_t e = cudaMemcpy(p->nbr_dev, nbr.data(), nbr.size() * sizeof(int), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "curl plan: copy");
    }
    *out = ctx->cplans.insert(std::move(p), ctx->counters.epoch, [&] { before_evict(ctx); },
                              &ctx->counters.plans_evicted);
    return LGF_OK;
}

// out = scale * stencil_D(in) for D = dir (see the file comment); in on the
// plan's source blocks, out on its target blocks, nrhs vector fields.
lgf_status curl_run(lgf_ctx *ctx, const CurlPlan *pl, const void *in, void *out, int nrhs, double scale,
                    cudaStream_t s)
{
    const int lb = log2_exact(pl->b);
    const int64_t b3 = (int64_t)pl->b * pl->b * pl->b;
    const int64_t ntgt = (int64_t)pl->tgt.size() / 3, nsrc = (int64_t)pl->src.size() / 3;
    if (ntgt == 0) return LGF_OK;
    const int64_t ncell = ntgt * b3;
    if (ctx->prec == LGF_F64) {
        return pl->dir < 0 ? launch_curl_t<double, -1>(ctx, lb, (const double *)in, (double *)out, pl->nbr_dev, ncell,
                                                       nsrc * b3, ntgt * b3, nrhs, scale, s)
                           : launch_curl_t<double, 1>(ctx, lb, (const double *)in, (double *)out, pl->nbr_dev, ncell,
                                                      nsrc * b3, ntgt * b3, nrhs, scale, s);
    }
    return pl->dir < 0 ? launch_curl_t<float, -1>(ctx, lb, (const float *)in, (float *)out, pl->nbr_dev, ncell,
                                                  nsrc * b3, ntgt * b3, nrhs, (float)scale, s)
                       : launch_curl_t<float, 1>(ctx, lb, (const float *)in, (float *)out, pl->nbr_dev, ncell,
                                                 nsrc * b3, ntgt * b3, nrhs, (float)scale, s);
}

// Target blocks and their +x, +y, +z neighbours, sorted.
std::vector<int32_t> grown_forward(const lgf_blockset *tgt)
{
    std::set<std::array<int, 3>> out;
    for (int t = 0; t < tgt->nblocks; ++t) {
        const int x = tgt->coords[3 * t], y = tgt->coords[3 * t + 1], z = tgt->coords[3 * t + 2];
        out.insert({x, y, z});
        out.insert({x + 1, y, z});
        out.insert({x, y + 1, z});
        out.insert({x, y, z + 1});
    }
    std::vector<int32_t> v;
    v.reserve(3 * out.size());
    for (auto &c : out) v.insert(v.end(), c.begin(), c.end());
    return v;
}

}  // namespace lgf
