// Fused y and x inverse passes of the Poisson apply (FP32), one target plane
// per thread-block cluster.
//
// Unfused, the y inverse writes the array A (the target rows of every plane,
// half spectra along x) to global memory and the x inverse reads it back.
// Here a cluster of NCL CTAs takes one (field, target plane): the Lt_y target
// rows of the plane stay in the distributed shared memory of the cluster,
// rows [c RPB, (c + 1) RPB) in CTA c (RPB even, so a line pair never
// straddles two CTAs).
//   phase 1: the CTAs share out the plane's kx columns in tiles of W; each
//            column's inverse transform along y runs as in k_col_inverse, and
//            its target rows are stored into the owning CTA's shared memory
//            (st.shared::cluster through the cluster's address map);
//   cluster barrier;
//   phase 2: each CTA runs the x inverse of its own rows, line pair by line
//            pair as in k_row_inverse, and scatters to the target blocks.
// The arithmetic of every line is that of the two unfused kernels, in the
// same order, so the results are equal bit for bit.  Both lengths are
// compile-time (the radix plans); the half-output variants of both stages are
// chosen at run time.
#pragma once
#include <cooperative_groups.h>

#include "lgf_poisson_kernels.cuh"

namespace lgf {
namespace pk {

// One problem of a fused launch.  The CTAs of a job: nf * Lt_z * NCL, cluster
// by cluster (field-major, then plane).
struct YXJob {
    PoissonGeom g;               // scale = dx^2; Bstride set
    const Cx<float> *B;          // after the z pass: [field][tz][ky][kx]
    float *u;
    const Cx<float> *twy, *twx;  // twiddles of My and Mx
    int nf, lb, rpb;             // fields, log2 b, rows per CTA (even)
    int cta0, gx;                // gx: CTAs per field (Lt_z * NCL)
};

template <int MY, int MX>
struct YXCfg {
    using CY = ColCfg<float, MY>;
    using CX = RowCfg<float, MX>;
    static constexpr int TY = CY::W * CY::TPC;
    static constexpr int TX = CX::LPC * CX::TPC;
    static constexpr int THREADS = TY > TX ? TY : TX;
    // the work area of the two phases (they run one after the other)
    static constexpr size_t WORK = CY::SMEM > CX::SMEM ? CY::SMEM : CX::SMEM;
};

// Shared-memory bytes of a fused CTA with `rpb` rows of K complex values.
template <int MY, int MX>
constexpr size_t yx_smem(int rpb)
{
    return (size_t)rpb * (MX / 2 + 1) * sizeof(Cx<float>) + YXCfg<MY, MX>::WORK;
}

// A complex value of the (read-only) B array through the non-coherent path,
// so that the compiler may move the loads across the shared-memory stores.
__device__ __forceinline__ Cx<float> ldg_cx(const Cx<float> *p)
{
    const float2 v = __ldg(reinterpret_cast<const float2 *>(p));
    return {v.x, v.y};
}

template <int MY, int MX, int NCL>
__global__ void __cluster_dims__(NCL, 1, 1) __launch_bounds__(YXCfg<MY, MX>::THREADS)
    k_yx_inverse_rag(const __grid_constant__ RagTable<YXJob> tab)
{
    namespace cg = cooperative_groups;
    using T = float;
    using CY = ColCfg<T, MY>;
    using CX = RowCfg<T, MX>;
    using PY = Plan<MY>;
    constexpr int W = CY::W;
    // threads beyond a phase's own count take part in its barriers only
    constexpr bool GY = YXCfg<MY, MX>::THREADS > YXCfg<MY, MX>::TY;
    constexpr bool GX = YXCfg<MY, MX>::THREADS > YXCfg<MY, MX>::TX;
    const YXJob &J = rag_job(tab);
    const PoissonGeom &g = J.g;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int c = (int)blockIdx.x - J.cta0;
    const int field = c / J.gx;
    const int zi = (c % J.gx) / NCL;
    const int K = g.Kx, lb = J.lb, rpb = J.rpb;
    const int lo = g.t0[1], n = g.Lt[1];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx<T> *band = reinterpret_cast<Cx<T> *>(smem_raw);    // [rpb][K]: target rows rank*rpb ...
    Cx<T> *work = band + (size_t)rpb * K;
    // a plane without target blocks has nothing to compute (uniform over the
    // cluster: every CTA still reaches the cluster barrier)
    const bool plane_live = !g.tgtrow || g.tgtrow[zi >> lb] != 0ull;

    // ---- phase 1: inverse along y of the plane's columns, tile by tile ----
    if (plane_live) {
        Cx<T> *tw = work;
        Cx<T> *s = tw + MY;
        load_twiddles(tw, J.twy, MY);
        const ColAddrW ad{W};
        const int w = threadIdx.x % W, t = threadIdx.x / W;
        const bool act = !GY || t < PY::TPC;
        const Cx<T> *plane = J.B + field * g.Bstride + (int64_t)zi * MY * K;
        const bool half = lo + n <= MY / 2;
        constexpr int RL = PY::RL, R0 = PY::R0;
        constexpr int NGL = PY::GL / PY::TPC;
        const int64_t istep = (int64_t)(MY / RL) * K;
        const int ntile = (K + W - 1) / W;
#pragma unroll 1
        for (int tile = rank; tile < ntile; tile += NCL) {
            const int kx = tile * W + w;
            const bool live = act && kx < K;
            const Cx<T> *ib = plane + kx;
            Cx<T> cc[NGL][RL];
#pragma unroll
            for (int i = 0; i < NGL; ++i) {
                const int gg = t + i * PY::TPC;
                int64_t off = (int64_t)freq_of<MY>(gg * RL) * K;
#pragma unroll
                for (int q = 0; q < RL; ++q) {
                    cc[i][q] = live ? ldg_cx(ib + off) : Cx<T>{T(0), T(0)};
                    off += istep;
                }
            }
            if (act) {
#pragma unroll
                for (int i = 0; i < NGL; ++i) {
                    const int gg = t + i * PY::TPC;
                    Dft<RL, 1, T>::run(cc[i]);
#pragma unroll
                    for (int q = 0; q < RL; ++q) s[ad(w, (gg * RL) + q)] = cc[i][q];
                }
            }
            __syncthreads();
            if constexpr (PY::NST == 3) {
                if (act) middle_stage<MY, 1>(s, ad, w, t, tw);
                __syncthreads();
            }
            if (act) {
#pragma unroll
                for (int gg = t; gg < PY::G0; gg += PY::TPC) {
                    Cx<T> a[R0];
#pragma unroll
                    for (int q = 0; q < R0; ++q) a[q] = s[ad(w, q * PY::G0 + gg)];
                    if (half)
                        dit_group<R0, 1, true>(a, gg, tw);
                    else
                        dit_group<R0, 1, false>(a, gg, tw);
                    if (live) {
                        const int r = gg - lo;
#pragma unroll
                        for (int p = 0; p < R0; ++p) {
                            const int yr = r + p * PY::G0;
                            if ((half && p >= R0 / 2) || (unsigned)yr >= (unsigned)n) continue;
                            Cx<T> *dst = cl.map_shared_rank(band, yr / rpb);
                            dst[(yr % rpb) * K + kx] = a[p];
                        }
                    }
                }
            }
            __syncthreads();   // s is reused by the next tile
        }
    }
    cl.sync();   // every row of every CTA of the cluster is written

    // ---- phase 2: inverse along x of this CTA's rows ----
    if (!plane_live) return;
    using PX = Plan<MX>;
    constexpr int LPC = CX::LPC;
    Cx<T> *tw = work;
    Cx<T> *s = tw + MX;
    load_twiddles(tw, J.twx, MX);
    const int t = threadIdx.x % PX::TPC, l = threadIdx.x / PX::TPC;
    const int r0 = rank * rpb;
    const int r1 = min(n, r0 + rpb);
    const int np = r1 > r0 ? (r1 - r0) / 2 : 0;   // at most LPC (the host keeps rpb <= 2 LPC)
    T *uu = J.u + field * g.ustride;
    // one line pair per slot, no loop: every address stays a function of the
    // thread, as in k_row_inverse
    const bool live = (!GX || l < LPC) && l < np;
    const int yi = r0 + 2 * (live ? l : 0);
    if (g.tgtrow && !__syncthreads_or(live && ((g.tgtrow[zi >> lb] >> (yi >> lb)) & 1ull))) return;
    const Cx<T> *row = band + (size_t)(yi - r0) * K;
    row_inverse_line<T, MX, LPC, false, true>(t, l, live, zi, yi, row, uu, g, tw, s, lb);
}

}  // namespace pk
}  // namespace lgf

namespace lgf {
namespace pk {

// Host side: one fused launch (tables of kRagJobs) for jobs of one (MY, MX,
// NCL); each job's rpb set, gx filled here.
template <int MY, int MX, int NCL>
lgf_status yx_m(lgf_ctx *ctx, YXJob *jobs, int n, cudaStream_t s)
{
    int rmax = 2;
    for (int i = 0; i < n; ++i) {
        if (jobs[i].g.M[1] != MY || jobs[i].g.M[0] != MX || jobs[i].rpb * NCL < jobs[i].g.Lt[1] || jobs[i].rpb % 2 ||
            jobs[i].rpb > 2 * RowCfg<float, MX>::LPC)
            return fail(ctx, LGF_EINVAL, "fused inverse: job does not match the launch");
        jobs[i].gx = jobs[i].g.Lt[2] * NCL;
        rmax = jobs[i].rpb > rmax ? jobs[i].rpb : rmax;
    }
    const size_t smem = yx_smem<MY, MX>(rmax);
    auto kern = k_yx_inverse_rag<MY, MX, NCL>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaFuncSetAttribute");
    return rag_send(ctx, kern, YXCfg<MY, MX>::THREADS, smem, jobs, n, s, "poisson_yx_inverse");
}

// The lengths along x in two parts (PART 0: up to 384, PART 1: above), each
// part of each length along y its own translation unit.
template <int MY, int PART, int NCL>
lgf_status yx_mx(lgf_ctx *ctx, int Mx, YXJob *jobs, int n, cudaStream_t s)
{
    if constexpr (PART == 0) {
        switch (Mx) {
        case 32: return yx_m<MY, 32, NCL>(ctx, jobs, n, s);
        case 64: return yx_m<MY, 64, NCL>(ctx, jobs, n, s);
        case 80: return yx_m<MY, 80, NCL>(ctx, jobs, n, s);
        case 96: return yx_m<MY, 96, NCL>(ctx, jobs, n, s);
        case 128: return yx_m<MY, 128, NCL>(ctx, jobs, n, s);
        case 160: return yx_m<MY, 160, NCL>(ctx, jobs, n, s);
        case 192: return yx_m<MY, 192, NCL>(ctx, jobs, n, s);
        case 256: return yx_m<MY, 256, NCL>(ctx, jobs, n, s);
        case 320: return yx_m<MY, 320, NCL>(ctx, jobs, n, s);
        case 384: return yx_m<MY, 384, NCL>(ctx, jobs, n, s);
        default: break;
        }
    } else {
        switch (Mx) {
        case 512: return yx_m<MY, 512, NCL>(ctx, jobs, n, s);
        case 640: return yx_m<MY, 640, NCL>(ctx, jobs, n, s);
        case 768: return yx_m<MY, 768, NCL>(ctx, jobs, n, s);
        case 1024: return yx_m<MY, 1024, NCL>(ctx, jobs, n, s);
        case 1280: return yx_m<MY, 1280, NCL>(ctx, jobs, n, s);
        case 1536: return yx_m<MY, 1536, NCL>(ctx, jobs, n, s);
        case 2048: return yx_m<MY, 2048, NCL>(ctx, jobs, n, s);
        case 2560: return yx_m<MY, 2560, NCL>(ctx, jobs, n, s);
        case 3072: return yx_m<MY, 3072, NCL>(ctx, jobs, n, s);
        case 4096: return yx_m<MY, 4096, NCL>(ctx, jobs, n, s);
        default: break;
        }
    }
    return fail(ctx, LGF_EUNSUPPORTED, "fused inverse: length along x not in this part");
}

// Part of a length along x.
inline int yx_part(int Mx) { return Mx <= 384 ? 0 : 1; }

template <int MY, int PART>
lgf_status yx_launch_my(lgf_ctx *ctx, int Mx, int ncl, YXJob *jobs, int n, cudaStream_t s)
{
    switch (ncl) {
    case 1: return yx_mx<MY, PART, 1>(ctx, Mx, jobs, n, s);
    case 2: return yx_mx<MY, PART, 2>(ctx, Mx, jobs, n, s);
    case 4: return yx_mx<MY, PART, 4>(ctx, Mx, jobs, n, s);
    default: return fail(ctx, LGF_EINVAL, "fused inverse: cluster size 1, 2 or 4");
    }
}

// Work-area bytes of the pair and line pairs per CTA of its x inverse (for
// the host's choice of the cluster size); false for a length not supported.
template <int MY>
bool yx_info_my(int Mx, size_t *work, int *lpc)
{
    switch (Mx) {
#define LGF_YX_I(L)                              \
    case L:                                      \
        *work = YXCfg<MY, L>::WORK;              \
        *lpc = RowCfg<float, L>::LPC;            \
        return true;
        LGF_YX_I(32) LGF_YX_I(64) LGF_YX_I(80) LGF_YX_I(96) LGF_YX_I(128) LGF_YX_I(160) LGF_YX_I(192)
        LGF_YX_I(256) LGF_YX_I(320) LGF_YX_I(384) LGF_YX_I(512) LGF_YX_I(640) LGF_YX_I(768) LGF_YX_I(1024)
        LGF_YX_I(1280) LGF_YX_I(1536) LGF_YX_I(2048) LGF_YX_I(2560) LGF_YX_I(3072) LGF_YX_I(4096)
#undef LGF_YX_I
    default: return false;
    }
}

}  // namespace pk
}  // namespace lgf
