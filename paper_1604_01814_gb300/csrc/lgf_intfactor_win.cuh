// Integrating-factor pass with a register window (radius bound RMAX fixed at
// compile time, actual radius R <= RMAX at run time; weights past R are zero).
//
// A CTA stages one slab of an output block plus a halo of RMAX points along
// the pass axis (16-byte loads from the neighbour blocks, zero where a block
// is absent).  Each thread then produces V outputs along the axis for NV
// adjacent x values: it streams the V + 2 RMAX staged inputs once, and every
// input feeds the V accumulators it touches with the weight w(|d|) held in a
// register (the distance d is a compile-time constant after unrolling).
// Shared-memory traffic per output is (V + 2 RMAX) / V values instead of
// 2R + 1.  In FP32 the accumulators go in pairs through the packed FP32x2 FMA
// (two lane-wise fma.rn per instruction, the scalar loop's bits): adjacent x
// values in the y and z passes, adjacent y rows in the x pass of the fused
// x+y kernel.
#pragma once
#include <algorithm>
#include <type_traits>

#include "lgf_async.cuh"
#include "lgf_internal.cuh"

namespace lgf {
namespace win {

template <typename T>
struct Vec;
template <>
struct Vec<float> {
    using V = float4;
    static constexpr int N = 4;
};
template <>
struct Vec<double> {
    using V = double2;
    static constexpr int N = 2;
};

constexpr int kV = 4;   // outputs per thread along the pass axis

// Register copy of the weights w_0 .. w_RMAX (zero past the job's radius).
// In FP32 each weight is held as the pair (w_k, w_k), the operand of the packed
// FP32x2 FMA: one instruction forms two lane-wise fma.rn, each rounded exactly
// as a scalar FFMA, so the packed loops give the scalar loops' bits.
template <typename T, int RMAX>
struct WinW {
    T w[RMAX + 1];
};
template <int RMAX>
struct WinW<float, RMAX> {
    float2 w[RMAX + 1];
};

template <typename T, int RMAX>
__device__ __forceinline__ void load_weights(WinW<T, RMAX> &W, const T *__restrict__ wg, int R)
{
#pragma unroll
    for (int k = 0; k <= RMAX; ++k) {
        const T v = k <= R ? wg[k] : T(0);
        if constexpr (std::is_same<T, float>::value) W.w[k] = make_float2(v, v);
        else W.w[k] = v;
    }
}

template <int RMAX>
__device__ __forceinline__ float wscalar(const WinW<float, RMAX> &W, int k) { return W.w[k].x; }
template <int RMAX>
__device__ __forceinline__ double wscalar(const WinW<double, RMAX> &W, int k) { return W.w[k]; }

// kV consecutive outputs along a column of staged inputs (stride st between
// axis positions; the window starts RMAX before the first output) for the
// Vec<T>::N adjacent x values of one 16-byte vector.
template <int RMAX>
__device__ __forceinline__ void col_window(const float *col, int st, const WinW<float, RMAX> &W, float4 (&out)[kV])
{
    float2 acc[kV][2];
#pragma unroll
    for (int v = 0; v < kV; ++v) acc[v][0] = acc[v][1] = make_float2(0.f, 0.f);
#pragma unroll
    for (int pos = 0; pos < kV + 2 * RMAX; ++pos) {
        const float4 val = *reinterpret_cast<const float4 *>(col + pos * st);
        const float2 lo = make_float2(val.x, val.y), hi = make_float2(val.z, val.w);
#pragma unroll
        for (int v = 0; v < kV; ++v) {
            const int d = pos - RMAX - v;
            if (d >= -RMAX && d <= RMAX) {
                acc[v][0] = __ffma2_rn(W.w[d < 0 ? -d : d], lo, acc[v][0]);
                acc[v][1] = __ffma2_rn(W.w[d < 0 ? -d : d], hi, acc[v][1]);
            }
        }
    }
#pragma unroll
    for (int v = 0; v < kV; ++v) out[v] = make_float4(acc[v][0].x, acc[v][0].y, acc[v][1].x, acc[v][1].y);
}

template <int RMAX>
__device__ __forceinline__ void col_window(const double *col, int st, const WinW<double, RMAX> &W,
                                           double2 (&out)[kV])
{
    double acc[kV][2];
#pragma unroll
    for (int v = 0; v < kV; ++v) acc[v][0] = acc[v][1] = 0.0;
#pragma unroll
    for (int pos = 0; pos < kV + 2 * RMAX; ++pos) {
        const double2 val = *reinterpret_cast<const double2 *>(col + pos * st);
#pragma unroll
        for (int v = 0; v < kV; ++v) {
            const int d = pos - RMAX - v;
            if (d >= -RMAX && d <= RMAX) {
                acc[v][0] += W.w[d < 0 ? -d : d] * val.x;
                acc[v][1] += W.w[d < 0 ? -d : d] * val.y;
            }
        }
    }
#pragma unroll
    for (int v = 0; v < kV; ++v) out[v] = make_double2(acc[v][0], acc[v][1]);
}

}  // namespace win

// One integrating-factor apply inside a grouped launch: its own input,
// output, weights and radius; the block sets (neighbour tables) are shared.
template <typename T>
struct SepJob {
    const T *in;
    T *out;
    const T *w;
    int R;
    int pad;
    int64_t in_stride, out_stride;   // elements per field
};
constexpr int kMaxSepJobs = 8;
template <typename T>
struct SepJobs {
    SepJob<T> j[kMaxSepJobs];
    int n;    // jobs in this launch
    int nf;   // fields per job (grid.z = n * nf)
};

// Ragged launches (lgf_batch_apply's ragged mode): jobs of different plans
// (block sets) in one launch.  Job i carries its plan's tables and owns the
// CTAs [cta0_i, cta0_i + nitems_i * nf_i) along x (field-major); every CTA
// finds its job by a binary search over cta0.
constexpr int kSepRagJobs = 64;
template <typename T>
struct SepRagJob {
    SepJob<T> job;
    const int *nbr;     // the pass's neighbour table of the job's plan
    const int *items;   // fused x+y pass: the plan's output items
    int nr, nitems, nf, cta0;
};
template <typename T>
struct SepRag {
    SepRagJob<T> j[kSepRagJobs];
    int n;
};

// Where a CTA's work lies: its job, field and output item, and the plan
// tables to use.
template <typename T>
struct SepAt {
    const SepJob<T> *J;
    int field, item;
    const int *nbr, *items;
    int nr;
};
template <typename T>
__device__ __forceinline__ SepAt<T> sep_at(const SepJobs<T> &t, const int *nbr, const int *items, int nr)
{
    return {&t.j[blockIdx.z / t.nf], (int)blockIdx.z % t.nf, (int)blockIdx.x, nbr, items, nr};
}
template <typename T>
__device__ __forceinline__ SepAt<T> sep_at(const SepRag<T> &t, const int *, const int *, int)
{
    int lo = 0, hi = t.n - 1;
    const int c = blockIdx.x;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (t.j[mid].cta0 <= c) lo = mid;
        else hi = mid - 1;
    }
    const SepRagJob<T> &r = t.j[lo];
    const int k = c - r.cta0;
    return {&r.job, k / r.nitems, k % r.nitems, r.nbr, r.items, r.nr};
}

namespace win {

// Threads per CTA and slab extent for block edge b = 2^LB.
template <typename T, int LB, int AX>
struct Cfg {
    static constexpr int b = 1 << LB;
    static constexpr int NV = Vec<T>::N;
    // threads needed for one plane of the slab axis
    static constexpr int per_plane = AX == 0 ? b * (b / kV) : (b / NV) * (b / kV);
    static constexpr int NS0 = 256 / per_plane;
    static constexpr int NS = NS0 < 1 ? 1 : (NS0 > b ? b : NS0);
    static constexpr int THREADS = NS * per_plane;
};

template <typename T, int LB, int AX, int RMAX, class Tab = SepJobs<T>>
__global__ void __launch_bounds__(Cfg<T, LB, AX>::THREADS)
    k_sep_win(const __grid_constant__ Tab jobs, const int *__restrict__ nbr_arg, int nr_arg)
{
    const SepAt<T> at = sep_at(jobs, nbr_arg, nullptr, nr_arg);
    const SepJob<T> &J = *at.J;
    const int field = at.field;
    const int *__restrict__ nbr = at.nbr;
    const int nr = at.nr;
    const T *__restrict__ wg = J.w;
    const int R = J.R;
    using C = Cfg<T, LB, AX>;
    using VT = typename Vec<T>::V;
    constexpr int b = C::b, bm = b - 1, NV = C::NV, NS = C::NS, HL = RMAX, E = b + 2 * HL;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *s = reinterpret_cast<T *>(smem_raw);
    const int o = at.item;
    const int s0 = blockIdx.y * NS;
    const int nd = 2 * nr + 1;
    const int *nb = nbr + (int64_t)o * nd;
    const T *inf = J.in + field * J.in_stride;
    T *outf = J.out + field * J.out_stride;

    // ---- stage [slab + halo] with 16-byte loads ----
    constexpr int rowlen = AX == 0 ? E : b;
    constexpr int nrows = AX == 0 ? NS * b : NS * E;
    constexpr int vpr = rowlen / NV;
    constexpr int total = nrows * vpr;
    constexpr int U = 4;
    for (int base = threadIdx.x; base < total; base += U * C::THREADS) {
        VT v[U];
        int dst[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int it = base + u * C::THREADS;
            dst[u] = -1;
            v[u] = VT{};
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
                y = s0 + row % NS;
                e = row / NS - HL;
                z = e & bm;
            }
            dst[u] = it * NV;
            const int bi = nb[(e + nr * b) >> LB];
            if (bi >= 0)
                v[u] = *reinterpret_cast<const VT *>(inf + ((int64_t)bi << (3 * LB)) + (((z << LB) + y) << LB) + x);
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (dst[u] >= 0) *reinterpret_cast<VT *>(s + dst[u]) = v[u];
    }
    WinW<T, RMAX> W;
    load_weights(W, wg, R);
    __syncthreads();

    // ---- stencil through the register window ----
    const int tid = threadIdx.x;
    if constexpr (AX == 0) {
        // thread: kV consecutive x outputs of row (y, z)
        const int xv = tid % (b / kV);
        const int y = (tid / (b / kV)) & bm;
        const int sl = tid / (b * (b / kV));
        const int x0 = xv * kV;
        const T *row = s + (sl * b + y) * E + x0;      // window starts at x0 - HL
        T acc[kV];
#pragma unroll
        for (int v = 0; v < kV; ++v) acc[v] = T(0);
#pragma unroll
        for (int i = 0; i < (kV + 2 * RMAX) / NV; ++i) {
            const VT val = *reinterpret_cast<const VT *>(row + i * NV);
            const T *vs = reinterpret_cast<const T *>(&val);
#pragma unroll
            for (int e = 0; e < NV; ++e) {
                const int pos = i * NV + e;             // input at x0 - HL + pos
#pragma unroll
                for (int v = 0; v < kV; ++v) {
                    const int d = pos - HL - v;
                    if (d >= -RMAX && d <= RMAX) acc[v] += wscalar(W, d < 0 ? -d : d) * vs[e];
                }
            }
        }
        const int z = s0 + sl;
#pragma unroll
        for (int v = 0; v < kV; v += NV) {
            VT r;
            T *rr = reinterpret_cast<T *>(&r);
#pragma unroll
            for (int e = 0; e < NV; ++e) rr[e] = acc[v + e];
            *reinterpret_cast<VT *>(outf + ((int64_t)o << (3 * LB)) + (((z << LB) + y) << LB) + x0 + v) = r;
        }
    } else {
        // thread: NV adjacent x values, kV consecutive outputs along the axis.
        // z pass: the slab row (y) varies before the axis group, so the two
        // thread quads of a quarter-warp read adjacent rows (128 contiguous
        // bytes, every bank once) where the axis groups would be 64 floats
        // apart (the same banks); the output rows stay contiguous.
        const int xv = tid % (b / NV);
        const int av = AX == 2 ? tid / ((b / NV) * NS) : (tid / (b / NV)) % (b / kV);
        const int sl = AX == 2 ? (tid / (b / NV)) % NS : tid / ((b / NV) * (b / kV));
        const int x = xv * NV, a0 = av * kV;
        // element (axis position p in [-HL, b + HL), slab-local sl, x)
        const int st = AX == 1 ? b : NS * b;
        const T *col = AX == 1 ? s + (sl * E + a0) * b + x : s + (a0 * NS + sl) * b + x;
        VT r[kV];
        col_window<RMAX>(col, st, W, r);
#pragma unroll
        for (int v = 0; v < kV; ++v) {
            const int Y = AX == 1 ? a0 + v : s0 + sl;
            const int Z = AX == 1 ? s0 + sl : a0 + v;
            *reinterpret_cast<VT *>(outf + ((int64_t)o << (3 * LB)) + (((Z << LB) + Y) << LB) + x) = r[v];
        }
    }
}

// The z pass as a persistent kernel that stages with bulk asynchronous
// copies.  In the block layout every staged z-plane of a slab (NS rows of b)
// is one contiguous run, so a slab plus its halo is at most E bulk copies
// (cp.async.bulk, completed on an mbarrier); planes of absent blocks are
// zero-filled.  Each CTA walks the items (output block, slab, job, field)
// with a stride of the grid and keeps two slab buffers: the copies of item
// t + 1 are in flight while the stencil runs on item t.  Every wait is
// bounded; one that runs out sets a bit of *err, drains the other buffer's
// copies (again bounded) and ends the CTA (lgf_async.cuh).  Results equal
// those of k_sep_win<T, LB, 2, RMAX> bit for bit.
template <typename T, int LB, int RMAX>
__global__ void __launch_bounds__(Cfg<T, LB, 2>::THREADS)
    k_sep_z_bulk(const SepJobs<T> jobs, const int *__restrict__ nbr, int nr, int nout, int *err)
{
    using C = Cfg<T, LB, 2>;
    using VT = typename Vec<T>::V;
    constexpr int b = C::b, bm = b - 1, NV = C::NV, NS = C::NS, HL = RMAX, E = b + 2 * HL;
    constexpr int PV = NS * b;      // values per staged plane
    constexpr int NSL = b / NS;     // slabs per block
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *const sbuf = reinterpret_cast<T *>(smem_raw);   // [2][E][NS][b]
    __shared__ __align__(8) uint64_t bar[2];
    const int nd = 2 * nr + 1;
    const int nitems = nout * NSL * jobs.n * jobs.nf;
    if (threadIdx.x == 0) {
        async::mbar_init(&bar[0]);
        async::mbar_init(&bar[1]);
    }
    __syncthreads();
    // item -> output block o (fastest, for neighbour reuse in L2), slab, field, job
    auto decode = [&](int i, int &o, int &s0, int &fd, int &jb) {
        o = i % nout;
        int r = i / nout;
        s0 = (r % NSL) * NS;
        r /= NSL;
        fd = r % jobs.nf;
        jb = r / jobs.nf;
    };
    // stage item i into buffer k: zero the planes of absent blocks, then the
    // first warp announces the bytes and issues one bulk copy per present plane
    auto issue = [&](int i, int k) {
        int o, s0, fd, jb;
        decode(i, o, s0, fd, jb);
        const int *nb = nbr + (int64_t)o * nd;
        const T *inf = jobs.j[jb].in + fd * jobs.j[jb].in_stride;
        T *sb = sbuf + k * E * PV;
        for (int it = threadIdx.x; it < E * (PV / NV); it += C::THREADS)
            if (nb[(it / (PV / NV) - HL + nr * b) >> LB] < 0) *reinterpret_cast<VT *>(sb + it * NV) = VT{};
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            if (lane == 0) {
                uint32_t bytes = 0;
                for (int p = 0; p < E; ++p) bytes += nb[(p - HL + nr * b) >> LB] >= 0 ? PV * sizeof(T) : 0;
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                async::mbar_arrive_expect(&bar[k], bytes);
            }
            __syncwarp();
            for (int p = lane; p < E; p += 32) {
                const int e = p - HL;
                const int bi = nb[(e + nr * b) >> LB];
                if (bi >= 0)
                    async::bulk_copy(sb + p * PV, inf + ((int64_t)bi << (3 * LB)) + (((e & bm) << LB) + s0) * b,
                                     PV * sizeof(T), &bar[k]);
            }
        }
    };
    const int tid = threadIdx.x;
    const int xv = tid % (b / NV);
    const int sl = (tid / (b / NV)) % NS;
    const int av = tid / ((b / NV) * NS);
    const int x = xv * NV, a0 = av * kV;
    int t = 0;
    if ((int)blockIdx.x < nitems) issue(blockIdx.x, 0);
    for (int i = blockIdx.x; i < nitems; i += gridDim.x, ++t) {
        const int k = t & 1;
        const int inext = i + gridDim.x;
        if (inext < nitems) issue(inext, k ^ 1);
        const bool ok = async::mbar_wait(&bar[k], (t >> 1) & 1, err);
        if (!__syncthreads_and(ok)) {
            if (inext < nitems) async::mbar_wait(&bar[k ^ 1], ((t + 1) >> 1) & 1, nullptr);
            return;
        }
        int o, s0, fd, jb;
        decode(i, o, s0, fd, jb);
        const SepJob<T> &J = jobs.j[jb];
        WinW<T, RMAX> W;
        load_weights(W, J.w, J.R);
        const T *col = sbuf + k * E * PV + (a0 * NS + sl) * b + x;
        VT r[kV];
        col_window<RMAX>(col, NS * b, W, r);
        T *outf = J.out + fd * J.out_stride;
#pragma unroll
        for (int v = 0; v < kV; ++v)
            *reinterpret_cast<VT *>(outf + ((int64_t)o << (3 * LB)) + ((((a0 + v) << LB) + s0 + sl) << LB) + x) = r[v];
        __syncthreads();   // buffer k is read; the next iteration may refill it
    }
}

// Fused x and y passes.  A CTA owns one output block, or two that are
// neighbours in y (a pair shares the y halo between them: 2b + 2 RMAX staged
// rows for 2b outputs instead of 2 (b + 2 RMAX)), and NS z-planes.  It stages
// the neighbourhood from the xy neighbour blocks, runs the x stencil over
// every staged row into an intermediate [NS][EY][b] and then the y stencil to
// the output block(s).
template <typename T, int LB, int RMAX>
struct XYCfg {
    static constexpr int b = 1 << LB, E = b + 2 * RMAX;
    static constexpr int EY1 = b + 2 * RMAX, EY = 2 * b + 2 * RMAX;   // staged rows: single, pair
    // FP32 stages row pairs interleaved, [EY/2][P2], with a 16-byte skew per
    // row pair (pitch P2 = 2E + 4), so that the row pairs of a warp start on
    // different bank groups.
    static constexpr int P2 = 2 * E + 4;
    static constexpr int RG = sizeof(T) == 4 ? (EY / 2) * P2 : EY * E;   // staged elements per plane
    // pitch of the x stencil's output rows: 20 floats for FP32 16^3 blocks, so
    // that the y stencil's two thread quads (rows 4 apart) fall on the two
    // halves of the banks; b elsewhere
    static constexpr int IP = sizeof(T) == 4 && b == 16 ? 20 : b;
    static constexpr int per_plane = RG + EY * IP;
    static constexpr int NS0 = 12288 / per_plane;
    static constexpr int NS = NS0 >= 8 ? 8 : NS0 >= 4 ? 4 : NS0 >= 2 ? 2 : 1;
    static constexpr int NSB = NS > b ? b : NS;
    static constexpr size_t SMEM = sizeof(T) * (size_t)NSB * per_plane;
};

// items: [n][2] output blocks (second -1 for a single block); nbr: for every
// output block its (2nr+1)^2 xy neighbourhood of source blocks.
template <typename T, int LB, int RMAX, class Tab = SepJobs<T>>
__global__ void __launch_bounds__(256) k_sep_xy(const __grid_constant__ Tab jobs, const int *__restrict__ nbr_arg,
                                                const int *__restrict__ items_arg, int nr_arg)
{
    const SepAt<T> at = sep_at(jobs, nbr_arg, items_arg, nr_arg);
    const SepJob<T> &J = *at.J;
    const int field = at.field;
    const int *__restrict__ nbr = at.nbr;
    const int *__restrict__ items = at.items;
    const int nr = at.nr;
    const T *__restrict__ wg = J.w;
    const int R = J.R;
    using C = XYCfg<T, LB, RMAX>;
    using VT = typename Vec<T>::V;
    constexpr int b = C::b, bm = b - 1, NV = Vec<T>::N, NS = C::NSB, HL = RMAX, E = C::E, EY = C::EY;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *rg = reinterpret_cast<T *>(smem_raw);       // [NS][EY][E] (FP32: [NS][EY/2][P2])
    T *im = rg + NS * C::RG;                        // [NS][EY][IP] (row pitch IP >= b)
    constexpr int IP = C::IP;
    const int o1 = items[2 * at.item], o2 = items[2 * at.item + 1];
    const bool pair = o2 >= 0;                      // uniform over the CTA
    const int ny = pair ? 2 : 1;
    const int rows = pair ? C::EY : C::EY1;         // staged rows per plane
    const int s0 = blockIdx.y * NS;
    const int nd = 2 * nr + 1;
    const int *nb1 = nbr + (int64_t)o1 * nd * nd;
    const int *nb2 = pair ? nbr + (int64_t)o2 * nd * nd : nb1;
    const T *inf = J.in + field * J.in_stride;
    T *outf = J.out + field * J.out_stride;
    // plane-local row -> (z-plane, staged row) with compile-time divisors
    auto split = [&](int row, int &zl, int &yr) {
        zl = pair ? row / C::EY : row / C::EY1;
        yr = row - zl * rows;
    };
    // ---- stage ----
    // FP64: one staged row per item, layout [NS][EY][E].  FP32: rows 2j and
    // 2j + 1 per item (the same source block: block edges and the halo are
    // even), interleaved as [NS][EY/2][E][2] (row pairs P2 apart), so that the
    // x stencil runs on the packed pair (row 2j, row 2j + 1) with one FP32x2
    // FMA per weight.
    constexpr bool PACK = std::is_same<T, float>::value;
    constexpr int RPI = PACK ? 2 : 1;                  // staged rows per item
    constexpr int vpr = E / NV;
    const int total = NS * (rows / RPI) * vpr;
    constexpr int U = 4;
    for (int base = threadIdx.x; base < total; base += U * 256) {
        VT v[U][RPI];
        int dst[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int it = base + u * 256;
            dst[u] = -1;
#pragma unroll
            for (int q = 0; q < RPI; ++q) v[u][q] = VT{};
            if (it >= total) continue;
            const int rr = it / vpr, cv = it - rr * vpr;
            int zl, yr;
            split(rr * RPI, zl, yr);
            const int ex = cv * NV - HL, ey = yr - HL, z = s0 + zl;
            dst[u] = PACK ? (zl * (EY / 2) + yr / 2) * C::P2 + cv * NV * 2 : (zl * EY + yr) * E + cv * NV;
            // block row of ey relative to the first output block: -nr .. ny - 1 + nr
            const int dyb = (ey + nr * b) >> LB;
            const int *nbt = dyb <= 2 * nr ? nb1 + dyb * nd : nb2 + (dyb - 1) * nd;
            const int bi = nbt[(ex + nr * b) >> LB];
            if (bi >= 0) {
                const T *src = inf + ((int64_t)bi << (3 * LB)) + (((z << LB) + (ey & bm)) << LB) + (ex & bm);
#pragma unroll
                for (int q = 0; q < RPI; ++q) v[u][q] = *reinterpret_cast<const VT *>(src + q * b);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (dst[u] < 0) continue;
            if constexpr (PACK) {
                const float4 a = v[u][0], c = v[u][RPI - 1];
                *reinterpret_cast<float4 *>(rg + dst[u]) = make_float4(a.x, c.x, a.y, c.y);
                *reinterpret_cast<float4 *>(rg + dst[u] + 4) = make_float4(a.z, c.z, a.w, c.w);
            } else {
                *reinterpret_cast<VT *>(rg + dst[u]) = v[u][0];
            }
        }
    }
    WinW<T, RMAX> W;
    load_weights(W, wg, R);
    __syncthreads();
    // ---- x stencil: every staged row, kV outputs per item (two rows in FP32) ----
    // (Lanes 32 bytes apart in FP32: two-way bank conflicts on these loads.
    // Mapping the items of a quarter-warp onto distinct bank groups made this
    // kernel faster alone but the graph step, where it runs beside the FFT
    // passes, slower, presumably because the shared-memory-bound form leaves
    // their warps more issue slots.)
    const int xitems = NS * (rows / RPI) * (b / kV);
    for (int it = threadIdx.x; it < xitems; it += 256) {
        const int xv = it % (b / kV);
        int zl, yr;
        split(it / (b / kV) * RPI, zl, yr);
        const int x0 = xv * kV;
        const int row = zl * EY + yr;
        // staged x_ext = x0 - HL ...
        const T *r = PACK ? rg + (zl * (EY / 2) + yr / 2) * C::P2 + 2 * x0 : rg + row * E + x0;
        if constexpr (PACK) {
            float2 acc[kV];                                    // (row, row + 1)
#pragma unroll
            for (int v = 0; v < kV; ++v) acc[v] = make_float2(0.f, 0.f);
#pragma unroll
            for (int i = 0; i < (kV + 2 * RMAX) / 2; ++i) {
                const float4 val = *reinterpret_cast<const float4 *>(r + 4 * i);
                const float2 pr[2] = {make_float2(val.x, val.y), make_float2(val.z, val.w)};
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int pos = 2 * i + e;
#pragma unroll
                    for (int v = 0; v < kV; ++v) {
                        const int d = pos - HL - v;
                        if (d >= -RMAX && d <= RMAX) acc[v] = __ffma2_rn(W.w[d < 0 ? -d : d], pr[e], acc[v]);
                    }
                }
            }
            static_assert(kV == 4, "one float4 per row");
            *reinterpret_cast<float4 *>(im + row * IP + x0) = make_float4(acc[0].x, acc[1].x, acc[2].x, acc[3].x);
            *reinterpret_cast<float4 *>(im + (row + 1) * IP + x0) =
                make_float4(acc[0].y, acc[1].y, acc[2].y, acc[3].y);
        } else {
            T acc[kV];
#pragma unroll
            for (int v = 0; v < kV; ++v) acc[v] = T(0);
#pragma unroll
            for (int i = 0; i < (kV + 2 * RMAX) / NV; ++i) {
                const VT val = *reinterpret_cast<const VT *>(r + i * NV);
                const T *vs = reinterpret_cast<const T *>(&val);
#pragma unroll
                for (int e = 0; e < NV; ++e) {
                    const int pos = i * NV + e;
#pragma unroll
                    for (int v = 0; v < kV; ++v) {
                        const int d = pos - HL - v;
                        if (d >= -RMAX && d <= RMAX) acc[v] += wscalar(W, d < 0 ? -d : d) * vs[e];
                    }
                }
            }
#pragma unroll
            for (int v = 0; v < kV; v += NV) {
                VT q;
                T *qq = reinterpret_cast<T *>(&q);
#pragma unroll
                for (int e = 0; e < NV; ++e) qq[e] = acc[v + e];
                *reinterpret_cast<VT *>(im + row * IP + x0 + v) = q;
            }
        }
    }
    __syncthreads();
    // ---- y stencil: NV adjacent x, kV consecutive y outputs per item ----
    const int ypp = ny * (b / kV);                     // y items per plane and x column
    const int yitems = NS * (b / NV) * ypp;
    for (int it = threadIdx.x; it < yitems; it += 256) {
        const int xv = it % (b / NV);
        const int yv = (it / (b / NV)) % ypp;
        const int zl = it / ((b / NV) * ypp);
        const int x = xv * NV, y0 = yv * kV;                  // output row among the ny * b
        const T *col = im + (zl * EY + y0) * IP + x;          // y_ext = y0 - HL ...
        VT q[kV];
        col_window<RMAX>(col, IP, W, q);
        const int z = s0 + zl;
        const int o = y0 < b ? o1 : o2;
        const int yl = y0 & bm;
#pragma unroll
        for (int v = 0; v < kV; ++v)
            *reinterpret_cast<VT *>(outf + ((int64_t)o << (3 * LB)) + (((z << LB) + yl + v) << LB) + x) = q[v];
    }
}

template <typename T, int LB, int RMAX>
lgf_status launch_xy_m(lgf_ctx *ctx, int nitems, const SepJobs<T> &jobs, cudaStream_t s, const int *nbr,
                       const int *items, int nr)
{
    using C = XYCfg<T, LB, RMAX>;
    auto kern = k_sep_xy<T, LB, RMAX>;
    if (C::SMEM > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaFuncSetAttribute");
    }
    dim3 grid(nitems, C::b / C::NSB, jobs.n * jobs.nf);
    kern<<<grid, 256, C::SMEM, s>>>(jobs, nbr, items, nr);
    return LGF_OK;
}

template <typename T, int LB>
lgf_status launch_xy_r(lgf_ctx *ctx, int rmax, int nitems, const SepJobs<T> &jobs, cudaStream_t s, const int *nbr,
                       const int *items, int nr)
{
    switch (rmax) {
    case 4: return launch_xy_m<T, LB, 4>(ctx, nitems, jobs, s, nbr, items, nr);
    case 8: return launch_xy_m<T, LB, 8>(ctx, nitems, jobs, s, nbr, items, nr);
    case 12: return launch_xy_m<T, LB, 12>(ctx, nitems, jobs, s, nbr, items, nr);
    default: return launch_xy_m<T, LB, 16>(ctx, nitems, jobs, s, nbr, items, nr);
    }
}

template <typename T, int LB, int AX, int RMAX>
lgf_status launch_m(lgf_ctx *ctx, int nout, const SepJobs<T> &jobs, cudaStream_t s, const int *nbr, int nr)
{
    using C = Cfg<T, LB, AX>;
    constexpr int b = 1 << LB, E = b + 2 * RMAX;
    constexpr size_t smem = sizeof(T) * (size_t)C::NS * b * E;
    auto kern = k_sep_win<T, LB, AX, RMAX>;
    // the z pass stages with bulk copies when every job's input is 16-byte
    // aligned (the copies' requirement; block and plane offsets keep it) and
    // the context has a device error word for the bounded waits
    bool aligned = AX == 2 && ctx != nullptr && ctx->err_dev != nullptr && ctx->opt_bulk;
    for (int i = 0; i < jobs.n; ++i)
        aligned = aligned && (reinterpret_cast<uintptr_t>(jobs.j[i].in) % 16 == 0) &&
                  ((jobs.j[i].in_stride * (int64_t)sizeof(T)) % 16 == 0);
    if constexpr (AX == 2) {
        if (aligned) {
            auto kb = k_sep_z_bulk<T, LB, RMAX>;
            const size_t sm2 = 2 * smem;
            cudaError_t e = cudaFuncSetAttribute(kb, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2);
            int per_sm = 0;
            if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kb, C::THREADS, sm2);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "bulk z pass set-up");
            int nsm = 0;
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device);
            const int64_t nitems = (int64_t)nout * (b / C::NS) * jobs.n * jobs.nf;
            const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(nitems, (int64_t)std::max(1, per_sm) * nsm));
            kb<<<grid, C::THREADS, sm2, s>>>(jobs, nbr, nr, nout, ctx->err_dev);
            return LGF_OK;
        }
    }
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaFuncSetAttribute");
    }
    dim3 grid(nout, b / C::NS, jobs.n * jobs.nf);
    kern<<<grid, C::THREADS, smem, s>>>(jobs, nbr, nr);
    return LGF_OK;
}

// Ragged launches: every job field but cta0 set; sent in tables of
// kSepRagJobs, each table by launch(grid.x, table).
template <typename T, class Launch>
lgf_status rag_send_sep(lgf_ctx *ctx, SepRagJob<T> *jobs, int n, Launch launch)
{
    static_assert(sizeof(SepRag<T>) <= 32000, "job table beyond the kernel parameter space");
    for (int c0 = 0; c0 < n;) {
        SepRag<T> t;
        t.n = 0;
        int64_t ctas = 0;
        for (; c0 < n && t.n < kSepRagJobs; ++c0) {
            SepRagJob<T> &j = jobs[c0];
            const int64_t nc = (int64_t)j.nitems * j.nf;
            if (nc <= 0) continue;
            j.cta0 = (int)ctas;
            t.j[t.n++] = j;
            ctas += nc;
        }
        if (t.n == 0) continue;
        if (ctas > 0x7fffffff) return fail(ctx, LGF_EUNSUPPORTED, "ragged integrating factor: too many CTAs");
        launch((unsigned)ctas, t);
    }
    return LGF_OK;
}

template <typename T, int LB, int RMAX>
lgf_status launch_xy_rag_m(lgf_ctx *ctx, SepRagJob<T> *jobs, int n, cudaStream_t s)
{
    using C = XYCfg<T, LB, RMAX>;
    auto kern = k_sep_xy<T, LB, RMAX, SepRag<T>>;
    if (C::SMEM > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaFuncSetAttribute");
    }
    return rag_send_sep<T>(ctx, jobs, n, [&](unsigned gx, const SepRag<T> &t) {
        kern<<<dim3(gx, C::b / C::NSB, 1), 256, C::SMEM, s>>>(t, nullptr, nullptr, 0);
    });
}

template <typename T, int LB, int RMAX>
lgf_status launch_z_rag_m(lgf_ctx *ctx, SepRagJob<T> *jobs, int n, cudaStream_t s)
{
    using C = Cfg<T, LB, 2>;
    constexpr int b = 1 << LB, E = b + 2 * RMAX;
    constexpr size_t smem = sizeof(T) * (size_t)C::NS * b * E;
    auto kern = k_sep_win<T, LB, 2, RMAX, SepRag<T>>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaFuncSetAttribute");
    }
    return rag_send_sep<T>(ctx, jobs, n, [&](unsigned gx, const SepRag<T> &t) {
        kern<<<dim3(gx, b / C::NS, 1), C::THREADS, smem, s>>>(t, nullptr, 0);
    });
}

template <typename T, int LB, int AX>
lgf_status launch_r(lgf_ctx *ctx, int rmax, int nout, const SepJobs<T> &jobs, cudaStream_t s, const int *nbr, int nr)
{
    switch (rmax) {
    case 4: return launch_m<T, LB, AX, 4>(ctx, nout, jobs, s, nbr, nr);
    case 8: return launch_m<T, LB, AX, 8>(ctx, nout, jobs, s, nbr, nr);
    case 12:
        if constexpr (AX == 2) return launch_m<T, LB, AX, 12>(ctx, nout, jobs, s, nbr, nr);
        return launch_m<T, LB, AX, 16>(ctx, nout, jobs, s, nbr, nr);
    default: return launch_m<T, LB, AX, 16>(ctx, nout, jobs, s, nbr, nr);
    }
}

}  // namespace win

// Window bound for a radius: the smallest of 4, 8, 12, 16 that covers it (0: none).
inline int window_class(int R) { return R <= 4 ? 4 : R <= 8 ? 8 : R <= 12 ? 12 : R <= 16 ? 16 : 0; }

// Largest radius of a job list, rounded up to a window bound (0: none fits).
template <typename T>
inline int window_rmax(const SepJobs<T> &jobs, int b, int nr)
{
    int R = 0;
    for (int i = 0; i < jobs.n; ++i) R = jobs.j[i].R > R ? jobs.j[i].R : R;
    const int rmax = window_class(R);
    if (rmax == 0 || rmax > nr * b || (b != 8 && b != 16 && b != 32)) return 0;
    return rmax;
}

// Fused x+y pass (S -> Y2 with the (2nr+1)^2 xy neighbour table, over the
// single and y-paired output items) for a job list; *done tells whether the
// window kernels applied.
template <typename T>
lgf_status launch_sep_xy(lgf_ctx *ctx, int b, int nitems, const SepJobs<T> &jobs, cudaStream_t s, const int *nbr,
                         const int *items, int nr, bool *done)
{
    const int rmax = window_rmax(jobs, b, nr);
    *done = rmax > 0;
    if (!*done) return LGF_OK;
    switch (b) {
    case 8: return win::launch_xy_r<T, 3>(ctx, rmax, nitems, jobs, s, nbr, items, nr);
    case 16: return win::launch_xy_r<T, 4>(ctx, rmax, nitems, jobs, s, nbr, items, nr);
    default: return win::launch_xy_r<T, 5>(ctx, rmax, nitems, jobs, s, nbr, items, nr);
    }
}

// Single-axis window pass for a job list.
template <typename T>
lgf_status launch_sep_window(lgf_ctx *ctx, int ax, int b, int nout, const SepJobs<T> &jobs, cudaStream_t s,
                             const int *nbr, int nr, bool *done)
{
    const int rmax = window_rmax(jobs, b, nr);
    *done = rmax > 0;
    if (!*done) return LGF_OK;
    const int lb = b == 8 ? 3 : b == 16 ? 4 : 5;
#define LGF_WIN_AX(AXV)                                                                           \
    switch (lb) {                                                                                 \
    case 3: return win::launch_r<T, 3, AXV>(ctx, rmax, nout, jobs, s, nbr, nr);                   \
    case 4: return win::launch_r<T, 4, AXV>(ctx, rmax, nout, jobs, s, nbr, nr);                   \
    default: return win::launch_r<T, 5, AXV>(ctx, rmax, nout, jobs, s, nbr, nr);                  \
    }
    if (ax == 0) {
        LGF_WIN_AX(0)
    } else if (ax == 1) {
        LGF_WIN_AX(1)
    } else {
        LGF_WIN_AX(2)
    }
#undef LGF_WIN_AX
}

// Ragged fused x+y pass (xy = true) or z pass over jobs of several plans
// that share the block edge b and the window bound rmax (4, 8, 12, 16, at
// most nr * b of every job's plan).
template <typename T>
lgf_status launch_sep_rag(lgf_ctx *ctx, bool xy, int b, int rmax, SepRagJob<T> *jobs, int n, cudaStream_t s)
{
#define LGF_RAG_R(LBV)                                                                                   \
    switch (rmax) {                                                                                      \
    case 4: return xy ? win::launch_xy_rag_m<T, LBV, 4>(ctx, jobs, n, s) : win::launch_z_rag_m<T, LBV, 4>(ctx, jobs, n, s);     \
    case 8: return xy ? win::launch_xy_rag_m<T, LBV, 8>(ctx, jobs, n, s) : win::launch_z_rag_m<T, LBV, 8>(ctx, jobs, n, s);     \
    case 12: return xy ? win::launch_xy_rag_m<T, LBV, 12>(ctx, jobs, n, s) : win::launch_z_rag_m<T, LBV, 12>(ctx, jobs, n, s);  \
    default: return xy ? win::launch_xy_rag_m<T, LBV, 16>(ctx, jobs, n, s) : win::launch_z_rag_m<T, LBV, 16>(ctx, jobs, n, s);  \
    }
    switch (b) {
    case 8: LGF_RAG_R(3)
    case 16: LGF_RAG_R(4)
    default: LGF_RAG_R(5)
    }
#undef LGF_RAG_R
}

}  // namespace lgf
