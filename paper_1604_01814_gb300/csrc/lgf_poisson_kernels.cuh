// Pass kernels of the Poisson apply, specialised on the transform length.
//
// Every length M = 2^k, 3 * 2^k or 5 * 2^k (32..4096) has a fixed plan of two
// or three DIF stages (radix <= 20), see Plan below.  A line (a column of W adjacent kx
// values, or one packed pair of x rows) is handled by TPC threads:
//   - the first forward stage loads its operands straight from global memory
//     into registers (all loads of a thread in flight together), does the
//     butterflies and writes the stage result to shared memory;
//   - the middle stage (three-stage plans only) works in shared memory;
//   - the last forward stage reads shared memory into registers; its outputs
//     are final spectrum values, stored straight to global memory (y pass) or
//     multiplied by the kernel spectrum and sent straight into the first
//     inverse stage (z pass).
// The inverse sweep mirrors this (adjoint stages, conjugate twiddles).  One
// shared-memory transpose per stage boundary, one __syncthreads per boundary.
#pragma once
#include <type_traits>

#include "lgf_internal.cuh"

namespace lgf {
namespace pk {

constexpr int cgcd(int a, int b) { return b == 0 ? a : cgcd(b, a % b); }

// Stage plan of a length M (2^k, 3 * 2^k or 5 * 2^k, 32..4096): a first stage
// of radix R0, for M >= 512 and most 3 * 2^k, 5 * 2^k a middle stage of radix
// R1 (R0, R1 powers of two; the middle stage keeps more threads per line),
// and a last stage of radix RL (16, 8 or 4; 12 when M = 3 * 2^k, 20 when
// M = 5 * 2^k).  Every stage
// before the last splits off a power of two, so its twiddle index stays
// j q M/N with M/N a power of two.  TPC threads share a line: the greatest
// common divisor of the stages' group counts, so that every thread owns a
// whole number of groups in every stage.
template <int ML>
struct Plan {
    static constexpr int M = ML;
    static constexpr int R0 = M == 80 || M == 96 || M == 192 || M == 320 ? 4
                            : M == 32 || M == 64 || M == 160 || M == 384 || M == 512 || M == 640 || M == 768 ||
                                      M == 1280
                                  ? 8
                                  : 16;
    static constexpr int R1 = M == 96 ? 2
                            : M == 192 || M == 320 || M == 384 || M == 640 ? 4
                            : M == 512 || M == 768 || M == 1024 || M == 1280 || M == 1536 || M == 2560 ? 8
                            : M == 2048 || M == 3072 || M == 4096 ? 16 : 1;
    static constexpr int RL = M / (R0 * R1);
    static constexpr int NST = R1 > 1 ? 3 : 2;
    static constexpr int N1 = M / R0;                             // sub-problem size entering stage 1
    static constexpr int G0 = M / R0, G1 = M / R1, GL = M / RL;   // groups per stage
    static constexpr int TPC = cgcd(cgcd(G0, NST == 3 ? G1 : G0), GL);
    static_assert(R0 * R1 * RL == M && RL <= 20 && RL >= 4, "plan must cover the length");
    static_assert(G0 % TPC == 0 && G1 % TPC == 0 && GL % TPC == 0, "whole groups per thread");
};

// Position of frequency k after the forward sweep, and back: position
// q0 M/R0 + q1 RL + qL holds frequency q0 + R0 q1 + R0 R1 qL.
template <int ML>
__device__ __forceinline__ int pos_of(int k)
{
    using P = Plan<ML>;
    const int q0 = k % P::R0;
    k /= P::R0;
    const int q1 = k % P::R1;
    const int qL = k / P::R1;
    return q0 * (ML / P::R0) + q1 * P::RL + qL;
}

template <int ML>
__device__ __forceinline__ int freq_of(int pos)
{
    using P = Plan<ML>;
    const int q0 = pos / (ML / P::R0);
    const int r0 = pos % (ML / P::R0);
    return q0 + P::R0 * (r0 / P::RL) + P::R0 * P::R1 * (r0 % P::RL);
}

// Forward butterfly of one group of a stage that is not the last: DFT then
// twiddles w_N^{j q} = tw[j q TWS] (TWS = M/N).  HALF: the inputs
// a[R/2..R) are zero (not read).
template <int R, int TWS, bool HALF = false, typename T>
__device__ __forceinline__ void dif_group(Cx<T> *a, int j, const Cx<T> *tw)
{
    if constexpr (HALF)
        dft_half_in<R, -1, T>(a);
    else
        Dft<R, -1, T>::run(a);
#pragma unroll
    for (int q = 1; q < R; ++q) a[q] = cmul(a[q], tw[j * q * TWS]);
}

// A group whose only nonzero input is a[0] (the data of the line end before
// M/R): the DFT gives a[0] at every output, so the stage is the twiddles.
template <int R, int TWS, typename T>
__device__ __forceinline__ void dif_group_single(Cx<T> *a, int j, const Cx<T> *tw)
{
#pragma unroll
    for (int q = 1; q < R; ++q) a[q] = cmul(a[0], tw[j * q * TWS]);
}

// Its adjoint.  HALF: only the outputs a[0..R/2) are formed.
template <int R, int TWS, bool HALF = false, typename T>
__device__ __forceinline__ void dit_group(Cx<T> *a, int j, const Cx<T> *tw)
{
#pragma unroll
    for (int q = 1; q < R; ++q) a[q] = cmulc(a[q], tw[j * q * TWS]);
    if constexpr (HALF)
        dft_half_out<R, 1, T>(a);
    else
        Dft<R, 1, T>::run(a);
}

// Middle stage (three-stage plans): shared memory to shared memory.
template <int ML, int DIR, typename T, class Addr>
__device__ __forceinline__ void middle_stage(Cx<T> *s, const Addr &ad, int line, int t, const Cx<T> *tw)
{
    using P = Plan<ML>;
    if constexpr (P::NST == 3) {
        constexpr int N = P::N1, R = P::R1, NP = N / R;
#pragma unroll
        for (int g = t; g < P::G1; g += P::TPC) {
            const int sub = g / NP, j = g % NP, o = sub * N;
            Cx<T> a[R];
            if (DIR < 0) {
#pragma unroll
                for (int p = 0; p < R; ++p) a[p] = s[ad(line, o + j + p * NP)];
                dif_group<R, P::R0>(a, j, tw);
#pragma unroll
                for (int q = 0; q < R; ++q) s[ad(line, o + q * NP + j)] = a[q];
            } else {
#pragma unroll
                for (int q = 0; q < R; ++q) a[q] = s[ad(line, o + q * NP + j)];
                dit_group<R, P::R0>(a, j, tw);
#pragma unroll
                for (int p = 0; p < R; ++p) s[ad(line, o + j + p * NP)] = a[p];
            }
        }
    }
}

// Shared-memory layouts.
struct ColAddrW {   // element m of column w: m * W + w
    int W;
    __device__ __forceinline__ int operator()(int w, int m) const { return m * W + w; }
};
// Row-pass layout of element m of line l, chosen per length so that the
// 8-byte accesses of every stage (first-stage stores at q G0 + g, middle
// stage, last-stage groups at g RL + q, the Hermitian packing at the
// digit-reversed positions) spread over the 16 bank pairs of a half-warp:
// either padding, m + (m >> A) + (m >> B), or a swizzle of the low four
// bits, m ^ (((m >> A) ^ (m >> B)) & 15) (a permutation inside each aligned
// run of 16).  The (kind, A, B) per length came from a model of those
// accesses that counts shared-memory wavefronts per half-warp; it cuts them
// from 2.3x to 1.5x the conflict-free count on average.  B = 0: no second term.
template <int ML>
struct RowAddr {
    static constexpr int KIND = ML == 512 || ML == 768 || ML == 1280 || ML == 1536 || ML == 2560 || ML == 3072 ||
                                        ML == 4096
                                    ? 1
                                    : 0;   // 0 padding, 1 swizzle
    static constexpr int A = ML == 32 || ML == 96 || ML == 160 || ML == 256 || ML == 512 || ML == 2048 || ML == 4096
                                 ? 4
                             : ML == 80 || ML == 1024 ? 3
                             : ML == 768 || ML == 1536 || ML == 2560 || ML == 3072 ? 5
                             : ML == 1280 ? 6
                                          : 2;
    static constexpr int B = ML == 80 || ML == 96 || ML == 512 || ML == 3072 ? 6
                             : ML == 160 || ML == 1024 ? 7
                             : ML == 2048 || ML == 4096 ? 8
                                                        : 0;
    // line stride: the largest index of a line plus one, plus one to offset lines
    static constexpr int LD = (KIND == 0 ? ML + (ML >> A) + (B ? (ML >> B) : 0) : ML) + 1;
    __device__ __forceinline__ int operator()(int l, int m) const
    {
        if constexpr (KIND == 0)
            return l * LD + m + (m >> A) + (B ? (m >> B) : 0);
        else
            return l * LD + (m ^ (((m >> A) ^ (B ? (m >> B) : 0)) & 15));
    }
};

template <typename T>
__device__ __forceinline__ void load_twiddles(Cx<T> *tw, const Cx<T> *__restrict__ twg, int M)
{
    for (int i = threadIdx.x; i < M; i += blockDim.x) tw[i] = twg[i];
}

// ---------------------------------------------------------------------------
// Column passes.  Data in global memory: rows of K complex values (kx), row
// `r` of the current column set at base + r * rs.  Most CTAs own W adjacent
// kx of one plane; the K mod W leftover kx of every plane (the Nyquist column
// kx = M/2 when K = M/2 + 1) are packed W (plane, kx) pairs per CTA, so no
// CTA runs mostly empty columns.  Those CTAs come first in the grid: their
// scattered accesses are slower, and they then overlap the rest instead of
// trailing it.
// ---------------------------------------------------------------------------
// Row-block occupancy for the y-forward pass: row y of plane pl (both
// relative to the source region) holds data unless its (z, y) row block has
// no block along x (the x-forward pass then skipped it); bit y >> lb of
// mask[pl >> lb].
struct RowFlags {
    const unsigned long long *mask = nullptr;   // nullptr: every row holds data
    int lb = 0;
    __device__ __forceinline__ unsigned long long plane(int pl) const { return mask ? mask[pl >> lb] : ~0ull; }
    // only with a mask: every region then has at most 64 row blocks, so the
    // shift stays below 64
    __device__ __forceinline__ bool row(unsigned long long pm, int y) const { return (pm >> (y >> lb)) & 1ull; }
};

template <int W>
__host__ __device__ __forceinline__ int col_ctas(int K, int nplanes)
{
    const int nfull = K / W, rem = K - nfull * W;
    return nfull * nplanes + (rem * nplanes + W - 1) / W;
}

// Column (kx, plane) of lane w of CTA `cta`; false for padding lanes of the
// last packed CTA (kx, plane set to 0 so that addresses stay in range).
template <int W>
__device__ __forceinline__ bool column_of(int cta, int w, int K, int nplanes, int &kx, int &pl)
{
    const int nfull = K / W, rem = K - nfull * W;
    const int ntail = (rem * nplanes + W - 1) / W;
    if (cta >= ntail) {
        const int c = cta - ntail;
        pl = c / nfull;
        kx = (c - pl * nfull) * W + w;
        return true;
    }
    const int i = cta * W + w;
    pl = i / rem;
    kx = nfull * W + (i - pl * rem);
    if (pl < nplanes) return true;
    pl = 0;
    kx = 0;
    return false;
}

// Forward along the column: rows [lo, lo + n) hold data (row m at
// in + (m - lo) * rs), others are zero; the spectrum (natural order) goes to
// out + k * os.  Used by the y pass and by the spectrum build's z pass.
// HALF: the data rows lie in [0, M/2), which holds for every pass of an
// apply (the transform length is at least twice the box), so the first
// stage's upper inputs are zero at compile time and its first butterfly
// layer is skipped.  Row addresses advance by a fixed stride per radix digit
// (the last stage's digit is the top digit of the frequency).
// (The body of every pass kernel takes its CTA coordinates as arguments: the
// kernels below run it at their own blockIdx, the ragged kernels at the
// coordinates of a CTA inside one job of a job table.)
template <typename T, int ML, int W, bool HALF>
__device__ __forceinline__ void col_forward_body(int bx, int by, const Cx<T> *__restrict__ in, Cx<T> *__restrict__ out,
                                                 int K, int nplanes, int lo, int n, int64_t rs, int64_t os,
                                                 int64_t in_plane, int64_t out_plane, int64_t in_field,
                                                 int64_t out_field, const Cx<T> *__restrict__ twg, RowFlags rf)
{
    using P = Plan<ML>;
    constexpr int M = P::M;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx<T> *tw = reinterpret_cast<Cx<T> *>(smem_raw);
    Cx<T> *s = tw + M;
    load_twiddles(tw, twg, M);
    const int w = threadIdx.x % W, t = threadIdx.x / W;
    int kx, pl;
    const bool live = column_of<W>(bx, w, K, nplanes, kx, pl);
    const Cx<T> *ib = in + by * in_field + pl * in_plane + kx;
    Cx<T> *ob = out + by * out_field + pl * out_plane + kx;
    const ColAddrW ad{W};
    constexpr int R0 = P::R0;
    constexpr int NG0 = P::G0 / P::TPC;
    constexpr int NP = HALF ? R0 / 2 : R0;
    const int64_t istep = (int64_t)P::G0 * rs;
    Cx<T> a[NG0][R0];
    if (rf.mask == nullptr) {   // every row holds data (uniform branch)
#pragma unroll
        for (int i = 0; i < NG0; ++i) {
            const int r = t + i * P::TPC - lo;   // data row of digit p = 0
            int64_t off = (int64_t)r * rs;
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const bool ok = live && (unsigned)(r + p * P::G0) < (unsigned)n;
                a[i][p] = ok ? ib[off] : Cx<T>{T(0), T(0)};
                off += istep;
            }
        }
    } else {
        const unsigned long long pm = rf.plane(pl);
#pragma unroll
        for (int i = 0; i < NG0; ++i) {
            const int r = t + i * P::TPC - lo;
            int64_t off = (int64_t)r * rs;
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const int y = r + p * P::G0;
                const bool ok = live && (unsigned)y < (unsigned)n && rf.row(pm, y);
                a[i][p] = ok ? ib[off] : Cx<T>{T(0), T(0)};
                off += istep;
            }
        }
    }
    __syncthreads();   // twiddles
#pragma unroll
    for (int i = 0; i < NG0; ++i) {
        const int g = t + i * P::TPC;
        dif_group<P::R0, 1, HALF>(a[i], g, tw);
#pragma unroll
        for (int q = 0; q < R0; ++q) s[ad(w, q * P::G0 + g)] = a[i][q];
    }
    __syncthreads();
    if constexpr (P::NST == 3) {
        middle_stage<ML, -1>(s, ad, w, t, tw);
        __syncthreads();
    }
    constexpr int RL = P::RL;
    const int64_t ostep = (int64_t)(M / RL) * os;
#pragma unroll
    for (int g = t; g < P::GL; g += P::TPC) {
        Cx<T> c[RL];
#pragma unroll
        for (int q = 0; q < RL; ++q) c[q] = s[ad(w, (g * P::RL) + q)];
        Dft<RL, -1, T>::run(c);
        if (live) {
            int64_t off = (int64_t)freq_of<ML>(g * P::RL) * os;
#pragma unroll
            for (int q = 0; q < RL; ++q) {
                ob[off] = c[q];
                off += ostep;
            }
        }
    }
}

template <typename T, int ML, int W, bool HALF>
__global__ void __launch_bounds__(W * Plan<ML>::TPC) k_col_forward(const Cx<T> *__restrict__ in, Cx<T> *__restrict__ out,
                                                                     int K, int nplanes, int lo, int n, int64_t rs,
                                                                     int64_t os, int64_t in_plane, int64_t out_plane,
                                                                     int64_t in_field, int64_t out_field,
                                                                     const Cx<T> *__restrict__ twg, RowFlags rf)
{
    col_forward_body<T, ML, W, HALF>(blockIdx.x, blockIdx.y, in, out, K, nplanes, lo, n, rs, os, in_plane, out_plane,
                                     in_field, out_field, twg, rf);
}

// Inverse along the column: spectrum rows (natural order, row k at
// in + k * rs) in; rows [lo, lo + n) of the result written to
// out + (m - lo) * os.  HALF_OUT: the written rows lie in [0, M/2), so the
// last stage forms only the lower half of its outputs (otherwise, the
// shifted y window with targets past M/2, all of them).
template <typename T, int ML, int W, bool HALF_OUT>
__device__ __forceinline__ void col_inverse_body(int bx, int by, const Cx<T> *__restrict__ in, Cx<T> *__restrict__ out,
                                                 int K, int nplanes, int lo, int n, int64_t rs, int64_t os,
                                                 int64_t in_plane, int64_t out_plane, int64_t in_field,
                                                 int64_t out_field, const Cx<T> *__restrict__ twg)
{
    using P = Plan<ML>;
    constexpr int M = P::M;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx<T> *tw = reinterpret_cast<Cx<T> *>(smem_raw);
    Cx<T> *s = tw + M;
    load_twiddles(tw, twg, M);
    const int w = threadIdx.x % W, t = threadIdx.x / W;
    int kx, pl;
    const bool live = column_of<W>(bx, w, K, nplanes, kx, pl);
    const Cx<T> *ib = in + by * in_field + pl * in_plane + kx;
    Cx<T> *ob = out + by * out_field + pl * out_plane + kx;
    const ColAddrW ad{W};
    constexpr int RL = P::RL;
    constexpr int NGL = P::GL / P::TPC;
    const int64_t istep = (int64_t)(M / RL) * rs;
    Cx<T> c[NGL][RL];
#pragma unroll
    for (int i = 0; i < NGL; ++i) {
        const int g = t + i * P::TPC;
        int64_t off = (int64_t)freq_of<ML>(g * P::RL) * rs;
#pragma unroll
        for (int q = 0; q < RL; ++q) {
            c[i][q] = live ? ib[off] : Cx<T>{T(0), T(0)};
            off += istep;
        }
    }
#pragma unroll
    for (int i = 0; i < NGL; ++i) {
        const int g = t + i * P::TPC;
        Dft<RL, 1, T>::run(c[i]);
#pragma unroll
        for (int q = 0; q < RL; ++q) s[ad(w, (g * P::RL) + q)] = c[i][q];
    }
    __syncthreads();
    if constexpr (P::NST == 3) {
        middle_stage<ML, 1>(s, ad, w, t, tw);
        __syncthreads();
    }
    constexpr int R0 = P::R0;
    constexpr int NOUT = HALF_OUT ? R0 / 2 : R0;
    const int64_t ostep = (int64_t)P::G0 * os;
#pragma unroll
    for (int g = t; g < P::G0; g += P::TPC) {
        Cx<T> a[R0];
#pragma unroll
        for (int q = 0; q < R0; ++q) a[q] = s[ad(w, q * P::G0 + g)];
        dit_group<P::R0, 1, HALF_OUT>(a, g, tw);
        if (live) {
            const int r = g - lo;
            int64_t off = (int64_t)r * os;
#pragma unroll
            for (int p = 0; p < NOUT; ++p) {
                if ((unsigned)(r + p * P::G0) < (unsigned)n) ob[off] = a[p];
                off += ostep;
            }
        }
    }
}

template <typename T, int ML, int W, bool HALF_OUT>
__global__ void __launch_bounds__(W * Plan<ML>::TPC) k_col_inverse(const Cx<T> *__restrict__ in, Cx<T> *__restrict__ out,
                                                                     int K, int nplanes, int lo, int n, int64_t rs,
                                                                     int64_t os, int64_t in_plane, int64_t out_plane,
                                                                     int64_t in_field, int64_t out_field,
                                                                     const Cx<T> *__restrict__ twg)
{
    col_inverse_body<T, ML, W, HALF_OUT>(blockIdx.x, blockIdx.y, in, out, K, nplanes, lo, n, rs, os, in_plane,
                                         out_plane, in_field, out_field, twg);
}

// z pass: forward along z over the source planes, times the real even kernel
// spectrum, inverse along z, target planes written back in place.  The field
// is the fastest part of the CTA index, so the CTAs of every field of one
// column set run back to back and read that part of the spectrum from L2:
// for big boxes the spectrum is larger than L2.  Source and target planes
// lie in [0, M/2): the first stage skips its zero upper inputs and the last
// stage forms only its lower outputs.
// Resident CTAs per SM that the register allocation must allow (FP32 at the
// lengths 256 (32 warps), 320, 384 and 512 (24 warps) and the long mixed
// lengths (2 CTAs); no spills).
// ZV = 1 (the tuner's alternative, FP32 only) asks for one more resident CTA
// per SM than the default, i.e. a tighter register cap (where the default
// leaves the choice to the compiler: 4 up to length 192, 3 above).
template <typename T, int ML, int ZV = 0>
struct ConvOcc {
    static constexpr int base = sizeof(T) == 4 ? (ML == 256 ? 4 : ML == 320 || ML == 384 || ML == 512 ? 3 : ML == 640 || ML == 1536 || ML == 2560 || ML == 3072 ? 2 : 1) : 1;
    static constexpr int value = ZV == 0 ? base : (base == 1 ? (ML <= 192 ? 4 : 3) : base + 1);
};

// SPEC: 0 the real spectrum of the even embedding ([kz][ky <= My/2][kx]);
// 1 the complex spectrum of the shifted x window (same layout); 2 the complex
// spectrum of the shifted y window ([kz][ky < My][kx], no mirror in ky).
template <typename T, int ML, int W, int SPEC>
__device__ __forceinline__ void col_convolve_body(int bx, int nf, Cx<T> *__restrict__ B, const void *__restrict__ specv,
                                                  int K, int My, int s0, int ns, int t0, int nt, int64_t field,
                                                  const Cx<T> *__restrict__ twg)
{
    constexpr bool CPLX = SPEC > 0;
    using SpecT = typename std::conditional<CPLX, Cx<T>, T>::type;
    const SpecT *__restrict__ spec = reinterpret_cast<const SpecT *>(specv);
    using P = Plan<ML>;
    constexpr int M = P::M;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx<T> *tw = reinterpret_cast<Cx<T> *>(smem_raw);
    Cx<T> *s = tw + M;
    load_twiddles(tw, twg, M);
    const int w = threadIdx.x % W, t = threadIdx.x / W;
    int kx, ky;
    const int field_i = bx % nf;
    const bool live = column_of<W>(bx / nf, w, K, My, kx, ky);
    const int64_t plane = (int64_t)My * K;
    Cx<T> *bb = B + field_i * field + (int64_t)ky * K + kx;
    const ColAddrW ad{W};
    constexpr int R0 = P::R0;
    constexpr int NG0 = P::G0 / P::TPC;
    const int64_t step0 = (int64_t)P::G0 * plane;
    {
        Cx<T> a[NG0][R0];
#pragma unroll
        for (int i = 0; i < NG0; ++i) {
            const int r = t + i * P::TPC - s0;
            int64_t off = (int64_t)r * plane;
#pragma unroll
            for (int p = 0; p < R0 / 2; ++p) {
                const bool ok = live && (unsigned)(r + p * P::G0) < (unsigned)ns;
                a[i][p] = ok ? bb[off] : Cx<T>{T(0), T(0)};
                off += step0;
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < NG0; ++i) {
            const int g = t + i * P::TPC;
            dif_group<P::R0, 1, true>(a[i], g, tw);
#pragma unroll
            for (int q = 0; q < R0; ++q) s[ad(w, q * P::G0 + g)] = a[i][q];
        }
    }
    __syncthreads();
    if constexpr (P::NST == 3) {
        middle_stage<ML, -1>(s, ad, w, t, tw);
        __syncthreads();
    }
    constexpr int RL = P::RL;
    constexpr int S = M / RL;   // frequency step of the last stage's digit
    const int Khy = SPEC == 2 ? My : My / 2 + 1;
    const int kyr = SPEC == 2 ? ky : (ky <= My - ky ? ky : My - ky);
    const SpecT *sp = spec + (int64_t)kyr * K + kx;
    const int64_t sp_plane = (int64_t)Khy * K;
#pragma unroll
    for (int g = t; g < P::GL; g += P::TPC) {
        // frequency of digit q: kb + q S; its mirror M - kb - q S once past M/2
        const int kb = freq_of<ML>(g * P::RL);
        const SpecT *spl = sp + (int64_t)kb * sp_plane;
        const SpecT *sph = sp + (int64_t)(M - kb) * sp_plane;
        Cx<T> c[RL];
        SpecT gk[RL];
#pragma unroll
        for (int q = 0; q < RL; ++q) {
            gk[q] = q < RL / 2 ? spl[(int64_t)(q * S) * sp_plane] : sph[-(int64_t)(q * S) * sp_plane];
            c[q] = s[ad(w, (g * P::RL) + q)];
        }
        Dft<RL, -1, T>::run(c);
#pragma unroll
        for (int q = 0; q < RL; ++q) {
            if constexpr (CPLX) {
                c[q] = cmul(c[q], gk[q]);
            } else {
                c[q].x *= gk[q];
                c[q].y *= gk[q];
            }
        }
        Dft<RL, 1, T>::run(c);
#pragma unroll
        for (int q = 0; q < RL; ++q) s[ad(w, (g * P::RL) + q)] = c[q];
    }
    __syncthreads();
    if constexpr (P::NST == 3) {
        middle_stage<ML, 1>(s, ad, w, t, tw);
        __syncthreads();
    }
    const int64_t step1 = (int64_t)P::G0 * plane;
#pragma unroll
    for (int g = t; g < P::G0; g += P::TPC) {
        Cx<T> a[R0];
#pragma unroll
        for (int q = 0; q < R0; ++q) a[q] = s[ad(w, q * P::G0 + g)];
        dit_group<P::R0, 1, true>(a, g, tw);
        if (live) {
            const int r = g - t0;
            int64_t off = (int64_t)r * plane;
#pragma unroll
            for (int p = 0; p < R0 / 2; ++p) {
                if ((unsigned)(r + p * P::G0) < (unsigned)nt) bb[off] = a[p];
                off += step1;
            }
        }
    }
}

template <typename T, int ML, int W, int SPEC, int ZV>
__global__ void __launch_bounds__(W * Plan<ML>::TPC, ConvOcc<T, ML, ZV>::value) k_col_convolve(Cx<T> *__restrict__ B, const void *__restrict__ specv,
                                                                      int K, int My, int s0, int ns, int t0, int nt,
                                                                      int64_t field, const Cx<T> *__restrict__ twg)
{
    col_convolve_body<T, ML, W, SPEC>(blockIdx.x, gridDim.x / col_ctas<W>(K, My), B, specv, K, My, s0, ns, t0, nt,
                                      field, twg);
}

// ---------------------------------------------------------------------------
// Row passes along x (real <-> half complex), two real rows per complex line.
// ---------------------------------------------------------------------------
// Forward: rows (y, y+1) of source plane z, x in [s0x, s0x + Lsx), from the
// block layout (HALF: the apply, where the row lies in [0, M/2) so the first
// stage's upper inputs are zero at compile time) or from a dense box with row
// length dense_ld (the spectrum build, full rows).
template <typename T, int ML, int LPC, bool HALF>
__device__ __forceinline__ void row_forward_body(int bx, int by, const T *__restrict__ f, Cx<T> *__restrict__ A,
                                                 const PoissonGeom &g, const Cx<T> *__restrict__ twg, int npairs,
                                                 int lb, int dense_ld)
{
    using P = Plan<ML>;
    constexpr int M = P::M;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx<T> *tw = reinterpret_cast<Cx<T> *>(smem_raw);
    Cx<T> *s = tw + M;
    load_twiddles(tw, twg, M);
    const int t = threadIdx.x % P::TPC, l = threadIdx.x / P::TPC;
    const int pr = bx * LPC + l;
    const bool live = pr < npairs;
    const int hp = g.Ls[1] >> 1;
    const int zi = live ? pr / hp : 0, yi = live ? 2 * (pr - zi * hp) : 0;
    // a CTA whose lines all lie in row blocks without source blocks has
    // nothing to transform (the y pass does not read those rows)
    if (g.srcrow && !__syncthreads_or(live && ((g.srcrow[zi >> lb] >> (yi >> lb)) & 1ull))) return;
    const T *ff = f + by * g.fstride;
    const RowAddr<ML> ad{};
    constexpr int R0 = P::R0;
    constexpr int NG0 = P::G0 / P::TPC;
    Cx<T> a[NG0][R0];
    if constexpr (HALF) {
        // the block-map row and the in-block offset of rows (y, y+1) are
        // fixed per line; y is even and b >= 2, so both rows share a block
        const int bm = (1 << lb) - 1;
        const int *mrow = g.srcmap + ((zi >> lb) * g.nbs[1] + (yi >> lb)) * g.nbs[0];
        const int inner = (((zi & bm) << lb) + (yi & bm)) << lb;
#pragma unroll
        for (int i = 0; i < NG0; ++i) {
            const int xr = t + i * P::TPC - g.s0[0];
#pragma unroll
            for (int p = 0; p < R0 / 2; ++p) {
                const int x = xr + p * P::G0;
                Cx<T> v{T(0), T(0)};
                if (live && (unsigned)x < (unsigned)g.Ls[0]) {
                    const int bi = mrow[x >> lb];
                    if (bi >= 0) {
                        const T *q = ff + ((int64_t)bi << (3 * lb)) + inner + (x & bm);
                        v.x = q[0];
                        v.y = q[1 << lb];
                    }
                }
                a[i][p] = v;
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < NG0; ++i) {
            const int gg = t + i * P::TPC;
            const T *row = ff + ((int64_t)(g.s0[2] + zi) * g.M[1] + (g.s0[1] + yi)) * dense_ld;
#pragma unroll
            for (int p = 0; p < R0; ++p) {
                const int x = gg + p * P::G0;
                Cx<T> v{T(0), T(0)};
                if (live && x >= g.s0[0] && x < g.s0[0] + g.Ls[0]) {
                    v.x = row[x];
                    v.y = row[dense_ld + x];
                }
                a[i][p] = v;
            }
        }
    }
    __syncthreads();
    // source rows that end before M/R0 (a small body in a long box): one
    // nonzero input per first-stage group (uniform over the launch)
    const bool single = HALF && g.s0[0] + g.Ls[0] <= P::G0;
#pragma unroll
    for (int i = 0; i < NG0; ++i) {
        const int gg = t + i * P::TPC;
        if (single)
            dif_group_single<P::R0, 1>(a[i], gg, tw);
        else
            dif_group<P::R0, 1, HALF>(a[i], gg, tw);
#pragma unroll
        for (int q = 0; q < R0; ++q) s[ad(l, q * P::G0 + gg)] = a[i][q];
    }
    __syncthreads();
    if constexpr (P::NST == 3) {
        middle_stage<ML, -1>(s, ad, l, t, tw);
        __syncthreads();
    }
    constexpr int RL = P::RL;
#pragma unroll
    for (int gg = t; gg < P::GL; gg += P::TPC) {
        Cx<T> c[RL];
#pragma unroll
        for (int q = 0; q < RL; ++q) c[q] = s[ad(l, (gg * P::RL) + q)];
        Dft<RL, -1, T>::run(c);
#pragma unroll
        for (int q = 0; q < RL; ++q) s[ad(l, (gg * P::RL) + q)] = c[q];
    }
    __syncthreads();
    if (!live) return;
    const int K = g.Kx;
    Cx<T> *row = A + by * g.Astride + ((int64_t)zi * g.ldA_y + yi) * K;
    for (int k = t; k < K; k += P::TPC) {
        const Cx<T> zk = s[ad(l, pos_of<ML>(k))];
        const Cx<T> zm = s[ad(l, pos_of<ML>(k == 0 ? 0 : M - k))];
        row[k] = Cx<T>{T(0.5) * (zk.x + zm.x), T(0.5) * (zk.y - zm.y)};
        row[K + k] = Cx<T>{T(0.5) * (zk.y + zm.y), T(-0.5) * (zk.x - zm.x)};
    }
}

template <typename T, int ML, int LPC, bool HALF>
__global__ void __launch_bounds__(LPC * Plan<ML>::TPC) k_row_forward(const T *__restrict__ f, Cx<T> *__restrict__ A,
                                                                       PoissonGeom g, const Cx<T> *__restrict__ twg,
                                                                       int npairs, int lb, int dense_ld)
{
    row_forward_body<T, ML, LPC, HALF>(blockIdx.x, blockIdx.y, f, A, g, twg, npairs, lb, dense_ld);
}

// Inverse: rows (y, y+1) of target plane z from their half spectra; x in
// [t0x, t0x + Ltx) scaled by dx^2 and scattered to the target block layout.
// HALF_OUT: the target x lies in [0, M/2) (even embedding), so only the
// lower half of the last stage's outputs is formed; otherwise (the shifted x
// window, targets up to M) every output is.
// One line pair per slot l < LPC (thread t of TPC in it): rows (yi, yi+1)
// of target plane zi, their half spectra at row[0..K) and row[K..2K), in any
// memory; the Hermitian extension goes to s, the inverse sweep runs, and x in
// [t0x, t0x + Ltx) scaled by dx^2 is scattered to the target blocks of uu.
// tw holds the M twiddles in shared memory.  GUARD (the fused inverse, rows
// in shared memory): the CTA may have threads beyond the LPC slots, which
// take part in the barriers only.
template <typename T, int ML, int LPC, bool HALF_OUT, bool GUARD = false>
__device__ __forceinline__ void row_inverse_line(int t, int l, bool live, int zi, int yi,
                                                 const Cx<T> *__restrict__ row, T *__restrict__ uu,
                                                 const PoissonGeom &g, const Cx<T> *__restrict__ tw,
                                                 Cx<T> *__restrict__ s, int lb)
{
    using P = Plan<ML>;
    constexpr int M = P::M;
    const bool act = !GUARD || l < LPC;
    if (GUARD) live = live && act;
    const int K = g.Kx;
    const RowAddr<ML> ad{};
    // Hermitian extension of the two half spectra, packed as Z = G1 + i G2,
    // stored at the digit-reversed positions the inverse sweep expects.
    constexpr int NPT = M / P::TPC;
    if constexpr (GUARD) {
        // (row may lie in shared memory: each value is stored right after its
        // load, so no long run of loads is held in registers)
        if (act) {
#pragma unroll
            for (int i = 0; i < NPT; ++i) {
                const int k = t + i * P::TPC;
                const int kk = k <= M / 2 ? k : M - k;
                Cx<T> g1 = live ? row[kk] : Cx<T>{T(0), T(0)};
                Cx<T> g2 = live ? row[K + kk] : Cx<T>{T(0), T(0)};
                if (k == 0 || k == M / 2) {
                    g1.y = T(0);
                    g2.y = T(0);
                }
                s[ad(l, pos_of<ML>(k))] = k <= M / 2 ? Cx<T>{g1.x - g2.y, g1.y + g2.x} : Cx<T>{g1.x + g2.y, g2.x - g1.y};
            }
        }
    } else {
        Cx<T> g1[NPT], g2[NPT];
#pragma unroll
        for (int i = 0; i < NPT; ++i) {
            const int k = t + i * P::TPC;
            const int kk = k <= M / 2 ? k : M - k;
            g1[i] = live ? row[kk] : Cx<T>{T(0), T(0)};
            g2[i] = live ? row[K + kk] : Cx<T>{T(0), T(0)};
        }
#pragma unroll
        for (int i = 0; i < NPT; ++i) {
            const int k = t + i * P::TPC;
            Cx<T> v;
            if (k <= M / 2) {
                if (k == 0 || k == M / 2) {
                    g1[i].y = T(0);
                    g2[i].y = T(0);
                }
                v = {g1[i].x - g2[i].y, g1[i].y + g2[i].x};
            } else {
                v = {g1[i].x + g2[i].y, g2[i].x - g1[i].y};
            }
            s[ad(l, pos_of<ML>(k))] = v;
        }
    }
    __syncthreads();
    constexpr int RL = P::RL;
    if (act) {
#pragma unroll
        for (int gg = t; gg < P::GL; gg += P::TPC) {
            Cx<T> c[RL];
#pragma unroll
            for (int q = 0; q < RL; ++q) c[q] = s[ad(l, (gg * P::RL) + q)];
            Dft<RL, 1, T>::run(c);
#pragma unroll
            for (int q = 0; q < RL; ++q) s[ad(l, (gg * P::RL) + q)] = c[q];
        }
    }
    __syncthreads();
    if constexpr (P::NST == 3) {
        if (act) middle_stage<ML, 1>(s, ad, l, t, tw);
        __syncthreads();
    }
    if (!live) return;
    const T sc = T(g.scale);
    const int bm = g.b - 1;
    const int *mrow = g.tgtmap + ((zi >> lb) * g.nbt[1] + (yi >> lb)) * g.nbt[0];
    const int inner = (((zi & bm) << lb) + (yi & bm)) << lb;
    constexpr int R0 = P::R0;
    constexpr int NOUT = HALF_OUT ? R0 / 2 : R0;
#pragma unroll
    for (int gg = t; gg < P::G0; gg += P::TPC) {
        Cx<T> a[R0];
#pragma unroll
        for (int q = 0; q < R0; ++q) a[q] = s[ad(l, q * P::G0 + gg)];
        dit_group<P::R0, 1, HALF_OUT>(a, gg, tw);
        const int xr = gg - g.t0[0];
#pragma unroll
        for (int p = 0; p < NOUT; ++p) {
            const int xi = xr + p * P::G0;
            if ((unsigned)xi >= (unsigned)g.Lt[0]) continue;
            const int bi0 = mrow[xi >> lb];
            if (bi0 < 0) continue;
            T *q = uu + ((int64_t)bi0 << (3 * lb)) + inner + (xi & bm);
            q[0] = sc * a[p].x;
            q[1 << lb] = sc * a[p].y;   // row y + 1 of the same block (y is even, b >= 2)
        }
    }
}

template <typename T, int ML, int LPC, bool HALF_OUT>
__device__ __forceinline__ void row_inverse_body(int bx, int by, const Cx<T> *__restrict__ A, T *__restrict__ u,
                                                 const PoissonGeom &g, const Cx<T> *__restrict__ twg, int npairs,
                                                 int lb)
{
    using P = Plan<ML>;
    constexpr int M = P::M;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx<T> *tw = reinterpret_cast<Cx<T> *>(smem_raw);
    Cx<T> *s = tw + M;
    load_twiddles(tw, twg, M);
    const int t = threadIdx.x % P::TPC, l = threadIdx.x / P::TPC;
    const int pr = bx * LPC + l;
    const bool live = pr < npairs;
    const int hp = g.Lt[1] >> 1;
    const int zi = live ? pr / hp : 0, yi = live ? 2 * (pr - zi * hp) : 0;
    // a CTA whose lines all lie in row blocks without target blocks has
    // nothing to write
    if (g.tgtrow && !__syncthreads_or(live && ((g.tgtrow[zi >> lb] >> (yi >> lb)) & 1ull))) return;
    const Cx<T> *row = A + by * g.Astride + ((int64_t)zi * g.ldA_y + yi) * g.Kx;
    row_inverse_line<T, ML, LPC, HALF_OUT>(t, l, live, zi, yi, row, u + by * g.ustride, g, tw, s, lb);
}

template <typename T, int ML, int LPC, bool HALF_OUT>
__global__ void __launch_bounds__(LPC * Plan<ML>::TPC) k_row_inverse(const Cx<T> *__restrict__ A, T *__restrict__ u,
                                                                       PoissonGeom g, const Cx<T> *__restrict__ twg,
                                                                       int npairs, int lb)
{
    row_inverse_body<T, ML, LPC, HALF_OUT>(blockIdx.x, blockIdx.y, A, u, g, twg, npairs, lb);
}

// ---------------------------------------------------------------------------
// Ragged launches: one pass of many independent problems that share the
// transform length (and the kernel's compile-time variant) in one launch.
// The job table travels in the kernel's parameter space; job j owns the CTAs
// [cta0_j, cta0_{j+1}) of the one-dimensional grid, and every CTA finds its
// job by a binary search over cta0 (the same for all threads of a CTA), then
// runs the pass body at its coordinates inside that job.  No CTA waits on
// another, so problems of any size mix in one launch.
// ---------------------------------------------------------------------------
constexpr int kRagJobs = 64;   // jobs per launch (longer lists go in several launches)

template <class J>
struct RagTable {
    J j[kRagJobs];
    int n;
};

template <class J>
__device__ __forceinline__ const J &rag_job(const RagTable<J> &t)
{
    int lo = 0, hi = t.n - 1;
    const int c = blockIdx.x;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (t.j[mid].cta0 <= c) lo = mid;
        else hi = mid - 1;
    }
    return t.j[lo];
}

// x passes: in = f (forward) or A (inverse), out = A or u; CTAs (gx, nf).
template <typename T>
struct RowJob {
    PoissonGeom g;
    const void *in;
    void *out;
    const Cx<T> *tw;
    int npairs, lb, nf;
    int cta0, gx;
};
// y passes: the argument list of k_col_forward / k_col_inverse; CTAs (gx, nf).
template <typename T>
struct ColJob {
    const Cx<T> *in;
    Cx<T> *out;
    const Cx<T> *tw;
    RowFlags rf;
    int64_t rs, os, in_plane, out_plane, in_field, out_field;
    int K, nplanes, lo, n, nf;
    int cta0, gx;
};
// z pass: the argument list of k_col_convolve; CTAs nf * col_ctas.
template <typename T>
struct ConvJob {
    Cx<T> *B;
    const void *spec;
    const Cx<T> *tw;
    int64_t field;
    int K, My, s0, ns, t0, nt, nf;
    int cta0, gx;
};

template <typename T, int ML, int LPC, bool HALF>
__global__ void __launch_bounds__(LPC * Plan<ML>::TPC) k_row_forward_rag(const __grid_constant__ RagTable<RowJob<T>> t)
{
    const RowJob<T> &J = rag_job(t);
    const int c = (int)blockIdx.x - J.cta0;
    row_forward_body<T, ML, LPC, HALF>(c % J.gx, c / J.gx, (const T *)J.in, (Cx<T> *)J.out, J.g, J.tw, J.npairs, J.lb,
                                       0);
}

template <typename T, int ML, int LPC, bool HALF_OUT>
__global__ void __launch_bounds__(LPC * Plan<ML>::TPC) k_row_inverse_rag(const __grid_constant__ RagTable<RowJob<T>> t)
{
    const RowJob<T> &J = rag_job(t);
    const int c = (int)blockIdx.x - J.cta0;
    row_inverse_body<T, ML, LPC, HALF_OUT>(c % J.gx, c / J.gx, (const Cx<T> *)J.in, (T *)J.out, J.g, J.tw, J.npairs,
                                           J.lb);
}

template <typename T, int ML, int W>
__global__ void __launch_bounds__(W * Plan<ML>::TPC) k_col_forward_rag(const __grid_constant__ RagTable<ColJob<T>> t)
{
    const ColJob<T> &J = rag_job(t);
    const int c = (int)blockIdx.x - J.cta0;
    col_forward_body<T, ML, W, true>(c % J.gx, c / J.gx, J.in, J.out, J.K, J.nplanes, J.lo, J.n, J.rs, J.os,
                                     J.in_plane, J.out_plane, J.in_field, J.out_field, J.tw, J.rf);
}

template <typename T, int ML, int W, bool HALF_OUT>
__global__ void __launch_bounds__(W * Plan<ML>::TPC) k_col_inverse_rag(const __grid_constant__ RagTable<ColJob<T>> t)
{
    const ColJob<T> &J = rag_job(t);
    const int c = (int)blockIdx.x - J.cta0;
    col_inverse_body<T, ML, W, HALF_OUT>(c % J.gx, c / J.gx, J.in, J.out, J.K, J.nplanes, J.lo, J.n, J.rs, J.os,
                                         J.in_plane, J.out_plane, J.in_field, J.out_field, J.tw);
}

template <typename T, int ML, int W, int SPEC, int ZV>
__global__ void __launch_bounds__(W * Plan<ML>::TPC, ConvOcc<T, ML, ZV>::value) k_col_convolve_rag(
    const __grid_constant__ RagTable<ConvJob<T>> t)
{
    const ConvJob<T> &J = rag_job(t);
    col_convolve_body<T, ML, W, SPEC>((int)blockIdx.x - J.cta0, J.nf, J.B, J.spec, J.K, J.My, J.s0, J.ns, J.t0, J.nt,
                                      J.field, J.tw);
}

// ---------------------------------------------------------------------------
// Host-side launch helpers.
// ---------------------------------------------------------------------------
template <typename T, int ML>
struct ColCfg {
    static constexpr int TPC = Plan<ML>::TPC;
    static constexpr int W0 = 256 / TPC < 8 ? 8 : (256 / TPC > 32 ? 32 : 256 / TPC);
    static constexpr int WMAX = int(98304 / (sizeof(Cx<T>) * ML)) < 1 ? 1 : int(98304 / (sizeof(Cx<T>) * ML));
    static constexpr int W = W0 < WMAX ? W0 : WMAX;
    static constexpr size_t SMEM = sizeof(Cx<T>) * (((size_t)ML) * (W + 1));
};

template <typename T, int ML>
struct RowCfg {
    static constexpr int TPC = Plan<ML>::TPC;
    static constexpr int L0 = 256 / TPC < 1 ? 1 : (256 / TPC > 32 ? 32 : 256 / TPC);
    static constexpr int LD = RowAddr<ML>::LD;
    static constexpr int LMAX = int(98304 / (sizeof(Cx<T>) * LD)) < 1 ? 1 : int(98304 / (sizeof(Cx<T>) * LD));
    static constexpr int LPC = L0 < LMAX ? L0 : LMAX;
    static constexpr size_t SMEM = sizeof(Cx<T>) * (((size_t)ML) + (size_t)LPC * LD);
};

}  // namespace pk

// Launch entry points (one set per precision, instantiated in
// lgf_poisson_f32.cu / lgf_poisson_f64.cu).
template <typename T>
lgf_status launch_row_forward(lgf_ctx *ctx, const PoissonGeom &g, const T *f, Cx<T> *A, const Cx<T> *tw, int nfields,
                              int lb, int dense_ld, cudaStream_t s);
template <typename T>
lgf_status launch_row_inverse(lgf_ctx *ctx, const PoissonGeom &g, const Cx<T> *A, T *u, const Cx<T> *tw, int nfields,
                              int lb, cudaStream_t s);
template <typename T>
lgf_status launch_col_forward(lgf_ctx *ctx, int M, int K, int nplanes, int nfields, const Cx<T> *in, Cx<T> *out,
                              int lo, int n, int64_t rs, int64_t os, int64_t in_plane, int64_t out_plane,
                              int64_t in_field, int64_t out_field, const Cx<T> *tw, pk::RowFlags rf, cudaStream_t s,
                              const char *name);
template <typename T>
lgf_status launch_col_inverse(lgf_ctx *ctx, int M, int K, int nplanes, int nfields, const Cx<T> *in, Cx<T> *out,
                              int lo, int n, int64_t rs, int64_t os, int64_t in_plane, int64_t out_plane,
                              int64_t in_field, int64_t out_field, const Cx<T> *tw, cudaStream_t s, const char *name);
template <typename T, int SPEC>
lgf_status launch_col_convolve(lgf_ctx *ctx, const PoissonGeom &g, Cx<T> *B, const T *spec, const Cx<T> *tw,
                               int nfields, cudaStream_t s);
// Ragged launches of one pass over jobs that share the transform length M
// (and the variant named by the other arguments); every job field but cta0
// and gx is set by the caller.
template <typename T>
lgf_status launch_row_forward_rag(lgf_ctx *ctx, int M, pk::RowJob<T> *jobs, int n, cudaStream_t s);
template <typename T>
lgf_status launch_row_inverse_rag(lgf_ctx *ctx, int M, bool half_out, pk::RowJob<T> *jobs, int n, cudaStream_t s);
template <typename T>
lgf_status launch_col_forward_rag(lgf_ctx *ctx, int M, pk::ColJob<T> *jobs, int n, cudaStream_t s);
template <typename T>
lgf_status launch_col_inverse_rag(lgf_ctx *ctx, int M, bool half_out, pk::ColJob<T> *jobs, int n, cudaStream_t s);
template <typename T, int SPEC>
lgf_status launch_col_convolve_rag(lgf_ctx *ctx, int M, int zvar, pk::ConvJob<T> *jobs, int n, cudaStream_t s);

}  // namespace lgf

namespace lgf {
namespace pk {

template <class K>
inline lgf_status set_smem(lgf_ctx *ctx, K kern, size_t smem)
{
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaFuncSetAttribute");
    }
    return LGF_OK;
}

template <typename T, int ML>
lgf_status row_forward_m(lgf_ctx *ctx, const PoissonGeom &g, const T *f, Cx<T> *A, const Cx<T> *tw, int nfields,
                         int lb, int dense_ld, cudaStream_t s)
{
    using C = RowCfg<T, ML>;
    auto kern = k_row_forward<T, ML, C::LPC, true>;
    if (dense_ld) {
        // full dense rows: only the FP64 spectrum build
        if constexpr (sizeof(T) == 8)
            kern = k_row_forward<T, ML, C::LPC, false>;
        else
            return fail(ctx, LGF_EINVAL, "row forward: FP32 dense rows");
    } else if (g.s0[0] < 0 || 2 * (g.s0[0] + g.Ls[0]) > g.M[0]) {
        return fail(ctx, LGF_EINVAL, "row forward: source beyond half the transform length");
    }
    lgf_status st = set_smem(ctx, kern, C::SMEM);
    if (st != LGF_OK) return st;
    const int npairs = (g.Ls[1] / 2) * g.Ls[2];
    dim3 grid((npairs + C::LPC - 1) / C::LPC, nfields);
    const int ph = prof_begin(ctx, s, dense_ld ? "spectrum_x_forward" : "poisson_x_forward");
    kern<<<grid, C::LPC * C::TPC, C::SMEM, s>>>(f, A, g, tw, npairs, lb, dense_ld);
    LGF_CHECK_LAUNCH(ctx, "poisson x-forward");
    prof_end(ctx, s, ph);
    return LGF_OK;
}

template <typename T, int ML>
lgf_status row_inverse_m(lgf_ctx *ctx, const PoissonGeom &g, const Cx<T> *A, T *u, const Cx<T> *tw, int nfields,
                         int lb, cudaStream_t s)
{
    using C = RowCfg<T, ML>;
    auto kern = k_row_inverse<T, ML, C::LPC, true>;
    if (g.t0[0] < 0 || g.t0[0] + g.Lt[0] > g.M[0])
        return fail(ctx, LGF_EINVAL, "row inverse: target beyond the transform length");
    if (2 * (g.t0[0] + g.Lt[0]) > g.M[0]) kern = k_row_inverse<T, ML, C::LPC, false>;
    lgf_status st = set_smem(ctx, kern, C::SMEM);
    if (st != LGF_OK) return st;
    const int npairs = (g.Lt[1] / 2) * g.Lt[2];
    dim3 grid((npairs + C::LPC - 1) / C::LPC, nfields);
    const int ph = prof_begin(ctx, s, "poisson_x_inverse");
    kern<<<grid, C::LPC * C::TPC, C::SMEM, s>>>(A, u, g, tw, npairs, lb);
    LGF_CHECK_LAUNCH(ctx, "poisson x-inverse");
    prof_end(ctx, s, ph);
    return LGF_OK;
}

template <typename T, int ML>
lgf_status col_forward_m(lgf_ctx *ctx, int K, int nplanes, int nfields, const Cx<T> *in, Cx<T> *out, int lo, int n,
                         int64_t rs, int64_t os, int64_t in_plane, int64_t out_plane, int64_t in_field,
                         int64_t out_field, const Cx<T> *tw, RowFlags rf, cudaStream_t s, const char *name)
{
    using C = ColCfg<T, ML>;
    auto kern = k_col_forward<T, ML, C::W, true>;
    if (lo + n > ML / 2) {
        // full-length input: only the FP64 spectrum build's z pass
        if constexpr (sizeof(T) == 8)
            kern = k_col_forward<T, ML, C::W, false>;
        else
            return fail(ctx, LGF_EINVAL, "column forward: FP32 input beyond half the transform length");
    }
    lgf_status st = set_smem(ctx, kern, C::SMEM);
    if (st != LGF_OK) return st;
    dim3 grid(col_ctas<C::W>(K, nplanes), nfields);
    const int ph = prof_begin(ctx, s, name);
    kern<<<grid, C::W * C::TPC, C::SMEM, s>>>(in, out, K, nplanes, lo, n, rs, os, in_plane, out_plane, in_field,
                                              out_field, tw, rf);
    LGF_CHECK_LAUNCH(ctx, name);
    prof_end(ctx, s, ph);
    return LGF_OK;
}

template <typename T, int ML>
lgf_status col_inverse_m(lgf_ctx *ctx, int K, int nplanes, int nfields, const Cx<T> *in, Cx<T> *out, int lo, int n,
                         int64_t rs, int64_t os, int64_t in_plane, int64_t out_plane, int64_t in_field,
                         int64_t out_field, const Cx<T> *tw, cudaStream_t s, const char *name)
{
    using C = ColCfg<T, ML>;
    auto kern = k_col_inverse<T, ML, C::W, true>;
    if (lo < 0 || lo + n > ML) return fail(ctx, LGF_EINVAL, "column inverse: rows beyond the length");
    if (lo + n > ML / 2) kern = k_col_inverse<T, ML, C::W, false>;
    lgf_status st = set_smem(ctx, kern, C::SMEM);
    if (st != LGF_OK) return st;
    dim3 grid(col_ctas<C::W>(K, nplanes), nfields);
    const int ph = prof_begin(ctx, s, name);
    kern<<<grid, C::W * C::TPC, C::SMEM, s>>>(in, out, K, nplanes, lo, n, rs, os, in_plane, out_plane, in_field,
                                              out_field, tw);
    LGF_CHECK_LAUNCH(ctx, name);
    prof_end(ctx, s, ph);
    return LGF_OK;
}

template <typename T, int ML, int SPEC>
lgf_status col_convolve_m(lgf_ctx *ctx, const PoissonGeom &g, Cx<T> *B, const T *spec, const Cx<T> *tw, int nfields,
                          cudaStream_t s)
{
    using C = ColCfg<T, ML>;
    // the register variant is an FP32 choice (FP64 runs one CTA per SM)
    auto kern = (sizeof(T) == 4 && g.zvar) ? k_col_convolve<T, ML, C::W, SPEC, sizeof(T) == 4 ? 1 : 0>
                                           : k_col_convolve<T, ML, C::W, SPEC, 0>;
    if (g.s0[2] < 0 || g.t0[2] < 0 || 2 * (g.s0[2] + g.Ls[2]) > g.M[2] || 2 * (g.t0[2] + g.Lt[2]) > g.M[2])
        return fail(ctx, LGF_EINVAL, "z pass: planes beyond half the transform length");
    lgf_status st = set_smem(ctx, kern, C::SMEM);
    if (st != LGF_OK) return st;
    dim3 grid(nfields * col_ctas<C::W>(g.Kx, g.M[1]));
    const int ph = prof_begin(ctx, s, "poisson_z_convolve");
    kern<<<grid, C::W * C::TPC, C::SMEM, s>>>(B, spec, g.Kx, g.M[1], g.s0[2], g.Ls[2], g.t0[2], g.Lt[2], g.Bstride,
                                              tw);
    LGF_CHECK_LAUNCH(ctx, "poisson z-convolve");
    prof_end(ctx, s, ph);
    return LGF_OK;
}

// Send jobs in tables of kRagJobs, CTA ranges assigned in order; jobs with
// no CTAs are skipped.
template <class J, class Kern>
lgf_status rag_send(lgf_ctx *ctx, Kern kern, int threads, size_t smem, J *jobs, int n, cudaStream_t s,
                    const char *name)
{
    static_assert(sizeof(RagTable<J>) <= 32000, "job table beyond the kernel parameter space");
    for (int c0 = 0; c0 < n;) {
        RagTable<J> t;
        t.n = 0;
        int64_t ctas = 0;
        for (; c0 < n && t.n < kRagJobs; ++c0) {
            J &j = jobs[c0];
            const int64_t nc = (int64_t)j.gx * j.nf;
            if (nc <= 0) continue;
            j.cta0 = (int)ctas;
            t.j[t.n++] = j;
            ctas += nc;
        }
        if (t.n == 0) continue;
        if (ctas > 0x7fffffff) return fail(ctx, LGF_EUNSUPPORTED, "ragged launch: too many CTAs");
        const int ph = prof_begin(ctx, s, name);
        kern<<<(unsigned)ctas, threads, smem, s>>>(t);
        LGF_CHECK_LAUNCH(ctx, name);
        prof_end(ctx, s, ph);
    }
    return LGF_OK;
}

template <typename T, int ML>
lgf_status row_forward_rag_m(lgf_ctx *ctx, RowJob<T> *jobs, int n, cudaStream_t s)
{
    using C = RowCfg<T, ML>;
    auto kern = k_row_forward_rag<T, ML, C::LPC, true>;
    for (int i = 0; i < n; ++i) {
        const PoissonGeom &g = jobs[i].g;
        if (g.M[0] != ML || g.s0[0] < 0 || 2 * (g.s0[0] + g.Ls[0]) > g.M[0])
            return fail(ctx, LGF_EINVAL, "ragged row forward: source beyond half the transform length");
        jobs[i].gx = (jobs[i].npairs + C::LPC - 1) / C::LPC;
    }
    lgf_status st = set_smem(ctx, kern, C::SMEM);
    if (st != LGF_OK) return st;
    return rag_send(ctx, kern, C::LPC * C::TPC, C::SMEM, jobs, n, s, "poisson_x_forward");
}

template <typename T, int ML>
lgf_status row_inverse_rag_m(lgf_ctx *ctx, bool half_out, RowJob<T> *jobs, int n, cudaStream_t s)
{
    using C = RowCfg<T, ML>;
    auto kern = half_out ? k_row_inverse_rag<T, ML, C::LPC, true> : k_row_inverse_rag<T, ML, C::LPC, false>;
    for (int i = 0; i < n; ++i) {
        const PoissonGeom &g = jobs[i].g;
        if (g.M[0] != ML || g.t0[0] < 0 || g.t0[0] + g.Lt[0] > g.M[0] ||
            (half_out && 2 * (g.t0[0] + g.Lt[0]) > g.M[0]))
            return fail(ctx, LGF_EINVAL, "ragged row inverse: target beyond the transform length");
        jobs[i].gx = (jobs[i].npairs + C::LPC - 1) / C::LPC;
    }
    lgf_status st = set_smem(ctx, kern, C::SMEM);
    if (st != LGF_OK) return st;
    return rag_send(ctx, kern, C::LPC * C::TPC, C::SMEM, jobs, n, s, "poisson_x_inverse");
}

template <typename T, int ML>
lgf_status col_forward_rag_m(lgf_ctx *ctx, ColJob<T> *jobs, int n, cudaStream_t s)
{
    using C = ColCfg<T, ML>;
    auto kern = k_col_forward_rag<T, ML, C::W>;
    for (int i = 0; i < n; ++i) {
        if (jobs[i].lo < 0 || jobs[i].lo + jobs[i].n > ML / 2)
            return fail(ctx, LGF_EINVAL, "ragged column forward: input beyond half the transform length");
        jobs[i].gx = col_ctas<C::W>(jobs[i].K, jobs[i].nplanes);
    }
    lgf_status st = set_smem(ctx, kern, C::SMEM);
    if (st != LGF_OK) return st;
    return rag_send(ctx, kern, C::W * C::TPC, C::SMEM, jobs, n, s, "poisson_y_forward");
}

template <typename T, int ML>
lgf_status col_inverse_rag_m(lgf_ctx *ctx, bool half_out, ColJob<T> *jobs, int n, cudaStream_t s)
{
    using C = ColCfg<T, ML>;
    auto kern = half_out ? k_col_inverse_rag<T, ML, C::W, true> : k_col_inverse_rag<T, ML, C::W, false>;
    for (int i = 0; i < n; ++i) {
        if (jobs[i].lo < 0 || jobs[i].lo + jobs[i].n > (half_out ? ML / 2 : ML))
            return fail(ctx, LGF_EINVAL, "ragged column inverse: rows beyond the length");
        jobs[i].gx = col_ctas<C::W>(jobs[i].K, jobs[i].nplanes);
    }
    lgf_status st = set_smem(ctx, kern, C::SMEM);
    if (st != LGF_OK) return st;
    return rag_send(ctx, kern, C::W * C::TPC, C::SMEM, jobs, n, s, "poisson_y_inverse");
}

template <typename T, int ML, int SPEC>
lgf_status col_convolve_rag_m(lgf_ctx *ctx, int zvar, ConvJob<T> *jobs, int n, cudaStream_t s)
{
    using C = ColCfg<T, ML>;
    auto kern = (sizeof(T) == 4 && zvar) ? k_col_convolve_rag<T, ML, C::W, SPEC, sizeof(T) == 4 ? 1 : 0>
                                         : k_col_convolve_rag<T, ML, C::W, SPEC, 0>;
    for (int i = 0; i < n; ++i) {
        const ConvJob<T> &j = jobs[i];
        if (j.s0 < 0 || j.t0 < 0 || 2 * (j.s0 + j.ns) > ML || 2 * (j.t0 + j.nt) > ML)
            return fail(ctx, LGF_EINVAL, "ragged z pass: planes beyond half the transform length");
        jobs[i].gx = col_ctas<C::W>(j.K, j.My);
    }
    lgf_status st = set_smem(ctx, kern, C::SMEM);
    if (st != LGF_OK) return st;
    return rag_send(ctx, kern, C::W * C::TPC, C::SMEM, jobs, n, s, "poisson_z_convolve");
}

#define LGF_DISPATCH_ML(M_RT, CALL)                                             \
    switch (M_RT) {                                                             \
    case 32: { constexpr int LM = 32; return CALL; }                            \
    case 64: { constexpr int LM = 64; return CALL; }                            \
    case 80: { constexpr int LM = 80; return CALL; }                            \
    case 160: { constexpr int LM = 160; return CALL; }                          \
    case 320: { constexpr int LM = 320; return CALL; }                          \
    case 640: { constexpr int LM = 640; return CALL; }                          \
    case 1280: { constexpr int LM = 1280; return CALL; }                        \
    case 2560: { constexpr int LM = 2560; return CALL; }                        \
    case 96: { constexpr int LM = 96; return CALL; }                            \
    case 128: { constexpr int LM = 128; return CALL; }                          \
    case 192: { constexpr int LM = 192; return CALL; }                          \
    case 256: { constexpr int LM = 256; return CALL; }                          \
    case 384: { constexpr int LM = 384; return CALL; }                          \
    case 512: { constexpr int LM = 512; return CALL; }                          \
    case 768: { constexpr int LM = 768; return CALL; }                          \
    case 1024: { constexpr int LM = 1024; return CALL; }                        \
    case 1536: { constexpr int LM = 1536; return CALL; }                        \
    case 2048: { constexpr int LM = 2048; return CALL; }                        \
    case 3072: { constexpr int LM = 3072; return CALL; }                        \
    case 4096: { constexpr int LM = 4096; return CALL; }                        \
    default: return fail(ctx, LGF_EUNSUPPORTED, "transform length not 2^k, 3*2^k or 5*2^k in 32..4096"); \
    }

}  // namespace pk

template <typename T>
lgf_status launch_row_forward(lgf_ctx *ctx, const PoissonGeom &g, const T *f, Cx<T> *A, const Cx<T> *tw, int nfields,
                              int lb, int dense_ld, cudaStream_t s)
{
    LGF_DISPATCH_ML(g.M[0], (pk::row_forward_m<T, LM>(ctx, g, f, A, tw, nfields, lb, dense_ld, s)));
}

template <typename T>
lgf_status launch_row_inverse(lgf_ctx *ctx, const PoissonGeom &g, const Cx<T> *A, T *u, const Cx<T> *tw, int nfields,
                              int lb, cudaStream_t s)
{
    LGF_DISPATCH_ML(g.M[0], (pk::row_inverse_m<T, LM>(ctx, g, A, u, tw, nfields, lb, s)));
}

template <typename T>
lgf_status launch_col_forward(lgf_ctx *ctx, int M, int K, int nplanes, int nfields, const Cx<T> *in, Cx<T> *out,
                              int lo, int n, int64_t rs, int64_t os, int64_t in_plane, int64_t out_plane,
                              int64_t in_field, int64_t out_field, const Cx<T> *tw, pk::RowFlags rf, cudaStream_t s,
                              const char *name)
{
    LGF_DISPATCH_ML(M, (pk::col_forward_m<T, LM>(ctx, K, nplanes, nfields, in, out, lo, n, rs, os,
                                                               in_plane, out_plane, in_field, out_field, tw, rf,
                                                               s, name)));
}

template <typename T>
lgf_status launch_col_inverse(lgf_ctx *ctx, int M, int K, int nplanes, int nfields, const Cx<T> *in, Cx<T> *out,
                              int lo, int n, int64_t rs, int64_t os, int64_t in_plane, int64_t out_plane,
                              int64_t in_field, int64_t out_field, const Cx<T> *tw, cudaStream_t s, const char *name)
{
    LGF_DISPATCH_ML(M, (pk::col_inverse_m<T, LM>(ctx, K, nplanes, nfields, in, out, lo, n, rs, os,
                                                               in_plane, out_plane, in_field, out_field, tw,
                                                               s, name)));
}

template <typename T, int SPEC>
lgf_status launch_col_convolve(lgf_ctx *ctx, const PoissonGeom &g, Cx<T> *B, const T *spec, const Cx<T> *tw,
                               int nfields, cudaStream_t s)
{
    LGF_DISPATCH_ML(g.M[2], (pk::col_convolve_m<T, LM, SPEC>(ctx, g, B, spec, tw, nfields, s)));
}

template <typename T>
lgf_status launch_row_forward_rag(lgf_ctx *ctx, int M, pk::RowJob<T> *jobs, int n, cudaStream_t s)
{
    LGF_DISPATCH_ML(M, (pk::row_forward_rag_m<T, LM>(ctx, jobs, n, s)));
}

template <typename T>
lgf_status launch_row_inverse_rag(lgf_ctx *ctx, int M, bool half_out, pk::RowJob<T> *jobs, int n, cudaStream_t s)
{
    LGF_DISPATCH_ML(M, (pk::row_inverse_rag_m<T, LM>(ctx, half_out, jobs, n, s)));
}

template <typename T>
lgf_status launch_col_forward_rag(lgf_ctx *ctx, int M, pk::ColJob<T> *jobs, int n, cudaStream_t s)
{
    LGF_DISPATCH_ML(M, (pk::col_forward_rag_m<T, LM>(ctx, jobs, n, s)));
}

template <typename T>
lgf_status launch_col_inverse_rag(lgf_ctx *ctx, int M, bool half_out, pk::ColJob<T> *jobs, int n, cudaStream_t s)
{
    LGF_DISPATCH_ML(M, (pk::col_inverse_rag_m<T, LM>(ctx, half_out, jobs, n, s)));
}

template <typename T, int SPEC>
lgf_status launch_col_convolve_rag(lgf_ctx *ctx, int M, int zvar, pk::ConvJob<T> *jobs, int n, cudaStream_t s)
{
    LGF_DISPATCH_ML(M, (pk::col_convolve_rag_m<T, LM, SPEC>(ctx, zvar, jobs, n, s)));
}

}  // namespace lgf
