// Shared-memory FFTs of power-of-two length M (32..4096) for many lines at once.
//
// A line is factored into radix-16/8/4/2 stages.  The forward transform is a
// decimation-in-frequency sweep: each stage reads R elements at stride N/R of
// a sub-problem of size N, does the R-point DFT in registers, multiplies by
// the twiddles w_N^{j q} and writes the results back to the same R slots, so
// sub-problem q occupies a contiguous range afterwards.  The spectrum ends in
// mixed-radix digit-reversed order; pos_of_freq/freq_of_pos convert.  The
// inverse is the exact adjoint sweep (conjugate twiddles, stages reversed),
// which takes digit-reversed input to natural-order output.  A z-pass can
// therefore run forward -> pointwise multiply -> inverse with no permutation.
//
// Sign convention: forward X[k] = sum_n x[n] e^{-2 pi i n k / M};
// inverse x[n] = sum_k X[k] e^{+2 pi i n k / M} (unnormalised).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lgf {

template <typename R>
struct __align__(2 * sizeof(R)) Cx {
    R x, y;
};

template <typename R>
__device__ __forceinline__ Cx<R> cadd(Cx<R> a, Cx<R> b) { return {a.x + b.x, a.y + b.y}; }
template <typename R>
__device__ __forceinline__ Cx<R> csub(Cx<R> a, Cx<R> b) { return {a.x - b.x, a.y - b.y}; }
template <typename R>
__device__ __forceinline__ Cx<R> cmul(Cx<R> a, Cx<R> b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
// a * conj(b)
template <typename R>
__device__ __forceinline__ Cx<R> cmulc(Cx<R> a, Cx<R> b) { return {a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y}; }
template <typename R>
__device__ __forceinline__ Cx<R> cconj(Cx<R> a) { return {a.x, -a.y}; }

// Radix factorisation of a power-of-two length, passed to kernels by value.
struct FftShape {
    int M;       // length
    int logM;    // log2(M)
    int nst;     // number of stages
    int lg[4];   // log2 of each stage's radix, first stage first
};

// cos(pi k / 8) and sin(pi k / 8), k = 0..8 (the 16th roots of unity).
__host__ __device__ constexpr double c16(int k)
{
    return k == 0 ? 1.0 : k == 1 ? 0.92387953251128675613 : k == 2 ? 0.70710678118654752440
         : k == 3 ? 0.38268343236508977173 : k == 4 ? 0.0 : k == 5 ? -0.38268343236508977173
         : k == 6 ? -0.70710678118654752440 : k == 7 ? -0.92387953251128675613 : -1.0;
}
__host__ __device__ constexpr double s16(int k) { return c16(k < 4 ? 4 - k : k - 4) * (k <= 8 ? 1.0 : -1.0); }

// v * exp(DIR * 2 pi i k / R) for compile-time R, k.
template <int R, int K, int DIR, typename T>
__device__ __forceinline__ Cx<T> rot(Cx<T> v)
{
    constexpr int q = (16 / R) * K;   // angle = pi q / 8
    if constexpr (q == 0) {
        return v;
    } else if constexpr (q == 4) {    // multiply by DIR * i
        return {T(-DIR) * v.y, T(DIR) * v.x};
    } else {
        const T c = T(c16(q)), s = T(DIR) * T(s16(q));
        return {v.x * c - v.y * s, v.x * s + v.y * c};
    }
}

// In-register DFT of R points (natural order in, natural order out), by
// recursive even/odd splitting unrolled at compile time.
template <int R, int DIR, typename T>
struct Dft {
    template <int K>
    static __device__ __forceinline__ void combine(Cx<T> *a, const Cx<T> *e, const Cx<T> *o)
    {
        if constexpr (K < R / 2) {
            const Cx<T> t = rot<R, K, DIR, T>(o[K]);
            a[K] = cadd(e[K], t);
            a[K + R / 2] = csub(e[K], t);
            combine<K + 1>(a, e, o);
        }
    }
    static __device__ __forceinline__ void run(Cx<T> *a)
    {
        Cx<T> e[R / 2], o[R / 2];
#pragma unroll
        for (int k = 0; k < R / 2; ++k) {
            e[k] = a[2 * k];
            o[k] = a[2 * k + 1];
        }
        Dft<R / 2, DIR, T>::run(e);
        Dft<R / 2, DIR, T>::run(o);
        combine<0>(a, e, o);
    }
};
template <int DIR, typename T>
struct Dft<1, DIR, T> {
    static __device__ __forceinline__ void run(Cx<T> *) {}
};

// DFT of R points whose upper half a[R/2..R) is zero (only a[0..R/2) is
// read): the even outputs are the (R/2)-point DFT of a[p], the odd ones the
// (R/2)-point DFT of a[p] w_R^p.  Saves the first butterfly layer.
template <int R, int DIR, typename T, int P = 0>
__device__ __forceinline__ void twist_half(Cx<T> *o, const Cx<T> *a)
{
    if constexpr (P < R / 2) {
        o[P] = rot<R, P, DIR, T>(a[P]);
        twist_half<R, DIR, T, P + 1>(o, a);
    }
}
template <int R, int DIR, typename T>
__device__ __forceinline__ void dft_half_in(Cx<T> *a)
{
    Cx<T> e[R / 2], o[R / 2];
#pragma unroll
    for (int p = 0; p < R / 2; ++p) e[p] = a[p];
    twist_half<R, DIR, T>(o, a);
    Dft<R / 2, DIR, T>::run(e);
    Dft<R / 2, DIR, T>::run(o);
#pragma unroll
    for (int k = 0; k < R / 2; ++k) {
        a[2 * k] = e[k];
        a[2 * k + 1] = o[k];
    }
}

// DFT of R points of which only the outputs a[0..R/2) are wanted: the last
// butterfly layer keeps its sums and drops its differences.
template <int R, int DIR, typename T, int K = 0>
__device__ __forceinline__ void combine_low(Cx<T> *a, const Cx<T> *e, const Cx<T> *o)
{
    if constexpr (K < R / 2) {
        a[K] = cadd(e[K], rot<R, K, DIR, T>(o[K]));
        combine_low<R, DIR, T, K + 1>(a, e, o);
    }
}
template <int R, int DIR, typename T>
__device__ __forceinline__ void dft_half_out(Cx<T> *a)
{
    Cx<T> e[R / 2], o[R / 2];
#pragma unroll
    for (int k = 0; k < R / 2; ++k) {
        e[k] = a[2 * k];
        o[k] = a[2 * k + 1];
    }
    Dft<R / 2, DIR, T>::run(e);
    Dft<R / 2, DIR, T>::run(o);
    combine_low<R, DIR, T>(a, e, o);
}

// Shared-memory addressing of lines.
// Rows: line-major, each line contiguous, one padding slot per 16 elements
// (keeps stride-R accesses of late stages off a single bank).
struct RowAddr {
    int ld;  // = M + M / 16
    __device__ __forceinline__ int operator()(int line, int m) const { return line * ld + m + (m >> 4); }
};
// Columns: element m of line w at m * W + w (consecutive threads -> consecutive w).
struct ColAddr {
    int W;
    __device__ __forceinline__ int operator()(int line, int m) const { return m * W + line; }
};

// One stage.  Forward (DIR = -1): butterfly then twiddle.  Adjoint (DIR = +1):
// conjugate twiddle then butterfly, data movement reversed.
// tw[m] = exp(-2 pi i m / M), m < M.  LINE_FAST selects the thread -> (line,
// group) mapping so that consecutive threads touch consecutive addresses.
template <int LOGR, int DIR, bool LINE_FAST, typename T, class Addr>
__device__ __forceinline__ void fft_stage(Cx<T> *s, const Addr &ad, int nlines, int logM, int logN,
                                          const Cx<T> *tw)
{
    constexpr int R = 1 << LOGR;
    const int logNp = logN - LOGR;                 // sub-problem size after this stage
    const int Np = 1 << logNp;
    const int logG = logM - LOGR;                  // groups per line
    const int items = nlines << logG;
    const int twshift = logM - logN;               // twiddle index = (M/N) * j * q
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
        int line, g;
        if (LINE_FAST) {
            line = it % nlines;
            g = it / nlines;
        } else {
            g = it & ((1 << logG) - 1);
            line = it >> logG;
        }
        const int sub = g >> logNp, j = g & (Np - 1);
        const int o = sub << logN;
        Cx<T> a[R];
        if (DIR < 0) {
#pragma unroll
            for (int p = 0; p < R; ++p) a[p] = s[ad(line, o + j + (p << logNp))];
            Dft<R, -1, T>::run(a);
#pragma unroll
            for (int q = 1; q < R; ++q) a[q] = cmul(a[q], tw[(j * q) << twshift]);
#pragma unroll
            for (int q = 0; q < R; ++q) s[ad(line, o + (q << logNp) + j)] = a[q];
        } else {
#pragma unroll
            for (int q = 0; q < R; ++q) a[q] = s[ad(line, o + (q << logNp) + j)];
#pragma unroll
            for (int q = 1; q < R; ++q) a[q] = cmulc(a[q], tw[(j * q) << twshift]);
            Dft<R, 1, T>::run(a);
#pragma unroll
            for (int p = 0; p < R; ++p) s[ad(line, o + j + (p << logNp))] = a[p];
        }
    }
}

template <int DIR, bool LINE_FAST, typename T, class Addr>
__device__ __forceinline__ void fft_stage_any(int lgR, Cx<T> *s, const Addr &ad, int nlines, int logM, int logN,
                                              const Cx<T> *tw)
{
    switch (lgR) {
    case 4: fft_stage<4, DIR, LINE_FAST>(s, ad, nlines, logM, logN, tw); break;
    case 3: fft_stage<3, DIR, LINE_FAST>(s, ad, nlines, logM, logN, tw); break;
    case 2: fft_stage<2, DIR, LINE_FAST>(s, ad, nlines, logM, logN, tw); break;
    default: fft_stage<1, DIR, LINE_FAST>(s, ad, nlines, logM, logN, tw); break;
    }
}

// Forward transform of `nlines` lines: natural order in, digit-reversed out.
// Every thread of the block must call it (it synchronises between stages).
template <bool LINE_FAST, typename T, class Addr>
__device__ void fft_forward(Cx<T> *s, const Addr &ad, int nlines, const FftShape &sh, const Cx<T> *tw)
{
    int logN = sh.logM;
    for (int st = 0; st < sh.nst; ++st) {
        fft_stage_any<-1, LINE_FAST>(sh.lg[st], s, ad, nlines, sh.logM, logN, tw);
        __syncthreads();
        logN -= sh.lg[st];
    }
}

// Inverse (adjoint) transform: digit-reversed in, natural order out.
template <bool LINE_FAST, typename T, class Addr>
__device__ void fft_inverse(Cx<T> *s, const Addr &ad, int nlines, const FftShape &sh, const Cx<T> *tw)
{
    int logN[4];
    int l = sh.logM;
    for (int st = 0; st < sh.nst; ++st) {
        logN[st] = l;
        l -= sh.lg[st];
    }
    for (int st = sh.nst - 1; st >= 0; --st) {
        fft_stage_any<1, LINE_FAST>(sh.lg[st], s, ad, nlines, sh.logM, logN[st], tw);
        __syncthreads();
    }
}

// Position in the forward output of frequency k.
__device__ __forceinline__ int pos_of_freq(int k, const FftShape &sh)
{
    int P = 0, logN = sh.logM;
    for (int st = 0; st < sh.nst; ++st) {
        const int lgR = sh.lg[st];
        const int q = k & ((1 << lgR) - 1);
        k >>= lgR;
        logN -= lgR;
        P += q << logN;
    }
    return P;
}

// Frequency held at position P of the forward output.
__device__ __forceinline__ int freq_of_pos(int P, const FftShape &sh)
{
    int k = 0, shift = 0, logN = sh.logM;
    for (int st = 0; st < sh.nst; ++st) {
        const int lgR = sh.lg[st];
        logN -= lgR;
        const int q = P >> logN;
        P &= (1 << logN) - 1;
        k += q << shift;
        shift += lgR;
    }
    return k;
}

}  // namespace lgf
