// In-register DFT building blocks of the pass kernels (lgf_poisson_kernels.cuh).
//
// A line of length M (2^k, or 3 * 2^k) is transformed by decimation in
// frequency: each stage reads R elements at stride N/R of a sub-problem of
// size N, does the R-point DFT in registers, multiplies by the twiddles
// w_N^{j q} and writes the results back to the same R slots, so sub-problem q
// occupies a contiguous range afterwards.  The spectrum ends in mixed-radix
// digit-reversed order.  The inverse is the exact adjoint sweep (conjugate
// twiddles, stages reversed), which takes digit-reversed input to
// natural-order output, so a z pass can run forward -> pointwise multiply ->
// inverse with no permutation.
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

// cos(pi m / 24) for m = 0..12 (every twiddle angle of the register DFTs,
// radices 2..16 and 3 * 2^j up to 48, is a multiple of pi / 24).
__host__ __device__ constexpr double c24q(int m)
{
    return m == 0 ? 1.0 : m == 1 ? 0.99144486137381041114 : m == 2 ? 0.96592582628906828675
         : m == 3 ? 0.92387953251128675613 : m == 4 ? 0.86602540378443864676 : m == 5 ? 0.79335334029123516458
         : m == 6 ? 0.70710678118654752440 : m == 7 ? 0.60876142900872063942 : m == 8 ? 0.5
         : m == 9 ? 0.38268343236508977173 : m == 10 ? 0.25881904510252076235 : m == 11 ? 0.13052619222005159155
         : 0.0;
}
// cos(pi m / 24) and sin(pi m / 24) for any integer m.
__host__ __device__ constexpr double c24(int m)
{
    return (m = ((m % 48) + 48) % 48, m > 24 ? c24(48 - m) : m > 12 ? -c24q(24 - m) : c24q(m));
}
__host__ __device__ constexpr double s24(int m) { return c24(m - 12); }

// v * exp(DIR * 2 pi i k / R) for compile-time R (a divisor of 48 times k), k.
template <int R, int K, int DIR, typename T>
__device__ __forceinline__ Cx<T> rot(Cx<T> v)
{
    static_assert((48 * K) % R == 0, "twiddle angle must be a multiple of pi/24");
    constexpr int m = 48 * K / R;   // angle = pi m / 24
    if constexpr (m % 48 == 0) {
        return v;
    } else if constexpr (m % 48 == 12) {   // multiply by DIR * i
        return {T(-DIR) * v.y, T(DIR) * v.x};
    } else {
        const T c = T(c24(m)), s = T(DIR) * T(s24(m));
        return {v.x * c - v.y * s, v.x * s + v.y * c};
    }
}

// In-register DFT of R points (natural order in, natural order out), by
// recursive even/odd splitting unrolled at compile time (R = 2^j or 3 * 2^j).
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
// Three points: X0 = a0 + t, X1,2 = a0 - t/2 +- DIR i (sqrt(3)/2)(a1 - a2), t = a1 + a2.
template <int DIR, typename T>
struct Dft<3, DIR, T> {
    static __device__ __forceinline__ void run(Cx<T> *a)
    {
        const T h = T(0.86602540378443864676);
        const Cx<T> t = cadd(a[1], a[2]), d = csub(a[1], a[2]);
        const Cx<T> m = {a[0].x - T(0.5) * t.x, a[0].y - T(0.5) * t.y};
        const Cx<T> sd = {T(-DIR) * h * d.y, T(DIR) * h * d.x};
        a[0] = cadd(a[0], t);
        a[1] = cadd(m, sd);
        a[2] = csub(m, sd);
    }
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

}  // namespace lgf
