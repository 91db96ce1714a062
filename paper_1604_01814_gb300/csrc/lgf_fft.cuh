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

// cos(pi m / 120) for m = 0..60: every twiddle angle of the register DFTs
// (radices 2..16, 3 * 2^j and 5 * 2^j up to 20) is a multiple of pi / 120.
constexpr double kCos120[61] = {
    1.0, 0.99965732497555728004, 0.99862953475457387378, 0.99691733373312797620,
    0.99452189536827333692, 0.99144486137381041114, 0.98768834059513772619, 0.98325490756395458455,
    0.97814760073380563793, 0.97236992039767660183, 0.96592582628906828675, 0.95881973486819304976,
    0.95105651629515357212, 0.94264149109217839478, 0.93358042649720174899, 0.92387953251128675613,
    0.91354545764260089550, 0.90258528434986060676, 0.89100652418836786236, 0.87881711266196537413,
    0.86602540378443864676, 0.85264016435409222152, 0.83867056794542402964, 0.82412618862201566173,
    0.80901699437494742410, 0.79335334029123516458, 0.77714596145697087998, 0.76040596560003093817,
    0.74314482547739423501, 0.72537437101228763799, 0.70710678118654752440, 0.68835457569375398439,
    0.66913060635885821383, 0.64944804833018365573, 0.62932039104983745271, 0.60876142900872063942,
    0.58778525229247312917, 0.56640623692483283182, 0.54463903501502708222, 0.52249856471594886499,
    0.50000000000000000000, 0.47715876025960841505, 0.45399049973954679156, 0.43051109680829514438,
    0.40673664307580020775, 0.38268343236508977173, 0.35836794954530027348, 0.33380685923377092883,
    0.30901699437494742410, 0.28401534470392261744, 0.25881904510252076235, 0.23344536385590541177,
    0.20791169081775933710, 0.18223552549214745660, 0.15643446504023086901, 0.13052619222005159155,
    0.10452846326765347140, 0.07845909572784494503, 0.05233595624294383272, 0.02617694830787315261,
    0.0,
};
// cos(pi m / 120) and sin(pi m / 120) for any integer m.
__host__ __device__ constexpr double c120(int m)
{
    return (m = ((m % 240) + 240) % 240, m > 120 ? c120(240 - m) : m > 60 ? -kCos120[120 - m] : kCos120[m]);
}
__host__ __device__ constexpr double s120(int m) { return c120(m - 60); }

// v * exp(DIR * 2 pi i k / R) for compile-time R, k (2k/R a multiple of 1/120).
template <int R, int K, int DIR, typename T>
__device__ __forceinline__ Cx<T> rot(Cx<T> v)
{
    static_assert((240 * K) % R == 0, "twiddle angle must be a multiple of pi/120");
    constexpr int m = 240 * K / R;   // angle = pi m / 120
    if constexpr (m % 240 == 0) {
        return v;
    } else if constexpr (m % 240 == 60) {   // multiply by DIR * i
        return {T(-DIR) * v.y, T(DIR) * v.x};
    } else {
        constexpr double cd = c120(m), sd = s120(m);
        const T c = T(cd), s = T(DIR) * T(sd);
        return {v.x * c - v.y * s, v.x * s + v.y * c};
    }
}

// In-register DFT of R points (natural order in, natural order out), by
// recursive even/odd splitting unrolled at compile time (R = 2^j, 3 * 2^j or
// 5 * 2^j).
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
// Five points: with t1 = a1 + a4, t2 = a2 + a3, t3 = a1 - a4, t4 = a2 - a3 and
// w = exp(DIR 2 pi i / 5), X1,4 = a0 + c1 t1 + c2 t2 +- DIR i (s1 t3 + s2 t4),
// X2,3 = a0 + c2 t1 + c1 t2 +- DIR i (s2 t3 - s1 t4) (c_k = cos 2 pi k/5,
// s_k = sin 2 pi k/5), since w^4 and w^3 are the conjugates of w and w^2.
template <int DIR, typename T>
struct Dft<5, DIR, T> {
    static __device__ __forceinline__ void run(Cx<T> *a)
    {
        constexpr double c1d = c120(48), c2d = c120(96), s1d = s120(48), s2d = s120(96);
        const T c1 = T(c1d), c2 = T(c2d), s1 = T(DIR) * T(s1d), s2 = T(DIR) * T(s2d);
        const Cx<T> t1 = cadd(a[1], a[4]), t2 = cadd(a[2], a[3]), t3 = csub(a[1], a[4]), t4 = csub(a[2], a[3]);
        const Cx<T> m1 = {a[0].x + c1 * t1.x + c2 * t2.x, a[0].y + c1 * t1.y + c2 * t2.y};
        const Cx<T> m2 = {a[0].x + c2 * t1.x + c1 * t2.x, a[0].y + c2 * t1.y + c1 * t2.y};
        // i (s1 t3 + s2 t4) and i (s2 t3 - s1 t4)
        const Cx<T> n1 = {-(s1 * t3.y + s2 * t4.y), s1 * t3.x + s2 * t4.x};
        const Cx<T> n2 = {-(s2 * t3.y - s1 * t4.y), s2 * t3.x - s1 * t4.x};
        a[0] = cadd(a[0], cadd(t1, t2));
        a[1] = cadd(m1, n1);
        a[4] = csub(m1, n1);
        a[2] = cadd(m2, n2);
        a[3] = csub(m2, n2);
    }
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
