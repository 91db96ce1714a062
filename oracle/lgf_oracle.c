/*
 * CPU oracle for the LGF Poisson apply and the viscous integrating factor.
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, slow, FP64 C.  Only tests/, the smoke
 * check and the benchmark's CPU-baseline leg may load this library.  It shares
 * no code, header, table or constant generator with the CUDA path.
 *
 * What it computes (Liska & Colonius, arXiv:1604.01814):
 *   - e^{-z} I_n(z) by Miller's backward recurrence, normalised with
 *     e^{-z} (I_0(z) + 2 sum_{k>=1} I_k(z)) = 1 (the generating function of I_n
 *     at unit argument).                                        [App. A, Eq. lgf_intfac]
 *   - G_L(n) = -int_0^inf prod_i e^{-2t} I_{|n_i|}(2t) dt by adaptive
 *     Gauss-Kronrod (7/15) on doubling panels of [0, T] plus the term-by-term
 *     integral of the large-argument series of the three Bessel factors on
 *     [T, inf).                                                  [App. A, Eq. lgf_lap]
 *   - the far-field expansion G_L ~ -1/(4 pi r) + T3 + T5 + T7 (derivation in
 *     derive_asymptotic.py).                          [Sec. 2.2; App. A footnote]
 *   - u(n) = dx^2 sum_{m in D} G_L(n - m) f(m), direct summation with Neumaier
 *     compensation.                                        [Sec. 2.2, Eq. dpoisson_conv]
 *   - u = E(alpha) f with E(n) = prod_i e^{-2 alpha} I_{|n_i|}(2 alpha),
 *     untruncated, as three exact one-dimensional sums over a dense box.
 *                                    [Sec. 2.3 footnote; App. A, Eq. lgf_intfac]
 *   - G_K(alpha)(n) = -int_alpha^inf prod_i e^{-2t} I_{|n_i|}(2t) dt, split as
 *     G_L(n) + R(alpha)(n) with R(alpha)(n) = int_0^alpha (same integrand) dt
 *     by adaptive Gauss-Kronrod (7/15) on unit panels of [0, alpha].
 *                               [App. A, Eq. lgf_iflap and the partition of G_K]
 *
 * Parity pins for every function live in tests/test_oracle_pins.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.141592653589793238462643383279502884

/* ------------------------------------------------------------------------ */
/* Scaled modified Bessel functions e^{-z} I_k(z), k = 0..nmax.              */
/* ------------------------------------------------------------------------ */
int orc_ive_all(int nmax, double z, double *out)
{
    if (nmax < 0 || !(z >= 0.0) || out == NULL) return -1;
    if (z == 0.0) {
        for (int k = 0; k <= nmax; ++k) out[k] = (k == 0) ? 1.0 : 0.0;
        return 0;
    }
    /* Start far enough above both nmax and the bulk of the normalising sum:
       for large z the terms fall like exp(-k^2 / (2 z)). */
    int N = nmax + 40 + (int)(10.0 * sqrt(z));
    double ikp1 = 0.0, ik = 1e-300, sum = 0.0;
    for (int k = N; k >= 1; --k) {
        double ikm1 = (2.0 * k / z) * ik + ikp1; /* I_{k-1} = (2k/z) I_k + I_{k+1} */
        if (k <= nmax) out[k] = ik;
        sum += 2.0 * ik;
        ikp1 = ik;
        ik = ikm1;
        if (fabs(ik) > 1e250) { /* rescale everything kept so far */
            const double s = 1e-250;
            ik *= s; ikp1 *= s; sum *= s;
            for (int j = k; j <= nmax; ++j) out[j] *= s;
        }
    }
    /* ik now holds I_0 */
    sum += ik;
    out[0] = ik;
    for (int k = 0; k <= nmax; ++k) out[k] /= sum;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Gauss-Kronrod 7/15 rule (QUADPACK qk15 abscissae and weights).            */
/* ------------------------------------------------------------------------ */
static const double GK_X[8] = {
    0.991455371120812639206854697526329, 0.949107912342758524526189684047851,
    0.864864423359769072789712788640926, 0.741531185599394439863864773280788,
    0.586087235467691130294144845693013, 0.405845151377397166906606412076961,
    0.207784955007898467600689403773245, 0.000000000000000000000000000000000};
static const double GK_WK[8] = {
    0.022935322010529224963732008058970, 0.063092092629978553290700663189204,
    0.104790010322250183839876322541518, 0.140653259715525918745189590510238,
    0.169004726639267902826583426598550, 0.190350578064785409913256402421014,
    0.204432940075298892414161999234649, 0.209482141084727828012999174891714};
/* Gauss 7-point weights for the nodes GK_X[1], GK_X[3], GK_X[5], GK_X[7]. */
static const double GK_WG[4] = {
    0.129484966168869693270611432679082, 0.279705391489276667901467771423780,
    0.381830050505118944950369775488975, 0.417959183673469387755102040816327};

typedef double (*orc_fn)(double t, void *ctx);

static void gk15(orc_fn f, void *ctx, double a, double b, double *k15, double *g7)
{
    const double c = 0.5 * (a + b), h = 0.5 * (b - a);
    double fc = f(c, ctx);
    double sk = GK_WK[7] * fc, sg = GK_WG[3] * fc;
    for (int i = 0; i < 7; ++i) {
        double f1 = f(c - h * GK_X[i], ctx), f2 = f(c + h * GK_X[i], ctx);
        sk += GK_WK[i] * (f1 + f2);
        if (i & 1) sg += GK_WG[i >> 1] * (f1 + f2);
    }
    *k15 = sk * h;
    *g7 = sg * h;
}

/* Exposed for the quadrature-rule pin: integral of x^k over [-1, 1]. */
static double poly_fn(double t, void *ctx) { return pow(t, *(int *)ctx); }
int orc_gk15_poly(int k, double *k15, double *g7)
{
    gk15(poly_fn, &k, -1.0, 1.0, k15, g7);
    return 0;
}

/* Bisect until the Gauss-7 and Kronrod-15 values agree to tol.  The Kronrod
   value is kept; for analytic integrands its error is far below |K15 - G7|
   (roughly |K15 - G7|^{3/2}), so tol = 1e-11 of the result's scale leaves a
   per-panel error near 1e-16. */
static double adapt(orc_fn f, void *ctx, double a, double b, double tol, int depth)
{
    double k15, g7;
    gk15(f, ctx, a, b, &k15, &g7);
    if (fabs(k15 - g7) <= tol || depth >= 30) return k15;
    const double m = 0.5 * (a + b);
    return adapt(f, ctx, a, m, tol, depth + 1) + adapt(f, ctx, m, b, tol, depth + 1);
}

/* ------------------------------------------------------------------------ */
/* G_L by quadrature of the Bessel form.                                     */
/* ------------------------------------------------------------------------ */
typedef struct { int n[3]; int nmax; double *buf; } lgf_q;

static double lgf_integrand(double t, void *vctx)
{
    lgf_q *q = (lgf_q *)vctx;
    orc_ive_all(q->nmax, 2.0 * t, q->buf);
    return q->buf[q->n[0]] * q->buf[q->n[1]] * q->buf[q->n[2]];
}

/* Coefficients of e^{-z} I_n(z) ~ (2 pi z)^{-1/2} sum_k a_k z^{-k} (large z):
   a_k = (-1)^k prod_{j=1..k} (4n^2 - (2j-1)^2) / (k! 8^k). */
static void ive_series(int n, int K, double *a)
{
    const double mu = 4.0 * (double)n * (double)n;
    a[0] = 1.0;
    for (int k = 1; k <= K; ++k) {
        const double f = mu - (double)(2 * k - 1) * (double)(2 * k - 1);
        a[k] = -a[k - 1] * f / (8.0 * k);
    }
}

/* int_T^inf prod_i e^{-2t} I_{n_i}(2t) dt from the product of the three
   large-argument series (z = 2t):  (4 pi t)^{-3/2} sum_K C_K (2t)^{-K}. */
static double lgf_tail(const int n[3], double T)
{
    enum { K = 16 };
    double a[3][K + 1], ab[K + 1], c[K + 1];
    for (int i = 0; i < 3; ++i) ive_series(n[i], K, a[i]);
    for (int k = 0; k <= K; ++k) {
        ab[k] = 0.0;
        for (int j = 0; j <= k; ++j) ab[k] += a[0][j] * a[1][k - j];
    }
    for (int k = 0; k <= K; ++k) {
        c[k] = 0.0;
        for (int j = 0; j <= k; ++j) c[k] += ab[j] * a[2][k - j];
    }
    /* int_T^inf t^{-3/2} (2t)^{-k} dt = 2^{-k} T^{-k-1/2} / (k + 1/2) */
    double s = 0.0;
    for (int k = K; k >= 0; --k)
        s += c[k] * pow(2.0 * T, -(double)k) / (k + 0.5);
    return s * pow(4.0 * ORC_PI, -1.5) / sqrt(T);
}

double orc_lgf_quad(int n1, int n2, int n3)
{
    lgf_q q;
    q.n[0] = abs(n1); q.n[1] = abs(n2); q.n[2] = abs(n3);
    q.nmax = q.n[0];
    if (q.n[1] > q.nmax) q.nmax = q.n[1];
    if (q.n[2] > q.nmax) q.nmax = q.n[2];
    q.buf = (double *)malloc(sizeof(double) * (q.nmax + 1));
    if (!q.buf) return NAN;
    /* Past T the series of each factor converges fast: the term ratio is
       about n^2 / (2 z) <= 1/64 with z = 2T. */
    const double T = 16.0 * ((double)q.nmax * q.nmax + 8.0);
    const double scale = 1.0 / (4.0 * ORC_PI * (1.0 + sqrt((double)q.n[0] * q.n[0] + (double)q.n[1] * q.n[1] + (double)q.n[2] * q.n[2])));
    double s = 0.0, a = 0.0, b = 1.0;
    while (a < T) {
        if (b > T) b = T;
        s += adapt(lgf_integrand, &q, a, b, 1e-11 * scale, 0);
        a = b;
        b = 2.0 * b;
    }
    s += lgf_tail(q.n, T);
    free(q.buf);
    return -s;
}

/* ------------------------------------------------------------------------ */
/* G_K(alpha) = G_L + R(alpha), R(alpha)(n) = int_0^alpha G_E(t)(n) dt.      */
/* ------------------------------------------------------------------------ */
double orc_lgf_r(double alpha, int n1, int n2, int n3)
{
    if (!(alpha >= 0.0) || isinf(alpha)) return NAN;
    if (alpha == 0.0) return 0.0;
    lgf_q q;
    q.n[0] = abs(n1); q.n[1] = abs(n2); q.n[2] = abs(n3);
    q.nmax = q.n[0];
    if (q.n[1] > q.nmax) q.nmax = q.n[1];
    if (q.n[2] > q.nmax) q.nmax = q.n[2];
    q.buf = (double *)malloc(sizeof(double) * (q.nmax + 1));
    if (!q.buf) return NAN;
    /* same absolute scale as the G_L quadrature, so that G_K = G_L + R keeps
       the accuracy of G_L */
    const double scale = 1.0 / (4.0 * ORC_PI * (1.0 + sqrt((double)q.n[0] * q.n[0] + (double)q.n[1] * q.n[1] + (double)q.n[2] * q.n[2])));
    double s = 0.0;
    for (double a = 0.0; a < alpha; a += 1.0) {
        const double b = a + 1.0 < alpha ? a + 1.0 : alpha;
        s += adapt(lgf_integrand, &q, a, b, 1e-11 * scale, 0);
    }
    free(q.buf);
    return s;
}

double orc_gk_quad(double alpha, int n1, int n2, int n3)
{
    return orc_lgf_quad(n1, n2, n3) + orc_lgf_r(alpha, n1, n2, n3);
}

/* ------------------------------------------------------------------------ */
/* Far-field asymptotic expansion (monomials in X = n1^2, Y = n2^2, Z = n3^2). */
/* ------------------------------------------------------------------------ */
typedef struct { int a, b, c; double v; } mono;
static const mono T3M[] = {{2,0,0,-1}, {1,1,0,3}, {1,0,1,3}, {0,2,0,-1}, {0,1,1,3}, {0,0,2,-1}};
static const mono T5M[] = {{4,0,0,-23}, {3,1,0,244}, {3,0,1,244}, {2,2,0,-621}, {2,1,1,228}, {2,0,2,-621},
                           {1,3,0,244}, {1,2,1,228}, {1,1,2,228}, {1,0,3,244}, {0,4,0,-23}, {0,3,1,244},
                           {0,2,2,-621}, {0,1,3,244}, {0,0,4,-23}};
static const mono T7M[] = {{6,0,0,-647}, {5,1,0,16419}, {5,0,1,16419}, {4,2,0,-106536}, {4,1,1,15723},
                           {4,0,2,-106536}, {3,3,0,178221}, {3,2,1,74469}, {3,1,2,74469}, {3,0,3,178221},
                           {2,4,0,-106536}, {2,3,1,74469}, {2,2,2,-626835}, {2,1,3,74469}, {2,0,4,-106536},
                           {1,5,0,16419}, {1,4,1,15723}, {1,3,2,74469}, {1,2,3,74469}, {1,1,4,15723},
                           {1,0,5,16419}, {0,6,0,-647}, {0,5,1,16419}, {0,4,2,-106536}, {0,3,3,178221},
                           {0,2,4,-106536}, {0,1,5,16419}, {0,0,6,-647}};

static double mono_sum(const mono *m, int count, double X, double Y, double Z)
{
    double px[7], py[7], pz[7];   /* X^k, Y^k, Z^k for k <= 6 */
    px[0] = py[0] = pz[0] = 1.0;
    for (int k = 1; k < 7; ++k) {
        px[k] = px[k - 1] * X;
        py[k] = py[k - 1] * Y;
        pz[k] = pz[k - 1] * Z;
    }
    double s = 0.0;
    for (int i = 0; i < count; ++i)
        s += m[i].v * px[m[i].a] * py[m[i].b] * pz[m[i].c];
    return s;
}

/* order = 1, 3, 5 or 7: include terms up to |n|^-order. */
double orc_lgf_asym(int n1, int n2, int n3, int order)
{
    const double X = (double)n1 * n1, Y = (double)n2 * n2, Z = (double)n3 * n3;
    const double r2 = X + Y + Z, r = sqrt(r2);
    if (r2 == 0.0) return NAN;
    double g = -1.0 / (4.0 * ORC_PI * r);
    const double r6 = r2 * r2 * r2, r7 = r6 * r;
    if (order >= 3) g += mono_sum(T3M, 6, X, Y, Z) / (16.0 * ORC_PI * r7);
    if (order >= 5) g += mono_sum(T5M, 15, X, Y, Z) / (128.0 * ORC_PI * r7 * r6);
    if (order >= 7) g += mono_sum(T7M, 28, X, Y, Z) / (512.0 * ORC_PI * r7 * r6 * r6);
    return g;
}

/* ------------------------------------------------------------------------ */
/* Table of G_L over sorted offsets a >= b >= c >= 0, a <= R.                */
/* ------------------------------------------------------------------------ */
int64_t orc_table_index(int a, int b, int c)
{
    return (int64_t)a * (a + 1) * (a + 2) / 6 + (int64_t)b * (b + 1) / 2 + c;
}

int64_t orc_table_size(int R) { return orc_table_index(R + 1, 0, 0); }

int orc_lgf_table(int R, double *out)
{
    if (R < 0 || !out) return -1;
    const int64_t n = orc_table_size(R);
    int *abc = (int *)malloc(sizeof(int) * 3 * (size_t)n);
    if (!abc) return -2;
    for (int a = 0; a <= R; ++a)
        for (int b = 0; b <= a; ++b)
            for (int c = 0; c <= b; ++c) {
                int64_t i = orc_table_index(a, b, c);
                abc[3 * i] = a; abc[3 * i + 1] = b; abc[3 * i + 2] = c;
            }
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < n; ++i)
        out[i] = orc_lgf_quad(abc[3 * i], abc[3 * i + 1], abc[3 * i + 2]);
    free(abc);
    return 0;
}

/* Table of R(alpha) over the same sorted offsets (G_K = G_L table + this). */
int orc_r_table(double alpha, int R, double *out)
{
    if (R < 0 || !out || !(alpha >= 0.0)) return -1;
    const int64_t n = orc_table_size(R);
    int *abc = (int *)malloc(sizeof(int) * 3 * (size_t)n);
    if (!abc) return -2;
    for (int a = 0; a <= R; ++a)
        for (int b = 0; b <= a; ++b)
            for (int c = 0; c <= b; ++c) {
                int64_t i = orc_table_index(a, b, c);
                abc[3 * i] = a; abc[3 * i + 1] = b; abc[3 * i + 2] = c;
            }
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < n; ++i)
        out[i] = orc_lgf_r(alpha, abc[3 * i], abc[3 * i + 1], abc[3 * i + 2]);
    free(abc);
    return 0;
}

static inline void sort3(int *a, int *b, int *c)
{
    int t;
    if (*a < *b) { t = *a; *a = *b; *b = t; }
    if (*b < *c) { t = *b; *b = *c; *c = t; }
    if (*a < *b) { t = *a; *a = *b; *b = t; }
}

/* G_L(n): table when max|n_i| <= R, the order-7 expansion otherwise. */
double orc_lgf(const double *table, int R, int n1, int n2, int n3)
{
    int a = abs(n1), b = abs(n2), c = abs(n3);
    sort3(&a, &b, &c);
    if (a <= R) return table[orc_table_index(a, b, c)];
    return orc_lgf_asym(a, b, c, 7);
}

/* ------------------------------------------------------------------------ */
/* Direct-sum Poisson apply over block sets.                                 */
/* ------------------------------------------------------------------------ */
/* src_coords: [nsrc][3] block coordinates; block B holds lattice points
   b*B + [0,b)^3, values f[B][(z*b + y)*b + x].  tgt_pts: [ntgt][3] lattice
   points.  out[i] = dx^2 sum_m G_L(tgt_i - m) f(m). */
int orc_poisson_direct(int b, int nsrc, const int32_t *src_coords, const double *f,
                       int64_t ntgt, const int32_t *tgt_pts, double dx,
                       const double *table, int R, double *out)
{
    if (b <= 0 || nsrc < 0 || ntgt < 0) return -1;
    const int64_t b3 = (int64_t)b * b * b;
    /* compact the non-zero sources */
    int64_t nnz = 0;
    for (int64_t i = 0; i < (int64_t)nsrc * b3; ++i) nnz += (f[i] != 0.0);
    int32_t *pos = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)(nnz + 1));
    double *val = (double *)malloc(sizeof(double) * (size_t)(nnz + 1));
    if (!pos || !val) { free(pos); free(val); return -2; }
    int64_t k = 0;
    for (int s = 0; s < nsrc; ++s)
        for (int z = 0; z < b; ++z)
            for (int y = 0; y < b; ++y)
                for (int x = 0; x < b; ++x) {
                    double v = f[s * b3 + ((int64_t)z * b + y) * b + x];
                    if (v == 0.0) continue;
                    pos[3 * k] = src_coords[3 * s] * b + x;
                    pos[3 * k + 1] = src_coords[3 * s + 1] * b + y;
                    pos[3 * k + 2] = src_coords[3 * s + 2] * b + z;
                    val[k++] = v;
                }
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < ntgt; ++t) {
        const int tx = tgt_pts[3 * t], ty = tgt_pts[3 * t + 1], tz = tgt_pts[3 * t + 2];
        double s = 0.0, c = 0.0; /* Neumaier */
        for (int64_t m = 0; m < nnz; ++m) {
            const double term = orc_lgf(table, R, tx - pos[3 * m], ty - pos[3 * m + 1], tz - pos[3 * m + 2]) * val[m];
            const double t2 = s + term;
            if (fabs(s) >= fabs(term)) c += (s - t2) + term;
            else c += (term - t2) + s;
            s = t2;
        }
        out[t] = dx * dx * (s + c);
    }
    free(pos);
    free(val);
    return 0;
}

/* The same sum for nf fields on one source block set at once (the fields'
   values at a point share one evaluation of G_L): f [nf][nsrc][b^3],
   out [nf][ntgt].  Points where every field is zero are skipped.
   G_L depends only on (|n1|, |n2|, |n3|), so its values over the offsets the
   targets and sources span are taken once from orc_lgf into a dense table
   (the same numbers; skipped when the table would exceed 2^26 entries).  Each
   field is summed with compensation: the exact rounding error of every
   addition is formed by Knuth's TwoSum (branch-free, the same error that the
   Neumaier branches form) and the errors are added up beside the sum. */
int orc_poisson_direct_multi(int b, int nsrc, const int32_t *src_coords, int nf, const double *f,
                             int64_t ntgt, const int32_t *tgt_pts, double dx,
                             const double *table, int R, double *out)
{
    if (b <= 0 || nsrc < 0 || ntgt < 0 || nf < 1 || nf > 64) return -1;
    const int64_t b3 = (int64_t)b * b * b;
    const int64_t npts = (int64_t)nsrc * b3;
    int64_t nnz = 0;
    for (int64_t i = 0; i < npts; ++i) {
        int any = 0;
        for (int j = 0; j < nf; ++j) any |= (f[j * npts + i] != 0.0);
        nnz += any;
    }
    int32_t *pos = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)(nnz + 1));
    double *val = (double *)malloc(sizeof(double) * (size_t)nf * (size_t)(nnz + 1));
    if (!pos || !val) { free(pos); free(val); return -2; }
    int64_t k = 0;
    for (int s = 0; s < nsrc; ++s)
        for (int z = 0; z < b; ++z)
            for (int y = 0; y < b; ++y)
                for (int x = 0; x < b; ++x) {
                    const int64_t i = s * b3 + ((int64_t)z * b + y) * b + x;
                    int any = 0;
                    for (int j = 0; j < nf; ++j) any |= (f[j * npts + i] != 0.0);
                    if (!any) continue;
                    pos[3 * k] = src_coords[3 * s] * b + x;
                    pos[3 * k + 1] = src_coords[3 * s + 1] * b + y;
                    pos[3 * k + 2] = src_coords[3 * s + 2] * b + z;
                    for (int j = 0; j < nf; ++j) val[k * nf + j] = f[j * npts + i];
                    ++k;
                }
    /* largest |offset| per axis between any target and any source point */
    int64_t ext[3] = {0, 0, 0};
    if (nnz > 0 && ntgt > 0)
        for (int d = 0; d < 3; ++d) {
            int32_t slo = pos[d], shi = pos[d], tlo = tgt_pts[d], thi = tgt_pts[d];
            for (int64_t m = 1; m < nnz; ++m) {
                if (pos[3 * m + d] < slo) slo = pos[3 * m + d];
                if (pos[3 * m + d] > shi) shi = pos[3 * m + d];
            }
            for (int64_t t = 1; t < ntgt; ++t) {
                if (tgt_pts[3 * t + d] < tlo) tlo = tgt_pts[3 * t + d];
                if (tgt_pts[3 * t + d] > thi) thi = tgt_pts[3 * t + d];
            }
            const int64_t a1 = (int64_t)thi - slo, a2 = (int64_t)shi - tlo;
            const int64_t m1 = a1 < 0 ? -a1 : a1, m2 = a2 < 0 ? -a2 : a2;
            ext[d] = (m1 > m2 ? m1 : m2) + 1;
        }
    double *gd = NULL;
    const int64_t ngd = ext[0] * ext[1] * ext[2];
    if (ngd > 0 && ngd <= ((int64_t)1 << 26)) {
        gd = (double *)malloc(sizeof(double) * (size_t)ngd);
        if (gd) {
#pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < ngd; ++i)
                gd[i] = orc_lgf(table, R, (int)(i % ext[0]), (int)((i / ext[0]) % ext[1]),
                                (int)(i / (ext[0] * ext[1])));
        }
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < ntgt; ++t) {
        const int tx = tgt_pts[3 * t], ty = tgt_pts[3 * t + 1], tz = tgt_pts[3 * t + 2];
        double sum[64], cmp[64];
        for (int j = 0; j < nf; ++j) sum[j] = cmp[j] = 0.0;
        for (int64_t m = 0; m < nnz; ++m) {
            const int d0 = abs(tx - pos[3 * m]), d1 = abs(ty - pos[3 * m + 1]), d2 = abs(tz - pos[3 * m + 2]);
            const double g = gd ? gd[((int64_t)d2 * ext[1] + d1) * ext[0] + d0] : orc_lgf(table, R, d0, d1, d2);
            const double *v = val + m * nf;
            for (int j = 0; j < nf; ++j) {
                const double term = g * v[j];
                const double s2 = sum[j] + term;       /* TwoSum: s2 + e == sum + term exactly */
                const double bv = s2 - sum[j];
                const double e = (sum[j] - (s2 - bv)) + (term - bv);
                sum[j] = s2;
                cmp[j] += e;
            }
        }
        for (int j = 0; j < nf; ++j) out[j * ntgt + t] = dx * dx * (sum[j] + cmp[j]);
    }
    free(gd);
    free(pos);
    free(val);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Integrating factor.                                                       */
/* ------------------------------------------------------------------------ */
int orc_intfactor_weights(double alpha, int nmax, double *w)
{
    if (!(alpha >= 0.0)) return -1;
    return orc_ive_all(nmax, 2.0 * alpha, w);
}

/* u = E(alpha) f on a dense nx*ny*nz box (x fastest), every offset kept. */
int orc_intfactor_box(double alpha, int nx, int ny, int nz, const double *f, double *u)
{
    if (nx <= 0 || ny <= 0 || nz <= 0) return -1;
    int nmax = nx;
    if (ny > nmax) nmax = ny;
    if (nz > nmax) nmax = nz;
    double *w = (double *)malloc(sizeof(double) * (size_t)nmax);
    const size_t n = (size_t)nx * ny * nz;
    double *t1 = (double *)malloc(sizeof(double) * n);
    double *t2 = (double *)malloc(sizeof(double) * n);
    if (!w || !t1 || !t2) { free(w); free(t1); free(t2); return -2; }
    orc_intfactor_weights(alpha, nmax - 1, w);
#pragma omp parallel for collapse(2)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                double s = 0.0;
                for (int m = 0; m < nx; ++m) s += w[abs(x - m)] * f[((size_t)z * ny + y) * nx + m];
                t1[((size_t)z * ny + y) * nx + x] = s;
            }
#pragma omp parallel for collapse(2)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                double s = 0.0;
                for (int m = 0; m < ny; ++m) s += w[abs(y - m)] * t1[((size_t)z * ny + m) * nx + x];
                t2[((size_t)z * ny + y) * nx + x] = s;
            }
#pragma omp parallel for collapse(2)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                double s = 0.0;
                for (int m = 0; m < nz; ++m) s += w[abs(z - m)] * t2[((size_t)m * ny + y) * nx + x];
                u[((size_t)z * ny + y) * nx + x] = s;
            }
    free(w); free(t1); free(t2);
    return 0;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
