/*
 * lgf.h -- C ABI of the GB300 lattice-Green's-function library.
 *
 * Operations (Liska & Colonius, "A fast immersed boundary method for external
 * incompressible viscous flows using lattice Green's functions",
 * arXiv:1604.01814):
 *
 *   Poisson apply   u(n) = dx^2 * sum_{m in D} G_L(n - m) f(m)
 *                   -- the solution of the discrete 7-point Poisson problem
 *                   L u = f with supp(f) in D, evaluated as the lattice
 *                   convolution of Sec. 2.2, Eq. dpoisson / dpoisson_conv.
 *                   G_L is the LGF of the 7-point Laplacian, App. A, Eq. lgf_lap:
 *                   G_L(n) = -int_0^inf prod_i e^{-2t} I_{|n_i|}(2t) dt.
 *   Integrating     u(n) = sum_m E_alpha(n - m) f(m),
 *   factor          E_alpha(n) = prod_i e^{-2 alpha} I_{|n_i|}(2 alpha)
 *                   -- the solution operator exp(alpha L) of the discrete heat
 *                   equation (Sec. 2.3 footnote; App. A, Eq. lgf_intfac).
 *
 * Sources and targets live on the active blocks of a block-structured lattice
 * (Sec. 4.1): a block set lists block coordinates B, and block B with edge b
 * covers the lattice points b*B + [0, b)^3.  Sources outside the source block
 * set are exactly zero (the truncation of Table 1); results are produced on
 * the target block set only.
 *
 * Conventions shared by every entry point
 *   - Every call returns an lgf_status; nothing aborts.  On failure the
 *     context keeps a message readable with lgf_last_error().  Calls on one
 *     context are not thread safe (use one context per host thread).
 *   - Field layout: [nrhs][ncomp][nblocks][b^3], x fastest inside a block
 *     (index ((r*ncomp + c)*nblocks + k)*b^3 + (z*b + y)*b + x).  The element
 *     type is float for LGF_F32 contexts and double for LGF_F64 contexts.
 *   - Device pointers must stay valid until the stream reaches the work.  The
 *     caller owns every buffer it passes; the library owns its context memory
 *     (tables, spectra, plans, scratch) and frees it in lgf_ctx_destroy().
 *   - Block lists are host arrays; they are read during the call and copied
 *     into cached plans, so the caller may free them when the call returns.
 *   - Outputs are overwritten, never accumulated.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Work is enqueued asynchronously on it.
 */
#ifndef LGF_H
#define LGF_H

#include <stdint.h>

#if defined(__GNUC__)
#define LGF_API __attribute__((visibility("default")))
#else
#define LGF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lgf_ctx lgf_ctx;

typedef enum {
    LGF_OK = 0,
    LGF_EINVAL = 1,        /* bad argument: null pointer, size, duplicate block, ... */
    LGF_ENOMEM = 2,        /* device or host allocation failed */
    LGF_ECUDA = 3,         /* a CUDA runtime call or kernel launch failed */
    LGF_ETIMEOUT = 4,      /* a bounded device-side wait ran out */
    LGF_EUNSUPPORTED = 5,  /* a size beyond the library's limits */
    LGF_ENOTABLE = 6       /* lgf_table_build has not covered the offsets needed */
} lgf_status;

typedef enum { LGF_F32 = 0, LGF_F64 = 1 } lgf_prec;

/* A block set: `nblocks` distinct block coordinates (x, y, z), host memory. */
typedef struct {
    int32_t b;               /* block edge in lattice points: 4, 8, 16, 32 or 64 */
    int32_t nblocks;         /* >= 0 */
    const int32_t *coords;   /* [nblocks][3], host pointer */
} lgf_blockset;

/* Context options.  Zero fields take the defaults noted. */
typedef struct {
    double tol;              /* target relative accuracy; default 1e-7 (F32), 1e-13 (F64).
                                Sets the E_alpha truncation radius. */
    int32_t prec;            /* lgf_prec of every field passed to this context */
    int32_t table_radius;    /* G_L by quadrature for max|n_i| <= table_radius, by the
                                far-field expansion beyond; default 48, range 8..96 */
    int32_t stencil_radius;  /* fixed E_alpha truncation radius; 0 = from tol */
    int32_t device;          /* CUDA device ordinal used by this context */
    int32_t flags;           /* LGF_FLAG_* below; 0 = defaults */
    int32_t reserved[3];     /* must be zero */
} lgf_options;

/* Stage the integrating factor's z pass with bulk asynchronous copies (the
   TMA engine's cp.async.bulk, double-buffered in a persistent kernel, waits
   bounded) instead of per-thread 16-byte loads.  Off by default: on the
   measured workloads the per-thread loads were faster. */
#define LGF_FLAG_BULK_STAGING 1

/* Execution of lgf_batch_apply where the autotuner has not chosen one for
   the batch's shape: by default the ragged mode (one launch per pass and
   transform length across the batch's Poisson parts) when the batch has two
   or more Poisson parts, per-problem launches otherwise.  BATCH_RAGGED asks
   for the ragged mode also with one Poisson part; BATCH_PER_PROBLEM for
   per-problem launches always (not both). */
#define LGF_FLAG_BATCH_RAGGED 2
#define LGF_FLAG_BATCH_PER_PROBLEM 4

/* Create a context on opt->device (NULL opt = defaults, device 0).
   Errors: LGF_EINVAL (bad option), LGF_ECUDA, LGF_ENOMEM. */
LGF_API lgf_status lgf_ctx_create(lgf_ctx **out, const lgf_options *opt);

/* Free every resource of the context (synchronises the device first). */
LGF_API lgf_status lgf_ctx_destroy(lgf_ctx *ctx);

/* Build the FP64 G_L table on the GPU: quadrature of the Bessel form of
   App. A, Eq. lgf_lap, for sorted offsets |n1| >= |n2| >= |n3| up to
   table_radius, with the far-field expansion -1/(4 pi |n|) + O(|n|^-3)
   (Sec. 2.2 and App. A footnote) beyond.  The table is computed once per
   context, a pre-processing step as in App. A.  `max_offset` (>= 0) is the
   largest per-axis lattice offset the caller expects; the quadrature radius
   is min(table_radius, max(max_offset, 24)), since the expansion is accurate
   to 1e-9 relative beyond 24.  A later call with a larger max_offset extends
   the table.  Synchronous with respect to `stream`.
   Errors: LGF_EINVAL, LGF_ECUDA, LGF_ENOMEM. */
LGF_API lgf_status lgf_table_build(lgf_ctx *ctx, int32_t max_offset, void *stream);

/* Report the table: quadrature radius and the largest relative mismatch
   between quadrature and expansion on the shell table_radius-3..table_radius
   (the near/far matching check).  Either pointer may be NULL.
   Errors: LGF_ENOTABLE before lgf_table_build. */
LGF_API lgf_status lgf_table_info(lgf_ctx *ctx, int32_t *table_radius, double *shell_mismatch);

/* G_L at `n` integer offsets: offsets_dev [n][3] int32 (device), out_dev [n]
   double (device).  Uses the table inside its radius and the expansion
   outside, exactly as the Poisson apply does.  Errors: LGF_ENOTABLE, LGF_EINVAL. */
LGF_API lgf_status lgf_table_lookup(lgf_ctx *ctx, const int32_t *offsets_dev, int64_t n, double *out_dev,
                            void *stream);

/* Poisson apply (Sec. 2.2, Eq. dpoisson_conv):
     u[r][c][t] = dx^2 * sum_{s in src} G_L(n_t - m_s) f[r][c][s]
   for every target point n_t of `tgt` and every rhs r < nrhs, component
   c < ncomp (each component is an independent scalar convolution with the
   same kernel).  f_dev: [nrhs][ncomp][src.nblocks][b^3]; u_dev:
   [nrhs][ncomp][tgt.nblocks][b^3].  src.b must equal tgt.b.  The result is
   the exact convolution up to floating-point rounding (no far-field
   approximation).  Errors: LGF_EINVAL (null pointers, b mismatch, duplicate
   blocks, nblocks == 0 is allowed and writes nothing / zeros),
   LGF_EUNSUPPORTED (extent beyond 2048 lattice points per axis),
   LGF_ENOTABLE, LGF_ENOMEM, LGF_ECUDA. */
LGF_API lgf_status lgf_poisson_apply(lgf_ctx *ctx, const lgf_blockset *src, const lgf_blockset *tgt,
                             const void *f_dev, void *u_dev, int32_t ncomp, int32_t nrhs, double dx,
                             void *stream);

/* G_K(alpha) at `n` integer offsets (App. A, Eq. lgf_iflap):
     G_K(alpha)(n) = -int_alpha^inf prod_i e^{-2t} I_{|n_i|}(2t) dt
                   = G_L(n) + R(alpha)(n),  R(alpha)(n) = int_0^alpha (same) dt,
   the kernel of K(alpha)^{-1} = [E(-alpha) L]^{-1} (Sec. 2.2).  The context
   builds one FP64 table per alpha on first use: R(alpha) by Gauss-Legendre
   quadrature on the GPU over the offsets of the G_L table, added to it;
   beyond the table radius the G_L expansion is used, and the build fails with
   LGF_EUNSUPPORTED when R(alpha) on the table's outer shell exceeds
   2.5e-16 (alpha too large for the radius: build a larger table).  alpha = 0
   gives G_L.  offsets_dev [n][3] int32 and out_dev [n] double are device
   pointers.  Errors: LGF_ENOTABLE, LGF_EINVAL (alpha < 0 or not finite),
   LGF_EUNSUPPORTED (alpha > 64 or the shell check), LGF_ENOMEM, LGF_ECUDA. */
LGF_API lgf_status lgf_kinv_lookup(lgf_ctx *ctx, double alpha, const int32_t *offsets_dev, int64_t n,
                                   double *out_dev, void *stream);

/* K(alpha)^{-1} apply (Sec. 2.2, the action of [E(-alpha) L]^{-1} through the
   LGF G_K(alpha) of App. A):
     u[r][c][t] = dx^2 * sum_{s in src} G_K(alpha)(n_t - m_s) f[r][c][s]
   with the layouts, engine and errors of lgf_poisson_apply (only the kernel
   spectrum differs; it is cached per transform shape and alpha).  alpha = 0
   equals lgf_poisson_apply. */
LGF_API lgf_status lgf_kinv_apply(lgf_ctx *ctx, double alpha, const lgf_blockset *src, const lgf_blockset *tgt,
                                  const void *f_dev, void *u_dev, int32_t ncomp, int32_t nrhs, double dx,
                                  void *stream);

/* Integrating-factor apply (Sec. 2.3 footnote; App. A, Eq. lgf_intfac):
     u[r][c][t] = sum_{s in src} E_alpha(n_t - m_s) f[r][c][s],  alpha >= 0,
   with E_alpha truncated at the radius R where the 1-D factor falls below
   tol/8 of its central value (or at opt.stencil_radius).  Same layouts as
   lgf_poisson_apply.  alpha = 0 copies sources onto coinciding targets.
   Errors: LGF_EINVAL (alpha < 0 or not finite, ...), LGF_EUNSUPPORTED
   (alpha so large that the radius would exceed 128), LGF_ENOMEM, LGF_ECUDA. */
LGF_API lgf_status lgf_intfactor_apply(lgf_ctx *ctx, double alpha, const lgf_blockset *src, const lgf_blockset *tgt,
                               const void *f_dev, void *u_dev, int32_t ncomp, int32_t nrhs, void *stream);

/* The 1-D factor e^{-2 alpha} I_n(2 alpha), n = 0..R, that lgf_intfactor_apply
   uses (FP64, computed on the GPU by Miller's recurrence); w_dev holds cap
   doubles; *radius receives R.  Errors: LGF_EINVAL (cap <= R). */
LGF_API lgf_status lgf_intfactor_weights(lgf_ctx *ctx, double alpha, double *w_dev, int32_t cap, int32_t *radius,
                                 void *stream);

/* Batched applies.  Operations: */
enum { LGF_OP_POISSON = 0, LGF_OP_INTFACTOR = 1, LGF_OP_POISSON_THEN_INTFACTOR = 2, LGF_OP_KINV = 3 };

typedef struct {
    lgf_blockset src, tgt;   /* as in lgf_poisson_apply; for POISSON_THEN_INTFACTOR
                                the integrating factor maps tgt -> tgt */
    const void *f_dev;       /* [nrhs][ncomp][src.nblocks][b^3] */
    void *u_dev;             /* [nrhs][ncomp][tgt.nblocks][b^3] */
    int32_t ncomp, nrhs;
    int32_t op;              /* LGF_OP_* */
    int32_t reserved;        /* must be zero */
    double alpha, dx;
} lgf_problem;

/* Apply `nprob` independent problems (the per-stage right-hand sides of
   Sec. 2.3 and many uneven block-adaptive problems) as one batch.  All plans,
   spectra and weights are prepared first.  Integrating factors on the same
   block sets with the same field count form one group that runs as one
   launch per pass (up to 8 problems per launch, different alphas and buffers
   allowed).  The Poisson parts (each with its own integrating factor when no
   other problem shares its group) and the groups that read only batch inputs
   are independent units.  With per-problem launches they are spread over up
   to 4 concurrent branches
   (8 when the autotuner finds that faster)
   (context streams forked from and joined back to the caller's stream, each
   with its own scratch), longest first onto the least loaded branch.
   Groups of several
   POISSON_THEN_INTFACTOR problems run after the branches join.  In the
   ragged mode (see LGF_FLAG_BATCH_RAGGED) the Poisson parts of all
   problems instead run together: one launch per pass and transform length
   (each CTA finds its problem in a job table passed with the launch, up to
   64 problems per launch), the lengths of a pass on 2 concurrent branches
   (4 when the autotuner finds that faster),
   every part with its own slice of one scratch; the integrating-factor
   groups that read Poisson results follow, their jobs of all block sets
   together in one launch per pass (and block edge and stencil radius
   class); the groups that read only batch inputs run likewise on a branch
   alongside the Poisson passes.  The autotuner times both modes.  On a
   non-default stream the whole batch is captured once into a CUDA graph,
   and later calls with an identical batch (same block lists, pointers,
   alphas, stream) replay it; the context keeps the graphs of the 8 most
   recently used batches (so, e.g., double-buffered batches alternate
   without recapture).  u buffers must not alias one another or any f
   buffer of the same batch.  POISSON_THEN_INTFACTOR writes
   E_alpha(G_L * f) into u_dev; KINV writes dx^2 G_K(alpha) * f (alpha is
   the kernel's, no integrating factor follows).  Results equal those of the single applies
   bit for bit.  Errors: as the single applies. */
LGF_API lgf_status lgf_batch_apply(lgf_ctx *ctx, const lgf_problem *probs, int32_t nprob, void *stream);

/* Staggered-grid curl C: faces -> edges (Sec. 2.1, operator list).  Cell n
   holds face k at (n + (1 - e_k)/2) dx and edge k at (n + e_k/2) dx; with
   (k, i, j) cyclic,
     w_k(n) = ([u_j(n) - u_j(n - e_i)] - [u_i(n) - u_i(n - e_j)]) / dx
   at every cell of `tgt`, u read on `src` and zero elsewhere.  u_dev:
   [nrhs][3][src.nblocks][b^3], w_dev: [nrhs][3][tgt.nblocks][b^3], context
   precision, component k of cell n in the cell's slot.  The paper lists C but
   prints no stencil: this is the second-order finite-volume one, which
   satisfies the mimetic identity L_F = -G G^dagger - C^dagger C of Sec. 2.1.
   Errors: LGF_EINVAL (b mismatch, null pointers, dx <= 0), LGF_ENOMEM,
   LGF_ECUDA. */
LGF_API lgf_status lgf_curl(lgf_ctx *ctx, const lgf_blockset *src, const lgf_blockset *tgt, const void *u_dev,
                            void *w_dev, int32_t nrhs, double dx, void *stream);

/* Adjoint curl C^dagger: edges -> faces, the transpose of lgf_curl under the
   sum over cells:
     u_k(n) = -([w_j(n) - w_j(n + e_i)] - [w_i(n) - w_i(n + e_j)]) / dx.
   Same layouts and errors as lgf_curl (w on `src`, u on `tgt`). */
LGF_API lgf_status lgf_curl_adjoint(lgf_ctx *ctx, const lgf_blockset *src, const lgf_blockset *tgt,
                                    const void *w_dev, void *u_dev, int32_t nrhs, double dx, void *stream);

/* Velocity refresh (Sec. 4.1, Eq. vel_refresh): w = C u on the source blocks,
   s = L^{-1} w = dx^2 G_L * w (each edge component a scalar convolution, the
   exact box convolution of lgf_poisson_apply) on the target blocks and their
   +x, +y, +z neighbours, and u_out = -C^dagger s on the target blocks.  The
   printed composition C^dagger L^{-1} C returns -u for a divergence-free u
   under the paper's L_F = -G G^dagger - C^dagger C; the minus sign is the
   reading that refreshes u.  u_dev: [nrhs][3][src.nblocks][b^3] (zero
   outside the source blocks); u_out_dev: [nrhs][3][tgt.nblocks][b^3].  The
   result does not depend on dx.  Errors: as lgf_poisson_apply and lgf_curl. */
LGF_API lgf_status lgf_velocity_refresh(lgf_ctx *ctx, const lgf_blockset *src, const lgf_blockset *tgt,
                                        const void *u_dev, void *u_out_dev, int32_t nrhs, double dx, void *stream);

/* One IF-HERK stage's linear solve by the nested projection of Sec. 3.1,
   Eq. nested_proj (the operator-block LU of Eq. ibifherk_linsys_full):
     ip:  L_C d* = -G^dagger r                       (Dbar = -G^dagger)
     f :  C f_hat = I^i H [r - G d*] - u_Gamma,      f_hat = W2 (W1 rhs)
     pc:  d_hat = d* + L_C^{-1} G^dagger (I^{i-1})^dagger f_hat
     vc:  u = H [r - G d_hat - (I^{i-1})^dagger f_hat]
   with H = E(alpha) (the stage's integrating factor, Eq. ibifherk_aux_1:
   alpha = (c_i - c_{i-1}) dt / (dx^2 Re)), L_C^{-1} = dx^2 G_L * (the
   Poisson engine), G and Dbar the staggered gradient and divergence of
   Sec. 2.1 (cell n holds face k at (n + (1 - e_k)/2) dx:
   (G q)_k(n) = [q(n) - q(n - e_k)] / dx, (Dbar u)(n) = sum_k [u_k(n + e_k)
   - u_k(n)] / dx), I = dx^3 R^dagger and I^dagger = dx^3 R the IB operators
   of lgf_ib_interp / lgf_ib_spread at the markers of stage i and i-1.  The
   force Schur complement C is not formed: the caller passes the factors of
   its inverse (Sec. 3.2 stores W = L^{-1} from the Cholesky factor of C, so
   C^{-1} = W^T W: pass W1 = W, W2 = NULL; a moving body, whose C is not
   symmetric, passes any two factors with C^{-1} = W2 W1).
   Printed readings: Eq. nested_proj-f prints H_C [r - G^dagger d*]; the face
   field r - G d* under the face operator H is the reading that follows from
   Eq. nested_proj_naive.
   Regions (the truncation of Table 1): every field lives on the one block
   set `flow` (D); r is zero outside D; every Poisson problem has its sources
   on the cells of D and its results on D and its -x, -y, -z neighbour blocks
   (the cells G reads); H maps D to D; the IB operators act on the faces of D.
   The GPU forms d_hat as L_C^{-1} Dbar (r - (I^{i-1})^dagger f_hat), equal to
   pc by linearity.  Layouts: r_dev, u_dev [3][nD][b^3]; d_dev [nD][b^3]
   (d_hat on the cells of D; may be NULL); X_prev_dev, X_dev [nm][3] double in
   units of dx (device); ub_dev and f_dev [3][nm]; W1_dev, W2_dev [3nm][3nm]
   row-major, rows and columns in the [3][nm] order.  Fields, ub, W and f in
   the context precision.  nmarkers = 0 gives the plain projection
   u = H [r - G d*].  Errors: LGF_EINVAL, LGF_ENOTABLE, LGF_EUNSUPPORTED,
   LGF_ENOMEM, LGF_ECUDA. */
typedef struct {
    lgf_blockset flow;          /* D */
    int64_t nmarkers;           /* nm >= 0 */
    const double *X_prev_dev;   /* markers of stage i-1 (I^{i-1}) */
    const double *X_dev;        /* markers of stage i (I^i) */
    const void *ub_dev;         /* u_Gamma at stage i */
    const void *W1_dev;         /* first factor of C^{-1} */
    const void *W2_dev;         /* second factor, or NULL for W1^T */
    const void *r_dev;          /* right-hand side r_k^i (faces of D) */
    void *u_dev;                /* u_k^i (faces of D) */
    void *d_dev;                /* pressure d_hat (cells of D) or NULL */
    void *f_dev;                /* marker forces f_hat or NULL */
    double alpha, dx;
    int32_t reserved[4];        /* must be zero */
} lgf_stage;

LGF_API lgf_status lgf_nested_projection_stage(lgf_ctx *ctx, const lgf_stage *stage, void *stream);

/* Immersed-boundary regularisation R (Sec. 2.1):
     f^k(n) = dx^-3 sum_i g^k(i) prod_d phi(x_F^k(n)_d - X_i,d)
   on the face lattices of `set` (face k of cell n at n + (1 - e_k)/2, in
   units of dx), with the three-point kernel phi(r) = (1 + sqrt(1 - 3 r^2)) / 3
   for |r| <= 1/2, (5 - 3|r| - sqrt(1 - 3 (1 - |r|)^2)) / 6 for
   1/2 <= |r| <= 3/2, 0 beyond (the paper cites a smoothed three-point kernel
   without printing it; this is the Roma-Peskin-Berger one).  X_dev:
   [nmarkers][3] double, marker positions in units of dx; g_dev:
   [nrhs][3][nmarkers]; f_dev: [nrhs][3][set.nblocks][b^3] (overwritten;
   points outside the set are dropped).  Context precision for g and f.  The
   additions are atomic, so the last bits vary between runs.  Errors:
   LGF_EINVAL, LGF_EUNSUPPORTED (bounding box of the set above 2^26 blocks),
   LGF_ENOMEM, LGF_ECUDA. */
LGF_API lgf_status lgf_ib_spread(lgf_ctx *ctx, const lgf_blockset *set, int64_t nmarkers, const double *X_dev,
                                 const void *g_dev, void *f_dev, int32_t nrhs, double dx, void *stream);

/* Immersed-boundary interpolation I = dx^3 R^dagger (Sec. 2.1):
     U^k(i) = sum_n v^k(n) prod_d phi(x_F^k(n)_d - X_i,d)
   (dx^3 delta_dx is the bare product of phi, so dx does not enter).  v_dev:
   [nrhs][3][set.nblocks][b^3] (absent blocks read as zero); U_dev:
   [nrhs][3][nmarkers].  Deterministic.  Errors: as lgf_ib_spread. */
LGF_API lgf_status lgf_ib_interp(lgf_ctx *ctx, const lgf_blockset *set, int64_t nmarkers, const double *X_dev,
                                 const void *v_dev, void *U_dev, int32_t nrhs, void *stream);

/* FP64 residual check of the discrete Poisson problem (Sec. 2.2, Eq. dpoisson):
     r = (L_h u)(n) - f(n),  L_h u = (sum_{+-e_i} u(n +- e) - 6 u(n)) / dx^2,
   at every point of `set` whose six neighbours are in `set`; r = 0 elsewhere.
   u_dev, f_dev: one field each on `set` in the context precision (f is the
   source restricted to `set`: zero where the source set has no block);
   r_dev: [set.nblocks][b^3] double.  *max_abs (host, may be NULL) receives
   max |r| over the checked points and *max_f the largest |f| (for relative
   reporting).  Synchronous.  Errors: LGF_EINVAL, LGF_ECUDA, LGF_ENOMEM. */
LGF_API lgf_status lgf_residual(lgf_ctx *ctx, const lgf_blockset *set, const void *u_dev, const void *f_dev,
                        double dx, double *r_dev, double *max_abs, double *max_f, void *stream);

/* Per-kernel timing.  While enabled, every kernel the context launches is
   bracketed by two CUDA events recorded on its launch stream, and
   lgf_batch_apply runs without a CUDA graph (direct launches).  Enabling or
   disabling synchronises the device and clears the statistics. */
LGF_API lgf_status lgf_profile_enable(lgf_ctx *ctx, int32_t enable);

typedef struct {
    char name[48];           /* kernel role, e.g. "poisson_z_convolve" */
    int64_t launches;        /* launches since the last read */
    double total_ms;         /* summed event-to-event time of those launches */
} lgf_kernel_stat;

/* Synchronise the device, fold the recorded events into per-kernel totals,
   copy up to `cap` of them into `out` (host), set *n to the number of kernels
   seen, and reset the totals. */
LGF_API lgf_status lgf_profile_read(lgf_ctx *ctx, lgf_kernel_stat *out, int32_t cap, int32_t *n);

/* Cache state of a context (host-side bookkeeping; no device work).
   The context caches plans (block maps and neighbour tables per block-set
   pair), kernel spectra (per transform shape and kernel) and the CUDA graphs
   of recent batches.  A captured graph holds the device addresses of the
   scratch buffers, plans and spectra it was captured with, so every cached
   graph is destroyed whenever any such buffer is freed or reallocated
   (scratch growth, an eviction, a table rebuild); `generation` counts those
   invalidations and a later batch is captured afresh.  Plan and spectrum
   caches are bounded (least recently used evicted first, never an entry the
   running call uses), so an active set that changes every step (Sec. 4.1)
   does not grow device memory without bound. */
typedef struct {
    int64_t graphs_cached;      /* captured batch graphs held now */
    int64_t poisson_plans, intfactor_plans, curl_plans, ib_plans;
    int64_t spectra;            /* kernel spectra held now */
    int64_t generation;         /* graph-cache invalidations so far */
    int64_t graphs_dropped;     /* graphs destroyed (invalidation or LRU bound) */
    int64_t evictions;          /* plans and spectra released by the LRU bounds */
    int64_t scratch_reallocs;   /* scratch buffers (re)allocated */
    int64_t scratch_bytes;      /* bytes of scratch held now */
    int64_t reserved[5];
} lgf_stats;

/* Fill *out with the context's cache state.  Errors: LGF_EINVAL (null). */
LGF_API lgf_status lgf_ctx_stats(lgf_ctx *ctx, lgf_stats *out);

/* Set the cache bounds: max_plans (per plan kind, >= 1; default 256 Poisson
   and integrating-factor plans, 64 curl and IB plans), max_spectra (>= 1,
   default 32) and max_graphs (>= 0, default 8; 0 runs every batch with direct
   launches).  -1 keeps a bound.  Lowering a bound takes effect at the next
   insertion.  Changing max_graphs drops the cached graphs.
   Errors: LGF_EINVAL. */
LGF_API lgf_status lgf_cache_limits(lgf_ctx *ctx, int32_t max_plans, int32_t max_spectra, int32_t max_graphs);

/* A-posteriori error estimate of a Poisson result (the diagnostic of the
   scope table's boundary): at `nsample` target points spread evenly over the
   target blocks, the exact sum dx^2 sum_m G_L(n - m) f(m) of Sec. 2.2,
   Eq. dpoisson_conv, is formed in FP64 on the GPU (one CTA per point over
   every source point, G_L from the context's table and expansion), and
   *max_rel_err (host) receives the largest over the fields of
   max |u - exact| / max |exact| at those points.  f_dev and u_dev are as in
   lgf_poisson_apply (u its result).  Cost: nsample x sources FP64 terms per
   field.  Synchronous.  Errors: as lgf_poisson_apply; LGF_EINVAL (nsample
   outside 1..65536). */
LGF_API lgf_status lgf_poisson_error_estimate(lgf_ctx *ctx, const lgf_blockset *src, const lgf_blockset *tgt,
                                              const void *f_dev, const void *u_dev, int32_t ncomp, int32_t nrhs,
                                              double dx, int32_t nsample, double *max_rel_err, void *stream);

/* Save the context's FP64 G_L table (the App. A pre-processing) to a file,
   and load one back into a context (skipping the quadrature): a versioned
   header ("LGFTAB01", radius, entry count, near/far shell mismatch), the
   values, and a 64-bit hash of them.  A load replaces the table and drops the
   spectra, G_K tables and graphs built from the old one; a file that fails
   any check is refused.  Errors: LGF_EINVAL (path, file), LGF_ENOTABLE
   (save before a build), LGF_ENOMEM, LGF_ECUDA. */
LGF_API lgf_status lgf_table_save(lgf_ctx *ctx, const char *path);
LGF_API lgf_status lgf_table_load(lgf_ctx *ctx, const char *path);

/* Device-side status.  Kernels that wait on the GPU (the integrating
   factor's z pass stages its slab with bulk asynchronous copies completed on
   an mbarrier) bound every wait to about one second; a wait that runs out
   sets a bit of the context's device error word and its CTA returns without
   output, so nothing traps and the context stays usable.  This call
   synchronises the device, stores the word in *word (may be NULL), clears
   it, and returns LGF_ETIMEOUT when it was set.  Errors: LGF_ETIMEOUT,
   LGF_ECUDA. */
LGF_API lgf_status lgf_device_status(lgf_ctx *ctx, int32_t *word);

/* Exercise the timeout path: one CTA waits on an mbarrier that no copy
   completes, with a limit of `cycles` SM clock cycles (1 .. 4e9), so the wait
   runs out and sets the device error word that lgf_device_status reports.
   Nothing faults; the context stays usable.  Errors: LGF_EINVAL, LGF_ECUDA. */
LGF_API lgf_status lgf_wait_selftest(lgf_ctx *ctx, int64_t cycles, void *stream);

/* Autotuner.  A Poisson plan's geometry has free choices that the method
   leaves open (Sec. 2.2 fixes only the convolution): the embedding of x and
   of y (the even circular embedding of G_L, M >= 2L - 1 on the union extent
   L, or the shifted window, M >= Ls + Lt - 1), the transform length along
   each axis (the smallest supported length, or the next one, whose radix
   plan may run faster) and the register cap of the z pass (FP32); a batch
   also has its branch count (1, 2, 4 or 8 concurrent streams).  With tuning on,
   each new plan's first apply times candidates on the caller's stream
   (coordinate descent from the default: one knob changed at a time, a change
   kept when it cuts the median time of the passes by at least 3 %), and each
   new batch shape times its branch counts; the choices are kept in the
   context and, when `cache_path` names a file (NULL: the LGF_TUNE_CACHE
   environment variable, if set), appended to it as "key -> value" lines and
   read back by later contexts.  A plan value ends in "f0" or "f1": with
   "f1" (FP32, lengths 64, 80, 96 and 128 along y) the y and x inverses run
   fused, one thread-block cluster per target plane holding the plane's rows
   in distributed shared memory; the tuner keeps "f0", which measured faster
   inside batches.  LGF_TUNE_CACHED uses the file's choices and
   the defaults elsewhere, timing nothing.  Results do not depend on the
   choices beyond floating-point rounding.  Tuning runs synchronously in the
   call that first meets a plan, so tune before capturing a stream into a
   CUDA graph.  Errors: LGF_EINVAL (mode), LGF_ECUDA. */
enum { LGF_TUNE_OFF = 0, LGF_TUNE_ON = 1, LGF_TUNE_CACHED = 2 };

LGF_API lgf_status lgf_autotune(lgf_ctx *ctx, int32_t mode, const char *cache_path);

typedef struct {
    int64_t plans_tuned;        /* plans whose choice was timed in this context */
    int64_t plans_from_cache;   /* plans whose choice came from the file */
    int64_t candidates_timed;   /* candidate geometries timed */
    int64_t batches_tuned;      /* batch shapes whose branch count was chosen */
    int64_t last_branches;      /* branch count of the last batch */
    int64_t shifted_x, shifted_y, longer_x, longer_y, longer_z, z_variant;   /* counts over the context's plans */
    double tune_ms;             /* GPU time spent timing candidates */
    int64_t last_ragged;        /* 1: the last batch ran its Poisson parts ragged (one launch per pass and length) */
    int64_t fused_inverse;      /* plans whose y and x inverses run as one cluster kernel */
    int64_t reserved[2];
} lgf_tune_info;

/* The tuner's counters and a summary of the choices of the context's plans.
   Errors: LGF_EINVAL. */
LGF_API lgf_status lgf_tune_report(lgf_ctx *ctx, lgf_tune_info *out);

/* Allocation-free integrating-factor apply.  The paper has no counterpart:
   this entry point exists for callers that must not allocate device memory
   while they run -- for example a time-stepping loop whose device memory is
   reserved up front by another allocator (a framework's caching allocator),
   where a cudaMalloc could fail or synchronise the whole device.  It computes
   what lgf_intfactor_apply computes -- the same truncation rule with `tol`
   (0 = 1e-7 for LGF_F32, 1e-13 for LGF_F64) and the same separable stencil --
   on the current device, without a context and without calling cudaMalloc,
   cudaFree or any allocating routine.  It always runs three single-axis
   passes (x, y, z), whereas the context path may fuse the x and y passes, so
   FP32 results agree with lgf_intfactor_apply to rounding, not bit for bit.
   Its scratch (weights, neighbour tables and the two intermediate fields) is
   one 32 MiB __device__ array that every GPU which loads the library holds
   until the process exits; planning uses fixed host arrays, so the function
   is not thread safe.
   Limits (LGF_EUNSUPPORTED beyond them): at most 1024 source and 1024 target
   blocks, block sets within a 64-block box (after growing by the stencil
   reach), at most 8192 blocks per intermediate set, intermediate fields of
   at most about 32 MiB in total (nfields x blocks x b^3 x element size), and
   device ordinals below 64.
   The first call on each device takes the device address of the array with
   cudaGetSymbolAddress.  Every call reads the weights back to the host and
   synchronises `stream` once (to choose the radius), so it cannot be called
   while `stream` is being captured into a CUDA graph.  Every call reuses the
   same array: calls whose work overlaps on the GPU (different streams, or
   the same array from two host threads) race.  err_msg (host, err_cap bytes,
   may be NULL) receives a message on failure. */
LGF_API lgf_status lgf_intfactor_apply_noalloc(int32_t prec, double tol, double alpha, const lgf_blockset *src,
                                               const lgf_blockset *tgt, const void *f_dev, void *u_dev,
                                               int32_t ncomp, int32_t nrhs, void *stream, char *err_msg,
                                               int32_t err_cap);

/* Static text for a status code. */
LGF_API const char *lgf_status_string(lgf_status s);

/* Message of the last failed call on this context ("" if none). */
LGF_API const char *lgf_last_error(lgf_ctx *ctx);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
LGF_API int32_t lgf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LGF_H */
