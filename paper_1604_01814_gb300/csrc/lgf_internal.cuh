// Internal declarations shared by the translation units of the CUDA library.
#pragma once
#include <cuda_runtime.h>

#include <array>
#include <cstdint>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "lgf.h"
#include "lgf_cache.h"
#include "lgf_fft.cuh"

namespace lgf {

constexpr int kMaxFft = 4096;        // largest transform length per axis
constexpr int kMinTableRadius = 24;  // expansion error at |n| > 24 is below 1e-9 relative

// --------------------------------------------------------------------------
// Transform lengths: 2^k, 3 * 2^k and 5 * 2^k from 32 to 4096.
// --------------------------------------------------------------------------
int next_fft_size(int n);   // smallest supported length >= n
// --------------------------------------------------------------------------
// Poisson plan: one problem's padded transform box.
// Box coordinates are lattice coordinates minus `lo` (the union bounding box
// corner of the source and target block sets).
// --------------------------------------------------------------------------
struct PoissonGeom {
    int M[3];           // transform lengths (x, y, z)
    int Kx;             // Mx / 2 + 1 (half spectrum along x)
    int s0[3], Ls[3];   // source region [s0, s0 + Ls) in box coordinates
    int t0[3], Lt[3];   // target region
    int b;
    int nbs[3], nbt[3]; // region extents in blocks
    const int *srcmap;  // [nbs_z][nbs_y][nbs_x] -> source block index or -1
    const int *tgtmap;  // [nbt_z][nbt_y][nbt_x] -> target block index or -1
    // row-block occupancy per plane block: bit y of [nbs_z] (source) and
    // [nbt_z] (target) set where some block lies along x in row block y (the
    // x passes skip CTAs in empty row blocks, the y-forward pass their rows);
    // nullptr when every row block is occupied or a region has more than 64
    // row blocks
    const unsigned long long *srcrow, *tgtrow;
    int64_t fstride;    // elements per field in f (nsrc * b^3)
    int64_t ustride;    // elements per field in u (ntgt * b^3)
    int64_t Astride;    // complex elements per field in scratch A
    int64_t Bstride;    // complex elements per field in scratch B
    int ldA_y;          // rows per z-plane in A (max(Ls_y, Lt_y))
    // embedding along x and y: 0 = even (M >= 2L - 1 on the union extent,
    // real spectrum along that axis); 1 = shifted window (M >= Ls + Lt - 1,
    // source and target both placed at 0, complex spectrum):
    // h[m] = G_L(m + c) for m < P, G_L(m - M + c) above.  z is always even.
    int xasym, xc, xP;
    int yasym, yc, yP;
    int zvar;           // z-pass variant: 0 default, 1 one more CTA per SM (tighter register cap)
    int fuse;           // FP32: the y and x inverses as one cluster kernel where available
    double scale;       // dx^2
};

// The free choices of a Poisson plan (the tuner's knobs).
struct PoissonChoice {
    int shift[2] = {0, 0};   // x, y: shifted window instead of the even embedding
    int bump[3] = {0, 0, 0}; // transform length: the bump-th supported length above the smallest valid one
    int zvar = 0;
    int fuse = 0;            // fused y+x inverse (FP32, where instantiated; the tuner's alternative)
    bool operator==(const PoissonChoice &o) const
    {
        return shift[0] == o.shift[0] && shift[1] == o.shift[1] && bump[0] == o.bump[0] && bump[1] == o.bump[1] &&
               bump[2] == o.bump[2] && zvar == o.zvar && fuse == o.fuse;
    }
};

struct PoissonPlan {
    int b = 0;
    std::vector<int32_t> src, tgt;   // block coordinates, for cache matching
    int slo[3], shi[3], tlo[3], thi[3];   // block extents of the source and target sets
    PoissonChoice choice;            // the geometry's free choices (default or tuned)
    int tuned_nf = 0;                // field count the choice was tuned for (0: not tuned)
    PoissonGeom g{};
    int *srcmap_dev = nullptr, *tgtmap_dev = nullptr;
    unsigned long long *srcrow_dev = nullptr, *tgtrow_dev = nullptr;
    int64_t A_elems = 0, B_elems = 0; // complex elements per field
    uint64_t used = 0;                // epoch of the last call that used it
    ~PoissonPlan();
};

// --------------------------------------------------------------------------
// Integrating-factor plan: three separable passes over block sets.
// --------------------------------------------------------------------------
struct IntfPass {
    int nout = 0;             // output blocks
    int *nbr_dev = nullptr;   // [nout][2*nr+1] input block index or -1
};

struct IntfPlan {
    int b = 0, nr = 0;
    std::vector<int32_t> src, tgt;
    int n1 = 0, n2 = 0;       // sizes of the two intermediate block sets
    IntfPass pass[3];
    int *nbr_xy_dev = nullptr; // [n2][(2nr+1)^2] source block at xy offset of each Y2 block, or -1
    int *xy_items_dev = nullptr; // [n_xy_items][2] Y2 blocks of each fused-pass CTA (second -1: single)
    int n_xy_items = 0;
    uint64_t used = 0;
    ~IntfPlan();
};

struct IntfWeights {
    double alpha = 0;
    int R = 0;
    double *w64 = nullptr;    // [R+1]
    float *w32 = nullptr;     // [R+1]
};

struct Spectrum {
    std::array<int, 3> M{};
    double alpha = 0.0;       // 0: G_L; > 0: G_K(alpha)
    int xasym = 0, xc = 0, xP = 0;   // the x and y embeddings of PoissonGeom
    int yasym = 0, yc = 0, yP = 0;
    // (Mz/2+1)(My/2+1)(Mx/2+1) values, context precision, scaled by
    // 1/(MxMyMz): reals for the even x embedding, complex for the shifted one
    void *dev = nullptr;
    uint64_t used = 0;
    Spectrum() = default;
    Spectrum(const Spectrum &) = delete;
    Spectrum &operator=(const Spectrum &) = delete;
    ~Spectrum();
};

// Grow-only scratch buffers: A, B for the Poisson passes, C, D for the
// integrating factor (separate, so the two may run on concurrent branches).
struct Scratch {
    void *A = nullptr, *B = nullptr, *C = nullptr, *D = nullptr;
    size_t a = 0, b = 0, c = 0, d = 0;
    void *E = nullptr, *F = nullptr;   // velocity refresh: vorticity and its potential
    size_t e = 0, f = 0;
    void *G = nullptr;                 // nested-projection stage: its fields and marker vectors
    size_t g = 0;
};

// Block look-up for the immersed-boundary operators: dense table over the
// bounding box of the block set.
struct IBPlan {
    int b = 0, lo[3] = {0, 0, 0}, ext[3] = {1, 1, 1};
    std::vector<int32_t> coords;
    int *lut_dev = nullptr;
    uint64_t used = 0;
    ~IBPlan();
};

// Curl stencil plan: for every target block, the source blocks at the block
// itself and at +dir along x, y, z (-1 where absent).
struct CurlPlan {
    int b = 0, dir = 0;
    std::vector<int32_t> src, tgt;
    int *nbr_dev = nullptr;   // [ntgt][4]
    uint64_t used = 0;
    ~CurlPlan();
};
constexpr int kBranches = 8;        // most concurrent branches of a batch
constexpr int kDefaultBranches = 4; // branches of an untuned batch

}  // namespace lgf

struct lgf_ctx {
    lgf_options opt{};
    bool opt_xshift = true;   // allow the shifted x embedding in new Poisson plans
    int device = 0;
    int prec = LGF_F32;
    double tol = 1e-7;
    std::string last_error;

    // G_L table (FP64, sorted offsets a >= b >= c up to table_radius)
    double *table_dev = nullptr;
    int table_radius = -1;
    double shell_mismatch = 0.0;

    // twiddles per log2 length: exp(-2 pi i m / M), m < M
    std::map<int, void *> tw32, tw64;

    // G_K(alpha) tables (alpha > 0) over the same offsets as the G_L table
    std::map<double, double *> gk_tables;

    // kernel spectra per transform-box shape and kernel (alpha = 0: G_L,
    // alpha > 0: G_K(alpha)) and the plans, each cache bounded (least
    // recently used evicted; entries of the current call are kept)
    lgf::LruCache<lgf::Spectrum> spectra{128};
    lgf::LruCache<lgf::PoissonPlan> pplans{256};
    lgf::LruCache<lgf::IntfPlan> iplans{256};
    std::vector<std::unique_ptr<lgf::IntfWeights>> weights;
    lgf::LruCache<lgf::CurlPlan> cplans{64};
    lgf::LruCache<lgf::IBPlan> ibplans{64};
    lgf::CacheCounters counters;

    // grow-only scratch, one set per concurrent branch of lgf_batch_apply
    // (branch 0 also serves the single applies); `cur` is the set the next
    // enqueued work uses
    lgf::Scratch scr[lgf::kBranches];
    lgf::Scratch *cur = &scr[0];

    // branch streams and the fork/join events on the caller's stream
    cudaStream_t br[lgf::kBranches] = {};
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_join[lgf::kBranches] = {};

    // batch graph cache: the most recently used batches (key = everything that
    // shapes the work), least recently used evicted; dropped whole whenever a
    // buffer that a graph may have captured is freed or reallocated
    lgf::GraphCache<cudaGraphExec_t> graphs{8};
    uint64_t graph_clock = 0;

    double *red_dev = nullptr;   // small reduction buffer (residual, table mismatch)
    int *err_dev = nullptr;      // device error word: bits set by bounded waits that ran out
    bool opt_bulk = false;       // stage the E z pass with bulk asynchronous copies (LGF_FLAG_BULK_STAGING)
    bool opt_rag = false;        // batches in the ragged mode unless tuned otherwise (LGF_FLAG_BATCH_RAGGED)
    bool opt_units = false;      // batches in per-problem launches unless tuned otherwise (LGF_FLAG_BATCH_PER_PROBLEM)

    // autotuner: mode (LGF_TUNE_*), persisted choices (key -> value lines of
    // lgf_tune.h, loaded from and appended to tune_path), counters, the
    // branch count per batch shape, and the timing runs' input/output buffers
    int tune_mode = 0;
    int tune_reps = 5;
    std::string tune_path;
    std::map<std::string, std::string> tune_db;
    int64_t tune_plans = 0, tune_plans_cached = 0, tune_candidates = 0, tune_batches = 0;
    double tune_ms = 0.0;
    int tune_last_branches = 0;
    int tune_last_ragged = 0;
    void *tune_f = nullptr, *tune_u = nullptr;
    size_t tune_fb = 0, tune_ub = 0;

    // optional per-kernel timing with CUDA events on the launch stream
    bool prof = false;
    struct ProfRec {
        int name;
        cudaEvent_t a, b;
    };
    std::vector<ProfRec> prof_pending;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::string> prof_names;
    std::vector<int64_t> prof_launches;
    std::vector<double> prof_ms;
};

namespace lgf {

lgf_status fail(lgf_ctx *ctx, lgf_status st, const std::string &msg);
lgf_status cuda_fail(lgf_ctx *ctx, cudaError_t e, const char *what);
lgf_status ensure_scratch(lgf_ctx *ctx, void **p, size_t *have, size_t need);
// Drop every captured graph (their buffers are about to change).
void invalidate_graphs(lgf_ctx *ctx);
// Called before a cache evicts entries: drop the graphs and wait for the
// device, so no queued or replayed work still reads what is freed.
void before_evict(lgf_ctx *ctx);
const void *twiddles(lgf_ctx *ctx, int M, bool dbl, lgf_status *st);

#define LGF_CUDA(ctx, call)                                   \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return lgf::cuda_fail((ctx), e_, #call); \
    } while (0)

#define LGF_CHECK_LAUNCH(ctx, what)                           \
    do {                                                      \
        cudaError_t e_ = cudaGetLastError();                  \
        if (e_ != cudaSuccess) return lgf::cuda_fail((ctx), e_, (what)); \
    } while (0)

// Per-kernel timing (lgf_capi.cu): prof_begin records a start event and
// returns a handle (-1 when profiling is off); prof_end records the stop event.
int prof_begin(lgf_ctx *ctx, cudaStream_t s, const char *name);
void prof_end(lgf_ctx *ctx, cudaStream_t s, int handle);

// Table (lgf_table.cu)
lgf_status table_build(lgf_ctx *ctx, int radius, cudaStream_t s);
lgf_status gk_table(lgf_ctx *ctx, double alpha, const double **out, cudaStream_t s);
lgf_status table_lookup(lgf_ctx *ctx, const double *table, const int32_t *off, int64_t n, double *out,
                        cudaStream_t s);
lgf_status kernel_window(lgf_ctx *ctx, const double *table, const int M[3], int xc, int xP, int yc, int yP,
                         double *box, cudaStream_t s);
lgf_status bessel_weights(lgf_ctx *ctx, double z, int nmax, double *out_dev, cudaStream_t s);
// FP64 direct sums dx^2 sum_m G_L(t - m) f(m) of one source field at npts
// lattice points (host [npts][3]); values to host out.  Synchronous.
lgf_status direct_samples(lgf_ctx *ctx, const lgf_blockset *src, const void *f_field, const int32_t *pts_host,
                          int npts, double dx, double *out_host, cudaStream_t s);
// Values of a field at element indices (host), to host doubles.  Synchronous.
lgf_status gather_values(lgf_ctx *ctx, const void *field, const int64_t *idx_host, int n, double *out_host,
                         cudaStream_t s);
lgf_status table_save(lgf_ctx *ctx, const char *path);
lgf_status table_load(lgf_ctx *ctx, const char *path);

// Poisson (lgf_poisson.cu)
lgf_status poisson_plan(lgf_ctx *ctx, const lgf_blockset *src, const lgf_blockset *tgt, PoissonPlan **out);
// The geometry of `ch` for the plan's block extents (false: the choice is not
// valid for them); fills g's sizes, offsets and embeddings, *A, *B the
// scratch elements per field.
bool poisson_geometry(const PoissonPlan &pl, const PoissonChoice &ch, PoissonGeom *g, int64_t *A, int64_t *B);
// Default choice: the shifted window on x and y where it is shorter.
PoissonChoice poisson_default_choice(const PoissonPlan &pl, bool allow_shift);
// Apply a choice to the plan (geometry and scratch sizes).
void poisson_set_choice(PoissonPlan *pl, const PoissonChoice &ch);
lgf_status poisson_spectrum(lgf_ctx *ctx, const PoissonGeom &pg, double alpha, Spectrum **out, cudaStream_t s);
lgf_status poisson_run(lgf_ctx *ctx, PoissonPlan *pl, const Spectrum *sp, const void *f, void *u, int nfields,
                       double dx, cudaStream_t s);
lgf_status poisson_prepare_scratch(lgf_ctx *ctx, const PoissonPlan *pl, int nfields);
// Cluster size of the fused y+x inverse for a geometry (0: not available:
// FP64, a length pair not instantiated, or rows that do not fit), and the
// rows per CTA.
int poisson_fused_ncl(const PoissonGeom &g, int *rpb);
// Many Poisson parts at once (lgf_batch_apply): one launch per pass and
// transform length, the length groups of a pass spread over `nbr` branch
// streams of the context (nbr <= 1: all on s).  Every part's A and B are
// slices of the scratch of branch 0, which poisson_ragged_scratch sizes.
struct RagPart {
    const PoissonPlan *plan;
    const Spectrum *sp;
    const void *f;
    void *u;
    int nf;
    double dx;
};
lgf_status poisson_ragged_scratch(lgf_ctx *ctx, const RagPart *parts, int n);
lgf_status poisson_run_ragged(lgf_ctx *ctx, const RagPart *parts, int n, cudaStream_t s, int nbr);

// Integrating factor (lgf_intfactor.cu)
lgf_status intf_weights(lgf_ctx *ctx, double alpha, IntfWeights **out, cudaStream_t s);
lgf_status intf_plan(lgf_ctx *ctx, const lgf_blockset *src, const lgf_blockset *tgt, int R, IntfPlan **out);
lgf_status intf_prepare_scratch(lgf_ctx *ctx, const IntfPlan *pl, int nfields, int njobs);
struct IntfJob {
    const IntfWeights *w;
    const void *f;
    void *u;
};
lgf_status intf_run_jobs(lgf_ctx *ctx, IntfPlan *pl, const IntfJob *jobs, int njobs, int nfields, cudaStream_t s);
lgf_status intf_run(lgf_ctx *ctx, IntfPlan *pl, const IntfWeights *w, const void *f, void *u, int nfields,
                    cudaStream_t s);
// Integrating-factor groups of several plans at once (lgf_batch_apply's
// ragged mode): the fused x+y pass of all their jobs in one launch per block
// edge and window bound, then the z pass likewise, each job's intermediate a
// slice of scratch D of `sc` (intf_ragged_scratch sizes it); groups the
// window kernels do not cover run one after another as intf_run_jobs (with
// the scratch of `sc`).
struct IntfGroupRef {
    IntfPlan *plan;
    const IntfJob *jobs;
    int njobs;
    int nf;
};
lgf_status intf_ragged_scratch(lgf_ctx *ctx, const IntfGroupRef *gs, int n, Scratch *sc);
lgf_status intf_run_ragged(lgf_ctx *ctx, const IntfGroupRef *gs, int n, cudaStream_t s, Scratch *sc);

// Curl and velocity refresh (lgf_curl.cu)
lgf_status curl_plan(lgf_ctx *ctx, const lgf_blockset *src, const lgf_blockset *tgt, int dir, CurlPlan **out);
lgf_status curl_run(lgf_ctx *ctx, const CurlPlan *pl, const void *in, void *out, int nrhs, double scale,
                    cudaStream_t s);
std::vector<int32_t> grown_forward(const lgf_blockset *tgt);

// Nested-projection stage kernels (lgf_stage.cu)
lgf_status stage_div(lgf_ctx *ctx, const CurlPlan *pl, const void *a, const void *c, void *out, double dx,
                     cudaStream_t s);
lgf_status stage_grad(lgf_ctx *ctx, const CurlPlan *pl, const void *d, const void *a, const void *c, void *out,
                      double dx, cudaStream_t s);
lgf_status stage_force(lgf_ctx *ctx, const void *U, const void *ub, const void *W1, const void *W2, void *rhs, void *y,
                       void *fh, int n, cudaStream_t s);

// Immersed-boundary operators (lgf_ib.cu)
lgf_status ib_plan(lgf_ctx *ctx, const lgf_blockset *set, IBPlan **out);
lgf_status ib_run(lgf_ctx *ctx, const IBPlan *pl, bool spread, int64_t nm, const double *X, const void *in, void *out,
                  int nrhs, double dx, cudaStream_t s);

// Residual (lgf_residual.cu)
lgf_status residual_run(lgf_ctx *ctx, const lgf_blockset *set, const void *u, const void *f, double dx,
                        double *r, double *max_abs, double *max_f, cudaStream_t s);

// Autotuner (lgf_tune.cu): choose the plan's geometry for nf fields (timed
// candidates, or the persisted choice); no-op when tuning is off or the plan
// is tuned.
lgf_status tune_poisson(lgf_ctx *ctx, PoissonPlan *pl, int nf, double kalpha, cudaStream_t s);
// Time the five passes of `pl` under choice `ch` (median of the context's
// repetitions, ms); builds the spectrum the choice needs.
lgf_status poisson_time_choice(lgf_ctx *ctx, PoissonPlan *pl, const PoissonChoice &ch, int nf, double kalpha,
                               cudaStream_t s, float *ms);
// Record a tuned item (in memory and appended to the persisted file).
void tune_record(lgf_ctx *ctx, const std::string &key, const std::string &value);

// A single CTA waiting on an mbarrier that no copy completes, with a limit of
// `cycles`: the wait runs out and sets the device error word (lgf_stage.cu).
lgf_status wait_selftest(lgf_ctx *ctx, long long cycles, cudaStream_t s);

// Block-set validation shared by the entry points.
lgf_status check_blockset(lgf_ctx *ctx, const lgf_blockset *bs, const char *name);

}  // namespace lgf
