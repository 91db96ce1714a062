// Poisson pass kernels instantiated for double (compiled as its own translation unit).
#include "lgf_poisson_kernels.cuh"

namespace lgf {
template lgf_status launch_row_forward<double>(lgf_ctx *, const PoissonGeom &, const double *, Cx<double> *, const Cx<double> *, int,
                                          int, int, cudaStream_t);
template lgf_status launch_row_inverse<double>(lgf_ctx *, const PoissonGeom &, const Cx<double> *, double *, const Cx<double> *, int,
                                          int, cudaStream_t);
template lgf_status launch_col_forward<double>(lgf_ctx *, int, int, int, int, const Cx<double> *, Cx<double> *, int, int, int64_t,
                                          int64_t, int64_t, int64_t, int64_t, int64_t, const Cx<double> *, cudaStream_t,
                                          const char *);
template lgf_status launch_col_inverse<double>(lgf_ctx *, int, int, int, int, const Cx<double> *, Cx<double> *, int, int, int64_t,
                                          int64_t, int64_t, int64_t, int64_t, int64_t, const Cx<double> *, cudaStream_t,
                                          const char *);
template lgf_status launch_col_convolve<double>(lgf_ctx *, const PoissonGeom &, Cx<double> *, const double *, const Cx<double> *, int,
                                           cudaStream_t);
}  // namespace lgf
