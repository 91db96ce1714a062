// Poisson pass kernels instantiated for float (compiled as its own translation unit).
#include "lgf_poisson_kernels.cuh"

namespace lgf {
template lgf_status launch_row_forward<float>(lgf_ctx *, const PoissonGeom &, const float *, Cx<float> *, const Cx<float> *, int,
                                          int, int, cudaStream_t);
template lgf_status launch_row_inverse<float>(lgf_ctx *, const PoissonGeom &, const Cx<float> *, float *, const Cx<float> *, int,
                                          int, cudaStream_t);
template lgf_status launch_col_forward<float>(lgf_ctx *, int, int, int, int, const Cx<float> *, Cx<float> *, int, int, int64_t,
                                          int64_t, int64_t, int64_t, int64_t, int64_t, const Cx<float> *, cudaStream_t,
                                          const char *);
template lgf_status launch_col_inverse<float>(lgf_ctx *, int, int, int, int, const Cx<float> *, Cx<float> *, int, int, int64_t,
                                          int64_t, int64_t, int64_t, int64_t, int64_t, const Cx<float> *, cudaStream_t,
                                          const char *);
template lgf_status launch_col_convolve<float>(lgf_ctx *, const PoissonGeom &, Cx<float> *, const float *, const Cx<float> *, int,
                                           cudaStream_t);
}  // namespace lgf
