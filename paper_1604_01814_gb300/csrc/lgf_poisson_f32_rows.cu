// Poisson x passes instantiated for float: one translation unit per pass family
// and precision, so that the many transform lengths compile in parallel.
#include "lgf_poisson_kernels.cuh"

namespace lgf {
template lgf_status launch_row_forward<float>(lgf_ctx *, const PoissonGeom &, const float *, Cx<float> *, const Cx<float> *,
                                           int, int, int, cudaStream_t);
template lgf_status launch_row_inverse<float>(lgf_ctx *, const PoissonGeom &, const Cx<float> *, float *, const Cx<float> *,
                                           int, int, cudaStream_t);
template lgf_status launch_row_forward_rag<float>(lgf_ctx *, int, pk::RowJob<float> *, int, cudaStream_t);
template lgf_status launch_row_inverse_rag<float>(lgf_ctx *, int, bool, pk::RowJob<float> *, int, cudaStream_t);
}  // namespace lgf
