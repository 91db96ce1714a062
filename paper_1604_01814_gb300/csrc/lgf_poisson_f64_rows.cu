// Poisson x passes instantiated for double: one translation unit per pass family
// and precision, so that the many transform lengths compile in parallel.
#include "lgf_poisson_kernels.cuh"

namespace lgf {
template lgf_status launch_row_forward<double>(lgf_ctx *, const PoissonGeom &, const double *, Cx<double> *, const Cx<double> *,
                                           int, int, int, cudaStream_t);
template lgf_status launch_row_inverse<double>(lgf_ctx *, const PoissonGeom &, const Cx<double> *, double *, const Cx<double> *,
                                           int, int, cudaStream_t);
template lgf_status launch_row_forward_rag<double>(lgf_ctx *, int, pk::RowJob<double> *, int, cudaStream_t);
template lgf_status launch_row_inverse_rag<double>(lgf_ctx *, int, bool, pk::RowJob<double> *, int, cudaStream_t);
}  // namespace lgf
