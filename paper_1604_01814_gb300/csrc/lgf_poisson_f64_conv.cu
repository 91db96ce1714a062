// Poisson z pass instantiated for double with the even embedding's real spectrum: one translation unit per
// pass family, precision and spectrum layout, so that the many transform
// lengths compile in parallel.
#include "lgf_poisson_kernels.cuh"

namespace lgf {
template lgf_status launch_col_convolve<double, 0>(lgf_ctx *, const PoissonGeom &, Cx<double> *, const double *,
                                              const Cx<double> *, int, cudaStream_t);
template lgf_status launch_col_convolve_rag<double, 0>(lgf_ctx *, int, int, pk::ConvJob<double> *, int, cudaStream_t);
}  // namespace lgf
