// Poisson z pass instantiated for float with the shifted y window's complex spectrum: one translation unit per
// pass family, precision and spectrum layout, so that the many transform
// lengths compile in parallel.
#include "lgf_poisson_kernels.cuh"

namespace lgf {
template lgf_status launch_col_convolve<float, 2>(lgf_ctx *, const PoissonGeom &, Cx<float> *, const float *,
                                              const Cx<float> *, int, cudaStream_t);
template lgf_status launch_col_convolve_rag<float, 2>(lgf_ctx *, int, int, pk::ConvJob<float> *, int, cudaStream_t);
}  // namespace lgf
