// Poisson z pass instantiated for float: one translation unit per pass family
// and precision, so that the many transform lengths compile in parallel.
#include "lgf_poisson_kernels.cuh"

namespace lgf {
template lgf_status launch_col_convolve<float>(lgf_ctx *, const PoissonGeom &, Cx<float> *, const float *,
                                            const Cx<float> *, int, cudaStream_t);
}  // namespace lgf
