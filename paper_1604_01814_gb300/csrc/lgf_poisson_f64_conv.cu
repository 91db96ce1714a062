// Poisson z pass instantiated for double: one translation unit per pass family
// and precision, so that the many transform lengths compile in parallel.
#include "lgf_poisson_kernels.cuh"

namespace lgf {
template lgf_status launch_col_convolve<double>(lgf_ctx *, const PoissonGeom &, Cx<double> *, const double *,
                                            const Cx<double> *, int, cudaStream_t);
}  // namespace lgf
