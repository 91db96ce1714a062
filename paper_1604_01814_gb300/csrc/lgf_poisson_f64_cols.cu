// Poisson y passes (and the spectrum build's z pass) instantiated for double: one translation unit per pass family
// and precision, so that the many transform lengths compile in parallel.
#include "lgf_poisson_kernels.cuh"

namespace lgf {
template lgf_status launch_col_forward<double>(lgf_ctx *, int, int, int, int, const Cx<double> *, Cx<double> *, int, int,
                                           int64_t, int64_t, int64_t, int64_t, int64_t, int64_t, const Cx<double> *,
                                           pk::RowFlags, cudaStream_t, const char *);
template lgf_status launch_col_inverse<double>(lgf_ctx *, int, int, int, int, const Cx<double> *, Cx<double> *, int, int,
                                           int64_t, int64_t, int64_t, int64_t, int64_t, int64_t, const Cx<double> *,
                                           cudaStream_t, const char *);
template lgf_status launch_col_forward_rag<double>(lgf_ctx *, int, pk::ColJob<double> *, int, cudaStream_t);
template lgf_status launch_col_inverse_rag<double>(lgf_ctx *, int, bool, pk::ColJob<double> *, int, cudaStream_t);
}  // namespace lgf
