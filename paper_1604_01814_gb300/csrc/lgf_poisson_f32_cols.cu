// Poisson y passes (and the spectrum build's z pass) instantiated for float: one translation unit per pass family
// and precision, so that the many transform lengths compile in parallel.
#include "lgf_poisson_kernels.cuh"

namespace lgf {
template lgf_status launch_col_forward<float>(lgf_ctx *, int, int, int, int, const Cx<float> *, Cx<float> *, int, int,
                                           int64_t, int64_t, int64_t, int64_t, int64_t, int64_t, const Cx<float> *,
                                           pk::RowFlags, cudaStream_t, const char *);
template lgf_status launch_col_inverse<float>(lgf_ctx *, int, int, int, int, const Cx<float> *, Cx<float> *, int, int,
                                           int64_t, int64_t, int64_t, int64_t, int64_t, int64_t, const Cx<float> *,
                                           cudaStream_t, const char *);
template lgf_status launch_col_forward_rag<float>(lgf_ctx *, int, pk::ColJob<float> *, int, cudaStream_t);
template lgf_status launch_col_inverse_rag<float>(lgf_ctx *, int, bool, pk::ColJob<float> *, int, cudaStream_t);
}  // namespace lgf
