// Register-window integrating-factor passes instantiated for float.
#include "lgf_intfactor_win.cuh"

namespace lgf {
template lgf_status launch_sep_window<float>(lgf_ctx *, int, int, int, const SepJobs<float> &, cudaStream_t, const int *,
                                         int, bool *);
template lgf_status launch_sep_xy<float>(lgf_ctx *, int, int, const SepJobs<float> &, cudaStream_t, const int *,
                                     const int *, int, bool *);
template lgf_status launch_sep_rag<float>(lgf_ctx *, bool, int, int, SepRagJob<float> *, int, cudaStream_t);
}  // namespace lgf
