// Register-window integrating-factor passes instantiated for double.
#include "lgf_intfactor_win.cuh"

namespace lgf {
template lgf_status launch_sep_window<double>(lgf_ctx *, int, int, int, const SepJobs<double> &, cudaStream_t, const int *,
                                         int, bool *);
template lgf_status launch_sep_xy<double>(lgf_ctx *, int, int, const SepJobs<double> &, cudaStream_t, const int *,
                                     const int *, int, bool *);
template lgf_status launch_sep_rag<double>(lgf_ctx *, bool, int, int, SepRagJob<double> *, int, cudaStream_t);
}  // namespace lgf
