// Register-window integrating-factor passes instantiated for double.
#include "lgf_intfactor_win.cuh"

namespace lgf {
template lgf_status launch_sep_window<double>(lgf_ctx *, int, int, int, int, cudaStream_t, const double *, double *, const int *,
                                         const double *, int, int, int64_t, int64_t, bool *);
template lgf_status launch_sep_xy<double>(lgf_ctx *, int, int, int, cudaStream_t, const double *, double *, const int *,
                                     const double *, int, int, int64_t, int64_t, bool *);
}  // namespace lgf
