// Register-window integrating-factor passes instantiated for float.
#include "lgf_intfactor_win.cuh"

namespace lgf {
template lgf_status launch_sep_window<float>(lgf_ctx *, int, int, int, int, cudaStream_t, const float *, float *, const int *,
                                         const float *, int, int, int64_t, int64_t, bool *);
template lgf_status launch_sep_xy<float>(lgf_ctx *, int, int, int, cudaStream_t, const float *, float *, const int *,
                                     const float *, int, int, int64_t, int64_t, bool *);
}  // namespace lgf
