// Fused y+x inverse instantiated for length 64 along y (every length along x,
// clusters of 1, 2 and 4 CTAs): one translation unit per y length, so that
// the pairs compile in parallel.
#include "lgf_poisson_fused.cuh"

namespace lgf {
namespace pk {
template lgf_status yx_launch_my<64>(lgf_ctx *, int, int, YXJob *, int, cudaStream_t);
template bool yx_info_my<64>(int, size_t *, int *);
}  // namespace pk
}  // namespace lgf
