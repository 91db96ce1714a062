// Fused y+x inverse instantiated for length 128 along y and lengths 32 to 384 along x
// (clusters of 1, 2 and 4 CTAs): one translation unit per length along y and
// part of the lengths along x, so that the pairs compile in parallel.
#include "lgf_poisson_fused.cuh"

namespace lgf {
namespace pk {
template lgf_status yx_launch_my<128, 0>(lgf_ctx *, int, int, YXJob *, int, cudaStream_t);
}  // namespace pk
}  // namespace lgf
