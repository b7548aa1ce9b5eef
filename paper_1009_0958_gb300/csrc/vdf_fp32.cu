// vdf_fp32.cu -- dispatch of the FP32 tile kernel over its tile shapes.  The
// shapes are instantiated in vdf_fp32_s<k>.cu; the autotuner picks one per
// (window, filter, distance mode).
#include "vdf_dispatch.h"

namespace vdf {

cudaError_t run_fp32_s0(const TileParams &prm, int R, int filter, int dist, cudaStream_t st);
cudaError_t run_fp32_s1(const TileParams &prm, int R, int filter, int dist, cudaStream_t st);
cudaError_t run_fp32_s2(const TileParams &prm, int R, int filter, int dist, cudaStream_t st);
cudaError_t run_fp32_s3(const TileParams &prm, int R, int filter, int dist, cudaStream_t st);

cudaError_t run_fp32(const TileParams &prm, int R, int filter, int dist, int shape, cudaStream_t st)
{
    switch (shape) {
    case 0: return run_fp32_s0(prm, R, filter, dist, st);
    case 1: return run_fp32_s1(prm, R, filter, dist, st);
    case 2: return run_fp32_s2(prm, R, filter, dist, st);
    case 3: return run_fp32_s3(prm, R, filter, dist, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace vdf
