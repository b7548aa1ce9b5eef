// vdf_fp32_s3.cu -- FP32 tile kernel instantiations for tile shape 3 (kShapes32[3]).
#include "vdf_fp32_inst.cuh"

namespace vdf {

cudaError_t run_fp32_s3(const TileParams &prm, int R, int filter, int dist, cudaStream_t st)
{
    return run_fp32_shape<kShapes32[3].tw, kShapes32[3].th>(prm, R, filter, dist, st);
}

}  // namespace vdf
