// vdf_fp32_s1.cu -- FP32 tile kernel instantiations for tile shape 1 (kShapes32[1]).
#include "vdf_fp32_inst.cuh"

namespace vdf {

cudaError_t run_fp32_s1(const TileParams &prm, int R, int filter, int dist, cudaStream_t st)
{
    return run_fp32_shape<kShapes32[1].tw, kShapes32[1].th>(prm, R, filter, dist, st);
}

}  // namespace vdf
