// vdf_fp32_s2.cu -- FP32 tile kernel instantiations for tile shape 2 (kShapes32[2]).
#include "vdf_fp32_inst.cuh"

namespace vdf {

cudaError_t run_fp32_s2(const TileParams &prm, int R, int filter, int dist, cudaStream_t st)
{
    return run_fp32_shape<kShapes32[2].tw, kShapes32[2].th>(prm, R, filter, dist, st);
}

}  // namespace vdf
