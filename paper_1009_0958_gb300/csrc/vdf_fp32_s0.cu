// vdf_fp32_s0.cu -- FP32 tile kernel instantiations for tile shape 0 (kShapes32[0]).
#include "vdf_fp32_inst.cuh"

namespace vdf {

cudaError_t run_fp32_s0(const TileParams &prm, int R, int filter, int dist, cudaStream_t st)
{
    return run_fp32_shape<kShapes32[0].tw, kShapes32[0].th>(prm, R, filter, dist, st);
}

}  // namespace vdf
