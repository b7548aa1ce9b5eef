// vdf_fp32f.cu -- FP32 certified tile kernel for float32 input (exact
// mode), one 32x16 tile shape; built with flush-to-zero like the uint8 FP32
// units (the float bounds and the safe-pixel test do not depend on it).
#include "vdf_dispatch.h"

namespace vdf {

cudaError_t run_fp32_f32in(const TileParams &prm, int R, int filter, cudaStream_t st)
{
    if (R == 1)
        return filter == DDF ? launch_tile<TileCfg<1, DDF, EXACT, false, true, 32, 16>>(prm, st)
                             : launch_tile<TileCfg<1, BVDF, EXACT, false, true, 32, 16>>(prm, st);
    if (R == 2)
        return filter == DDF ? launch_tile<TileCfg<2, DDF, EXACT, false, true, 32, 16>>(prm, st)
                             : launch_tile<TileCfg<2, BVDF, EXACT, false, true, 32, 16>>(prm, st);
    return cudaErrorInvalidValue;
}

}  // namespace vdf
