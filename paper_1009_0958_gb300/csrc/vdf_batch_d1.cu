// vdf_batch_d1.cu -- batch kernels of distance mode MINIMAX (vdf_batch_kernels.cuh).
#define VDF_BATCH_INSTANTIATE
#include "vdf_batch_kernels.cuh"

namespace vdf {

template struct BatchOps<MINIMAX>;

}  // namespace vdf
