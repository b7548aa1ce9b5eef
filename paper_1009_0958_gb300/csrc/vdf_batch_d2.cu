// vdf_batch_d2.cu -- batch kernels of distance mode RGB (vdf_batch_kernels.cuh).
#define VDF_BATCH_INSTANTIATE
#include "vdf_batch_kernels.cuh"

namespace vdf {

template struct BatchOps<RGB>;

}  // namespace vdf
