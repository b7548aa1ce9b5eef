// vdf_batch_d0.cu -- batch kernels of distance mode EXACT (vdf_batch_kernels.cuh).
#define VDF_BATCH_INSTANTIATE
#include "vdf_batch_kernels.cuh"

namespace vdf {

template struct BatchOps<EXACT>;

}  // namespace vdf
