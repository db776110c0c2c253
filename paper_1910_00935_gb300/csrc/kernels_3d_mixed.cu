// kernels_3d_mixed.cu -- 3D per-particle materials (solid + liquid), FP32 sums: the
// particle passes and the persistent pass interpreters (templates in kernels_launch.cuh;
// one variant per translation unit so that the variants compile in parallel).
#include "kernels_launch.cuh"

namespace mpm {

template cudaError_t step_variant<3, kMixed, false>(int, const SimParams&, const StepArgs&, int,
                                                     cudaStream_t);
template cudaError_t adj_variant<3, kMixed, false>(int, const SimParams&, const AdjArgs&, int,
                                                    cudaStream_t);
template cudaError_t persistent_variant<3, kMixed, false>(int, const SimParams&, const PassEntry*,
                                                           int, int, const PersistCtl&, cudaStream_t,
                                                           int*);

}  // namespace mpm
