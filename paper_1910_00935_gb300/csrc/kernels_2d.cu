// kernels_2d.cu -- 2D instantiations of the particle passes, the persistent pass
// interpreters and the grid clear (templates in kernels_launch.cuh).
#include "kernels_launch.cuh"

namespace mpm {

#define MPM_INSTANTIATE(D, MAT, DET)                                                              \
  template cudaError_t step_variant<D, MAT, DET>(int, const SimParams&, const StepArgs&, int,       \
                                                 cudaStream_t);                                   \
  template cudaError_t adj_variant<D, MAT, DET>(int, const SimParams&, const AdjArgs&, int,         \
                                                cudaStream_t);                                    \
  template cudaError_t persistent_variant<D, MAT, DET>(int, const SimParams&, const PassEntry*, int, \
                                                       int, const PersistCtl&, cudaStream_t, int*);

MPM_INSTANTIATE(2, kFixedCorotated, false)
MPM_INSTANTIATE(2, kNeoHookean, false)
MPM_INSTANTIATE(2, kFixedCorotated, true)
MPM_INSTANTIATE(2, kNeoHookean, true)
MPM_INSTANTIATE(2, kLiquid, false)
MPM_INSTANTIATE(2, kLiquid, true)
MPM_INSTANTIATE(2, kMixed, false)
MPM_INSTANTIATE(2, kMixed, true)
template cudaError_t launch_clear<2>(const Clears&, int, int, int, int, cudaStream_t);
template cudaError_t launch_clear<3>(const Clears&, int, int, int, int, cudaStream_t);

}  // namespace mpm
