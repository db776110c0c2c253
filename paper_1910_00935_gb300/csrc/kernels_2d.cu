// kernels_2d.cu -- 2D instantiations of the particle passes, the persistent pass
// interpreters and the grid clear (templates in kernels_launch.cuh).
#include "kernels_launch.cuh"

namespace mpm {

template cudaError_t launch_step<2>(int, int, const SimParams&, const StepArgs&, int, cudaStream_t);
template cudaError_t launch_adjoint<2>(int, int, const SimParams&, const AdjArgs&, int, cudaStream_t);
template cudaError_t launch_persistent<2>(int, int, const SimParams&, const PassEntry*, int, int,
                                             const PersistCtl&, cudaStream_t, int*);
template cudaError_t launch_clear<2>(const Clears&, int, int, int, int, cudaStream_t);

}  // namespace mpm
