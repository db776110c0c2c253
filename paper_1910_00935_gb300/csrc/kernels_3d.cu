// kernels_3d.cu -- 3D instantiations of the particle passes and the grid clear and their
// launch wrappers (material and mode are compile-time, dispatched here).
#include "mpm_internal.h"
#include "mpm_kernels.cuh"

namespace mpm {

namespace {
template <int MAT, int MODE>
cudaError_t step_one(const SimParams& P, const StepArgs& A, int n_tiles, cudaStream_t s) {
  const size_t smem = pass_smem_bytes<3>(P.tile_capacity, P.gather_capacity);
  auto k = step_kernel<3, MAT, MODE>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k<<<n_tiles, kTile, smem, s>>>(P, A);
  return cudaGetLastError();
}

template <int MAT, int MODE>
cudaError_t adj_one(const SimParams& P, const AdjArgs& A, int n_tiles, cudaStream_t s) {
  const size_t smem = pass_smem_bytes<3>(P.tile_capacity, P.gather_capacity);
  auto k = adjoint_kernel<3, MAT, MODE>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k<<<n_tiles, kTile, smem, s>>>(P, A);
  return cudaGetLastError();
}

template <int MAT>
cudaError_t step_mat(int mode, const SimParams& P, const StepArgs& A, int n_tiles, cudaStream_t s) {
  switch (mode) {
    case kP2GOnly: return step_one<MAT, kP2GOnly>(P, A, n_tiles, s);
    case kG2PP2G: return step_one<MAT, kG2PP2G>(P, A, n_tiles, s);
    case kG2PP2GFull: return step_one<MAT, kG2PP2GFull>(P, A, n_tiles, s);
    case kG2POnlyFull: return step_one<MAT, kG2POnlyFull>(P, A, n_tiles, s);
  }
  return cudaErrorInvalidValue;
}

template <int MAT>
cudaError_t adj_mat(int mode, const SimParams& P, const AdjArgs& A, int n_tiles, cudaStream_t s) {
  switch (mode) {
    case kAdjG2P: return adj_one<MAT, kAdjG2P>(P, A, n_tiles, s);
    case kAdjFused: return adj_one<MAT, kAdjFused>(P, A, n_tiles, s);
    case kAdjP2G: return adj_one<MAT, kAdjP2G>(P, A, n_tiles, s);
  }
  return cudaErrorInvalidValue;
}
}  // namespace

template <>
cudaError_t launch_step<3>(int material, int mode, const SimParams& P, const StepArgs& A,
                             int n_tiles, cudaStream_t s) {
  return material == kFixedCorotated ? step_mat<kFixedCorotated>(mode, P, A, n_tiles, s)
                                     : step_mat<kNeoHookean>(mode, P, A, n_tiles, s);
}

template <>
cudaError_t launch_adjoint<3>(int material, int mode, const SimParams& P, const AdjArgs& A,
                                int n_tiles, cudaStream_t s) {
  return material == kFixedCorotated ? adj_mat<kFixedCorotated>(mode, P, A, n_tiles, s)
                                     : adj_mat<kNeoHookean>(mode, P, A, n_tiles, s);
}

template <>
cudaError_t launch_clear<3>(const Clears& C, int nnodes, int n_grid, int n_scenes, int blocks_per_scene,
                          cudaStream_t s) {
  clear_kernel<3><<<dim3(blocks_per_scene, n_scenes), 256, 0, s>>>(C, nnodes, n_grid);
  return cudaGetLastError();
}

}  // namespace mpm
