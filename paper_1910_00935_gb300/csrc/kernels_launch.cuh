// kernels_launch.cuh -- launch wrappers of the particle passes, the persistent pass
// interpreters and the grid clear, templated on dimension, material and accumulation
// (FP32 or deterministic fixed point).  The kernels_*.cu translation units each
// instantiate a share of the variants so that they compile in parallel; the dispatch on
// the runtime material and mode is in mpm_internal.h and here.
#pragma once

#include "mpm_internal.h"
#include "mpm_kernels.cuh"

namespace mpm {

namespace {
// Raise a kernel's dynamic shared-memory limit when static + dynamic may pass the default
// 48 KB: the passes' static shared memory (box slots, bucket table, group sums, the
// persistent forms' pass entry) stays below 8 KB, so any dynamic size above 32 KB sets it.
template <typename K>
cudaError_t allow_smem(K k, size_t smem) {
  if (smem <= 32 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <int D, int MAT, int MODE, bool DET>
cudaError_t step_one(const SimParams& P, const StepArgs& A, int n_tiles, cudaStream_t s) {
  const size_t smem = step_smem_bytes<D>(P.tile_capacity, P.gather_capacity);
  auto k = step_kernel<D, MAT, MODE, DET>;
  cudaError_t e = allow_smem(k, smem);
  if (e != cudaSuccess) {
    note_launch_failure("step_kernel", D, MAT, MODE, smem, e);
    return e;
  }
  if (n_tiles <= 0) {  // no tiles: only make sure the kernel's module is loaded
    cudaFuncAttributes attr;
    return cudaFuncGetAttributes(&attr, k);
  }
  k<<<n_tiles, kTile, smem, s>>>(P, A);
  e = cudaGetLastError();
  if (e != cudaSuccess) note_launch_failure("step_kernel", D, MAT, MODE, smem, cudaSuccess);
  return e;
}

template <int D, int MAT, int MODE, bool DET>
cudaError_t adj_one(const SimParams& P, const AdjArgs& A, int n_tiles, cudaStream_t s) {
  const size_t smem = adj_smem_bytes<D>(P.tile_capacity, P.gather_capacity);
  auto k = adjoint_kernel<D, MAT, MODE, DET>;
  cudaError_t e = allow_smem(k, smem);
  if (e != cudaSuccess) {
    note_launch_failure("adjoint_kernel", D, MAT, MODE, smem, e);
    return e;
  }
  if (n_tiles <= 0) {  // no tiles: only make sure the kernel's module is loaded
    cudaFuncAttributes attr;
    return cudaFuncGetAttributes(&attr, k);
  }
  k<<<n_tiles, kTile, smem, s>>>(P, A);
  e = cudaGetLastError();
  if (e != cudaSuccess) note_launch_failure("adjoint_kernel", D, MAT, MODE, smem, cudaSuccess);
  return e;
}

// Cooperative launch of a persistent pass interpreter: as many CTAs as can be resident
// at once (occupancy x SMs), at most one per tile.
template <typename K>
cudaError_t persistent_one(K k, size_t smem, const PassEntry* plan, int n_pass, int n_tiles,
                           const PersistCtl& ctl, cudaStream_t s, int* grid_out) {
  cudaError_t e = allow_smem(k, smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kTile, smem)) != cudaSuccess)
    return e;
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
  int grid = per_sm * sms;
  if (grid > n_tiles) grid = n_tiles;
  if (grid_out) *grid_out = grid;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kTile);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, plan, n_pass, n_tiles, ctl);
}
}  // namespace

template <int D, int MAT, bool DET>
cudaError_t step_variant(int mode, const SimParams& P, const StepArgs& A, int n_tiles, cudaStream_t s) {
  switch (mode) {
    case kP2GOnly: return step_one<D, MAT, kP2GOnly, DET>(P, A, n_tiles, s);
    case kG2PP2G: return step_one<D, MAT, kG2PP2G, DET>(P, A, n_tiles, s);
    case kG2PP2GFull: return step_one<D, MAT, kG2PP2GFull, DET>(P, A, n_tiles, s);
    case kG2POnlyFull: return step_one<D, MAT, kG2POnlyFull, DET>(P, A, n_tiles, s);
  }
  return cudaErrorInvalidValue;
}

template <int D, int MAT, bool DET>
cudaError_t adj_variant(int mode, const SimParams& P, const AdjArgs& A, int n_tiles, cudaStream_t s) {
  switch (mode) {
    case kAdjG2P: return adj_one<D, MAT, kAdjG2P, DET>(P, A, n_tiles, s);
    case kAdjFused: return adj_one<D, MAT, kAdjFused, DET>(P, A, n_tiles, s);
    case kAdjP2G: return adj_one<D, MAT, kAdjP2G, DET>(P, A, n_tiles, s);
  }
  return cudaErrorInvalidValue;
}

// kind_mode = PassKind * 8 + the run's pass mode (StepMode or AdjMode)
template <int D, int MAT, bool DET>
cudaError_t persistent_variant(int kind_mode, const SimParams& P, const PassEntry* plan, int n_pass,
                               int n_tiles, const PersistCtl& ctl, cudaStream_t s, int* grid_out) {
  const size_t ss = step_smem_bytes<D>(P.tile_capacity, P.gather_capacity);
  const size_t as = adj_smem_bytes<D>(P.tile_capacity, P.gather_capacity);
  switch (kind_mode) {
    case kPassStep * 8 + kP2GOnly:
      return persistent_one(step_persistent_kernel<D, MAT, kP2GOnly, DET>, ss, plan, n_pass, n_tiles, ctl, s, grid_out);
    case kPassStep * 8 + kG2PP2G:
      return persistent_one(step_persistent_kernel<D, MAT, kG2PP2G, DET>, ss, plan, n_pass, n_tiles, ctl, s, grid_out);
    case kPassStep * 8 + kG2PP2GFull:
      return persistent_one(step_persistent_kernel<D, MAT, kG2PP2GFull, DET>, ss, plan, n_pass, n_tiles, ctl, s, grid_out);
    case kPassStep * 8 + kG2POnlyFull:
      return persistent_one(step_persistent_kernel<D, MAT, kG2POnlyFull, DET>, ss, plan, n_pass, n_tiles, ctl, s, grid_out);
    case kPassAdjoint * 8 + kAdjG2P:
      return persistent_one(adjoint_persistent_kernel<D, MAT, kAdjG2P, DET>, as, plan, n_pass, n_tiles, ctl, s, grid_out);
    case kPassAdjoint * 8 + kAdjFused:
      return persistent_one(adjoint_persistent_kernel<D, MAT, kAdjFused, DET>, as, plan, n_pass, n_tiles, ctl, s, grid_out);
    case kPassAdjoint * 8 + kAdjP2G:
      return persistent_one(adjoint_persistent_kernel<D, MAT, kAdjP2G, DET>, as, plan, n_pass, n_tiles, ctl, s, grid_out);
  }
  return cudaErrorInvalidValue;
}

template <int D>
cudaError_t launch_clear(const Clears& C, int nnodes, int n_grid, int n_scenes, int blocks_per_scene,
                         cudaStream_t s) {
  clear_kernel<D><<<dim3(blocks_per_scene, n_scenes), 256, 0, s>>>(C, nnodes, n_grid);
  return cudaGetLastError();
}

}  // namespace mpm
