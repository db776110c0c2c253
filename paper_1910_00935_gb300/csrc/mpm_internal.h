// mpm_internal.h -- host-side declarations shared by the C-ABI and the kernel
// translation units (launch wrappers; no device code).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <cuda_runtime.h>

#include "mpm_common.cuh"

namespace mpm {

struct StepArgs;
struct AdjArgs;
struct Clears;
struct PassEntry;
struct PersistCtl;

// kernels_*.cu (templates in kernels_launch.cuh; DET: deterministic fixed-point grids)
template <int D, int MAT, bool DET>
cudaError_t step_variant(int mode, const SimParams& P, const StepArgs& A, int n_tiles, cudaStream_t s);
template <int D, int MAT, bool DET>
cudaError_t adj_variant(int mode, const SimParams& P, const AdjArgs& A, int n_tiles, cudaStream_t s);
// one cooperative launch running plan[0..n_pass) (all of PassKind `kind`) with a bounded
// grid barrier between passes; P supplies the shared-memory capacities; *grid_out gets
// the CTA count
template <int D, int MAT, bool DET>
cudaError_t persistent_variant(int kind, const SimParams& P, const PassEntry* plan, int n_pass,
                               int n_tiles, const PersistCtl& ctl, cudaStream_t s, int* grid_out);
template <int D>
cudaError_t launch_clear(const Clears& C, int nnodes, int n_grid, int n_scenes, int blocks_per_scene,
                         cudaStream_t s);

// the message mpm_last_error(NULL) returns (per host thread)
void set_static_error(const char* msg);
// detail of the last failed kernel launch on this host thread (which pass, its dynamic
// shared memory), appended to the next CUDA error message and then cleared
void note_launch_failure(const char* kernel, int dim, int material, int mode, size_t smem,
                         cudaError_t attr_rc);
std::string take_launch_failure();

// dispatch on the runtime material and accumulation mode (P.det)
#define MPM_DISPATCH_MATERIAL(FN, ...)                                                   \
  switch (material) {                                                                   \
    case kFixedCorotated:                                                               \
      return P.det ? FN<D, kFixedCorotated, true>(__VA_ARGS__)                          \
                   : FN<D, kFixedCorotated, false>(__VA_ARGS__);                        \
    case kNeoHookean:                                                                   \
      return P.det ? FN<D, kNeoHookean, true>(__VA_ARGS__) : FN<D, kNeoHookean, false>(__VA_ARGS__); \
    case kLiquid:                                                                       \
      return P.det ? FN<D, kLiquid, true>(__VA_ARGS__) : FN<D, kLiquid, false>(__VA_ARGS__); \
    case kMixed:                                                                        \
      return P.det ? FN<D, kMixed, true>(__VA_ARGS__) : FN<D, kMixed, false>(__VA_ARGS__); \
  }                                                                                     \
  return cudaErrorInvalidValue;

template <int D>
inline cudaError_t launch_step(int material, int mode, const SimParams& P, const StepArgs& A,
                               int n_tiles, cudaStream_t s) {
  MPM_DISPATCH_MATERIAL(step_variant, mode, P, A, n_tiles, s)
}
template <int D>
inline cudaError_t launch_adjoint(int material, int mode, const SimParams& P, const AdjArgs& A,
                                  int n_tiles, cudaStream_t s) {
  MPM_DISPATCH_MATERIAL(adj_variant, mode, P, A, n_tiles, s)
}
template <int D>
inline cudaError_t launch_persistent(int kind, int material, const SimParams& P, const PassEntry* plan,
                                     int n_pass, int n_tiles, const PersistCtl& ctl, cudaStream_t s,
                                     int* grid_out) {
  MPM_DISPATCH_MATERIAL(persistent_variant, kind, P, plan, n_pass, n_tiles, ctl, s, grid_out)
}
#undef MPM_DISPATCH_MATERIAL

// setup.cu
size_t sort_temp_bytes(int64_t n);
cudaError_t launch_sort_keys(int dim, int n_grid, int n_scenes, const int64_t* scene_off, int64_t N,
                             const float* x0, int order, uint64_t* keys, int* idx, cudaStream_t s);
cudaError_t launch_sort(void* tmp, size_t tmp_bytes, const uint64_t* keys_in, uint64_t* keys_out,
                        const int* idx_in, int* idx_out, int64_t N, int end_bit, cudaStream_t s);
cudaError_t launch_gather_initial(int dim, int64_t N, const int* perm, const float* x0,
                                  const float* v0, const float* C0, const float* F0, const float* E,
                                  const float* nu, const int* group_in, float* state, float* mu,
                                  float* la, float* Eo, float* nuo, int* group_out, cudaStream_t s);
// reset n_boxes consecutive [8]-int boxes to empty (lo = INT_MAX, hi = INT_MIN)
cudaError_t launch_reset_boxes(int* boxes, int64_t n_boxes, cudaStream_t s);
cudaError_t launch_gather_rows(int rows, int64_t N, const int* perm, const float* src_caller,
                               float* dst_internal, cudaStream_t s);
// dst[i] = src[perm[i]] for int32 rows (per-particle material ids)
cudaError_t launch_gather_int(int64_t N, const int* perm, const int* src_caller, int* dst_internal,
                              cudaStream_t s);
// identity_dim > 0: rows are a dim x dim matrix per particle and I is added on the way out;
// the first fix_rows rows hold fixed-point positions, converted to FP32 on the way out
cudaError_t launch_scatter_rows(int rows, int64_t N, const int* perm, const float* src_internal,
                                float* dst_caller, int identity_dim, int fix_rows, cudaStream_t s);
cudaError_t launch_material_grad(int64_t N, const int* perm, const float* E, const float* nu,
                                 const float2* mubar, const float2* labar, float* gE, float* gnu,
                                 cudaStream_t s);
// per-scene sums of x_T and x_0 (state rows, fixed-point positions) into com[scene][6];
// part: com_scratch_doubles(n_scenes)
size_t com_scratch_doubles(int n_scenes);
cudaError_t launch_com(int dim, int64_t N, int n_scenes, const int64_t* scene_off, const int* perm,
                       const float* xT, const float* x0, double* part, double* com, cudaStream_t s);
// out[scene][gk] = sum over the scene's tiles (tile_off[scene] .. tile_off[scene+1]) in order
cudaError_t launch_wbar_reduce(int n_scenes, int gk, const int* tile_off, const float* wbar_tile,
                               float* out, cudaStream_t s);
cudaError_t launch_loss_seed(int dim, int kind, int64_t N, int n_scenes, const int64_t* scene_off,
                             const int* perm, const double* com, const float* target, float* loss,
                             float* dL_dxT, float* dL_dx0, cudaStream_t s);

// controller.cu (closed-loop controller): sensing + MLP of one forward step, writing the
// step's inputs u, hidden h, pre-scale outputs y, actuation act[scene][G] and group sizes
// cnt[scene][G+1]; part: n_tiles x (G+1) x 7 doubles
cudaError_t launch_ctrl_forward(const CtrlStep& cs, int n_scenes, int n_tiles, int64_t N,
                                const int4* tiles, const int* tile_off, const float* st,
                                const int* group, double* part, const float* theta, double* u,
                                double* h, double* y, float* act, double* cnt, cudaStream_t s);
// reverse of one step: reads (and clears) the per-tile actuation adjoints abar_tile[tile][G],
// accumulates dL/dtheta into thbar (FP64) and adds the sensor terms to the x and v rows of
// the state adjoint adj; add: n_scenes x (G+1) x 2 dim floats of scratch
cudaError_t launch_ctrl_backward(const CtrlStep& cs, int n_scenes, int n_tiles, int64_t N,
                                 const int4* tiles, const int* tile_off, const int* group,
                                 float* abar_tile, const float* theta, const double* u,
                                 const double* h, const double* y, const double* cnt,
                                 double* thbar, float* add, float* adj, cudaStream_t s);
cudaError_t launch_ctrl_grad_out(int64_t n, const double* thbar, float* gw, cudaStream_t s);

}  // namespace mpm
