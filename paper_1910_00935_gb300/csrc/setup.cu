// setup.cu -- one-time set-up, permutation, loss and output kernels.
//
// Particles are reordered once per mpm_set_initial by (scene, Morton code of the
// initial stencil base) so that every P2G tile covers a compact block of cells; an elastic
// body keeps its neighbours, so the order stays coherent for the whole run and the
// tape never has to record a permutation.  Every input is gathered into that order
// and every output scattered back to the caller's.
#include <climits>
#include <cub/device/device_radix_sort.cuh>

#include "mpm_internal.h"

namespace mpm {

namespace {

__device__ __forceinline__ uint32_t spread2(uint32_t v) {  // 16 bits -> every 2nd bit
  v &= 0xFFFFu;
  v = (v | (v << 8)) & 0x00FF00FFu;
  v = (v | (v << 4)) & 0x0F0F0F0Fu;
  v = (v | (v << 2)) & 0x33333333u;
  v = (v | (v << 1)) & 0x55555555u;
  return v;
}

__device__ __forceinline__ uint32_t spread3(uint32_t v) {  // 10 bits -> every 3rd bit
  v &= 0x3FFu;
  v = (v | (v << 16)) & 0x030000FFu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

__device__ __forceinline__ int scene_of(const int64_t* off, int n_scenes, int64_t p) {
  int lo = 0, hi = n_scenes - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= p) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Sort keys (`order`, MPM_OPT_SORT_ORDER).  Every order is (scene, a grid coordinate c per
// axis, which half of that coordinate's cell the particle sits in along each axis), with the
// coordinates in runs of 8 along the last axis (the grid's contiguous one) and the runs in
// Morton order of (other axes, run index), the second axis lowest: a 3D tile of 128 lattice
// particles then covers 1 x 2 x 8 coordinates, and the lanes of a reduction instruction hit
// nodes in z-runs (fewer L2 requests than a 2 x 2 x 4 Morton block, measured).  The half
// bits vary fastest, the last axis's first.
//  0: c = the cell floor(x/dx) on every axis.
//  1: c = the stencil base floor(x/dx - 0.5) on every axis: the particles sharing a base (the
//     ones that scatter to the same 3^D nodes) are contiguous.
//  2: cells on the other axes, the base on the last: consecutive pairs (last-axis halves 0, 1)
//     share their whole base, which the pair-merged scatter exploits, while the tile's lanes
//     still spread over the cells' distinct bases.
__global__ void sort_keys_kernel(int dim, int n_grid, int n_scenes, const int64_t* off, int64_t N,
                                 const float* x0, int order, uint64_t* keys, int* idx) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N;
       p += (int64_t)gridDim.x * blockDim.x) {
    uint32_t c[3] = {0, 0, 0}, half = 0;
    for (int a = 0; a < dim; ++a) {
      const bool by_base = order == 1 || (order == 2 && a == dim - 1);
      float X = x0[a * N + p] * (float)n_grid - (by_base ? 0.5f : 0.0f);
      int ci = 0, h = 0;
      if (X == X) {
        const float b = fminf(fmaxf(floorf(X), 0.0f), (float)(n_grid - 1));
        ci = (int)b;
        h = X - b >= 0.5f ? 1 : 0;
      }
      c[a] = (uint32_t)ci;
      half = (half << 1) | (uint32_t)h;
    }
    const uint32_t last = c[dim - 1];
    uint64_t m = dim == 2 ? (spread2(last >> 3) | (spread2(c[0]) << 1))
                          : (spread3(c[1]) | (spread3(c[0]) << 1) | (spread3(last >> 3) << 2));
    m = (m << 3) | (last & 7u);
    keys[p] = ((uint64_t)scene_of(off, n_scenes, p) << 36) | (m << 3) | half;
    idx[p] = (int)p;
  }
}

__global__ void gather_initial_kernel(int dim, int64_t N, const int* perm, const float* x0,
                                      const float* v0, const float* C0, const float* F0,
                                      const float* E, const float* nu, const int* group_in,
                                      float* st, float* mu, float* la, float* Eo, float* nuo,
                                      int* group_out) {
  const int dd = dim * dim;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = perm[i];
    for (int a = 0; a < dim; ++a) {
      st[a * N + i] = pos_to_fix(x0[a * N + e]);  // positions in fixed point (mpm_common.cuh)
      st[(dim + a) * N + i] = v0[a * N + e];
    }
    for (int k = 0; k < dd; ++k) {
      // the deformation gradient is stored as E = F - I
      const float id = (k / dim == k % dim) ? 1.0f : 0.0f;
      st[(2 * dim + k) * N + i] = C0 ? C0[k * N + e] : 0.0f;
      st[(2 * dim + dd + k) * N + i] = F0 ? F0[k * N + e] - id : 0.0f;
    }
    float Ee = E[e], ne = nu[e];
    Eo[i] = Ee;
    nuo[i] = ne;
    // Lame parameters of Young's modulus and Poisson ratio
    mu[i] = Ee / (2.0f * (1.0f + ne));
    la[i] = Ee * ne / ((1.0f + ne) * (1.0f - 2.0f * ne));
    group_out[i] = group_in ? group_in[e] : 0;
  }
}

__global__ void reset_boxes_kernel(int* boxes, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n * 8;
       i += (int64_t)gridDim.x * blockDim.x)
    boxes[i] = (i % 8) < 4 ? INT_MAX : INT_MIN;
}

__global__ void gather_int_kernel(int64_t N, const int* perm, const int* src, int* dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[perm[i]];
}

__global__ void gather_rows_kernel(int rows, int64_t N, const int* perm, const float* src,
                                   float* dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = perm[i];
    for (int r = 0; r < rows; ++r) dst[r * N + i] = src ? src[r * N + e] : 0.0f;
  }
}

__global__ void scatter_rows_kernel(int rows, int64_t N, const int* perm, const float* src,
                                    float* dst, int identity_dim, int fix_rows) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = perm[i];
    for (int r = 0; r < rows; ++r) {
      if (r < fix_rows) {
        dst[r * N + e] = (float)pos_from_fix(src[r * N + i]);
        continue;
      }
      float add = (identity_dim > 0 && r / identity_dim == r % identity_dim) ? 1.0f : 0.0f;
      dst[r * N + e] = src[r * N + i] + add;
    }
  }
}

// chain rule of the Lame parameters: (mubar, labar) -> (Ebar, nubar), in FP64 (the two
// terms of dL/dnu have opposite signs and nearly cancel); the sums arrive as compensated FP32
// (value, correction) pairs
__global__ void material_grad_kernel(int64_t N, const int* perm, const float* E, const float* nu,
                                     const float2* mubar, const float2* labar, float* gE,
                                     float* gnu) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = perm[i];
    const double Ee = E[i], v = nu[i];
    const double q = (1.0 + v) * (1.0 - 2.0 * v);
    const double mb = (double)mubar[i].x + (double)mubar[i].y;
    const double lb = (double)labar[i].x + (double)labar[i].y;
    if (gE) gE[e] = (float)(mb / (2.0 * (1.0 + v)) + lb * v / q);
    if (gnu) gnu[e] = (float)(-mb * Ee / (2.0 * (1.0 + v) * (1.0 + v)) + lb * Ee * (1.0 + 2.0 * v * v) / (q * q));
  }
}

// per-scene sums of x_T and x_0 (FP64): one CTA per (scene, chunk) writes its partial
// sums part[scene][chunk][6]; com_final_kernel adds the chunks in order (no atomics, so
// the sums do not depend on scheduling)
constexpr int kComChunks = 64;
__global__ void com_kernel(int dim, int n_scenes, const int64_t* off, int64_t N, const float* xT,
                           const float* x0, double* part) {
  __shared__ double red[6][256 / 32];
  const int s = blockIdx.y;
  const int64_t b = off[s], e = off[s + 1];
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t i = b + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < e;
       i += (int64_t)gridDim.x * blockDim.x)
    for (int a = 0; a < dim; ++a) {  // the state rows hold fixed-point positions
      acc[a] += pos_from_fix(xT[a * N + i]);
      acc[3 + a] += pos_from_fix(x0[a * N + i]);
    }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c = 0; c < 6; ++c) {
    double v = acc[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[c][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[threadIdx.x][w];
    part[((int64_t)s * kComChunks + blockIdx.x) * 6 + threadIdx.x] = v;
  }
}

__global__ void com_final_kernel(int n_scenes, const double* part, double* com) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_scenes * 6) return;
  const int s = i / 6, c = i % 6;
  double v = 0.0;
  for (int k = 0; k < kComChunks; ++k) v += part[((int64_t)s * kComChunks + k) * 6 + c];
  com[i] = v;
}

// dL/dw[scene][g][k] = sum over the scene's tiles, in tile order, of the per-tile partials
__global__ void wbar_reduce_kernel(int n_scenes, int gk, const int* tile_off, const float* wbar_tile,
                                   float* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_scenes * gk) return;
  const int s = i / gk, c = i % gk;
  float v = 0.0f;
  for (int t = tile_off[s]; t < tile_off[s + 1]; ++t) v += wbar_tile[(int64_t)t * gk + c];
  out[i] = v;
}

__global__ void loss_seed_kernel(int dim, int kind, int64_t N, int n_scenes, const int64_t* off,
                                 const int* perm, const double* com, const float* target,
                                 float* loss, float* gT, float* g0) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int s = scene_of(off, n_scenes, i);
    const double n_s = (double)(off[s + 1] - off[s]);
    const int64_t e = perm[i];
    double L = 0.0;
    for (int a = 0; a < dim; ++a) {
      double c = com[s * 6 + a] / n_s, c0 = com[s * 6 + 3 + a] / n_s;
      double seedT = 0.0, seed0 = 0.0;
      if (kind == 0) {
        double r = c - (double)target[s * dim + a];
        L += r * r;
        seedT = 2.0 * r / n_s;
      } else if (a == 0) {
        L = -(c - c0);
        seedT = -1.0 / n_s;
        seed0 = 1.0 / n_s;
      }
      gT[a * N + e] = (float)seedT;
      if (g0) g0[a * N + e] = (float)seed0;
    }
    if (i == off[s] && loss) loss[s] = (float)L;
  }
}

inline int grid_for(int64_t n, int threads = 256) {
  int64_t b = (n + threads - 1) / threads;
  return (int)(b < 1 ? 1 : (b > 65535 ? 65535 : b));
}

}  // namespace

size_t sort_temp_bytes(int64_t n) {
  size_t bytes = 0;
  cudaError_t e = cub::DeviceRadixSort::SortPairs(nullptr, bytes, (const uint64_t*)nullptr,
                                                  (uint64_t*)nullptr, (const int*)nullptr,
                                                  (int*)nullptr, (int)n, 0, 64, (cudaStream_t)0);
  if (e != cudaSuccess) {
    // no device to query (size-only call on a host without a GPU): a safe upper bound
    cudaGetLastError();
    bytes = (size_t)32 * 1024 * 1024 + (size_t)n * 16;
  }
  return bytes;
}

cudaError_t launch_sort_keys(int dim, int n_grid, int n_scenes, const int64_t* scene_off, int64_t N,
                             const float* x0, int order, uint64_t* keys, int* idx,
                             cudaStream_t s) {
  sort_keys_kernel<<<grid_for(N), 256, 0, s>>>(dim, n_grid, n_scenes, scene_off, N, x0, order, keys, idx);
  return cudaGetLastError();
}

cudaError_t launch_sort(void* tmp, size_t tmp_bytes, const uint64_t* keys_in, uint64_t* keys_out,
                        const int* idx_in, int* idx_out, int64_t N, int end_bit, cudaStream_t s) {
  return cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, keys_in, keys_out, idx_in, idx_out, (int)N,
                                         0, end_bit, s);
}

cudaError_t launch_gather_initial(int dim, int64_t N, const int* perm, const float* x0,
                                  const float* v0, const float* C0, const float* F0, const float* E,
                                  const float* nu, const int* group_in, float* state, float* mu,
                                  float* la, float* Eo, float* nuo, int* group_out, cudaStream_t s) {
  gather_initial_kernel<<<grid_for(N), 256, 0, s>>>(dim, N, perm, x0, v0, C0, F0, E, nu, group_in,
                                                    state, mu, la, Eo, nuo, group_out);
  return cudaGetLastError();
}

cudaError_t launch_reset_boxes(int* boxes, int64_t n_boxes, cudaStream_t s) {
  reset_boxes_kernel<<<grid_for(n_boxes * 8), 256, 0, s>>>(boxes, n_boxes);
  return cudaGetLastError();
}

cudaError_t launch_gather_rows(int rows, int64_t N, const int* perm, const float* src_caller,
                               float* dst_internal, cudaStream_t s) {
  gather_rows_kernel<<<grid_for(N), 256, 0, s>>>(rows, N, perm, src_caller, dst_internal);
  return cudaGetLastError();
}

cudaError_t launch_gather_int(int64_t N, const int* perm, const int* src_caller, int* dst_internal,
                              cudaStream_t s) {
  gather_int_kernel<<<grid_for(N), 256, 0, s>>>(N, perm, src_caller, dst_internal);
  return cudaGetLastError();
}

cudaError_t launch_scatter_rows(int rows, int64_t N, const int* perm, const float* src_internal,
                                float* dst_caller, int identity_dim, int fix_rows, cudaStream_t s) {
  scatter_rows_kernel<<<grid_for(N), 256, 0, s>>>(rows, N, perm, src_internal, dst_caller,
                                                  identity_dim, fix_rows);
  return cudaGetLastError();
}

cudaError_t launch_material_grad(int64_t N, const int* perm, const float* E, const float* nu,
                                 const float2* mubar, const float2* labar, float* gE, float* gnu,
                                 cudaStream_t s) {
  material_grad_kernel<<<grid_for(N), 256, 0, s>>>(N, perm, E, nu, mubar, labar, gE, gnu);
  return cudaGetLastError();
}

size_t com_scratch_doubles(int n_scenes) { return (size_t)n_scenes * kComChunks * 6; }

cudaError_t launch_com(int dim, int64_t N, int n_scenes, const int64_t* scene_off, const int* perm,
                       const float* xT, const float* x0, double* part, double* com, cudaStream_t s) {
  (void)perm;
  com_kernel<<<dim3(kComChunks, n_scenes), 256, 0, s>>>(dim, n_scenes, scene_off, N, xT, x0, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  com_final_kernel<<<(n_scenes * 6 + 255) / 256, 256, 0, s>>>(n_scenes, part, com);
  return cudaGetLastError();
}

cudaError_t launch_wbar_reduce(int n_scenes, int gk, const int* tile_off, const float* wbar_tile,
                               float* out, cudaStream_t s) {
  wbar_reduce_kernel<<<(n_scenes * gk + 255) / 256, 256, 0, s>>>(n_scenes, gk, tile_off, wbar_tile, out);
  return cudaGetLastError();
}

cudaError_t launch_loss_seed(int dim, int kind, int64_t N, int n_scenes, const int64_t* scene_off,
                             const int* perm, const double* com, const float* target, float* loss,
                             float* dL_dxT, float* dL_dx0, cudaStream_t s) {
  loss_seed_kernel<<<grid_for(N), 256, 0, s>>>(dim, kind, N, n_scenes, scene_off, perm, com, target,
                                               loss, dL_dxT, dL_dx0);
  return cudaGetLastError();
}

}  // namespace mpm
