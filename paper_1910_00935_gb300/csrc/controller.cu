// controller.cu -- the closed-loop controller of the actuated bodies (the neural-network
// controllers of Section 4.1): at every step the sensors of the current state feed a
// small MLP whose outputs are the actuation of the groups, and the reverse pass carries
// the actuation adjoint back through the MLP to its weights and to the sensed state.
//
//   inputs u (n_in = K + 2 d G): sin(2 pi k t / P + phi) for k = 1..K, then per group g
//     the offset of its centre of mass from the body's (d values) and its mean velocity
//     (d values); an empty group reads zeros
//   h = tanh(W1 u + b1) (H units), a_g = scale tanh(W2 h + b2)_g
//   theta per scene = [W1 (H x n_in, row-major) | b1 (H) | W2 (G x H, row-major) | b2 (G)]
//
// Weights arrive in FP32; a tile's sensor sums are FP32, the sums over tiles, the inputs and
// the MLP's dot products FP64 (a few thousand operations per scene and step, one warp per
// dot product), the activations tanh in FP32.  Every sum runs in a fixed order (a
// tile's particles in order, a scene's tiles in order), so the controller adds nothing
// order-dependent to a deterministic run.
#include "mpm_internal.h"

namespace mpm {

namespace {

constexpr int kSenseThreads = kTile;  // one CTA per particle tile
static_assert(kTile <= 512, "the sensing CTA stages a tile's values in static shared memory");
constexpr int kCtrlThreads = 1024;    // one CTA per scene for the MLP passes
constexpr int kSenseVals = 7;       // x (d), v (d), count: at most 7
constexpr int kSenseSlots = kMaxGroups + 1;  // slot 0: particles in no group

// out[j] = sum over t in [t0, t1) of a[t * stride + j] for j < nv, by the whole CTA: thread
// (j, r) sums rows t0 + r, t0 + r + R, ... (R = blockDim / nv) with four independent
// accumulators (loads in flight together), then each out[j] adds its R partials in order.
// The order depends only on (t0, t1), so the sums are reproducible.  clear: zero every
// element read (the per-tile actuation adjoints are consumed).  scratch: blockDim doubles;
// out: shared, nv doubles.  Ends with a barrier.
template <typename T>
__device__ void block_tile_sums(T* a, int t0, int t1, int stride, int nv, bool clear,
                                double* scratch, double* out) {
  const int R = blockDim.x / nv;
  const int j = threadIdx.x % nv, r = threadIdx.x / nv;
  double acc = 0.0;
  if (r < R) {
    double q[4] = {0.0, 0.0, 0.0, 0.0};
    int t = t0 + r;
    for (; t + 3 * R < t1; t += 4 * R) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        T* e = a + (int64_t)(t + u * R) * stride + j;
        q[u] += (double)*e;
        if (clear) *e = T(0);
      }
    }
    for (; t < t1; t += R) {
      T* e = a + (int64_t)t * stride + j;
      q[0] += (double)*e;
      if (clear) *e = T(0);
    }
    acc = (q[0] + q[1]) + (q[2] + q[3]);
  }
  scratch[threadIdx.x] = acc;
  __syncthreads();
  if ((int)threadIdx.x < nv) {
    double v = 0.0;
    for (int k = 0; k < R; ++k) v += scratch[k * nv + threadIdx.x];
    out[threadIdx.x] = v;
  }
  __syncthreads();
}

// sum of v over the 32 lanes of the warp, the same butterfly order on every run (all lanes
// must call it)
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Per-tile sums of x, v and the particle count by group slot, in particle order:
// part[tile][slot][value], value = x_0..x_{d-1}, v_0..v_{d-1}, count.  A tile's at most 128
// terms are summed in FP32 (FP64 adds run at 1/64 of the FP32 rate and made this the
// controller's slowest step); the sums over a scene's tiles are FP64.
__global__ void ctrl_sense_kernel(int dim, int G, int64_t N, const int4* tiles, const float* st,
                                  const int* group, double* part) {
  // rows padded by one: the threads summing different values of the same particle then
  // read different banks
  __shared__ float vals[kSenseVals][kSenseThreads + 1];
  __shared__ int slot[kSenseThreads];
  const int4 tile = tiles[blockIdx.x];
  const int i = threadIdx.x;
  const int nv = 2 * dim + 1, ns = G + 1;
  if (i < tile.z) {
    const int64_t p = (int64_t)tile.y + i;
    const int g = group[p];
    slot[i] = (g >= 0 && g < G) ? g + 1 : 0;
    for (int a = 0; a < dim; ++a) {
      vals[a][i] = (float)pos_from_fix(st[(int64_t)a * N + p]);  // fixed-point position rows
      vals[dim + a][i] = st[(int64_t)(dim + a) * N + p];
    }
    vals[2 * dim][i] = 1.0f;
  }
  __syncthreads();
  for (int j = i; j < ns * nv; j += blockDim.x) {
    const int sl = j / nv, c = j % nv;
    float acc = 0.0f;
    for (int q = 0; q < tile.z; ++q)
      if (slot[q] == sl) acc += vals[c][q];
    part[(int64_t)blockIdx.x * ns * nv + j] = (double)acc;
  }
}

// One CTA per scene: reduce the scene's tile sums in order, form the inputs, run the MLP
// and store u, h, y = tanh(W2 h + b2) (kept for the reverse pass), the actuation
// a = scale y, and the group sizes.
__global__ void __launch_bounds__(kCtrlThreads) ctrl_forward_kernel(CtrlStep cs, const int* tile_off, const double* part,
                                    const float* theta, double* u_out, double* h_out,
                                    double* y_out, float* act_out, double* cnt_out) {
  __shared__ double sums[kSenseSlots * kSenseVals];
  __shared__ double u[kCtrlMaxInputs];
  __shared__ double hs[kCtrlMaxHidden];
  const int s = blockIdx.x;
  const int dim = cs.dim, G = cs.G, K = cs.K, H = cs.H;
  const int nv = 2 * dim + 1, ns = G + 1;
  const int n_in = K + 2 * dim * G;
  const int n_par = H * n_in + H + G * H + G;
  const float* th = theta + (int64_t)s * n_par;
  __shared__ double scratch[kCtrlThreads];
  block_tile_sums(const_cast<double*>(part), tile_off[s], tile_off[s + 1], ns * nv, ns * nv, false,
                  scratch, sums);
  // inputs: the time basis, then per group (centre offset, mean velocity)
  for (int i = threadIdx.x; i < n_in; i += blockDim.x) {
    double val;
    if (i < K) {
      val = cs.basis[i];
    } else {
      const int r = i - K, g = r / (2 * dim), c = r % (2 * dim);
      const double n_g = sums[(g + 1) * nv + 2 * dim];
      if (n_g <= 0.0) {
        val = 0.0;
      } else if (c < dim) {
        double tot = 0.0, cnt = 0.0;
        for (int q = 0; q < ns; ++q) {
          tot += sums[q * nv + c];
          cnt += sums[q * nv + 2 * dim];
        }
        val = sums[(g + 1) * nv + c] / n_g - tot / cnt;
      } else {
        val = sums[(g + 1) * nv + c] / n_g;
      }
    }
    u[i] = val;
    u_out[(int64_t)s * n_in + i] = val;
  }
  if ((int)threadIdx.x < ns) cnt_out[s * ns + threadIdx.x] = sums[threadIdx.x * nv + 2 * dim];
  __syncthreads();
  const float* W1 = th;
  const float* b1 = th + H * n_in;
  const float* W2 = b1 + H;
  const float* b2 = W2 + G * H;
  // one warp per hidden unit (then per output): its lanes take the dot product's terms and
  // a butterfly sums them, instead of one thread running the whole chain while the CTA
  // waits at the barrier
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, n_warps = blockDim.x >> 5;
  for (int j = warp; j < H; j += n_warps) {
    double z = 0.0;
    for (int i = lane; i < n_in; i += 32) z += (double)W1[j * n_in + i] * u[i];
    z = warp_sum(z);
    if (lane == 0) {
      // the activation in FP32: FP64 transcendentals run on the FP64 pipe (1/64 of the FP32
      // rate here) and made these one-CTA-per-scene kernels latency chains
      const double hj = (double)tanhf((float)(z + (double)b1[j]));
      hs[j] = hj;
      h_out[(int64_t)s * H + j] = hj;
    }
  }
  __syncthreads();
  for (int g = warp; g < G; g += n_warps) {
    double z = 0.0;
    for (int j = lane; j < H; j += 32) z += (double)W2[g * H + j] * hs[j];
    z = warp_sum(z);
    if (lane == 0) {
      const double y = (double)tanhf((float)(z + (double)b2[g]));
      y_out[(int64_t)s * G + g] = y;
      act_out[(int64_t)s * G + g] = (float)((double)cs.scale * y);
    }
  }
}

// One CTA per scene, reverse of the controller at one step: abar_g = the scene's per-tile
// actuation adjoints summed in tile order (and the tile slots cleared for the next step);
// dL/dtheta accumulates in FP64 (thbar); the sensor adjoint becomes per-slot additions to
// the state adjoint: add[scene][slot][0..d) to xbar, [d..2d) to vbar.
__global__ void __launch_bounds__(kCtrlThreads) ctrl_backward_kernel(CtrlStep cs, const int* tile_off, float* abar_tile,
                                     const float* theta, const double* u_in, const double* h_in,
                                     const double* y_in, const double* cnt, double* thbar,
                                     float* add) {
  __shared__ double z2b[kMaxGroups];
  __shared__ double z1b[kCtrlMaxHidden];
  __shared__ double ub[kCtrlMaxInputs];
  __shared__ double body[3];
  const int s = blockIdx.x;
  const int dim = cs.dim, G = cs.G, K = cs.K, H = cs.H;
  const int ns = G + 1;
  const int n_in = K + 2 * dim * G;
  const int n_par = H * n_in + H + G * H + G;
  const float* th = theta + (int64_t)s * n_par;
  const float* W1 = th;
  const float* W2 = th + H * n_in + H;
  double* W1b = thbar + (int64_t)s * n_par;
  double* b1b = W1b + H * n_in;
  double* W2b = b1b + H;
  double* b2b = W2b + G * H;
  const double* u = u_in + (int64_t)s * n_in;
  const double* h = h_in + (int64_t)s * H;
  // the scene's per-tile actuation adjoints, summed and cleared for the next step
  __shared__ double scratch[kCtrlThreads];
  __shared__ double abar[kMaxGroups];
  block_tile_sums(abar_tile, tile_off[s], tile_off[s + 1], G, G, true, scratch, abar);
  if ((int)threadIdx.x < G) {
    const int g = threadIdx.x;
    const double y = y_in[(int64_t)s * G + g];
    const double zb = abar[g] * (double)cs.scale * (1.0 - y * y);
    z2b[g] = zb;
    b2b[g] += zb;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < H; j += blockDim.x) {
    double hb = 0.0;
    for (int g = 0; g < G; ++g) {
      W2b[g * H + j] += z2b[g] * h[j];
      hb += (double)W2[g * H + j] * z2b[g];
    }
    const double zb = hb * (1.0 - h[j] * h[j]);
    z1b[j] = zb;
    b1b[j] += zb;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < H * n_in; e += blockDim.x) W1b[e] += z1b[e / n_in] * u[e % n_in];
  {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, n_warps = blockDim.x >> 5;
    for (int i = warp; i < n_in; i += n_warps) {  // one warp per input, as in the forward
      double acc = 0.0;
      for (int j = lane; j < H; j += 32) acc += (double)W1[j * n_in + i] * z1b[j];
      acc = warp_sum(acc);
      if (lane == 0) ub[i] = acc;
    }
  }
  __syncthreads();
  // u_xg = mean_{p in g} x_p - mean_p x_p: every particle carries -sum_g ub_xg / N, and
  // its own group's ub_xg / N_g; u_vg = mean_{p in g} v_p: ub_vg / N_g
  if ((int)threadIdx.x < dim) {
    const int a = threadIdx.x;
    double tot = 0.0, n = 0.0;
    for (int q = 0; q < ns; ++q) n += cnt[s * ns + q];
    for (int g = 0; g < G; ++g)
      if (cnt[s * ns + g + 1] > 0.0) tot += ub[K + g * 2 * dim + a];
    body[a] = n > 0.0 ? tot / n : 0.0;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < ns * 2 * dim; j += blockDim.x) {
    const int sl = j / (2 * dim), c = j % (2 * dim);
    double v = 0.0;
    if (c < dim) v = -body[c];
    if (sl > 0) {
      const double n_g = cnt[s * ns + sl];
      if (n_g > 0.0) v += ub[K + (sl - 1) * 2 * dim + c] / n_g;
    }
    add[((int64_t)s * ns + sl) * 2 * dim + c] = (float)v;
  }
}

// xbar_p += add[scene][slot(p)][0..d), vbar_p += add[scene][slot(p)][d..2d): one CTA per
// particle tile
__global__ void ctrl_sensor_adjoint_kernel(int dim, int G, int64_t N, const int4* tiles,
                                           const int* group, const float* add, float* adj) {
  const int4 tile = tiles[blockIdx.x];
  if ((int)threadIdx.x >= tile.z) return;
  const int64_t p = (int64_t)tile.y + threadIdx.x;
  const int g = group[p];
  const int sl = (g >= 0 && g < G) ? g + 1 : 0;
  const float* a = add + ((int64_t)tile.x * (G + 1) + sl) * 2 * dim;
  for (int c = 0; c < 2 * dim; ++c) adj[(int64_t)c * N + p] += a[c];
}

// gw[scene][i] = thbar[scene][i] (FP64 -> FP32)
__global__ void ctrl_grad_out_kernel(int64_t n, const double* thbar, float* gw) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    gw[i] = (float)thbar[i];
}

}  // namespace

cudaError_t launch_ctrl_forward(const CtrlStep& cs, int n_scenes, int n_tiles, int64_t N,
                                const int4* tiles, const int* tile_off, const float* st,
                                const int* group, double* part, const float* theta, double* u,
                                double* h, double* y, float* act, double* cnt, cudaStream_t s) {
  ctrl_sense_kernel<<<n_tiles, kSenseThreads, 0, s>>>(cs.dim, cs.G, N, tiles, st, group, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  ctrl_forward_kernel<<<n_scenes, kCtrlThreads, 0, s>>>(cs, tile_off, part, theta, u, h, y, act, cnt);
  return cudaGetLastError();
}

cudaError_t launch_ctrl_backward(const CtrlStep& cs, int n_scenes, int n_tiles, int64_t N,
                                 const int4* tiles, const int* tile_off, const int* group,
                                 float* abar_tile, const float* theta, const double* u,
                                 const double* h, const double* y, const double* cnt,
                                 double* thbar, float* add, float* adj, cudaStream_t s) {
  ctrl_backward_kernel<<<n_scenes, kCtrlThreads, 0, s>>>(cs, tile_off, abar_tile, theta, u, h, y,
                                                         cnt, thbar, add);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  ctrl_sensor_adjoint_kernel<<<n_tiles, kSenseThreads, 0, s>>>(cs.dim, cs.G, N, tiles, group, add, adj);
  return cudaGetLastError();
}

cudaError_t launch_ctrl_grad_out(int64_t n, const double* thbar, float* gw, cudaStream_t s) {
  ctrl_grad_out_kernel<<<(int)((n + 255) / 256 > 1024 ? 1024 : (n + 255) / 256), 256, 0, s>>>(n, thbar, gw);
  return cudaGetLastError();
}

}  // namespace mpm
