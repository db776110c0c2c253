// mpm_kernels.cuh -- the particle and grid passes of one MLS-MPM step and of its
// adjoint (Appendix D: p2g, grid_op, g2p and their .grad counterparts).
//
// Particle passes run one CTA per tile of up to kTile particles of one scene
// (particles are Morton-sorted per scene at set-up, so a tile covers a compact
// block of cells).  Scatters (P2G mass/momentum, G2P-adjoint grid-velocity
// adjoint) accumulate into a shared-memory copy of the tile's node box and flush
// it with one float4 atomic per non-empty node; a tile whose box exceeds the
// shared capacity scatters with global float4 atomics instead.  Node passes sweep
// the bounding box of the nodes touched in each scene.
#pragma once

#include <climits>

#include "mpm_common.cuh"

namespace mpm {

// particle-pass modes
enum StepMode : int {
  kP2GOnly = 0,      // full state in -> P2G
  kG2PP2G = 1,       // G2P (writes x, F) then P2G of the new state
  kG2PP2GFull = 2,   // same, also writes v and C
  kG2POnlyFull = 3,  // G2P, writes the full state
};
enum AdjMode : int {
  kAdjG2P = 0,    // G2P-adjoint of step s from the full adjoint of state s+1
  kAdjFused = 1,  // P2G-adjoint of step s+1, then G2P-adjoint of step s
  kAdjP2G = 2,    // P2G-adjoint of step s+1 only (s+1 = 0), writes the full adjoint
};

struct StepArgs {
  const int4* tiles;  // {scene, first particle, count, 0}
  int N;              // row stride (total particles)
  const float* in;    // state rows x, v, C, F (component-major)
  float* out;
  const float* mu;
  const float* la;
  const int* group;
  const float* wact;  // [scene][group][basis]
  const float4* U;    // (u, m) per node, scene-major
  float4* PM;         // (m, p) accumulation per node
  int* bbox;          // [scene][8]: lo[3], hi[3] of touched nodes
  unsigned* err;
};

struct AdjArgs {
  const int4* tiles;
  int N;
  const float* st1;  // state s+1 (full)
  const float* st0;  // state s (x and F rows)
  float* adj;        // adjoint rows x, v, C, F
  const float* mu;
  const float* la;
  float* mubar;
  float* labar;
  const int* group;
  const float* wact;
  float* wbar;        // [scene][group][basis]
  const float4* PBM;  // (pbar, mbar) of step s+1
  const float4* U;    // (u, m) of step s
  float4* UB;         // grid-velocity adjoint of step s (accumulated)
  unsigned* err;
};

template <int D>
struct Rows {
  static constexpr int X = 0, V = D, C = 2 * D, F = 2 * D + D * D, Q = 2 * D + 2 * D * D;
};

template <int D>
__device__ __forceinline__ int64_t node_flat(const int idx[D], int n) {
  int64_t r = idx[0];
#pragma unroll
  for (int a = 1; a < D; ++a) r = r * n + idx[a];
  return r;
}

// flat index of the stencil's centre node base + (1, ..., 1)
template <int D>
__device__ __forceinline__ int64_t centre_flat(const int base[D], int n) {
  int idx[D];
#pragma unroll
  for (int a = 0; a < D; ++a) idx[a] = base[a] + 1;
  return node_flat<D>(idx, n);
}

// ---------------------------------------------------------------------------
// CTA-cooperative scatter into a shared-memory node box
// ---------------------------------------------------------------------------
template <int D>
struct BoxInfo {
  int lo[D], dim[D];
  int vol;
  bool use_tile;
};

// Every thread of the CTA must call this (it synchronises).  valid: this thread's
// particle scatters; base: its stencil base.  Zeroes the box when it fits.
template <int D>
__device__ __forceinline__ BoxInfo<D> box_begin(bool valid, const int base[D], int cap, float* sm,
                                                int* s_box) {
  if (threadIdx.x < D) {
    s_box[threadIdx.x] = INT_MAX;
    s_box[4 + threadIdx.x] = INT_MIN;
  }
  __syncthreads();
  const unsigned lane = threadIdx.x & 31u;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    int lo = valid ? base[a] : INT_MAX;
    int hi = valid ? base[a] + 2 : INT_MIN;
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    if (lane == 0) {
      atomicMin(&s_box[a], lo);
      atomicMax(&s_box[4 + a], hi);
    }
  }
  __syncthreads();
  BoxInfo<D> b;
  int vol = 1;
  bool any = true;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    b.lo[a] = s_box[a];
    int hi = s_box[4 + a];
    any = any && hi >= b.lo[a];
    b.dim[a] = any ? hi - b.lo[a] + 1 : 0;
    vol *= b.dim[a];
  }
  b.vol = any ? vol : 0;
  b.use_tile = any && vol <= cap;
  if (b.use_tile)
    for (int l = threadIdx.x; l < b.vol; l += blockDim.x) {
      sm[l] = 0.0f;
      sm[cap + l] = 0.0f;
      sm[2 * cap + l] = 0.0f;
      sm[3 * cap + l] = 0.0f;
    }
  __syncthreads();
  return b;
}

template <int D>
__device__ __forceinline__ int box_local(const BoxInfo<D>& b, const int idx[D]) {
  int l = idx[0] - b.lo[0];
#pragma unroll
  for (int a = 1; a < D; ++a) l = l * b.dim[a] + (idx[a] - b.lo[a]);
  return l;
}

// add (c0..c3) at node idx (NC of them meaningful): into the shared box, or straight
// to global memory
template <int D, int NC>
__device__ __forceinline__ void box_add(const BoxInfo<D>& b, float* sm, int cap, float4* g,
                                        int64_t scene_off, int n, const int idx[D], float c0, float c1,
                                        float c2, float c3) {
  if (b.use_tile) {
    int l = box_local<D>(b, idx);
    atomicAdd(&sm[l], c0);
    atomicAdd(&sm[cap + l], c1);
    if (NC > 2) atomicAdd(&sm[2 * cap + l], c2);
    if (NC > 3) atomicAdd(&sm[3 * cap + l], c3);
  } else {
    atomicAdd(g + scene_off + node_flat<D>(idx, n), make_float4(c0, c1, c2, c3));
  }
}

template <int D>
__device__ __forceinline__ void box_flush(const BoxInfo<D>& b, const float* sm, int cap, float4* g,
                                          int64_t scene_off, int n) {
  __syncthreads();
  if (!b.use_tile) return;
  for (int l = threadIdx.x; l < b.vol; l += blockDim.x) {
    float4 v = make_float4(sm[l], sm[cap + l], sm[2 * cap + l], sm[3 * cap + l]);
    if (v.x != 0.0f || v.y != 0.0f || v.z != 0.0f || v.w != 0.0f) {
      int idx[D], r = l;
#pragma unroll
      for (int a = D - 1; a >= 0; --a) {
        idx[a] = b.lo[a] + r % b.dim[a];
        r /= b.dim[a];
      }
      atomicAdd(g + scene_off + node_flat<D>(idx, n), v);
    }
  }
}

__device__ __forceinline__ float particle_act(const SimParams& P, const int* group, const float* wact,
                                              int scene, int64_t p, int dim, int& axis) {
  axis = 0;
  if (P.n_groups <= 0) return 0.0f;
  int g = group[p];
  if (g < 0 || g >= P.n_groups) return 0.0f;
  axis = g % dim;
  const float* w = wact + ((int64_t)scene * P.n_groups + g) * P.n_basis;
  float a = 0.0f;
#pragma unroll
  for (int k = 0; k < kMaxBasis; ++k)
    if (k < P.n_basis) a += w[k] * P.basis[k];
  return a;
}

// ---------------------------------------------------------------------------
// forward particle pass
// ---------------------------------------------------------------------------
template <int D, int MAT, int MODE>
__global__ void __launch_bounds__(kTile) step_kernel(SimParams P, StepArgs A) {
  using R = Rows<D>;
  extern __shared__ float sm[];
  __shared__ int s_box[8];
  const int4 tile = A.tiles[blockIdx.x];
  const int scene = tile.x;
  const bool active = (int)threadIdx.x < tile.z;
  const int64_t p = (int64_t)tile.y + (active ? threadIdx.x : 0);
  const int64_t N = A.N;
  const int64_t soff = (int64_t)scene * P.nnodes;
  const int n = P.n_grid;
  unsigned err = 0;

  float x[D], v[D], C[D][D], F[D][D];
  if (MODE == kP2GOnly) {
#pragma unroll
    for (int a = 0; a < D; ++a) {
      x[a] = A.in[(R::X + a) * N + p];
      v[a] = A.in[(R::V + a) * N + p];
    }
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = 0; j < D; ++j) {
        C[i][j] = A.in[(R::C + i * D + j) * N + p];
        F[i][j] = A.in[(R::F + i * D + j) * N + p];
      }
  } else {
    // ---- G2P: gather u, build v' and C', advect, update F ----
    float xo[D], Fo[D][D];
#pragma unroll
    for (int a = 0; a < D; ++a) xo[a] = A.in[(R::X + a) * N + p];
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = 0; j < D; ++j) Fo[i][j] = A.in[(R::F + i * D + j) * N + p];
    Stencil<D> s;
    bool ok = make_stencil<D>(xo, P, s) && active;
    if (active && !ok) err |= kErrOOB;
    float B[D][D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      v[a] = 0.0f;
#pragma unroll
      for (int b = 0; b < D; ++b) B[a][b] = 0.0f;
    }
    if (ok) {
      // sum W u dpos^T is accumulated on u - u_c (u_c: the stencil's centre node); the
      // two are equal because sum W dpos = 0, and the centred form keeps FP32 accuracy
      // when u is nearly uniform over the stencil
      const float4 uc4 = __ldg(A.U + soff + centre_flat<D>(s.base, n));
      const float uc[3] = {uc4.x, uc4.y, uc4.z};
      constexpr int NS = D == 2 ? 9 : 27;
#pragma unroll
      for (int o = 0; o < NS; ++o) {
        int off[D], idx[D];
        offsets<D>(o, off);
        float W, gW[D], dpos[D];
        node_terms<D>(s, off, P, W, gW, dpos);
#pragma unroll
        for (int a = 0; a < D; ++a) idx[a] = s.base[a] + off[a];
        float4 u = __ldg(A.U + soff + node_flat<D>(idx, n));
        const float uu[3] = {u.x, u.y, u.z};
#pragma unroll
        for (int a = 0; a < D; ++a) {
          v[a] += W * uu[a];
          float wd = W * (uu[a] - uc[a]);
#pragma unroll
          for (int b = 0; b < D; ++b) B[a][b] += wd * dpos[b];
        }
      }
    }
    const float c4 = 4.0f * P.inv_dx * P.inv_dx;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int b = 0; b < D; ++b) C[a][b] = c4 * B[a][b];
#pragma unroll
    for (int a = 0; a < D; ++a) x[a] = xo[a] + P.dt * v[a];
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = 0; j < D; ++j) {
        float s2 = Fo[i][j];
#pragma unroll
        for (int k = 0; k < D; ++k) s2 += P.dt * C[i][k] * Fo[k][j];
        F[i][j] = s2;
      }
    if (active) {
#pragma unroll
      for (int a = 0; a < D; ++a) A.out[(R::X + a) * N + p] = x[a];
#pragma unroll
      for (int i = 0; i < D * D; ++i) A.out[(R::F + i) * N + p] = F[i / D][i % D];
      if (MODE == kG2PP2GFull || MODE == kG2POnlyFull) {
#pragma unroll
        for (int a = 0; a < D; ++a) A.out[(R::V + a) * N + p] = v[a];
#pragma unroll
        for (int i = 0; i < D * D; ++i) A.out[(R::C + i) * N + p] = C[i / D][i % D];
      }
    }
  }

  if (MODE != kG2POnlyFull) {
    // ---- P2G: stress, affine matrix, scatter (m, m v + A dpos) ----
    Stencil<D> s;
    bool ok = make_stencil<D>(x, P, s) && active;
    if (active && !ok) err |= kErrOOB;
    float Am[D][D], mv[D];
    if (ok) {
      int axis;
      float act = particle_act(P, A.group, A.wact, scene, p, D, axis);
      float tau[D][D];
      StressCache<D> sc;
      bool sok = kirchhoff<D, MAT>(F, A.mu[p], A.la[p], act, axis, tau, sc);
      if (!sok) {
        err |= kErrNonFinite;
        ok = false;
      }
#pragma unroll
      for (int i = 0; i < D; ++i) {
        mv[i] = P.p_mass * v[i];
#pragma unroll
        for (int j = 0; j < D; ++j) Am[i][j] = P.kappa * tau[i][j] + P.p_mass * C[i][j];
      }
    }
    BoxInfo<D> bx = box_begin<D>(ok, s.base, P.tile_capacity, sm, s_box);
    if (ok) {
      constexpr int NS = D == 2 ? 9 : 27;
#pragma unroll
      for (int o = 0; o < NS; ++o) {
        int off[D], idx[D];
        offsets<D>(o, off);
        float W, gW[D], dpos[D];
        node_terms<D>(s, off, P, W, gW, dpos);
#pragma unroll
        for (int a = 0; a < D; ++a) idx[a] = s.base[a] + off[a];
        float c[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int a = 0; a < D; ++a) {
          float q = mv[a];
#pragma unroll
          for (int b = 0; b < D; ++b) q += Am[a][b] * dpos[b];
          c[a] = W * q;
        }
        box_add<D, D + 1>(bx, sm, P.tile_capacity, A.PM, soff, n, idx, W * P.p_mass, c[0], c[1],
                              c[2]);
      }
    }
    box_flush<D>(bx, sm, P.tile_capacity, A.PM, soff, n);
    if (threadIdx.x == 0 && bx.vol > 0) {
#pragma unroll
      for (int a = 0; a < D; ++a) {
        atomicMin(&A.bbox[scene * 8 + a], bx.lo[a]);
        atomicMax(&A.bbox[scene * 8 + 4 + a], bx.lo[a] + bx.dim[a] - 1);
      }
    }
  }
  if (err) atomicOr(A.err, err);
}

// ---------------------------------------------------------------------------
// adjoint particle pass
// ---------------------------------------------------------------------------
template <int D, int MAT, int MODE>
__global__ void __launch_bounds__(kTile) adjoint_kernel(SimParams P, AdjArgs A) {
  using R = Rows<D>;
  extern __shared__ float sm[];
  __shared__ int s_box[8];
  __shared__ float s_wbar[kMaxGroups * kMaxBasis];
  const int4 tile = A.tiles[blockIdx.x];
  const int scene = tile.x;
  const bool active = (int)threadIdx.x < tile.z;
  const int64_t p = (int64_t)tile.y + (active ? threadIdx.x : 0);
  const int64_t N = A.N;
  const int64_t soff = (int64_t)scene * P.nnodes;
  const int n = P.n_grid;
  const float c4 = 4.0f * P.inv_dx * P.inv_dx;
  unsigned err = 0;

  // adjoint of state s+1: xb, vb, Cb, Fb
  float xb[D], vb[D], Cb[D][D], Fb[D][D];
  float C1[D][D];  // C of state s+1
#pragma unroll
  for (int a = 0; a < D; ++a) xb[a] = A.adj[(R::X + a) * N + p];
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) {
      Fb[i][j] = A.adj[(R::F + i * D + j) * N + p];
      C1[i][j] = A.st1[(R::C + i * D + j) * N + p];
    }

  if (MODE == kAdjG2P) {
#pragma unroll
    for (int a = 0; a < D; ++a) vb[a] = A.adj[(R::V + a) * N + p];
#pragma unroll
    for (int i = 0; i < D * D; ++i) Cb[i / D][i % D] = A.adj[(R::C + i) * N + p];
  } else {
    // ---- P2G adjoint of step s+1 (gather pbar, mbar) ----
    if (threadIdx.x < kMaxGroups * kMaxBasis) s_wbar[threadIdx.x] = 0.0f;
    float x[D], v[D], F[D][D], Am[D][D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      x[a] = A.st1[(R::X + a) * N + p];
      v[a] = A.st1[(R::V + a) * N + p];
    }
#pragma unroll
    for (int i = 0; i < D * D; ++i) F[i / D][i % D] = A.st1[(R::F + i) * N + p];
    Stencil<D> s;
    bool ok = make_stencil<D>(x, P, s) && active;
    if (active && !ok) err |= kErrOOB;
    int axis;
    float act = particle_act(P, A.group, A.wact, scene, p, D, axis);
    float mu = A.mu[p], la = A.la[p];
    float tau[D][D];
    StressCache<D> sc;
    if (!kirchhoff<D, MAT>(F, mu, la, act, axis, tau, sc) && ok) {
      err |= kErrNonFinite;
      ok = false;
    }
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = 0; j < D; ++j) Am[i][j] = P.kappa * tau[i][j] + P.p_mass * C1[i][j];
    float Ab[D][D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      vb[a] = 0.0f;
#pragma unroll
      for (int b = 0; b < D; ++b) Ab[a][b] = 0.0f;
    }
    if (ok) {
      // Abar and the x-adjoint use pbar - pbar_c and mbar - mbar_c (centre node): equal
      // to the plain sums because sum W dpos = 0, sum grad W = 0 and
      // sum grad W dpos^T = I, and free of the FP32 cancellation of a smooth pbar field
      const float4 gc = __ldg(A.PBM + soff + centre_flat<D>(s.base, n));
      const float pc[3] = {gc.x, gc.y, gc.z};
      constexpr int NS = D == 2 ? 9 : 27;
#pragma unroll
      for (int o = 0; o < NS; ++o) {
        int off[D], idx[D];
        offsets<D>(o, off);
        float W, gW[D], dpos[D];
        node_terms<D>(s, off, P, W, gW, dpos);
#pragma unroll
        for (int a = 0; a < D; ++a) idx[a] = s.base[a] + off[a];
        float4 g = __ldg(A.PBM + soff + node_flat<D>(idx, n));
        const float pb[3] = {g.x, g.y, g.z};
        float dp[D];
#pragma unroll
        for (int a = 0; a < D; ++a) dp[a] = pb[a] - pc[a];
        float Wbar = P.p_mass * (g.w - gc.w);
#pragma unroll
        for (int a = 0; a < D; ++a) {
          float q = P.p_mass * v[a];
#pragma unroll
          for (int b = 0; b < D; ++b) q += Am[a][b] * dpos[b];
          Wbar += dp[a] * q;
          vb[a] += W * P.p_mass * pb[a];
#pragma unroll
          for (int b = 0; b < D; ++b) Ab[a][b] += W * dp[a] * dpos[b];
        }
#pragma unroll
        for (int b = 0; b < D; ++b) {
          float atp = 0.0f;
#pragma unroll
          for (int a = 0; a < D; ++a) atp += Am[a][b] * dp[a];
          xb[b] += Wbar * gW[b] - W * atp;
        }
      }
    }
    float tb[D][D];
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = 0; j < D; ++j) {
        Cb[i][j] = P.p_mass * Ab[i][j];
        tb[i][j] = P.kappa * Ab[i][j];
      }
    float mub = 0.0f, lab = 0.0f, abar = 0.0f;
    if (ok) abar = kirchhoff_adjoint<D, MAT>(F, mu, la, act, axis, sc, tb, Fb, mub, lab);
    if (active) {
      A.mubar[p] += mub;
      A.labar[p] += lab;
    }
    __syncthreads();  // s_wbar zeroed
    if (P.n_groups > 0 && ok) {
      int g = A.group[p];
      if (g >= 0 && g < P.n_groups) {
#pragma unroll
        for (int k = 0; k < kMaxBasis; ++k)
          if (k < P.n_basis) atomicAdd(&s_wbar[g * P.n_basis + k], abar * P.basis[k]);
      }
    }
    __syncthreads();
    if (P.n_groups > 0 && (int)threadIdx.x < P.n_groups * P.n_basis) {
      float wv = s_wbar[threadIdx.x];
      if (wv != 0.0f) atomicAdd(&A.wbar[(int64_t)scene * P.n_groups * P.n_basis + threadIdx.x], wv);
    }
    if (MODE == kAdjP2G) {
      if (active) {
#pragma unroll
        for (int a = 0; a < D; ++a) {
          A.adj[(R::X + a) * N + p] = xb[a];
          A.adj[(R::V + a) * N + p] = vb[a];
        }
#pragma unroll
        for (int i = 0; i < D * D; ++i) {
          A.adj[(R::C + i) * N + p] = Cb[i / D][i % D];
          A.adj[(R::F + i) * N + p] = Fb[i / D][i % D];
        }
      }
      if (err) atomicOr(A.err, err);
      return;
    }
  }

  // ---- G2P adjoint of step s: x' = x + dt v', F' = (I + dt C') F ----
  {
    float x0[D], F0[D][D];
#pragma unroll
    for (int a = 0; a < D; ++a) x0[a] = A.st0[(R::X + a) * N + p];
#pragma unroll
    for (int i = 0; i < D * D; ++i) F0[i / D][i % D] = A.st0[(R::F + i) * N + p];
    float vt[D], Ct[D][D], Fb0[D][D], xb0[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      vt[a] = vb[a] + P.dt * xb[a];
      xb0[a] = xb[a];
    }
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = 0; j < D; ++j) {
        float g = Fb[i][j], h = Cb[i][j];
#pragma unroll
        for (int k = 0; k < D; ++k) {
          g += P.dt * C1[k][i] * Fb[k][j];  // (I + dt C')^T Fbar'
          h += P.dt * Fb[i][k] * F0[j][k];  // Cbar' + dt Fbar' F^T
        }
        Fb0[i][j] = g;
        Ct[i][j] = h;
      }
    Stencil<D> s;
    bool ok = make_stencil<D>(x0, P, s) && active;
    if (active && !ok) err |= kErrOOB;
    BoxInfo<D> bx = box_begin<D>(ok, s.base, P.tile_capacity, sm, s_box);
    if (ok) {
      // x-adjoint terms on u - u_c (centre node): equal to the plain sums by the same
      // B-spline identities, without the FP32 cancellation of a smooth u field
      const float4 uc4 = __ldg(A.U + soff + centre_flat<D>(s.base, n));
      const float uc[3] = {uc4.x, uc4.y, uc4.z};
      constexpr int NS = D == 2 ? 9 : 27;
#pragma unroll
      for (int o = 0; o < NS; ++o) {
        int off[D], idx[D];
        offsets<D>(o, off);
        float W, gW[D], dpos[D];
        node_terms<D>(s, off, P, W, gW, dpos);
#pragma unroll
        for (int a = 0; a < D; ++a) idx[a] = s.base[a] + off[a];
        float4 u4 = __ldg(A.U + soff + node_flat<D>(idx, n));
        const float u[3] = {u4.x - uc[0], u4.y - uc[1], u4.z - uc[2]};
        float Wbar = 0.0f, ub[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int a = 0; a < D; ++a) {
          float cd = 0.0f;
#pragma unroll
          for (int b = 0; b < D; ++b) cd += Ct[a][b] * dpos[b];
          ub[a] = W * (vt[a] + c4 * cd);
          Wbar += u[a] * (vt[a] + c4 * cd);
        }
#pragma unroll
        for (int b = 0; b < D; ++b) {
          float ctu = 0.0f;
#pragma unroll
          for (int a = 0; a < D; ++a) ctu += Ct[a][b] * u[a];
          xb0[b] += Wbar * gW[b] - c4 * W * ctu;
        }
        box_add<D, D>(bx, sm, P.tile_capacity, A.UB, soff, n, idx, ub[0], ub[1], ub[2], 0.0f);
      }
    }
    box_flush<D>(bx, sm, P.tile_capacity, A.UB, soff, n);
    if (active) {
#pragma unroll
      for (int a = 0; a < D; ++a) A.adj[(R::X + a) * N + p] = xb0[a];
#pragma unroll
      for (int i = 0; i < D * D; ++i) A.adj[(R::F + i) * N + p] = Fb0[i / D][i % D];
    }
  }
  if (err) atomicOr(A.err, err);
}

// ---------------------------------------------------------------------------
// node passes over each scene's touched box (blockIdx.y = scene)
// ---------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ bool box_node(const int* bb, int l, int idx[D]) {
  int r = l;
#pragma unroll
  for (int a = D - 1; a >= 0; --a) {
    int ext = bb[4 + a] - bb[a] + 1;
    idx[a] = bb[a] + r % ext;
    r /= ext;
  }
  return true;
}

template <int D>
__device__ __forceinline__ int box_volume(const int* bb) {
  int vol = 1;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    if (bb[4 + a] < bb[a]) return 0;  // reset box (lo = INT_MAX, hi = INT_MIN)
    vol *= bb[4 + a] - bb[a] + 1;
  }
  return vol;
}

// grid_op: u = p/m + dt g for m > 0 off the walls, else 0; store (u, m); clear PM.
// The last CTA to finish copies the box to bbox_u (used by the grid adjoint of this
// step) and resets the accumulation box for the next P2G.
template <int D>
__global__ void grid_update_kernel(SimParams P, float4* PM, float4* U, int* bbox, int* bbox_u,
                                   unsigned* done) {
  __shared__ int bb[8];
  __shared__ bool last;
  const int scene = blockIdx.y;
  if (threadIdx.x < 8) bb[threadIdx.x] = bbox[scene * 8 + threadIdx.x];
  __syncthreads();
  const int vol = box_volume<D>(bb);
  const int64_t soff = (int64_t)scene * P.nnodes;
  const int n = P.n_grid;
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < vol; l += gridDim.x * blockDim.x) {
    int idx[D];
    box_node<D>(bb, l, idx);
    const int64_t g = soff + node_flat<D>(idx, n);
    float4 pm = PM[g];
    bool wall = false;
#pragma unroll
    for (int a = 0; a < D; ++a) wall = wall || idx[a] < P.wall || idx[a] >= n - P.wall;
    float4 u = make_float4(0.0f, 0.0f, 0.0f, pm.x);
    if (pm.x > 0.0f && !wall) {
      float im = 1.0f / pm.x;
      u.x = pm.y * im + P.dt * P.gravity[0];
      u.y = pm.z * im + P.dt * P.gravity[1];
      if (D == 3) u.z = pm.w * im + P.dt * P.gravity[2];
    }
    U[g] = u;
    PM[g] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  }
  // last-CTA hand-off of the box (threadfence-reduction pattern)
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned total = gridDim.x * gridDim.y;
    last = atomicAdd(done, 1u) == total - 1;
  }
  __syncthreads();
  if (last) {
    __threadfence();
    for (int i = threadIdx.x; i < (int)gridDim.y * 8; i += blockDim.x) {
      int v = bbox[i];
      bbox_u[i] = v;
      bbox[i] = (i % 8) < 4 ? INT_MAX : INT_MIN;
    }
    if (threadIdx.x == 0) *done = 0u;
  }
}

// grid_op.grad: pbar = ubar / m, mbar = -ubar . (u - dt g) / m on non-wall nodes with
// m > 0, else 0; clear the accumulated ubar.
template <int D>
__global__ void grid_adjoint_kernel(SimParams P, float4* UB, const float4* U, float4* PBM,
                                    const int* bbox_u) {
  __shared__ int bb[8];
  const int scene = blockIdx.y;
  if (threadIdx.x < 8) bb[threadIdx.x] = bbox_u[scene * 8 + threadIdx.x];
  __syncthreads();
  const int vol = box_volume<D>(bb);
  const int64_t soff = (int64_t)scene * P.nnodes;
  const int n = P.n_grid;
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < vol; l += gridDim.x * blockDim.x) {
    int idx[D];
    box_node<D>(bb, l, idx);
    const int64_t g = soff + node_flat<D>(idx, n);
    float4 ub = UB[g];
    float4 u = U[g];
    bool wall = false;
#pragma unroll
    for (int a = 0; a < D; ++a) wall = wall || idx[a] < P.wall || idx[a] >= n - P.wall;
    float4 r = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (u.w > 0.0f && !wall) {
      float im = 1.0f / u.w;
      r.x = ub.x * im;
      r.y = ub.y * im;
      float dot = ub.x * (u.x - P.dt * P.gravity[0]) + ub.y * (u.y - P.dt * P.gravity[1]);
      if (D == 3) {
        r.z = ub.z * im;
        dot += ub.z * (u.z - P.dt * P.gravity[2]);
      }
      r.w = -dot * im;
    }
    PBM[g] = r;
    UB[g] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  }
}

}  // namespace mpm
