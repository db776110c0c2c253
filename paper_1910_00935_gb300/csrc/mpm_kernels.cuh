// mpm_kernels.cuh -- the particle passes of one MLS-MPM step and of its adjoint
// (Appendix D: p2g, grid_op, g2p and their .grad counterparts).
//
// There are no separate grid passes.  grid_op (v = p/m + dt g, sticky walls) and its
// adjoint (pbar = ubar/m, mbar = -ubar.p/m^2) are node-local, so the particle pass that
// consumes a grid applies them to every node it gathers.  Grids are accumulation
// buffers handed out by the host's ring allocator: a pass scatters into a clean buffer,
// records the touched box per scene, and a later pass zeroes that box once the buffer's
// last reader has finished (each buffer keeps two parity copies of its box so that a box
// is never reset while another CTA may still read it).
//
// Particle passes run one CTA per tile of up to kTile particles of one scene
// (particles are Morton-sorted per scene at set-up, so a tile covers a compact block
// of cells, ~8 particles per cell in 3D).  Each pass works in two orders:
//   - gathers, stress and state I/O run in tile order (thread t = particle t), so the
//     state rows are read and written coalesced;
//   - scatters run in an interleaved order (warp w takes particles w, w+8, w+16, ...),
//     so that the 32 lanes of a warp sit in 32 different cells and never hit the same
//     node in the same instruction.  The per-particle scatter record (stencil base, f,
//     and the affine pair a + B dpos) moves between the two orders through shared
//     memory.
// Scatters go to the grid with float4 reductions (default), or accumulate in a shared
// node box flushed once per node (MPM_OPT_SMEM_TILE).  Gathers read a shared gather box
// filled once per CTA (grid functions applied while filling), or the grid directly.
//
// Stencil loops are separable: the weight of node (i, j, k) is w0[i] w1[j] w2[k] and
// dpos = (dp0[i], dp1[j], dp2[k]), so partial products over (i) and (i, j) are hoisted.
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

// a dirty grid buffer to zero over its recorded per-scene boxes
struct ClearJob {
  float4* grid;     // scene-major dense grids
  const int* box;   // [scene][8]: lo[3], hi[3]
};
constexpr int kMaxClears = 3;
struct Clears {
  ClearJob job[kMaxClears];
  int n;
  int words;  // float4 slots per node (1, or 2 for fixed-point grids)
};

struct StepArgs {
  const int4* tiles;       // {scene, first particle, count, rank of the tile in its scene}
  const int* scene_tiles;  // tiles per scene
  int N;                   // row stride (total particles)
  const float* in;         // state rows x, v, C, F - f_diag I (component-major)
  float* out;
  const float* mu;
  const float* la;
  const int* group;
  const int* matid;        // per-particle material (kMixed scenes) or null
  const float* wact;       // [scene][group][basis]
  const float4* PMr;       // grid (m, p) of step t-1, read by G2P (null: P2G only)
  float4* PMw;             // grid of step t, accumulated by P2G (null: G2P only)
  double* Rw;              // [9][N] polar factors (R_hi, R_lo pairs) of the P2G's states, written (or null)
  int* box_w;              // [scene][8] box of PMw for this use
  int* box_reset;          // [scene][8] the other parity box of PMw, reset here (or null)
  Clears clears;
  unsigned* err;
  unsigned long long* box_stats;  // [2]: gather boxes staged, of which too large for the shared
                                  // box (read from the grid instead); null: not counted
};

struct AdjArgs {
  const int4* tiles;
  const int* scene_tiles;
  int N;
  const float* st1;   // state s+1 (full)
  const float* st0;   // state s (x and F rows)
  const float* stm;   // state s-1 (full) for the recomputed P2G of step s-1, or null
  float* adj;         // adjoint rows x, v, C, F
  const float* mu;
  const float* la;
  float2* mubar;      // dL/dmu, dL/dlambda per particle, summed over the steps as compensated
  float2* labar;      // FP32 (value, correction) pairs: the per-step terms oscillate in sign
                      // over a long run and mostly cancel, so the sum needs ~48 bits
  const int* group;
  const int* matid;   // per-particle material (kMixed scenes) or null
  const float* wact;
  float* wbar_tile;   // [tile][group][basis] per-tile dL/dw partial sums (this pass adds)
  const float4* PM1;  // grid (m, p) of step s+1 (P2G-adjoint)
  const float4* UB1;  // grid-velocity adjoint of step s+1
  const float4* PM0;  // grid of step s (G2P-adjoint)
  float4* UB0;        // grid-velocity adjoint of step s (accumulated)
  int* box_ub;
  int* box_ub_reset;
  float4* PMm;        // grid of step s-1 (recomputed P2G) or null
  unsigned* ub_m0;    // deterministic mode: largest velocity-adjoint contribution bound of
                      // the backward's first scatter (FP32 bits; the measuring pass raises it,
                      // every pass derives the fixed-point scale of the ubar grids from it)
  int measure;        // 1: this kAdjG2P pass only measures that bound (no scatter, no writes)
  const double* R1;   // [9][N] cached polar factors of state s+1 (or null: recompute)
  const double* Rm;   // same for state s-1
  int* box_m;
  int* box_m_reset;
  Clears clears;
  unsigned* err;
};

// Grid reads in the particle passes.  A grid written by an earlier launch is read through
// the read-only data path (NC); inside a persistent launch the grid was written by an
// earlier pass of the same launch, so it is read with coherent loads, which the barrier's
// acquire makes current.
template <bool NC>
__device__ __forceinline__ float4 grid_load(const float4* p) {
  if (NC) return __ldg(p);
  return *p;
}

// node `node` of a scene's (m, p) grid as floats (DET: fixed-point grid)
template <bool NC, bool DET>
__device__ __forceinline__ float4 pm_load(const float4* g, int64_t node, const SimParams& P) {
  if (DET) return fix_load<NC>(g, node, P.unfix_m, P.unfix_p);
  return grid_load<NC>(g + node);
}
// fixed-point scale pair of this backward's velocity-adjoint grids (deterministic mode)
__device__ __forceinline__ void ub_scales(const unsigned* m0, float& fix, float& unfix) {
  fix_scales_from(__uint_as_float(*(const volatile unsigned*)m0), fix, unfix);
}
// node of a scene's velocity-adjoint grid
template <bool NC, bool DET>
__device__ __forceinline__ float4 ub_load(const float4* g, int64_t node, const SimParams& P,
                                          const unsigned* m0) {
  if (DET) {
    float fix, unfix;
    ub_scales(m0, fix, unfix);
    return fix_load<NC>(g, node, unfix, unfix);
  }
  return grid_load<NC>(g + node);
}
// a scene's grid inside a buffer of per-scene grids
__device__ __forceinline__ float4* scene_grid(float4* g, int scene, const SimParams& P) {
  return g + (int64_t)scene * P.nnodes * P.node_words;
}
__device__ __forceinline__ const float4* scene_grid(const float4* g, int scene, const SimParams& P) {
  return g + (int64_t)scene * P.nnodes * P.node_words;
}

template <int D>
struct Rows {
  static constexpr int X = 0, V = D, C = 2 * D, F = 2 * D + D * D, Q = 2 * D + 2 * D * D;
};

// scatter records: packed base, f[D], a[D], B[D][D]
template <int D>
struct Xch {
  static constexpr int kWidth = 1 + 2 * D + D * D;
  static constexpr int kStride = kTile + kTile / 8;  // padded: conflict-free in both orders
};

// per-warp group sums of the dL/dw reduction
constexpr int kWbarSlots = (kTile / 32) * kMaxGroups;

// Particle rows staged ahead of use with asynchronous copies (cp.async, no registers held
// while in flight): stage row r holds component r of the CTA's particles at
// [r * kTile + threadIdx.x]; each thread copies and later reads only its own column.
template <int D>
struct Stage {
  static constexpr int kStep = 2;                   // mu, la (read by the P2G stress)
  static constexpr int kAdjB = D + D * D;           // x, F rows of state s (G2P-adjoint)
  static constexpr int kAdjC = 2 * D + 2 * D * D;   // full state s-1 (recomputed P2G)
  static constexpr int kAdj = kAdjB + kAdjC + 2;    // + mu, la
};
__device__ __forceinline__ void stage_row(float* stage, int r, const float* src) {
  const unsigned dst = (unsigned)__cvta_generic_to_shared(stage + r * kTile + threadIdx.x);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void stage_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// wait until at most N of this thread's copy groups are still in flight (the passes use
// N = 0 before the first read of any staged row)
template <int N>
__device__ __forceinline__ void stage_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ float staged(const float* stage, int r) { return stage[r * kTile + threadIdx.x]; }

__device__ __forceinline__ int scatter_slot(int t) { return (t & 31) * (kTile / 32) + (t >> 5); }
__device__ __forceinline__ int xidx(int j) { return j + (j >> 3); }

// dynamic shared memory of a particle pass: node box (4 floats per node, shared by the
// gather box and the scatter box) + scatter records
__host__ __device__ inline int box_floats(int scatter_cap, int gather_cap) {
  int c = scatter_cap > gather_cap ? scatter_cap : gather_cap;
  return 4 * (c > 0 ? c : 1);
}
template <int D>
inline size_t pass_smem_bytes(int scatter_cap, int gather_cap) {
  return sizeof(float) * ((size_t)box_floats(scatter_cap, gather_cap) +
                          (size_t)Xch<D>::kWidth * Xch<D>::kStride);
}
// + the staged rows of a forward / adjoint pass
template <int D>
inline size_t step_smem_bytes(int scatter_cap, int gather_cap) {
  return pass_smem_bytes<D>(scatter_cap, gather_cap) + sizeof(float) * Stage<D>::kStep * kTile;
}
template <int D>
inline size_t adj_smem_bytes(int scatter_cap, int gather_cap) {
  return pass_smem_bytes<D>(scatter_cap, gather_cap) + sizeof(float) * Stage<D>::kAdj * kTile;
}

// Scene bounding box of the nodes a scatter touches: each warp reduces its valid lanes
// into s_bbox (shared int atomics, native); after the CTA's next barrier thread 0 folds
// s_bbox into the scene box with one set of global atomics (cta_bbox_flush).
// s_bbox must have been reset (cta_bbox_reset) before a barrier preceding this call.
__device__ __forceinline__ void cta_bbox_reset(int* s_bbox) {
  if (threadIdx.x < 8) s_bbox[threadIdx.x] = (threadIdx.x & 4) ? INT_MIN : INT_MAX;
}
template <int D>
__device__ __forceinline__ void warp_bbox(bool valid, const int base[D], int* s_bbox) {
  const unsigned lane = threadIdx.x & 31u;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    int lo = __reduce_min_sync(0xffffffffu, valid ? base[a] : INT_MAX);
    int hi = __reduce_max_sync(0xffffffffu, valid ? base[a] + 2 : INT_MIN);
    if (lane == 0 && hi >= lo) {
      atomicMin(&s_bbox[a], lo);
      atomicMax(&s_bbox[4 + a], hi);
    }
  }
}
template <int D>
__device__ __forceinline__ void cta_bbox_flush(const int* s_bbox, int* bbox_scene) {
  if (threadIdx.x == 0 && s_bbox[4] >= s_bbox[0]) {
#pragma unroll
    for (int a = 0; a < D; ++a) {
      atomicMin(&bbox_scene[a], s_bbox[a]);
      atomicMax(&bbox_scene[4 + a], s_bbox[4 + a]);
    }
  }
}

template <int D>
__device__ __forceinline__ int pack_base(const int b[D]) {
  return D == 2 ? (b[0] << 16) | b[D - 1] : (b[0] << 20) | (b[1] << 10) | b[D - 1];
}
template <int D>
__device__ __forceinline__ void unpack_base(int v, int b[D]) {
  if (D == 2) {
    b[0] = v >> 16;
    b[D - 1] = v & 0xFFFF;
  } else {
    b[0] = v >> 20;
    b[1] = (v >> 10) & 0x3FF;
    b[D - 1] = v & 0x3FF;
  }
}

// flat node index inside one scene grid
template <int D>
__device__ __forceinline__ int node_flat(const int idx[D], int n) {
  int r = idx[0];
#pragma unroll
  for (int a = 1; a < D; ++a) r = r * n + idx[a];
  return r;
}

// flat offset of stencil node (i, j, k) from the stencil base
template <int D>
__device__ __forceinline__ int stencil_off(int i, int j, int k, int n) {
  return D == 2 ? i * n + j : (i * n + j) * n + k;
}

// Calls fn(i, j, k, W) for the 3^D stencil nodes (k = 0 in 2D); indices are
// compile-time after unrolling.
template <int D, typename Fn>
__device__ __forceinline__ void for_nodes(const float w[D][3], Fn&& fn) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float wij = w[0][i] * w[1][j];
      if (D == 2) {
        fn(i, j, 0, wij);
      } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) fn(i, j, k, wij * w[D - 1][k]);
      }
    }
}

// ---------------------------------------------------------------------------
// CTA-cooperative node box in shared memory
// ---------------------------------------------------------------------------
template <int D>
struct BoxInfo {
  int lo[D], dim[D];
  int vol;
  bool use_tile;
};

// Each box computation of a tile has its own 8-int slot of s_box (kBoxSlots slots, reset
// together by reset_box_slots before the tile's first barrier), so a box costs one barrier.
constexpr int kBoxSlots = 3;
__device__ __forceinline__ void reset_box_slots(int* s_box) {
  if (threadIdx.x < 8 * kBoxSlots) s_box[threadIdx.x] = (threadIdx.x & 4) ? INT_MIN : INT_MAX;
}

// Extent of the node box covering the stencils of the CTA's valid particles.  Every
// thread of the CTA must call this; s_box is a slot reset before an earlier barrier and
// not used since.  Ends with a barrier, which also orders every earlier read of the
// shared node box before the box_load that follows.
template <int D>
__device__ __forceinline__ BoxInfo<D> box_extent(bool valid, const int base[D], int cap, int* s_box) {
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
  return b;
}

// Zero the SoA accumulation box (4 arrays of cap floats).  Synchronises on both sides.
template <int D>
__device__ __forceinline__ void box_zero(const BoxInfo<D>& b, float* sm, int cap) {
  __syncthreads();
  if (b.use_tile)
    for (int l = threadIdx.x; l < b.vol; l += blockDim.x) {
      sm[l] = 0.0f;
      sm[cap + l] = 0.0f;
      sm[2 * cap + l] = 0.0f;
      sm[3 * cap + l] = 0.0f;
    }
  __syncthreads();
}

// Fill the shared gather box (float4 per node, box-local order) with value(idx) for every
// node idx of the box, one node per thread.  Called right after box_extent (whose barrier
// separates it from earlier readers of the box); synchronises after.
template <int D, typename Value>
__device__ __forceinline__ void box_load(const BoxInfo<D>& b, float4* sm4, Value&& value) {
  if (b.use_tile)
    for (int l = threadIdx.x; l < b.vol; l += blockDim.x) {
      int idx[D], r = l;
#pragma unroll
      for (int a = D - 1; a >= 0; --a) {
        idx[a] = b.lo[a] + r % b.dim[a];
        r /= b.dim[a];
      }
      sm4[l] = value(idx);
    }
  __syncthreads();
}

// Run body(load) with load(i, j, k) returning value(base + (i, j, k)): from the shared
// gather box when it holds the CTA's stencils, else computed from global memory.
template <int D, typename Value, typename Body>
__device__ __forceinline__ void with_nodes(const BoxInfo<D>& b, const float4* sm4, const int base[D],
                                           Value&& value, Body&& body) {
  if (b.use_tile) {
    int lb = base[0] - b.lo[0];
#pragma unroll
    for (int c = 1; c < D; ++c) lb = lb * b.dim[c] + (base[c] - b.lo[c]);
    const int s1 = D == 2 ? 1 : b.dim[D - 1];
    const int s0 = b.dim[1] * s1;
    const float4* p = sm4 + lb;
    body([&](int i, int j, int k) { return p[i * s0 + j * s1 + k]; });
  } else {
    body([&](int i, int j, int k) {
      int idx[D];
      idx[0] = base[0] + i;
      idx[1] = base[1] + j;
      if (D == 3) idx[D - 1] = base[D - 1] + k;
      return value(idx);
    });
  }
}

template <int D>
__device__ __forceinline__ void box_flush(const BoxInfo<D>& b, const float* sm, int cap, float4* g,
                                          int n) {
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
      atomicAdd(g + node_flat<D>(idx, n), v);
    }
  }
}

// Write this thread's scatter record (tile order).  A negative base marks "no scatter".
template <int D>
__device__ __forceinline__ void put_record(float* xr, bool valid, const int base[D], const float f[D],
                                           const float a[D], const float B[D][D]) {
  constexpr int S = Xch<D>::kStride;
  const int i = xidx(threadIdx.x);
  xr[i] = __int_as_float(valid ? pack_base<D>(base) : -1);
#pragma unroll
  for (int c = 0; c < D; ++c) {
    xr[(1 + c) * S + i] = f[c];
    xr[(1 + D + c) * S + i] = a[c];
  }
#pragma unroll
  for (int c = 0; c < D * D; ++c) xr[(1 + 2 * D + c) * S + i] = B[c / D][c % D];
}

// quadratic B-spline weight of stencil offset o (compile-time after unrolling) at f = x/dx - base
__device__ __forceinline__ float bspline_w(int o, float f) {
  if (o == 0) {
    const float r = 1.5f - f;
    return 0.5f * r * r;
  }
  if (o == 1) {
    const float r = f - 1.0f;
    return 0.75f - r * r;
  }
  const float r = f - 0.5f;
  return 0.5f * r * r;
}

// Reversed stencil walk.  Particles sorted by stencil base put ~8 particles (3D) of a base in
// one tile, so two lanes of a reduction instruction often share a base; if both walk the 27
// nodes in the same order they reduce into the same node in the same instruction, which the
// L2 serialises.  A lane with rev walks them in reverse: by the B-spline symmetry
// w_o(f) = w_(2-o)(2 - f) and dpos_o(f) = -dpos_(2-o)(2 - f), the contribution for the loop's
// offset o, computed from f' = 2 - f and -B, belongs to node base + 2 - o.  This rewrites f
// and B in place and returns the grid pointer of node base + 2 rev and the offset sign.
template <int D>
__device__ __forceinline__ float4* reversed_stencil(bool rev, float4* g, int n, const int base[D],
                                                    float f[D], float B[D][D], int& sgn) {
  int b[D];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    f[a] = rev ? 2.0f - f[a] : f[a];
    b[a] = base[a] + (rev ? 2 : 0);
  }
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) B[i][j] = rev ? -B[i][j] : B[i][j];
  sgn = rev ? -1 : 1;
  return g + node_flat<D>(b, n);
}

// Pair-merged scatter (FP32 sums, reductions straight to the grid).  On GB300 a pass's
// time grows with its count of scattered float4 reductions (measured on the fused forward
// pass of a 262,144-particle cube: 51 us with 27 per particle, 26 us with none and the
// arithmetic kept).  Particles are sorted by stencil base with the last axis's half-cell
// varying fastest, so particles 2j and 2j+1 of a tile usually share their base: two
// threads take such a pair, each one half of the 3^D nodes, and sum the pair's two
// contributions to a node before one reduction -- half the reductions for the same
// arithmetic.  A pair whose bases differ scatters each particle's contributions on their
// own.  The node half is uniform per warp (no divergence); each thread reads two records.
template <int D, bool WITH_MASS>
__device__ __noinline__ void scatter_pairs(const float* xr, int count, float4* g, int n,
                                           const SimParams& P, float mass_c) {
  static_assert(kTile % 64 == 0, "pairs: two node halves of whole warps");
  constexpr int S = Xch<D>::kStride;
  constexpr int NN = D == 3 ? 27 : 9;
  constexpr int SPLIT = D == 3 ? 15 : 5;   // nodes of the first half (whole columns in 3D)
  constexpr int HW = kTile / 64;           // warps per node half
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int h = warp >= HW ? 1 : 0;
  // lanes of a warp take every second pair, so fewer of them share a base (and nodes)
  const int j = lane * HW + (warp - h * HW);  // 0 .. kTile/2 - 1
  const int ia = 2 * j, ib = 2 * j + 1;
  const int pa = ia < count ? __float_as_int(xr[xidx(ia)]) : -1;
  const int pb = ib < count ? __float_as_int(xr[xidx(ib)]) : -1;
  const bool va = pa >= 0, vb = pb >= 0;
  if (!va && !vb) return;
  const bool merged = va && vb && pa == pb;
  float fa[D], fb[D], aa[D], ab[D], Ba[D][D], Bb[D][D];
#pragma unroll
  for (int c = 0; c < D; ++c) {
    fa[c] = va ? xr[(1 + c) * S + xidx(ia)] : 1.0f;
    aa[c] = va ? xr[(1 + D + c) * S + xidx(ia)] : 0.0f;
    fb[c] = vb ? xr[(1 + c) * S + xidx(ib)] : 1.0f;
    ab[c] = vb ? xr[(1 + D + c) * S + xidx(ib)] : 0.0f;
  }
#pragma unroll
  for (int c = 0; c < D * D; ++c) {
    Ba[c / D][c % D] = va ? xr[(1 + 2 * D + c) * S + xidx(ia)] : 0.0f;
    Bb[c / D][c % D] = vb ? xr[(1 + 2 * D + c) * S + xidx(ib)] : 0.0f;
  }
  int base_a[D], base_b[D];
  unpack_base<D>(va ? pa : 0, base_a);
  unpack_base<D>(vb ? pb : 0, base_b);
  // odd lanes walk their pair's stencils in reverse (reversed_stencil)
  const bool rev = (lane & 1) != 0;
  int sgn;
  float4* ga = reversed_stencil<D>(rev, g, n, base_a, fa, Ba, sgn);
  float4* gb = reversed_stencil<D>(rev, g, n, base_b, fb, Bb, sgn);
  // weights and dpos are formed where they are used (few registers: the pair's records
  // already hold 2 (2D + D^2) values)
#pragma unroll
  for (int col = 0; col < (D == 3 ? 9 : 3); ++col) {
    // column: (i, jj) in 3D (nodes k = 0..2), i in 2D (nodes jj = 0..2)
    const int i = D == 3 ? col / 3 : col;
    const int jj = D == 3 ? col % 3 : 0;
    const int o0 = D == 3 ? col * 3 : col * 3;  // first node of the column
    // the column's nodes all lie in one half (3D: 15 = 5 columns; 2D: split inside col 1)
    if (D == 3 && ((o0 < SPLIT) != (h == 0))) continue;
    float wca = bspline_w(i, fa[0]), wcb = bspline_w(i, fb[0]);
    float qca[D], qcb[D];
    const float dia = ((float)i - fa[0]) * P.dx, dib = ((float)i - fb[0]) * P.dx;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      qca[c] = aa[c] + Ba[c][0] * dia;
      qcb[c] = ab[c] + Bb[c][0] * dib;
    }
    if (D == 3) {
      const float dja = ((float)jj - fa[1]) * P.dx, djb = ((float)jj - fb[1]) * P.dx;
      wca *= bspline_w(jj, fa[1]);
      wcb *= bspline_w(jj, fb[1]);
#pragma unroll
      for (int c = 0; c < D; ++c) {
        qca[c] += Ba[c][1] * dja;
        qcb[c] += Bb[c][1] * djb;
      }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int o = o0 + k;
      if (D == 2 && ((o < SPLIT) != (h == 0))) continue;
      const float Wa = wca * bspline_w(k, fa[D - 1]), Wb = wcb * bspline_w(k, fb[D - 1]);
      const float dza = ((float)k - fa[D - 1]) * P.dx, dzb = ((float)k - fb[D - 1]) * P.dx;
      float q_a[3] = {0.0f, 0.0f, 0.0f}, q_b[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int c = 0; c < D; ++c) {
        q_a[c] = qca[c] + Ba[c][D - 1] * dza;
        q_b[c] = qcb[c] + Bb[c][D - 1] * dzb;
      }
      const float4 ca = WITH_MASS ? make_float4(Wa * mass_c, Wa * q_a[0], Wa * q_a[1], D == 3 ? Wa * q_a[2] : 0.0f)
                                  : make_float4(Wa * q_a[0], Wa * q_a[1], D == 3 ? Wa * q_a[2] : 0.0f, 0.0f);
      const float4 cb = WITH_MASS ? make_float4(Wb * mass_c, Wb * q_b[0], Wb * q_b[1], D == 3 ? Wb * q_b[2] : 0.0f)
                                  : make_float4(Wb * q_b[0], Wb * q_b[1], D == 3 ? Wb * q_b[2] : 0.0f, 0.0f);
      const int off = sgn * (D == 3 ? stencil_off<D>(i, jj, k, n) : stencil_off<D>(i, k, 0, n));
      if (merged) {
        atomicAdd(ga + off, make_float4(ca.x + cb.x, ca.y + cb.y, ca.z + cb.z, ca.w + cb.w));
      } else {
        if (va) atomicAdd(ga + off, ca);
        if (vb) atomicAdd(gb + off, cb);
      }
    }
  }
}

// Interleaved scatter of the records: node (i, j, k) receives
//   mass  W * mass_c                      (when WITH_MASS)
//   vec   W * (a + B dpos)
// into the shared box (or global memory g when the box did not fit).
template <int D, bool WITH_MASS, bool DET>
__device__ __forceinline__ void scatter_records(const float* xr, int count, const BoxInfo<D>& bx,
                                                float* sm, int cap, float4* g, int n,
                                                const SimParams& P, float mass_c, float fix0,
                                                float fix1, unsigned& err, bool pair) {
  constexpr int S = Xch<D>::kStride;
  if (!DET && !bx.use_tile && pair) {
    scatter_pairs<D, WITH_MASS>(xr, count, g, n, P, mass_c);
    return;
  }
  const int j = scatter_slot(threadIdx.x);
  if (j >= count) return;
  const int xi = xidx(j);
  const int packed = __float_as_int(xr[xi]);
  if (packed < 0) return;
  int base[D];
  unpack_base<D>(packed, base);
  float f[D], a[D], B[D][D];
#pragma unroll
  for (int c = 0; c < D; ++c) {
    f[c] = xr[(1 + c) * S + xi];
    a[c] = xr[(1 + D + c) * S + xi];
  }
#pragma unroll
  for (int c = 0; c < D * D; ++c) B[c / D][c % D] = xr[(1 + 2 * D + c) * S + xi];
  float w[D][3], dp[D][3];
  if (bx.use_tile || DET) axes_from_f<D>(f, P, w, dp);
  if (bx.use_tile) {
    int lb = base[0] - bx.lo[0];
#pragma unroll
    for (int c = 1; c < D; ++c) lb = lb * bx.dim[c] + (base[c] - bx.lo[c]);
    const int s1 = D == 2 ? 1 : bx.dim[D - 1];
    const int s0 = bx.dim[1] * s1;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      float qi[D];
#pragma unroll
      for (int c = 0; c < D; ++c) qi[c] = a[c] + B[c][0] * dp[0][i];
#pragma unroll
      for (int jj = 0; jj < 3; ++jj) {
        const float wij = w[0][i] * w[1][jj];
        float qij[D];
#pragma unroll
        for (int c = 0; c < D; ++c) qij[c] = qi[c] + B[c][1] * dp[1][jj];
        if (D == 2) {
          const int l = lb + i * s0 + jj;
          if (WITH_MASS) {
            atomicAdd(&sm[l], wij * mass_c);
            atomicAdd(&sm[cap + l], wij * qij[0]);
            atomicAdd(&sm[2 * cap + l], wij * qij[1]);
          } else {
            atomicAdd(&sm[l], wij * qij[0]);
            atomicAdd(&sm[cap + l], wij * qij[1]);
          }
        } else {
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const float W = wij * w[D - 1][k];
            const int l = lb + i * s0 + jj * s1 + k;
            float q[D];
#pragma unroll
            for (int c = 0; c < D; ++c) q[c] = qij[c] + B[c][D - 1] * dp[D - 1][k];
            if (WITH_MASS) {
              atomicAdd(&sm[l], W * mass_c);
              atomicAdd(&sm[cap + l], W * q[0]);
              atomicAdd(&sm[2 * cap + l], W * q[1]);
              atomicAdd(&sm[3 * cap + l], W * q[D - 1]);
            } else {
              atomicAdd(&sm[l], W * q[0]);
              atomicAdd(&sm[cap + l], W * q[1]);
              atomicAdd(&sm[2 * cap + l], W * q[D - 1]);
            }
          }
        }
      }
    }
  } else if (DET) {
    const int64_t nb = node_flat<D>(base, n);
    for_nodes<D>(w, [&](int i, int jj, int k, float W) {
      float q[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int c = 0; c < D; ++c) {
        q[c] = a[c] + B[c][0] * dp[0][i] + B[c][1] * dp[1][jj];
        if (D == 3) q[c] += B[c][D - 1] * dp[D - 1][k];
      }
      float4 v = WITH_MASS ? make_float4(W * mass_c, W * q[0], W * q[1], D == 3 ? W * q[2] : 0.0f)
                           : make_float4(W * q[0], W * q[1], D == 3 ? W * q[2] : 0.0f, 0.0f);
      fix_red(g, nb + stencil_off<D>(i, jj, k, n), v, fix0, fix1, WITH_MASS ? D + 1 : D, err);
    });
  } else {
    // odd lanes walk the stencil in reverse (see reversed_stencil), so two lanes that share
    // a base hit different nodes in each reduction instruction
    const bool rev = (threadIdx.x & 1) != 0;
    int sgn;
    float4* gb = reversed_stencil<D>(rev, g, n, base, f, B, sgn);
    float wr[D][3], dpr[D][3];
    axes_from_f<D>(f, P, wr, dpr);
    for_nodes<D>(wr, [&](int i, int jj, int k, float W) {
      float q[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int c = 0; c < D; ++c) {
        q[c] = a[c] + B[c][0] * dpr[0][i] + B[c][1] * dpr[1][jj];
        if (D == 3) q[c] += B[c][D - 1] * dpr[D - 1][k];
      }
      float4 v = WITH_MASS ? make_float4(W * mass_c, W * q[0], W * q[1], D == 3 ? W * q[2] : 0.0f)
                           : make_float4(W * q[0], W * q[1], D == 3 ? W * q[2] : 0.0f, 0.0f);
      atomicAdd(gb + sgn * stencil_off<D>(i, jj, k, n), v);
    });
  }
}

// ---------------------------------------------------------------------------
// Bucketed scatter (FP32 sums).  A scattered float4 reduction costs the SM's L1/L2 path far
// more than the arithmetic that produces it (measured on GB300: ~1.5 SM cycles per lane,
// the equivalent of ~6 warp-wide FMA instructions), and a 128-particle tile sends ~3,500
// of them into a box of ~200 nodes.  Particles that share a stencil base touch the same
// 3^D nodes, so the tile's particles are grouped by base in a shared table, and one warp
// takes a whole group: lane o < 3^D owns node base + o, sums the group's contributions in
// registers and issues one reduction.  In 3D a tile holds ~16-64 bases of ~2-8 particles,
// so the reductions drop 2-3x for ~30 extra FMA-class instructions per particle.  Bases
// whose group overflows the table's slots, and tiles whose base box exceeds its keys, go
// through the per-particle path.  Not used in the deterministic mode (its sums are
// fixed point and order-free already).  Measured on GB300 it is slower than the per-particle
// reductions (cube3d fused forward 53.2 vs 50.8 us): each group step is a chain of
// dependent shared-memory reads (slot, then record) and the pass was already limited by
// its shared-memory instruction queue as much as by the reductions; the pair-merged
// scatter (scatter_pairs) halves the reductions without that cost.  It stays an option.
// ---------------------------------------------------------------------------
constexpr int kBucketKeys = 256;  // bases of one tile's base box the table can hold
constexpr int kBucketSlots = 8;   // particles per base held in the table
static_assert(kTile <= 256, "bucket entries hold tile-local indices in one byte");
struct Buckets {
  int count[kBucketKeys];                           // particles per base (kept zero between uses)
  unsigned char order[kBucketKeys * kBucketSlots];  // their tile-local indices
};
__device__ __forceinline__ void buckets_zero(Buckets& b) {
  for (int i = threadIdx.x; i < kBucketKeys; i += blockDim.x) b.count[i] = 0;
}

// array-of-structures scatter record of one particle: f[D], a[D], B[D][D], padded to float4s
template <int D>
struct Aos {
  static constexpr int kFloats = D == 3 ? 16 : 8;
};
static_assert(Aos<3>::kFloats * kTile <= Xch<3>::kWidth * Xch<3>::kStride, "record area");
static_assert(Aos<2>::kFloats * kTile <= Xch<2>::kWidth * Xch<2>::kStride, "record area");

template <int D>
__device__ __forceinline__ void put_record_aos(float* xr, const float f[D], const float a[D],
                                               const float B[D][D]) {
  float r[Aos<D>::kFloats];
  int c = 0;
#pragma unroll
  for (int i = 0; i < D; ++i) r[c++] = f[i];
#pragma unroll
  for (int i = 0; i < D; ++i) r[c++] = a[i];
#pragma unroll
  for (int i = 0; i < D * D; ++i) r[c++] = B[i / D][i % D];
#pragma unroll
  for (; c < Aos<D>::kFloats; ++c) r[c] = 0.0f;
  float4* dst = reinterpret_cast<float4*>(xr) + threadIdx.x * (Aos<D>::kFloats / 4);
#pragma unroll
  for (int i = 0; i < Aos<D>::kFloats / 4; ++i)
    dst[i] = make_float4(r[4 * i], r[4 * i + 1], r[4 * i + 2], r[4 * i + 3]);
}

// keys of the tile's base box: the stencil box bx less its 2-node margin
template <int D>
__device__ __forceinline__ int bucket_keys(const BoxInfo<D>& bx) {
  if (bx.vol <= 0) return 0;
  int K = 1;
#pragma unroll
  for (int a = 0; a < D; ++a) K *= bx.dim[a] - 2;
  return K;
}
template <int D>
__device__ __forceinline__ int bucket_key(const BoxInfo<D>& bx, const int base[D]) {
  int k = base[0] - bx.lo[0];
#pragma unroll
  for (int a = 1; a < D; ++a) k = k * (bx.dim[a] - 2) + (base[a] - bx.lo[a]);
  return k;
}

// Enter this thread's particle in the table (valid particles only); returns true when its
// base's slots were full and the particle must scatter on its own.
template <int D>
__device__ __forceinline__ bool bucket_fill(Buckets& bk, const BoxInfo<D>& bx, bool valid,
                                            const int base[D]) {
  if (!valid) return false;
  const int key = bucket_key<D>(bx, base);
  const int slot = atomicAdd(&bk.count[key], 1);
  if (slot < kBucketSlots) {
    bk.order[key * kBucketSlots + slot] = (unsigned char)threadIdx.x;
    return false;
  }
  return true;
}

// One particle's 3^D reductions (mass W * mass_c when WITH_MASS, vector W (a + B dpos)) into
// grid g from its own registers (the per-particle path)
template <int D, bool WITH_MASS>
__device__ __forceinline__ void scatter_one(float4* g, int n, const Axes<D>& s, const float a[D],
                                            const float B[D][D], float mass_c) {
  float4* gb = g + node_flat<D>(s.base, n);
  for_nodes<D>(s.w, [&](int i, int jj, int k, float W) {
    float q[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int c = 0; c < D; ++c) {
      q[c] = a[c] + B[c][0] * s.dp[0][i] + B[c][1] * s.dp[1][jj];
      if (D == 3) q[c] += B[c][D - 1] * s.dp[D - 1][k];
    }
    float4 v = WITH_MASS ? make_float4(W * mass_c, W * q[0], W * q[1], D == 3 ? W * q[2] : 0.0f)
                         : make_float4(W * q[0], W * q[1], D == 3 ? W * q[2] : 0.0f, 0.0f);
    atomicAdd(gb + stencil_off<D>(i, jj, k, n), v);
  });
}

// Every warp takes groups of the table in turn (3D: one group per warp step, lanes 0..26;
// 2D: three groups, lanes 0..26 in threes of nine), sums each group's records into its
// lane's node and issues one reduction per node; a group's count is reset to zero once
// read, so the table is empty again for its next use.  The caller synchronised the CTA
// after filling the table and writing the records.
template <int D, bool WITH_MASS>
__device__ __forceinline__ void scatter_buckets(Buckets& bk, int K, const BoxInfo<D>& bx,
                                                const float* xr, float4* g, int n, const SimParams& P,
                                                float mass_c) {
  constexpr int L = D == 3 ? 27 : 9;  // nodes of a stencil = lanes per group
  constexpr int PER = 32 / L;         // groups per warp step
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int sub = lane / L, o = lane - sub * L;
  const bool lane_on = sub < PER;
  int off[3];
  off[0] = D == 3 ? o / 9 : o / 3;
  off[1] = D == 3 ? (o / 3) % 3 : o % 3;
  off[2] = D == 3 ? o % 3 : 0;
  // the quadratic B-spline weight of stencil offset off_a as alpha (f - beta)^2 + gamma
  float alpha[D], beta[D], gamma[D], odx[D];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    alpha[a] = off[a] == 1 ? -1.0f : 0.5f;
    beta[a] = off[a] == 0 ? 1.5f : (off[a] == 1 ? 1.0f : 0.5f);
    gamma[a] = off[a] == 1 ? 0.75f : 0.0f;
    odx[a] = (float)off[a];
  }
  int kd[D];
#pragma unroll
  for (int a = 0; a < D; ++a) kd[a] = bx.dim[a] - 2;
  for (int k0 = warp * PER; k0 < K; k0 += nwarps * PER) {
    const int key = k0 + sub;
    const bool on = lane_on && key < K;
    int cnt = on ? bk.count[key] : 0;
    if (!__any_sync(0xffffffffu, cnt > 0)) continue;
    const int m = cnt < kBucketSlots ? cnt : kBucketSlots;
    float am = 0.0f, aq[3] = {0.0f, 0.0f, 0.0f};
    for (int s = 0; s < m; ++s) {
      const int q = bk.order[key * kBucketSlots + s];
      const float4* r4 = reinterpret_cast<const float4*>(xr) + q * (Aos<D>::kFloats / 4);
      float r[Aos<D>::kFloats];
#pragma unroll
      for (int i = 0; i < Aos<D>::kFloats / 4; ++i) {
        const float4 v = r4[i];
        r[4 * i] = v.x;
        r[4 * i + 1] = v.y;
        r[4 * i + 2] = v.z;
        r[4 * i + 3] = v.w;
      }
      float W = 1.0f, dp[D];
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const float f = r[a];
        const float t = f - beta[a];
        W *= fmaf(alpha[a] * t, t, gamma[a]);
        dp[a] = (odx[a] - f) * P.dx;
      }
#pragma unroll
      for (int c = 0; c < D; ++c) {
        float qc = r[D + c];
#pragma unroll
        for (int b = 0; b < D; ++b) qc = fmaf(r[2 * D + c * D + b], dp[b], qc);
        aq[c] = fmaf(W, qc, aq[c]);
      }
      am += W;
    }
    if (on && cnt > 0) {
      int base[D], r = key;
#pragma unroll
      for (int a = D - 1; a >= 0; --a) {
        base[a] = bx.lo[a] + r % kd[a] + off[a];
        r /= kd[a];
      }
      const float4 v = WITH_MASS ? make_float4(am * mass_c, aq[0], aq[1], D == 3 ? aq[2] : 0.0f)
                                 : make_float4(aq[0], aq[1], D == 3 ? aq[2] : 0.0f, 0.0f);
      atomicAdd(g + node_flat<D>(base, n), v);
    }
    __syncwarp();
    if (on && o == 0 && cnt > 0) bk.count[key] = 0;
  }
}

// The bucketed form of one tile's scatter, from the CTA's stencil box bx (every thread
// calls it; bx came from box_extent, whose barrier separates this from the table's
// previous use).  Writes the records, fills the table, synchronises, scatters by group and
// lets overflowing particles scatter on their own.  Returns false (nothing done, no
// barrier) when the tile's base box exceeds the table; the caller then takes the
// per-particle path.
template <int D, bool WITH_MASS>
__device__ __forceinline__ bool bucket_scatter_tile(Buckets& bk, const BoxInfo<D>& bx, bool valid,
                                                    const Axes<D>& s, const float a[D],
                                                    const float B[D][D], float* xr, float4* g,
                                                    int n, const SimParams& P, float mass_c) {
  const int K = bucket_keys<D>(bx);
  if (K > kBucketKeys) return false;
  if (valid) put_record_aos<D>(xr, s.f, a, B);
  const bool over = bucket_fill<D>(bk, bx, valid, s.base);
  __syncthreads();
  scatter_buckets<D, WITH_MASS>(bk, K, bx, xr, g, n, P, mass_c);
  if (over) scatter_one<D, WITH_MASS>(g, n, s, a, B, mass_c);
  return true;
}

__device__ __forceinline__ float particle_act(const SimParams& P, const float* basis, const int* group,
                                              const float* wact, int scene, int64_t p, int dim,
                                              int& axis) {
  axis = 0;
  if (P.n_groups <= 0) return 0.0f;
  int g = group[p];
  if (g < 0 || g >= P.n_groups) return 0.0f;
  axis = g % dim;
  const float* w = wact + ((int64_t)scene * P.n_groups + g) * P.n_basis;
  float a = 0.0f;
#pragma unroll
  for (int k = 0; k < kMaxBasis; ++k)
    if (k < P.n_basis) a += w[k] * basis[k];
  return a;
}

template <int D>
__device__ __forceinline__ void load_E(const float* rows, int64_t N, int64_t p, float f_diag,
                                       float E[D][D]) {
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j)
      E[i][j] = rows[(Rows<D>::F + i * D + j) * N + p] - (i == j ? f_diag : 0.0f);
}

// ---------------------------------------------------------------------------
// grid functions applied at gather time
// ---------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ bool is_wall(const int idx[D], const SimParams& P) {
  bool wall = false;
#pragma unroll
  for (int a = 0; a < D; ++a) wall = wall || idx[a] < P.wall || idx[a] >= P.n_grid - P.wall;
  return wall;
}

// grid_op: v = p/m + dt g for m > 0 off the sticky walls, else 0 (w keeps m).  Rounding is
// spelled out (no compiler-chosen contraction), so a node gives the same bits whether it
// is staged in the shared gather box or read directly.
template <int D>
__device__ __forceinline__ float4 node_velocity(float4 pm, const int idx[D], const SimParams& P) {
  float4 u = make_float4(0.0f, 0.0f, 0.0f, pm.x);
  if (pm.x > 0.0f && !is_wall<D>(idx, P)) {
    const float im = __fdiv_rn(1.0f, pm.x);
    u.x = __fmaf_rn(pm.y, im, __fmul_rn(P.dt, P.gravity[0]));
    u.y = __fmaf_rn(pm.z, im, __fmul_rn(P.dt, P.gravity[1]));
    if (D == 3) u.z = __fmaf_rn(pm.w, im, __fmul_rn(P.dt, P.gravity[2]));
  }
  return u;
}

// grid_op.grad: pbar = ubar / m and mbar = -ubar . (p / m) / m for m > 0 off the walls
// (rounding spelled out as in node_velocity)
template <int D>
__device__ __forceinline__ float4 node_adjoint(float4 ub, float4 pm, const int idx[D],
                                               const SimParams& P) {
  float4 r = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  if (pm.x > 0.0f && !is_wall<D>(idx, P)) {
    const float im = __fdiv_rn(1.0f, pm.x);
    r.x = __fmul_rn(ub.x, im);
    r.y = __fmul_rn(ub.y, im);
    float dot = __fmaf_rn(ub.y, pm.z, __fmul_rn(ub.x, pm.y));
    if (D == 3) {
      r.z = __fmul_rn(ub.z, im);
      dot = __fmaf_rn(ub.z, pm.w, dot);
    }
    r.w = __fmul_rn(__fmul_rn(-dot, im), im);
  }
  return r;
}

// ---------------------------------------------------------------------------
// clears and box resets (each CTA takes its share of its own scene)
// ---------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ void run_clears(const Clears& C, int scene, int rank, int nranks,
                                           int nnodes, int n) {
  for (int c = 0; c < C.n; ++c) {
    const int* bb = C.job[c].box + scene * 8;
    // An empty box (lo = INT_MAX, hi = INT_MIN: a buffer that was allocated but never
    // scattered into, e.g. after a pass that gave up) clears nothing; hi - lo is formed
    // only for a non-empty box, and the box is clipped to the grid.
    int lo[D], ext[D], vol = 1;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      lo[a] = bb[a] > 0 ? bb[a] : 0;
      const int hi = bb[4 + a] < n - 1 ? bb[4 + a] : n - 1;
      ext[a] = hi >= lo[a] ? hi - lo[a] + 1 : 0;
      vol *= ext[a];
    }
    const int w = C.words;
    float4* g = C.job[c].grid + (int64_t)scene * nnodes * w;
    for (int l = rank * blockDim.x + threadIdx.x; l < vol; l += nranks * blockDim.x) {
      int idx[D], r = l;
#pragma unroll
      for (int a = D - 1; a >= 0; --a) {
        idx[a] = lo[a] + r % ext[a];
        r /= ext[a];
      }
      float4* q = g + (int64_t)node_flat<D>(idx, n) * w;
      q[0] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      if (w == 2) q[1] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
  }
}

__device__ __forceinline__ void reset_box(int* box, int scene) {
  if (box && threadIdx.x < 8) box[scene * 8 + threadIdx.x] = (threadIdx.x & 4) ? INT_MIN : INT_MAX;
}

// ---------------------------------------------------------------------------
// P2G of the CTA's particles: stress, affine matrix A = kappa tau + m C, scatter
// (m, m v + A dpos) into the scene grid g, fold the touched box into box_scene.
// Every thread calls it; s_bbox must have been reset before an earlier barrier.
// ---------------------------------------------------------------------------
template <int D, int MAT, bool DET>
__device__ __forceinline__ void p2g_pass(const SimParams& P, const float* basis, bool active, int scene,
                                         int64_t p, int count, const float x[D], const float v[D],
                                         const float C[D][D], const float E[D][D], float mu_p,
                                         float la_p, int mat_p, const int* group, const float* wact,
                                         float4* g, int* box_scene, float* sm, float* xr,
                                         int* s_box, int* s_bbox, Buckets& bk, unsigned& err,
                                         const double* R_in, double* R_out, int64_t N, bool pair) {
  Axes<D> s;
  bool ok = make_axes<D>(x, P, s) && active;
  if (active && !ok) err |= kErrOOB;
  float Am[D][D], mv[D];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    mv[i] = 0.0f;
#pragma unroll
    for (int j = 0; j < D; ++j) Am[i][j] = 0.0f;
  }
  if (ok) {
    int axis;
    const float act = particle_act(P, basis, group, wact, scene, p, D, axis);
    float tau[D][D];
    StressCache<D> sc;
    if (!kirchhoff<D, MAT>(E, mu_p, la_p, act, axis, tau, sc, R_in, N, p, mat_p)) {
      err |= kErrNonFinite;
      ok = false;
    }
    // the polar cache is a 3D fixed-corotated feature
    if (D == 3 && (MAT == kFixedCorotated || (MAT == kMixed && mat_p == kFixedCorotated)) && R_out && active)
      polar_to_cache<D>(R_out, N, p, sc.pol);
#pragma unroll
    for (int i = 0; i < D; ++i) {
      mv[i] = P.p_mass * v[i];
#pragma unroll
      for (int j = 0; j < D; ++j) Am[i][j] = P.kappa * tau[i][j] + P.p_mass * C[i][j];
    }
  }
  __syncthreads();  // the record area may still be read by an earlier scatter
  if (!DET && P.bucket && P.tile_capacity == 0) {
    const BoxInfo<D> bx = box_extent<D>(ok, s.base, INT_MAX, s_box + 16);
    if (bucket_scatter_tile<D, true>(bk, bx, ok, s, mv, Am, xr, g, P.n_grid, P, P.p_mass)) {
      if (threadIdx.x == 0 && bx.vol > 0) {
#pragma unroll
        for (int a = 0; a < D; ++a) {
          atomicMin(&box_scene[a], bx.lo[a]);
          atomicMax(&box_scene[4 + a], bx.lo[a] + bx.dim[a] - 1);
        }
      }
      return;
    }
  }
  put_record<D>(xr, ok, s.base, s.f, mv, Am);
  if (P.tile_capacity > 0) {
    const BoxInfo<D> bx = box_extent<D>(ok, s.base, P.tile_capacity, s_box + 16);
    box_zero<D>(bx, sm, P.tile_capacity);
    scatter_records<D, true, DET>(xr, count, bx, sm, P.tile_capacity, g, P.n_grid, P, P.p_mass, P.fix_m,
                             P.fix_p, err, pair);
    box_flush<D>(bx, sm, P.tile_capacity, g, P.n_grid);
    if (threadIdx.x == 0 && bx.vol > 0) {
#pragma unroll
      for (int a = 0; a < D; ++a) {
        atomicMin(&box_scene[a], bx.lo[a]);
        atomicMax(&box_scene[4 + a], bx.lo[a] + bx.dim[a] - 1);
      }
    }
  } else {
    warp_bbox<D>(ok, s.base, s_bbox);
    __syncthreads();
    cta_bbox_flush<D>(s_bbox, box_scene);
    BoxInfo<D> none;
    none.use_tile = false;
    scatter_records<D, true, DET>(xr, count, none, sm, 0, g, P.n_grid, P, P.p_mass, P.fix_m, P.fix_p, err,
                                  pair);
  }
}

// ---------------------------------------------------------------------------
// forward particle pass: [G2P of step t-1] then [P2G of step t]
// ---------------------------------------------------------------------------
// One tile of a forward pass; every thread of the CTA calls it.  sm: dynamic shared memory
// (step_smem_bytes), s_box: 8 * kBoxSlots ints, s_bbox: 8 ints.  A CTA that runs several tiles must
// synchronise between them.
template <int D, int MAT, int MODE, bool NC, bool DET>
__device__ __forceinline__ void step_tile(const SimParams& P, const StepArgs& A, int tile_index,
                                          float* sm, int* s_box, int* s_bbox, Buckets& bk) {
  using R = Rows<D>;
  cta_bbox_reset(s_bbox);
  reset_box_slots(s_box);
  float* xr = sm + box_floats(P.tile_capacity, P.gather_capacity);
  const int4 tile = A.tiles[tile_index];
  const int scene = tile.x;
  const bool active = (int)threadIdx.x < tile.z;
  const int64_t p = (int64_t)tile.y + (active ? threadIdx.x : 0);
  const int64_t N = A.N;
  const int n = P.n_grid;
  unsigned err = 0;
  run_clears<D>(A.clears, scene, tile.w, A.scene_tiles[scene], P.nnodes, n);
  if (tile.w == 0) reset_box(A.box_reset, scene);
  float* stage = xr + Xch<D>::kWidth * Xch<D>::kStride;
  if (MODE != kG2POnlyFull) {
    stage_row(stage, 0, A.mu + p);
    stage_row(stage, 1, A.la + p);
  }
  stage_commit();
  __syncthreads();  // s_bbox reset

  float x[D], v[D], C[D][D], E[D][D];
  if (MODE == kP2GOnly) {
#pragma unroll
    for (int a = 0; a < D; ++a) {
      x[a] = A.in[(R::X + a) * N + p];
      v[a] = A.in[(R::V + a) * N + p];
    }
#pragma unroll
    for (int i = 0; i < D * D; ++i) C[i / D][i % D] = A.in[(R::C + i) * N + p];
    load_E<D>(A.in, N, p, P.f_diag, E);
  } else {
    // ---- G2P: v' = sum W u, C' = 4/dx^2 sum W (u - u_c) dpos^T, x' = x + dt v',
    //      E' = E + dt C' (I + E), with u = grid_op(PM of step t-1) at each node
    float xo[D], Eo[D][D];
#pragma unroll
    for (int a = 0; a < D; ++a) xo[a] = A.in[(R::X + a) * N + p];
    load_E<D>(A.in, N, p, P.f_diag, Eo);
    Axes<D> s;
    const bool ok = make_axes<D>(xo, P, s) && active;
    if (active && !ok) err |= kErrOOB;
    float B[D][D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      v[a] = 0.0f;
#pragma unroll
      for (int b = 0; b < D; ++b) B[a][b] = 0.0f;
    }
    const float4* PMg = scene_grid(A.PMr, scene, P);
    auto velocity = [&](const int idx[D]) { return node_velocity<D>(pm_load<NC, DET>(PMg, node_flat<D>(idx, n), P), idx, P); };
    BoxInfo<D> gbx;
    gbx.use_tile = false;
    if (P.gather_capacity > 0) {
      gbx = box_extent<D>(ok, s.base, P.gather_capacity, s_box);  // slot 0
      if (A.box_stats && threadIdx.x == 0 && gbx.vol > 0) {
        atomicAdd(A.box_stats, 1ull);
        if (!gbx.use_tile) atomicAdd(A.box_stats + 1, 1ull);
      }
      box_load<D>(gbx, reinterpret_cast<float4*>(sm), velocity);
    }
    if (ok) {
      // centred on the stencil's centre node: equal because sum W dpos = 0, and
      // accurate in FP32 when u is nearly uniform over the stencil
      with_nodes<D>(gbx, reinterpret_cast<const float4*>(sm), s.base, velocity, [&](auto load) {
        const float4 uc4 = load(1, 1, D == 3 ? 1 : 0);
        const float uc[3] = {uc4.x, uc4.y, uc4.z};
        for_nodes<D>(s.w, [&](int i, int j, int k, float W) {
          const float4 u4 = load(i, j, k);
          const float u[3] = {u4.x, u4.y, u4.z};
          const float dpos[3] = {s.dp[0][i], s.dp[1][j], D == 3 ? s.dp[D - 1][k] : 0.0f};
#pragma unroll
          for (int a = 0; a < D; ++a) {
            v[a] += W * u[a];
            const float wd = W * (u[a] - uc[a]);
#pragma unroll
            for (int b = 0; b < D; ++b) B[a][b] += wd * dpos[b];
          }
        });
      });
    }
    const float c4 = 4.0f * P.inv_dx * P.inv_dx;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int b = 0; b < D; ++b) C[a][b] = c4 * B[a][b];
#pragma unroll
    for (int a = 0; a < D; ++a) x[a] = P.xfix ? pos_advance(xo[a], P.dt * v[a]) : xo[a] + P.dt * v[a];
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = 0; j < D; ++j) {
        float g = P.dt * C[i][j];  // dt C' (I + E)
#pragma unroll
        for (int k = 0; k < D; ++k) g += P.dt * C[i][k] * Eo[k][j];
        E[i][j] = Eo[i][j] + g;
      }
    if (active) {
#pragma unroll
      for (int a = 0; a < D; ++a) A.out[(R::X + a) * N + p] = x[a];
#pragma unroll
      for (int i = 0; i < D * D; ++i)
        A.out[(R::F + i) * N + p] = E[i / D][i % D] + (i / D == i % D ? P.f_diag : 0.0f);
      if (MODE == kG2PP2GFull || MODE == kG2POnlyFull) {
#pragma unroll
        for (int a = 0; a < D; ++a) A.out[(R::V + a) * N + p] = v[a];
#pragma unroll
        for (int i = 0; i < D * D; ++i) A.out[(R::C + i) * N + p] = C[i / D][i % D];
      }
    }
  }

  if (MODE != kG2POnlyFull) {
    stage_wait<0>();
    p2g_pass<D, MAT, DET>(P, P.basis, active, scene, p, tile.z, x, v, C, E, staged(stage, 0),
                          staged(stage, 1), MAT == kMixed ? A.matid[p] : MAT, A.group, A.wact,
                     scene_grid(A.PMw, scene, P), A.box_w + scene * 8, sm, xr, s_box, s_bbox,
                     bk, err, nullptr, A.Rw, N, (P.pair & 1) != 0);
  }
  if (err) atomicOr(A.err, err);
}

// resident CTAs per SM the forward passes are compiled for
template <int D, int MAT>
constexpr int step_ctas_per_sm() {
  return D == 2 ? MPM_STEP_CTAS_PER_SM_2D
                : (MAT == kFixedCorotated || MAT == kMixed) ? MPM_STEP_CTAS_PER_SM_3D_POLAR
                                                           : MPM_STEP_CTAS_PER_SM_3D;
}

template <int D, int MAT, int MODE, bool DET>
__global__ void __launch_bounds__(kTile, step_ctas_per_sm<D, MAT>())
    step_kernel(const __grid_constant__ SimParams P, const __grid_constant__ StepArgs A) {
  extern __shared__ __align__(16) float sm[];
  __shared__ int s_box[8 * kBoxSlots];
  __shared__ int s_bbox[8];
  __shared__ Buckets s_bk;
  buckets_zero(s_bk);  // ordered before its first use by the tile's first barrier
  step_tile<D, MAT, MODE, true, DET>(P, A, blockIdx.x, sm, s_box, s_bbox, s_bk);
}

// ---------------------------------------------------------------------------
// adjoint particle pass: [P2G-adjoint of step s+1] [G2P-adjoint of step s]
// [recomputed P2G of step s-1, the grid the next adjoint pass needs (Appendix D.1)]
// ---------------------------------------------------------------------------
// One tile of an adjoint pass (same calling rules as step_tile; s_wbar: kWbarSlots floats).
template <int D, int MAT, int MODE, bool NC, bool DET>
__device__ __forceinline__ void adjoint_tile(const SimParams& P, const AdjArgs& A, int tile_index,
                                             float* sm, int* s_box, int* s_bbox_ub, int* s_bbox_pm,
                                             float* s_wbar, Buckets& bk) {
  using R = Rows<D>;
  cta_bbox_reset(s_bbox_ub);
  cta_bbox_reset(s_bbox_pm);
  reset_box_slots(s_box);
  float* xr = sm + box_floats(P.tile_capacity, P.gather_capacity);
  const int4 tile = A.tiles[tile_index];
  const int scene = tile.x;
  const bool active = (int)threadIdx.x < tile.z;
  const int64_t p = (int64_t)tile.y + (active ? threadIdx.x : 0);
  const int64_t N = A.N;
  const int n = P.n_grid;
  const float c4 = 4.0f * P.inv_dx * P.inv_dx;
  unsigned err = 0;
  run_clears<D>(A.clears, scene, tile.w, A.scene_tiles[scene], P.nnodes, n);
  if (tile.w == 0) {
    reset_box(A.box_ub_reset, scene);
    reset_box(A.box_m_reset, scene);
  }
  __syncthreads();  // shared boxes reset
  // stage what the G2P-adjoint (state s: x, F) and the recomputed P2G (state s-1, mu, la)
  // read, so that those loads are in flight during the P2G-adjoint
  float* stage = xr + Xch<D>::kWidth * Xch<D>::kStride;
  if (MODE != kAdjP2G) {
#pragma unroll
    for (int a = 0; a < D; ++a) stage_row(stage, a, A.st0 + (int64_t)(R::X + a) * N + p);
#pragma unroll
    for (int i = 0; i < D * D; ++i) stage_row(stage, D + i, A.st0 + (int64_t)(R::F + i) * N + p);
  }
  stage_commit();
  if (MODE != kAdjP2G && A.stm) {  // the recomputed P2G runs whenever state s-1 is given
#pragma unroll
    for (int r = 0; r < R::Q; ++r) stage_row(stage, Stage<D>::kAdjB + r, A.stm + (int64_t)r * N + p);
    stage_row(stage, Stage<D>::kAdjB + R::Q, A.mu + p);
    stage_row(stage, Stage<D>::kAdjB + R::Q + 1, A.la + p);
  }
  stage_commit();

  // adjoint of state s+1: xb, vb, Cb, Fb (Fb = dL/dE = dL/dF); C1 = C of state s+1.  In 3D,
  // after a P2G-adjoint the carried xb, Fb and the rows of state s+1 needed again (C, E,
  // mu, la, the polar factor) are read after its gather -- fresh loads, as the gather's
  // barriers order them -- so that none of them holds a register across the gather (in 2D
  // they fit: loaded once, before it)
  constexpr bool kLate = D == 3;
  float xb[D], vb[D], Cb[D][D], Fb[D][D];
  float C1[D][D];
  auto load_carried = [&]() {
#pragma unroll
    for (int a = 0; a < D; ++a) xb[a] = A.adj[(R::X + a) * N + p];
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = 0; j < D; ++j) {
        Fb[i][j] = A.adj[(R::F + i * D + j) * N + p];
        C1[i][j] = A.st1[(R::C + i * D + j) * N + p];
      }
  };

  if (MODE == kAdjG2P || !kLate) load_carried();
  if (MODE == kAdjG2P) {
#pragma unroll
    for (int a = 0; a < D; ++a) vb[a] = A.adj[(R::V + a) * N + p];
#pragma unroll
    for (int i = 0; i < D * D; ++i) Cb[i / D][i % D] = A.adj[(R::C + i) * N + p];
  } else {
    // ---- P2G adjoint of step s+1: gather (pbar, mbar) = grid_op.grad(ubar, (m, p)) ----
    float x[D], v[D], E[D][D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      x[a] = A.st1[(R::X + a) * N + p];
      v[a] = A.st1[(R::V + a) * N + p];
    }
    load_E<D>(A.st1, N, p, P.f_diag, E);
    Axes<D> s;
    bool ok = make_axes<D>(x, P, s) && active;
    if (active && !ok) err |= kErrOOB;
    int axis;
    const float act = particle_act(P, P.basis, A.group, A.wact, scene, p, D, axis);
    const float mu = A.mu[p], la = A.la[p];
    float tau[D][D];
    StressCache<D> sc;
    const int mat_p = MAT == kMixed ? A.matid[p] : MAT;
    if (!kirchhoff<D, MAT>(E, mu, la, act, axis, tau, sc, A.R1, N, p, mat_p) && ok) {
      err |= kErrNonFinite;
      ok = false;
    }
    float Am[D][D], mv[D];
#pragma unroll
    for (int i = 0; i < D; ++i) {
      mv[i] = P.p_mass * v[i];
#pragma unroll
      for (int j = 0; j < D; ++j)
        Am[i][j] = P.kappa * tau[i][j] + P.p_mass * (kLate ? A.st1[(R::C + i * D + j) * N + p] : C1[i][j]);
    }
    float Ab[D][D], xg[D], sw[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      vb[a] = 0.0f;
      xg[a] = 0.0f;
      sw[a] = 0.0f;
#pragma unroll
      for (int b = 0; b < D; ++b) Ab[a][b] = 0.0f;
    }
    const float4* UBg = scene_grid(A.UB1, scene, P);
    const float4* PMg = scene_grid(A.PM1, scene, P);
    auto pbar = [&](const int idx[D]) {
      const int f = node_flat<D>(idx, n);
      return node_adjoint<D>(ub_load<NC, DET>(UBg, f, P, A.ub_m0), pm_load<NC, DET>(PMg, f, P), idx, P);
    };
    BoxInfo<D> gbx;
    gbx.use_tile = false;
    if (P.gather_capacity > 0) {
      gbx = box_extent<D>(ok, s.base, P.gather_capacity, s_box);  // slot 0
      box_load<D>(gbx, reinterpret_cast<float4*>(sm), pbar);
    }
    if (ok) with_nodes<D>(gbx, reinterpret_cast<const float4*>(sm), s.base, pbar, [&](auto load) {
      // pbar - pbar_c and mbar - mbar_c (centre node) in the moment and weight-gradient
      // terms: equal to the plain sums because sum W dpos = 0, sum grad W = 0 and
      // sum grad W dpos^T = I, without the FP32 cancellation of a smooth pbar field
      const float4 gc = load(1, 1, D == 3 ? 1 : 0);
      const float pc[3] = {gc.x, gc.y, gc.z};
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        float qi[D];
#pragma unroll
        for (int c = 0; c < D; ++c) qi[c] = mv[c] + Am[c][0] * s.dp[0][i];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const float wij = s.w[0][i] * s.w[1][j];
          const float dwij0 = s.dw[0][i] * s.w[1][j];
          const float dwij1 = s.w[0][i] * s.dw[1][j];
          float qij[D];
#pragma unroll
          for (int c = 0; c < D; ++c) qij[c] = qi[c] + Am[c][1] * s.dp[1][j];
#pragma unroll
          for (int k = 0; k < (D == 3 ? 3 : 1); ++k) {
            const float wk = D == 3 ? s.w[D - 1][k] : 1.0f;
            const float W = wij * wk;
            float gW[D];
            gW[0] = dwij0 * wk;
            gW[1] = dwij1 * wk;
            if (D == 3) gW[D - 1] = wij * s.dw[D - 1][k];
            float q[D];
#pragma unroll
            for (int c = 0; c < D; ++c)
              q[c] = D == 3 ? qij[c] + Am[c][D - 1] * s.dp[D - 1][k] : qij[c];
            const float dpos[3] = {s.dp[0][i], s.dp[1][j], D == 3 ? s.dp[D - 1][k] : 0.0f};
            const float4 g4 = load(i, j, k);
            const float pb[3] = {g4.x, g4.y, g4.z};
            float Wbar = P.p_mass * (g4.w - gc.w);
#pragma unroll
            for (int c = 0; c < D; ++c) {
              const float dpb = pb[c] - pc[c];
              Wbar += dpb * q[c];
              vb[c] += W * pb[c];
              sw[c] += W * dpb;
#pragma unroll
              for (int b = 0; b < D; ++b) Ab[c][b] += W * dpb * dpos[b];
            }
#pragma unroll
            for (int b = 0; b < D; ++b) xg[b] += Wbar * gW[b];
          }
        }
      }
    });
    if (kLate) load_carried();
    // x += inv_dx sum Wbar gradW - A^T sum W dpbar
#pragma unroll
    for (int b = 0; b < D; ++b) {
      float atw = 0.0f;
#pragma unroll
      for (int a = 0; a < D; ++a) atw += Am[a][b] * sw[a];
      xb[b] += P.inv_dx * xg[b] - atw;
      vb[b] *= P.p_mass;
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
    if (kLate) load_E<D>(A.st1, N, p, P.f_diag, E);
    if (kLate && (MAT == kFixedCorotated || MAT == kMixed)) {
      // the polar factor again (from the cache, or recomputed where the state has no cached
      // factor: one adjoint pass per segment), so that it holds no registers across the
      // gather; the stress itself is not needed again
      float tau_again[D][D];
      kirchhoff<D, MAT>(E, A.mu[p], A.la[p], act, axis, tau_again, sc, A.R1, N, p, mat_p);
    }
    if (ok) abar = kirchhoff_adjoint<D, MAT>(E, A.mu[p], A.la[p], act, axis, sc, tb, Fb, mub, lab, mat_p);
    if (active) {
      float2 ms = A.mubar[p], ls = A.labar[p];
      compensated_add(ms, mub);
      compensated_add(ls, lab);
      A.mubar[p] = ms;
      A.labar[p] = ls;
    }
    if (P.n_groups > 0) {
      // dL/dw_gk += basis_k * sum of abar over this tile's particles of group g, reduced in
      // a fixed order (warp butterfly, then warps in order) into the tile's own slot, so
      // the result does not depend on scheduling; the tiles are summed in order at the end
      int g = -1;
      if (ok) {
        g = A.group[p];
        if (g < 0 || g >= P.n_groups) g = -1;
      }
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
      for (int gg = 0; gg < kMaxGroups; ++gg) {
        if (gg < P.n_groups) {
          float v = (g == gg) ? abar : 0.0f;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
          if (lane == 0) s_wbar[warp * kMaxGroups + gg] = v;
        }
      }
      __syncthreads();
      const int GK = P.n_groups * P.n_basis;
      if ((int)threadIdx.x < GK) {
        const int gg = threadIdx.x / P.n_basis, k = threadIdx.x % P.n_basis;
        float sum = 0.0f;
        for (int w = 0; w < kTile / 32; ++w) sum += s_wbar[w * kMaxGroups + gg];
        A.wbar_tile[(int64_t)tile_index * GK + threadIdx.x] += sum * P.basis[k];
      }
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

  // ---- G2P adjoint of step s: x' = x + dt v', E' = E + dt C' (I + E) ----
  {
    float x0[D], E0[D][D];
#pragma unroll
    stage_wait<0>();
#pragma unroll
    for (int a = 0; a < D; ++a) x0[a] = staged(stage, a);
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = 0; j < D; ++j) E0[i][j] = staged(stage, D + i * D + j) - (i == j ? P.f_diag : 0.0f);
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
        float g = Fb[i][j], h = Cb[i][j] + P.dt * Fb[i][j];
#pragma unroll
        for (int k = 0; k < D; ++k) {
          g += P.dt * C1[k][i] * Fb[k][j];  // (I + dt C')^T Fbar'
          h += P.dt * Fb[i][k] * E0[j][k];  // Cbar' + dt Fbar' (I + E)^T
        }
        Fb0[i][j] = g;
        Ct[i][j] = h;
      }
    Axes<D> s;
    const bool ok = make_axes<D>(x0, P, s) && active;
    if (active && !ok) err |= kErrOOB;
    if (MODE == kAdjG2P && DET && A.measure) {
      // bound of this particle's ubar contributions W (vt + c4 Ct dpos), W <= 1, |dpos| <= 1.5 dx
      float bound = 0.0f;
      if (ok) {
#pragma unroll
        for (int a = 0; a < D; ++a) {
          float r = fabsf(vt[a]);
#pragma unroll
          for (int b = 0; b < D; ++b) r += 1.5f * P.dx * c4 * fabsf(Ct[a][b]);
          bound = fmaxf(bound, r);
        }
        if (!(bound <= 3.0e38f)) {
          err |= kErrNonFinite;
          bound = 0.0f;
        }
      }
      // non-negative floats order like their bit patterns
      const unsigned mb = __reduce_max_sync(0xffffffffu, __float_as_uint(bound));
      if ((threadIdx.x & 31) == 0 && mb != 0u) atomicMax(A.ub_m0, mb);
      if (err) atomicOr(A.err, err);
      return;
    }
    const float4* PMg = scene_grid(A.PM0, scene, P);
    auto velocity = [&](const int idx[D]) { return node_velocity<D>(pm_load<NC, DET>(PMg, node_flat<D>(idx, n), P), idx, P); };
    const int cap_box = P.tile_capacity > P.gather_capacity ? P.tile_capacity : P.gather_capacity;
    BoxInfo<D> bx;
    bx.use_tile = false;
    if (cap_box > 0) bx = box_extent<D>(ok, s.base, cap_box, s_box + 8);
    BoxInfo<D> gbx = bx;
    gbx.use_tile = bx.use_tile && P.gather_capacity > 0 && bx.vol <= P.gather_capacity;
    if (P.gather_capacity > 0) box_load<D>(gbx, reinterpret_cast<float4*>(sm), velocity);
    if (ok) with_nodes<D>(gbx, reinterpret_cast<const float4*>(sm), s.base, velocity, [&](auto load) {
      // x-adjoint terms on u - u_c (centre node), by the same B-spline identities
      const float4 uc4 = load(1, 1, D == 3 ? 1 : 0);
      const float uc[3] = {uc4.x, uc4.y, uc4.z};
      float xg[D], sw[D];
#pragma unroll
      for (int a = 0; a < D; ++a) xg[a] = sw[a] = 0.0f;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        float qi[D];
#pragma unroll
        for (int c = 0; c < D; ++c) qi[c] = vt[c] + c4 * Ct[c][0] * s.dp[0][i];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const float wij = s.w[0][i] * s.w[1][j];
          const float dwij0 = s.dw[0][i] * s.w[1][j];
          const float dwij1 = s.w[0][i] * s.dw[1][j];
          float qij[D];
#pragma unroll
          for (int c = 0; c < D; ++c) qij[c] = qi[c] + c4 * Ct[c][1] * s.dp[1][j];
#pragma unroll
          for (int k = 0; k < (D == 3 ? 3 : 1); ++k) {
            const float wk = D == 3 ? s.w[D - 1][k] : 1.0f;
            const float W = wij * wk;
            float gW[D];
            gW[0] = dwij0 * wk;
            gW[1] = dwij1 * wk;
            if (D == 3) gW[D - 1] = wij * s.dw[D - 1][k];
            const float4 u4 = load(i, j, k);
            const float du[3] = {u4.x - uc[0], u4.y - uc[1], u4.z - uc[2]};
            float Wbar = 0.0f;
#pragma unroll
            for (int c = 0; c < D; ++c) {
              const float q = D == 3 ? qij[c] + c4 * Ct[c][D - 1] * s.dp[D - 1][k] : qij[c];
              Wbar += du[c] * q;
              sw[c] += W * du[c];
            }
#pragma unroll
            for (int b = 0; b < D; ++b) xg[b] += Wbar * gW[b];
          }
        }
      }
#pragma unroll
      for (int b = 0; b < D; ++b) {
        float ctu = 0.0f;
#pragma unroll
        for (int a = 0; a < D; ++a) ctu += Ct[a][b] * sw[a];
        xb0[b] += P.inv_dx * xg[b] - c4 * ctu;
      }
    });
    if (active) {
#pragma unroll
      for (int a = 0; a < D; ++a) A.adj[(R::X + a) * N + p] = xb0[a];
#pragma unroll
      for (int i = 0; i < D * D; ++i) A.adj[(R::F + i) * N + p] = Fb0[i / D][i % D];
    }
    // ---- scatter ubar_i += W (vt + c4 Ct dpos) ----
    float Bs[D][D];
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = 0; j < D; ++j) Bs[i][j] = c4 * Ct[i][j];
    float4* UBs = scene_grid(A.UB0, scene, P);
    float fix_u = 1.0f, unfix_u = 1.0f;
    if (DET) ub_scales(A.ub_m0, fix_u, unfix_u);
    if (!DET && P.bucket && P.tile_capacity == 0 && cap_box > 0 &&
        bucket_scatter_tile<D, false>(bk, bx, ok, s, vt, Bs, xr, UBs, n, P, 0.0f)) {
      if (threadIdx.x == 0 && bx.vol > 0) {
#pragma unroll
        for (int a = 0; a < D; ++a) {
          atomicMin(&A.box_ub[scene * 8 + a], bx.lo[a]);
          atomicMax(&A.box_ub[scene * 8 + 4 + a], bx.lo[a] + bx.dim[a] - 1);
        }
      }
    } else if (P.tile_capacity > 0) {
      put_record<D>(xr, ok, s.base, s.f, vt, Bs);
      BoxInfo<D> sbx = bx;
      sbx.use_tile = bx.use_tile && bx.vol <= P.tile_capacity;
      box_zero<D>(sbx, sm, P.tile_capacity);  // same extent as the gather box
      scatter_records<D, false, DET>(xr, tile.z, sbx, sm, P.tile_capacity, UBs, n, P, 0.0f, fix_u, fix_u, err,
                                     false);
      box_flush<D>(sbx, sm, P.tile_capacity, UBs, n);
      if (threadIdx.x == 0 && sbx.vol > 0) {
#pragma unroll
        for (int a = 0; a < D; ++a) {
          atomicMin(&A.box_ub[scene * 8 + a], sbx.lo[a]);
          atomicMax(&A.box_ub[scene * 8 + 4 + a], sbx.lo[a] + sbx.dim[a] - 1);
        }
      }
    } else {
      put_record<D>(xr, ok, s.base, s.f, vt, Bs);
      warp_bbox<D>(ok, s.base, s_bbox_ub);
      __syncthreads();
      cta_bbox_flush<D>(s_bbox_ub, A.box_ub + scene * 8);
      BoxInfo<D> none;
      none.use_tile = false;
      scatter_records<D, false, DET>(xr, tile.z, none, sm, 0, UBs, n, P, 0.0f, fix_u, fix_u, err,
                                     (P.pair & 2) != 0);
    }
  }

  // ---- recomputed P2G of step s-1 (the grid of the next adjoint pass) ----
  if (A.stm) {
    float x[D], v[D], C[D][D], E[D][D];
    stage_wait<0>();
    constexpr int b = Stage<D>::kAdjB;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      x[a] = staged(stage, b + R::X + a);
      v[a] = staged(stage, b + R::V + a);
    }
#pragma unroll
    for (int i = 0; i < D * D; ++i) C[i / D][i % D] = staged(stage, b + R::C + i);
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = 0; j < D; ++j) E[i][j] = staged(stage, b + R::F + i * D + j) - (i == j ? P.f_diag : 0.0f);
    p2g_pass<D, MAT, DET>(P, P.basis2, active, scene, p, tile.z, x, v, C, E, staged(stage, b + R::Q),
                          staged(stage, b + R::Q + 1), MAT == kMixed ? A.matid[p] : MAT, A.group,
                          A.wact,
                     scene_grid(A.PMm, scene, P), A.box_m + scene * 8, sm, xr, s_box, s_bbox_pm,
                     bk, err, A.Rm, nullptr, N, (P.pair & 2) != 0);
  }
  if (err) atomicOr(A.err, err);
}

template <int D, int MAT, int MODE, bool DET>
__global__ void __launch_bounds__(kTile, MPM_ADJ_CTAS_PER_SM)
    adjoint_kernel(const __grid_constant__ SimParams P, const __grid_constant__ AdjArgs A) {
  extern __shared__ __align__(16) float sm[];
  __shared__ int s_box[8 * kBoxSlots];
  __shared__ int s_bbox_ub[8];
  __shared__ int s_bbox_pm[8];
  __shared__ float s_wbar[kWbarSlots];
  __shared__ Buckets s_bk;
  buckets_zero(s_bk);  // ordered before its first use by the tile's first barrier
  adjoint_tile<D, MAT, MODE, true, DET>(P, A, blockIdx.x, sm, s_box, s_bbox_ub, s_bbox_pm, s_wbar,
                                        s_bk);
}

// ---------------------------------------------------------------------------
// persistent launches: one co-resident (cooperative) grid runs a list of passes of one
// kind with a grid-wide barrier between consecutive passes.  The list is recorded on the
// host by the same code that issues the one-launch-per-pass form, so the two run the
// same passes on the same buffers in the same order.
// ---------------------------------------------------------------------------
enum PassKind : int { kPassStep = 0, kPassAdjoint = 1 };

struct __align__(16) PassEntry {
  int kind;  // PassKind
  int mode;  // StepMode or AdjMode
  int pad[2];
  SimParams P;
  StepArgs S;  // kPassStep
  AdjArgs A;   // kPassAdjoint
};

struct GridSync {
  unsigned arrived;  // CTA arrivals at the barriers of this launch (reset before it)
  unsigned abort;    // set by a CTA whose wait ran out; every CTA then leaves
};

struct PersistCtl {
  GridSync* sync;
  unsigned* tickets;     // [n_pass] tile tickets (reset before the launch)
  unsigned* err;
  long long timeout_ns;  // limit of one barrier wait
  unsigned extra;        // arrivals a barrier waits for beyond the grid's own (0; a nonzero
                         // value makes every wait run out: the timeout path's test hook)
};

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned ld_relaxed_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier: returns when `target` arrivals have been counted, or false when the
// wait ran out (err |= kErrTimeout, abort raised) or another CTA aborted.  The wait is
// bounded twice: by the global nanosecond timer and by the SM cycle counter (4 cycles per
// ns of limit, at least twice the limit at any SM clock up to 2 GHz), so it ends even if
// one of the two clocks stalls.
__device__ __forceinline__ bool grid_barrier(const PersistCtl& c, unsigned target, int* s_go) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();  // this CTA's grid and state writes before its arrival
    atomicAdd(&c.sync->arrived, 1u);
    int go = 1;
    const unsigned long long t0 = globaltimer_ns();
    const long long c0 = clock64();
    const long long cycle_limit = 4 * c.timeout_ns;
    for (unsigned it = 1;; ++it) {
      if (ld_acquire_gpu(&c.sync->arrived) >= target) break;
      if (ld_relaxed_gpu(&c.sync->abort)) {
        go = 0;
        break;
      }
      if ((it & 15u) == 0 && ((long long)(globaltimer_ns() - t0) > c.timeout_ns ||
                              clock64() - c0 > cycle_limit)) {
        atomicExch(&c.sync->abort, 1u);
        atomicOr(c.err, kErrTimeout);
        go = 0;
        break;
      }
      __nanosleep(128);
    }
    __threadfence();
    *s_go = go;
  }
  __syncthreads();
  return *s_go != 0;
}

// Copy a 16-byte-multiple object to shared memory with the whole CTA (no barrier).
template <typename T>
__device__ __forceinline__ void cta_copy(T* dst, const T* src) {
  static_assert(sizeof(T) % 16 == 0, "16-byte multiple");
  const int4* s4 = reinterpret_cast<const int4*>(src);
  int4* d4 = reinterpret_cast<int4*>(dst);
  for (int i = threadIdx.x; i < (int)(sizeof(T) / 16); i += blockDim.x) d4[i] = s4[i];
}

// Next tile of pass i for this CTA (tickets in tile order, so tiles are taken in the order
// the hardware would dispatch one CTA per tile, and a CTA that finishes early takes more);
// a value >= n_tiles ends the pass.  Synchronises the CTA.
__device__ __forceinline__ int next_tile(const PersistCtl& c, int i, int* s_tile) {
  if (threadIdx.x == 0) *s_tile = (int)atomicAdd(&c.tickets[i], 1u);
  __syncthreads();
  return *s_tile;
}

// Forward-kind passes plan[0..n_pass), all of pass mode MODE (the launcher splits runs at
// mode changes, so each interpreter compiles one pass body, as the one-launch-per-pass kernel
// does), tiles handed out by tickets.
template <int D, int MAT, int MODE, bool DET>
__global__ void __launch_bounds__(kTile, step_ctas_per_sm<D, MAT>())
    step_persistent_kernel(const PassEntry* plan, int n_pass, int n_tiles, PersistCtl ctl) {
  extern __shared__ __align__(16) float sm[];
  __shared__ int s_box[8 * kBoxSlots];
  __shared__ int s_bbox[8];
  __shared__ int s_go, s_tile;
  __shared__ PassEntry e;
  __shared__ Buckets s_bk;
  buckets_zero(s_bk);  // ordered before its first use by the barriers that follow
  // a barrier of an earlier launch of this sequence gave up: its passes never finished, so
  // this launch would only run on an incomplete state
  if (*(volatile unsigned*)ctl.err & kErrTimeout) return;
  for (int i = 0; i < n_pass; ++i) {
    if (i > 0 && !grid_barrier(ctl, (unsigned)i * gridDim.x + ctl.extra, &s_go)) return;
    __syncthreads();
    cta_copy(&e, plan + i);
    for (int t; (t = next_tile(ctl, i, &s_tile)) < n_tiles;) {
      step_tile<D, MAT, MODE, false, DET>(e.P, e.S, t, sm, s_box, s_bbox, s_bk);
      __syncthreads();
    }
  }
}

// Adjoint-kind passes plan[0..n_pass), all of mode MODE.
template <int D, int MAT, int MODE, bool DET>
__global__ void __launch_bounds__(kTile, MPM_ADJ_CTAS_PER_SM)
    adjoint_persistent_kernel(const PassEntry* plan, int n_pass, int n_tiles, PersistCtl ctl) {
  extern __shared__ __align__(16) float sm[];
  __shared__ int s_box[8 * kBoxSlots];
  __shared__ int s_bbox_ub[8];
  __shared__ int s_bbox_pm[8];
  __shared__ float s_wbar[kWbarSlots];
  __shared__ int s_go, s_tile;
  __shared__ PassEntry e;
  __shared__ Buckets s_bk;
  buckets_zero(s_bk);  // ordered before its first use by the barriers that follow
  // a barrier of an earlier launch of this sequence gave up: its passes never finished, so
  // this launch would only run on an incomplete state
  if (*(volatile unsigned*)ctl.err & kErrTimeout) return;
  for (int i = 0; i < n_pass; ++i) {
    if (i > 0 && !grid_barrier(ctl, (unsigned)i * gridDim.x + ctl.extra, &s_go)) return;
    __syncthreads();
    cta_copy(&e, plan + i);
    for (int t; (t = next_tile(ctl, i, &s_tile)) < n_tiles;) {
      adjoint_tile<D, MAT, MODE, false, DET>(e.P, e.A, t, sm, s_box, s_bbox_ub, s_bbox_pm, s_wbar, s_bk);
      __syncthreads();
    }
  }
}

// Zero the dirty boxes of the clear jobs (end of a launch sequence); blockIdx.y = scene.
template <int D>
__global__ void clear_kernel(const __grid_constant__ Clears C, int nnodes, int n) {
  run_clears<D>(C, blockIdx.y, blockIdx.x, gridDim.x, nnodes, n);
}

}  // namespace mpm
