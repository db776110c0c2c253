// mpm_common.cuh -- per-particle device math of the MLS-MPM step and its adjoint.
//
// Quadratic B-spline stencil, Kirchhoff stress (fixed-corotated / neo-Hookean,
// plus the actuation fibre stress of diffmpm's open-loop controller, Section 4.1),
// the stress adjoint, and the polar decomposition with its adjoint (the hand-written
// SVD/polar gradient of Appendix C).  Bulk arithmetic is FP32; the polar factor R and F - R
// are resolved to ~1e-14 in compensated FP32; the polar adjoint is FP32.
//
// The deformation gradient is carried as E = F - I: an FP32 F close to a rotation-free
// identity keeps only ~1e-7/|strain| relative precision on the strain, E keeps 1e-7.
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>

namespace mpm {

// Build-time launch shape (defaults measured on GB300): particles (= threads) per CTA of
// the particle passes, and the CTAs per SM each pass is compiled to fit (register cap).
// 128-particle tiles: measured 5-14% faster fwd+bwd than 256 (cube3d, robots3d, rects2d)
// at the same register budget (80 per thread in the forward passes); the adjoint at 5 CTAs
// per SM (96 registers) measured 1-6% faster than at 4 (128 registers).
#ifndef MPM_TILE
#define MPM_TILE 128
#endif
// 3D forward passes: 7 CTAs per SM (72 registers, a few spills; 2,048 cube3d tiles then run in
// 1.9 waves instead of 2.25) measured 3% faster than 6 for neo-Hookean, and 2% faster for the
// fixed-corotated passes once their polar refinement left the FP64 pipe
#ifndef MPM_STEP_CTAS_PER_SM_3D
#define MPM_STEP_CTAS_PER_SM_3D (896 / MPM_TILE)
#endif
#ifndef MPM_STEP_CTAS_PER_SM_3D_POLAR
#define MPM_STEP_CTAS_PER_SM_3D_POLAR (896 / MPM_TILE)
#endif
#ifndef MPM_STEP_CTAS_PER_SM_2D
#define MPM_STEP_CTAS_PER_SM_2D (1024 / MPM_TILE)
#endif
// Precision of the fixed-corotated polar factor's refinement and adjoint: 0 (default) =
// compensated FP32 refinement (R to ~1e-14) and an FP32 adjoint; 1 = both in FP64 (a build
// variant, `build(polar_fp64=True)`, kept to compare against and for users who want the FP64
// forms; ~3x slower on this part, whose FP64 pipe runs at 1/64 of the FP32 rate)
#ifndef MPM_POLAR_FP64
#define MPM_POLAR_FP64 0
#endif
#ifndef MPM_ADJ_CTAS_PER_SM
#define MPM_ADJ_CTAS_PER_SM (640 / MPM_TILE)  // 96 registers: a few spills, 25% more warps
#endif
constexpr int kTile = MPM_TILE;   // particles (= threads) per CTA in particle passes
static_assert(kTile % 32 == 0 && kTile >= 64 && kTile <= 1024, "tile must be whole warps");
constexpr int kMaxBasis = 8;
constexpr int kMaxGroups = 8;
// closed-loop controller (mpm_scene_desc.ctrl_hidden > 0): hidden units, and inputs
// (time basis, then per group the centre offset and mean velocity)
constexpr int kCtrlMaxHidden = 64;
constexpr int kCtrlMaxInputs = kMaxBasis + 2 * 3 * kMaxGroups;

// what the controller kernels of one step need (passed by value)
struct CtrlStep {
  int dim, G, K, H;   // dimension, groups, time-basis inputs, hidden units
  float scale;        // output scale: a_g = scale tanh(.)
  double basis[kMaxBasis];  // sin(2 pi k t / P + phi), k = 1..K, at this step
};

// device error bits (sticky, OR-ed into the handle's error word)
constexpr unsigned kErrOOB = 1u;
constexpr unsigned kErrNonFinite = 2u;
constexpr unsigned kErrTimeout = 4u;
constexpr unsigned kErrRange = 8u;  // a fixed-point grid contribution left its range

// kMixed: each particle carries one of the other three (a solid and a liquid coupled
// through one grid)
enum Material : int { kFixedCorotated = 0, kNeoHookean = 1, kLiquid = 3, kMixed = 4 };
// weakly compressible liquid (Tait form of the model the paper's liquid simulator follows,
// Tampubolon et al. 2017): tau = kappa (J - J^(1-g)) I, kappa = la + 2 mu / d, g = 7
constexpr float kLiquidGamma = 7.0f;

// Scalars every kernel of one launch needs (passed by value).
struct SimParams {
  int n_grid;
  int nnodes;        // n_grid^dim, nodes per scene grid
  float dx, inv_dx, dt;
  float gravity[3];
  int wall;
  float p_mass;      // rho * (dx/2)^dim
  float kappa;       // -dt * V0 * 4 / dx^2 (stress term of the affine matrix)
  int n_groups, n_basis;
  float basis[kMaxBasis];  // sin(2 pi k t / P + phi), k = 1..n_basis, at this pass's step
  float basis2[kMaxBasis]; // same at the step of an adjoint pass's recomputed P2G
  int tile_capacity;       // max nodes of a CTA's shared scatter box (0 = global reductions)
  int gather_capacity;     // max nodes of a CTA's shared gather box (0 = gathers through L1)
  int bucket;              // 1: FP32 scatters go through the per-base bucket table (one
                           // reduction per base and node); 0: one per particle and node
  int xfix;                // 1: the state's x rows hold positions in 32-bit fixed point
                           // (the float bits are the int32 x * 2^31), 0: FP32 positions
  int pair;                // FP32 reductions straight to the grid merge pairs of particles
                           // that share a stencil base (one per pair and node): bit 0 in
                           // the forward passes, bit 1 in the adjoint passes
  float f_diag;            // the F rows of the state hold F - f_diag I (0: E = F - I, 1: F)
  // deterministic accumulation: grids hold 64-bit fixed-point sums (node_words = 2 float4
  // slots per node), channel c of a contribution v enters as round(v * fix_c); mass uses
  // fix_m, momentum fix_p (the velocity adjoint's scale is set per backward on the device)
  int det;
  int node_words;          // float4 slots per grid node: 1 (FP32 sums) or 2 (fixed point)
  float fix_m, fix_p, unfix_m, unfix_p;
};

// ---------------------------------------------------------------------------
// 64-bit fixed-point grid nodes (deterministic mode).  Integer addition is associative,
// so the node sums, and everything computed from them, do not depend on the order in
// which particles add their contributions.  A contribution is rounded once,
// round(v * 2^e); a contribution beyond 2^55 (so that 256 of them cannot overflow the
// 64-bit sum) is refused and flagged instead.
// ---------------------------------------------------------------------------
constexpr float kFixLimit = 36028797018963968.0f;  // 2^55

// bit and conversion primitives of the fixed-point helpers below, with host versions so
// that those helpers can be checked on the host
__host__ __device__ __forceinline__ unsigned fx_float_bits(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  unsigned u;
  memcpy(&u, &f, 4);
  return u;
#endif
}
__host__ __device__ __forceinline__ float fx_bits_float(unsigned u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  memcpy(&f, &u, 4);
  return f;
#endif
}
__host__ __device__ __forceinline__ int fx_f2i_rn(float f) {  // |f| < 2^31, ties to even
#ifdef __CUDA_ARCH__
  return __float2int_rn(f);
#else
  return (int)nearbyintf(f);
#endif
}
__host__ __device__ __forceinline__ float fx_u2f_rn(unsigned u) {
#ifdef __CUDA_ARCH__
  return __uint2float_rn(u);
#else
  return (float)u;
#endif
}
__host__ __device__ __forceinline__ int fx_clzll(unsigned long long u) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)u);
#else
  return u ? __builtin_clzll(u) : 64;
#endif
}

// round(c) as a 64-bit integer for |c| <= 2^55, equal to __float2ll_rn(c) but without the
// 64-bit conversion, which issues on the FP64 pipe (1/64 of the FP32 rate here): below 2^23
// the 32-bit conversion rounds; from 2^23 on a float is an integer, its mantissa shifted by
// its exponent
__host__ __device__ __forceinline__ long long fix_round(float c) {
  if (fabsf(c) < 8388608.0f) return (long long)fx_f2i_rn(c);
  const unsigned b = fx_float_bits(c);
  const int sh = (int)((b >> 23) & 0xFFu) - 150;  // 0 <= sh <= 32 for 2^23 <= |c| <= 2^55
  const long long m = (long long)((b & 0x7FFFFFu) | 0x800000u) << sh;
  return (b >> 31) ? -m : m;
}

// channels 0..nch-1 of v into the fixed-point node `node` of grid g (two float4 slots
// per node); channel 0 is scaled by f0, the others by f1
__device__ __forceinline__ void fix_red(float4* g, int64_t node, float4 v, float f0, float f1,
                                        int nch, unsigned& err) {
  unsigned long long* q = reinterpret_cast<unsigned long long*>(g + 2 * node);
  const float c[4] = {v.x * f0, v.y * f1, v.z * f1, v.w * f1};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (k >= nch || c[k] == 0.0f) continue;
    if (!(fabsf(c[k]) <= kFixLimit)) {
      err |= kErrRange;
      continue;
    }
    atomicAdd(q + k, (unsigned long long)fix_round(c[k]));
  }
}

// a 64-bit integer rounded to the nearest float (ties to even) with 32-bit integer and
// conversion instructions only (the 64-bit conversion issues on the FP64 pipe)
__host__ __device__ __forceinline__ float ll_to_float_rn(long long a) {
  const bool neg = a < 0;
  const unsigned long long u = neg ? 0ull - (unsigned long long)a : (unsigned long long)a;
  if (u < (1ull << 24)) {
    const float f = fx_u2f_rn((unsigned)u);  // exact
    return neg ? -f : f;
  }
  const int sh = 40 - fx_clzll(u);  // bits below a 24-bit mantissa, 1..40
  unsigned long long m = u >> sh;
  const unsigned long long rem = u & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
  if (rem > half || (rem == half && (m & 1ull))) ++m;  // may reach 2^24: still exact below
  const float f = fx_u2f_rn((unsigned)m) * fx_bits_float((unsigned)(127 + sh) << 23);
  return neg ? -f : f;
}

// the fixed-point node as floats: channel 0 times u0, the others times u1 (powers of two,
// so each product is exact and the node value is rounded once, in ll_to_float_rn)
template <bool NC>
__device__ __forceinline__ float4 fix_load(const float4* g, int64_t node, float u0, float u1) {
  const longlong2* q = reinterpret_cast<const longlong2*>(g + 2 * node);
  longlong2 a, b;
  if (NC) {
    a = __ldg(q);
    b = __ldg(q + 1);
  } else {
    a = q[0];
    b = q[1];
  }
  return make_float4(ll_to_float_rn(a.x) * u0, ll_to_float_rn(a.y) * u1, ll_to_float_rn(b.x) * u1,
                     ll_to_float_rn(b.y) * u1);
}

// scale pair of the velocity-adjoint grids of one backward from the largest contribution
// bound m0 of its first scatter: m0 maps to below 2^36, leaving 2^19 of growth before the
// 2^55 limit and 2^-36 m0 resolution
__device__ __forceinline__ void fix_scales_from(float m0, float& fix, float& unfix) {
  int k = 0;
  if (m0 > 0.0f && m0 <= 3.0e38f) {
    k = 36 - (ilogbf(m0) + 1);
    k = k > 120 ? 120 : (k < -120 ? -120 : k);
  }
  fix = ldexpf(1.0f, k);
  unfix = ldexpf(1.0f, -k);
}

// ---------------------------------------------------------------------------
// Fixed-point positions.  An FP32 position in [0, 1) carries ~6e-8 of absolute precision,
// and rounding it at every step is what bounds the accuracy of long runs: emulated in the
// FP64 oracle on a 4,096-particle cube over 1,024 steps, rounding x alone to FP32 after each
// step moves dL/dmu by 7.4e-4 and dL/dF0 by 1.5e-4 (relative L2), while 32-bit fixed point
// (resolution 2^-31 = 4.7e-10) moves them by 1.6e-5 and 5e-7 -- at the same 4 bytes.  The
// state's x rows therefore hold int32(x * 2^31) in their float bits; the stencil base and
// fraction are formed exactly from the integer, and the step's advance x += dt v adds the
// rounded increment in integer arithmetic.  A particle that leaves [-1, 1) saturates (it left
// the grid long before, and its stencil check reports it).
// ---------------------------------------------------------------------------
constexpr float kFixPos = 2147483648.0f;              // 2^31
constexpr double kFixPosInv = 4.656612873077392578e-10;  // 2^-31

__device__ __forceinline__ int fix_saturate(long long v) {
  return v > 2147483647LL ? 2147483647 : (v < -2147483648LL ? (int)(-2147483647 - 1) : (int)v);
}
// FP32 position -> fixed-point bits
__device__ __forceinline__ float pos_to_fix(float x) {
  return __int_as_float(fix_saturate(__float2ll_rn(x * kFixPos)));
}
// fixed-point bits -> position (FP64 is exact; FP32 rounds to the nearest float)
__device__ __forceinline__ double pos_from_fix(float raw) {
  return (double)__float_as_int(raw) * kFixPosInv;
}
// x + delta on fixed-point bits (delta rounded once to the 2^-31 grid).  A step moves a
// particle by less than the unit domain, so delta * 2^31 fits 32 bits and converts without
// the 64-bit conversion (which issues on the FP64 pipe); a larger delta saturates, and that
// particle has left the grid anyway (the stencil check reports it).
__device__ __forceinline__ float pos_advance(float raw, float delta) {
  return __int_as_float(fix_saturate((long long)__float_as_int(raw) + (long long)__float2int_rn(delta * kFixPos)));
}

// ---------------------------------------------------------------------------
// quadratic B-spline stencil (MLS-MPM, Hu et al. 2018), kept per axis: the weight of
// node base + (i, j, k) is w[0][i] w[1][j] w[2][k] and dpos = (dp[0][i], dp[1][j], dp[2][k])
// ---------------------------------------------------------------------------
template <int D>
struct Axes {
  int base[D];
  float f[D];      // x/dx - base in [0.5, 1.5)
  float w[D][3];
  float dw[D][3];  // dw/df
  float dp[D][3];  // (o - f) dx
};

// Returns false (and leaves a harmless in-range base) when the stencil would leave
// [0, n-1] or x is not finite; such a particle must not touch the grid.
template <int D>
__device__ __forceinline__ bool make_axes(const float* x, const SimParams& P, Axes<D>& s) {
  bool ok = true;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    float b, f;
    bool good;
    if (P.xfix) {
      // X = x / dx with 31 fractional bits, exact in 64-bit integers
      const long long X = (long long)__float_as_int(x[a]) * (long long)P.n_grid;
      const long long bi = (X - (1LL << 30)) >> 31;  // floor(X - 0.5)
      good = bi >= 0 && bi <= (long long)(P.n_grid - 3);
      // a 32-bit conversion (0 <= bi <= n_grid - 3): the 64-bit one issues on the FP64 pipe
      // (measured 0.3-0.6% faster passes on cube3d, rects2d and robots3d)
      b = good ? (float)(int)bi : 0.0f;
      // the fraction X - base in [0.5, 1.5): below 2^32 in units of 2^-31 (FP32 rounds it once)
      f = good ? __uint2float_rn((unsigned)(X - (bi << 31))) * (1.0f / kFixPos) : 1.0f;
    } else {
      const float Xf = x[a] * P.inv_dx;
      b = floorf(Xf - 0.5f);
      good = (Xf == Xf) && b >= 0.0f && b <= (float)(P.n_grid - 3);
      b = good ? b : 0.0f;
      f = good ? Xf - b : 1.0f;
    }
    ok = ok && good;
    s.base[a] = (int)b;
    s.f[a] = f;
    float r0 = 1.5f - f, r1 = f - 1.0f, r2 = f - 0.5f;
    s.w[a][0] = 0.5f * r0 * r0;
    s.w[a][1] = 0.75f - r1 * r1;
    s.w[a][2] = 0.5f * r2 * r2;
    s.dw[a][0] = -r0;
    s.dw[a][1] = -2.0f * r1;
    s.dw[a][2] = r2;
    s.dp[a][0] = -f * P.dx;
    s.dp[a][1] = (1.0f - f) * P.dx;
    s.dp[a][2] = (2.0f - f) * P.dx;
  }
  return ok;
}

// weights only, from f (used by scatters that receive f from another thread)
template <int D>
__device__ __forceinline__ void axes_from_f(const float f[D], const SimParams& P, float w[D][3],
                                            float dp[D][3]) {
#pragma unroll
  for (int a = 0; a < D; ++a) {
    float r0 = 1.5f - f[a], r1 = f[a] - 1.0f, r2 = f[a] - 0.5f;
    w[a][0] = 0.5f * r0 * r0;
    w[a][1] = 0.75f - r1 * r1;
    w[a][2] = 0.5f * r2 * r2;
    dp[a][0] = -f[a] * P.dx;
    dp[a][1] = (1.0f - f[a]) * P.dx;
    dp[a][2] = (2.0f - f[a]) * P.dx;
  }
}

// ---------------------------------------------------------------------------
// small matrix helpers (row-major D x D)
// ---------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ void cofactor(const float A[D][D], float c[D][D]) {
  if (D == 2) {
    c[0][0] = A[1][1];
    c[0][1] = -A[1][0];
    c[1][0] = -A[0][1];
    c[1][1] = A[0][0];
  } else {
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = 0; j < D; ++j) {
        const int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
        c[i][j] = A[i1][j1] * A[i2][j2] - A[i1][j2] * A[i2][j1];
      }
  }
}

// J - 1 for F = I + E, summed by invariants (trace, principal minors, det E) so that it
// keeps its relative accuracy when F is close to the identity.
template <int D>
__device__ __forceinline__ float det_minus_one(const float E[D][D]) {
  if (D == 2) {
    return E[0][0] + E[1][1] + (E[0][0] * E[1][1] - E[0][1] * E[1][0]);
  } else {
    float m2 = (E[0][0] * E[1][1] - E[0][1] * E[1][0]) + (E[0][0] * E[2][2] - E[0][2] * E[2][0]) +
               (E[1][1] * E[2][2] - E[1][2] * E[2][1]);
    float d3 = E[0][0] * (E[1][1] * E[2][2] - E[1][2] * E[2][1]) -
               E[0][1] * (E[1][0] * E[2][2] - E[1][2] * E[2][0]) +
               E[0][2] * (E[1][0] * E[2][1] - E[1][1] * E[2][0]);
    return (E[0][0] + E[1][1] + E[2][2]) + m2 + d3;
  }
}

template <int D>
__device__ __forceinline__ void plus_identity(const float E[D][D], float F[D][D]) {
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) F[i][j] = E[i][j] + (i == j ? 1.0f : 0.0f);
}

// ---------------------------------------------------------------------------
// Polar decomposition F = R S (R in SO(d), S symmetric positive definite)
// ---------------------------------------------------------------------------
template <int D>
struct Polar {
  float Rh[D][D], Rl[D][D];  // R = Rh + Rl to ~1e-14 (the per-segment cache stores both)
  float Rf[D][D];            // R rounded to FP32
  float Df[D][D];            // F - R formed from the exact parts, rounded once
};

// 3x3 cofactor matrix (c[i][j] = cofactor of X[i][j]; X^-T = c / det X)
template <typename T>
__host__ __device__ __forceinline__ void cofactor3(const T X[3][3], T c[3][3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
      c[i][j] = X[i1][j1] * X[i2][j2] - X[i1][j2] * X[i2][j1];
    }
}

// Newton's iteration X <- (X + X^-T)/2 (Higham 1986) in precision T from X = F: converges
// quadratically to the orthogonal polar factor and keeps det X > 0.  Stops once the
// squared update norm is below `tol`; false for det <= 0, overflow or no convergence.
template <typename T>
__host__ __device__ __forceinline__ bool polar_newton3(T X[3][3], T tol, int max_it) {
  for (int it = 0; it < max_it; ++it) {
    T c[3][3];
    cofactor3<T>(X, c);
    const T det = X[0][0] * c[0][0] + X[0][1] * c[0][1] + X[0][2] * c[0][2];
    if (!(det > T(0)) || !(det < T(1e30))) return false;
    const T hid = T(0.5) / det;
    T diff = T(0);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const T xn = T(0.5) * X[i][j] + c[i][j] * hid;
        const T dd = xn - X[i][j];
        diff += dd * dd;
        X[i][j] = xn;
      }
    if (diff < tol) return true;
  }
  return false;
}

#if MPM_POLAR_FP64
// One Newton-Schulz step toward the nearest orthogonal matrix, Q <- Q (3I - Q^T Q)/2, in
// FP64 (quadratic: an orthogonality error e becomes ~e^2)
__device__ __forceinline__ void orthonormalize_step(double Q[3][3]) {
  double G[3][3];  // symmetric: six entries
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      double g = 0.0;
#pragma unroll
      for (int k = 0; k < 3; ++k) g += Q[k][i] * Q[k][j];
      G[i][j] = G[j][i] = 0.5 * ((i == j ? 3.0 : 0.0) - g);
    }
  double Qn[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double q = 0.0;
#pragma unroll
      for (int k = 0; k < 3; ++k) q += Q[i][k] * G[k][j];
      Qn[i][j] = q;
    }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) Q[i][j] = Qn[i][j];
}
#endif

// Error-free transformations in FP32: a + b = s + e exactly (Knuth's TwoSum) and
// a * b = p + e exactly (the fused multiply-add gives the product's rounding error).  The
// _rn intrinsics keep the compiler from fusing or reordering these operations.
__host__ __device__ __forceinline__ float ef_add(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
__host__ __device__ __forceinline__ float ef_mul(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
__host__ __device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = ef_add(a, b);
  const float bb = ef_add(s, -a);
  e = ef_add(ef_add(a, -ef_add(s, -bb)), ef_add(b, -bb));
}
// acc.x + acc.y += v: the rounding error of the sum goes to the correction term (a
// compensated sum: over n terms its error is ~n ulp^2 of the total, FP64-like for n ~ 1e3)
__host__ __device__ __forceinline__ void compensated_add(float2& acc, float v) {
  float s, e;
  two_sum(acc.x, v, s, e);
  acc.x = s;
  acc.y += e;
}
__host__ __device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = ef_mul(a, b);
  e = fmaf(a, b, -p);
}

// (delta + e) - (rh + rl) rounded once: delta + e = fh + fl and fh - rh = g + ge exactly
__host__ __device__ __forceinline__ float f_minus_r(float delta, float e, float rh, float rl) {
  float fh, fl, g, ge;
  two_sum(delta, e, fh, fl);
  two_sum(fh, -rh, g, ge);
  return g + ((ge + fl) - rl);
}

// 2D polar factor R = [[c, -s], [s, c]] / r, c = F00 + F11, s = F10 - F01, r = |(c, s)|,
// without FP64 arithmetic: c, s, c^2 + s^2, r and 1/r are carried as value + correction pairs
// (exact sums and products; one correction of the FP32 square root from its exact residual,
// and of the FP32 reciprocal from r0 i0 - 1, exact in one fused multiply-add), so cos = c / r
// and sin = s / r are resolved to ~1e-14 and F - R is formed from the exact parts.  Returns
// false (R = I) for det F <= 0 or a degenerate (c, s).
__host__ __device__ __forceinline__ bool polar_refine2(const float E[2][2], float Rh[2][2], float Rl[2][2],
                                                       float Df[2][2]) {
  float ch, cl, sh, sl;
  {
    float t, e1, e2;
    two_sum(2.0f, E[0][0], t, e1);
    two_sum(t, E[1][1], ch, e2);
    cl = e1 + e2;
  }
  two_sum(E[1][0], -E[0][1], sh, sl);
  float p1, e1, p2, e2, qh, e3;
  two_prod(ch, ch, p1, e1);
  two_prod(sh, sh, p2, e2);
  two_sum(p1, p2, qh, e3);
  const float ql = e1 + e2 + e3 + 2.0f * (ch * cl + sh * sl);
  const float det = (1.0f + E[0][0]) * (1.0f + E[1][1]) - E[0][1] * E[1][0];
  if (!(det > 0.0f) || !(qh > 1e-30f) || !(qh < 1e30f)) {
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        Rh[i][j] = i == j ? 1.0f : 0.0f;
        Rl[i][j] = 0.0f;
        Df[i][j] = E[i][j];
      }
    return false;
  }
  const float r0 = sqrtf(qh);
  float pp, ee;
  two_prod(r0, r0, pp, ee);
  const float rl = ((ef_add(qh, -pp) - ee) + ql) / (2.0f * r0);  // r = r0 + rl
  const float i0 = 1.0f / r0;
  const float ie = fmaf(r0, i0, -1.0f);                           // r0 i0 - 1, exact
  const float il = -i0 * (ie + rl * i0);                          // 1 / r = i0 + il
  float ah, al, bh, bl;
  two_prod(ch, i0, ah, al);
  al += ch * il + cl * i0;
  two_prod(sh, i0, bh, bl);
  bl += sh * il + sl * i0;
  Rh[0][0] = Rh[1][1] = ah;
  Rl[0][0] = Rl[1][1] = al;
  Rh[1][0] = bh;
  Rl[1][0] = bl;
  Rh[0][1] = -bh;
  Rl[0][1] = -bl;
  Df[0][0] = f_minus_r(1.0f, E[0][0], ah, al);
  Df[1][1] = f_minus_r(1.0f, E[1][1], ah, al);
  Df[1][0] = f_minus_r(0.0f, E[1][0], bh, bl);
  Df[0][1] = f_minus_r(0.0f, E[0][1], -bh, -bl);
  return true;
}

// 3D polar factor refined from an FP32 one without FP64 arithmetic (the FP64 pipe runs at
// 1/64 of the FP32 rate on this part).  Q is Newton's FP32 iterate, orthogonal and equal to R
// to within FP32 resolution (~1e-7), so every correction below is of that size and needs only
// FP32 relative precision, provided the quantities it is formed from are exact to ~1e-14:
//  1. orthonormalise: X = Q (3I - Q^T Q)/2 = Q + Q H, H = (I - Q^T Q)/2, with Q^T Q summed
//     from exact products and sums (its deviation from I is the small part);
//  2. M = X^T F = X^T + X^T E, again from exact products and sums, as a value and a
//     correction (M_hi, M_lo);
//  3. the small rotation X^T R = exp(W) that makes X^T F symmetric solves
//     (tr(S) I - S) w = (M32 - M23, M13 - M31, M21 - M12) for the axial vector w of W
//     (S = sym(M); eigenvalues sigma_i + sigma_j > 0): an FP32 solve, |w| ~ 1e-7;
//  4. R = X (I + W) = Q + (Q H + Q W) to first order (the dropped terms are ~|w|^2, 1e-14):
//     kept as R_hi = Q and R_lo = Q (H + W);
//  5. F - R = (I + E) - (R_hi + R_lo) with exact sums, rounded once.
// R = R_hi + R_lo agrees with an FP64 polar decomposition to ~1e-14 (checked against an
// SVD on random F with strains up to 0.6), far below what the FP32 stress resolves.
// Returns false when the solve of step 3 is singular (then the caller falls back).
__host__ __device__ __forceinline__ bool polar_refine3(const float E[3][3], const float Q[3][3],
                                                       float Rh[3][3], float Rl[3][3], float Df[3][3]) {
  float H[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      float sh = 0.0f, sl = 0.0f;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        float pk, ek, t, et;
        two_prod(Q[k][i], Q[k][j], pk, ek);
        two_sum(sh, pk, t, et);
        sh = t;
        sl += ek + et;
      }
      // 1 - sh is exact (sh within 1e-6 of 1), 0 - sh trivially
      H[i][j] = H[j][i] = 0.5f * (ef_add(i == j ? 1.0f : 0.0f, -sh) - sl);
    }
  float Xl[3][3];  // X = Q + Xl, Xl = Q H
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) Xl[i][j] = Q[i][0] * H[0][j] + Q[i][1] * H[1][j] + Q[i][2] * H[2][j];
  float Mh[3][3], Ml[3][3];  // M = X^T (I + E)
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      float sh = Q[j][i], sl = Xl[j][i];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        float pk, ek, t, et;
        two_prod(Q[k][i], E[k][j], pk, ek);
        two_sum(sh, pk, t, et);
        sh = t;
        sl += ek + et + Xl[k][i] * E[k][j];
      }
      Mh[i][j] = sh;
      Ml[i][j] = sl;
    }
  // right-hand side: the skew part of M (the hi differences are exact or carry only a
  // relative rounding of their own result)
  const float b0 = ef_add(Mh[2][1], -Mh[1][2]) + (Ml[2][1] - Ml[1][2]);
  const float b1 = ef_add(Mh[0][2], -Mh[2][0]) + (Ml[0][2] - Ml[2][0]);
  const float b2 = ef_add(Mh[1][0], -Mh[0][1]) + (Ml[1][0] - Ml[0][1]);
  const float tr = Mh[0][0] + Mh[1][1] + Mh[2][2];
  float A[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) A[i][j] = (i == j ? tr : 0.0f) - 0.5f * (Mh[i][j] + Mh[j][i]);
  float c[3][3];
  cofactor3<float>(A, c);
  const float det = A[0][0] * c[0][0] + A[0][1] * c[0][1] + A[0][2] * c[0][2];
  if (!(det > 1e-30f) || !(det < 1e30f)) return false;
  const float id = 1.0f / det;
  const float w0 = (c[0][0] * b0 + c[1][0] * b1 + c[2][0] * b2) * id;
  const float w1 = (c[0][1] * b0 + c[1][1] * b1 + c[2][1] * b2) * id;
  const float w2 = (c[0][2] * b0 + c[1][2] * b1 + c[2][2] * b2) * id;
  // H + W, W = [[0, -w2, w1], [w2, 0, -w0], [-w1, w0, 0]]
  const float K[3][3] = {{H[0][0], H[0][1] - w2, H[0][2] + w1},
                         {H[1][0] + w2, H[1][1], H[1][2] - w0},
                         {H[2][0] - w1, H[2][1] + w0, H[2][2]}};
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Rh[i][j] = Q[i][j];
      Rl[i][j] = Q[i][0] * K[0][j] + Q[i][1] * K[1][j] + Q[i][2] * K[2][j];
      Df[i][j] = f_minus_r(i == j ? 1.0f : 0.0f, E[i][j], Rh[i][j], Rl[i][j]);
    }
  return true;
}

// 2D: R is the rotation by atan2(F10 - F01, F00 + F11), formed without a transcendental
// as (c, s) / |(c, s)| in compensated FP32 (polar_refine2).
// 3D: Newton's iteration in FP32 gives Q within FP32 resolution of R, refined without FP64
// arithmetic (polar_refine3) to R = R_hi + R_lo and F - R; R in FP64 is formed from the pair
// only where a pass needs it (the polar adjoint, the per-segment cache).  When the FP32 stage
// fails (near-singular F) Newton's iteration runs in FP64 from F.
// Returns false for det F <= 0 or non-finite input.
template <int D>
__device__ __forceinline__ bool polar_factor(const float E[D][D], Polar<D>& p) {
  double Fd[D][D];  // F = I + E, exact in FP64
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) Fd[i][j] = (double)E[i][j] + (i == j ? 1.0 : 0.0);
  if constexpr (D == 2) {
#if !MPM_POLAR_FP64
    const bool ok = polar_refine2(E, p.Rh, p.Rl, p.Df);
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) p.Rf[i][j] = p.Rh[i][j] + p.Rl[i][j];
    return ok;
#else
    double c = Fd[0][0] + Fd[1][1];
    double s = Fd[1][0] - Fd[0][1];
    double r = sqrt(c * c + s * s);
    double det = Fd[0][0] * Fd[1][1] - Fd[0][1] * Fd[1][0];
    if (!(det > 0.0) || !(r > 0.0)) {
      c = 1.0; s = 0.0; r = 1.0;
    }
    double ir = 1.0 / r;
    const double R[2][2] = {{c * ir, -s * ir}, {s * ir, c * ir}};
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = 0; j < D; ++j) {
        p.Rh[i][j] = p.Rf[i][j] = (float)R[i][j];
        p.Rl[i][j] = (float)(R[i][j] - (double)p.Rh[i][j]);
        p.Df[i][j] = (float)(Fd[i][j] - R[i][j]);
      }
    return det > 0.0 && r > 0.0;
#endif
  } else {
    float Xf[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) Xf[i][j] = E[i][j] + (i == j ? 1.0f : 0.0f);
    bool ok = polar_newton3<float>(Xf, 1e-12f, 20);
#if !MPM_POLAR_FP64
    if (ok) {
      ok = polar_refine3(E, Xf, p.Rh, p.Rl, p.Df);
      if (ok) {
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) p.Rf[i][j] = p.Rh[i][j] + p.Rl[i][j];
        return true;
      }
    }
    double X[3][3];
#else
    // FP64 refinement: orthonormalise Q (one Newton-Schulz step), then rotate it by the small
    // rotation that makes Q^T F symmetric, all in FP64
    double X[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) X[i][j] = (double)Xf[i][j];
    if (ok) {
      orthonormalize_step(X);
      double M[3][3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          double m = 0.0;
#pragma unroll
          for (int k = 0; k < 3; ++k) m += X[k][i] * Fd[k][j];
          M[i][j] = m;
        }
      const double tr = M[0][0] + M[1][1] + M[2][2];
      double A[3][3];  // tr(S) I - S, S = sym(M)
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) A[i][j] = (i == j ? tr : 0.0) - 0.5 * (M[i][j] + M[j][i]);
      const double b[3] = {M[2][1] - M[1][2], M[0][2] - M[2][0], M[1][0] - M[0][1]};
      double c[3][3];
      cofactor3<double>(A, c);
      const double det = A[0][0] * c[0][0] + A[0][1] * c[0][1] + A[0][2] * c[0][2];
      ok = det > 1e-30 && det < 1e30;
      if (ok) {
        // 1/det: FP32 reciprocal, two FP64 Newton steps (relative error ~1e-28 -> FP64 ulps)
        double id = (double)__frcp_rn((float)det);
        id = id * (2.0 - det * id);
        id = id * (2.0 - det * id);
        double w[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) w[i] = (c[0][i] * b[0] + c[1][i] * b[1] + c[2][i] * b[2]) * id;
        // G = I + W + W^2/2 with W the cross-product matrix of w (W^2 = w w^T - |w|^2 I)
        const double ww = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
        const double Wm[3][3] = {{0.0, -w[2], w[1]}, {w[2], 0.0, -w[0]}, {-w[1], w[0], 0.0}};
        double G[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j)
            G[i][j] = (i == j ? 1.0 - 0.5 * ww : 0.0) + Wm[i][j] + 0.5 * w[i] * w[j];
        double Rn[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            double r = 0.0;
#pragma unroll
            for (int k = 0; k < 3; ++k) r += X[i][k] * G[k][j];
            Rn[i][j] = r;
          }
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) X[i][j] = Rn[i][j];
      }
    }
#endif
    if (!ok) {
      // near-singular F: Newton's iteration in FP64 from F
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) X[i][j] = Fd[i][j];
      // stop when the next update would be below FP64 resolution
      ok = polar_newton3<double>(X, 1e-20, 24);
    }
    if (!ok) {
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) X[i][j] = (i == j) ? 1.0 : 0.0;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        p.Rh[i][j] = p.Rf[i][j] = (float)X[i][j];
        p.Rl[i][j] = (float)(X[i][j] - (double)p.Rh[i][j]);
        p.Df[i][j] = (float)(Fd[i][j] - X[i][j]);
      }
    return ok;
  }
}

// The per-segment polar cache holds R_hi and R_lo as FP32 rows [2 D^2][N] (rows i*D + j,
// then D^2 + i*D + j), in the footprint of [D^2][N] FP64 values; F - R is re-formed from them
// exactly as the factorisation forms it.
template <int D>
__device__ __forceinline__ void polar_from_cache(const double* Rc, int64_t N, int64_t p,
                                                 const float E[D][D], Polar<D>& pol) {
  const float* r = reinterpret_cast<const float*>(Rc);
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const float rh = r[(int64_t)(i * D + j) * N + p];
      const float rl = r[(int64_t)(D * D + i * D + j) * N + p];
      pol.Rh[i][j] = rh;
      pol.Rl[i][j] = rl;
      pol.Rf[i][j] = rh + rl;
      pol.Df[i][j] = f_minus_r(i == j ? 1.0f : 0.0f, E[i][j], rh, rl);
    }
}

template <int D>
__device__ __forceinline__ void polar_to_cache(double* Rc, int64_t N, int64_t p, const Polar<D>& pol) {
  float* r = reinterpret_cast<float*>(Rc);
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) {
      r[(int64_t)(i * D + j) * N + p] = pol.Rh[i][j];
      r[(int64_t)(D * D + i * D + j) * N + p] = pol.Rl[i][j];
    }
}

// Fbar += dR/dF^T [Rbar].  With F = R S, dR = R W (W antisymmetric) and
// W S + S W = R^T dF - dF^T R; the adjoint is Fbar += 2 R Y where Y is the
// antisymmetric solution of Y S + S Y = skew(R^T Rbar).  In 3D that equation is
// (tr(S) I - S) y = b on axial vectors (eigenvalues sigma_i + sigma_j > 0), in 2D
// y = b / tr(S); no singular-value differences appear.  It runs in FP32 on R rounded to
// FP32: Rbar is an FP32 value, so R^T Rbar carries its rounding whatever the precision of
// the product, and the solve is well conditioned (tr(S) I - S ~ 2 I at small strain).
#if !MPM_POLAR_FP64
template <int D>
__device__ __forceinline__ void polar_adjoint(const float E[D][D], const Polar<D>& p,
                                              const float Rbar[D][D], float Fbar[D][D]) {
  float M[D][D], S[D][D];
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) {
      float m = 0.0f, sv = 0.0f;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        m += p.Rf[k][i] * Rbar[k][j];
        sv += p.Rf[k][i] * (E[k][j] + (k == j ? 1.0f : 0.0f));
      }
      M[i][j] = m;
      S[i][j] = sv;
    }
  if constexpr (D == 2) {
    const float b = 0.5f * (M[1][0] - M[0][1]);
    const float tr = S[0][0] + S[1][1];
    const float y2 = 2.0f * b / fmaxf(tr, 1e-6f);
    // 2 R Y, Y = [[0, -y], [y, 0]]
    Fbar[0][0] += p.Rf[0][1] * y2;
    Fbar[0][1] -= p.Rf[0][0] * y2;
    Fbar[1][0] += p.Rf[1][1] * y2;
    Fbar[1][1] -= p.Rf[1][0] * y2;
  } else {
    const float b0 = 0.5f * (M[2][1] - M[1][2]);
    const float b1 = 0.5f * (M[0][2] - M[2][0]);
    const float b2 = 0.5f * (M[1][0] - M[0][1]);
    const float tr = S[0][0] + S[1][1] + S[2][2];
    // G = tr(S) I - sym(S)
    const float g00 = tr - S[0][0], g11 = tr - S[1][1], g22 = tr - S[2][2];
    const float g01 = -0.5f * (S[0][1] + S[1][0]);
    const float g02 = -0.5f * (S[0][2] + S[2][0]);
    const float g12 = -0.5f * (S[1][2] + S[2][1]);
    const float c00 = g11 * g22 - g12 * g12, c01 = g02 * g12 - g01 * g22, c02 = g01 * g12 - g02 * g11;
    const float c11 = g00 * g22 - g02 * g02, c12 = g01 * g02 - g00 * g12, c22 = g00 * g11 - g01 * g01;
    const float id = 2.0f / fmaxf(g00 * c00 + g01 * c01 + g02 * c02, 1e-30f);
    const float y0 = (c00 * b0 + c01 * b1 + c02 * b2) * id;  // 2y
    const float y1 = (c01 * b0 + c11 * b1 + c12 * b2) * id;
    const float y2 = (c02 * b0 + c12 * b1 + c22 * b2) * id;
    // (R Y)[i][j] with Y = [[0, -y2, y1], [y2, 0, -y0], [-y1, y0, 0]]
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      Fbar[i][0] += p.Rf[i][1] * y2 - p.Rf[i][2] * y1;
      Fbar[i][1] += p.Rf[i][2] * y0 - p.Rf[i][0] * y2;
      Fbar[i][2] += p.Rf[i][0] * y1 - p.Rf[i][1] * y0;
    }
  }
}
#else
// FP64 form: the products and the solve in FP64 on R = R_hi + R_lo
template <int D>
__device__ __forceinline__ void polar_adjoint(const float E[D][D], const Polar<D>& p,
                                                  const float Rbar[D][D], float Fbar[D][D]) {
  double Rd[D][D];
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) Rd[i][j] = (double)p.Rh[i][j] + (double)p.Rl[i][j];
  double M[D][D], S[D][D];
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) {
      double m = 0.0, s = 0.0;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        m += Rd[k][i] * (double)Rbar[k][j];
        s += Rd[k][i] * ((double)E[k][j] + (k == j ? 1.0 : 0.0));
      }
      M[i][j] = m;
      S[i][j] = s;
    }
  if constexpr (D == 2) {
    double b = 0.5 * (M[1][0] - M[0][1]);
    double tr = S[0][0] + S[1][1];
    double y = b / fmax(tr, 1e-6);
    // 2 R Y, Y = [[0, -y], [y, 0]]
    Fbar[0][0] += (float)(2.0 * Rd[0][1] * y);
    Fbar[0][1] += (float)(-2.0 * Rd[0][0] * y);
    Fbar[1][0] += (float)(2.0 * Rd[1][1] * y);
    Fbar[1][1] += (float)(-2.0 * Rd[1][0] * y);
  } else {
    double b0 = 0.5 * (M[2][1] - M[1][2]);
    double b1 = 0.5 * (M[0][2] - M[2][0]);
    double b2 = 0.5 * (M[1][0] - M[0][1]);
    double tr = S[0][0] + S[1][1] + S[2][2];
    // G = tr(S) I - sym(S)
    double g00 = tr - S[0][0], g11 = tr - S[1][1], g22 = tr - S[2][2];
    double g01 = -0.5 * (S[0][1] + S[1][0]);
    double g02 = -0.5 * (S[0][2] + S[2][0]);
    double g12 = -0.5 * (S[1][2] + S[2][1]);
    double c00 = g11 * g22 - g12 * g12, c01 = g02 * g12 - g01 * g22, c02 = g01 * g12 - g02 * g11;
    double c11 = g00 * g22 - g02 * g02, c12 = g01 * g02 - g00 * g12, c22 = g00 * g11 - g01 * g01;
    const double det = fmax(g00 * c00 + g01 * c01 + g02 * c02, 1e-18);
    // 1/det: FP32 reciprocal, two FP64 Newton steps (relative error ~1e-28 -> FP64 ulps);
    // a plain division beyond the FP32 seed's range
    double id;
    if (det < 1e30) {
      id = (double)__frcp_rn((float)det);
      id = id * (2.0 - det * id);
      id = id * (2.0 - det * id);
    } else {
      id = 1.0 / det;
    }
    // 2y, rounded once: the rotation 2 R Y below is well conditioned (|2 R Y| = 2|y|), so it
    // runs in FP32 on R rounded to FP32, with the error of the FP32 accumulation into Fbar
    const float y0 = (float)(2.0 * (c00 * b0 + c01 * b1 + c02 * b2) * id);
    const float y1 = (float)(2.0 * (c01 * b0 + c11 * b1 + c12 * b2) * id);
    const float y2 = (float)(2.0 * (c02 * b0 + c12 * b1 + c22 * b2) * id);
    // (R Y)[i][j] with Y = [[0, -y2, y1], [y2, 0, -y0], [-y1, y0, 0]]
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      Fbar[i][0] += p.Rf[i][1] * y2 - p.Rf[i][2] * y1;
      Fbar[i][1] += p.Rf[i][2] * y0 - p.Rf[i][0] * y2;
      Fbar[i][2] += p.Rf[i][0] * y1 - p.Rf[i][1] * y0;
    }
  }
}
#endif

// ---------------------------------------------------------------------------
// Kirchhoff stress tau(F) and its adjoint
// ---------------------------------------------------------------------------
template <int D>
struct StressCache {
  float J, Jm1;
  Polar<D> pol;  // fixed-corotated only
};

// tau = 2 mu (F - R) F^T + la (J - 1) J I        (fixed-corotated)
// tau = mu (F F^T - I) + la ln(J) I               (neo-Hookean)
// tau = kappa (J - J^(1-g)) I                     (liquid; no shear stress)
// row[axis] by selects: an array indexed with a runtime value would be placed in local
// memory (stores of the whole matrix on every stress evaluation)
template <int D>
__device__ __forceinline__ float column_of(const float row[D], int axis) {
  float v = row[0];
  if (axis == 1) v = row[1];
  if (D == 3 && axis == 2) v = row[D - 1];
  return v;
}

// tau += act (F e)(F e)^T, e = unit vector of `axis` (actuation fibre)
// with F = I + E; every product is formed on E (or on F - R) so small strains keep
// their relative precision.
// Rc (fixed-corotated only, may be null): the cached polar factor of this particle (R_hi and
// R_lo rows, particle p), used instead of recomputing it.
template <int D, int MAT>
__device__ __forceinline__ bool kirchhoff(const float E[D][D], float mu, float la, float act, int axis,
                                          float tau[D][D], StressCache<D>& sc,
                                          const double* Rc = nullptr, int64_t N = 0, int64_t p = 0,
                                          int mat_p = MAT) {
  if (MAT == kMixed) {  // the particle's own model (mat_p)
    if (mat_p == kFixedCorotated)
      return kirchhoff<D, kFixedCorotated>(E, mu, la, act, axis, tau, sc, Rc, N, p);
    if (mat_p == kNeoHookean) return kirchhoff<D, kNeoHookean>(E, mu, la, act, axis, tau, sc);
    return kirchhoff<D, kLiquid>(E, mu, la, act, axis, tau, sc);
  }
  bool ok = true;
  sc.Jm1 = det_minus_one<D>(E);
  sc.J = 1.0f + sc.Jm1;
  if (MAT == kFixedCorotated) {
    if (D == 3 && Rc) {  // the cache is kept for 3D only
      polar_from_cache<D>(Rc, N, p, E, sc.pol);
      ok = sc.J > 0.0f;
    } else {
      ok = polar_factor<D>(E, sc.pol);
    }
    // (F - R) F^T = Df + Df E^T
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = 0; j < D; ++j) {
        float s = sc.pol.Df[i][j];
#pragma unroll
        for (int k = 0; k < D; ++k) s += sc.pol.Df[i][k] * E[j][k];
        tau[i][j] = 2.0f * mu * s;
      }
    float vol = la * sc.Jm1 * sc.J;
#pragma unroll
    for (int i = 0; i < D; ++i) tau[i][i] += vol;
  } else if (MAT == kLiquid) {
    ok = sc.J > 0.0f;
    // J - J^(1-g) = (J - 1) - (J^(1-g) - 1), both terms from J - 1 (no cancellation at J ~ 1)
    const float kap = la + 2.0f * mu / (float)D;
    const float g = sc.Jm1 - expm1f((1.0f - kLiquidGamma) * log1pf(sc.Jm1));
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = 0; j < D; ++j) tau[i][j] = (i == j) ? kap * g : 0.0f;
  } else {
    ok = sc.J > 0.0f;
    // F F^T - I = E + E^T + E E^T
    float lnJ = log1pf(sc.Jm1);
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = 0; j < D; ++j) {
        float s = E[i][j] + E[j][i];
#pragma unroll
        for (int k = 0; k < D; ++k) s += E[i][k] * E[j][k];
        tau[i][j] = mu * s + (i == j ? la * lnJ : 0.0f);
      }
  }
  if (act != 0.0f) {
    float fe[D];
#pragma unroll
    for (int i = 0; i < D; ++i) fe[i] = column_of<D>(E[i], axis) + (i == axis ? 1.0f : 0.0f);
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = 0; j < D; ++j) tau[i][j] += act * fe[i] * fe[j];
  }
  return ok && (sc.J == sc.J);
}

// Given taubar = dL/dtau, accumulate Fbar (= dL/dE), mubar, labar and return abar = dL/dact.
template <int D, int MAT>
__device__ __forceinline__ float kirchhoff_adjoint(const float E[D][D], float mu, float la, float act,
                                                   int axis, const StressCache<D>& sc,
                                                   const float tb[D][D], float Fbar[D][D],
                                                   float& mubar, float& labar, int mat_p = MAT) {
  if (MAT == kMixed) {
    if (mat_p == kFixedCorotated)
      return kirchhoff_adjoint<D, kFixedCorotated>(E, mu, la, act, axis, sc, tb, Fbar, mubar, labar);
    if (mat_p == kNeoHookean)
      return kirchhoff_adjoint<D, kNeoHookean>(E, mu, la, act, axis, sc, tb, Fbar, mubar, labar);
    return kirchhoff_adjoint<D, kLiquid>(E, mu, la, act, axis, sc, tb, Fbar, mubar, labar);
  }
  float trtb = 0.0f;
#pragma unroll
  for (int i = 0; i < D; ++i) trtb += tb[i][i];
  float F[D][D], cof[D][D];
  plus_identity<D>(E, F);
  cofactor<D>(F, cof);
  if (MAT == kFixedCorotated) {
    // d/dF [2 mu (F F^T - R F^T)] at fixed R: 2 mu (tb F + tb^T (F - R));  Rbar = -2 mu tb F
    float Rbar[D][D];
    float mub = 0.0f;
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = 0; j < D; ++j) {
        float tF = tb[i][j], tD = 0.0f, DFt = sc.pol.Df[i][j];
#pragma unroll
        for (int k = 0; k < D; ++k) {
          tF += tb[i][k] * E[k][j];
          tD += tb[k][i] * sc.pol.Df[k][j];
          DFt += sc.pol.Df[i][k] * E[j][k];
        }
        Fbar[i][j] += 2.0f * mu * (tF + tD);
        Rbar[i][j] = -2.0f * mu * tF;
        // <tb, (F - R) F^T>: (F - R) F^T = F F^T - R S R^T is symmetric; symmetrise tb first
        // (its antisymmetric part then cancels exactly)
        if (j >= i) mub += (i == j ? tb[i][j] : tb[i][j] + tb[j][i]) * DFt;
      }
    polar_adjoint<D>(E, sc.pol, Rbar, Fbar);
    float c = la * (2.0f * sc.J - 1.0f) * trtb;
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = 0; j < D; ++j) Fbar[i][j] += c * cof[i][j];
    mubar += 2.0f * mub;
    labar += trtb * sc.Jm1 * sc.J;
  } else if (MAT == kLiquid) {
    // tau = kappa g(J) I: Fbar += tr(tb) kappa g'(J) cof F, g'(J) = 1 + (g - 1) J^-g;
    // kappa-bar = tr(tb) g(J) -> labar += kappa-bar, mubar += 2 kappa-bar / d
    const float kap = la + 2.0f * mu / (float)D;
    const float lj = log1pf(sc.Jm1);
    const float g = sc.Jm1 - expm1f((1.0f - kLiquidGamma) * lj);
    const float gp = 1.0f + (kLiquidGamma - 1.0f) * expf(-kLiquidGamma * lj);
    const float c = trtb * kap * gp;
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = 0; j < D; ++j) Fbar[i][j] += c * cof[i][j];
    const float kbar = trtb * g;
    labar += kbar;
    mubar += 2.0f * kbar / (float)D;
  } else {
    float iJ = 1.0f / sc.J;
    float c = la * trtb * iJ;
    float mub = 0.0f;
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = 0; j < D; ++j) {
        float s = tb[i][j] + tb[j][i];  // (tb + tb^T) F = (tb + tb^T) + (tb + tb^T) E
#pragma unroll
        for (int k = 0; k < D; ++k) s += (tb[i][k] + tb[k][i]) * E[k][j];
        Fbar[i][j] += mu * s + c * cof[i][j];
        if (j < i) continue;
        // <tb, F F^T - I> over the symmetric g = E + E^T + E E^T, pairing tb_ij + tb_ji
        // first: a large antisymmetric part of tb then cancels exactly instead of in the sum
        float g = E[i][j] + E[j][i];
#pragma unroll
        for (int k = 0; k < D; ++k) g += E[i][k] * E[j][k];
        mub += (i == j ? tb[i][j] : tb[i][j] + tb[j][i]) * g;
      }
    mubar += mub;
    labar += trtb * log1pf(sc.Jm1);
  }
  // actuation: abar = (F e)^T tb (F e);  Fbar[:, axis] += act (tb + tb^T) F e
  float fe[D];
#pragma unroll
  for (int i = 0; i < D; ++i) fe[i] = column_of<D>(F[i], axis);
  float abar = 0.0f;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    float s = 0.0f, r = 0.0f;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      r += tb[i][j] * fe[j];
      s += (tb[i][j] + tb[j][i]) * fe[j];
    }
    abar += fe[i] * r;
#pragma unroll
    for (int j = 0; j < D; ++j) Fbar[i][j] += j == axis ? act * s : 0.0f;
  }
  return abar;
}

}  // namespace mpm
