// mass_spring.cu -- batched differentiable mass-spring systems (the C ABI of
// include/mass_spring.h): the introductory example of Section 2 and the tape
// demonstration of Section 3, for many independent systems at once.
//
// One thread owns one system for the whole run: its positions, velocities and forces live
// in shared memory (rows indexed by the springs' anchors; in registers for systems of at
// most 4 masses and 4 springs), its rest lengths in registers,
// and every step streams the new state to the tape in HBM (coalesced across systems); the
// backward thread walks the tape in reverse.  The tape is the only memory traffic, so the
// passes are bound by HBM bandwidth: 2 * n * dim floats written per system-step forward,
// n * dim read backward.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mass_spring.h"
#include "../../include/mpm.h"

namespace {

constexpr int kMsThreads = 128;
constexpr float kMsEps = 1e-4f;  // the example's guard: len = |d| + 1e-4
constexpr size_t kAlign = 256;

struct MsParams {
  int n, ns, S;          // masses, springs, systems
  float k, s, dt, inv_m;  // stiffness, exp(-dt alpha), time step, 1 / mass
  signed char a[MS_MAX_SPRINGS], b[MS_MAX_SPRINGS];
};

// Forward: state 0 from (x0, v0), states 1 .. steps-1 by the example's two kernels
// (apply_spring_force, time_integrate), each written to the tape X, V [t][row][system].
// Per-thread rows live in dynamic shared memory, row r of a thread at [r * blockDim + tid]
// (R = n * dim rows per array, so a small system takes little shared memory); MAXS bounds
// the springs a thread keeps in registers (the rest lengths, their gradients).
template <int D, int MAXS>
__global__ void __launch_bounds__(kMsThreads)
    ms_forward_kernel(const __grid_constant__ MsParams P, const float* x0, const float* v0,
                      const float* rest, float* X, float* V, int steps) {
  extern __shared__ float ms_sm[];
  const int sys = blockIdx.x * blockDim.x + threadIdx.x;
  if (sys >= P.S) return;  // no barrier below: each thread works alone
  const int tid = threadIdx.x;
  const int R = P.n * D;
  const int64_t S = P.S;
  const int B = blockDim.x;
  auto sx = [&](int r) -> float& { return ms_sm[r * B + tid]; };
  auto sv = [&](int r) -> float& { return ms_sm[(R + r) * B + tid]; };
  auto sf = [&](int r) -> float& { return ms_sm[(2 * R + r) * B + tid]; };
  for (int r = 0; r < R; ++r) {
    sx(r) = x0[r * S + sys];
    sv(r) = v0[r * S + sys];
    X[r * S + sys] = sx(r);
    V[r * S + sys] = sv(r);
  }
  float l0[MAXS];
#pragma unroll
  for (int j = 0; j < MAXS; ++j) l0[j] = j < P.ns ? rest[j * S + sys] : 0.0f;
  for (int t = 1; t < steps; ++t) {
    for (int r = 0; r < R; ++r) sf(r) = 0.0f;
#pragma unroll
    for (int j = 0; j < MAXS; ++j) {
      if (j >= P.ns) break;
      const int a = P.a[j] * D, b = P.b[j] * D;
      float d[D], nrm = 0.0f;
#pragma unroll
      for (int c = 0; c < D; ++c) {
        d[c] = sx(a + c) - sx(b + c);
        nrm += d[c] * d[c];
      }
      const float len = sqrtf(nrm) + kMsEps;
      const float coef = P.k * (len - l0[j]) / len;
#pragma unroll
      for (int c = 0; c < D; ++c) {
        sf(a + c) -= coef * d[c];
        sf(b + c) += coef * d[c];
      }
    }
    float* Xt = X + (int64_t)t * R * S;
    float* Vt = V + (int64_t)t * R * S;
    for (int r = 0; r < R; ++r) {
      const float v = P.s * sv(r) + P.dt * sf(r) * P.inv_m;
      const float x = sx(r) + P.dt * v;
      sv(r) = v;
      sx(r) = x;
      Xt[r * S + sys] = x;
      Vt[r * S + sys] = v;
    }
  }
}

// Backward: the step adjoints in reverse over the recorded positions (velocities are not
// needed): x_t = x_{t-1} + dt v_t, v_t = s v_{t-1} + dt f(x_{t-1}) / m.  The positions of
// step t-1 are copied from the tape into shared memory kMsAhead steps before they are
// needed (asynchronous copies, a ring of kMsAhead + 1 buffers per thread), so the tape's
// DRAM latency overlaps the arithmetic of the steps in between.
constexpr int kMsBwdThreads = 64;
constexpr int kMsAhead = 3;

__device__ __forceinline__ void ms_copy_async(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void ms_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void ms_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int D, int MAXS>
__global__ void __launch_bounds__(kMsBwdThreads)
    ms_backward_kernel(const __grid_constant__ MsParams P, const float* rest, const float* X,
                       const float* xbT, const float* vbT, float* gx0, float* gv0,
                       float* grest, int steps) {
  extern __shared__ float ms_sm[];
  const int sys = blockIdx.x * blockDim.x + threadIdx.x;
  if (sys >= P.S) return;  // no barrier below: each thread works alone
  const int tid = threadIdx.x;
  const int R = P.n * D;
  const int64_t S = P.S;
  const int B = blockDim.x;
  auto sxb = [&](int r) -> float& { return ms_sm[r * B + tid]; };
  auto svb = [&](int r) -> float& { return ms_sm[(R + r) * B + tid]; };
  // ring buffer q (q < kMsAhead + 1) of recorded positions
  auto sxp = [&](int q, int r) -> float& { return ms_sm[((2 + q) * R + r) * B + tid]; };
  // positions of state u into ring buffer u mod (kMsAhead + 1)
  auto fetch = [&](int u) {
    if (u < 0) return;
    const float* Xu = X + (int64_t)u * R * S;
    const int q = u % (kMsAhead + 1);
    for (int r = 0; r < R; ++r) ms_copy_async(&sxp(q, r), Xu + r * S + sys);
  };
#pragma unroll
  for (int q = 0; q < kMsAhead; ++q) {  // states steps-2, ..., steps-1-kMsAhead
    fetch(steps - 2 - q);
    ms_commit();
  }
  for (int r = 0; r < R; ++r) {
    sxb(r) = xbT ? xbT[r * S + sys] : 0.0f;
    svb(r) = vbT ? vbT[r * S + sys] : 0.0f;
  }
  float l0[MAXS], gl[MAXS];
#pragma unroll
  for (int j = 0; j < MAXS; ++j) {
    l0[j] = j < P.ns ? rest[j * S + sys] : 0.0f;
    gl[j] = 0.0f;
  }
  const float fscale = P.dt * P.inv_m;
  for (int t = steps - 1; t >= 1; --t) {
    fetch(t - 1 - kMsAhead);
    ms_commit();
    ms_wait<kMsAhead>();  // the copy of state t-1, issued kMsAhead steps ago, has landed
    const int q = (t - 1) % (kMsAhead + 1);
    for (int r = 0; r < R; ++r) svb(r) += P.dt * sxb(r);  // dL/dv_t, complete
    // dL/df_t = dt/m dL/dv_t; the springs carry it to x_{t-1} and the rest lengths
#pragma unroll
    for (int j = 0; j < MAXS; ++j) {
      if (j >= P.ns) break;
      const int a = P.a[j] * D, b = P.b[j] * D;
      float d[D], Fb[D], nrm = 0.0f, dFb = 0.0f;
#pragma unroll
      for (int c = 0; c < D; ++c) {
        d[c] = sxp(q, a + c) - sxp(q, b + c);
        nrm += d[c] * d[c];
        Fb[c] = fscale * (svb(b + c) - svb(a + c));  // f_a -= F, f_b += F
        dFb += d[c] * Fb[c];
      }
      // F = k (1 - l0/len) d, dlen/dd = d / r: one reciprocal square root and one division
      // (the reverse pass needs no bit-exact match with the forward's rounding)
      const float rinv = nrm > 0.0f ? rsqrtf(nrm) : 0.0f;
      const float r = nrm * rinv, inv = 1.0f / (r + kMsEps);
      gl[j] -= P.k * dFb * inv;
      const float c1 = P.k * (1.0f - l0[j] * inv);
      const float c2 = P.k * l0[j] * inv * inv * dFb * rinv;
#pragma unroll
      for (int c = 0; c < D; ++c) {
        const float db = c1 * Fb[c] + c2 * d[c];
        sxb(a + c) += db;
        sxb(b + c) -= db;
      }
    }
    for (int r = 0; r < R; ++r) svb(r) *= P.s;  // dL/dv_{t-1}
  }
  ms_wait<0>();  // no copy is left in flight when the thread exits
  for (int r = 0; r < R; ++r) {
    if (gx0) gx0[r * S + sys] = sxb(r);
    if (gv0) gv0[r * S + sys] = svb(r);
  }
  if (grest)
#pragma unroll
    for (int j = 0; j < MAXS; ++j)
      if (j < P.ns) grest[j * S + sys] = gl[j];
}

// Small systems (at most 4 masses and 4 springs, the paper's triangle among them): the whole
// state of a thread's system in registers.  A spring's anchors are runtime values, so its
// end points are picked from the register rows by compares (mass i of row i is a
// compile-time index in every unrolled access) instead of indexing shared memory, which
// keeps each step free of shared-memory round trips.
constexpr int kMsSmallMasses = 4;

template <int D>
__device__ __forceinline__ float ms_pick(const float (&x)[kMsSmallMasses][D], int a, int c) {
  float r = x[0][c];
#pragma unroll
  for (int i = 1; i < kMsSmallMasses; ++i)
    if (a == i) r = x[i][c];
  return r;
}
template <int D>
__device__ __forceinline__ void ms_add(float (&x)[kMsSmallMasses][D], int a, int c, float v) {
#pragma unroll
  for (int i = 0; i < kMsSmallMasses; ++i)
    if (a == i) x[i][c] += v;
}

template <int D>
__global__ void __launch_bounds__(kMsThreads)
    ms_forward_small(const __grid_constant__ MsParams P, const float* x0, const float* v0,
                     const float* rest, float* X, float* V, int steps) {
  const int sys = blockIdx.x * blockDim.x + threadIdx.x;
  if (sys >= P.S) return;
  const int n = P.n;
  const int64_t S = P.S, RS = (int64_t)n * D * S;
  float x[kMsSmallMasses][D], v[kMsSmallMasses][D], l0[4];
#pragma unroll
  for (int i = 0; i < kMsSmallMasses; ++i)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      const bool on = i < n;
      x[i][c] = on ? x0[(i * D + c) * S + sys] : 0.0f;
      v[i][c] = on ? v0[(i * D + c) * S + sys] : 0.0f;
      if (on) {
        X[(i * D + c) * S + sys] = x[i][c];
        V[(i * D + c) * S + sys] = v[i][c];
      }
    }
#pragma unroll
  for (int j = 0; j < 4; ++j) l0[j] = j < P.ns ? rest[j * S + sys] : 0.0f;
  for (int t = 1; t < steps; ++t) {
    float f[kMsSmallMasses][D];
#pragma unroll
    for (int i = 0; i < kMsSmallMasses; ++i)
#pragma unroll
      for (int c = 0; c < D; ++c) f[i][c] = 0.0f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (j >= P.ns) break;
      const int a = P.a[j], b = P.b[j];
      float d[D], nrm = 0.0f;
#pragma unroll
      for (int c = 0; c < D; ++c) {
        d[c] = ms_pick<D>(x, a, c) - ms_pick<D>(x, b, c);
        nrm += d[c] * d[c];
      }
      const float len = sqrtf(nrm) + kMsEps;
      const float coef = P.k * (len - l0[j]) / len;
#pragma unroll
      for (int c = 0; c < D; ++c) {
        ms_add<D>(f, a, c, -coef * d[c]);
        ms_add<D>(f, b, c, coef * d[c]);
      }
    }
    float* Xt = X + t * RS;
    float* Vt = V + t * RS;
#pragma unroll
    for (int i = 0; i < kMsSmallMasses; ++i)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        v[i][c] = P.s * v[i][c] + P.dt * f[i][c] * P.inv_m;
        x[i][c] = x[i][c] + P.dt * v[i][c];
        if (i < n) {
          Xt[(i * D + c) * S + sys] = x[i][c];
          Vt[(i * D + c) * S + sys] = v[i][c];
        }
      }
  }
}

template <int D>
__global__ void __launch_bounds__(kMsBwdThreads)
    ms_backward_small(const __grid_constant__ MsParams P, const float* rest, const float* X,
                      const float* xbT, const float* vbT, float* gx0, float* gv0, float* grest,
                      int steps) {
  extern __shared__ float ms_sm[];  // the prefetch ring: (kMsAhead + 1) x R rows
  const int sys = blockIdx.x * blockDim.x + threadIdx.x;
  if (sys >= P.S) return;  // no barrier below: each thread works alone
  const int tid = threadIdx.x, B = blockDim.x;
  const int n = P.n, R = n * D;
  const int64_t S = P.S;
  auto ring = [&](int q, int r) -> float& { return ms_sm[(q * R + r) * B + tid]; };
  auto fetch = [&](int u) {
    if (u < 0) return;
    const float* Xu = X + (int64_t)u * R * S;
    const int q = u % (kMsAhead + 1);
    for (int r = 0; r < R; ++r) ms_copy_async(&ring(q, r), Xu + r * S + sys);
  };
#pragma unroll
  for (int q = 0; q < kMsAhead; ++q) {
    fetch(steps - 2 - q);
    ms_commit();
  }
  float xb[kMsSmallMasses][D], vb[kMsSmallMasses][D], l0[4], gl[4];
#pragma unroll
  for (int i = 0; i < kMsSmallMasses; ++i)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      const bool on = i < n;
      xb[i][c] = on && xbT ? xbT[(i * D + c) * S + sys] : 0.0f;
      vb[i][c] = on && vbT ? vbT[(i * D + c) * S + sys] : 0.0f;
    }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    l0[j] = j < P.ns ? rest[j * S + sys] : 0.0f;
    gl[j] = 0.0f;
  }
  const float fscale = P.dt * P.inv_m;
  for (int t = steps - 1; t >= 1; --t) {
    fetch(t - 1 - kMsAhead);
    ms_commit();
    ms_wait<kMsAhead>();  // the copy of state t-1, issued kMsAhead steps ago, has landed
    const int q = (t - 1) % (kMsAhead + 1);
    float xp[kMsSmallMasses][D];
#pragma unroll
    for (int i = 0; i < kMsSmallMasses; ++i)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        xp[i][c] = i < n ? ring(q, i * D + c) : 0.0f;
        vb[i][c] += P.dt * xb[i][c];  // dL/dv_t, complete
      }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (j >= P.ns) break;
      const int a = P.a[j], b = P.b[j];
      float d[D], Fb[D], nrm = 0.0f, dFb = 0.0f;
#pragma unroll
      for (int c = 0; c < D; ++c) {
        d[c] = ms_pick<D>(xp, a, c) - ms_pick<D>(xp, b, c);
        nrm += d[c] * d[c];
        Fb[c] = fscale * (ms_pick<D>(vb, b, c) - ms_pick<D>(vb, a, c));  // f_a -= F, f_b += F
        dFb += d[c] * Fb[c];
      }
      // F = k (1 - l0/len) d, dlen/dd = d / r: one reciprocal square root and one division
      const float rinv = nrm > 0.0f ? rsqrtf(nrm) : 0.0f;
      const float r = nrm * rinv, inv = 1.0f / (r + kMsEps);
      gl[j] -= P.k * dFb * inv;
      const float c1 = P.k * (1.0f - l0[j] * inv);
      const float c2 = P.k * l0[j] * inv * inv * dFb * rinv;
#pragma unroll
      for (int c = 0; c < D; ++c) {
        const float db = c1 * Fb[c] + c2 * d[c];
        ms_add<D>(xb, a, c, db);
        ms_add<D>(xb, b, c, -db);
      }
    }
#pragma unroll
    for (int i = 0; i < kMsSmallMasses; ++i)
#pragma unroll
      for (int c = 0; c < D; ++c) vb[i][c] *= P.s;  // dL/dv_{t-1}
  }
  ms_wait<0>();
#pragma unroll
  for (int i = 0; i < kMsSmallMasses; ++i)
#pragma unroll
    for (int c = 0; c < D; ++c)
      if (i < n) {
        if (gx0) gx0[(i * D + c) * S + sys] = xb[i][c];
        if (gv0) gv0[(i * D + c) * S + sys] = vb[i][c];
      }
  if (grest)
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (j < P.ns) grest[j * S + sys] = gl[j];
}

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct MsLayout {
  size_t X, V, rest, total;
};

MsLayout ms_layout(const ms_desc* d, int steps) {
  const size_t rows = (size_t)d->n_masses * d->dim, S = (size_t)d->n_systems;
  MsLayout L;
  size_t o = 0;
  L.X = o;
  o = align_up(o + (size_t)steps * rows * S * 4);
  L.V = o;
  o = align_up(o + (size_t)steps * rows * S * 4);
  L.rest = o;
  o = align_up(o + (size_t)(d->n_springs > 0 ? d->n_springs : 1) * S * 4);
  L.total = o;
  return L;
}

thread_local std::string g_ms_error;

bool ms_valid(const ms_desc* d, int steps, std::string* why) {
  auto fail = [&](const char* m) {
    *why = m;
    return false;
  };
  if (!d) return fail("desc is NULL");
  if (d->dim != 2 && d->dim != 3) return fail("dim must be 2 or 3");
  if (d->n_masses < 1 || d->n_masses > MS_MAX_MASSES) return fail("n_masses must be in [1, 8]");
  if (d->n_springs < 0 || d->n_springs > MS_MAX_SPRINGS) return fail("n_springs must be in [0, 32]");
  if (d->n_springs > 0 && (!d->spring_a || !d->spring_b)) return fail("spring anchors are NULL");
  for (int j = 0; j < d->n_springs; ++j) {
    const int a = d->spring_a[j], b = d->spring_b[j];
    if (a < 0 || b < 0 || a >= d->n_masses || b >= d->n_masses || a == b)
      return fail("a spring's anchors must be two different masses");
  }
  if (d->n_systems < 1) return fail("n_systems must be >= 1");
  if (!(d->dt > 0.0f) || !std::isfinite(d->dt)) return fail("dt must be > 0");
  if (!(d->mass > 0.0f) || !std::isfinite(d->mass)) return fail("mass must be > 0");
  if (!std::isfinite(d->stiffness) || !std::isfinite(d->damping)) return fail("stiffness and damping must be finite");
  if (steps < 1) return fail("steps must be >= 1");
  const double bytes = 2.0 * steps * d->n_masses * d->dim * (double)d->n_systems * 4.0;
  if (bytes > 1.0e12) return fail("the tape would exceed 1 TB");
  return true;
}

}  // namespace

struct ms_handle {
  ms_desc desc;
  std::vector<int32_t> sa, sb;
  int steps_max = 0;
  int steps_rec = 0;
  MsLayout L;
  char* ws = nullptr;
  std::string last_error;
  cudaStream_t last_stream = nullptr;
  MsParams P;
};

namespace {

int ms_fail(ms_handle* h, int code, const std::string& m) {
  if (h) h->last_error = m; else g_ms_error = m;
  return code;
}

#define MS_CK(expr)                                                                   \
  do {                                                                                \
    cudaError_t e_ = (expr);                                                          \
    if (e_ != cudaSuccess) return ms_fail(h, MPM_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

int blocks_for(int S, int threads) { return (S + threads - 1) / threads; }

// dispatch on the dimension and the springs kept in registers (4 or MS_MAX_SPRINGS)
template <int D, int MAXS>
cudaError_t ms_fwd(const MsParams& P, const float* x0, const float* v0, const float* R, float* X,
                   float* V, int steps, cudaStream_t s) {
  const size_t smem = (size_t)3 * P.n * D * kMsThreads * sizeof(float);
  ms_forward_kernel<D, MAXS><<<blocks_for(P.S, kMsThreads), kMsThreads, smem, s>>>(P, x0, v0, R, X, V, steps);
  return cudaGetLastError();
}
template <int D, int MAXS>
cudaError_t ms_bwd(const MsParams& P, const float* R, const float* X, const float* xb,
                   const float* vb, float* gx, float* gv, float* gl, int steps, cudaStream_t s) {
  const size_t smem = (size_t)(2 + kMsAhead + 1) * P.n * D * kMsBwdThreads * sizeof(float);
  ms_backward_kernel<D, MAXS><<<blocks_for(P.S, kMsBwdThreads), kMsBwdThreads, smem, s>>>(P, R, X, xb, vb, gx, gv, gl, steps);
  return cudaGetLastError();
}
bool ms_small(const MsParams& P) { return P.n <= kMsSmallMasses && P.ns <= 4; }

cudaError_t ms_launch_forward(int dim, const MsParams& P, const float* x0, const float* v0,
                              const float* R, float* X, float* V, int steps, cudaStream_t s) {
  if (ms_small(P)) {
    if (dim == 2) ms_forward_small<2><<<blocks_for(P.S, kMsThreads), kMsThreads, 0, s>>>(P, x0, v0, R, X, V, steps);
    else ms_forward_small<3><<<blocks_for(P.S, kMsThreads), kMsThreads, 0, s>>>(P, x0, v0, R, X, V, steps);
    return cudaGetLastError();
  }
  if (dim == 2) return P.ns <= 4 ? ms_fwd<2, 4>(P, x0, v0, R, X, V, steps, s) : ms_fwd<2, MS_MAX_SPRINGS>(P, x0, v0, R, X, V, steps, s);
  return P.ns <= 4 ? ms_fwd<3, 4>(P, x0, v0, R, X, V, steps, s) : ms_fwd<3, MS_MAX_SPRINGS>(P, x0, v0, R, X, V, steps, s);
}
cudaError_t ms_launch_backward(int dim, const MsParams& P, const float* R, const float* X,
                               const float* xb, const float* vb, float* gx, float* gv, float* gl,
                               int steps, cudaStream_t s) {
  if (ms_small(P)) {
    const size_t smem = (size_t)(kMsAhead + 1) * P.n * dim * kMsBwdThreads * sizeof(float);
    if (dim == 2)
      ms_backward_small<2><<<blocks_for(P.S, kMsBwdThreads), kMsBwdThreads, smem, s>>>(P, R, X, xb, vb, gx, gv, gl, steps);
    else
      ms_backward_small<3><<<blocks_for(P.S, kMsBwdThreads), kMsBwdThreads, smem, s>>>(P, R, X, xb, vb, gx, gv, gl, steps);
    return cudaGetLastError();
  }
  if (dim == 2) return P.ns <= 4 ? ms_bwd<2, 4>(P, R, X, xb, vb, gx, gv, gl, steps, s) : ms_bwd<2, MS_MAX_SPRINGS>(P, R, X, xb, vb, gx, gv, gl, steps, s);
  return P.ns <= 4 ? ms_bwd<3, 4>(P, R, X, xb, vb, gx, gv, gl, steps, s) : ms_bwd<3, MS_MAX_SPRINGS>(P, R, X, xb, vb, gx, gv, gl, steps, s);
}

}  // namespace

extern "C" {

int ms_workspace_bytes(const ms_desc* desc, int32_t steps, size_t* out_bytes) {
  std::string why;
  if (!out_bytes) return ms_fail(nullptr, MPM_ERR_ARG, "out_bytes is NULL");
  if (!ms_valid(desc, steps, &why)) return ms_fail(nullptr, MPM_ERR_ARG, why);
  *out_bytes = ms_layout(desc, steps).total;
  return MPM_OK;
}

int ms_create(const ms_desc* desc, void* workspace, size_t workspace_bytes, int32_t steps,
              ms_handle** out) {
  std::string why;
  if (!out) return ms_fail(nullptr, MPM_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!ms_valid(desc, steps, &why)) return ms_fail(nullptr, MPM_ERR_ARG, why);
  const MsLayout L = ms_layout(desc, steps);
  if (!workspace || reinterpret_cast<uintptr_t>(workspace) % kAlign != 0)
    return ms_fail(nullptr, MPM_ERR_WORKSPACE, "workspace must be a 256-byte aligned device pointer");
  if (workspace_bytes < L.total)
    return ms_fail(nullptr, MPM_ERR_WORKSPACE, "workspace smaller than ms_workspace_bytes");
  ms_handle* h = new ms_handle();
  h->desc = *desc;
  h->sa.assign(desc->spring_a, desc->spring_a + desc->n_springs);
  h->sb.assign(desc->spring_b, desc->spring_b + desc->n_springs);
  h->desc.spring_a = h->sa.data();
  h->desc.spring_b = h->sb.data();
  h->steps_max = steps;
  h->L = L;
  h->ws = static_cast<char*>(workspace);
  MsParams& P = h->P;
  memset(&P, 0, sizeof(P));
  P.n = desc->n_masses;
  P.ns = desc->n_springs;
  P.S = desc->n_systems;
  P.k = desc->stiffness;
  P.s = (float)std::exp(-(double)desc->dt * (double)desc->damping);
  P.dt = desc->dt;
  P.inv_m = 1.0f / desc->mass;
  for (int j = 0; j < desc->n_springs; ++j) {
    P.a[j] = (signed char)desc->spring_a[j];
    P.b[j] = (signed char)desc->spring_b[j];
  }
  *out = h;
  return MPM_OK;
}

int ms_forward(ms_handle* h, const float* x0, const float* v0, const float* rest, int32_t steps,
               void* stream) {
  if (!h) return ms_fail(nullptr, MPM_ERR_ARG, "handle is NULL");
  if (!x0 || !v0 || (h->desc.n_springs > 0 && !rest)) return ms_fail(h, MPM_ERR_ARG, "x0, v0 and rest are required");
  if (steps < 1 || steps > h->steps_max) return ms_fail(h, MPM_ERR_STATE, "steps must be in [1, create-time steps]");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  h->last_stream = s;
  float* R = reinterpret_cast<float*>(h->ws + h->L.rest);
  if (h->desc.n_springs > 0)
    MS_CK(cudaMemcpyAsync(R, rest, (size_t)h->desc.n_springs * h->desc.n_systems * 4,
                          cudaMemcpyDeviceToDevice, s));
  float* X = reinterpret_cast<float*>(h->ws + h->L.X);
  float* V = reinterpret_cast<float*>(h->ws + h->L.V);
  MS_CK(ms_launch_forward(h->desc.dim, h->P, x0, v0, R, X, V, steps, s));
  h->steps_rec = steps;
  return MPM_OK;
}

int ms_get_state(ms_handle* h, int32_t t, float* x, float* v, void* stream) {
  if (!h) return ms_fail(nullptr, MPM_ERR_ARG, "handle is NULL");
  if (!h->steps_rec) return ms_fail(h, MPM_ERR_STATE, "no forward recorded");
  if (t < 0 || t >= h->steps_rec) return ms_fail(h, MPM_ERR_ARG, "t must be in [0, steps)");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  h->last_stream = s;
  const size_t row = (size_t)h->desc.n_masses * h->desc.dim * h->desc.n_systems;
  if (x) MS_CK(cudaMemcpyAsync(x, reinterpret_cast<float*>(h->ws + h->L.X) + t * row, row * 4, cudaMemcpyDeviceToDevice, s));
  if (v) MS_CK(cudaMemcpyAsync(v, reinterpret_cast<float*>(h->ws + h->L.V) + t * row, row * 4, cudaMemcpyDeviceToDevice, s));
  return MPM_OK;
}

int ms_backward(ms_handle* h, const float* dL_dx, const float* dL_dv, float* gx0, float* gv0,
                float* grest, void* stream) {
  if (!h) return ms_fail(nullptr, MPM_ERR_ARG, "handle is NULL");
  if (!h->steps_rec) return ms_fail(h, MPM_ERR_STATE, "backward needs a recorded forward");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  h->last_stream = s;
  const float* R = reinterpret_cast<const float*>(h->ws + h->L.rest);
  const float* X = reinterpret_cast<const float*>(h->ws + h->L.X);
  MS_CK(ms_launch_backward(h->desc.dim, h->P, R, X, dL_dx, dL_dv, gx0, gv0, grest, h->steps_rec, s));
  return MPM_OK;
}

int ms_sync(ms_handle* h) {
  if (!h) return ms_fail(nullptr, MPM_ERR_ARG, "handle is NULL");
  cudaError_t e = cudaStreamSynchronize(h->last_stream);
  if (e != cudaSuccess) return ms_fail(h, MPM_ERR_CUDA, std::string("cudaStreamSynchronize: ") + cudaGetErrorString(e));
  return MPM_OK;
}

const char* ms_last_error(ms_handle* h) { return h ? h->last_error.c_str() : g_ms_error.c_str(); }

void ms_destroy(ms_handle* h) { delete h; }

}  // extern "C"
