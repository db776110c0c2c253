/*
 * mass_spring.h -- C ABI of the batched differentiable mass-spring system in libmpm.so:
 * the introductory example of "DiffTaichi: Differentiable Programming for Physical
 * Simulation" (Section 2) and the tape demonstration of Section 3, for many independent
 * systems at once.
 *
 * What it computes (per system, states 0 .. steps-1; step t >= 1 from state t-1):
 *   d_j = x_a - x_b,  len_j = |d_j| + 1e-4,  F_j = k (len_j - l0_j) d_j / len_j
 *   (Hooke's law with the example's guard against a zero length),  f_a -= F_j, f_b += F_j,
 *   v_t = exp(-dt alpha) v_{t-1} + dt f / m,   x_t = x_{t-1} + dt v_t
 *   (semi-implicit Euler with damping).  The forward records every state (the example's
 *   tensors of size steps x n); ms_backward replays the step adjoints in reverse (the tape
 *   of Section 3) and returns dL/dx0, dL/dv0 and dL/dl0 (the rest lengths the example
 *   optimises).
 *
 * Conventions: int status codes (MPM_OK = 0, MPM_ERR_* of mpm.h); "device" pointers are
 * CUDA device pointers; every per-system array is float32, component-major over systems:
 * a[r * n_systems + s] for row r of system s.  Positions and velocities have rows
 * i * dim + c (mass i, component c); rest lengths have rows j (spring j).  All work is
 * asynchronous on `stream` (a cudaStream_t; NULL = legacy default stream).  The library
 * owns nothing beyond the caller's workspace and a small host handle.
 */
#ifndef MASS_SPRING_H
#define MASS_SPRING_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MS_MAX_MASSES 8   /* mass points per system */
#define MS_MAX_SPRINGS 32 /* springs per system */

typedef struct ms_handle ms_handle;

/* Shared by every system of the batch; copied at create. */
typedef struct ms_desc {
  int32_t dim;              /* 2 or 3 */
  int32_t n_masses;         /* 1 .. MS_MAX_MASSES */
  int32_t n_springs;        /* 0 .. MS_MAX_SPRINGS */
  const int32_t* spring_a;  /* host [n_springs]: first mass of each spring */
  const int32_t* spring_b;  /* host [n_springs]: second mass (a != b, both < n_masses) */
  int32_t n_systems;        /* independent systems, >= 1 */
  float stiffness;          /* k */
  float damping;            /* alpha: velocities scale by exp(-dt alpha) per step */
  float dt;                 /* > 0 */
  float mass;               /* m > 0, every mass point */
} ms_desc;

/* Device bytes for this description and at most `steps` states (the tape of positions
 * and velocities, the rest lengths).  out_bytes: host. */
int ms_workspace_bytes(const ms_desc* desc, int32_t steps, size_t* out_bytes);

/* workspace: device, >= ms_workspace_bytes, 256-byte aligned, owned by the caller.
 * out: host.  MPM_ERR_ARG on a bad description, MPM_ERR_WORKSPACE on a bad workspace. */
int ms_create(const ms_desc* desc, void* workspace, size_t workspace_bytes, int32_t steps,
              ms_handle** out);

/* Run from state 0 = (x0, v0) (device [n_masses*dim][n_systems]) with rest lengths
 * rest (device [n_springs][n_systems], copied in) to state steps-1 (1 <= steps <= the
 * create-time steps; steps = 1 records state 0 only), recording every state. */
int ms_forward(ms_handle* h, const float* x0, const float* v0, const float* rest, int32_t steps,
               void* stream);

/* Copy state t (0 <= t < steps of the last forward) to device x, v (either may be NULL). */
int ms_get_state(ms_handle* h, int32_t t, float* x, float* v, void* stream);

/* Reverse of the last forward: given dL/dx and dL/dv of its last state (device, either may
 * be NULL = 0), write dL/dx0, dL/dv0 (device [n_masses*dim][n_systems]) and dL/drest
 * (device [n_springs][n_systems]); any output may be NULL.  MPM_ERR_STATE before a forward.
 * May be called more than once per forward. */
int ms_backward(ms_handle* h, const float* dL_dx, const float* dL_dv, float* gx0, float* gv0,
                float* grest, void* stream);

/* Wait for the handle's last stream; MPM_OK or MPM_ERR_CUDA. */
int ms_sync(ms_handle* h);

/* Message of the last failure of a call on h (NULL: of a call without a handle). */
const char* ms_last_error(ms_handle* h);

void ms_destroy(ms_handle* h);

#ifdef __cplusplus
}
#endif

#endif /* MASS_SPRING_H */
