/*
 * mpm.h -- C ABI of libmpm.so, the GB300 (sm_103a) differentiable MLS-MPM
 * elastic-object simulator: the hot path of DiffTaichi's diffmpm (Section 4.1 and
 * Appendix D of "DiffTaichi: Differentiable Programming for Physical Simulation").
 *
 * What the library computes
 *   One time step (Appendix D, "advance"): clear the grid, P2G scatter of mass and
 *   APIC/MLS momentum with quadratic B-spline weights and the Kirchhoff stress
 *   folded into the affine matrix, grid update (momentum/mass + dt g, sticky walls),
 *   G2P gather of velocity and affine matrix C, x' = x + dt v', F' = (I + dt C') F.
 *   The reverse pass is the light-weight tape of Section 3.2: the forward stores
 *   the full particle state every ckpt_every steps (Appendix D.2); mpm_backward
 *   re-simulates each segment and replays the step adjoints in reverse order,
 *   recomputing each step's grid (Appendix D.1, "advance_grad").
 *   Materials: fixed-corotated (polar factor resolved to FP64 accuracy with
 *   compensated FP32 arithmetic, FP32 adjoint; the build variant MPM_POLAR_FP64=1
 *   forms both in FP64) or neo-Hookean; optional actuation stress a_g(t) (F e)(F e)^T with
 *   a_g(t) = sum_k w_gk sin(2 pi k t / act_period + act_phase), k = 1..n_basis
 *   (open loop), or a_g(t) = the output of a closed-loop controller evaluated on
 *   state t (the neural-network controllers of Section 4.1; see ctrl_hidden).
 *
 * Conventions (every entry point)
 *   - Returns an int status (MPM_OK = 0 or an MPM_ERR_* code); no exception
 *     crosses the ABI.  mpm_last_error() gives a message for the last failure.
 *   - Pointers named "device" are CUDA device pointers; "host" are host pointers.
 *   - Per-particle arrays are float32, component-major: a[c * N + p] with N the
 *     total particle count; scenes are concatenated in particle order.  Vectors
 *     have dim components, matrices dim*dim (row-major within a particle: C[i][j]
 *     is component i*dim + j).
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  All work is
 *     asynchronous on that stream; device-side errors (a particle's stencil
 *     leaving the grid, non-finite values, det F <= 0, a bounded wait running out)
 *     are sticky in the handle and reported by mpm_sync_status().
 *   - Ownership: the library allocates no device memory.  The caller provides one
 *     device workspace (size from mpm_workspace_bytes) at create time and owns it;
 *     it must outlive the handle.  Inputs are copied into the workspace; outputs
 *     go to caller-allocated buffers.  The handle itself is a small host object.
 */
#ifndef MPM_H_
#define MPM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define MPM_OK 0
#define MPM_ERR_ARG 1        /* invalid argument (NULL handle, bad size, ...) */
#define MPM_ERR_CUDA 2       /* a CUDA runtime call failed */
#define MPM_ERR_OOB 3        /* a particle's 3^dim stencil left [0, n_grid-1] */
#define MPM_ERR_NONFINITE 4  /* non-finite state or det F <= 0 */
#define MPM_ERR_TIMEOUT 5    /* a bounded device-side wait gave up */
#define MPM_ERR_STATE 6      /* call out of order (backward before forward, T > max) */
#define MPM_ERR_WORKSPACE 7  /* workspace NULL, misaligned or too small */
#define MPM_ERR_TOO_LARGE 8  /* mpm_step_noalloc: problem larger than its fixed scratch */
#define MPM_ERR_RANGE 9      /* deterministic mode: a grid contribution left the fixed-point range */

/* materials */
#define MPM_FIXED_COROTATED 0
#define MPM_NEO_HOOKEAN 1
#define MPM_LIQUID 3 /* weakly compressible liquid: the paper's liquid simulator follows the
                        weakly compressible model of Tampubolon et al. 2017; here in Tait form,
                        Kirchhoff stress kappa (J - J^(1-7)) I with kappa = lambda + 2 mu / dim
                        the bulk modulus of the particle's (E, nu); no shear stress */
#define MPM_MIXED 4  /* each particle carries its own material id (MPM_FIXED_COROTATED,
                        MPM_NEO_HOOKEAN or MPM_LIQUID; any other id acts as MPM_LIQUID), set
                        with mpm_set_particle_materials: a solid and a liquid two-way coupled
                        through one grid, as in the paper's robot-in-liquid experiment */

/* losses computed by mpm_loss (the compute_loss pattern of Section 3.2) */
#define MPM_LOSS_COM_TARGET 0 /* L_s = |COM_s(x_T) - target_s|^2 */
#define MPM_LOSS_COM_X_DISP 1 /* L_s = -(COM_s,x(x_T) - COM_s,x(x_0)) */

/* options for mpm_set_option (tuning knobs; defaults in brackets) */
#define MPM_OPT_USE_GRAPHS 1      /* capture forward/backward into CUDA graphs [1] */
#define MPM_OPT_SMEM_TILE 2       /* 1: scatters accumulate in a shared-memory node box and
                                     flush once per node; 0: float4 reductions straight to
                                     the L2-resident grid [0, faster on GB300] */
#define MPM_OPT_TILE_CAPACITY 3   /* max nodes of one CTA's shared tile [1024]; this and
                                     MPM_OPT_GATHER_CAPACITY / MPM_OPT_SMEM_TILE return
                                     MPM_ERR_ARG (option unchanged) when the node boxes would
                                     not fit the device's shared memory per CTA */
#define MPM_OPT_PROFILE 4         /* 1: time every kernel launch with CUDA events on its
                                     stream (launches go unbatched, no graphs) [0];
                                     setting it clears the collected timings */

#define MPM_OPT_GATHER_CAPACITY 5 /* max nodes of a CTA's shared gather box; 0 = gathers
                                     read the grid through L1 [512] */
#define MPM_OPT_POLAR_CACHE 7     /* 3D fixed-corotated: the re-simulation stores each state's
                                     polar factor (as an FP32 value + correction pair) for the
                                     two backward passes that need it instead of recomputing
                                     it [1] */
#define MPM_OPT_GRID_BLOCKS 6     /* CTAs per scene of the end-of-sequence grid clear; 0 = automatic [0] */
#define MPM_OPT_PERSISTENT 8      /* 1: each run of passes of one kind and one pass mode (the
                                     fused steps of a forward; the re-simulation and the
                                     adjoint passes of each backward segment, each split at
                                     its first and last pass) is one cooperative launch of
                                     resident CTAs that step through a recorded pass plan
                                     with a grid-wide barrier between passes [0].  Results
                                     equal the one-launch-per-pass form up to FP32 atomic
                                     order; slower than it on this GPU (the interpreter spills
                                     the parameters the per-pass kernels read as constants). */
#define MPM_OPT_BARRIER_TIMEOUT_US 9 /* limit of one grid-barrier wait in the persistent form,
                                     microseconds, 1..6e8 [2000000].  A wait that runs out sets
                                     MPM_ERR_TIMEOUT (reported by mpm_sync_status, after which the
                                     handle needs mpm_set_initial) and every CTA returns. */
#define MPM_OPT_GRID_RECOMPUTE 12 /* 1: every adjoint pass recomputes the grid of the step before
                                     (Appendix D.1) even when the re-simulated segment's grids fit
                                     in the workspace (K + 4 grid buffers within 8 GiB, decided at
                                     create); 0: keep them [0] */
#define MPM_OPT_OVERLAP_RESIM 13  /* 1: mpm_backward re-simulates segment j-1 on a second stream
                                     while the adjoint passes of segment j run (independent
                                     work that shares the SMs; results are the same as with 0,
                                     bitwise in the deterministic mode).  Not used in the
                                     persistent form, with a controller, or while profiling [1] */
#define MPM_OPT_PERSISTENT_CHUNK 11 /* persistent form: at most this many passes per launch
                                     (0 = a whole run of same-kind passes) [0]; bounds the
                                     duration of any one launch */
#define MPM_OPT_BUCKET_SCATTER 14  /* 1: a particle pass groups its tile's particles by stencil
                                     base and scatters each group with one warp, one float4
                                     reduction per (base, node) summed in registers, instead of
                                     one per (particle, node) [0: on GB300 the extra shared-
                                     memory traffic of the group loop outweighed the saved
                                     reductions].  FP32 sums only (ignored in the deterministic
                                     mode and with MPM_OPT_SMEM_TILE). */
#define MPM_OPT_PAIR_SCATTER 15    /* bit mask, 0..3: float4 reductions straight to the grid
                                     merge the two contributions of a pair of particles
                                     (consecutive in the set-up's base order) that share a
                                     stencil base, one reduction per pair and node -- bit 0 in
                                     the forward and re-simulation passes, bit 1 in the adjoint
                                     passes [0; pairs share a base only in MPM_OPT_SORT_ORDER 1].
                                     FP32 sums only. */
#define MPM_OPT_SORT_ORDER 16      /* particle order chosen by mpm_set_initial (takes effect at
                                     the next mpm_set_initial), by a grid coordinate per axis
                                     in runs of 8 along the last axis: 0 the cell; 1 the
                                     stencil base; 2 the cell, but the base on the last axis,
                                     so that consecutive pairs of particles share their base
                                     (what MPM_OPT_PAIR_SCATTER merges) [0: the adjoint passes'
                                     gathers run fastest over the cell order's tiles] */
#define MPM_OPT_BARRIER_TEST_EXTRA 10 /* test hook, 0..1024 [0]: arrivals every grid barrier
                                     waits for beyond the launch's own CTAs.  Nonzero values
                                     can never be met, so each persistent launch ends through
                                     the timeout path; nothing else changes. */

/* kernel categories for mpm_get_profile */
#define MPM_KERNEL_P2G 1          /* P2G from a full state (segment starts, grid recompute) */
#define MPM_KERNEL_G2P_P2G 2      /* fused G2P of step t-1 + P2G of step t, x and F written */
#define MPM_KERNEL_G2P_P2G_FULL 3 /* same, full state written (checkpoints, re-simulation) */
#define MPM_KERNEL_G2P 4          /* last G2P of a run or segment, full state written */
#define MPM_KERNEL_GRID_CLEAR 5   /* zeroing of grid buffers at the end of a launch sequence */
#define MPM_KERNEL_ADJ_G2P 6      /* G2P adjoint from the seeds (step T-1) */
#define MPM_KERNEL_ADJ_FUSED 7    /* P2G adjoint of step s+1 + G2P adjoint of step s +
                                     recomputed P2G of step s-1 */
#define MPM_KERNEL_ADJ_P2G 8      /* P2G adjoint of step 0 */
#define MPM_KERNEL_PERSISTENT_STEP 9 /* persistent launch of forward-kind passes (categories 1-4) */
#define MPM_KERNEL_PERSISTENT_ADJ 10 /* persistent launch of adjoint passes (categories 6-8) */
#define MPM_KERNEL_CONTROLLER 11  /* closed-loop controller: sensing + MLP, or its reverse */


/* queries for mpm_get_info */
#define MPM_INFO_KERNEL_LAUNCHES 1 /* kernels launched by this handle so far */
#define MPM_INFO_N_TOTAL 2         /* total particles N */
#define MPM_INFO_STEPS_RECORDED 3  /* T of the last mpm_forward (0 = none) */
#define MPM_INFO_KEEPS_SEGMENT_GRIDS 4 /* 1: a re-simulated segment's grids are kept for its
                                          adjoint passes (see MPM_OPT_GRID_RECOMPUTE) */
#define MPM_INFO_ACT_PARAMS 5      /* actuation parameters per scene: n_groups * n_basis, or
                                      the controller's theta when ctrl_hidden > 0 */
#define MPM_INFO_CKPT_EVERY 6      /* the checkpoint interval k in use */
#define MPM_INFO_GATHER_BOXES 8    /* forward gathers (one per CTA and G2P pass) since the last
                                      mpm_set_initial, and of them ... (waits for the handle's
                                      last stream) */
#define MPM_INFO_GATHER_BOX_OVERFLOWS 9 /* ... those whose stencil box exceeded the shared gather
                                      box (MPM_OPT_GATHER_CAPACITY) and read the grid through L1:
                                      the particle order's decay as a body flows */
#define MPM_INFO_POLAR_FP64 7      /* 1: this library was built with MPM_POLAR_FP64=1 (the
                                      fixed-corotated polar refinement and adjoint in FP64);
                                      0: compensated FP32 refinement, FP32 adjoint */

typedef struct mpm_handle mpm_handle;

/* Scene description, copied at create.  Every scene of a batch shares these
 * scalars; each has its own dense n_grid^dim grid on [0,1]^dim. */
typedef struct mpm_scene_desc {
  int32_t dim;                 /* 2 or 3 */
  int32_t n_grid;              /* grid nodes per axis, 8..1024; dx = 1/n_grid */
  int32_t n_scenes;            /* >= 1 independent scenes */
  const int64_t* n_particles;  /* host [n_scenes], each >= 1 */
  float dt;                    /* time step */
  float gravity[3];            /* added as dt*g in the grid update */
  int32_t wall_cells;          /* sticky walls: node i with any i_k < wall or i_k >= n-wall gets v = 0 */
  int32_t material;            /* MPM_FIXED_COROTATED, MPM_NEO_HOOKEAN, MPM_LIQUID or MPM_MIXED */
  float rho;                   /* density; particle volume (dx/2)^dim, mass rho*volume */
  int32_t ckpt_every;          /* k: full state stored every k steps (Appendix D.2), >= 1; 0:
                                  ceil(sqrt(max_steps)), the interval that minimises the stored
                                  states (T/k checkpoints + k segment states, Appendix D's
                                  O(sqrt(T)) memory) */
  int32_t n_groups;            /* actuator groups, 0..8 (0 = no actuation) */
  int32_t n_basis;             /* sine terms per group, 0..8 */
  float act_period;            /* P of sin(2 pi k t / P + phase), t = step index */
  float act_phase;
  int32_t deterministic_p2g;   /* 1: every grid sum (P2G, the recomputed P2G, the velocity-
                                  adjoint scatter) is accumulated in 64-bit fixed point, so the
                                  forward and backward are bitwise reproducible whatever the
                                  order of the atomic adds (run to run, graphs or not, persistent
                                  or not).  Grids take twice the memory and four 64-bit integer
                                  adds replace one float4 add per contribution.  Scales: mass
                                  m_p -> 2^40, momentum m_p dx/dt -> 2^40, velocity adjoint: its
                                  first scatter's largest contribution -> below 2^36 (a measuring
                                  pass per backward); a contribution beyond 2^55 is refused with
                                  MPM_ERR_RANGE.  The shared scatter box is not used.  0: FP32
                                  atomic sums (default, faster).  No counterpart in the paper,
                                  whose GPU atomics are order-dependent as well. */
  int32_t ctrl_hidden;         /* 0: open-loop sine actuation (w = sine weights).  H in 1..64:
                                  closed-loop controller with H hidden units, evaluated at every
                                  step on the current state: inputs u = [sin(2 pi k t / P +
                                  phase), k = 1..n_basis] followed, for each group g, by the
                                  offset of g's centre of mass from the scene's (dim values) and
                                  g's mean velocity (dim values; an empty group reads zeros);
                                  h = tanh(W1 u + b1), a_g = ctrl_scale tanh(W2 h + b2)_g.  w is
                                  then theta = [W1 (H x n_in, row-major) | b1 (H) | W2 (n_groups x
                                  H) | b2 (n_groups)] per scene, n_in = n_basis + 2 dim n_groups
                                  (MPM_INFO_ACT_PARAMS gives the count).  Needs n_groups >= 1;
                                  n_basis may be 0.  The forward splits each fused particle pass
                                  around the controller, the backward each fused adjoint pass
                                  around its reverse; the persistent form is not used. */
  float ctrl_scale;            /* controller output scale (ctrl_hidden > 0) */
  int32_t ckpt_coarse;         /* 0 or 1: one level of checkpoints (every k = ckpt_every steps).
                                  M >= 2: two levels -- the forward keeps the state every k*M
                                  steps only, and mpm_backward re-simulates each such coarse
                                  segment once to rebuild its states every k steps before the
                                  usual per-segment re-simulation: about T/(kM) + M + 2k states
                                  stored instead of T/k + 2k, for one more forward's worth of
                                  re-simulation (Appendix D's recursive checkpointing, one level
                                  deeper).  The re-simulation then runs on the main stream. */
} mpm_scene_desc;

/* Device bytes the workspace needs for this description and at most max_steps
 * steps per forward (checkpoints, one segment buffer, adjoints, four grids per
 * scene, sort scratch).  out_bytes: host. */
int mpm_workspace_bytes(const mpm_scene_desc* desc, int32_t max_steps, size_t* out_bytes);

/* Create a handle.  workspace: device, >= mpm_workspace_bytes bytes, 256-byte
 * aligned, owned by the caller.  out: host, receives the handle. */
int mpm_create(const mpm_scene_desc* desc, void* workspace, size_t workspace_bytes,
               int32_t max_steps, mpm_handle** out);

/* Copy the initial state in (device pointers, component-major, N particles).
 * C0 may be NULL (zero), F0 NULL (identity).  E, nu: Young's modulus and Poisson
 * ratio per particle.  group: int32 [N] actuator group in [0, n_groups) (NULL if
 * n_groups == 0); w: float [n_scenes][n_groups][n_basis] actuation weights, or
 * [n_scenes][MPM_INFO_ACT_PARAMS] controller parameters theta when ctrl_hidden > 0.
 * Particles are reordered internally by a spatial (Morton) key per scene so that
 * P2G tiles are compact; all outputs come back in the caller's order.
 * Invalidates any recorded forward. */
int mpm_set_initial(mpm_handle* h, const float* x0, const float* v0, const float* C0,
                    const float* F0, const float* E, const float* nu, const int32_t* group,
                    const float* w, void* stream);

/* MPM_MIXED scenes: the material of every particle (device int32 [N], caller order:
 * MPM_FIXED_COROTATED, MPM_NEO_HOOKEAN or MPM_LIQUID), copied in and permuted like the
 * state.  Call after each mpm_set_initial and before mpm_forward (which otherwise fails
 * with MPM_ERR_STATE); discards any recorded forward.  MPM_ERR_ARG when the scene is not
 * MPM_MIXED or material is NULL.  The paper couples its 3D robot with its liquid simulator
 * in one grid; its own API has no separate call for this (materials are fields there). */
int mpm_set_particle_materials(mpm_handle* h, const int32_t* material, void* stream);

/* Run T steps (1 <= T <= max_steps) from the initial state and record the tape.
 * Stores the full state at steps 0, k, 2k, ... (k = ckpt_every). */
int mpm_forward(mpm_handle* h, int32_t T, void* stream);

/* Copy the state at step T of the last forward to caller buffers (device,
 * component-major, caller order).  Any pointer may be NULL. */
int mpm_get_state(mpm_handle* h, float* x, float* v, float* C, float* F, void* stream);

/* Centre-of-mass loss of every scene on the state at step T (FP64 accumulation).
 * target: device float [n_scenes][dim] (MPM_LOSS_COM_TARGET; else may be NULL).
 * loss: device float [n_scenes].  dL_dxT: device float [dim][N], the seed of
 * dL/dx_T.  dL_dx0: device float [dim][N] or NULL, the direct dependence of the
 * loss on x_0 (nonzero only for MPM_LOSS_COM_X_DISP; add it to mpm_backward's gx0). */
int mpm_loss(mpm_handle* h, int32_t kind, const float* target, float* loss, float* dL_dxT,
             float* dL_dx0, void* stream);

/* Reverse pass of the last forward (the tape is replayed in reverse, Section 3.2):
 * given dL/dstate_T (device, caller order; any of the four may be NULL = zero),
 * write dL/dstate_0 (gx0, gv0, gC0, gF0: device [dim|dim*dim][N]), dL/dE and dL/dnu
 * (device [N]) and dL/dw (device [n_scenes][n_groups][n_basis], or dL/dtheta
 * [n_scenes][MPM_INFO_ACT_PARAMS] with the controller).  Any output may be NULL.  May
 * be called more than once per forward. */
int mpm_backward(mpm_handle* h, const float* dL_dx, const float* dL_dv, const float* dL_dC,
                 const float* dL_dF, float* gx0, float* gv0, float* gC0, float* gF0,
                 float* gE, float* gnu, float* gw, void* stream);

/* Wait for the handle's last stream and return the first sticky device error
 * (MPM_OK, MPM_ERR_OOB, MPM_ERR_NONFINITE, MPM_ERR_TIMEOUT) or MPM_ERR_CUDA;
 * clears the device error word. */
int mpm_sync_status(mpm_handle* h);

/* Set a tuning knob (MPM_OPT_*); drops any cached CUDA graphs. */
int mpm_set_option(mpm_handle* h, int32_t key, int64_t value);

/* Read a counter (MPM_INFO_*). value: host. */
int mpm_get_info(mpm_handle* h, int32_t key, int64_t* value);

/* Timings collected while MPM_OPT_PROFILE is on: launches of kernel category
 * `kind` (MPM_KERNEL_*) and their summed device time in milliseconds.  Waits for the
 * recorded events.  launches, total_ms: host. */
int mpm_get_profile(mpm_handle* h, int32_t kind, int64_t* launches, double* total_ms);

/* Diagnostics (sub-stage tests): the (m, p) grid that P2G scatters from the initial state
 * (the first pass of a forward), copied densely to grid: device float [n_scenes][n_grid^dim]
 * [4] = (m, p_0, .., p_{dim-1}, 0 ...), node (i0, i1[, i2]) at (i0 n + i1)[n + i2].  Needs
 * mpm_set_initial; leaves any recorded forward intact.  MPM_ERR_ARG in the deterministic mode
 * (its grids are fixed point) or with a controller. */
int mpm_initial_p2g_grid(mpm_handle* h, float* grid, void* stream);

/* Checkpoint schedule for a workspace budget (the memory/recompute trade of Appendix D.2,
 * generalised to two levels): among intervals k (every k up to 4096, powers of two, and
 * max_steps itself, which re-simulates nothing) and second-level multipliers M (1, i.e. one
 * level, or 2..1024), the schedule whose mpm_workspace_bytes fits budget_bytes with the
 * fewest particle passes per forward + backward: 2T, plus the steps before the last
 * segment's start (re-simulated once), plus those before the last coarse segment's start
 * for a second level, plus T/2 when a segment's grids cannot be kept (every adjoint
 * pass then recomputes a P2G pass); ties go to the smaller workspace.  desc: host (its
 * ckpt_every and ckpt_coarse are ignored); outputs: host, the values to put in
 * desc->ckpt_every and desc->ckpt_coarse and the resulting workspace bytes (ws_bytes may be
 * NULL).  Host-only arithmetic, no GPU needed.  Returns MPM_OK, MPM_ERR_ARG, or
 * MPM_ERR_WORKSPACE when no schedule fits. */
int mpm_plan_checkpoints(const mpm_scene_desc* desc, int32_t max_steps, size_t budget_bytes,
                         int32_t* ckpt_every, int32_t* ckpt_coarse, size_t* ws_bytes);

/* Peaks of the current GPU, measured with the library's own kernels (best of three timed
 * launches after a warm-up, CUDA events on `stream`, 8 CTAs of 256 threads per SM), the
 * denominators of the ALU and scatter rooflines of the particle passes.  kind:
 *   MPM_PEAK_FP64_FMA / MPM_PEAK_FP32_FMA: FLOP/s of 8 independent fused multiply-add
 *     chains per thread (an FMA counts 2 FLOP);
 *   MPM_PEAK_RED_F32X4: float4 reductions per second (atomicAdd(float4*), result unused)
 *     into an L2-resident array of 2^18 nodes, the 32 lanes of an instruction on 32
 *     consecutive nodes (4 cache lines: the best case);
 *   MPM_PEAK_RED_F32X4_SPREAD: the same with the 32 lanes on 32 different cache lines.
 * flops_per_s (host) receives the rate.  The reduction kernels write a fixed 4 MiB device
 * array of the library (no allocation).  Blocks until the launches finish (a diagnostic,
 * ~0.1 s).  Returns MPM_OK, MPM_ERR_ARG or MPM_ERR_CUDA (message in mpm_last_error(NULL)). */
#define MPM_PEAK_FP64_FMA 0
#define MPM_PEAK_FP32_FMA 1
#define MPM_PEAK_RED_F32X4 2
#define MPM_PEAK_RED_F32X4_SPREAD 3
int mpm_measure_peak(int32_t kind, double* flops_per_s, void* stream);

/* Message of the last failure on this handle (static storage if h is NULL). */
const char* mpm_last_error(mpm_handle* h);

/* Destroy the handle (host objects and CUDA graphs; the workspace stays the caller's). */
void mpm_destroy(mpm_handle* h);

/* ---------------------------------------------------------------------------
 * mpm_step_noalloc -- one forward MLS-MPM step with no workspace and no allocation.
 * The paper has no counterpart: this entry point exists for callers that cannot
 * allocate device memory at all -- code embedded in a host application that owns the
 * device memory budget and forbids allocation after start-up (plugins, real-time
 * control loops where an allocation could stall or fail), or a small C caller with no
 * allocator to hand for a workspace.  It calls no cudaMalloc, cudaFree or allocating
 * library routine.
 *
 * The grid scratch lives in one fixed device array inside the library (about 6 MiB:
 * one float4 grid of MPM_NOALLOC_MAX_NODES nodes plus per-particle Lame parameters and
 * the tile table), held by every GPU that loads the library until the process exits.
 * Limits: one scene, no actuation, n_grid^dim <= MPM_NOALLOC_MAX_NODES and
 * n_particles[0] <= MPM_NOALLOC_MAX_PARTICLES; larger problems return
 * MPM_ERR_TOO_LARGE and launch nothing.
 *
 * desc: host; dim, n_grid, n_scenes (must be 1), n_particles[0], dt, gravity,
 *   wall_cells, material and rho are used (ckpt_every is ignored, n_groups must be 0).
 * state_in / state_out: device float, one component-major block [Q][N] with
 *   Q = 2 dim + 2 dim^2 rows in the order x, v, C, F (C and F row-major per
 *   particle); state_in holds step s, state_out receives step s+1 (distinct buffers).
 * E, nu: device float [N].  device_err: device uint32 or NULL; when given, the
 *   step ORs its device error bits into it (1 = a stencil left the grid, 2 =
 *   non-finite value or det F <= 0); when NULL those bits go to the fixed array
 *   and are not reported.  A particle whose stencil leaves the grid is skipped by
 *   the kernels' own bounds check (no access outside the grid) and sets bit 1.
 * Results equal mpm_forward with T = 1 up to FP32 atomic-order rounding, and one more
 *   rounding: the rows hold F itself, and each call forms F - I in FP32 and adds I back,
 *   so a caller that chains calls rounds the small strain to FP32's spacing near 1 on
 *   every step (the workspace path keeps F - I between steps and does not).
 *
 * Set-up and memory: CUDA loads modules lazily, so the device memory of the fixed array
 * and the modules of the step kernels are committed on first use.  A call with
 * n_particles[0] == 0 (the pointers may then be any non-NULL values; nothing is read or
 * written) does only that set-up for desc's dim and material and returns MPM_OK: make
 * it at start-up, before the caller's memory budget is spent and before any stream
 * capture, once per device and per (dim, material) to be used.  Without it the first
 * real call on a device does the set-up.  The device address of the array is looked up
 * (cudaGetSymbolAddress, no allocation) on every call, with the calling thread's
 * current device and context.  Every call on a device shares the one array and each
 * call clears what must start at zero; calls that overlap on the GPU (two streams, or
 * two threads) race on it and must be serialised by the caller.
 * Returns MPM_OK, MPM_ERR_ARG, MPM_ERR_TOO_LARGE or MPM_ERR_CUDA; on failure
 * mpm_last_error(NULL) names the check or the CUDA call that failed (this host thread). */
#define MPM_NOALLOC_MAX_NODES (1 << 18)     /* 64^3 in 3D, 512^2 in 2D */
#define MPM_NOALLOC_MAX_PARTICLES (1 << 18) /* 262,144 */
int mpm_step_noalloc(const mpm_scene_desc* desc, const float* state_in, const float* E,
                     const float* nu, float* state_out, uint32_t* device_err, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MPM_H_ */
