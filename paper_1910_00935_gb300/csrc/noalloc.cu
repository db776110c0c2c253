// noalloc.cu -- mpm_step_noalloc: one MLS-MPM step of one scene with no workspace.
//
// For callers that cannot allocate device memory at all: code embedded in a host
// application that owns the whole device memory budget and forbids allocation after
// start-up (plugins, real-time control loops where an allocation could stall or fail),
// and small C callers that have no allocator to hand for a workspace.  Such a caller
// passes only its inputs and outputs; the grid scratch of the step lives in the
// file-scope array below, which every GPU that loads the library holds until the
// process exits.
//
// The step runs the library's own kernels (P2G from the full input state, then G2P
// writing the full output state, grid_op applied as it gathers) with pointers into that
// array, so its results equal those of mpm_forward with T = 1 up to FP32 atomic-order
// rounding and the rounding of F - I noted in mpm.h.
//
// Device memory for the array, and the kernels' modules, are committed when they are first
// used (CUDA loads modules lazily): a call with n_particles[0] == 0 does only that set-up,
// so a caller can make it at start-up, before its memory budget is spent and before any
// stream capture.
#include <climits>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/mpm.h"
#include "mpm_internal.h"
#include "mpm_kernels.cuh"

using namespace mpm;

namespace {

constexpr int64_t kMaxNodes = MPM_NOALLOC_MAX_NODES;
constexpr int64_t kMaxParticles = MPM_NOALLOC_MAX_PARTICLES;
constexpr int64_t kMaxTiles = (kMaxParticles + kTile - 1) / kTile;

// byte offsets inside the scratch array (each 256-byte aligned)
constexpr size_t kOffPM = 0;                                    // float4 (m, p) per node
constexpr size_t kOffMu = kOffPM + (size_t)kMaxNodes * 16;     // float per particle
constexpr size_t kOffLa = kOffMu + (size_t)kMaxParticles * 4;  // float per particle
constexpr size_t kOffTiles = kOffLa + (size_t)kMaxParticles * 4;
constexpr size_t kOffMisc = kOffTiles + (size_t)kMaxTiles * 16;  // box[8], tile count, err
constexpr size_t kScratchBytes = kOffMisc + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
bool g_setup_done[kMaxDevices] = {};

__global__ void noalloc_prepare_kernel(int64_t N, const float* E, const float* nu, float* mu,
                                       float* la, int4* tiles, int* n_tiles, int* box) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    float e = E[i], v = nu[i];
    mu[i] = e / (2.0f * (1.0f + v));
    la[i] = e * v / ((1.0f + v) * (1.0f - 2.0f * v));
    if (i % kTile == 0) {
      int64_t cnt = N - i < kTile ? N - i : kTile;
      tiles[i / kTile] = make_int4(0, (int)i, (int)cnt, (int)(i / kTile));
    }
  }
  if (blockIdx.x == 0 && threadIdx.x < 8) {
    box[threadIdx.x] = (threadIdx.x & 4) ? INT_MIN : INT_MAX;
    if (threadIdx.x == 0) *n_tiles = (int)((N + kTile - 1) / kTile);
  }
}

// a rejection's message goes where mpm_last_error(NULL) reads it (this host thread)
int reject(int code, const char* why) {
  set_static_error(why);
  return code;
}

// message of a failed CUDA call
int reject_cuda(const char* where, cudaError_t e) {
  std::string m = std::string("mpm_step_noalloc: ") + where + ": " + cudaGetErrorString(e);
  set_static_error(m.c_str());
  return MPM_ERR_CUDA;
}

}  // namespace

extern "C" int mpm_step_noalloc(const mpm_scene_desc* d, const float* state_in, const float* E,
                                const float* nu, float* state_out, uint32_t* device_err,
                                void* stream) {
  if (!d || !state_in || !E || !nu || !state_out)
    return reject(MPM_ERR_ARG, "mpm_step_noalloc: NULL argument");
  if (d->dim != 2 && d->dim != 3) return reject(MPM_ERR_ARG, "mpm_step_noalloc: dim must be 2 or 3");
  if (d->n_scenes != 1 || !d->n_particles)
    return reject(MPM_ERR_ARG, "mpm_step_noalloc: exactly one scene");
  if (d->n_groups != 0 || d->ctrl_hidden != 0) return reject(MPM_ERR_ARG, "mpm_step_noalloc: no actuation");
  if (d->deterministic_p2g != 0)
    return reject(MPM_ERR_ARG, "mpm_step_noalloc: the deterministic mode needs the workspace form");
  if (d->material != MPM_FIXED_COROTATED && d->material != MPM_NEO_HOOKEAN &&
      d->material != MPM_LIQUID)
    return reject(MPM_ERR_ARG, "mpm_step_noalloc: unknown material");
  if (d->n_grid < 8 || !(d->dt > 0.0f) || !(d->rho > 0.0f) || d->wall_cells < 0 ||
      2 * d->wall_cells >= d->n_grid)
    return reject(MPM_ERR_ARG, "mpm_step_noalloc: bad n_grid, dt, rho or wall_cells");
  int64_t nnodes = 1;
  for (int a = 0; a < d->dim; ++a) nnodes *= d->n_grid;
  const int64_t N = d->n_particles[0];
  if (N < 0) return reject(MPM_ERR_ARG, "mpm_step_noalloc: negative particle count");
  if (nnodes > kMaxNodes)
    return reject(MPM_ERR_TOO_LARGE, "mpm_step_noalloc: n_grid^dim exceeds MPM_NOALLOC_MAX_NODES");
  if (N > kMaxParticles)
    return reject(MPM_ERR_TOO_LARGE, "mpm_step_noalloc: more than MPM_NOALLOC_MAX_PARTICLES");

  // the device address of the scratch array, looked up on every call (cheap, allocates
  // nothing) so that it is always that of the current context; the first lookup on a
  // device also commits the array's memory and loads this file's module
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return reject(MPM_ERR_CUDA, "mpm_step_noalloc: no current CUDA device");
  }
  void* scratch = nullptr;
  e = cudaGetSymbolAddress(&scratch, g_noalloc_scratch);
  if (e != cudaSuccess || !scratch) {
    cudaGetLastError();
    return reject_cuda("cudaGetSymbolAddress", e);
  }
  char* base = static_cast<char*>(scratch);

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  {
    // set-up: once per device, load the modules of the two step kernels this problem
    // launches (a zero-tile launch only loads); a call with no particles stops here
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_setup_done[dev] || N == 0) {
      SimParams Q;
      memset(&Q, 0, sizeof(Q));
      Q.tile_capacity = 1024;
      StepArgs Z;
      memset(&Z, 0, sizeof(Z));
      e = d->dim == 2 ? launch_step<2>(d->material, kP2GOnly, Q, Z, 0, s)
                      : launch_step<3>(d->material, kP2GOnly, Q, Z, 0, s);
      if (e == cudaSuccess)
        e = d->dim == 2 ? launch_step<2>(d->material, kG2POnlyFull, Q, Z, 0, s)
                        : launch_step<3>(d->material, kG2POnlyFull, Q, Z, 0, s);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return reject_cuda("loading the step kernels", e);
      }
      g_setup_done[dev] = true;
    }
  }
  if (N == 0) return MPM_OK;

  float4* PM = reinterpret_cast<float4*>(base + kOffPM);
  float* mu = reinterpret_cast<float*>(base + kOffMu);
  float* la = reinterpret_cast<float*>(base + kOffLa);
  int4* tiles = reinterpret_cast<int4*>(base + kOffTiles);
  int* box = reinterpret_cast<int*>(base + kOffMisc);
  int* n_tiles_dev = box + 8;
  unsigned* err = device_err ? reinterpret_cast<unsigned*>(device_err)
                             : reinterpret_cast<unsigned*>(box + 9);

  // the array keeps the previous call's contents: clear what must start at zero (the
  // mass/momentum grid; the prepare kernel rewrites the box, tiles and Lame parameters)
  e = cudaMemsetAsync(PM, 0, (size_t)nnodes * sizeof(float4), s);
  if (e == cudaSuccess && !device_err) e = cudaMemsetAsync(err, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) {
    int blocks = (int)((N + 255) / 256);
    noalloc_prepare_kernel<<<blocks, 256, 0, s>>>(N, E, nu, mu, la, tiles, n_tiles_dev, box);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return reject_cuda("clearing the grid", e);

  SimParams P;
  memset(&P, 0, sizeof(P));
  P.n_grid = d->n_grid;
  P.nnodes = (int)nnodes;
  P.dx = 1.0f / (float)d->n_grid;
  P.inv_dx = (float)d->n_grid;
  P.dt = d->dt;
  for (int a = 0; a < 3; ++a) P.gravity[a] = d->gravity[a];
  P.wall = d->wall_cells;
  const double dx = 1.0 / d->n_grid;
  const double vol = d->dim == 2 ? 0.25 * dx * dx : 0.125 * dx * dx * dx;
  P.p_mass = (float)(d->rho * vol);
  P.kappa = (float)(-(double)d->dt * vol * 4.0 / (dx * dx));
  P.tile_capacity = 1024;
  P.f_diag = 1.0f;  // the caller's state rows hold F itself
  P.node_words = 1;

  StepArgs A;
  memset(&A, 0, sizeof(A));
  A.tiles = tiles;
  A.scene_tiles = n_tiles_dev;
  A.N = (int)N;
  A.in = state_in;
  A.out = state_out;
  A.mu = mu;
  A.la = la;
  A.PMw = PM;  // P2G pass
  A.box_w = box;
  A.err = err;
  const int n_tiles = (int)((N + kTile - 1) / kTile);
  StepArgs G = A;  // G2P pass reads the same grid
  G.PMr = PM;
  G.PMw = nullptr;
  G.box_w = nullptr;
  if (d->dim == 2) {
    e = launch_step<2>(d->material, kP2GOnly, P, A, n_tiles, s);
    if (e == cudaSuccess) e = launch_step<2>(d->material, kG2POnlyFull, P, G, n_tiles, s);
  } else {
    e = launch_step<3>(d->material, kP2GOnly, P, A, n_tiles, s);
    if (e == cudaSuccess) e = launch_step<3>(d->material, kG2POnlyFull, P, G, n_tiles, s);
  }
  if (e != cudaSuccess) return reject_cuda("launching the step", e);
  set_static_error("");
  return MPM_OK;
}
