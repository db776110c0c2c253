// mpm_api.cu -- the C ABI of libmpm.so (declared in include/mpm.h): workspace
// layout, handle, and the light-weight tape of Section 3.2 with the checkpointing
// of Appendix D.
//
// Tape.  The forward of T steps only records T (and therefore the actuation time
// of every step); the particle state itself is stored every k = ckpt_every steps
// (Appendix D.2, segment-wise recomputation).  The backward walks s = T-1 .. 0;
// entering a segment it re-simulates the segment from its checkpoint into one
// segment buffer; then each adjoint pass runs [P2G-adjoint of step s+1 | G2P-adjoint
// of step s | recomputed P2G of step s-1] -- the grid of each step is recomputed once,
// one pass before it is needed (Appendix D.1).  One particle pass per step in every
// phase; grid_op and its adjoint are applied by the consuming pass.
//
// Grids.  The per-step grids are accumulation buffers from two rings (mass/momentum,
// velocity adjoint) managed on the host: a pass scatters into a free clean buffer, the
// buffer stays live until its last reader, and the next pass zeroes its recorded box.
// Each buffer has two parity boxes so that resetting a box never races with a reader.
// Every launch sequence starts and ends with all buffers clean.
//
// Launch sequences are captured into CUDA graphs (one per forward length T and one
// per backward length), cached on the handle and replayed on the caller's stream.
//
// Persistent form (MPM_OPT_PERSISTENT).  The same issue code runs first in record mode,
// which collects every pass (kernel parameters included) into a plan; the plan is copied
// to the workspace when it differs from the copy already there, and the sequence then
// runs each maximal run of same-kind passes as one cooperative launch that steps
// through the plan with a bounded grid barrier between passes: one launch for a forward,
// two per segment for a backward.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/mpm.h"
#include "mpm_internal.h"
#include "mpm_kernels.cuh"

using namespace mpm;

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

constexpr int kPMSlots = 6;  // mass/momentum grids in flight (measured need: 4)
constexpr int kUBSlots = 4;  // velocity-adjoint grids in flight (need: 3)
// Grids of a re-simulated segment are kept for its adjoint passes (instead of each adjoint
// pass recomputing the grid of the step before, Appendix D.1) when two pools of K + 3 grid
// buffers (one per segment parity, see issue_backward_overlap) fit this budget; otherwise
// the per-step recompute is used.
constexpr size_t kStoredGridBudget = (size_t)16 << 30;

struct Layout {
  size_t perm, keys0, keys1, idx0, sort_tmp, sort_tmp_bytes;
  size_t tiles, scene_off, scene_tiles, scene_tile_off;
  size_t mu, la, E, nu, group, matid, wact, wbar_tile, mubar, labar;
  size_t fin, cur, ckpt, fine, seg, adj;
  size_t rcache;  // 2 x (K+1) x [9][N] polar factors of a segment (3D FCR; R_hi, R_lo as FP32 pairs), by parity
  size_t grids;  // pm_slots + kUBSlots dense grids
  size_t boxes;  // (pm_slots + kUBSlots) x 2 parities x [scene][8]
  size_t err, box_stats, com, com_part, ub_m0;
  size_t plan_fwd, plan_bwd, gsync;  // persistent-form pass plans and barrier counters
  // closed-loop controller: per-tile sensor sums, per-step inputs / hidden / outputs /
  // actuation, group sizes, dL/dtheta (FP64) and the per-slot sensor adjoints
  size_t ctrl_part, ctrl_u, ctrl_h, ctrl_y, act_tab, ctrl_cnt, ctrl_thbar, ctrl_add;
  size_t total;
};

struct Dims {
  int D, Q, S, K, n_ckpt, n_tiles, n_grid;
  int M;  // coarse checkpoint multiplier: 1 (one level) or >= 2 (states every K*M, then K)
  int64_t N, nnodes;
  bool polar_cache;  // 3D fixed-corotated: polar factors are cached per segment
  bool store_grids;  // a re-simulated segment's grids stay live for its adjoint passes
  int pm_slots;      // (m, p) grid buffers: two pools of pm_pool
  int pm_pool;       // kPMSlots, or K + 3 when store_grids
  int words;         // float4 slots per grid node: 2 for fixed-point grids (deterministic)
  int T_max;         // max_steps
  int G;             // actuation groups
  int ctrl_H;        // controller hidden units (0: open-loop sine actuation)
  int ctrl_in;       // controller inputs K + 2 D G
  int64_t n_act;     // actuation parameters per scene: G K (open loop) or the controller's
};

// passes of the longest forward (T + 1) and backward (re-simulation T + segments, adjoint
// T + 1, plus the measuring pass of the deterministic mode) sequences
int64_t plan_fwd_cap(const Dims& m) { return (int64_t)m.T_max + 1; }
int64_t plan_bwd_cap(const Dims& m) { return 3 * (int64_t)m.T_max + m.n_ckpt + 2; }

bool valid_desc(const mpm_scene_desc* d, int32_t max_steps, std::string* why) {
  auto fail = [&](const char* m) {
    if (why) *why = m;
    return false;
  };
  if (!d) return fail("desc is NULL");
  if (d->dim != 2 && d->dim != 3) return fail("dim must be 2 or 3");
  if (d->n_grid < 8 || d->n_grid > 1024) return fail("n_grid must be in [8, 1024]");
  if (d->n_scenes < 1 || d->n_scenes > 65535) return fail("n_scenes must be in [1, 65535]");
  if (!d->n_particles) return fail("n_particles is NULL");
  int64_t N = 0;
  for (int s = 0; s < d->n_scenes; ++s) {
    if (d->n_particles[s] < 1) return fail("every scene needs >= 1 particle");
    N += d->n_particles[s];
  }
  if (N > (int64_t)INT32_MAX / 32) return fail("too many particles");
  if (!(d->dt > 0.0f) || !std::isfinite(d->dt)) return fail("dt must be > 0");
  if (d->wall_cells < 0 || 2 * d->wall_cells >= d->n_grid) return fail("bad wall_cells");
  if (d->material != MPM_FIXED_COROTATED && d->material != MPM_NEO_HOOKEAN &&
      d->material != MPM_LIQUID && d->material != MPM_MIXED)
    return fail("unknown material");
  if (!(d->rho > 0.0f)) return fail("rho must be > 0");
  if (d->ckpt_every < 0) return fail("ckpt_every must be >= 0 (0: ceil(sqrt(max_steps)))");
  if (d->ckpt_coarse < 0 || d->ckpt_coarse > 4096) return fail("ckpt_coarse must be in [0, 4096]");
  if (d->n_groups < 0 || d->n_groups > kMaxGroups) return fail("n_groups must be in [0, 8]");
  if (d->n_basis < 0 || d->n_basis > kMaxBasis) return fail("n_basis must be in [0, 8]");
  if (d->ctrl_hidden < 0 || d->ctrl_hidden > kCtrlMaxHidden)
    return fail("ctrl_hidden must be in [0, 64]");
  if (d->ctrl_hidden > 0) {
    if (d->n_groups < 1) return fail("the controller needs n_groups >= 1");
    if (!std::isfinite(d->ctrl_scale)) return fail("ctrl_scale must be finite");
    if (d->n_basis > 0 && !(d->act_period != 0.0f)) return fail("time inputs need act_period != 0");
  } else if (d->n_groups > 0 && (d->n_basis < 1 || !(d->act_period != 0.0f))) {
    return fail("actuation needs n_basis >= 1 and act_period != 0");
  }
  if (d->deterministic_p2g != 0 && d->deterministic_p2g != 1) return fail("deterministic_p2g must be 0 or 1");
  if (max_steps < 1) return fail("max_steps must be >= 1");
  if (max_steps > (1 << 24)) return fail("max_steps too large");
  return true;
}

Dims make_dims(const mpm_scene_desc* d, int32_t max_steps) {
  Dims m;
  m.D = d->dim;
  m.Q = 2 * m.D + 2 * m.D * m.D;
  m.S = d->n_scenes;
  // 0: the interval that minimises the stored states, T/k checkpoints + k segment states
  // (Appendix D's O(sqrt(T)) memory)
  int k = d->ckpt_every;
  if (k == 0) k = (int)std::ceil(std::sqrt((double)max_steps));
  m.K = k < max_steps ? k : max_steps;
  m.M = d->ckpt_coarse >= 2 ? d->ckpt_coarse : 1;
  m.n_ckpt = (max_steps - 1) / (m.K * m.M) + 1;  // states 0, KM, 2KM, ... < max_steps
  m.n_grid = d->n_grid;
  m.polar_cache = d->dim == 3 && (d->material == MPM_FIXED_COROTATED || d->material == MPM_MIXED);
  m.T_max = max_steps;
  m.words = d->deterministic_p2g ? 2 : 1;
  m.G = d->n_groups;
  m.ctrl_H = d->ctrl_hidden;
  m.ctrl_in = d->ctrl_hidden > 0 ? d->n_basis + 2 * d->dim * d->n_groups : 0;
  m.n_act = d->ctrl_hidden > 0
                ? (int64_t)m.ctrl_H * m.ctrl_in + m.ctrl_H + (int64_t)m.G * m.ctrl_H + m.G
                : (int64_t)d->n_groups * d->n_basis;
  {
    int64_t nn = 1;
    for (int a = 0; a < d->dim; ++a) nn *= d->n_grid;
    const size_t grid_bytes = (size_t)d->n_scenes * nn * 16 * m.words;
    m.store_grids = (size_t)2 * std::max(m.K + 3, kPMSlots) * grid_bytes <= kStoredGridBudget;
    m.pm_pool = m.store_grids ? std::max(m.K + 3, kPMSlots) : kPMSlots;
    m.pm_slots = 2 * m.pm_pool;
  }
  m.nnodes = 1;
  for (int a = 0; a < m.D; ++a) m.nnodes *= d->n_grid;
  m.N = 0;
  m.n_tiles = 0;
  for (int s = 0; s < m.S; ++s) {
    m.N += d->n_particles[s];
    m.n_tiles += (int)((d->n_particles[s] + kTile - 1) / kTile);
  }
  return m;
}

Layout make_layout(const Dims& m) {
  Layout L;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align_up(o + (bytes ? bytes : 1));
    return at;
  };
  const size_t N = (size_t)m.N, Q = (size_t)m.Q, S = (size_t)m.S;
  L.perm = take(N * 4);
  L.keys0 = take(N * 8);
  L.keys1 = take(N * 8);
  L.idx0 = take(N * 4);
  L.sort_tmp_bytes = sort_temp_bytes(m.N);
  L.sort_tmp = take(L.sort_tmp_bytes);
  L.tiles = take((size_t)m.n_tiles * sizeof(int4));
  L.scene_off = take((S + 1) * 8);
  L.scene_tiles = take(S * 4);
  L.scene_tile_off = take((S + 1) * 4);
  L.mu = take(N * 4);
  L.la = take(N * 4);
  L.E = take(N * 4);
  L.nu = take(N * 4);
  L.group = take(N * 4);
  L.matid = take(N * 4);
  L.wact = take(S * (size_t)std::max<int64_t>(kMaxGroups * kMaxBasis, m.n_act) * 4);
  L.wbar_tile = take((size_t)m.n_tiles * kMaxGroups * kMaxBasis * 4);
  L.mubar = take(N * 8);  // compensated FP32 sums over the steps (see AdjArgs::mubar)
  L.labar = take(N * 8);
  L.fin = take(Q * N * 4);
  L.cur = take(Q * N * 4);
  L.ckpt = take((size_t)m.n_ckpt * Q * N * 4);
  L.fine = take(m.M > 1 ? (size_t)m.M * Q * N * 4 : 0);  // states every K of one coarse segment
  L.seg = take((size_t)2 * (m.K + 1) * Q * N * 4);  // two segment buffers (by parity)
  L.adj = take(Q * N * 4);
  L.rcache = m.polar_cache ? take((size_t)2 * (m.K + 1) * 9 * N * 8) : take(0);
  const size_t grid = S * (size_t)m.nnodes * sizeof(float4) * m.words;
  L.grids = take(grid * (m.pm_slots + kUBSlots));
  L.boxes = take((size_t)(m.pm_slots + kUBSlots) * 2 * S * 8 * 4);
  L.err = take(4);
  L.box_stats = take(16);
  L.ub_m0 = take(4);
  L.com = take(S * 6 * 8);
  L.com_part = take(com_scratch_doubles(m.S) * 8);
  L.plan_fwd = take((size_t)plan_fwd_cap(m) * sizeof(PassEntry));
  L.plan_bwd = take((size_t)plan_bwd_cap(m) * sizeof(PassEntry));
  // barrier counters, then one tile-ticket counter per pass of the longest plan
  L.gsync = take(16 + 4 * (size_t)std::max(plan_fwd_cap(m), plan_bwd_cap(m)));
  {
    const bool c = m.ctrl_H > 0;
    const size_t steps = (size_t)m.T_max + 1, slots = (size_t)kMaxGroups + 1;
    L.ctrl_part = take(c ? (size_t)m.n_tiles * slots * 7 * 8 : 0);
    L.ctrl_u = take(c ? steps * S * m.ctrl_in * 8 : 0);
    L.ctrl_h = take(c ? steps * S * m.ctrl_H * 8 : 0);
    L.ctrl_y = take(c ? steps * S * m.G * 8 : 0);
    L.act_tab = take(c ? steps * S * m.G * 4 : 0);
    L.ctrl_cnt = take(c ? S * slots * 8 : 0);
    L.ctrl_thbar = take(c ? S * (size_t)m.n_act * 8 : 0);
    L.ctrl_add = take(c ? S * slots * 6 * 4 : 0);
  }
  L.total = o;
  return L;
}

}  // namespace

struct mpm_handle {
  mpm_scene_desc desc;
  std::vector<int64_t> n_particles;
  int32_t max_steps = 0;
  Dims m;
  Layout L;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  int smem_optin = 0;  // the device's per-CTA shared-memory limit (bytes)
  bool initialized = false;
  bool materials_set = false;  // MPM_MIXED: per-particle materials given since the last set-up
  int32_t T_recorded = 0;
  int32_t resident_T = 0;  // T of the forward whose last segment is still in the segment buffer
  // options
  bool use_graphs = true;
  bool smem_tile = false;  // measured on GB300: global float4 reductions beat shared FP32 atomics
  bool bucket_scatter = false;  // one reduction per (base, node) of a tile (measured slower: off)
  // one reduction per (pair sharing a base, node): bit 0 forward passes, bit 1 adjoint passes.
  // Off by default: it needs the base order (sort_order 1), whose tiles make the adjoint
  // passes' gathers slower than the cell order's (measured on GB300, cube3d: forward pass
  // 43.6 vs 46.3 us, adjoint 88.9 vs 77.1 us)
  int pair_scatter = 0;
  int sort_order = 0;  // particle order of mpm_set_initial: 0 cells, 1 stencil bases, 2 cells
                       // with the base on the last axis
  int tile_capacity = 1024;
  int gather_capacity = 512;  // nodes; a 128-particle tile's stencil box is ~150-300
  int grid_blocks = 0;  // CTAs per scene of the end-of-sequence grid clear (0 = automatic)
  bool use_polar_cache = true;
  bool grid_recompute = false;           // MPM_OPT_GRID_RECOMPUTE
  bool persistent = false;               // MPM_OPT_PERSISTENT
  int64_t barrier_timeout_us = 2000000;  // MPM_OPT_BARRIER_TIMEOUT_US
  unsigned barrier_extra = 0;            // MPM_OPT_BARRIER_TEST_EXTRA
  int persistent_chunk = 0;              // MPM_OPT_PERSISTENT_CHUNK (0: unlimited)
  std::vector<PassEntry> plan_copy[2];   // what the workspace plan regions hold (fwd, bwd)
  // graphs
  cudaStream_t cap_stream = nullptr;
  std::map<int64_t, std::pair<cudaGraphExec_t, int64_t>> graphs;  // key -> (exec, launches)
  int64_t launches = 0;
  // grid rings (host bookkeeping of the launch sequence being issued)
  struct Ring {
    int first;               // index of the ring's first buffer among all grid buffers
    int n;
    std::vector<int> use;    // writes so far (box parity)
    std::vector<int> state;  // 0 free, 1 live, 2 pending clear, 3 clearing in this launch
    std::vector<int> owner;  // stream (0 main, 1 side) that released it: it clears it
    int sid = 0;             // stream of the passes being issued
  } pm{0, kPMSlots, {}, {}, {}}, ub{kPMSlots, kUBSlots, {}, {}, {}};
  cudaStream_t side_stream = nullptr;  // re-simulation overlapped with the adjoint passes
  cudaEvent_t ev_fork = nullptr, ev_free = nullptr, ev_resim = nullptr, ev_join = nullptr;
  bool overlap = true;  // MPM_OPT_OVERLAP_RESIM
  // live per-launch timing (MPM_OPT_PROFILE)
  bool profile = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_records;
  std::string last_error;
  cudaStream_t last_stream = nullptr;

  template <typename T>
  T* at(size_t off) const {
    return reinterpret_cast<T*>(ws + off);
  }
  float* state(size_t base, int slot) const {
    return at<float>(base) + (size_t)slot * m.Q * m.N;
  }
  // the checkpoint of segment j (state j K): a stored checkpoint, or with two levels
  // (M > 1) a coarse one (j a multiple of M) or one rebuilt for the coarse segment being
  // processed
  float* ckpt(int j) const {
    if (m.M == 1) return state(L.ckpt, j);
    if (j % m.M == 0) return state(L.ckpt, j / m.M);
    return state(L.fine, j % m.M);
  }
  // state s0 + i of segment j (s0 = j K) in the segment buffer of j's parity
  float* seg(int j, int i) const {
    return at<float>(L.seg) + ((size_t)(j & 1) * (m.K + 1) + i) * m.Q * m.N;
  }
  // the cached polar factor of that state (3D fixed-corotated), or null
  double* rslot(int j, int i) const {
    return m.polar_cache && use_polar_cache
               ? at<double>(L.rcache) + ((size_t)(j & 1) * (m.K + 1) + i) * 9 * m.N
               : nullptr;
  }
};

namespace {

thread_local std::string g_static_error;

int fail(mpm_handle* h, int code, const std::string& msg) {
  if (h) h->last_error = msg; else g_static_error = msg;
  return code;
}

}  // namespace

void mpm::set_static_error(const char* msg) { g_static_error = msg ? msg : ""; }

static thread_local std::string g_launch_failure;
void mpm::note_launch_failure(const char* kernel, int dim, int material, int mode, size_t smem,
                              cudaError_t attr_rc) {
  char buf[256];
  snprintf(buf, sizeof(buf), " [%s<dim %d, material %d, mode %d>: %zu B dynamic shared memory%s%s]",
           kernel, dim, material, mode, smem, attr_rc != cudaSuccess ? ", raising its limit failed: " : "",
           attr_rc != cudaSuccess ? cudaGetErrorString(attr_rc) : "");
  g_launch_failure = buf;
}
std::string mpm::take_launch_failure() {
  std::string s;
  s.swap(g_launch_failure);
  return s;
}

namespace {

int cuda_fail(mpm_handle* h, cudaError_t e, const char* where) {
  return fail(h, MPM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e) + take_launch_failure());
}

#define CK(expr)                                   \
  do {                                             \
    cudaError_t e_ = (expr);                       \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #expr); \
  } while (0)

SimParams params_for(const mpm_handle* h, int t) {
  const mpm_scene_desc& d = h->desc;
  SimParams P;
  memset(&P, 0, sizeof(P));
  P.n_grid = d.n_grid;
  P.nnodes = (int)h->m.nnodes;
  P.dx = 1.0f / (float)d.n_grid;
  P.inv_dx = (float)d.n_grid;
  P.dt = d.dt;
  for (int a = 0; a < 3; ++a) P.gravity[a] = d.gravity[a];
  P.wall = d.wall_cells;
  const double dx = 1.0 / d.n_grid;
  const double vol = std::pow(0.5 * dx, (double)d.dim);
  P.p_mass = (float)(d.rho * vol);
  P.kappa = (float)(-(double)d.dt * vol * 4.0 / (dx * dx));
  P.n_groups = d.n_groups;
  P.n_basis = d.n_basis;
  const double two_pi = 6.283185307179586476925286766559;
  if (d.ctrl_hidden > 0) {
    // closed loop: a particle's actuation is its group's entry of this step's row of the
    // controller's actuation table (one "basis" value of 1)
    P.n_basis = 1;
    P.basis[0] = 1.0f;
  } else {
    for (int k = 1; k <= d.n_basis; ++k)
      P.basis[k - 1] =
          (float)std::sin(two_pi * k * (double)t / (double)d.act_period + (double)d.act_phase);
  }
  // the shared scatter box sums in FP32 in arbitrary order: not in the deterministic mode
  P.tile_capacity = h->smem_tile && !d.deterministic_p2g ? h->tile_capacity : 0;
  P.gather_capacity = h->gather_capacity;
  // the bucketed scatter sums a base's particles in FP32 registers: not in the deterministic mode
  P.bucket = h->bucket_scatter && !d.deterministic_p2g ? 1 : 0;
  P.pair = d.deterministic_p2g ? 0 : h->pair_scatter;
  P.f_diag = 0.0f;  // the workspace holds E = F - I
  P.xfix = 1;       // and positions in 32-bit fixed point
  P.det = d.deterministic_p2g;
  P.node_words = h->m.words;
  if (P.det) {
    // fixed-point scales: a particle's mass maps to 2^40, momentum at the grid speed dx/dt
    // to 2^40 (2^15 of headroom before the 2^55 limit, resolution 2^-40 of the unit)
    const int em = 40 - (std::ilogb((double)P.p_mass) + 1);
    const int ep = 40 - (std::ilogb((double)P.p_mass * (double)P.dx / (double)P.dt) + 1);
    P.fix_m = std::ldexp(1.0f, em);
    P.unfix_m = std::ldexp(1.0f, -em);
    P.fix_p = std::ldexp(1.0f, ep);
    P.unfix_p = std::ldexp(1.0f, -ep);
  }
  return P;
}

// the actuation parameters a pass reads at step t: the open-loop weights, or row t of the
// closed-loop controller's actuation table [step][scene][group]
const float* act_ptr(const mpm_handle* h, int t) {
  if (h->m.ctrl_H > 0) return h->at<float>(h->L.act_tab) + (size_t)t * h->m.S * h->m.G;
  return h->at<float>(h->L.wact);
}

CtrlStep ctrl_step(const mpm_handle* h, int t) {
  const mpm_scene_desc& d = h->desc;
  CtrlStep c;
  memset(&c, 0, sizeof(c));
  c.dim = d.dim;
  c.G = d.n_groups;
  c.K = d.n_basis;
  c.H = d.ctrl_hidden;
  c.scale = d.ctrl_scale;
  const double two_pi = 6.283185307179586476925286766559;
  for (int k = 1; k <= d.n_basis; ++k)
    c.basis[k - 1] = std::sin(two_pi * k * (double)t / (double)d.act_period + (double)d.act_phase);
  return c;
}

int grid_blocks_per_scene(const mpm_handle* h) {
  if (h->grid_blocks > 0) return h->grid_blocks;
  // enough CTAs to cover a typical active box; the kernels stride over the rest
  int64_t per_scene = 304 / h->m.S;
  if (per_scene < 2) per_scene = 2;
  if (per_scene > 256) per_scene = 256;
  return (int)per_scene;
}

// ------------------------------ grid rings ---------------------------------

using Ring = mpm_handle::Ring;

void ring_reset(Ring& r) {
  r.use.assign(r.n, 0);
  r.state.assign(r.n, 0);
  r.owner.assign(r.n, 0);
  r.sid = 0;
}

float4* ring_grid(const mpm_handle* h, const Ring& r, int id) {
  return h->at<float4>(h->L.grids) + (size_t)(r.first + id) * h->m.S * h->m.nnodes * h->m.words;
}

int* ring_box(const mpm_handle* h, const Ring& r, int id, int parity) {
  return h->at<int>(h->L.boxes) + ((size_t)(r.first + id) * 2 + (parity & 1)) * h->m.S * 8;
}

// A buffer to scatter into: its box for this use and the other parity box to reset.
struct WriteSlot {
  int id = -1;
  float4* grid = nullptr;
  int* box = nullptr;
  int* box_reset = nullptr;
};

// a free buffer among [lo, hi) (hi < 0: the whole ring)
bool ring_alloc(mpm_handle* h, Ring& r, WriteSlot& w, int lo = 0, int hi = -1) {
  if (hi < 0 || hi > r.n) hi = r.n;
  for (int i = lo; i < hi; ++i)
    if (r.state[i] == 0) {
      r.state[i] = 1;
      w.id = i;
      w.grid = ring_grid(h, r, i);
      w.box = ring_box(h, r, i, r.use[i]);
      w.box_reset = ring_box(h, r, i, r.use[i] + 1);
      return true;
    }
  return false;
}

// the buffer's last reader has been issued: it is cleared by a later launch on the same
// stream (the stream that issued the release)
void ring_release(Ring& r, int id) {
  if (id >= 0 && r.state[id] == 1) {
    r.state[id] = 2;
    r.owner[id] = r.sid;
  }
}

// Hand up to kMaxClears pending buffers released on the issuing stream to the next launch.
Clears take_clears(mpm_handle* h) {
  Clears C;
  memset(&C, 0, sizeof(C));
  C.words = h->m.words;
  for (Ring* r : {&h->pm, &h->ub})
    for (int i = 0; i < r->n && C.n < kMaxClears; ++i)
      if (r->state[i] == 2 && r->owner[i] == r->sid) {
        C.job[C.n].grid = ring_grid(h, *r, i);
        C.job[C.n].box = ring_box(h, *r, i, r->use[i]);
        ++C.n;
        r->state[i] = 3;
      }
  return C;
}

// After a launch: buffers cleared by it are clean and free again.
void after_launch(mpm_handle* h) {
  for (Ring* r : {&h->pm, &h->ub})
    for (int i = 0; i < r->n; ++i)
      if (r->state[i] == 3) {
        r->state[i] = 0;
        r->use[i] += 1;
      }
}

// ------------------------------ launch helpers ------------------------------

enum LaunchMode : int {
  kDirect = 0,     // one kernel launch per pass
  kRecord = 1,     // append every pass to *rec, launch nothing (ring bookkeeping still runs)
  kPersistent = 2  // run the recorded plan (dplan, same order) as cooperative launches
};

struct Launcher {
  mpm_handle* h;
  cudaStream_t s;
  int64_t count = 0;
  int mode = kDirect;
  std::vector<PassEntry>* rec = nullptr;
  const PassEntry* dplan = nullptr;
  int next = 0;        // passes issued so far (kPersistent)
  int run_kind = -1;   // kind of the pending run of passes
  int run_mode = -1;   // and its pass mode (a persistent launch runs one kind and mode)
  int run_first = 0;   // its first pass
  // two-stream backward (issue_backward_overlap): the stream passes go to, and the range
  // of (m, p) grid buffers they allocate from
  cudaStream_t main_s = nullptr;  // (the caller's stream may be the legacy default, null)
  bool main_known = false;
  int pm_lo = 0, pm_hi = -1;

  // issue on the main (0) or the side (1) stream from now on
  void use_stream(int sid) {
    if (!main_known) {
      main_s = s;
      main_known = true;
    }
    s = sid ? h->side_stream : main_s;
    h->pm.sid = h->ub.sid = sid;
  }
  void use_pool(int p) {
    pm_lo = p * h->m.pm_pool;
    pm_hi = pm_lo + h->m.pm_pool;
  }
  cudaError_t signal(cudaEvent_t ev) { return cudaEventRecord(ev, s); }
  cudaError_t wait(cudaEvent_t ev) { return cudaStreamWaitEvent(s, ev, 0); }

  // clear, on the current stream, every buffer released on it and not yet cleared
  cudaError_t flush_clears() {
    for (;;) {
      Clears C = take_clears(h);
      if (C.n == 0) return cudaSuccess;
      ++count;
      cudaError_t e = timed(MPM_KERNEL_GRID_CLEAR, [&] {
        return h->m.D == 2 ? launch_clear<2>(C, (int)h->m.nnodes, h->m.n_grid, h->m.S, grid_blocks_per_scene(h), s)
                           : launch_clear<3>(C, (int)h->m.nnodes, h->m.n_grid, h->m.S, grid_blocks_per_scene(h), s);
      });
      after_launch(h);
      if (e != cudaSuccess) return e;
    }
  }

  // one pass: launched, recorded, or queued into the pending persistent run
  template <typename Args>
  cudaError_t pass(int kind, int pmode, int category, const SimParams& P, const Args& A) {
    if (mode == kRecord) {
      PassEntry e;
      memset(&e, 0, sizeof(e));
      e.kind = kind;
      e.mode = pmode;
      e.P = P;
      if constexpr (std::is_same<Args, StepArgs>::value) e.S = A;
      else e.A = A;
      rec->push_back(e);
      return cudaSuccess;
    }
    if (mode == kPersistent) {
      if (run_kind != kind || run_mode != pmode) {
        cudaError_t e = flush();
        if (e != cudaSuccess) return e;
        run_kind = kind;
        run_mode = pmode;
        run_first = next;
      }
      ++next;
      return cudaSuccess;
    }
    ++count;
    const Dims& m = h->m;
    return timed(category, [&] {
      if constexpr (std::is_same<Args, StepArgs>::value)
        return m.D == 2 ? launch_step<2>(h->desc.material, pmode, P, A, m.n_tiles, s)
                        : launch_step<3>(h->desc.material, pmode, P, A, m.n_tiles, s);
      else
        return m.D == 2 ? launch_adjoint<2>(h->desc.material, pmode, P, A, m.n_tiles, s)
                        : launch_adjoint<3>(h->desc.material, pmode, P, A, m.n_tiles, s);
    });
  }

  // launch the pending run of same-kind passes as persistent launches of at most
  // persistent_chunk passes each (one launch when the chunk is 0)
  cudaError_t flush() {
    while (mode == kPersistent && next > run_first) {
      int n = next - run_first;
      if (h->persistent_chunk > 0 && n > h->persistent_chunk) n = h->persistent_chunk;
      cudaError_t e = launch_run(n);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }

  cudaError_t launch_run(int n) {
    static_assert(sizeof(GridSync) <= 16, "barrier counters fit the first 16 bytes");
    GridSync* gs = h->at<GridSync>(h->L.gsync);
    cudaError_t e = cudaMemsetAsync(gs, 0, 16 + 4 * (size_t)n, s);
    if (e != cudaSuccess) return e;
    PersistCtl c;
    c.sync = gs;
    c.tickets = reinterpret_cast<unsigned*>(h->at<char>(h->L.gsync) + 16);
    c.err = h->at<unsigned>(h->L.err);
    c.timeout_ns = h->barrier_timeout_us * 1000;
    c.extra = h->barrier_extra;
    const SimParams P = params_for(h, 0);  // shared-memory capacities
    const int kind = run_kind;
    const int kind_mode = run_kind * 8 + run_mode;
    const PassEntry* plan = dplan + run_first;
    const Dims& m = h->m;
    ++count;
    e = timed(kind == kPassStep ? MPM_KERNEL_PERSISTENT_STEP : MPM_KERNEL_PERSISTENT_ADJ, [&] {
      return m.D == 2 ? launch_persistent<2>(kind_mode, h->desc.material, P, plan, n, m.n_tiles, c, s, nullptr)
                      : launch_persistent<3>(kind_mode, h->desc.material, P, plan, n, m.n_tiles, c, s, nullptr);
    });
    run_first += n;
    return e;
  }

  // bracket one launch with events when profiling (category = MPM_KERNEL_*)
  template <typename Fn>
  cudaError_t timed(int category, Fn&& launch) {
    if (!h->profile) return launch();
    size_t used = h->ev_records.size() * 2;
    while (h->ev_pool.size() < used + 2) {
      cudaEvent_t e;
      cudaError_t ce = cudaEventCreate(&e);
      if (ce != cudaSuccess) return ce;
      h->ev_pool.push_back(e);
    }
    cudaEvent_t a = h->ev_pool[used], b = h->ev_pool[used + 1];
    cudaError_t e = cudaEventRecord(a, s);
    if (e == cudaSuccess) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(b, s);
    if (e == cudaSuccess) h->ev_records.push_back({category, {a, b}});
    return e;
  }

  // one forward particle pass: G2P of step t-1 from grid `read` (-1: none), P2G of step
  // t into a new grid (returned in *written, -1 for G2P only)
  cudaError_t step(int smode, int t, const float* in, float* out, int read, int* written,
                   double* R_out = nullptr) {
    const Dims& m = h->m;
    SimParams P = params_for(h, t);
    StepArgs A;
    memset(&A, 0, sizeof(A));
    A.tiles = h->at<int4>(h->L.tiles);
    A.scene_tiles = h->at<int>(h->L.scene_tiles);
    A.N = (int)m.N;
    A.in = in;
    A.out = out;
    A.mu = h->at<float>(h->L.mu);
    A.la = h->at<float>(h->L.la);
    A.group = h->at<int>(h->L.group);
    A.matid = h->at<int>(h->L.matid);
    A.wact = act_ptr(h, t);
    A.err = h->at<unsigned>(h->L.err);
    A.box_stats = h->at<unsigned long long>(h->L.box_stats);
    if (read >= 0) A.PMr = ring_grid(h, h->pm, read);
    A.Rw = R_out;
    if (written) {
      WriteSlot w;
      if (!ring_alloc(h, h->pm, w, pm_lo, pm_hi)) return cudaErrorMemoryAllocation;
      A.PMw = w.grid;
      A.box_w = w.box;
      A.box_reset = w.box_reset;
      *written = w.id;
    }
    A.clears = take_clears(h);
    const int cat = smode == kP2GOnly ? MPM_KERNEL_P2G
                    : smode == kG2PP2G ? MPM_KERNEL_G2P_P2G
                    : smode == kG2PP2GFull ? MPM_KERNEL_G2P_P2G_FULL : MPM_KERNEL_G2P;
    cudaError_t e = pass(kPassStep, smode, cat, P, A);
    after_launch(h);
    return e;
  }

  // one adjoint pass (see the file comment); pm1/ub1: grids of step s+1 (-1 in kAdjG2P
  // mode), pm0: grid of step s; writes the velocity adjoint of step s (*ub_written) and,
  // when stm != null, the recomputed grid of step s-1 (*pm_written)
  cudaError_t adjoint(int amode, int s_step, const float* st1, const float* st0, const float* stm,
                      int pm1, int ub1, int pm0, int* ub_written, int* pm_written,
                      const double* R1 = nullptr, const double* Rm = nullptr, int measure = 0) {
    const Dims& m = h->m;
    SimParams P = params_for(h, s_step + 1);
    SimParams P2 = params_for(h, s_step - 1 >= 0 ? s_step - 1 : 0);
    memcpy(P.basis2, P2.basis, sizeof(P.basis2));
    AdjArgs A;
    memset(&A, 0, sizeof(A));
    A.tiles = h->at<int4>(h->L.tiles);
    A.scene_tiles = h->at<int>(h->L.scene_tiles);
    A.N = (int)m.N;
    A.st1 = st1;
    A.st0 = st0;
    A.stm = stm;
    A.adj = h->at<float>(h->L.adj);
    A.mu = h->at<float>(h->L.mu);
    A.la = h->at<float>(h->L.la);
    A.mubar = h->at<float2>(h->L.mubar);
    A.labar = h->at<float2>(h->L.labar);
    A.group = h->at<int>(h->L.group);
    A.matid = h->at<int>(h->L.matid);
    A.wact = act_ptr(h, s_step + 1);
    A.wbar_tile = h->at<float>(h->L.wbar_tile);
    A.err = h->at<unsigned>(h->L.err);
    A.R1 = R1;
    A.Rm = Rm;
    A.ub_m0 = h->at<unsigned>(h->L.ub_m0);
    A.measure = measure;
    if (pm1 >= 0) A.PM1 = ring_grid(h, h->pm, pm1);
    if (ub1 >= 0) A.UB1 = ring_grid(h, h->ub, ub1);
    if (pm0 >= 0) A.PM0 = ring_grid(h, h->pm, pm0);
    if (ub_written) {
      WriteSlot w;
      if (!ring_alloc(h, h->ub, w)) return cudaErrorMemoryAllocation;
      A.UB0 = w.grid;
      A.box_ub = w.box;
      A.box_ub_reset = w.box_reset;
      *ub_written = w.id;
    }
    if (stm && pm_written) {
      WriteSlot w;
      if (!ring_alloc(h, h->pm, w, pm_lo, pm_hi)) return cudaErrorMemoryAllocation;
      A.PMm = w.grid;
      A.box_m = w.box;
      A.box_m_reset = w.box_reset;
      *pm_written = w.id;
    } else {
      A.stm = nullptr;
    }
    A.clears = take_clears(h);
    const int cat = amode == kAdjG2P ? MPM_KERNEL_ADJ_G2P
                    : amode == kAdjFused ? MPM_KERNEL_ADJ_FUSED : MPM_KERNEL_ADJ_P2G;
    cudaError_t e = pass(kPassAdjoint, amode, cat, P, A);
    after_launch(h);
    return e;
  }

  // closed-loop controller at step t: sense state st and evaluate the MLP, giving row t of
  // the actuation table (direct launches only: the persistent form is off with a controller)
  cudaError_t ctrl_forward(int t, const float* st) {
    if (mode != kDirect) return cudaErrorNotSupported;
    const Dims& m = h->m;
    const Layout& L = h->L;
    const CtrlStep c = ctrl_step(h, t);
    count += 2;
    return timed(MPM_KERNEL_CONTROLLER, [&] {
      return launch_ctrl_forward(c, m.S, m.n_tiles, m.N, h->at<int4>(L.tiles), h->at<int>(L.scene_tile_off), st,
                                 h->at<int>(L.group), h->at<double>(L.ctrl_part), h->at<float>(L.wact),
                                 h->at<double>(L.ctrl_u) + (size_t)t * m.S * m.ctrl_in,
                                 h->at<double>(L.ctrl_h) + (size_t)t * m.S * m.ctrl_H,
                                 h->at<double>(L.ctrl_y) + (size_t)t * m.S * m.G,
                                 h->at<float>(L.act_tab) + (size_t)t * m.S * m.G, h->at<double>(L.ctrl_cnt), s);
    });
  }

  // reverse of the controller at step t, after the P2G adjoint of step t left the
  // per-tile actuation adjoints in wbar_tile and the adjoint of state t in adj
  cudaError_t ctrl_backward(int t) {
    if (mode != kDirect) return cudaErrorNotSupported;
    const Dims& m = h->m;
    const Layout& L = h->L;
    const CtrlStep c = ctrl_step(h, t);
    count += 2;
    return timed(MPM_KERNEL_CONTROLLER, [&] {
      return launch_ctrl_backward(c, m.S, m.n_tiles, m.N, h->at<int4>(L.tiles), h->at<int>(L.scene_tile_off),
                                  h->at<int>(L.group), h->at<float>(L.wbar_tile), h->at<float>(L.wact),
                                  h->at<double>(L.ctrl_u) + (size_t)t * m.S * m.ctrl_in,
                                  h->at<double>(L.ctrl_h) + (size_t)t * m.S * m.ctrl_H,
                                  h->at<double>(L.ctrl_y) + (size_t)t * m.S * m.G, h->at<double>(L.ctrl_cnt),
                                  h->at<double>(L.ctrl_thbar), h->at<float>(L.ctrl_add), h->at<float>(L.adj), s);
    });
  }

  // End of a launch sequence (on the main stream, after any side-stream work has been
  // joined): zero every dirty buffer, reset every box.
  cudaError_t finish() {
    cudaError_t e = flush();
    if (e != cudaSuccess) return e;
    for (Ring* r : {&h->pm, &h->ub})
      for (int i = 0; i < r->n; ++i)
        if (r->state[i] == 1 || r->state[i] == 2) {
          r->state[i] = 2;
          r->owner[i] = r->sid;
        }
    for (;;) {
      Clears C = take_clears(h);
      if (C.n == 0) break;
      if (mode != kRecord) {
        ++count;
        e = timed(MPM_KERNEL_GRID_CLEAR, [&] {
          return h->m.D == 2 ? launch_clear<2>(C, (int)h->m.nnodes, h->m.n_grid, h->m.S, grid_blocks_per_scene(h), s)
                             : launch_clear<3>(C, (int)h->m.nnodes, h->m.n_grid, h->m.S, grid_blocks_per_scene(h), s);
        });
      }
      after_launch(h);
      if (e != cudaSuccess) return e;
    }
    if (mode != kRecord) {
      ++count;
      e = launch_reset_boxes(h->at<int>(h->L.boxes), (int64_t)(h->m.pm_slots + kUBSlots) * 2 * h->m.S, s);
    }
    ring_reset(h->pm);
    ring_reset(h->ub);
    return e;
  }
};

#define LK(expr)                                        \
  do {                                                  \
    cudaError_t e_ = (expr);                            \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #expr); \
  } while (0)

// forward: states 0..T; full state stored at multiples of K and at T (fin)
// first step of the last segment of a T-step run: the forward leaves that segment's states
// (and their polar factors) in the segment buffer, so the backward starts without
// re-simulating it -- with ckpt_every >= T nothing is re-simulated at all
int last_segment_start(const mpm_handle* h, int T) { return ((T - 1) / h->m.K) * h->m.K; }

// whether the forward stores state t as a checkpoint: every K steps with one level; with two,
// every K*M steps, and every K steps over the last coarse segment (left for the backward
// like the last segment's states)
bool forward_stores_ckpt(const mpm_handle* h, int T, int t) {
  const int K = h->m.K, KM = h->m.K * h->m.M;
  if (t % K != 0) return false;
  return h->m.M == 1 || t % KM == 0 || t >= ((T - 1) / KM) * KM;
}

// Two levels: rebuild the checkpoints every K steps of coarse segment Jc (states
// Jc K M + m K, m = 1 .. M-1 below T) by re-simulating it from its coarse checkpoint.
int issue_coarse_resim(mpm_handle* h, Launcher& Lc, int Jc, int T) {
  const int K = h->m.K, M = h->m.M;
  const int s0 = Jc * K * M;
  const int last = std::min(s0 + (M - 1) * K, ((T - 1) / K) * K);  // last checkpoint to rebuild
  if (last <= s0) return MPM_OK;
  const float* src = h->ckpt(s0 / K);
  float* cur = h->at<float>(h->L.cur);
  int g = -1;
  LK(Lc.step(kP2GOnly, s0, src, nullptr, -1, &g));
  for (int t = s0 + 1; t < last; ++t) {
    const bool ck = (t - s0) % K == 0;
    float* dst = ck ? h->ckpt(t / K) : cur;
    int g_next = -1;
    LK(Lc.step(ck ? kG2PP2GFull : kG2PP2G, t, src, dst, g, &g_next));
    ring_release(h->pm, g);
    g = g_next;
    src = dst;
  }
  LK(Lc.step(kG2POnlyFull, last, src, h->ckpt(last / K), g, nullptr));
  ring_release(h->pm, g);
  return MPM_OK;
}

int issue_forward(mpm_handle* h, Launcher& Lc, int T) {
  const int K = h->m.K;
  const int sL = last_segment_start(h, T);
  ring_reset(h->pm);
  ring_reset(h->ub);
  const float* src = h->state(h->L.ckpt, 0);
  float* cur = h->at<float>(h->L.cur);
  int g = -1;
  LK(Lc.step(kP2GOnly, 0, src, nullptr, -1, &g, sL == 0 ? h->rslot(sL / K, 0) : nullptr));
  for (int t = 1; t < T; ++t) {
    float* dst;
    int mode;
    if (forward_stores_ckpt(h, T, t)) {
      dst = h->ckpt(t / K);
      mode = kG2PP2GFull;
    } else if (t > sL) {
      dst = h->seg(sL / K, t - sL);
      mode = kG2PP2GFull;
    } else {
      dst = cur;
      mode = kG2PP2G;
    }
    int g_next = -1;
    LK(Lc.step(mode, t, src, dst, g, &g_next, t >= sL ? h->rslot(sL / K, t - sL) : nullptr));
    ring_release(h->pm, g);
    g = g_next;
    src = dst;
  }
  LK(Lc.step(kG2POnlyFull, T, src, h->at<float>(h->L.fin), g, nullptr));
  ring_release(h->pm, g);
  LK(Lc.finish());
  return MPM_OK;
}

// re-simulate segment [s0, top): seg slot i <- state s0 + i (i = 1..top-s0); returns the
// grid of step top-1 (kept live for the adjoint passes)
// re-simulate segment [s0, top): seg slot i <- state s0 + i (i = 1..top-s0); returns the
// grid of step top-1 (kept live for the adjoint passes); with seg_grids, every grid of the
// segment is kept live too (seg_grids[t - s0] = grid of step t)
int issue_resim(mpm_handle* h, Launcher& Lc, int s0, int top, int* grid_top_minus_1,
                int* seg_grids) {
  const float* ck = h->ckpt(s0 / h->m.K);
  int g = -1;
  LK(Lc.step(kP2GOnly, s0, ck, nullptr, -1, &g, h->rslot(s0 / h->m.K, 0)));
  const float* prev = ck;
  for (int t = s0 + 1; t < top; ++t) {
    float* dst = h->seg(s0 / h->m.K, t - s0);
    int g_next = -1;
    LK(Lc.step(kG2PP2GFull, t, prev, dst, g, &g_next, h->rslot(s0 / h->m.K, t - s0)));
    if (seg_grids) seg_grids[t - 1 - s0] = g;
    else ring_release(h->pm, g);
    g = g_next;
    prev = dst;
  }
  LK(Lc.step(kG2POnlyFull, top, prev, h->seg(s0 / h->m.K, top - s0), g, nullptr));
  if (seg_grids) seg_grids[top - 1 - s0] = g;
  *grid_top_minus_1 = g;
  return MPM_OK;
}

// Backward.  With `overlap`, segment j-1 is re-simulated on the side stream while the
// adjoint passes of segment j run on the main stream: the two are independent (the
// re-simulation reads only checkpoint j-1) and latency-bound, so they share the SMs
// better than they run one after the other.  Segments alternate between two segment
// buffers, polar caches and (m, p) grid pools by parity.  Hand-offs: the side stream
// starts re-simulating segment j-1 (parity of j+1) once the first adjoint pass of segment
// j has released the last grid of segment j+1 and the main stream has cleared that pool
// (ev_free); the adjoint passes of segment j-1 start after its re-simulation (ev_resim).
// A buffer released on a stream is cleared by a later launch on the same stream.
int issue_backward(mpm_handle* h, Launcher& Lc, int T, bool resident, bool overlap) {
  const int K = h->m.K;
  ring_reset(h->pm);
  ring_reset(h->ub);
  const bool kept = h->m.store_grids && !h->grid_recompute;
  // live grids: PM of steps s+1 and s, UB of step s+1
  int pm_s1 = -1, pm_s = -1, ub_s1 = -1;
  std::vector<int> seg_grids[2] = {std::vector<int>(K, -1), std::vector<int>(K, -1)};
  int side_top[2] = {-1, -1};  // grid of step top-1 of a segment re-simulated on the side
  bool stored = false;         // this segment's grids were kept by its re-simulation
  if (overlap) {
    LK(Lc.signal(h->ev_fork));
    Lc.use_stream(1);
    LK(Lc.wait(h->ev_fork));
    Lc.use_stream(0);
  }
  int coarse = resident ? (T - 1) / (K * h->m.M) : -1;  // coarse segment whose checkpoints are built
  for (int s = T - 1; s >= 0; --s) {
    const int j = s / K, s0 = j * K, pj = j & 1;
    const int top = (s0 + K < T) ? s0 + K : T;
    if (overlap) Lc.use_pool(pj);
    if (h->m.M > 1 && j / h->m.M != coarse) {
      coarse = j / h->m.M;
      int rc = issue_coarse_resim(h, Lc, coarse, T);
      if (rc) return rc;
    }
    if (s == T - 1 && resident) {
      // the forward left this segment's states in place: only the grid of step T-1
      const float* st = (s == s0) ? h->ckpt(j) : h->seg(j, s - s0);
      LK(Lc.step(kP2GOnly, s, st, nullptr, -1, &pm_s));
      stored = false;
    } else if (s == top - 1) {
      stored = kept;
      if (overlap && s != T - 1) {  // re-simulated on the side stream meanwhile
        LK(Lc.wait(h->ev_resim));
        pm_s = side_top[pj];
      } else {
        int rc = issue_resim(h, Lc, s0, top, &pm_s, stored ? seg_grids[pj].data() : nullptr);
        if (rc) return rc;
      }
    }
    const float* st_s = (s == s0) ? h->ckpt(j) : h->seg(j, s - s0);
    const float* st_s1 = (s + 1 == T) ? h->at<float>(h->L.fin) : h->seg(j, s + 1 - s0);
    // the recomputed P2G of step s-1 runs only when this segment's grids were not kept
    const float* st_sm = (s - 1 >= s0 && !stored)
                             ? ((s - 1 == s0) ? h->ckpt(j) : h->seg(j, s - 1 - s0))
                             : nullptr;
    int ub_s = -1, pm_sm = -1;
    // cached polar factors: state s+1 only inside this segment (the segment's top state
    // was never the P2G input of this re-simulation), state s-1 always when present
    const double* R1 = (s + 1 < top) ? h->rslot(j, s + 1 - s0) : nullptr;
    const double* Rm = (s - 1 >= s0) ? h->rslot(j, s - 1 - s0) : nullptr;
    if (s == T - 1 && h->m.words == 2)  // deterministic: bound of the first ubar scatter
      LK(Lc.adjoint(kAdjG2P, s, st_s1, st_s, nullptr, -1, -1, pm_s, nullptr, nullptr, nullptr,
                    nullptr, 1));
    LK(Lc.adjoint(s == T - 1 ? kAdjG2P : kAdjFused, s, st_s1, st_s, st_sm,
                  s == T - 1 ? -1 : pm_s1, s == T - 1 ? -1 : ub_s1, pm_s, &ub_s, &pm_sm, R1, Rm));
    ring_release(h->pm, pm_s1);
    ring_release(h->ub, ub_s1);
    pm_s1 = pm_s;
    ub_s1 = ub_s;
    // the grid of step s-1: kept, recomputed by this pass, or (at a segment start) provided
    // by the next segment's re-simulation
    pm_s = stored ? (s - 1 >= s0 ? seg_grids[pj][s - 1 - s0] : -1) : pm_sm;
    if (overlap && s == top - 1 && j >= 1) {
      // segment j+1's last grid is released: clear its pool, then re-simulate segment j-1
      // into that pool and segment buffer on the side stream
      LK(Lc.flush_clears());
      LK(Lc.signal(h->ev_free));
      Lc.use_stream(1);
      Lc.use_pool(1 - pj);
      LK(Lc.wait(h->ev_free));
      int rc = issue_resim(h, Lc, s0 - K, s0, &side_top[1 - pj], kept ? seg_grids[1 - pj].data() : nullptr);
      if (rc) return rc;
      LK(Lc.flush_clears());
      LK(Lc.signal(h->ev_resim));
      Lc.use_stream(0);
      Lc.use_pool(pj);
    }
  }
  const float* st0 = h->state(h->L.ckpt, 0);
  LK(Lc.adjoint(kAdjP2G, -1, st0, st0, nullptr, pm_s1, ub_s1, -1, nullptr, nullptr));
  ring_release(h->pm, pm_s1);
  ring_release(h->ub, ub_s1);
  if (overlap) {  // join (the side stream's last work is already waited for)
    Lc.use_stream(1);
    LK(Lc.signal(h->ev_join));
    Lc.use_stream(0);
    LK(Lc.wait(h->ev_join));
  }
  LK(Lc.finish());
  return MPM_OK;
}

// Closed-loop controller (desc.ctrl_hidden > 0).  The actuation of step t depends on
// state t through the controller's sensors, so P2G of step t waits for the whole of
// G2P of step t-1 and for the controller: the forward splits the fused pass into G2P
// (state t written in full), the controller, and P2G.  The storage of states (checkpoints,
// the resident last segment, the polar factors) is that of issue_forward, and the
// actuation table the forward writes is what every later pass of that step reads.
int issue_forward_ctrl(mpm_handle* h, Launcher& Lc, int T) {
  const int K = h->m.K;
  const int sL = last_segment_start(h, T);
  ring_reset(h->pm);
  ring_reset(h->ub);
  const float* src = h->state(h->L.ckpt, 0);
  float* cur = h->at<float>(h->L.cur);
  int g = -1;
  LK(Lc.ctrl_forward(0, src));
  LK(Lc.step(kP2GOnly, 0, src, nullptr, -1, &g, sL == 0 ? h->rslot(sL / K, 0) : nullptr));
  for (int t = 1; t < T; ++t) {
    float* dst = forward_stores_ckpt(h, T, t) ? h->ckpt(t / K) : (t > sL) ? h->seg(sL / K, t - sL) : cur;
    LK(Lc.step(kG2POnlyFull, t, src, dst, g, nullptr));
    ring_release(h->pm, g);
    LK(Lc.ctrl_forward(t, dst));
    LK(Lc.step(kP2GOnly, t, dst, nullptr, -1, &g, t >= sL ? h->rslot(sL / K, t - sL) : nullptr));
    src = dst;
  }
  LK(Lc.step(kG2POnlyFull, T, src, h->at<float>(h->L.fin), g, nullptr));
  ring_release(h->pm, g);
  LK(Lc.finish());
  return MPM_OK;
}

// Backward with the controller: the sensor adjoint of state s+1 needs the actuation
// adjoint of step s+1 summed over every particle, so the fused adjoint pass splits into
// the P2G adjoint of step s+1 (adjoint of state s+1 written in full), the controller's
// reverse (which adds the sensor terms to it), and the G2P adjoint of step s read from
// it.  Re-simulation reads the recorded actuation table; a grid that is neither kept nor
// re-simulated is recomputed by its own P2G pass.
int issue_backward_ctrl(mpm_handle* h, Launcher& Lc, int T, bool resident) {
  const int K = h->m.K;
  ring_reset(h->pm);
  ring_reset(h->ub);
  int pm_s1 = -1, pm_s = -1, ub_s1 = -1;
  std::vector<int> seg_grids(K, -1);
  bool stored = false;
  int coarse = resident ? (T - 1) / (K * h->m.M) : -1;  // coarse segment whose checkpoints are built
  for (int s = T - 1; s >= 0; --s) {
    const int j = s / K, s0 = j * K;
    const int top = (s0 + K < T) ? s0 + K : T;
    if (h->m.M > 1 && j / h->m.M != coarse) {
      coarse = j / h->m.M;
      int rc = issue_coarse_resim(h, Lc, coarse, T);
      if (rc) return rc;
    }
    const float* st_s = (s == s0) ? h->ckpt(j) : h->seg(j, s - s0);
    const float* st_s1 = (s + 1 == T) ? h->at<float>(h->L.fin) : h->seg(j, s + 1 - s0);
    const double* R1 = (s + 1 < top) ? h->rslot(j, s + 1 - s0) : nullptr;
    if (s == T - 1 && resident) {
      LK(Lc.step(kP2GOnly, s, st_s, nullptr, -1, &pm_s));
      stored = false;
    } else if (s == top - 1) {
      stored = h->m.store_grids && !h->grid_recompute;
      int rc = issue_resim(h, Lc, s0, top, &pm_s, stored ? seg_grids.data() : nullptr);
      if (rc) return rc;
    } else if (stored) {
      pm_s = seg_grids[s - s0];
    } else {
      LK(Lc.step(kP2GOnly, s, st_s, nullptr, -1, &pm_s, nullptr));
    }
    if (s < T - 1) {
      LK(Lc.adjoint(kAdjP2G, s, st_s1, st_s1, nullptr, pm_s1, ub_s1, -1, nullptr, nullptr, R1));
      ring_release(h->pm, pm_s1);
      ring_release(h->ub, ub_s1);
      LK(Lc.ctrl_backward(s + 1));
    } else if (h->m.words == 2) {  // deterministic: bound of the first ubar scatter
      LK(Lc.adjoint(kAdjG2P, s, st_s1, st_s, nullptr, -1, -1, pm_s, nullptr, nullptr, nullptr,
                    nullptr, 1));
    }
    int ub_s = -1;
    LK(Lc.adjoint(kAdjG2P, s, st_s1, st_s, nullptr, -1, -1, pm_s, &ub_s, nullptr));
    pm_s1 = pm_s;
    ub_s1 = ub_s;
  }
  const float* st0 = h->state(h->L.ckpt, 0);
  LK(Lc.adjoint(kAdjP2G, -1, st0, st0, nullptr, pm_s1, ub_s1, -1, nullptr, nullptr));
  ring_release(h->pm, pm_s1);
  ring_release(h->ub, ub_s1);
  LK(Lc.ctrl_backward(0));
  LK(Lc.finish());
  return MPM_OK;
}

void drop_graphs(mpm_handle* h) {
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second.first);
  h->graphs.clear();
}

// After a failed issue inside a capture: join the side stream back into the capturing
// stream if a fork left it in the capture, so that ending the capture takes both streams out
// of capture mode (the event is destroyed by the caller after the capture ends).
void unjoin_side_stream(mpm_handle* h, cudaEvent_t* join) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (!h->side_stream || cudaStreamIsCapturing(h->side_stream, &st) != cudaSuccess ||
      st == cudaStreamCaptureStatusNone)
    return;
  if (cudaEventCreateWithFlags(join, cudaEventDisableTiming) != cudaSuccess) {
    *join = nullptr;
    return;
  }
  cudaEventRecord(*join, h->side_stream);
  cudaStreamWaitEvent(h->cap_stream, *join, 0);
}

// Run a launch sequence on `stream`, through a cached CUDA graph when enabled.
template <typename Fn>
int run_sequence_impl(mpm_handle* h, int64_t key, cudaStream_t stream, Fn&& issue) {
  const PassEntry* dplan = nullptr;
  if (h->persistent && h->m.ctrl_H == 0) {  // the controller's kernels are not plan passes
    // record the plan (forward keys are even, backward keys odd), refresh its device copy
    const int region = (int)(key & 1);
    std::vector<PassEntry> plan;
    Launcher R{h, stream};
    R.mode = kRecord;
    R.rec = &plan;
    int rc = issue(R);
    if (rc) return rc;
    const int64_t cap = region ? plan_bwd_cap(h->m) : plan_fwd_cap(h->m);
    if ((int64_t)plan.size() > cap) return fail(h, MPM_ERR_STATE, "pass plan exceeds its workspace region");
    PassEntry* dst = h->at<PassEntry>(region ? h->L.plan_bwd : h->L.plan_fwd);
    std::vector<PassEntry>& have = h->plan_copy[region];
    if (have.size() != plan.size() ||
        memcmp(have.data(), plan.data(), plan.size() * sizeof(PassEntry)) != 0) {
      drop_graphs(h);  // captured persistent launches read the region being replaced
      // pageable source: the call returns once the bytes are staged, and the copy runs in
      // stream order before the launches that read it
      CK(cudaMemcpyAsync(dst, plan.data(), plan.size() * sizeof(PassEntry), cudaMemcpyHostToDevice,
                         stream));
      have.swap(plan);
    }
    dplan = dst;
  }
  auto configure = [&](Launcher& Lc) {
    if (dplan) {
      Lc.mode = kPersistent;
      Lc.dplan = dplan;
    }
  };
  if (!h->use_graphs || h->profile) {
    Launcher Lc{h, stream};
    configure(Lc);
    int rc = issue(Lc);
    h->launches += Lc.count;
    return rc;
  }
  auto it = h->graphs.find(key);
  if (it == h->graphs.end()) {
    if (!h->cap_stream) CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    Launcher Lc{h, h->cap_stream};
    configure(Lc);
    int rc = issue(Lc);
    cudaEvent_t join = nullptr;
    if (rc) unjoin_side_stream(h, &join);  // a failed issue may leave the side stream forked
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
    if (join) cudaEventDestroy(join);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();  // the capture's own errors are not the caller's
      return rc;
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
    it = h->graphs.emplace(key, std::make_pair(ex, Lc.count)).first;
  }
  CK(cudaGraphLaunch(it->second.first, stream));
  h->launches += it->second.second;
  return MPM_OK;
}

// A failed sequence may leave grid buffers dirty: the handle then needs mpm_set_initial
// (which clears every buffer) before the next forward.
template <typename Fn>
int run_sequence(mpm_handle* h, int64_t key, cudaStream_t stream, Fn&& issue) {
  int rc = run_sequence_impl(h, key, stream, issue);
  if (rc != MPM_OK) {
    h->initialized = false;
    h->T_recorded = 0;
  }
  return rc;
}

// Dynamic shared memory the particle passes need with the handle's capacities, plus the
// passes' static shared memory (below 8 KB), against the device's per-CTA limit.
bool capacities_fit(const mpm_handle* h, std::string* why) {
  if (h->smem_optin <= 0) return true;
  const SimParams P = params_for(h, 0);
  const size_t need = (h->m.D == 2 ? std::max(step_smem_bytes<2>(P.tile_capacity, P.gather_capacity),
                                              adj_smem_bytes<2>(P.tile_capacity, P.gather_capacity))
                                   : std::max(step_smem_bytes<3>(P.tile_capacity, P.gather_capacity),
                                              adj_smem_bytes<3>(P.tile_capacity, P.gather_capacity))) +
                      8 * 1024;
  if (need <= (size_t)h->smem_optin) return true;
  char buf[160];
  snprintf(buf, sizeof(buf), "the shared node boxes need %zu B of shared memory per CTA, the device allows %d B",
           need, h->smem_optin);
  *why = buf;
  return false;
}

}  // namespace

// =============================== C ABI ======================================

extern "C" {

int mpm_workspace_bytes(const mpm_scene_desc* desc, int32_t max_steps, size_t* out_bytes) {
  std::string why;
  if (!out_bytes) return fail(nullptr, MPM_ERR_ARG, "out_bytes is NULL");
  if (!valid_desc(desc, max_steps, &why)) return fail(nullptr, MPM_ERR_ARG, why);
  Dims m = make_dims(desc, max_steps);
  *out_bytes = make_layout(m).total;
  return MPM_OK;
}

int mpm_plan_checkpoints(const mpm_scene_desc* desc, int32_t max_steps, size_t budget_bytes,
                         int32_t* ckpt_every, int32_t* ckpt_coarse, size_t* ws_bytes) {
  std::string why;
  if (!ckpt_every || !ckpt_coarse) return fail(nullptr, MPM_ERR_ARG, "NULL output");
  if (!valid_desc(desc, max_steps, &why)) return fail(nullptr, MPM_ERR_ARG, why);
  const int64_t T = max_steps;
  // candidate intervals: every k up to 4096, then powers of two, and T itself (no re-simulation)
  std::vector<int64_t> ks;
  for (int64_t k = 1; k <= std::min<int64_t>(T, 4096); ++k) ks.push_back(k);
  for (int64_t k = 8192; k < T; k *= 2) ks.push_back(k);
  if (T > 4096) ks.push_back(T);
  const int coarse[] = {1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64, 96, 128, 256, 512, 1024};
  mpm_scene_desc d = *desc;
  double best_cost = 0.0;
  size_t best_bytes = 0;
  int64_t best_k = -1, best_M = 0;
  for (int M : coarse) {
    for (int64_t k : ks) {
      if (M > 1 && k * M >= T) break;  // a second level needs more than one coarse segment
      d.ckpt_every = (int32_t)k;
      d.ckpt_coarse = M > 1 ? M : 0;
      const Dims m = make_dims(&d, max_steps);
      const size_t bytes = make_layout(m).total;
      if (bytes > budget_bytes) continue;
      // cost in particle passes of one forward + backward: T forward, T adjoint, every
      // segment but the last re-simulated once (the steps before the last segment's start),
      // a second level re-simulates every coarse segment but the last once more, and an
      // adjoint pass that cannot keep its segment's grids recomputes one P2G pass (about
      // half an adjoint pass)
      const int64_t K = m.K;
      double cost = 2.0 * (double)T + (double)(((T - 1) / K) * K);
      if (M > 1) cost += (double)(((T - 1) / (K * M)) * (K * M));
      if (!m.store_grids) cost += 0.5 * (double)T;
      if (best_k < 0 || cost < best_cost || (cost == best_cost && bytes < best_bytes)) {
        best_cost = cost;
        best_bytes = bytes;
        best_k = K;
        best_M = M;
      }
    }
  }
  if (best_k < 0)
    return fail(nullptr, MPM_ERR_WORKSPACE, "no checkpoint schedule fits the workspace budget");
  *ckpt_every = (int32_t)best_k;
  *ckpt_coarse = best_M > 1 ? (int32_t)best_M : 0;
  if (ws_bytes) *ws_bytes = best_bytes;
  return MPM_OK;
}

int mpm_create(const mpm_scene_desc* desc, void* workspace, size_t workspace_bytes,
               int32_t max_steps, mpm_handle** out) {
  std::string why;
  if (!out) return fail(nullptr, MPM_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!valid_desc(desc, max_steps, &why)) return fail(nullptr, MPM_ERR_ARG, why);
  Dims m = make_dims(desc, max_steps);
  Layout L = make_layout(m);
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) % kAlign) != 0)
    return fail(nullptr, MPM_ERR_WORKSPACE, "workspace must be a 256-byte aligned device pointer");
  if (workspace_bytes < L.total)
    return fail(nullptr, MPM_ERR_WORKSPACE, "workspace smaller than mpm_workspace_bytes");
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, workspace) != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    return fail(nullptr, MPM_ERR_WORKSPACE, "workspace is not device memory");
  }
  mpm_handle* h = new mpm_handle();
  h->desc = *desc;
  h->n_particles.assign(desc->n_particles, desc->n_particles + desc->n_scenes);
  h->desc.n_particles = h->n_particles.data();
  h->max_steps = max_steps;
  h->m = m;
  h->L = L;
  h->ws = static_cast<char*>(workspace);
  h->smem_optin = 0;
  if (cudaDeviceGetAttribute(&h->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, attr.device) != cudaSuccess) {
    cudaGetLastError();
    h->smem_optin = 0;  // unknown: capacities are then checked by the launches alone
  }
  h->pm.n = m.pm_slots;
  h->ub.first = m.pm_slots;
  {
    cudaError_t es = cudaStreamCreateWithFlags(&h->side_stream, cudaStreamNonBlocking);
    for (cudaEvent_t* ev : {&h->ev_fork, &h->ev_free, &h->ev_resim, &h->ev_join})
      if (es == cudaSuccess) es = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (es != cudaSuccess) {
      mpm_destroy(h);
      return fail(nullptr, MPM_ERR_CUDA, std::string("mpm_create: ") + cudaGetErrorString(es));
    }
  }
  h->ws_bytes = workspace_bytes;
  // tile table and scene offsets (host -> device once)
  std::vector<int4> tiles;
  std::vector<int64_t> off(m.S + 1, 0);
  std::vector<int> scene_tiles(m.S, 0);
  for (int s = 0; s < m.S; ++s) {
    off[s + 1] = off[s] + h->n_particles[s];
    for (int64_t b = off[s]; b < off[s + 1]; b += kTile) {
      int cnt = (int)((off[s + 1] - b) < kTile ? (off[s + 1] - b) : kTile);
      tiles.push_back(make_int4(s, (int)b, cnt, scene_tiles[s]++));
    }
  }
  cudaError_t e = cudaMemcpy(h->at<int4>(L.tiles), tiles.data(), tiles.size() * sizeof(int4),
                             cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(h->at<int64_t>(L.scene_off), off.data(), off.size() * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(h->at<int>(L.scene_tiles), scene_tiles.data(), scene_tiles.size() * 4,
                   cudaMemcpyHostToDevice);
  std::vector<int> tile_off(m.S + 1, 0);
  for (int s = 0; s < m.S; ++s) tile_off[s + 1] = tile_off[s] + scene_tiles[s];
  if (e == cudaSuccess)
    e = cudaMemcpy(h->at<int>(L.scene_tile_off), tile_off.data(), tile_off.size() * 4,
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(h->at<char>(L.err), 0, 4);
  if (e != cudaSuccess) {
    delete h;
    return fail(nullptr, MPM_ERR_CUDA, std::string("mpm_create: ") + cudaGetErrorString(e));
  }
  *out = h;
  return MPM_OK;
}

int mpm_set_initial(mpm_handle* h, const float* x0, const float* v0, const float* C0,
                    const float* F0, const float* E, const float* nu, const int32_t* group,
                    const float* w, void* stream) {
  if (!h) return fail(nullptr, MPM_ERR_ARG, "handle is NULL");
  if (!x0 || !v0 || !E || !nu) return fail(h, MPM_ERR_ARG, "x0, v0, E and nu are required");
  if (h->desc.n_groups > 0 && (!group || !w))
    return fail(h, MPM_ERR_ARG, "group and w are required when n_groups > 0");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  h->last_stream = s;
  const Dims& m = h->m;
  const Layout& L = h->L;
  int end_bit = 36;  // scene id above 36 bits of base Morton code and half-cell bits
  while ((1ll << (end_bit - 36)) < m.S) ++end_bit;
  CK(launch_sort_keys(m.D, m.n_grid, m.S, h->at<int64_t>(L.scene_off), m.N, x0, h->sort_order,
                      h->at<uint64_t>(L.keys0), h->at<int>(L.idx0), s));
  CK(launch_sort(h->at<void>(L.sort_tmp), L.sort_tmp_bytes, h->at<uint64_t>(L.keys0),
                 h->at<uint64_t>(L.keys1), h->at<int>(L.idx0), h->at<int>(L.perm), m.N, end_bit, s));
  CK(launch_gather_initial(m.D, m.N, h->at<int>(L.perm), x0, v0, C0, F0, E, nu, group,
                           h->state(L.ckpt, 0), h->at<float>(L.mu), h->at<float>(L.la),
                           h->at<float>(L.E), h->at<float>(L.nu), h->at<int>(L.group), s));
  const size_t wbytes = (size_t)m.S * m.n_act * sizeof(float);
  if (wbytes) CK(cudaMemcpyAsync(h->at<float>(L.wact), w, wbytes, cudaMemcpyDeviceToDevice, s));
  const size_t grid = (size_t)m.S * m.nnodes * sizeof(float4) * m.words;
  CK(cudaMemsetAsync(h->at<char>(L.grids), 0, grid * (m.pm_slots + kUBSlots), s));
  CK(cudaMemsetAsync(h->at<char>(L.box_stats), 0, 16, s));
  CK(launch_reset_boxes(h->at<int>(L.boxes), (int64_t)(m.pm_slots + kUBSlots) * 2 * m.S, s));
  ring_reset(h->pm);
  ring_reset(h->ub);
  h->launches += 3;
  h->initialized = true;
  h->materials_set = false;
  h->T_recorded = 0;
  return MPM_OK;
}

int mpm_set_particle_materials(mpm_handle* h, const int32_t* material, void* stream) {
  if (!h) return fail(nullptr, MPM_ERR_ARG, "handle is NULL");
  if (!material) return fail(h, MPM_ERR_ARG, "material is NULL");
  if (h->desc.material != MPM_MIXED) return fail(h, MPM_ERR_ARG, "the scene is not MPM_MIXED");
  if (!h->initialized) return fail(h, MPM_ERR_STATE, "mpm_set_initial has not been called");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  h->last_stream = s;
  CK(launch_gather_int(h->m.N, h->at<int>(h->L.perm), material, h->at<int>(h->L.matid), s));
  ++h->launches;
  h->T_recorded = 0;
  h->materials_set = true;
  return MPM_OK;
}

int mpm_forward(mpm_handle* h, int32_t T, void* stream) {
  if (!h) return fail(nullptr, MPM_ERR_ARG, "handle is NULL");
  if (!h->initialized) return fail(h, MPM_ERR_STATE, "mpm_set_initial has not been called");
  if (h->desc.material == MPM_MIXED && !h->materials_set)
    return fail(h, MPM_ERR_STATE, "MPM_MIXED: mpm_set_particle_materials has not been called");
  if (T < 1 || T > h->max_steps) return fail(h, MPM_ERR_STATE, "T must be in [1, max_steps]");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  h->last_stream = s;
  int rc = run_sequence(h, (int64_t)T * 2, s, [&](Launcher& Lc) {
    return h->m.ctrl_H > 0 ? issue_forward_ctrl(h, Lc, T) : issue_forward(h, Lc, T);
  });
  if (rc) return rc;
  h->T_recorded = T;
  h->resident_T = T;
  return MPM_OK;
}

int mpm_get_state(mpm_handle* h, float* x, float* v, float* C, float* F, void* stream) {
  if (!h) return fail(nullptr, MPM_ERR_ARG, "handle is NULL");
  if (!h->T_recorded) return fail(h, MPM_ERR_STATE, "no forward recorded");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  h->last_stream = s;
  const Dims& m = h->m;
  const float* fin = h->at<float>(h->L.fin);
  const int* perm = h->at<int>(h->L.perm);
  const int D = m.D;
  float* outs[4] = {x, v, C, F};
  const int rows[4] = {D, D, D * D, D * D};
  int r0 = 0;
  for (int k = 0; k < 4; ++k) {
    if (outs[k]) {
      // the workspace holds E = F - I; the caller gets F
      CK(launch_scatter_rows(rows[k], m.N, perm, fin + (size_t)r0 * m.N, outs[k], k == 3 ? D : 0,
                             k == 0 ? D : 0, s));
      ++h->launches;
    }
    r0 += rows[k];
  }
  return MPM_OK;
}

int mpm_loss(mpm_handle* h, int32_t kind, const float* target, float* loss, float* dL_dxT,
             float* dL_dx0, void* stream) {
  if (!h) return fail(nullptr, MPM_ERR_ARG, "handle is NULL");
  if (!h->T_recorded) return fail(h, MPM_ERR_STATE, "no forward recorded");
  if (kind != MPM_LOSS_COM_TARGET && kind != MPM_LOSS_COM_X_DISP)
    return fail(h, MPM_ERR_ARG, "unknown loss kind");
  if (kind == MPM_LOSS_COM_TARGET && !target) return fail(h, MPM_ERR_ARG, "target is NULL");
  if (!dL_dxT) return fail(h, MPM_ERR_ARG, "dL_dxT is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  h->last_stream = s;
  const Dims& m = h->m;
  double* com = h->at<double>(h->L.com);
  CK(launch_com(m.D, m.N, m.S, h->at<int64_t>(h->L.scene_off), h->at<int>(h->L.perm),
                h->at<float>(h->L.fin), h->state(h->L.ckpt, 0), h->at<double>(h->L.com_part), com, s));
  CK(launch_loss_seed(m.D, kind, m.N, m.S, h->at<int64_t>(h->L.scene_off), h->at<int>(h->L.perm),
                      com, target, loss, dL_dxT, dL_dx0, s));
  h->launches += 2;
  return MPM_OK;
}

int mpm_backward(mpm_handle* h, const float* dL_dx, const float* dL_dv, const float* dL_dC,
                 const float* dL_dF, float* gx0, float* gv0, float* gC0, float* gF0, float* gE,
                 float* gnu, float* gw, void* stream) {
  if (!h) return fail(nullptr, MPM_ERR_ARG, "handle is NULL");
  if (!h->T_recorded) return fail(h, MPM_ERR_STATE, "backward needs a recorded forward");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  h->last_stream = s;
  const Dims& m = h->m;
  const Layout& L = h->L;
  const int D = m.D;
  const int* perm = h->at<int>(L.perm);
  float* adj = h->at<float>(L.adj);
  const float* seeds[4] = {dL_dx, dL_dv, dL_dC, dL_dF};
  const int rows[4] = {D, D, D * D, D * D};
  int r0 = 0;
  for (int k = 0; k < 4; ++k) {
    CK(launch_gather_rows(rows[k], m.N, perm, seeds[k], adj + (size_t)r0 * m.N, s));
    r0 += rows[k];
  }
  CK(cudaMemsetAsync(h->at<double>(L.mubar), 0, (size_t)m.N * 8, s));
  CK(cudaMemsetAsync(h->at<double>(L.labar), 0, (size_t)m.N * 8, s));
  const bool ctrl = m.ctrl_H > 0;
  // per-tile sums of the actuation adjoint: times the sine basis (open loop), or per step
  // and group for the controller (cleared again by each controller reverse)
  const int GK = ctrl ? m.G : h->desc.n_groups * h->desc.n_basis;
  if (m.words == 2) CK(cudaMemsetAsync(h->at<unsigned>(L.ub_m0), 0, 4, s));
  if (GK) CK(cudaMemsetAsync(h->at<float>(L.wbar_tile), 0, (size_t)m.n_tiles * GK * 4, s));
  if (ctrl) CK(cudaMemsetAsync(h->at<double>(L.ctrl_thbar), 0, (size_t)m.S * m.n_act * 8, s));
  h->launches += 4;
  const int T = h->T_recorded;
  const bool resident = h->resident_T == T;
  // the re-simulation overlaps the adjoint passes when there is a segment to re-simulate,
  // except in the persistent form (one stream of plan passes) and while profiling (each
  // launch timed alone)
  const bool overlap = h->overlap && !h->persistent && !h->profile && !ctrl && m.M == 1 &&
                       last_segment_start(h, T) > 0;
  const int64_t key = (int64_t)T * 2 + 1 + (resident ? 0 : ((int64_t)1 << 40)) +
                      (overlap ? ((int64_t)1 << 41) : 0);
  int rc = run_sequence(h, key, s, [&](Launcher& Lc) {
    return ctrl ? issue_backward_ctrl(h, Lc, T, resident) : issue_backward(h, Lc, T, resident, overlap);
  });
  if (rc) return rc;
  // re-simulating the earlier segments reused the segment buffer: a later backward of
  // the same forward re-simulates the last segment as well
  if (last_segment_start(h, T) > 0) h->resident_T = 0;
  float* outs[4] = {gx0, gv0, gC0, gF0};
  r0 = 0;
  for (int k = 0; k < 4; ++k) {
    if (outs[k]) {
      CK(launch_scatter_rows(rows[k], m.N, perm, adj + (size_t)r0 * m.N, outs[k], 0, 0, s));
      ++h->launches;
    }
    r0 += rows[k];
  }
  if (gE || gnu) {
    CK(launch_material_grad(m.N, perm, h->at<float>(L.E), h->at<float>(L.nu), h->at<float2>(L.mubar),
                            h->at<float2>(L.labar), gE, gnu, s));
    ++h->launches;
  }
  if (gw && ctrl) {
    CK(launch_ctrl_grad_out((int64_t)m.S * m.n_act, h->at<double>(L.ctrl_thbar), gw, s));
    ++h->launches;
  } else if (gw && GK) {
    CK(launch_wbar_reduce(m.S, GK, h->at<int>(L.scene_tile_off), h->at<float>(L.wbar_tile), gw, s));
    ++h->launches;
  }
  return MPM_OK;
}

int mpm_initial_p2g_grid(mpm_handle* h, float* grid, void* stream) {
  if (!h) return fail(nullptr, MPM_ERR_ARG, "handle is NULL");
  if (!grid) return fail(h, MPM_ERR_ARG, "grid is NULL");
  if (!h->initialized) return fail(h, MPM_ERR_STATE, "mpm_set_initial has not been called");
  if (h->m.words != 1 || h->m.ctrl_H > 0)
    return fail(h, MPM_ERR_ARG, "not available in the deterministic mode or with a controller");
  if (h->desc.material == MPM_MIXED && !h->materials_set)
    return fail(h, MPM_ERR_STATE, "MPM_MIXED: mpm_set_particle_materials has not been called");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  h->last_stream = s;
  Launcher Lc{h, s};
  ring_reset(h->pm);
  ring_reset(h->ub);
  int g = -1;
  LK(Lc.step(kP2GOnly, 0, h->ckpt(0), nullptr, -1, &g));
  CK(cudaMemcpyAsync(grid, ring_grid(h, h->pm, g), (size_t)h->m.S * h->m.nnodes * sizeof(float4),
                     cudaMemcpyDeviceToDevice, s));
  ring_release(h->pm, g);
  LK(Lc.finish());
  h->launches += Lc.count;
  return MPM_OK;
}

int mpm_sync_status(mpm_handle* h) {
  if (!h) return fail(nullptr, MPM_ERR_ARG, "handle is NULL");
  cudaError_t e = cudaStreamSynchronize(h->last_stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
  unsigned err = 0;
  e = cudaMemcpy(&err, h->at<unsigned>(h->L.err), 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e, "read error word");
  if (err) {
    cudaMemset(h->at<unsigned>(h->L.err), 0, 4);
    // a timeout first: the passes after the barrier that gave up never ran, so whatever else
    // the word holds may follow from the incomplete state
    if (err & kErrTimeout) {
      // grid buffers may be dirty
      h->initialized = false;
      h->T_recorded = 0;
      return fail(h, MPM_ERR_TIMEOUT, "a bounded device wait gave up (call mpm_set_initial again)");
    }
    if (err & kErrOOB) return fail(h, MPM_ERR_OOB, "a particle's stencil left the grid");
    if (err & kErrNonFinite) return fail(h, MPM_ERR_NONFINITE, "non-finite value or det F <= 0");
    if (err & kErrRange)
      return fail(h, MPM_ERR_RANGE, "deterministic mode: a fixed-point grid contribution left its range");
  }
  return MPM_OK;
}

int mpm_set_option(mpm_handle* h, int32_t key, int64_t value) {
  if (!h) return fail(nullptr, MPM_ERR_ARG, "handle is NULL");
  if (key == MPM_OPT_GATHER_CAPACITY || key == MPM_OPT_TILE_CAPACITY || key == MPM_OPT_SMEM_TILE) {
    // try the value on a copy of the capacities first: a size the device cannot hold is
    // refused here rather than by a launch
    const int g0 = h->gather_capacity, t0 = h->tile_capacity;
    const bool s0 = h->smem_tile;
    if (key == MPM_OPT_GATHER_CAPACITY && (value == 0 || (value >= 27 && value <= 12288))) h->gather_capacity = (int)value;
    if (key == MPM_OPT_TILE_CAPACITY && value >= 27 && value <= 12288) h->tile_capacity = (int)value;
    if (key == MPM_OPT_SMEM_TILE) h->smem_tile = value != 0;
    std::string why;
    const bool ok = capacities_fit(h, &why);
    h->gather_capacity = g0;
    h->tile_capacity = t0;
    h->smem_tile = s0;
    if (!ok) return fail(h, MPM_ERR_ARG, why);
  }
  switch (key) {
    case MPM_OPT_USE_GRAPHS: h->use_graphs = value != 0; break;
    case MPM_OPT_SMEM_TILE: h->smem_tile = value != 0; break;
    case MPM_OPT_BUCKET_SCATTER: h->bucket_scatter = value != 0; break;
    case MPM_OPT_SORT_ORDER:
      if (value < 0 || value > 2) return fail(h, MPM_ERR_ARG, "sort order must be 0, 1 or 2");
      h->sort_order = (int)value;
      break;
    case MPM_OPT_PAIR_SCATTER:
      if (value < 0 || value > 3) return fail(h, MPM_ERR_ARG, "pair scatter must be in [0, 3]");
      h->pair_scatter = (int)value;
      break;
    case MPM_OPT_GATHER_CAPACITY:
      if (value != 0 && (value < 27 || value > 12288))
        return fail(h, MPM_ERR_ARG, "gather capacity must be 0 or in [27, 12288]");
      h->gather_capacity = (int)value;
      break;
    case MPM_OPT_GRID_BLOCKS:
      if (value < 0 || value > 65535) return fail(h, MPM_ERR_ARG, "grid blocks must be in [0, 65535]");
      h->grid_blocks = (int)value;
      break;
    case MPM_OPT_POLAR_CACHE: h->use_polar_cache = value != 0; break;
    case MPM_OPT_GRID_RECOMPUTE: h->grid_recompute = value != 0; break;
    case MPM_OPT_PERSISTENT: h->persistent = value != 0; break;
    case MPM_OPT_OVERLAP_RESIM: h->overlap = value != 0; break;
    case MPM_OPT_PERSISTENT_CHUNK:
      if (value < 0 || value > (1 << 30)) return fail(h, MPM_ERR_ARG, "persistent chunk must be >= 0");
      h->persistent_chunk = (int)value;
      break;
    case MPM_OPT_BARRIER_TIMEOUT_US:
      if (value < 1 || value > 600000000) return fail(h, MPM_ERR_ARG, "barrier timeout must be in [1 us, 600 s]");
      h->barrier_timeout_us = value;
      break;
    case MPM_OPT_BARRIER_TEST_EXTRA:
      if (value < 0 || value > 1024) return fail(h, MPM_ERR_ARG, "barrier test arrivals must be in [0, 1024]");
      h->barrier_extra = (unsigned)value;
      break;
    case MPM_OPT_PROFILE:
      h->profile = value != 0;
      h->ev_records.clear();
      break;
    case MPM_OPT_TILE_CAPACITY:
      if (value < 27 || value > 12288) return fail(h, MPM_ERR_ARG, "tile capacity must be in [27, 12288]");
      h->tile_capacity = (int)value;
      break;
    default: return fail(h, MPM_ERR_ARG, "unknown option");
  }
  drop_graphs(h);
  return MPM_OK;
}

int mpm_get_info(mpm_handle* h, int32_t key, int64_t* value) {
  if (!h || !value) return fail(h, MPM_ERR_ARG, "NULL argument");
  switch (key) {
    case MPM_INFO_KERNEL_LAUNCHES: *value = h->launches; return MPM_OK;
    case MPM_INFO_N_TOTAL: *value = h->m.N; return MPM_OK;
    case MPM_INFO_STEPS_RECORDED: *value = h->T_recorded; return MPM_OK;
    case MPM_INFO_KEEPS_SEGMENT_GRIDS: *value = h->m.store_grids && !h->grid_recompute; return MPM_OK;
    case MPM_INFO_ACT_PARAMS: *value = h->m.n_act; return MPM_OK;
    case MPM_INFO_CKPT_EVERY: *value = h->m.K; return MPM_OK;
    case MPM_INFO_POLAR_FP64: *value = MPM_POLAR_FP64; return MPM_OK;
    case MPM_INFO_GATHER_BOXES:
    case MPM_INFO_GATHER_BOX_OVERFLOWS: {
      unsigned long long st[2] = {0, 0};
      cudaError_t e = cudaStreamSynchronize(h->last_stream);
      if (e == cudaSuccess) e = cudaMemcpy(st, h->at<char>(h->L.box_stats), 16, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return cuda_fail(h, e, "read gather-box counters");
      *value = (int64_t)st[key == MPM_INFO_GATHER_BOXES ? 0 : 1];
      return MPM_OK;
    }
  }
  return fail(h, MPM_ERR_ARG, "unknown info key");
}

int mpm_get_profile(mpm_handle* h, int32_t kind, int64_t* launches, double* total_ms) {
  if (!h || !launches || !total_ms) return fail(h, MPM_ERR_ARG, "NULL argument");
  int64_t n = 0;
  double ms = 0.0;
  for (auto& r : h->ev_records) {
    if (r.first != kind) continue;
    cudaError_t e = cudaEventSynchronize(r.second.second);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaEventSynchronize");
    float t = 0.0f;
    e = cudaEventElapsedTime(&t, r.second.first, r.second.second);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaEventElapsedTime");
    ++n;
    ms += t;
  }
  *launches = n;
  *total_ms = ms;
  return MPM_OK;
}

const char* mpm_last_error(mpm_handle* h) {
  return h ? h->last_error.c_str() : g_static_error.c_str();
}

void mpm_destroy(mpm_handle* h) {
  if (!h) return;
  drop_graphs(h);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->side_stream) {
    cudaStreamSynchronize(h->side_stream);  // normally idle: its work is joined into the main stream
    cudaStreamDestroy(h->side_stream);
  }
  for (cudaEvent_t ev : {h->ev_fork, h->ev_free, h->ev_resim, h->ev_join})
    if (ev) cudaEventDestroy(ev);
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  delete h;
}

}  // extern "C"
