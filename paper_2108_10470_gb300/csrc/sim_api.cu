// C ABI of the GB300 articulated-body step (declared in include/sim.h): model validation,
// flattening of environments into env-type tables, device buffers, views, launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <vector>

#include "../../include/sim.h"
#include "sim_internal.h"
#include "launch.h"

using namespace artsim;

namespace {

thread_local std::string g_last_error;

struct TypePlan {
  EnvTypeTable tab;
  SmemLayout lay;
  std::vector<int> envs;
  int G = 32;                 // lanes per env (8, 16 or 32)
  int G_min = 32;             // fewest lanes that hold the type's links, DOFs and shapes
  int warps_per_cta = 4;      // per-type launches
  int groups_per_block = 4;
  size_t smem_bytes = 0;
  int env_off = 0;            // offset into the concatenated env-id array
  float* scratch = nullptr;   // global rows, per-type launches: one slot per group of the launch
  size_t scratch_floats = 0;
  float* pscratch = nullptr;  // global rows, persistent launch: one slot per resident group
  size_t pscratch_floats = 0;
  float* ybg = nullptr;       // reverse pass with Y outside the arena: Y's adjoint, one slot per env
  size_t ybg_floats = 0;
  double env_cost = 0.0;      // relative cost of one env (persistent tile order)
};

}  // namespace

struct sim_s {
  uint32_t magic = 0x5349414du;
  int device = 0;
  cudaStream_t stream = nullptr;
  int n_envs = 0, actors_per_env = 0;
  int64_t N_A = 0, N_D = 0, N_B = 0;
  int pair_stride = 0, cache_stride = 0, dof_row_stride = 0;
  sim_params params{};
  std::vector<TypePlan> types;
  bool contiguous_single_type = false;
  EnvTypeTable* d_types = nullptr;
  int* d_env_ids = nullptr;
  int* d_dof_base = nullptr;    // n_envs + 1
  int* d_body_base = nullptr;   // n_envs + 1
  int* d_actor_base = nullptr;  // n_envs + 1: first root-state row of each env
  int* d_actor_env = nullptr;   // N_A: env of each actor
  float* root = nullptr;
  float* dof = nullptr;
  float* act = nullptr;
  float* net_force = nullptr;
  float* cache = nullptr;
  int* pairs = nullptr;
  int* n_pairs = nullptr;
  unsigned* sig = nullptr;
  int* status = nullptr;
  float* pos_target = nullptr;   // (N_D,) drive targets
  float* vel_target = nullptr;
  float* dof_force = nullptr;    // (N_D,) out
  float* body_state = nullptr;   // (N_B, 13) out
  float* body_force = nullptr;   // (N_B, 6) external force, torque
  // persistent heterogeneous launch (SIM_FLAG_PERSISTENT)
  bool persistent = false;
  int p_grid = 0, p_warps = 0, p_warp_words = 0;
  bool p_ball = false;  // the persistent instantiation with the ball-joint code
  size_t p_smem = 0;
  std::vector<int> p_order;       // env types, costliest first
  unsigned* d_counter = nullptr;  // tile counter and finished-warp counter
  // per-type launches of a step with several env types run concurrently: type 0 on the step's
  // stream, type t >= 1 on type_streams[t - 1], forked from and joined back into the step's stream
  std::vector<cudaStream_t> type_streams;
  std::vector<cudaEvent_t> type_events;  // [0] fork, [t] join of type t
  // CUDA graph of one step (SIM_FLAG_GRAPH), captured on cap_stream, replayed on stream
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  float graph_dt = 0.f;
  int graph_substeps = 0;
  // sim_step_vjp by the reverse pass: a copy of the step's input state stepped by the taped step,
  // and the tape (allocated on first use)
  // sim_step_host with pinned host buffers: their device addresses, for the duration of the call
  const float* zc_act = nullptr;
  float* zc_root = nullptr;
  float* zc_dof = nullptr;
  float* rv_state = nullptr;
  size_t rv_state_floats = 0;
  float* rv_tape = nullptr;
  size_t rv_tape_floats = 0;
};

namespace {

std::mutex g_handles_mu;
std::set<const sim_s*> g_handles;

bool valid_handle(const sim_s* h) {
  std::lock_guard<std::mutex> lk(g_handles_mu);
  return h && g_handles.count(h) && h->magic == 0x5349414du;
}

int cuda_fail(cudaError_t e, const char* what) {
  char buf[256];
  snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
  g_last_error = buf;
  return SIM_ERR_CUDA;
}
#define CK(call)                                   \
  do {                                             \
    cudaError_t e__ = (call);                      \
    if (e__ != cudaSuccess) return cuda_fail(e__, #call); \
  } while (0)

bool finite(float x) { return std::isfinite(x); }

void quat_to_rot(const float* qin, float* R) {
  double q[4] = {qin[0], qin[1], qin[2], qin[3]};
  const double n = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  for (double& x : q) x /= n;
  const double x = q[0], y = q[1], z = q[2], w = q[3];
  const double m[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w),
                       2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w),
                       2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)};
  for (int k = 0; k < 9; ++k) R[k] = (float)m[k];
}

int validate_model(const sim_model_desc& m) {
  if (m.n_links < 1 || m.n_links > kMaxLinks || m.n_shapes < 0 || m.n_shapes > kMaxShapes) return SIM_ERR_CAPACITY;
  if (!m.parent || !m.joint_type || !m.joint_axis || !m.parent_pos || !m.parent_quat || !m.mass || !m.com ||
      !m.inertia || !m.armature || !m.damping || !m.limit_lo || !m.limit_hi || !m.has_limit || !m.is_virtual)
    return SIM_ERR_INVALID_ARG;
  if (m.n_shapes > 0 && (!m.shape_link || !m.shape_type || !m.shape_size || !m.shape_pos || !m.shape_quat ||
                         !m.shape_friction))
    return SIM_ERR_INVALID_ARG;
  if (m.parent[0] != -1) return SIM_ERR_TOPOLOGY;
  if (m.joint_type[0] != SIM_JOINT_FREE && m.joint_type[0] != SIM_JOINT_FIXED) return SIM_ERR_TOPOLOGY;
  for (int i = 0; i < m.n_links; ++i) {
    if (i > 0) {
      if (m.parent[i] < 0 || m.parent[i] >= i) return SIM_ERR_TOPOLOGY;
      const int jt = m.joint_type[i];
      if (jt != SIM_JOINT_FIXED && jt != SIM_JOINT_REVOLUTE && jt != SIM_JOINT_PRISMATIC && jt != SIM_JOINT_SPHERICAL)
        return SIM_ERR_TOPOLOGY;
    }
    for (int k = 0; k < 3; ++k)
      if (!finite(m.joint_axis[3 * i + k]) || !finite(m.parent_pos[3 * i + k]) || !finite(m.com[3 * i + k]))
        return SIM_ERR_INVALID_ARG;
    double qn = 0;
    for (int k = 0; k < 4; ++k) {
      if (!finite(m.parent_quat[4 * i + k])) return SIM_ERR_INVALID_ARG;
      qn += (double)m.parent_quat[4 * i + k] * m.parent_quat[4 * i + k];
    }
    if (qn < 1e-12) return SIM_ERR_INVALID_ARG;
    if (!(m.mass[i] >= 0.f) || !finite(m.mass[i])) return SIM_ERR_INVALID_ARG;
    if (i == 0 && m.joint_type[0] == SIM_JOINT_FREE && !(m.mass[0] > 0.f)) return SIM_ERR_INVALID_ARG;
    const float* I = m.inertia + 6 * i;
    for (int k = 0; k < 6; ++k)
      if (!finite(I[k])) return SIM_ERR_INVALID_ARG;
    // positive semi-definite: leading minors and diagonal non-negative (small tolerance)
    const double a = I[0], b = I[1], c = I[2], xy = I[3], xz = I[4], yz = I[5];
    const double tol = 1e-9 * (std::fabs(a) + std::fabs(b) + std::fabs(c) + 1e-12);
    const double det = a * (b * c - yz * yz) - xy * (xy * c - yz * xz) + xz * (xy * yz - b * xz);
    if (a < -tol || b < -tol || c < -tol || a * b - xy * xy < -tol * tol || det < -tol * tol * tol)
      return SIM_ERR_INVALID_ARG;
    if (i == 0 && m.joint_type[0] == SIM_JOINT_FREE && !(a > 0 && b > 0 && c > 0)) return SIM_ERR_INVALID_ARG;
    if (!(m.armature[i] >= 0.f) || !(m.damping[i] >= 0.f) || !finite(m.armature[i]) || !finite(m.damping[i]))
      return SIM_ERR_INVALID_ARG;
    const int jt = m.joint_type[i];
    if (i > 0 && (jt == SIM_JOINT_REVOLUTE || jt == SIM_JOINT_PRISMATIC)) {
      const float* ax = m.joint_axis + 3 * i;
      const double an = std::sqrt((double)ax[0] * ax[0] + (double)ax[1] * ax[1] + (double)ax[2] * ax[2]);
      if (an < 1e-6) return SIM_ERR_INVALID_ARG;
      if (m.has_limit[i] && (!finite(m.limit_lo[i]) || !finite(m.limit_hi[i]) || m.limit_lo[i] > m.limit_hi[i]))
        return SIM_ERR_INVALID_ARG;
    }
    if (m.has_limit[i] > 1 || m.is_virtual[i] > 1) return SIM_ERR_INVALID_ARG;
    if (jt == SIM_JOINT_SPHERICAL &&  // ball joints take no limits and no drives
        (m.has_limit[i] || (m.drive_stiffness && m.drive_stiffness[i] != 0.f) || (m.drive_damping && m.drive_damping[i] != 0.f)))
      return SIM_ERR_INVALID_ARG;
    if (m.drive_stiffness && !(m.drive_stiffness[i] >= 0.f && finite(m.drive_stiffness[i]))) return SIM_ERR_INVALID_ARG;
    if (m.drive_damping && !(m.drive_damping[i] >= 0.f && finite(m.drive_damping[i]))) return SIM_ERR_INVALID_ARG;
  }
  if (m.n_tendons < 0 || m.n_tendons > kMaxTendons) return SIM_ERR_CAPACITY;
  if (m.n_tendons > 0) {
    if (!m.tendon_joint_count || !m.tendon_link || !m.tendon_coef || !m.tendon_stiffness || !m.tendon_damping ||
        !m.tendon_rest_length || !m.tendon_limit_lo || !m.tendon_limit_hi || !m.tendon_has_limit)
      return SIM_ERR_INVALID_ARG;
    int e = 0;
    for (int t = 0; t < m.n_tendons; ++t) {
      const int cnt = m.tendon_joint_count[t];
      if (cnt < 1 || cnt > kMaxTendonJoints) return SIM_ERR_CAPACITY;
      for (int k = 0; k < cnt; ++k, ++e) {
        const int li = m.tendon_link[e];
        if (li < 1 || li >= m.n_links) return SIM_ERR_INVALID_ARG;
        if (m.joint_type[li] != SIM_JOINT_REVOLUTE && m.joint_type[li] != SIM_JOINT_PRISMATIC) return SIM_ERR_INVALID_ARG;
        if (!finite(m.tendon_coef[e])) return SIM_ERR_INVALID_ARG;
      }
      if (!(m.tendon_stiffness[t] >= 0.f) || !(m.tendon_damping[t] >= 0.f) || !finite(m.tendon_stiffness[t]) ||
          !finite(m.tendon_damping[t]) || !finite(m.tendon_rest_length[t]) || m.tendon_has_limit[t] > 1)
        return SIM_ERR_INVALID_ARG;
      if (m.tendon_has_limit[t] && (!finite(m.tendon_limit_lo[t]) || !finite(m.tendon_limit_hi[t]) ||
                                    m.tendon_limit_lo[t] > m.tendon_limit_hi[t]))
        return SIM_ERR_INVALID_ARG;
    }
  }
  for (int s = 0; s < m.n_shapes; ++s) {
    const int li = m.shape_link[s];
    if (li < 0 || li >= m.n_links || m.is_virtual[li]) return SIM_ERR_INVALID_ARG;
    const int st = m.shape_type[s];
    if (st != SIM_SHAPE_SPHERE && st != SIM_SHAPE_CAPSULE && st != SIM_SHAPE_BOX) return SIM_ERR_INVALID_ARG;
    const float* sz = m.shape_size + 3 * s;
    const int need = (st == SIM_SHAPE_SPHERE) ? 1 : (st == SIM_SHAPE_CAPSULE ? 2 : 3);
    for (int k = 0; k < need; ++k)
      if (!(sz[k] > 0.f) || !finite(sz[k])) return SIM_ERR_INVALID_ARG;
    if (!(m.shape_friction[s] >= 0.f) || !finite(m.shape_friction[s])) return SIM_ERR_INVALID_ARG;
    for (int k = 0; k < 3; ++k)
      if (!finite(m.shape_pos[3 * s + k]) || !finite(sz[k])) return SIM_ERR_INVALID_ARG;
    double qn = 0;
    for (int k = 0; k < 4; ++k) {
      if (!finite(m.shape_quat[4 * s + k])) return SIM_ERR_INVALID_ARG;
      qn += (double)m.shape_quat[4 * s + k] * m.shape_quat[4 * s + k];
    }
    if (qn < 1e-12) return SIM_ERR_INVALID_ARG;
  }
  return SIM_OK;
}

int ndof_of(const sim_model_desc& m, int i) {
  const int jt = m.joint_type[i];
  if (i == 0) return jt == SIM_JOINT_FREE ? 6 : 0;
  if (jt == SIM_JOINT_SPHERICAL) return 3;
  return (jt == SIM_JOINT_REVOLUTE || jt == SIM_JOINT_PRISMATIC) ? 1 : 0;
}

// Flatten the actors of one environment type into a forest of links.
int build_type(const sim_model_desc* models, const std::vector<int>& actor_models, const sim_params& p,
               EnvTypeTable& T) {
  std::memset(&T, 0, sizeof(T));
  int L = 0, n = 0, nj = 0, ns = 0, nc = 0, nb = 0;
  for (int k = 0; k < kMaxLinks; ++k) { T.first_child[k] = -1; T.next_sibling[k] = -1; T.gdof[k] = -1; T.jdof[k] = -1; T.body[k] = -1; }
  if ((int)actor_models.size() > kMaxActors) return SIM_ERR_CAPACITY;
  for (size_t a = 0; a < actor_models.size(); ++a) {
    const sim_model_desc& m = models[actor_models[a]];
    const int base = L;
    if (L + m.n_links > kMaxLinks || ns + m.n_shapes > kMaxShapes) return SIM_ERR_CAPACITY;
    for (int i = 0; i < m.n_links; ++i) {
      const int l = base + i;
      const int nd = ndof_of(m, i);
      if (n + nd > kMaxGen) return SIM_ERR_CAPACITY;
      T.parent[l] = (i == 0) ? -1 : base + m.parent[i];
      T.jtype[l] = m.joint_type[i];
      T.depth[l] = (i == 0) ? 0 : T.depth[T.parent[l]] + 1;
      T.actor[l] = (int)a;
      T.aroot[l] = base;
      T.gdof[l] = nd ? n : -1;
      if (nd == 6) {
        for (int k = 0; k < 6; ++k) { T.dof_link[n + k] = l; T.dof_comp[n + k] = k; }
      } else if (nd == 1 || nd == 3) {  // a joint's DOFs (armature on each)
        for (int k = 0; k < nd; ++k) { T.dof_link[n + k] = l; T.dof_comp[n + k] = -1; }
        T.jdof[l] = nj;
        nj += nd;
        if (nd == 3) T.has_ball = 1;
      }
      n += nd;
      double an = 1.0;
      const float* ax = m.joint_axis + 3 * i;
      if (nd == 1) an = std::sqrt((double)ax[0] * ax[0] + (double)ax[1] * ax[1] + (double)ax[2] * ax[2]);
      for (int k = 0; k < 3; ++k) {
        T.axis[k][l] = nd == 1 ? (float)(ax[k] / an) : 0.f;
        T.ppos[k][l] = m.parent_pos[3 * i + k];
        T.com[k][l] = m.com[3 * i + k];
      }
      float R[9];
      quat_to_rot(m.parent_quat + 4 * i, R);
      for (int k = 0; k < 9; ++k) T.prot[k][l] = R[k];
      T.mass[l] = m.mass[i];
      for (int k = 0; k < 6; ++k) T.inertia[k][l] = m.inertia[6 * i + k];
      T.armature[l] = m.armature[i];
      T.damping[l] = m.damping[i];
      T.has_limit[l] = (nd == 1 && m.has_limit[i]) ? 1 : 0;
      T.drive_kp[l] = (nd == 1 && i > 0 && m.drive_stiffness) ? m.drive_stiffness[i] : 0.f;
      T.drive_kd[l] = (nd == 1 && i > 0 && m.drive_damping) ? m.drive_damping[i] : 0.f;
      if (T.drive_kp[l] != 0.f || T.drive_kd[l] != 0.f) T.has_drives = 1;
      T.lo[l] = m.limit_lo[i];
      T.hi[l] = m.limit_hi[i];
      // both rows of a joint can be active only if its range is below twice the margin; the
      // slack covers rounding of the two float comparisons near that boundary
      T.lim_slots[l] = T.has_limit[l] ? ((T.hi[l] - T.lo[l] < 2.f * p.limit_margin + 1e-4f) ? 2 : 1) : 0;
      T.body[l] = m.is_virtual[i] ? -1 : nb++;
    }
    for (int s = 0; s < m.n_shapes; ++s) {
      const int e = ns + s;
      T.shape_link[e] = base + m.shape_link[s];
      T.shape_type[e] = m.shape_type[s];
      T.cand_off[e] = nc;
      nc += (m.shape_type[s] == SIM_SHAPE_SPHERE) ? 1 : (m.shape_type[s] == SIM_SHAPE_CAPSULE ? 2 : 8);
      for (int k = 0; k < 3; ++k) {
        T.shape_size[k][e] = m.shape_size[3 * s + k];
        T.shape_pos[k][e] = m.shape_pos[3 * s + k];
      }
      float R[9];
      quat_to_rot(m.shape_quat + 4 * s, R);
      for (int k = 0; k < 9; ++k) T.shape_rot[k][e] = R[k];
      T.shape_mu[e] = std::max(m.shape_friction[s], p.ground_friction);
      T.shape_fr[e] = m.shape_friction[s];
    }
    int e = 0;
    for (int t = 0; t < m.n_tendons; ++t) {
      if (T.n_tendons >= kMaxTendons) return SIM_ERR_CAPACITY;
      const int k = T.n_tendons++;
      T.ten_n[k] = m.tendon_joint_count[t];
      for (int j = 0; j < T.ten_n[k]; ++j, ++e) {
        T.ten_link[k][j] = base + m.tendon_link[e];
        T.ten_coef[k][j] = m.tendon_coef[e];
      }
      T.ten_k[k] = m.tendon_stiffness[t];
      T.ten_d[k] = m.tendon_damping[t];
      T.ten_rest[k] = m.tendon_rest_length[t];
      T.ten_has_limit[k] = m.tendon_has_limit[t];
      T.ten_lo[k] = m.tendon_limit_lo[t];
      T.ten_hi[k] = m.tendon_limit_hi[t];
    }
    L += m.n_links;
    ns += m.n_shapes;
  }
  // capsule-box pairs across actors (a < b), candidates after every ground candidate
  T.n_ground_cand = nc;
  int np = 0;
  for (int sa = 0; sa < ns; ++sa)
    for (int sb = sa + 1; sb < ns; ++sb) {
      if (T.actor[T.shape_link[sa]] == T.actor[T.shape_link[sb]]) continue;
      const int ta = T.shape_type[sa], tb = T.shape_type[sb];
      if (!((ta == kCapsule && tb == kBox) || (ta == kBox && tb == kCapsule))) continue;
      if (np >= kMaxPairs) return SIM_ERR_CAPACITY;
      T.pair_a[np] = sa;
      T.pair_b[np] = sb;
      ++np;
    }
  T.n_pairs = np;
  nc += kPairSlots * np;
  if (nc > kMaxCand) return SIM_ERR_CAPACITY;
  // children lists (ascending), ancestor DOF masks, depth
  int maxd = 0;
  for (int l = L - 1; l >= 0; --l) {
    const int pa = T.parent[l];
    if (pa >= 0) { T.next_sibling[l] = T.first_child[pa]; T.first_child[pa] = l; }
  }
  int lim_cap = 0;
  for (int l = 0; l < L; ++l) {
    unsigned mask = 0u;
    for (int a = l; a >= 0; a = T.parent[a]) {
      const int nd = (T.parent[a] < 0) ? (T.jtype[a] == kFree ? 6 : 0)
                                        : (T.jtype[a] == kSpherical ? 3
                                                                    : ((T.jtype[a] == kRevolute || T.jtype[a] == kPrismatic) ? 1 : 0));
      for (int k = 0; k < nd; ++k) mask |= 1u << (T.gdof[a] + k);
    }
    T.anc[l] = mask;
    maxd = std::max(maxd, T.depth[l]);
    lim_cap += T.lim_slots[l];
  }
  T.n_links = L;
  T.n_gen = n;
  T.n_jdof = nj;
  T.n_shapes = ns;
  T.n_cand = nc;
  T.n_body = nb;
  T.n_actors = (int)actor_models.size();
  T.max_depth = maxd;
  for (int t = 0; t < T.n_tendons; ++t) lim_cap += T.ten_has_limit[t] ? 2 : 0;
  T.lim_cap = lim_cap;
  T.row_cap = lim_cap + 3 * nc;
  T.cache_len = 3 * nc + 2 * nj + 2 * T.n_tendons;
  const int need = std::max(std::max(L, n), std::max(ns, 1));
  T.group = need <= 8 ? 8 : (need <= 16 ? 16 : 32);
  return SIM_OK;
}

// Largest per-env shared arena sized to the row capacity; bigger worst cases, and every env type
// with shape pairs, keep their contact / row blocks in global scratch (the Humanoid's 18 KB stays
// in shared memory, the hand-with-cube's ~60 KB does not).
constexpr int kSharedArenaLimit = 24 * 1024;

// Per-CTA dynamic shared memory cap used by the planner.
constexpr size_t kMaxSmemPerCta = 220 * 1024;

// Residency of the step kernels: 128 registers x 128 threads (__launch_bounds__(128, 4)) leave 16
// warps per SM; the SM's shared memory and the part of it reserved per CTA.
constexpr int kStepWarpsPerSm = 16;
constexpr int kSmemPerSm = 228 * 1024;
constexpr int kSmemReservedPerCta = 1024;

// Layout of one env's arena for G lanes per env; rows_global puts the contact and row blocks in a
// per-env slot of global scratch instead of shared memory. envs_per_cta > 0 lets a shared-rows
// layout at G = 32 size its Y region below the type's row capacity (a global Y slot per group
// then serves the substeps with more rows); 0 keeps the whole capacity in shared memory.
SmemLayout make_layout(const EnvTypeTable& T, int G, bool rows_global, int envs_per_cta) {
  SmemLayout Ly{};
  const int n = std::max(T.n_gen, 1);
  const int L = T.n_links;
  Ly.rcap = std::max(T.row_cap, 1);
  Ly.RS = Ly.rcap | 1;
  Ly.MS = n | 1;
  Ly.ccap = std::max(T.n_cand, 1);
  auto al4 = [](int x) { return (x + 3) & ~3; };
  // ground-only env types keep the 9-word contact record (no body b, normal +z)
  const int conw = T.n_pairs > 0 ? kConWords : 9;
  int o = 0;
  if (!rows_global) {
    const int full = n * Ly.RS;
    int phase = std::max(L * kLinkWords, full);
    if (envs_per_cta > 0 && G == 32) {
      // The Y region (Y of the substep's R rows at stride R | 1, then the Delassus block when it
      // fits) is sized to what the shared memory of the register-limited residency leaves per env,
      // not to the row capacity, which most substeps use a fraction of (the Humanoid: 96 rows of
      // capacity, fewer than 42 in every substep of a 128-env, 140-step oracle rollout, 17.5 on
      // average). Its arena: 18.1 -> 14.0 KB per env, four 4-env CTAs per SM instead of three; Y
      // fits for up to 61 rows, W too for up to 29. It holds at least the link slots and Y of 32 rows.
      const int rest = al4(al4(6 * n + n * Ly.MS + 5 * n + conw * Ly.ccap) + 6 * Ly.rcap + 3 * L);
      const int ctas = std::max(1, kStepWarpsPerSm / (envs_per_cta * G / 32));
      const int budget = (((kSmemPerSm / ctas - kSmemReservedPerCta) / 4) / envs_per_cta - rest) & ~3;
      const int lo = al4(std::max(L * kLinkWords, n * 33));
      if (lo < phase && budget < phase) phase = std::max(lo, budget);
    }
    if (phase < full) Ly.scratch_words = al4(full);  // the global Y slot of the substeps past it
    Ly.link = o;
    Ly.Y = o;
    Ly.ywords = phase;
    o += phase;
    Ly.SD = o; o += 6 * n;
    Ly.M = o; o += n * Ly.MS;
    Ly.vec = o; o += 5 * n;
    Ly.con = o; o += conw * Ly.ccap;
    o = al4(o);
    Ly.rowc = o; o += 4 * Ly.rcap;
    Ly.lam = o; o += Ly.rcap;
    Ly.rowa = o; o += Ly.rcap;
    Ly.frc = o; o += 3 * L;
    Ly.total = al4(o);
  } else {
    Ly.grows = 1;
    int g = 0;
    Ly.con = g; g += conw * Ly.ccap;
    g = al4(g);
    Ly.rowc = g; g += 4 * Ly.rcap;
    Ly.lam = g; g += Ly.rcap;
    Ly.rowa = g; g += Ly.rcap;
    Ly.Y = g; g += n * Ly.RS;
    Ly.scratch_words = al4(g);
    Ly.ywords = Ly.scratch_words - Ly.Y;
    Ly.link = o; o += L * kLinkWords;
    Ly.SD = o; o += 6 * n;
    Ly.M = o; o += n * Ly.MS;
    Ly.vec = o; o += 5 * n;
    Ly.frc = o; o += 3 * L;
    Ly.ball = o; o += T.has_ball ? kBallWords * L : 0;
    Ly.total = al4(o);
  }
  // Groups that share a warp (G < 32) must not share banks: pad the per-group stride to G mod 32
  // so the g-th group of a warp is shifted by g * G banks (the row stride RS is odd, so each
  // group's lanes also fall on distinct banks).
  if (G < 32)
    while (Ly.total % 32 != G) Ly.total += 4;
  return Ly;
}

// Default placement: rows in global scratch when the all-shared arena would exceed
// kSharedArenaLimit, and always for env types with shape pairs or ball joints (the pair phase and
// the 3-DOF joint blocks are compiled into the global-rows variant only).
bool default_rows_global(const EnvTypeTable& T, int G) {
  return T.n_pairs > 0 || T.has_ball || make_layout(T, G, false, 0).total * 4 > kSharedArenaLimit;
}

cudaError_t launch_type(const TypePlan& tp, const StepArgs& a, const TypeArgs& ta, cudaStream_t st) {
  return launch_step_kernel(tp.G, tp.lay.grows != 0, tp.tab.has_ball != 0, a, ta, tp.groups_per_block, tp.smem_bytes, st);
}

int variant_of(const TypePlan& tp) {
  return (tp.G == 8 ? kVar8 : (tp.G == 16 ? kVar16 : kVar32)) | (tp.lay.grows ? kVarRowsGlobal : 0);
}

int grow_buffer(float** buf, size_t* have, size_t need, const char* what) {
  if (need <= *have) return SIM_OK;
  float* p = nullptr;
  const cudaError_t e = cudaMalloc(&p, need * sizeof(float));
  if (e != cudaSuccess) return cuda_fail(e, what);
  if (*buf) cudaFree(*buf);
  *buf = p;
  *have = need;
  return SIM_OK;
}

// Lay out one env type for G lanes per env, its rows in shared or global memory, and `warps`
// warps per CTA of its per-type launch; allocates the per-type scratch that launch needs.
int configure_type(TypePlan& tp, int G, bool rows_global, int warps, bool per_type_scratch) {
  if ((G != 8 && G != 16 && G != 32) || G < tp.G_min || (warps != 1 && warps != 2 && warps != 4)) {
    g_last_error = "type config: lanes per env must be 8, 16 or 32 and hold the type; warps 1, 2 or 4";
    return SIM_ERR_INVALID_ARG;
  }
  if ((tp.tab.n_pairs > 0 || tp.tab.has_ball) && !rows_global) {
    g_last_error = "type config: env types with shape pairs or ball joints keep their rows in global memory";
    return SIM_ERR_INVALID_ARG;
  }
  const int gpb = warps * 32 / G;
  const SmemLayout Ly = make_layout(tp.tab, G, rows_global, gpb);
  const size_t smem = (size_t)gpb * Ly.total * 4;
  if (smem > kMaxSmemPerCta) {
    g_last_error = "type config: the CTA's shared arena exceeds 220 KB";
    return SIM_ERR_CAPACITY;
  }
  if (Ly.scratch_words && per_type_scratch) {  // global rows, or a shared-rows layout's Y slots
    const size_t slots = (tp.envs.size() + gpb - 1) / gpb * gpb;
    const int rc = grow_buffer(&tp.scratch, &tp.scratch_floats, slots * (size_t)Ly.scratch_words,
                               "cudaMalloc (global rows scratch)");
    if (rc != SIM_OK) return rc;
  }
  // the attribute is a cap per kernel instantiation, shared by every type that uses it: set the
  // planner's maximum rather than this type's size
  const cudaError_t e = set_step_kernel_smem_cap(G, Ly.grows != 0, tp.tab.has_ball != 0, kMaxSmemPerCta);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
  tp.G = G;
  tp.lay = Ly;
  tp.warps_per_cta = warps;
  tp.groups_per_block = gpb;
  tp.smem_bytes = smem;
  return SIM_OK;
}

// Resident grid, per-warp arena, global-rows slots and tile order of the persistent launch.
int plan_persistent(sim_s* h) {
  if (h->types.size() > (size_t)kMaxPersistTypes) {
    g_last_error = "persistent launch: more than 8 env types";
    return SIM_ERR_CAPACITY;
  }
  int warp_words = 0;
  for (const TypePlan& tp : h->types) warp_words = std::max(warp_words, (32 / tp.G) * tp.lay.total);
  const size_t smem = 4 * (size_t)warp_words * sizeof(float);
  if (smem > kMaxSmemPerCta) {
    g_last_error = "persistent launch: four warps' arenas exceed 220 KB";
    return SIM_ERR_CAPACITY;
  }
  bool ball = false;
  for (const TypePlan& tp : h->types) ball = ball || tp.tab.has_ball;
  h->p_ball = ball;
  CK(set_persistent_kernel_smem_cap(ball, kMaxSmemPerCta));
  int per_sm = 0, sms = 0;
  CK(persistent_kernel_occupancy(ball, &per_sm, smem));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
  if (per_sm < 1) {
    g_last_error = "persistent launch: no CTA fits on an SM";
    return SIM_ERR_CAPACITY;
  }
  h->p_grid = per_sm * sms;
  h->p_warps = h->p_grid * 4;
  h->p_smem = smem;
  h->p_warp_words = warp_words;
  for (TypePlan& tp : h->types)
    if (tp.lay.scratch_words) {
      const size_t need = (size_t)h->p_warps * (32 / tp.G) * tp.lay.scratch_words;
      const int rc = grow_buffer(&tp.pscratch, &tp.pscratch_floats, need, "cudaMalloc (persistent rows scratch)");
      if (rc != SIM_OK) return rc;
    }
  h->p_order.resize(h->types.size());
  for (size_t t = 0; t < h->types.size(); ++t) h->p_order[t] = (int)t;
  std::stable_sort(h->p_order.begin(), h->p_order.end(),
                   [&](int a, int b) { return h->types[a].env_cost > h->types[b].env_cost; });
  return SIM_OK;
}

// The derivative kernel covers env types with a bounded impulse cache.
int tangent_supported(const sim_s* h) {
  for (const TypePlan& tp : h->types)
    if (tp.tab.cache_len > 448) {
      g_last_error = "step derivative: env types with more than 448 impulse-cache entries are not supported";
      return SIM_ERR_CAPACITY;
    }
  return SIM_OK;
}

void drop_graph(sim_s* h) {
  if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
  h->graph_exec = nullptr;
}

void fill_common(const sim_s* h, float dt, int substeps, StepArgs& a) {
  const sim_params& p = h->params;
  a = StepArgs{};
  a.root = h->root; a.dof = h->dof; a.act = h->act; a.net_force = h->net_force; a.cache = h->cache;
  a.pairs = h->pairs; a.n_pairs = h->n_pairs; a.sig = h->sig; a.status = h->status;
  a.env_dof_base = h->d_dof_base; a.env_body_base = h->d_body_base; a.env_actor_base = h->d_actor_base;
  a.pos_target = h->pos_target; a.vel_target = h->vel_target; a.body_force = h->body_force;
  a.dof_force = h->dof_force; a.body_state = h->body_state;
  if (h->zc_act) { a.act = h->zc_act; a.act_copy = h->act; }
  a.root_out = h->zc_root; a.dof_out = h->zc_dof;
  a.cache_stride = h->cache_stride; a.pair_stride = h->pair_stride;
  a.dt = dt; a.h = dt / (float)substeps; a.substeps = substeps;
  a.gx = p.gravity[0]; a.gy = p.gravity[1]; a.gz = p.gravity[2];
  a.pos_iters = p.pos_iters; a.vel_iters = p.vel_iters;
  a.contact_offset = p.contact_offset; a.limit_margin = p.limit_margin;
  a.bias_coef = p.bias_coef; a.max_depen_vel = p.max_depen_vel; a.flags = p.flags;
}

void fill_type(const sim_s* h, size_t t, TypeArgs& ta) {
  const TypePlan& tp = h->types[t];
  ta = TypeArgs{};
  ta.type = h->d_types + t;
  ta.env_ids = h->contiguous_single_type ? nullptr : h->d_env_ids + tp.env_off;
  ta.env_first = 0;
  ta.n_launch_envs = (int)tp.envs.size();
  ta.scratch = tp.scratch;
  ta.lay = tp.lay;
}

// Enqueue one step on stream st: one persistent launch, or one launch per env type.
int launch_step(sim_s* h, cudaStream_t st, float dt, int substeps) {
  if (h->persistent) {
    PersistArgs P{};
    fill_common(h, dt, substeps, P.common);
    int acc = 0;
    for (size_t s = 0; s < h->p_order.size(); ++s) {
      const int k = h->p_order[s];
      const TypePlan& tp = h->types[k];
      fill_type(h, (size_t)k, P.types[k]);
      P.types[k].scratch = tp.lay.scratch_words ? tp.pscratch : nullptr;
      P.variant[k] = variant_of(tp);
      P.order[s] = k;
      const int per = 32 / tp.G;  // envs per warp tile
      acc += ((int)tp.envs.size() + per - 1) / per;
      P.tile_end[s] = acc;
    }
    P.n_tiles = acc;
    P.n_warps = h->p_warps;
    P.warp_words = h->p_warp_words;
    P.counter = h->d_counter;
    const cudaError_t e = launch_persistent_kernel(P, h->p_ball, h->p_grid, h->p_smem, st);
    if (e != cudaSuccess) return cuda_fail(e, "persistent_step_kernel launch");
    return SIM_OK;
  }
  StepArgs a;
  fill_common(h, dt, substeps, a);
  const size_t nt = h->types.size();
  if (nt > 1) {
    // the types write disjoint envs: launch them side by side (the smaller ones fill the SMs the
    // larger ones leave idle in their last wave), joined before the step's stream goes on; the
    // mixed 16384-env batch steps in 1.12 ms instead of 1.20 ms one type after another
    if (h->type_streams.size() < nt - 1) {
      while (h->type_streams.size() < nt - 1) {
        cudaStream_t s = nullptr;
        CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        h->type_streams.push_back(s);
      }
      while (h->type_events.size() < nt) {
        cudaEvent_t e = nullptr;
        CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        h->type_events.push_back(e);
      }
    }
    CK(cudaEventRecord(h->type_events[0], st));
    for (size_t t = 1; t < nt; ++t) CK(cudaStreamWaitEvent(h->type_streams[t - 1], h->type_events[0], 0));
    for (size_t t = 0; t < nt; ++t) {
      TypeArgs ta;
      fill_type(h, t, ta);
      const cudaError_t e = launch_type(h->types[t], a, ta, t == 0 ? st : h->type_streams[t - 1]);
      if (e != cudaSuccess) return cuda_fail(e, "step_kernel launch");
    }
    for (size_t t = 1; t < nt; ++t) {
      CK(cudaEventRecord(h->type_events[t], h->type_streams[t - 1]));
      CK(cudaStreamWaitEvent(st, h->type_events[t], 0));
    }
    return SIM_OK;
  }
  for (size_t t = 0; t < nt; ++t) {
    TypeArgs ta;
    fill_type(h, t, ta);
    const cudaError_t e = launch_type(h->types[t], a, ta, st);
    if (e != cudaSuccess) return cuda_fail(e, "step_kernel launch");
  }
  return SIM_OK;
}

// Capture one step (for this dt / substeps) into a graph on the handle's capture stream.
int capture_step(sim_s* h, float dt, int substeps) {
  drop_graph(h);
  if (!h->cap_stream) CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
  const int rc = launch_step(h, h->cap_stream, dt, substeps);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
  if (rc != SIM_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  const cudaError_t e2 = cudaGraphInstantiate(&h->graph_exec, g, 0);
  cudaGraphDestroy(g);
  if (e2 != cudaSuccess) {
    h->graph_exec = nullptr;
    return cuda_fail(e2, "cudaGraphInstantiate");
  }
  h->graph_dt = dt;
  h->graph_substeps = substeps;
  return SIM_OK;
}

void free_all(sim_s* h) {
  void* ptrs[] = {h->d_types, h->d_env_ids, h->d_dof_base, h->d_body_base, h->d_actor_base, h->d_actor_env,
                  h->root, h->dof, h->act, h->net_force, h->cache, h->pairs, h->n_pairs, h->sig, h->status,
                  h->pos_target, h->vel_target, h->dof_force, h->body_state, h->body_force};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (auto& tp : h->types) {
    if (tp.scratch) cudaFree(tp.scratch);
    if (tp.pscratch) cudaFree(tp.pscratch);
    if (tp.ybg) cudaFree(tp.ybg);
  }
  if (h->rv_state) cudaFree(h->rv_state);
  if (h->rv_tape) cudaFree(h->rv_tape);
  drop_graph(h);
  if (h->d_counter) cudaFree(h->d_counter);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  for (cudaStream_t s : h->type_streams) cudaStreamDestroy(s);
  for (cudaEvent_t e : h->type_events) cudaEventDestroy(e);
}

__global__ void set_root_kernel(float* root, const float* src, const int* idx, int n, int64_t N_A,
                                const int* actor_env, float* cache, int cache_stride) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int a = idx[i];
  if (a < 0 || a >= N_A) return;
  for (int k = 0; k < 13; ++k) root[(size_t)a * 13 + k] = src[(size_t)i * 13 + k];
  const int env = actor_env[a];
  for (int k = 0; k < cache_stride; ++k) cache[(size_t)env * cache_stride + k] = 0.f;
}

__global__ void set_dof_kernel(float* dof, const float* src, const int* idx, int n, int n_envs, const int* dof_base,
                               int row_stride, float* cache, int cache_stride) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int e = idx[i];
  if (e < 0 || e >= n_envs) return;
  const int b0 = dof_base[e], b1 = dof_base[e + 1];
  for (int k = 0; k < 2 * (b1 - b0); ++k) dof[(size_t)b0 * 2 + k] = src[(size_t)i * row_stride + k];
  for (int k = 0; k < cache_stride; ++k) cache[(size_t)e * cache_stride + k] = 0.f;
}

__global__ void fma_probe_kernel(float* out, int iters, float seed) {
  float a0 = seed + threadIdx.x, a1 = a0 + 1.f, a2 = a0 + 2.f, a3 = a0 + 3.f;
  float a4 = a0 + 4.f, a5 = a0 + 5.f, a6 = a0 + 6.f, a7 = a0 + 7.f;
  const float b = 0.999999f, c = 1e-7f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      a0 = fmaf(a0, b, c); a1 = fmaf(a1, b, c); a2 = fmaf(a2, b, c); a3 = fmaf(a3, b, c);
      a4 = fmaf(a4, b, c); a5 = fmaf(a5, b, c); a6 = fmaf(a6, b, c); a7 = fmaf(a7, b, c);
    }
  }
  const float s = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
  if (s == 123.456f) out[blockIdx.x] = s;  // keeps the loop alive
}

}  // namespace

// ================================================================================================
// ---- scratch of sim_step_static_scratch ---------------------------------------------------------
// Env types whose contact and row blocks do not fit in shared memory keep them in global scratch.
// sim_step uses the per-type buffers that sim_create allocated; sim_step_static_scratch uses this
// file-scope array instead, so that call allocates nothing. The array (64 MiB) exists on every
// device where the library's device code is loaded, from that load until the process exits. In
// host code its name is a stand-in for the device symbol, never an address: the address on each
// device comes from cudaGetSymbolAddress.
constexpr size_t kStaticScratchBytes = size_t(64) << 20;
static __device__ __align__(256) float g_static_scratch[kStaticScratchBytes / sizeof(float)];

namespace {

constexpr int kMaxStaticDevices = 64;
std::mutex g_static_mu;
float* g_static_addr[kMaxStaticDevices] = {};

// Device address of g_static_scratch on device `dev`, looked up with that device current (the
// caller's current device is restored afterwards). Outside a stream capture every call looks the
// address up again, so a context the caller destroyed and re-created between calls (the module
// reloaded, possibly elsewhere) is followed; during a capture the address of the last call on the
// device is reused (a lookup could load the module, which a capture does not allow).
int static_scratch_address(int dev, cudaStream_t st, float** out) {
  if (dev < 0 || dev >= kMaxStaticDevices) {
    g_last_error = "sim_step_static_scratch: device ordinal out of range";
    return SIM_ERR_CAPACITY;
  }
  std::lock_guard<std::mutex> lk(g_static_mu);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(st, &cs));
  if (cs != cudaStreamCaptureStatusNone) {
    if (!g_static_addr[dev]) {
      g_last_error = "sim_step_static_scratch: the first call on a device must come before any stream capture";
      return SIM_ERR_INVALID_ARG;
    }
    *out = g_static_addr[dev];
    return SIM_OK;
  }
  int prev = 0;
  CK(cudaGetDevice(&prev));
  CK(cudaSetDevice(dev));
  float* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress((void**)&p, g_static_scratch);
  const cudaError_t e2 = cudaSetDevice(prev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_static_scratch)");
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaSetDevice (restoring the caller's device)");
  g_static_addr[dev] = p;
  *out = p;
  return SIM_OK;
}

}  // namespace

extern "C" {

const char* sim_error_string(int code) {
  switch (code) {
    case SIM_OK: return "ok";
    case SIM_ERR_INVALID_ARG: return "invalid argument";
    case SIM_ERR_TOPOLOGY: return "invalid articulation topology";
    case SIM_ERR_CUDA: return "CUDA error";
    case SIM_ERR_CAPACITY: return "environment exceeds kernel capacity";
    case SIM_ERR_TIMEOUT: return "device wait timed out";
    case SIM_ERR_NONFINITE: return "non-finite state in some environment";
    case SIM_ERR_HANDLE: return "invalid handle";
    case SIM_ERR_NO_DEVICE: return "no CUDA device";
    default: return "unknown error";
  }
}

const char* sim_last_error_message(void) { return g_last_error.c_str(); }

int sim_create(const sim_model_desc* models, int32_t n_models, const int32_t* env_actor_model, int32_t actors_per_env,
               int32_t n_envs, const sim_params* params, void* cuda_stream, sim_handle* out) {
  if (!models || n_models < 1 || !env_actor_model || actors_per_env < 1 || actors_per_env > kMaxActors ||
      n_envs < 1 || !params || !out)
    return SIM_ERR_INVALID_ARG;
  const sim_params& p = *params;
  for (int k = 0; k < 3; ++k)
    if (!finite(p.gravity[k])) return SIM_ERR_INVALID_ARG;
  if (p.pos_iters < 1 || p.vel_iters < 0 || !finite(p.contact_offset) || !finite(p.limit_margin) ||
      !(p.bias_coef >= 0.f) || !(p.max_depen_vel >= 0.f) || !(p.ground_friction >= 0.f) ||
      !finite(p.max_depen_vel) || !finite(p.ground_friction) || !finite(p.bias_coef))
    return SIM_ERR_INVALID_ARG;
  for (int m = 0; m < n_models; ++m) {
    const int rc = validate_model(models[m]);
    if (rc != SIM_OK) return rc;
  }
  // entries of -1 pad envs with fewer actors; every env needs at least one actor
  for (int64_t e = 0; e < n_envs; ++e) {
    int cnt = 0;
    for (int a = 0; a < actors_per_env; ++a) {
      const int m = env_actor_model[e * actors_per_env + a];
      if (m < -1 || m >= n_models) return SIM_ERR_INVALID_ARG;
      cnt += m >= 0;
    }
    if (cnt == 0) return SIM_ERR_INVALID_ARG;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return SIM_ERR_NO_DEVICE;
  }

  sim_s* h = new sim_s();
  h->stream = (cudaStream_t)cuda_stream;
  h->n_envs = n_envs;
  h->actors_per_env = actors_per_env;
  h->params = p;
  cudaGetDevice(&h->device);
  // env types
  std::map<std::vector<int>, int> type_of;
  std::vector<int> env_type(n_envs);
  std::vector<int> actor_base(n_envs + 1, 0);
  for (int e = 0; e < n_envs; ++e) {
    std::vector<int> key;
    for (int a = 0; a < actors_per_env; ++a) {
      const int m = env_actor_model[(int64_t)e * actors_per_env + a];
      if (m >= 0) key.push_back(m);
    }
    actor_base[e + 1] = actor_base[e] + (int)key.size();
    auto it = type_of.find(key);
    if (it == type_of.end()) {
      TypePlan tp;
      const int rc = build_type(models, key, p, tp.tab);
      if (rc != SIM_OK) { delete h; return rc; }
      tp.G_min = tp.G = tp.tab.group;
      // relative per-env cost for the persistent tile order: factorisation plus the row solves
      tp.env_cost = (double)tp.tab.n_gen * (tp.tab.n_gen + tp.tab.row_cap) + 8.0 * tp.tab.n_links;
      it = type_of.emplace(key, (int)h->types.size()).first;
      h->types.push_back(tp);
    }
    env_type[e] = it->second;
    h->types[it->second].envs.push_back(e);
  }
  // per-env bases
  std::vector<int> dof_base(n_envs + 1, 0), body_base(n_envs + 1, 0);
  int max_cache = 1, max_pairs = 1, max_jdof = 0;
  for (int e = 0; e < n_envs; ++e) {
    const EnvTypeTable& T = h->types[env_type[e]].tab;
    dof_base[e + 1] = dof_base[e] + T.n_jdof;
    body_base[e + 1] = body_base[e] + T.n_body;
    max_cache = std::max(max_cache, T.cache_len);
    max_pairs = std::max(max_pairs, T.n_cand);
    max_jdof = std::max(max_jdof, T.n_jdof);
  }
  h->N_A = actor_base[n_envs];
  h->N_D = dof_base[n_envs];
  h->N_B = body_base[n_envs];
  h->cache_stride = max_cache;
  h->pair_stride = max_pairs;
  h->dof_row_stride = 2 * max_jdof;
  h->contiguous_single_type = h->types.size() == 1;
  std::vector<int> env_ids;
  for (auto& tp : h->types) {
    tp.env_off = (int)env_ids.size();
    env_ids.insert(env_ids.end(), tp.envs.begin(), tp.envs.end());
  }
  std::vector<EnvTypeTable> tabs;
  for (auto& tp : h->types) tabs.push_back(tp.tab);

  auto fail = [&](cudaError_t e, const char* what) {
    cuda_fail(e, what);
    free_all(h);
    delete h;
    return SIM_ERR_CUDA;
  };
#define CKC(call)                                    \
  do {                                               \
    cudaError_t e__ = (call);                        \
    if (e__ != cudaSuccess) return fail(e__, #call); \
  } while (0)
  CKC(cudaMalloc(&h->d_types, sizeof(EnvTypeTable) * tabs.size()));
  CKC(cudaMalloc(&h->d_env_ids, sizeof(int) * env_ids.size()));
  CKC(cudaMalloc(&h->d_dof_base, sizeof(int) * (n_envs + 1)));
  CKC(cudaMalloc(&h->d_body_base, sizeof(int) * (n_envs + 1)));
  CKC(cudaMalloc(&h->d_actor_base, sizeof(int) * (n_envs + 1)));
  CKC(cudaMalloc(&h->d_actor_env, sizeof(int) * h->N_A));
  CKC(cudaMalloc(&h->d_counter, 2 * sizeof(unsigned)));
  CKC(cudaMemset(h->d_counter, 0, 2 * sizeof(unsigned)));
  h->persistent = (p.flags & SIM_FLAG_PERSISTENT) != 0;
  // default plan per env type: fewest lanes, rows in shared memory when the arena is small,
  // 4 warps per CTA (fewer when the arena does not fit)
  for (auto& tp : h->types) {
    const bool rg = default_rows_global(tp.tab, tp.G_min);
    int rc = SIM_ERR_CAPACITY;
    for (int warps = 4; warps >= 1 && rc == SIM_ERR_CAPACITY; warps /= 2)
      rc = configure_type(tp, tp.G_min, rg, warps, !h->persistent);
    if (rc != SIM_OK) {
      free_all(h);
      delete h;
      return rc;
    }
  }
  if (h->persistent) {
    const int rc = plan_persistent(h);
    if (rc != SIM_OK) {
      free_all(h);
      delete h;
      return rc;
    }
  }
  CKC(cudaMalloc(&h->root, sizeof(float) * h->N_A * 13));
  CKC(cudaMalloc(&h->dof, sizeof(float) * std::max<int64_t>(h->N_D * 2, 1)));
  CKC(cudaMalloc(&h->act, sizeof(float) * std::max<int64_t>(h->N_D, 1)));
  CKC(cudaMalloc(&h->net_force, sizeof(float) * std::max<int64_t>(h->N_B * 3, 1)));
  CKC(cudaMalloc(&h->cache, sizeof(float) * (size_t)n_envs * h->cache_stride));
  CKC(cudaMalloc(&h->pairs, sizeof(int) * (size_t)n_envs * h->pair_stride * 3));
  CKC(cudaMalloc(&h->n_pairs, sizeof(int) * n_envs));
  CKC(cudaMalloc(&h->sig, sizeof(unsigned) * n_envs));
  CKC(cudaMalloc(&h->status, sizeof(int) * n_envs));
  {
    const size_t nd = (size_t)std::max<int64_t>(h->N_D, 1), nb = (size_t)std::max<int64_t>(h->N_B, 1);
    CKC(cudaMalloc(&h->pos_target, sizeof(float) * nd));
    CKC(cudaMalloc(&h->vel_target, sizeof(float) * nd));
    CKC(cudaMalloc(&h->dof_force, sizeof(float) * nd));
    CKC(cudaMalloc(&h->body_state, sizeof(float) * nb * 13));
    CKC(cudaMalloc(&h->body_force, sizeof(float) * nb * 6));
    CKC(cudaMemset(h->pos_target, 0, sizeof(float) * nd));
    CKC(cudaMemset(h->vel_target, 0, sizeof(float) * nd));
    CKC(cudaMemset(h->dof_force, 0, sizeof(float) * nd));
    CKC(cudaMemset(h->body_state, 0, sizeof(float) * nb * 13));
    CKC(cudaMemset(h->body_force, 0, sizeof(float) * nb * 6));
  }
  CKC(cudaMemcpy(h->d_types, tabs.data(), sizeof(EnvTypeTable) * tabs.size(), cudaMemcpyHostToDevice));
  CKC(cudaMemcpy(h->d_env_ids, env_ids.data(), sizeof(int) * env_ids.size(), cudaMemcpyHostToDevice));
  CKC(cudaMemcpy(h->d_dof_base, dof_base.data(), sizeof(int) * (n_envs + 1), cudaMemcpyHostToDevice));
  CKC(cudaMemcpy(h->d_body_base, body_base.data(), sizeof(int) * (n_envs + 1), cudaMemcpyHostToDevice));
  CKC(cudaMemcpy(h->d_actor_base, actor_base.data(), sizeof(int) * (n_envs + 1), cudaMemcpyHostToDevice));
  {
    std::vector<int> actor_env(h->N_A);
    for (int e = 0; e < n_envs; ++e)
      for (int a = actor_base[e]; a < actor_base[e + 1]; ++a) actor_env[a] = e;
    CKC(cudaMemcpy(h->d_actor_env, actor_env.data(), sizeof(int) * h->N_A, cudaMemcpyHostToDevice));
  }
  std::vector<float> root0((size_t)h->N_A * 13, 0.f);
  for (int64_t a = 0; a < h->N_A; ++a) root0[a * 13 + 6] = 1.f;
  CKC(cudaMemcpy(h->root, root0.data(), sizeof(float) * root0.size(), cudaMemcpyHostToDevice));
  CKC(cudaMemset(h->dof, 0, sizeof(float) * std::max<int64_t>(h->N_D * 2, 1)));
  CKC(cudaMemset(h->act, 0, sizeof(float) * std::max<int64_t>(h->N_D, 1)));
  CKC(cudaMemset(h->net_force, 0, sizeof(float) * std::max<int64_t>(h->N_B * 3, 1)));
  CKC(cudaMemset(h->cache, 0, sizeof(float) * (size_t)n_envs * h->cache_stride));
  CKC(cudaMemset(h->pairs, 0xff, sizeof(int) * (size_t)n_envs * h->pair_stride * 3));
  CKC(cudaMemset(h->n_pairs, 0, sizeof(int) * n_envs));
  CKC(cudaMemset(h->sig, 0, sizeof(unsigned) * n_envs));
  CKC(cudaMemset(h->status, 0, sizeof(int) * n_envs));
  CKC(cudaGetLastError());
#undef CKC
  {
    std::lock_guard<std::mutex> lk(g_handles_mu);
    g_handles.insert(h);
  }
  *out = h;
  return SIM_OK;
}

int sim_step(sim_handle h, float dt, int32_t substeps) {
  if (!valid_handle(h)) return SIM_ERR_HANDLE;
  if (!(dt > 0.f) || !finite(dt) || substeps < 1) return SIM_ERR_INVALID_ARG;
  if (!(h->params.flags & SIM_FLAG_GRAPH)) return launch_step(h, h->stream, dt, substeps);
  if (!h->graph_exec || h->graph_dt != dt || h->graph_substeps != substeps) {
    const int rc = capture_step(h, dt, substeps);
    if (rc != SIM_OK) return rc;
  }
  CK(cudaGraphLaunch(h->graph_exec, h->stream));
  return SIM_OK;
}

int sim_step_static_scratch(sim_handle h, const sim_state_buffers* io, float dt, int32_t substeps) {
  if (!valid_handle(h)) return SIM_ERR_HANDLE;
  if (!io || !io->root_state || !io->dof_state || !io->dof_actuation || !io->net_contact_force ||
      !io->impulse_cache || !io->contact_pairs || !io->contact_count || !io->signature || !io->status)
    return SIM_ERR_INVALID_ARG;
  if (!(dt > 0.f) || !finite(dt) || substeps < 1) return SIM_ERR_INVALID_ARG;
  // the call reads and writes only *io: steps that would read the handle's control views (drive
  // targets, body forces) or write its output views (DOF forces, rigid-body states) are refused
  if (h->params.flags & (SIM_FLAG_BODY_FORCES | SIM_FLAG_RIGID_BODY_STATE | SIM_FLAG_DOF_FORCE)) {
    g_last_error = "sim_step_static_scratch: handles created with SIM_FLAG_BODY_FORCES, SIM_FLAG_RIGID_BODY_STATE "
                   "or SIM_FLAG_DOF_FORCE are refused (those steps use the handle's views)";
    return SIM_ERR_INVALID_ARG;
  }
  for (const TypePlan& tp : h->types)
    if (tp.tab.has_drives) {
      g_last_error = "sim_step_static_scratch: env types with joint drives are refused (their targets are the "
                     "handle's views)";
      return SIM_ERR_INVALID_ARG;
    }
  // the types launch one after another on the handle's stream, so each may use the whole array
  for (const TypePlan& tp : h->types) {
    if (!tp.lay.grows) continue;
    const size_t gpb = (size_t)tp.groups_per_block;
    const size_t slot_bytes = sizeof(float) * (size_t)tp.lay.scratch_words;
    const size_t slots = (tp.envs.size() + gpb - 1) / gpb * gpb;
    if (slots * slot_bytes > kStaticScratchBytes) {
      char buf[320];
      snprintf(buf, sizeof(buf),
               "sim_step_static_scratch: an env type of %zu envs needs %zu bytes of scratch (%zu per env), more "
               "than the %zu-byte static array; at most %zu envs of this type fit",
               tp.envs.size(), slots * slot_bytes, slot_bytes, kStaticScratchBytes,
               kStaticScratchBytes / (slot_bytes * gpb) * gpb);
      g_last_error = buf;
      return SIM_ERR_CAPACITY;
    }
  }
  float* scratch = nullptr;
  const int rc = static_scratch_address(h->device, h->stream, &scratch);
  if (rc != SIM_OK) return rc;
  StepArgs a;
  fill_common(h, dt, substeps, a);
  a.root = io->root_state; a.dof = io->dof_state; a.act = io->dof_actuation; a.net_force = io->net_contact_force;
  a.cache = io->impulse_cache; a.pairs = io->contact_pairs; a.n_pairs = io->contact_count;
  a.sig = io->signature; a.status = io->status;
  a.pos_target = nullptr; a.vel_target = nullptr; a.body_force = nullptr;  // refused above: never read
  a.dof_force = nullptr; a.body_state = nullptr;                          // nor written
  for (size_t t = 0; t < h->types.size(); ++t) {
    const TypePlan& tp = h->types[t];
    TypeArgs ta;
    fill_type(h, t, ta);
    ta.scratch = tp.lay.grows ? scratch : nullptr;
    size_t smem = tp.smem_bytes;
    if (!tp.lay.grows && tp.lay.scratch_words) {
      // a shared-rows type whose Y region is sized below its row capacity: step it with the whole
      // capacity in shared memory (no global Y slots), so the array serves only global-rows types
      ta.lay = make_layout(tp.tab, tp.G, false, 0);
      smem = (size_t)tp.groups_per_block * ta.lay.total * 4;
      if (smem > kMaxSmemPerCta) {
        g_last_error = "sim_step_static_scratch: an env type's shared arena without global Y slots exceeds 220 KB "
                       "(use fewer warps per CTA for it)";
        return SIM_ERR_CAPACITY;
      }
    }
    const cudaError_t e = launch_step_kernel(tp.G, tp.lay.grows != 0, tp.tab.has_ball != 0, a, ta,
                                             tp.groups_per_block, smem, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "step_kernel launch (static scratch)");
  }
  return SIM_OK;
}

namespace {
// Device address of a pinned host buffer (CUDA-allocated or registered), or null for pageable memory.
void* device_view_of_host(const void* p) {
  if (!p) return nullptr;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();  // not an error of the step: the buffer is copied instead
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}
}  // namespace

int sim_step_actuated(sim_handle h, const float* actuation, float dt, int32_t substeps) {
  if (!valid_handle(h)) return SIM_ERR_HANDLE;
  if (!actuation && h->N_D > 0) return SIM_ERR_INVALID_ARG;
  if (!(dt > 0.f) || !finite(dt) || substeps < 1) return SIM_ERR_INVALID_ARG;
  // The step kernel of a single-type handle loads the forces from the caller's buffer wherever the
  // device can address it (its own memory, managed memory, pinned host memory) and stores them
  // into the actuation view (Ant 4096: 0.1038 -> 0.1000 ms per control step against the copy and
  // sim_step); pageable host memory, another device's memory, graph and persistent handles, and
  // handles of several env types get one copy into the view first (the concurrent per-type
  // launches of the mixed 16384-env batch measured 1.206 ms reading in place against 1.140 ms
  // after the copy, while each type's envs alone were faster in place).
  const bool direct = !(h->params.flags & (SIM_FLAG_GRAPH | SIM_FLAG_PERSISTENT)) && h->types.size() == 1;
  const float* za = nullptr;
  if (h->N_D > 0) {
    if (direct) {
      cudaPointerAttributes at{};
      if (cudaPointerGetAttributes(&at, actuation) == cudaSuccess) {
        if ((at.type == cudaMemoryTypeDevice && at.device == h->device) || at.type == cudaMemoryTypeManaged)
          za = actuation;
        else if (at.type == cudaMemoryTypeHost)
          za = static_cast<const float*>(at.devicePointer);
      } else {
        cudaGetLastError();  // not an error of the step: the buffer is copied instead
      }
    }
    if (!za) CK(cudaMemcpyAsync(h->act, actuation, sizeof(float) * h->N_D, cudaMemcpyDefault, h->stream));
  }
  h->zc_act = za;
  const int rc = sim_step(h, dt, substeps);
  h->zc_act = nullptr;
  return rc;
}

int sim_step_host(sim_handle h, const float* host_actuation, float* host_root_out, float* host_dof_out, float dt,
                  int32_t substeps) {
  if (!valid_handle(h)) return SIM_ERR_HANDLE;
  if (!host_actuation && h->N_D > 0) return SIM_ERR_INVALID_ARG;
  if (!(dt > 0.f) || !finite(dt) || substeps < 1) return SIM_ERR_INVALID_ARG;
  // Pinned buffers are read and written by the step kernels themselves (the actuation loads, the
  // final state stores), with no copy launch; pageable buffers, graph handles (whose captured
  // launches have fixed arguments) and persistent handles (whose kernel is compiled without these
  // accesses) are copied.
  const bool direct = !(h->params.flags & (SIM_FLAG_GRAPH | SIM_FLAG_PERSISTENT));
  const float* za = (direct && h->N_D > 0) ? static_cast<const float*>(device_view_of_host(host_actuation)) : nullptr;
  float* zr = direct ? static_cast<float*>(device_view_of_host(host_root_out)) : nullptr;
  float* zd = (direct && h->N_D > 0) ? static_cast<float*>(device_view_of_host(host_dof_out)) : nullptr;
  if (h->N_D > 0 && !za)
    CK(cudaMemcpyAsync(h->act, host_actuation, sizeof(float) * h->N_D, cudaMemcpyHostToDevice, h->stream));
  h->zc_act = za; h->zc_root = zr; h->zc_dof = zd;
  const int rc = sim_step(h, dt, substeps);
  h->zc_act = nullptr; h->zc_root = nullptr; h->zc_dof = nullptr;
  if (rc != SIM_OK) return rc;
  if (host_root_out && !zr)
    CK(cudaMemcpyAsync(host_root_out, h->root, sizeof(float) * h->N_A * 13, cudaMemcpyDeviceToHost, h->stream));
  if (host_dof_out && h->N_D > 0 && !zd)
    CK(cudaMemcpyAsync(host_dof_out, h->dof, sizeof(float) * h->N_D * 2, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return SIM_OK;
}

// ---- reverse pass ---------------------------------------------------------------------------------
namespace {

int al4i(int x) { return (x + 3) & ~3; }

// Tape of one env-substep of type tp (offsets in words; see TapeLayout).
TapeLayout tape_layout(const TypePlan& tp, int npos, int nvel) {
  const EnvTypeTable& T = tp.tab;
  TapeLayout t{};
  t.n = std::max(T.n_gen, 1);
  t.rcap = tp.lay.rcap;
  t.ccap = tp.lay.ccap;
  t.npos = npos;
  t.iters = npos + nvel;
  const int n = t.n;
  int o = 0;
  t.hdr = o; o += 4;
  t.st = o; o += 2 * T.n_jdof + 13 * T.n_actors;
  o = al4i(o);
  t.LT = n | 1;
  t.YT = t.rcap | 1;
  t.vec = o; o += 7 * n;
  t.L = o; o += n * t.LT;
  t.Linv = o; o += n;
  t.cw = T.n_pairs > 0 ? kTapeConPairWords : 5;
  t.con = o; o += t.cw * t.ccap;
  o = al4i(o);
  t.rowc = o; o += 4 * t.rcap;
  t.rowa = o; o += t.rcap;
  t.lam0 = o; o += t.rcap;
  t.lamf = o; o += t.rcap;
  o = al4i(o);  // a reverse arena without room for the row history copies the block up to here
  t.lamb = o; o += t.iters * t.rcap;
  t.seps = o; o += (npos + 1) * t.rcap;
  // the adjoint reuses these two blocks, once read, as 7 words per row (14 with shape pairs: the
  // rows act on two bodies), then as 18 words per pair contact: keep at least that many
  o = std::max(o, t.lamb + (T.n_pairs > 0 ? 14 : 7) * t.rcap);
  o = al4i(o);
  t.Y = o; o += n * t.YT;
  t.words = al4i(o);
  return t;
}

constexpr int kAdjThreads = 64;  // threads per CTA of the adjoint kernel

// Arena of one env in the adjoint kernel (offsets in words; see AdjLayout).
AdjLayout adj_layout(const TypePlan& tp, int npos, int nvel) {
  const EnvTypeTable& T = tp.tab;
  const TapeLayout tl = tape_layout(tp, npos, nvel);
  AdjLayout a{};
  const int n = std::max(T.n_gen, 1), rc = tp.lay.rcap;
  a.YS = tl.YT;
  a.LS = tl.LT;
  const bool pairs = T.n_pairs > 0;
  for (int gY = 0; gY < 2; ++gY) {
    int o = 0;
    a.gY = gY;
    a.imgw = gY ? tl.lamb : tl.words;
    a.frw = std::max(14 * rc, 18 * tl.ccap);
    a.rw = gY ? a.frw + 9 * rc : 0;
    a.img = o; o += a.imgw;
    a.bar = o; o += 4;
    a.Yb = o; o += gY ? 0 : n * a.YS;
    a.Mb = o; o += n * a.LS;
    a.lamb = o; o += rc;
    a.db = o; o += rc;
    a.invAb = o; o += rc;
    a.xbw = pairs ? 9 : 3;
    a.xb = o; o += gY ? 0 : a.xbw * rc;
    a.vec = o; o += kAdjVecs * n;
    a.SD = o; o += 7 * n;   // 6-vectors at an odd stride of 7
    a.FM = o; o += 7 * n;
    a.FMb = o; o += 7 * n;
    a.Sb = o; o += 7 * n;
    a.link = o; o += kAdjLinkWords * T.n_links;
    a.pose = o; o += pairs ? 12 * T.n_links : 0;
    a.total = al4i(o);
    // Y and its adjoint in shared memory while the CTA's envs (64 threads / G) fit (the option of
    // reading them from global memory is compiled into the kernels for env types with shape pairs)
    if (!pairs || (size_t)(kAdjThreads / tp.G) * a.total * sizeof(float) <= kMaxSmemPerCta) break;
  }
  return a;
}

// The reverse pass covers every env type whose adjoint arena fits a CTA.
int reverse_supported(const sim_s* h) {
  for (const TypePlan& tp : h->types) {
    const AdjLayout al = adj_layout(tp, h->params.pos_iters, h->params.vel_iters);
    if ((size_t)(kAdjThreads / tp.G) * al.total * sizeof(float) > kMaxSmemPerCta) {
      g_last_error = "reverse pass: the env type's adjoint arena exceeds a CTA's shared memory";
      return SIM_ERR_CAPACITY;
    }
  }
  return SIM_OK;
}

// Floats of one step's tape over all env types, and each type's offset.
int64_t tape_floats(const sim_s* h, int substeps, std::vector<int64_t>* offs) {
  int64_t total = 0;
  for (const TypePlan& tp : h->types) {
    if (offs) offs->push_back(total);
    total += (int64_t)tp.envs.size() * substeps * tape_layout(tp, h->params.pos_iters, h->params.vel_iters).words;
  }
  return total;
}

// One taped step: the per-type step kernels, given the tape pointer, advance the state buffers of
// `a` exactly as sim_step's per-type launches do (the same kernels and arithmetic; the tape stores
// are their only difference) and write each env-substep's tape to `tape`.
int launch_taped(sim_s* h, StepArgs a, float* tape, cudaStream_t st) {
  std::vector<int64_t> offs;
  tape_floats(h, a.substeps, &offs);
  for (size_t t = 0; t < h->types.size(); ++t) {
    TypePlan& tp = h->types[t];
    if (tp.lay.scratch_words) {  // a persistent handle steps without per-type scratch (no-op when it fits)
      const size_t gpb = (size_t)tp.groups_per_block;
      const int rc = grow_buffer(&tp.scratch, &tp.scratch_floats,
                                 (tp.envs.size() + gpb - 1) / gpb * gpb * (size_t)tp.lay.scratch_words,
                                 "cudaMalloc (global rows scratch)");
      if (rc != SIM_OK) return rc;
    }
    TypeArgs ta;
    fill_type(h, t, ta);
    ta.tape = tape + offs[t];
    ta.tl = tape_layout(tp, a.pos_iters, a.vel_iters);
    const cudaError_t e = launch_type(tp, a, ta, st);  // the per-type step kernel, recording the tape
    if (e != cudaSuccess) return cuda_fail(e, "step_kernel launch (taped)");
  }
  return SIM_OK;
}

// The adjoint of a taped step: one launch per env type.
int launch_adjoint(sim_s* h, const StepArgs& a, const float* tape, AdjArgs j, cudaStream_t st) {
  std::vector<int64_t> offs;
  tape_floats(h, a.substeps, &offs);
  for (size_t t = 0; t < h->types.size(); ++t) {
    TypePlan& tp = h->types[t];
    TypeArgs ta;
    fill_type(h, t, ta);
    ta.tl = tape_layout(tp, a.pos_iters, a.vel_iters);
    j.tape = tape + offs[t];
    j.al = adj_layout(tp, a.pos_iters, a.vel_iters);
    j.ybg = nullptr;
    j.rwg = nullptr;
    if (j.al.gY) {  // one slot per group of the launch (the dead groups of the last CTA own theirs)
      const size_t gpb = kAdjThreads / tp.G, groups = (tp.envs.size() + gpb - 1) / gpb * gpb;
      const size_t yb = groups * (size_t)std::max(tp.tab.n_gen, 1) * j.al.YS;
      const int rc = grow_buffer(&tp.ybg, &tp.ybg_floats, yb + groups * (size_t)j.al.rw,
                                 "cudaMalloc (reverse-pass Y adjoint and row work)");
      if (rc != SIM_OK) return rc;
      j.ybg = tp.ybg;
      j.rwg = tp.ybg + yb;
    }
    CK(set_adjoint_kernel_smem_cap(tp.G, kMaxSmemPerCta));
    const cudaError_t e = launch_adjoint_kernel(tp.G, tp.tab.has_ball != 0, a, ta, j, st);
    if (e != cudaSuccess) return cuda_fail(e, "adjoint_kernel launch");
  }
  return SIM_OK;
}

}  // namespace

int sim_tape_size(sim_handle h, int32_t substeps, int64_t* floats) {
  if (!valid_handle(h)) return SIM_ERR_HANDLE;
  if (!floats || substeps < 1) return SIM_ERR_INVALID_ARG;
  const int rc = reverse_supported(h);
  if (rc != SIM_OK) return rc;
  *floats = tape_floats(h, substeps, nullptr);
  return SIM_OK;
}

int sim_step_taped(sim_handle h, float* tape, float dt, int32_t substeps) {
  if (!valid_handle(h)) return SIM_ERR_HANDLE;
  if (!tape || !(dt > 0.f) || !finite(dt) || substeps < 1) return SIM_ERR_INVALID_ARG;
  const int rc = reverse_supported(h);
  if (rc != SIM_OK) return rc;
  StepArgs a;
  fill_common(h, dt, substeps, a);
  return launch_taped(h, a, tape, h->stream);
}

int sim_step_adjoint(sim_handle h, const float* tape, const sim_adjoint_buffers* b, float dt, int32_t substeps) {
  if (!valid_handle(h)) return SIM_ERR_HANDLE;
  const bool jd = h->N_D > 0;  // the DOF buffers are required only when there are joint DOFs
  if (!tape || !b || !b->grad_root_state_in || (jd && (!b->grad_dof_state_in || !b->grad_dof_actuation)) ||
      !b->grad_impulse_cache_in)
    return SIM_ERR_INVALID_ARG;
  if (!(dt > 0.f) || !finite(dt) || substeps < 1) return SIM_ERR_INVALID_ARG;
  const int rc = reverse_supported(h);
  if (rc != SIM_OK) return rc;
  StepArgs a;
  fill_common(h, dt, substeps, a);
  AdjArgs j{};
  j.g_root = b->grad_root_state; j.g_dof = b->grad_dof_state; j.g_cache = b->grad_impulse_cache;
  j.gi_root = b->grad_root_state_in; j.gi_dof = b->grad_dof_state_in; j.gi_act = b->grad_dof_actuation;
  j.gi_cache = b->grad_impulse_cache_in;
  j.status = b->status;
  return launch_adjoint(h, a, tape, j, h->stream);
}

int sim_step_vjp(sim_handle h, const sim_vjp_buffers* b, float dt, int32_t substeps) {
  if (!valid_handle(h)) return SIM_ERR_HANDLE;
  const bool jd = h->N_D > 0;  // the DOF buffers are required only when there are joint DOFs
  if (!b || !b->root_state || (jd && (!b->dof_state || !b->dof_actuation || !b->grad_dof_state_in ||
                                      !b->grad_dof_actuation)) ||
      !b->impulse_cache || !b->grad_root_state_in || !b->grad_impulse_cache_in)
    return SIM_ERR_INVALID_ARG;
  if (!(dt > 0.f) || !finite(dt) || substeps < 1) return SIM_ERR_INVALID_ARG;
  if (!(h->params.flags & SIM_FLAG_TANGENT_VJP) && reverse_supported(h) == SIM_OK) {
    // the reverse pass: the taped step on a copy of the input state, then its adjoint
    g_last_error.clear();
    const size_t nr = 13 * (size_t)h->N_A, nd = 2 * (size_t)h->N_D, nc = (size_t)h->n_envs * h->cache_stride;
    const size_t nn = 3 * (size_t)h->N_B, np = (size_t)h->n_envs * h->pair_stride * 3, ne = (size_t)h->n_envs;
    int rc = grow_buffer(&h->rv_state, &h->rv_state_floats, nr + nd + nc + nn + np + 3 * ne + 4,
                         "cudaMalloc (reverse-pass state)");
    if (rc != SIM_OK) return rc;
    const int64_t tf = tape_floats(h, substeps, nullptr);
    rc = grow_buffer(&h->rv_tape, &h->rv_tape_floats, (size_t)std::max<int64_t>(tf, 4), "cudaMalloc (reverse-pass tape)");
    if (rc != SIM_OK) return rc;
    float* st_root = h->rv_state;
    float* st_dof = st_root + nr;
    float* st_cache = st_dof + nd;
    float* st_net = st_cache + nc;
    int* st_pairs = reinterpret_cast<int*>(st_net + nn);
    int* st_np = st_pairs + np;
    unsigned* st_sig = reinterpret_cast<unsigned*>(st_np + ne);
    int* st_status = reinterpret_cast<int*>(st_sig + ne);
    CK(cudaMemcpyAsync(st_root, b->root_state, sizeof(float) * nr, cudaMemcpyDeviceToDevice, h->stream));
    if (nd) CK(cudaMemcpyAsync(st_dof, b->dof_state, sizeof(float) * nd, cudaMemcpyDeviceToDevice, h->stream));
    CK(cudaMemcpyAsync(st_cache, b->impulse_cache, sizeof(float) * nc, cudaMemcpyDeviceToDevice, h->stream));
    StepArgs a;
    fill_common(h, dt, substeps, a);
    a.root = st_root; a.dof = st_dof; a.act = b->dof_actuation; a.cache = st_cache; a.net_force = st_net;
    a.pairs = st_pairs; a.n_pairs = st_np; a.sig = st_sig; a.status = st_status;
    a.flags &= ~(SIM_FLAG_RIGID_BODY_STATE | SIM_FLAG_DOF_FORCE);  // no writes to the handle's views
    a.dof_force = nullptr; a.body_state = nullptr;
    rc = launch_taped(h, a, h->rv_tape, h->stream);
    if (rc != SIM_OK) return rc;
    AdjArgs j{};
    j.g_root = b->grad_root_state; j.g_dof = b->grad_dof_state; j.g_cache = b->grad_impulse_cache;
    j.gi_root = b->grad_root_state_in; j.gi_dof = b->grad_dof_state_in; j.gi_act = b->grad_dof_actuation;
    j.gi_cache = b->grad_impulse_cache_in;
    j.status = b->status;
    return launch_adjoint(h, a, h->rv_tape, j, h->stream);
  }
  int rc = tangent_supported(h);
  if (rc != SIM_OK) return rc;
  StepArgs a;
  fill_common(h, dt, substeps, a);
  TangentArgs v{};
  v.root = b->root_state; v.dof = b->dof_state; v.act = b->dof_actuation; v.cache = b->impulse_cache;
  v.g_root = b->grad_root_state; v.g_dof = b->grad_dof_state; v.g_cache = b->grad_impulse_cache;
  v.gi_root = b->grad_root_state_in; v.gi_dof = b->grad_dof_state_in; v.gi_act = b->grad_dof_actuation;
  v.gi_cache = b->grad_impulse_cache_in;
  v.status = b->status;
  v.mode = 0;
  for (size_t t = 0; t < h->types.size(); ++t) {
    const EnvTypeTable& T = h->types[t].tab;
    TypeArgs ta;
    fill_type(h, t, ta);
    // directions: state and actuation, plus the impulse-cache slots the env's first substep reads
    // (known only in the kernel; budgeted here at 24, more run as further passes in the kernel)
    const int K = tangent_lanes_per_dir(13 * T.n_actors + 3 * T.n_jdof + 24);
    v.dir_base = 0;
    const cudaError_t e = launch_tangent_kernel(K, a, ta, v, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "tangent_step_kernel launch (adjoint)");
  }
  return SIM_OK;
}

int sim_step_jvp(sim_handle h, const sim_jvp_buffers* b, float dt, int32_t substeps) {
  if (!valid_handle(h)) return SIM_ERR_HANDLE;
  const bool jd = h->N_D > 0;  // the DOF buffers are required only when there are joint DOFs
  if (!b || !b->root_state || !b->impulse_cache || !b->tan_root_state || !b->tan_impulse_cache ||
      !b->root_state_out || !b->impulse_cache_out || !b->tan_root_state_out || !b->tan_impulse_cache_out ||
      (jd && (!b->dof_state || !b->dof_actuation || !b->tan_dof_state || !b->tan_dof_actuation ||
              !b->dof_state_out || !b->tan_dof_state_out)))
    return SIM_ERR_INVALID_ARG;
  if (!(dt > 0.f) || !finite(dt) || substeps < 1) return SIM_ERR_INVALID_ARG;
  int rc = tangent_supported(h);
  if (rc != SIM_OK) return rc;
  StepArgs a;
  fill_common(h, dt, substeps, a);
  TangentArgs v{};
  v.root = b->root_state; v.dof = b->dof_state; v.act = b->dof_actuation; v.cache = b->impulse_cache;
  v.t_root = b->tan_root_state; v.t_dof = b->tan_dof_state; v.t_act = b->tan_dof_actuation;
  v.t_cache = b->tan_impulse_cache;
  v.o_root = b->root_state_out; v.o_dof = b->dof_state_out; v.o_cache = b->impulse_cache_out;
  v.to_root = b->tan_root_state_out; v.to_dof = b->tan_dof_state_out; v.to_cache = b->tan_impulse_cache_out;
  v.status = b->status;
  v.mode = 1;
  for (size_t t = 0; t < h->types.size(); ++t) {
    TypeArgs ta;
    fill_type(h, t, ta);
    const cudaError_t e = launch_tangent_kernel(1, a, ta, v, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "tangent_step_kernel launch (tangent)");
  }
  return SIM_OK;
}

int sim_get_max_dims(sim_handle h, int32_t* n_max, int32_t* l_max) {
  if (!valid_handle(h)) return SIM_ERR_HANDLE;
  if (!n_max || !l_max) return SIM_ERR_INVALID_ARG;
  int nm = 1, lm = 1;
  for (const TypePlan& tp : h->types) { nm = std::max(nm, tp.tab.n_gen); lm = std::max(lm, tp.tab.n_links); }
  *n_max = nm;
  *l_max = lm;
  return SIM_OK;
}

static int run_query(sim_handle h, float* out, int what) {
  if (!valid_handle(h)) return SIM_ERR_HANDLE;
  if (!out) return SIM_ERR_INVALID_ARG;
  int nm = 1, lm = 1;
  sim_get_max_dims(h, &nm, &lm);
  StepArgs a;
  fill_common(h, 1.f, 1, a);
  for (size_t t = 0; t < h->types.size(); ++t) {
    TypeArgs ta;
    fill_type(h, t, ta);
    const cudaError_t e = launch_query_kernel(what, a, ta, out, nm, lm, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "dynamics query kernel launch");
  }
  return SIM_OK;
}

int sim_compute_mass_matrix(sim_handle h, float* out) { return run_query(h, out, 0); }
int sim_compute_jacobian(sim_handle h, float* out) { return run_query(h, out, 1); }

int sim_get_type_config(sim_handle h, int32_t type, int32_t* out) {
  if (!valid_handle(h)) return SIM_ERR_HANDLE;
  if (!out || type < 0 || type >= (int)h->types.size()) return SIM_ERR_INVALID_ARG;
  const TypePlan& tp = h->types[type];
  out[0] = tp.G; out[1] = tp.lay.grows; out[2] = tp.warps_per_cta; out[3] = (int32_t)tp.envs.size();
  out[4] = tp.G_min; out[5] = tp.envs.empty() ? -1 : tp.envs[0];
  return SIM_OK;
}

int sim_set_type_config(sim_handle h, int32_t type, int32_t lanes_per_env, int32_t rows_global,
                        int32_t warps_per_cta) {
  if (!valid_handle(h)) return SIM_ERR_HANDLE;
  if (type < 0 || type >= (int)h->types.size() || (rows_global != 0 && rows_global != 1)) return SIM_ERR_INVALID_ARG;
  TypePlan& tp = h->types[type];
  const int G0 = tp.G, w0 = tp.warps_per_cta;
  const bool r0 = tp.lay.grows != 0;
  int rc = configure_type(tp, lanes_per_env, rows_global != 0, warps_per_cta, !h->persistent);
  if (rc != SIM_OK) return rc;
  drop_graph(h);
  if (h->persistent) {
    rc = plan_persistent(h);
    if (rc != SIM_OK) {  // restore the previous, working plan
      const std::string msg = g_last_error;
      configure_type(tp, G0, r0, w0, false);
      plan_persistent(h);
      g_last_error = msg;
      return rc;
    }
  }
  return SIM_OK;
}

// A candidate replaces the knobs the autotuner holds only when its median step is this much
// faster, so that timing noise on the tuning state (a snapshot, possibly early in the trajectory)
// does not pick the plan: on the mixed 16384-env batch a persistent plan chosen on a snapshot of
// step 10 (the Humanoid's rows moved to global scratch) ran 11 % slower than the default knobs
// over steps 20 to 119.
constexpr double kAutotuneMargin = 0.03;

int sim_autotune(sim_handle h, float dt, int32_t substeps, int32_t reps, double* ms_per_step) {
  if (!valid_handle(h)) return SIM_ERR_HANDLE;
  if (!(dt > 0.f) || !finite(dt) || substeps < 1 || reps < 1 || reps > 1000 || !ms_per_step)
    return SIM_ERR_INVALID_ARG;
  cudaStream_t st = h->stream;
  struct Snap { void* live; void* save; size_t bytes; };
  std::vector<Snap> snaps = {
      {h->root, nullptr, sizeof(float) * (size_t)h->N_A * 13},
      {h->dof, nullptr, sizeof(float) * (size_t)std::max<int64_t>(h->N_D * 2, 1)},
      {h->net_force, nullptr, sizeof(float) * (size_t)std::max<int64_t>(h->N_B * 3, 1)},
      {h->cache, nullptr, sizeof(float) * (size_t)h->n_envs * h->cache_stride},
      {h->pairs, nullptr, sizeof(int) * (size_t)h->n_envs * h->pair_stride * 3},
      {h->n_pairs, nullptr, sizeof(int) * (size_t)h->n_envs},
      {h->sig, nullptr, sizeof(unsigned) * (size_t)h->n_envs},
      {h->status, nullptr, sizeof(int) * (size_t)h->n_envs}};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = SIM_OK;
  auto cleanup = [&]() {
    for (Snap& sn : snaps)
      if (sn.save) cudaFree(sn.save);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
#define CKT(call)                                   \
  do {                                              \
    cudaError_t e__ = (call);                       \
    if (e__ != cudaSuccess) {                       \
      cleanup();                                    \
      return cuda_fail(e__, #call);                 \
    }                                               \
  } while (0)
  for (Snap& sn : snaps) {
    CKT(cudaMalloc(&sn.save, sn.bytes));
    CKT(cudaMemcpyAsync(sn.save, sn.live, sn.bytes, cudaMemcpyDeviceToDevice, st));
  }
  CKT(cudaEventCreate(&e0));
  CKT(cudaEventCreate(&e1));
  auto restore = [&]() {
    for (Snap& sn : snaps) cudaMemcpyAsync(sn.live, sn.save, sn.bytes, cudaMemcpyDeviceToDevice, st);
  };
  // median time of `enqueue` over reps runs, each from the snapshot, after one warm-up run
  auto time_it = [&](auto&& enqueue, double* ms) -> int {
    std::vector<float> ts;
    for (int r = -1; r < reps; ++r) {
      restore();
      cudaEventRecord(e0, st);
      const int erc = enqueue();
      if (erc != SIM_OK) return erc;
      cudaEventRecord(e1, st);
      const cudaError_t e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) return cuda_fail(e, "autotune step");
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      if (r >= 0) ts.push_back(t);
    }
    std::sort(ts.begin(), ts.end());
    *ms = ts[ts.size() / 2];
    return SIM_OK;
  };
  auto step = [&]() { return launch_step(h, st, dt, substeps); };
  drop_graph(h);
  double best_step = 0.0;
  if (!h->persistent) {
    for (size_t t = 0; t < h->types.size() && rc == SIM_OK; ++t) {
      TypePlan& tp = h->types[t];
      int bG = tp.G, bw = tp.warps_per_cta;
      bool br = tp.lay.grows != 0;
      auto one = [&]() {
        StepArgs a;
        TypeArgs ta;
        fill_common(h, dt, substeps, a);
        fill_type(h, t, ta);
        const cudaError_t e = launch_type(tp, a, ta, st);
        return e == cudaSuccess ? SIM_OK : cuda_fail(e, "step_kernel launch (autotune)");
      };
      double best = 1e30;  // the current knobs first: a candidate must beat them by the margin
      rc = time_it(one, &best);
      for (int G = tp.G_min; G <= 32 && rc == SIM_OK; G *= 2)
        for (int rg = 0; rg < 2 && rc == SIM_OK; ++rg)
          for (int w = 2; w <= 4 && rc == SIM_OK; w += 2) {
            if (G == bG && (rg != 0) == br && w == bw) continue;
            const int crc = configure_type(tp, G, rg != 0, w, true);
            if (crc == SIM_ERR_CUDA) rc = crc;
            if (crc != SIM_OK) continue;
            double ms = 0.0;
            rc = time_it(one, &ms);
            if (rc == SIM_OK && ms < best * (1.0 - kAutotuneMargin)) { best = ms; bG = G; br = rg != 0; bw = w; }
          }
      if (rc == SIM_OK) rc = configure_type(tp, bG, br, bw, true);
    }
    if (rc == SIM_OK) rc = time_it(step, &best_step);
  } else {
    rc = time_it(step, &best_step);
    for (int pass = 0; pass < 2 && rc == SIM_OK; ++pass)
      for (size_t t = 0; t < h->types.size() && rc == SIM_OK; ++t) {
        TypePlan& tp = h->types[t];
        for (int G = tp.G_min; G <= 32 && rc == SIM_OK; G *= 2)
          for (int rg = 0; rg < 2 && rc == SIM_OK; ++rg) {
            const int G0 = tp.G;
            const bool r0 = tp.lay.grows != 0;
            if (G == G0 && (rg != 0) == r0) continue;
            int crc = configure_type(tp, G, rg != 0, 4, false);
            if (crc == SIM_OK) crc = plan_persistent(h);
            if (crc == SIM_ERR_CUDA) rc = crc;
            double ms = 1e30;
            if (crc == SIM_OK) rc = time_it(step, &ms);
            if (rc == SIM_OK && ms < best_step * (1.0 - kAutotuneMargin)) {
              best_step = ms;
            } else if (rc == SIM_OK) {
              configure_type(tp, G0, r0, 4, false);
              rc = plan_persistent(h);
            }
          }
      }
  }
#undef CKT
  restore();
  const cudaError_t e = cudaStreamSynchronize(st);
  cleanup();
  if (rc != SIM_OK) return rc;
  if (e != cudaSuccess) return cuda_fail(e, "autotune restore");
  *ms_per_step = best_step;
  return SIM_OK;
}

int sim_get_view(sim_handle h, int32_t which, sim_view* out) {
  if (!valid_handle(h)) return SIM_ERR_HANDLE;
  if (!out) return SIM_ERR_INVALID_ARG;
  sim_view v{};
  v.device = h->device;
  auto set = [&](void* d, int nd, int64_t s0, int64_t s1, int64_t s2, int dt) {
    v.data = d; v.ndim = nd; v.shape[0] = s0; v.shape[1] = s1; v.shape[2] = s2; v.dtype = dt;
    if (nd == 1) { v.strides[0] = 1; }
    if (nd == 2) { v.strides[0] = s1; v.strides[1] = 1; }
    if (nd == 3) { v.strides[0] = s1 * s2; v.strides[1] = s2; v.strides[2] = 1; }
  };
  switch (which) {
    case SIM_VIEW_ROOT_STATE: set(h->root, 2, h->N_A, 13, 0, SIM_DTYPE_F32); break;
    case SIM_VIEW_DOF_STATE: set(h->dof, 2, h->N_D, 2, 0, SIM_DTYPE_F32); break;
    case SIM_VIEW_DOF_ACTUATION: set(h->act, 1, h->N_D, 0, 0, SIM_DTYPE_F32); break;
    case SIM_VIEW_NET_CONTACT_FORCE: set(h->net_force, 2, h->N_B, 3, 0, SIM_DTYPE_F32); break;
    case SIM_VIEW_CONTACT_PAIRS: set(h->pairs, 3, h->n_envs, h->pair_stride, 3, SIM_DTYPE_I32); break;
    case SIM_VIEW_CONTACT_COUNT: set(h->n_pairs, 1, h->n_envs, 0, 0, SIM_DTYPE_I32); break;
    case SIM_VIEW_SIGNATURE: set(h->sig, 1, h->n_envs, 0, 0, SIM_DTYPE_U32); break;
    case SIM_VIEW_STATUS: set(h->status, 1, h->n_envs, 0, 0, SIM_DTYPE_I32); break;
    case SIM_VIEW_IMPULSE_CACHE: set(h->cache, 2, h->n_envs, h->cache_stride, 0, SIM_DTYPE_F32); break;
    case SIM_VIEW_DOF_POSITION_TARGET: set(h->pos_target, 1, h->N_D, 0, 0, SIM_DTYPE_F32); break;
    case SIM_VIEW_DOF_VELOCITY_TARGET: set(h->vel_target, 1, h->N_D, 0, 0, SIM_DTYPE_F32); break;
    case SIM_VIEW_DOF_FORCE: set(h->dof_force, 1, h->N_D, 0, 0, SIM_DTYPE_F32); break;
    case SIM_VIEW_RIGID_BODY_STATE: set(h->body_state, 2, h->N_B, 13, 0, SIM_DTYPE_F32); break;
    case SIM_VIEW_RIGID_BODY_FORCE: set(h->body_force, 2, h->N_B, 6, 0, SIM_DTYPE_F32); break;
    default: return SIM_ERR_INVALID_ARG;
  }
  *out = v;
  return SIM_OK;
}

int sim_set_root_state_indexed(sim_handle h, const float* dev_src, const int32_t* dev_actor_idx, int32_t n) {
  if (!valid_handle(h)) return SIM_ERR_HANDLE;
  if (n < 0 || (n > 0 && (!dev_src || !dev_actor_idx))) return SIM_ERR_INVALID_ARG;
  if (n == 0) return SIM_OK;
  set_root_kernel<<<(n + 127) / 128, 128, 0, h->stream>>>(h->root, dev_src, dev_actor_idx, n, h->N_A,
                                                          h->d_actor_env, h->cache, h->cache_stride);
  CK(cudaGetLastError());
  return SIM_OK;
}

int sim_set_dof_state_indexed(sim_handle h, const float* dev_src, const int32_t* dev_env_idx, int32_t n) {
  if (!valid_handle(h)) return SIM_ERR_HANDLE;
  if (n < 0 || (n > 0 && (!dev_src || !dev_env_idx))) return SIM_ERR_INVALID_ARG;
  if (n == 0) return SIM_OK;
  set_dof_kernel<<<(n + 127) / 128, 128, 0, h->stream>>>(h->dof, dev_src, dev_env_idx, n, h->n_envs, h->d_dof_base,
                                                         std::max(h->dof_row_stride, 1), h->cache, h->cache_stride);
  CK(cudaGetLastError());
  return SIM_OK;
}

int sim_set_stream(sim_handle h, void* cuda_stream) {
  if (!valid_handle(h)) return SIM_ERR_HANDLE;
  h->stream = (cudaStream_t)cuda_stream;
  return SIM_OK;
}

int sim_sync_status(sim_handle h, int32_t* n_bad_envs) {
  if (!valid_handle(h)) return SIM_ERR_HANDLE;
  std::vector<int> st(h->n_envs);
  CK(cudaMemcpyAsync(st.data(), h->status, sizeof(int) * h->n_envs, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  int bad = 0;
  for (int s : st) bad += (s != 0);
  if (n_bad_envs) *n_bad_envs = bad;
  return bad ? SIM_ERR_NONFINITE : SIM_OK;
}

int sim_get_sizes(sim_handle h, int64_t* out) {
  if (!valid_handle(h)) return SIM_ERR_HANDLE;
  if (!out) return SIM_ERR_INVALID_ARG;
  out[0] = h->N_A; out[1] = h->N_D; out[2] = h->N_B; out[3] = h->pair_stride; out[4] = h->cache_stride;
  out[5] = (int64_t)h->types.size(); out[6] = h->persistent ? 1 : (int64_t)h->types.size();
  return SIM_OK;
}

int sim_destroy(sim_handle h) {
  {
    std::lock_guard<std::mutex> lk(g_handles_mu);
    if (!h || !g_handles.count(h)) return SIM_ERR_HANDLE;
    g_handles.erase(h);
  }
  cudaStreamSynchronize(h->stream);
  free_all(h);
  h->magic = 0;
  delete h;
  return SIM_OK;
}

int sim_probe_fp32_peak(void* cuda_stream, int32_t iters, double* flops_per_s) {
  if (iters < 1 || !flops_per_s) return SIM_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  float* out = nullptr;
  const int blocks = sms * 8, threads = 256;
  CK(cudaMalloc(&out, sizeof(float) * blocks));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  fma_probe_kernel<<<blocks, threads, 0, st>>>(out, std::max(1, iters / 10), 1.f);  // warm-up
  CK(cudaEventRecord(e0, st));
  fma_probe_kernel<<<blocks, threads, 0, st>>>(out, iters, 1.f);
  CK(cudaEventRecord(e1, st));
  CK(cudaEventSynchronize(e1));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  *flops_per_s = 2.0 * 8.0 * 16.0 * (double)iters * blocks * threads / (ms * 1e-3);
  return SIM_OK;
}

}  // extern "C"
