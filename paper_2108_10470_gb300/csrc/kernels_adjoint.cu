// The env-step's derivative on the GPU: tangent_step_kernel<K> evaluates one env per warp in dual
// arithmetic (tangent_step.cuh). In the adjoint mode each lane seeds K input directions of the env
// (root state, DOF state, actuation, impulse cache, in that order) and contracts its output
// tangents with the caller's output gradient, so the warp writes 32 K entries of the input
// gradient J^T g; in the tangent mode every lane propagates the caller's input tangent and lane 0
// writes the output value and tangent.
#include "launch.h"
#include "tangent_step.cuh"

namespace artsim {

namespace {

// Input component of direction `dir` of an env with na actors and nj joint DOFs: root state (13
// per actor), DOF state (2 per joint DOF), actuation, then the read impulse-cache slots.
template <int K>
__device__ __forceinline__ Dn<K>* input_slot(TanState<K>& s, int dir, int na, int nj, const int* slots, int nread,
                                             int* where) {
  if (dir < 13 * na) {
    const int a = dir / 13, c = dir % 13;
    *where = 0;
    if (c < 3) return &s.rp[a][c];
    if (c < 7) return &s.rq[a][c - 3];
    if (c < 10) return &s.rv[a][c - 7];
    return &s.rw[a][c - 10];
  }
  dir -= 13 * na;
  if (dir < 2 * nj) { *where = 1; return (dir & 1) ? &s.qd[dir >> 1] : &s.q[dir >> 1]; }
  dir -= 2 * nj;
  if (dir < nj) { *where = 2; return &s.act[dir]; }
  dir -= nj;
  if (dir < nread) { *where = 3; return &s.cache[slots[dir]]; }
  *where = -1;
  return nullptr;
}

template <int K>
__global__ void __launch_bounds__(64) tangent_step_kernel(const __grid_constant__ StepArgs A,
                                                          const __grid_constant__ TypeArgs TA,
                                                          const __grid_constant__ TangentArgs V) {
  const int lane = threadIdx.x & 31;
  const int grp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (grp >= TA.n_launch_envs) return;
  const int env = TA.env_ids ? TA.env_ids[grp] : TA.env_first + grp;
  const EnvTypeTable* T = TA.type;
  const int na = T->n_actors, nj = T->n_jdof, nc = T->cache_len;
  const int abase = A.env_actor_base[env], dbase = A.env_dof_base[env];
  const size_t cbase = (size_t)env * A.cache_stride;

  TanState<K> s;
  TanWork<K> w;
  // a fixed root's velocity is not part of the state: the step reads zeros and writes zeros
  unsigned free_mask = 0u;
  for (int l = 0; l < T->n_links; ++l)
    if (T->parent[l] < 0 && T->jtype[l] == kFree) free_mask |= 1u << T->actor[l];
  auto load = [&]() {
    for (int a = 0; a < na; ++a) {
      const float* r = V.root + (size_t)(abase + a) * 13;
      const bool fr = (free_mask >> a) & 1u;
      for (int k = 0; k < 3; ++k) {
        s.rp[a][k] = Dn<K>(r[k]);
        s.rv[a][k] = Dn<K>(fr ? r[7 + k] : 0.f);
        s.rw[a][k] = Dn<K>(fr ? r[10 + k] : 0.f);
      }
      for (int k = 0; k < 4; ++k) s.rq[a][k] = Dn<K>(r[3 + k]);
    }
    for (int j = 0; j < nj; ++j) {
      s.q[j] = Dn<K>(V.dof[(size_t)(dbase + j) * 2]);
      s.qd[j] = Dn<K>(V.dof[(size_t)(dbase + j) * 2 + 1]);
      s.act[j] = Dn<K>(V.act[dbase + j]);
      // drive targets: the handle's target views, as in the forward step
      s.qt[j] = T->has_drives ? A.pos_target[dbase + j] : 0.f;
      s.vt[j] = T->has_drives ? A.vel_target[dbase + j] : 0.f;
    }
    for (int i = 0; i < nc; ++i) s.cache[i] = Dn<K>(V.cache[cbase + i]);
    s.bf = (A.flags & 8) ? A.body_force + (size_t)A.env_body_base[env] * 6 : nullptr;
  };
  bool ok = true;

  if (V.mode == 1) {  // tangent: the caller's direction in slot 0
    load();
    for (int a = 0; a < na; ++a) {
      const float* t = V.t_root + (size_t)(abase + a) * 13;
      const bool fr = (free_mask >> a) & 1u;
      for (int k = 0; k < 3; ++k) {
        s.rp[a][k].d[0] = t[k];
        s.rv[a][k].d[0] = fr ? t[7 + k] : 0.f;
        s.rw[a][k].d[0] = fr ? t[10 + k] : 0.f;
      }
      for (int k = 0; k < 4; ++k) s.rq[a][k].d[0] = t[3 + k];
    }
    for (int j = 0; j < nj; ++j) {
      s.q[j].d[0] = V.t_dof[(size_t)(dbase + j) * 2];
      s.qd[j].d[0] = V.t_dof[(size_t)(dbase + j) * 2 + 1];
      s.act[j].d[0] = V.t_act[dbase + j];
    }
    for (int i = 0; i < nc; ++i) s.cache[i].d[0] = V.t_cache[cbase + i];
    for (int sub = 0; sub < A.substeps && ok; ++sub) ok = tangent_substep<K>(A, T, s, w);
  } else {
    // adjoint. Directions: the state and actuation components, then only the impulse-cache slots
    // the first substep reads (the others cannot affect the step); passes of 32 K directions.
    load();
    int slots[kTanMaxRows];
    int nread = read_slots<K>(A, T, s, w, slots);
    if (nread < 0) { ok = false; nread = 0; }
    const int n_dirs = 13 * na + 3 * nj + nread;
    for (int i = lane; i < A.cache_stride; i += 32) V.gi_cache[cbase + i] = 0.f;
    __syncwarp();
    for (int base = 0; base < n_dirs && ok; base += 32 * K) {
      load();
      for (int k = 0; k < K; ++k) {
        const int dir = base + k * 32 + lane;
        int where;
        Dn<K>* x = input_slot<K>(s, dir, na, nj, slots, nread, &where);
        const bool fixed_vel = where == 0 && (dir % 13) >= 7 && !((free_mask >> (dir / 13)) & 1u);
        if (x && !fixed_vel) x->d[k] = 1.f;
      }
      for (int sub = 0; sub < A.substeps && ok; ++sub) ok = tangent_substep<K>(A, T, s, w);
      // input gradient of each seeded direction: sum over outputs of g_out * d(output)/d(direction)
      for (int k = 0; k < K; ++k) {
        const int dir = base + k * 32 + lane;
        int where;
        if (!input_slot<K>(s, dir, na, nj, slots, nread, &where)) continue;
        float g = 0.f;
        if (V.g_root)
          for (int a = 0; a < na; ++a) {
            const float* gr = V.g_root + (size_t)(abase + a) * 13;
            for (int c = 0; c < 3; ++c) g += gr[c] * s.rp[a][c].d[k] + gr[7 + c] * s.rv[a][c].d[k] + gr[10 + c] * s.rw[a][c].d[k];
            for (int c = 0; c < 4; ++c) g += gr[3 + c] * s.rq[a][c].d[k];
          }
        if (V.g_dof)
          for (int j = 0; j < nj; ++j)
            g += V.g_dof[(size_t)(dbase + j) * 2] * s.q[j].d[k] + V.g_dof[(size_t)(dbase + j) * 2 + 1] * s.qd[j].d[k];
        if (V.g_cache)
          for (int i = 0; i < nc; ++i) g += V.g_cache[cbase + i] * s.cache[i].d[k];
        if (!ok) g = 0.f;
        int d = dir;
        if (where == 0) V.gi_root[(size_t)(abase + d / 13) * 13 + d % 13] = g;
        d -= 13 * na;
        if (where == 1) V.gi_dof[(size_t)(dbase + (d >> 1)) * 2 + (d & 1)] = g;
        d -= 2 * nj;
        if (where == 2) V.gi_act[dbase + d] = g;
        d -= nj;
        if (where == 3) V.gi_cache[cbase + slots[d]] = g;
      }
    }
    if (!ok) {  // a failed step has no derivative: every input gradient of the env is zero
      __syncwarp();
      for (int i = lane; i < 13 * na; i += 32) V.gi_root[(size_t)abase * 13 + i] = 0.f;
      for (int i = lane; i < 2 * nj; i += 32) V.gi_dof[(size_t)dbase * 2 + i] = 0.f;
      for (int i = lane; i < nj; i += 32) V.gi_act[dbase + i] = 0.f;
      __syncwarp();
      for (int i = lane; i < A.cache_stride; i += 32) V.gi_cache[cbase + i] = 0.f;
    }
  }
  if (lane == 0) {
    for (int a = 0; a < na; ++a) {
      const size_t o = (size_t)(abase + a) * 13;
      for (int c = 0; c < 3; ++c) {
        if (V.o_root) { V.o_root[o + c] = s.rp[a][c].v; V.o_root[o + 7 + c] = s.rv[a][c].v; V.o_root[o + 10 + c] = s.rw[a][c].v; }
        if (V.to_root) { V.to_root[o + c] = s.rp[a][c].d[0]; V.to_root[o + 7 + c] = s.rv[a][c].d[0]; V.to_root[o + 10 + c] = s.rw[a][c].d[0]; }
      }
      for (int c = 0; c < 4; ++c) {
        if (V.o_root) V.o_root[o + 3 + c] = s.rq[a][c].v;
        if (V.to_root) V.to_root[o + 3 + c] = s.rq[a][c].d[0];
      }
    }
    for (int j = 0; j < nj; ++j) {
      const size_t o = (size_t)(dbase + j) * 2;
      if (V.o_dof) { V.o_dof[o] = s.q[j].v; V.o_dof[o + 1] = s.qd[j].v; }
      if (V.to_dof) { V.to_dof[o] = s.q[j].d[0]; V.to_dof[o + 1] = s.qd[j].d[0]; }
    }
    for (int i = 0; i < A.cache_stride; ++i) {
      if (V.o_cache) V.o_cache[cbase + i] = i < nc ? s.cache[i].v : 0.f;
      if (V.to_cache) V.to_cache[cbase + i] = i < nc ? s.cache[i].d[0] : 0.f;
    }
    if (V.status) V.status[env] = ok ? 0 : 2;
  }
}

}  // namespace

namespace {

// Mass matrices (what = 0) or link Jacobians (what = 1) at the current state, one thread per env.
__global__ void __launch_bounds__(64) query_kernel(const __grid_constant__ StepArgs A,
                                                   const __grid_constant__ TypeArgs TA, float* out, int what,
                                                   int n_max, int l_max) {
  const int grp = blockIdx.x * blockDim.x + threadIdx.x;
  if (grp >= TA.n_launch_envs) return;
  const int env = TA.env_ids ? TA.env_ids[grp] : TA.env_first + grp;
  const EnvTypeTable* T = TA.type;
  const int na = T->n_actors, nj = T->n_jdof, n = T->n_gen, L = T->n_links;
  const int abase = A.env_actor_base[env], dbase = A.env_dof_base[env];
  TanState<1> s;
  TanWork<1> w;
  unsigned free_mask = 0u;
  for (int l = 0; l < L; ++l)
    if (T->parent[l] < 0 && T->jtype[l] == kFree) free_mask |= 1u << T->actor[l];
  for (int a = 0; a < na; ++a) {
    const float* r = A.root + (size_t)(abase + a) * 13;
    const bool fr = (free_mask >> a) & 1u;
    for (int k = 0; k < 3; ++k) {
      s.rp[a][k] = Dn<1>(r[k]);
      s.rv[a][k] = Dn<1>(fr ? r[7 + k] : 0.f);
      s.rw[a][k] = Dn<1>(fr ? r[10 + k] : 0.f);
    }
    for (int k = 0; k < 4; ++k) s.rq[a][k] = Dn<1>(r[3 + k]);
  }
  for (int j = 0; j < nj; ++j) {
    s.q[j] = Dn<1>(A.dof[(size_t)(dbase + j) * 2]);
    s.qd[j] = Dn<1>(A.dof[(size_t)(dbase + j) * 2 + 1]);
    s.act[j] = Dn<1>(0.f);
  }
  tangent_dynamics<1>(A, T, s, w, false);  // the physical M: no implicit drive term
  if (what == 0) {
    float* o = out + (size_t)env * n_max * n_max;
    for (int i = 0; i < n_max; ++i)
      for (int j = 0; j < n_max; ++j)
        o[i * n_max + j] = (i < n && j < n) ? (i >= j ? w.L[tri(i, j)].v : w.L[tri(j, i)].v) : 0.f;
  } else {
    float* o = out + (size_t)env * l_max * 6 * n_max;
    for (int l = 0; l < l_max; ++l)
      for (int g = 0; g < n_max; ++g) {
        float col[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (l < L && g < n && ((T->anc[l] >> g) & 1u)) {
          // [S_ang; S_lin + S_ang x P]: the motion subspace moved from the actor origin to the link origin
          const float sw0 = w.S[g][0].v, sw1 = w.S[g][1].v, sw2 = w.S[g][2].v;
          const float p0 = w.P[l][0].v, p1 = w.P[l][1].v, p2 = w.P[l][2].v;
          col[0] = sw0; col[1] = sw1; col[2] = sw2;
          col[3] = w.S[g][3].v + sw1 * p2 - sw2 * p1;
          col[4] = w.S[g][4].v + sw2 * p0 - sw0 * p2;
          col[5] = w.S[g][5].v + sw0 * p1 - sw1 * p0;
        }
        for (int r = 0; r < 6; ++r) o[((size_t)l * 6 + r) * n_max + g] = col[r];
      }
  }
}

}  // namespace

cudaError_t launch_query_kernel(int what, const StepArgs& a, const TypeArgs& ta, float* out, int n_max, int l_max,
                                cudaStream_t st) {
  query_kernel<<<(ta.n_launch_envs + 63) / 64, 64, 0, st>>>(a, ta, out, what, n_max, l_max);
  return cudaGetLastError();
}

int tangent_lanes_per_dir(int n_dirs) {
  if (n_dirs <= 32) return 1;
  if (n_dirs <= 64) return 2;
  if (n_dirs <= 128) return 4;
  return 8;
}

namespace {
// The kernel keeps its dual work space in local memory and uses no shared memory: prefer L1.
template <int K> void prefer_l1() {
  static bool done = false;
  if (!done) {
    cudaFuncSetAttribute(tangent_step_kernel<K>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
    done = true;
  }
}
}  // namespace

cudaError_t launch_tangent_kernel(int K, const StepArgs& a, const TypeArgs& ta, const TangentArgs& v, cudaStream_t st) {
  if (K == 1) prefer_l1<1>();
  else if (K == 2) prefer_l1<2>();
  else if (K == 4) prefer_l1<4>();
  else prefer_l1<8>();
  const int blocks = (ta.n_launch_envs + 1) / 2;
  if (K == 1) tangent_step_kernel<1><<<blocks, 64, 0, st>>>(a, ta, v);
  else if (K == 2) tangent_step_kernel<2><<<blocks, 64, 0, st>>>(a, ta, v);
  else if (K == 4) tangent_step_kernel<4><<<blocks, 64, 0, st>>>(a, ta, v);
  else tangent_step_kernel<8><<<blocks, 64, 0, st>>>(a, ta, v);
  return cudaGetLastError();
}

}  // namespace artsim
