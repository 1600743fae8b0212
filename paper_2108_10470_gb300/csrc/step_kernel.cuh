// Fused env-step kernel for sm_103a: every substep of one environment (controls, forward
// kinematics, articulated-body forward dynamics, joint-space inertia, ground contacts and joint
// limits, constraint Jacobian and response, warm-started TGS-style Gauss-Seidel, integration)
// runs inside one group of G lanes, with the environment's tree, contact list and constraint
// rows staged in shared memory and its state in registers between substeps. HBM is touched once
// per env-step: state, actuation and impulse cache in; state, forces, contacts and cache out.
//
// Formulation. Each actor is expressed in world axes about its own reference point O_a = the
// actor root's origin at the start of the substep. Spatial quantities (RBDA ch. 2) are then
// plain sums along the tree with no coordinate transforms between links:
//   * a revolute joint with world axis a through the link origin p has S = [a; p x a], a
//     prismatic joint S = [0; a] (p relative to O_a);
//   * the floating root's generalized velocity is nu = [omega; p_dot] (world axes, root-origin
//     velocity): S = identity at the instant, and its velocity-product term is [0; p_dot x omega];
//   * the articulated-body algorithm (RBDA Table 7.1) runs its three sweeps with per-link
//     rigid-body inertias about O_a and gravity as an external force; the composite-rigid-body
//     inertias of RBDA Table 6.2 are accumulated in the same inward sweep and give the
//     joint-space inertia M_ij = S_i . (I^c_link(i) S_j) for DOF j on the path of DOF i.
// The TGS-style solve follows the paper's TGS paragraph: position iterations accumulate
// h/n_pos * v into the delta buffer dq, which is projected onto each row's Jacobian and added to
// its bias; velocity iterations are unbiased.
//
// Lane roles: "link mode" lane l = env link l; "DOF mode" lane g = generalized DOF g; "row mode"
// lane r = constraint row r (strided by G); "shape mode" lane s = shape s. Every loop whose body
// shuffles has a warp-uniform trip count (maxima over the warp's groups), so the groups of one
// warp stay converged.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "sim_internal.h"

namespace artsim {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------------------------
// Small vector helpers.
struct V3 {
  float x, y, z;
};
__device__ __forceinline__ V3 v3(float x, float y, float z) { return V3{x, y, z}; }
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ V3 operator*(V3 a, float s) { return v3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 cross(V3 a, V3 b) {
  return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
// row-major 3x3
__device__ __forceinline__ V3 mv(const float* R, V3 x) {
  return v3(R[0] * x.x + R[1] * x.y + R[2] * x.z, R[3] * x.x + R[4] * x.y + R[5] * x.z,
            R[6] * x.x + R[7] * x.y + R[8] * x.z);
}
__device__ __forceinline__ void mm(const float* A, const float* B, float* C) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) C[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
}
__device__ __forceinline__ void quat_to_mat(const float* q, float* R) {
  const float x = q[0], y = q[1], z = q[2], w = q[3];
  R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - z * w);       R[2] = 2.f * (x * z + y * w);
  R[3] = 2.f * (x * y + z * w);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - x * w);
  R[6] = 2.f * (x * z - y * w);       R[7] = 2.f * (y * z + x * w);       R[8] = 1.f - 2.f * (x * x + y * y);
}
// Rotation by angle th about unit axis a (Rodrigues), child -> joint coordinates.
__device__ __forceinline__ void axis_angle(V3 a, float th, float* R) {
  float s, c;
  sincosf(th, &s, &c);
  const float t = 1.f - c;
  R[0] = t * a.x * a.x + c;       R[1] = t * a.x * a.y - s * a.z; R[2] = t * a.x * a.z + s * a.y;
  R[3] = t * a.x * a.y + s * a.z; R[4] = t * a.y * a.y + c;       R[5] = t * a.y * a.z - s * a.x;
  R[6] = t * a.x * a.z - s * a.y; R[7] = t * a.y * a.z + s * a.x; R[8] = t * a.z * a.z + c;
}

// Symmetric 6x6 stored as its upper triangle, row-major (21 words).
__host__ __device__ constexpr int sidx(int i, int j) {
  return (i <= j) ? (i * 6 - (i * (i - 1)) / 2 + (j - i)) : (j * 6 - (j * (j - 1)) / 2 + (i - j));
}

// Group-level collectives over G lanes (G = 8, 16 or 32; groups never straddle a warp).
template <int G> struct Grp {
  static __device__ __forceinline__ float sum(float x) {
#pragma unroll
    for (int m = G / 2; m >= 1; m >>= 1) x += __shfl_xor_sync(kFull, x, m, G);
    return x;
  }
  static __device__ __forceinline__ float get(float x, int src) { return __shfl_sync(kFull, x, src, G); }
  static __device__ __forceinline__ int geti(int x, int src) { return __shfl_sync(kFull, x, src, G); }
  static __device__ __forceinline__ int any(int x) {
#pragma unroll
    for (int m = G / 2; m >= 1; m >>= 1) x |= __shfl_xor_sync(kFull, x, m, G);
    return x;
  }
  // exclusive prefix sum over the group's lanes; *total receives the group sum
  static __device__ __forceinline__ int excl_scan(int x, int lane, int* total) {
    int inc = x;
#pragma unroll
    for (int d = 1; d < G; d <<= 1) {
      const int y = __shfl_up_sync(kFull, inc, d, G);
      if (lane >= d) inc += y;
    }
    *total = __shfl_sync(kFull, inc, G - 1, G);
    return inc - x;
  }
};

__device__ __forceinline__ void fnv1a(unsigned& h, int v) {
  const unsigned u = (unsigned)v;
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    h ^= (u >> (8 * b)) & 0xffu;
    h *= 16777619u;
  }
}

// ---------------------------------------------------------------------------------------------
template <int G>
__global__ void __launch_bounds__(128) step_kernel(const StepArgs A) {
  extern __shared__ __align__(16) float smem[];
  const EnvTypeTable* __restrict__ T = A.type;
  const int lane = threadIdx.x & (G - 1);
  const int grp_blk = threadIdx.x / G;
  const int grp = blockIdx.x * (blockDim.x / G) + grp_blk;
  const bool live = grp < A.n_launch_envs;
  const int gi = live ? grp : A.n_launch_envs - 1;  // dead groups shadow the last env, never store
  const int env = A.env_ids ? A.env_ids[gi] : A.env_first + gi;
  const SmemLayout& Ly = A.lay;
  float* sm = smem + grp_blk * Ly.total;
  int* smi = reinterpret_cast<int*>(sm);

  const int L = T->n_links, n = T->n_gen, NS = T->n_shapes;
  const int maxdepth = T->max_depth;
  const int RS = Ly.RS, MS = Ly.MS, CC = Ly.ccap, RC = Ly.rcap;
  float* s_link = sm + Ly.link;
  float* s_J = sm + Ly.J;
  float* s_W = sm + Ly.W;
  float* s_S = sm + Ly.S;
  float* s_M = sm + Ly.M;
  float* s_qdd = sm + Ly.vec;
  float* s_v0 = s_qdd + n;
  float* s_vf = s_v0 + n;
  float* s_dq = s_vf + n;
  float* s_Linv = s_dq + n;
  float* s_con = sm + Ly.con;
  float* s_row = sm + Ly.rowh;
  int* s_rowi = smi + Ly.rowh;
  int* s_coni = smi + Ly.con;
  float* s_cache = sm + Ly.cache;
  float* s_frc = sm + Ly.frc;

  // ---- per-link constants (link mode) ----
  const bool isl = lane < L;
  const int l = isl ? lane : 0;
  const int par = isl ? T->parent[l] : -1;
  const int jt = T->jtype[l];
  const int dep = isl ? T->depth[l] : -1;
  const int gd = T->gdof[l];
  const int jd = T->jdof[l];
  const int ar = T->aroot[l];
  const bool is_root = isl && par < 0;
  const bool free_root = is_root && jt == kFree;
  const bool has_dof = isl && (jt == kRevolute || jt == kPrismatic);
  const V3 jaxis = v3(T->axis[0][l], T->axis[1][l], T->axis[2][l]);
  const float damping = T->damping[l], armature = T->armature[l];

  // ---- load state (one HBM read per env-step) ----
  const int dof_base = A.env_dof_base[env];
  float rq[4] = {0.f, 0.f, 0.f, 1.f};
  V3 rp = v3(0.f, 0.f, 0.f), rw = rp, rv = rp;  // root pose / velocity (root lanes)
  float q = 0.f, qd = 0.f, f = 0.f;
  if (is_root) {
    const float* r = A.root + (size_t)(env * A.actors_per_env + T->actor[l]) * 13;
    rp = v3(r[0], r[1], r[2]);
    rq[0] = r[3]; rq[1] = r[4]; rq[2] = r[5]; rq[3] = r[6];
    rv = v3(r[7], r[8], r[9]);
    rw = v3(r[10], r[11], r[12]);
    if (!free_root) { rv = v3(0.f, 0.f, 0.f); rw = rv; }
  }
  if (has_dof) {
    q = A.dof[(size_t)(dof_base + jd) * 2];
    qd = A.dof[(size_t)(dof_base + jd) * 2 + 1];
    f = A.act[dof_base + jd];
  }
  for (int i = lane; i < T->cache_len; i += G) s_cache[i] = A.cache[(size_t)env * A.cache_stride + i];
  for (int i = lane; i < 3 * L; i += G) s_frc[i] = 0.f;
  const float tau = f;  // joint force; damping is applied with the substep's velocity below

  unsigned sig = 2166136261u;
  int status = 0;
  const float h = A.h;
  const int npos = A.pos_iters, nvel = A.vel_iters;
  const float hit = h / (float)npos;
  const V3 g = v3(A.gx, A.gy, A.gz);
  int n_con = 0, n_lim = 0, R = 0;

  for (int sub = 0; sub < A.substeps; ++sub) {
    // ======== (a2) forward kinematics + velocities, level-synchronous (link mode) ========
    float Rw[9];  // link -> world rotation
    V3 P = v3(0.f, 0.f, 0.f);  // link origin relative to the actor origin O_a
    V3 Ow = rp;                // actor origin in world (root lanes; others fetch below)
    float vs[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // link spatial velocity [w; v] about O_a
    float Sa[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // joint motion subspace about O_a
    float cc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // velocity-product acceleration
    quat_to_mat(rq, Rw);
    if (is_root) {
      vs[0] = rw.x; vs[1] = rw.y; vs[2] = rw.z; vs[3] = rv.x; vs[4] = rv.y; vs[5] = rv.z;
      const V3 pxw = cross(rv, rw);  // d/dt S_root * nu = [0; p_dot x omega]
      cc[3] = pxw.x; cc[4] = pxw.y; cc[5] = pxw.z;
    }
    {
      const float ox = Grp<G>::get(rp.x, ar), oy = Grp<G>::get(rp.y, ar), oz = Grp<G>::get(rp.z, ar);
      Ow = v3(ox, oy, oz);
    }
    for (int d = 1; d <= maxdepth; ++d) {
      float Rp[9], vp[6];
      const int src = par >= 0 ? par : lane;
#pragma unroll
      for (int k = 0; k < 9; ++k) Rp[k] = Grp<G>::get(Rw[k], src);
#pragma unroll
      for (int k = 0; k < 6; ++k) vp[k] = Grp<G>::get(vs[k], src);
      const float ppx = Grp<G>::get(P.x, src), ppy = Grp<G>::get(P.y, src), ppz = Grp<G>::get(P.z, src);
      if (dep == d) {
        const V3 Pp = v3(ppx, ppy, ppz);
        float Rpj[9], RB[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) Rpj[k] = T->prot[k][l];
        mm(Rp, Rpj, RB);
        const V3 pp = v3(T->ppos[0][l], T->ppos[1][l], T->ppos[2][l]);
        const V3 aw = mv(RB, jaxis);
        if (jt == kRevolute) {
          float RJ[9];
          axis_angle(jaxis, q, RJ);
          mm(RB, RJ, Rw);
          P = Pp + mv(Rp, pp);
          const V3 pxa = cross(P, aw);
          Sa[0] = aw.x; Sa[1] = aw.y; Sa[2] = aw.z; Sa[3] = pxa.x; Sa[4] = pxa.y; Sa[5] = pxa.z;
        } else if (jt == kPrismatic) {
#pragma unroll
          for (int k = 0; k < 9; ++k) Rw[k] = RB[k];
          P = Pp + mv(Rp, pp + mv(Rpj, jaxis * q));
          Sa[3] = aw.x; Sa[4] = aw.y; Sa[5] = aw.z;
        } else {
#pragma unroll
          for (int k = 0; k < 9; ++k) Rw[k] = RB[k];
          P = Pp + mv(Rp, pp);
        }
        float sq[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) { sq[k] = Sa[k] * qd; vs[k] = vp[k] + sq[k]; }
        // c = v x (S qd) (motion cross product)
        const V3 w = v3(vs[0], vs[1], vs[2]), vl = v3(vs[3], vs[4], vs[5]);
        const V3 sa = v3(sq[0], sq[1], sq[2]), sl = v3(sq[3], sq[4], sq[5]);
        const V3 c0 = cross(w, sa), c1 = cross(w, sl) + cross(vl, sa);
        cc[0] = c0.x; cc[1] = c0.y; cc[2] = c0.z; cc[3] = c1.x; cc[4] = c1.y; cc[5] = c1.z;
      }
    }
    if (isl) {
#pragma unroll
      for (int k = 0; k < 6; ++k) s_S[6 * l + k] = Sa[k];
    }

    // ======== (a3) rigid-body inertias about O_a, bias forces: p = v x* I v - f_gravity ========
    float U[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, Dinv = 0.f, uu = 0.f;
    if (isl) {
      const float m = T->mass[l];
      const V3 cw = P + mv(Rw, v3(T->com[0][l], T->com[1][l], T->com[2][l]));
      // rotational inertia about the COM in world axes: R Ic R^T
      float Ic[9] = {T->inertia[0][l], T->inertia[3][l], T->inertia[4][l], T->inertia[3][l], T->inertia[1][l],
                     T->inertia[5][l], T->inertia[4][l], T->inertia[5][l], T->inertia[2][l]};
      float RI[9], RIRt[9], Rt[9];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Rt[3 * i + j] = Rw[3 * j + i];
      mm(Rw, Ic, RI);
      mm(RI, Rt, RIRt);
      // I_O = Ic_w + m (|c|^2 1 - c c^T); h = m c
      const float c2 = dot(cw, cw);
      const float Ixx = RIRt[0] + m * (c2 - cw.x * cw.x), Iyy = RIRt[4] + m * (c2 - cw.y * cw.y),
                  Izz = RIRt[8] + m * (c2 - cw.z * cw.z);
      const float Ixy = RIRt[1] - m * cw.x * cw.y, Ixz = RIRt[2] - m * cw.x * cw.z, Iyz = RIRt[5] - m * cw.y * cw.z;
      const V3 hh = cw * m;
      // I v = [I_O w + h x v; m v + w x h]
      const V3 w = v3(vs[0], vs[1], vs[2]), vl = v3(vs[3], vs[4], vs[5]);
      const V3 Iw = v3(Ixx * w.x + Ixy * w.y + Ixz * w.z, Ixy * w.x + Iyy * w.y + Iyz * w.z,
                       Ixz * w.x + Iyz * w.y + Izz * w.z);
      const V3 Fa = Iw + cross(hh, vl), Fl = vl * m + cross(w, hh);
      // v x* F = [w x Fa + v x Fl; w x Fl]; gravity force I [0; g] = [h x g; m g]
      const V3 pa = cross(w, Fa) + cross(vl, Fl) - cross(hh, g);
      const V3 pl = cross(w, Fl) - g * m;
      float* sl = s_link + kLinkWords * l;
      // articulated inertia starts as the rigid inertia: [[I_O, h~], [h~^T, m 1]]
      sl[sidx(0, 0)] = Ixx; sl[sidx(0, 1)] = Ixy; sl[sidx(0, 2)] = Ixz;
      sl[sidx(1, 1)] = Iyy; sl[sidx(1, 2)] = Iyz; sl[sidx(2, 2)] = Izz;
      sl[sidx(0, 3)] = 0.f;    sl[sidx(0, 4)] = -hh.z; sl[sidx(0, 5)] = hh.y;
      sl[sidx(1, 3)] = hh.z;   sl[sidx(1, 4)] = 0.f;   sl[sidx(1, 5)] = -hh.x;
      sl[sidx(2, 3)] = -hh.y;  sl[sidx(2, 4)] = hh.x;  sl[sidx(2, 5)] = 0.f;
      sl[sidx(3, 3)] = m; sl[sidx(3, 4)] = 0.f; sl[sidx(3, 5)] = 0.f;
      sl[sidx(4, 4)] = m; sl[sidx(4, 5)] = 0.f; sl[sidx(5, 5)] = m;
      sl[21] = pa.x; sl[22] = pa.y; sl[23] = pa.z; sl[24] = pl.x; sl[25] = pl.y; sl[26] = pl.z;
      // composite rigid inertia (m, h, I_O)
      sl[27] = m; sl[28] = hh.x; sl[29] = hh.y; sl[30] = hh.z;
      sl[31] = Ixx; sl[32] = Iyy; sl[33] = Izz; sl[34] = Ixy; sl[35] = Ixz; sl[36] = Iyz;
    }
    __syncwarp();

    // ======== inward sweep: articulated inertias (ABA pass 2) and composite inertias ========
    const float tau_sub = tau - damping * qd;
    for (int d = maxdepth; d >= 1; --d) {
      if (dep == d && has_dof) {
        float* sl = s_link + kLinkWords * l;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
          float s = 0.f;
#pragma unroll
          for (int j = 0; j < 6; ++j) s += sl[sidx(i, j)] * Sa[j];
          U[i] = s;
        }
        float D = armature, sp = 0.f;
#pragma unroll
        for (int i = 0; i < 6; ++i) { D += Sa[i] * U[i]; sp += Sa[i] * sl[21 + i]; }
        Dinv = 1.f / D;
        uu = tau_sub - sp;
        if (!(D > 0.f)) status |= 2;
        // Ia = IA - U U^T / D ; pa = pA + Ia c + U u / D
#pragma unroll
        for (int i = 0; i < 6; ++i)
#pragma unroll
          for (int j = i; j < 6; ++j) sl[sidx(i, j)] -= U[i] * U[j] * Dinv;
        float pa[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
          float s = sl[21 + i] + U[i] * uu * Dinv;
#pragma unroll
          for (int j = 0; j < 6; ++j) s += sl[sidx(i, j)] * cc[j];
          pa[i] = s;
        }
#pragma unroll
        for (int i = 0; i < 6; ++i) sl[21 + i] = pa[i];
      }
      __syncwarp();
      if (dep == d - 1) {
        float* sl = s_link + kLinkWords * l;
        for (int ch = T->first_child[l]; ch >= 0; ch = T->next_sibling[ch]) {
          const float* sc = s_link + kLinkWords * ch;
#pragma unroll
          for (int k = 0; k < kLinkWords; ++k) sl[k] += sc[k];
        }
      }
      __syncwarp();
    }

    // ======== root acceleration, outward sweep (ABA pass 3) ========
    float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float qdd = 0.f;
    if (free_root) {
      // a0 = -(IA)^-1 pA by a 6x6 Cholesky solve in registers
      const float* sl = s_link + kLinkWords * l;
      float Lc[21], y[6];
#pragma unroll
      for (int k = 0; k < 21; ++k) Lc[k] = sl[k];
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        float s = Lc[sidx(j, j)];
#pragma unroll
        for (int k = 0; k < j; ++k) s -= Lc[sidx(j, k)] * Lc[sidx(j, k)];
        if (!(s > 0.f)) { status |= 2; s = 1.f; }
        const float ljj = sqrtf(s), inv = 1.f / ljj;
        Lc[sidx(j, j)] = ljj;
#pragma unroll
        for (int i = j + 1; i < 6; ++i) {
          float t = Lc[sidx(i, j)];
#pragma unroll
          for (int k = 0; k < j; ++k) t -= Lc[sidx(i, k)] * Lc[sidx(j, k)];
          Lc[sidx(i, j)] = t * inv;
        }
      }
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        float s = -sl[21 + i];
#pragma unroll
        for (int k = 0; k < i; ++k) s -= Lc[sidx(i, k)] * y[k];
        y[i] = s / Lc[sidx(i, i)];
      }
#pragma unroll
      for (int i = 5; i >= 0; --i) {
        float s = y[i];
#pragma unroll
        for (int k = i + 1; k < 6; ++k) s -= Lc[sidx(k, i)] * acc[k];
        acc[i] = s / Lc[sidx(i, i)];
      }
    }
    for (int d = 1; d <= maxdepth; ++d) {
      float ap[6];
      const int src = par >= 0 ? par : lane;
#pragma unroll
      for (int k = 0; k < 6; ++k) ap[k] = Grp<G>::get(acc[k], src);
      if (dep == d) {
#pragma unroll
        for (int k = 0; k < 6; ++k) acc[k] = ap[k] + cc[k];
        if (has_dof) {
          float ua = 0.f;
#pragma unroll
          for (int k = 0; k < 6; ++k) ua += U[k] * acc[k];
          qdd = (uu - ua) * Dinv;
#pragma unroll
          for (int k = 0; k < 6; ++k) acc[k] += Sa[k] * qdd;
        }
      }
    }
    // generalized velocity and its rate (root: nu_dot = a0 - [0; p_dot x omega])
    if (has_dof) { s_qdd[gd] = qdd; s_v0[gd] = qd; }
    if (free_root) {
#pragma unroll
      for (int k = 0; k < 6; ++k) { s_qdd[gd + k] = acc[k] - cc[k]; s_v0[gd + k] = vs[k]; }
    }
    __syncwarp();

    // ======== joint-space inertia M (DOF mode) ========
    const bool isg = lane < n;
    const int gl = isg ? T->dof_link[lane] : 0;
    const int gcomp = isg ? T->dof_comp[lane] : -1;
    float Sg[6];
    if (gcomp >= 0) {
#pragma unroll
      for (int k = 0; k < 6; ++k) Sg[k] = (k == gcomp) ? 1.f : 0.f;
    } else {
#pragma unroll
      for (int k = 0; k < 6; ++k) Sg[k] = s_S[6 * gl + k];
    }
    if (isg) {
      const float* ic = s_link + kLinkWords * gl + 27;
      const float m = ic[0];
      const V3 hh = v3(ic[1], ic[2], ic[3]);
      const V3 w = v3(Sg[0], Sg[1], Sg[2]), vl = v3(Sg[3], Sg[4], Sg[5]);
      const V3 Iw = v3(ic[4] * w.x + ic[7] * w.y + ic[8] * w.z, ic[7] * w.x + ic[5] * w.y + ic[9] * w.z,
                       ic[8] * w.x + ic[9] * w.y + ic[6] * w.z);
      const V3 Fa = Iw + cross(hh, vl), Fl = vl * m + cross(w, hh);
      const float F[6] = {Fa.x, Fa.y, Fa.z, Fl.x, Fl.y, Fl.z};
      const unsigned anc = T->anc[gl];
      for (int j = 0; j <= lane; ++j) {
        float mij = 0.f;
        if ((anc >> j) & 1u) {
          const int jc = T->dof_comp[j];
          if (jc >= 0) {
            mij = F[jc];
          } else {
            const float* Sj = s_S + 6 * T->dof_link[j];
#pragma unroll
            for (int k = 0; k < 6; ++k) mij += Sj[k] * F[k];
          }
        }
        if (j == lane && gcomp < 0) mij += T->armature[gl];
        s_M[lane * MS + j] = mij;
      }
    }
    __syncwarp();
    // ======== dense Cholesky M = L L^T (lanes = rows; lower triangle in place) ========
    for (int k = 0; k < n; ++k) {
      float akk = s_M[k * MS + k];
      if (!(akk > 0.f)) { status |= 2; akk = 1.f; }
      const float lkk = sqrtf(akk), inv = 1.f / lkk;
      __syncwarp();
      if (lane > k && lane < n) s_M[lane * MS + k] *= inv;
      if (lane == k) { s_M[k * MS + k] = lkk; s_Linv[k] = inv; }
      __syncwarp();
      if (lane > k && lane < n) {
        const float lik = s_M[lane * MS + k];
        for (int j = k + 1; j <= lane; ++j) s_M[lane * MS + j] -= lik * s_M[j * MS + k];
      }
      __syncwarp();
    }

    // ======== (a4) ground contacts (shape mode) and limit rows (link mode) ========
    {
      // shape lanes fetch their link's pose
      const int sl_link = (lane < NS) ? T->shape_link[lane] : 0;
      float Rl[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) Rl[k] = Grp<G>::get(Rw[k], sl_link);
      const float plx = Grp<G>::get(P.x, sl_link), ply = Grp<G>::get(P.y, sl_link), plz = Grp<G>::get(P.z, sl_link);
      const float oz = Grp<G>::get(Ow.z, sl_link);
      int nk = 0;
      unsigned keep = 0u;
      float zc[8];
      V3 xs[8];
      const int st = (lane < NS) ? T->shape_type[lane] : -1;
      const float coff = A.contact_offset;
      if (lane < NS) {
        float Rsh[9], Rs[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) Rsh[k] = T->shape_rot[k][lane];
        mm(Rl, Rsh, Rs);
        const V3 cs = v3(plx, ply, plz) + mv(Rl, v3(T->shape_pos[0][lane], T->shape_pos[1][lane], T->shape_pos[2][lane]));
        const float s0 = T->shape_size[0][lane], s1 = T->shape_size[1][lane], s2 = T->shape_size[2][lane];
        if (st == kSphere) {
          xs[0] = v3(cs.x, cs.y, cs.z - s0);
          zc[0] = (oz + cs.z) - s0;
          nk = 1;
        } else if (st == kCapsule) {
          const V3 ax = v3(Rs[0], Rs[3], Rs[6]);
          const V3 e0 = cs - ax * s1, e1 = cs + ax * s1;
          xs[0] = v3(e0.x, e0.y, e0.z - s0);
          xs[1] = v3(e1.x, e1.y, e1.z - s0);
          zc[0] = (oz + e0.z) - s0;
          zc[1] = (oz + e1.z) - s0;
          nk = 2;
        } else {
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const V3 loc = v3((k & 4) ? s0 : -s0, (k & 2) ? s1 : -s1, (k & 1) ? s2 : -s2);
            xs[k] = cs + mv(Rs, loc);
            zc[k] = oz + xs[k].z;
          }
          nk = 8;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k)
          if (k < nk && zc[k] < coff) keep |= 1u << k;
      }
      const int cnt = __popc(keep);
      const int base = Grp<G>::excl_scan(cnt, lane, &n_con);
      if (lane < NS) {
        int o = base;
        const float mu = T->shape_mu[lane];
        const int coff_s = T->cand_off[lane];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          if ((keep >> k) & 1u) {
            s_con[0 * CC + o] = xs[k].x;
            s_con[1 * CC + o] = xs[k].y;
            s_con[2 * CC + o] = xs[k].z;
            s_con[3 * CC + o] = zc[k];
            s_con[4 * CC + o] = mu;
            s_coni[5 * CC + o] = sl_link;
            s_coni[6 * CC + o] = coff_s + k;
            s_coni[7 * CC + o] = lane;
            s_coni[8 * CC + o] = k;
            ++o;
          }
        }
      }
      // limit rows in DOF order: link lanes with a limited joint
      int lf = 0;
      float dlo = 0.f, dhi = 0.f;
      if (has_dof && T->has_limit[l]) {
        dlo = q - T->lo[l];
        dhi = T->hi[l] - q;
        if (dlo < A.limit_margin) lf |= 1;
        if (dhi < A.limit_margin) lf |= 2;
      }
      const int lbase = Grp<G>::excl_scan(__popc(lf), lane, &n_lim);
      if (lf) {
        int o = lbase;
        if (lf & 1) {
          s_rowi[0 * RC + o] = kRowLimit; s_rowi[1 * RC + o] = gd; s_row[2 * RC + o] = dlo;
          s_row[5 * RC + o] = 1.f; s_rowi[6 * RC + o] = 3 * T->n_cand + 2 * jd; ++o;
        }
        if (lf & 2) {
          s_rowi[0 * RC + o] = kRowLimit; s_rowi[1 * RC + o] = gd | (1 << 16); s_row[2 * RC + o] = dhi;
          s_row[5 * RC + o] = -1.f; s_rowi[6 * RC + o] = 3 * T->n_cand + 2 * jd + 1;
        }
      }
      R = n_lim + 3 * n_con;
      __syncwarp();
      // contact rows: normal rows then friction pairs
      for (int c = lane; c < n_con; c += G) {
        const int cand = s_coni[6 * CC + c];
        const float mu = s_con[4 * CC + c];
        const int rn = n_lim + c;
        s_rowi[0 * RC + rn] = kRowNormal; s_rowi[1 * RC + rn] = c; s_row[2 * RC + rn] = s_con[3 * CC + c];
        s_row[5 * RC + rn] = mu; s_rowi[6 * RC + rn] = 3 * cand;
        for (int t = 0; t < 2; ++t) {
          const int rf = n_lim + n_con + 2 * c + t;
          s_rowi[0 * RC + rf] = kRowFriction; s_rowi[1 * RC + rf] = c | (t << 16); s_row[2 * RC + rf] = 0.f;
          s_row[5 * RC + rf] = mu; s_rowi[6 * RC + rf] = 3 * cand + 1 + t;
        }
      }
      if ((A.flags & 1) && lane == 0) {
        fnv1a(sig, n_lim);
        for (int r = 0; r < n_lim; ++r) {
          const int aux = s_rowi[1 * RC + r];
          // env joint-DOF index of the limited DOF: the row's cache slot encodes it
          const int slot = s_rowi[6 * RC + r] - 3 * T->n_cand;
          fnv1a(sig, slot >> 1);
          fnv1a(sig, (aux >> 16) & 1);
        }
        fnv1a(sig, n_con);
        for (int c = 0; c < n_con; ++c) {
          fnv1a(sig, s_coni[7 * CC + c]);
          fnv1a(sig, -1);
          fnv1a(sig, s_coni[8 * CC + c]);
        }
      }
      __syncwarp();
    }

    // ======== (a5) constraint Jacobian rows (DOF mode) ========
    const int Rw_max = __reduce_max_sync(kFull, R);
    {
      const unsigned gbit = 1u << (lane & 31);
      for (int r = 0; r < R; ++r) {
        const int kind = s_rowi[0 * RC + r];
        const int aux = s_rowi[1 * RC + r];
        float jv = 0.f;
        if (kind == kRowLimit) {
          jv = ((aux & 0xffff) == lane) ? s_row[5 * RC + r] : 0.f;
        } else {
          const int c = aux & 0xffff;
          const int la = s_coni[5 * CC + c];
          if (isg && (T->anc[la] & gbit)) {
            const V3 x = v3(s_con[0 * CC + c], s_con[1 * CC + c], s_con[2 * CC + c]);
            // k = e_z (normal), e_x / e_y (friction t = 0 / 1); f = [x x k; k]
            float fr[6];
            if (kind == kRowNormal) { fr[0] = x.y; fr[1] = -x.x; fr[2] = 0.f; fr[3] = 0.f; fr[4] = 0.f; fr[5] = 1.f; }
            else if ((aux >> 16) == 0) { fr[0] = 0.f; fr[1] = x.z; fr[2] = -x.y; fr[3] = 1.f; fr[4] = 0.f; fr[5] = 0.f; }
            else { fr[0] = -x.z; fr[1] = 0.f; fr[2] = x.x; fr[3] = 0.f; fr[4] = 1.f; fr[5] = 0.f; }
#pragma unroll
            for (int k = 0; k < 6; ++k) jv += Sg[k] * fr[k];
          }
        }
        if (isg) s_J[lane * RS + r] = jv;
      }
    }
    __syncwarp();
    // ======== response W = M^-1 J^T, A = J W, warm start (row mode) ========
    for (int r = lane; r < R; r += G) {
      for (int i = 0; i < n; ++i) {
        float y = s_J[i * RS + r];
        for (int k = 0; k < i; ++k) y -= s_M[i * MS + k] * s_W[k * RS + r];
        s_W[i * RS + r] = y * s_Linv[i];
      }
      for (int i = n - 1; i >= 0; --i) {
        float y = s_W[i * RS + r];
        for (int k = i + 1; k < n; ++k) y -= s_M[k * MS + i] * s_W[k * RS + r];
        s_W[i * RS + r] = y * s_Linv[i];
      }
      float a = 0.f;
      for (int i = 0; i < n; ++i) a += s_J[i * RS + r] * s_W[i * RS + r];
      const bool act = a > 1e-12f;
      s_row[3 * RC + r] = act ? 1.f / a : 0.f;
      s_row[4 * RC + r] = act ? s_cache[s_rowi[6 * RC + r]] : 0.f;
    }
    __syncwarp();

    // ======== (a6) TGS-style projected Gauss-Seidel (DOF mode) ========
    float v = 0.f, dq = 0.f;
    if (isg) {
      v = s_v0[lane] + h * s_qdd[lane];
      for (int r = 0; r < R; ++r) v += s_W[lane * RS + r] * s_row[4 * RC + r];
    }
    {
      const float inv_hit = 1.f / hit, inv_h = 1.f / h;
      const float beta = A.bias_coef, vmax = A.max_depen_vel;
      for (int it = 0; it < npos + nvel; ++it) {
        const bool pos = it < npos;
        for (int r = 0; r < Rw_max; ++r) {
          const bool rv = r < R;
          float jj = 0.f, ww = 0.f;
          if (rv && isg) { jj = s_J[lane * RS + r]; ww = s_W[lane * RS + r]; }
          const float jv = Grp<G>::sum(jj * v);
          const float jdq = Grp<G>::sum(jj * dq);
          if (rv) {
            const float invA = s_row[3 * RC + r];
            if (invA > 0.f) {
              const int kind = s_rowi[0 * RC + r];
              const float lam = s_row[4 * RC + r];
              float lnew;
              if (kind == kRowFriction) {
                const int c = s_rowi[1 * RC + r] & 0xffff;
                const float lim = s_row[5 * RC + r] * s_row[4 * RC + (n_lim + c)];
                lnew = fminf(fmaxf(lam - jv * invA, -lim), lim);
              } else {
                const float sep = s_row[2 * RC + r] + jdq;
                float target;
                if (pos) target = (sep >= 0.f) ? -sep * inv_hit : fminf(-beta * sep * inv_hit, vmax);
                else target = (sep > 0.f) ? -sep * inv_h : 0.f;
                lnew = fmaxf(lam + (target - jv) * invA, 0.f);
              }
              v += ww * (lnew - lam);
              s_row[4 * RC + r] = lnew;  // every lane stores the same value
            }
          }
        }
        if (pos) dq += hit * v;
      }
    }
    if (isg) { s_vf[lane] = v; s_dq[lane] = dq; }
    __syncwarp();

    // ======== impulse cache, contact impulses per link ========
    for (int i = lane; i < T->cache_len; i += G) s_cache[i] = 0.f;
    __syncwarp();
    for (int r = lane; r < R; r += G) s_cache[s_rowi[6 * RC + r]] = s_row[4 * RC + r];
    if (isl) {
      float fx = 0.f, fy = 0.f, fz = 0.f;
      for (int c = 0; c < n_con; ++c) {
        if (s_coni[5 * CC + c] == l) {
          fz += s_row[4 * RC + (n_lim + c)];
          fx += s_row[4 * RC + (n_lim + n_con + 2 * c)];
          fy += s_row[4 * RC + (n_lim + n_con + 2 * c + 1)];
        }
      }
      s_frc[3 * l] += fx; s_frc[3 * l + 1] += fy; s_frc[3 * l + 2] += fz;
    }
    __syncwarp();

    // ======== (a7) integrate (link mode) ========
    if (has_dof) { q += s_dq[gd]; qd = s_vf[gd]; }
    if (free_root) {
      const V3 da = v3(s_dq[gd], s_dq[gd + 1], s_dq[gd + 2]);
      rp = rp + v3(s_dq[gd + 3], s_dq[gd + 4], s_dq[gd + 5]);
      rw = v3(s_vf[gd], s_vf[gd + 1], s_vf[gd + 2]);
      rv = v3(s_vf[gd + 3], s_vf[gd + 4], s_vf[gd + 5]);
      // quat <- exp(da) * quat, exact exponential, then normalise
      const float a2 = dot(da, da);
      float e[4];
      if (a2 < 1e-30f) { e[0] = 0.5f * da.x; e[1] = 0.5f * da.y; e[2] = 0.5f * da.z; e[3] = 1.f; }
      else {
        const float an = sqrtf(a2);
        float sn, cs;
        sincosf(0.5f * an, &sn, &cs);
        const float s = sn / an;
        e[0] = da.x * s; e[1] = da.y * s; e[2] = da.z * s; e[3] = cs;
      }
      const float x = e[3] * rq[0] + e[0] * rq[3] + e[1] * rq[2] - e[2] * rq[1];
      const float y = e[3] * rq[1] - e[0] * rq[2] + e[1] * rq[3] + e[2] * rq[0];
      const float z = e[3] * rq[2] + e[0] * rq[1] - e[1] * rq[0] + e[2] * rq[3];
      const float w = e[3] * rq[3] - e[0] * rq[0] - e[1] * rq[1] - e[2] * rq[2];
      const float nr = sqrtf(x * x + y * y + z * z + w * w);
      rq[0] = x / nr; rq[1] = y / nr; rq[2] = z / nr; rq[3] = w / nr;
    }
    __syncwarp();
  }  // substeps

  // ======== outputs (one HBM write per env-step) ========
  if (is_root) {
    if (!(isfinite(rp.x) && isfinite(rp.y) && isfinite(rp.z) && isfinite(rq[0]) && isfinite(rq[1]) &&
          isfinite(rq[2]) && isfinite(rq[3]) && isfinite(rv.x) && isfinite(rv.y) && isfinite(rv.z) &&
          isfinite(rw.x) && isfinite(rw.y) && isfinite(rw.z)))
      status |= 1;
  }
  if (has_dof && !(isfinite(q) && isfinite(qd))) status |= 1;
  status = Grp<G>::any(status);
  if (live) {
    if (is_root) {
      float* r = A.root + (size_t)(env * A.actors_per_env + T->actor[l]) * 13;
      r[0] = rp.x; r[1] = rp.y; r[2] = rp.z;
      r[3] = rq[0]; r[4] = rq[1]; r[5] = rq[2]; r[6] = rq[3];
      r[7] = rv.x; r[8] = rv.y; r[9] = rv.z;
      r[10] = rw.x; r[11] = rw.y; r[12] = rw.z;
    }
    if (has_dof) {
      A.dof[(size_t)(dof_base + jd) * 2] = q;
      A.dof[(size_t)(dof_base + jd) * 2 + 1] = qd;
    }
    const int bd = isl ? T->body[l] : -1;
    if (bd >= 0) {
      const float inv_dt = 1.f / A.dt;
      float* nf = A.net_force + (size_t)(A.env_body_base[env] + bd) * 3;
      nf[0] = s_frc[3 * l] * inv_dt; nf[1] = s_frc[3 * l + 1] * inv_dt; nf[2] = s_frc[3 * l + 2] * inv_dt;
    }
    for (int i = lane; i < T->cache_len; i += G) A.cache[(size_t)env * A.cache_stride + i] = s_cache[i];
    int* pr = A.pairs + (size_t)env * A.pair_stride * 3;
    for (int c = lane; c < A.pair_stride; c += G) {
      const bool vc = c < n_con;
      pr[3 * c + 0] = vc ? s_coni[7 * CC + c] : -1;
      pr[3 * c + 1] = -1;
      pr[3 * c + 2] = vc ? s_coni[8 * CC + c] : -1;
    }
    if (lane == 0) {
      A.n_pairs[env] = n_con;
      A.status[env] = status;
      if (A.flags & 1) A.sig[env] = sig;
    }
  }
}

}  // namespace artsim
