// Forward-mode derivative of the env-step on the GPU: the step of step_kernel.cuh evaluated by one
// lane in dual arithmetic (a value and K tangents), serially over the env's links, DOFs, contacts
// and rows. Every lane of a warp evaluates the same env with its own K input directions seeded, so
// a warp yields 32 K columns of the env-step's Jacobian; contracting them with an output gradient
// gives the vector-Jacobian product (the adjoint) without communication between lanes.
//
// The discrete step is the forward kernel's (joint forces, forward kinematics, articulated-body
// dynamics, ground contacts and joint-limit rows, the TGS-style projected Gauss-Seidel solve in
// z = L^T v, integration), written here in its joint-space form: M qdd = tau - b with the
// joint-space inertia M from composite inertias and the bias b from a recursive Newton-Euler pass,
// both in world axes about each actor's root origin. Branches (contact and limit decisions, clamps,
// the speculative / biased target) follow the value, so the derivative is that of the step with its
// constraint and active sets held fixed. Capsule-box pair contacts go through a dual version of the
// forward step's pair geometry (segment-box closest point, face clip, sphere-box) with two-body rows.
#pragma once
#include "sim_internal.h"

namespace artsim {

// ---- dual numbers ------------------------------------------------------------------------------
template <int K> struct Dn {
  float v;
  float d[K];
  __device__ __forceinline__ Dn() {}
  __device__ __forceinline__ Dn(float x) : v(x) {
#pragma unroll
    for (int k = 0; k < K; ++k) d[k] = 0.f;
  }
};
template <int K> __device__ __forceinline__ Dn<K> operator+(const Dn<K>& a, const Dn<K>& b) {
  Dn<K> r; r.v = a.v + b.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] + b.d[k];
  return r;
}
template <int K> __device__ __forceinline__ Dn<K> operator-(const Dn<K>& a, const Dn<K>& b) {
  Dn<K> r; r.v = a.v - b.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] - b.d[k];
  return r;
}
template <int K> __device__ __forceinline__ Dn<K> operator-(const Dn<K>& a) {
  Dn<K> r; r.v = -a.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = -a.d[k];
  return r;
}
template <int K> __device__ __forceinline__ Dn<K> operator*(const Dn<K>& a, const Dn<K>& b) {
  Dn<K> r; r.v = a.v * b.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
  return r;
}
template <int K> __device__ __forceinline__ Dn<K> operator*(const Dn<K>& a, float s) {
  Dn<K> r; r.v = a.v * s;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] * s;
  return r;
}
template <int K> __device__ __forceinline__ Dn<K> operator/(const Dn<K>& a, const Dn<K>& b) {
  Dn<K> r; r.v = a.v / b.v;
  const float ib = 1.f / b.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
  return r;
}
template <int K> __device__ __forceinline__ Dn<K> dsqrt(const Dn<K>& a) {
  Dn<K> r; r.v = sqrtf(a.v);
  const float h = 0.5f / r.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] * h;
  return r;
}
template <int K> __device__ __forceinline__ void dsincos(const Dn<K>& a, Dn<K>& s, Dn<K>& c) {
  float sv, cv;
  sincosf(a.v, &sv, &cv);
  s.v = sv; c.v = cv;
#pragma unroll
  for (int k = 0; k < K; ++k) { s.d[k] = cv * a.d[k]; c.d[k] = -sv * a.d[k]; }
}
// a + b * c
template <int K> __device__ __forceinline__ Dn<K> dfma(const Dn<K>& b, const Dn<K>& c, const Dn<K>& a) {
  Dn<K> r; r.v = fmaf(b.v, c.v, a.v);
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] + b.d[k] * c.v + b.v * c.d[k];
  return r;
}

template <int K> struct DV3 { Dn<K> x, y, z; };
template <int K> __device__ __forceinline__ DV3<K> dv3(const Dn<K>& x, const Dn<K>& y, const Dn<K>& z) {
  DV3<K> r; r.x = x; r.y = y; r.z = z; return r;
}
template <int K> __device__ __forceinline__ DV3<K> operator+(const DV3<K>& a, const DV3<K>& b) {
  return dv3<K>(a.x + b.x, a.y + b.y, a.z + b.z);
}
template <int K> __device__ __forceinline__ DV3<K> operator-(const DV3<K>& a, const DV3<K>& b) {
  return dv3<K>(a.x - b.x, a.y - b.y, a.z - b.z);
}
template <int K> __device__ __forceinline__ DV3<K> operator*(const DV3<K>& a, const Dn<K>& s) {
  return dv3<K>(a.x * s, a.y * s, a.z * s);
}
template <int K> __device__ __forceinline__ Dn<K> ddot(const DV3<K>& a, const DV3<K>& b) {
  return a.x * b.x + a.y * b.y + a.z * b.z;
}
template <int K> __device__ __forceinline__ DV3<K> dcross(const DV3<K>& a, const DV3<K>& b) {
  return dv3<K>(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
// 3x3 row-major matrix times vector / matrix
template <int K> __device__ __forceinline__ DV3<K> dmv(const Dn<K>* R, const DV3<K>& v) {
  return dv3<K>(R[0] * v.x + R[1] * v.y + R[2] * v.z, R[3] * v.x + R[4] * v.y + R[5] * v.z,
                R[6] * v.x + R[7] * v.y + R[8] * v.z);
}
template <int K> __device__ __forceinline__ void dmm(const Dn<K>* A, const Dn<K>* B, Dn<K>* C) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) C[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
}

// ---- per-lane work space (local memory) --------------------------------------------------------
constexpr int kTanMaxCon = 64;                       // kept contacts per env (ground and pairs)
constexpr int kTanMaxRows = 2 * (kMaxGen + kMaxTendons) + 3 * kTanMaxCon;
constexpr int kTanMaxCache = 448;                    // impulse-cache entries per env

template <int K> struct TanWork {
  Dn<K> R[kMaxLinks][9];     // link -> world rotation
  Dn<K> P[kMaxLinks][3];     // link origin relative to its actor's origin
  Dn<K> V[kMaxLinks][6];     // spatial velocity [w; v] about the actor origin
  Dn<K> Ab[kMaxLinks][6];    // velocity-product (bias) acceleration; later the subtree bias force
  Dn<K> Ic[kMaxLinks][10];   // rigid, then composite inertia about the actor origin: m, h (3), I (6)
  Dn<K> S[kMaxGen][6];       // motion subspace of each generalized DOF
  Dn<K> L[kMaxGen * (kMaxGen + 1) / 2];  // joint-space inertia, then its Cholesky factor (lower, packed)
  Dn<K> nu[kMaxGen], rhs[kMaxGen], z[kMaxGen], dz[kMaxGen];
  Dn<K> cx[kTanMaxCon][3], cd[kTanMaxCon];
  int clink[kTanMaxCon], ccand[kTanMaxCon];
  float cmu[kTanMaxCon];
  int clb[kTanMaxCon];          // body b of a pair contact (its link), -1 for the ground
  Dn<K> cn[kTanMaxCon][3];      // pair contact normal (world, from b to a); the ground's is +z
  Dn<K> lam[kTanMaxRows];
};

// packed lower-triangular index (i >= j)
__device__ __forceinline__ int tri(int i, int j) { return i * (i + 1) / 2 + j; }

template <int K> __device__ __forceinline__ void dquat_to_mat(const Dn<K>* q, Dn<K>* R) {
  const Dn<K> x = q[0], y = q[1], z = q[2], w = q[3];
  const Dn<K> two(2.f), one(1.f);
  R[0] = one - two * (y * y + z * z); R[1] = two * (x * y - z * w); R[2] = two * (x * z + y * w);
  R[3] = two * (x * y + z * w); R[4] = one - two * (x * x + z * z); R[5] = two * (y * z - x * w);
  R[6] = two * (x * z - y * w); R[7] = two * (y * z + x * w); R[8] = one - two * (x * x + y * y);
}

// Quaternion (x, y, z, w) of the rotation vector r (exact exponential).
template <int K> __device__ __forceinline__ void drotvec_quat(const Dn<K>& rx, const Dn<K>& ry, const Dn<K>& rz, Dn<K>* e) {
  const Dn<K> a2 = rx * rx + ry * ry + rz * rz;
  if (a2.v < 1e-30f) {
    e[0] = rx * 0.5f; e[1] = ry * 0.5f; e[2] = rz * 0.5f; e[3] = Dn<K>(1.f);
    return;
  }
  const Dn<K> an = dsqrt(a2);
  Dn<K> sn, cs;
  dsincos<K>(an * 0.5f, sn, cs);
  const Dn<K> sc = sn / an;
  e[0] = rx * sc; e[1] = ry * sc; e[2] = rz * sc; e[3] = cs;
}
// atan2 with its derivative (x dy - y dx) / (x^2 + y^2).
template <int K> __device__ __forceinline__ Dn<K> datan2(const Dn<K>& y, const Dn<K>& x) {
  Dn<K> r(atan2f(y.v, x.v));
  const float id = 1.f / (x.v * x.v + y.v * y.v);
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = (x.v * y.d[k] - y.v * x.d[k]) * id;
  return r;
}
// Rotation vector of the quaternion q (need not be exactly unit): the shorter rotation.
template <int K> __device__ __forceinline__ void dquat_rotvec(const Dn<K>* q, Dn<K>* r) {
  const float sg = q[3].v < 0.f ? -1.f : 1.f;
  const Dn<K> x = q[0] * sg, y = q[1] * sg, z = q[2] * sg, w = q[3] * sg;
  const Dn<K> s2 = x * x + y * y + z * z;
  Dn<K> f;
  if (s2.v < 1e-30f) {
    f = Dn<K>(2.f) / w;
  } else {
    const Dn<K> sn = dsqrt(s2);
    f = datan2<K>(sn, w) * 2.f / sn;
  }
  r[0] = x * f; r[1] = y * f; r[2] = z * f;
}

// Per-env state of the tangent step (per actor: root p, quat, v, w; per joint DOF: q, qd; the env's
// actuation and impulse cache). Arrays are indexed env-locally.
template <int K> struct TanState {
  Dn<K> rp[kMaxActors][3], rq[kMaxActors][4], rv[kMaxActors][3], rw[kMaxActors][3];
  Dn<K> q[kMaxGen], qd[kMaxGen], act[kMaxGen];
  Dn<K> cache[kTanMaxCache];
  float qt[kMaxGen], vt[kMaxGen];  // drive position / velocity targets (constants of the derivative)
  const float* bf = nullptr;       // the env's external body forces (N_B rows of 6) or null (constants)
};

// Kinematics and dynamics of the substep's start state: link poses, velocities, motion subspaces,
// the joint-space inertia M (armature included; packed lower in w.L) and tau - b in w.rhs. With
// drives (a step, not a query: `drives`), each driven DOF adds kp (q* - q - h qd) + kd (v* - qd) to
// tau and h (h kp + kd) to its diagonal of M (the implicit drive of the forward step).
template <int K> __device__ void tangent_dynamics(const StepArgs& A, const EnvTypeTable* T, TanState<K>& s,
                                                  TanWork<K>& w, const bool drives = true) {
  const int L = T->n_links, n = T->n_gen;
  const float gx = A.gx, gy = A.gy, gz = A.gz;
  // ---- forward kinematics, velocities, bias accelerations, rigid inertias (links in order) ----
  for (int l = 0; l < L; ++l) {
    const int par = T->parent[l], jt = T->jtype[l], a = T->actor[l], gd = T->gdof[l], jd = T->jdof[l];
    if (par < 0) {
      dquat_to_mat<K>(s.rq[a], w.R[l]);
#pragma unroll
      for (int k = 0; k < 3; ++k) w.P[l][k] = Dn<K>(0.f);
      if (jt == kFree) {
        for (int k = 0; k < 3; ++k) { w.V[l][k] = s.rw[a][k]; w.V[l][3 + k] = s.rv[a][k]; }
        // d/dt (S_root nu) = [0; p_dot x omega]
        const DV3<K> pxw = dcross(dv3<K>(s.rv[a][0], s.rv[a][1], s.rv[a][2]), dv3<K>(s.rw[a][0], s.rw[a][1], s.rw[a][2]));
        w.Ab[l][0] = Dn<K>(0.f); w.Ab[l][1] = Dn<K>(0.f); w.Ab[l][2] = Dn<K>(0.f);
        w.Ab[l][3] = pxw.x; w.Ab[l][4] = pxw.y; w.Ab[l][5] = pxw.z;
        for (int c = 0; c < 6; ++c)
          for (int k = 0; k < 6; ++k) w.S[gd + c][k] = Dn<K>(c == k ? 1.f : 0.f);
        for (int k = 0; k < 3; ++k) { w.nu[gd + k] = s.rw[a][k]; w.nu[gd + 3 + k] = s.rv[a][k]; }
      } else {
        for (int k = 0; k < 6; ++k) { w.V[l][k] = Dn<K>(0.f); w.Ab[l][k] = Dn<K>(0.f); }
      }
    } else {
      Dn<K> Rpj[9], RB[9];
      for (int k = 0; k < 9; ++k) Rpj[k] = Dn<K>(T->prot[k][l]);
      dmm<K>(w.R[par], Rpj, RB);
      const DV3<K> jax = dv3<K>(Dn<K>(T->axis[0][l]), Dn<K>(T->axis[1][l]), Dn<K>(T->axis[2][l]));
      const DV3<K> pp = dv3<K>(Dn<K>(T->ppos[0][l]), Dn<K>(T->ppos[1][l]), Dn<K>(T->ppos[2][l]));
      const DV3<K> Pp = dv3<K>(w.P[par][0], w.P[par][1], w.P[par][2]);
      const DV3<K> aw = dmv<K>(RB, jax);
      DV3<K> Pl;
      Dn<K> Sa[6];
      for (int k = 0; k < 6; ++k) Sa[k] = Dn<K>(0.f);
      if (jt == kRevolute) {
        // R_J = rotation by q about the joint axis (Rodrigues)
        Dn<K> sn, cs;
        dsincos<K>(s.q[jd], sn, cs);
        const Dn<K> t = Dn<K>(1.f) - cs;
        const float ax = T->axis[0][l], ay = T->axis[1][l], az = T->axis[2][l];
        Dn<K> RJ[9];
        RJ[0] = t * (ax * ax) + cs;      RJ[1] = t * (ax * ay) - sn * az; RJ[2] = t * (ax * az) + sn * ay;
        RJ[3] = t * (ax * ay) + sn * az; RJ[4] = t * (ay * ay) + cs;      RJ[5] = t * (ay * az) - sn * ax;
        RJ[6] = t * (ax * az) - sn * ay; RJ[7] = t * (ay * az) + sn * ax; RJ[8] = t * (az * az) + cs;
        dmm<K>(RB, RJ, w.R[l]);
        Pl = Pp + dmv<K>(w.R[par], pp);
        const DV3<K> pxa = dcross(Pl, aw);
        Sa[0] = aw.x; Sa[1] = aw.y; Sa[2] = aw.z; Sa[3] = pxa.x; Sa[4] = pxa.y; Sa[5] = pxa.z;
      } else if (jt == kPrismatic) {
        for (int k = 0; k < 9; ++k) w.R[l][k] = RB[k];
        Pl = Pp + dmv<K>(w.R[par], pp + dmv<K>(Rpj, jax * s.q[jd]));
        Sa[3] = aw.x; Sa[4] = aw.y; Sa[5] = aw.z;
      } else if (jt == kSpherical) {  // ball joint: R_J = exp([r]x), r = (q[jd], q[jd+1], q[jd+2])
        Dn<K> e[4], RJ[9];
        drotvec_quat<K>(s.q[jd], s.q[jd + 1], s.q[jd + 2], e);
        dquat_to_mat<K>(e, RJ);
        dmm<K>(RB, RJ, w.R[l]);
        Pl = Pp + dmv<K>(w.R[par], pp);
      } else {
        for (int k = 0; k < 9; ++k) w.R[l][k] = RB[k];
        Pl = Pp + dmv<K>(w.R[par], pp);
      }
      w.P[l][0] = Pl.x; w.P[l][1] = Pl.y; w.P[l][2] = Pl.z;
      Dn<K> sq[6];
      const Dn<K> qd = (jd >= 0 && jt != kSpherical) ? s.qd[jd] : Dn<K>(0.f);
      for (int k = 0; k < 6; ++k) sq[k] = Sa[k] * qd;
      if (jt == kSpherical) {
        // the child's axes in world coordinates about the actor origin, one column per DOF
        for (int c = 0; c < 3; ++c) {
          const DV3<K> ax = dv3<K>(w.R[l][c], w.R[l][3 + c], w.R[l][6 + c]);
          const DV3<K> px = dcross(Pl, ax);
          w.S[gd + c][0] = ax.x; w.S[gd + c][1] = ax.y; w.S[gd + c][2] = ax.z;
          w.S[gd + c][3] = px.x; w.S[gd + c][4] = px.y; w.S[gd + c][5] = px.z;
          w.nu[gd + c] = s.qd[jd + c];
          for (int k = 0; k < 6; ++k) sq[k] = sq[k] + w.S[gd + c][k] * s.qd[jd + c];
        }
      }
      for (int k = 0; k < 6; ++k) w.V[l][k] = w.V[par][k] + sq[k];
      // c = v x (S qd); bias acceleration accumulates down the tree
      const DV3<K> wv = dv3<K>(w.V[l][0], w.V[l][1], w.V[l][2]), vl = dv3<K>(w.V[l][3], w.V[l][4], w.V[l][5]);
      const DV3<K> sa = dv3<K>(sq[0], sq[1], sq[2]), sl = dv3<K>(sq[3], sq[4], sq[5]);
      const DV3<K> c0 = dcross(wv, sa), c1 = dcross(wv, sl) + dcross(vl, sa);
      w.Ab[l][0] = w.Ab[par][0] + c0.x; w.Ab[l][1] = w.Ab[par][1] + c0.y; w.Ab[l][2] = w.Ab[par][2] + c0.z;
      w.Ab[l][3] = w.Ab[par][3] + c1.x; w.Ab[l][4] = w.Ab[par][4] + c1.y; w.Ab[l][5] = w.Ab[par][5] + c1.z;
      if (gd >= 0 && jt != kSpherical) {
        for (int k = 0; k < 6; ++k) w.S[gd][k] = Sa[k];
        w.nu[gd] = qd;
      }
    }
    // rigid inertia about the actor origin: I_O = R I_c R^T + m (|c|^2 1 - c c^T), h = m c
    const float m = T->mass[l];
    const DV3<K> cw = dv3<K>(w.P[l][0], w.P[l][1], w.P[l][2]) +
                      dmv<K>(w.R[l], dv3<K>(Dn<K>(T->com[0][l]), Dn<K>(T->com[1][l]), Dn<K>(T->com[2][l])));
    Dn<K> In[9], RI[9], RIRt[9], Rt[9];
    const float ii[9] = {T->inertia[0][l], T->inertia[3][l], T->inertia[4][l], T->inertia[3][l], T->inertia[1][l],
                         T->inertia[5][l], T->inertia[4][l], T->inertia[5][l], T->inertia[2][l]};
    for (int k = 0; k < 9; ++k) In[k] = Dn<K>(ii[k]);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) Rt[3 * i + j] = w.R[l][3 * j + i];
    dmm<K>(w.R[l], In, RI);
    dmm<K>(RI, Rt, RIRt);
    const Dn<K> c2 = ddot(cw, cw);
    w.Ic[l][0] = Dn<K>(m);
    w.Ic[l][1] = cw.x * m; w.Ic[l][2] = cw.y * m; w.Ic[l][3] = cw.z * m;
    w.Ic[l][4] = RIRt[0] + (c2 - cw.x * cw.x) * m;
    w.Ic[l][5] = RIRt[4] + (c2 - cw.y * cw.y) * m;
    w.Ic[l][6] = RIRt[8] + (c2 - cw.z * cw.z) * m;
    w.Ic[l][7] = RIRt[1] - cw.x * cw.y * m;
    w.Ic[l][8] = RIRt[2] - cw.x * cw.z * m;
    w.Ic[l][9] = RIRt[5] - cw.y * cw.z * m;
  }
  // ---- bias forces f = I a_bias + v x* I v - f_gravity (stored in Ab) ----
  for (int l = 0; l < L; ++l) {
    const Dn<K>* I = w.Ic[l];
    const DV3<K> hh = dv3<K>(I[1], I[2], I[3]);
    auto Imul = [&](const Dn<K>* x, DV3<K>& fa, DV3<K>& fl) {
      const DV3<K> xw = dv3<K>(x[0], x[1], x[2]), xv = dv3<K>(x[3], x[4], x[5]);
      const DV3<K> Iw = dv3<K>(I[4] * xw.x + I[7] * xw.y + I[8] * xw.z, I[7] * xw.x + I[5] * xw.y + I[9] * xw.z,
                               I[8] * xw.x + I[9] * xw.y + I[6] * xw.z);
      fa = Iw + dcross(hh, xv);
      fl = xv * I[0] + dcross(xw, hh);
    };
    DV3<K> Fa, Fl, Ga, Gl;
    Imul(w.V[l], Fa, Fl);
    Imul(w.Ab[l], Ga, Gl);
    const DV3<K> wv = dv3<K>(w.V[l][0], w.V[l][1], w.V[l][2]), vl = dv3<K>(w.V[l][3], w.V[l][4], w.V[l][5]);
    const DV3<K> g = dv3<K>(Dn<K>(gx), Dn<K>(gy), Dn<K>(gz));
    DV3<K> pa = Ga + dcross(wv, Fa) + dcross(vl, Fl) - dcross(hh, g);
    DV3<K> pl = Gl + dcross(wv, Fl) - g * I[0];
    if (s.bf && T->body[l] >= 0) {
      // external force F and torque at the COM c (world axes): c x F + torque about the origin
      const float* f = s.bf + (size_t)T->body[l] * 6;
      const DV3<K> cw = dv3<K>(w.P[l][0], w.P[l][1], w.P[l][2]) +
                        dmv<K>(w.R[l], dv3<K>(Dn<K>(T->com[0][l]), Dn<K>(T->com[1][l]), Dn<K>(T->com[2][l])));
      const DV3<K> F = dv3<K>(Dn<K>(f[0]), Dn<K>(f[1]), Dn<K>(f[2]));
      pa = pa - (dcross(cw, F) + dv3<K>(Dn<K>(f[3]), Dn<K>(f[4]), Dn<K>(f[5])));
      pl = pl - F;
    }
    w.Ab[l][0] = pa.x; w.Ab[l][1] = pa.y; w.Ab[l][2] = pa.z; w.Ab[l][3] = pl.x; w.Ab[l][4] = pl.y; w.Ab[l][5] = pl.z;
  }
  // ---- subtree sums (children after parents: sweep links backwards) ----
  for (int l = L - 1; l >= 0; --l) {
    const int par = T->parent[l];
    if (par >= 0) {
      for (int k = 0; k < 6; ++k) w.Ab[par][k] = w.Ab[par][k] + w.Ab[l][k];
      for (int k = 0; k < 10; ++k) w.Ic[par][k] = w.Ic[par][k] + w.Ic[l][k];
    }
  }
  // ---- joint-space inertia M (composite inertias) and bias b = S^T F ----
  for (int i = 0; i < n; ++i) {
    const int li = T->dof_link[i];
    // f = Ic(li) S_i ... M_ij = S_j^T Ic(deeper) S_i for j an ancestor-or-self DOF of i
    const Dn<K>* I = w.Ic[li];
    const DV3<K> hh = dv3<K>(I[1], I[2], I[3]);
    const DV3<K> xw = dv3<K>(w.S[i][0], w.S[i][1], w.S[i][2]), xv = dv3<K>(w.S[i][3], w.S[i][4], w.S[i][5]);
    const DV3<K> Iw = dv3<K>(I[4] * xw.x + I[7] * xw.y + I[8] * xw.z, I[7] * xw.x + I[5] * xw.y + I[9] * xw.z,
                             I[8] * xw.x + I[9] * xw.y + I[6] * xw.z);
    const DV3<K> fa = Iw + dcross(hh, xv), fl = xv * I[0] + dcross(xw, hh);
    const unsigned anc = T->anc[li];
    for (int j = 0; j <= i; ++j) {
      if (!((anc >> j) & 1u)) { w.L[tri(i, j)] = Dn<K>(0.f); continue; }
      w.L[tri(i, j)] = w.S[j][0] * fa.x + w.S[j][1] * fa.y + w.S[j][2] * fa.z + w.S[j][3] * fl.x +
                       w.S[j][4] * fl.y + w.S[j][5] * fl.z;
    }
    Dn<K> bi(0.f);
    for (int k = 0; k < 6; ++k) bi = bi + w.S[i][k] * w.Ab[li][k];
    // joint force of the substep (damping at the substep-start velocity); a floating root has none
    const int comp = T->dof_comp[i];
    Dn<K> tau(0.f);
    if (comp < 0) {
      const int jd = T->jdof[li] + (i - T->gdof[li]);  // the DOF's row (a ball joint has three)
      tau = s.act[jd] - s.qd[jd] * T->damping[li];
      w.L[tri(i, i)] = w.L[tri(i, i)] + Dn<K>(T->armature[li]);
      if (drives && T->has_drives) {
        const float kp = T->drive_kp[li], kd = T->drive_kd[li], h = A.h;
        tau = tau + (Dn<K>(s.qt[jd]) - s.q[jd] - s.qd[jd] * h) * kp + (Dn<K>(s.vt[jd]) - s.qd[jd]) * kd;
        w.L[tri(i, i)] = w.L[tri(i, i)] + Dn<K>(h * (h * kp + kd));
      }
      // fixed tendons: F = -k (l - rest) - d l_dot on the length l = sum c q (substep start),
      // applied to each of the tendon's joints as c F
      for (int t = 0; t < T->n_tendons; ++t) {
        Dn<K> len(0.f), rate(0.f);
        float mine = 0.f;
        for (int k = 0; k < T->ten_n[t]; ++k) {
          const int lk = T->ten_link[t][k], jk = T->jdof[lk];
          const float c = T->ten_coef[t][k];
          len = len + s.q[jk] * c;
          rate = rate + s.qd[jk] * c;
          if (lk == li) mine += c;
        }
        if (mine != 0.f)
          tau = tau + ((len - Dn<K>(T->ten_rest[t])) * (-T->ten_k[t]) - rate * T->ten_d[t]) * mine;
      }
    }
    w.rhs[i] = tau - bi;
  }
}

// ---- capsule-box geometry in dual arithmetic (box frame): the forward step's definitions, every
// branch (inside / outside, breakpoint order, clamps, the face and the friction anchor) taken on the
// value ----
template <int K> __device__ __forceinline__ const Dn<K>& dcomp(const DV3<K>& v, int k) {
  return k == 0 ? v.x : (k == 1 ? v.y : v.z);
}
template <int K> __device__ __forceinline__ Dn<K> dabs(const Dn<K>& a) { return a.v < 0.f ? -a : a; }
template <int K> __device__ Dn<K> dbox_dist2(const DV3<K>& p, const float* e) {
  Dn<K> f(0.f);
  for (int k = 0; k < 3; ++k) {
    const Dn<K> o = dabs(dcomp(p, k)) - Dn<K>(e[k]);
    if (o.v > 0.f) f = f + o * o;
  }
  return f;
}
// minimiser over [0, 1] of the squared distance from p0 + t dv to the box (pieces between the
// breakpoints |p_k(t)| = e_k, each piece's stationary point clamped into it; ties to the smaller t)
template <int K> __device__ Dn<K> dsegment_box_closest_t(const DV3<K>& p0, const DV3<K>& dv, const float* e) {
  Dn<K> ts[8];
  int nt = 0;
  ts[nt++] = Dn<K>(0.f);
  ts[nt++] = Dn<K>(1.f);
  for (int k = 0; k < 3; ++k) {
    const Dn<K>& dk = dcomp(dv, k);
    if (dk.v == 0.f) continue;
    for (int sg = -1; sg <= 1; sg += 2) {
      const Dn<K> t = (Dn<K>((float)sg * e[k]) - dcomp(p0, k)) / dk;
      if (t.v > 0.f && t.v < 1.f) ts[nt++] = t;
    }
  }
  for (int i = 1; i < nt; ++i) {  // insertion sort on the values
    const Dn<K> x = ts[i];
    int j = i - 1;
    while (j >= 0 && x.v < ts[j].v) { ts[j + 1] = ts[j]; --j; }
    ts[j + 1] = x;
  }
  Dn<K> best_t(0.f);
  float best_f = dbox_dist2<K>(p0, e).v;
  for (int i = 0; i + 1 < nt; ++i) {
    const Dn<K> ta = ts[i], tb = ts[i + 1];
    const DV3<K> pm = p0 + dv * ((ta + tb) * 0.5f);
    Dn<K> num(0.f), den(0.f);
    for (int k = 0; k < 3; ++k) {
      const Dn<K>& pk = dcomp(pm, k);
      if (!(e[k] < fabsf(pk.v))) continue;
      const float sg = (pk.v > 0.f) ? 1.f : -1.f;
      const Dn<K>& dk = dcomp(dv, k);
      num = num + dk * (Dn<K>(sg * e[k]) - dcomp(p0, k));
      den = den + dk * dk;
    }
    Dn<K> t = ta;
    if (den.v > 0.f) {
      t = num / den;
      if (t.v < ta.v) t = ta;
      if (t.v > tb.v) t = tb;
    }
    const float f = dbox_dist2<K>(p0 + dv * t, e).v;
    if (f < best_f) { best_f = f; best_t = t; }
  }
  if (dbox_dist2<K>(p0 + dv, e).v < best_f) best_t = Dn<K>(1.f);
  return best_t;
}
// a sphere of radius r at p against the box: normal (box -> sphere), separation, and the point
// halfway between the two surfaces
template <int K> __device__ void dsphere_box(const DV3<K>& p, float r, const float* e, DV3<K>& n, Dn<K>& d,
                                             DV3<K>& x) {
  const bool inside = fabsf(p.x.v) <= e[0] && fabsf(p.y.v) <= e[1] && fabsf(p.z.v) <= e[2];
  if (!inside) {
    Dn<K> q[3];
    for (int k = 0; k < 3; ++k) {
      const Dn<K>& pk = dcomp(p, k);
      q[k] = pk.v > e[k] ? Dn<K>(e[k]) : (pk.v < -e[k] ? Dn<K>(-e[k]) : pk);
    }
    const DV3<K> dl = p - dv3<K>(q[0], q[1], q[2]);
    const Dn<K> dist = dsqrt(ddot(dl, dl));
    n = dv3<K>(dl.x / dist, dl.y / dist, dl.z / dist);
    d = dist - Dn<K>(r);
  } else {
    int kb = 0;
    float best = e[0] - fabsf(p.x.v);
    if (e[1] - fabsf(p.y.v) < best) { best = e[1] - fabsf(p.y.v); kb = 1; }
    if (e[2] - fabsf(p.z.v) < best) { best = e[2] - fabsf(p.z.v); kb = 2; }
    const float sg = (dcomp(p, kb).v < 0.f) ? -1.f : 1.f;
    n = dv3<K>(Dn<K>(kb == 0 ? sg : 0.f), Dn<K>(kb == 1 ? sg : 0.f), Dn<K>(kb == 2 ? sg : 0.f));
    d = -(Dn<K>(e[kb]) - dabs(dcomp(p, kb))) - Dn<K>(r);
  }
  x = p - n * (Dn<K>(r) + d * 0.5f);
}
// the part of the segment over the box face selected by the closest point t*
template <int K> __device__ bool dface_clip(const DV3<K>& p0, const DV3<K>& dv, const float* e, float r,
                                           const Dn<K>& tstar, Dn<K>& ta, Dn<K>& tb) {
  DV3<K> n, x;
  Dn<K> d;
  dsphere_box<K>(p0 + dv * tstar, r, e, n, d, x);
  int kn = 0;
  if (fabsf(n.x.v) < fabsf(n.y.v)) kn = 1;
  if (fabsf(dcomp(n, kn).v) < fabsf(n.z.v)) kn = 2;
  ta = Dn<K>(0.f);
  tb = Dn<K>(1.f);
  for (int j = 0; j < 3; ++j) {
    if (j == kn) continue;
    const Dn<K>& dj = dcomp(dv, j);
    const Dn<K>& pj = dcomp(p0, j);
    if (dj.v == 0.f) {
      if (e[j] < fabsf(pj.v)) return false;
      continue;
    }
    Dn<K> t0 = (Dn<K>(-e[j]) - pj) / dj, t1 = (Dn<K>(e[j]) - pj) / dj;
    if (t1.v < t0.v) { const Dn<K> sw = t0; t0 = t1; t1 = sw; }
    if (t0.v > ta.v) ta = t0;
    if (t1.v < tb.v) tb = t1;
  }
  return !(tb.v < ta.v);
}
// friction directions of a contact normal (anchor e_x, e_y or e_z chosen on the value)
template <int K> __device__ void dtangent_basis(const DV3<K>& n, DV3<K>& t1, DV3<K>& t2) {
  const float ax = fabsf(n.x.v) < 0.57735f ? 1.f : 0.f;
  const float ay = ax == 0.f && fabsf(n.y.v) < 0.57735f ? 1.f : 0.f;
  const float az = (ax == 0.f && ay == 0.f) ? 1.f : 0.f;
  const DV3<K> an = dv3<K>(Dn<K>(ax), Dn<K>(ay), Dn<K>(az));
  const DV3<K> t = an - n * ddot(an, n);
  const Dn<K> tn = dsqrt(ddot(t, t));
  t1 = dv3<K>(t.x / tn, t.y / tn, t.z / tn);
  t2 = dcross(n, t1);
}

// Spatial forces of a pair contact row (direction k: the normal from b to a, or one of its friction
// directions): body a sees f = [x x k; k] about its actor origin, body b -[x_b x k; k] with x_b the
// point about b's actor origin. Out of line: it keeps the pair geometry out of the solver loop.
template <int K> __device__ __noinline__ void pair_row_forces(const EnvTypeTable* T, const TanState<K>& s,
                                                              const TanWork<K>& w, int c, int dir, Dn<K>* fr,
                                                              Dn<K>* fb) {
  const DV3<K> nrm = dv3<K>(w.cn[c][0], w.cn[c][1], w.cn[c][2]);
  DV3<K> k = nrm;
  if (dir != 0) {
    DV3<K> t1, t2;
    dtangent_basis<K>(nrm, t1, t2);
    k = (dir == 1) ? t1 : t2;
  }
  const DV3<K> x = dv3<K>(w.cx[c][0], w.cx[c][1], w.cx[c][2]);
  const int aa = T->actor[w.clink[c]], ab = T->actor[w.clb[c]];
  const DV3<K> dob = dv3<K>(s.rp[ab][0] - s.rp[aa][0], s.rp[ab][1] - s.rp[aa][1], s.rp[ab][2] - s.rp[aa][2]);
  const DV3<K> xk = dcross(x, k), xbk = dcross(x - dob, k);
  fr[0] = xk.x; fr[1] = xk.y; fr[2] = xk.z; fr[3] = k.x; fr[4] = k.y; fr[5] = k.z;
  fb[0] = -xbk.x; fb[1] = -xbk.y; fb[2] = -xbk.z; fb[3] = -k.x; fb[4] = -k.y; fb[5] = -k.z;
}

// Row r's J^T solved through L: y = L^-1 J_r^T (n entries). Row kinds as in the forward kernel:
// limit rows (unit +-1 on one DOF), tendon rows (+-c on the tendon's DOFs), ground contact normal /
// friction rows along e_z, e_x, e_y, and pair contact rows on two bodies along the pair normal and
// its friction directions.
template <int K> __device__ void row_response(const EnvTypeTable* T, const TanState<K>& s, const TanWork<K>& w, int n,
                                              int kind, int gdof, float sgn, int c, int dir, Dn<K>* y) {
  const bool jrow = kind == kRowLimit || kind == kRowTendon;  // rows on joint coordinates
  const bool pair = !jrow && w.clb[c] >= 0;                   // a contact between two bodies
  const unsigned anc = jrow ? 0u : T->anc[w.clink[c]];
  const unsigned ancb = pair ? T->anc[w.clb[c]] : 0u;
  Dn<K> fr[6], fb[6];
  if (pair) {
    pair_row_forces<K>(T, s, w, c, dir, fr, fb);
  } else if (!jrow) {
    // ground: k = e_z (normal), e_x, e_y (friction); f = [x x k; k]
    const Dn<K>& x0 = w.cx[c][0];
    const Dn<K>& x1 = w.cx[c][1];
    const Dn<K>& x2 = w.cx[c][2];
    const Dn<K> zero(0.f);
    if (dir == 0) { fr[0] = x1; fr[1] = -x0; fr[2] = zero; fr[3] = zero; fr[4] = zero; fr[5] = Dn<K>(1.f); }
    else if (dir == 1) { fr[0] = zero; fr[1] = x2; fr[2] = -x1; fr[3] = Dn<K>(1.f); fr[4] = zero; fr[5] = zero; }
    else { fr[0] = -x2; fr[1] = zero; fr[2] = x0; fr[3] = zero; fr[4] = Dn<K>(1.f); fr[5] = zero; }
  }
  for (int i = 0; i < n; ++i) {
    Dn<K> ji(0.f);
    if (kind == kRowLimit) {
      if (i == gdof) ji = Dn<K>(sgn);
    } else if (kind == kRowTendon) {  // gdof holds the tendon: J = +-c over its joints
      float jt = 0.f;
      for (int k = 0; k < T->ten_n[gdof]; ++k)
        if (T->gdof[T->ten_link[gdof][k]] == i) jt += sgn * T->ten_coef[gdof][k];
      ji = Dn<K>(jt);
    } else {
      if ((anc >> i) & 1u) {
#pragma unroll
        for (int k = 0; k < 6; ++k) ji = ji + w.S[i][k] * fr[k];
      }
      if ((ancb >> i) & 1u) {
#pragma unroll
        for (int k = 0; k < 6; ++k) ji = ji + w.S[i][k] * fb[k];
      }
    }
    for (int k = 0; k < i; ++k) ji = ji - w.L[tri(i, k)] * y[k];
    y[i] = ji / w.L[tri(i, i)];
  }
}

// Capsule-box pair contacts appended after the nc ground contacts in pair / slot order (everything
// relative to the box actor's origin; the stored point relative to body a's actor origin); returns
// the new count, or -1 past kTanMaxCon. Out of line: it runs once per substep.
template <int K> __device__ __noinline__ int tangent_pair_contacts(const StepArgs& A, const EnvTypeTable* T,
                                                                   const TanState<K>& s, TanWork<K>& w, int nc) {
  const float coff = A.contact_offset;
  for (int p = 0; p < T->n_pairs; ++p) {
    const int sa = T->pair_a[p], sb = T->pair_b[p];
    const bool a_cap = T->shape_type[sa] == kCapsule;
    const int sc = a_cap ? sa : sb, sx = a_cap ? sb : sa;
    const int lc = T->shape_link[sc], lx = T->shape_link[sx];
    const int ac = T->actor[lc], axr = T->actor[lx];
    const DV3<K> Oc = dv3<K>(s.rp[ac][0], s.rp[ac][1], s.rp[ac][2]);
    const DV3<K> Ox = dv3<K>(s.rp[axr][0], s.rp[axr][1], s.rp[axr][2]);
    Dn<K> Rsh[9], Rcs[9], Rb[9];
    for (int k = 0; k < 9; ++k) Rsh[k] = Dn<K>(T->shape_rot[k][sc]);
    dmm<K>(w.R[lc], Rsh, Rcs);
    for (int k = 0; k < 9; ++k) Rsh[k] = Dn<K>(T->shape_rot[k][sx]);
    dmm<K>(w.R[lx], Rsh, Rb);
    const DV3<K> cc = dv3<K>(w.P[lc][0], w.P[lc][1], w.P[lc][2]) +
                      dmv<K>(w.R[lc], dv3<K>(Dn<K>(T->shape_pos[0][sc]), Dn<K>(T->shape_pos[1][sc]),
                                             Dn<K>(T->shape_pos[2][sc]))) + (Oc - Ox);
    const DV3<K> cb = dv3<K>(w.P[lx][0], w.P[lx][1], w.P[lx][2]) +
                      dmv<K>(w.R[lx], dv3<K>(Dn<K>(T->shape_pos[0][sx]), Dn<K>(T->shape_pos[1][sx]),
                                             Dn<K>(T->shape_pos[2][sx])));
    const float r = T->shape_size[0][sc], hl = T->shape_size[1][sc];
    const float e[3] = {T->shape_size[0][sx], T->shape_size[1][sx], T->shape_size[2][sx]};
    const DV3<K> ax = dv3<K>(Rcs[0], Rcs[3], Rcs[6]);
    const DV3<K> b0 = dv3<K>(Rb[0], Rb[3], Rb[6]), b1 = dv3<K>(Rb[1], Rb[4], Rb[7]), b2 = dv3<K>(Rb[2], Rb[5], Rb[8]);
    const DV3<K> w0 = cc - ax * Dn<K>(hl) - cb, w1 = cc + ax * Dn<K>(hl) - cb;
    const DV3<K> p0 = dv3<K>(ddot(b0, w0), ddot(b1, w0), ddot(b2, w0));
    const DV3<K> dv = dv3<K>(ddot(b0, w1), ddot(b1, w1), ddot(b2, w1)) - p0;
    const Dn<K> tstar = dsegment_box_closest_t<K>(p0, dv, e);
    Dn<K> ta, tb;
    const bool clip = dface_clip<K>(p0, dv, e, r, tstar, ta, tb);
    const DV3<K> Oa = a_cap ? Oc : Ox;
    for (int slot = 0; slot < kPairSlots; ++slot) {
      const Dn<K> t = slot == 0 ? Dn<K>(0.f) : (slot == 1 ? Dn<K>(1.f) : (slot == 2 ? ta : (slot == 3 ? tb : tstar)));
      if (slot >= 2) {
        if (slot < 4 && !clip) continue;
        if (slot == 3 && !(ta.v < tb.v)) continue;
        if (!(t.v > 0.f && t.v < 1.f)) continue;
      }
      DV3<K> pn, px;
      Dn<K> pd;
      dsphere_box<K>(p0 + dv * t, r, e, pn, pd, px);
      if (!(pd.v < coff)) continue;
      if (nc >= kTanMaxCon) return -1;
      DV3<K> nw = b0 * pn.x + b1 * pn.y + b2 * pn.z;  // box -> capsule
      if (!a_cap) nw = dv3<K>(-nw.x, -nw.y, -nw.z);
      const DV3<K> xw = cb + b0 * px.x + b1 * px.y + b2 * px.z + (Ox - Oa);
      w.cx[nc][0] = xw.x; w.cx[nc][1] = xw.y; w.cx[nc][2] = xw.z;
      w.cn[nc][0] = nw.x; w.cn[nc][1] = nw.y; w.cn[nc][2] = nw.z;
      w.cd[nc] = pd;
      w.clink[nc] = a_cap ? lc : lx;
      w.clb[nc] = a_cap ? lx : lc;
      w.ccand[nc] = T->n_ground_cand + kPairSlots * p + slot;
      w.cmu[nc] = fmaxf(T->shape_fr[sa], T->shape_fr[sb]);
      ++nc;
    }
  }
  return nc;
}

// Contacts of the current poses (w.R, w.P): ground contacts in shape / slot order, then capsule-box
// pair contacts, into w.cx, w.cd, w.clink, w.ccand, w.cmu, w.clb (and w.cn for pairs); returns their
// count, or -1 past kTanMaxCon.
template <int K> __device__ int tangent_contacts(const StepArgs& A, const EnvTypeTable* T, const TanState<K>& s,
                                                 TanWork<K>& w) {
  const float coff = A.contact_offset;
  int nc = 0;
  for (int sh = 0; sh < T->n_shapes; ++sh) {
    const int l = T->shape_link[sh], st = T->shape_type[sh], a = T->actor[l];
    Dn<K> Rsh[9], Rs[9];
    for (int k = 0; k < 9; ++k) Rsh[k] = Dn<K>(T->shape_rot[k][sh]);
    dmm<K>(w.R[l], Rsh, Rs);
    const DV3<K> cs = dv3<K>(w.P[l][0], w.P[l][1], w.P[l][2]) +
                      dmv<K>(w.R[l], dv3<K>(Dn<K>(T->shape_pos[0][sh]), Dn<K>(T->shape_pos[1][sh]), Dn<K>(T->shape_pos[2][sh])));
    const Dn<K> oz = s.rp[a][2];
    const float s0 = T->shape_size[0][sh], s1 = T->shape_size[1][sh], s2 = T->shape_size[2][sh];
    const int nk = (st == kSphere) ? 1 : (st == kCapsule ? 2 : 8);
    for (int k = 0; k < nk; ++k) {
      DV3<K> x;
      Dn<K> zc;
      if (st == kSphere) {
        x = dv3<K>(cs.x, cs.y, cs.z - Dn<K>(s0));
        zc = (oz + cs.z) - Dn<K>(s0);
      } else if (st == kCapsule) {
        const DV3<K> ax = dv3<K>(Rs[0], Rs[3], Rs[6]);
        const DV3<K> e = (k == 0) ? cs - ax * Dn<K>(s1) : cs + ax * Dn<K>(s1);
        x = dv3<K>(e.x, e.y, e.z - Dn<K>(s0));
        zc = (oz + e.z) - Dn<K>(s0);
      } else {
        const DV3<K> loc = dv3<K>(Dn<K>((k & 4) ? s0 : -s0), Dn<K>((k & 2) ? s1 : -s1), Dn<K>((k & 1) ? s2 : -s2));
        x = cs + dmv<K>(Rs, loc);
        zc = oz + x.z;
      }
      if (zc.v < coff) {
        if (nc >= kTanMaxCon) return -1;
        w.cx[nc][0] = x.x; w.cx[nc][1] = x.y; w.cx[nc][2] = x.z;
        w.cd[nc] = zc;
        w.clink[nc] = l;
        w.ccand[nc] = T->cand_off[sh] + k;
        w.cmu[nc] = T->shape_mu[sh];
        w.clb[nc] = -1;
        ++nc;
      }
    }
  }
  return T->n_pairs > 0 ? tangent_pair_contacts<K>(A, T, s, w, nc) : nc;
}

// Link poses only (w.R, w.P), as in tangent_dynamics.
template <int K> __device__ void tangent_poses(const EnvTypeTable* T, const TanState<K>& s, TanWork<K>& w) {
  for (int l = 0; l < T->n_links; ++l) {
    const int par = T->parent[l], jt = T->jtype[l], jd = T->jdof[l];
    if (par < 0) {
      dquat_to_mat<K>(s.rq[T->actor[l]], w.R[l]);
      for (int k = 0; k < 3; ++k) w.P[l][k] = Dn<K>(0.f);
      continue;
    }
    Dn<K> Rpj[9], RB[9];
    for (int k = 0; k < 9; ++k) Rpj[k] = Dn<K>(T->prot[k][l]);
    dmm<K>(w.R[par], Rpj, RB);
    const DV3<K> jax = dv3<K>(Dn<K>(T->axis[0][l]), Dn<K>(T->axis[1][l]), Dn<K>(T->axis[2][l]));
    const DV3<K> pp = dv3<K>(Dn<K>(T->ppos[0][l]), Dn<K>(T->ppos[1][l]), Dn<K>(T->ppos[2][l]));
    const DV3<K> Pp = dv3<K>(w.P[par][0], w.P[par][1], w.P[par][2]);
    DV3<K> Pl;
    if (jt == kRevolute) {
      Dn<K> sn, cs;
      dsincos<K>(s.q[jd], sn, cs);
      const Dn<K> t = Dn<K>(1.f) - cs;
      const float ax = T->axis[0][l], ay = T->axis[1][l], az = T->axis[2][l];
      Dn<K> RJ[9];
      RJ[0] = t * (ax * ax) + cs;      RJ[1] = t * (ax * ay) - sn * az; RJ[2] = t * (ax * az) + sn * ay;
      RJ[3] = t * (ax * ay) + sn * az; RJ[4] = t * (ay * ay) + cs;      RJ[5] = t * (ay * az) - sn * ax;
      RJ[6] = t * (ax * az) - sn * ay; RJ[7] = t * (ay * az) + sn * ax; RJ[8] = t * (az * az) + cs;
      dmm<K>(RB, RJ, w.R[l]);
      Pl = Pp + dmv<K>(w.R[par], pp);
    } else if (jt == kPrismatic) {
      for (int k = 0; k < 9; ++k) w.R[l][k] = RB[k];
      Pl = Pp + dmv<K>(w.R[par], pp + dmv<K>(Rpj, jax * s.q[jd]));
    } else if (jt == kSpherical) {
      Dn<K> e[4], RJ[9];
      drotvec_quat<K>(s.q[jd], s.q[jd + 1], s.q[jd + 2], e);
      dquat_to_mat<K>(e, RJ);
      dmm<K>(RB, RJ, w.R[l]);
      Pl = Pp + dmv<K>(w.R[par], pp);
    } else {
      for (int k = 0; k < 9; ++k) w.R[l][k] = RB[k];
      Pl = Pp + dmv<K>(w.R[par], pp);
    }
    w.P[l][0] = Pl.x; w.P[l][1] = Pl.y; w.P[l][2] = Pl.z;
  }
}

// Impulse-cache slots the step's first substep reads (the warm start of each of its constraint
// rows: joint limits, then contacts' normal and friction rows), into slots[]; returns their count,
// or -1 past the capacities.
template <int K> __device__ int read_slots(const StepArgs& A, const EnvTypeTable* T, const TanState<K>& s,
                                           TanWork<K>& w, int* slots) {
  tangent_poses<K>(T, s, w);
  const int nc = tangent_contacts<K>(A, T, s, w);
  if (nc < 0) return -1;
  int m = 0;
  for (int l = 0; l < T->n_links; ++l) {
    const int jt = T->jtype[l];
    if (T->parent[l] < 0 || !(jt == kRevolute || jt == kPrismatic) || !T->has_limit[l]) continue;
    const int jd = T->jdof[l];
    if (s.q[jd].v - T->lo[l] < A.limit_margin) slots[m++] = 3 * T->n_cand + 2 * jd;
    if (T->hi[l] - s.q[jd].v < A.limit_margin) slots[m++] = 3 * T->n_cand + 2 * jd + 1;
  }
  for (int t = 0; t < T->n_tendons; ++t) {
    if (!T->ten_has_limit[t]) continue;
    float tl = 0.f;
    for (int k = 0; k < T->ten_n[t]; ++k) tl += T->ten_coef[t][k] * s.q[T->jdof[T->ten_link[t][k]]].v;
    const int slot0 = 3 * T->n_cand + 2 * T->n_jdof + 2 * t;
    if (tl - T->ten_lo[t] < A.limit_margin) slots[m++] = slot0;
    if (T->ten_hi[t] - tl < A.limit_margin) slots[m++] = slot0 + 1;
  }
  for (int c = 0; c < nc; ++c)
    for (int d = 0; d < 3; ++d) slots[m++] = 3 * w.ccand[c] + d;
  return m;
}

// One substep in dual arithmetic. Returns false if a pivot or a capacity check fails.
template <int K> __device__ bool tangent_substep(const StepArgs& A, const EnvTypeTable* T, TanState<K>& s,
                                                 TanWork<K>& w) {
  tangent_dynamics<K>(A, T, s, w);
  const int L = T->n_links, n = T->n_gen;
  const float h = A.h;
  const int npos = A.pos_iters, nvel = A.vel_iters;
  const float hit = h / (float)npos;
  // ---- Cholesky M = L L^T (in place, packed lower) ----
  for (int j = 0; j < n; ++j) {
    Dn<K> djj = w.L[tri(j, j)];
    for (int k = 0; k < j; ++k) djj = djj - w.L[tri(j, k)] * w.L[tri(j, k)];
    if (!(djj.v > 0.f)) return false;
    const Dn<K> ljj = dsqrt(djj);
    w.L[tri(j, j)] = ljj;
    for (int i = j + 1; i < n; ++i) {
      Dn<K> x = w.L[tri(i, j)];
      for (int k = 0; k < j; ++k) x = x - w.L[tri(i, k)] * w.L[tri(j, k)];
      w.L[tri(i, j)] = x / ljj;
    }
  }
  // qdd = M^-1 (tau - b): y = L^-1 rhs, then v_free = nu + h L^-T y; z = L^T v_free = L^T nu + h y
  for (int i = 0; i < n; ++i) {
    Dn<K> x = w.rhs[i];
    for (int k = 0; k < i; ++k) x = x - w.L[tri(i, k)] * w.rhs[k];
    w.rhs[i] = x / w.L[tri(i, i)];
  }
  for (int i = 0; i < n; ++i) {
    Dn<K> x(0.f);
    for (int k = i; k < n; ++k) x = x + w.L[tri(k, i)] * w.nu[k];
    w.z[i] = x + w.rhs[i] * h;
    w.dz[i] = Dn<K>(0.f);
  }
  const int nc = tangent_contacts<K>(A, T, s, w);
  if (nc < 0) return false;
  // ---- rows: joint limits (link order, lower before upper), tendon limits (tendon order), normals,
  // friction pairs. Row r is described on the fly: r < nl: limit list; then contact normals; then
  // frictions. A tendon row keeps its tendon in lim_g and -1 - slot offset in lim_jd.
  int lim_g[2 * (kMaxGen + kMaxTendons)], lim_side[2 * (kMaxGen + kMaxTendons)], lim_jd[2 * (kMaxGen + kMaxTendons)];
  Dn<K> lim_d[2 * (kMaxGen + kMaxTendons)];
  int nl = 0;
  for (int l = 0; l < L; ++l) {
    const int jt = T->jtype[l];
    if (T->parent[l] < 0 || !(jt == kRevolute || jt == kPrismatic) || !T->has_limit[l]) continue;
    const int jd = T->jdof[l];
    const Dn<K> dlo = s.q[jd] - Dn<K>(T->lo[l]), dhi = Dn<K>(T->hi[l]) - s.q[jd];
    if (dlo.v < A.limit_margin) { lim_g[nl] = T->gdof[l]; lim_side[nl] = 0; lim_jd[nl] = jd; lim_d[nl] = dlo; ++nl; }
    if (dhi.v < A.limit_margin) { lim_g[nl] = T->gdof[l]; lim_side[nl] = 1; lim_jd[nl] = jd; lim_d[nl] = dhi; ++nl; }
  }
  for (int t = 0; t < T->n_tendons; ++t) {
    if (!T->ten_has_limit[t]) continue;
    Dn<K> tl(0.f);
    for (int k = 0; k < T->ten_n[t]; ++k) tl = tl + s.q[T->jdof[T->ten_link[t][k]]] * T->ten_coef[t][k];
    const Dn<K> dlo = tl - Dn<K>(T->ten_lo[t]), dhi = Dn<K>(T->ten_hi[t]) - tl;
    if (dlo.v < A.limit_margin) { lim_g[nl] = t; lim_side[nl] = 0; lim_jd[nl] = -1; lim_d[nl] = dlo; ++nl; }
    if (dhi.v < A.limit_margin) { lim_g[nl] = t; lim_side[nl] = 1; lim_jd[nl] = -1; lim_d[nl] = dhi; ++nl; }
  }
  const int R = nl + 3 * nc;
  if (R > kTanMaxRows) return false;
  Dn<K> y[kMaxGen];
  auto describe = [&](int r, int& kind, int& g, float& sgn, int& c, int& dir, int& slot) {
    if (r < nl) {
      kind = lim_jd[r] >= 0 ? kRowLimit : kRowTendon; g = lim_g[r]; sgn = lim_side[r] ? -1.f : 1.f; c = 0; dir = 0;
      slot = 3 * T->n_cand + 2 * (lim_jd[r] >= 0 ? lim_jd[r] : T->n_jdof + lim_g[r]) + lim_side[r];
    } else if (r < nl + nc) {
      kind = kRowNormal; c = r - nl; dir = 0; g = 0; sgn = 0.f; slot = 3 * w.ccand[c];
    } else {
      kind = kRowFriction; c = (r - nl - nc) >> 1; dir = 1 + ((r - nl - nc) & 1); g = 0; sgn = 0.f;
      slot = 3 * w.ccand[c] + dir;
    }
  };
  // warm start from the cache
  for (int r = 0; r < R; ++r) {
    int kind, g, c, dir, slot;
    float sgn;
    describe(r, kind, g, sgn, c, dir, slot);
    row_response<K>(T, s, w, n, kind, g, sgn, c, dir, y);
    Dn<K> a2(0.f);
    for (int i = 0; i < n; ++i) a2 = a2 + y[i] * y[i];
    w.lam[r] = (a2.v > 1e-12f) ? s.cache[slot] : Dn<K>(0.f);
    for (int i = 0; i < n; ++i) w.z[i] = w.z[i] + y[i] * w.lam[r];
  }
  // ---- projected Gauss-Seidel in z = L^T v ----
  const float beta = A.bias_coef, vmax = A.max_depen_vel;
  for (int it = 0; it < npos + nvel; ++it) {
    const bool pos = it < npos;
    for (int r = 0; r < R; ++r) {
      int kind, g, c, dir, slot;
      float sgn;
      describe(r, kind, g, sgn, c, dir, slot);
      row_response<K>(T, s, w, n, kind, g, sgn, c, dir, y);
      Dn<K> a2(0.f), yz(0.f), ydz(0.f);
      for (int i = 0; i < n; ++i) { a2 = a2 + y[i] * y[i]; yz = yz + y[i] * w.z[i]; ydz = ydz + y[i] * w.dz[i]; }
      if (!(a2.v > 1e-12f)) continue;
      const Dn<K> dr = (kind == kRowLimit || kind == kRowTendon) ? lim_d[r] : w.cd[c];
      const Dn<K> sep = dr + ydz;
      const Dn<K> lam = w.lam[r];
      Dn<K> lnew;
      if (kind == kRowFriction) {
        const Dn<K> lim = w.lam[nl + c] * w.cmu[c];
        lnew = lam - yz / a2;
        if (lnew.v > lim.v) lnew = lim;
        if (lnew.v < -lim.v) lnew = -lim;
      } else {
        Dn<K> target(0.f);
        if (pos) {
          if (sep.v >= 0.f) target = -sep * (1.f / hit);
          else {
            target = -sep * (beta / hit);
            if (target.v > vmax) target = Dn<K>(vmax);
          }
        } else if (sep.v > 0.f) {
          target = -sep * (1.f / h);
        }
        lnew = lam + (target - yz) / a2;
        if (lnew.v < 0.f) lnew = Dn<K>(0.f);
      }
      const Dn<K> dl = lnew - lam;
      for (int i = 0; i < n; ++i) w.z[i] = w.z[i] + y[i] * dl;
      w.lam[r] = lnew;
    }
    if (pos)
      for (int i = 0; i < n; ++i) w.dz[i] = w.dz[i] + w.z[i] * hit;
  }
  // v = L^-T z, dq = L^-T dz (overwrite z, dz)
  for (int i = n - 1; i >= 0; --i) {
    Dn<K> a = w.z[i], b = w.dz[i];
    for (int k = i + 1; k < n; ++k) { a = a - w.L[tri(k, i)] * w.z[k]; b = b - w.L[tri(k, i)] * w.dz[k]; }
    w.z[i] = a / w.L[tri(i, i)];
    w.dz[i] = b / w.L[tri(i, i)];
  }
  // ---- impulse cache: cleared, then every row's impulse at its slot ----
  for (int i = 0; i < T->cache_len; ++i) s.cache[i] = Dn<K>(0.f);
  for (int r = 0; r < R; ++r) {
    int kind, g, c, dir, slot;
    float sgn;
    describe(r, kind, g, sgn, c, dir, slot);
    s.cache[slot] = w.lam[r];
  }
  // ---- integrate ----
  for (int l = 0; l < L; ++l) {
    const int gd = T->gdof[l], jd = T->jdof[l], a = T->actor[l];
    if (T->parent[l] >= 0 && T->jtype[l] == kSpherical) {
      // R_J <- R_J exp([dq]x), back to the shorter rotation vector
      Dn<K> e1[4], e2[4], qn[4];
      drotvec_quat<K>(s.q[jd], s.q[jd + 1], s.q[jd + 2], e1);
      drotvec_quat<K>(w.dz[gd], w.dz[gd + 1], w.dz[gd + 2], e2);
      qn[0] = e1[3] * e2[0] + e1[0] * e2[3] + e1[1] * e2[2] - e1[2] * e2[1];
      qn[1] = e1[3] * e2[1] - e1[0] * e2[2] + e1[1] * e2[3] + e1[2] * e2[0];
      qn[2] = e1[3] * e2[2] + e1[0] * e2[1] - e1[1] * e2[0] + e1[2] * e2[3];
      qn[3] = e1[3] * e2[3] - e1[0] * e2[0] - e1[1] * e2[1] - e1[2] * e2[2];
      Dn<K> r[3];
      dquat_rotvec<K>(qn, r);
      for (int c = 0; c < 3; ++c) { s.q[jd + c] = r[c]; s.qd[jd + c] = w.z[gd + c]; }
    } else if (T->parent[l] >= 0) {
      if (jd >= 0) { s.q[jd] = s.q[jd] + w.dz[gd]; s.qd[jd] = w.z[gd]; }
    } else if (T->jtype[l] == kFree) {
      for (int k = 0; k < 3; ++k) {
        s.rp[a][k] = s.rp[a][k] + w.dz[gd + 3 + k];
        s.rw[a][k] = w.z[gd + k];
        s.rv[a][k] = w.z[gd + 3 + k];
      }
      // quat <- exp(da) * quat (exact exponential), normalised
      const DV3<K> da = dv3<K>(w.dz[gd], w.dz[gd + 1], w.dz[gd + 2]);
      const Dn<K> a2 = ddot(da, da);
      Dn<K> e[4];
      if (a2.v < 1e-30f) {
        e[0] = da.x * 0.5f; e[1] = da.y * 0.5f; e[2] = da.z * 0.5f; e[3] = Dn<K>(1.f);
      } else {
        const Dn<K> an = dsqrt(a2);
        Dn<K> sn, cs;
        dsincos<K>(an * 0.5f, sn, cs);
        const Dn<K> sc = sn / an;
        e[0] = da.x * sc; e[1] = da.y * sc; e[2] = da.z * sc; e[3] = cs;
      }
      const Dn<K>* q = s.rq[a];
      const Dn<K> x = e[3] * q[0] + e[0] * q[3] + e[1] * q[2] - e[2] * q[1];
      const Dn<K> yq = e[3] * q[1] - e[0] * q[2] + e[1] * q[3] + e[2] * q[0];
      const Dn<K> zq = e[3] * q[2] + e[0] * q[1] - e[1] * q[0] + e[2] * q[3];
      const Dn<K> wq = e[3] * q[3] - e[0] * q[0] - e[1] * q[1] - e[2] * q[2];
      const Dn<K> nr = dsqrt(x * x + yq * yq + zq * zq + wq * wq);
      s.rq[a][0] = x / nr; s.rq[a][1] = yq / nr; s.rq[a][2] = zq / nr; s.rq[a][3] = wq / nr;
    }
  }
  return true;
}

}  // namespace artsim
