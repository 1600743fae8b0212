// Test infrastructure only: the FP64 CPU oracle of the batched articulated-body physics step
// (Isaac Gym, arXiv 2108.10470: reduced-coordinate articulations, Sec. "Physics Simulation"; TGS
// solver, same section; tensor layout, Tables "Physics state tensors" / "Physics control tensors").
// Only tests, the smoke check and the benchmark's CPU-baseline leg may load this library; the
// CUDA product path shares no code with it.
//
// The paper gives no equations for the step, so the oracle executes the textbook algorithms named
// below, in the order and notation of their sources:
//   * forward kinematics and spatial inertias: Featherstone RBDA (2008) ch. 2-4;
//   * forward dynamics: articulated-body algorithm, RBDA Table 7.1, gravity applied as an external
//     force on every link, multi-DOF (free) root handled by the general joint formulas;
//   * joint-space inertia: composite-rigid-body algorithm, RBDA Table 6.2;
//   * inverse dynamics (for pins only): recursive Newton-Euler, RBDA Table 5.1;
//   * contacts, constraint rows and the TGS-style projected Gauss-Seidel solve: the paper's TGS
//     paragraph (velocities accumulated, scaled by dt/N, into a delta buffer that is projected onto
//     the constraint Jacobians and added to the bias), with every unstated detail fixed by an
//     explicit reading (contact offset, tangent choice, row order, bias formula) documented beside
//     the code that applies it.
// Generalized velocity of a free root: nu = [omega; v] in world axes, v being the velocity of the
// root origin. At any instant nu equals the world-axis spatial velocity about the point that
// coincides with the root origin, so the root motion subspace in link coordinates is
// S0 = rot(R0^T); its rate, however, is [omega_dot; a_lin + omega x v] where a is the spatial
// acceleration about that (fixed) point, which is what the ABA returns.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <thread>

#include "oracle_math.hpp"
#include "oracle_dual.hpp"
#include "oracle_opcount.hpp"

namespace orc {

enum { JOINT_FREE = 0, JOINT_FIXED = 1, JOINT_REVOLUTE = 2, JOINT_PRISMATIC = 3, JOINT_SPHERICAL = 4 };
enum { SHAPE_SPHERE = 0, SHAPE_CAPSULE = 1, SHAPE_BOX = 2 };
enum { ROW_LIMIT = 0, ROW_NORMAL = 1, ROW_FRICTION = 2 };

struct LinkD {
  int parent, jtype;
  double axis[3], ppos[3], pquat[4];
  double mass, com[3], inertia[6];
  double armature, damping, lo, hi;
  int has_limit, is_virtual;
  double kp = 0.0, kd = 0.0;  // joint drive stiffness and damping
};
struct ShapeD {
  int link, type;
  double size[3], pos[3], quat[4], friction;
};
// Fixed tendon: length l = sum_k coef_k q_{link_k} over 1-DOF joints of one articulation; a spring
// -damper on the length and optional length limits.
struct TendonD {
  std::vector<int> links;     // model-local link of each joint
  std::vector<double> coef;
  double stiffness = 0.0, damping = 0.0, rest = 0.0, lo = 0.0, hi = 0.0;
  int has_limit = 0;
};
struct ModelD {
  std::vector<LinkD> links;
  std::vector<ShapeD> shapes;
  std::vector<TendonD> tendons;
  std::vector<int> ndof;   // DOFs of each link's joint (0, 1, 3 for a ball joint, or 6)
  std::vector<int> goff;   // offset of each link's DOFs in the model's generalized vector
  std::vector<int> jdof;   // first joint-DOF index (DOF state tensor row within the model) or -1
  int n_gen = 0, n_jdof = 0, n_body = 0, contact_cap = 0;
  bool free_root = false;
};
struct Params {
  double gravity[3];
  int pos_iters, vel_iters;
  double contact_offset, limit_margin, bias_coef, max_depen_vel, ground_friction;
};

struct Oracle {
  std::vector<ModelD> models;
  std::vector<std::vector<int>> env_actors;  // per env: model index of each actor (padding dropped)
  std::vector<int64_t> actor_off;           // per env: first row of its actors in the root tensor
  std::vector<std::vector<std::pair<int, int>>> env_pairs;  // per env: shape-shape candidate pairs
  int n_envs = 0;
  Params prm;
  // per env prefix offsets into the global tensors
  std::vector<int64_t> jdof_off, body_off;
  std::vector<int> n_gen, contact_cap;
  int64_t N_A = 0, N_D = 0, N_B = 0;
  int max_contact_cap = 0, max_gen = 0;
  int cache_len = 0;  // per env: 3 * contact candidates + 2 * joint DOFs + 2 * tendons (max over envs)
  const ModelD& actor_model(int env, int a) const { return models[env_actors[env][a]]; }
  int n_act(int env) const { return (int)env_actors[env].size(); }
};

// ------------------------------------------------------------------------------------------------
// Per-actor state and kinematics.
template <class T> struct ActorState {
  Vec3<T> p;
  T quat[4];
  Vec3<T> w, v;  // world angular velocity, world velocity of the root origin
  std::vector<T> q, qd;
};

template <class T> struct ActorKin {
  std::vector<SMat<T>> Xup;           // i_X_parent(i)
  std::vector<Mat3<T>> R;             // link -> world rotation
  std::vector<Vec3<T>> p;             // link origin in world
  std::vector<std::vector<SVec<T>>> S;  // motion subspace columns, link coordinates
  std::vector<SMat<T>> I;             // spatial inertia, link coordinates
  std::vector<SVec<T>> v, c;          // link velocity and velocity-product acceleration
};

template <class T> Vec3<T> vec3_of(const double* a) { return mk3<T>(T(a[0]), T(a[1]), T(a[2])); }

template <class T> Mat3<T> inertia_matrix(const double* in6) {  // xx, yy, zz, xy, xz, yz
  Mat3<T> m;
  m(0, 0) = T(in6[0]); m(1, 1) = T(in6[1]); m(2, 2) = T(in6[2]);
  m(0, 1) = m(1, 0) = T(in6[3]);
  m(0, 2) = m(2, 0) = T(in6[4]);
  m(1, 2) = m(2, 1) = T(in6[5]);
  return m;
}

// The model's generalized velocity: [omega; v] of a free root followed by the joint rates.
template <class T> std::vector<T> gen_velocity(const ModelD& M, const ActorState<T>& s) {
  std::vector<T> g(M.n_gen, T(0.0));
  if (M.free_root)
    for (int k = 0; k < 3; ++k) { g[k] = s.w[k]; g[3 + k] = s.v[k]; }
  for (size_t i = 0; i < M.links.size(); ++i)
    if (M.jdof[i] >= 0)
      for (int k = 0; k < M.ndof[i]; ++k) g[M.goff[i] + k] = s.qd[M.jdof[i] + k];
  return g;
}

// Forward kinematics, motion subspaces, spatial inertias and velocities (RBDA ch. 4, Table 7.1
// first pass). gv is the model's generalized velocity.
template <class T> void kinematics(const ModelD& M, const ActorState<T>& s, const std::vector<T>& gv, ActorKin<T>& K) {
  const int L = (int)M.links.size();
  K.Xup.assign(L, szeroM<T>());
  K.R.resize(L); K.p.resize(L); K.S.assign(L, {}); K.I.resize(L); K.v.resize(L); K.c.resize(L);
  for (int i = 0; i < L; ++i) {
    const LinkD& lk = M.links[i];
    const Vec3<T> com = vec3_of<T>(lk.com);
    K.I[i] = mcI<T>(T(lk.mass), com, inertia_matrix<T>(lk.inertia));
    if (i == 0) {
      K.R[0] = quat_to_mat<T>(s.quat);
      K.p[0] = s.p;
      if (lk.jtype == JOINT_FREE) {
        // S0 = rot(R0^T): columns map world-axis [omega; v at root origin] to link coordinates.
        const SMat<T> S0 = plux<T>(transpose(K.R[0]), zero3<T>());
        for (int k = 0; k < 6; ++k) {
          SVec<T> col;
          for (int r = 0; r < 6; ++r) col[r] = S0(r, k);
          K.S[0].push_back(col);
        }
      }
      continue;
    }
    const int par = lk.parent;
    const Mat3<T> Rpj = quat_to_mat<T>(std::vector<T>{T(lk.pquat[0]), T(lk.pquat[1]), T(lk.pquat[2]), T(lk.pquat[3])}.data());
    const Vec3<T> r = vec3_of<T>(lk.ppos);
    const SMat<T> XT = plux<T>(transpose(Rpj), r);  // parent -> joint frame
    const Vec3<T> a = vec3_of<T>(lk.axis);
    SMat<T> XJ;
    Mat3<T> Rj = ident3<T>();
    Vec3<T> tj = zero3<T>();
    const T qi = (M.jdof[i] >= 0) ? s.q[M.jdof[i]] : T(0.0);
    if (lk.jtype == JOINT_REVOLUTE) {
      Rj = axis_angle<T>(a, qi);
      XJ = plux<T>(transpose(Rj), zero3<T>());
      K.S[i].push_back(smk<T>(a, zero3<T>()));
    } else if (lk.jtype == JOINT_SPHERICAL) {
      // ball joint (RBDA Table 4.1): position = rotation vector r, R_J = exp([r]x); velocity =
      // the child's angular velocity relative to the parent in child coordinates, S = [I; 0]
      const int j0 = M.jdof[i];
      const Vec3<T> rv = mk3<T>(s.q[j0], s.q[j0 + 1], s.q[j0 + 2]);
      T qj[4];
      quat_exp(rv, qj);
      Rj = quat_to_mat<T>(qj);
      XJ = plux<T>(transpose(Rj), zero3<T>());
      for (int k = 0; k < 3; ++k) {
        Vec3<T> e = zero3<T>();
        e[k] = T(1.0);
        K.S[i].push_back(smk<T>(e, zero3<T>()));
      }
    } else if (lk.jtype == JOINT_PRISMATIC) {
      tj = scale(a, qi);
      XJ = plux<T>(ident3<T>(), tj);
      K.S[i].push_back(smk<T>(zero3<T>(), a));
    } else {
      XJ = plux<T>(ident3<T>(), zero3<T>());
    }
    K.Xup[i] = smul(XJ, XT);
    K.R[i] = mul(mul(K.R[par], Rpj), Rj);
    K.p[i] = add(K.p[par], mul(K.R[par], add(r, mul(Rpj, tj))));
  }
  // velocities (outward)
  for (int i = 0; i < L; ++i) {
    SVec<T> vJ = szero<T>();
    for (size_t k = 0; k < K.S[i].size(); ++k) vJ = sadd(vJ, sscale(K.S[i][k], gv[M.goff[i] + k]));
    if (i == 0) {
      K.v[0] = vJ;  // zero for a fixed root
      K.c[0] = szero<T>();  // d/dt rot(R0^T) * nu = -v0 x v0 = 0
    } else {
      K.v[i] = sadd(smul(K.Xup[i], K.v[M.links[i].parent]), vJ);
      K.c[i] = smul(crm(K.v[i]), vJ);
    }
  }
}

// Gravity as a spatial force on link i in link coordinates: I_i * [0; R_i^T g].
template <class T> SVec<T> gravity_force(const ActorKin<T>& K, int i, const Params& P) {
  const Vec3<T> g = mul(transpose(K.R[i]), mk3<T>(T(P.gravity[0]), T(P.gravity[1]), T(P.gravity[2])));
  return smul(K.I[i], smk<T>(zero3<T>(), g));
}

// Small dense helpers for the (0, 1 or 6)-DOF joint blocks of the ABA.
template <class T> bool small_inverse_spd(std::vector<T> A, int n, std::vector<T>& inv) {
  inv.assign(n * n, T(0.0));
  if (!cholesky_factor(A, n)) return false;
  for (int c = 0; c < n; ++c) {
    std::vector<T> e(n, T(0.0));
    e[c] = T(1.0);
    cholesky_solve(A, n, e.data());
    for (int r = 0; r < n; ++r) inv[r * n + c] = e[r];
  }
  return true;
}

// Articulated-body algorithm (RBDA Table 7.1) with external gravity forces; tau is the model's
// generalized force vector. Returns the generalized acceleration.
// diag (optional): extra joint-space inertia on each 1-DOF joint's diagonal (the implicit drive
// term); fext (optional): external spatial force on each link, in link coordinates.
template <class T> bool aba(const ModelD& M, const ActorKin<T>& K, const std::vector<T>& tau, const Params& P,
                            std::vector<T>& qdd, const std::vector<T>* diag = nullptr,
                            const std::vector<SVec<T>>* fext = nullptr) {
  const int L = (int)M.links.size();
  qdd.assign(M.n_gen, T(std::nan("")));  // stays NaN if a pivot fails (the env is reported failed)
  std::vector<SMat<T>> IA(L);
  std::vector<SVec<T>> pA(L);
  for (int i = 0; i < L; ++i) {
    IA[i] = K.I[i];
    pA[i] = ssub(smul(crf(K.v[i]), smul(K.I[i], K.v[i])), gravity_force(K, i, P));
    if (fext) pA[i] = ssub(pA[i], (*fext)[i]);
  }
  std::vector<std::vector<SVec<T>>> U(L);
  std::vector<std::vector<T>> Dinv(L), u(L);
  for (int i = L - 1; i >= 0; --i) {
    const int nd = (int)K.S[i].size();
    U[i].resize(nd);
    std::vector<T> D(nd * nd, T(0.0));
    u[i].assign(nd, T(0.0));
    for (int k = 0; k < nd; ++k) U[i][k] = smul(IA[i], K.S[i][k]);
    for (int a = 0; a < nd; ++a) {
      for (int b = 0; b < nd; ++b) D[a * nd + b] = sdot(K.S[i][a], U[i][b]);
      u[i][a] = tau[M.goff[i] + a] - sdot(K.S[i][a], pA[i]);
    }
    if (nd == 1 || nd == 3)  // armature on every joint DOF (not on a free root)
      for (int k = 0; k < nd; ++k) D[k * nd + k] = D[k * nd + k] + T(M.links[i].armature);
    if (nd == 1 && diag) D[0] = D[0] + (*diag)[M.goff[i]];
    if (!small_inverse_spd(D, nd, Dinv[i])) return false;
    const int par = M.links[i].parent;
    if (par < 0) continue;
    SMat<T> Ia = IA[i];
    SVec<T> pa = pA[i];
    // Ia = IA - U Dinv U^T ; pa = pA + Ia c + U Dinv u
    for (int a = 0; a < nd; ++a)
      for (int b = 0; b < nd; ++b)
        for (int r = 0; r < 6; ++r)
          for (int cc = 0; cc < 6; ++cc) Ia(r, cc) = Ia(r, cc) - U[i][a][r] * Dinv[i][a * nd + b] * U[i][b][cc];
    pa = sadd(pa, smul(Ia, K.c[i]));
    for (int a = 0; a < nd; ++a) {
      T s = T(0.0);
      for (int b = 0; b < nd; ++b) s = s + Dinv[i][a * nd + b] * u[i][b];
      pa = sadd(pa, sscale(U[i][a], s));
    }
    const SMat<T> XT = stranspose(K.Xup[i]);
    IA[par] = saddM(IA[par], smul(smul(XT, Ia), K.Xup[i]));
    pA[par] = sadd(pA[par], smul(XT, pa));
  }
  qdd.assign(M.n_gen, T(0.0));
  std::vector<SVec<T>> acc(L);
  for (int i = 0; i < L; ++i) {
    const int par = M.links[i].parent;
    SVec<T> ap = K.c[i];
    if (par >= 0) ap = sadd(smul(K.Xup[i], acc[par]), K.c[i]);
    const int nd = (int)K.S[i].size();
    std::vector<T> rhs(nd);
    for (int a = 0; a < nd; ++a) rhs[a] = u[i][a] - sdot(U[i][a], ap);
    acc[i] = ap;
    for (int a = 0; a < nd; ++a) {
      T s = T(0.0);
      for (int b = 0; b < nd; ++b) s = s + Dinv[i][a * nd + b] * rhs[b];
      qdd[M.goff[i] + a] = s;
      acc[i] = sadd(acc[i], sscale(K.S[i][a], s));
    }
  }
  return true;
}

// Composite-rigid-body algorithm (RBDA Table 6.2), armature added on the joint diagonal.
template <class T> void crba(const ModelD& M, const ActorKin<T>& K, std::vector<T>& H, const std::vector<T>* diag = nullptr) {
  const int L = (int)M.links.size(), n = M.n_gen;
  H.assign(n * n, T(0.0));
  std::vector<SMat<T>> Ic(K.I);
  for (int i = L - 1; i >= 1; --i) {
    const int par = M.links[i].parent;
    Ic[par] = saddM(Ic[par], smul(smul(stranspose(K.Xup[i]), Ic[i]), K.Xup[i]));
  }
  for (int i = 0; i < L; ++i) {
    const int nd = (int)K.S[i].size();
    for (int a = 0; a < nd; ++a) {
      SVec<T> F = smul(Ic[i], K.S[i][a]);
      const int row = M.goff[i] + a;
      for (int b = 0; b < nd; ++b) H[row * n + M.goff[i] + b] = sdot(F, K.S[i][b]);
      int j = i;
      while (M.links[j].parent >= 0) {
        F = smul(stranspose(K.Xup[j]), F);
        j = M.links[j].parent;
        for (int b = 0; b < (int)K.S[j].size(); ++b) {
          const T hv = sdot(F, K.S[j][b]);
          H[row * n + M.goff[j] + b] = hv;
          H[(M.goff[j] + b) * n + row] = hv;
        }
      }
    }
    if (nd == 1 || nd == 3)
      for (int k = 0; k < nd; ++k) {
        const int g = M.goff[i] + k;
        H[g * n + g] = H[g * n + g] + T(M.links[i].armature);
      }
    if (nd == 1 && diag) H[M.goff[i] * n + M.goff[i]] = H[M.goff[i] * n + M.goff[i]] + (*diag)[M.goff[i]];
  }
}

// Recursive Newton-Euler inverse dynamics (RBDA Table 5.1) with gravity as an external force and
// armature torques; returns the generalized force that produces qdd.
template <class T> void rnea(const ModelD& M, const ActorKin<T>& K, const std::vector<T>& qdd, const Params& P,
                             std::vector<T>& tau) {
  const int L = (int)M.links.size();
  std::vector<SVec<T>> a(L), f(L);
  for (int i = 0; i < L; ++i) {
    SVec<T> aJ = szero<T>();
    for (size_t k = 0; k < K.S[i].size(); ++k) aJ = sadd(aJ, sscale(K.S[i][k], qdd[M.goff[i] + k]));
    const int par = M.links[i].parent;
    a[i] = sadd(aJ, K.c[i]);
    if (par >= 0) a[i] = sadd(a[i], smul(K.Xup[i], a[par]));
    f[i] = ssub(sadd(smul(K.I[i], a[i]), smul(crf(K.v[i]), smul(K.I[i], K.v[i]))), gravity_force(K, i, P));
  }
  tau.assign(M.n_gen, T(0.0));
  for (int i = L - 1; i >= 0; --i) {
    for (size_t k = 0; k < K.S[i].size(); ++k) tau[M.goff[i] + k] = sdot(K.S[i][k], f[i]);
    if (K.S[i].size() == 1 || K.S[i].size() == 3)
      for (size_t k = 0; k < K.S[i].size(); ++k)
        tau[M.goff[i] + k] = tau[M.goff[i] + k] + T(M.links[i].armature) * qdd[M.goff[i] + k];
    const int par = M.links[i].parent;
    if (par >= 0) f[par] = sadd(f[par], smul(stranspose(K.Xup[i]), f[i]));
  }
}

// ------------------------------------------------------------------------------------------------
// Contact generation against the ground plane z = 0 (normal +z). A candidate point is kept iff its
// separation d is strictly below the contact offset. Canonical order: env-local shape index, then
// slot (sphere: 0; capsule: 0 = centre - h*axis, 1 = centre + h*axis; box: k = 4[sx>0] + 2[sy>0] +
// [sz>0]).
template <class T> struct ContactPt {
  int shape_a, shape_b, slot;
  int cand;  // env-level candidate index (ground candidates shape by shape, then 3 per shape pair)
  int actor_a, link_a;
  int actor_b, link_b;  // -1: the ground
  Vec3<T> x;            // contact point (world)
  T d;                  // signed separation
  T mu;
  Vec3<T> n, t1, t2;    // normal from b to a, friction directions
};

// Friction directions for a contact normal n [reading]: anchor = e_x if |n_x| < 0.57735, else e_y if
// |n_y| < 0.57735, else e_z; t1 = normalise(anchor - (anchor . n) n), t2 = n x t1. For the ground
// normal e_z this gives t1 = e_x, t2 = e_y.
template <class T> void tangent_basis(const Vec3<T>& n, Vec3<T>& t1, Vec3<T>& t2) {
  const T lim = T(0.57735);
  Vec3<T> an;
  if (fabs(n[0]) < lim) an = mk3<T>(T(1.0), T(0.0), T(0.0));
  else if (fabs(n[1]) < lim) an = mk3<T>(T(0.0), T(1.0), T(0.0));
  else an = mk3<T>(T(0.0), T(0.0), T(1.0));
  const Vec3<T> t = sub(an, scale(n, dot(an, n)));
  t1 = scale(t, T(1.0) / sqrt(dot(t, t)));
  t2 = cross(n, t1);
}

// World pose (rotation, centre) of a shape.
template <class T> void shape_pose(const ActorKin<T>& K, const ShapeD& sh, Mat3<T>& Rs, Vec3<T>& cs) {
  const int li = sh.link;
  const T q[4] = {T(sh.quat[0]), T(sh.quat[1]), T(sh.quat[2]), T(sh.quat[3])};
  Rs = mul(K.R[li], quat_to_mat<T>(q));
  cs = add(K.p[li], mul(K.R[li], vec3_of<T>(sh.pos)));
}

// Squared distance from the point p (box frame) to the box of half extents e.
template <class T> T box_dist2(const Vec3<T>& p, const Vec3<T>& e) {
  T f = T(0.0);
  for (int k = 0; k < 3; ++k) {
    const T o = fabs(p[k]) - e[k];
    if (T(0.0) < o) f = f + o * o;
  }
  return f;
}

// Exact minimiser over t in [0, 1] of the squared distance from p0 + t dv to the box (convex,
// piecewise quadratic): split [0, 1] at the breakpoints p_k(t) = +-e_k, take each piece's
// stationary point clamped into the piece (the piece's start if the distance is constant there),
// and keep the smallest value, ties to the smallest t.
template <class T> T segment_box_closest_t(const Vec3<T>& p0, const Vec3<T>& dv, const Vec3<T>& e) {
  std::vector<T> ts = {T(0.0), T(1.0)};
  for (int k = 0; k < 3; ++k) {
    if (dv[k] == T(0.0)) continue;
    for (int s = -1; s <= 1; s += 2) {
      const T t = (T((double)s) * e[k] - p0[k]) / dv[k];
      if (T(0.0) < t && t < T(1.0)) ts.push_back(t);
    }
  }
  std::sort(ts.begin(), ts.end(), [](const T& a, const T& b) { return a < b; });
  auto at = [&](const T& t) { return add(p0, scale(dv, t)); };
  T best_t = T(0.0), best_f = box_dist2(at(T(0.0)), e);
  for (size_t i = 0; i + 1 < ts.size(); ++i) {
    const T ta = ts[i], tb = ts[i + 1];
    const Vec3<T> pm = at((ta + tb) * T(0.5));
    T num = T(0.0), den = T(0.0);
    for (int k = 0; k < 3; ++k) {
      if (!(e[k] < fabs(pm[k]))) continue;  // inside this slab on the whole piece
      const T s = (T(0.0) < pm[k]) ? T(1.0) : T(-1.0);
      num = num + dv[k] * (s * e[k] - p0[k]);
      den = den + dv[k] * dv[k];
    }
    T t = ta;
    if (T(0.0) < den) t = tmin(tmax(num / den, ta), tb);
    const T f = box_dist2(at(t), e);
    if (f < best_f) { best_f = f; best_t = t; }
  }
  const T f1 = box_dist2(at(T(1.0)), e);
  if (f1 < best_f) best_t = T(1.0);
  return best_t;
}

constexpr int kPairSlots = 5;  // capsule-box samples: t = 0, t = 1, face-clip entry / exit, closest point

// The part of the segment over the box face selected by the closest point [reading]: let k be the
// box axis along which the normal at the closest point t* is largest (ties: lowest k); clip the
// segment to the slabs |x_j| <= e_j of the two other axes. Returns false if nothing remains,
// else the parameter interval [ta, tb] within [0, 1]. Its ends are the extra samples that give a
// capsule lying along a face two supporting points.
template <class T> bool face_clip(const Vec3<T>& p0, const Vec3<T>& dv, const Vec3<T>& e, const T& r, const T& tstar,
                                  T& ta, T& tb);

// A sphere of radius r at p (box frame) against the box of half extents e: normal from the box to
// the sphere, separation d, and the contact point halfway between the two surfaces.
template <class T> void sphere_box(const Vec3<T>& p, const T& r, const Vec3<T>& e, Vec3<T>& n, T& d, Vec3<T>& x) {
  bool inside = true;
  for (int k = 0; k < 3; ++k)
    if (e[k] < fabs(p[k])) inside = false;
  if (!inside) {
    Vec3<T> q;
    for (int k = 0; k < 3; ++k) q[k] = tmin(tmax(p[k], T(0.0) - e[k]), e[k]);
    const Vec3<T> dl = sub(p, q);
    const T dist = sqrt(dot(dl, dl));
    n = scale(dl, T(1.0) / dist);
    d = dist - r;
  } else {
    int kb = 0;
    T best = e[0] - fabs(p[0]);
    for (int k = 1; k < 3; ++k)
      if (e[k] - fabs(p[k]) < best) { best = e[k] - fabs(p[k]); kb = k; }
    n = zero3<T>();
    n[kb] = (p[kb] < T(0.0)) ? T(-1.0) : T(1.0);
    d = T(0.0) - best - r;
  }
  x = sub(p, scale(n, r + d * T(0.5)));
}

template <class T> bool face_clip(const Vec3<T>& p0, const Vec3<T>& dv, const Vec3<T>& e, const T& r, const T& tstar,
                                  T& ta, T& tb) {
  Vec3<T> n, x;
  T d;
  sphere_box(add(p0, scale(dv, tstar)), r, e, n, d, x);
  int kn = 0;
  for (int k = 1; k < 3; ++k)
    if (fabs(n[kn]) < fabs(n[k])) kn = k;
  ta = T(0.0);
  tb = T(1.0);
  for (int j = 0; j < 3; ++j) {
    if (j == kn) continue;
    if (dv[j] == T(0.0)) {
      if (e[j] < fabs(p0[j])) return false;
      continue;
    }
    T t0 = (T(0.0) - e[j] - p0[j]) / dv[j], t1 = (e[j] - p0[j]) / dv[j];
    if (t1 < t0) { const T s = t0; t0 = t1; t1 = s; }
    ta = tmax(ta, t0);
    tb = tmin(tb, t1);
  }
  return !(tb < ta);
}

// Contact generation at the substep-start configuration. Ground (plane z = 0, normal +z): a
// candidate point is kept iff its separation d is strictly below the contact offset; candidates
// are numbered shape by shape (sphere: 0; capsule: 0 = centre - h*axis, 1 = centre + h*axis; box:
// k = 4[sx>0] + 2[sy>0] + [sz>0]). Then every capsule-box pair of shapes of different actors
// (env-local shape indices a < b, in order): the capsule's endpoints (slots 0, 1), the ends of its
// face clip (slots 2, 3) and the closest point of its segment to the box (slot 4), the last three
// only if strictly inside the segment, each treated as a sphere of the capsule's radius against
// the box.
template <class T> void env_contacts(const Oracle& O, int env, const std::vector<ActorKin<T>>& K,
                                     std::vector<ContactPt<T>>& out) {
  out.clear();
  const T coff = T(O.prm.contact_offset);
  const Vec3<T> ez = mk3<T>(T(0.0), T(0.0), T(1.0)), ex = mk3<T>(T(1.0), T(0.0), T(0.0)),
                ey = mk3<T>(T(0.0), T(1.0), T(0.0));
  int shape_base = 0, cand_base = 0;
  std::vector<std::pair<int, int>> shape_ref;  // env-local shape -> (actor, shape within actor)
  for (int a = 0; a < O.n_act(env); ++a) {
    const ModelD& M = O.actor_model(env, a);
    for (size_t s = 0; s < M.shapes.size(); ++s) {
      shape_ref.push_back({a, (int)s});
      const ShapeD& sh = M.shapes[s];
      const int ncand = (sh.type == SHAPE_SPHERE) ? 1 : (sh.type == SHAPE_CAPSULE ? 2 : 8);
      const int li = sh.link;
      Mat3<T> Rs;
      Vec3<T> cs;
      shape_pose(K[a], sh, Rs, cs);
      const T mu = tmax(T(sh.friction), T(O.prm.ground_friction));
      auto push = [&](int slot, const Vec3<T>& x, const T& d) {
        if (d < coff)
          out.push_back(ContactPt<T>{shape_base + (int)s, -1, slot, cand_base + slot, a, li, -1, -1, x, d, mu, ez, ex, ey});
      };
      if (sh.type == SHAPE_SPHERE) {
        const T r = T(sh.size[0]);
        push(0, mk3<T>(cs[0], cs[1], cs[2] - r), cs[2] - r);
      } else if (sh.type == SHAPE_CAPSULE) {
        const T r = T(sh.size[0]), hl = T(sh.size[1]);
        const Vec3<T> ax = mk3<T>(Rs(0, 0), Rs(1, 0), Rs(2, 0));  // local x axis in world
        for (int k = 0; k < 2; ++k) {
          const Vec3<T> e = (k == 0) ? sub(cs, scale(ax, hl)) : add(cs, scale(ax, hl));
          push(k, mk3<T>(e[0], e[1], e[2] - r), e[2] - r);
        }
      } else if (sh.type == SHAPE_BOX) {
        for (int k = 0; k < 8; ++k) {
          const T sx = (k & 4) ? T(1.0) : T(-1.0), sy = (k & 2) ? T(1.0) : T(-1.0), sz = (k & 1) ? T(1.0) : T(-1.0);
          const Vec3<T> loc = mk3<T>(sx * T(sh.size[0]), sy * T(sh.size[1]), sz * T(sh.size[2]));
          const Vec3<T> vtx = add(cs, mul(Rs, loc));
          push(k, vtx, vtx[2]);
        }
      }
      cand_base += ncand;
    }
    shape_base += (int)M.shapes.size();
  }
  // capsule-box pairs
  for (size_t pi = 0; pi < O.env_pairs[env].size(); ++pi) {
    const int sa = O.env_pairs[env][pi].first, sb = O.env_pairs[env][pi].second;
    const int aa = shape_ref[sa].first, ab = shape_ref[sb].first;
    const ShapeD& sha = O.actor_model(env, aa).shapes[shape_ref[sa].second];
    const ShapeD& shb = O.actor_model(env, ab).shapes[shape_ref[sb].second];
    const bool a_is_capsule = sha.type == SHAPE_CAPSULE;
    const ShapeD& cap = a_is_capsule ? sha : shb;
    const ShapeD& box = a_is_capsule ? shb : sha;
    Mat3<T> Rc, Rb;
    Vec3<T> cc, cb;
    shape_pose(K[a_is_capsule ? aa : ab], cap, Rc, cc);
    shape_pose(K[a_is_capsule ? ab : aa], box, Rb, cb);
    const T r = T(cap.size[0]), hl = T(cap.size[1]);
    const Vec3<T> ax = mk3<T>(Rc(0, 0), Rc(1, 0), Rc(2, 0));
    const Mat3<T> RbT = transpose(Rb);
    const Vec3<T> p0 = mul(RbT, sub(sub(cc, scale(ax, hl)), cb));
    const Vec3<T> p1 = mul(RbT, sub(add(cc, scale(ax, hl)), cb));
    const Vec3<T> dv = sub(p1, p0);
    const Vec3<T> ext = vec3_of<T>(box.size);
    const T tstar = segment_box_closest_t(p0, dv, ext);
    T ta, tb;
    const bool clip = face_clip(p0, dv, ext, r, tstar, ta, tb);
    const T mu = tmax(T(sha.friction), T(shb.friction));
    for (int slot = 0; slot < kPairSlots; ++slot) {
      T t;
      if (slot == 0) t = T(0.0);
      else if (slot == 1) t = T(1.0);
      else {
        t = (slot == 2) ? ta : ((slot == 3) ? tb : tstar);
        if (slot < 4 && !clip) continue;
        if (slot == 3 && !(ta < tb)) continue;
        if (!(T(0.0) < t && t < T(1.0))) continue;
      }
      Vec3<T> nb, xb;
      T d;
      sphere_box(add(p0, scale(dv, t)), r, ext, nb, d, xb);
      if (!(d < coff)) continue;
      Vec3<T> n = mul(Rb, nb);  // from the box to the capsule
      if (!a_is_capsule) n = scale(n, T(-1.0));
      ContactPt<T> c{sa, sb, slot, cand_base + kPairSlots * (int)pi + slot, aa, sha.link, ab, shb.link,
                     add(cb, mul(Rb, xb)), d, mu, n, n, n};
      tangent_basis(n, c.t1, c.t2);
      out.push_back(c);
    }
  }
}

// FNV-1a (32 bit) over the little-endian bytes of 32-bit integers; used to record the active
// constraint set of every substep so that integer decisions can be compared exactly.
inline void fnv1a_int(uint32_t& h, int32_t v) {
  const uint32_t u = (uint32_t)v;
  for (int b = 0; b < 4; ++b) {
    h ^= (u >> (8 * b)) & 0xffu;
    h *= 16777619u;
  }
}

template <class T> struct Row {
  int kind;
  std::vector<T> J;  // env generalized space
  T d;               // separation (normal and limit rows)
  int normal_row;    // for friction rows, index of the normal row
  T mu;
  int contact;       // contact index or -1
  Vec3<T> k;         // direction (contact rows)
  std::vector<T> W;  // M^-1 J^T
  T A;               // J M^-1 J^T
  int cache;         // slot of this constraint in the env's impulse cache
};

struct EnvLayout {
  std::vector<int> gen_off;    // per actor offset in the env generalized vector
  std::vector<int> body_off;   // per actor offset of its first non-virtual link (net force rows)
  int n_gen = 0;
};

inline EnvLayout env_layout(const Oracle& O, int env) {
  EnvLayout E;
  int g = 0, b = 0;
  for (int a = 0; a < O.n_act(env); ++a) {
    const ModelD& M = O.actor_model(env, a);
    E.gen_off.push_back(g);
    E.body_off.push_back(b);
    g += M.n_gen;
    b += M.n_body;
  }
  E.n_gen = g;
  return E;
}

// Jacobian row of a world direction k at world point x on link li of actor a: k . d(x_dot)/d(nu).
template <class T> void point_row(const Oracle& O, int env, const EnvLayout& E, const std::vector<ActorKin<T>>& K,
                                  int a, int li, const Vec3<T>& x, const Vec3<T>& k, const T& sign, std::vector<T>& J) {
  const ModelD& M = O.actor_model(env, a);
  int l = li;
  while (l >= 0) {
    const LinkD& lk = M.links[l];
    const int g = E.gen_off[a] + M.goff[l];
    if (l == 0 && lk.jtype == JOINT_FREE) {
      const Vec3<T> rxk = cross(sub(x, K[a].p[0]), k);
      for (int m = 0; m < 3; ++m) {
        J[g + m] = J[g + m] + sign * rxk[m];
        J[g + 3 + m] = J[g + 3 + m] + sign * k[m];
      }
    } else if (lk.jtype == JOINT_REVOLUTE) {
      const Vec3<T> ax = mul(K[a].R[l], vec3_of<T>(lk.axis));
      J[g] = J[g] + sign * dot(k, cross(ax, sub(x, K[a].p[l])));
    } else if (lk.jtype == JOINT_PRISMATIC) {
      const Vec3<T> ax = mul(K[a].R[l], vec3_of<T>(lk.axis));
      J[g] = J[g] + sign * dot(k, ax);
    } else if (lk.jtype == JOINT_SPHERICAL) {  // rotation about each child axis through the joint
      for (int c = 0; c < 3; ++c) {
        const Vec3<T> ax = mk3<T>(K[a].R[l](0, c), K[a].R[l](1, c), K[a].R[l](2, c));
        J[g + c] = J[g + c] + sign * dot(k, cross(ax, sub(x, K[a].p[l])));
      }
    }
    l = lk.parent;
  }
}

// Build all constraint rows of one env at the substep-start configuration. Row order: joint-limit
// rows (env DOF ascending, lower before upper), then every contact's normal row, then every
// contact's two friction rows (t1 = e_x, t2 = e_y for the ground).
template <class T> void build_rows(const Oracle& O, int env, const EnvLayout& E, const std::vector<ActorState<T>>& st,
                                   const std::vector<ActorKin<T>>& K, const std::vector<ContactPt<T>>& C,
                                   std::vector<Row<T>>& rows, uint32_t* sig) {
  rows.clear();
  const int n = E.n_gen;
  const T margin = T(O.prm.limit_margin);
  std::vector<int32_t> lim_ids;
  int jbase = 0;
  for (int a = 0; a < O.n_act(env); ++a) {
    const ModelD& M = O.actor_model(env, a);
    for (size_t l = 0; l < M.links.size(); ++l) {
      const LinkD& lk = M.links[l];
      if (M.jdof[l] < 0 || M.ndof[l] != 1 || !lk.has_limit) continue;
      const T q = st[a].q[M.jdof[l]];
      const int g = E.gen_off[a] + M.goff[l];
      if (q - T(lk.lo) < margin) {
        Row<T> r{ROW_LIMIT, std::vector<T>(n, T(0.0)), q - T(lk.lo), -1, T(0.0), -1, zero3<T>(), {}, T(0.0),
                 3 * O.contact_cap[env] + 2 * (jbase + M.jdof[l])};
        r.J[g] = T(1.0);
        rows.push_back(r);
        lim_ids.push_back(jbase + M.jdof[l]);
        lim_ids.push_back(0);
      }
      if (T(lk.hi) - q < margin) {
        Row<T> r{ROW_LIMIT, std::vector<T>(n, T(0.0)), T(lk.hi) - q, -1, T(0.0), -1, zero3<T>(), {}, T(0.0),
                 3 * O.contact_cap[env] + 2 * (jbase + M.jdof[l]) + 1};
        r.J[g] = T(-1.0);
        rows.push_back(r);
        lim_ids.push_back(jbase + M.jdof[l]);
        lim_ids.push_back(1);
      }
    }
    jbase += M.n_jdof;
  }
  // tendon length limits (after every joint limit): J = +-c over the tendon's joints, slots after
  // the joint-limit slots
  std::vector<int32_t> ten_ids;
  int tbase = 0;
  for (int a = 0; a < O.n_act(env); ++a) {
    const ModelD& M = O.actor_model(env, a);
    for (size_t t = 0; t < M.tendons.size(); ++t) {
      const TendonD& td = M.tendons[t];
      if (!td.has_limit) continue;
      T len(0.0);
      for (size_t k = 0; k < td.links.size(); ++k) len = len + T(td.coef[k]) * st[a].q[M.jdof[td.links[k]]];
      for (int side = 0; side < 2; ++side) {
        const T dist = side == 0 ? len - T(td.lo) : T(td.hi) - len;
        if (!(dist < margin)) continue;
        Row<T> r{ROW_LIMIT, std::vector<T>(n, T(0.0)), dist, -1, T(0.0), -1, zero3<T>(), {}, T(0.0),
                 3 * O.contact_cap[env] + 2 * jbase + 2 * (tbase + (int)t) + side};
        for (size_t k = 0; k < td.links.size(); ++k)
          r.J[E.gen_off[a] + M.goff[td.links[k]]] = r.J[E.gen_off[a] + M.goff[td.links[k]]] +
                                                   T(side == 0 ? td.coef[k] : -td.coef[k]);
        rows.push_back(r);
        ten_ids.push_back(tbase + (int)t);
        ten_ids.push_back(side);
      }
    }
    tbase += (int)M.tendons.size();
  }
  if (sig) {
    fnv1a_int(*sig, (int32_t)(lim_ids.size() / 2));
    for (int32_t v : lim_ids) fnv1a_int(*sig, v);
    if (tbase > 0) {  // envs with tendons also hash their tendon-limit rows
      fnv1a_int(*sig, (int32_t)(ten_ids.size() / 2));
      for (int32_t v : ten_ids) fnv1a_int(*sig, v);
    }
    fnv1a_int(*sig, (int32_t)C.size());
    for (const auto& c : C) { fnv1a_int(*sig, c.shape_a); fnv1a_int(*sig, c.shape_b); fnv1a_int(*sig, c.slot); }
  }
  // J = k . d(x_dot on body a)/d(nu) - k . d(x_dot on body b)/d(nu) at the contact point
  auto contact_row = [&](const ContactPt<T>& c, const Vec3<T>& k, std::vector<T>& J) {
    point_row(O, env, E, K, c.actor_a, c.link_a, c.x, k, T(1.0), J);
    if (c.actor_b >= 0) point_row(O, env, E, K, c.actor_b, c.link_b, c.x, k, T(-1.0), J);
  };
  const int first_normal = (int)rows.size();
  for (size_t c = 0; c < C.size(); ++c) {
    Row<T> r{ROW_NORMAL, std::vector<T>(n, T(0.0)), C[c].d, -1, C[c].mu, (int)c, C[c].n, {}, T(0.0), 3 * C[c].cand};
    contact_row(C[c], C[c].n, r.J);
    rows.push_back(r);
  }
  for (size_t c = 0; c < C.size(); ++c) {
    for (int t = 0; t < 2; ++t) {
      const Vec3<T> k = (t == 0) ? C[c].t1 : C[c].t2;
      Row<T> r{ROW_FRICTION, std::vector<T>(n, T(0.0)), T(0.0), first_normal + (int)c, C[c].mu, (int)c, k, {}, T(0.0),
               3 * C[c].cand + 1 + t};
      contact_row(C[c], k, r.J);
      rows.push_back(r);
    }
  }
}

// Read/write one env's actors from/to the global tensors (paper layout: root (N_A, 13) =
// [p 3 | quat xyzw 4 | v 3 | omega 3], DOF state (N_D, 2) = [q, qd]).
template <class T> void load_env(const Oracle& O, int env, const double* root, const double* dof,
                                 std::vector<ActorState<T>>& st) {
  st.resize(O.n_act(env));
  int64_t jd = O.jdof_off[env];
  for (int a = 0; a < O.n_act(env); ++a) {
    const ModelD& M = O.actor_model(env, a);
    const double* r = root + (int64_t)(O.actor_off[env] + a) * 13;
    ActorState<T>& s = st[a];
    s.p = vec3_of<T>(r);
    for (int k = 0; k < 4; ++k) s.quat[k] = T(r[3 + k]);
    s.v = vec3_of<T>(r + 7);
    s.w = vec3_of<T>(r + 10);
    s.q.assign(M.n_jdof, T(0.0));
    s.qd.assign(M.n_jdof, T(0.0));
    for (int j = 0; j < M.n_jdof; ++j) { s.q[j] = T(dof[(jd + j) * 2]); s.qd[j] = T(dof[(jd + j) * 2 + 1]); }
    jd += M.n_jdof;
  }
}

template <class T> void store_env(const Oracle& O, int env, const std::vector<ActorState<T>>& st, double* root, double* dof) {
  int64_t jd = O.jdof_off[env];
  for (int a = 0; a < O.n_act(env); ++a) {
    const ModelD& M = O.actor_model(env, a);
    double* r = root + (int64_t)(O.actor_off[env] + a) * 13;
    const ActorState<T>& s = st[a];
    for (int k = 0; k < 3; ++k) { r[k] = val(s.p[k]); r[7 + k] = val(s.v[k]); r[10 + k] = val(s.w[k]); }
    for (int k = 0; k < 4; ++k) r[3 + k] = val(s.quat[k]);
    for (int j = 0; j < M.n_jdof; ++j) { dof[(jd + j) * 2] = val(s.q[j]); dof[(jd + j) * 2 + 1] = val(s.qd[j]); }
    jd += M.n_jdof;
  }
}

// Per-env accumulators of one sim step.
template <class T> struct StepOut {
  std::vector<Vec3<T>> impulse;  // per env link (actor-major), sum of lambda * k over substeps
  std::vector<ContactPt<T>> last_contacts;
  std::vector<T> dof_force;      // per env joint DOF: joint force of the last substep
  uint32_t sig = 2166136261u;
  bool ok = true;
};

// Per-step controls beyond the actuation (env-local arrays, null when absent): joint drive targets
// per joint DOF, and an external force and torque (world axes, at the body's COM) per body.
struct Controls {
  const double* pos_target = nullptr;
  const double* vel_target = nullptr;
  const double* body_force = nullptr;  // [env bodies * 6]: force (3), torque (3)
};

// One substep of one env (steps a1-a7 of the method).
template <class T> void env_substep(const Oracle& O, int env, std::vector<ActorState<T>>& st, const T* act,
                                    const T& h, std::vector<T>& cache, StepOut<T>& out, const Controls& ctl = {}) {
  const Params& P = O.prm;
  const EnvLayout E = env_layout(O, env);
  const int n = E.n_gen, A = O.n_act(env);
  // a1 + a2 + a3: controls, kinematics, ABA -> v_free = nu + h * qdd
  std::vector<ActorKin<T>> K(A);
  std::vector<T> nu(n, T(0.0)), vfree(n, T(0.0));
  std::vector<T> Mfull(n * n, T(0.0));
  int jbase = 0, bbase = 0;
  for (int a = 0; a < A; ++a) {
    const ModelD& M = O.actor_model(env, a);
    const std::vector<T> gv = gen_velocity(M, st[a]);
    kinematics(M, st[a], gv, K[a]);
    // joint forces of the substep: actuation, damping at the substep-start velocity, and the
    // implicit drive kp (q* - q - h qd) + kd (qd* - qd), whose h (h kp + kd) joins the joint's
    // diagonal of the joint-space inertia (implicit Euler of the spring-damper)
    std::vector<T> tau(M.n_gen, T(0.0)), diag(M.n_gen, T(0.0));
    for (size_t l = 0; l < M.links.size(); ++l)
      for (int k = 1; k < M.ndof[l] && M.jdof[l] >= 0; ++k) {  // ball-joint DOFs 1, 2 (no drives)
        const int j = M.jdof[l] + k;
        const T f = act[jbase + j] - T(M.links[l].damping) * st[a].qd[j];
        tau[M.goff[l] + k] = f;
        if (out.dof_force.size() > (size_t)(jbase + j)) out.dof_force[jbase + j] = f;
      }
    for (size_t l = 0; l < M.links.size(); ++l)
      if (M.jdof[l] >= 0) {
        const int j = M.jdof[l];
        const LinkD& lk = M.links[l];
        T f = act[jbase + j] - T(lk.damping) * st[a].qd[j];
        if (lk.kp != 0.0 || lk.kd != 0.0) {
          const T qt = ctl.pos_target ? T(ctl.pos_target[jbase + j]) : T(0.0);
          const T vt = ctl.vel_target ? T(ctl.vel_target[jbase + j]) : T(0.0);
          f = f + T(lk.kp) * (qt - st[a].q[j] - h * st[a].qd[j]) + T(lk.kd) * (vt - st[a].qd[j]);
          diag[M.goff[l]] = h * (h * T(lk.kp) + T(lk.kd));
        }
        tau[M.goff[l]] = f;
        if (out.dof_force.size() > (size_t)(jbase + j)) out.dof_force[jbase + j] = f;
      }
    // fixed tendons: spring-damper on the length l = sum c_k q_k, force F = -k (l - rest) - d l_dot
    // at the substep start, applied to each joint as c_k F
    for (const TendonD& td : M.tendons) {
      T len(0.0), rate(0.0);
      for (size_t k = 0; k < td.links.size(); ++k) {
        const int j = M.jdof[td.links[k]];
        len = len + T(td.coef[k]) * st[a].q[j];
        rate = rate + T(td.coef[k]) * st[a].qd[j];
      }
      const T F = T(0.0) - T(td.stiffness) * (len - T(td.rest)) - T(td.damping) * rate;
      for (size_t k = 0; k < td.links.size(); ++k) {
        const int l = td.links[k];
        tau[M.goff[l]] = tau[M.goff[l]] + T(td.coef[k]) * F;
        if (out.dof_force.size() > (size_t)(jbase + M.jdof[l]))
          out.dof_force[jbase + M.jdof[l]] = out.dof_force[jbase + M.jdof[l]] + T(td.coef[k]) * F;
      }
    }
    // external force and torque per body (world axes, at the COM) as link-coordinate spatial forces
    std::vector<SVec<T>> fext;
    if (ctl.body_force) {
      fext.assign(M.links.size(), szero<T>());
      int b = bbase;
      for (size_t l = 0; l < M.links.size(); ++l) {
        if (M.links[l].is_virtual) continue;
        const double* bf = ctl.body_force + (int64_t)b * 6;
        ++b;
        const Mat3<T> Rt = transpose(K[a].R[l]);
        const Vec3<T> F = mul(Rt, mk3<T>(T(bf[0]), T(bf[1]), T(bf[2])));
        const Vec3<T> Tq = mul(Rt, mk3<T>(T(bf[3]), T(bf[4]), T(bf[5])));
        fext[l] = smk<T>(add(Tq, cross(vec3_of<T>(M.links[l].com), F)), F);
      }
    }
    bbase += M.n_body;
    std::vector<T> qdd;
    if (!aba(M, K[a], tau, P, qdd, &diag, ctl.body_force ? &fext : nullptr)) out.ok = false;
    if (M.free_root) {  // rate of the root-origin velocity: a_lin + omega x v
      const Vec3<T> wxv = cross(st[a].w, st[a].v);
      for (int k = 0; k < 3; ++k) qdd[3 + k] = qdd[3 + k] + wxv[k];
    }
    std::vector<T> H;
    crba(M, K[a], H, &diag);
    for (int i = 0; i < M.n_gen; ++i) {
      nu[E.gen_off[a] + i] = gv[i];
      vfree[E.gen_off[a] + i] = gv[i] + h * (i < (int)qdd.size() ? qdd[i] : T(0.0));
      for (int j = 0; j < M.n_gen; ++j) Mfull[(E.gen_off[a] + i) * n + E.gen_off[a] + j] = H[i * M.n_gen + j];
    }
    jbase += M.n_jdof;
  }
  // a4: contacts at the substep-start configuration; a5: rows, W = M^-1 J^T, A = J W
  std::vector<ContactPt<T>> C;
  env_contacts(O, env, K, C);
  std::vector<Row<T>> rows;
  build_rows(O, env, E, st, K, C, rows, &out.sig);
  if (n > 0 && !cholesky_factor(Mfull, n)) out.ok = false;
  for (auto& r : rows) {
    r.W = r.J;
    if (n > 0) cholesky_solve(Mfull, n, r.W.data());
    T Arr = T(0.0);
    for (int i = 0; i < n; ++i) Arr = Arr + r.J[i] * r.W[i];
    r.A = Arr;
  }
  // a6: TGS-style projected Gauss-Seidel. h_it = h / n_pos; Delta q starts at 0. Each row's impulse
  // starts from the cached impulse of the same constraint in the previous substep (zero if that
  // constraint was not active), applied in row order: v = v_free + sum_r W_r lambda_r.
  const int npos = P.pos_iters, nvel = P.vel_iters;
  const T hit = h / T((double)npos);
  const T beta = T(P.bias_coef), vmax = T(P.max_depen_vel);
  const T eps_A = T(1e-12);  // rows with no response are skipped (lambda stays 0)
  std::vector<T> v = vfree, dq(n, T(0.0)), lam(rows.size(), T(0.0));
  for (size_t ri = 0; ri < rows.size(); ++ri) {
    if (!(eps_A < rows[ri].A)) continue;
    lam[ri] = cache[rows[ri].cache];
    for (int i = 0; i < n; ++i) v[i] = v[i] + rows[ri].W[i] * lam[ri];
  }
  auto Jdot = [&](const Row<T>& r, const std::vector<T>& x) {
    T s = T(0.0);
    for (int i = 0; i < n; ++i) s = s + r.J[i] * x[i];
    return s;
  };
  auto apply = [&](size_t ri, const T& lnew) {
    const T dl = lnew - lam[ri];
    for (int i = 0; i < n; ++i) v[i] = v[i] + rows[ri].W[i] * dl;
    lam[ri] = lnew;
  };
  for (int it = 0; it < npos + nvel; ++it) {
    const bool pos = it < npos;
    for (size_t ri = 0; ri < rows.size(); ++ri) {
      const Row<T>& r = rows[ri];
      if (!(eps_A < r.A)) continue;
      if (r.kind == ROW_FRICTION) {
        const T lim = r.mu * lam[r.normal_row];
        T lnew = lam[ri] + (T(0.0) - Jdot(r, v)) / r.A;
        lnew = tmin(tmax(lnew, T(0.0) - lim), lim);
        apply(ri, lnew);
      } else {
        const T sep = r.d + Jdot(r, dq);
        T target;
        if (pos) {
          if (!(sep < T(0.0))) target = (T(0.0) - sep) / hit;      // speculative: close the gap
          else target = tmin((T(0.0) - beta * sep) / hit, vmax);    // biased push-out
        } else {
          target = (T(0.0) < sep) ? (T(0.0) - sep) / h : T(0.0);
        }
        const T lnew = tmax(lam[ri] + (target - Jdot(r, v)) / r.A, T(0.0));
        apply(ri, lnew);
      }
    }
    if (pos)
      for (int i = 0; i < n; ++i) dq[i] = dq[i] + hit * v[i];
  }
  // the cache keeps exactly this substep's active constraints
  for (auto& c : cache) c = T(0.0);
  for (size_t ri = 0; ri < rows.size(); ++ri) cache[rows[ri].cache] = lam[ri];
  // contact impulses per env link
  {
    std::vector<int> link_base(A, 0);
    int lb = 0;
    for (int a = 0; a < A; ++a) { link_base[a] = lb; lb += (int)O.actor_model(env, a).links.size(); }
    for (size_t ri = 0; ri < rows.size(); ++ri) {
      if (rows[ri].contact < 0) continue;
      const ContactPt<T>& c = C[rows[ri].contact];
      Vec3<T>& acc = out.impulse[link_base[c.actor_a] + c.link_a];
      acc = add(acc, scale(rows[ri].k, lam[ri]));
      if (c.actor_b >= 0) {  // equal and opposite on body b; ground reactions are not reported
        Vec3<T>& accb = out.impulse[link_base[c.actor_b] + c.link_b];
        accb = sub(accb, scale(rows[ri].k, lam[ri]));
      }
    }
  }
  out.last_contacts = C;
  // a7: integrate. Joints: q += dq, qd = v. Free root: p += dq_lin, quat = exp(dq_ang) * quat,
  // omega = v_ang, v_root = v_lin.
  for (int a = 0; a < A; ++a) {
    const ModelD& M = O.actor_model(env, a);
    ActorState<T>& s = st[a];
    const int g0 = E.gen_off[a];
    if (M.free_root) {
      const Vec3<T> dang = mk3<T>(dq[g0], dq[g0 + 1], dq[g0 + 2]);
      const Vec3<T> dlin = mk3<T>(dq[g0 + 3], dq[g0 + 4], dq[g0 + 5]);
      const Vec3<T> wn = mk3<T>(v[g0], v[g0 + 1], v[g0 + 2]);
      const Vec3<T> vn = mk3<T>(v[g0 + 3], v[g0 + 4], v[g0 + 5]);
      s.p = add(s.p, dlin);
      T e[4], qn[4];
      quat_exp(dang, e);
      quat_mul(e, s.quat, qn);
      const T nrm = sqrt(qn[0] * qn[0] + qn[1] * qn[1] + qn[2] * qn[2] + qn[3] * qn[3]);
      for (int k = 0; k < 4; ++k) s.quat[k] = qn[k] / nrm;
      s.w = wn;
      s.v = vn;
    } else {
      s.w = zero3<T>();
      s.v = zero3<T>();
    }
    for (size_t l = 0; l < M.links.size(); ++l)
      if (M.ndof[l] == 3) {
        // ball joint: R_J <- R_J exp([dq]x) (dq in child coordinates), back to a rotation vector
        const int j = M.jdof[l], g = g0 + M.goff[l];
        T qj[4], e[4], qn[4];
        quat_exp(mk3<T>(s.q[j], s.q[j + 1], s.q[j + 2]), qj);
        quat_exp(mk3<T>(dq[g], dq[g + 1], dq[g + 2]), e);
        quat_mul(qj, e, qn);
        const Vec3<T> r = quat_log(qn);
        for (int k = 0; k < 3; ++k) {
          s.q[j + k] = r[k];
          s.qd[j + k] = v[g + k];
        }
      } else if (M.jdof[l] >= 0) {
        const int j = M.jdof[l], g = g0 + M.goff[l];
        s.q[j] = s.q[j] + dq[g];
        s.qd[j] = v[g];
      }
  }
}

template <class T> struct Outputs {
  double* cache;       // [n_envs * cache_len] impulse cache, in/out (required)
  double* net_force;   // [N_B * 3] or null
  int32_t* contacts;   // [n_envs * max_contact_cap * 3] or null
  int32_t* n_contacts; // [n_envs] or null
  uint32_t* sig;       // [n_envs] or null
  int32_t* status;     // [n_envs] or null
  const double* pos_target = nullptr;  // [N_D] drive position targets or null (0)
  const double* vel_target = nullptr;  // [N_D] drive velocity targets or null (0)
  const double* body_force = nullptr;  // [N_B * 6] external force, torque per body or null
  double* dof_force = nullptr;         // [N_D] out: joint force of the last substep, or null
  double* body_state = nullptr;        // [N_B * 13] out: body poses and velocities after the step, or null
};

// Unit quaternion (x, y, z, w), w >= 0, of a rotation matrix (Shepperd's method: the largest of
// 4w^2, 4x^2, 4y^2, 4z^2 picks the square root taken).
inline void mat_to_quat(const Mat3<double>& R, double q[4]) {
  const double tr = R(0, 0) + R(1, 1) + R(2, 2);
  double x, y, z, w;
  if (tr > 0.0) {
    const double s = std::sqrt(tr + 1.0) * 2.0;
    w = 0.25 * s; x = (R(2, 1) - R(1, 2)) / s; y = (R(0, 2) - R(2, 0)) / s; z = (R(1, 0) - R(0, 1)) / s;
  } else if (R(0, 0) > R(1, 1) && R(0, 0) > R(2, 2)) {
    const double s = std::sqrt(1.0 + R(0, 0) - R(1, 1) - R(2, 2)) * 2.0;
    w = (R(2, 1) - R(1, 2)) / s; x = 0.25 * s; y = (R(0, 1) + R(1, 0)) / s; z = (R(0, 2) + R(2, 0)) / s;
  } else if (R(1, 1) > R(2, 2)) {
    const double s = std::sqrt(1.0 + R(1, 1) - R(0, 0) - R(2, 2)) * 2.0;
    w = (R(0, 2) - R(2, 0)) / s; x = (R(0, 1) + R(1, 0)) / s; y = 0.25 * s; z = (R(1, 2) + R(2, 1)) / s;
  } else {
    const double s = std::sqrt(1.0 + R(2, 2) - R(0, 0) - R(1, 1)) * 2.0;
    w = (R(1, 0) - R(0, 1)) / s; x = (R(0, 2) + R(2, 0)) / s; y = (R(1, 2) + R(2, 1)) / s; z = 0.25 * s;
  }
  const double sg = (w < 0.0) ? -1.0 : 1.0;
  q[0] = sg * x; q[1] = sg * y; q[2] = sg * z; q[3] = sg * w;
}

template <class T> int env_step(const Oracle& O, int env, double* root, double* dof, const double* act, double dt,
                                int substeps, const Outputs<T>& o) {
  std::vector<ActorState<T>> st;
  load_env(O, env, root, dof, st);
  int nlinks = 0;
  for (int a = 0; a < O.n_act(env); ++a) nlinks += (int)O.actor_model(env, a).links.size();
  StepOut<T> out;
  out.impulse.assign(nlinks, zero3<T>());
  const T h = T(dt) / T((double)substeps);
  const double* act_env = act + O.jdof_off[env];
  double* cache_env = o.cache + (int64_t)env * O.cache_len;
  std::vector<T> cache(O.cache_len), actv(O.jdof_off[env + 1] - O.jdof_off[env]);
  for (int i = 0; i < O.cache_len; ++i) cache[i] = T(cache_env[i]);
  for (size_t j = 0; j < actv.size(); ++j) actv[j] = T(act_env[j]);
  Controls ctl;
  if (o.pos_target) ctl.pos_target = o.pos_target + O.jdof_off[env];
  if (o.vel_target) ctl.vel_target = o.vel_target + O.jdof_off[env];
  if (o.body_force) ctl.body_force = o.body_force + O.body_off[env] * 6;
  if (o.dof_force) out.dof_force.assign(actv.size(), T(0.0));
  for (int s = 0; s < substeps; ++s) env_substep(O, env, st, actv.data(), h, cache, out, ctl);
  if (o.dof_force)
    for (size_t j = 0; j < actv.size(); ++j) o.dof_force[O.jdof_off[env] + j] = val(out.dof_force[j]);
  if (o.body_state) {
    // poses and velocities of the env's bodies after the step: link origin, link rotation, world
    // angular velocity and the velocity of the link origin
    int64_t b = O.body_off[env];
    for (int a = 0; a < O.n_act(env); ++a) {
      const ModelD& M = O.actor_model(env, a);
      const std::vector<T> gv = gen_velocity(M, st[a]);
      ActorKin<T> K;
      kinematics(M, st[a], gv, K);
      for (size_t l = 0; l < M.links.size(); ++l) {
        if (M.links[l].is_virtual) continue;
        double* bs = o.body_state + b * 13;
        ++b;
        Mat3<double> R;
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) R(i, j) = val(K.R[l](i, j));
        double q[4];
        mat_to_quat(R, q);
        for (int k = 0; k < 3; ++k) bs[k] = val(K.p[l][k]);
        for (int k = 0; k < 4; ++k) bs[3 + k] = q[k];
        for (int i = 0; i < 3; ++i) {
          double wv = 0.0, vv = 0.0;
          for (int j = 0; j < 3; ++j) { wv += R(i, j) * val(K.v[l][j]); vv += R(i, j) * val(K.v[l][3 + j]); }
          bs[7 + i] = vv;
          bs[10 + i] = wv;
        }
      }
    }
  }
  for (int i = 0; i < O.cache_len; ++i) cache_env[i] = val(cache[i]);
  store_env(O, env, st, root, dof);
  if (o.net_force) {
    int li = 0;
    int64_t b = O.body_off[env];
    for (int a = 0; a < O.n_act(env); ++a) {
      const ModelD& M = O.actor_model(env, a);
      for (size_t l = 0; l < M.links.size(); ++l, ++li) {
        if (M.links[l].is_virtual) continue;
        for (int k = 0; k < 3; ++k) o.net_force[b * 3 + k] = val(out.impulse[li][k]) / dt;
        ++b;
      }
    }
  }
  if (o.contacts) {
    int32_t* c = o.contacts + (int64_t)env * O.max_contact_cap * 3;
    for (int i = 0; i < O.max_contact_cap * 3; ++i) c[i] = -1;
    for (size_t i = 0; i < out.last_contacts.size(); ++i) {
      c[i * 3 + 0] = out.last_contacts[i].shape_a;
      c[i * 3 + 1] = out.last_contacts[i].shape_b;
      c[i * 3 + 2] = out.last_contacts[i].slot;
    }
  }
  if (o.n_contacts) o.n_contacts[env] = (int32_t)out.last_contacts.size();
  if (o.sig) o.sig[env] = out.sig;
  if (o.status) o.status[env] = out.ok ? 0 : 1;
  return out.ok ? 0 : 1;
}

// ------------------------------------------------------------------------------------------------
// Contact-free RK4 (test integrator for the energy and momentum pins). The state derivative of a
// free root: p_dot = v_root, quat_dot = 0.5 [omega; 0] * quat, omega_dot = a_ang,
// v_root_dot = a_lin + omega x v_root (a = world spatial acceleration at the root origin).
template <class T> void deriv(const ModelD& M, const ActorState<T>& s, const std::vector<T>& tau_j, const Params& P,
                              ActorState<T>& ds) {
  const std::vector<T> gv = gen_velocity(M, s);
  ActorKin<T> K;
  kinematics(M, s, gv, K);
  std::vector<T> tau(M.n_gen, T(0.0)), qdd;
  for (size_t l = 0; l < M.links.size(); ++l)
    if (M.jdof[l] >= 0) tau[M.goff[l]] = tau_j[M.jdof[l]] - T(M.links[l].damping) * s.qd[M.jdof[l]];
  aba(M, K, tau, P, qdd);
  ds = s;
  if (M.free_root) {
    ds.p = s.v;
    const T wq[4] = {s.w[0], s.w[1], s.w[2], T(0.0)};
    T qd[4];
    quat_mul(wq, s.quat, qd);
    for (int k = 0; k < 4; ++k) ds.quat[k] = qd[k] * T(0.5);
    ds.w = mk3<T>(qdd[0], qdd[1], qdd[2]);
    ds.v = add(mk3<T>(qdd[3], qdd[4], qdd[5]), cross(s.w, s.v));
  } else {
    ds.p = zero3<T>();
    for (int k = 0; k < 4; ++k) ds.quat[k] = T(0.0);
    ds.w = zero3<T>();
    ds.v = zero3<T>();
  }
  for (size_t l = 0; l < M.links.size(); ++l)
    if (M.jdof[l] >= 0) {
      ds.q[M.jdof[l]] = s.qd[M.jdof[l]];
      ds.qd[M.jdof[l]] = qdd[M.goff[l]];
    }
}
template <class T> ActorState<T> axpy_state(const ActorState<T>& s, const ActorState<T>& d, const T& h) {
  ActorState<T> o = s;
  o.p = add(s.p, scale(d.p, h));
  for (int k = 0; k < 4; ++k) o.quat[k] = s.quat[k] + d.quat[k] * h;
  o.w = add(s.w, scale(d.w, h));
  o.v = add(s.v, scale(d.v, h));
  for (size_t j = 0; j < s.q.size(); ++j) { o.q[j] = s.q[j] + d.q[j] * h; o.qd[j] = s.qd[j] + d.qd[j] * h; }
  return o;
}

}  // namespace orc

namespace orc {

template <class D> int32_t step_tangent_t(void* h, double* root, double* dof, double* cache, const double* act,
                                         double* droot, double* ddof, double* dcache, const double* dact, double dt,
                                         int32_t substeps, int32_t n_threads, const double* pos_target = nullptr,
                                         const double* vel_target = nullptr, const double* body_force = nullptr) {
  const Oracle* O = (const Oracle*)h;
  std::atomic<int> bad{0};
  if (n_threads < 1) n_threads = 1;
  auto one = [&](int env) {
    Controls ctl;  // the env's drive targets and body forces (constants of the derivative; zero when absent)
    if (pos_target) ctl.pos_target = pos_target + O->jdof_off[env];
    if (vel_target) ctl.vel_target = vel_target + O->jdof_off[env];
    if (body_force) ctl.body_force = body_force + O->body_off[env] * 6;
    std::vector<ActorState<D>> st;
    load_env(*O, env, root, dof, st);
    int64_t jd = O->jdof_off[env];
    for (int a = 0; a < O->n_act(env); ++a) {
      const double* dr = droot + (int64_t)(O->actor_off[env] + a) * 13;
      ActorState<D>& x = st[a];
      for (int k = 0; k < 3; ++k) { x.p[k].d = dr[k]; x.v[k].d = dr[7 + k]; x.w[k].d = dr[10 + k]; }
      for (int k = 0; k < 4; ++k) x.quat[k].d = dr[3 + k];
      for (size_t j = 0; j < x.q.size(); ++j) { x.q[j].d = ddof[(jd + j) * 2]; x.qd[j].d = ddof[(jd + j) * 2 + 1]; }
      jd += (int64_t)x.q.size();
    }
    int nlinks = 0;
    for (int a = 0; a < O->n_act(env); ++a) nlinks += (int)O->actor_model(env, a).links.size();
    StepOut<D> out;
    out.impulse.assign(nlinks, zero3<D>());
    const D hs = D(dt) / D((double)substeps);
    const int64_t j0 = O->jdof_off[env], nj = O->jdof_off[env + 1] - j0;
    std::vector<D> actv(nj), cv(O->cache_len);
    for (int64_t j = 0; j < nj; ++j) { actv[j] = D(act[j0 + j]); actv[j].d = dact[j0 + j]; }
    double* c_env = cache + (int64_t)env * O->cache_len;
    double* dc_env = dcache + (int64_t)env * O->cache_len;
    for (int i = 0; i < O->cache_len; ++i) { cv[i] = D(c_env[i]); cv[i].d = dc_env[i]; }
    for (int s = 0; s < substeps; ++s) env_substep(*O, env, st, actv.data(), hs, cv, out, ctl);
    for (int i = 0; i < O->cache_len; ++i) { c_env[i] = (double)cv[i].v; dc_env[i] = (double)cv[i].d; }
    store_env(*O, env, st, root, dof);
    jd = O->jdof_off[env];
    for (int a = 0; a < O->n_act(env); ++a) {
      double* dr = droot + (int64_t)(O->actor_off[env] + a) * 13;
      const ActorState<D>& x = st[a];
      for (int k = 0; k < 3; ++k) { dr[k] = (double)x.p[k].d; dr[7 + k] = (double)x.v[k].d; dr[10 + k] = (double)x.w[k].d; }
      for (int k = 0; k < 4; ++k) dr[3 + k] = (double)x.quat[k].d;
      for (size_t j = 0; j < x.q.size(); ++j) { ddof[(jd + j) * 2] = (double)x.q[j].d; ddof[(jd + j) * 2 + 1] = (double)x.qd[j].d; }
      jd += (int64_t)x.q.size();
    }
    if (!out.ok) bad++;
  };
  auto work = [&](int t) {
    for (int e = t; e < O->n_envs; e += n_threads) one(e);
  };
  if (n_threads == 1) work(0);
  else {
    std::vector<std::thread> th;
    for (int t = 0; t < n_threads; ++t) th.emplace_back(work, t);
    for (auto& x : th) x.join();
  }
  return bad.load();
}

}  // namespace orc

// ==================================================================================================
// C entry points (ctypes).
using namespace orc;

extern "C" {

struct OracleModels {
  int32_t n_models;
  const int32_t* link_off;   // [n_models + 1]
  const int32_t* shape_off;  // [n_models + 1]
  const int32_t* parent;
  const int32_t* jtype;
  const double* axis;
  const double* ppos;
  const double* pquat;
  const double* mass;
  const double* com;
  const double* inertia;
  const double* armature;
  const double* damping;
  const double* lo;
  const double* hi;
  const int32_t* has_limit;
  const int32_t* is_virtual;
  const int32_t* shape_link;
  const int32_t* shape_type;
  const double* shape_size;
  const double* shape_pos;
  const double* shape_quat;
  const double* shape_friction;
  const double* drive_kp;  // [links] or null (no drives)
  const double* drive_kd;  // [links] or null
  // fixed tendons (all null: none): model m owns tendons tendon_off[m] .. tendon_off[m+1]-1,
  // tendon t owns entries entry_off[t] .. entry_off[t+1]-1 (model-local link, coefficient)
  const int32_t* tendon_off;
  const int32_t* tendon_entry_off;
  const int32_t* tendon_link;
  const double* tendon_coef;
  const double* tendon_stiffness;
  const double* tendon_damping;
  const double* tendon_rest;
  const double* tendon_lo;
  const double* tendon_hi;
  const int32_t* tendon_has_limit;
};
struct OracleParams {
  double gravity[3];
  int32_t pos_iters, vel_iters;
  double contact_offset, limit_margin, bias_coef, max_depen_vel, ground_friction;
};

void* oracle_create(const OracleModels* md, const int32_t* env_actor_model, int32_t actors_per_env, int32_t n_envs,
                    const OracleParams* p) {
  Oracle* O = new Oracle();
  for (int m = 0; m < md->n_models; ++m) {
    ModelD M;
    for (int i = md->link_off[m]; i < md->link_off[m + 1]; ++i) {
      LinkD L;
      L.parent = md->parent[i];
      L.jtype = md->jtype[i];
      for (int k = 0; k < 3; ++k) { L.axis[k] = md->axis[3 * i + k]; L.ppos[k] = md->ppos[3 * i + k]; L.com[k] = md->com[3 * i + k]; }
      for (int k = 0; k < 4; ++k) L.pquat[k] = md->pquat[4 * i + k];
      for (int k = 0; k < 6; ++k) L.inertia[k] = md->inertia[6 * i + k];
      L.mass = md->mass[i];
      L.armature = md->armature[i];
      L.damping = md->damping[i];
      L.lo = md->lo[i];
      L.hi = md->hi[i];
      L.has_limit = md->has_limit[i];
      L.is_virtual = md->is_virtual[i];
      L.kp = md->drive_kp ? md->drive_kp[i] : 0.0;
      L.kd = md->drive_kd ? md->drive_kd[i] : 0.0;
      M.links.push_back(L);
    }
    for (int s = md->shape_off[m]; s < md->shape_off[m + 1]; ++s) {
      ShapeD S;
      S.link = md->shape_link[s];
      S.type = md->shape_type[s];
      for (int k = 0; k < 3; ++k) { S.size[k] = md->shape_size[3 * s + k]; S.pos[k] = md->shape_pos[3 * s + k]; }
      for (int k = 0; k < 4; ++k) S.quat[k] = md->shape_quat[4 * s + k];
      S.friction = md->shape_friction[s];
      M.shapes.push_back(S);
      M.contact_cap += (S.type == SHAPE_SPHERE) ? 1 : (S.type == SHAPE_CAPSULE ? 2 : 8);
    }
    const int L = (int)M.links.size();
    M.ndof.assign(L, 0);
    M.goff.assign(L, 0);
    M.jdof.assign(L, -1);
    int g = 0, j = 0;
    for (int i = 0; i < L; ++i) {
      const int jt = M.links[i].jtype;
      M.goff[i] = g;
      if (i == 0 && jt == JOINT_FREE) { M.ndof[i] = 6; M.free_root = true; }
      else if (jt == JOINT_REVOLUTE || jt == JOINT_PRISMATIC) { M.ndof[i] = 1; M.jdof[i] = j++; }
      else if (jt == JOINT_SPHERICAL && i > 0) { M.ndof[i] = 3; M.jdof[i] = j; j += 3; }
      g += M.ndof[i];
      if (!M.links[i].is_virtual) M.n_body++;
    }
    M.n_gen = g;
    M.n_jdof = j;
    if (md->tendon_off)
      for (int t = md->tendon_off[m]; t < md->tendon_off[m + 1]; ++t) {
        TendonD td;
        for (int e = md->tendon_entry_off[t]; e < md->tendon_entry_off[t + 1]; ++e) {
          td.links.push_back(md->tendon_link[e]);
          td.coef.push_back(md->tendon_coef[e]);
        }
        td.stiffness = md->tendon_stiffness[t];
        td.damping = md->tendon_damping[t];
        td.rest = md->tendon_rest[t];
        td.lo = md->tendon_lo[t];
        td.hi = md->tendon_hi[t];
        td.has_limit = md->tendon_has_limit[t];
        M.tendons.push_back(td);
      }
    O->models.push_back(M);
  }
  O->n_envs = n_envs;
  O->env_actors.assign(n_envs, {});
  O->actor_off.assign(n_envs + 1, 0);
  for (int e = 0; e < n_envs; ++e) {
    for (int a = 0; a < actors_per_env; ++a) {
      const int m = env_actor_model[(int64_t)e * actors_per_env + a];
      if (m >= 0) O->env_actors[e].push_back(m);  // -1 pads envs with fewer actors
    }
    O->actor_off[e + 1] = O->actor_off[e] + (int64_t)O->env_actors[e].size();
  }
  // shape-shape candidate pairs of every env: (a < b), different actors, capsule vs box
  O->env_pairs.assign(n_envs, {});
  for (int e = 0; e < n_envs; ++e) {
    std::vector<std::pair<int, int>> shp;  // (actor, type) per env-local shape
    for (int a = 0; a < O->n_act(e); ++a)
      for (const ShapeD& s : O->actor_model(e, a).shapes) shp.push_back({a, s.type});
    for (int sa = 0; sa < (int)shp.size(); ++sa)
      for (int sb = sa + 1; sb < (int)shp.size(); ++sb) {
        if (shp[sa].first == shp[sb].first) continue;
        const int ta = shp[sa].second, tb = shp[sb].second;
        if ((ta == SHAPE_CAPSULE && tb == SHAPE_BOX) || (ta == SHAPE_BOX && tb == SHAPE_CAPSULE))
          O->env_pairs[e].push_back({sa, sb});
      }
  }
  std::memcpy(O->prm.gravity, p->gravity, sizeof(double) * 3);
  O->prm.pos_iters = p->pos_iters;
  O->prm.vel_iters = p->vel_iters;
  O->prm.contact_offset = p->contact_offset;
  O->prm.limit_margin = p->limit_margin;
  O->prm.bias_coef = p->bias_coef;
  O->prm.max_depen_vel = p->max_depen_vel;
  O->prm.ground_friction = p->ground_friction;
  O->jdof_off.assign(n_envs + 1, 0);
  O->body_off.assign(n_envs + 1, 0);
  O->n_gen.assign(n_envs, 0);
  O->contact_cap.assign(n_envs, 0);
  for (int e = 0; e < n_envs; ++e) {
    int jd = 0, nb = 0, ng = 0, nt = 0, cc = kPairSlots * (int)O->env_pairs[e].size();
    for (int a = 0; a < O->n_act(e); ++a) {
      const ModelD& M = O->actor_model(e, a);
      jd += M.n_jdof; nb += M.n_body; ng += M.n_gen; cc += M.contact_cap; nt += (int)M.tendons.size();
    }
    O->jdof_off[e + 1] = O->jdof_off[e] + jd;
    O->body_off[e + 1] = O->body_off[e] + nb;
    O->n_gen[e] = ng;
    O->contact_cap[e] = cc;
    O->max_contact_cap = std::max(O->max_contact_cap, cc);
    O->max_gen = std::max(O->max_gen, ng);
    O->cache_len = std::max(O->cache_len, 3 * cc + 2 * jd + 2 * nt);
  }
  O->N_A = O->actor_off[n_envs];
  O->N_D = O->jdof_off[n_envs];
  O->N_B = O->body_off[n_envs];
  return O;
}

void oracle_destroy(void* h) { delete (Oracle*)h; }

// out: N_A, N_D, N_B, max contact capacity per env, max generalized DOFs per env, impulse-cache
// length per env
void oracle_sizes(void* h, int64_t* out) {
  const Oracle* O = (const Oracle*)h;
  out[0] = O->N_A; out[1] = O->N_D; out[2] = O->N_B; out[3] = O->max_contact_cap; out[4] = O->max_gen;
  out[5] = O->cache_len;
}
int32_t oracle_env_ngen(void* h, int32_t env) { return ((const Oracle*)h)->n_gen[env]; }

// One env-step (substeps substeps of dt/substeps) for every env, in place on root/dof. Returns
// the number of envs whose step failed (non-SPD articulated inertia or mass matrix).
int32_t oracle_step(void* h, double* root, double* dof, double* cache, const double* act, double dt, int32_t substeps,
                    double* net_force, int32_t* contacts, int32_t* n_contacts, uint32_t* sig, int32_t n_threads) {
  const Oracle* O = (const Oracle*)h;
  Outputs<double> o{cache, net_force, contacts, n_contacts, sig, nullptr};
  std::atomic<int> bad{0};
  if (n_threads < 1) n_threads = 1;
  auto work = [&](int t) {
    for (int e = t; e < O->n_envs; e += n_threads)
      if (env_step<double>(*O, e, root, dof, act, dt, substeps, o)) bad++;
  };
  if (n_threads == 1) work(0);
  else {
    std::vector<std::thread> th;
    for (int t = 0; t < n_threads; ++t) th.emplace_back(work, t);
    for (auto& x : th) x.join();
  }
  return bad.load();
}

// The step with the per-step controls and outputs beyond oracle_step: drive targets (N_D each, or
// null = 0), external body forces and torques (N_B x 6, world axes at the COM, or null), the joint
// force of the last substep (N_D, or null) and body states after the step (N_B x 13, or null).
int32_t oracle_step_ext(void* h, double* root, double* dof, double* cache, const double* act, const double* pos_target,
                        const double* vel_target, const double* body_force, double dt, int32_t substeps,
                        double* net_force, double* dof_force, double* body_state, int32_t* contacts,
                        int32_t* n_contacts, uint32_t* sig, int32_t n_threads) {
  const Oracle* O = (const Oracle*)h;
  Outputs<double> o{cache, net_force, contacts, n_contacts, sig, nullptr};
  o.pos_target = pos_target; o.vel_target = vel_target; o.body_force = body_force;
  o.dof_force = dof_force; o.body_state = body_state;
  std::atomic<int> bad{0};
  if (n_threads < 1) n_threads = 1;
  auto work = [&](int t) {
    for (int e = t; e < O->n_envs; e += n_threads)
      if (env_step<double>(*O, e, root, dof, act, dt, substeps, o)) bad++;
  };
  if (n_threads == 1) work(0);
  else {
    std::vector<std::thread> th;
    for (int t = 0; t < n_threads; ++t) th.emplace_back(work, t);
    for (auto& x : th) x.join();
  }
  return bad.load();
}

// Same step evaluated with the operation-counting scalar; returns the floating-point operations
// (add, sub, mul, div, sqrt, sin, cos) it performed. State is advanced like oracle_step.
double oracle_step_flops(void* h, double* root, double* dof, double* cache, const double* act, double dt,
                         int32_t substeps) {
  const Oracle* O = (const Oracle*)h;
  OpCount::reset();
  Outputs<OpCount> o{cache, nullptr, nullptr, nullptr, nullptr, nullptr};
  for (int e = 0; e < O->n_envs; ++e) env_step<OpCount>(*O, e, root, dof, act, dt, substeps, o);
  return (double)OpCount::count();
}

// The same step evaluated with forward-mode dual numbers: root, dof and cache advance like
// oracle_step, and droot, ddof, dcache (same layouts) carry the input tangent in and the output
// tangent out, with dact the actuation tangent. The derivative is exact for the discrete FP64 step
// with its constraint and active sets held at the values' choices. Returns the failed-env count.
int32_t oracle_step_tangent(void* h, double* root, double* dof, double* cache, const double* act, double* droot,
                            double* ddof, double* dcache, const double* dact, double dt, int32_t substeps,
                            int32_t n_threads, const double* pos_target, const double* vel_target,
                            const double* body_force) {
  return step_tangent_t<Dual>(h, root, dof, cache, act, droot, ddof, dcache, dact, dt, substeps, n_threads, pos_target,
                              vel_target, body_force);
}

// The same derivative evaluated in single precision (conditioning probe for the GPU derivative).
int32_t oracle_step_tangent_f32(void* h, double* root, double* dof, double* cache, const double* act,
                                double* droot, double* ddof, double* dcache, const double* dact, double dt,
                                int32_t substeps, const double* pos_target, const double* vel_target,
                                const double* body_force) {
  return step_tangent_t<DualF>(h, root, dof, cache, act, droot, ddof, dcache, dact, dt, substeps, 1, pos_target,
                               vel_target, body_force);
}

// The same step evaluated in single precision (a conditioning probe for the parity tests: it
// shows how far a plain FP32 evaluation of the identical algorithm lands from the FP64 result).
int32_t oracle_step_f32(void* h, double* root, double* dof, double* cache, const double* act, double dt,
                        int32_t substeps, double* net_force) {
  const Oracle* O = (const Oracle*)h;
  Outputs<float> o{cache, net_force, nullptr, nullptr, nullptr, nullptr};
  int bad = 0;
  for (int e = 0; e < O->n_envs; ++e) bad += env_step<float>(*O, e, root, dof, act, dt, substeps, o);
  return bad;
}

// Capsule-box geometry for the pins, in the box frame: segment p0 -> p1, radius r, half extents e.
// out[0] = t* (closest point of the segment); then for t = 0, 1, t*: n (3), d, x (3); out[22] = 1 if
// the face clip is non-empty, out[23], out[24] = its ends.
void oracle_capsule_box(const double* p0, const double* p1, double r, const double* e, double* out) {
  const Vec3<double> a = vec3_of<double>(p0), b = vec3_of<double>(p1), ext = vec3_of<double>(e);
  const Vec3<double> dv = sub(b, a);
  const double ts = segment_box_closest_t(a, dv, ext);
  out[0] = ts;
  double ta = 0.0, tb = 0.0;
  out[22] = face_clip(a, dv, ext, r, ts, ta, tb) ? 1.0 : 0.0;
  out[23] = ta;
  out[24] = tb;
  const double tt[3] = {0.0, 1.0, ts};
  for (int s = 0; s < 3; ++s) {
    Vec3<double> n, x;
    double d;
    sphere_box(add(a, scale(dv, tt[s])), r, ext, n, d, x);
    double* o = out + 1 + 7 * s;
    for (int k = 0; k < 3; ++k) { o[k] = n[k]; o[4 + k] = x[k]; }
    o[3] = d;
  }
}

// --- single-env helpers for the pins. root/dof point at this env's rows (actors_per_env x 13 and
// its joint DOFs x 2); generalized vectors are env-level ([free root 6] + joints, actor by actor).
static void env_kin(const Oracle& O, int env, const double* root, const double* dof, std::vector<ActorState<double>>& st,
                    std::vector<ActorKin<double>>& K, std::vector<std::vector<double>>& gv) {
  // load from env-local pointers: build a temporary view with offset 0
  st.resize(O.n_act(env));
  int jd = 0;
  for (int a = 0; a < O.n_act(env); ++a) {
    const ModelD& M = O.actor_model(env, a);
    const double* r = root + a * 13;
    ActorState<double>& s = st[a];
    s.p = vec3_of<double>(r);
    for (int k = 0; k < 4; ++k) s.quat[k] = r[3 + k];
    s.v = vec3_of<double>(r + 7);
    s.w = vec3_of<double>(r + 10);
    s.q.assign(M.n_jdof, 0.0);
    s.qd.assign(M.n_jdof, 0.0);
    for (int j = 0; j < M.n_jdof; ++j) { s.q[j] = dof[(jd + j) * 2]; s.qd[j] = dof[(jd + j) * 2 + 1]; }
    jd += M.n_jdof;
  }
  K.resize(O.n_act(env));
  gv.resize(O.n_act(env));
  for (int a = 0; a < O.n_act(env); ++a) {
    gv[a] = gen_velocity(O.actor_model(env, a), st[a]);
    kinematics(O.actor_model(env, a), st[a], gv[a], K[a]);
  }
}

int32_t oracle_aba(void* h, int32_t env, const double* root, const double* dof, const double* tau, double* qdd) {
  const Oracle& O = *(const Oracle*)h;
  std::vector<ActorState<double>> st; std::vector<ActorKin<double>> K; std::vector<std::vector<double>> gv;
  env_kin(O, env, root, dof, st, K, gv);
  const EnvLayout E = env_layout(O, env);
  for (int a = 0; a < O.n_act(env); ++a) {
    const ModelD& M = O.actor_model(env, a);
    std::vector<double> t(tau + E.gen_off[a], tau + E.gen_off[a] + M.n_gen), q;
    if (!aba(M, K[a], t, O.prm, q)) return 1;
    for (int i = 0; i < M.n_gen; ++i) qdd[E.gen_off[a] + i] = q[i];
  }
  return 0;
}

int32_t oracle_crba(void* h, int32_t env, const double* root, const double* dof, double* Hout) {
  const Oracle& O = *(const Oracle*)h;
  std::vector<ActorState<double>> st; std::vector<ActorKin<double>> K; std::vector<std::vector<double>> gv;
  env_kin(O, env, root, dof, st, K, gv);
  const EnvLayout E = env_layout(O, env);
  const int n = E.n_gen;
  for (int i = 0; i < n * n; ++i) Hout[i] = 0.0;
  for (int a = 0; a < O.n_act(env); ++a) {
    const ModelD& M = O.actor_model(env, a);
    std::vector<double> H;
    crba(M, K[a], H);
    for (int i = 0; i < M.n_gen; ++i)
      for (int j = 0; j < M.n_gen; ++j) Hout[(E.gen_off[a] + i) * n + E.gen_off[a] + j] = H[i * M.n_gen + j];
  }
  return 0;
}

int32_t oracle_rnea(void* h, int32_t env, const double* root, const double* dof, const double* qdd, double* tau) {
  const Oracle& O = *(const Oracle*)h;
  std::vector<ActorState<double>> st; std::vector<ActorKin<double>> K; std::vector<std::vector<double>> gv;
  env_kin(O, env, root, dof, st, K, gv);
  const EnvLayout E = env_layout(O, env);
  for (int a = 0; a < O.n_act(env); ++a) {
    const ModelD& M = O.actor_model(env, a);
    std::vector<double> q(qdd + E.gen_off[a], qdd + E.gen_off[a] + M.n_gen), t;
    rnea(M, K[a], q, O.prm, t);
    for (int i = 0; i < M.n_gen; ++i) tau[E.gen_off[a] + i] = t[i];
  }
  return 0;
}

// out[0] = kinetic energy (incl. armature), out[1] = gravitational potential energy.
int32_t oracle_energy(void* h, int32_t env, const double* root, const double* dof, double* out) {
  const Oracle& O = *(const Oracle*)h;
  std::vector<ActorState<double>> st; std::vector<ActorKin<double>> K; std::vector<std::vector<double>> gv;
  env_kin(O, env, root, dof, st, K, gv);
  const Vec3<double> g = mk3<double>(O.prm.gravity[0], O.prm.gravity[1], O.prm.gravity[2]);
  double T = 0.0, V = 0.0;
  for (int a = 0; a < O.n_act(env); ++a) {
    const ModelD& M = O.actor_model(env, a);
    for (size_t i = 0; i < M.links.size(); ++i) {
      T += 0.5 * sdot(K[a].v[i], smul(K[a].I[i], K[a].v[i]));
      for (int k = 0; k < M.ndof[i] && M.jdof[i] >= 0; ++k)
        T += 0.5 * M.links[i].armature * st[a].qd[M.jdof[i] + k] * st[a].qd[M.jdof[i] + k];
      const Vec3<double> c = add(K[a].p[i], mul(K[a].R[i], vec3_of<double>(M.links[i].com)));
      V -= M.links[i].mass * dot(g, c);
    }
  }
  out[0] = T;
  out[1] = V;
  return 0;
}

// Total spatial momentum about the world origin (world axes), and its rate of change for the
// generalized acceleration qdd (out[0..5] = h, out[6..11] = h_dot).
int32_t oracle_momentum(void* h, int32_t env, const double* root, const double* dof, const double* qdd, double* out) {
  const Oracle& O = *(const Oracle*)h;
  std::vector<ActorState<double>> st; std::vector<ActorKin<double>> K; std::vector<std::vector<double>> gv;
  env_kin(O, env, root, dof, st, K, gv);
  const EnvLayout E = env_layout(O, env);
  SVec<double> hm = szero<double>(), hd = szero<double>();
  for (int a = 0; a < O.n_act(env); ++a) {
    const ModelD& M = O.actor_model(env, a);
    const int L = (int)M.links.size();
    std::vector<SVec<double>> acc(L);
    for (int i = 0; i < L; ++i) {
      SVec<double> aJ = szero<double>();
      for (size_t k = 0; k < K[a].S[i].size(); ++k) aJ = sadd(aJ, sscale(K[a].S[i][k], qdd[E.gen_off[a] + M.goff[i] + k]));
      acc[i] = sadd(aJ, K[a].c[i]);
      if (M.links[i].parent >= 0) acc[i] = sadd(acc[i], smul(K[a].Xup[i], acc[M.links[i].parent]));
      // link -> world force transform is (i_X_0)^T with i_X_0 = plux(R_i^T, p_i)
      const SMat<double> XT = stranspose(plux<double>(transpose(K[a].R[i]), K[a].p[i]));
      const SVec<double> hi = smul(K[a].I[i], K[a].v[i]);
      hm = sadd(hm, smul(XT, hi));
      hd = sadd(hd, smul(XT, sadd(smul(K[a].I[i], acc[i]), smul(crf(K[a].v[i]), hi))));
    }
  }
  for (int k = 0; k < 6; ++k) { out[k] = hm[k]; out[6 + k] = hd[k]; }
  return 0;
}

// Contact-free RK4 steps of every env (tau = act - damping * qd), in place.
int32_t oracle_rk4(void* h, double* root, double* dof, const double* act, double dt, int32_t nsteps) {
  const Oracle& O = *(const Oracle*)h;
  // the reference integrator advances joint positions by q_dot = qd: hinges and sliders only
  for (const ModelD& M : O.models)
    for (int nd : M.ndof)
      if (nd == 3) return -2;
  for (int e = 0; e < O.n_envs; ++e) {
    std::vector<ActorState<double>> st;
    load_env(O, e, root, dof, st);
    int jb = 0;
    for (int a = 0; a < O.n_act(e); ++a) {
      const ModelD& M = O.actor_model(e, a);
      std::vector<double> tj(act + O.jdof_off[e] + jb, act + O.jdof_off[e] + jb + M.n_jdof);
      for (int s = 0; s < nsteps; ++s) {
        ActorState<double> k1, k2, k3, k4;
        deriv(M, st[a], tj, O.prm, k1);
        deriv(M, axpy_state(st[a], k1, 0.5 * dt), tj, O.prm, k2);
        deriv(M, axpy_state(st[a], k2, 0.5 * dt), tj, O.prm, k3);
        deriv(M, axpy_state(st[a], k3, dt), tj, O.prm, k4);
        ActorState<double> n = st[a];
        n = axpy_state(n, k1, dt / 6.0);
        n = axpy_state(n, k2, dt / 3.0);
        n = axpy_state(n, k3, dt / 3.0);
        n = axpy_state(n, k4, dt / 6.0);
        const double nr = std::sqrt(n.quat[0] * n.quat[0] + n.quat[1] * n.quat[1] + n.quat[2] * n.quat[2] + n.quat[3] * n.quat[3]);
        for (int k = 0; k < 4; ++k) n.quat[k] /= nr;
        st[a] = n;
      }
      jb += M.n_jdof;
    }
    store_env(O, e, st, root, dof);
  }
  return 0;
}

// World pose of env link `link` (actor-major numbering): out = R (9, row-major) then p (3).
int32_t oracle_link_pose(void* h, int32_t env, const double* root, const double* dof, int32_t link, double* out) {
  const Oracle& O = *(const Oracle*)h;
  std::vector<ActorState<double>> st; std::vector<ActorKin<double>> K; std::vector<std::vector<double>> gv;
  env_kin(O, env, root, dof, st, K, gv);
  int l = link;
  for (int a = 0; a < O.n_act(env); ++a) {
    const int L = (int)O.actor_model(env, a).links.size();
    if (l < L) {
      for (int k = 0; k < 9; ++k) out[k] = K[a].R[l].e[k];
      for (int k = 0; k < 3; ++k) out[9 + k] = K[a].p[l][k];
      return 0;
    }
    l -= L;
  }
  return 1;
}

// World-axis Jacobian of env-local link `link` (6 x the env's generalized DOFs, row-major; env-local
// root and DOF arrays as for oracle_link_pose): rows [angular velocity; velocity of the link
// origin] as a linear map of the env's generalized velocity. Column g is the link's velocity for a
// unit generalized velocity g, by the same outward recursion as the state's velocities.
int32_t oracle_jacobian(void* h, int32_t env, const double* root, const double* dof, int32_t link, double* out) {
  const Oracle& O = *(const Oracle*)h;
  std::vector<ActorState<double>> st; std::vector<ActorKin<double>> K; std::vector<std::vector<double>> gv;
  env_kin(O, env, root, dof, st, K, gv);
  const EnvLayout E = env_layout(O, env);
  const int n = E.n_gen;
  for (int i = 0; i < 6 * n; ++i) out[i] = 0.0;
  int l = link;
  for (int a = 0; a < O.n_act(env); ++a) {
    const ModelD& M = O.actor_model(env, a);
    const int L = (int)M.links.size();
    if (l >= L) { l -= L; continue; }
    for (int g = 0; g < M.n_gen; ++g) {
      std::vector<SVec<double>> v(L);
      for (int i = 0; i < L; ++i) {
        SVec<double> vJ = szero<double>();
        for (size_t k = 0; k < K[a].S[i].size(); ++k)
          if (M.goff[i] + (int)k == g) vJ = sadd(vJ, K[a].S[i][k]);
        v[i] = (i == 0) ? vJ : sadd(smul(K[a].Xup[i], v[M.links[i].parent]), vJ);
      }
      for (int r = 0; r < 3; ++r) {
        double wv = 0.0, vv = 0.0;
        for (int c = 0; c < 3; ++c) { wv += K[a].R[l](r, c) * v[l][c]; vv += K[a].R[l](r, c) * v[l][3 + c]; }
        out[r * n + E.gen_off[a] + g] = wv;
        out[(3 + r) * n + E.gen_off[a] + g] = vv;
      }
    }
    return 0;
  }
  return -1;
}

// Constraint rows of one env at the given configuration (no solve). Returns the row count R (or
// -1 if cap is too small). J is R x n_gen; kind: 0 limit, 1 normal, 2 friction; link is the env
// link (actor-major) the row acts on (-1 for limits); x, k: contact point and direction.
int32_t oracle_rows(void* h, int32_t env, const double* root, const double* dof, int32_t cap, double* J, double* d,
                    int32_t* kind, int32_t* link, double* x, double* k, double* A, int32_t* info) {
  const Oracle& O = *(const Oracle*)h;
  std::vector<ActorState<double>> st; std::vector<ActorKin<double>> K; std::vector<std::vector<double>> gv;
  env_kin(O, env, root, dof, st, K, gv);
  const EnvLayout E = env_layout(O, env);
  std::vector<ContactPt<double>> C;
  env_contacts(O, env, K, C);
  std::vector<Row<double>> rows;
  build_rows(O, env, E, st, K, C, rows, nullptr);
  if ((int)rows.size() > cap) return -1;
  const int n = E.n_gen;
  std::vector<double> Mfull(n * n, 0.0);
  for (int a = 0; a < O.n_act(env); ++a) {
    const ModelD& M = O.actor_model(env, a);
    std::vector<double> H;
    crba(M, K[a], H);
    for (int i = 0; i < M.n_gen; ++i)
      for (int j = 0; j < M.n_gen; ++j) Mfull[(E.gen_off[a] + i) * n + E.gen_off[a] + j] = H[i * M.n_gen + j];
  }
  if (n > 0) cholesky_factor(Mfull, n);
  std::vector<int> link_base(O.n_act(env), 0);
  int lb = 0;
  for (int a = 0; a < O.n_act(env); ++a) { link_base[a] = lb; lb += (int)O.actor_model(env, a).links.size(); }
  for (size_t r = 0; r < rows.size(); ++r) {
    for (int i = 0; i < n; ++i) J[r * n + i] = rows[r].J[i];
    std::vector<double> w = rows[r].J;
    if (n > 0) cholesky_solve(Mfull, n, w.data());
    double a = 0.0;
    for (int i = 0; i < n; ++i) a += rows[r].J[i] * w[i];
    A[r] = a;
    d[r] = rows[r].d;
    kind[r] = rows[r].kind;
    if (rows[r].contact >= 0) {
      const ContactPt<double>& c = C[rows[r].contact];
      link[r] = link_base[c.actor_a] + c.link_a;
      for (int m = 0; m < 3; ++m) { x[r * 3 + m] = c.x[m]; k[r * 3 + m] = rows[r].k[m]; }
      info[r * 3 + 0] = c.shape_a; info[r * 3 + 1] = c.shape_b; info[r * 3 + 2] = c.slot;
    } else {
      link[r] = -1;
      for (int m = 0; m < 3; ++m) { x[r * 3 + m] = 0.0; k[r * 3 + m] = 0.0; info[r * 3 + m] = -1; }
    }
  }
  return (int32_t)rows.size();
}

// Operation count of one primitive evaluated on the counting scalar (the pins of the counter
// itself): which = 0..7 one add, sub, mul, div, sqrt, sin, cos, atan2; 8 a negation; 9 fabs; 10 a
// comparison; 20 dot; 21 cross; 22 3x3 matrix times vector; 23 3x3 matrix product; 24 quaternion
// product; 25 quaternion exponential of a rotation vector of length 0.3; 26 6x6 matrix times
// spatial vector; 27 6x6 matrix product; 28 spatial dot product; 29 Cholesky factor of an n x n SPD
// matrix; 30 the two triangular solves with that factor. Returns -1 for an unknown `which`.
double oracle_opcount_probe(int32_t which, int32_t n) {
  using C = OpCount;
  const C a(0.7), b(1.3);
  Vec3<C> u = mk3<C>(C(0.1), C(0.2), C(0.3)), w = mk3<C>(C(-0.4), C(0.5), C(0.6));
  Mat3<C> R, S;
  SMat<C> X, Y;
  SVec<C> sv;
  for (int i = 0; i < 9; ++i) { R.e[i] = C(0.1 * i + 0.05); S.e[i] = C(0.3 - 0.02 * i); }
  for (int i = 0; i < 36; ++i) { X.e[i] = C(0.01 * i); Y.e[i] = C(0.5 - 0.01 * i); }
  for (int i = 0; i < 6; ++i) sv[i] = C(0.2 * i - 0.4);
  const C q1[4] = {C(0.1), C(0.2), C(0.3), C(0.9)}, q2[4] = {C(-0.2), C(0.1), C(0.4), C(0.8)};
  C qo[4];
  // SPD matrix for the Cholesky probes: n I + (all ones)
  std::vector<C> A((size_t)std::max(n, 1) * std::max(n, 1));
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) A[i * n + j] = C((i == j ? (double)n : 0.0) + 1.0);
  if (which == 29 || which == 30) {
    if (n < 1) return -1.0;
    if (which == 30) cholesky_factor(A, n);
  }
  std::vector<C> rhs((size_t)std::max(n, 1), C(1.0));
  volatile double sink = 0.0;
  OpCount::reset();
  switch (which) {
    case 0: sink = val(a + b); break;
    case 1: sink = val(a - b); break;
    case 2: sink = val(a * b); break;
    case 3: sink = val(a / b); break;
    case 4: sink = val(sqrt(a)); break;
    case 5: sink = val(sin(a)); break;
    case 6: sink = val(cos(a)); break;
    case 7: sink = val(atan2(a, b)); break;
    case 8: sink = val(-a); break;
    case 9: sink = val(fabs(a)); break;
    case 10: sink = (a < b) ? 1.0 : 0.0; break;
    case 20: sink = val(dot(u, w)); break;
    case 21: sink = val(cross(u, w)[0]); break;
    case 22: sink = val(mul(R, u)[1]); break;
    case 23: sink = val(mul(R, S).e[4]); break;
    case 24: quat_mul(q1, q2, qo); sink = val(qo[3]); break;
    case 25: quat_exp(mk3<C>(C(0.1), C(0.2), C(std::sqrt(0.09 - 0.05))), qo); sink = val(qo[3]); break;
    case 26: sink = val(smul(X, sv)[2]); break;
    case 27: sink = val(smul(X, Y).e[7]); break;
    case 28: sink = val(sdot(sv, sv)); break;
    case 29: cholesky_factor(A, n); sink = val(A[0]); break;
    case 30: cholesky_solve(A, n, rhs.data()); sink = val(rhs[0]); break;
    default: return -1.0;
  }
  (void)sink;
  return (double)OpCount::count();
}

}  // extern "C"
