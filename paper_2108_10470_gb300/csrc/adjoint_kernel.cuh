// Reverse (adjoint) pass of the env-step for sm_103a: the vector-Jacobian product of one recorded
// step, one environment per group of G lanes, substeps in reverse order. The forward step's
// discrete choices (contact set, limit rows, every projection and target branch of the solve) are
// held fixed, as in the forward-mode derivative; the step kernels, given a tape, record what the
// reverse needs (TapeLayout in sim_internal.h), and everything else is recomputed.
//
// Formulation. The forward step computes qdd = M^-1 (tau - b) (articulated-body algorithm), a
// Gauss-Seidel solve in z = L^T v with Y = L^-1 J^T, and integration. Its adjoint is taken in the
// same coordinates:
//  * integration: hinge and slider joints are additive; a ball joint's rotation update
//    log(exp(q) exp(dq)) is differentiated locally in forward mode; the root quaternion's adjoint
//    is carried as the adjoint of
//    a world-axis rotation th (q_bar = 2 [th_bar; 0] (x) q, the component along q is dropped: the
//    step's output quaternion is normalised), through the exact exponential by the left Jacobian
//    of SO(3);
//  * v = L^-T z, dq = L^-T dz: z_bar = L^-1 v_bar, dz_bar = L^-1 dq_bar;
//  * the solve: row updates in reverse order, z reconstructed from its final value by subtracting
//    each update (z_before = z_after - Y_r dlambda), the taped impulses giving dlambda and the
//    branches (a normal impulse at 0, a friction impulse at +-mu lambda_n, the biased target's cap);
//  * M through its factor: with L_bar the adjoint of L, M_bar = sym(L^-T Phi(L^T L_bar) L^-1)
//    (Phi: lower triangle, halved diagonal); L^T L_bar is formed in z coordinates,
//    -Y_bar Y^T - z z_bar^T - dz dz_bar^T + z0 z0_bar^T, without L^-T Y_bar;
//  * qdd: c_bar = M^-1 qdd_bar, tau_bar = c_bar, and the pose and velocity adjoints of
//    -c_bar . (M qdd + b) come from the reverse of the recursive Newton-Euler algorithm (RBDA Table
//    5.1) at the recorded qdd; those of M_bar . M from the reverse of the composite-rigid-body
//    algorithm (RBDA Table 6.2);
//  * configuration: every pose-dependent quantity (motion subspaces, spatial inertias about the
//    actor origin, contact points) is attached to a link; its adjoint becomes a wrench on that link
//    (a motion subspace S: S x* S_bar; a point x: [x x x_bar; x_bar]; an inertia: from its COM
//    position and rotational inertia), and a joint's position adjoint is S . (wrenches summed over
//    its subtree) (for a ball joint through the right Jacobian of SO(3): J_r(q)^T S^T W), the root
//    rotation's the angular part over the whole actor;
//  * capsule-box pair contacts: two-body rows, and each contact's point, normal and separation
//    differentiated locally in forward mode over the pair geometry (three passes of six tangents).
// Supported: floating and fixed roots, revolute, prismatic, ball and fixed joints, ground contacts
// of spheres, capsules and boxes, capsule-box pairs, joint limits, damping, armature, joint drives,
// fixed tendons (springs and length-limit rows) and external body forces (their values constants of
// the derivative). The pair and ball-joint paths are separate instantiations (template flags).
#pragma once
#include "step_kernel.cuh"
#include "tangent_step.cuh"

namespace artsim {

// Hamilton product and conjugate of quaternions stored (x, y, z, w).
__device__ __forceinline__ void qmul4(const float* a, const float* b, float* o) {
  o[0] = a[3] * b[0] + a[0] * b[3] + a[1] * b[2] - a[2] * b[1];
  o[1] = a[3] * b[1] - a[0] * b[2] + a[1] * b[3] + a[2] * b[0];
  o[2] = a[3] * b[2] + a[0] * b[1] - a[1] * b[0] + a[2] * b[3];
  o[3] = a[3] * b[3] - a[0] * b[0] - a[1] * b[1] - a[2] * b[2];
}
// spatial inertia (m, h, I_O about the actor origin, I_O as xx yy zz xy xz yz) times a motion vector:
// [I_O w + h x v; m v + w x h]
__device__ __forceinline__ void inertia_mul(const float m, const V3 h, const float* IO, const float* x, float* o) {
  const V3 w = v3(x[0], x[1], x[2]), vl = v3(x[3], x[4], x[5]);
  const V3 Iw = v3(IO[0] * w.x + IO[3] * w.y + IO[4] * w.z, IO[3] * w.x + IO[1] * w.y + IO[5] * w.z,
                   IO[4] * w.x + IO[5] * w.y + IO[2] * w.z);
  const V3 a = Iw + cross(h, vl), l = vl * m + cross(w, h);
  o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = l.x; o[4] = l.y; o[5] = l.z;
}
// motion cross product v x m = [w x m_a; w x m_l + v_l x m_a]
__device__ __forceinline__ void crm6(const float* v, const float* m, float* o) {
  const V3 w = v3(v[0], v[1], v[2]), vl = v3(v[3], v[4], v[5]);
  const V3 ma = v3(m[0], m[1], m[2]), ml = v3(m[3], m[4], m[5]);
  const V3 a = cross(w, ma), l = cross(w, ml) + cross(vl, ma);
  o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = l.x; o[4] = l.y; o[5] = l.z;
}
// force cross product v x* f = [w x f_a + v_l x f_l; w x f_l]
__device__ __forceinline__ void crf6(const float* v, const float* f, float* o) {
  const V3 w = v3(v[0], v[1], v[2]), vl = v3(v[3], v[4], v[5]);
  const V3 fa = v3(f[0], f[1], f[2]), fl = v3(f[3], f[4], f[5]);
  const V3 a = cross(w, fa) + cross(vl, fl), l = cross(w, fl);
  o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = l.x; o[4] = l.y; o[5] = l.z;
}
// adjoint of an inertia (I_O sym as xx yy zz xy xz yz, h) from an outer product a b^T of 6-vectors:
// the symmetric part of the angular block, and h_bar = b_l x a_a - b_a x a_l
__device__ __forceinline__ void inertia_outer(const float* a, const float* b, float* IOb, float* hb) {
  IOb[0] += a[0] * b[0];
  IOb[1] += a[1] * b[1];
  IOb[2] += a[2] * b[2];
  IOb[3] += 0.5f * (a[0] * b[1] + a[1] * b[0]);
  IOb[4] += 0.5f * (a[0] * b[2] + a[2] * b[0]);
  IOb[5] += 0.5f * (a[1] * b[2] + a[2] * b[1]);
  const V3 aa = v3(a[0], a[1], a[2]), al = v3(a[3], a[4], a[5]);
  const V3 ba = v3(b[0], b[1], b[2]), bl = v3(b[3], b[4], b[5]);
  const V3 t = cross(bl, aa) - cross(ba, al);
  hb[0] += t.x; hb[1] += t.y; hb[2] += t.z;
}
// 3x3 symmetric (xx yy zz xy xz yz) times vector
__device__ __forceinline__ V3 sym_mv(const float* S, V3 x) {
  return v3(S[0] * x.x + S[3] * x.y + S[4] * x.z, S[3] * x.x + S[1] * x.y + S[5] * x.z,
            S[4] * x.x + S[5] * x.y + S[2] * x.z);
}

// Stride of the per-DOF 6-vectors of the reverse arena (odd: the lanes of a group that each hold one
// DOF's vector fall on distinct banks).
constexpr int kSDS = 7;

constexpr int SIM_STEP_BODY_FORCES = 8;  // StepArgs::flags bit: external body forces every substep

// Per-link record of the reverse arena (kAdjLinkWords words, odd for the same reason).
enum : int {
  kRecVs = 0, kRecCc = 6, kRecIO = 12, kRecH = 18, kRecCw = 21, kRecIcw = 24, kRecM = 30, kRecS = 31,
  kRecIc = 37,   // composite inertia m | h 3 | I_O 6 (10 words)
  kRecSlot = 47  // 6-word hand-off slot of the inward sweeps
};
// Vectors (n words each): the tape's (in the image) and the reverse's own (kAdjVecs in the arena).
enum : int {
  kVQdd = 0, kVFree = 1, kVZ0 = 2, kVZf = 3, kVDzf = 4, kVV = 5, kVDq = 6, kVLinv = 7,
  kVVb = 8, kVDqb = 9, kVZb6 = 10, kVDzb6 = 11, kVZb0 = 12, kVCb = 13
};

// Bulk asynchronous copy (the TMA engine) of `bytes` (a multiple of 16, both addresses 16-byte
// aligned) from global memory into shared memory, completing on the mbarrier at `bar`.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, void* bar) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst), b = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // earlier writes to dst come first
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(d),
               "l"(src), "r"(bytes), "r"(b)
               : "memory");
}
__device__ __forceinline__ void mbar_init(void* bar) {
  const unsigned b = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Wait for the phase `parity` of the mbarrier, giving up after a bounded number of tries (each
// try suspends for at most a hardware time limit): false means the copy did not complete.
__device__ __forceinline__ bool mbar_wait(void* bar, unsigned parity) {
  const unsigned b = (unsigned)__cvta_generic_to_shared(bar);
  for (int i = 0; i < (1 << 20); ++i) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(b), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// Back substitution L^T x = b by one lane for one right-hand side: b_i at base[i * stride] in,
// x_k written there (right-looking, the remaining right-hand side in registers: y[0] holds b_k).
template <int G>
__device__ __forceinline__ void lt_solve_lane(const float* L, const int LS, const float* linv, const int n, float* base,
                                              const int stride) {
  float y[G];
#pragma unroll
  for (int m = 0; m < G; ++m) y[m] = (m < n) ? base[(n - 1 - m) * stride] : 0.f;
  for (int k = n - 1; k >= 0; --k) {
    const float xk = y[0] * linv[k];
    base[k * stride] = xk;
    const float* Lk = L + k * LS;
    // every register shifts down one place; the m <= k ones also take their L_k,k-m term (the
    // others are past the solution's start: no branch, the load clamped inside row k)
#pragma unroll
    for (int m = 1; m < G; ++m) y[m - 1] = y[m] - ((m <= k) ? Lk[m <= k ? k - m : 0] * xk : 0.f);
  }
}

// Group-parallel forward substitution L x = b (lane k holds b_k in, x_k out); two right-hand sides.
template <int G>
__device__ __forceinline__ void fwd_subst2(const float* sL, const int LS, const float* linv, const int n,
                                           const int lane, float& b0, float& b1) {
  float x0 = 0.f, x1 = 0.f;
  for (int k = 0; k < n; ++k) {
    const float li = linv[k];
    const float y0 = Grp<G>::get(b0 * li, k), y1 = Grp<G>::get(b1 * li, k);
    if (lane == k) { x0 = y0; x1 = y1; }
    if (lane > k && lane < n) {
      const float lik = sL[lane * LS + k];
      b0 -= lik * y0;
      b1 -= lik * y1;
    }
  }
  b0 = x0;
  b1 = x1;
}
// Group-parallel back substitution L^T x = b (lane k holds b_k in, x_k out).
template <int G>
__device__ __forceinline__ float back_subst(const float* sL, const int LS, const float* linv, const int n,
                                            const int lane, float b) {
  float x = 0.f;
  for (int k = n - 1; k >= 0; --k) {
    const float xk = Grp<G>::get(b * linv[k], k);
    if (lane == k) x = xk;
    if (lane < k) b -= sL[k * LS + lane] * xk;
  }
  return x;
}

// ---------------------------------------------------------------------------------------------
// Adjoint of a ball joint's rotation update q' = log(exp(q) exp(dq)) (rotation vectors, dq in the
// child frame; the step keeps the shorter rotation), in forward mode with six tangents (q, dq):
// qb = (dq'/dq)^T ob, dqb = (dq'/d dq)^T ob. qb and dqb may alias the inputs.
__device__ __noinline__ void ball_integration_adjoint(const float* q, const float* dq, const float* ob, float* qb,
                                                      float* dqb) {
  constexpr int K = 6;
  Dn<K> a0(q[0]), a1(q[1]), a2(q[2]), b0(dq[0]), b1(dq[1]), b2(dq[2]);
  a0.d[0] = 1.f; a1.d[1] = 1.f; a2.d[2] = 1.f; b0.d[3] = 1.f; b1.d[4] = 1.f; b2.d[5] = 1.f;
  Dn<K> e1[4], e2[4], qn[4], r[3];
  drotvec_quat<K>(a0, a1, a2, e1);
  drotvec_quat<K>(b0, b1, b2, e2);
  qn[0] = e1[3] * e2[0] + e1[0] * e2[3] + e1[1] * e2[2] - e1[2] * e2[1];
  qn[1] = e1[3] * e2[1] - e1[0] * e2[2] + e1[1] * e2[3] + e1[2] * e2[0];
  qn[2] = e1[3] * e2[2] + e1[0] * e2[1] - e1[1] * e2[0] + e1[2] * e2[3];
  qn[3] = e1[3] * e2[3] - e1[0] * e2[0] - e1[1] * e2[1] - e1[2] * e2[2];
  dquat_rotvec<K>(qn, r);
  float o[K];
#pragma unroll
  for (int j = 0; j < K; ++j) o[j] = ob[0] * r[0].d[j] + ob[1] * r[1].d[j] + ob[2] * r[2].d[j];
#pragma unroll
  for (int c = 0; c < 3; ++c) { qb[c] = o[c]; dqb[c] = o[3 + c]; }
}

// ---------------------------------------------------------------------------------------------
// One kept capsule-box sample (pair p, slot) in forward mode over the step's pair geometry, with six
// tangents seeded by `mode`: 0 the capsule link's twist about its actor origin (rotation [w]x R,
// link origin w x P + v), 1 the box link's, 2 the two actor origins (the capsule's, then the box's).
// out[j] = xb . dx/ds_j + nb . dn/ds_j + t1b . dt1/ds_j + t2b . dt2/ds_j + db dd/ds_j for the
// sample's contact point x (relative to body a's actor origin), normal n (from b to a), its
// friction directions and separation d. Out of line: it runs once per pair contact and pass.
__device__ __noinline__ void pair_sample_adjoint(const EnvTypeTable* __restrict__ T, const int p, const int slot,
                                                 const float* Rc, const float* Pc, const float* Oc, const float* Rx,
                                                 const float* Px, const float* Ox, const int mode, const V3 xb,
                                                 const V3 nb, const V3 t1b, const V3 t2b, const float db, float* out) {
  constexpr int K = 6;
  const int sa = T->pair_a[p], sb = T->pair_b[p];
  const bool a_cap = T->shape_type[sa] == kCapsule;
  const int sc = a_cap ? sa : sb, sx = a_cap ? sb : sa;
  Dn<K> Rcd[9], Rxd[9];
  DV3<K> Pcd, Pxd, Ocd, Oxd;
#pragma unroll
  for (int k = 0; k < 9; ++k) { Rcd[k] = Dn<K>(Rc[k]); Rxd[k] = Dn<K>(Rx[k]); }
  Pcd = dv3<K>(Dn<K>(Pc[0]), Dn<K>(Pc[1]), Dn<K>(Pc[2]));
  Pxd = dv3<K>(Dn<K>(Px[0]), Dn<K>(Px[1]), Dn<K>(Px[2]));
  Ocd = dv3<K>(Dn<K>(Oc[0]), Dn<K>(Oc[1]), Dn<K>(Oc[2]));
  Oxd = dv3<K>(Dn<K>(Ox[0]), Dn<K>(Ox[1]), Dn<K>(Ox[2]));
  if (mode < 2) {  // a twist of one link: d R = [e_j]x R (columns rotate), d P = e_j x P; d P = e_(j-3)
    Dn<K>* R = mode == 0 ? Rcd : Rxd;
    DV3<K>& P = mode == 0 ? Pcd : Pxd;
    const float* Rv = mode == 0 ? Rc : Rx;
    const float* Pv = mode == 0 ? Pc : Px;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const V3 e = v3(j == 0 ? 1.f : 0.f, j == 1 ? 1.f : 0.f, j == 2 ? 1.f : 0.f);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const V3 dc = cross(e, v3(Rv[k], Rv[3 + k], Rv[6 + k]));
        R[k].d[j] = dc.x; R[3 + k].d[j] = dc.y; R[6 + k].d[j] = dc.z;
      }
      const V3 dp = cross(e, v3(Pv[0], Pv[1], Pv[2]));
      P.x.d[j] = dp.x; P.y.d[j] = dp.y; P.z.d[j] = dp.z;
    }
    P.x.d[3] = 1.f; P.y.d[4] = 1.f; P.z.d[5] = 1.f;
  } else {
    Ocd.x.d[0] = 1.f; Ocd.y.d[1] = 1.f; Ocd.z.d[2] = 1.f;
    Oxd.x.d[3] = 1.f; Oxd.y.d[4] = 1.f; Oxd.z.d[5] = 1.f;
  }
  // the geometry of the step's pair phase (relative to the box actor's origin)
  Dn<K> Rsh[9], Rcs[9], Rb[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) Rsh[k] = Dn<K>(T->shape_rot[k][sc]);
  dmm<K>(Rcd, Rsh, Rcs);
#pragma unroll
  for (int k = 0; k < 9; ++k) Rsh[k] = Dn<K>(T->shape_rot[k][sx]);
  dmm<K>(Rxd, Rsh, Rb);
  const DV3<K> cc = Pcd + dmv<K>(Rcd, dv3<K>(Dn<K>(T->shape_pos[0][sc]), Dn<K>(T->shape_pos[1][sc]),
                                             Dn<K>(T->shape_pos[2][sc]))) + (Ocd - Oxd);
  const DV3<K> cb = Pxd + dmv<K>(Rxd, dv3<K>(Dn<K>(T->shape_pos[0][sx]), Dn<K>(T->shape_pos[1][sx]),
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
  const Dn<K> t = slot == 0 ? Dn<K>(0.f) : (slot == 1 ? Dn<K>(1.f) : (slot == 2 ? ta : (slot == 3 ? tb : tstar)));
  bool ok = true;  // the step kept this sample; its recomputation must find it valid too
  if (slot >= 2) {
    if (slot < 4 && !clip) ok = false;
    if (slot == 3 && !(ta.v < tb.v)) ok = false;
    if (!(t.v > 0.f && t.v < 1.f)) ok = false;
  }
#pragma unroll
  for (int j = 0; j < K; ++j) out[j] = 0.f;
  if (!ok) return;
  DV3<K> pn, px;
  Dn<K> pd;
  dsphere_box<K>(p0 + dv * t, r, e, pn, pd, px);
  DV3<K> nw = b0 * pn.x + b1 * pn.y + b2 * pn.z;  // box -> capsule
  if (!a_cap) nw = dv3<K>(-nw.x, -nw.y, -nw.z);
  const DV3<K> Oa = a_cap ? Ocd : Oxd;
  const DV3<K> xw = cb + b0 * px.x + b1 * px.y + b2 * px.z + (Oxd - Oa);
  DV3<K> t1, t2;
  dtangent_basis<K>(nw, t1, t2);
#pragma unroll
  for (int j = 0; j < K; ++j)
    out[j] = xb.x * xw.x.d[j] + xb.y * xw.y.d[j] + xb.z * xw.z.d[j] + nb.x * nw.x.d[j] + nb.y * nw.y.d[j] +
             nb.z * nw.z.d[j] + t1b.x * t1.x.d[j] + t1b.y * t1.y.d[j] + t1b.z * t1.z.d[j] + t2b.x * t2.x.d[j] +
             t2b.y * t2.y.d[j] + t2b.z * t2.z.d[j] + db * pd.d[j];
}

// ---------------------------------------------------------------------------------------------
// The reverse pass of one env (group of G lanes): sm is the group's arena (AdjLayout), gi its index
// in the launch (the tape block), live false for the dead groups of the last CTA (they shadow the
// last env and store nothing).
template <int G, bool PAIRS, bool BALL>
__device__ __forceinline__ void adjoint_group(const StepArgs& A, const TypeArgs& TA, const AdjArgs& J, const int grp,
                                              float* sm) {
  const EnvTypeTable* __restrict__ T = TA.type;
  const int lane = threadIdx.x & (G - 1);
  const bool live = grp < TA.n_launch_envs;
  const int gi = live ? grp : TA.n_launch_envs - 1;
  const int env = TA.env_ids ? TA.env_ids[gi] : TA.env_first + gi;
  const AdjLayout& al = J.al;
  const TapeLayout& TL = TA.tl;
  const int L = T->n_links, n = T->n_gen;
  const int maxdepth = T->max_depth;
  const int YS = al.YS, LS = al.LS, RC = TL.rcap;
  // the substep's tape image (read in place; its final impulses are rewound during the solve); Y
  // is the image's last block, or, when the arena has no room for it, read in place from the tape
  float* img = sm + al.img;
  void* bar = sm + al.bar;
  const float* s_Y = img + TL.Y;
  float* s_L = img + TL.L;
  float4* s_rowc = reinterpret_cast<float4*>(img + TL.rowc);
  int* s_rowa = reinterpret_cast<int*>(img + TL.rowa);
  float* s_lam = img + TL.lamf;
  float* s_lam0 = img + TL.lam0;
  // the row history (read in the solve's reverse): in the image, or with gY in place in the tape
  const float* s_lambef = img + TL.lamb;
  const float* s_seps = img + TL.seps;
  // row work blocks, once the history is dead: the image's history block, or a global slot
  float* rws = (PAIRS && al.gY) ? J.rwg + (size_t)grp * al.rw : img + TL.lamb;
  float* s_con = img + TL.con;
  int* s_coni = reinterpret_cast<int*>(s_con);
  const float* s_linv = img + TL.Linv;
  // Y's adjoint outside the arena: env types with shape pairs only (a global slot per group: the
  // dead groups own one too); elsewhere both stay shared-memory pointers the compiler can see
  float* s_Yb = (PAIRS && al.gY) ? J.ybg + (size_t)grp * (size_t)n * YS : sm + al.Yb;
  float* s_Mb = sm + al.Mb;
  float* s_lamb = sm + al.lamb;
  float* s_db = sm + al.db;
  float* s_invAb = sm + al.invAb;
  float* s_xb = (PAIRS && al.gY) ? rws + al.frw : sm + al.xb;
  constexpr int XW = PAIRS ? 9 : 3;  // words per row of s_xb (AdjLayout::xbw)
  constexpr bool pairs_t = PAIRS;    // the type has capsule-box shape pairs (TL.cw > 5)
  float* s_pose = sm + al.pose;      // pairs: rotation 9 | origin 3 of each link
  float* s_vec = sm + al.vec;
  float* s_SD = sm + al.SD;
  float* s_FM = sm + al.FM;
  float* s_FMb = sm + al.FMb;
  float* s_Sb = sm + al.Sb;
  float* s_link = sm + al.link;
  float* s_sink = sm + al.bar + 2;  // a scratch word after the mbarrier (the arena reserves 4 words there)
  auto V = [&](int k) -> float* {
    return k < 7 ? img + TL.vec + k * n : (k == kVLinv ? img + TL.Linv : s_vec + (k - kVVb) * n);
  };

  // ---- per-link constants (link mode) ----
  const bool isl = lane < L;
  const int l = isl ? lane : 0;
  const int par = isl ? T->parent[l] : -1;
  const int jt = T->jtype[l];
  const int dep = isl ? T->depth[l] : -1;
  const int gd = T->gdof[l];
  const int jd = T->jdof[l];
  const bool is_root = isl && par < 0;
  const bool free_root = is_root && jt == kFree;
  const bool has_dof = isl && (jt == kRevolute || jt == kPrismatic);
  // ball joint (three generalized DOFs from gd: rotation vector, angular velocity in the child
  // frame), compiled into the BALL instantiation only
  const bool is_ball = BALL && isl && jt == kSpherical;
  const bool isg = lane < n;
  float* rec = s_link + kAdjLinkWords * l;
  float* slot = rec + kRecSlot;
  const int dof_base = A.env_dof_base[env];
  const int actor_row = isl ? A.env_actor_base[env] + T->actor[l] : 0;
  const float h = A.h;
  const int npos = A.pos_iters, nvel = A.vel_iters;
  const float hit = h / (float)npos;
  const float inv_hit = 1.f / hit, inv_h = 1.f / h;
  const float beta = A.bias_coef, vmax = A.max_depen_vel;
  const V3 g = v3(A.gx, A.gy, A.gz);
  float* cacheb = J.gi_cache + (size_t)env * A.cache_stride;

  // inward sum of a 6-vector over each link's subtree (children in the fixed sibling order)
  auto inward6 = [&](float* x) {
    for (int d = maxdepth; d >= 1; --d) {
      if (dep == d) {
#pragma unroll
        for (int k = 0; k < 6; ++k) slot[k] = x[k];
      }
      __syncwarp();
      if (dep == d - 1)
        for (int ch = T->first_child[l]; ch >= 0; ch = T->next_sibling[ch]) {
          const float* sc = s_link + kAdjLinkWords * ch + kRecSlot;
#pragma unroll
          for (int k = 0; k < 6; ++k) x[k] += sc[k];
        }
      __syncwarp();
    }
  };
  // outward prefix sum of a K-vector over each link's ancestors (root first)
  auto outward = [&](float* x, const int K) {
    for (int d = 1; d <= maxdepth; ++d) {
      const int src = par >= 0 ? par : lane;
      for (int k = 0; k < K; ++k) {
        const float pv = Grp<G>::get(x[k], src);
        if (dep == d) x[k] += pv;
      }
    }
  };

  // ---- carried adjoints: the output gradient of the step ----
  float qb = 0.f, qdb = 0.f, actb = 0.f;
  float rpb[3] = {0.f, 0.f, 0.f}, rqb[4] = {0.f, 0.f, 0.f, 0.f}, rwb[3] = {0.f, 0.f, 0.f}, rvb[3] = {0.f, 0.f, 0.f};
  if (has_dof && J.g_dof) {
    qb = J.g_dof[(size_t)(dof_base + jd) * 2];
    qdb = J.g_dof[(size_t)(dof_base + jd) * 2 + 1];
  }
  float bqb[3] = {0.f, 0.f, 0.f}, bwb[3] = {0.f, 0.f, 0.f}, bab[3] = {0.f, 0.f, 0.f};  // ball: q, qd, act
  if (is_ball && J.g_dof) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      bqb[c] = J.g_dof[(size_t)(dof_base + jd + c) * 2];
      bwb[c] = J.g_dof[(size_t)(dof_base + jd + c) * 2 + 1];
    }
  }
  if (is_root && J.g_root) {
    const float* gr = J.g_root + (size_t)actor_row * 13;
#pragma unroll
    for (int k = 0; k < 3; ++k) { rpb[k] = gr[k]; rvb[k] = free_root ? gr[7 + k] : 0.f; rwb[k] = free_root ? gr[10 + k] : 0.f; }
#pragma unroll
    for (int k = 0; k < 4; ++k) rqb[k] = gr[3 + k];
  }
  if (live)
    for (int i = lane; i < A.cache_stride; i += G) cacheb[i] = J.g_cache ? J.g_cache[(size_t)env * A.cache_stride + i] : 0.f;
  if (lane == 0) mbar_init(bar);
  __syncwarp();
  unsigned parity = 0;
  bool failed = false;  // a tape copy that did not complete: the env's gradient is not computed

  for (int sub = A.substeps - 1; sub >= 0; --sub) {
    const float* tp = J.tape + ((size_t)gi * A.substeps + sub) * TL.words;
    if (PAIRS && al.gY) { s_Y = tp + TL.Y; s_lambef = tp + TL.lamb; s_seps = tp + TL.seps; }
    // ---- the tape block into the arena: one bulk copy by the TMA engine ----
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // this lane's writes to the image first
    __syncwarp();
    if (lane == 0) bulk_copy_g2s(img, tp, 4u * (unsigned)al.imgw, bar);
    const bool arrived = mbar_wait(bar, parity);
    parity ^= 1u;
    if (__any_sync(kFull, !arrived)) {  // warp-uniform: both groups of the warp stop here
      failed = true;
      mbar_wait(bar, parity ^ 1u);  // once more for the copy in flight, then no further use
      break;
    }
    const int* th = reinterpret_cast<const int*>(img + TL.hdr);
    const int n_con = th[0], n_lim = th[1], R = th[2];
    for (int i = 0; i < n; ++i)
      for (int r = lane; r < R; r += G) s_Yb[i * YS + r] = 0.f;
    for (int r = lane; r < R; r += G) {
      const float4 hc = s_rowc[r];
      s_lamb[r] = (hc.y > 0.f) ? cacheb[__float_as_int(hc.w)] : 0.f;
      s_db[r] = 0.f;
      s_invAb[r] = 0.f;
    }
    // the substep's input state
    float q = 0.f, qd = 0.f, rq[4] = {0.f, 0.f, 0.f, 1.f};
    V3 rp = v3(0.f, 0.f, 0.f), rw = rp, rv = rp;
    if (has_dof) { q = img[TL.st + 2 * jd]; qd = img[TL.st + 2 * jd + 1]; }
    float bq[3] = {0.f, 0.f, 0.f}, bw[3] = {0.f, 0.f, 0.f};  // ball: rotation vector, angular velocity
    if (is_ball) {
#pragma unroll
      for (int c = 0; c < 3; ++c) { bq[c] = img[TL.st + 2 * (jd + c)]; bw[c] = img[TL.st + 2 * (jd + c) + 1]; }
    }
    if (is_root) {
      const float* r = img + TL.st + 2 * T->n_jdof + 13 * T->actor[l];
      rp = v3(r[0], r[1], r[2]);
      rq[0] = r[3]; rq[1] = r[4]; rq[2] = r[5]; rq[3] = r[6];
      rv = v3(r[7], r[8], r[9]);
      rw = v3(r[10], r[11], r[12]);
    }
    __syncwarp();

    // ---- kinematics and inertias of the substep's input state (as in the forward step) ----
    float S[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    {
      float Rw[9];
      V3 P = v3(0.f, 0.f, 0.f);
      float vs[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, cc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      quat_to_mat(rq, Rw);
      if (is_root) {
        vs[0] = rw.x; vs[1] = rw.y; vs[2] = rw.z; vs[3] = rv.x; vs[4] = rv.y; vs[5] = rv.z;
        const V3 pxw = cross(rv, rw);
        cc[3] = pxw.x; cc[4] = pxw.y; cc[5] = pxw.z;
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
          const V3 jaxis = v3(T->axis[0][l], T->axis[1][l], T->axis[2][l]);
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
            S[0] = aw.x; S[1] = aw.y; S[2] = aw.z; S[3] = pxa.x; S[4] = pxa.y; S[5] = pxa.z;
          } else if (jt == kPrismatic) {
#pragma unroll
            for (int k = 0; k < 9; ++k) Rw[k] = RB[k];
            P = Pp + mv(Rp, pp + mv(Rpj, jaxis * q));
            S[3] = aw.x; S[4] = aw.y; S[5] = aw.z;
          } else if (BALL && jt == kSpherical) {
            float qj[4], RJ[9];
            rotvec_quat(bq[0], bq[1], bq[2], qj);
            quat_to_mat(qj, RJ);
            mm(RB, RJ, Rw);
            P = Pp + mv(Rp, pp);
          } else {
#pragma unroll
            for (int k = 0; k < 9; ++k) Rw[k] = RB[k];
            P = Pp + mv(Rp, pp);
          }
          float sq[6];
#pragma unroll
          for (int k = 0; k < 6; ++k) sq[k] = S[k] * qd;
          if (BALL && jt == kSpherical) {  // the child's axes about the actor origin, one per DOF
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              const V3 ax = v3(Rw[c], Rw[3 + c], Rw[6 + c]), px = cross(P, ax);
              sq[0] += ax.x * bw[c]; sq[1] += ax.y * bw[c]; sq[2] += ax.z * bw[c];
              sq[3] += px.x * bw[c]; sq[4] += px.y * bw[c]; sq[5] += px.z * bw[c];
            }
          }
#pragma unroll
          for (int k = 0; k < 6; ++k) vs[k] = vp[k] + sq[k];
          crm6(vs, sq, cc);
        }
      }
      if (isl) {
#pragma unroll
        for (int k = 0; k < 6; ++k) { rec[kRecVs + k] = vs[k]; rec[kRecCc + k] = cc[k]; rec[kRecS + k] = S[k]; }
        // rigid inertia about the actor origin: m, h = m c, I_O = R I_c R^T + m (|c|^2 1 - c c^T)
        const float m = T->mass[l];
        const V3 cw = P + mv(Rw, v3(T->com[0][l], T->com[1][l], T->com[2][l]));
        const float In[9] = {T->inertia[0][l], T->inertia[3][l], T->inertia[4][l], T->inertia[3][l], T->inertia[1][l],
                             T->inertia[5][l], T->inertia[4][l], T->inertia[5][l], T->inertia[2][l]};
        float RI[9], Rt[9], Ic9[9];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) Rt[3 * i + j] = Rw[3 * j + i];
        mm(Rw, In, RI);
        mm(RI, Rt, Ic9);
        const float c2 = dot(cw, cw);
        const float icw[6] = {Ic9[0], Ic9[4], Ic9[8], Ic9[1], Ic9[2], Ic9[5]};
        const float io[6] = {icw[0] + m * (c2 - cw.x * cw.x), icw[1] + m * (c2 - cw.y * cw.y),
                             icw[2] + m * (c2 - cw.z * cw.z), icw[3] - m * cw.x * cw.y, icw[4] - m * cw.x * cw.z,
                             icw[5] - m * cw.y * cw.z};
#pragma unroll
        for (int k = 0; k < 6; ++k) { rec[kRecIcw + k] = icw[k]; rec[kRecIO + k] = io[k]; }
        rec[kRecH] = m * cw.x; rec[kRecH + 1] = m * cw.y; rec[kRecH + 2] = m * cw.z;
        rec[kRecCw] = cw.x; rec[kRecCw + 1] = cw.y; rec[kRecCw + 2] = cw.z;
        rec[kRecM] = m;
        if (pairs_t) {  // the link's pose, for the pair contacts' geometry
#pragma unroll
          for (int k = 0; k < 9; ++k) s_pose[12 * l + k] = Rw[k];
          s_pose[12 * l + 9] = P.x; s_pose[12 * l + 10] = P.y; s_pose[12 * l + 11] = P.z;
        }
      }
      // motion subspace per generalized DOF (unit columns for a floating root)
      if (has_dof) {
#pragma unroll
        for (int k = 0; k < 6; ++k) s_SD[kSDS * gd + k] = S[k];
      }
      if (is_ball) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const V3 ax = v3(Rw[c], Rw[3 + c], Rw[6 + c]), px = cross(P, ax);
          float* Sc = s_SD + kSDS * (gd + c);
          Sc[0] = ax.x; Sc[1] = ax.y; Sc[2] = ax.z; Sc[3] = px.x; Sc[4] = px.y; Sc[5] = px.z;
        }
      }
      if (free_root) {
#pragma unroll
        for (int c = 0; c < 6; ++c)
#pragma unroll
          for (int k = 0; k < 6; ++k) s_SD[kSDS * (gd + c) + k] = (k == c) ? 1.f : 0.f;
      }
    }

    // ---- integration reverse: v_bar, dq_bar from the output adjoints ----
    float thb[3] = {0.f, 0.f, 0.f};  // adjoint of the input root rotation (world axes)
    if (has_dof) {
      V(kVDqb)[gd] = qb;   // q' = q + dq (qb stays: the identity path)
      V(kVVb)[gd] = qdb;   // qd' = v
      qdb = 0.f;
    }
    if (is_ball) {  // q' = log(exp(q) exp(dq)) (the shorter rotation), qd' = v
      float dqv[3], qin[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) dqv[c] = V(kVDq)[gd + c];
      ball_integration_adjoint(bq, dqv, bqb, qin, dqv);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        V(kVDqb)[gd + c] = dqv[c];
        V(kVVb)[gd + c] = bwb[c];
        bqb[c] = qin[c];
        bwb[c] = 0.f;
      }
    }
    if (is_root) {
      // rotation adjoint of the output quaternion q' (its component along q' is dropped)
      float qo[4] = {rq[0], rq[1], rq[2], rq[3]};
      float E[9] = {1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 1.f};
      V3 phi = v3(0.f, 0.f, 0.f);
      if (free_root) {
        phi = v3(V(kVDq)[gd], V(kVDq)[gd + 1], V(kVDq)[gd + 2]);
        float e[4];
        rotvec_quat(phi.x, phi.y, phi.z, e);
        quat_to_mat(e, E);
        float qn[4];
        qmul4(e, rq, qn);
        const float nr = sqrtf(qn[0] * qn[0] + qn[1] * qn[1] + qn[2] * qn[2] + qn[3] * qn[3]);
#pragma unroll
        for (int k = 0; k < 4; ++k) qo[k] = qn[k] / nr;
      }
      const float qc[4] = {-qo[0], -qo[1], -qo[2], qo[3]};
      float t4[4];
      qmul4(rqb, qc, t4);
      const V3 tho = v3(0.5f * t4[0], 0.5f * t4[1], 0.5f * t4[2]);
      // th_in = E^T th_out (q' = e (x) q: a world rotation of q is rotated by e)
      const V3 ti = v3(E[0] * tho.x + E[3] * tho.y + E[6] * tho.z, E[1] * tho.x + E[4] * tho.y + E[7] * tho.z,
                       E[2] * tho.x + E[5] * tho.y + E[8] * tho.z);
      thb[0] = ti.x; thb[1] = ti.y; thb[2] = ti.z;
      if (free_root) {
        // dq_ang_bar = J_l(phi)^T th_out, J_l^T x = x - a phi x x + b phi x (phi x x)
        const float a2 = dot(phi, phi);
        float ca, cb;
        if (a2 < 1e-8f) {
          ca = 0.5f - a2 / 24.f;
          cb = 1.f / 6.f - a2 / 120.f;
        } else {
          const float an = sqrtf(a2);
          float sn, cs;
          sincosf(an, &sn, &cs);
          ca = (1.f - cs) / a2;
          cb = (an - sn) / (a2 * an);
        }
        const V3 px = cross(phi, tho);
        const V3 jt3 = tho - px * ca + cross(phi, px) * cb;
        V(kVDqb)[gd] = jt3.x; V(kVDqb)[gd + 1] = jt3.y; V(kVDqb)[gd + 2] = jt3.z;
        // p' = p + dq_lin (rpb stays), omega' = v_ang, p_dot' = v_lin
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          V(kVDqb)[gd + 3 + k] = rpb[k];
          V(kVVb)[gd + k] = rwb[k];
          V(kVVb)[gd + 3 + k] = rvb[k];
          rwb[k] = 0.f;
          rvb[k] = 0.f;
        }
      }
    }
    __syncwarp();

    // ---- v = L^-T z, dq = L^-T dz: z_bar = L^-1 v_bar, dz_bar = L^-1 dq_bar (DOF mode) ----
    float zb = isg ? V(kVVb)[lane] : 0.f, dzb = isg ? V(kVDqb)[lane] : 0.f;
    fwd_subst2<G>(s_L, LS, s_linv, n, lane, zb, dzb);
    if (isg) { V(kVZb6)[lane] = zb; V(kVDzb6)[lane] = dzb; }

    // ---- the Gauss-Seidel solve in reverse (DOF mode: lane g holds z_g, z_bar_g, dz_g, dz_bar_g) ----
    {
      float z = isg ? V(kVZf)[lane] : 0.f, dz = isg ? V(kVDzf)[lane] : 0.f;
      const float dzf = dz;
      const int Rw_max = __reduce_max_sync(kFull, R);
      for (int it = npos + nvel - 1; it >= 0; --it) {
        const bool pos = it < npos;
        if (pos) {  // forward: dz(it + 1) = dz(it) + h_it z after the iteration's rows
          zb += hit * dzb;
          dz -= hit * z;
        }
        const float dzs = pos ? dz : dzf;  // the dz this iteration's separations used
        const float* sp = s_seps + (pos ? it : npos) * RC;
        const float* lb = s_lambef + it * RC;
        for (int r = Rw_max - 1; r >= 0; --r) {
          const bool inr = r < R;
          const int rr = inr ? r : 0;
          const float4 hc = s_rowc[rr];
          const float invA = inr ? hc.y : 0.f;
          const bool valid = invA > 0.f;
          const int kb = __float_as_int(hc.z);
          const bool fric = (kb & 3) == kRowFriction;
          const int nrow = (valid && fric) ? (kb >> 2) : 0;
          // every value this row's update reads, before any lane stores (the stores below write
          // the same value from every lane of the group)
          const float la = s_lam[rr], lbf = lb[rr], lbar = s_lamb[rr], sep = sp[rr];
          const float dbr = s_db[rr], iab = s_invAb[rr], ln_cur = s_lam[nrow], lbn = s_lamb[nrow];
          const float D = valid ? la - lbf : 0.f;
          const float y = (isg && inr) ? s_Y[lane * YS + rr] : 0.f;
          const float ybar = isg ? s_Yb[lane * YS + rr] : 0.f;  // (rr's own value: written back unchanged)
          const float zbef = z - y * D;
          // two group reductions in one pass: Y_r . z_bar and Y_r . z (before the update)
          float Db = y * zb, yz = y * zbef;
#pragma unroll
          for (int m = G / 2; m >= 1; m >>= 1) {
            Db += __shfl_xor_sync(kFull, Db, m, G);
            yz += __shfl_xor_sync(kFull, yz, m, G);
          }
          const float ap = lbar + Db;  // adjoint of the impulse after the update
          // friction: clamped at +lim or -lim (lim = mu lambda_n; at lim = 0 the argument's sign)
          const float lim = hc.x * ln_cur;
          const float arg_f = lbf - yz * invA;
          const bool zl = (lim == 0.f);
          const bool hi = fric && (la == lim) && (!zl || arg_f > 0.f);
          const bool lo = fric && !hi && (la == -lim) && (!zl || arg_f < 0.f);
          // normal and limit rows: max(arg, 0) at 0 is the clamped side; the target and its slope
          const bool clamped = fric ? (hi || lo) : (la == 0.f);
          const float t1 = -beta * sep * inv_hit;
          const bool cap = !(t1 < vmax);
          const float tgt = pos ? ((sep >= 0.f) ? -sep * inv_hit : (cap ? vmax : t1)) : ((sep > 0.f) ? -sep * inv_h : 0.f);
          const float dts = pos ? ((sep >= 0.f) ? -inv_hit : (cap ? 0.f : -beta * inv_hit)) : ((sep > 0.f) ? -inv_h : 0.f);
          const float argb = (clamped || !valid) ? 0.f : ap;
          const float nbar = hi ? hc.x * ap : (lo ? -hc.x * ap : 0.f);
          const float yzb = -argb * invA;
          const float iadd = argb * ((fric ? 0.f : tgt) - yz);
          const float sepb = fric ? 0.f : argb * invA * dts;
          // (an invalid row, y = 0 and argb = 0, leaves every value as it was: the stores below are
          // unconditional, the friction store of a non-friction row goes to a sink word)
          if (isg) s_Yb[lane * YS + rr] = valid ? ybar + D * zb + yzb * zbef + sepb * dzs : ybar;
          zb += yzb * y;
          dzb += sepb * y;
          z = zbef;
          __syncwarp();  // every lane has read what the stores below overwrite
          s_lam[rr] = valid ? lbf : la;
          s_lamb[rr] = valid ? argb - Db : lbar;
          s_db[rr] = dbr + sepb;
          s_invAb[rr] = iab + iadd;
          *((valid && fric) ? s_lamb + nrow : s_sink) = lbn + nbar;
          __syncwarp();
        }
      }
      if (isg) V(kVZb0)[lane] = zb;  // adjoint of z0 = L^T v_free (after the warm start)
    }
    __syncwarp();

    // ---- warm start z = z0 + sum Y_r lambda0_r and A_r = |Y_r|^2 (row mode) ----
    for (int r = lane; r < R; r += G) {
      const float4 hc = s_rowc[r];
      if (!(hc.y > 0.f)) { s_lamb[r] = 0.f; continue; }
      const float l0 = s_lam0[r], ia = hc.y, ca = -2.f * s_invAb[r] * ia * ia;
      float acc = 0.f;
      for (int i = 0; i < n; ++i) {
        const float yi = s_Y[i * YS + r], zbi = V(kVZb0)[i];
        acc += yi * zbi;
        s_Yb[i * YS + r] += l0 * zbi + ca * yi;
      }
      s_lamb[r] += acc;  // adjoint of the warm-start impulse: the input impulse cache
    }
    __syncwarp();

    // ---- v_free_bar = L z0_bar; c_bar = M^-1 (h v_free_bar) (DOF mode) ----
    float vfb = 0.f;
    if (isg)
      for (int j = 0; j <= lane; ++j) vfb += s_L[lane * LS + j] * V(kVZb0)[j];
    {
      float b = h * vfb, dummy = 0.f;
      fwd_subst2<G>(s_L, LS, s_linv, n, lane, b, dummy);
      const float cb = back_subst<G>(s_L, LS, s_linv, n, lane, b);
      if (isg) V(kVCb)[lane] = cb;
    }
    // ---- P = Phi(L^T L_bar) = Phi(-Y_bar Y^T - z z_bar^T - dz dz_bar^T + z0 z0_bar^T) (lane = row) ----
    if (isg) {
      float p[G];
#pragma unroll
      for (int j = 0; j < G; ++j) p[j] = 0.f;
      for (int r = 0; r < R; ++r) {
        const float yb = s_Yb[lane * YS + r];
#pragma unroll
        for (int j = 0; j < G; ++j) p[j] -= yb * s_Y[(j < n ? j : 0) * YS + r];  // j >= n: unused
      }
      const float zf = V(kVZf)[lane], dzf = V(kVDzf)[lane], z0 = V(kVZ0)[lane];
#pragma unroll
      for (int j = 0; j < G; ++j) {
        const int jj = j < n ? j : 0;
        const float v = p[j] - zf * V(kVZb6)[jj] - dzf * V(kVDzb6)[jj] + z0 * V(kVZb0)[jj];
        if (j < n) s_Mb[lane * LS + j] = (j < lane) ? v : ((j == lane) ? 0.5f * v : 0.f);
      }
    }
    __syncwarp();
    // ---- Jacobian-row adjoints J_bar_r = L^-T Y_bar_r, in place (row mode, contact rows) ----
    for (int r = lane; r < R; r += G) {
      const int kind = __float_as_int(s_rowc[r].z) & 3;
      if (!(s_rowc[r].y > 0.f) || kind == kRowLimit || kind == kRowTendon) continue;  // constant J
      lt_solve_lane<G>(s_L, LS, s_linv, n, s_Yb + r, YS);
    }
    // ---- M_bar' = L^-T P L^-1 (its symmetric part is the joint-space inertia's adjoint) ----
    if (isg) lt_solve_lane<G>(s_L, LS, s_linv, n, s_Mb + lane, LS);  // X = L^-T P, lane = column
    __syncwarp();
    if (isg) lt_solve_lane<G>(s_L, LS, s_linv, n, s_Mb + lane * LS, 1);  // M_bar'^T solves L^T: lane = row
    __syncwarp();

    // ---- composite inertias (inward sweep of m, h, I_O) and F_i = Ic S_i (DOF mode) ----
    {
      float ic[10];
      if (isl) {
        ic[0] = rec[kRecM];
#pragma unroll
        for (int k = 0; k < 3; ++k) ic[1 + k] = rec[kRecH + k];
#pragma unroll
        for (int k = 0; k < 6; ++k) ic[4 + k] = rec[kRecIO + k];
      }
      for (int d = maxdepth; d >= 1; --d) {
        if (dep == d) {
#pragma unroll
          for (int k = 0; k < 10; ++k) rec[kRecIc + k] = ic[k];
        }
        __syncwarp();
        if (dep == d - 1)
          for (int ch = T->first_child[l]; ch >= 0; ch = T->next_sibling[ch]) {
            const float* sc = s_link + kAdjLinkWords * ch + kRecIc;
#pragma unroll
            for (int k = 0; k < 10; ++k) ic[k] += sc[k];
          }
        __syncwarp();
      }
      if (is_root) {
#pragma unroll
        for (int k = 0; k < 10; ++k) rec[kRecIc + k] = ic[k];
      }
    }
    __syncwarp();
    if (isg) {
      const float* ic = s_link + kAdjLinkWords * T->dof_link[lane] + kRecIc;
      inertia_mul(ic[0], v3(ic[1], ic[2], ic[3]), ic + 4, s_SD + kSDS * lane, s_FM + kSDS * lane);
    }
    __syncwarp();
    // ---- contact rows (row mode): the contact-point adjoint x_bar = sum_g J_bar_rg (k x a_g), + d_bar
    // e_z for a ground normal row; and, for the gather below, the row's [x x k; k] and the mask of the
    // generalized DOFs it acts on (0 for a row without response), in the dead impulse-history block.
    // A pair row acts on two bodies, J_r = S . [x x k; k] on a's path and -S . [x_b x k; k] on b's
    // (x_b = x - o_b, o_b b's actor origin relative to a's; k the pair normal or a friction direction
    // of it): its adjoints of x, o_b and k go to the pair phase below ----
    float* s_fr = rws;  // 7 x RC words: [x x k; k] (6) | DOF mask; with shape pairs 7 more: b's
    for (int r = n_lim + lane; r < R; r += G) {
      const float4 hc = s_rowc[r];
      const int a = s_rowa[r];
      const int c = a & 0xff, dir = (a >> 8) & 3;
      const bool act = hc.y > 0.f;
      const int lbk = pairs_t ? s_coni[5 * TL.ccap + c] : -1;  // body b of a pair contact
      const unsigned anc = act ? T->anc[s_coni[3 * TL.ccap + c]] : 0u;
      const unsigned ancb = (act && lbk >= 0) ? T->anc[lbk] : 0u;
      const V3 x = v3(s_con[c], s_con[TL.ccap + c], s_con[2 * TL.ccap + c]);
      V3 k = dir == 0 ? v3(0.f, 0.f, 1.f) : (dir == 1 ? v3(1.f, 0.f, 0.f) : v3(0.f, 1.f, 0.f));
      V3 dob = v3(0.f, 0.f, 0.f);
      if (lbk >= 0) {
        const V3 nrm = v3(s_con[7 * TL.ccap + c], s_con[8 * TL.ccap + c], s_con[9 * TL.ccap + c]);
        dob = v3(s_con[10 * TL.ccap + c], s_con[11 * TL.ccap + c], s_con[12 * TL.ccap + c]);
        k = nrm;
        if (dir != 0) {
          V3 t1, t2;
          tangent_basis(nrm, t1, t2);
          k = (dir == 1) ? t1 : t2;
        }
      }
      V3 sa = v3(0.f, 0.f, 0.f), la = sa, sb = sa, lb = sa;  // sums of J_bar_rg S_g (angular, linear)
      for (int gg = 0; gg < n; ++gg) {
        const float jr = s_Yb[gg * YS + r];
        const float ja = ((anc >> gg) & 1u) ? jr : 0.f, jb = ((ancb >> gg) & 1u) ? jr : 0.f;
        const V3 Sa = v3(s_SD[kSDS * gg], s_SD[kSDS * gg + 1], s_SD[kSDS * gg + 2]);
        sa = sa + Sa * ja;
        sb = sb + Sa * jb;
        if (pairs_t) {
          const V3 Sl = v3(s_SD[kSDS * gg + 3], s_SD[kSDS * gg + 4], s_SD[kSDS * gg + 5]);
          la = la + Sl * ja;
          lb = lb + Sl * jb;
        }
      }
      V3 xb = cross(k, sa);
      if (lbk < 0 && dir == 0 && act) xb.z += s_db[r];  // ground: d = O_z + x_z (a pair's d: below)
      const V3 xk = cross(x, k);
      s_fr[r] = xk.x; s_fr[RC + r] = xk.y; s_fr[2 * RC + r] = xk.z;
      s_fr[3 * RC + r] = k.x; s_fr[4 * RC + r] = k.y; s_fr[5 * RC + r] = k.z;
      s_fr[6 * RC + r] = __uint_as_float(anc);
      if (pairs_t) {
        const V3 xq = x - dob;                      // the point about b's actor origin
        const V3 kxb = cross(k, sb);
        xb = xb - kxb;                              // d/dx through x_b
        const V3 kb = cross(sa, x) + la - cross(sb, xq) - lb;  // d/dk of both bodies' terms
        s_xb[XW * r + 3] = kxb.x; s_xb[XW * r + 4] = kxb.y; s_xb[XW * r + 5] = kxb.z;  // d/do_b
        s_xb[XW * r + 6] = kb.x; s_xb[XW * r + 7] = kb.y; s_xb[XW * r + 8] = kb.z;
        const V3 xqk = cross(xq, k);
        s_fr[7 * RC + r] = -xqk.x; s_fr[8 * RC + r] = -xqk.y; s_fr[9 * RC + r] = -xqk.z;
        s_fr[10 * RC + r] = -k.x; s_fr[11 * RC + r] = -k.y; s_fr[12 * RC + r] = -k.z;
        s_fr[13 * RC + r] = __uint_as_float(ancb);
      }
      s_xb[XW * r] = xb.x; s_xb[XW * r + 1] = xb.y; s_xb[XW * r + 2] = xb.z;
    }
    __syncwarp();
    // ---- reverse of the composite-rigid-body algorithm and the contact rows' S adjoints (DOF mode;
    // uniform trip counts, masks instead of branches) ----
    if (isg) {
      const int i = lane;
      const unsigned anc_i = T->anc[T->dof_link[i]];
      float Fb[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, Sb[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      for (int j = 0; j < n; ++j) {
        // F_bar_i = sum_{j <= i on i's path} w_ij S_j; S_bar_i = sum_{k >= i, i on k's path} w_ki F_k
        const float mij = s_Mb[i * LS + j], mji = s_Mb[j * LS + i];
        const float w = (j == i) ? mij : mij + mji;
        const float wf = (j <= i && ((anc_i >> j) & 1u)) ? w : 0.f;
        const float ws = (j >= i && ((T->anc[T->dof_link[j]] >> i) & 1u)) ? w : 0.f;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          Fb[k] += wf * s_SD[kSDS * j + k];
          Sb[k] += ws * s_FM[kSDS * j + k];
        }
      }
      {
        const float* ic = s_link + kAdjLinkWords * T->dof_link[i] + kRecIc;
        float t[6];
        inertia_mul(ic[0], v3(ic[1], ic[2], ic[3]), ic + 4, Fb, t);
#pragma unroll
        for (int k = 0; k < 6; ++k) Sb[k] += t[k];
      }
      // contact rows: J_ri = S_i . [x x k; k] on the contact link's path (and for a pair row
      // -S_i . [x_b x k; k] on body b's)
      for (int r = n_lim; r < R; ++r) {
        const unsigned mask = __float_as_uint(s_fr[6 * RC + r]);
        const float jb = ((mask >> i) & 1u) ? s_Yb[i * YS + r] : 0.f;
#pragma unroll
        for (int k = 0; k < 6; ++k) Sb[k] += jb * s_fr[k * RC + r];
        if (pairs_t) {
          const unsigned maskb = __float_as_uint(s_fr[13 * RC + r]);
          const float jbb = ((maskb >> i) & 1u) ? s_Yb[i * YS + r] : 0.f;
#pragma unroll
          for (int k = 0; k < 6; ++k) Sb[k] += jbb * s_fr[(7 + k) * RC + r];
        }
      }
#pragma unroll
      for (int k = 0; k < 6; ++k) { s_Sb[kSDS * i + k] = Sb[k]; s_FMb[kSDS * i + k] = Fb[k]; }
    }
    __syncwarp();

    // ---- capsule-box pair contacts (contact mode): the adjoints of each pair contact's point,
    // normal, friction directions, b's actor offset and separation, carried to the poses of its two
    // links and to the two actor origins by three forward-mode passes over the pair geometry (the
    // capsule link's twist, the box link's, the origins), into 18 words per contact: wrench on link
    // a (6) | on link b (6) | adjoint of a's actor origin (3) | of b's (3) ----
    float* s_pw = rws;  // (the row vectors of the gather above are dead)
    if (pairs_t) {
      for (int c = lane; c < n_con; c += G) {
        const int lbk = s_coni[5 * TL.ccap + c];
        if (lbk < 0) continue;
        const int rn = n_lim + c, rf = n_lim + n_con + 2 * c;
        V3 xa = v3(0.f, 0.f, 0.f), ob = xa;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const int r = q == 0 ? rn : rf + q - 1;
          xa = xa + v3(s_xb[XW * r], s_xb[XW * r + 1], s_xb[XW * r + 2]);
          ob = ob + v3(s_xb[XW * r + 3], s_xb[XW * r + 4], s_xb[XW * r + 5]);
        }
        const V3 nb = v3(s_xb[XW * rn + 6], s_xb[XW * rn + 7], s_xb[XW * rn + 8]);
        const V3 t1b = v3(s_xb[XW * rf + 6], s_xb[XW * rf + 7], s_xb[XW * rf + 8]);
        const V3 t2b = v3(s_xb[XW * (rf + 1) + 6], s_xb[XW * (rf + 1) + 7], s_xb[XW * (rf + 1) + 8]);
        const float dbn = s_db[rn];
        const int cand = s_coni[6 * TL.ccap + c] - T->n_ground_cand;
        const int p = cand / kPairSlots, slot = cand - kPairSlots * p;
        const bool a_cap = T->shape_type[T->pair_a[p]] == kCapsule;
        const int la_ = s_coni[3 * TL.ccap + c];
        const int lc = a_cap ? la_ : lbk, lx = a_cap ? lbk : la_;
        const float* Oc = img + TL.st + 2 * T->n_jdof + 13 * T->actor[lc];
        const float* Ox = img + TL.st + 2 * T->n_jdof + 13 * T->actor[lx];
        float w[3][6];
#pragma unroll 1
        for (int mode = 0; mode < 3; ++mode)
          pair_sample_adjoint(T, p, slot, s_pose + 12 * lc, s_pose + 12 * lc + 9, Oc, s_pose + 12 * lx,
                              s_pose + 12 * lx + 9, Ox, mode, xa, nb, t1b, t2b, dbn, w[mode]);
        float* o = s_pw + 18 * c;
#pragma unroll
        for (int k = 0; k < 6; ++k) { o[k] = a_cap ? w[0][k] : w[1][k]; o[6 + k] = a_cap ? w[1][k] : w[0][k]; }
        // origins: through the geometry, and o_b = O_b - O_a directly
        const V3 oc = v3(w[2][0], w[2][1], w[2][2]), ox = v3(w[2][3], w[2][4], w[2][5]);
        const V3 oa = (a_cap ? oc : ox) - ob, obb = (a_cap ? ox : oc) + ob;
        o[12] = oa.x; o[13] = oa.y; o[14] = oa.z; o[15] = obb.x; o[16] = obb.y; o[17] = obb.z;
      }
    }
    __syncwarp();

    // ---- link mode: gathers of the DOF- and row-level adjoints ----
    float IOb[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, hbar[3] = {0.f, 0.f, 0.f};  // composite inertia adjoint
    float wr[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // pose wrench of the link's attached quantities
    if (isl) {
      for (int gg = 0; gg < n; ++gg)
        if (T->dof_link[gg] == l) inertia_outer(s_FMb + kSDS * gg, s_SD + kSDS * gg, IOb, hbar);
      for (int c = 0; c < n_con; ++c) {
        const int la_ = s_coni[3 * TL.ccap + c];
        const int lbk = pairs_t ? s_coni[5 * TL.ccap + c] : -1;
        if (lbk >= 0) {  // a pair contact: the wrenches of the pair phase
          const float* o = s_pw + 18 * c;
          if (la_ == l)
#pragma unroll
            for (int k = 0; k < 6; ++k) wr[k] += o[k];
          if (lbk == l)
#pragma unroll
            for (int k = 0; k < 6; ++k) wr[k] += o[6 + k];
          continue;
        }
        if (la_ != l) continue;
        const int rn = n_lim + c, rf = n_lim + n_con + 2 * c;
        const V3 xb = v3(s_xb[XW * rn] + s_xb[XW * rf] + s_xb[XW * (rf + 1)],
                         s_xb[XW * rn + 1] + s_xb[XW * rf + 1] + s_xb[XW * (rf + 1) + 1],
                         s_xb[XW * rn + 2] + s_xb[XW * rf + 2] + s_xb[XW * (rf + 1) + 2]);
        const int sh = s_coni[4 * TL.ccap + c];
        const float rad = (T->shape_type[sh] == kBox) ? 0.f : T->shape_size[0][sh];
        // the body-fixed point: the contact point lies one radius straight below it
        const V3 xf = v3(s_con[c], s_con[TL.ccap + c], s_con[2 * TL.ccap + c] + rad);
        const V3 m = cross(xf, xb);
        wr[0] += m.x; wr[1] += m.y; wr[2] += m.z; wr[3] += xb.x; wr[4] += xb.y; wr[5] += xb.z;
      }
      if (has_dof) {
        for (int r = 0; r < n_lim; ++r) {  // joint limits: d = q - lo or hi - q
          const int a = s_rowa[r];
          if ((__float_as_int(s_rowc[r].z) & 3) == kRowLimit && (a & 0xff) == gd && s_rowc[r].y > 0.f)
            qb += ((a >> 8) & 1) ? -s_db[r] : s_db[r];
        }
        // fixed tendons (length l = sum c q): the limit rows' d = l - lo or hi - l, and the spring
        // -k (l - rest) - d l_dot acting on each of the tendon's joints with its coefficient
        for (int t = 0; t < T->n_tendons; ++t) {
          float mine = 0.f, fbar = 0.f;
          for (int k = 0; k < T->ten_n[t]; ++k) {
            const int lk = T->ten_link[t][k];
            const float c = T->ten_coef[t][k];
            if (lk == l) mine += c;
            fbar += c * V(kVCb)[T->gdof[lk]];  // adjoint of the tendon force: sum of c tau_bar
          }
          if (mine == 0.f) continue;
          qb -= T->ten_k[t] * mine * fbar;
          qdb -= T->ten_d[t] * mine * fbar;
          for (int r = 0; r < n_lim; ++r) {
            const int a = s_rowa[r];
            if ((__float_as_int(s_rowc[r].z) & 3) == kRowTendon && (a & 0xff) == t && s_rowc[r].y > 0.f)
              qb += ((a >> 8) & 1) ? -mine * s_db[r] : mine * s_db[r];
          }
        }
      }
      if (is_root)
        for (int c = 0; c < n_con; ++c) {
          const int la_ = s_coni[3 * TL.ccap + c];
          const int lbk = pairs_t ? s_coni[5 * TL.ccap + c] : -1;
          if (lbk >= 0) {  // the pair phase's origin adjoints
            const float* o = s_pw + 18 * c;
            if (T->actor[la_] == T->actor[l])
#pragma unroll
              for (int k = 0; k < 3; ++k) rpb[k] += o[12 + k];
            if (T->actor[lbk] == T->actor[l])
#pragma unroll
              for (int k = 0; k < 3; ++k) rpb[k] += o[15 + k];
          } else if (T->actor[la_] == T->actor[l]) {
            rpb[2] += s_db[n_lim + c];
          }
        }
    }
    {  // composite-inertia adjoints reach every link of the subtree: outward prefix over ancestors
      float t9[9] = {IOb[0], IOb[1], IOb[2], IOb[3], IOb[4], IOb[5], hbar[0], hbar[1], hbar[2]};
      outward(t9, 9);
#pragma unroll
      for (int k = 0; k < 6; ++k) IOb[k] = t9[k];
#pragma unroll
      for (int k = 0; k < 3; ++k) hbar[k] = t9[6 + k];
    }

    // ---- reverse of the recursive Newton-Euler algorithm at the recorded qdd, seeded -c_bar ----
    float Sbar[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (has_dof) {
#pragma unroll
      for (int k = 0; k < 6; ++k) Sbar[k] = s_Sb[kSDS * gd + k];
    }
    float vs[6], cc[6], io[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) { vs[k] = rec[kRecVs + k]; cc[k] = rec[kRecCc + k]; io[k] = rec[kRecIO + k]; }
    const float m_l = isl ? rec[kRecM] : 0.f;
    const V3 h_l = isl ? v3(rec[kRecH], rec[kRecH + 1], rec[kRecH + 2]) : v3(0.f, 0.f, 0.f);
    const float qdd_l = has_dof ? V(kVQdd)[gd] : 0.f;
    float acc[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) acc[k] = isl ? cc[k] + S[k] * qdd_l : 0.f;
    if (free_root) {
#pragma unroll
      for (int k = 0; k < 6; ++k) acc[k] += V(kVQdd)[gd + k];
    }
    float bSb[3][6];  // ball: the three columns' S adjoints
    if (BALL) {
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int k = 0; k < 6; ++k) bSb[c][k] = is_ball ? s_Sb[kSDS * (gd + c) + k] : 0.f;
      if (is_ball)
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int k = 0; k < 6; ++k) acc[k] += s_SD[kSDS * (gd + c) + k] * V(kVQdd)[gd + c];
    }
    outward(acc, 6);
    float ag[6] = {acc[0], acc[1], acc[2], acc[3] - g.x, acc[4] - g.y, acc[5] - g.z};
    float u[6], Fc[6];
    inertia_mul(m_l, h_l, io, vs, u);
    // external force and torque at the COM (world axes; constants of the derivative), as in the step
    V3 fe = v3(0.f, 0.f, 0.f), te = fe;
    const int bdy = isl ? T->body[l] : -1;
    if ((A.flags & SIM_STEP_BODY_FORCES) && bdy >= 0) {
      const float* bf = A.body_force + (size_t)(A.env_body_base[env] + bdy) * 6;
      fe = v3(bf[0], bf[1], bf[2]);
      te = v3(bf[3], bf[4], bf[5]);
    }
    {
      float ia[6], vu[6];
      inertia_mul(m_l, h_l, io, ag, ia);
      crf6(vs, u, vu);
      const V3 cwl = isl ? v3(rec[kRecCw], rec[kRecCw + 1], rec[kRecCw + 2]) : v3(0.f, 0.f, 0.f);
      const V3 na = cross(cwl, fe) + te;
      const float fx[6] = {na.x, na.y, na.z, fe.x, fe.y, fe.z};
#pragma unroll
      for (int k = 0; k < 6; ++k) Fc[k] = isl ? ia[k] + vu[k] - fx[k] : 0.f;
    }
    inward6(Fc);
    float fb[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (has_dof) {
      const float cb = V(kVCb)[gd];
#pragma unroll
      for (int k = 0; k < 6; ++k) { fb[k] = -cb * S[k]; Sbar[k] -= cb * Fc[k]; }
    }
    if (free_root) {
#pragma unroll
      for (int k = 0; k < 6; ++k) fb[k] = -V(kVCb)[gd + k];
    }
    if (is_ball) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float cb = V(kVCb)[gd + c];
#pragma unroll
        for (int k = 0; k < 6; ++k) { fb[k] -= cb * s_SD[kSDS * (gd + c) + k]; bSb[c][k] -= cb * Fc[k]; }
      }
    }
    outward(fb, 6);
    float accb[6], vsb[6];
    // adjoint of the COM position from the external force's moment -(c x F): f_bar_ang x F
    const V3 cwb_ext = cross(v3(fb[0], fb[1], fb[2]), fe);
    {
      float ub[6], t[6];
      crm6(vs, fb, ub);
#pragma unroll
      for (int k = 0; k < 6; ++k) ub[k] = -ub[k];
      inertia_outer(fb, ag, IOb, hbar);
      inertia_outer(ub, vs, IOb, hbar);
      inertia_mul(m_l, h_l, io, fb, accb);
      inertia_mul(m_l, h_l, io, ub, t);
      const V3 ua = v3(u[0], u[1], u[2]), ul = v3(u[3], u[4], u[5]);
      const V3 fa = v3(fb[0], fb[1], fb[2]), fl = v3(fb[3], fb[4], fb[5]);
      const V3 b0 = cross(ua, fa) + cross(ul, fl), b1 = cross(ul, fa);
      vsb[0] = b0.x + t[0]; vsb[1] = b0.y + t[1]; vsb[2] = b0.z + t[2];
      vsb[3] = b1.x + t[3]; vsb[4] = b1.y + t[4]; vsb[5] = b1.z + t[5];
      if (!isl) {
#pragma unroll
        for (int k = 0; k < 6; ++k) { accb[k] = 0.f; vsb[k] = 0.f; }
      }
    }
    inward6(accb);  // acc_bar summed over the subtree: the adjoint of c and of S qdd
    if (has_dof) {
#pragma unroll
      for (int k = 0; k < 6; ++k) Sbar[k] += accb[k] * qdd_l;
      // c = v x (S qd): v_bar += (S qd) x* c_bar, (S qd)_bar = -v x* c_bar
      float sq[6], t[6], sqb[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) sq[k] = S[k] * qd;
      crf6(sq, accb, t);
      crf6(vs, accb, sqb);
#pragma unroll
      for (int k = 0; k < 6; ++k) { vsb[k] += t[k]; Sbar[k] -= sqb[k] * qd; qdb -= S[k] * sqb[k]; }
    }
    if (is_ball) {
      float sq[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, t[6], sqb[6];
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          const float Sck = s_SD[kSDS * (gd + c) + k];
          sq[k] += Sck * bw[c];
          bSb[c][k] += accb[k] * V(kVQdd)[gd + c];
        }
      crf6(sq, accb, t);
      crf6(vs, accb, sqb);
#pragma unroll
      for (int k = 0; k < 6; ++k) vsb[k] += t[k];
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int k = 0; k < 6; ++k) { bSb[c][k] -= sqb[k] * bw[c]; bwb[c] -= s_SD[kSDS * (gd + c) + k] * sqb[k]; }
    }
    if (free_root) {  // c_root = [0; p_dot x omega]
      const V3 cb = v3(accb[3], accb[4], accb[5]);
      const V3 a = cross(rw, cb), b = cross(cb, rv);
      rvb[0] += a.x; rvb[1] += a.y; rvb[2] += a.z;
      rwb[0] += b.x; rwb[1] += b.y; rwb[2] += b.z;
    }
    inward6(vsb);  // v = v_parent + S qd
    if (has_dof) {
#pragma unroll
      for (int k = 0; k < 6; ++k) { Sbar[k] += vsb[k] * qd; qdb += S[k] * vsb[k]; }
    }
    if (is_ball) {
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int k = 0; k < 6; ++k) { bSb[c][k] += vsb[k] * bw[c]; bwb[c] += s_SD[kSDS * (gd + c) + k] * vsb[k]; }
    }
    if (free_root) {
#pragma unroll
      for (int k = 0; k < 3; ++k) { rwb[k] += vsb[k]; rvb[k] += vsb[3 + k]; }
    }

    // ---- configuration: wrenches of S, the inertia and the contact points, summed over subtrees ----
    if (isl) {
      if (has_dof) {
        float t[6];
        crf6(S, Sbar, t);
#pragma unroll
        for (int k = 0; k < 6; ++k) wr[k] += t[k];
      }
      if (is_ball) {  // the columns are the child's axes: they turn with the link
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          float t[6], Sc[6];
#pragma unroll
          for (int k = 0; k < 6; ++k) Sc[k] = s_SD[kSDS * (gd + c) + k];
          crf6(Sc, bSb[c], t);
#pragma unroll
          for (int k = 0; k < 6; ++k) wr[k] += t[k];
        }
      }
      const V3 cw = v3(rec[kRecCw], rec[kRecCw + 1], rec[kRecCw + 2]);
      const float* icw = rec + kRecIcw;
      const float tr = IOb[0] + IOb[1] + IOb[2];
      const V3 gc = (cw * (2.f * tr) - sym_mv(IOb, cw) * 2.f) * m_l + v3(hbar[0], hbar[1], hbar[2]) * m_l + cwb_ext;
      // B = IOb Icw; vee(B - B^T) = 2 (B21 - B12, B02 - B20, B10 - B01)
      const float B01 = IOb[0] * icw[3] + IOb[3] * icw[1] + IOb[4] * icw[5];
      const float B02 = IOb[0] * icw[4] + IOb[3] * icw[5] + IOb[4] * icw[2];
      const float B10 = IOb[3] * icw[0] + IOb[1] * icw[3] + IOb[5] * icw[4];
      const float B12 = IOb[3] * icw[4] + IOb[1] * icw[5] + IOb[5] * icw[2];
      const float B20 = IOb[4] * icw[0] + IOb[5] * icw[3] + IOb[2] * icw[4];
      const float B21 = IOb[4] * icw[3] + IOb[5] * icw[1] + IOb[2] * icw[5];
      const V3 nrot = v3(2.f * (B21 - B12), 2.f * (B02 - B20), 2.f * (B10 - B01)) + cross(cw, gc);
      wr[0] += nrot.x; wr[1] += nrot.y; wr[2] += nrot.z; wr[3] += gc.x; wr[4] += gc.y; wr[5] += gc.z;
    }
    inward6(wr);
    if (has_dof) {
#pragma unroll
      for (int k = 0; k < 6; ++k) qb += S[k] * wr[k];
    }
    if (is_ball) {
      // the subtree turns about the child's axes by J_r(q) dq (exp(q + dq) = exp(q) exp(J_r dq)):
      // q_bar += J_r^T p, p_c = S_c . wr, J_r^T p = p + a q x p + b q x (q x p)
      V3 pp = v3(0.f, 0.f, 0.f);
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        pp.x += s_SD[kSDS * gd + k] * wr[k];
        pp.y += s_SD[kSDS * (gd + 1) + k] * wr[k];
        pp.z += s_SD[kSDS * (gd + 2) + k] * wr[k];
      }
      const V3 qv = v3(bq[0], bq[1], bq[2]);
      const float a2 = dot(qv, qv);
      float ca, cb;
      if (a2 < 1e-8f) {
        ca = 0.5f - a2 / 24.f;
        cb = 1.f / 6.f - a2 / 120.f;
      } else {
        const float an = sqrtf(a2);
        float sn, cs;
        sincosf(an, &sn, &cs);
        ca = (1.f - cs) / a2;
        cb = (an - sn) / (a2 * an);
      }
      const V3 qp = cross(qv, pp);
      const V3 jt3 = pp + qp * ca + cross(qv, qp) * cb;
      bqb[0] += jt3.x; bqb[1] += jt3.y; bqb[2] += jt3.z;
    }
    if (is_root) { thb[0] += wr[0]; thb[1] += wr[1]; thb[2] += wr[2]; }

    // ---- joint forces (actuation, damping, drives) and v_free = nu + h qdd ----
    if (isg) V(kVVb)[lane] = vfb;
    __syncwarp();
    if (has_dof) {
      const float cb = V(kVCb)[gd];
      actb += cb;
      float dq_damp = T->damping[l];
      if (T->has_drives) {
        const float kp = T->drive_kp[l], kd = T->drive_kd[l];
        dq_damp += kd + h * kp;
        qb -= kp * cb;
      }
      qdb -= dq_damp * cb;
      qdb += V(kVVb)[gd];
    }
    if (free_root) {
#pragma unroll
      for (int k = 0; k < 3; ++k) { rwb[k] += V(kVVb)[gd + k]; rvb[k] += V(kVVb)[gd + 3 + k]; }
    }
    if (is_ball) {  // tau = actuation - damping qd per DOF
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float cb = V(kVCb)[gd + c];
        bab[c] += cb;
        bwb[c] -= T->damping[l] * cb;
        bwb[c] += V(kVVb)[gd + c];
      }
    }
    // ---- input impulse cache adjoint: the warm-start impulses' adjoints at their slots ----
    if (live)
      for (int i = lane; i < A.cache_stride; i += G) cacheb[i] = 0.f;
    __syncwarp();
    if (live)
      for (int r = lane; r < R; r += G)
        if (s_rowc[r].y > 0.f) cacheb[__float_as_int(s_rowc[r].w)] = s_lamb[r];
    __syncwarp();
    // ---- the input quaternion's adjoint from the rotation adjoint: q_bar = 2 [th_bar; 0] (x) q ----
    if (is_root) {
      const float t4[4] = {thb[0], thb[1], thb[2], 0.f};
      float o4[4];
      qmul4(t4, rq, o4);
#pragma unroll
      for (int k = 0; k < 4; ++k) rqb[k] = 2.f * o4[k];
    }
    __syncwarp();
  }  // substeps

  // ---- outputs ----
  int status = failed ? 4 : 0;
  if (failed) {  // no gradient for an env whose tape did not arrive
    qb = qdb = actb = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) { bqb[c] = 0.f; bwb[c] = 0.f; bab[c] = 0.f; }
#pragma unroll
    for (int k = 0; k < 3; ++k) { rpb[k] = 0.f; rwb[k] = 0.f; rvb[k] = 0.f; }
#pragma unroll
    for (int k = 0; k < 4; ++k) rqb[k] = 0.f;
  }
  if (has_dof && !(isfinite(qb) && isfinite(qdb) && isfinite(actb))) status = 2;
  if (is_ball && !(isfinite(bqb[0] + bqb[1] + bqb[2]) && isfinite(bwb[0] + bwb[1] + bwb[2]) &&
                   isfinite(bab[0] + bab[1] + bab[2])))
    status = 2;
  if (is_root && !(isfinite(rpb[0] + rpb[1] + rpb[2]) && isfinite(rqb[0] + rqb[1] + rqb[2] + rqb[3]) &&
                   isfinite(rwb[0] + rwb[1] + rwb[2]) && isfinite(rvb[0] + rvb[1] + rvb[2])))
    status = 2;
  status = Grp<G>::any(status);
  if (live) {
    if (has_dof) {
      J.gi_dof[(size_t)(dof_base + jd) * 2] = qb;
      J.gi_dof[(size_t)(dof_base + jd) * 2 + 1] = qdb;
      J.gi_act[dof_base + jd] = actb;
    }
    if (is_ball) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        J.gi_dof[(size_t)(dof_base + jd + c) * 2] = bqb[c];
        J.gi_dof[(size_t)(dof_base + jd + c) * 2 + 1] = bwb[c];
        J.gi_act[dof_base + jd + c] = bab[c];
      }
    }
    if (is_root) {
      float* o = J.gi_root + (size_t)actor_row * 13;
#pragma unroll
      for (int k = 0; k < 3; ++k) { o[k] = rpb[k]; o[7 + k] = free_root ? rvb[k] : 0.f; o[10 + k] = free_root ? rwb[k] : 0.f; }
#pragma unroll
      for (int k = 0; k < 4; ++k) o[3 + k] = rqb[k];
    }
    if (lane == 0 && J.status) J.status[env] = status;
  }
}

// One launch per env type: blocks of blockDim / G groups, one env per group.
template <int G, bool PAIRS, bool BALL>
__global__ void __launch_bounds__(64) adjoint_kernel(const __grid_constant__ StepArgs A,
                                                    const __grid_constant__ TypeArgs TA,
                                                    const __grid_constant__ AdjArgs J) {
  extern __shared__ __align__(16) float smem[];
  const int grp_blk = threadIdx.x / G;
  const int grp = blockIdx.x * (blockDim.x / G) + grp_blk;
  adjoint_group<G, PAIRS, BALL>(A, TA, J, grp, smem + grp_blk * J.al.total);
}

}  // namespace artsim
