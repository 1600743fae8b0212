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
// Constraint response. With M = L L^T (Cholesky) and Y = L^-1 J^T, the solve runs in the
// coordinates z = L^T v: J_r v = Y_r . z, the impulse update v += M^-1 J_r^T dl becomes
// z += Y_r dl, and J_r M^-1 J_r^T = |Y_r|^2. Only Y (n x R) is stored; v = L^-T z at the end.
// The TGS-style solve follows the paper's TGS paragraph: position iterations accumulate
// h/n_pos * v into the delta buffer dq (here dz = L^T dq), which is projected onto each row's
// Jacobian and added to its bias; velocity iterations are unbiased.
//
// Lane roles: "link mode" lane l = env link l; "DOF mode" lane g = generalized DOF g; "row mode"
// lane r = constraint row r (strided by G); "shape mode" lane s = shape s. Every loop whose body
// shuffles or synchronises has a warp-uniform trip count (the groups of one launch share one env
// type; row loops use the maximum over the warp), so the groups of one warp stay converged.
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
// Unit quaternion (x, y, z, w), w >= 0, of a row-major rotation matrix (Shepperd's method: the
// largest of 4w^2, 4x^2, 4y^2, 4z^2 picks the square root taken).
__device__ __forceinline__ void mat_to_quat(const float* R, float* q) {
  const float tr = R[0] + R[4] + R[8];
  float x, y, z, w;
  if (tr > 0.f) {
    const float s = sqrtf(tr + 1.f) * 2.f;
    w = 0.25f * s; x = (R[7] - R[5]) / s; y = (R[2] - R[6]) / s; z = (R[3] - R[1]) / s;
  } else if (R[0] > R[4] && R[0] > R[8]) {
    const float s = sqrtf(1.f + R[0] - R[4] - R[8]) * 2.f;
    w = (R[7] - R[5]) / s; x = 0.25f * s; y = (R[1] + R[3]) / s; z = (R[2] + R[6]) / s;
  } else if (R[4] > R[8]) {
    const float s = sqrtf(1.f + R[4] - R[0] - R[8]) * 2.f;
    w = (R[2] - R[6]) / s; x = (R[1] + R[3]) / s; y = 0.25f * s; z = (R[5] + R[7]) / s;
  } else {
    const float s = sqrtf(1.f + R[8] - R[0] - R[4]) * 2.f;
    w = (R[3] - R[1]) / s; x = (R[2] + R[6]) / s; y = (R[5] + R[7]) / s; z = 0.25f * s;
  }
  const float sg = (w < 0.f) ? -1.f : 1.f;
  q[0] = sg * x; q[1] = sg * y; q[2] = sg * z; q[3] = sg * w;
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

// Unit quaternion (x, y, z, w) of the rotation vector r: rotation by |r| about r / |r|.
__device__ __forceinline__ void rotvec_quat(float rx, float ry, float rz, float* e) {
  const float a2 = rx * rx + ry * ry + rz * rz;
  if (a2 < 1e-30f) {  // sin(a/2)/a -> 1/2
    e[0] = 0.5f * rx; e[1] = 0.5f * ry; e[2] = 0.5f * rz; e[3] = 1.f;
    return;
  }
  const float an = sqrtf(a2);
  float sn, cs;
  sincosf(0.5f * an, &sn, &cs);
  const float sc = sn / an;
  e[0] = rx * sc; e[1] = ry * sc; e[2] = rz * sc; e[3] = cs;
}
// Rotation vector of the quaternion q (need not be exactly unit): the shorter rotation (w >= 0),
// angle 2 atan2(|v|, w) about v / |v|.
__device__ __forceinline__ void quat_rotvec(const float* q, float* r) {
  const float sg = q[3] < 0.f ? -1.f : 1.f;
  const float x = sg * q[0], y = sg * q[1], z = sg * q[2], w = sg * q[3];
  const float s2 = x * x + y * y + z * z;
  float f;
  if (s2 < 1e-30f) {
    f = 2.f / w;
  } else {
    const float sn = sqrtf(s2);
    f = 2.f * atan2f(sn, w) / sn;
  }
  r[0] = x * f; r[1] = y * f; r[2] = z * f;
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
// Capsule-box geometry (box frame). All three follow the definitions the FP64 oracle applies.
__device__ __forceinline__ float comp(V3 v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : v.z); }
__device__ __forceinline__ float box_dist2(V3 p, V3 e) {
  const float ox = fmaxf(fabsf(p.x) - e.x, 0.f), oy = fmaxf(fabsf(p.y) - e.y, 0.f), oz = fmaxf(fabsf(p.z) - e.z, 0.f);
  return ox * ox + oy * oy + oz * oz;
}
// Exact minimiser over [0, 1] of the squared distance from p0 + t dv to the box: pieces between the
// breakpoints |p_k(t)| = e_k, each piece's stationary point clamped into it (its start if the
// distance is constant there); smallest value wins, ties to the smallest t.
__device__ inline float segment_box_closest_t(V3 p0, V3 dv, V3 e) {
  float ts[8];
  int nt = 0;
  ts[nt++] = 0.f;
  ts[nt++] = 1.f;
  for (int k = 0; k < 3; ++k) {
    const float dk = comp(dv, k), pk = comp(p0, k), ek = comp(e, k);
    if (dk == 0.f) continue;
    for (int s = -1; s <= 1; s += 2) {
      const float t = ((float)s * ek - pk) / dk;
      if (t > 0.f && t < 1.f) ts[nt++] = t;
    }
  }
  for (int i = 1; i < nt; ++i) {  // insertion sort
    const float x = ts[i];
    int j = i - 1;
    while (j >= 0 && x < ts[j]) { ts[j + 1] = ts[j]; --j; }
    ts[j + 1] = x;
  }
  float best_t = 0.f, best_f = box_dist2(p0, e);
  for (int i = 0; i + 1 < nt; ++i) {
    const float ta = ts[i], tb = ts[i + 1];
    const V3 pm = p0 + dv * ((ta + tb) * 0.5f);
    float num = 0.f, den = 0.f;
    for (int k = 0; k < 3; ++k) {
      const float pk = comp(pm, k), ek = comp(e, k), dk = comp(dv, k);
      if (!(ek < fabsf(pk))) continue;
      const float s = (pk > 0.f) ? 1.f : -1.f;
      num += dk * (s * ek - comp(p0, k));
      den += dk * dk;
    }
    float t = ta;
    if (den > 0.f) t = fminf(fmaxf(num / den, ta), tb);
    const float f = box_dist2(p0 + dv * t, e);
    if (f < best_f) { best_f = f; best_t = t; }
  }
  if (box_dist2(p0 + dv, e) < best_f) best_t = 1.f;
  return best_t;
}
// A sphere of radius r at p against the box: normal from the box to the sphere, separation, and
// the point halfway between the two surfaces.
__device__ __forceinline__ void sphere_box(V3 p, float r, V3 e, V3& n, float& d, V3& x) {
  const bool inside = fabsf(p.x) <= e.x && fabsf(p.y) <= e.y && fabsf(p.z) <= e.z;
  if (!inside) {
    const V3 q = v3(fminf(fmaxf(p.x, -e.x), e.x), fminf(fmaxf(p.y, -e.y), e.y), fminf(fmaxf(p.z, -e.z), e.z));
    const V3 dl = p - q;
    const float dist = sqrtf(dot(dl, dl));
    n = dl * (1.f / dist);
    d = dist - r;
  } else {
    int kb = 0;
    float best = e.x - fabsf(p.x);
    if (e.y - fabsf(p.y) < best) { best = e.y - fabsf(p.y); kb = 1; }
    if (e.z - fabsf(p.z) < best) { best = e.z - fabsf(p.z); kb = 2; }
    const float s = (comp(p, kb) < 0.f) ? -1.f : 1.f;
    n = v3(kb == 0 ? s : 0.f, kb == 1 ? s : 0.f, kb == 2 ? s : 0.f);
    d = -best - r;
  }
  x = p - n * (r + 0.5f * d);
}
// The part of the segment over the box face selected by the closest point: clip to the slabs of
// the two axes other than the one along which the normal at t* is largest.
__device__ __forceinline__ bool face_clip(V3 p0, V3 dv, V3 e, float r, float tstar, float& ta, float& tb) {
  V3 n, x;
  float d;
  sphere_box(p0 + dv * tstar, r, e, n, d, x);
  int kn = 0;
  if (fabsf(n.x) < fabsf(n.y)) kn = 1;
  if (fabsf(comp(n, kn)) < fabsf(n.z)) kn = 2;
  ta = 0.f;
  tb = 1.f;
  for (int j = 0; j < 3; ++j) {
    if (j == kn) continue;
    const float dj = comp(dv, j), pj = comp(p0, j), ej = comp(e, j);
    if (dj == 0.f) {
      if (ej < fabsf(pj)) return false;
      continue;
    }
    float t0 = (-ej - pj) / dj, t1 = (ej - pj) / dj;
    if (t1 < t0) { const float s = t0; t0 = t1; t1 = s; }
    ta = fmaxf(ta, t0);
    tb = fminf(tb, t1);
  }
  return !(tb < ta);
}
// Friction directions of a contact normal: anchor e_x if |n_x| < 0.57735, else e_y if
// |n_y| < 0.57735, else e_z; t1 = normalise(anchor - (anchor . n) n), t2 = n x t1.
__device__ __forceinline__ void tangent_basis(V3 n, V3& t1, V3& t2) {
  V3 an = (fabsf(n.x) < 0.57735f) ? v3(1.f, 0.f, 0.f) : ((fabsf(n.y) < 0.57735f) ? v3(0.f, 1.f, 0.f) : v3(0.f, 0.f, 1.f));
  const V3 t = an - n * dot(an, n);
  t1 = t * (1.f / sqrtf(dot(t, t)));
  t2 = cross(n, t1);
}

// Row header words (float4 per row, constant during the solve):
//   x: separation d (limit / normal rows) or friction coefficient (friction rows)
//   y: 1 / (J M^-1 J^T), 0 for a row without response (skipped)
//   z: int bits: kind | normal_row << 2
//   w: int bits: impulse-cache slot
// rowa (int per row): limit rows: g | side << 8 | jd << 16; contact rows: c | dir << 8
// (dir 0 = normal e_z, 1 = e_x, 2 = e_y).

struct Mat9 { float m[9]; };

// Capsule-box pair contacts of one env (lane = pair, in chunks of G), appended to the contact
// records after the n_con ground contacts in pair / slot order; returns the new count. A separate
// function (not inlined) so its register pressure does not spill into the rest of the step.
template <int G>
__device__ __noinline__ int pair_contacts(const EnvTypeTable* __restrict__ T, const int lane, const Mat9 Rw, const V3 P,
                                          const V3 rp, float* s_con, int* s_coni, const int CC, int n_con,
                                          const float coff) {
  for (int pc = 0; pc < T->n_pairs; pc += G) {
    const int p = pc + lane;
    const bool isp = p < T->n_pairs;
    const int sa = isp ? T->pair_a[p] : 0, sb = isp ? T->pair_b[p] : 0;
    const bool a_cap = T->shape_type[sa] == kCapsule;
    const int sc = a_cap ? sa : sb, sx = a_cap ? sb : sa;  // the capsule and the box
    const int lc = T->shape_link[sc], lx = T->shape_link[sx];
    const int rc = T->aroot[lc], rxl = T->aroot[lx];
    float Rc[9], Rx[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) { Rc[k] = Grp<G>::get(Rw.m[k], lc); Rx[k] = Grp<G>::get(Rw.m[k], lx); }
    const V3 Pc = v3(Grp<G>::get(P.x, lc), Grp<G>::get(P.y, lc), Grp<G>::get(P.z, lc));
    const V3 Px = v3(Grp<G>::get(P.x, lx), Grp<G>::get(P.y, lx), Grp<G>::get(P.z, lx));
    const V3 Oc = v3(Grp<G>::get(rp.x, rc), Grp<G>::get(rp.y, rc), Grp<G>::get(rp.z, rc));
    const V3 Ox = v3(Grp<G>::get(rp.x, rxl), Grp<G>::get(rp.y, rxl), Grp<G>::get(rp.z, rxl));
    unsigned pk = 0u;
    V3 pn[kPairSlots], px[kPairSlots];
    float pd[kPairSlots];
    V3 Rb3[3];
    V3 cb = v3(0.f, 0.f, 0.f);
    if (isp) {
      float Rsh[9], Rcs[9], Rb[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) Rsh[k] = T->shape_rot[k][sc];
      mm(Rc, Rsh, Rcs);
#pragma unroll
      for (int k = 0; k < 9; ++k) Rsh[k] = T->shape_rot[k][sx];
      mm(Rx, Rsh, Rb);
      // everything relative to the box actor's origin
      const V3 cc = Pc + mv(Rc, v3(T->shape_pos[0][sc], T->shape_pos[1][sc], T->shape_pos[2][sc])) + (Oc - Ox);
      cb = Px + mv(Rx, v3(T->shape_pos[0][sx], T->shape_pos[1][sx], T->shape_pos[2][sx]));
      const float r = T->shape_size[0][sc], hl = T->shape_size[1][sc];
      const V3 ax = v3(Rcs[0], Rcs[3], Rcs[6]);
      const V3 e = v3(T->shape_size[0][sx], T->shape_size[1][sx], T->shape_size[2][sx]);
      Rb3[0] = v3(Rb[0], Rb[3], Rb[6]);  // box axes (columns) in world
      Rb3[1] = v3(Rb[1], Rb[4], Rb[7]);
      Rb3[2] = v3(Rb[2], Rb[5], Rb[8]);
      const V3 w0 = cc - ax * hl - cb, w1 = cc + ax * hl - cb;
      const V3 p0 = v3(dot(Rb3[0], w0), dot(Rb3[1], w0), dot(Rb3[2], w0));
      const V3 p1 = v3(dot(Rb3[0], w1), dot(Rb3[1], w1), dot(Rb3[2], w1));
      const V3 dv = p1 - p0;
      const float tstar = segment_box_closest_t(p0, dv, e);
      float ta, tb;
      const bool clip = face_clip(p0, dv, e, r, tstar, ta, tb);
#pragma unroll
      for (int slot = 0; slot < kPairSlots; ++slot) {
        float t = (slot == 0) ? 0.f : ((slot == 1) ? 1.f : ((slot == 2) ? ta : ((slot == 3) ? tb : tstar)));
        bool ok = true;
        if (slot >= 2) {
          if (slot < 4 && !clip) ok = false;
          if (slot == 3 && !(ta < tb)) ok = false;
          if (!(t > 0.f && t < 1.f)) ok = false;
        }
        if (ok) {
          sphere_box(p0 + dv * t, r, e, pn[slot], pd[slot], px[slot]);
          if (pd[slot] < coff) pk |= 1u << slot;
        }
      }
    }
    int nchunk;
    const int pbase = n_con + Grp<G>::excl_scan(__popc(pk), lane, &nchunk);
    if (isp && pk) {
      int o = pbase;
      const int ao = a_cap ? rc : rxl, bo = a_cap ? rxl : rc;   // actor roots of bodies a and b
      const V3 Oa = a_cap ? Oc : Ox, Ob = a_cap ? Ox : Oc;
      const float mu = fmaxf(T->shape_fr[sa], T->shape_fr[sb]);
      (void)ao; (void)bo;
#pragma unroll
      for (int slot = 0; slot < kPairSlots; ++slot) {
        if (!((pk >> slot) & 1u)) continue;
        V3 nw = Rb3[0] * pn[slot].x + Rb3[1] * pn[slot].y + Rb3[2] * pn[slot].z;  // box -> capsule
        if (!a_cap) nw = nw * -1.f;
        const V3 xw = cb + Rb3[0] * px[slot].x + Rb3[1] * px[slot].y + Rb3[2] * px[slot].z + (Ox - Oa);
        const V3 dob = Ob - Oa;
        s_con[0 * CC + o] = xw.x;
        s_con[1 * CC + o] = xw.y;
        s_con[2 * CC + o] = xw.z;
        s_con[3 * CC + o] = pd[slot];
        s_con[4 * CC + o] = mu;
        s_coni[5 * CC + o] = a_cap ? lc : lx;
        s_coni[6 * CC + o] = T->n_ground_cand + kPairSlots * p + slot;
        s_coni[7 * CC + o] = sa;
        s_coni[8 * CC + o] = slot;
        s_coni[9 * CC + o] = a_cap ? lx : lc;
        s_coni[10 * CC + o] = sb;
        s_con[11 * CC + o] = nw.x;
        s_con[12 * CC + o] = nw.y;
        s_con[13 * CC + o] = nw.z;
        s_con[14 * CC + o] = dob.x;
        s_con[15 * CC + o] = dob.y;
        s_con[16 * CC + o] = dob.z;
        ++o;
      }
    }
    n_con += nchunk;
  }
  return n_con;
}

// ---------------------------------------------------------------------------------------------
// Ball-joint block of the articulated-body inward sweep (RBDA Table 7.1, a 3-DOF joint): with IA,
// pA the link's articulated inertia (packed symmetric, 21) and bias (6) in its hand-off slot sl and
// S the joint's three motion-subspace columns (world axes about the actor origin), U = IA S,
// D = S^T U + armature I, u = tau - S^T pA with tau = actuation - damping qd (bl's state words);
// the slot becomes Ia = IA - U D^-1 U^T and pa = pA + Ia c + U D^-1 u, and U, D^-1 (00 11 22 01
// 02 12) and u go to bl for the outward sweep.
// Returns the status bit 2 if D is not positive definite (D^-1 = I is used then).
static __device__ __noinline__ int ball_joint_block(float* sl, float* bl, const float* S, const float c0, const float c1,
                                             const float c2, const float c3, const float c4, const float c5,
                                             const float damping, const float arm) {
  const float cc[6] = {c0, c1, c2, c3, c4, c5};
  float tau3[3];  // actuation - damping qd (from the joint's state words of bl)
#pragma unroll
  for (int k = 0; k < 3; ++k) tau3[k] = bl[33 + k] - damping * bl[30 + k];
  int st = 0;
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      float t = 0.f;
#pragma unroll
      for (int j = 0; j < 6; ++j) t += sl[sidx(i, j)] * S[6 * c + j];
      bl[6 * c + i] = t;
    }
  float Dm[9], u3[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float sp = 0.f;
#pragma unroll
    for (int i = 0; i < 6; ++i) sp += S[6 * c + i] * sl[21 + i];
    u3[c] = tau3[c] - sp;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      float t = 0.f;
#pragma unroll
      for (int i = 0; i < 6; ++i) t += S[6 * c + i] * bl[6 * m + i];
      Dm[3 * c + m] = t;
    }
    Dm[4 * c] += arm;
  }
  // symmetric inverse by cofactors
  const float a = Dm[0], b = Dm[4], cz = Dm[8];
  const float dxy = 0.5f * (Dm[1] + Dm[3]), dxz = 0.5f * (Dm[2] + Dm[6]), dyz = 0.5f * (Dm[5] + Dm[7]);
  const float k00 = b * cz - dyz * dyz, k01 = dxz * dyz - dxy * cz, k02 = dxy * dyz - b * dxz;
  const float k11 = a * cz - dxz * dxz, k12 = dxy * dxz - a * dyz, k22 = a * b - dxy * dxy;
  const float det = a * k00 + dxy * k01 + dxz * k02;
  float Di[6];
  if (!(a > 0.f && k22 > 0.f && det > 0.f)) {
    st = 2;
    Di[0] = 1.f; Di[1] = 1.f; Di[2] = 1.f; Di[3] = 0.f; Di[4] = 0.f; Di[5] = 0.f;
  } else {
    const float id = 1.f / det;
    Di[0] = k00 * id; Di[1] = k11 * id; Di[2] = k22 * id; Di[3] = k01 * id; Di[4] = k02 * id; Di[5] = k12 * id;
  }
  const float D9[9] = {Di[0], Di[3], Di[4], Di[3], Di[1], Di[5], Di[4], Di[5], Di[2]};
#pragma unroll
  for (int k = 0; k < 6; ++k) bl[18 + k] = Di[k];
#pragma unroll
  for (int k = 0; k < 3; ++k) bl[24 + k] = u3[k];
  float w3[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) w3[c] = D9[3 * c] * u3[0] + D9[3 * c + 1] * u3[1] + D9[3 * c + 2] * u3[2];
  // Ia = IA - sum_c U_c V_c^T, V_c = sum_m D^-1_cm U_m
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float Uc[6], Vc[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      Uc[i] = bl[6 * c + i];
      Vc[i] = D9[3 * c] * bl[i] + D9[3 * c + 1] * bl[6 + i] + D9[3 * c + 2] * bl[12 + i];
    }
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int j = i; j < 6; ++j) sl[sidx(i, j)] -= Uc[i] * Vc[j];
  }
  float pa[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    float t = sl[21 + i] + bl[i] * w3[0] + bl[6 + i] * w3[1] + bl[12 + i] * w3[2];
#pragma unroll
    for (int j = 0; j < 6; ++j) t += sl[sidx(i, j)] * cc[j];
    pa[i] = t;
  }
#pragma unroll
  for (int i = 0; i < 6; ++i) sl[21 + i] = pa[i];
  return st;
}

// ---------------------------------------------------------------------------------------------
// Row form of the projected Gauss-Seidel solve in z = L^T v: per row, J_r v = Y_r . z comes from
// a group reduction, and z moves by Y_r dl; the separations d_r + Y_r . dz are formed once per
// iteration into s_sep (R words; s_dz, n words, is scratch). Starts from z_free (z0 of the DOF
// lane) plus the warm start; returns (z, dz) of the lane. The impulses are updated in s_lam.
template <int G>
__device__ __noinline__ float2 pgs_row_form(const float* s_Y, const int YS, const float4* s_rowc, float* s_lam,
                                            float* s_dz, float* s_sep, const int R, const int Rw_max, const int n,
                                            const bool isg, const int lane, const int npos, const int nvel,
                                            const float h, const float hit, const float beta, const float vmax,
                                            const float z0, float* t_lamb, float* t_seps, const int t_rcap) {
  float z = z0, dz = 0.f;
  if (isg)
    for (int r = 0; r < R; ++r) z += s_Y[lane * YS + r] * s_lam[r];  // warm start
  const float inv_hit = 1.f / hit, inv_h = 1.f / h;
  for (int it = 0; it < npos + nvel; ++it) {
    const bool pos = it < npos;
    // separations d_r + Y_r . dz (lane r): dz changes only at the end of a position iteration,
    // so they are formed once per iteration instead of by a reduction per row (dz = 0 before the
    // first iteration, and the velocity iterations all see the final dz)
    if (it >= 1 && it <= npos) {
      if (isg) s_dz[lane] = dz;
      __syncwarp();
      for (int r = lane; r < R; r += G) {
        float acc = 0.f;
        for (int i = 0; i < n; ++i) acc += s_Y[i * YS + r] * s_dz[i];
        s_sep[r] = s_rowc[r].x + acc;
      }
      __syncwarp();
    }
    if (t_lamb) {  // taped step: every row's impulse before this iteration and its separation
        for (int r = lane; r < R; r += G) {
          t_lamb[it * t_rcap + r] = s_lam[r];
          if (it <= npos) t_seps[it * t_rcap + r] = (it == 0) ? s_rowc[r].x : s_sep[r];
        }
    }
    // one group reduction per row, then a branch-free update (selects: measured 7 % faster on the
    // Ant step than a branch around it)
    for (int r = 0; r < Rw_max; ++r) {
      const float y = (isg && r < R) ? s_Y[lane * YS + r] : 0.f;
      const float4 hc = s_rowc[r];
      const float yz = Grp<G>::sum(y * z);
      const float sep = (it == 0) ? hc.x : s_sep[r];
      const int kb = __float_as_int(hc.z);
      const bool valid = (r < R) && (hc.y > 0.f);
      const bool fric = (kb & 3) == kRowFriction;
      const float lam = s_lam[r];
      const float lim = hc.x * s_lam[(valid && fric) ? (kb >> 2) : 0];
      const float lf = fminf(fmaxf(lam - yz * hc.y, -lim), lim);
      const float tp = (sep >= 0.f) ? -sep * inv_hit : fminf(-beta * sep * inv_hit, vmax);
      const float tv = (sep > 0.f) ? -sep * inv_h : 0.f;
      const float ln = fmaxf(lam + ((pos ? tp : tv) - yz) * hc.y, 0.f);
      const float lnew = fric ? lf : ln;
      const float dl = valid ? lnew - lam : 0.f;
      z += y * dl;
      if (valid) s_lam[r] = lnew;  // every lane stores the same value
    }
    if (pos) dz += hit * z;
  }
  return make_float2(z, dz);
}

// ---------------------------------------------------------------------------------------------
// Delassus form of the same solve, for substeps with at most one row per lane whose W fits in
// s_W (R * R + R words): lane s holds w_s = Y_s . z, d_s = Y_s . dz, the impulse lambda_s and its
// sum over the position iterations. A row reads w_r, d_r and lambda_r from lane r (one shuffle
// each, no reduction) and every lane adds W_sr dl to w_s, with W = Y^T Y = J M^-1 J^T formed once
// per substep; z and dz are rebuilt from the impulses at the end. Returns (z, dz) of the lane and
// leaves the impulses in s_lam; s_dq is used as scratch. Out of line, like the row form, so the
// loop gets its own register allocation.
template <int G>
__device__ __noinline__ float2 pgs_delassus_form(const float* s_Y, const int YS, float* s_W, const float4* s_rowc,
                                                 float* s_lam, float* s_dq, const int R, const int Rw_max,
                                                 const int n, const bool isg, const int lane, const int npos,
                                                 const int nvel, const float h, const float hit, const float beta,
                                                 const float vmax, const float z0, float* t_lamb, float* t_seps,
                                                 const int t_rcap) {
  float* s_acc = s_W + R * R;  // W: row r at r * R; then the impulses summed over the position iterations
  float zw = z0;               // z after the warm start
  if (isg)
    for (int r = 0; r < R; ++r) zw += s_Y[lane * YS + r] * s_lam[r];
  if (isg) s_dq[lane] = zw;
  // W is symmetric: lane s forms W_sm for m = s + d (mod R), d = 0 .. R/2, and stores both
  // triangles (for even R the pair d = R/2 is formed by two lanes, with identical values)
  if (lane < R) {
    for (int d = 0; d <= R / 2; ++d) {
      const int m = (lane + d < R) ? lane + d : lane + d - R;
      float acc = 0.f;
      for (int i = 0; i < n; ++i) acc += s_Y[i * YS + lane] * s_Y[i * YS + m];
      s_W[m * R + lane] = acc;
      s_W[lane * R + m] = acc;
    }
  }
  __syncwarp();
  float wv = 0.f, dv = 0.f, lv = 0.f, av = 0.f;
  if (lane < R) {
    for (int i = 0; i < n; ++i) wv += s_Y[i * YS + lane] * s_dq[i];
    lv = s_lam[lane];
  }
  const float inv_hit = 1.f / hit, inv_h = 1.f / h;
  for (int it = 0; it < npos + nvel; ++it) {
    const bool pos = it < npos;
    if (t_lamb) {  // taped step: lane s, its row's impulse before this iteration and its separation
      if (lane < R) {
        t_lamb[it * t_rcap + lane] = lv;
        if (it <= npos) t_seps[it * t_rcap + lane] = s_rowc[lane].x + dv;
      }
    }
    for (int r = 0; r < Rw_max; ++r) {
      const bool inr = r < R;
      const float4 hc = s_rowc[r];
      const float wc = (inr && lane < R) ? s_W[r * R + lane] : 0.f;  // W_sr of this lane's row
      const int kb = __float_as_int(hc.z);
      const float yz = Grp<G>::get(wv, r), ydz = Grp<G>::get(dv, r);
      // friction rows: the normal impulse of their contact, from its row's lane
      const float lam = Grp<G>::get(lv, r), lam_n = Grp<G>::get(lv, (kb >> 2) & (G - 1));
      const float sep = hc.x + ydz;
      const bool valid = inr && (hc.y > 0.f);
      const bool fric = (kb & 3) == kRowFriction;
      const float lim = hc.x * lam_n;
      const float lf = fminf(fmaxf(lam - yz * hc.y, -lim), lim);
      const float tp = (sep >= 0.f) ? -sep * inv_hit : fminf(-beta * sep * inv_hit, vmax);
      const float tv = (sep > 0.f) ? -sep * inv_h : 0.f;
      const float ln = fmaxf(lam + ((pos ? tp : tv) - yz) * hc.y, 0.f);
      const float lnew = fric ? lf : ln;
      const float dl = valid ? lnew - lam : 0.f;
      wv += wc * dl;
      if (valid && lane == r) lv = lnew;
    }
    if (pos) {
      dv += hit * wv;
      av += lv;
    }
  }
  if (lane < R) { s_lam[lane] = lv; s_acc[lane] = av; }
  __syncwarp();
  // z = z_free + Y lambda; dz = sum over the position iterations of h_it z
  float z = 0.f, dz = 0.f;
  if (isg) {
    float zs = 0.f, as = 0.f;
    for (int r = 0; r < R; ++r) {
      const float y = s_Y[lane * YS + r];
      zs += y * s_lam[r];
      as += y * s_acc[r];
    }
    z = z0 + zs;
    dz = hit * ((float)npos * z0 + as);
  }
  return make_float2(z, dz);
}

// ---------------------------------------------------------------------------------------------
// One substep loop of one environment by one group of G lanes. grp indexes the launch's env list
// (grp >= n_launch_envs: a dead group, which shadows the last env and never stores); sm is the
// group's shared arena and rb the base of its contact and row blocks (sm itself, or a private
// slot of global scratch in the GROWS variant). yg (shared-rows layouts whose Y region is sized
// below the type's row capacity, else null) is the group's global slot for Y in the substeps whose
// rows do not fit that region.
template <int G, bool GROWS, bool BALL = false, bool PER_TYPE = true>
__device__ __forceinline__ void step_group(const StepArgs& A, const TypeArgs& TA, const int grp, float* sm,
                                           float* rb, float* yg) {
  const EnvTypeTable* __restrict__ T = TA.type;
  const int lane = threadIdx.x & (G - 1);
  const bool live = grp < TA.n_launch_envs;
  const int gi = live ? grp : TA.n_launch_envs - 1;
  const int env = TA.env_ids ? TA.env_ids[gi] : TA.env_first + gi;
  const SmemLayout& Ly = TA.lay;
  // sim_step_taped: record the reverse pass's tape. PER_TYPE false (the persistent kernel's tile
  // bodies: taped steps and sim_step_host's direct buffers always use the per-type kernels)
  // compiles without the tape stores and the direct host-buffer loads and stores.
  const bool tape_on = PER_TYPE && TA.tape != nullptr;
  const bool direct_io = PER_TYPE;
  int* smi = reinterpret_cast<int*>(sm);
  int* rbi = reinterpret_cast<int*>(rb);

  const int L = T->n_links, n = T->n_gen, NS = T->n_shapes;
  const int maxdepth = T->max_depth;
  const int MS = Ly.MS, CC = Ly.ccap;
  float* s_link = sm + Ly.link;  // phase 1: per-link hand-off slots of the inward sweep
  float* const s_Yr = rb + Ly.Y;  // phase 2 (aliases phase 1 in shared memory): Y = L^-1 J^T, n x (R | 1)
  float* s_SD = sm + Ly.SD;      // motion subspace column of every generalized DOF
  float* s_M = sm + Ly.M;        // Cholesky factor L (lower), n x MS
  float* s_qdd = sm + Ly.vec;
  float* s_v0 = s_qdd + n;
  float* s_vf = s_v0 + n;
  float* s_dq = s_vf + n;
  float* s_Linv = s_dq + n;
  float* s_con = rb + Ly.con;
  int* s_coni = rbi + Ly.con;
  float4* s_rowc = reinterpret_cast<float4*>(rb + Ly.rowc);
  float* s_lam = rb + Ly.lam;
  int* s_rowa = rbi + Ly.rowa;
  float* s_frc = sm + Ly.frc;
  (void)smi;
  // warm-start impulse cache of this env, read and rewritten in place in global memory (each
  // entry is touched once per substep; only live groups store)
  float* gcache = A.cache + (size_t)env * A.cache_stride;

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
  // ball joint (3 DOF from joint-DOF row jd: rotation vector, angular velocity in the child
  // frame; compiled into the global-rows variant with BALL only, which env types with ball
  // joints use: the other kernels carry none of its code)
  const bool is_ball = BALL && GROWS && isl && jt == kSpherical;
  const bool isg = lane < n;
  // 17-word contact records (body b, normal, offset); shape pairs exist only in the global-rows
  // variant, so the shared-memory variant compiles without the pair phase
  const bool has_pairs = GROWS && T->n_pairs > 0;

  // ---- load state (one HBM read per env-step) ----
  const int dof_base = A.env_dof_base[env];
  float rq[4] = {0.f, 0.f, 0.f, 1.f};
  V3 rp = v3(0.f, 0.f, 0.f), rw = rp, rv = rp;  // root pose / velocity (root lanes)
  float q = 0.f, qd = 0.f, tau = 0.f;
  if (is_root) {
    const float* r = A.root + (size_t)(A.env_actor_base[env] + T->actor[l]) * 13;
    rp = v3(r[0], r[1], r[2]);
    rq[0] = r[3]; rq[1] = r[4]; rq[2] = r[5]; rq[3] = r[6];
    if (free_root) {
      rv = v3(r[7], r[8], r[9]);
      rw = v3(r[10], r[11], r[12]);
    }
  }
  if (has_dof) {
    q = A.dof[(size_t)(dof_base + jd) * 2];
    qd = A.dof[(size_t)(dof_base + jd) * 2 + 1];
    tau = A.act[dof_base + jd];  // joint force of the step; damping is added per substep
    if (direct_io && A.act_copy && live) A.act_copy[dof_base + jd] = tau;
  }
  // ball-joint links keep their state in a shared slot of kBallWords (not in registers, which the
  // rest of the global-rows variant needs): U (3 x 6) | D^-1 (sym 3 x 3) | u (3) | q (3) | qd (3) | tau (3)
  float* s_ball = sm + Ly.ball;
  float* bst = s_ball + kBallWords * l + 27;  // q | qd | tau of this lane's ball joint
  if (is_ball) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      bst[k] = A.dof[(size_t)(dof_base + jd + k) * 2];
      bst[3 + k] = A.dof[(size_t)(dof_base + jd + k) * 2 + 1];
      bst[6 + k] = A.act[dof_base + jd + k];
      if (direct_io && A.act_copy && live) A.act_copy[dof_base + jd + k] = bst[6 + k];
    }
  }
  float q_t = 0.f, v_t = 0.f;  // drive targets
  if (has_dof && T->has_drives) {
    q_t = A.pos_target[dof_base + jd];
    v_t = A.vel_target[dof_base + jd];
  }
  for (int i = lane; i < 3 * L; i += G) s_frc[i] = 0.f;

  unsigned sig = 2166136261u;
  int status = 0;
  const float h = A.h;
  const int npos = A.pos_iters, nvel = A.vel_iters;
  const float hit = h / (float)npos;
  const V3 g = v3(A.gx, A.gy, A.gz);
  int n_con = 0, n_lim = 0, R = 0;

  // (a2) forward kinematics + velocities of the current state, level-synchronous (link mode): link
  // rotation Rw, origin P relative to the actor origin, spatial velocity vs = [w; v] about it, the
  // joint's motion subspace Sa and velocity-product acceleration cc
  auto kinematics = [&](float* Rw, V3& P, float* vs, float* Sa, float* cc) {
    quat_to_mat(rq, Rw);
    if (is_root) {
      vs[0] = rw.x; vs[1] = rw.y; vs[2] = rw.z; vs[3] = rv.x; vs[4] = rv.y; vs[5] = rv.z;
      const V3 pxw = cross(rv, rw);  // d/dt S_root * nu = [0; p_dot x omega]
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
          Sa[0] = aw.x; Sa[1] = aw.y; Sa[2] = aw.z; Sa[3] = pxa.x; Sa[4] = pxa.y; Sa[5] = pxa.z;
        } else if (jt == kPrismatic) {
#pragma unroll
          for (int k = 0; k < 9; ++k) Rw[k] = RB[k];
          P = Pp + mv(Rp, pp + mv(Rpj, jaxis * q));
          Sa[3] = aw.x; Sa[4] = aw.y; Sa[5] = aw.z;
        } else if (BALL && jt == kSpherical) {
          float qj[4], RJ[9];
          rotvec_quat(bst[0], bst[1], bst[2], qj);
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
        for (int k = 0; k < 6; ++k) sq[k] = Sa[k] * qd;
        if (BALL && jt == kSpherical) {
          // motion subspace: the child's axes in world coordinates about O_a, one column per DOF
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const V3 ax = v3(Rw[c], Rw[3 + c], Rw[6 + c]);
            const V3 px = cross(P, ax);
            float* Sc = s_SD + 6 * (gd + c);
            Sc[0] = ax.x; Sc[1] = ax.y; Sc[2] = ax.z; Sc[3] = px.x; Sc[4] = px.y; Sc[5] = px.z;
            const float w = bst[3 + c];
            sq[0] += ax.x * w; sq[1] += ax.y * w; sq[2] += ax.z * w;
            sq[3] += px.x * w; sq[4] += px.y * w; sq[5] += px.z * w;
          }
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) vs[k] = vp[k] + sq[k];
        // c = v x (S qd) (motion cross product)
        const V3 w = v3(vs[0], vs[1], vs[2]), vl = v3(vs[3], vs[4], vs[5]);
        const V3 sa = v3(sq[0], sq[1], sq[2]), sl = v3(sq[3], sq[4], sq[5]);
        const V3 c0 = cross(w, sa), c1 = cross(w, sl) + cross(vl, sa);
        cc[0] = c0.x; cc[1] = c0.y; cc[2] = c0.z; cc[3] = c1.x; cc[4] = c1.y; cc[5] = c1.z;
      }
    }
  };

  for (int sub = 0; sub < A.substeps; ++sub) {
    // taped step (a tape given): this env-substep's block of the tape, written by live groups only
    // (the same code and arithmetic as the plain step: the stores are its only difference)
    float* tp = nullptr;
    const TapeLayout& TL = TA.tl;
    if (tape_on) {
      tp = TA.tape + ((size_t)gi * A.substeps + sub) * TL.words;
      if (live) {
        if (has_dof) { tp[TL.st + 2 * jd] = q; tp[TL.st + 2 * jd + 1] = qd; }
        if (is_ball) {
#pragma unroll
          for (int c = 0; c < 3; ++c) { tp[TL.st + 2 * (jd + c)] = bst[c]; tp[TL.st + 2 * (jd + c) + 1] = bst[3 + c]; }
        }
        if (is_root) {
          float* r = tp + TL.st + 2 * T->n_jdof + 13 * T->actor[l];
          r[0] = rp.x; r[1] = rp.y; r[2] = rp.z; r[3] = rq[0]; r[4] = rq[1]; r[5] = rq[2]; r[6] = rq[3];
          r[7] = rv.x; r[8] = rv.y; r[9] = rv.z; r[10] = rw.x; r[11] = rw.y; r[12] = rw.z;
        }
      }
    }
    // ======== (a2) forward kinematics + velocities, level-synchronous (link mode) ========
    float Rw[9];               // link -> world rotation
    V3 P = v3(0.f, 0.f, 0.f);  // link origin relative to the actor origin O_a
    float vs[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // link spatial velocity [w; v] about O_a
    float Sa[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // joint motion subspace about O_a
    float cc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // velocity-product acceleration
    kinematics(Rw, P, vs, Sa, cc);
    const float Oz = Grp<G>::get(rp.z, ar);  // actor origin height (world)
    // motion subspace per generalized DOF (unit columns for a floating root)
    if (has_dof) {
#pragma unroll
      for (int k = 0; k < 6; ++k) s_SD[6 * gd + k] = Sa[k];
    }
    if (free_root) {
#pragma unroll
      for (int c = 0; c < 6; ++c)
#pragma unroll
        for (int k = 0; k < 6; ++k) s_SD[6 * (gd + c) + k] = (k == c) ? 1.f : 0.f;
    }

    // ======== (a3) rigid-body inertia about O_a and bias force, in registers ========
    // articulated inertia IA (sym 6x6), bias pA, composite inertia Ic = (m, h, I_O)
    float IA[21], pA[6], Ic[10];
    {
      const float m = isl ? T->mass[l] : 0.f;
      const V3 cw = P + mv(Rw, v3(T->com[0][l], T->com[1][l], T->com[2][l]));
      float In[9] = {T->inertia[0][l], T->inertia[3][l], T->inertia[4][l], T->inertia[3][l], T->inertia[1][l],
                     T->inertia[5][l], T->inertia[4][l], T->inertia[5][l], T->inertia[2][l]};
      if (!isl) {
#pragma unroll
        for (int k = 0; k < 9; ++k) In[k] = 0.f;
      }
      float RI[9], RIRt[9], Rt[9];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Rt[3 * i + j] = Rw[3 * j + i];
      mm(Rw, In, RI);
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
      V3 pa = cross(w, Fa) + cross(vl, Fl) - cross(hh, g);
      V3 pl = cross(w, Fl) - g * m;
      if ((A.flags & 8) && isl) {  // external force and torque at the COM (world axes)
        const int bd = T->body[l];
        if (bd >= 0) {
          const float* bf = A.body_force + (size_t)(A.env_body_base[env] + bd) * 6;
          const V3 F = v3(bf[0], bf[1], bf[2]);
          pa = pa - (cross(cw, F) + v3(bf[3], bf[4], bf[5]));
          pl = pl - F;
        }
      }
      // articulated inertia starts as the rigid inertia: [[I_O, h~], [h~^T, m 1]]
      IA[sidx(0, 0)] = Ixx; IA[sidx(0, 1)] = Ixy; IA[sidx(0, 2)] = Ixz;
      IA[sidx(1, 1)] = Iyy; IA[sidx(1, 2)] = Iyz; IA[sidx(2, 2)] = Izz;
      IA[sidx(0, 3)] = 0.f;   IA[sidx(0, 4)] = -hh.z; IA[sidx(0, 5)] = hh.y;
      IA[sidx(1, 3)] = hh.z;  IA[sidx(1, 4)] = 0.f;   IA[sidx(1, 5)] = -hh.x;
      IA[sidx(2, 3)] = -hh.y; IA[sidx(2, 4)] = hh.x;  IA[sidx(2, 5)] = 0.f;
      IA[sidx(3, 3)] = m; IA[sidx(3, 4)] = 0.f; IA[sidx(3, 5)] = 0.f;
      IA[sidx(4, 4)] = m; IA[sidx(4, 5)] = 0.f; IA[sidx(5, 5)] = m;
      pA[0] = pa.x; pA[1] = pa.y; pA[2] = pa.z; pA[3] = pl.x; pA[4] = pl.y; pA[5] = pl.z;
      Ic[0] = m; Ic[1] = hh.x; Ic[2] = hh.y; Ic[3] = hh.z;
      Ic[4] = Ixx; Ic[5] = Iyy; Ic[6] = Izz; Ic[7] = Ixy; Ic[8] = Ixz; Ic[9] = Iyz;
    }

    // ======== (a4) ground contacts (shape mode) and limit rows (link mode) ========
    {
      const int sl_link = (lane < NS) ? T->shape_link[lane] : 0;
      float Rl[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) Rl[k] = Grp<G>::get(Rw[k], sl_link);
      const float plx = Grp<G>::get(P.x, sl_link), ply = Grp<G>::get(P.y, sl_link), plz = Grp<G>::get(P.z, sl_link);
      const float oz = Grp<G>::get(Oz, sl_link);
      unsigned keep = 0u;
      float zc[8];
      V3 xs[8];
      const float coff = A.contact_offset;
      if (lane < NS) {
        const int st = T->shape_type[lane];
        float Rsh[9], Rs[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) Rsh[k] = T->shape_rot[k][lane];
        mm(Rl, Rsh, Rs);
        const V3 cs = v3(plx, ply, plz) + mv(Rl, v3(T->shape_pos[0][lane], T->shape_pos[1][lane], T->shape_pos[2][lane]));
        const float s0 = T->shape_size[0][lane], s1 = T->shape_size[1][lane], s2 = T->shape_size[2][lane];
        int nk;
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
      const int base = Grp<G>::excl_scan(__popc(keep), lane, &n_con);
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
            if (has_pairs) {  // ground-only types use the 9-word record: body b = ground, n = +z
              s_coni[9 * CC + o] = -1;
              s_coni[10 * CC + o] = -1;
              s_con[11 * CC + o] = 0.f;
              s_con[12 * CC + o] = 0.f;
              s_con[13 * CC + o] = 1.f;
              s_con[14 * CC + o] = 0.f;
              s_con[15 * CC + o] = 0.f;
              s_con[16 * CC + o] = 0.f;
            }
            ++o;
          }
        }
      }
      // ---- capsule-box pairs, appended in pair / slot order ----
      if (has_pairs) {
        Mat9 rw9;
#pragma unroll
        for (int k = 0; k < 9; ++k) rw9.m[k] = Rw[k];
        n_con = pair_contacts<G>(T, lane, rw9, P, rp, s_con, s_coni, CC, n_con, coff);
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
        const int slot0 = 3 * T->n_cand + 2 * jd;
        if (lf & 1) {
          s_rowc[o] = make_float4(dlo, 0.f, __int_as_float(kRowLimit), __int_as_float(slot0));
          s_rowa[o] = gd | (jd << 16);
          ++o;
        }
        if (lf & 2) {
          s_rowc[o] = make_float4(dhi, 0.f, __int_as_float(kRowLimit), __int_as_float(slot0 + 1));
          s_rowa[o] = gd | (1 << 8) | (jd << 16);
        }
      }
      // tendon length limits after the joint limits (lane t: tendon t); J = +-c over its joints
      const int n_jlim = n_lim;
      int n_tlim = 0;
      if (T->n_tendons > 0) {
        float tl = 0.f;
        for (int t = 0; t < T->n_tendons; ++t)
          for (int k = 0; k < T->ten_n[t]; ++k) {
            const float qk = Grp<G>::get(q, T->ten_link[t][k]);
            if (lane == t) tl += T->ten_coef[t][k] * qk;
          }
        int tf = 0;
        float tdlo = 0.f, tdhi = 0.f;
        if (lane < T->n_tendons && T->ten_has_limit[lane]) {
          tdlo = tl - T->ten_lo[lane];
          tdhi = T->ten_hi[lane] - tl;
          if (tdlo < A.limit_margin) tf |= 1;
          if (tdhi < A.limit_margin) tf |= 2;
        }
        int o = n_jlim + Grp<G>::excl_scan(__popc(tf), lane, &n_tlim);
        const int slot0 = 3 * T->n_cand + 2 * T->n_jdof + 2 * lane;
        if (tf & 1) {
          s_rowc[o] = make_float4(tdlo, 0.f, __int_as_float(kRowTendon), __int_as_float(slot0));
          s_rowa[o] = lane;
          ++o;
        }
        if (tf & 2) {
          s_rowc[o] = make_float4(tdhi, 0.f, __int_as_float(kRowTendon), __int_as_float(slot0 + 1));
          s_rowa[o] = lane | (1 << 8);
        }
      }
      n_lim = n_jlim + n_tlim;
      R = n_lim + 3 * n_con;
      __syncwarp();
      // contact rows: every contact's normal row, then every contact's two friction rows
      for (int c = lane; c < n_con; c += G) {
        const int cand = s_coni[6 * CC + c];
        const float mu = s_con[4 * CC + c];
        const int rn = n_lim + c;
        s_rowc[rn] = make_float4(s_con[3 * CC + c], 0.f, __int_as_float(kRowNormal), __int_as_float(3 * cand));
        s_rowa[rn] = c;
        for (int t = 0; t < 2; ++t) {
          const int rf = n_lim + n_con + 2 * c + t;
          s_rowc[rf] = make_float4(mu, 0.f, __int_as_float(kRowFriction | (rn << 2)), __int_as_float(3 * cand + 1 + t));
          s_rowa[rf] = c | ((1 + t) << 8);
        }
      }
      __syncwarp();
      if ((A.flags & 1) && lane == 0) {
        fnv1a(sig, n_jlim);
        for (int r = 0; r < n_jlim; ++r) {
          const int a = s_rowa[r];
          fnv1a(sig, a >> 16);
          fnv1a(sig, (a >> 8) & 1);
        }
        if (T->n_tendons > 0) {  // envs with tendons also hash their tendon-limit rows
          fnv1a(sig, n_tlim);
          for (int r = n_jlim; r < n_lim; ++r) {
            const int a = s_rowa[r];
            fnv1a(sig, a & 0xff);
            fnv1a(sig, (a >> 8) & 1);
          }
        }
        fnv1a(sig, n_con);
        for (int c = 0; c < n_con; ++c) {
          fnv1a(sig, s_coni[7 * CC + c]);
          fnv1a(sig, has_pairs ? s_coni[10 * CC + c] : -1);
          fnv1a(sig, s_coni[8 * CC + c]);
        }
      }
    }

    // ======== inward sweep: articulated inertias (ABA pass 2) and composite inertias ========
    float U[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, Dinv = 0.f, uu = 0.f;
    {
      // joint force of the substep: actuation, damping, and the implicit drive kp (q* - q - h qd)
      // + kd (qd* - qd) whose h (h kp + kd) joins the pivot (and the joint-space inertia diagonal)
      float tau_sub = tau - T->damping[l] * qd, drive_d = 0.f;
      if (T->has_drives) {
        const float kp = T->drive_kp[l], kd = T->drive_kd[l];
        tau_sub += kp * (q_t - q - h * qd) + kd * (v_t - qd);
        drive_d = h * (h * kp + kd);
      }
      // fixed tendons: force -k (l - rest) - d l_dot on the length l = sum c q, applied as c F
      for (int t = 0; t < T->n_tendons; ++t) {
        float len = 0.f, rate = 0.f, mine = 0.f;
        for (int k = 0; k < T->ten_n[t]; ++k) {
          const int lk = T->ten_link[t][k];
          const float c = T->ten_coef[t][k];
          len += c * Grp<G>::get(q, lk);
          rate += c * Grp<G>::get(qd, lk);
          if (lk == l && has_dof) mine += c;
        }
        tau_sub += mine * (-T->ten_k[t] * (len - T->ten_rest[t]) - T->ten_d[t] * rate);
      }
      if ((A.flags & 32) && live && has_dof && sub == A.substeps - 1) A.dof_force[dof_base + jd] = tau_sub;
      if ((A.flags & 32) && live && is_ball && sub == A.substeps - 1) {  // ball joint: actuation - damping qd
#pragma unroll
        for (int k = 0; k < 3; ++k) A.dof_force[dof_base + jd + k] = bst[6 + k] - T->damping[l] * bst[3 + k];
      }
      for (int d = maxdepth; d >= 1; --d) {
        if (dep == d) {
          if (has_dof) {
#pragma unroll
            for (int i = 0; i < 6; ++i) {
              float s = 0.f;
#pragma unroll
              for (int j = 0; j < 6; ++j) s += IA[sidx(i, j)] * Sa[j];
              U[i] = s;
            }
            float D = T->armature[l] + drive_d, sp = 0.f;
#pragma unroll
            for (int i = 0; i < 6; ++i) { D += Sa[i] * U[i]; sp += Sa[i] * pA[i]; }
            if (!(D > 0.f)) { status |= 2; D = 1.f; }
            Dinv = 1.f / D;
            uu = tau_sub - sp;
            // Ia = IA - U U^T / D ; pa = pA + Ia c + U u / D
#pragma unroll
            for (int i = 0; i < 6; ++i)
#pragma unroll
              for (int j = i; j < 6; ++j) IA[sidx(i, j)] -= U[i] * U[j] * Dinv;
            float pa[6];
#pragma unroll
            for (int i = 0; i < 6; ++i) {
              float s = pA[i] + U[i] * uu * Dinv;
#pragma unroll
              for (int j = 0; j < 6; ++j) s += IA[sidx(i, j)] * cc[j];
              pa[i] = s;
            }
#pragma unroll
            for (int i = 0; i < 6; ++i) pA[i] = pa[i];
          }
          float* sl = s_link + kLinkWords * l;
          if (is_ball) {
            // the 3-DOF block works on the link's hand-off slot (out of line: its temporaries
            // stay out of the register allocation of the whole step)
#pragma unroll
            for (int k = 0; k < 21; ++k) sl[k] = IA[k];
#pragma unroll
            for (int k = 0; k < 6; ++k) sl[21 + k] = pA[k];
            status |= ball_joint_block(sl, s_ball + kBallWords * l, s_SD + 6 * gd, cc[0], cc[1], cc[2], cc[3], cc[4],
                                       cc[5], T->damping[l], T->armature[l]);
          } else {
#pragma unroll
            for (int k = 0; k < 21; ++k) sl[k] = IA[k];
#pragma unroll
            for (int k = 0; k < 6; ++k) sl[21 + k] = pA[k];
          }
#pragma unroll
          for (int k = 0; k < 10; ++k) sl[27 + k] = Ic[k];
        }
        __syncwarp();
        if (dep == d - 1) {
          for (int ch = T->first_child[l]; ch >= 0; ch = T->next_sibling[ch]) {
            const float* sc = s_link + kLinkWords * ch;
#pragma unroll
            for (int k = 0; k < 21; ++k) IA[k] += sc[k];
#pragma unroll
            for (int k = 0; k < 6; ++k) pA[k] += sc[21 + k];
#pragma unroll
            for (int k = 0; k < 10; ++k) Ic[k] += sc[27 + k];
          }
        }
      }
      // final composite inertias for the joint-space inertia (roots were never handed off)
      if (is_root) {
        float* sl = s_link + kLinkWords * l;
#pragma unroll
        for (int k = 0; k < 10; ++k) sl[27 + k] = Ic[k];
      }
    }

    // ======== root acceleration, outward sweep (ABA pass 3) ========
    float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float qdd = 0.f, qdd3[3] = {0.f, 0.f, 0.f};
    if (free_root) {
      // a0 = -(IA)^-1 pA by a 6x6 Cholesky solve in registers
      float y[6];
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        float s = IA[sidx(j, j)];
#pragma unroll
        for (int k = 0; k < j; ++k) s -= IA[sidx(j, k)] * IA[sidx(j, k)];
        if (!(s > 0.f)) { status |= 2; s = 1.f; }
        const float ljj = sqrtf(s), inv = 1.f / ljj;
        IA[sidx(j, j)] = ljj;
#pragma unroll
        for (int i = j + 1; i < 6; ++i) {
          float t = IA[sidx(i, j)];
#pragma unroll
          for (int k = 0; k < j; ++k) t -= IA[sidx(i, k)] * IA[sidx(j, k)];
          IA[sidx(i, j)] = t * inv;
        }
      }
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        float s = -pA[i];
#pragma unroll
        for (int k = 0; k < i; ++k) s -= IA[sidx(i, k)] * y[k];
        y[i] = s / IA[sidx(i, i)];
      }
#pragma unroll
      for (int i = 5; i >= 0; --i) {
        float s = y[i];
#pragma unroll
        for (int k = i + 1; k < 6; ++k) s -= IA[sidx(k, i)] * acc[k];
        acc[i] = s / IA[sidx(i, i)];
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
        if (is_ball) {  // qdd = D^-1 (u - U^T a), a += S qdd
          const float* bl = s_ball + kBallWords * l;
          float r3[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            float ua = 0.f;
#pragma unroll
            for (int k = 0; k < 6; ++k) ua += bl[6 * c + k] * acc[k];
            r3[c] = bl[24 + c] - ua;
          }
          const float* Di = bl + 18;  // 00 11 22 01 02 12
          qdd3[0] = Di[0] * r3[0] + Di[3] * r3[1] + Di[4] * r3[2];
          qdd3[1] = Di[3] * r3[0] + Di[1] * r3[1] + Di[5] * r3[2];
          qdd3[2] = Di[4] * r3[0] + Di[5] * r3[1] + Di[2] * r3[2];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const float* Sc = s_SD + 6 * (gd + c);
#pragma unroll
            for (int k = 0; k < 6; ++k) acc[k] += Sc[k] * qdd3[c];
          }
        }
      }
    }
    // generalized velocity and its rate (root: nu_dot = a0 - [0; p_dot x omega])
    if (has_dof) { s_qdd[gd] = qdd; s_v0[gd] = qd; }
    if (is_ball) {
#pragma unroll
      for (int c = 0; c < 3; ++c) { s_qdd[gd + c] = qdd3[c]; s_v0[gd + c] = bst[3 + c]; }
    }
    if (free_root) {
#pragma unroll
      for (int k = 0; k < 6; ++k) { s_qdd[gd + k] = acc[k] - cc[k]; s_v0[gd + k] = vs[k]; }
    }
    __syncwarp();
    if (tape_on) {
      if (live && isg) tp[TL.vec + lane] = s_qdd[lane];
    }

    // ======== joint-space inertia (rows in registers) and its Cholesky factor (DOF mode) ========
    {
      float m[G];
      const int gl = isg ? T->dof_link[lane] : 0;
      const unsigned anc = isg ? T->anc[gl] : 0u;
      float F[6];
      {
        const float* ic = s_link + kLinkWords * gl + 27;
        const float mm_ = ic[0];
        const V3 hh = v3(ic[1], ic[2], ic[3]);
        const float* Sg = s_SD + 6 * (isg ? lane : 0);
        const V3 w = v3(Sg[0], Sg[1], Sg[2]), vl = v3(Sg[3], Sg[4], Sg[5]);
        const V3 Iw = v3(ic[4] * w.x + ic[7] * w.y + ic[8] * w.z, ic[7] * w.x + ic[5] * w.y + ic[9] * w.z,
                         ic[8] * w.x + ic[9] * w.y + ic[6] * w.z);
        const V3 Fa = Iw + cross(hh, vl), Fl = vl * mm_ + cross(w, hh);
        F[0] = Fa.x; F[1] = Fa.y; F[2] = Fa.z; F[3] = Fl.x; F[4] = Fl.y; F[5] = Fl.z;
      }
      float arm = 0.f;
      if (isg && T->dof_comp[lane] < 0) {
        arm = T->armature[gl];
        if (T->has_drives) arm += h * (h * T->drive_kp[gl] + T->drive_kd[gl]);
      }
      // row i of M through its shared row (a loop, not unrolled: less code), then into registers
      if (isg) {
        for (int j = 0; j <= lane; ++j) {
          float mij = 0.f;
          if ((anc >> j) & 1u) {
            const float* Sj = s_SD + 6 * j;
#pragma unroll
            for (int k = 0; k < 6; ++k) mij += Sj[k] * F[k];
          }
          if (j == lane) mij += arm;
          s_M[lane * MS + j] = mij;
        }
      }
      __syncwarp();
#pragma unroll
      for (int j = 0; j < G; ++j) m[j] = (isg && j <= lane) ? s_M[lane * MS + j] : 0.f;
      // right-looking Cholesky, lane i owns row i: L_ik = M_ik / L_kk, M_ij -= L_ik L_jk. The
      // column loop is not unrolled: the row shifts down one register per column (m[0] holds
      // M_ik at step k), which keeps the code a few hundred bytes at any G (the unrolled
      // triangle was 60 KB at G = 32 and the instruction fetch stalled); same operations, same order
      float linv = 1.f;
      for (int k = 0; k < n; ++k) {
        float dkk = Grp<G>::get(m[0], k);
        if (!(dkk > 0.f)) { status |= 2; dkk = 1.f; }
        const float lkk = sqrtf(dkk), inv = 1.f / lkk;
        const float lik = (lane > k) ? m[0] * inv : ((lane == k) ? lkk : 0.f);
        if (lane == k) linv = inv;
        if (isg && lane >= k) s_M[lane * MS + k] = lik;
#pragma unroll
        for (int j = 1; j < G; ++j) {
          if (j >= n - k) break;
          const float ljk = Grp<G>::get(lik, k + j);
          m[j - 1] = (k + j <= lane) ? m[j] - lik * ljk : m[j];
        }
      }
      if (isg) s_Linv[lane] = linv;
    }
    __syncwarp();

    // ======== (a5) Jacobian rows and Y = L^-1 J^T, A = |Y_r|^2, warm start (row mode) ========
    // Y is n x YS with the odd stride YS = R | 1 of this substep's rows, so that the rest of the
    // region can hold the Delassus block of the solve below
    const int YS = R | 1;
    // A shared-rows layout at G = 32 may size the Y region for the rows a substep usually has (the
    // Delassus form's 32 rows and more; the Humanoid's substeps rarely pass 40 of its 114) rather
    // than the type's row capacity; a substep with more rows puts Y in the group's global slot.
    float* const s_Y = (!GROWS && G == 32 && n * YS > Ly.ywords) ? yg : s_Yr;
    for (int r = lane; r < R; r += G) {
      const float4 hc = s_rowc[r];
      const int a = s_rowa[r];
      const int kind = __float_as_int(hc.z) & 3;
      // contact rows: J_i = S_i . [x_a x k; k] on body a's path, - S_i . [x_b x k; k] on body b's
      // (x_a, x_b: the contact point relative to each actor's origin; the paths never overlap)
      float fr[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, fb[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      unsigned anc = 0u, ancb = 0u;
      int gl = -1;
      float sgn = 0.f;
      int tt = -1;
      if (kind == kRowLimit) {
        gl = a & 0xff;
        sgn = ((a >> 8) & 1) ? -1.f : 1.f;
      } else if (kind == kRowTendon) {
        tt = a & 0xff;
        sgn = ((a >> 8) & 1) ? -1.f : 1.f;
      } else {
        const int c = a & 0xff, dir = (a >> 8) & 3;
        anc = T->anc[s_coni[5 * CC + c]];
        const int lb = has_pairs ? s_coni[9 * CC + c] : -1;
        const V3 x = v3(s_con[0 * CC + c], s_con[1 * CC + c], s_con[2 * CC + c]);
        const V3 nrm = has_pairs ? v3(s_con[11 * CC + c], s_con[12 * CC + c], s_con[13 * CC + c]) : v3(0.f, 0.f, 1.f);
        V3 k = nrm;
        if (dir != 0) {
          V3 t1, t2;
          tangent_basis(nrm, t1, t2);
          k = (dir == 1) ? t1 : t2;
        }
        const V3 xk = cross(x, k);
        fr[0] = xk.x; fr[1] = xk.y; fr[2] = xk.z; fr[3] = k.x; fr[4] = k.y; fr[5] = k.z;
        if (lb >= 0) {
          ancb = T->anc[lb];
          const V3 xb = x - v3(s_con[14 * CC + c], s_con[15 * CC + c], s_con[16 * CC + c]);
          const V3 xbk = cross(xb, k);
          fb[0] = -xbk.x; fb[1] = -xbk.y; fb[2] = -xbk.z; fb[3] = -k.x; fb[4] = -k.y; fb[5] = -k.z;
        }
      }
      float y[G];
      float asum = 0.f;
      if (kind == kRowTendon) {
        // (rare) tendon rows: J from the tendon's coefficients, forward substitution through the
        // row's column of Y in shared memory (kept out of the unrolled loop below)
        for (int i = 0; i < n; ++i) {
          float ji = 0.f;
          for (int k = 0; k < T->ten_n[tt]; ++k)
            if (T->gdof[T->ten_link[tt][k]] == i) ji += sgn * T->ten_coef[tt][k];
          for (int k = 0; k < i; ++k) ji -= s_M[i * MS + k] * s_Y[k * YS + r];
          const float yi = ji * s_Linv[i];
          s_Y[i * YS + r] = yi;
          asum += yi * yi;
        }
      } else {
        // J_r in registers, then a right-looking forward substitution: y_k = b_k / L_kk and
        // b_i -= L_ik y_k for i > k (the subtractions of the row-by-row form, in the same order).
        // The vector shifts down one register per step (y[0] holds b_k), so the loop over k is
        // not unrolled (the unrolled triangle was 25 KB of code at G = 32)
        // J_r through the row's column of Y (a loop, not unrolled: less code), then into registers
        for (int i = 0; i < n; ++i) {
          float ji = 0.f;
          if (kind == kRowLimit) {
            ji = (i == gl) ? sgn : 0.f;
          } else if ((anc >> i) & 1u) {
            const float* Si = s_SD + 6 * i;
#pragma unroll
            for (int k = 0; k < 6; ++k) ji += Si[k] * fr[k];
          } else if ((ancb >> i) & 1u) {
            const float* Si = s_SD + 6 * i;
#pragma unroll
            for (int k = 0; k < 6; ++k) ji += Si[k] * fb[k];
          }
          s_Y[i * YS + r] = ji;
        }
#pragma unroll
        for (int i = 0; i < G; ++i) y[i] = (i < n) ? s_Y[i * YS + r] : 0.f;
        for (int k = 0; k < n; ++k) {
          const float yk = y[0] * s_Linv[k];
          s_Y[k * YS + r] = yk;
          asum += yk * yk;
#pragma unroll
          for (int j = 1; j < G; ++j) {
            if (j >= n - k) break;
            y[j - 1] = y[j] - s_M[(k + j) * MS + k] * yk;
          }
        }
      }
      const bool act = asum > 1e-12f;
      const float invA = act ? 1.f / asum : 0.f;
      s_rowc[r].y = invA;
      s_lam[r] = act ? gcache[__float_as_int(hc.w)] : 0.f;
    }
    __syncwarp();
    if (tape_on) {  // contact and row lists, L, Y and the warm-start impulses
      if (live) {
        if (lane == 0) {
          int* th = reinterpret_cast<int*>(tp + TL.hdr);
          th[0] = n_con; th[1] = n_lim; th[2] = R; th[3] = 0;
        }
        for (int c = lane; c < n_con; c += G) {
          tp[TL.con + c] = s_con[c];
          tp[TL.con + TL.ccap + c] = s_con[CC + c];
          tp[TL.con + 2 * TL.ccap + c] = s_con[2 * CC + c];
          tp[TL.con + 3 * TL.ccap + c] = __int_as_float(s_coni[5 * CC + c]);
          tp[TL.con + 4 * TL.ccap + c] = __int_as_float(s_coni[7 * CC + c]);
          if (has_pairs) {  // body b (-1: the ground), candidate, normal, b's actor offset
            tp[TL.con + 5 * TL.ccap + c] = __int_as_float(s_coni[9 * CC + c]);
            tp[TL.con + 6 * TL.ccap + c] = __int_as_float(s_coni[6 * CC + c]);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
              tp[TL.con + (7 + k) * TL.ccap + c] = s_con[(11 + k) * CC + c];
              tp[TL.con + (10 + k) * TL.ccap + c] = s_con[(14 + k) * CC + c];
            }
          }
        }
        for (int r = lane; r < R; r += G) {
          reinterpret_cast<float4*>(tp + TL.rowc)[r] = s_rowc[r];
          tp[TL.rowa + r] = __int_as_float(s_rowa[r]);
          tp[TL.lam0 + r] = s_lam[r];
          for (int i = 0; i < n; ++i) tp[TL.Y + i * TL.YT + r] = s_Y[i * YS + r];
        }
        if (isg) {
          for (int k = 0; k <= lane; ++k) tp[TL.L + lane * TL.LT + k] = s_M[lane * MS + k];
          tp[TL.Linv + lane] = s_Linv[lane];
        }
      }
    }

    // ======== (a6) TGS-style projected Gauss-Seidel in z = L^T v ========
    // With v = L^-T z, row r's velocity is J_r v = Y_r . z and its separation d_r + J_r dq =
    // d_r + Y_r . dz; an impulse change dl on row r moves z by Y_r dl.
    float z0 = 0.f;  // z of the free velocity (DOF lanes)
    if (isg) s_vf[lane] = s_v0[lane] + h * s_qdd[lane];  // v_free
    __syncwarp();
    if (isg)
      for (int k = lane; k < n; ++k) z0 += s_M[k * MS + lane] * s_vf[k];  // z = L^T v_free
    if (tape_on) {
      if (live && isg) { tp[TL.vec + n + lane] = s_vf[lane]; tp[TL.vec + 2 * n + lane] = z0; }
    }
    float* t_lamb = nullptr;
    float* t_seps = nullptr;
    if (tape_on && live) { t_lamb = tp + TL.lamb; t_seps = tp + TL.seps; }
    const int Rw_max = __reduce_max_sync(kFull, R);
    float z = 0.f, dz = 0.f;
    // The Delassus form serves one env per warp (G = 32: five-level reductions, nothing to share
    // the warp's issue slots with); at G <= 16 forming W costs more than it saves (measured on the
    // Ant: 3 % slower, 8 % with two rows per lane so that every Ant substep fits). W and the
    // impulse sums go after Y in its region, or, with the rows in global
    // scratch, into the shared link slots (free from the inertia pass to the next substep's
    // inward sweep); flag 64 keeps every substep in the row form.
    float* s_W = GROWS ? s_link : s_Y + n * YS;
    const int wcap = GROWS ? L * kLinkWords : Ly.ywords - n * YS;
    const bool delassus = G == 32 && !(A.flags & 64) && __all_sync(kFull, R <= G && R * R + R <= wcap);
    if (delassus) {
      const float2 zd = pgs_delassus_form<G>(s_Y, YS, s_W, s_rowc, s_lam, s_dq, R, Rw_max, n, isg, lane, npos,
                                                   nvel, h, hit, A.bias_coef, A.max_depen_vel, z0,
                                                   t_lamb, t_seps, TL.rcap);
      z = zd.x;
      dz = zd.y;
    } else {
      // s_dq and the row aux words (dead after the Jacobian rows) are the form's scratch
      const float2 zd = pgs_row_form<G>(s_Y, YS, s_rowc, s_lam, s_dq, reinterpret_cast<float*>(s_rowa), R,
                                              Rw_max, n, isg, lane, npos, nvel, h, hit, A.bias_coef,
                                              A.max_depen_vel, z0, t_lamb, t_seps, TL.rcap);
      z = zd.x;
      dz = zd.y;
    }
    // back to joint space: v = L^-T z, dq = L^-T dz (lane k finalises DOF k, highest first)
    {
      float bz = z, bd = dz, xz = 0.f, xd = 0.f;
      for (int k = n - 1; k >= 0; --k) {
        const float li = s_Linv[k];
        const float xzk = Grp<G>::get(bz * li, k), xdk = Grp<G>::get(bd * li, k);
        if (lane == k) { xz = xzk; xd = xdk; }
        if (lane < k) {
          const float lki = s_M[k * MS + lane];
          bz -= lki * xzk;
          bd -= lki * xdk;
        }
      }
      if (isg) { s_vf[lane] = xz; s_dq[lane] = xd; }
    }
    __syncwarp();
    if (tape_on) {  // the solve's result in both coordinates, and the final impulses
      if (live) {
        if (isg) {
          tp[TL.vec + 3 * n + lane] = z;
          tp[TL.vec + 4 * n + lane] = dz;
          tp[TL.vec + 5 * n + lane] = s_vf[lane];
          tp[TL.vec + 6 * n + lane] = s_dq[lane];
        }
        for (int r = lane; r < R; r += G) tp[TL.lamf + r] = s_lam[r];
      }
    }

    // ======== impulse cache, contact impulses per link ========
    if (live)
      for (int i = lane; i < T->cache_len; i += G) gcache[i] = 0.f;
    __syncwarp();
    if (live)
      for (int r = lane; r < R; r += G) gcache[__float_as_int(s_rowc[r].w)] = s_lam[r];
    if (isl) {
      // impulse lambda_n n + lambda_1 t1 + lambda_2 t2 on body a, the opposite on body b
      V3 fsum = v3(0.f, 0.f, 0.f);
      for (int c = 0; c < n_con; ++c) {
        const int la = s_coni[5 * CC + c], lb = has_pairs ? s_coni[9 * CC + c] : -1;
        if (la != l && lb != l) continue;
        const V3 nrm = has_pairs ? v3(s_con[11 * CC + c], s_con[12 * CC + c], s_con[13 * CC + c]) : v3(0.f, 0.f, 1.f);
        V3 t1, t2;
        tangent_basis(nrm, t1, t2);
        const V3 imp = nrm * s_lam[n_lim + c] + t1 * s_lam[n_lim + n_con + 2 * c] + t2 * s_lam[n_lim + n_con + 2 * c + 1];
        fsum = (la == l) ? fsum + imp : fsum - imp;
      }
      s_frc[3 * l] += fsum.x; s_frc[3 * l + 1] += fsum.y; s_frc[3 * l + 2] += fsum.z;
    }
    __syncwarp();

    // ======== (a7) integrate (link mode) ========
    if (has_dof) { q += s_dq[gd]; qd = s_vf[gd]; }
    if (is_ball) {  // R_J <- R_J exp([dq]x), dq in child coordinates; stored as the shorter rotation
      float e1[4], e2[4], qn[4];
      rotvec_quat(bst[0], bst[1], bst[2], e1);
      rotvec_quat(s_dq[gd], s_dq[gd + 1], s_dq[gd + 2], e2);
      qn[0] = e1[3] * e2[0] + e1[0] * e2[3] + e1[1] * e2[2] - e1[2] * e2[1];
      qn[1] = e1[3] * e2[1] - e1[0] * e2[2] + e1[1] * e2[3] + e1[2] * e2[0];
      qn[2] = e1[3] * e2[2] + e1[0] * e2[1] - e1[1] * e2[0] + e1[2] * e2[3];
      qn[3] = e1[3] * e2[3] - e1[0] * e2[0] - e1[1] * e2[1] - e1[2] * e2[2];
      quat_rotvec(qn, bst);
#pragma unroll
      for (int c = 0; c < 3; ++c) bst[3 + c] = s_vf[gd + c];
    }
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
      const float yq = e[3] * rq[1] - e[0] * rq[2] + e[1] * rq[3] + e[2] * rq[0];
      const float zq = e[3] * rq[2] + e[0] * rq[1] - e[1] * rq[0] + e[2] * rq[3];
      const float w = e[3] * rq[3] - e[0] * rq[0] - e[1] * rq[1] - e[2] * rq[2];
      const float nr = sqrtf(x * x + yq * yq + zq * zq + w * w);
      rq[0] = x / nr; rq[1] = yq / nr; rq[2] = zq / nr; rq[3] = w / nr;
    }
    __syncwarp();
  }  // substeps

  // ======== body states after the step (flag 16): one more kinematics pass ========
  if (A.flags & 16) {
    float Rw[9];
    V3 P = v3(0.f, 0.f, 0.f);
    float vs[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, Sa[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float cc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    kinematics(Rw, P, vs, Sa, cc);
    const V3 O = v3(Grp<G>::get(rp.x, ar), Grp<G>::get(rp.y, ar), Grp<G>::get(rp.z, ar));
    const int bd = isl ? T->body[l] : -1;
    if (live && bd >= 0) {
      float* bs = A.body_state + (size_t)(A.env_body_base[env] + bd) * 13;
      float qb[4];
      mat_to_quat(Rw, qb);
      const V3 w = v3(vs[0], vs[1], vs[2]);
      const V3 vp = v3(vs[3], vs[4], vs[5]) + cross(w, P);  // velocity of the link origin
      bs[0] = O.x + P.x; bs[1] = O.y + P.y; bs[2] = O.z + P.z;
      bs[3] = qb[0]; bs[4] = qb[1]; bs[5] = qb[2]; bs[6] = qb[3];
      bs[7] = vp.x; bs[8] = vp.y; bs[9] = vp.z;
      bs[10] = w.x; bs[11] = w.y; bs[12] = w.z;
    }
  }

  // ======== outputs (one HBM write per env-step) ========
  if (is_root) {
    if (!(isfinite(rp.x) && isfinite(rp.y) && isfinite(rp.z) && isfinite(rq[0]) && isfinite(rq[1]) &&
          isfinite(rq[2]) && isfinite(rq[3]) && isfinite(rv.x) && isfinite(rv.y) && isfinite(rv.z) &&
          isfinite(rw.x) && isfinite(rw.y) && isfinite(rw.z)))
      status |= 1;
  }
  if (has_dof && !(isfinite(q) && isfinite(qd))) status |= 1;
  if (is_ball && !(isfinite(bst[0]) && isfinite(bst[1]) && isfinite(bst[2]) && isfinite(bst[3]) && isfinite(bst[4]) &&
                   isfinite(bst[5])))
    status |= 1;
  status = Grp<G>::any(status);
  if (live) {
    if (is_root) {
      float* r = A.root + (size_t)(A.env_actor_base[env] + T->actor[l]) * 13;
      r[0] = rp.x; r[1] = rp.y; r[2] = rp.z;
      r[3] = rq[0]; r[4] = rq[1]; r[5] = rq[2]; r[6] = rq[3];
      r[7] = rv.x; r[8] = rv.y; r[9] = rv.z;
      r[10] = rw.x; r[11] = rw.y; r[12] = rw.z;
      if (direct_io && A.root_out) {  // sim_step_host with a pinned output buffer: the row goes there too
        float* o = A.root_out + (size_t)(A.env_actor_base[env] + T->actor[l]) * 13;
        o[0] = rp.x; o[1] = rp.y; o[2] = rp.z;
        o[3] = rq[0]; o[4] = rq[1]; o[5] = rq[2]; o[6] = rq[3];
        o[7] = rv.x; o[8] = rv.y; o[9] = rv.z;
        o[10] = rw.x; o[11] = rw.y; o[12] = rw.z;
      }
    }
    if (has_dof) {
      A.dof[(size_t)(dof_base + jd) * 2] = q;
      A.dof[(size_t)(dof_base + jd) * 2 + 1] = qd;
      if (direct_io && A.dof_out) {
        A.dof_out[(size_t)(dof_base + jd) * 2] = q;
        A.dof_out[(size_t)(dof_base + jd) * 2 + 1] = qd;
      }
    }
    if (is_ball) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        A.dof[(size_t)(dof_base + jd + c) * 2] = bst[c];
        A.dof[(size_t)(dof_base + jd + c) * 2 + 1] = bst[3 + c];
        if (direct_io && A.dof_out) {
          A.dof_out[(size_t)(dof_base + jd + c) * 2] = bst[c];
          A.dof_out[(size_t)(dof_base + jd + c) * 2 + 1] = bst[3 + c];
        }
      }
    }
    const int bd = isl ? T->body[l] : -1;
    if (bd >= 0) {
      const float inv_dt = 1.f / A.dt;
      float* nf = A.net_force + (size_t)(A.env_body_base[env] + bd) * 3;
      nf[0] = s_frc[3 * l] * inv_dt; nf[1] = s_frc[3 * l + 1] * inv_dt; nf[2] = s_frc[3 * l + 2] * inv_dt;
    }
    int* pr = A.pairs + (size_t)env * A.pair_stride * 3;
    for (int c = lane; c < A.pair_stride; c += G) {
      const bool vc = c < n_con;
      pr[3 * c + 0] = vc ? s_coni[7 * CC + c] : -1;
      pr[3 * c + 1] = (vc && has_pairs) ? s_coni[10 * CC + c] : -1;
      pr[3 * c + 2] = vc ? s_coni[8 * CC + c] : -1;
    }
    if (lane == 0) {
      A.n_pairs[env] = n_con;
      A.status[env] = status;
      if (A.flags & 1) A.sig[env] = sig;
    }
  }
}

// One launch per env type: blocks of 128 / G groups, one env per group. In the GROWS variant the
// group's scratch slot is its index in the launch (the dead groups of the last block own the
// slots past the launched envs); so is a shared-rows layout's Y overflow slot.
template <int G, bool GROWS, bool BALL = false>
__global__ void __launch_bounds__(128, 4) step_kernel(const __grid_constant__ StepArgs A,
                                                     const __grid_constant__ TypeArgs TA) {
  extern __shared__ __align__(16) float smem[];
  const int grp_blk = threadIdx.x / G;
  const int grp = blockIdx.x * (blockDim.x / G) + grp_blk;
  float* sm = smem + grp_blk * TA.lay.total;
  float* rb = GROWS ? TA.scratch + (size_t)grp * TA.lay.scratch_words : sm;
  float* yg = (!GROWS && TA.lay.scratch_words) ? TA.scratch + (size_t)grp * TA.lay.scratch_words : nullptr;
  // The type's model table (9.5 KB) is read by every phase, each phase first touching lines of its
  // own; after a cold L2 each first touch is a DRAM round trip on some env's dependent chain. One
  // warp of the first CTA requests all of its lines into L2 at the start (measured with L2 flushed
  // between steps: cartpole 64 envs 7 % faster, Ant 4096 1 %; every warp prefetching instead made
  // the Ant step 5 % slower).
  if (blockIdx.x == 0 && threadIdx.x < 32) {
    const char* tb = reinterpret_cast<const char*>(TA.type);
    for (int o = threadIdx.x * 128; o < (int)sizeof(EnvTypeTable); o += 32 * 128)
      asm volatile("prefetch.global.L2 [%0];" ::"l"(__cvta_generic_to_global(tb + o)));
  }
  step_group<G, GROWS, BALL>(A, TA, grp, sm, rb, yg);
}

}  // namespace artsim
