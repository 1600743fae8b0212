// Test infrastructure only: part of the FP64 CPU oracle for the batched articulated-body step.
// Nothing in the product path may include, link or call this file.
//
// Small fixed-size linear algebra and spatial (6-D) algebra, written out directly from
// R. Featherstone, "Rigid Body Dynamics Algorithms" (2008), ch. 2:
//   * a spatial motion / force vector is [angular(3); linear(3)];
//   * crm(v) is the motion cross-product matrix v x, crf(v) = -crm(v)^T is v x*;
//   * plux(E, r) is the Plücker transform B_X_A for a frame B at position r (A coords) with
//     rotation E (B coords = E * A coords): [[E, 0], [-E r~, E]];
//   * mcI(m, c, Ic) is the spatial inertia about the frame origin of a body of mass m with centre of
//     mass c and rotational inertia Ic about the centre of mass.
// Every routine is templated on the scalar so the oracle can run in double, in an operation
// counting type, or in a forward-mode dual type.
#pragma once
#include <cmath>
#include <cstdint>
#include <vector>

namespace orc {

// ----------------------------------------------------------------------------------------------
// Scalar helpers. The templates below call sqrt/sin/cos/fabs unqualified so that a custom scalar
// type can provide them by argument-dependent lookup.
using std::sqrt;
using std::sin;
using std::cos;
using std::fabs;
using std::atan2;

inline double val(double x) { return x; }
inline double val(float x) { return (double)x; }
template <class T> inline T tmax(const T& a, const T& b) { return (a < b) ? b : a; }
template <class T> inline T tmin(const T& a, const T& b) { return (b < a) ? b : a; }

// ----------------------------------------------------------------------------------------------
// 3-vectors and row-major 3x3 matrices.
template <class T> struct Vec3 {
  T e[3];
  T& operator[](int i) { return e[i]; }
  const T& operator[](int i) const { return e[i]; }
};
template <class T> struct Mat3 {
  T e[9];
  T& operator()(int i, int j) { return e[3 * i + j]; }
  const T& operator()(int i, int j) const { return e[3 * i + j]; }
};

template <class T> Vec3<T> mk3(const T& a, const T& b, const T& c) { return Vec3<T>{{a, b, c}}; }
template <class T> Vec3<T> zero3() { return mk3<T>(T(0.0), T(0.0), T(0.0)); }
template <class T> Vec3<T> add(const Vec3<T>& a, const Vec3<T>& b) { return mk3<T>(a[0] + b[0], a[1] + b[1], a[2] + b[2]); }
template <class T> Vec3<T> sub(const Vec3<T>& a, const Vec3<T>& b) { return mk3<T>(a[0] - b[0], a[1] - b[1], a[2] - b[2]); }
template <class T> Vec3<T> scale(const Vec3<T>& a, const T& s) { return mk3<T>(a[0] * s, a[1] * s, a[2] * s); }
template <class T> T dot(const Vec3<T>& a, const Vec3<T>& b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
template <class T> Vec3<T> cross(const Vec3<T>& a, const Vec3<T>& b) {
  return mk3<T>(a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]);
}

template <class T> Mat3<T> ident3() {
  Mat3<T> m;
  for (int i = 0; i < 9; ++i) m.e[i] = T(0.0);
  m(0, 0) = m(1, 1) = m(2, 2) = T(1.0);
  return m;
}
template <class T> Mat3<T> mul(const Mat3<T>& a, const Mat3<T>& b) {
  Mat3<T> m;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) m(i, j) = a(i, 0) * b(0, j) + a(i, 1) * b(1, j) + a(i, 2) * b(2, j);
  return m;
}
template <class T> Vec3<T> mul(const Mat3<T>& a, const Vec3<T>& x) {
  return mk3<T>(a(0, 0) * x[0] + a(0, 1) * x[1] + a(0, 2) * x[2], a(1, 0) * x[0] + a(1, 1) * x[1] + a(1, 2) * x[2],
                a(2, 0) * x[0] + a(2, 1) * x[1] + a(2, 2) * x[2]);
}
template <class T> Mat3<T> transpose(const Mat3<T>& a) {
  Mat3<T> m;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) m(i, j) = a(j, i);
  return m;
}
template <class T> Mat3<T> madd(const Mat3<T>& a, const Mat3<T>& b) {
  Mat3<T> m;
  for (int i = 0; i < 9; ++i) m.e[i] = a.e[i] + b.e[i];
  return m;
}
template <class T> Mat3<T> mscale(const Mat3<T>& a, const T& s) {
  Mat3<T> m;
  for (int i = 0; i < 9; ++i) m.e[i] = a.e[i] * s;
  return m;
}
// skew(v) * x = v x x
template <class T> Mat3<T> skew(const Vec3<T>& v) {
  Mat3<T> m;
  m(0, 0) = T(0.0); m(0, 1) = -v[2]; m(0, 2) = v[1];
  m(1, 0) = v[2];  m(1, 1) = T(0.0); m(1, 2) = -v[0];
  m(2, 0) = -v[1]; m(2, 1) = v[0];  m(2, 2) = T(0.0);
  return m;
}

// Rotation matrix (body -> world) of the unit quaternion q = (x, y, z, w).
template <class T> Mat3<T> quat_to_mat(const T q[4]) {
  const T x = q[0], y = q[1], z = q[2], w = q[3];
  Mat3<T> m;
  m(0, 0) = T(1.0) - T(2.0) * (y * y + z * z); m(0, 1) = T(2.0) * (x * y - z * w); m(0, 2) = T(2.0) * (x * z + y * w);
  m(1, 0) = T(2.0) * (x * y + z * w); m(1, 1) = T(1.0) - T(2.0) * (x * x + z * z); m(1, 2) = T(2.0) * (y * z - x * w);
  m(2, 0) = T(2.0) * (x * z - y * w); m(2, 1) = T(2.0) * (y * z + x * w); m(2, 2) = T(1.0) - T(2.0) * (x * x + y * y);
  return m;
}
// Hamilton product a*b of quaternions stored (x, y, z, w).
template <class T> void quat_mul(const T a[4], const T b[4], T out[4]) {
  const T x = a[3] * b[0] + a[0] * b[3] + a[1] * b[2] - a[2] * b[1];
  const T y = a[3] * b[1] - a[0] * b[2] + a[1] * b[3] + a[2] * b[0];
  const T z = a[3] * b[2] + a[0] * b[1] - a[1] * b[0] + a[2] * b[3];
  const T w = a[3] * b[3] - a[0] * b[0] - a[1] * b[1] - a[2] * b[2];
  out[0] = x; out[1] = y; out[2] = z; out[3] = w;
}
// Exact quaternion exponential of a rotation vector th (rotation by |th| about th/|th|).
template <class T> void quat_exp(const Vec3<T>& th, T out[4]) {
  const T ang2 = dot(th, th);
  if (ang2 < T(1e-30)) {  // limit of sin(a/2)/a is 1/2
    out[0] = th[0] * T(0.5); out[1] = th[1] * T(0.5); out[2] = th[2] * T(0.5); out[3] = T(1.0);
    return;
  }
  const T ang = sqrt(ang2);
  const T s = sin(ang * T(0.5)) / ang;
  out[0] = th[0] * s; out[1] = th[1] * s; out[2] = th[2] * s; out[3] = cos(ang * T(0.5));
}
// Rotation vector of the quaternion q = (x, y, z, w) (need not be exactly unit): the shorter
// rotation (w >= 0), angle 2 atan2(|v|, w) about v / |v|; r = 2 v / w in the limit |v| -> 0.
template <class T> Vec3<T> quat_log(const T qin[4]) {
  T q[4] = {qin[0], qin[1], qin[2], qin[3]};
  if (q[3] < T(0.0))
    for (int k = 0; k < 4; ++k) q[k] = T(0.0) - q[k];
  const T s2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
  T f;
  if (s2 < T(1e-30)) {
    f = T(2.0) / q[3];
  } else {
    const T sn = sqrt(s2);
    f = T(2.0) * atan2(sn, q[3]) / sn;
  }
  Vec3<T> r = zero3<T>();
  r[0] = q[0] * f; r[1] = q[1] * f; r[2] = q[2] * f;
  return r;
}
// Rotation by angle th about the unit axis a (Rodrigues' formula): maps rotated-frame coords to
// original-frame coords.
template <class T> Mat3<T> axis_angle(const Vec3<T>& a, const T& th) {
  const T c = cos(th), s = sin(th), t = T(1.0) - c;
  Mat3<T> m;
  m(0, 0) = t * a[0] * a[0] + c;        m(0, 1) = t * a[0] * a[1] - s * a[2]; m(0, 2) = t * a[0] * a[2] + s * a[1];
  m(1, 0) = t * a[0] * a[1] + s * a[2]; m(1, 1) = t * a[1] * a[1] + c;        m(1, 2) = t * a[1] * a[2] - s * a[0];
  m(2, 0) = t * a[0] * a[2] - s * a[1]; m(2, 1) = t * a[1] * a[2] + s * a[0]; m(2, 2) = t * a[2] * a[2] + c;
  return m;
}

// ----------------------------------------------------------------------------------------------
// Spatial vectors [angular; linear] and row-major 6x6 matrices.
template <class T> struct SVec {
  T e[6];
  T& operator[](int i) { return e[i]; }
  const T& operator[](int i) const { return e[i]; }
};
template <class T> struct SMat {
  T e[36];
  T& operator()(int i, int j) { return e[6 * i + j]; }
  const T& operator()(int i, int j) const { return e[6 * i + j]; }
};

template <class T> SVec<T> szero() {
  SVec<T> v;
  for (int i = 0; i < 6; ++i) v[i] = T(0.0);
  return v;
}
template <class T> SVec<T> smk(const Vec3<T>& ang, const Vec3<T>& lin) {
  SVec<T> v;
  for (int i = 0; i < 3; ++i) { v[i] = ang[i]; v[3 + i] = lin[i]; }
  return v;
}
template <class T> Vec3<T> sang(const SVec<T>& v) { return mk3<T>(v[0], v[1], v[2]); }
template <class T> Vec3<T> slin(const SVec<T>& v) { return mk3<T>(v[3], v[4], v[5]); }
template <class T> SVec<T> sadd(const SVec<T>& a, const SVec<T>& b) {
  SVec<T> v;
  for (int i = 0; i < 6; ++i) v[i] = a[i] + b[i];
  return v;
}
template <class T> SVec<T> ssub(const SVec<T>& a, const SVec<T>& b) {
  SVec<T> v;
  for (int i = 0; i < 6; ++i) v[i] = a[i] - b[i];
  return v;
}
template <class T> SVec<T> sscale(const SVec<T>& a, const T& s) {
  SVec<T> v;
  for (int i = 0; i < 6; ++i) v[i] = a[i] * s;
  return v;
}
template <class T> T sdot(const SVec<T>& a, const SVec<T>& b) {
  T s = T(0.0);
  for (int i = 0; i < 6; ++i) s = s + a[i] * b[i];
  return s;
}
template <class T> SMat<T> szeroM() {
  SMat<T> m;
  for (int i = 0; i < 36; ++i) m.e[i] = T(0.0);
  return m;
}
template <class T> SMat<T> smul(const SMat<T>& a, const SMat<T>& b) {
  SMat<T> m;
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      T s = T(0.0);
      for (int k = 0; k < 6; ++k) s = s + a(i, k) * b(k, j);
      m(i, j) = s;
    }
  return m;
}
template <class T> SVec<T> smul(const SMat<T>& a, const SVec<T>& x) {
  SVec<T> v;
  for (int i = 0; i < 6; ++i) {
    T s = T(0.0);
    for (int k = 0; k < 6; ++k) s = s + a(i, k) * x[k];
    v[i] = s;
  }
  return v;
}
template <class T> SMat<T> stranspose(const SMat<T>& a) {
  SMat<T> m;
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) m(i, j) = a(j, i);
  return m;
}
template <class T> SMat<T> saddM(const SMat<T>& a, const SMat<T>& b) {
  SMat<T> m;
  for (int i = 0; i < 36; ++i) m.e[i] = a.e[i] + b.e[i];
  return m;
}
template <class T> SMat<T> ssubM(const SMat<T>& a, const SMat<T>& b) {
  SMat<T> m;
  for (int i = 0; i < 36; ++i) m.e[i] = a.e[i] - b.e[i];
  return m;
}
// Fill one 3x3 block (bi, bj in {0, 1}) of a 6x6 matrix.
template <class T> void set_block(SMat<T>& m, int bi, int bj, const Mat3<T>& b) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) m(3 * bi + i, 3 * bj + j) = b(i, j);
}
// Motion cross-product matrix: crm(v) * m = v x m.
template <class T> SMat<T> crm(const SVec<T>& v) {
  SMat<T> m = szeroM<T>();
  const Mat3<T> w = skew(sang(v)), l = skew(slin(v));
  set_block(m, 0, 0, w);
  set_block(m, 1, 0, l);
  set_block(m, 1, 1, w);
  return m;
}
// Force cross-product matrix: crf(v) * f = v x* f = -crm(v)^T f.
template <class T> SMat<T> crf(const SVec<T>& v) {
  SMat<T> m = szeroM<T>();
  const Mat3<T> w = skew(sang(v)), l = skew(slin(v));
  set_block(m, 0, 0, w);
  set_block(m, 0, 1, l);
  set_block(m, 1, 1, w);
  return m;
}
// Plücker transform rot(E) * xlt(r) = [[E, 0], [-E r~, E]].
template <class T> SMat<T> plux(const Mat3<T>& E, const Vec3<T>& r) {
  SMat<T> m = szeroM<T>();
  set_block(m, 0, 0, E);
  set_block(m, 1, 1, E);
  set_block(m, 1, 0, mscale(mul(E, skew(r)), T(-1.0)));
  return m;
}
// Spatial inertia about the frame origin: [[Ic + m c~ c~^T, m c~], [m c~^T, m 1]].
template <class T> SMat<T> mcI(const T& m, const Vec3<T>& c, const Mat3<T>& Ic) {
  SMat<T> I = szeroM<T>();
  const Mat3<T> C = skew(c);
  const Mat3<T> CT = transpose(C);
  set_block(I, 0, 0, madd(Ic, mscale(mul(C, CT), m)));
  set_block(I, 0, 1, mscale(C, m));
  set_block(I, 1, 0, mscale(CT, m));
  set_block(I, 1, 1, mscale(ident3<T>(), m));
  return I;
}

// ----------------------------------------------------------------------------------------------
// Dense symmetric positive-definite solve by Cholesky factorisation A = L L^T (row-major n x n).
// Returns false if a pivot is not positive.
template <class T> bool cholesky_factor(std::vector<T>& A, int n) {
  for (int j = 0; j < n; ++j) {
    T s = A[j * n + j];
    for (int k = 0; k < j; ++k) s = s - A[j * n + k] * A[j * n + k];
    if (!(T(0.0) < s)) return false;
    const T ljj = sqrt(s);
    A[j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      T t = A[i * n + j];
      for (int k = 0; k < j; ++k) t = t - A[i * n + k] * A[j * n + k];
      A[i * n + j] = t / ljj;
    }
    for (int i = 0; i < j; ++i) A[i * n + j] = T(0.0);  // keep only the lower triangle
  }
  return true;
}
// Solve L L^T x = b in place given the factor from cholesky_factor.
template <class T> void cholesky_solve(const std::vector<T>& L, int n, T* b) {
  for (int i = 0; i < n; ++i) {
    T s = b[i];
    for (int k = 0; k < i; ++k) s = s - L[i * n + k] * b[k];
    b[i] = s / L[i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    T s = b[i];
    for (int k = i + 1; k < n; ++k) s = s - L[k * n + i] * b[k];
    b[i] = s / L[i * n + i];
  }
}

}  // namespace orc
