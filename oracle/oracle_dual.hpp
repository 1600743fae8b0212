// Test infrastructure only: a forward-mode dual number (value, one tangent) for the FP64 oracle.
// Running the oracle's step on it gives the exact directional derivative of the discrete FP64 step
// along the seeded input tangent: each elementary operation carries its derivative by the chain
// rule; comparisons and branches (contact and limit decisions, clamps, the speculative / biased
// target choice) follow the value, so the derivative is that of the step with its constraint and
// active sets held fixed. This is the oracle gradient the adjoint of the CUDA path is checked
// against.
#pragma once
#include <cmath>

namespace orc {

template <class F> struct DualT {
  F v, d;
  DualT() : v(F(0)), d(F(0)) {}
  DualT(double x) : v(F(x)), d(F(0)) {}  // NOLINT: implicit by design (constants)
  DualT(F x, F dx, int) : v(x), d(dx) {}
  friend DualT operator+(const DualT& a, const DualT& b) { return DualT(a.v + b.v, a.d + b.d, 0); }
  friend DualT operator-(const DualT& a, const DualT& b) { return DualT(a.v - b.v, a.d - b.d, 0); }
  friend DualT operator*(const DualT& a, const DualT& b) { return DualT(a.v * b.v, a.d * b.v + a.v * b.d, 0); }
  friend DualT operator/(const DualT& a, const DualT& b) {
    const F q = a.v / b.v;
    return DualT(q, (a.d - q * b.d) / b.v, 0);
  }
  DualT operator-() const { return DualT(-v, -d, 0); }
  friend bool operator<(const DualT& a, const DualT& b) { return a.v < b.v; }
  friend bool operator==(const DualT& a, const DualT& b) { return a.v == b.v; }
};
template <class F> inline DualT<F> sqrt(const DualT<F>& a) {
  const F s = std::sqrt(a.v);
  return DualT<F>(s, a.d / (F(2) * s), 0);
}
template <class F> inline DualT<F> sin(const DualT<F>& a) { return DualT<F>(std::sin(a.v), std::cos(a.v) * a.d, 0); }
template <class F> inline DualT<F> cos(const DualT<F>& a) { return DualT<F>(std::cos(a.v), -std::sin(a.v) * a.d, 0); }
template <class F> inline DualT<F> fabs(const DualT<F>& a) { return a.v < F(0) ? -a : a; }
template <class F> inline DualT<F> atan2(const DualT<F>& y, const DualT<F>& x) {
  const F r2 = x.v * x.v + y.v * y.v;
  return DualT<F>(std::atan2(y.v, x.v), (x.v * y.d - y.v * x.d) / r2, 0);
}
template <class F> inline double val(const DualT<F>& a) { return (double)a.v; }

using Dual = DualT<double>;   // the FP64 oracle derivative
using DualF = DualT<float>;   // the same arithmetic in single precision (conditioning probe)

}  // namespace orc
